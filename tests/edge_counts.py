"""Window-edge argmin counts taken from the oracle's recorded argmins (test
helper: the expected value of hjlo_counters.window_edge_hits)."""
import numpy as np

from oracle import oracle as O


def edge_hits(u0, dx, h, P, W, V, n):
    """Outputs whose oracle argmin is the first or last displacement of a
    partial window (2W+1 < N), summed over the steps and axes."""
    _, am = O.run(u0, dx, h, P, W, V, n, record_argmin=True)
    shape = np.shape(u0)
    nd = len(shape)
    dxv = np.broadcast_to(np.asarray(dx, dtype=np.float64), (nd,))
    Pv = np.broadcast_to(np.asarray(P, dtype=np.float64), (nd,))
    Wv = np.broadcast_to(np.asarray(W, dtype=np.int64), (nd,))
    tot = 0
    for a in range(nd):
        N, w = shape[a], int(Wv[a])
        if w <= 0 or 2 * w + 1 >= N:
            continue
        lo, hi = O.window(N, float(dxv[a]), h, float(Pv[a]), w)
        tot += int(np.count_nonzero((am[:, a] == lo) | (am[:, a] == hi)))
    return tot
