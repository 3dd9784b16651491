"""The five steps of the whole-period decomposition across CTAs (classify,
chunk-local cuts, stitch, per-piece running maxima, per-block vertex
emission), written out plainly in Python and checked on the CPU against the
oracle's decomposition method (Sec. 4.3: one greedy cut per period, every
component convolved, the minimum taken): the same starts, the same
component count and the same values bit for bit, over random lines, windows,
tolerances, chunk sizes and output blocks.  This pins the algorithm the CUDA
kernels implement (a piece's vertex is (A(p), p + 1) when its component is
convex and (A(p), p), (A(p), p + 1) when concave; a point's vertices fill an
interval fixed by A at its two pieces and whether it starts or ends its
component); the kernels themselves are compared with the oracle on the GPU."""
import numpy as np
import pytest

from oracle import oracle as O


def model(src, k, eta, CH, vR):
    """(outputs, component count, starts) of one lifted line src (N + n
    points, k the n + 1 kernel values) by the five steps, with chunks of CH
    points and output blocks of vR rows."""
    n = len(k) - 1
    L = len(src)
    N = L - n
    slopes = np.diff(k)
    # 1. classify: convex / concave rule at every interior point, F per piece
    cv = np.zeros(L + CH, bool)
    cc = np.zeros(L + CH, bool)
    F = np.zeros(L, np.int64)
    for q in range(L - 1):
        r1 = src[q + 1] - src[q]
        F[q] = int(np.searchsorted(slopes, r1, side="left"))   # kernel slopes strictly below
        if q >= 1:
            inc = r1 - (src[q] - src[q - 1])
            cv[q] = inc >= -eta
            cc[q] = inc <= 0.0

    def next_start(s):
        """The greedy cut's next start after a component starting at s."""
        if s + 1 >= L - 1:
            return L - 1
        bits = cv if cv[s + 1] else cc
        q = s + 2
        while q < L - 1 and bits[q]:
            q += 1
        return min(q, L - 1)

    # 2. local cuts: each chunk cut from its first point
    B = (L + CH - 1) // CH
    local = np.zeros(B * CH, bool)
    X = [0] * B
    for b in range(B):
        s = b * CH
        while s < (b + 1) * CH and s < L - 1:
            local[s] = True
            s = next_start(s)
        X[b] = s
    # 3. stitch: walk the true cut, jumping along a chunk's local cut once on it
    entry = [-1] * B
    single = np.zeros(B * CH, bool)
    s = 0
    while s < L - 1:
        b = s // CH
        if local[s]:
            entry[b] = s
            s = X[b]
        else:
            single[s] = True
            s = next_start(s)
    starts = np.array([(local[q] and 0 <= entry[q // CH] <= q) or single[q] for q in range(B * CH)])
    # 4. pieces: component kind and A (running max of F if convex, else F)
    A = np.zeros(L, np.int64)
    convex = np.zeros(L, bool)
    comp, run = 0, 0
    for q in range(L - 1):
        if starts[q]:
            comp, run = q, F[q]
        else:
            run = max(run, F[q])
        convex[q] = cv[comp + 1] if comp + 1 < L - 1 else True
        A[q] = run if convex[q] else F[q]
    # 5. emit per block of outputs x in [x0, x1) (vertex z = x + n)
    out = np.full(N, np.inf)
    for x0 in range(0, N, vR):
        x1 = min(N, x0 + vR)
        zlo, zhi = x0 + n, x1 + n
        keys = np.full(x1 - x0, np.inf)

        def vertex(y, d):
            z = y + d
            assert 0 <= d <= n
            if zlo <= z < zhi:
                keys[z - zlo] = min(keys[z - zlo], k[d] + src[y])

        for q in range(max(0, x0 - 1), min(L - 2, x1 + n - 1) + 1):
            if convex[q]:
                vertex(q + 1, A[q])
            else:
                vertex(q, A[q])
                vertex(q + 1, A[q])
        for y in range(x0, min(L - 1, x1 + n - 1) + 1):
            is_start = y == 0 or (y < L - 1 and starts[y])
            is_end = y == L - 1 or (y > 0 and starts[y])
            spans = []
            if is_start and y <= L - 2:
                spans.append((0, A[y] + 1))
            if is_end and y >= 1:
                spans.append((A[y - 1] + (1 if convex[y - 1] else 0), n + 1))
            if not (is_start or is_end) and convex[y]:
                spans.append((A[y - 1] + 1, A[y] + 1))
            for d0, d1 in spans:
                for d in range(d0, d1):
                    vertex(y, d)
        out[x0:x1] = keys
    return out, int(starts[:L - 1].sum()), [q for q in range(L - 1) if starts[q]]


@pytest.mark.parametrize("seed", range(4))
def test_split_steps_equal_the_method(seed):
    rng = np.random.default_rng(500 + seed)
    for trial in range(20):
        N = int(rng.integers(2, 260))
        W = int(rng.integers(0, max(1, N // 2)))
        dx = 1.0 / N
        h = float(rng.uniform(0.01, 0.2))
        P = float(rng.uniform(-0.5, 0.5))
        dlo, dhi, k = O.table(N, dx, h, P, W)
        n = dhi - dlo
        x = np.arange(N) * dx
        kind = trial % 3
        if kind == 0:
            u = rng.normal(size=N) * 0.3
        elif kind == 1:
            u = np.cos(2 * np.pi * x) + 0.01 * rng.normal(size=N)
        else:
            u = np.abs(np.sin(3 * np.pi * x)) * 0.2
        src = u[(np.arange(N + n) - dhi) % N]
        eta = float(rng.choice([0.0, dx, 10 * dx, 1e3]))
        ref, nc = O.decomp_line(src, k, eta)
        CH = int(rng.choice([32, 64, 96, 128]))
        vR = int(rng.integers(1, N + 1))
        got, ncg, starts = model(src, k, eta, CH, vR)
        assert starts == [c[0] for c in O.decompose(src, eta)], (seed, trial)
        assert ncg == nc, (seed, trial)
        assert np.array_equal(got.view(np.int64), ref.view(np.int64)), (seed, trial, N, W, eta, CH, vR)
