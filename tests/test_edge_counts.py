"""The window-edge count used as the expected value of
hjlo_counters.window_edge_hits, checked on the CPU oracle.

A window of 2W+1 displacements centred on the kernel minimiser (Sec. 4.2)
truncates the lift-minimised torus window (eq. los).  A steep ramp moves the
minimiser of u[i-d] + k[d] beyond the window for every row away from the
ramp's jump, so those argmins sit on the window's edge and the truncated step
differs from the full one; a gentle field keeps every argmin inside."""
import numpy as np

from edge_counts import edge_hits
from oracle import oracle as O


def test_steep_ramp_hits_the_edge():
    N, W, h = 64, 3, 0.05
    dx = 1.0 / N
    x = np.arange(N) * dx
    u0 = 40.0 * x                      # slope 40: the unwindowed minimiser is ~ h*40/dx = 128 cells away
    hits = edge_hits(u0, dx, h, 0.0, W, None, 1)
    assert hits >= N - 2 * W - 2
    windowed = O.run(u0, dx, h, 0.0, W, None, 1)
    full = O.run(u0, dx, h, 0.0, 0, None, 1)
    assert np.all(full <= windowed) and np.any(full < windowed)


def test_gentle_field_stays_inside():
    N, W, h = 128, 16, 0.02
    dx = 1.0 / N
    x = np.arange(N) * dx
    u0 = 0.05 * np.sin(2 * np.pi * x)
    V = 0.1 * np.cos(2 * np.pi * x)
    assert edge_hits(u0, dx, h, 0.3, W, V, 5) == 0
    assert np.array_equal(O.run(u0, dx, h, 0.3, W, V, 5), O.run(u0, dx, h, 0.3, 0, V, 5))


def test_full_window_counts_nothing():
    rng = np.random.default_rng(0)
    u0 = rng.normal(size=(12, 10))
    assert edge_hits(u0, (1 / 12, 1 / 10), 0.1, (0.2, -0.4), (0, 5), None, 3) == 0
