"""The discrete effective Hamiltonian as a (min,plus) eigenvalue (Remark
after Prop. prop:klm): the one-step matrix of the scheme, Karp's minimum
cycle mean, and the long-time slope of the scheme itself, checked against
each other and against brute force and closed forms."""
import itertools

import numpy as np
import pytest

from oracle import oracle as O


def _brute_cycle_mean(B):
    """Minimum mean over all simple cycles (every ordered subset), n <= 5."""
    n = B.shape[0]
    best = np.inf
    for m in range(1, n + 1):
        for cyc in itertools.permutations(range(n), m):
            if cyc[0] != min(cyc):
                continue
            w = sum(B[cyc[i], cyc[(i + 1) % m]] for i in range(m))
            best = min(best, w / m)
    return best


@pytest.mark.parametrize("seed", range(6))
def test_karp_equals_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 6))
    B = rng.normal(size=(n, n))
    if seed % 2:
        B[rng.random((n, n)) < 0.3] = np.inf        # sparse but keep a Hamiltonian cycle
        for i in range(n):
            B[i, (i + 1) % n] = rng.normal()
    assert abs(O.minplus_eigenvalue(B) - _brute_cycle_mean(B)) < 1e-12


def test_karp_closed_forms():
    # one cheap self-loop dominates; a uniform matrix has its entry as mean
    B = np.full((4, 4), 3.0)
    B[2, 2] = -1.5
    assert O.minplus_eigenvalue(B) == -1.5
    assert O.minplus_eigenvalue(np.full((3, 3), 0.25)) == 0.25


@pytest.mark.parametrize("shape,dx,h,P,W", [
    ((7,), 1 / 7, 0.1, 0.9, 0),
    ((6, 5), (1 / 6, 1 / 5), 0.08, (0.5, -1.2), (0, 0)),
    ((9,), 1 / 9, 0.05, -0.4, 2),
])
def test_zero_potential_eigenvalue_is_sum_of_kernel_minima(shape, dx, h, P, W):
    """V = 0: the cheapest cycle repeats the kernel minimiser on every axis,
    so lambda = sum_a min_d k_a[d] (pin P1 of the closed forms)."""
    B = O.step_matrix(shape, dx, h, P, W)
    ndim = len(shape)
    want = sum(O.table(shape[a], np.atleast_1d(dx)[a] if ndim > 1 else dx, h,
                       np.atleast_1d(P)[a] if ndim > 1 else P,
                       np.atleast_1d(W)[a] if ndim > 1 else W)[2].min() for a in range(ndim))
    assert abs(O.minplus_eigenvalue(B) - want) <= 1e-15 * (1 + abs(want)) * 8


@pytest.mark.parametrize("shape,dx,h,P,W", [
    ((8,), 1 / 8, 0.1, 0.3, 0),
    ((5, 6), (1 / 5, 1 / 6), 0.07, (0.4, -0.2), (0, 2)),
])
def test_step_matrix_is_one_step_of_the_scheme(shape, dx, h, P, W):
    rng = np.random.default_rng(1)
    u = rng.normal(size=shape) * 0.3
    V = rng.normal(size=shape) * 0.2
    B = O.step_matrix(shape, dx, h, P, W, V)
    got = np.min(u.reshape(-1)[:, None] + B, axis=0).reshape(shape)
    ref = O.run(u, dx, h, P, W, V, 1)
    assert np.max(np.abs(got - ref)) <= 1e-14


@pytest.mark.parametrize("shape,dx,h,P,W", [
    ((8,), 1 / 8, 0.1, 0.3, 0),
    ((12,), 1 / 12, 0.05, -0.7, 3),
    ((4, 5), (1 / 4, 1 / 5), 0.07, (0.4, -0.2), (0, 0)),
])
def test_long_time_slope_is_the_eigenvalue(shape, dx, h, P, W):
    """Prop. prop:klm: u^n / n -> lambda; past the transient the (min,plus)
    powers are periodic (Remark rem38), so the slope over many steps matches
    Karp's value to rounding divided by the step count."""
    rng = np.random.default_rng(7)
    u0 = rng.normal(size=shape) * 0.3
    V = rng.normal(size=shape) * 0.3
    lam = O.minplus_eigenvalue(O.step_matrix(shape, dx, h, P, W, V))
    n1, n2 = 400, 1200
    u1 = O.run(u0, dx, h, P, W, V, n1)
    u2 = O.run(u1, dx, h, P, W, V, n2 - n1)
    slope = (u2 - u1) / (n2 - n1)
    assert np.max(np.abs(slope - lam)) < 1e-9 * (1 + abs(lam))
    hb = O.hbar_estimate(u1, u2, n2 - n1, h)
    assert abs(hb[0] - (-lam / h)) < 1e-8 * (1 + abs(lam / h))
