"""Pins of the oracle's first discrete semigroup (Sec. 2.2, eq. cost1): the
exact path integral of a Fourier-series potential against numerical
quadrature, the action of a straight path against its definition, the
reductions to the fully discrete scheme (V = 0, constant V) on exact dyadic
data, monotonicity and contraction, and the two semigroups approaching each
other under refinement."""
import numpy as np
import pytest

from oracle import oracle as O


def series(x, modes, coef, L):
    x = np.atleast_2d(x)
    v = np.zeros(x.shape[0])
    for k, c in zip(np.asarray(modes).reshape(len(coef), -1), coef):
        ph = 2 * np.pi * (x / L) @ k
        v += np.real(c) * np.cos(ph) - np.imag(c) * np.sin(ph)
    return v


def gauss_integral(f, tau, n=48):
    t, w = np.polynomial.legendre.leggauss(n)
    s = 0.5 * tau * (t + 1)
    return 0.5 * tau * np.sum(w * np.array([f(si) for si in s]))


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_path_integral_against_quadrature(ndim):
    rng = np.random.default_rng(ndim)
    modes = rng.integers(-3, 4, size=(5, ndim))
    modes[0] = 0                                    # the constant mode
    coef = rng.normal(size=5) + 1j * rng.normal(size=5)
    L = rng.uniform(0.5, 2.0, size=ndim)
    tau = 0.07
    for _ in range(5):
        y = rng.uniform(0, 1, size=ndim) * L
        D = rng.normal(size=ndim) * 0.3
        got = O.path_integral(modes, coef, y[None], D[None], tau, L)[0]
        want = gauss_integral(lambda s: series(y + s * D / tau, modes, coef, L)[0], tau)
        assert abs(got - want) < 1e-13 * (1 + abs(want))


def test_trig_values_on_the_grid():
    modes = np.array([[1, 0], [2, -1]])
    coef = np.array([0.5 - 0.25j, 0.1 + 0.3j])
    V = O.trig_values((8, 6), modes, coef)
    i, j = np.meshgrid(np.arange(8), np.arange(6), indexing="ij")
    x = np.stack([i / 8, j / 6], -1).reshape(-1, 2)
    assert np.allclose(V.ravel(), series(x, modes, coef, np.ones(2)), atol=1e-15)


def test_step_cost_is_the_path_action():
    """One candidate of one step, recomputed as the definition: tau K*(v)
    minus the quadrature of V along the straight path from y to x."""
    shape, dx, h, P, W = (10,), 0.1, 0.05, 0.3, 0
    modes, coef = np.array([[1], [3]]), np.array([0.4 + 0.1j, -0.2j])
    u0 = np.zeros(shape)
    u0[3] = -50.0                                   # the source y = 3 wins every row
    out = O.integral_run(u0, dx, h, P, W, modes, coef, 1)
    for x in range(10):
        dlo, dhi, _ = O.table(10, dx, h, P, W)
        ds = [dd for dd in range(dlo, dhi + 1) if (x - dd) % 10 == 3]
        best = np.inf
        for dd in ds:
            v = dd * dx / h
            kin = h * (0.5 * v * v - P * v)
            pot = gauss_integral(lambda s: series(np.array([[3 * dx + s * dd * dx / h]]), modes, coef,
                                                  np.array([1.0]))[0], h)
            best = min(best, -50.0 + kin - pot)
        assert abs(out[x] - best) < 1e-12


CASES = [((16,), 1 / 32, 0.125, 0.25, 3), ((12, 16), (1 / 32, 1 / 32), 0.125, (0.25, -0.5), (2, 3)),
         ((6, 8, 10), (1 / 32,) * 3, 0.125, (0.5, 0.25, -0.25), (1, 2, 0))]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[0])))
def test_reduces_to_the_scheme_on_dyadic_data(case):
    shape, dx, h, P, W = case
    rng = np.random.default_rng(4)
    u0 = rng.integers(-2048, 2048, size=shape) / 1024.0
    nd = len(shape)
    none = np.zeros((0, nd), dtype=int)
    assert np.array_equal(O.integral_run(u0, dx, h, P, W, none, [], 2), O.run(u0, dx, h, P, W, None, 2))
    c = 0.375                                        # constant potential: the k = 0 mode
    got = O.integral_run(u0, dx, h, P, W, np.zeros((1, nd), dtype=int), [c], 2)
    assert np.array_equal(got, O.run(u0, dx, h, P, W, np.full(shape, c), 2))


def test_monotone_and_contracting():
    rng = np.random.default_rng(5)
    shape, dx, h, P, W = (20,), 0.05, 0.05, 0.2, 6
    modes, coef = np.array([[1], [2]]), np.array([0.5 + 0.2j, 0.1 - 0.3j])
    u = rng.normal(size=shape) * 0.2
    v = u + np.abs(rng.normal(size=shape)) * 0.1
    Tu = O.integral_run(u, dx, h, P, W, modes, coef, 3)
    Tv = O.integral_run(v, dx, h, P, W, modes, coef, 3)
    assert np.all(Tu <= Tv)
    w = u + rng.normal(size=shape) * 0.1
    Tw = O.integral_run(w, dx, h, P, W, modes, coef, 3)
    assert np.max(np.abs(Tu - Tw)) <= np.max(np.abs(u - w)) + 1e-15


def test_the_two_semigroups_approach_each_other():
    """Both are consistent discretisations of the same equation: at T = 0.5
    the sup distance between them shrinks under refinement (dx, tau ~ sqrt dx)."""
    modes, coef = np.array([[1], [2]]), np.array([0.5 + 0.2j, 0.1 - 0.3j])
    gaps = []
    for N in (16, 64, 256):
        dx = 1.0 / N
        n = int(np.ceil(0.5 / np.sqrt(dx)))
        h = 0.5 / n
        W = int(np.ceil(3 * h / dx)) + 1
        x = np.arange(N) / N
        u0 = 0.3 * np.cos(2 * np.pi * x)
        V = O.trig_values((N,), modes, coef)
        a = O.integral_run(u0, dx, h, 0.3, W, modes, coef, n)
        b = O.run(u0, dx, h, 0.3, W, V, n)
        gaps.append(np.max(np.abs(a - b)))
    assert gaps[2] < gaps[1] < gaps[0], gaps
