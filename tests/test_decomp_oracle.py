"""Pins of the oracle's version of the paper's own fast (min,plus)
convolution (Sec. 4): Algorithm 1 (convex by convex, Theorem th:convex), the
three-part convex-by-concave convolution (Lemmas lm:seg, lm:simplif,
Theorem th:ccc, Algorithm 2) and the convex/concave decomposition with its
tolerance eta (Sec. 4.3-4.4), each against the plain definition of the
(min,plus) convolution and against the scheme."""
import numpy as np
import pytest

from oracle import oracle as O


def brute_conv(f, g):
    """(f conv g)(x) = min_{i + j = x} f(i) + g(j), the definition (eq. convolfg)."""
    n, m = len(f) - 1, len(g) - 1
    h = np.full(n + m + 1, np.inf)
    for i in range(n + 1):
        for j in range(m + 1):
            h[i + j] = min(h[i + j], f[i] + g[j])
    return h


def dyadic_convex(rng, n, scale=64):
    """Exact binary64 convex sequence: cumulative sums of sorted dyadic slopes."""
    slopes = np.sort(rng.integers(-scale, scale, size=n)) / 16.0
    return rng.integers(-64, 64) / 16.0 + np.concatenate([[0.0], np.cumsum(slopes)])


@pytest.mark.parametrize("seed", range(25))
def test_convex_convex_is_the_convolution(seed):
    rng = np.random.default_rng(seed)
    f = dyadic_convex(rng, int(rng.integers(0, 9)))
    g = dyadic_convex(rng, int(rng.integers(0, 9)))
    h = O.convex_convex(f, g)
    assert np.array_equal(h, brute_conv(f, g))
    s = np.diff(h)
    assert np.all(np.diff(s) >= 0)           # Theorem th:convex: the result is convex


@pytest.mark.parametrize("seed", range(40))
def test_convex_concave_is_the_convolution(seed):
    rng = np.random.default_rng(100 + seed)
    f = dyadic_convex(rng, int(rng.integers(0, 10)))
    g = -dyadic_convex(rng, int(rng.integers(1, 10)))          # concave
    h = O.convex_concave(f, g)
    assert np.array_equal(h, brute_conv(f, g))


def test_convex_concave_with_equal_slopes_and_affine_pieces():
    f = np.array([0.0, 0.0, 0.0, 1.0, 3.0])          # flat start: ties in alpha
    g = np.array([2.0, 2.5, 3.0, 3.0, 1.0])          # concave with an affine run
    assert np.array_equal(O.convex_concave(f, g), brute_conv(f, g))
    assert np.array_equal(O.convex_convex(f, np.array([1.0, 1.0])), brute_conv(f, np.array([1.0, 1.0])))


@pytest.mark.parametrize("eta", [0.0, 0.05, 1e9])
def test_decompose_components(eta):
    rng = np.random.default_rng(3)
    g = rng.normal(size=60)
    comps = O.decompose(g, eta)
    assert comps[0][0] == 0 and comps[-1][1] == len(g) - 1
    for (s, e, cvx), nxt in zip(comps, comps[1:] + [None]):
        assert e > s
        if nxt is not None:
            assert nxt[0] == e                         # consecutive, sharing end points
        inc = np.diff(np.diff(g[s:e + 1]))
        assert np.all(inc >= -eta) if cvx else np.all(inc <= 0)
    if eta >= 1e9:
        assert len(comps) == 1                          # everything is "convex enough"
    x = np.linspace(0, 1, 30)
    assert len(O.decompose(x ** 2, 0.0)) == 1 and len(O.decompose(-x ** 2, 0.0)) == 1


CASES = [
    ((48,), 1 / 32, 0.125, 0.25, 6),
    ((40,), 1 / 32, 0.125, -0.5, 0),
    ((12, 20), (1 / 32, 1 / 32), 0.125, (0.25, -0.5), (3, 0)),
    ((6, 8, 10), (1 / 32,) * 3, 0.125, (0.5, 0.25, -0.25), (2, 0, 3)),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[0])))
def test_decomposition_method_equals_scheme_on_dyadic_data(case):
    """eta = 0: Sec. 4 computes the convolution exactly; with dyadic data every
    sum is exact, so the method equals the scheme bit for bit."""
    shape, dx, h, P, W = case
    rng = np.random.default_rng(5)
    u0 = rng.integers(-2048, 2048, size=shape) / 1024.0
    V = rng.integers(-256, 256, size=shape) / 256.0
    ref = O.run(u0, dx, h, P, W, V, 3)
    got, ncomp = O.decomp_run(u0, dx, h, P, W, V, 3)
    assert np.array_equal(got, ref) and ncomp > 0


@pytest.mark.parametrize("eta", [0.0, 1e-3, 1e-1])
def test_every_output_is_a_candidate(eta):
    """One pass: each output is one candidate u(y) + k(d) of the scheme's set,
    so it is never below the scheme's minimum; at eta = 0 it equals it
    wherever rounding does not reorder near-ties."""
    rng = np.random.default_rng(9)
    shape, dx, h, P, W = (300,), 1 / 300, 0.05, 0.4, 25
    u0 = np.cumsum(rng.normal(size=shape)) * 0.02
    ref = O.run(u0, dx, h, P, W, None, 1)
    got, _ = O.decomp_run(u0, dx, h, P, W, None, 1, eta)
    assert np.all(got >= ref)
    if eta == 0.0:
        assert np.max(np.abs(got - ref)) <= 4 * np.spacing(np.max(np.abs(ref)))


def test_error_grows_with_eta_and_components_shrink():
    rng = np.random.default_rng(4)
    shape, dx, h, P, W = (256,), 1 / 256, 0.05, 0.3, 20
    u0 = np.cumsum(rng.normal(size=shape)) * 0.01
    ref = O.run(u0, dx, h, P, W, None, 4)
    errs, comps = [], []
    for eta in (0.0, 1e-4, 1e-3, 1e-2):
        got, c = O.decomp_run(u0, dx, h, P, W, None, 4, eta)
        errs.append(np.max(np.abs(got - ref)))
        comps.append(c)
    assert errs[0] <= 1e-14
    assert comps == sorted(comps, reverse=True) and comps[-1] < comps[0]
    assert errs[-1] >= errs[0]


def test_zero_tolerance_equals_the_scheme_for_any_start():
    """At eta = 0 every component is exactly convex or concave and the method
    is exact (Theorem th:convex, Theorem th:ccc), so the result does not
    depend on where the decomposition of the periodic line starts: lines
    rotated before the pass give the scheme's values rotated."""
    N, W, h = 300, 12, 0.01
    x = np.arange(N) / N
    rng = np.random.default_rng(5)
    u0 = 0.3 * np.sin(6 * np.pi * x) + 0.01 * rng.normal(size=N)
    ref = O.run(u0, 1.0 / N, h, 0.2, W, None, 1)
    for shift in (0, 24, 77, 151):
        got, _ = O.decomp_run(np.roll(u0, shift), 1.0 / N, h, 0.2, W, None, 1, 0.0)
        assert np.array_equal(np.roll(got, -shift).view(np.int64), ref.view(np.int64)), shift


def test_tolerance_outputs_stay_candidates():
    """With eta > 0 every output is still one candidate of the scheme (a value
    f(i) + g(j) of the components' convolutions), so never below the exact
    scheme's value, and the gap grows with eta."""
    N, W, h = 300, 12, 0.01
    x = np.arange(N) / N
    rng = np.random.default_rng(6)
    u0 = 0.3 * np.sin(6 * np.pi * x) + 0.01 * np.cumsum(rng.normal(size=N)) / np.sqrt(N)
    exact = O.run(u0, 1.0 / N, h, 0.2, W, None, 1)
    gaps = []
    for eta in (0.5, 5.0, 50.0):
        got, _ = O.decomp_run(u0, 1.0 / N, h, 0.2, W, None, 1, eta)
        assert np.all(got >= exact), eta
        gaps.append(float(np.max(got - exact)))
    assert gaps[0] <= gaps[1] <= gaps[2], gaps
