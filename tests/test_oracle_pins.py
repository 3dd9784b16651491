"""Pins for the CPU oracle: every check ties it to something other than itself.

The paper (Bouillard, Faou & Zavidovique) fixes: the kernel (eq. cost2 with
L = v^2/2 - P.v, Sec. 2.1), the torus scheme with lift-minimised cost (eq.
los), the min-plus structure of one step (eq. eqconvol), axis splitting
(Remark rk28), the N-step composition (eq. uN), monotonicity (remark after
eq. uN), the discrete optimal path (eq. raslebol), convex-by-convex
convolution (Theorem th:convex), the weak-KAM limit (Prop. prop:klm) and its
error bound (theorem after prop:klm).  Pins used below:
  * exact rational arithmetic (fractions) for kernel values and windows;
  * dyadic parameters where binary64 arithmetic is exact, so brute force over
    paths / lifts / full n-D minima must agree bit for bit;
  * closed forms: V=0 constant data, n-fold convex convolution, 1D effective
    Hamiltonian of the cell problem;
  * invariants: monotonicity, shift/reflection equivariance, semigroup,
    bounded oscillation, cotangent mass conservation, finite differences.
All CPU; no GPU and no CUDA library involved.
"""
import itertools
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_1210_4090_gb300 import workloads as WL

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ helpers

def exact_k(d, dx, h, P):
    """h * (v^2/2 - P v), v = d dx / h, in exact rational arithmetic."""
    dx, h, P = Fraction(dx), Fraction(h), Fraction(P)
    v = d * dx / h
    return h * (v * v / 2 - P * v)


def dyadic_problem(shape, seed, nsteps=3, P=None, W=None, per_step=False):
    """Parameters and data for which every binary64 operation of the scheme is exact."""
    rng = np.random.default_rng(seed)
    nd = len(shape)
    dx = tuple(1.0 / 32 for _ in shape)           # 2^-5
    h = 0.125                                     # v = d/4 exactly
    P = P if P is not None else tuple(float(x) for x in rng.choice([-0.5, -0.25, 0.25, 0.5, 0.75], nd))
    W = W if W is not None else tuple(0 for _ in shape)
    u0 = rng.integers(-2048, 2048, size=shape) / 1024.0          # multiples of 2^-10
    vshape = (nsteps, *shape) if per_step else shape
    V = rng.integers(-256, 256, size=vshape) / 256.0              # h*V = V/8 exact
    return dx, h, P, W, u0, V


def generic_problem(shape, seed, W=None):
    rng = np.random.default_rng(seed)
    nd = len(shape)
    dx = tuple(1.0 / n for n in shape)
    h = 0.07
    P = tuple(float(x) for x in rng.uniform(-0.8, 0.8, nd))
    W = W if W is not None else tuple(max(1, n // 4) for n in shape)
    u0 = rng.normal(size=shape) * 0.3
    V = rng.normal(size=shape) * 0.2
    return dx, h, P, W, u0, V


def lift_min_cost(N, dx, h, P, residue):
    """kappa~ for one residue: min over lifts of the exact kernel (eq. los)."""
    best, arg = None, None
    for m in range(-4, 5):
        d = residue + m * N
        k = exact_k(d, dx, h, P)
        if best is None or k < best:
            best, arg = k, d
    return best, arg


# ------------------------------------------------------------------ kernel table

PARAMS = [  # (N, dx, h, P, W) from the workloads and some awkward ones
    (256, 1 / 256, 0.05, 0.3, 0), (1024, 1 / 1024, 0.02, 0.3, 64), (1024, 1 / 1024, 0.02, 0.1, 64),
    (256, 1 / 256, 0.02, 0.2, 32), (256, 1 / 256, 0.02, -0.1, 32), (256, 1 / 256, 0.02, 0.35, 32),
    (512, 1 / 512, 0.02, 0.3, 32), (128, 1 / 128, 0.02, -0.93, 8), (17, 1 / 17, 0.3, 2.7, 0),
    (16, 1 / 16, 0.11, -1.3, 0), (7, 1 / 7, 0.5, 0.0, 2), (1, 1.0, 0.1, 0.4, 0),
]


@pytest.mark.parametrize("N,dx,h,P,W", PARAMS)
def test_kernel_matches_exact_rationals(N, dx, h, P, W):
    dlo, dhi, k = O.table(N, dx, h, P, W)
    for d in range(dlo, dhi + 1):
        ex = exact_k(d, dx, h, P)
        v = abs(d * dx / h)
        bound = 8 * 2.0 ** -53 * h * (v * v / 2 + abs(P * v)) + 1e-300
        assert abs(Fraction(k[d - dlo]) - ex) <= Fraction(bound), (d, k[d - dlo], float(ex))


@pytest.mark.parametrize("N,dx,h,P,W", PARAMS)
def test_window_centre_and_lift_minimisation(N, dx, h, P, W):
    dlo, dhi = O.window(N, dx, h, P, W)
    ds = int(np.floor(P * h / dx))
    cands = list(range(ds - 6, ds + 8))
    vals = [exact_k(d, dx, h, P) for d in cands]
    kmin = min(vals)
    c = max(d for d, v in zip(cands, vals) if v == kmin)          # largest minimiser
    if W > 0 and 2 * W + 1 < N:
        assert (dlo, dhi) == (c - W, c + W)
    else:
        assert dhi - dlo + 1 == N and dlo <= c <= dhi
        for d in range(dlo, dhi + 1):                               # one lift per residue ...
            best, _ = lift_min_cost(N, dx, h, P, d % N)
            assert exact_k(d, dx, h, P) == best                     # ... and the cheapest one


def test_workload_centres():
    # integer minimisers of h L(d dx/h): nearest integer to P h / dx.  Full window
    # of line256: the 256 integers nearest the continuous minimiser 3.84, i.e.
    # those in (3.84 - 128, 3.84 + 128).
    assert O.window(256, 1 / 256, 0.05, 0.3, 300) == (-124, 131)
    for (N, P, c) in [(1024, 0.3, 6), (1024, 0.1, 2), (256, 0.2, 1), (256, -0.1, -1),
                      (256, 0.35, 2), (512, 0.3, 3), (512, 0.1, 1)]:
        W = 64 if N == 1024 else 32
        assert O.window(N, 1 / N, 0.02, P, W) == (c - W, c + W)


# ------------------------------------------------------------------ V = 0 closed forms

def _golden_hbar():
    out = {}
    with open(os.path.join(GOLDEN, "vzero_hbar.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, val = line.split()
                out[name] = float(val)
    return out


@pytest.mark.parametrize("name", ["line256", "grid1024", "cube256", "adjoint512"])
def test_vzero_constant_data_hbar(name):
    """u0 = const, V = 0: every candidate of a line is const + k[d], so one step adds
    sum_a min_d k_a[d] exactly once per axis; the discrete effective Hamiltonian is
    -sum_a kmin_a / h (Prop. prop:klm), within (dx/h)^2/8 per axis of |P|^2/2."""
    N = {"line256": 9, "grid1024": 11, "cube256": 6, "adjoint512": 10}[name]
    # same h, P and dx as the workload; a small grid of the same dx keeps it cheap
    full = {"line256": (256,), "grid1024": (1024, 1024), "cube256": (256,) * 3,
            "adjoint512": (512, 512)}[name]
    h = {"line256": 0.05}.get(name, 0.02)
    P = {"line256": (0.3,), "grid1024": (0.3, 0.1), "cube256": (0.2, -0.1, 0.35),
         "adjoint512": (0.3, 0.1)}[name]
    dx = tuple(1.0 / n for n in full)
    nd = len(full)
    shape = (N,) * nd
    W = tuple(0 for _ in shape)
    u0 = np.full(shape, 0.375)
    n = 7
    un = O.run(u0, dx, h, P, W, None, n)
    kmins = []
    for a in range(nd):
        # exact minimum over the integers near P h / dx
        ds = int(np.floor(P[a] * h / dx[a]))
        kmins.append(min(exact_k(d, dx[a], h, P[a]) for d in range(ds - 3, ds + 5)))
    # binary64 replay: u <- fl(u + fl(kmin_a)) per axis per step
    expect = 0.375
    for _ in range(n):
        for km in kmins:
            expect = expect + float(km)
    assert np.all(un == expect)
    hbar = -sum(kmins) / Fraction(h)
    golden = _golden_hbar()[name]
    assert abs(float(hbar) - golden) <= 1e-15
    half_p2 = sum(Fraction(x) ** 2 for x in P) / 2
    assert abs(hbar - half_p2) <= sum(Fraction(d) ** 2 / Fraction(h) ** 2 / 8 for d in dx)
    est, lo, hi = O.hbar_estimate(u0, un, n, h)
    assert abs(est - float(hbar)) < 1e-12 and lo == hi == est


def test_vzero_convolution_power_dyadic():
    """V = 0: n steps equal one min-plus convolution with the n-fold kernel, which for
    a convex kernel puts the slopes end to end (Theorem th:convex): with D = n q + r,
    k^{(+)n}(D) = (n - r) k(q) + r k(q+1).  Dyadic data: exact, so bitwise."""
    for N, P, n in [(32, 0.25, 1), (32, 0.5, 3), (31, -0.75, 4), (12, 0.25, 5)]:
        dx, h = 1.0 / 32, 0.125
        rng = np.random.default_rng(N + n)
        u0 = rng.integers(-4096, 4096, size=N) / 1024.0
        un = O.run(u0, dx, h, P, 0, None, n)
        for x in range(N):
            best = None
            for D in range(-4 * N * n, 4 * N * n + 1):
                q, r = divmod(D, n)
                kn = (n - r) * exact_k(q, dx, h, P) + r * exact_k(q + 1, dx, h, P)
                c = Fraction(u0[(x - D) % N]) + kn
                best = c if best is None or c < best else best
            assert Fraction(un[x]) == best, (N, P, n, x)


# ------------------------------------------------------------------ invariants

SHAPES = [(40,), (13, 9), (6, 7, 5)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("windowed", [False, True])
def test_monotone(shape, windowed):
    """u <= v implies T^n u <= T^n v (remark after eq. uN); rounding is monotone too."""
    dx, h, P, W, u0, V = generic_problem(shape, 11)
    if not windowed:
        W = tuple(0 for _ in shape)
    rng = np.random.default_rng(5)
    v0 = u0 + np.abs(rng.normal(size=shape)) * rng.integers(0, 2, size=shape)
    a = O.run(u0, dx, h, P, W, V, 4)
    b = O.run(v0, dx, h, P, W, V, 4)
    assert np.all(a <= b)
    c = O.run(u0 + 1e-9, dx, h, P, W, V, 4)     # sup-norm contraction
    assert np.max(np.abs(c - a)) <= 1e-9 * (1 + 1e-6) + 1e-14


@pytest.mark.parametrize("shape", SHAPES)
def test_commutes_with_constants_dyadic(shape):
    dx, h, P, W, u0, V = dyadic_problem(shape, 2)
    a = O.run(u0, dx, h, P, W, V, 3)
    b = O.run(u0 + 2.0 ** -6, dx, h, P, W, V, 3)
    assert np.array_equal(b, a + 2.0 ** -6)


@pytest.mark.parametrize("shape", SHAPES)
def test_shift_equivariance(shape):
    dx, h, P, W, u0, V = generic_problem(shape, 3)
    a = O.run(u0, dx, h, P, W, V, 3)
    for ax in range(len(shape)):
        for s in (1, shape[ax] - 2):
            b = O.run(np.roll(u0, s, ax), dx, h, P, W, np.roll(V, s, ax), 3)
            assert np.array_equal(b, np.roll(a, s, ax))


@pytest.mark.parametrize("shape", [(41,), (13, 9), (7, 5, 9)])
def test_reflection_equivariance(shape):
    """x -> -x with P -> -P: k_{-P}(-d) = k_P(d) exactly (negation is exact)."""
    dx, h, P, W, u0, V = generic_problem(shape, 4)
    idx = np.ix_(*[(-np.arange(n)) % n for n in shape])
    a = O.run(u0, dx, h, P, W, V, 3)
    b = O.run(u0[idx], dx, h, tuple(-p for p in P), W, V[idx], 3)
    assert np.array_equal(b, a[idx])


def test_semigroup_time_dependent():
    """run(n+m) = run(m) after run(n), with the potential of step n at t_n (eq. uN)."""
    shape = (12, 10)
    dx, h, P, W, u0, _ = generic_problem(shape, 6)
    V = np.random.default_rng(1).normal(size=(9, *shape))
    full = O.run(u0, dx, h, P, W, V, 9, V_per_step=True)
    mid = O.run(u0, dx, h, P, W, V[:4], 4, V_per_step=True)
    rest = O.run(mid, dx, h, P, W, V[4:], 5, V_per_step=True)
    assert np.array_equal(full, rest)


# ------------------------------------------------------------------ brute force

def _product_cost(shape, dx, h, P, W):
    """Full n-D cost table C[x - y] = sum_a k_a(d_a) over the per-axis window
    (a candidate displacement vector per residue tuple), exact rationals."""
    per_axis = []
    for a, n in enumerate(shape):
        dlo, dhi = O.window(n, dx[a], h, P[a], W[a])
        per_axis.append({d % n: exact_k(d, dx[a], h, P[a]) for d in range(dlo, dhi + 1)})
    return per_axis


@pytest.mark.parametrize("shape", [(6, 5), (4, 3, 5)])
@pytest.mark.parametrize("windowed", [False, True])
def test_axis_splitting_equals_full_minimum_dyadic(shape, windowed):
    """Remark rk28: the n-D minimum over y of u(y) + sum_a k_a(x_a - y_a) equals the
    composition of 1D passes.  Exact data, so equal bit for bit."""
    W = tuple(1 for _ in shape) if windowed else None
    dx, h, P, W, u0, V = dyadic_problem(shape, 7, W=W)
    got = O.run(u0, dx, h, P, W, V, 1)
    costs = _product_cost(shape, dx, h, P, W)
    for x in itertools.product(*[range(n) for n in shape]):
        best = None
        for y in itertools.product(*[range(n) for n in shape]):
            c = Fraction(u0[y])
            ok = True
            for a in range(len(shape)):
                r = (x[a] - y[a]) % shape[a]
                if r not in costs[a]:
                    ok = False
                    break
                c += costs[a][r]
            if ok and (best is None or c < best):
                best = c
        best -= Fraction(h) * Fraction(V[x])
        assert Fraction(got[x]) == best


@pytest.mark.parametrize("shape,n", [((5,), 3), ((3, 4), 2)])
def test_optimal_path_brute_force_dyadic(shape, n):
    """eq. raslebol: T^n u(x) = min over grid paths y_0..y_n = x of
    u(y_0) + sum_i [kappa~(y_i, y_{i+1}) - h V(t_i, y_{i+1})], kappa~ minimised over
    lifts (eq. los).  All paths enumerated; time-dependent V; exact data.  The
    recorded argmins must trace an optimal path."""
    dx, h, P, W, u0, V = dyadic_problem(shape, 8, nsteps=n, per_step=True)
    got, amin = O.run(u0, dx, h, P, W, V, n, V_per_step=True, record_argmin=True)
    pts = list(itertools.product(*[range(s) for s in shape]))
    kt = [{r: lift_min_cost(shape[a], dx[a], h, P[a], r)[0] for r in range(shape[a])}
          for a in range(len(shape))]

    def kap(y, x):
        return sum(kt[a][(x[a] - y[a]) % shape[a]] for a in range(len(shape)))

    for x in pts:
        best = None
        for path in itertools.product(pts, repeat=n):
            seq = list(path) + [x]
            c = Fraction(u0[seq[0]])
            for i in range(n):
                c += kap(seq[i], seq[i + 1]) - Fraction(h) * Fraction(V[i][seq[i + 1]])
            best = c if best is None or c < best else best
        assert Fraction(got[x]) == best
        # backtrack the recorded argmins: the same cost along that path
        y = list(x)
        cost = Fraction(0)
        for i in reversed(range(n)):
            cost -= Fraction(h) * Fraction(V[i][tuple(y)])
            for a in reversed(range(len(shape))):
                d = int(amin[i, a][tuple(y)])
                cost += exact_k(d, dx[a], h, P[a])
                y[a] = (y[a] - d) % shape[a]
        cost += Fraction(u0[tuple(y)])
        assert cost == best


# ------------------------------------------------------------------ long time

def _hbar_cell_1d(P, a):
    """Effective Hamiltonian of H = (p+P)^2/2 + a cos(2 pi x) (1D cell problem):
    max V if |P| <= int sqrt(2(max V - V)), else the root of |P| = int sqrt(2(H - V))."""
    from scipy.integrate import quad
    from scipy.optimize import brentq

    def I(H):
        return quad(lambda x: np.sqrt(max(0.0, 2 * (H - a * np.cos(2 * np.pi * x)))), 0, 1,
                    limit=200)[0]
    vmax = abs(a)
    if abs(P) <= I(vmax):
        return vmax
    return brentq(lambda H: I(H) - abs(P), vmax, vmax + P * P + 1.0, xtol=1e-14)


@pytest.mark.parametrize("P,a", [(0.8, 0.1), (0.1, 0.1), (1.2, -0.3)])
def test_effective_hamiltonian_1d_converges(P, a):
    """Prop. prop:klm and the theorem after it: the discrete constant is within
    M (dx/h + h) of Hbar; refining dx and h with dx/h -> 0 shrinks the error."""
    Hb = _hbar_cell_1d(P, a)
    errs = []
    for N, h in [(128, 1 / 8), (512, 1 / 16), (2048, 1 / 32)]:
        dx = 1.0 / N
        x = np.arange(N) / N
        V = a * np.cos(2 * np.pi * x)
        W = int(np.ceil((abs(P) + 2 * np.sqrt(2 * abs(a)) + 0.5) * h / dx)) + 2
        n1 = int(round(20 / h))
        n2 = 2 * n1
        u1 = O.run(np.zeros(N), dx, h, P, W, V, n1)
        u2 = O.run(u1, dx, h, P, W, V, n2 - n1)
        est = -float(np.mean(u2 - u1)) / ((n2 - n1) * h)
        errs.append(abs(est - Hb))
        assert errs[-1] <= 0.05 * (dx / h + h)
    if errs[0] > 1e-4:      # the discretisation error dominates: it must shrink
        assert errs[-1] < errs[0] / 3


def test_weak_kam_bounded_oscillation():
    """Prop. prop:klm: u^n - n h Hbar_disc stays bounded (no linear drift)."""
    p = WL.line256(N=128)
    dx, h = p.dx, p.h
    u = p.u0.copy()
    est = None
    amps = []
    for n in (100, 200, 400, 800):
        u = O.run(p.u0, dx, h, p.P, p.W, p.V, n)
        if est is None:
            u_ref = O.run(p.u0, dx, h, p.P, p.W, p.V, 2000)
            u_ref2 = O.run(u_ref, dx, h, p.P, p.W, p.V, 1000)
            est = -float(np.mean(u_ref2 - u_ref)) / (1000 * h)
        amps.append(np.max(np.abs(u + n * h * est)))
    assert max(amps) < 1.0 and amps[-1] <= amps[0] + 0.05


# ------------------------------------------------------------------ binary32 storage

@pytest.mark.parametrize("shape", SHAPES)
def test_fp32_storage_bound(shape):
    dx, h, P, W, u0, V = generic_problem(shape, 9)
    a = O.run(u0, dx, h, P, W, V, 20)
    b = O.run(u0.astype(np.float32), dx, h, P, W, V, 20)
    assert b.dtype == np.float32
    assert np.max(np.abs(b.astype(np.float64) - a)) <= 1e-4 * (1 + np.max(np.abs(a)))


@pytest.mark.parametrize("shape", SHAPES)
def test_fp32_storage_exact_on_dyadic(shape):
    dx, h, P, W, u0, V = dyadic_problem(shape, 10)
    a = O.run(u0, dx, h, P, W, V, 3)
    b = O.run(u0.astype(np.float32), dx, h, P, W, V, 3)
    assert np.array_equal(b.astype(np.float64), a)


# ------------------------------------------------------------------ adjoint

def test_adjoint_vzero_closed_form():
    """V = 0, u0 const: loss = mean(u^n - u^0)/(n h) = sum_a kmin_a / h, so
    d loss / d P_a = -c_a dx_a / h (d k/d P = -d dx at the minimiser c_a)."""
    shape, n, h = (16, 12), 5, 0.02
    dx = (1 / 512, 1 / 512)
    P = (0.3, 0.1)
    u0 = np.zeros(shape)
    ub = np.full(shape, 1.0 / (u0.size * n * h))
    g0, gP, gV = O.adjoint(u0, dx, h, P, (0, 0), None, n, ub)
    for a, c in enumerate((3, 1)):
        assert abs(gP[a] - (-c * dx[a] / h)) <= 1e-12
    assert abs(g0.sum() - ub.sum()) <= 1e-14


@pytest.mark.parametrize("shape,W", [((15, 11), (3, 4)), ((24,), (0,)), ((5, 6, 4), (1, 0, 2))])
def test_adjoint_finite_differences(shape, W):
    """The scheme is piecewise linear in (u0, P, V) (min of sums, k linear in P);
    where no argmin changes inside the bracket, central differences are exact up
    to rounding.  Cotangent mass is conserved (each value has exactly one source)."""
    dx, h, P, _, u0, V = generic_problem(shape, 12)
    n = 4
    rng = np.random.default_rng(2)
    ub = rng.normal(size=shape)
    g0, gP, gV = O.adjoint(u0, dx, h, P, W, V, n, ub)
    assert abs(g0.sum() - ub.sum()) <= 1e-12 * np.abs(ub).sum()
    eps = 1e-6

    def J(u0_, P_, V_):
        u, am = O.run(u0_, dx, h, P_, W, V_, n, record_argmin=True)
        return float(np.sum(ub * u)), am

    _, am0 = J(u0, P, V)
    for a in range(len(shape)):
        Pp = list(P); Pp[a] += eps
        Pm = list(P); Pm[a] -= eps
        jp, amp = J(u0, tuple(Pp), V)
        jm, amm = J(u0, tuple(Pm), V)
        if np.array_equal(amp, am0) and np.array_equal(amm, am0):
            assert abs((jp - jm) / (2 * eps) - gP[a]) <= 1e-6 * (1 + abs(gP[a]))
    for idx in [tuple(0 for _ in shape), tuple(s // 2 for s in shape), tuple(s - 1 for s in shape)]:
        for arr, g in ((u0, g0), (V, gV)):
            ap, am_ = arr.copy(), arr.copy()
            ap[idx] += eps
            am_[idx] -= eps
            if arr is u0:
                jp, amp = J(ap, P, V); jm, amm = J(am_, P, V)
            else:
                jp, amp = J(u0, P, ap); jm, amm = J(u0, P, am_)
            if np.array_equal(amp, am0) and np.array_equal(amm, am0):
                assert abs((jp - jm) / (2 * eps) - g[idx]) <= 1e-6 * (1 + abs(g[idx]))


def test_tie_conventions_dyadic():
    """The paper leaves ties open (its Algorithm 1 uses a strict '<').  Convention:
    equal costs keep the larger displacement d, i.e. the smallest lifted source
    j = i - d.  Constructed exact ties (dx = 1/32, h = 1/8, so v = d/4):
      P = 1/8: k(0) = k(1) = 0 exactly -> centre c = 1, and with constant u every
               pass ties between d = 0 and d = 1 -> argmin d = 1;
      P = 1/4: the minimiser d = 1 is an integer, so for even N the two lifts
               1 - N/2 and 1 + N/2 of the antipodal residue cost the same -> the
               full window keeps 1 + N/2."""
    dx, h = 1.0 / 32, 0.125
    assert exact_k(0, dx, h, 0.125) == exact_k(1, dx, h, 0.125) == 0
    assert O.window(16, dx, h, 0.125, 3) == (1 - 3, 1 + 3)
    u0 = np.full((6, 8), 0.5)
    _, am = O.run(u0, (dx, dx), h, (0.125, 0.125), (2, 2), None, 2, record_argmin=True)
    assert np.all(am == 1)
    for N in (8, 12):
        assert exact_k(1 - N // 2, dx, h, 0.25) == exact_k(1 + N // 2, dx, h, 0.25)
        assert O.window(N, dx, h, 0.25, 0) == (1 - N // 2 + 1, 1 + N // 2)
    # odd N has no antipodal tie: the window is symmetric about the minimiser
    assert O.window(9, dx, h, 0.25, 0) == (1 - 4, 1 + 4)


@pytest.mark.parametrize("shape", [(6, 5), (4, 3, 5)])
def test_sampled_step_equals_full_minimum_dyadic(shape):
    """The point-wise evaluation (used to check large grids by sampling) is the
    same n-D minimum of Remark rk28, checked by brute force on exact data."""
    dx, h, P, W, u0, V = dyadic_problem(shape, 13, W=tuple(1 for _ in shape))
    costs = _product_cost(shape, dx, h, P, W)
    pts = np.arange(u0.size)
    got = O.step_points(u0, dx, h, P, W, V, pts)
    for q, x in enumerate(itertools.product(*[range(n) for n in shape])):
        best = None
        for y in itertools.product(*[range(n) for n in shape]):
            c = Fraction(u0[y])
            ok = True
            for a in range(len(shape)):
                r = (x[a] - y[a]) % shape[a]
                if r not in costs[a]:
                    ok = False
                    break
                c += costs[a][r]
            if ok and (best is None or c < best):
                best = c
        assert Fraction(got[q]) == best - Fraction(h) * Fraction(V[x])
