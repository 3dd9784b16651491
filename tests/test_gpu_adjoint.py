"""Reverse mode (hjlo_adjoint) vs the CPU oracle's adjoint and finite differences.

dJ/du0 and dJ/dV are summed in the definition's order (ascending target per
source, reverse steps), so they must equal the oracle's bit for bit; dJ/dP is
a global sum in another order (rtol 1e-11).  Cases: 1D/2D/3D, windowed and
full windows, contiguous axes in row blocks, several checkpoint intervals,
the adjoint512 law on a 64^2 copy with the 64 coefficient gradients,
|u| ~ 1e14 (non-monotone argmins take the sequential path), finite
differences through the forward kernels, and the torch.autograd binding.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1210_4090_gb300 import workloads as WL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _case(shape, seed, W, offset=0.0):
    rng = np.random.default_rng(seed)
    dx = tuple(1.0 / n for n in shape)
    P = tuple(float(x) for x in rng.uniform(-0.7, 0.7, len(shape)))
    u0 = rng.normal(size=shape) * 0.3 + offset
    V = rng.normal(size=shape) * 0.2
    ub = rng.normal(size=shape)
    return dx, 0.07, P, W, u0, V, ub


def _gpu_adjoint(shape, dx, h, P, W, u0, V, n, ub, S):
    from paper_1210_4090_gb300 import hjlo
    plan = hjlo.Plan(shape, dx, h, P, W)
    t = lambda a: torch.tensor(a, device="cuda")
    g0, gP, gV, un = plan.adjoint(t(u0), None if V is None else t(V), n, t(ub), S, want_un=True)
    cnt = plan.sync()
    return g0.cpu().numpy(), gP.cpu().numpy(), None if gV is None else gV.cpu().numpy(), un.cpu().numpy(), cnt


# the last two run their contiguous axis in row blocks (one or three lines)
CASES = [((40,), (0,), 9), ((24, 30), (4, 5), 7), ((9, 10, 12), (2, 0, 3), 5), ((33, 18), (0, 3), 6),
         ((300,), (12,), 6), ((3, 200), (1, 10), 5)]


@pytest.mark.parametrize("shape,W,n", CASES, ids=lambda c: str(c))
@pytest.mark.parametrize("S", [0, 1, 3])
def test_adjoint_matches_oracle(shape, W, n, S):
    dx, h, P, W, u0, V, ub = _case(shape, 7, W)
    g0, gP, gV, un, _ = _gpu_adjoint(shape, dx, h, P, W, u0, V, n, ub, S)
    r0, rP, rV = O.adjoint(u0, dx, h, P, W, V, n, ub)
    assert np.array_equal(un.view(np.int64), O.run(u0, dx, h, P, W, V, n).view(np.int64))
    assert np.array_equal(g0.view(np.int64), r0.view(np.int64))
    assert np.array_equal(gV.view(np.int64), rV.view(np.int64))
    assert np.allclose(gP, rP, rtol=1e-11, atol=1e-12 * np.abs(ub).sum())


def test_adjoint_without_potential_and_huge_values():
    shape, W, n = (20, 28), (3, 4), 4
    dx, h, P, W, u0, V, ub = _case(shape, 9, W, offset=1e14)
    g0, gP, gV, _, cnt = _gpu_adjoint(shape, dx, h, P, W, u0, None, n, ub, 2)
    r0, rP, rV = O.adjoint(u0, dx, h, P, W, None, n, ub)
    assert cnt["brute_fallback_lines"] > 0
    assert np.array_equal(g0.view(np.int64), r0.view(np.int64))
    assert np.allclose(gP, rP, rtol=1e-11, atol=1e-12 * np.abs(ub).sum())


def test_adjoint512_law_on_64_copy_with_coefficients():
    """The adjoint workload's law (64 learnable coefficients, loss =
    mean (u^n - u^0)/(n h)) on a 64^2 copy with checkpoints, against the CPU
    adjoint; coefficient gradients through hjlo_project."""
    from paper_1210_4090_gb300 import hjlo
    p = WL.adjoint512(N=64, nsteps=120, W=4)
    n, S = p.nsteps, 25
    ub = np.full(p.shape, 1.0 / (p.npts * n * p.h))
    plan = hjlo.Plan(p.shape, p.dx, p.h, p.P, p.W)
    t = lambda a: torch.tensor(a, device="cuda")
    g0, gP, gV, _ = plan.adjoint(t(p.u0), t(p.V), n, t(ub), S)
    r0, rP, rV = O.adjoint(p.u0, p.dx, p.h, p.P, p.W, p.V, n, ub)
    assert np.array_equal(g0.cpu().numpy().view(np.int64), r0.view(np.int64))
    assert np.array_equal(gV.cpu().numpy().view(np.int64), rV.view(np.int64))
    assert np.allclose(gP.cpu().numpy(), rP, rtol=1e-11, atol=1e-14)
    B = WL.adjoint_basis(64)
    gc = plan.project(gV, t(B)).cpu().numpy()
    want = np.tensordot(B, rV, axes=([1, 2], [0, 1]))
    assert np.allclose(gc, want, rtol=1e-12, atol=1e-15)


def test_adjoint_finite_differences_on_gpu():
    """Central differences of J = <ubar, u^n> through the forward kernels; the
    scheme is piecewise linear in (P, V), so where no argmin changes in the
    bracket the difference quotient equals the gradient up to rounding."""
    from paper_1210_4090_gb300 import hjlo
    shape, W, n = (32, 40), (4, 5), 6
    dx, h, P, W, u0, V, ub = _case(shape, 21, W)
    g0, gP, gV, _, _ = _gpu_adjoint(shape, dx, h, P, W, u0, V, n, ub, 0)
    eps = 1e-6

    def J(P_, V_):
        plan = hjlo.Plan(shape, dx, h, P_, W)
        u = torch.tensor(u0, device="cuda")
        ams = []
        for _ in range(n):
            a = torch.empty(len(shape) * u.numel(), dtype=torch.int32, device="cuda")
            plan.step(u, u, torch.tensor(V_, device="cuda"), argmin=a)
            ams.append(a.cpu().numpy())
        return float(np.sum(ub * u.cpu().numpy())), np.concatenate(ams)

    _, am0 = J(P, V)
    checked = 0
    for a in range(len(shape)):
        Pp = list(P); Pp[a] += eps
        Pm = list(P); Pm[a] -= eps
        jp, amp = J(Pp, V)
        jm, amm = J(Pm, V)
        if np.array_equal(amp, am0) and np.array_equal(amm, am0):
            assert abs((jp - jm) / (2 * eps) - gP[a]) <= 1e-6 * (1 + abs(gP[a]))
            checked += 1
    for idx in [(0, 0), (13, 17), (31, 39)]:
        Vp, Vm = V.copy(), V.copy()
        Vp[idx] += eps
        Vm[idx] -= eps
        jp, amp = J(P, Vp)
        jm, amm = J(P, Vm)
        if np.array_equal(amp, am0) and np.array_equal(amm, am0):
            assert abs((jp - jm) / (2 * eps) - gV[idx]) <= 1e-6 * (1 + abs(gV[idx]))
            checked += 1
    assert checked >= 2


def test_autograd_function():
    from paper_1210_4090_gb300.autograd import LaxOleinik, Spec
    shape, W, n = (20, 24), (3, 3), 5
    dx, h, P, W, u0, V, ub = _case(shape, 4, W)
    spec = Spec(shape, dx, h, W, n, 2)
    u0t = torch.tensor(u0, device="cuda", requires_grad=True)
    Pt = torch.tensor(P, dtype=torch.float64, requires_grad=True)
    Vt = torch.tensor(V, device="cuda", requires_grad=True)
    un = LaxOleinik.apply(u0t, Pt, Vt, spec)
    (un * torch.tensor(ub, device="cuda")).sum().backward()
    r0, rP, rV = O.adjoint(u0, dx, h, P, W, V, n, ub)
    assert np.array_equal(u0t.grad.cpu().numpy(), r0)
    assert np.array_equal(Vt.grad.cpu().numpy(), rV)
    assert np.allclose(Pt.grad.numpy(), rP, rtol=1e-11)
