"""The paper's 1D experiments (Sec. 5) on the CPU oracle: grids, window
margins and the order-1/2 convergence that Theorem approx2 predicts with
tau = sqrt(dx) (the paper observes it against WENO5; here the reference is the
scheme on a finer nested grid)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1210_4090_gb300 import experiments as E
from paper_1210_4090_gb300 import workloads as WL


def _solve(p):
    return O.run(p.u0, p.dx, p.h, p.P, p.W, p.V, p.nsteps, V_per_step=p.V_per_step)


def test_grids_are_nested_and_end_at_T():
    for K in (4, 64, 1024):
        p = WL.pendulum(K)
        assert p.shape == (2 * K,) and abs(p.dx[0] - np.pi / K) < 1e-15
        assert abs(p.h * p.nsteps - 8.0) < 1e-12 and p.h <= np.sqrt(p.dx[0]) + 1e-15
        x = p.extra["x"]
        assert abs(x[-1] - 2 * np.pi) < 1e-12 and abs(x[0] - p.dx[0]) < 1e-15
        fine = WL.pendulum(4 * K).extra["x"]
        assert np.allclose(E.restrict(fine, 4 * K, K), x, rtol=0, atol=1e-12)
    q = WL.tdep(32)
    assert q.V.shape == (q.nsteps, 64) and q.V_per_step
    t = np.arange(q.nsteps) * q.h
    assert np.array_equal(q.V[3], np.sin(t[3]) * np.cos(2 * q.extra["x"]))


@pytest.mark.parametrize("law", ["pendulum", "tdep"])
def test_window_holds_every_argmin(law):
    """Velocities stay well inside the window (|v| <= 2.6 < 4), so the windowed
    scheme equals the full periodic one: no argmin on the window's edge."""
    p = E.LAWS[law](256)
    _, am = O.run(p.u0, p.dx, p.h, p.P, p.W, p.V, p.nsteps, V_per_step=p.V_per_step, record_argmin=True)
    dlo, dhi = O.window(p.shape[0], p.dx[0], p.h, p.P[0], p.W[0])
    assert dlo < am.min() and am.max() < dhi
    assert np.max(np.abs(am)) * p.dx[0] / p.h < 3.0


@pytest.mark.parametrize("law", ["pendulum", "tdep"])
def test_order_one_half(law):
    r = E.convergence(law, [4, 8, 16, 32, 64, 128], 1024, solve=_solve)
    err = [row["error"] for row in r["rows"]]
    assert all(b < a for a, b in zip(err, err[1:])), err
    assert 0.4 <= r["order"] <= 0.9, r["order"]


def test_pendulum_drift_is_max_V():
    """P = 0 lies in the flat part of the effective Hamiltonian of the
    pendulum (|P| <= int sqrt(2 (max V - V))), so Hbar = max V = 2 and u drifts
    like -2 t (Sec. 3, 1D cell problem)."""
    p = WL.pendulum(256)
    u = _solve(p)
    drift = -(u - p.u0) / (p.h * p.nsteps)
    assert abs(np.mean(drift) - 2.0) < 0.3
