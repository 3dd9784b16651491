"""The paper's 1D experiments (Sec. 5) through the CUDA path: bit-exact
against the oracle (static V through hjlo_run, the time-dependent V through
hjlo_run_tv, one row per step) and the order-1/2 convergence at sizes the
oracle would take minutes for."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1210_4090_gb300 import experiments as E

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("law", ["pendulum", "tdep"])
@pytest.mark.parametrize("K", [2, 8, 64, 512])
def test_bitwise_vs_oracle(law, K):
    p = E.LAWS[law](K)
    ref = O.run(p.u0, p.dx, p.h, p.P, p.W, p.V, p.nsteps, V_per_step=p.V_per_step)
    got = E.solve_gpu(p)
    assert np.array_equal(got.view(np.int64), ref.view(np.int64))


def test_long_line_runs_in_row_blocks():
    """2 x 8192 points on one line: the monotone search runs it as blocks of
    rows spread over the GPU (a whole line would not fit one CTA's shared
    memory), still exact."""
    from paper_1210_4090_gb300 import hjlo
    p = E.LAWS["tdep"](8192)
    n = 4
    plan = hjlo.Plan(p.shape, p.dx, p.h, p.P, p.W)
    info = plan.info()
    assert info["algo"] == "monge" and info["row_blocks"][0] > 1, info
    u = torch.tensor(p.u0, device="cuda")
    plan.run_tv(u, torch.tensor(p.V[:n], device="cuda"), n)
    plan.close()
    ref = O.run(p.u0, p.dx, p.h, p.P, p.W, p.V[:n], n, V_per_step=True)
    assert np.array_equal(u.cpu().numpy().view(np.int64), ref.view(np.int64))


def test_paper_size_pendulum_line():
    """The paper's largest run (Sec. 5.1 footnote): 2^18 points, tau = sqrt(dx),
    one line in row blocks; the first steps bit-exact against the oracle."""
    from paper_1210_4090_gb300 import hjlo
    p = E.LAWS["pendulum"](2 ** 17)
    n = 2
    plan = hjlo.Plan(p.shape, p.dx, p.h, p.P, p.W)
    info = plan.info()
    assert info["algo"] == "monge" and info["row_blocks"][0] > 1, info
    u = torch.tensor(p.u0, device="cuda")
    plan.run(u, torch.tensor(p.V, device="cuda"), n)
    cnt = plan.sync()
    plan.close()
    assert cnt["error_flags"] == 0 and cnt["window_edge_hits"] == 0
    ref = O.run(p.u0, p.dx, p.h, p.P, p.W, p.V, n)
    assert np.array_equal(u.cpu().numpy().view(np.int64), ref.view(np.int64))


@pytest.mark.parametrize("law", ["pendulum", "tdep"])
def test_order_one_half_on_gpu(law):
    r = E.convergence(law, [16, 32, 64, 128, 256, 512, 1024], 4096)
    err = [row["error"] for row in r["rows"]]
    assert all(b < a for a, b in zip(err, err[1:])), err
    assert 0.4 <= r["order"] <= 0.9, r["order"]


@pytest.mark.parametrize("shape,dx,h,P,W", [
    ((12,), 1 / 12, 0.05, -0.7, 3),
    ((6, 7), (1 / 6, 1 / 7), 0.07, (0.4, -0.2), (0, 2)),
    ((3, 4, 5), (1 / 3, 1 / 4, 1 / 5), 0.1, (0.2, 0.5, -0.3), (0, 0, 0)),
])
def test_hbar_readout_matches_minplus_eigenvalue(shape, dx, h, P, W):
    """The GPU's long-run Hbar readout (hjlo_hbar over a late window of steps)
    equals -lambda/h, lambda the (min,plus) eigenvalue of the one-step matrix
    (Karp's minimum cycle mean on the CPU)."""
    from paper_1210_4090_gb300 import hjlo
    rng = np.random.default_rng(11)
    u0 = rng.normal(size=shape) * 0.3
    V = rng.normal(size=shape) * 0.3
    lam = O.minplus_eigenvalue(O.step_matrix(shape, dx, h, P, W, V))
    plan = hjlo.Plan(shape, dx, h, P, W)
    u = torch.tensor(u0, device="cuda")
    Vt = torch.tensor(V, device="cuda")
    plan.run(u, Vt, 400)
    u1 = u.clone()
    plan.run(u, Vt, 800)
    est = plan.hbar(u1, u, 800)
    plan.close()
    assert abs(est[0] - (-lam / h)) < 1e-8 * (1 + abs(lam / h))
    assert abs(est[1] - est[2]) < 1e-8 * (1 + abs(lam / h))
