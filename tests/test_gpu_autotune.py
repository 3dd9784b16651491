"""The launch-shape autotuner (hjlo_plan_autotune / hjlo_batch_autotune):
tuning leaves the caller's data untouched, reports a valid choice, and the
tuned plan or batch is still bit-exact against the oracle (results never
depend on the launch shape)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1210_4090_gb300 import workloads as WL

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("wl,kw,n", [
    ("grid1024", {"N": 192, "W": 16}, 12),
    ("cube256", {"N": 40, "W": 5}, 6),
])
def test_plan_autotune_keeps_exactness(wl, kw, n):
    from paper_1210_4090_gb300 import hjlo
    p = WL.WORKLOADS[wl](nsteps=n, **kw)
    plan = hjlo.Plan(p.shape, p.dx, p.h, p.P, p.W)
    u = torch.tensor(p.u0, device="cuda")
    Vt = torch.tensor(p.V, device="cuda")
    before = u.clone()
    rep = plan.autotune(u, Vt, 4)
    assert torch.equal(u, before)
    assert rep["trials"] >= 1 and rep["ms_tuned"] > 0 and rep["ms_initial"] > 0
    for a in range(len(p.shape)):
        lpl, C = rep["lanes_per_line"][a], rep["lines_per_tile"][a]
        assert lpl >= 1 and (lpl & (lpl - 1)) == 0 and lpl <= p.shape[a]
        assert C >= 1 and (C & (C - 1)) == 0
    plan.run(u, Vt, n)                    # > 16 steps would use the rebuilt graph; both paths are covered below
    plan.run(u, Vt, 40)
    ref = O.run(p.u0, p.dx, p.h, p.P, p.W, p.V, n + 40)
    assert np.array_equal(u.cpu().numpy().view(np.int64), ref.view(np.int64))
    assert plan.sync()["error_flags"] == 0
    plan.close()


def test_batch_autotune_keeps_exactness():
    from paper_1210_4090_gb300 import hjlo
    probs = WL.sweep512(count=6, nsteps=10, sizes=(48, 64, 96), first=60)
    b = hjlo.Batch([(p.shape, p.dx, p.h, p.P, p.W) for p in probs])
    us = [torch.tensor(p.u0 + 0.01 * np.arange(p.u0.size).reshape(p.u0.shape) / p.u0.size, device="cuda")
          for p in probs]
    Vs = [torch.tensor(p.V, device="cuda") for p in probs]
    keep = [u.clone() for u in us]
    rep = b.autotune(us, Vs, 3)
    assert all(torch.equal(u, k) for u, k in zip(us, keep))
    assert rep["trials"] >= 1
    b.run(us, Vs, 10)
    cnt = b.sync()
    assert cnt["steps"] == 10 and cnt["error_flags"] == 0
    for p, u, k in zip(probs, us, keep):
        ref = O.run(k.cpu().numpy(), p.dx, p.h, p.P, p.W, p.V, 10)
        assert np.array_equal(u.cpu().numpy().view(np.int64), ref.view(np.int64))
    b.close()


def test_autotune_binary32_storage():
    """Tuning a binary32-storage plan keeps it bit-exact against the oracle's
    binary32-storage scheme."""
    from paper_1210_4090_gb300 import hjlo
    p = WL.grid1024(N=160, nsteps=20, W=12)
    u0 = p.u0.astype(np.float32)
    plan = hjlo.Plan(p.shape, p.dx, p.h, p.P, p.W, dtype=hjlo.F32_STORAGE)
    u = torch.tensor(u0, device="cuda")
    Vt = torch.tensor(p.V, device="cuda")
    rep = plan.autotune(u, Vt, 4)
    assert rep["trials"] >= 1
    plan.run(u, Vt, 20)
    ref = O.run(u0, p.dx, p.h, p.P, p.W, p.V, 20)
    assert np.array_equal(u.cpu().numpy().view(np.int32), ref.view(np.int32))
    plan.close()


def test_autotune_row_blocks():
    """A single 1D line in row blocks: the tuner also varies the rows per
    block; whatever it keeps, the run stays bit-exact, the counters are the
    run's own (trials leave them untouched) and the data is untouched."""
    from paper_1210_4090_gb300 import hjlo
    from edge_counts import edge_hits
    N, W, h, P, n = 20000, 30, 1e-4, 0.2, 3
    x = np.arange(N) / N
    rng = np.random.default_rng(12)
    u0 = 0.3 * np.sin(6 * np.pi * x) + 0.01 * rng.normal(size=N)
    V = 0.2 * np.cos(4 * np.pi * x)
    plan = hjlo.Plan((N,), 1.0 / N, h, P, W)
    assert plan.info()["row_blocks"][0] > 1
    u = torch.tensor(u0, device="cuda")
    Vt = torch.tensor(V, device="cuda")
    before = u.clone()
    rep = plan.autotune(u, Vt, 4)
    assert torch.equal(u, before) and rep["trials"] >= 3
    assert plan.info()["row_blocks"][0] > 1
    plan.run(u, Vt, n)
    cnt = plan.sync()
    plan.close()
    ref = O.run(u0, 1.0 / N, h, P, W, V, n)
    assert np.array_equal(u.cpu().numpy().view(np.int64), ref.view(np.int64))
    assert cnt["steps"] == n and cnt["window_edge_hits"] == edge_hits(u0, 1.0 / N, h, P, W, V, n)
