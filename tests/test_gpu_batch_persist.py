"""The persistent batched pass (hjlo_batch_set_persistent): every instance
of a batch advanced by one launch per time step whose CTAs take tiles from a
device queue, a pass of axis a >= 1 waiting on its instance's axis a - 1
tile counter.  Bit for bit against the CPU oracle instance by instance (several
launch groups, 2D and 3D, binary64 and binary32 storage, step counts through
both captured graphs, modes switched between runs), and the bounded
dependency wait made to run out by a test knob reported as HJLO_ETIMEOUT."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1210_4090_gb300 import workloads as WL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _bits(a):
    return a.view(np.int64) if a.dtype == np.float64 else a.view(np.int32)


def _batch(probs, dtype="f64", persistent=True, algo=2):
    from paper_1210_4090_gb300 import hjlo
    code = hjlo.F64 if dtype == "f64" else hjlo.F32_STORAGE
    tdt = torch.float64 if dtype == "f64" else torch.float32
    b = hjlo.Batch([(p.shape, p.dx, p.h, p.P, p.W) for p in probs], dtype=code, algo=algo)
    if persistent:
        b.set_persistent(True)
    us = [torch.tensor(p.u0, dtype=tdt, device="cuda") for p in probs]
    Vs = [torch.tensor(p.V, device="cuda") for p in probs]
    return b, us, Vs


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_persistent_bitwise_vs_oracle(dtype):
    probs = WL.sweep512(count=12, nsteps=19, sizes=(48, 64, 80))
    b, us, Vs = _batch(probs, dtype)
    b.run(us, Vs, 19)                  # two 8-step graphs and three single steps
    cnt = b.sync()
    assert b.groups() >= 2 and cnt["error_flags"] == 0
    for p, u in zip(probs, us):
        u0 = p.u0 if dtype == "f64" else p.u0.astype(np.float32)
        ref = O.run(u0, p.dx, p.h, p.P, p.W, p.V, 19)
        assert np.array_equal(_bits(u.cpu().numpy()), _bits(ref)), p.name
    b.close()


def test_persistent_3d_and_mode_switch():
    """3D instances of two sizes: 8 steps grouped, then 7 persistent on the
    same tensors, then 2 grouped again; equal to the oracle's 17 steps."""
    rng = np.random.default_rng(3)
    probs = []
    for i, N in enumerate((12, 16, 12, 20)):
        p = WL.cube256(N=N, nsteps=17, W=2 + i % 2, seed=30 + i)
        p.u0 = rng.normal(size=p.shape) * 0.2
        probs.append(p)
    b, us, Vs = _batch(probs, persistent=False)
    b.run(us, Vs, 8)
    b.set_persistent(True)
    b.run(us, Vs, 7)
    b.set_persistent(False)
    b.run(us, Vs, 2)
    assert b.sync()["error_flags"] == 0
    for p, u in zip(probs, us):
        assert np.array_equal(_bits(u.cpu().numpy()), _bits(O.run(p.u0, p.dx, p.h, p.P, p.W, p.V, 17))), p.name
    b.close()


def test_persistent_refused_with_brute_force():
    from paper_1210_4090_gb300 import hjlo
    probs = WL.sweep512(count=3, nsteps=2, sizes=(32,))
    b = hjlo.Batch([(p.shape, p.dx, p.h, p.P, p.W) for p in probs], algo=hjlo.ALGO_BRUTE)
    with pytest.raises(hjlo.HjloError) as e:
        b.set_persistent(True)
    assert e.value.status == 6
    b.close()


def test_persistent_dependency_wait_runs_out(monkeypatch):
    """HJLO_TEST_EXTRA_DEP makes every dependency wait expect one tile more
    than the previous pass has: the first wait gives up after
    HJLO_TEST_WAIT_NS, raises the timeout flag, every later wait sees it and
    skips, and the launch ends.  hjlo_batch_sync reports HJLO_ETIMEOUT; a new
    batch without the knob is exact."""
    from paper_1210_4090_gb300 import hjlo
    probs = WL.sweep512(count=6, nsteps=3, sizes=(48, 64))
    monkeypatch.setenv("HJLO_TEST_EXTRA_DEP", "1")
    monkeypatch.setenv("HJLO_TEST_WAIT_NS", "2000000")
    b, us, Vs = _batch(probs)
    b.run(us, Vs, 1)
    with pytest.raises(hjlo.HjloError) as e:
        b.sync()
    assert e.value.name == "HJLO_ETIMEOUT"
    b.close()
    monkeypatch.delenv("HJLO_TEST_EXTRA_DEP")
    monkeypatch.delenv("HJLO_TEST_WAIT_NS")
    b, us, Vs = _batch(probs)
    b.run(us, Vs, 3)
    assert b.sync()["error_flags"] == 0
    for p, u in zip(probs, us):
        assert np.array_equal(_bits(u.cpu().numpy()), _bits(O.run(p.u0, p.dx, p.h, p.P, p.W, p.V, 3)))
    b.close()
