"""Batched grids (hjlo_batch_*) vs the CPU oracle, instance by instance.

Instances of the sweep law (P ~ U([-1,1]^2), random trig potentials, W = N/16)
at sizes the oracle runs in seconds, several launch groups (different N and
windows), step counts that exercise both captured graphs (8 steps and 1 step),
repeated runs on new tensors, binary32 storage and 3D grids.  Every instance
must equal the oracle bit for bit; the per-instance Hbar readout matches the
oracle's to rounding.
"""
import ctypes

import numpy as np
import pytest

from oracle import oracle as O
from paper_1210_4090_gb300 import workloads as WL


def _torch():
    return pytest.importorskip("torch")


def _problems(count, sizes=(48, 64, 80), nsteps=20, first=0):
    return WL.sweep512(count=count, nsteps=nsteps, sizes=sizes, first=first)


def _run_batch(probs, nsteps, dtype="f64", algo=0):
    torch = _torch()
    from paper_1210_4090_gb300 import hjlo
    code = hjlo.F64 if dtype == "f64" else hjlo.F32_STORAGE
    tdt = torch.float64 if dtype == "f64" else torch.float32
    b = hjlo.Batch([(p.shape, p.dx, p.h, p.P, p.W) for p in probs], dtype=code, algo=algo)
    us = [torch.tensor(p.u0, dtype=tdt, device="cuda") for p in probs]
    Vs = [torch.tensor(p.V, device="cuda") for p in probs]
    b.run(us, Vs, nsteps)
    cnt = b.sync()
    return b, us, Vs, cnt


@pytest.mark.gpu
@pytest.mark.parametrize("algo", [1, 2], ids=["brute", "monge"])
def test_batch_bitwise_vs_oracle(algo):
    from edge_counts import edge_hits
    probs = _problems(12)
    b, us, _, cnt = _run_batch(probs, 20, algo=algo)
    assert b.groups() >= 2 and cnt["error_flags"] == 0 and cnt["steps"] == 20
    for p, u in zip(probs, us):
        ref = O.run(p.u0, p.dx, p.h, p.P, p.W, p.V, 20)
        assert np.array_equal(u.cpu().numpy().view(np.int64), ref.view(np.int64)), p.name
    # window-edge argmins, all instances together
    assert cnt["window_edge_hits"] == sum(edge_hits(p.u0, p.dx, p.h, p.P, p.W, p.V, 20) for p in probs)
    b.close()


@pytest.mark.gpu
def test_batch_repeat_runs_new_tensors_and_hbar():
    torch = _torch()
    from paper_1210_4090_gb300 import hjlo
    probs = _problems(7, sizes=(32, 56), first=20)
    b = hjlo.Batch([(p.shape, p.dx, p.h, p.P, p.W) for p in probs])
    for rep, n in enumerate((5, 11)):
        us = [torch.tensor(p.u0 + rep, device="cuda") for p in probs]
        u0s = [u.clone() for u in us]
        Vs = [torch.tensor(p.V, device="cuda") for p in probs]
        b.run(us, Vs, n)
        hb = b.hbar(u0s, us, n)
        for k, (p, u) in enumerate(zip(probs, us)):
            ref = O.run(p.u0 + rep, p.dx, p.h, p.P, p.W, p.V, n)
            assert np.array_equal(u.cpu().numpy().view(np.int64), ref.view(np.int64))
            want = O.hbar_estimate(p.u0 + rep, ref, n, p.h)
            assert np.allclose(hb[k], want, rtol=1e-12, atol=1e-14)
    b.close()


@pytest.mark.gpu
def test_batch_f32_storage():
    probs = _problems(6, sizes=(40, 64), first=40)
    for p in probs:
        p.u0 = p.u0.astype(np.float32)
    b, us, _, _ = _run_batch(probs, 9, dtype="f32")
    for p, u in zip(probs, us):
        ref = O.run(p.u0, p.dx, p.h, p.P, p.W, p.V, 9)
        assert np.array_equal(u.cpu().numpy().view(np.int32), ref.view(np.int32))
    b.close()


@pytest.mark.gpu
def test_batch_3d_and_mixed_windows():
    torch = _torch()
    from paper_1210_4090_gb300 import hjlo
    rng = np.random.default_rng(3)
    probs = []
    for i, (shape, W) in enumerate([((10, 12, 16), (2, 3, 4)), ((10, 12, 16), (2, 3, 4)),
                                    ((8, 8, 8), (0, 0, 0)), ((10, 12, 16), (1, 1, 1))]):
        dx = tuple(1.0 / n for n in shape)
        P = tuple(rng.uniform(-0.7, 0.7, 3))
        probs.append((shape, dx, 0.06, P, W, rng.normal(size=shape) * 0.3, rng.normal(size=shape) * 0.2))
    b = hjlo.Batch([q[:5] for q in probs])
    assert b.groups() == 3
    us = [torch.tensor(q[5], device="cuda") for q in probs]
    Vs = [torch.tensor(q[6], device="cuda") for q in probs]
    Vs[1] = None
    b.run(us, Vs, 6)
    for k, (q, u) in enumerate(zip(probs, us)):
        ref = O.run(q[5], q[1], q[2], q[3], q[4], None if k == 1 else q[6], 6)
        assert np.array_equal(u.cpu().numpy().view(np.int64), ref.view(np.int64))
    b.close()


def test_batch_rejects_mixed_ndim_before_device_work():
    from paper_1210_4090_gb300 import hjlo
    descs = (hjlo.Desc * 2)()
    descs[0] = hjlo.make_desc((8, 8), 0.125, 0.1, (0.1, 0.2), (2, 2))
    descs[1] = hjlo.make_desc((8,), 0.125, 0.1, 0.1, 2)
    out = ctypes.c_void_p()
    assert hjlo.lib().hjlo_batch_create(descs, 2, None, ctypes.byref(out)) == 1
    assert hjlo.lib().hjlo_batch_create(descs, 0, None, ctypes.byref(out)) == 1
    assert hjlo.lib().hjlo_batch_destroy(None) == 0
