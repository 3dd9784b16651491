"""hjlo_step_noalloc: one step without a plan and without any allocation, for
callers that cannot allocate device memory (a framework allocator that owns
all device memory, code running next to a CUDA-graph capture).  Its scratch
(kernel tables, counters, an error word) is a static device array of the
library shared by all calls.  Checked here through the C ABI against the CPU
oracle and against hjlo_step on two calls in a row (the second call must not
see the first call's scratch contents): binary64 and binary32 storage,
in place and out of place, with and without V, the monotone and the
brute-force pass, the default and a created stream.  A bounded device wait
made to run out by the test knobs is reported by hjlo_noalloc_status as
HJLO_ETIMEOUT, after which the next step is exact again.  The size limit is
checked before any device work.  This file is collected last so that a
failure here leaves every other test already run."""
import ctypes

import numpy as np
import pytest

from oracle import oracle as O

torch = pytest.importorskip("torch")

CASES = [
    # shape, dx, h, P, W
    ((48, 72), (1 / 48, 1 / 72), 0.05, (0.3, -0.2), (6, 9)),
    ((12, 20, 24), (1 / 12, 1 / 20, 1 / 24), 0.08, (0.2, -0.1, 0.35), (3, 4, 0)),
    ((400,), 1 / 400, 0.05, 0.3, 20),                 # one line: the plan runs it in row blocks, this step whole
]


def _bits(a):
    return a.view(np.int64) if a.dtype == np.float64 else a.view(np.int32)


def test_noalloc_rejects_windows_beyond_the_limit():
    from paper_1210_4090_gb300 import hjlo
    N = 20000            # full window of 20000 displacements > HJLO_NOALLOC_MAX_WINDOW
    d = hjlo.make_desc((N,), 1.0 / N, 0.1, 0.3, 0)
    st = hjlo.lib().hjlo_step_noalloc(ctypes.byref(d), None, ctypes.c_void_p(16), ctypes.c_void_p(16), None)
    assert st == 6                                   # HJLO_EUNSUPPORTED
    assert b"no-allocation limit" in hjlo.lib().hjlo_last_error()


@pytest.mark.gpu
def test_noalloc_step_matches_planned_step_twice():
    from paper_1210_4090_gb300 import hjlo
    for k, (shape, dx, h, P, W) in enumerate(CASES):
        rng = np.random.default_rng(100 + k)
        u0 = rng.normal(size=shape) * 0.4
        V = rng.normal(size=shape) * 0.3
        plan = hjlo.Plan(shape, dx, h, P, W)
        Vt = torch.tensor(V, device="cuda")
        ref = torch.tensor(u0, device="cuda")
        got = torch.tensor(u0, device="cuda")
        out = torch.empty_like(got)
        for call in range(2):
            plan.step(ref, ref, Vt)
            hjlo.step_noalloc(got, out, Vt, shape, dx, h, P, W)
            torch.cuda.synchronize()
            assert torch.equal(out, ref), (shape, call)
            got.copy_(out)
        plan.close()
    assert hjlo.noalloc_status()["error_flags"] == 0


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("variant", ["out-of-place", "in-place", "no-V", "brute", "stream"])
def test_noalloc_step_matches_oracle_twice(dtype, variant):
    """Two no-allocation steps in a row equal two steps of the oracle, bit for
    bit (binary32 storage against the oracle's binary32-storage scheme)."""
    from paper_1210_4090_gb300 import hjlo
    code = hjlo.F64 if dtype == "f64" else hjlo.F32_STORAGE
    npdt = np.float64 if dtype == "f64" else np.float32
    tdt = torch.float64 if dtype == "f64" else torch.float32
    algo = hjlo.ALGO_BRUTE if variant == "brute" else hjlo.ALGO_MONGE
    stream = torch.cuda.Stream() if variant == "stream" else None
    for k, (shape, dx, h, P, W) in enumerate(CASES):
        rng = np.random.default_rng(200 + k)
        u0 = (rng.normal(size=shape) * 0.4).astype(npdt)
        V = None if variant == "no-V" else rng.normal(size=shape) * 0.3
        Vt = None if V is None else torch.tensor(V, device="cuda")
        u = torch.tensor(u0, dtype=tdt, device="cuda")
        torch.cuda.synchronize()                # u is ready before another stream reads it
        for call in range(2):
            if variant == "in-place":
                hjlo.step_noalloc(u, u, Vt, shape, dx, h, P, W, dtype=code, algo=algo)
            else:
                out = torch.empty_like(u)
                hjlo.step_noalloc(u, out, Vt, shape, dx, h, P, W, dtype=code, algo=algo, stream=stream)
                u = out
            if stream is not None:
                stream.synchronize()
            ref = O.run(u0, dx, h, P, W, V, call + 1)
            got = u.cpu().numpy()
            assert np.array_equal(_bits(got), _bits(ref)), (shape, call, variant, dtype)
        assert hjlo.noalloc_status(stream)["error_flags"] == 0


@pytest.mark.gpu
def test_noalloc_reports_a_wait_that_ran_out(monkeypatch):
    """The test knobs make every TMA barrier of the step expect 16 bytes more
    than its copy delivers: the kernel's bounded waits run out (its copies
    land; nothing is left in flight), it raises the timeout flag in the
    scratch's error word, and hjlo_noalloc_status returns HJLO_ETIMEOUT and
    clears it.  The next step, without the knobs, is exact."""
    from paper_1210_4090_gb300 import hjlo
    shape, dx, h, P, W = (64, 96), (1 / 64, 1 / 96), 0.05, (0.3, 0.1), (8, 12)
    rng = np.random.default_rng(7)
    u0, V = rng.normal(size=shape) * 0.3, rng.normal(size=shape) * 0.2
    Vt = torch.tensor(V, device="cuda")
    try:
        hjlo.noalloc_status()                   # start from a clear error word
    except hjlo.HjloError:
        pass
    monkeypatch.setenv("HJLO_TEST_EXTRA_TX", "16")
    monkeypatch.setenv("HJLO_TEST_WAIT_NS", "1000000")
    u = torch.tensor(u0, device="cuda")
    out = torch.empty_like(u)
    hjlo.step_noalloc(u, out, Vt, shape, dx, h, P, W)
    with pytest.raises(hjlo.HjloError) as ei:
        hjlo.noalloc_status()
    assert ei.value.name == "HJLO_ETIMEOUT"
    assert hjlo.noalloc_status()["error_flags"] == 0          # read and cleared
    monkeypatch.delenv("HJLO_TEST_EXTRA_TX")
    monkeypatch.delenv("HJLO_TEST_WAIT_NS")
    hjlo.step_noalloc(u, out, Vt, shape, dx, h, P, W)
    assert hjlo.noalloc_status()["error_flags"] == 0
    assert np.array_equal(_bits(out.cpu().numpy()), _bits(O.run(u0, dx, h, P, W, V, 1)))
