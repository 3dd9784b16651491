"""hjlo_step_noalloc: one step without a plan and without any allocation, for
callers that cannot allocate device memory (a framework allocator that owns
all device memory, code running next to a CUDA-graph capture).  Its scratch
(kernel tables, counters) is a static device array of the library shared by
all calls.  Checked here against hjlo_step through the C ABI on two calls in
a row (the second call must not see the first call's scratch contents), and
the size limit is checked before any device work.  This file is collected
last so that a failure here leaves every other test already run."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

CASES = [
    # shape, dx, h, P, W
    ((48, 72), (1 / 48, 1 / 72), 0.05, (0.3, -0.2), (6, 9)),
    ((12, 20, 24), (1 / 12, 1 / 20, 1 / 24), 0.08, (0.2, -0.1, 0.35), (3, 4, 0)),
    ((400,), 1 / 400, 0.05, 0.3, 20),                 # one line: the plan runs it in row blocks, this step whole
]


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
