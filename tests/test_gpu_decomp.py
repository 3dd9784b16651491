"""The paper's own fast convolution (Sec. 4, HJLO_ALGO_DECOMP) on the GPU
against the oracle's version of the same method: bit for bit (every output is
the same candidate minimum over the same components) and the same number of
components; on exact dyadic data also equal to the scheme itself."""
import ctypes

import numpy as np
import pytest

from oracle import oracle as O
from paper_1210_4090_gb300 import workloads as WL

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _hjlo():
    from paper_1210_4090_gb300 import hjlo
    return hjlo


def gpu_decomp(shape, dx, h, P, W, u0, V, nsteps, eta=0.0, V_per_step=False, facts=None):
    """Runs the decomposition pass; `facts`, a dict, receives the plan's facts
    (the rows per block of a contiguous axis in row blocks: the oracle must
    restart its decomposition at the same sources)."""
    H = _hjlo()
    plan = H.Plan(shape, dx, h, P, W, algo=H.ALGO_DECOMP)
    info = plan.info()
    assert info["algo"] == "decomp"
    if facts is not None:
        facts.update(info)
    if eta:
        plan.set_tolerance(eta)
    u = torch.tensor(u0, device="cuda")
    Vt = None if V is None else torch.tensor(V, device="cuda")
    if V_per_step:
        plan.run_tv(u, Vt, nsteps)
    else:
        plan.run(u, Vt, nsteps)
    cnt = plan.sync()
    plan.close()
    return u.cpu().numpy(), cnt


CASES = [
    ("1d-w", (200,), 1 / 200, 0.05, 0.4, 20),
    ("1d-full", (60,), 1 / 60, 0.1, -0.3, 0),
    ("1d-n1", (1,), 1.0, 0.1, 0.2, 0),
    ("1d-n2", (2,), 0.5, 0.1, 0.2, 0),
    ("2d", (24, 40), (1 / 24, 1 / 40), 0.06, (0.4, -0.2), (4, 6)),
    ("3d", (6, 8, 12), (1 / 6, 1 / 8, 1 / 12), 0.08, (0.3, -0.1, 0.5), (0, 2, 3)),
]


@pytest.mark.parametrize("eta", [0.0, 1e-4, 1e-2])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_bitwise_vs_oracle_method(case, eta):
    name, shape, dx, h, P, W = case
    rng = np.random.default_rng(len(name) * 7 + int(eta * 1e4))
    u0 = np.cumsum(rng.normal(size=shape), axis=-1) * 0.03
    V = rng.normal(size=shape) * 0.2
    n = 3
    facts = {}
    got, cnt = gpu_decomp(shape, dx, h, P, W, u0, V, n, eta, facts=facts)
    ref, ncomp = O.decomp_run(u0, dx, h, P, W, V, n, eta, block_rows=facts["block_rows"][-1])
    assert cnt["error_flags"] == 0
    assert np.array_equal(got.view(np.int64), ref.view(np.int64))
    assert cnt["components"] == ncomp


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_dyadic_equals_scheme(case):
    name, shape, dx, h, P, W = case
    dx = tuple(1 / 32 for _ in shape) if len(shape) > 1 else 1 / 32
    h, P = 0.125, (tuple(0.25 * (-1) ** a for a in range(len(shape))) if len(shape) > 1 else 0.25)
    rng = np.random.default_rng(2)
    u0 = rng.integers(-2048, 2048, size=shape) / 1024.0
    V = rng.integers(-256, 256, size=shape) / 256.0
    ref = O.run(u0, dx, h, P, W, V, 4)
    got, _ = gpu_decomp(shape, dx, h, P, W, u0, V, 4)
    assert np.array_equal(got.view(np.int64), ref.view(np.int64))


def test_graph_path_and_tolerance_change():
    """40 steps go through the captured graph; changing eta rebuilds it."""
    H = _hjlo()
    shape, dx, h, P, W = (96,), 1 / 96, 0.05, 0.3, 10
    rng = np.random.default_rng(4)
    u0 = np.cumsum(rng.normal(size=shape)) * 0.02
    V = rng.normal(size=shape) * 0.1
    plan = H.Plan(shape, dx, h, P, W, algo=H.ALGO_DECOMP)
    R = plan.info()["block_rows"][0]
    Vt = torch.tensor(V, device="cuda")
    for eta in (0.0, 5e-3, 0.0):
        plan.set_tolerance(eta)
        u = torch.tensor(u0, device="cuda")
        plan.run(u, Vt, 40)
        ref, _ = O.decomp_run(u0, dx, h, P, W, V, 40, eta, block_rows=R)
        assert np.array_equal(u.cpu().numpy().view(np.int64), ref.view(np.int64)), eta
    plan.close()


def test_paper_law_time_dependent():
    p = WL.tdep(32)
    ref, _ = O.decomp_run(p.u0, p.dx, p.h, p.P, p.W, p.V, p.nsteps, 0.0, V_per_step=True)
    got, _ = gpu_decomp(p.shape, p.dx, p.h, p.P, p.W, p.u0, p.V, p.nsteps, V_per_step=True)
    assert np.array_equal(got.view(np.int64), ref.view(np.int64))


def test_unsupported_uses_are_errors():
    H = _hjlo()
    d = H.make_desc((16,), 1 / 16, 0.1, 0.2, 3, dtype=H.F32_STORAGE, algo=H.ALGO_DECOMP)
    out = ctypes.c_void_p()
    assert H.lib().hjlo_plan_create(ctypes.byref(d), None, ctypes.byref(out)) == 6      # EUNSUPPORTED
    plan = H.Plan((16,), 1 / 16, 0.1, 0.2, 3, algo=H.ALGO_DECOMP)
    u = torch.zeros(16, dtype=torch.float64, device="cuda")
    am = torch.empty(16, dtype=torch.int32, device="cuda")
    with pytest.raises(H.HjloError):
        plan.step(u, u, None, argmin=am)
    with pytest.raises(H.HjloError):
        plan.set_tolerance(-1.0)
    plan.close()
    mono = H.Plan((16,), 1 / 16, 0.1, 0.2, 3, algo=H.ALGO_MONGE)
    with pytest.raises(H.HjloError):
        mono.set_tolerance(0.1)
    mono.close()


@pytest.mark.parametrize("eta", [0.0, 1.0, 10.0])
def test_row_blocks(eta):
    """A single long line in row blocks: each block is decomposed on its own
    span.  Bit for bit against the oracle's method restarted at the same
    blocks, the same number of components, and at eta = 0 equal to the
    scheme itself."""
    N, W, h, P, n = 12000, 40, 2e-3, 0.3, 4
    x = np.arange(N) / N
    rng = np.random.default_rng(13)
    u0 = 0.3 * np.sin(6 * np.pi * x) + 0.01 * np.cumsum(rng.normal(size=N)) / np.sqrt(N)
    V = 0.2 * np.cos(4 * np.pi * x)
    facts = {}
    got, cnt = gpu_decomp((N,), 1.0 / N, h, P, W, u0, V, n, eta, facts=facts)
    assert facts["row_blocks"][0] > 1 and cnt["error_flags"] == 0
    ref, ncomp = O.decomp_run(u0, 1.0 / N, h, P, W, V, n, eta, block_rows=facts["block_rows"][0])
    assert np.array_equal(got.view(np.int64), ref.view(np.int64))
    assert cnt["components"] == ncomp
    if eta == 0.0:
        assert np.array_equal(got.view(np.int64), O.run(u0, 1.0 / N, h, P, W, V, n).view(np.int64))


@pytest.mark.parametrize("eta", [0.0, 1.0])
def test_long_components_by_the_whole_block(eta):
    """Smooth lines of 1200 points decompose into components of 500 to 1260
    pieces (convolved by the whole CTA) next to short ones (a warp each):
    bit for bit against the oracle's method, the same component count."""
    shape = (80, 1200)
    x = np.arange(shape[0])[:, None] / shape[0]
    y = np.arange(shape[1])[None, :] / shape[1]
    u0 = np.cos(2 * np.pi * y) + 0.1 * np.cos(2 * np.pi * x)
    V = 0.1 * np.cos(2 * np.pi * x) + 0.05 * np.cos(2 * np.pi * y)
    dx, h, P, W, n = (1 / 80, 1 / 1200), 0.01, (0.2, 0.3), (4, 30), 3
    facts = {}
    got, cnt = gpu_decomp(shape, dx, h, P, W, u0, V, n, eta, facts=facts)
    assert facts["row_blocks"] == [1, 1] and cnt["error_flags"] == 0
    ref, ncomp = O.decomp_run(u0, dx, h, P, W, V, n, eta)
    assert np.array_equal(got.view(np.int64), ref.view(np.int64))
    assert cnt["components"] == ncomp
