"""The paper's own fast convolution (Sec. 4, HJLO_ALGO_DECOMP) on the GPU
against the oracle's version of the same method, which decomposes every line
once per pass (Sec. 4.2-4.3): bit for bit (every output is the same candidate
minimum over the same components) and the same number of components; at
eta = 0 (and on exact dyadic data) also equal to the scheme itself.  The
approximate option that restarts the decomposition at each row block of a
long line is checked against the scheme by what holds for it exactly: every
output is a candidate of the scheme, never below it, and within the bound
eta dx m^2 per pass that treating an eta-convex component of m pieces as
convex can add."""
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


def gpu_decomp(shape, dx, h, P, W, u0, V, nsteps, eta=0.0, V_per_step=False, restart=False):
    """Runs the decomposition pass; returns (u, counters, the plan's facts).
    The facts are only used to assert which launch shape a case exercises."""
    H = _hjlo()
    plan = H.Plan(shape, dx, h, P, W, algo=H.ALGO_DECOMP)
    if eta or restart:
        plan.set_tolerance(eta, restart_blocks=restart)
    info = plan.info()
    assert info["algo"] == "decomp"
    u = torch.tensor(u0, device="cuda")
    Vt = None if V is None else torch.tensor(V, device="cuda")
    if V_per_step:
        plan.run_tv(u, Vt, nsteps)
    else:
        plan.run(u, Vt, nsteps)
    cnt = plan.sync()
    plan.close()
    return u.cpu().numpy(), cnt, info


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
    got, cnt, info = gpu_decomp(shape, dx, h, P, W, u0, V, n, eta)
    ref, ncomp = O.decomp_run(u0, dx, h, P, W, V, n, eta)
    assert cnt["error_flags"] == 0
    assert np.array_equal(got.view(np.int64), ref.view(np.int64))
    if eta > 0:
        # whole lines: the same components as the oracle's
        assert info["row_blocks"] == [1] * len(shape)
        assert cnt["components"] == ncomp
    else:
        # at eta = 0 the method is exact: the scheme's values whatever the cut
        assert np.array_equal(got.view(np.int64), O.run(u0, dx, h, P, W, V, n).view(np.int64))


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_dyadic_equals_scheme(case):
    name, shape, dx, h, P, W = case
    dx = tuple(1 / 32 for _ in shape) if len(shape) > 1 else 1 / 32
    h, P = 0.125, (tuple(0.25 * (-1) ** a for a in range(len(shape))) if len(shape) > 1 else 0.25)
    rng = np.random.default_rng(2)
    u0 = rng.integers(-2048, 2048, size=shape) / 1024.0
    V = rng.integers(-256, 256, size=shape) / 256.0
    ref = O.run(u0, dx, h, P, W, V, 4)
    got, _, _ = gpu_decomp(shape, dx, h, P, W, u0, V, 4)
    assert np.array_equal(got.view(np.int64), ref.view(np.int64))


def test_graph_path_and_tolerance_change():
    """40 steps go through the captured graph; changing eta rebuilds it (and
    the launch shape: the single line runs in row blocks at eta = 0, whole at
    eta > 0)."""
    H = _hjlo()
    shape, dx, h, P, W = (96,), 1 / 96, 0.05, 0.3, 10
    rng = np.random.default_rng(4)
    u0 = np.cumsum(rng.normal(size=shape)) * 0.02
    V = rng.normal(size=shape) * 0.1
    plan = H.Plan(shape, dx, h, P, W, algo=H.ALGO_DECOMP)
    Vt = torch.tensor(V, device="cuda")
    for eta in (0.0, 5e-3, 0.0):
        plan.set_tolerance(eta)
        u = torch.tensor(u0, device="cuda")
        plan.run(u, Vt, 40)
        ref, _ = O.decomp_run(u0, dx, h, P, W, V, 40, eta)
        assert np.array_equal(u.cpu().numpy().view(np.int64), ref.view(np.int64)), eta
    plan.close()


def test_paper_law_time_dependent():
    p = WL.tdep(32)
    ref, _ = O.decomp_run(p.u0, p.dx, p.h, p.P, p.W, p.V, p.nsteps, 0.0, V_per_step=True)
    got, _, _ = gpu_decomp(p.shape, p.dx, p.h, p.P, p.W, p.u0, p.V, p.nsteps, V_per_step=True)
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
    assert H.lib().hjlo_plan_set_decomp(plan._h, 0.1, 2) == 1                            # EINVAL
    plan.close()
    mono = H.Plan((16,), 1 / 16, 0.1, 0.2, 3, algo=H.ALGO_MONGE)
    with pytest.raises(H.HjloError):
        mono.set_tolerance(0.1)
    mono.close()


def _long_line():
    N, W, h, P = 12000, 40, 2e-3, 0.3
    x = np.arange(N) / N
    rng = np.random.default_rng(13)
    u0 = 0.3 * np.sin(6 * np.pi * x) + 0.01 * np.cumsum(rng.normal(size=N)) / np.sqrt(N)
    V = 0.2 * np.cos(4 * np.pi * x)
    return N, W, h, P, u0, V


def test_row_blocks_at_zero_tolerance():
    """A single long line in row blocks, each block cut on its own span: at
    eta = 0 the method is exact, so bit for bit the oracle's whole-line
    decomposition and the scheme."""
    N, W, h, P, u0, V = _long_line()
    n = 4
    got, cnt, info = gpu_decomp((N,), 1.0 / N, h, P, W, u0, V, n, 0.0)
    assert info["row_blocks"][0] > 1 and cnt["error_flags"] == 0
    ref, _ = O.decomp_run(u0, 1.0 / N, h, P, W, V, n, 0.0)
    assert np.array_equal(got.view(np.int64), ref.view(np.int64))
    assert np.array_equal(got.view(np.int64), O.run(u0, 1.0 / N, h, P, W, V, n).view(np.int64))


def test_whole_line_at_positive_tolerance():
    """At eta > 0 a period is decomposed whole: a line longer than one CTA
    holds has its cut spread over CTAs (hjlo_split.cu) unless the caller asks
    for block restarts, which run it in row blocks."""
    H = _hjlo()
    N, W, h, P, u0, V = _long_line()
    plan = H.Plan((N,), 1.0 / N, h, P, W, algo=H.ALGO_DECOMP)
    assert plan.info()["row_blocks"][0] > 1 and plan.info()["split_chunks"][0] == 0
    plan.set_tolerance(1.0)
    assert plan.info()["row_blocks"][0] == 1 and plan.info()["split_chunks"][0] > 1
    plan.set_tolerance(1.0, restart_blocks=True)
    assert plan.info()["row_blocks"][0] > 1 and plan.info()["split_chunks"][0] == 0
    plan.close()


def _is_candidate(out, u, dx, h, P, W):
    """Every output of one pass on a line is one candidate fl(u(y) + k(d))."""
    dlo, dhi, k = O.table(len(u), dx, h, P, W)
    N = len(u)
    hit = np.zeros(N, dtype=bool)
    for i, d in enumerate(range(dlo, dhi + 1)):
        hit |= (np.roll(u, d) + k[i]) == out
    return hit


@pytest.mark.parametrize("eta", [1.0, 10.0])
@pytest.mark.parametrize("rows", [600, 2000])
def test_block_restart_option(eta, rows, monkeypatch):
    """The approximate option (hjlo_plan_set_decomp restart_blocks = 1) on the
    long line, blocks of `rows` rows chosen here: one pass is a candidate of
    the scheme at every output, never below it, and above it by at most
    eta dx m^2 with m <= rows + window - 1 (the longest component a block
    holds); n passes are never below the scheme's n steps (monotonicity) and
    within n such bounds (the scheme is a sup-norm contraction)."""
    monkeypatch.setenv("HJLO_BLOCK_ROWS", str(rows))
    N, W, h, P, u0, _ = _long_line()
    dx = 1.0 / N
    one, cnt, info = gpu_decomp((N,), dx, h, P, W, u0, None, 1, eta, restart=True)
    assert info["row_blocks"][0] > 1 and info["block_rows"][0] == rows and cnt["error_flags"] == 0
    exact = O.run(u0, dx, h, P, W, None, 1)
    assert np.all(_is_candidate(one, u0, dx, h, P, W))
    assert np.all(one >= exact)
    m = rows + (2 * W + 1) - 1
    bound = eta * dx * m * m
    assert float(np.max(one - exact)) <= bound
    n = 5
    many, _, _ = gpu_decomp((N,), dx, h, P, W, u0, None, n, eta, restart=True)
    exact_n = O.run(u0, dx, h, P, W, None, n)
    assert np.all(many >= exact_n)
    assert float(np.max(many - exact_n)) <= n * bound
    # the method itself (one decomposition per period) obeys the same bound
    # with m up to the whole lifted line
    whole, _ = O.decomp_run(u0, dx, h, P, W, None, 1, eta)
    assert np.all(whole >= exact)


def test_block_restart_at_zero_tolerance_is_exact(monkeypatch):
    monkeypatch.setenv("HJLO_BLOCK_ROWS", "700")
    N, W, h, P, u0, V = _long_line()
    got, _, info = gpu_decomp((N,), 1.0 / N, h, P, W, u0, V, 3, 0.0, restart=True)
    assert info["row_blocks"][0] > 1
    assert np.array_equal(got.view(np.int64), O.run(u0, 1.0 / N, h, P, W, V, 3).view(np.int64))


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
    got, cnt, info = gpu_decomp(shape, dx, h, P, W, u0, V, n, eta)
    assert info["row_blocks"] == [1, 1] and cnt["error_flags"] == 0
    ref, ncomp = O.decomp_run(u0, dx, h, P, W, V, n, eta)
    assert np.array_equal(got.view(np.int64), ref.view(np.int64))
    assert cnt["components"] == ncomp
