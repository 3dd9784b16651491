"""The decomposition method (Sec. 4) over whole periods of lines too long for
one CTA: the period's greedy cut (Sec. 4.3, tolerance eta of Sec. 4.4) is
made per chunk of the span and stitched into the one cut of the whole
period, and the components' convolutions are spread over blocks of outputs.
Checked bit for bit against the oracle's version of the method, which
decomposes every line once per pass, with the same number of components:
on long lines that take this path by themselves, and on short lines, many
lines, strided axes and ragged chunk and block tails with the path forced
(HJLO_DECOMP_SPLIT=1) and chunks and blocks made small.  At eta = 0 it is
also the scheme itself.  At the paper's size (2^18 points, eta = dx) the
components are counted against the oracle's cut of the same line and the
outputs checked to be candidates of the scheme, never below it."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1210_4090_gb300 import workloads as WL

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _hjlo():
    from paper_1210_4090_gb300 import hjlo
    return hjlo


def gpu_decomp(shape, dx, h, P, W, u0, V, nsteps, eta):
    """Runs the decomposition pass; returns (u, counters, the plan's facts).
    The facts are only used to assert which launch shape a case exercises."""
    H = _hjlo()
    plan = H.Plan(shape, dx, h, P, W, algo=H.ALGO_DECOMP)
    plan.set_tolerance(eta)
    info = plan.info()
    u = torch.tensor(u0, device="cuda")
    Vt = None if V is None else torch.tensor(V, device="cuda")
    plan.run(u, Vt, nsteps)
    cnt = plan.sync()
    plan.close()
    return u.cpu().numpy(), cnt, info


def _bits(a):
    return np.asarray(a).view(np.int64)


CASES = [
    ("1d-w", (200,), 1 / 200, 0.05, 0.4, 20),
    ("1d-full", (60,), 1 / 60, 0.1, -0.3, 0),
    ("1d-n1", (1,), 1.0, 0.1, 0.2, 0),
    ("1d-n2", (2,), 0.5, 0.1, 0.2, 0),
    ("1d-w0", (130,), 1 / 130, 0.05, 0.2, 1),
    ("2d", (24, 40), (1 / 24, 1 / 40), 0.06, (0.4, -0.2), (4, 6)),
    ("3d", (6, 8, 12), (1 / 6, 1 / 8, 1 / 12), 0.08, (0.3, -0.1, 0.5), (0, 2, 3)),
]


@pytest.mark.parametrize("chunk,rows", [(64, "7"), (96, "1"), (4096, "")])
@pytest.mark.parametrize("eta", [0.0, 1e-4, 1e-2, 1e3])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_forced_split_bitwise(case, eta, chunk, rows, monkeypatch):
    name, shape, dx, h, P, W = case
    monkeypatch.setenv("HJLO_DECOMP_SPLIT", "1")
    monkeypatch.setenv("HJLO_DECOMP_CHUNK", str(chunk))
    if rows:
        monkeypatch.setenv("HJLO_DECOMP_SPLIT_ROWS", rows)
    rng = np.random.default_rng(len(name) * 11 + int(eta * 1e4) + chunk)
    u0 = np.cumsum(rng.normal(size=shape), axis=-1) * 0.03
    V = rng.normal(size=shape) * 0.2
    n = 3
    got, cnt, info = gpu_decomp(shape, dx, h, P, W, u0, V, n, eta)
    assert all(c > 0 for c in info["split_chunks"]) and cnt["error_flags"] == 0
    ref, ncomp = O.decomp_run(u0, dx, h, P, W, V, n, eta)
    assert np.array_equal(_bits(got), _bits(ref))
    assert cnt["components"] == ncomp
    if eta == 0.0:
        assert np.array_equal(_bits(got), _bits(O.run(u0, dx, h, P, W, V, n)))


def test_forced_split_fuzz(monkeypatch):
    """Random geometries, data shapes, tolerances, chunk and block sizes."""
    monkeypatch.setenv("HJLO_DECOMP_SPLIT", "1")
    rng = np.random.default_rng(77)
    for trial in range(24):
        nd = int(rng.integers(1, 3))
        shape = tuple(int(rng.integers(2, 160 if nd == 1 else 40)) for _ in range(nd))
        dx = tuple(1.0 / s for s in shape)
        W = tuple(int(rng.integers(0, max(1, s // 2))) for s in shape)
        P = tuple(float(rng.uniform(-0.5, 0.5)) for _ in shape)
        h = float(rng.uniform(0.01, 0.2))
        monkeypatch.setenv("HJLO_DECOMP_CHUNK", str(int(rng.choice([64, 128, 160, 4096]))))
        monkeypatch.setenv("HJLO_DECOMP_SPLIT_ROWS", str(int(rng.integers(1, 200))))
        kind = trial % 3
        if kind == 0:
            u0 = rng.normal(size=shape) * 0.3
        elif kind == 1:
            u0 = np.cumsum(rng.normal(size=shape), axis=-1) * 0.02
        else:
            grids = np.meshgrid(*[np.arange(s) / s for s in shape], indexing="ij")
            u0 = np.abs(np.sin(3 * np.pi * sum(grids))) * 0.2
        eta = float(rng.choice([0.0, 1.0, 10.0, 1e4]))
        got, cnt, _ = gpu_decomp(shape, dx, h, P, W, u0, None, 2, eta)
        ref, ncomp = O.decomp_run(u0, dx, h, P, W, None, 2, eta)
        assert np.array_equal(_bits(got), _bits(ref)), (trial, shape, W, eta)
        assert cnt["components"] == ncomp and cnt["error_flags"] == 0, trial


def _long_line():
    N, W, h, P = 12000, 40, 2e-3, 0.3
    x = np.arange(N) / N
    rng = np.random.default_rng(13)
    u0 = 0.3 * np.sin(6 * np.pi * x) + 0.01 * np.cumsum(rng.normal(size=N)) / np.sqrt(N)
    V = 0.2 * np.cos(4 * np.pi * x)
    return N, W, h, P, u0, V


@pytest.mark.parametrize("eta", [1.0 / 12000, 1.0, 10.0])
def test_long_line_whole_period(eta):
    """A line longer than one CTA holds, at eta > 0, without restarts: its
    period is cut across CTAs, with the oracle's components and values."""
    N, W, h, P, u0, V = _long_line()
    n = 3
    got, cnt, info = gpu_decomp((N,), 1.0 / N, h, P, W, u0, V, n, eta)
    assert info["split_chunks"][0] > 1 and info["row_blocks"][0] == 1 and cnt["error_flags"] == 0
    ref, ncomp = O.decomp_run(u0, 1.0 / N, h, P, W, V, n, eta)
    assert np.array_equal(_bits(got), _bits(ref))
    assert cnt["components"] == ncomp


@pytest.mark.parametrize("eta", [0.0, 0.5])
@pytest.mark.parametrize("shape", [(2, 12000), (12000, 3)], ids=["contiguous", "strided"])
def test_long_lines_in_2d(shape, eta):
    """Long lines on a 2D grid: two contiguous lines (row blocks at eta = 0,
    whole periods across CTAs at eta > 0), and a strided long axis, which
    row blocks cannot serve, across CTAs at every tolerance."""
    rng = np.random.default_rng(sum(shape))
    dx = tuple(1.0 / s for s in shape)
    W = tuple(min(30, s // 3) for s in shape)
    P = (0.2, -0.3)
    u0 = np.cumsum(rng.normal(size=shape), axis=-1) * 0.01 + np.cumsum(rng.normal(size=shape), axis=0) * 0.01
    V = rng.normal(size=shape) * 0.1
    got, cnt, info = gpu_decomp(shape, dx, 2e-3, P, W, u0, V, 2, eta)
    long_axis = int(np.argmax(shape))
    if long_axis == 1 and eta == 0.0:
        assert info["row_blocks"][1] > 1 and info["split_chunks"][1] == 0
    else:
        assert info["split_chunks"][long_axis] > 1
    assert cnt["error_flags"] == 0
    ref, ncomp = O.decomp_run(u0, dx, 2e-3, P, W, V, 2, eta)
    assert np.array_equal(_bits(got), _bits(ref))
    if max(info["row_blocks"]) == 1:               # row blocks cut each block's span on its own
        assert cnt["components"] == ncomp
    if eta == 0.0:
        assert np.array_equal(_bits(got), _bits(O.run(u0, dx, 2e-3, P, W, V, 2)))


def test_paper_pendulum_whole_period():
    """The paper's pendulum (Sec. 5.1) on 2 x 8192 points at eta = dx, the
    tolerance of its timed run: the first steps by the method on whole
    periods, bit for bit the oracle's."""
    p = WL.pendulum(K=8192)
    n = 3
    eta = p.dx[0]
    got, cnt, info = gpu_decomp(p.shape, p.dx, p.h, p.P, p.W, p.u0, p.V, n, eta)
    assert info["split_chunks"][0] > 1 and cnt["error_flags"] == 0
    ref, ncomp = O.decomp_run(p.u0, p.dx, p.h, p.P, p.W, p.V, n, eta)
    assert np.array_equal(_bits(got), _bits(ref))
    assert cnt["components"] == ncomp


def test_paper_size_run_first_step(monkeypatch):
    """The paper's timed configuration (2^18 points, T = 8, tau = sqrt(dx),
    eta = dx) in the launch shape the benchmark times: one pass cuts the
    period into exactly the oracle's components, and every output is a
    candidate fl(u(y) + k(d)) of the scheme, never below the scheme's step
    (the scheme's minimum is over all candidates).  At eta = 0 the same
    path is the scheme bit for bit."""
    p = WL.pendulum(K=131072)
    N = p.shape[0]
    dx = p.dx[0]
    dlo, dhi, k = O.table(N, dx, p.h, p.P[0], p.W[0])
    n = dhi - dlo
    src = p.u0[(np.arange(N + n) - dhi) % N]
    got, cnt, info = gpu_decomp(p.shape, p.dx, p.h, p.P, p.W, p.u0, None, 1, dx)
    assert info["split_chunks"][0] > 1 and cnt["error_flags"] == 0
    assert cnt["components"] == len(O.decompose(src, dx * dx))      # second differences >= -eta dx
    exact = O.run(p.u0, p.dx, p.h, p.P, p.W, None, 1)
    assert np.all(got >= exact)
    hit = np.zeros(N, dtype=bool)
    for i, d in enumerate(range(dlo, dhi + 1)):
        hit |= (np.roll(p.u0, d) + k[i]) == got
    assert hit.all()
    monkeypatch.setenv("HJLO_DECOMP_SPLIT", "1")
    exact2, _, info2 = gpu_decomp(p.shape, p.dx, p.h, p.P, p.W, p.u0, p.V, 2, 0.0)
    assert info2["split_chunks"][0] > 1
    assert np.array_equal(_bits(exact2), _bits(O.run(p.u0, p.dx, p.h, p.P, p.W, p.V, 2)))


def test_whole_run_through_the_experiment_helper(monkeypatch):
    """The paper's pendulum on 2 x 256 points to T = 8 (73 steps) by the
    method at eta = dx, every pass on the split path: bit for bit the
    oracle's run, shocks and all."""
    from paper_1210_4090_gb300 import experiments as E
    monkeypatch.setenv("HJLO_DECOMP_SPLIT", "1")
    monkeypatch.setenv("HJLO_DECOMP_CHUNK", "128")
    p = WL.pendulum(256)
    got, comps = E.solve_decomp_gpu(p, p.dx[0])
    ref, ncomp = O.decomp_run(p.u0, p.dx, p.h, p.P, p.W, p.V, p.nsteps, p.dx[0])
    assert np.array_equal(_bits(got), _bits(ref))
    assert comps == ncomp / p.nsteps
