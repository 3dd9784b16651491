"""Row blocks: a contiguous axis whose lines are too long for one CTA's shared
memory, or too few to fill the GPU, is launched as blocks of rows, each staged
with the window span its rows need.  Results, argmins and the window-edge count
must equal the oracle's bit for bit, for both searches and both storage types,
including a ragged last block and a line of noise (argmin jumps everywhere)."""
import numpy as np
import pytest

from edge_counts import edge_hits
from oracle import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# name, shape, h, P, W, steps, noise-only data
CASES = [
    ("1d-40000", (40000,), 1e-4, 0.3, 50, 3, False),          # longer than one CTA's shared memory
    ("2d-3x30000", (3, 30000), 1e-4, (0.2, -0.4), (1, 40), 2, False),
    ("1d-4096", (4096,), 2e-3, -0.5, 60, 5, False),           # fits, but a single line
    ("1d-5003-ragged", (5003,), 1e-3, 0.1, 37, 4, False),
    ("1d-20000-noise", (20000,), 1e-4, 0.0, 30, 3, True),
]


def _data(shape, noise, seed):
    rng = np.random.default_rng(seed)
    grids = np.meshgrid(*[np.arange(n) / n for n in shape], indexing="ij")
    if noise:
        u0 = 0.05 * rng.normal(size=shape)
    else:
        u0 = 0.3 * np.sin(6 * np.pi * grids[-1]) + 0.002 * rng.normal(size=shape)
        for g in grids[:-1]:
            u0 = u0 + 0.1 * np.cos(2 * np.pi * g)
    V = 0.2 * np.cos(4 * np.pi * grids[-1]) + 0.05 * rng.normal(size=shape)
    return u0, V


def _plan_run(shape, dx, h, P, W, u0, V, n, algo, argmin=False):
    from paper_1210_4090_gb300 import hjlo
    f32 = u0.dtype == np.float32
    plan = hjlo.Plan(shape, dx, h, P, W, dtype=hjlo.F32_STORAGE if f32 else hjlo.F64, algo=algo)
    info = plan.info()
    u = torch.tensor(u0, device="cuda")
    Vt = torch.tensor(V, device="cuda")
    am = None
    if argmin:
        ams = []
        for _ in range(n):
            a = torch.empty(len(shape) * u0.size, dtype=torch.int32, device="cuda")
            plan.step(u, u, Vt, argmin=a)
            ams.append(a)
        am = torch.stack(ams).cpu().numpy().reshape(n, len(shape), *shape)
    else:
        plan.run(u, Vt, n)
    cnt = plan.sync()
    plan.close()
    return u.cpu().numpy(), am, cnt, info


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("algo", [1, 2], ids=["brute", "monge"])
def test_row_blocks_bitwise(case, algo):
    name, shape, h, P, W, n, noise = case
    dx = tuple(1.0 / s for s in shape)
    u0, V = _data(shape, noise, 7)
    ref = O.run(u0, dx, h, P, W, V, n)
    got, _, cnt, info = _plan_run(shape, dx, h, P, W, u0, V, n, algo)
    assert info["row_blocks"][-1] > 1, info
    assert cnt["error_flags"] == 0
    bad = np.flatnonzero(got.view(np.int64) != ref.view(np.int64))
    assert bad.size == 0, "%d mismatches, first at %d" % (bad.size, bad[0])
    assert cnt["window_edge_hits"] == edge_hits(u0, dx, h, P, W, V, n)


@pytest.mark.parametrize("case", [CASES[1], CASES[3], CASES[4]], ids=lambda c: c[0])
def test_row_blocks_argmins(case):
    name, shape, h, P, W, n, noise = case
    dx = tuple(1.0 / s for s in shape)
    u0, V = _data(shape, noise, 8)
    n = min(n, 2)
    ref, ref_am = O.run(u0, dx, h, P, W, V, n, record_argmin=True)
    for algo in (1, 2):
        got, am, _, _ = _plan_run(shape, dx, h, P, W, u0, V, n, algo, argmin=True)
        assert np.array_equal(got.view(np.int64), ref.view(np.int64))
        assert np.array_equal(am, ref_am)


@pytest.mark.parametrize("case", [CASES[0], CASES[2], CASES[4]], ids=lambda c: c[0])
def test_row_blocks_binary32_storage(case):
    name, shape, h, P, W, n, noise = case
    dx = tuple(1.0 / s for s in shape)
    u0, V = _data(shape, noise, 9)
    u32 = u0.astype(np.float32)
    ref = O.run(u32, dx, h, P, W, V, n)
    for algo in (1, 2):
        got, _, cnt, _ = _plan_run(shape, dx, h, P, W, u32, V, n, algo)
        assert got.dtype == np.float32 and cnt["error_flags"] == 0
        assert np.array_equal(got.view(np.int32), ref.view(np.int32))


def test_whole_lines_when_they_fill_the_gpu():
    """Many lines that fit: whole lines per CTA, as before."""
    from paper_1210_4090_gb300 import hjlo
    plan = hjlo.Plan((1024, 1024), (1 / 1024,) * 2, 0.02, (0.3, 0.1), (64, 64))
    assert plan.info()["row_blocks"] == [1, 1]
    plan.close()


def test_row_blocks_in_place_over_two_waves():
    """40 lines of 60000 points: 4 row blocks per line of ~15800 rows, 160
    CTAs of 1024 threads with ~220 KB of shared memory each -- more than one
    per SM, so some start after others have finished.  A block stages rows of
    its neighbours, so a pass in place (hjlo_run) must not write over rows a
    later block has yet to read: the plan routes it through its scratch."""
    shape, h, P, W, n = (40, 60000), 1e-4, (0.1, 0.2), (1, 30), 2
    dx = tuple(1.0 / s for s in shape)
    u0, V = _data(shape, False, 10)
    from paper_1210_4090_gb300 import hjlo
    plan = hjlo.Plan(shape, dx, h, P, W)
    info = plan.info()
    assert info["row_blocks"][1] > 1, info
    u = torch.tensor(u0, device="cuda")
    plan.run(u, torch.tensor(V, device="cuda"), n)
    assert plan.sync()["error_flags"] == 0
    plan.close()
    ref = O.run(u0, dx, h, P, W, V, n)
    bad = np.flatnonzero(u.cpu().numpy().view(np.int64) != ref.view(np.int64))
    assert bad.size == 0, "%d mismatches, first at %d" % (bad.size, bad[0])
