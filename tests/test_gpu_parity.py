"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Values are compared bit for bit (every candidate is one binary64 add in both
implementations, minima are exact, the potential term is one subtraction),
binary32 storage bit for bit against the oracle's binary32-storage scheme,
and argmins exactly (tie rule: smallest lifted source).  Cases span several
tiles with ragged tails, tiny and odd line lengths (non-TMA staging), full
torus windows, large P (window far from 0), exact ties and a grid whose
magnitude defeats the Monge rounding margin (brute-force fallback).  The
full-size workloads are checked on sampled outputs in the launch
configuration the benchmark times.
"""
import zlib

import numpy as np
import pytest

from oracle import oracle as O
from edge_counts import edge_hits
from paper_1210_4090_gb300 import workloads as WL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _hjlo():
    from paper_1210_4090_gb300 import hjlo
    return hjlo


def gen(shape, seed, *, dyadic=False, scale=0.3, offset=0.0):
    rng = np.random.default_rng(seed)
    if dyadic:
        u0 = rng.integers(-2048, 2048, size=shape) / 1024.0
        V = rng.integers(-256, 256, size=shape) / 256.0
    else:
        u0 = rng.normal(size=shape) * scale + offset
        V = rng.normal(size=shape) * 0.2
    return u0, V


def gpu_run(shape, dx, h, P, W, u0, V, nsteps, *, algo=0, dtype="f64", argmin=False):
    H = _hjlo()
    code = H.F64 if dtype == "f64" else H.F32_STORAGE
    plan = H.Plan(shape, dx, h, P, W, dtype=code, algo=algo)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    u = torch.tensor(u0, dtype=tdt, device="cuda").contiguous()
    Vt = None if V is None else torch.tensor(V, dtype=torch.float64, device="cuda").contiguous()
    am = None
    if argmin:
        ams = []
        for _ in range(nsteps):
            a = torch.empty(len(shape) * int(np.prod(shape)), dtype=torch.int32, device="cuda")
            plan.step(u, u, Vt, argmin=a)
            ams.append(a)
        am = torch.stack(ams).cpu().numpy().reshape(nsteps, len(shape), *shape)
    else:
        plan.run(u, Vt, nsteps)
    cnt = plan.sync()
    out = u.cpu().numpy()
    plan.close()
    return out, am, cnt


CASES = [
    # name, shape, dx, h, P, W, nsteps, data
    ("1d-n1", (1,), 1.0, 0.1, 0.4, 0, 3, "normal"),
    ("1d-n2", (2,), 0.5, 0.1, 0.4, 0, 3, "normal"),
    ("1d-n3-w1", (3,), 1 / 3, 0.1, -0.7, 1, 4, "normal"),
    ("1d-n31-full", (31,), 1 / 31, 0.07, 0.3, 0, 6, "normal"),
    ("1d-n33-w2", (33,), 1 / 33, 0.07, -1.1, 2, 6, "normal"),
    ("1d-n100-w9", (100,), 1 / 100, 0.05, 0.6, 9, 8, "normal"),
    ("1d-n1000-full", (1000,), 1e-3, 0.05, 0.3, 0, 4, "normal"),
    ("2d-odd", (37, 45), (1 / 37, 1 / 45), 0.06, (0.4, -0.2), (5, 7), 5, "normal"),
    ("2d-tma", (64, 96), (1 / 64, 1 / 96), 0.05, (0.3, 0.1), (8, 12), 5, "normal"),
    ("2d-ragged", (130, 258), (1 / 130, 1 / 258), 0.05, (-0.5, 0.8), (16, 20), 4, "normal"),
    ("2d-full", (24, 40), (1 / 24, 1 / 40), 0.1, (0.7, -0.4), (0, 0), 5, "normal"),
    ("2d-bigP", (64, 64), (1 / 64, 1 / 64), 0.1, (5.0, -7.3), (6, 6), 4, "normal"),
    ("2d-ties", (48, 64), (1 / 32, 1 / 32), 0.125, (0.25, -0.5), (6, 0), 5, "dyadic"),
    ("3d-small", (12, 20, 24), (1 / 12, 1 / 20, 1 / 24), 0.08, (0.2, -0.1, 0.35), (3, 4, 5), 4, "normal"),
    ("3d-tma", (16, 32, 48), (1 / 16, 1 / 32, 1 / 48), 0.05, (0.3, 0.2, -0.6), (4, 8, 4), 4, "normal"),
    ("3d-full-odd", (9, 11, 13), (1 / 9, 1 / 11, 1 / 13), 0.1, (0.5, -0.3, 0.1), (0, 0, 0), 3, "normal"),
    ("3d-ties", (8, 16, 32), (1 / 32,) * 3, 0.125, (0.25, 0.5, -0.25), (2, 3, 0), 3, "dyadic"),
]


def _data(case):
    name, shape, dx, h, P, W, n, kind = case
    u0, V = gen(shape, zlib.crc32(name.encode()) % 1000, dyadic=(kind == "dyadic"))
    return u0, V


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("algo", [1, 2], ids=["brute", "monge"])
def test_run_bitwise_f64(case, algo):
    name, shape, dx, h, P, W, n, kind = case
    u0, V = _data(case)
    ref = O.run(u0, dx, h, P, W, V, n)
    got, _, cnt = gpu_run(shape, dx, h, P, W, u0, V, n, algo=algo)
    assert cnt["error_flags"] == 0
    bad = np.flatnonzero(got.view(np.int64) != ref.view(np.int64))
    assert bad.size == 0, "%d mismatches, first at %s: gpu %r oracle %r" % (
        bad.size, np.unravel_index(bad[0], shape), got.ravel()[bad[0]], ref.ravel()[bad[0]])


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_argmins_exact(case):
    name, shape, dx, h, P, W, n, kind = case
    u0, V = _data(case)
    n = min(n, 3)
    ref, ref_am = O.run(u0, dx, h, P, W, V, n, record_argmin=True)
    for algo in (1, 2):
        got, am, _ = gpu_run(shape, dx, h, P, W, u0, V, n, algo=algo, argmin=True)
        assert np.array_equal(got.view(np.int64), ref.view(np.int64))
        assert np.array_equal(am, ref_am)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_window_edge_hits(case):
    """The plan's window_edge_hits counter equals the count taken from the
    oracle's argmins, for both searches (0 for full torus windows)."""
    name, shape, dx, h, P, W, n, kind = case
    u0, V = _data(case)
    n = min(n, 4)
    want = edge_hits(u0, dx, h, P, W, V, n)
    for algo in (1, 2):
        _, _, cnt = gpu_run(shape, dx, h, P, W, u0, V, n, algo=algo)
        assert cnt["window_edge_hits"] == want, (name, algo, cnt, want)


@pytest.mark.parametrize("case", [c for c in CASES if c[0] in
                                  ("1d-n33-w2", "2d-odd", "2d-tma", "2d-ragged", "3d-tma", "3d-full-odd",
                                   "2d-ties")], ids=lambda c: c[0])
def test_run_bitwise_f32_storage(case):
    name, shape, dx, h, P, W, n, kind = case
    u0, V = _data(case)
    u32 = u0.astype(np.float32)
    ref = O.run(u32, dx, h, P, W, V, n)
    for algo in (1, 2):
        got, _, _ = gpu_run(shape, dx, h, P, W, u32, V, n, algo=algo, dtype="f32")
        assert got.dtype == np.float32
        assert np.array_equal(got.view(np.int32), ref.view(np.int32))
    ref64 = O.run(u0, dx, h, P, W, V, n)
    assert np.max(np.abs(got.astype(np.float64) - ref64)) <= 1e-4 * (1 + np.max(np.abs(ref64)))


def test_monge_margin_fallback_is_exact():
    """|u| ~ 1e14 makes the rounding margin fail (curvature dx^2/h <= 0.0125 <
    8 ulp(1e14) ~ 0.125): the lines go to brute force (counted) and the result
    stays exact."""
    shape, dx, h, P, W = (40, 64), (1 / 40, 1 / 64), 0.05, (0.3, -0.2), (6, 8)
    u0, V = gen(shape, 5, offset=1e14)
    ref = O.run(u0, dx, h, P, W, V, 3)
    got, _, cnt = gpu_run(shape, dx, h, P, W, u0, V, 3, algo=2)
    assert np.array_equal(got.view(np.int64), ref.view(np.int64))
    assert cnt["brute_fallback_lines"] > 0


def test_ties_take_the_rescan_path():
    shape, dx, h, P, W = (48, 64), (1 / 32, 1 / 32), 0.125, (0.25, -0.5), (6, 0)
    u0, V = gen(shape, 3, dyadic=True)
    ref = O.run(u0, dx, h, P, W, V, 4)
    got, _, cnt = gpu_run(shape, dx, h, P, W, u0, V, 4, algo=2)
    assert np.array_equal(got.view(np.int64), ref.view(np.int64))
    assert cnt["exact_rescans"] > 0


def test_time_dependent_potential():
    shape, dx, h, P, W = (30, 52), (1 / 30, 1 / 52), 0.05, (0.4, 0.3), (4, 6)
    u0, _ = gen(shape, 8)
    n = 6
    V = np.random.default_rng(9).normal(size=(n, *shape)) * 0.3
    ref = O.run(u0, dx, h, P, W, V, n, V_per_step=True)
    H = _hjlo()
    plan = H.Plan(shape, dx, h, P, W)
    u = torch.tensor(u0, device="cuda")
    plan.run_tv(u, torch.tensor(V, device="cuda"), n)
    assert np.array_equal(u.cpu().numpy().view(np.int64), ref.view(np.int64))


def test_step_in_place_and_out_of_place_agree():
    shape, dx, h, P, W = (40, 72), (1 / 40, 1 / 72), 0.05, (0.2, -0.6), (5, 9)
    u0, V = gen(shape, 12)
    H = _hjlo()
    plan = H.Plan(shape, dx, h, P, W)
    a = torch.tensor(u0, device="cuda")
    b = torch.empty_like(a)
    Vt = torch.tensor(V, device="cuda")
    plan.step(a, b, Vt)
    plan.step(a, a, Vt)
    assert torch.equal(a, b)
    ref = O.run(u0, dx, h, P, W, V, 1)
    assert np.array_equal(a.cpu().numpy(), ref)


def test_run_host_end_to_end():
    p = WL.grid1024(N=96, nsteps=40, W=8)
    ref = O.run(p.u0, p.dx, p.h, p.P, p.W, p.V, p.nsteps)
    H = _hjlo()
    plan = H.Plan(p.shape, p.dx, p.h, p.P, p.W)
    u = p.u0.copy()
    plan.run_host(u, p.V, p.nsteps)
    assert np.array_equal(u.view(np.int64), ref.view(np.int64))


def test_hbar_readout():
    p = WL.line256()
    H = _hjlo()
    plan = H.Plan(p.shape, p.dx, p.h, p.P, p.W)
    u0 = torch.tensor(p.u0, device="cuda")
    u = u0.clone()
    plan.run(u, torch.tensor(p.V, device="cuda"), p.nsteps)
    est = plan.hbar(u0, u, p.nsteps)
    ref = O.run(p.u0, p.dx, p.h, p.P, p.W, p.V, p.nsteps)
    want = O.hbar_estimate(p.u0, ref, p.nsteps, p.h)
    assert np.allclose(est, want, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("wl,kw,n", [
    ("line256", {}, 200),
    ("grid1024", {"N": 160, "W": 12}, 40),
    ("cube256", {"N": 40, "W": 5}, 12),
    ("adjoint512", {"N": 96, "W": 6}, 30),
])
def test_workload_laws_small_bitwise(wl, kw, n):
    """The workload generators at sizes the oracle runs in seconds (several
    tiles, ragged tails), both algorithms."""
    p = WL.WORKLOADS[wl](nsteps=n, **kw)
    ref = O.run(p.u0, p.dx, p.h, p.P, p.W, p.V, n)
    for algo in (1, 2):
        got, _, cnt = gpu_run(p.shape, p.dx, p.h, p.P, p.W, p.u0, p.V, n, algo=algo)
        assert np.array_equal(got.view(np.int64), ref.view(np.int64)), (wl, algo)


def _sample_points(shape, rng, count):
    """Random points plus the corners and edges of tiles (first/last positions)."""
    npts = int(np.prod(shape))
    pts = set(rng.integers(0, npts, size=count).tolist())
    for corner in [(0,) * len(shape), tuple(s - 1 for s in shape)]:
        pts.add(int(np.ravel_multi_index(corner, shape)))
    for a, s in enumerate(shape):
        for pos in (0, 1, s // 2, s - 2, s - 1):
            c = [int(rng.integers(0, t)) for t in shape]
            c[a] = pos
            pts.add(int(np.ravel_multi_index(c, shape)))
    return np.array(sorted(pts), dtype=np.int64)


@pytest.mark.parametrize("wl,checkpoints,count", [
    ("grid1024", (0, 1, 499, 998), 400),
    ("cube256", (0, 1, 250, 498), 120),
])
def test_full_size_sampled(wl, checkpoints, count):
    """Full workload size, the benchmark's launch path (hjlo_run with its CUDA
    graph): at several step indices the GPU state u^n is read back, one more
    step is taken on the GPU, and sampled outputs of that step are recomputed by
    the oracle from u^n.  Every transition checked bit for bit."""
    p = WL.WORKLOADS[wl]()
    H = _hjlo()
    plan = H.Plan(p.shape, p.dx, p.h, p.P, p.W)
    info = plan.info()
    assert info["algo"] == "monge"
    u = torch.tensor(p.u0, device="cuda")
    Vt = torch.tensor(p.V, device="cuda")
    rng = np.random.default_rng(0)
    done = 0
    for cp in checkpoints:
        plan.run(u, Vt, cp - done)
        before = u.cpu().numpy()
        plan.run(u, Vt, 1)
        after = u.cpu().numpy()
        done = cp + 1
        pts = _sample_points(p.shape, rng, count)
        ref = O.step_points(before, p.dx, p.h, p.P, p.W, p.V, pts)
        got = after.ravel()[pts]
        assert np.array_equal(got.view(np.int64), ref.view(np.int64)), (wl, cp)
    plan.run(u, Vt, p.nsteps - done)
    cnt = plan.sync()
    assert cnt["error_flags"] == 0 and cnt["steps"] == p.nsteps
    assert np.isfinite(u.cpu().numpy()).all()


@pytest.mark.parametrize("lanes", [0, 2, 4, 8, 16, 32, 64], ids=lambda v: "lpl%d" % v if v else "auto")
@pytest.mark.parametrize("offload", ["", "0", "0,2"], ids=["offload-default", "offload-off", "offload-all"])
def test_segment_shapes_with_shocks(lanes, offload, monkeypatch):
    """Every segment length the monotone search can take (lanes per line forced
    from the environment), with the warp offload of wide brackets at its
    default rule, turned off, and taking every bracket of two or more offsets
    (groups of every size), on a developed solution with shocks (wide argmin
    jumps) and on a rough start (wide brackets everywhere)."""
    if lanes:
        monkeypatch.setenv("HJLO_LANES_PER_LINE", str(lanes))
    if offload:
        monkeypatch.setenv("HJLO_OFFLOAD", offload)
    p = WL.grid1024(N=160, nsteps=60, W=12)
    ref = O.run(p.u0, p.dx, p.h, p.P, p.W, p.V, p.nsteps)
    got, _, cnt = gpu_run(p.shape, p.dx, p.h, p.P, p.W, p.u0, p.V, p.nsteps, algo=2)
    assert cnt["error_flags"] == 0
    assert np.array_equal(got.view(np.int64), ref.view(np.int64))
    shape, dx, h, P, W = (24, 200), (1 / 24, 1 / 200), 0.05, (0.3, -0.2), (4, 40)
    u0, V = gen(shape, 17, scale=1.0)
    ref, ref_am = O.run(u0, dx, h, P, W, V, 2, record_argmin=True)
    got, am, _ = gpu_run(shape, dx, h, P, W, u0, V, 2, algo=2, argmin=True)
    assert np.array_equal(got.view(np.int64), ref.view(np.int64))
    assert np.array_equal(am, ref_am)


def test_resume_equals_uninterrupted_run():
    """Checkpoint and resume (the semigroup property of eq. uN): n steps, a
    copy of the state, then m more steps equal n + m steps bit for bit -- for
    a static V through the captured 16-step graphs and single steps, and for a
    time-dependent V whose rows continue where the first run stopped."""
    shape, dx, h, P, W = (40, 56), (1 / 40, 1 / 56), 0.05, (0.3, -0.2), (5, 7)
    u0, V = gen(shape, 21)
    H = _hjlo()
    plan = H.Plan(shape, dx, h, P, W)
    Vt = torch.tensor(V, device="cuda")
    whole = torch.tensor(u0, device="cuda")
    plan.run(whole, Vt, 37)
    part = torch.tensor(u0, device="cuda")
    plan.run(part, Vt, 20)
    resumed = part.clone()                       # the checkpoint
    plan.run(resumed, Vt, 17)
    assert torch.equal(whole, resumed)
    assert np.array_equal(whole.cpu().numpy().view(np.int64), O.run(u0, dx, h, P, W, V, 37).view(np.int64))
    Vs = np.random.default_rng(22).normal(size=(30, *shape)) * 0.2
    Vst = torch.tensor(Vs, device="cuda")
    a = torch.tensor(u0, device="cuda")
    plan.run_tv(a, Vst, 30)
    b = torch.tensor(u0, device="cuda")
    plan.run_tv(b, Vst[:11].contiguous(), 11)
    plan.run_tv(b, Vst[11:].contiguous(), 19)
    assert torch.equal(a, b)
    assert np.array_equal(a.cpu().numpy().view(np.int64),
                          O.run(u0, dx, h, P, W, Vs, 30, V_per_step=True).view(np.int64))
    assert plan.sync()["steps"] == 37 + 20 + 17 + 30 + 11 + 19
    plan.close()
