"""Seeded random geometries through every algorithm and storage type, bit for
bit against the oracle: shapes from 1 to 3 axes with odd and power-of-two
sizes, windows from 0 (full torus) to wide, P far from and near 0, and
potentials on and off.  Each case is small enough for the oracle to run in
well under a second."""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NCASES = 48


def _case(i):
    rng = np.random.default_rng([7, i])
    ndim = int(rng.integers(1, 4))
    cap = {1: 700, 2: 90, 3: 28}[ndim]
    shape = tuple(int(rng.integers(1, cap)) for _ in range(ndim))
    dx = tuple(float(1.0 / n) if n > 0 else 1.0 for n in shape)
    h = float(rng.uniform(0.02, 0.2))
    P = tuple(float(rng.choice([rng.uniform(-1, 1), rng.uniform(-6, 6)])) for _ in range(ndim))
    W = tuple(int(rng.choice([0, rng.integers(1, 6), rng.integers(4, 40)])) for _ in range(ndim))
    u0 = rng.normal(size=shape) * float(rng.choice([0.05, 0.3, 2.0]))
    V = rng.normal(size=shape) * 0.2 if rng.random() < 0.7 else None
    n = int(rng.integers(1, 6))
    algo = int(rng.choice([0, 1, 2]))
    f32 = bool(rng.random() < 0.25)
    return shape, dx, h, P, W, u0, V, n, algo, f32


@pytest.mark.parametrize("i", range(NCASES))
def test_random_geometry(i):
    from paper_1210_4090_gb300 import hjlo
    shape, dx, h, P, W, u0, V, n, algo, f32 = _case(i)
    if f32:
        u0 = u0.astype(np.float32)
    ref = O.run(u0, dx, h, P, W, V, n)
    try:
        plan = hjlo.Plan(shape, dx, h, P, W, dtype=hjlo.F32_STORAGE if f32 else hjlo.F64, algo=algo)
    except hjlo.HjloError as e:            # a window or line the library declines must say so
        assert e.status == 6, e
        return
    u = torch.tensor(u0, device="cuda")
    Vt = None if V is None else torch.tensor(V, device="cuda")
    plan.run(u, Vt, n)
    cnt = plan.sync()
    plan.close()
    assert cnt["error_flags"] == 0
    got = u.cpu().numpy()
    view = np.int32 if f32 else np.int64
    assert np.array_equal(got.view(view), ref.view(view)), (shape, W, P, algo, f32)
    if algo != 3:
        from edge_counts import edge_hits
        assert cnt["window_edge_hits"] == edge_hits(u0, dx, h, P, W, V, n)


NDECOMP = 16


def _decomp_case(i):
    rng = np.random.default_rng([11, i])
    ndim = int(rng.integers(1, 4))
    cap = {1: 600, 2: 60, 3: 20}[ndim]
    shape = tuple(int(rng.integers(1, cap)) for _ in range(ndim))
    dx = tuple(1.0 / n for n in shape)
    h = float(rng.uniform(0.02, 0.2))
    P = tuple(float(rng.uniform(-2, 2)) for _ in range(ndim))
    W = tuple(int(rng.choice([0, rng.integers(1, 6), rng.integers(4, 40)])) for _ in range(ndim))
    u0 = np.cumsum(rng.normal(size=shape), axis=-1) * float(rng.choice([0.01, 0.05]))
    V = rng.normal(size=shape) * 0.1 if rng.random() < 0.7 else None
    n = int(rng.integers(1, 4))
    eta = float(rng.choice([0.0, 0.0, 1.0, 10.0]))
    return shape, dx, h, P, W, u0, V, n, eta


@pytest.mark.parametrize("i", range(NDECOMP))
def test_random_geometry_decomposition(i):
    """The paper's Sec. 4 method on random geometries: bit for bit against the
    oracle's version of the method, with the same number of components when
    eta > 0 (at eta = 0 the values are the scheme's whatever the cut, and
    long or lonely lines may run in row blocks)."""
    from paper_1210_4090_gb300 import hjlo
    shape, dx, h, P, W, u0, V, n, eta = _decomp_case(i)
    try:
        plan = hjlo.Plan(shape, dx, h, P, W, algo=hjlo.ALGO_DECOMP)
        if eta:
            plan.set_tolerance(eta)
    except hjlo.HjloError as e:            # a non-strictly-convex table or a line too long
        assert e.status in (4, 6), e
        return
    u = torch.tensor(u0, device="cuda")
    plan.run(u, None if V is None else torch.tensor(V, device="cuda"), n)
    cnt = plan.sync()
    plan.close()
    ref, ncomp = O.decomp_run(u0, dx, h, P, W, V, n, eta)
    assert cnt["error_flags"] == 0
    assert np.array_equal(u.cpu().numpy().view(np.int64), ref.view(np.int64)), (shape, W, P, eta)
    if eta:
        assert cnt["components"] == ncomp
