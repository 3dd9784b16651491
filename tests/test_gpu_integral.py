"""The first discrete semigroup (eq. cost1) on the GPU against the oracle.

The kinetic part and the final add / multiply / subtract of a candidate are
the same binary64 operations on both sides; the path-integral sum S differs
in rounding (fused multiply-adds in two chains on the GPU, separate products
and one running sum in the oracle) and the trigonometric tables are formed
independently (the C library's sin / cos here, numpy's in the oracle), each
of which moves a candidate by at most a few ulps of its terms:
nmodes x 4 ulp x max|c| x h per step in all, far below the 1e-12 (1 + max|u|)
the values are compared to.  With V = 0 or a constant V there are no tables
and the result is bit for bit the oracle's, and on dyadic data the fully
discrete scheme's."""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def gpu_integral(shape, dx, h, P, W, modes, coef, u0, n):
    from paper_1210_4090_gb300 import hjlo
    plan = hjlo.IntegralPlan(shape, dx, h, P, W, modes, coef)
    u = torch.tensor(u0, device="cuda")
    plan.run(u, n)
    plan.sync()
    plan.close()
    return u.cpu().numpy()


CASES = [
    ("1d", (40,), 1 / 40, 0.05, 0.3, 6, 4),
    ("1d-full", (24,), 1 / 24, 0.08, -0.5, 0, 3),
    ("2d", (16, 20), (1 / 16, 1 / 20), 0.06, (0.4, -0.2), (2, 3), 3),
    ("2d-odd-steps", (12, 10), (1 / 12, 1 / 10), 0.06, (0.1, 0.2), (2, 2), 5),
    ("3d", (6, 8, 10), (1 / 6, 1 / 8, 1 / 10), 0.08, (0.3, -0.1, 0.5), (1, 2, 2), 2),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_against_oracle(case):
    name, shape, dx, h, P, W, n = case
    rng = np.random.default_rng(len(name))
    nd = len(shape)
    modes = rng.integers(-2, 3, size=(4, nd))
    modes[0] = 0
    coef = rng.normal(size=4) * 0.3 + 1j * rng.normal(size=4) * 0.3
    u0 = rng.normal(size=shape) * 0.2
    ref = O.integral_run(u0, dx, h, P, W, modes, coef, n)
    got = gpu_integral(shape, dx, h, P, W, modes, coef, u0, n)
    assert np.max(np.abs(got - ref)) <= 1e-12 * (1 + np.max(np.abs(ref)))


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_no_tables_bitwise(case):
    name, shape, dx, h, P, W, n = case
    nd = len(shape)
    dxd = tuple(1 / 32 for _ in shape) if nd > 1 else 1 / 32
    Pd = tuple(0.25 * (-1) ** a for a in range(nd)) if nd > 1 else 0.25
    rng = np.random.default_rng(3)
    u0 = rng.integers(-2048, 2048, size=shape) / 1024.0
    zero = np.zeros((0, nd), dtype=int)
    got = gpu_integral(shape, dxd, 0.125, Pd, W, zero, [], u0, n)
    assert np.array_equal(got.view(np.int64), O.integral_run(u0, dxd, 0.125, Pd, W, zero, [], n).view(np.int64))
    assert np.array_equal(got.view(np.int64), O.run(u0, dxd, 0.125, Pd, W, None, n).view(np.int64))
    c = np.zeros((1, nd), dtype=int)
    got = gpu_integral(shape, dxd, 0.125, Pd, W, c, [0.375], u0, n)
    assert np.array_equal(got.view(np.int64), O.run(u0, dxd, 0.125, Pd, W, np.full(shape, 0.375), n).view(np.int64))


def test_refused_forms():
    from paper_1210_4090_gb300 import hjlo
    import ctypes
    d = hjlo.make_desc((8,), 1 / 8, 0.1, 0.2, 2, dtype=hjlo.F32_STORAGE)
    out = ctypes.c_void_p()
    assert hjlo.lib().hjlo_integral_create(ctypes.byref(d), 0, None, None, None, ctypes.byref(out)) == 6
    d = hjlo.make_desc((8,), 1 / 8, 0.1, 0.2, 2, algo=hjlo.ALGO_MONGE)
    assert hjlo.lib().hjlo_integral_create(ctypes.byref(d), 0, None, None, None, ctypes.byref(out)) == 6
    assert hjlo.lib().hjlo_integral_destroy(None) == 0
