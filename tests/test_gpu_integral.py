"""The first discrete semigroup (eq. cost1) on the GPU against the oracle.

The kinetic part K and the final add, multiply and subtract of a candidate,
fl(fl(u(y) + K) - fl(h S)), are the same binary64 operations on both sides.
The path-integral sum S = sum_m (Are_m Pre_m - Aim_m Pim_m) is not: the
oracle forms each product, the difference and a running sum in mode order,
the kernel accumulates fused multiply-adds in two chains (even and odd
modes) added at the end, and the trigonometric tables come from different
libraries (the C library's sin / cos on the host, numpy's in the oracle).
The bound the values are compared to, per case:
  * |Are|, |Aim| <= |c_m| and |Pre|, |Pim| <= 1, so every partial sum and the
    sum of the terms' magnitudes are at most C = sum_m 2 |c_m|;
  * a sum of 2M products with one rounding per operation, in any order and
    with or without fusing, is within (2M + 1) u C of the exact S
    (u = 2^-53), for each side; the tables' libm results within 4 ulp each
    move a term by at most 9 u of its magnitude: |S_gpu - S_oracle| <=
    (4M + 2 + 9) u C, and h times that after the multiply by h;
  * the multiply by h, the subtract and the add of u(y) + K round on both
    sides: at most 2 ulp of the largest of |u| + |K| + h C;
  * a step is a sup-norm contraction (the minimum of the candidates), so the
    per-step differences add up over n steps.
With V = 0 or a constant V there are no tables and the result is bit for bit
the oracle's, and on dyadic data the fully discrete scheme's."""
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
    u, M = 2.0 ** -53, len(coef)
    C = 2.0 * float(np.sum(np.abs(coef)))
    dxv = dx if nd > 1 else (dx,)
    Pv = P if nd > 1 else (P,)
    Wv = W if nd > 1 else (W,)
    Kmax = sum(float(np.max(np.abs(O.table(shape[a], dxv[a], h, Pv[a], Wv[a])[2]))) for a in range(nd))
    umax = max(float(np.max(np.abs(u0))), float(np.max(np.abs(ref)))) + Kmax + h * C
    bound = n * (h * (4 * M + 11) * u * C + 4 * u * umax)
    assert np.max(np.abs(got - ref)) <= bound, (np.max(np.abs(got - ref)), bound)


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
