"""CPU oracle for the fully discrete Lax--Oleinik scheme (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
may import this module.  It wraps ``hjlo_oracle.c`` (plain C, binary64,
``-ffp-contract=off``) with ctypes and adds the few readouts the paper defines
on top of the scheme.  It shares no code with the CUDA library.

Paper: Bouillard, Faou & Zavidovique, "Fast weak-KAM integrators for separable
Hamiltonian systems".  Sec. 2.3 eq. cost2/eqconvol (one step), Remark rk28
(axis splitting), eq. uN (time loop), Sec. 3.3 eq. los (torus grid, lift-
minimised cost), Prop. prop:klm (discrete effective Hamiltonian), Appendix B
eq. raslebol (discrete optimal path; the adjoint follows it).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hjlo_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libhjlo_oracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (binary64, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            i64, f64, i32 = ctypes.c_int64, ctypes.c_double, ctypes.c_int
            P = ctypes.POINTER
            L.hjo_kernel.restype = f64
            L.hjo_kernel.argtypes = [i64, f64, f64, f64]
            L.hjo_window.restype = i32
            L.hjo_window.argtypes = [i64, f64, f64, f64, i64, P(i64), P(i64)]
            L.hjo_table.restype = None
            L.hjo_table.argtypes = [i64, i64, f64, f64, f64, P(f64)]
            run_args = [i32, P(i64), P(f64), f64, P(f64), P(i64), ctypes.c_void_p,
                        ctypes.c_void_p, i64, i64, ctypes.c_void_p, i32]
            L.hjo_run_f64.restype = i32
            L.hjo_run_f64.argtypes = run_args
            L.hjo_run_f32.restype = i32
            L.hjo_run_f32.argtypes = run_args
            L.hjo_adjoint_f64.restype = i32
            L.hjo_adjoint_f64.argtypes = [i32, P(i64), P(f64), f64, P(f64), P(i64), P(f64),
                                          ctypes.c_void_p, i64, i64, P(f64), P(f64), P(f64),
                                          P(f64), i32]
            L.hjo_step_points_f64.restype = i32
            L.hjo_step_points_f64.argtypes = [i32, P(i64), P(f64), f64, P(f64), P(i64), P(f64),
                                              ctypes.c_void_p, i64, P(i64), P(f64), i32]
            L.hjo_max_threads.restype = i32
            L.hjo_max_threads.argtypes = []
            _lib = L
    return _lib


def _vec(x, n, dtype):
    a = np.atleast_1d(np.asarray(x, dtype=dtype))
    if a.size == 1 and n > 1:
        a = np.repeat(a, n)
    if a.size != n:
        raise ValueError("expected %d per-axis values, got %d" % (n, a.size))
    return np.ascontiguousarray(a)


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def max_threads() -> int:
    return int(lib().hjo_max_threads())


def kernel(d: int, dx: float, h: float, P: float) -> float:
    """k[d] = h*L(d*dx/h), L(v) = v^2/2 - P v (eq. cost2, pinned binary64 order)."""
    return float(lib().hjo_kernel(int(d), float(dx), float(h), float(P)))


def window(N: int, dx: float, h: float, P: float, W: int) -> tuple[int, int]:
    """Displacement window [dlo, dhi]: 2W+1 centred on the kernel minimiser, or
    the N lift-minimising displacements when W <= 0 or 2W+1 >= N (eq. los)."""
    lo, hi = ctypes.c_int64(), ctypes.c_int64()
    if lib().hjo_window(int(N), float(dx), float(h), float(P), int(W), ctypes.byref(lo), ctypes.byref(hi)):
        raise ValueError("invalid window arguments")
    return lo.value, hi.value


def table(N: int, dx: float, h: float, P: float, W: int):
    """(dlo, dhi, k) with k[d - dlo] for d in [dlo, dhi]."""
    dlo, dhi = window(N, dx, h, P, W)
    k = np.empty(dhi - dlo + 1, dtype=np.float64)
    lib().hjo_table(dlo, dhi, float(dx), float(h), float(P), _ptr(k, ctypes.c_double))
    return dlo, dhi, k


def run(u0, dx, h, P, W, V=None, nsteps: int = 1, *, V_per_step: bool = False,
        record_argmin: bool = False, nthreads: int = 0):
    """nsteps of the scheme (eq. uN), returning u^nsteps (and argmins).

    u0: binary64 or binary32 array (1..3 dims, last axis contiguous); a
    binary32 array selects the binary32-storage scheme.  V: None, an array of
    u0's shape (time-independent) or, with V_per_step, shape (nsteps, *shape).
    Argmins are the displacement d of every pass, shape (nsteps, ndim, *shape).
    """
    u0 = np.asarray(u0)
    if u0.dtype not in (np.float64, np.float32):
        raise TypeError("u0 must be float64 or float32")
    ndim = u0.ndim
    shape = _vec(u0.shape, ndim, np.int64)
    dxv, Pv, Wv = _vec(dx, ndim, np.float64), _vec(P, ndim, np.float64), _vec(W, ndim, np.int64)
    u = np.array(u0, copy=True, order="C")
    npts = u.size
    vptr, vstride = None, 0
    if V is not None:
        Va = np.ascontiguousarray(V, dtype=np.float64)
        want = (nsteps, *u.shape) if V_per_step else u.shape
        if Va.shape != tuple(want):
            raise ValueError("V has shape %s, expected %s" % (Va.shape, want))
        vptr, vstride = Va.ctypes.data, (npts if V_per_step else 0)
    amin = None
    if record_argmin:
        amin = np.zeros((nsteps, ndim, *u.shape), dtype=np.int32)
    fn = lib().hjo_run_f64 if u.dtype == np.float64 else lib().hjo_run_f32
    rc = fn(ndim, _ptr(shape, ctypes.c_int64), _ptr(dxv, ctypes.c_double), float(h),
            _ptr(Pv, ctypes.c_double), _ptr(Wv, ctypes.c_int64), u.ctypes.data, vptr, vstride,
            int(nsteps), None if amin is None else amin.ctypes.data, int(nthreads))
    if rc:
        raise ValueError("oracle rejected its arguments")
    return (u, amin) if record_argmin else u


def step_points(u, dx, h, P, W, V, points, *, nthreads: int = 0):
    """One binary64 step evaluated only at the given flat indices (sampling)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    ndim = u.ndim
    shape = _vec(u.shape, ndim, np.int64)
    dxv, Pv, Wv = _vec(dx, ndim, np.float64), _vec(P, ndim, np.float64), _vec(W, ndim, np.int64)
    pts = np.ascontiguousarray(points, dtype=np.int64).ravel()
    out = np.empty(pts.size, dtype=np.float64)
    vptr = None
    if V is not None:
        Va = np.ascontiguousarray(V, dtype=np.float64)
        if Va.shape != u.shape:
            raise ValueError("V must have u's shape")
        vptr = Va.ctypes.data
    rc = lib().hjo_step_points_f64(ndim, _ptr(shape, ctypes.c_int64), _ptr(dxv, ctypes.c_double), float(h),
                                   _ptr(Pv, ctypes.c_double), _ptr(Wv, ctypes.c_int64),
                                   _ptr(u, ctypes.c_double), vptr, pts.size, _ptr(pts, ctypes.c_int64),
                                   _ptr(out, ctypes.c_double), int(nthreads))
    if rc:
        raise ValueError("oracle rejected its arguments")
    return out


def adjoint(u0, dx, h, P, W, V, nsteps: int, ubar_n, *, V_per_step: bool = False, nthreads: int = 0):
    """Gradient of J = <ubar_n, u^nsteps> w.r.t. u^0, P (per axis) and V.

    Follows the discrete optimal path (eq. raslebol): each value of a pass came
    from exactly one source, so the cotangent is routed back along the argmin.
    Returns (ubar0, Pbar, Vbar); Vbar has V's shape (static or per step).
    """
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    ndim = u0.ndim
    shape = _vec(u0.shape, ndim, np.int64)
    dxv, Pv, Wv = _vec(dx, ndim, np.float64), _vec(P, ndim, np.float64), _vec(W, ndim, np.int64)
    npts = u0.size
    if V is None:
        V = np.zeros(u0.shape)
        V_per_step = False
    Va = np.ascontiguousarray(V, dtype=np.float64)
    ub = np.ascontiguousarray(ubar_n, dtype=np.float64)
    ubar0 = np.zeros_like(u0)
    Pbar = np.zeros(ndim)
    Vbar = np.zeros(Va.shape)
    rc = lib().hjo_adjoint_f64(ndim, _ptr(shape, ctypes.c_int64), _ptr(dxv, ctypes.c_double), float(h),
                               _ptr(Pv, ctypes.c_double), _ptr(Wv, ctypes.c_int64),
                               _ptr(u0, ctypes.c_double), Va.ctypes.data, npts if V_per_step else 0,
                               int(nsteps), _ptr(ub, ctypes.c_double), _ptr(ubar0, ctypes.c_double),
                               _ptr(Pbar, ctypes.c_double), _ptr(Vbar, ctypes.c_double), int(nthreads))
    if rc:
        raise ValueError("oracle rejected its arguments")
    return ubar0, Pbar, Vbar


def hbar_estimate(u0, un, nsteps: int, h: float):
    """Discrete effective Hamiltonian readout (Prop. prop:klm, sign of u_t + H = 0):
    (-mean, -max, -min) of (u^n - u^0)/(n h) over the grid."""
    r = (np.asarray(un, dtype=np.float64) - np.asarray(u0, dtype=np.float64)) / (nsteps * h)
    return float(-r.mean()), float(-r.max()), float(-r.min())


def step_matrix(shape, dx, h, P, W, V=None) -> np.ndarray:
    """One time step as a (min,plus) matrix B (Remark after Prop. prop:klm):
    u^{n+1}(x) = min_y u^n(y) + B[y, x] with B[y, x] = sum_a k_a[d_a] - h V(x),
    d_a the displacement in axis a's window with d_a = x_a - y_a (mod N_a), and
    +inf where no displacement of the window reaches.  Row-major flat indices.
    The entries are sums in a different order from the scheme's passes, so the
    matrix product agrees with the scheme up to rounding."""
    shape = tuple(int(s) for s in np.atleast_1d(shape))
    ndim = len(shape)
    dxv, Pv, Wv = _vec(dx, ndim, np.float64), _vec(P, ndim, np.float64), _vec(W, ndim, np.int64)
    B = np.zeros([1] * (2 * ndim))
    for a, N in enumerate(shape):
        dlo, dhi, k = table(N, float(dxv[a]), float(h), float(Pv[a]), int(Wv[a]))
        Ka = np.full((N, N), np.inf)
        for d in range(dlo, dhi + 1):
            for y in range(N):
                x = (y + d) % N
                Ka[y, x] = min(Ka[y, x], k[d - dlo])
        sh = [1] * (2 * ndim)
        sh[a], sh[ndim + a] = N, N
        B = B + Ka.reshape(sh)                       # axes (y_0..y_n, x_0..x_n)
    npts = int(np.prod(shape))
    B = B.reshape(npts, npts)
    if V is not None:
        hV = float(h) * np.asarray(V, dtype=np.float64).reshape(npts)
        B = B - hV[None, :]
    return B


def minplus_eigenvalue(B: np.ndarray) -> float:
    """The (min,plus) eigenvalue of a matrix whose graph y -> x (weight
    B[y, x]) is strongly connected: its minimum cycle mean, by Karp's theorem
    (R. M. Karp, 1978), with walks allowed to start at any node:
    D_k(x) = min weight of a k-edge walk ending at x, and
    lambda = min_x max_{0 <= k < n} (D_n(x) - D_k(x)) / (n - k).
    For the step matrix, u^n / n -> lambda (Prop. prop:klm), so the discrete
    effective Hamiltonian of the readout is -lambda / h."""
    B = np.asarray(B, dtype=np.float64)
    n = B.shape[0]
    D = np.empty((n + 1, n))
    D[0] = 0.0
    for k in range(1, n + 1):
        D[k] = np.min(D[k - 1][:, None] + B, axis=0)
    best = np.inf
    for x in range(n):
        if not np.isfinite(D[n, x]):
            continue
        fin = np.isfinite(D[:n, x])
        ks = np.arange(n)[fin]
        worst = np.max((D[n, x] - D[ks, x]) / (n - ks))
        best = min(best, worst)
    return float(best)


# ---------------------------------------------------------------------------
# The paper's own fast (min,plus)-convolution (Sec. 4): decompose the source
# line into convex and concave components, convolve each with the convex
# kernel in linear time, take the minimum.  Plain Python loops (small cases).
# Every output value is one candidate u(y) + k(d), as in the scheme, so the
# result is never below the scheme's and equals it wherever the kept
# candidates include a minimiser (always, in exact arithmetic, at eta = 0).

def convex_convex(f, g):
    """f on [0, n] and g on [0, m] convex (Theorem th:convex, Algorithm 1):
    the pieces of f and g put end to end by increasing slope -- f's piece
    first when its slope is strictly smaller, as in Algorithm 1.  The vertex
    after i pieces of f and j of g has the value f(i) + g(j) (the telescoped
    running sum of Algorithm 1).  Returns h on [0, n + m]."""
    n, m = len(f) - 1, len(g) - 1
    h = np.empty(n + m + 1)
    i = j = 0
    h[0] = f[0] + g[0]
    while i + j < n + m:
        if i < n and (j == m or (f[i + 1] - f[i]) < (g[j + 1] - g[j])):
            i += 1
        else:
            j += 1
        h[i + j] = f[i] + g[j]
    return h


def convex_concave(f, g):
    """f on [0, n] convex, g on [0, m] concave, m >= 1 (Lemmas lm:seg and
    lm:simplif, Theorem th:ccc; Algorithm 2 walks the same three parts).
    With rho_j = g(j+1) - g(j) and alpha_j the first vertex of f whose next
    slope f(i+1) - f(i) is >= rho_j (n if none):
      (i)   f(x) + g(0)            for x in [0, alpha_0]          (first convex part)
      (ii)  f(alpha_j) + g(j), f(alpha_j) + g(j+1)
                                   at x = j + alpha_j, j + 1 + alpha_j  (concave part)
      (iii) f(x - m) + g(m)        for x in [m + alpha_{m-1}, m + n]  (last convex part)
    and h is their pointwise minimum on [0, n + m]."""
    n, m = len(f) - 1, len(g) - 1
    h = np.full(n + m + 1, np.inf)

    def alpha(rho):
        for i in range(n):
            if f[i + 1] - f[i] >= rho:
                return i
        return n

    a0 = alpha(g[1] - g[0])
    for x in range(a0 + 1):
        h[x] = min(h[x], f[x] + g[0])
    for j in range(m):
        a = alpha(g[j + 1] - g[j])
        h[j + a] = min(h[j + a], f[a] + g[j])
        h[j + 1 + a] = min(h[j + 1 + a], f[a] + g[j + 1])
        if j == m - 1:
            for x in range(m + a, m + n + 1):
                h[x] = min(h[x], f[x - m] + g[m])
    return h


def decompose(g, eta: float = 0.0):
    """Split g[0..L-1] into consecutive components sharing their end points
    (Sec. 4.3 step 1, with the tolerance of Sec. 4.4): the first slope
    increment of a component fixes its kind -- convex when it is >= -eta,
    concave otherwise -- and the component is extended while the following
    increments keep the kind (convex: >= -eta; concave: <= 0).  Returns
    [(start, end, convex)]; a single point is one convex component."""
    L = len(g)
    if L == 1:
        return [(0, 0, True)]
    rho = [g[p + 1] - g[p] for p in range(L - 1)]
    out = []
    s = 0
    while s < L - 1:
        e = s + 1
        if e == L - 1:
            out.append((s, e, True))
            break
        convex = (rho[s + 1] - rho[s]) >= -eta
        while e + 1 <= L - 1:
            inc = rho[e] - rho[e - 1]
            if not (inc >= -eta if convex else inc <= 0.0):
                break
            e += 1
        out.append((s, e, convex))
        s = e
    return out


def decomp_line(src, k, eta: float = 0.0):
    """One line of an axis pass by the decomposition method (Sec. 4.3).
    k[i] = k_a[dlo + i] for i in [0, n] (n = dhi - dlo) is the convex kernel;
    src[y'] = u((y' - dhi) mod N) for y' in [0, N + n) is the lifted source
    line, so that output x in [0, N) is the minimum over i of
    src[x + n - i] + k[i], i.e. entry x + n of the (min,plus) convolution of
    src and k.  Returns (the N outputs, the number of components)."""
    n = len(k) - 1
    L = len(src)
    N = L - n
    comps = decompose(src, eta)
    h = np.full(L + n, np.inf)
    for s, e, convex in comps:
        g = src[s:e + 1]
        part = convex_convex(k, g) if (convex or e == s) else convex_concave(k, g)
        h[s:s + len(part)] = np.minimum(h[s:s + len(part)], part)
    return h[n:n + N], len(comps)


def decomp_run(u0, dx, h, P, W, V=None, nsteps: int = 1, eta: float = 0.0, *, V_per_step: bool = False):
    """nsteps of the scheme with every axis pass computed by the decomposition
    method (axis 0 first, then fl(m - fl(h V)) as in the scheme).  eta is the
    tolerance on the increase of the slopes (u(i+1) - u(i)) / dx along the
    line, as the slopes of Sec. 4.1 are taken per unit length: on axis a the
    second differences are compared with -fl(eta * dx_a).  Each line is
    decomposed once per pass (Sec. 4.2-4.3 take the function over one period
    of the torus): the decomposition runs over the line's lifted span, from
    its first source.  Returns (u, total number of components over all lines
    and passes)."""
    u = np.array(u0, dtype=np.float64, copy=True)
    shape = u.shape
    ndim = u.ndim
    dxv, Pv, Wv = _vec(dx, ndim, np.float64), _vec(P, ndim, np.float64), _vec(W, ndim, np.int64)
    tabs = [table(shape[a], float(dxv[a]), float(h), float(Pv[a]), int(Wv[a])) for a in range(ndim)]
    ncomp = 0
    for step in range(nsteps):
        for a in range(ndim):
            dlo, dhi, k = tabs[a]
            N = shape[a]
            n = dhi - dlo
            v = np.moveaxis(u, a, -1)
            out = np.empty_like(v)
            for idx in np.ndindex(*v.shape[:-1]):
                src = v[idx][(np.arange(N + n) - dhi) % N]
                out[idx], c = decomp_line(src, k, float(eta) * float(dxv[a]))
                ncomp += c
            u = np.ascontiguousarray(np.moveaxis(out, -1, a))
        if V is not None:
            Vs = np.asarray(V, dtype=np.float64)
            Vn = Vs[step] if V_per_step else Vs
            u = u - float(h) * Vn
    return u, ncomp


# ---------------------------------------------------------------------------
# The first discrete semigroup (Sec. 2.2, eq. cost1): the cost of a step is
# the action of the straight path from the source y to the target x in time
# tau, c(y, x) = tau K*(v) - int_0^tau V(y + s v) ds, v = (x - y)/tau, and
# T u(x) = min_y u(y) + c(y, x) over the window box (the potential term no
# longer separates, so there is no axis splitting).  V is a finite Fourier
# series on the torus of side L_a = N_a dx_a,
# V(x) = Re sum_m c_m exp(2 pi i sum_a k_ma x_a / L_a), for which the path
# integral is exact:  tau Re sum_m c_m exp(i alpha_m(y)) phi(theta_m(D)),
# alpha_m(y) = 2 pi sum_a k_ma y_a / L_a, theta_m(D) = 2 pi sum_a k_ma D_a / L_a,
# D = x - y (lifted), phi(theta) = (exp(i theta) - 1)/(i theta), phi(0) = 1.

def trig_values(shape, modes, coef):
    """V on the grid points i_a dx_a of the torus (phases 2 pi k_a i_a / N_a)."""
    shape = tuple(int(s) for s in shape)
    grids = np.meshgrid(*[np.arange(n) / n for n in shape], indexing="ij")
    V = np.zeros(shape)
    for k, c in zip(np.asarray(modes).reshape(len(coef), -1), coef):
        th = 2 * np.pi * sum(int(ka) * g for ka, g in zip(k, grids))
        V = V + (np.real(c) * np.cos(th) - np.imag(c) * np.sin(th))
    return V


def path_integral(modes, coef, y, D, tau, L=1.0):
    """int_0^tau V(y + s D / tau) ds in closed form (points y, lifted
    displacements D, both (..., ndim) arrays; L: the torus sides)."""
    y = np.asarray(y, dtype=np.float64) / np.asarray(L, dtype=np.float64)
    D = np.asarray(D, dtype=np.float64) / np.asarray(L, dtype=np.float64)
    out = 0.0
    for k, c in zip(np.asarray(modes).reshape(len(coef), -1), coef):
        k = k.astype(np.float64)
        a = 2 * np.pi * (y @ k)
        th = 2 * np.pi * (D @ k)
        small = np.abs(th) < 1e-300
        ths = np.where(small, 1.0, th)
        pre = np.where(small, 1.0, np.sin(ths) / ths)
        pim = np.where(small, 0.0, (1 - np.cos(ths)) / ths)
        are = np.real(c) * np.cos(a) - np.imag(c) * np.sin(a)
        aim = np.real(c) * np.sin(a) + np.imag(c) * np.cos(a)
        out = out + (are * pre - aim * pim)
    return tau * out


def integral_run(u0, dx, h, P, W, modes, coef, nsteps: int = 1):
    """nsteps of the first discrete semigroup (eq. cost1, time-independent V
    as a Fourier series, exact path integral).  Per candidate, in binary64:
    fl(fl(u(y) + K(d)) - fl(h * S)), K(d) = k_0[d_0] + k_1[d_1] + ... (eq.
    cost2's kernel tables, left to right), S = sum over modes in order of
    fl(fl(Are Pre) - fl(Aim Pim)) with A = c_m exp(i alpha_m(y)) and
    (Pre, Pim) = phi(theta_m(D)) = (sin theta / theta, (1 - cos theta) / theta).
    Windows as in the scheme, per axis; the minimum runs over the whole box
    of displacements."""
    u = np.array(u0, dtype=np.float64, copy=True)
    shape = u.shape
    ndim = u.ndim
    dxv, Pv, Wv = _vec(dx, ndim, np.float64), _vec(P, ndim, np.float64), _vec(W, ndim, np.int64)
    tabs = [table(shape[a], float(dxv[a]), float(h), float(Pv[a]), int(Wv[a])) for a in range(ndim)]
    modes = np.asarray(modes, dtype=np.int64).reshape(len(coef), ndim)
    grids = np.meshgrid(*[np.arange(n) / n for n in shape], indexing="ij")
    A = []
    for k, c in zip(modes, coef):
        a = 2 * np.pi * sum(float(ka) * g for ka, g in zip(k, grids))
        ca, sa = np.cos(a), np.sin(a)
        A.append((np.real(c) * ca - np.imag(c) * sa, np.real(c) * sa + np.imag(c) * ca))
    ranges = [range(t[0], t[1] + 1) for t in tabs]
    idx = np.indices(shape)
    for _ in range(nsteps):
        best = np.full(shape, np.inf)
        for d in np.ndindex(*[len(r) for r in ranges]):
            dd = [ranges[a][d[a]] for a in range(ndim)]
            Kd = 0.0
            for a in range(ndim):
                Kd = Kd + tabs[a][2][d[a]]
            ys = tuple((idx[a] - dd[a]) % shape[a] for a in range(ndim))
            S = np.zeros(shape)
            for m, k in enumerate(modes):
                th = 2 * np.pi * sum(float(k[a]) * dd[a] / shape[a] for a in range(ndim))
                if th == 0.0:
                    pre, pim = 1.0, 0.0
                else:
                    pre, pim = np.sin(th) / th, (1.0 - np.cos(th)) / th
                S = S + (A[m][0][ys] * pre - A[m][1][ys] * pim)
            cand = (u[ys] + Kd) - float(h) * S
            best = np.minimum(best, cand)
        u = best
    return u
