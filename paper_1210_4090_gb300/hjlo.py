"""Python binding of the hjlo C ABI (include/hjlo.h): argument marshalling only.

Every step of the scheme runs in the library's sm_103a kernels; this module
checks tensors, passes raw device pointers and the torch stream handle, and
turns status codes into exceptions.  There is no CPU fallback: if the
compiled library cannot be loaded, importing it raises.

    plan = Plan(shape=(1024, 1024), dx=1/1024, h=0.02, P=(0.3, 0.1), W=64)
    plan.run(u, V, nsteps=1000)          # u: cuda float64 tensor, in place
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

__all__ = ["Plan", "Batch", "IntegralPlan", "HjloError", "lib", "library_path", "exported_symbols", "step_noalloc",
           "F64", "F32_STORAGE", "ALGO_AUTO", "ALGO_BRUTE", "ALGO_MONGE", "ALGO_DECOMP"]

F64, F32_STORAGE = 0, 1
ALGO_AUTO, ALGO_BRUTE, ALGO_MONGE, ALGO_DECOMP = 0, 1, 2, 3
_STATUS = {0: "HJLO_OK", 1: "HJLO_EINVAL", 2: "HJLO_ENOMEM", 3: "HJLO_ECUDA", 4: "HJLO_EPRECOND",
           5: "HJLO_ETIMEOUT", 6: "HJLO_EUNSUPPORTED"}

_i32, _i64, _f64, _vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p


class Desc(ctypes.Structure):
    _fields_ = [("ndim", _i32), ("dtype", _i32), ("algo", _i32), ("reserved", _i32),
                ("shape", _i64 * 3), ("dx", _f64 * 3), ("h", _f64), ("P", _f64 * 3),
                ("window", _i64 * 3)]


class Facts(ctypes.Structure):
    _fields_ = [("ndim", _i32), ("algo", _i32), ("dlo", _i64 * 3), ("dhi", _i64 * 3),
                ("centre", _i64 * 3), ("kmin", _f64 * 3), ("curvature", _f64 * 3), ("npts", _i64),
                ("row_blocks", _i64 * 3), ("block_rows", _i64 * 3), ("split_chunks", _i64 * 3)]


class Counters(ctypes.Structure):
    _fields_ = [("exact_rescans", _i64), ("brute_fallback_lines", _i64), ("steps", _i64),
                ("error_flags", _i32), ("reserved", _i32), ("components", _i64),
                ("window_edge_hits", _i64)]


class TuneReport(ctypes.Structure):
    _fields_ = [("lanes_per_line", _i32 * 3), ("lines_per_tile", _i32 * 3), ("offload", _i32 * 3),
                ("trials", _i32), ("ms_initial", _f64), ("ms_tuned", _f64)]

    def as_dict(self) -> dict:
        return {"lanes_per_line": list(self.lanes_per_line), "lines_per_tile": list(self.lines_per_tile),
                "offload": list(self.offload), "trials": self.trials, "ms_initial": self.ms_initial,
                "ms_tuned": self.ms_tuned}


class HjloError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        self.name = _STATUS.get(status, str(status))
        super().__init__("%s failed: %s (%s)" % (where, self.name, msg))


_lock = threading.Lock()
_lib = None

# (name, restype, argtypes) of every entry point declared in include/hjlo.h
class ShapeInfo(ctypes.Structure):
    _fields_ = [("lanes_per_line", _i32), ("segment_rows", _i32), ("lines_per_tile", _i32), ("threads", _i32),
                ("smem_bytes", _i64), ("tiles", _i64), ("row_blocks", _i64), ("block_rows", _i64),
                ("line_points", _i64), ("split_chunks", _i64), ("split_rows", _i64)]


_SIGS = [
    ("hjlo_version", _i32, []),
    ("hjlo_shape_query", _i32, [_i64, _i64, _i64, _i32, _i32, _i32, _i64, ctypes.POINTER(ShapeInfo)]),
    ("hjlo_last_error", ctypes.c_char_p, []),
    ("hjlo_plan_create", _i32, [ctypes.POINTER(Desc), _vp, ctypes.POINTER(_vp)]),
    ("hjlo_plan_destroy", _i32, [_vp]),
    ("hjlo_plan_info", _i32, [_vp, ctypes.POINTER(Facts)]),
    ("hjlo_plan_set_tolerance", _i32, [_vp, _f64]),
    ("hjlo_plan_set_decomp", _i32, [_vp, _f64, _i32]),
    ("hjlo_probe_fp64_add", _i32, [_i64, _vp, _vp]),
    ("hjlo_noalloc_status", _i32, [_vp, _vp]),
    ("hjlo_batch_set_persistent", _i32, [_vp, _i32]),
    ("hjlo_plan_autotune", _i32, [_vp, _vp, _vp, _i64, ctypes.POINTER(TuneReport)]),
    ("hjlo_integral_create", _i32, [ctypes.POINTER(Desc), _i32, ctypes.POINTER(_i32), ctypes.POINTER(_f64), _vp,
                                    ctypes.POINTER(_vp)]),
    ("hjlo_integral_run", _i32, [_vp, _vp, _i64]),
    ("hjlo_integral_sync", _i32, [_vp]),
    ("hjlo_integral_destroy", _i32, [_vp]),
    ("hjlo_batch_autotune", _i32, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i64,
                                   ctypes.POINTER(TuneReport)]),
    ("hjlo_step", _i32, [_vp, _vp, _vp, _vp, _vp]),
    ("hjlo_run", _i32, [_vp, _vp, _vp, _i64]),
    ("hjlo_run_tv", _i32, [_vp, _vp, _vp, _i64]),
    ("hjlo_run_host", _i32, [_vp, _vp, _vp, _i64]),
    ("hjlo_hbar", _i32, [_vp, _vp, _vp, _i64, ctypes.POINTER(_f64)]),
    ("hjlo_sync", _i32, [_vp, ctypes.POINTER(Counters)]),
    ("hjlo_step_noalloc", _i32, [ctypes.POINTER(Desc), _vp, _vp, _vp, _vp]),
    ("hjlo_batch_create", _i32, [ctypes.POINTER(Desc), _i32, _vp, ctypes.POINTER(_vp)]),
    ("hjlo_batch_destroy", _i32, [_vp]),
    ("hjlo_batch_run", _i32, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i64]),
    ("hjlo_batch_hbar", _i32, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i64, ctypes.POINTER(_f64)]),
    ("hjlo_batch_sync", _i32, [_vp, ctypes.POINTER(Counters)]),
    ("hjlo_batch_groups", _i32, [_vp]),
    ("hjlo_adjoint", _i32, [_vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp, _i64, _vp]),
    ("hjlo_project", _i32, [_vp, _vp, _vp, _i32, _vp]),
]


def library_path() -> str:
    return _build.LIB


def exported_symbols() -> list[str]:
    return [s[0] for s in _SIGS]


def shape_query(N, lines, weff, esize=8, algo=ALGO_MONGE, num_sms=152, smem_optin=232448) -> dict:
    """The launch shape a plan would use for a contiguous axis (hjlo_shape_query;
    host only, no device)."""
    out = ShapeInfo()
    _check(lib().hjlo_shape_query(int(N), int(lines), int(weff), int(esize), int(algo), int(num_sms),
                                  int(smem_optin), ctypes.byref(out)), "hjlo_shape_query")
    return {f: getattr(out, f) for f, _ in ShapeInfo._fields_}


def probe_fp64_add(iters: int = 1 << 16, stream=None) -> float:
    """The device's binary64 add rate in adds/s (hjlo_probe_fp64_add)."""
    out = ctypes.c_double(0.0)
    _check(lib().hjlo_probe_fp64_add(int(iters), stream, ctypes.byref(out)), "hjlo_probe_fp64_add")
    return float(out.value)


def lib() -> ctypes.CDLL:
    """Load (building first if needed) the compiled library."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            for name, res, args in _SIGS:
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(st: int, where: str):
    if st != 0:
        msg = lib().hjlo_last_error()
        raise HjloError(st, where, msg.decode() if msg else "")


def _per_axis(x, nd, typ):
    a = list(np.atleast_1d(np.asarray(x, dtype=typ)).tolist())
    if len(a) == 1 and nd > 1:
        a = a * nd
    if len(a) != nd:
        raise ValueError("expected %d per-axis values" % nd)
    return a + [typ(0)] * (3 - nd)


def make_desc(shape, dx, h, P, W, dtype=F64, algo=ALGO_AUTO) -> Desc:
    shape = tuple(int(s) for s in np.atleast_1d(shape))
    nd = len(shape)
    d = Desc()
    d.ndim = nd
    d.dtype = int(dtype)
    d.algo = int(algo)
    d.reserved = 0
    d.shape[:] = list(shape) + [1] * (3 - nd)
    d.dx[:] = _per_axis(dx, nd, float)
    d.h = float(h)
    d.P[:] = _per_axis(P, nd, float)
    d.window[:] = _per_axis(W, nd, int)
    return d


def _stream_handle(stream):
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def step_noalloc(u_in, u_out, V, shape, dx, h, P, W=0, dtype=F64, algo=ALGO_AUTO, stream=None):
    """One step through hjlo_step_noalloc (no plan, no allocation): the kernel
    tables live in the library's static device scratch array."""
    import torch
    desc = make_desc(shape, dx, h, P, W, dtype, algo)
    npts = int(np.prod(np.atleast_1d(shape)))
    want = torch.float64 if dtype == F64 else torch.float32
    for t, name in ((u_in, "u_in"), (u_out, "u_out")):
        if not t.is_cuda or t.dtype != want or t.numel() != npts or not t.is_contiguous():
            raise ValueError("%s must be a contiguous CUDA %s tensor with %d elements" % (name, want, npts))
    vp = None
    if V is not None:
        if not V.is_cuda or V.dtype != torch.float64 or V.numel() != npts or not V.is_contiguous():
            raise ValueError("V must be a contiguous CUDA float64 tensor with %d elements" % npts)
        vp = _vp(V.data_ptr())
    _check(lib().hjlo_step_noalloc(ctypes.byref(desc), _vp(_stream_handle(stream)), _vp(u_in.data_ptr()),
                                   _vp(u_out.data_ptr()), vp), "hjlo_step_noalloc")
    return u_out


def noalloc_status(stream=None) -> dict:
    """Device status of the no-allocation steps (hjlo_noalloc_status): waits for
    the stream, returns the counters of the most recent step and raises
    HjloError (HJLO_ETIMEOUT / HJLO_EPRECOND) if a step since the previous
    call raised a device error flag (the flag is cleared)."""
    c = Counters()
    st = lib().hjlo_noalloc_status(_vp(_stream_handle(stream)), ctypes.byref(c))
    res = {"exact_rescans": c.exact_rescans, "brute_fallback_lines": c.brute_fallback_lines,
           "error_flags": c.error_flags, "window_edge_hits": c.window_edge_hits}
    _check(st, "hjlo_noalloc_status")
    return res


class Plan:
    """One grid of the scheme (see hjlo_plan_create).  Tensors are torch CUDA
    tensors of the plan's storage dtype (float64, or float32 for F32_STORAGE);
    V is float64."""

    def __init__(self, shape, dx, h, P, W=0, dtype=F64, algo=ALGO_AUTO, stream=None):
        import torch
        self.shape = tuple(int(s) for s in np.atleast_1d(shape))
        self.ndim = len(self.shape)
        self.npts = int(np.prod(self.shape))
        self.h = float(h)
        self.dtype_code = int(dtype)
        self.torch_dtype = torch.float64 if dtype == F64 else torch.float32
        self._desc = make_desc(shape, dx, h, P, W, dtype, algo)
        self._stream = _stream_handle(stream)
        handle = _vp()
        _check(lib().hjlo_plan_create(ctypes.byref(self._desc), _vp(self._stream), ctypes.byref(handle)),
               "hjlo_plan_create")
        self._h = handle

    # -- helpers
    def _u(self, t, name):
        if not t.is_cuda or t.dtype != self.torch_dtype or t.numel() != self.npts or not t.is_contiguous():
            raise ValueError("%s must be a contiguous CUDA %s tensor with %d elements"
                             % (name, self.torch_dtype, self.npts))
        return _vp(t.data_ptr())

    def _v(self, V, count=1):
        import torch
        if V is None:
            return None
        if not V.is_cuda or V.dtype != torch.float64 or V.numel() != count * self.npts or not V.is_contiguous():
            raise ValueError("V must be a contiguous CUDA float64 tensor with %d elements" % (count * self.npts))
        return _vp(V.data_ptr())

    # -- API
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().hjlo_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def autotune(self, u, V=None, nsteps: int = 8) -> dict:
        """Time launch shapes of the monotone passes on nsteps steps from a copy
        of u and keep the fastest per axis (hjlo_plan_autotune); u is unchanged."""
        r = TuneReport()
        _check(lib().hjlo_plan_autotune(self._h, self._u(u, "u"), self._v(V), int(nsteps), ctypes.byref(r)),
               "hjlo_plan_autotune")
        return r.as_dict()

    def set_tolerance(self, eta: float, restart_blocks: bool = False):
        """Convexity tolerance of an ALGO_DECOMP plan (Sec. 4.4).  Each line is
        decomposed once per pass; restart_blocks=True lets lines too long for
        one CTA run in row blocks that restart the decomposition (an
        approximation, see hjlo_plan_set_decomp)."""
        _check(lib().hjlo_plan_set_decomp(self._h, float(eta), 1 if restart_blocks else 0), "hjlo_plan_set_decomp")

    def info(self) -> dict:
        f = Facts()
        _check(lib().hjlo_plan_info(self._h, ctypes.byref(f)), "hjlo_plan_info")
        nd = f.ndim
        return {"algo": {1: "brute", 2: "monge", 3: "decomp"}.get(f.algo, f.algo), "npts": f.npts,
                "dlo": list(f.dlo[:nd]), "dhi": list(f.dhi[:nd]), "centre": list(f.centre[:nd]),
                "kmin": list(f.kmin[:nd]), "curvature": list(f.curvature[:nd]),
                "row_blocks": list(f.row_blocks[:nd]), "block_rows": list(f.block_rows[:nd]),
                "split_chunks": list(f.split_chunks[:nd])}

    def step(self, u_in, u_out=None, V=None, argmin=None):
        """One step; returns u_out (u_in itself when u_out is None: in place)."""
        import torch
        if u_out is None:
            u_out = u_in
        am = None
        if argmin is not None:
            if argmin.dtype != torch.int32 or argmin.numel() != self.ndim * self.npts or not argmin.is_cuda \
                    or not argmin.is_contiguous():
                raise ValueError("argmin must be a contiguous CUDA int32 tensor of ndim*npts elements")
            am = _vp(argmin.data_ptr())
        _check(lib().hjlo_step(self._h, self._u(u_in, "u_in"), self._u(u_out, "u_out"), self._v(V), am),
               "hjlo_step")
        return u_out

    def run(self, u, V=None, nsteps=1):
        _check(lib().hjlo_run(self._h, self._u(u, "u"), self._v(V), int(nsteps)), "hjlo_run")
        return u

    def run_tv(self, u, V, nsteps):
        _check(lib().hjlo_run_tv(self._h, self._u(u, "u"), self._v(V, int(nsteps)), int(nsteps)), "hjlo_run_tv")
        return u

    def run_host(self, u: np.ndarray, V: np.ndarray | None, nsteps: int):
        """End to end from host arrays (in place on u)."""
        want = np.float64 if self.dtype_code == F64 else np.float32
        if u.dtype != want or u.size != self.npts or not u.flags.c_contiguous:
            raise ValueError("u must be a C-contiguous %s array of %d elements" % (want, self.npts))
        vp = None
        if V is not None:
            if V.dtype != np.float64 or V.size != self.npts or not V.flags.c_contiguous:
                raise ValueError("V must be a C-contiguous float64 array")
            vp = _vp(V.ctypes.data)
        _check(lib().hjlo_run_host(self._h, _vp(u.ctypes.data), vp, int(nsteps)), "hjlo_run_host")
        return u

    def adjoint(self, u0, V, nsteps, ubar_n, checkpoint_every=0, want_P=True, want_V=True, want_un=False):
        """Gradient of <ubar_n, u^nsteps> w.r.t. u0, P and V (hjlo_adjoint).
        Returns (ubar0, Pbar, Vbar, u_n) as CUDA tensors (None where not asked)."""
        import torch
        if self.dtype_code != F64:
            raise ValueError("the adjoint needs a float64 plan")
        ubar0 = torch.empty_like(u0)
        Pbar = torch.empty(self.ndim, dtype=torch.float64, device=u0.device) if want_P else None
        Vbar = torch.empty_like(u0) if want_V else None
        un = torch.empty_like(u0) if want_un else None
        ptr = (lambda t: None if t is None else _vp(t.data_ptr()))
        _check(lib().hjlo_adjoint(self._h, self._u(u0, "u0"), self._v(V), int(nsteps), self._u(ubar_n, "ubar_n"),
                                  ptr(ubar0), ptr(Pbar), ptr(Vbar), int(checkpoint_every), ptr(un)), "hjlo_adjoint")
        return ubar0, Pbar, Vbar, un

    def project(self, field, basis):
        """out[k] = sum_x field(x) basis[k](x) (hjlo_project)."""
        import torch
        nb = basis.shape[0]
        if basis.dtype != torch.float64 or not basis.is_cuda or basis.numel() != nb * self.npts \
                or not basis.is_contiguous():
            raise ValueError("basis must be a contiguous CUDA float64 tensor (nbasis, *shape)")
        out = torch.empty(nb, dtype=torch.float64, device=basis.device)
        _check(lib().hjlo_project(self._h, self._v(field), _vp(basis.data_ptr()), int(nb), _vp(out.data_ptr())),
               "hjlo_project")
        return out

    def hbar(self, u0, un, nsteps):
        out = (_f64 * 3)()
        _check(lib().hjlo_hbar(self._h, self._u(u0, "u0"), self._u(un, "un"), int(nsteps), out), "hjlo_hbar")
        return float(out[0]), float(out[1]), float(out[2])

    def sync(self) -> dict:
        c = Counters()
        st = lib().hjlo_sync(self._h, ctypes.byref(c))
        res = {"exact_rescans": c.exact_rescans, "brute_fallback_lines": c.brute_fallback_lines,
               "steps": c.steps, "error_flags": c.error_flags, "components": c.components,
               "window_edge_hits": c.window_edge_hits}
        _check(st, "hjlo_sync")
        return res


class Batch:
    """Many independent grids advanced together (hjlo_batch_*).  `problems` is a
    list of (shape, dx, h, P, W) tuples; tensors are passed as lists."""

    def __init__(self, problems, dtype=F64, algo=ALGO_AUTO, stream=None):
        import torch
        self.count = len(problems)
        descs = (Desc * self.count)()
        self.npts = []
        for i, (shape, dx, h, P, W) in enumerate(problems):
            descs[i] = make_desc(shape, dx, h, P, W, dtype, algo)
            self.npts.append(int(np.prod(np.atleast_1d(shape))))
        self._descs = descs
        self.torch_dtype = torch.float64 if dtype == F64 else torch.float32
        self._stream = _stream_handle(stream)
        handle = _vp()
        _check(lib().hjlo_batch_create(descs, self.count, _vp(self._stream), ctypes.byref(handle)),
               "hjlo_batch_create")
        self._h = handle

    def _ptrs(self, ts, dtype, name, allow_none=False):
        arr = (_vp * self.count)()
        for i, t in enumerate(ts):
            if t is None and allow_none:
                arr[i] = None
                continue
            if not t.is_cuda or t.dtype != dtype or t.numel() != self.npts[i] or not t.is_contiguous():
                raise ValueError("%s[%d] must be a contiguous CUDA %s tensor with %d elements"
                                 % (name, i, dtype, self.npts[i]))
            arr[i] = t.data_ptr()
        return arr

    def set_persistent(self, on: bool = True):
        """One persistent launch per time step over every instance and axis
        (True) or one launch per group and axis (False); see
        hjlo_batch_set_persistent.  Results are the same bit for bit."""
        _check(lib().hjlo_batch_set_persistent(self._h, 1 if on else 0), "hjlo_batch_set_persistent")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().hjlo_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def groups(self) -> int:
        return int(lib().hjlo_batch_groups(self._h))

    def run(self, us, Vs=None, nsteps=1):
        import torch
        up = self._ptrs(us, self.torch_dtype, "u")
        vp = None if Vs is None else self._ptrs(Vs, torch.float64, "V", allow_none=True)
        _check(lib().hjlo_batch_run(self._h, up, vp, int(nsteps)), "hjlo_batch_run")
        return us

    def autotune(self, us, Vs=None, nsteps: int = 8) -> dict:
        """hjlo_batch_autotune: tune every group's launch shapes on nsteps steps of
        the whole batch from copies of us (unchanged)."""
        import torch
        up = self._ptrs(us, self.torch_dtype, "u")
        vp = None if Vs is None else self._ptrs(Vs, torch.float64, "V", allow_none=True)
        r = TuneReport()
        _check(lib().hjlo_batch_autotune(self._h, up, vp, int(nsteps), ctypes.byref(r)), "hjlo_batch_autotune")
        return r.as_dict()

    def hbar(self, u0s, uns, nsteps):
        out = (_f64 * (3 * self.count))()
        _check(lib().hjlo_batch_hbar(self._h, self._ptrs(u0s, self.torch_dtype, "u0"),
                                     self._ptrs(uns, self.torch_dtype, "un"), int(nsteps), out), "hjlo_batch_hbar")
        return np.array(out[:]).reshape(self.count, 3)

    def sync(self) -> dict:
        c = Counters()
        st = lib().hjlo_batch_sync(self._h, ctypes.byref(c))
        res = {"exact_rescans": c.exact_rescans, "brute_fallback_lines": c.brute_fallback_lines,
               "steps": c.steps, "error_flags": c.error_flags, "window_edge_hits": c.window_edge_hits}
        _check(st, "hjlo_batch_sync")
        return res


class IntegralPlan:
    """The first discrete semigroup (eq. cost1) through hjlo_integral_*: the
    path integral of V = Re sum_m coef[m] exp(2 pi i modes[m] . x / L) is
    exact; every candidate of the window box is evaluated."""

    def __init__(self, shape, dx, h, P, W, modes, coef, stream=None):
        import torch
        self.shape = tuple(int(s) for s in np.atleast_1d(shape))
        nd = len(self.shape)
        self.npts = int(np.prod(self.shape))
        desc = make_desc(shape, dx, h, P, W, F64, ALGO_AUTO)
        modes = np.ascontiguousarray(np.asarray(modes, dtype=np.int32).reshape(-1, nd))
        coef = np.asarray(coef, dtype=np.complex128).reshape(-1)
        if modes.shape[0] != coef.size:
            raise ValueError("one coefficient per mode")
        cf = np.ascontiguousarray(np.stack([coef.real, coef.imag], -1).reshape(-1))
        st = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        h_ = _vp()
        _check(lib().hjlo_integral_create(ctypes.byref(desc), int(coef.size),
                                          modes.ctypes.data_as(ctypes.POINTER(_i32)),
                                          cf.ctypes.data_as(ctypes.POINTER(_f64)), _vp(st), ctypes.byref(h_)),
               "hjlo_integral_create")
        self._h = h_

    def run(self, u, nsteps: int):
        import torch
        if not u.is_cuda or u.dtype != torch.float64 or u.numel() != self.npts or not u.is_contiguous():
            raise ValueError("u must be a contiguous float64 CUDA tensor of %d elements" % self.npts)
        _check(lib().hjlo_integral_run(self._h, _vp(u.data_ptr()), int(nsteps)), "hjlo_integral_run")
        return u

    def sync(self):
        _check(lib().hjlo_integral_sync(self._h), "hjlo_integral_sync")

    def close(self):
        if getattr(self, "_h", None):
            lib().hjlo_integral_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
