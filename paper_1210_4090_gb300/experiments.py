"""The paper's two 1D experiments (Sec. 5) as convergence studies.

Both run the scheme on (0, 2 pi] with 2K points, tau ~ sqrt(dx) and T = 8:
the pendulum (P = 0, V = 1 - cos x) and the time-dependent potential
(P = 1, V = cos(2x) sin t), u0 = cos x.  Sec. 5 measures the relative sup-norm
error at T against a fifth-order WENO solution and observes order 1/2 in dx
(Theorem approx2 with tau = sqrt(dx)).  WENO is a third-party solver and is
not built here: the reference is the scheme itself on a finer nested grid
(coarse point x_i = (i+1) pi/K is fine point (i+1) K_ref/K - 1).

`solve` maps a workloads.Problem to u at its final time; the default runs the
CUDA library (hjlo_run, or hjlo_run_tv for a time-dependent V).
"""
from __future__ import annotations

import numpy as np

from . import workloads as WL

__all__ = ["solve_gpu", "solve_decomp_gpu", "restrict", "relative_error", "convergence", "LAWS"]

LAWS = {"pendulum": WL.pendulum, "tdep": WL.tdep}


def solve_gpu(p: WL.Problem) -> np.ndarray:
    """u at the problem's final time through the CUDA path."""
    import torch
    from . import hjlo
    plan = hjlo.Plan(p.shape, p.dx, p.h, p.P, p.W)
    try:
        u = torch.tensor(p.u0, dtype=torch.float64, device="cuda")
        V = torch.tensor(p.V, dtype=torch.float64, device="cuda")
        if p.V_per_step:
            plan.run_tv(u, V, p.nsteps)
        else:
            plan.run(u, V, p.nsteps)
        cnt = plan.sync()
        if cnt["error_flags"]:
            raise RuntimeError("device error flags %d" % cnt["error_flags"])
        return u.cpu().numpy()
    finally:
        plan.close()


def solve_decomp_gpu(p: WL.Problem, eta: float = 0.0, nsteps: int | None = None, restart_blocks: bool = False):
    """u after nsteps (default: to the problem's final time) by the paper's
    own method (Sec. 4, HJLO_ALGO_DECOMP) at tolerance eta on the slopes
    (per unit length, as Sec. 4.1 takes them; the paper's timed run uses
    eta = dx), and the components per line and pass.  Each period is
    decomposed whole unless restart_blocks asks for the row-block
    approximation."""
    import torch
    from . import hjlo
    n = p.nsteps if nsteps is None else int(nsteps)
    plan = hjlo.Plan(p.shape, p.dx, p.h, p.P, p.W, algo=hjlo.ALGO_DECOMP)
    try:
        plan.set_tolerance(float(eta), restart_blocks=restart_blocks)
        u = torch.tensor(p.u0, dtype=torch.float64, device="cuda")
        V = None if p.V is None else torch.tensor(p.V, dtype=torch.float64, device="cuda")
        if p.V_per_step:
            plan.run_tv(u, V, n)
        else:
            plan.run(u, V, n)
        cnt = plan.sync()
        if cnt["error_flags"]:
            raise RuntimeError("device error flags %d" % cnt["error_flags"])
        lines = sum(int(np.prod(p.shape)) // s for s in p.shape)
        return u.cpu().numpy(), cnt["components"] / max(1, n * lines)
    finally:
        plan.close()


def restrict(u_ref: np.ndarray, K_ref: int, K: int) -> np.ndarray:
    """Values of a solution on 2 K_ref points at the 2K points of the coarse
    grid (K divides K_ref; grids x_i = (i+1) pi/K are nested)."""
    if K_ref % K:
        raise ValueError("K must divide K_ref")
    r = K_ref // K
    return u_ref[(np.arange(2 * K) + 1) * r - 1]


def relative_error(u: np.ndarray, ref: np.ndarray) -> float:
    """Relative sup-norm error, the measure of Sec. 5."""
    return float(np.max(np.abs(u - ref)) / np.max(np.abs(ref)))


def convergence(law: str, Ks, K_ref: int, solve=solve_gpu, **kw) -> dict:
    """Errors at T of the scheme on 2K points (K in Ks) against the scheme on
    2 K_ref points, and the least-squares order in dx."""
    make = LAWS[law]
    pr = make(K_ref, **kw)
    ref = solve(pr)
    rows = []
    for K in Ks:
        p = make(K, **kw)
        u = solve(p)
        rows.append({"K": int(K), "N": int(p.shape[0]), "dx": float(p.dx[0]), "tau": float(p.h),
                     "nsteps": int(p.nsteps), "W": int(p.W[0]),
                     "error": relative_error(u, restrict(ref, K_ref, K))})
    dx = np.array([r["dx"] for r in rows])
    err = np.array([r["error"] for r in rows])
    order = float(np.polyfit(np.log(dx), np.log(err), 1)[0]) if len(rows) >= 2 else float("nan")
    return {"law": law, "K_ref": int(K_ref), "T": float(pr.extra["T"]), "rows": rows, "order": order}
