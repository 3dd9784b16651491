#!/usr/bin/env python3
"""Throughput of the fully discrete Lax--Oleinik scheme on GB300.

One benchmark step = one complete run of a workload from its initial data
(default: cube256, the 3D 256^3 torus, W = 32, 500 time steps, binary64, the
largest single-instance configuration) through the library's C ABI.  The metric is grid-point updates per second
(points x time steps / time); every result is bit-exact against the CPU
oracle (tests/test_gpu_parity.py).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload cube256|grid1024|line256|sweep512|adjoint512|paper1d|decomp|
                                integral128|peaks] [--algo monge|brute]

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events
on the plan's stream; before each timed step the state is reset to u0 and a
256 MiB buffer is written to flush L2 (cube256's fields, 134 MB each, exceed
L2; the 8 MiB grid of grid1024 is L2-resident within a step, as in any run of
that size).  Barrier and device
synchronisation on both sides of the timed region; the max over ranks is
reported.  Under torchrun every rank runs an independent replica (the single
grid does not shard: "replicas only"); value = all ranks' updates / max time.

The JSON line also carries: e2e (the same run through hjlo_run_host from
page-locked host buffers, copies inside the timed region), roofline of the
dominant kernel (the axis pass), the CPU oracle timed on a bounded sample of
the same workload (cpu_baseline), SM clocks sampled during the timed region
and the number of kernels launched.  --impl reference times the CPU oracle
alone (the reference arm: the paper publishes no code), each step one bounded
sample of the workload's time steps; steps and ms_per_step describe those
samples.  --workload peaks measures the binary64 add rate (the brute-force
pass's roofline) with a probe kernel.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1210_4090_gb300 import workloads as WL  # noqa: E402

METRIC = "grid-point updates/s"
UNIT = "updates/s"
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-autotune", action="store_true", help="keep the cost model's launch shapes")
    ap.add_argument("--workload", choices=["cube256", "grid1024", "line256", "sweep512", "adjoint512", "paper1d",
                                           "decomp", "integral128", "peaks"],
                    default="cube256")
    ap.add_argument("--loop-instances", type=int, default=28,
                    help="sweep512: instances timed one plan at a time for the per-instance loop")
    ap.add_argument("--algo", choices=["monge", "brute", "auto"], default="monge")
    ap.add_argument("--batch-mode", choices=["auto", "grouped", "persistent"], default="auto",
                    help="sweep512: launch mode (auto: the faster on a 64-step trial)")
    ap.add_argument("--dtype", choices=["f64", "f32"], default="f64")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="CPU-oracle sample budget")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(name):
    return WL.WORKLOADS[name]()


def kernel_source_hash() -> str:
    """Hash of the axis-pass kernel's device sources (the kernel an ncu summary
    describes): hjlo_device.cuh and the instantiation units."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1210_4090_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f == "hjlo_device.cuh" or f.startswith("hjlo_kern"):
            h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def profile_traffic(workload_name, algo, dtype):
    """DRAM bytes per pass launch from the committed ncu summary, if it was taken
    on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "pass_kernel_%s_%s_%s.txt" % (workload_name, algo, dtype))
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line and line.split(":", 1)[0].strip() in ("kernel_source_hash", "dram_bytes_per_launch"):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_hash") != kernel_source_hash():
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200"]
            if self.gpu_id:
                cmd += ["-i", self.gpu_id]
            self.proc = subprocess.Popen(cmd, stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    continue
        os.unlink(self.tmp.name)
        if not rows:
            return None
        sm = [r[0] for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower().startswith("active")})
        return {"sm_mhz": float(statistics.median(sm)), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": reasons}


def cpu_oracle_rate(p, budget_s):
    """The oracle as it stands on the host cores, on the first time steps of the
    same workload (after one step timed alone to size the sample); returns
    (updates/s, cores, sample description)."""
    from oracle import oracle as O
    cores = O.max_threads()
    t0 = time.perf_counter()
    u = O.run(p.u0, p.dx, p.h, p.P, p.W, p.V, 1)
    t1 = time.perf_counter() - t0
    n = int(max(1, min(p.nsteps - 1, budget_s / max(t1, 1e-9))))
    t0 = time.perf_counter()
    O.run(u, p.dx, p.h, p.P, p.W, p.V, n)
    dt = time.perf_counter() - t0
    rate = p.npts * n / dt
    sample = "%s %s, time steps 2..%d of %d (%d steps, %.1f s), %d OpenMP threads" % (
        p.name, "x".join(map(str, p.shape)), n + 1, p.nsteps, n, dt, cores)
    return rate, cores, sample


def run_reference(args):
    """The reference arm: the CPU oracle on the host cores.  Every step (warm-up
    or timed) is one bounded sample -- the next consecutive time steps of the
    workload, as many as fit the per-sample budget -- so steps and ms_per_step
    describe exactly the work timed; value = updates / time over the timed
    samples."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    p = workload(args.workload)
    from oracle import oracle as O
    O.build()
    per = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    # steps of the workload per sample, from a first step timed alone
    t0 = time.perf_counter()
    u = O.run(p.u0, p.dx, p.h, p.P, p.W, p.V, 1)
    first = time.perf_counter() - t0
    k = int(max(1, min(max(1, (p.nsteps - 1) // max(1, args.steps + args.warmup)), per / max(first, 1e-9))))
    done = 1
    cores = O.max_threads()
    secs, upd, samples = [], [], []
    for i in range(args.warmup + args.steps):
        if done + k > p.nsteps:                 # wrap: restart the run from u0 after its last step
            u = O.run(p.u0, p.dx, p.h, p.P, p.W, p.V, 1)
            done = 1
        t0 = time.perf_counter()
        u = O.run(u, p.dx, p.h, p.P, p.W, p.V, k)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            secs.append(dt)
            upd.append(p.npts * k)
            samples.append("time steps %d..%d" % (done + 1, done + k))
        done += k
    value = float(sum(upd) / sum(secs))
    sample = "%s %s, %d samples of %d consecutive time steps each (%s), %d OpenMP threads" % (
        p.name, "x".join(map(str, p.shape)), args.steps, k, ", ".join(samples[:3]) + (", ..." if len(samples) > 3 else ""),
        cores)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": float(np.mean(secs)) * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": p.name, "shape": list(p.shape), "nsteps": p.nsteps, "W": list(p.W),
                       "h": p.h, "P": list(p.P), "parallelism": "host cores",
                       "step": "one sample of %d of the workload's %d time steps (%d updates)"
                               % (k, p.nsteps, p.npts * k)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_peaks(args):
    """The binary64 add rate of the device (hjlo_probe_fp64_add), the peak the
    brute-force pass is measured against; best of K probes after W warm-ups."""
    import torch
    from paper_1210_4090_gb300 import hjlo
    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    for _ in range(max(3, args.warmup)):
        hjlo.probe_fp64_add(1 << 14)
    rates = [hjlo.probe_fp64_add(1 << 16) for _ in range(args.steps)]
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    best = max(rates)
    line = {"metric": "binary64 adds/s (probe)", "value": best, "unit": "adds/s", "n_gpus": 1,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "peaks", "kernel": "8 independent add chains per thread, 8 CTAs x 256 "
                                                      "threads per SM, 2^16 adds per chain"},
            "all": rates, "per_clock_per_sm_at_2070MHz": best / (sms * 2070.0e6)}
    print(json.dumps(line), flush=True)


def run_sweep(args):
    """sweep512: all instances in one batch (grouped launches, one CUDA graph)
    against the plain per-instance loop (one plan and hjlo_run per instance)."""
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1210_4090_gb300 import hjlo

    # instances are independent: each rank takes its LPT share of the work
    # (N_i^2 points per instance); the H-bar rows are gathered at the end
    from paper_1210_4090_gb300 import dist as D
    allp = WL.sweep512()
    idx = D.shard_indices(len(allp), rank, world, [p.npts for p in allp])
    probs = [allp[i] for i in idx]
    nsteps = probs[0].nsteps
    dev = torch.device("cuda", local)
    sizes = [p.npts for p in probs]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    u0_all = torch.tensor(np.concatenate([p.u0.ravel() for p in probs]), device=dev)
    V_all = torch.tensor(np.concatenate([p.V.ravel() for p in probs]), device=dev)
    u_all = torch.empty_like(u0_all)
    us = [u_all[offs[i]:offs[i + 1]] for i in range(len(probs))]
    u0s = [u0_all[offs[i]:offs[i + 1]] for i in range(len(probs))]
    Vs = [V_all[offs[i]:offs[i + 1]] for i in range(len(probs))]
    algo = {"monge": hjlo.ALGO_MONGE, "brute": hjlo.ALGO_BRUTE, "auto": hjlo.ALGO_AUTO}[args.algo]
    batch = hjlo.Batch([(p.shape, p.dx, p.h, p.P, p.W) for p in probs], algo=algo)
    # every group's launch shapes from the library's autotuner (untimed)
    tune = None if args.no_autotune else batch.autotune(u0s, Vs, 8)
    # launch mode: one launch per group and axis, or one persistent launch per
    # time step; both timed on 64 steps (untimed for the bench), the faster kept
    modes = {}
    for mode in ("grouped", "persistent"):
        try:
            batch.set_persistent(mode == "persistent")
        except hjlo.HjloError:
            continue
        ts = []
        for _ in range(3):
            u_all.copy_(u0_all)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(torch.cuda.current_stream())
            batch.run(us, Vs, 64)
            e1.record(torch.cuda.current_stream())
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        modes[mode] = min(ts[1:])
    if args.batch_mode != "auto" and args.batch_mode in modes:
        best_mode = args.batch_mode
    else:
        best_mode = min(modes, key=modes.get)
    batch.set_persistent(best_mode == "persistent")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        u_all.copy_(u0_all)
        batch.run(us, Vs, nsteps)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    try:
        gpu_uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        gpu_uuid = None
    clocks = ClockSampler(gpu_uuid)
    clocks.start()
    time.sleep(0.3)
    evs = []
    for _ in range(args.steps):
        u_all.copy_(u0_all)
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.run(us, Vs, nsteps)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    total_ms = float(sum(a.elapsed_time(b) for a, b in evs))
    updates_local = int(sum(sizes)) * nsteps
    total_ms, updates = D.reduce_step(total_ms, updates_local, dev)
    ms_per_step = total_ms / args.steps
    value = updates * args.steps / (total_ms * 1e-3)
    hb = D.gather_rows(batch.hbar(u0s, us, nsteps), idx, len(allp), dev)   # every instance, in order
    cnt = batch.sync()
    groups = batch.groups()

    # plain per-instance loop on a subset with the same size mix
    loop = None
    if rank == 0 and args.loop_instances > 0:
        sub = probs[:args.loop_instances]
        plans = [hjlo.Plan(p.shape, p.dx, p.h, p.P, p.W, algo=algo) for p in sub]
        for pl, i in zip(plans, range(len(sub))):
            us[i].copy_(u0s[i])
            pl.run(us[i], Vs[i], 2 * 16)          # warm: capture each plan's graph
        torch.cuda.synchronize()
        for i in range(len(sub)):
            us[i].copy_(u0s[i])
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for pl, i in zip(plans, range(len(sub))):
            pl.run(us[i], Vs[i], nsteps)
        e1.record(stream)
        torch.cuda.synchronize()
        lms = e0.elapsed_time(e1)
        lupd = sum(p.npts for p in sub) * nsteps
        loop = {"value": lupd / (lms * 1e-3), "unit": UNIT, "instances": len(sub), "ms": lms}
        for pl in plans:
            pl.close()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import oracle as O
        cores = O.max_threads()
        t0 = time.perf_counter()
        n_done = 0
        k = 0
        while time.perf_counter() - t0 < args.cpu_seconds and k < len(probs):
            p = probs[k]
            O.run(p.u0, p.dx, p.h, p.P, p.W, p.V, 50)
            n_done += p.npts * 50
            k += 1
        dt = time.perf_counter() - t0
        cpu = {"value": n_done / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "sweep512 instances 0..%d, first 50 of %d steps each, %d OpenMP threads"
                         % (k - 1, nsteps, cores)}

    launches = nsteps if best_mode == "persistent" else nsteps * 2 * groups
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    alg_bytes_run = updates_local * 40.0            # 2D binary64: 2 passes x 16 B + h*V 8 B
    avg_launch_s = ms_per_step * 1e-3 / launches
    achieved = alg_bytes_run / launches / avg_launch_s / 1e9
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "sweep512", "instances": len(allp), "nsteps": nsteps,
                           "sizes": sorted(set(p.shape[0] for p in allp)), "h": 0.02, "W": "N/16",
                           "launch_groups": groups, "updates_per_step": updates, "autotune": tune,
                           "batch_mode": best_mode,
                           "mode_trial_ms_per_64_steps": modes,
                           "l2": "256 MiB buffer written between timed steps",
                           "parallelism": ("instances sharded over ranks by LPT on N^2, H-bar rows gathered"
                                           if world > 1 else "single GPU")},
                "per_instance_loop": loop,
                "batched_vs_loop": (value / world / loop["value"]) if loop else None,
                "hbar": {"mean": float(hb[:, 0].mean()), "min": float(hb[:, 0].min()),
                         "max": float(hb[:, 0].max()), "first": [float(x) for x in hb[:4, 0]]},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                             "frac": achieved / hbm, "traffic": None,
                             "kernel": ("hjlo::pass_kernel_persist" if best_mode == "persistent"
                                        else "hjlo::pass_kernel_batch"), "peak_kind": peak_kind,
                             "alg_bytes_per_launch": alg_bytes_run / launches,
                             "avg_launch_us": avg_launch_s * 1e6},
                "cpu_baseline": cpu, "clocks": clk,
                "gpu_launches": int(args.steps * (len(probs) + launches)), "counters": cnt}
        print(json.dumps(line), flush=True)
    batch.close()
    if world > 1:
        dist.destroy_process_group()


def plain_adjoint_loop(p, plan, u0, V, ub_n, dev):
    """The plain per-step reverse loop: argmins of every step kept (no
    checkpoints), each pass transposed with torch's index_add_ (atomic
    scatter) -- the straightforward way to differentiate the scheme."""
    import torch
    nd, npts, n = p.ndim, p.npts, p.nsteps
    am = torch.empty((n, nd, npts), dtype=torch.int32, device=dev)
    u = u0.clone()
    for k in range(n):
        plan.step(u, u, V, argmin=am[k].view(-1))
    ub = ub_n.clone().view(p.shape)
    Vbar = torch.zeros_like(u)
    Pbar = torch.zeros(nd, dtype=torch.float64, device=dev)
    lin = torch.arange(npts, device=dev).view(p.shape)
    for k in range(n - 1, -1, -1):
        Vbar -= p.h * ub
        for a in range(nd - 1, -1, -1):
            d = am[k, a].view(p.shape).to(torch.int64)
            shp = [1] * nd
            shp[a] = p.shape[a]
            i_a = torch.arange(p.shape[a], device=dev).view(shp)
            src = torch.remainder(i_a - d, p.shape[a])
            Pbar[a] += (ub * (-d.to(torch.float64) * p.dx[a])).sum()
            stride = int(np.prod(p.shape[a + 1:])) if a + 1 < nd else 1
            srcflat = lin + (src - i_a) * stride
            nub = torch.zeros(npts, dtype=torch.float64, device=dev)
            nub.index_add_(0, srcflat.reshape(-1), ub.reshape(-1))
            ub = nub.view(p.shape)
    return ub, Pbar, Vbar


def run_adjoint(args):
    """adjoint512: gradient of loss = mean (u^n - u^0)/(n h) w.r.t. P and the 64
    coefficients of V through hjlo_adjoint (checkpoint every 100 steps), against
    the plain per-step loop."""
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    from paper_1210_4090_gb300 import hjlo

    p = WL.adjoint512()
    dev = torch.device("cuda", local)
    n, S = p.nsteps, p.extra["checkpoint_every"]
    plan = hjlo.Plan(p.shape, p.dx, p.h, p.P, p.W)
    u0 = torch.tensor(p.u0, device=dev)
    V = torch.tensor(p.V, device=dev)
    B = torch.tensor(WL.adjoint_basis(p.shape[0]), device=dev)
    ub_n = torch.full(p.shape, 1.0 / (p.npts * n * p.h), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    def one():
        g0, gP, gV, _ = plan.adjoint(u0, V, n, ub_n, S)
        return gP, plan.project(gV, B)

    for _ in range(max(3, args.warmup)):
        one()
    torch.cuda.synchronize()
    try:
        gpu_uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        gpu_uuid = None
    clocks = ClockSampler(gpu_uuid)
    clocks.start()
    time.sleep(0.3)
    evs = []
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gP, gc = one()
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = float(sum(a.elapsed_time(b) for a, b in evs)) / args.steps
    updates = p.npts * n
    gP, gc = gP.cpu().numpy(), gc.cpu().numpy()

    # the plain per-step loop, timed once after a warm-up on a short run
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    ub0, lP, lV = plain_adjoint_loop(p, plan, u0, V, ub_n, dev)
    lc = plan.project(lV.contiguous(), B)
    e1.record(stream)
    torch.cuda.synchronize()
    loop_ms = e0.elapsed_time(e1)
    lP, lc = lP.cpu().numpy(), lc.cpu().numpy()
    agree = {"Pbar_max_rel": float(np.max(np.abs(lP - gP) / np.maximum(np.abs(gP), 1e-300))),
             "coef_max_rel": float(np.max(np.abs(lc - gc)) / np.max(np.abs(gc)))}
    if rank == 0:
        line = {"metric": METRIC + " (adjoint: forward + reverse)", "value": updates / (ms * 1e-3), "unit": UNIT,
                "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": "adjoint512", "shape": list(p.shape), "nsteps": n, "W": list(p.W),
                           "checkpoint_every": S, "P": list(p.P), "coefficients": 64},
                "plain_loop": {"ms": loop_ms, "value": updates / (loop_ms * 1e-3), "unit": UNIT,
                               "how": "all argmins kept, torch index_add_ per pass"},
                "adjoint_vs_loop": loop_ms / ms, "gradients": {"Pbar": [float(x) for x in gP],
                                                               "coef_first": [float(x) for x in gc[:4]]},
                "agreement_with_loop": agree, "clocks": clk}
        print(json.dumps(line), flush=True)
    plan.close()


def run_paper1d(args):
    """The paper's two 1D experiments (Sec. 5) on the GPU.  The line's value is
    the paper's largest run (Sec. 5.1 footnote): the pendulum on 2^18 points,
    T = 8, tau = sqrt(dx) (1635 steps; one line launched in row blocks), timed
    with CUDA events like the other workloads; the paper reports ~19 min for
    it with its approximate decomposition method (eta = dx) in MATLAB on a
    laptop core, context only.  Also: the throughput of the time-dependent-V
    run (hjlo_run_tv, one row of V per step) on 2 x 4096 points, and the
    convergence table at T = 8 (2K points, K = 4 .. 4096) against the scheme
    on 2 x 16384 points."""
    import torch
    from paper_1210_4090_gb300 import experiments as E, hjlo
    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    conv = {}
    for law in ("pendulum", "tdep"):
        r = E.convergence(law, [2 ** k for k in range(2, 13)], 2 ** 14)
        conv[law] = {"order": r["order"], "K_ref": r["K_ref"],
                     "errors": [[row["K"], row["error"]] for row in r["rows"]]}
    # the time-dependent law on 2 x 4096 points
    p = WL.tdep(4096)
    plan = hjlo.Plan(p.shape, p.dx, p.h, p.P, p.W)
    ms_tv, _ = _time_run(plan, torch.tensor(p.u0, device=dev), torch.tensor(p.V, device=dev), p.nsteps,
                         args.steps, args.warmup, tv=True)
    tdep = {"shape": list(p.shape), "nsteps": p.nsteps, "W": list(p.W), "ms": ms_tv,
            "value": p.npts * p.nsteps / (ms_tv * 1e-3), "row_blocks": plan.info()["row_blocks"]}
    plan.close()
    # the paper's timed run (launch shapes tuned first, outside the timed region)
    q = WL.pendulum(2 ** 17)
    plan = hjlo.Plan(q.shape, q.dx, q.h, q.P, q.W)
    qu0, qV = torch.tensor(q.u0, device=dev), torch.tensor(q.V, device=dev)
    tune = None if args.no_autotune else plan.autotune(qu0, qV, 16)
    info = plan.info()
    ms, u = _time_run(plan, qu0, qV, q.nsteps, args.steps, args.warmup)
    cnt = plan.sync()
    plan.close()
    updates = q.npts * q.nsteps
    line = {"metric": METRIC + " (1D pendulum, 2^18 points)", "value": updates / (ms * 1e-3), "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (deterministic: the paper's Sec. 5 laws)",
            "config": {"workload": "pendulum_2^18", "shape": list(q.shape), "nsteps": q.nsteps, "W": list(q.W),
                       "h": q.h, "P": list(q.P), "T": q.extra["T"], "row_blocks": info["row_blocks"],
                       "autotune": tune,
                       "paper_context": "~19 min (1140 s) in MATLAB on a 2.3 GHz laptop core with the "
                                        "approximate decomposition method (eta = dx): another method and "
                                        "machine, not a target"},
            "tdep": tdep, "convergence": conv, "counters": cnt}
    print(json.dumps(line), flush=True)


def _time_run(plan, u0, V, nsteps, steps, warmup, tv=False):
    """Mean device time (ms) of `steps` runs of nsteps from u0, after warm-up."""
    import torch
    u = torch.empty_like(u0)
    stream = torch.cuda.current_stream()
    go = plan.run_tv if tv else plan.run
    for _ in range(max(3, warmup)):
        u.copy_(u0)
        go(u, V, nsteps)
    torch.cuda.synchronize()
    evs = []
    for _ in range(steps):
        u.copy_(u0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        go(u, V, nsteps)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in evs])), u


def run_decomp(args):
    """The paper's own fast convolution (Sec. 4, HJLO_ALGO_DECOMP) against the
    monotone pass on the same runs: the paper-size run (the pendulum of Sec.
    5.1 on 2^18 points, T = 8) at eta = 0 (exact: row blocks, the cut cannot
    change the result), at the paper's eta = dx by the method as the paper
    defines it (one decomposition per whole period, its cut spread over
    CTAs) and at eta = dx with the approximate block-restart option; the
    pendulum on 2 x 4096 points at eta = 0, dx and 10 dx (whole lines, one
    CTA each); the 1024^2 grid law for its first 100 steps at eta = 0 and dx
    (whole lines).  Reports time, updates/s, components per line and pass,
    and the relative sup-norm deviation from the exact scheme (the monotone
    pass is bit-exact)."""
    import torch
    from paper_1210_4090_gb300 import hjlo
    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cases = []
    big = WL.pendulum(2 ** 17)
    pend = WL.pendulum(4096)
    g = WL.grid1024(nsteps=100)
    plan_cases = ((big, ((big.dx[0], False), (0.0, False), (big.dx[0], True))),
                  (pend, ((0.0, False), (pend.dx[0], False), (10 * pend.dx[0], False))),
                  (g, ((0.0, False), (g.dx[0], False))))
    for p, etas in plan_cases:
        u0 = torch.tensor(p.u0, device=dev)
        V = torch.tensor(p.V, device=dev)
        mono = hjlo.Plan(p.shape, p.dx, p.h, p.P, p.W, algo=hjlo.ALGO_MONGE)
        ms_m, ref = _time_run(mono, u0, V, p.nsteps, args.steps, args.warmup)
        mono.close()
        ref = ref.cpu().numpy()
        lines_per_step = sum(p.npts // s for s in p.shape)
        for eta, restart in etas:
            dec = hjlo.Plan(p.shape, p.dx, p.h, p.P, p.W, algo=hjlo.ALGO_DECOMP)
            dec.set_tolerance(eta, restart_blocks=restart)
            info = dec.info()
            ms_d, got = _time_run(dec, u0, V, p.nsteps, args.steps, args.warmup)
            cnt = dec.sync()
            dec.close()
            got = got.cpu().numpy()
            runs = max(3, args.warmup) + args.steps
            cases.append({"workload": p.name, "shape": list(p.shape), "nsteps": p.nsteps, "W": list(p.W),
                          "eta": eta,
                          "method": ("block restarts (approximate)" if restart and eta > 0
                                     else "Sec. 4, one decomposition per period"),
                          "row_blocks": info["row_blocks"], "split_chunks": info["split_chunks"],
                          "decomp_ms": ms_d, "monge_ms": ms_m,
                          "decomp_updates_per_s": p.npts * p.nsteps / (ms_d * 1e-3),
                          "monge_updates_per_s": p.npts * p.nsteps / (ms_m * 1e-3),
                          "components_per_line_pass": cnt["components"] / (runs * p.nsteps * lines_per_step),
                          "rel_error_vs_exact": float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))})
    # the line's value: the paper's timed run (the pendulum with 2^18 points
    # to T = 8, tau = sqrt(dx), eta = dx) by the method as the paper defines
    # it; the paper reports ~19 min for it, 262144 x 1634 updates / 1140 s
    # (MATLAB, one 2.3 GHz laptop core: another machine, so the ratio is
    # context)
    head = cases[0]
    paper = 262144 * 1634 / 1140.0
    line = {"metric": METRIC + " (decomposition method of Sec. 4)", "value": head["decomp_updates_per_s"],
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup),
            "ms_per_step": head["decomp_ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": head["decomp_updates_per_s"] / paper, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "pendulum_2^18", "shape": head["shape"], "nsteps": head["nsteps"],
                       "eta_over_dx": 1.0, "W": head["W"], "split_chunks": head["split_chunks"],
                       "baseline": "the paper's ~19 min (MATLAB, 2.3 GHz laptop core) for this run: "
                                   "%.3g updates/s" % paper,
                       "note": "comparison method; the headline path is the monotone pass"},
            "cases": cases}
    print(json.dumps(line), flush=True)


def run_integral(args):
    """The first discrete semigroup (eq. cost1, hjlo_integral_*) on the 128^2
    law: every candidate of the 9 x 9 window box with the exact path integral
    of a 12-mode Fourier potential.  Bound by binary64 arithmetic:
    4 flops per mode and candidate plus 3 per candidate."""
    import torch
    from paper_1210_4090_gb300 import hjlo
    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    p = WL.integral128()
    modes, coef = p.extra["modes"], p.extra["coef"]
    plan = hjlo.IntegralPlan(p.shape, p.dx, p.h, p.P, p.W, modes, coef)
    dev = torch.device("cuda", local)
    u0 = torch.tensor(p.u0, device=dev)
    u = torch.empty_like(u0)
    stream = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        u.copy_(u0)
        plan.run(u, p.nsteps)
    torch.cuda.synchronize()
    evs = []
    for _ in range(args.steps):
        u.copy_(u0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.run(u, p.nsteps)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    plan.close()
    updates = p.npts * p.nsteps
    box = (2 * p.W[0] + 1) * (2 * p.W[1] + 1)
    # flops per candidate: two products and two adds per mode (fused in pairs
    # on the GPU) and three for the candidate; peak: 2 binary64 FMA per clock
    # per SM = 4 flops (the nominal 1.25 TFLOP/s)
    ops = float(updates) * box * (4 * len(coef) + 3)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak = 4.0 * sms * 2070.0e6 / 1e9
    ach = ops / (ms * 1e-3) / 1e9
    cpu = None
    if not args.no_cpu_baseline:
        from oracle import oracle as O
        t0 = time.perf_counter()
        O.integral_run(p.u0, p.dx, p.h, p.P, p.W, modes, coef, 2)
        dt = time.perf_counter() - t0
        cpu = {"value": p.npts * 2 / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "integral128, the first 2 time steps (numpy, %.1f s)" % dt}
    line = {"metric": METRIC + " (first discrete semigroup, eq. cost1)", "value": updates / (ms * 1e-3),
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "integral128", "shape": list(p.shape), "nsteps": p.nsteps, "W": list(p.W),
                       "modes": int(len(coef)), "box": box},
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "G fp64 flop/s", "frac": ach / peak,
                         "peak_kind": "derived (2 FMA = 4 flops/clk/SM x %d SMs x 2070 MHz)" % sms,
                         "fp64_flops_per_update": box * (4 * len(coef) + 3)},
            "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1210_4090_gb300 import hjlo

    p = workload(args.workload)
    algo = {"monge": hjlo.ALGO_MONGE, "brute": hjlo.ALGO_BRUTE, "auto": hjlo.ALGO_AUTO}[args.algo]
    code = hjlo.F64 if args.dtype == "f64" else hjlo.F32_STORAGE
    tdt = torch.float64 if args.dtype == "f64" else torch.float32
    plan = hjlo.Plan(p.shape, p.dx, p.h, p.P, p.W, dtype=code, algo=algo)
    info = plan.info()
    dev = torch.device("cuda", local)
    u0 = torch.tensor(p.u0, dtype=tdt, device=dev)
    Vt = torch.tensor(p.V, dtype=torch.float64, device=dev)
    u = torch.empty_like(u0)
    # launch shapes chosen by the library's autotuner on the first time steps
    # (outside the timed region; results do not depend on the shape)
    tune = plan.autotune(u0, Vt, 16) if (info["algo"] == "monge" and not args.no_autotune) else None
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device=dev)   # 256 MiB > L2
    stream = torch.cuda.current_stream()

    def one():
        plan.run(u, Vt, p.nsteps)

    for _ in range(max(3, args.warmup)):
        u.copy_(u0)
        one()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    try:
        gpu_uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        gpu_uuid = None
    clocks = ClockSampler(gpu_uuid)
    clocks.start()
    time.sleep(0.3)
    evs = []
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    for _ in range(args.steps):
        u.copy_(u0)
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        one()
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    from paper_1210_4090_gb300 import dist as D
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms, _ = D.reduce_step(float(sum(step_ms)), 0.0, dev)
    ms_per_step = total_ms / args.steps
    updates = p.npts * p.nsteps
    value = world * updates * args.steps / (total_ms * 1e-3)
    cnt = plan.sync()

    # roofline of the dominant kernel: the axis pass (ndim launches per time
    # step; the h*V kernel is one launch per run and is left in the average)
    launches_per_step = p.ndim * p.nsteps
    avg_launch_s = ms_per_step * 1e-3 / launches_per_step
    esize = 8 if args.dtype == "f64" else 4
    alg_bytes_step = p.npts * (p.ndim * 2 * esize + 8)          # per time step
    alg_bytes_launch = alg_bytes_step / p.ndim
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    achieved = alg_bytes_launch / avg_launch_s / 1e9
    traffic = profile_traffic(args.workload, info["algo"], args.dtype)
    if info["algo"] == "brute":
        # brute force is bound by binary64 adds: one per window candidate per
        # output and pass (+ the potential term); peak: the device's add rate
        # measured by the probe kernel (best of 3), next to the unit count's
        # 2 binary64 adds per clock per SM x SMs x max SM clock
        import torch
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        clk_mhz = (clk or {}).get("sm_max_mhz") or 2070.0
        derived = 2.0 * sms * clk_mhz * 1e6 / 1e9
        peak_gops = max(hjlo.probe_fp64_add(1 << 16) for _ in range(3)) / 1e9
        weffs = [info["dhi"][a] - info["dlo"][a] + 1 for a in range(p.ndim)]
        adds_launch = p.npts * (sum(weffs) + 1) / p.ndim
        ach = adds_launch / avg_launch_s / 1e9
        roof = {"bound": "alu", "achieved": ach, "peak": peak_gops, "unit": "G fp64 add/s",
                "frac": ach / peak_gops, "traffic": None, "kernel": "hjlo::pass_kernel (brute)",
                "peak_kind": "measured (hjlo_probe_fp64_add); derived 2 adds/clk/SM x %d SMs x %.0f MHz = %.0f"
                             % (sms, clk_mhz, derived),
                "fp64_adds_per_launch": adds_launch, "avg_launch_us": avg_launch_s * 1e6}
    else:
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic, "kernel": "hjlo::pass_kernel (%s)" % info["algo"],
                "peak_kind": peak_kind, "alg_bytes_per_launch": alg_bytes_launch,
                "avg_launch_us": avg_launch_s * 1e6,
                "fp64_ops_per_launch": p.npts * 1.0 + (p.npts / p.ndim)}

    e2e = None
    if not args.no_e2e:
        uh = torch.empty(p.shape, dtype=tdt).pin_memory().numpy()
        Vh = torch.empty(p.shape, dtype=torch.float64).pin_memory().numpy()
        Vh[...] = p.V
        ts = []
        for k in range(args.steps + 1):
            uh[...] = p.u0
            t0 = time.perf_counter()
            plan.run_host(uh, Vh, p.nsteps)
            dt = time.perf_counter() - t0
            if k:
                ts.append(dt)
        e2e = {"value": world * updates / float(np.mean(ts)), "unit": UNIT,
               "h2d_bytes_per_step": int(p.npts * esize + p.npts * 8),
               "d2h_bytes_per_step": int(p.npts * esize)}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, cores, sample = cpu_oracle_rate(p, args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
                "config": {"workload": p.name, "shape": list(p.shape), "nsteps": p.nsteps, "W": list(p.W),
                           "h": p.h, "P": list(p.P), "algo": info["algo"],
                           "updates_per_step": updates, "autotune": tune,
                           "l2": "256 MiB buffer written between timed steps; the grid is L2-resident "
                                 "within a step when it fits",
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "e2e": e2e, "roofline": roof, "cpu_baseline": cpu, "clocks": clk,
                "gpu_launches": int(args.steps * (1 + launches_per_step)),
                "counters": cnt}
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "sweep512":
        run_sweep(args)
    elif args.workload == "adjoint512":
        run_adjoint(args)
    elif args.workload == "paper1d":
        run_paper1d(args)
    elif args.workload == "decomp":
        run_decomp(args)
    elif args.workload == "integral128":
        run_integral(args)
    elif args.workload == "peaks":
        run_peaks(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
