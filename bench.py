"""Benchmark of the Lagrange-phase partial-assembly hot path on one B300 per rank.

Workload (default): 3D Taylor-Green vortex on [0,1]^3, 24^3 hexes, H1 Q2 / L2 Q1,
4^3 Gauss-Legendre points per element, ideal gas gamma = 5/3, FP64, RK2-average
with CFL 0.5 towards t = 0.1. One benchmark step = one RK2-average step (two
stages of: quadrature data, F.1, mass CG, F^T v with the energy solve, and the
state updates), i.e. one pass of the whole hot path.

Metric: MDOF/s = (vector H1 DOFs) x (steps) / (time), 1e6/s, higher is better.
The L2 cache (126 MB) is flushed before every timed step by writing a 512 MB
buffer, outside the timed events. Multi-GPU (torchrun): every rank advances its
own independent replica (the path needs no exchange for independent problems),
value = all ranks' DOF-steps / max-over-ranks time, scaling "weak".

--impl reference times the FP64 CPU oracle (the method's reference
implementation, full assembly) on this machine's host cores on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import ctypes
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

WORKLOADS = {
    # name: (dim, n, order, q1, jitter, t_end, cfl)
    "tg3d_24_q2": dict(dim=3, n=24, order=2, q1=4, jitter=0.0, t_end=0.1, cfl=0.5,
                       desc="3D Taylor-Green, 24^3 hexes, Q2/Q1, 4^3 Gauss points, CFL 0.5 to t=0.1"),
    "tg3d_32_q4_jit": dict(dim=3, n=32, order=4, q1=6, jitter=0.15, t_end=0.1, cfl=0.5,
                           desc="3D Taylor-Green, 32^3 hexes jittered +-0.15h (seed 3), Q4/Q3, 6^3 Gauss points"),
    "tg2d_8_q2": dict(dim=2, n=8, order=2, q1=4, jitter=0.0, t_end=0.02, cfl=0.5,
                      desc="2D Taylor-Green, 8^2 quads, Q2/Q1, 4^2 Gauss points"),
}
# DRAM bytes (read + write) of one launch of the roofline kernel, from one ncu
# capture of the current kernel (profiles/k_cg_tg3d24_q2_fp64.md,
# profiles/k_cg_ir_tg3d24_q2_fp32ir.md, profiles/k_cg_ir_tg3d32_q4_fp32ir.md); None
# where no capture of the current kernel exists.
TRAFFIC = {("tg3d_24_q2", "fp64"): 23394816, ("tg3d_24_q2", "fp32_ir"): 29678592,
           ("tg3d_32_q4_jit", "fp32_ir"): 10096740352}
METRIC = "MDOF/s of PA force+mass path (RK2-average step, H1 vector DOFs per second)"
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def max_over_ranks(t_local: float, world: int, device: str) -> float:
    """The slowest rank's timed duration (all ranks receive it)."""
    if world <= 1:
        return t_local
    import torch
    import torch.distributed as dist
    tt = torch.tensor([t_local], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_rate(nv_per_rank: int, steps: int, world: int, t_max: float) -> float:
    """Whole-job MDOF/s: every rank advanced nv_per_rank DOFs for `steps` steps."""
    return nv_per_rank * steps * world / t_max / 1e6


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# algorithmic work model (sum factorization, FP64)
# ---------------------------------------------------------------------------
def work_model(dim, p, q1, ne, nh1):
    D, Q, L = p + 1, q1, p
    nv = dim * nh1
    if dim == 3:
        interp = Q * D ** 3 + Q * Q * D * D + Q ** 3 * D
        grad = 2 * Q * D ** 3 + 3 * Q * Q * D * D + 3 * Q ** 3 * D
        l2i = Q * L ** 3 + Q * Q * L * L + Q ** 3 * L
    else:
        interp = Q * D * D + Q * Q * D
        grad = 2 * Q * D * D + 2 * Q * Q * D
        l2i = Q * L * L + Q * Q * L
    nq = Q ** dim
    mass_flops = 2 * ne * (2 * dim * interp) + ne * dim * nq          # FMA = 2 flops, D-scaling 1
    cg_iter_flops = mass_flops + 10 * nv
    cg_iter_bytes = 8 * (ne * nq + 2 * nv) + 56 * nv
    return dict(mass_flops=mass_flops, cg_iter_flops=cg_iter_flops, cg_iter_bytes=cg_iter_bytes,
                force_flops=2 * ne * dim * grad, force_bytes=8 * (dim * dim * ne * nq + nv),
                force_t_flops=2 * ne * (dim * grad + l2i) + 2 * ne * dim * dim * nq,
                force_t_bytes=8 * (dim * dim * ne * nq + nv + ne * L ** dim))


class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={CLOCK_QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1])]
        smax = max(num(r[2]) or 0 for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows), "power_w_max": max((num(r[3]) or 0) for r in rows)}


def probe_peaks():
    path = os.path.join(ROOT, "paper_2112_07075_b300", "probe", "libprobe_alu.so")
    lib = ctypes.CDLL(path)
    f64, f32 = ctypes.c_double(), ctypes.c_double()
    lib.probe_fma_tflops(ctypes.byref(f64), ctypes.byref(f32))
    return f64.value, f32.value


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_remap_only(args):
    """--remap-only: the remap report alone (one JSON line), for profiling the remap."""
    import torch
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    rep = remap_report(flush)
    if not args.no_cpu_baseline:
        rep["cpu_baseline"] = remap_cpu_baseline()
    print(json.dumps({"remap": rep}), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2112_07075_b300 import inputs
    from paper_2112_07075_b300.lh import Context

    wl = WORKLOADS[args.workload]
    dim, n, p, q1 = wl["dim"], wl["n"], wl["order"], wl["q1"]
    V = inputs.box_vertices(dim, n, jitter=wl["jitter"], seed=3 + rank)
    ctx = Context(dim, n, V, p, q1, cfl=wl["cfl"], precision=args.precision)
    sz = ctx.sizes
    x, v, e = ctx.init_state("taylor_green")
    info = ctx.new_step_info(0.0, wl["t_end"])
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    peak64, peak32 = probe_peaks()
    clk = ClockSampler(local).__enter__()
    for _ in range(args.warmup):
        ctx.rk2avg_step(x, v, e, 0.0, info)
    torch.cuda.synchronize()
    if ctx.sync_status() != 0:
        raise RuntimeError("device status after warm-up: " + ctx.lib.lh_last_error(ctx.h).decode())

    K = args.steps
    trajectory = K == 0   # time the whole configured run from t = 0 to t_end
    if trajectory:
        x, v, e = ctx.init_state("taylor_green")
        info = ctx.new_step_info(0.0, wl["t_end"])
    iters_before = ctx.read_step_info(info).cg_iters_total
    snap = (x.clone(), v.clone(), e.clone(), info.clone())   # e2e replays the same steps
    ctx.timing_enable(True)          # events around each solver launch, on the step's stream
    ev0, ev1 = [], []
    solver_ms, solver_launches = 0.0, 0
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    k = 0
    chunk = 16 if trajectory else min(16, K)
    while True:
        # chunks of up to 16 steps: the solver timing probe keeps 64 launches between
        # reads; near t_end the whole-run mode goes step by step to stop exactly there
        for _ in range(chunk):
            ev0.append(torch.cuda.Event(enable_timing=True))
            ev1.append(torch.cuda.Event(enable_timing=True))
            flush.fill_(float(k))
            ev0[-1].record(stream)
            ctx.rk2avg_step(x, v, e, 0.0, info)
            ev1[-1].record(stream)
            k += 1
        ms, ns = ctx.timing_read()
        solver_ms += ms
        solver_launches += ns
        if trajectory:
            si_ = ctx.read_step_info(info)
            left = wl["t_end"] - si_.t
            if left <= 1e-12 * wl["t_end"] or k >= 100000:
                break
            chunk = 16 if si_.dt > 0 and left > 20.0 * si_.dt else 1
        elif k >= K:
            break
        else:
            chunk = min(16, K - k)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    ctx.timing_enable(False)
    K = k
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    t_local = sum(step_ms) / 1e3
    si = ctx.read_step_info(info)
    timed_iters = int(si.cg_iters_total - iters_before)
    status = ctx.sync_status()
    t_max = max_over_ranks(t_local, world, "cuda")
    value = job_rate(sz.nv, K, world, t_max)

    # ---- per-kernel breakdown at the current state (same stream, CUDA events)
    W = work_model(dim, p, q1, sz.ne, sz.n_h1)
    reps = 5
    rhs, acc, out = ctx.h1_vector(), ctx.h1_vector(), ctx.l2_vector()
    cginfo = ctx.new_cg_info()

    def timed(fn):
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    t_q = timed(lambda: ctx.update_qdata(x, v, e, None))
    t_f = timed(lambda: ctx.force_mult(None, rhs))
    rhs.neg_()
    iters = []

    def cg():
        acc.zero_()
        ctx.mass_cg(rhs, acc, 1e-12, 1000, cginfo)
    t_cg = timed(cg)
    cgi = ctx.read_cg_info(cginfo)
    t_ft = timed(lambda: ctx.force_mult_t(v, out))
    cg_flops = cgi.iters * W["cg_iter_flops"] + W["mass_flops"]
    # rates in the mini-app's convention (H1 vector DOFs or qpoints per second, 1e6/s):
    # force = NV per (F.1, F^T v) pair, mass = NV x CG iterations, qdata = NQ per update
    kernels = {
        "mass_cg": {"ms": t_cg, "iters": cgi.iters, "gflop": cg_flops / 1e9,
                    "tflops": cg_flops / (t_cg * 1e-3) / 1e12,
                    "mass_rate_mdofs": sz.nv * cgi.iters / (t_cg * 1e-3) / 1e6},
        "qdata": {"ms": t_q, "rate_mqs": sz.nq / (t_q * 1e-3) / 1e6},
        "force_mult": {"ms": t_f, "tflops": W["force_flops"] / (t_f * 1e-3) / 1e12},
        "force_mult_t": {"ms": t_ft, "tflops": W["force_t_flops"] / (t_ft * 1e-3) / 1e12},
        "force_pair": {"rate_mdofs": sz.nv / ((t_f + t_ft) * 1e-3) / 1e6},
    }
    # the whole configured run beside the timed window (the headline workload only: the
    # other workloads' runs to t_end take minutes)
    whole = whole_run(ctx, wl, flush, stream) if (not trajectory and world == 1
                                                  and args.workload == "tg3d_24_q2") else None

    # Roofline of the dominant kernel, measured live over the timed steps: the
    # library's event pairs around each solver launch (same stream) give its
    # time; algorithmic FLOPs = iterations x CG-iteration FLOPs + one matvec per solve.
    # With fp32_ir the iterations are the FP32 inner ones and the peak is the FP32 one.
    timed_flops = timed_iters * W["cg_iter_flops"] + solver_launches * W["mass_flops"]
    achieved = timed_flops / (solver_ms * 1e-3) / 1e12 if solver_ms > 0 else 0.0
    peak = peak64 if args.precision == "fp64" else peak32
    roofline = {"bound": "alu", "kernel": "k_cg (persistent Jacobi-PCG on the PA mass operator)"
                if args.precision == "fp64" else "k_cg_ir (FP32 PCG under FP64 refinement)",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if peak > 0 else None,
                "traffic": TRAFFIC.get((args.workload, args.precision)),
                "peak_source": ("measured FP64 FMA-chain probe (paper_2112_07075_b300/probe/alu_peak.cu), "
                                "same run; derived 148 SM x 2 DFMA/clk x 2 flop x clock")
                if args.precision == "fp64" else
                "measured FP32 FMA-chain probe (paper_2112_07075_b300/probe/alu_peak.cu), same run",
                "launches": solver_launches, "launch_ms_avg": solver_ms / max(1, solver_launches),
                "flops_per_launch": timed_flops / max(1, solver_launches),
                "iters_per_launch": timed_iters / max(1, solver_launches),
                "share_of_step": solver_ms / max(1e-9, sum(step_ms)),
                "fp32_peak_tflops": peak32}

    # ---- end-to-end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        # the host copies start from the state of the first timed step, so the e2e
        # steps are the same steps (same CG iteration counts) as the timed ones
        x.copy_(snap[0])
        v.copy_(snap[1])
        e.copy_(snap[2])
        info.copy_(snap[3])
        xh = torch.empty_like(x, device="cpu").pin_memory()
        vh = torch.empty_like(v, device="cpu").pin_memory()
        eh = torch.empty_like(e, device="cpu").pin_memory()
        xh.copy_(x)
        vh.copy_(v)
        eh.copy_(e)
        Ke = max(3, K)   # the same number of steps as the timed region
        bytes_io = (xh.numel() + vh.numel() + eh.numel()) * 8
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ts = []
        for k in range(Ke):
            flush.fill_(2.0)
            a.record(stream)
            x.copy_(xh, non_blocking=True)
            v.copy_(vh, non_blocking=True)
            e.copy_(eh, non_blocking=True)
            ctx.rk2avg_step(x, v, e, 0.0, info)
            xh.copy_(x, non_blocking=True)
            vh.copy_(v, non_blocking=True)
            eh.copy_(e, non_blocking=True)
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        e2e = {"value": sz.nv * world / (statistics.mean(ts) * 1e-3) / 1e6, "unit": "MDOF/s",
               "h2d_bytes_per_step": bytes_io, "d2h_bytes_per_step": bytes_io, "steps": Ke}

    forms = None
    batching = None
    learned = None
    remap = None
    stiffness = None
    tmop = None
    shock = None
    if not args.no_forms and world == 1:
        which = ("precision", "batching", "learned", "remap", "stiffness", "tmop", "shock") \
            if args.forms == "all" \
            else (args.forms,)
        forms = forms_report(flush) if "precision" in which else None
        batching = batching_report(flush) if "batching" in which else None
        learned = learned_report(flush) if "learned" in which else None
        remap = remap_report(flush) if "remap" in which else None
        stiffness = stiffness_report(flush) if "stiffness" in which else None
        tmop = tmop_report(flush) if "tmop" in which else None
        shock = shock_report(flush) if "shock" in which else None
    clk.__exit__()
    clocks = clk.summary()
    clocks["window"] = "sampled every 200 ms from warm-up to the end of the GPU measurements"
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MDOF/s", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "fp32_ir": "f64+f32(inner CG)", "bf16tc_ir": "f64+bf16(tensor-core inner CG)"}[args.precision],
            "data": "synthetic",
            "config": {"workload": wl["desc"], "precision": args.precision,
                       "window": (f"whole run from t = 0 to t = {wl['t_end']} ({K} steps)" if trajectory
                                  else f"{K} steps after {args.warmup} warm-up steps from t = 0"), "dim": dim, "n": n, "order": p, "q1": q1, "cfl": wl["cfl"],
                       "t_end": wl["t_end"], "nv_per_gpu": sz.nv, "ne": sz.ne, "nq": sz.nq,
                       "l2_flush": "512 MB buffer written before every timed step",
                       "parallelism": f"replicas x{world} (independent problems, no exchange)"},
            "roofline": roofline,
            "cpu_baseline": None,
            "e2e": e2e,
            "gpu_launches": 13 * K,
            "clocks": clocks,
            "kernels": kernels,
            "whole_run": whole,
            "forms": {"precision": forms, "batching": batching, "learned": learned},
            "remap": remap,
            "stiffness": stiffness,
            "tmop": tmop,
            "shock": shock,
            "cg_iters_last_step": list(si.cg_iters), "sim_time": si.t, "dt_last": si.dt,
            "device_status": status, "wall_s_timed": wall,
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(wl, V)
            if REDUCED_STATES:
                line["forms_vs_oracle"] = forms_vs_oracle()
            if remap is not None:
                remap["cpu_baseline"] = remap_cpu_baseline()
            if stiffness is not None:
                stiffness["cpu_baseline"] = stiffness_cpu_baseline()
            if tmop is not None:
                tmop["cpu_baseline"] = tmop_cpu_baseline()
            if shock is not None:
                shock["cpu_baseline"] = shock_cpu_baseline()
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def measure_form(wl_name, precision, steps, warmup, flush, seed=3):
    """Per-step device time of one form on a workload, and the final state."""
    import torch
    from paper_2112_07075_b300 import inputs
    from paper_2112_07075_b300.lh import Context
    wl = WORKLOADS[wl_name]
    V = inputs.box_vertices(wl["dim"], wl["n"], jitter=wl["jitter"], seed=seed)
    ctx = Context(wl["dim"], wl["n"], V, wl["order"], wl["q1"], cfl=wl["cfl"], precision=precision)
    x, v, e = ctx.init_state("taylor_green")
    info = ctx.new_step_info(0.0, wl["t_end"])
    stream = torch.cuda.current_stream()
    ts, iters = [], []
    for k in range(warmup + steps):
        flush.fill_(3.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.rk2avg_step(x, v, e, 0.0, info)
        b.record(stream)
        b.synchronize()
        if k >= warmup:
            ts.append(a.elapsed_time(b))
            iters.append(list(ctx.read_step_info(info).cg_iters))
    st = ctx.sync_status()
    out = dict(ms_per_step=statistics.mean(ts), mdofs=ctx.sizes.nv / (statistics.mean(ts) * 1e-3) / 1e6,
               cg_iters=iters[-1], status=st, nv=ctx.sizes.nv)
    # mass-solve cost model at the final state: solves from a zero guess at several tolerances
    rhs, sol = ctx.h1_vector(), ctx.h1_vector()
    ctx.force_mult(None, rhs)
    rhs.neg_()
    cginfo = ctx.new_cg_info()
    solves = []
    for tol in (1e-4, 1e-8, 1e-12):
        best = None
        for _ in range(3):
            sol.zero_()
            flush.fill_(4.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.mass_cg(rhs, sol, tol, 5000, cginfo)
            b.record(stream)
            b.synchronize()
            t = a.elapsed_time(b)
            best = t if best is None else min(best, t)
        ci = ctx.read_cg_info(cginfo)
        solves.append(dict(tol=tol, ms=best, iters=ci.iters, refinements=ci.refinements, rel_res=ci.rel_res))
    out["solves_from_zero"] = solves
    state = tuple(t.cpu().numpy() for t in (x, v, e))
    ctx.close()
    return out, state


def whole_run(ctx, wl, flush, stream):
    """The configured run from t = 0 to t_end (CFL steps), every step timed with CUDA
    events after an L2 flush: the whole-run rate beside the timed window's."""
    import torch
    x, v, e = ctx.init_state("taylor_green")
    info = ctx.new_step_info(0.0, wl["t_end"])
    ev = []
    k = 0
    it0 = ctx.read_step_info(info).cg_iters_total
    while True:
        for _ in range(16):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.fill_(float(k))
            a.record(stream)
            ctx.rk2avg_step(x, v, e, 0.0, info)
            b.record(stream)
            ev.append((a, b))
            k += 1
        si = ctx.read_step_info(info)
        if wl["t_end"] - si.t <= 1e-12 * wl["t_end"] or k > 100000:
            break
        if si.dt > 0 and wl["t_end"] - si.t <= 20.0 * si.dt:
            while wl["t_end"] - ctx.read_step_info(info).t > 1e-12 * wl["t_end"]:
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                flush.fill_(float(k))
                a.record(stream)
                ctx.rk2avg_step(x, v, e, 0.0, info)
                b.record(stream)
                ev.append((a, b))
                k += 1
            break
    torch.cuda.synchronize()
    si = ctx.read_step_info(info)
    ms = [a.elapsed_time(b) for a, b in ev]
    tot = sum(ms) / 1e3
    return {"value": ctx.sizes.nv * k / tot / 1e6, "unit": "MDOF/s", "steps": k,
            "ms_per_step": 1e3 * tot / k, "t_final": si.t, "status": ctx.sync_status(),
            "cg_iters_per_solve": (si.cg_iters_total - it0) / (2.0 * k),
            "window": f"whole run from t = 0 to t = {wl['t_end']}, every step timed (L2 flushed)"}


# Reduced cases of the precision and learned workloads, small enough for the oracle:
# the same element families, jitter and seeds as the full-size configurations, on 6^3
# meshes, with CFL 0.5 steps from t = 0 (10 steps for the precision workload, 20 for
# the learned one). The GPU legs store their end states here; the CPU-baseline leg
# runs the oracle on the same cases and reports each form's error against it.
REDUCED = {
    "tg3d_6_q4_jit": dict(dim=3, n=6, order=4, q1=6, jitter=0.15, seed=3, steps=10,
                          desc="3D Taylor-Green 6^3 Q4/Q3 q6, jitter 0.15h (seed 3), 10 CFL steps"),
    "tg3d_6_q3_jit": dict(dim=3, n=6, order=3, q1=6, jitter=0.1, seed=9, steps=20,
                          desc="3D Taylor-Green 6^3 Q3/Q2 q6, jitter 0.1h (held-out seed 9), 20 CFL steps"),
}
REDUCED_STATES = {}   # (case, mode) -> (x, v, e) end state of the GPU run


def reduced_run(case, precision, net=None):
    """End state of a reduced case after its CFL steps, one form (net: learned guess)."""
    from paper_2112_07075_b300 import inputs
    from paper_2112_07075_b300.lh import Context, learn_attach
    rc = REDUCED[case]
    V = inputs.box_vertices(rc["dim"], rc["n"], jitter=rc["jitter"], seed=rc["seed"])
    c = Context(rc["dim"], rc["n"], V, rc["order"], rc["q1"], precision=precision)
    if net is not None:
        learn_attach(c, net, 2)
    x, v, e = c.init_state("taylor_green")
    info = c.new_step_info(0.0, 1.0)
    for _ in range(rc["steps"]):
        c.rk2avg_step(x, v, e, 0.0, info)
    si = c.read_step_info(info)
    out = tuple(t.cpu().numpy() for t in (x, v, e))
    st = c.sync_status()
    c.close()
    if st != 0 or si.steps != rc["steps"]:
        raise RuntimeError(f"reduced run {case}/{precision}: status {st}, {si.steps} steps")
    mode = precision + ("+learned" if net is not None else "")
    REDUCED_STATES[(case, mode)] = out
    return out


def forms_vs_oracle():
    """CPU-baseline leg: the oracle on every reduced case that has GPU end states, and the
    relative per-field error (x, v, e) of each form's end state against it."""
    from paper_2112_07075_b300 import inputs
    from oracle.hydro import Hydro, Params
    rep = {}
    for case in sorted({k[0] for k in REDUCED_STATES}):
        rc = REDUCED[case]
        V = inputs.box_vertices(rc["dim"], rc["n"], jitter=rc["jitter"], seed=rc["seed"])
        hy = Hydro(Params(dim=rc["dim"], n=rc["n"], order=rc["order"], q1=rc["q1"], vertices=V))
        x, v, e = hy.initial_state("taylor_green")
        t0 = time.perf_counter()
        t = 0.0
        for _ in range(rc["steps"]):
            x, v, e, oi = hy.rk2avg_step(x, v, e, dt=None, t=t, t_end=1.0)
            t += oi.dt
        el = time.perf_counter() - t0
        ref = (x, v, e.reshape(-1))
        errs = {}
        for (c2, mode), st in REDUCED_STATES.items():
            if c2 != case:
                continue
            errs[mode] = {f: float(np.linalg.norm(a.reshape(-1) - b) / np.linalg.norm(b))
                          for f, a, b in zip(("x", "v", "e"), st, (r.reshape(-1) for r in ref))}
            errs[mode]["max"] = max(errs[mode].values())
        rep[case] = {"workload": rc["desc"], "oracle_s": el, "cores": _cores(),
                     "rel_field_err_vs_oracle": errs, "bar": 1e-10}
    return rep


def forms_report(flush, steps=3, warmup=1):
    rep = {}
    for wl_name in ("tg3d_24_q2", "tg3d_32_q4_jit"):
        f64, s64 = measure_form(wl_name, "fp64", steps, warmup, flush)
        f32, s32 = measure_form(wl_name, "fp32_ir", steps, warmup, flush)
        err = max(float(np.linalg.norm(a - b) / np.linalg.norm(b)) for a, b in zip(s32, s64))
        rep[wl_name] = {"fp64": f64, "fp32_ir": f32, "speedup": f64["ms_per_step"] / f32["ms_per_step"],
                        "max_rel_field_diff_vs_fp64_gpu": err, "steps": warmup + steps,
                        "note": "same initial state, CFL steps from t=0; per-step CUDA-event time, L2 flushed"}
        if WORKLOADS[wl_name]["order"] >= 3:   # tensor-core inner operator (order >= 3)
            ftc, stc = measure_form(wl_name, "bf16tc_ir", steps, warmup, flush)
            rep[wl_name]["bf16tc_ir"] = ftc
            rep[wl_name]["bf16tc_ir"]["speedup_vs_fp64"] = f64["ms_per_step"] / ftc["ms_per_step"]
            rep[wl_name]["bf16tc_ir"]["max_rel_field_diff_vs_fp64_gpu"] = max(
                float(np.linalg.norm(a - b) / np.linalg.norm(b)) for a, b in zip(stc, s64))
    for prec in ("fp64", "fp32_ir", "bf16tc_ir"):
        reduced_run("tg3d_6_q4_jit", prec)
    rep["vs_oracle"] = "reduced case tg3d_6_q4_jit, filled in by the CPU-baseline leg (cpu_checks)"
    return rep


def batching_report(flush, steps=5, warmup=2, seed=4):
    """256 independent 2D problems (seeded orders 1..4, n in [8, 64], half Taylor-Green,
    half Gresho), fixed dt_i = 0.5 dt_est_i(S0): batched graph step vs one-by-one steps."""
    import torch
    from paper_2112_07075_b300 import inputs
    from paper_2112_07075_b300.lh import Batch, Context
    probs = inputs.batch_problems(seed)
    ctxs, states, dts, nv = [], [], [], 0
    t0 = time.perf_counter()
    est = torch.zeros(len(probs), dtype=torch.float64, device="cuda")
    for i, pr in enumerate(probs):
        V = inputs.box_vertices(2, pr["n"], pr["lo"], pr["hi"])
        src = "tg2d" if pr["kind"] == "taylor_green" else "none"
        ctx = Context(2, pr["n"], V, pr["order"], 2 * pr["order"], source=src)
        x, v, e = ctx.init_state(pr["kind"])
        ctx.update_qdata(x, v, e, est[i:i + 1])
        ctxs.append(ctx)
        states.append((x, v, e))
        nv += ctx.sizes.nv
    dts = (0.5 * est).cpu().tolist()
    setup_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    # one by one (each problem's own lh_rk2avg_step), on copies of the initial states
    copies = [tuple(t.clone() for t in st) for st in states]
    infos = [c.new_step_info() for c in ctxs]
    for _ in range(warmup):
        for c, (x, v, e), d, inf in zip(ctxs, copies, dts, infos):
            c.rk2avg_step(x, v, e, d, inf)
    flush.fill_(5.0)
    a, b = ev(), ev()
    a.record(stream)
    for _ in range(steps):
        for c, (x, v, e), d, inf in zip(ctxs, copies, dts, infos):
            c.rk2avg_step(x, v, e, d, inf)
    b.record(stream)
    b.synchronize()
    single_ms = a.elapsed_time(b) / steps
    # batched: one graph launch per step, first with the default tiles (all 1, 256
    # threads), then with the autotuned ones; both from the same initial states
    batch = Batch(ctxs, states, dts)
    init = [tuple(t.clone() for t in st) for st in states]
    info0 = batch.infos.clone()

    def run_batched():
        for st, st0 in zip(states, init):
            for t, t0 in zip(st, st0):
                t.copy_(t0)
        batch.infos.copy_(info0)
        for _ in range(warmup):
            batch.step()
        ts = []
        for _ in range(steps):
            flush.fill_(6.0)
            a, b = ev(), ev()
            a.record(stream)
            batch.step()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.mean(ts)

    batch.set_config()
    default_ms = run_batched()
    for st, st0 in zip(states, init):
        for t, t0 in zip(st, st0):
            t.copy_(t0)
    batch.infos.copy_(info0)
    t_tune = time.perf_counter()
    cfg = batch.autotune()
    tune_s = time.perf_counter() - t_tune
    batched_ms = run_batched()
    infos_b = batch.read_infos()
    st = max(i.status for i in infos_b)
    # algorithmic FP64 FLOPs of the timed steps: per problem and stage the qdata
    # contractions, F.1, F^T v and (iterations + 1) mass actions with the CG vector work
    flops = 0.0
    for c, inf in zip(ctxs, infos_b):
        W = work_model(2, c.order, c.q1, c.sizes.ne, c.sizes.n_h1)
        D_, Q_, L_ = c.order + 1, c.q1, c.order
        grad = 2 * Q_ * D_ * D_ + 2 * Q_ * Q_ * D_
        l2i = Q_ * L_ * L_ + Q_ * Q_ * L_
        qd = 2 * c.sizes.ne * (2 * 2 * grad + l2i)
        it = sum(inf.cg_iters)   # iterations of the last step's two solves
        flops += 2 * (qd + W["force_flops"] + W["force_t_flops"] + W["mass_flops"]) + it * W["cg_iter_flops"]
    peak64, _ = probe_peaks()
    achieved = flops / (batched_ms * 1e-3) / 1e12
    rep = {"problems": len(probs), "total_nv": nv, "orders": {p: sum(q["order"] == p for q in probs) for p in range(1, 5)},
           "setup_s": setup_s, "tile_config": cfg, "autotune_s": tune_s,
           "default_config_ms_per_step": default_ms, "autotune_gain": default_ms / batched_ms,
           "batched_ms_per_step": batched_ms, "batched_mdofs": nv / (batched_ms * 1e-3) / 1e6,
           "one_by_one_ms_per_step": single_ms, "one_by_one_mdofs": nv / (single_ms * 1e-3) / 1e6,
           "speedup": single_ms / batched_ms, "status": st,
           "cg_iters_max": max(max(i.cg_iters) for i in infos_b),
           "roofline": {"bound": "alu", "achieved": achieved, "peak": peak64, "unit": "TFLOP/s",
                        "frac": achieved / peak64, "flops_per_step": flops,
                        "note": "algorithmic FP64 FLOPs of the whole batched step (contractions and CG vector "
                                "work, last step's iteration counts) over its CUDA-event time; peak = the FP64 "
                                "FMA-chain probe"},
           "launches_per_step": 6, "note": "one CUDA-graph launch per batched step: per stage the fused "
                                           "qdata + F.1 element pass, one cooperative solver launch (rhs gather, "
                                           "solves, node update) and the F^T v element pass"}
    batch.close()
    for c in ctxs:
        c.close()
    return rep


LEARNED_WEIGHTS = os.path.join(ROOT, "paper_2112_07075_b300", "weights", "mlp_tg3d48_q3.npz")


def learned_report(flush, eval_steps=12, timed_from=2):
    """Learned workload: 3D Taylor-Green Q3/Q2, q1 = 6, 48^3 hexes jittered +-0.1h.
    The MLP carries the weights trained on the configured budget (2000 CFL steps from
    training seeds 1-8 on the 48^3 mesh, `python -m paper_2112_07075_b300.learned`,
    weights committed beside the package); the two held-out seeds 9 and 10 are
    stepped from t = 0 with CFL steps in six modes (FP64, FP32-IR and tensor-core IR,
    each with and without the learned guess); steps from `timed_from` on are timed
    (the guess needs three earlier solves). The warm-start analysis compares, on the
    same right-hand side, a CG solve from zero with the plain warm start."""
    import torch
    from paper_2112_07075_b300 import inputs
    from paper_2112_07075_b300.learned import HELD_OUT_SEEDS, LEARNED_N, load_weights
    from paper_2112_07075_b300.lh import Context, learn_attach, learn_stats
    import numpy as _np
    if not os.path.exists(LEARNED_WEIGHTS):
        return {"unavailable": "trained weights not found: " + LEARNED_WEIGHTS}
    w = _np.load(LEARNED_WEIGHTS)
    net = load_weights(LEARNED_WEIGHTS)
    n = LEARNED_N
    Ve = [inputs.box_vertices(3, n, jitter=0.1, seed=s) for s in HELD_OUT_SEEDS]
    stream = torch.cuda.current_stream()
    out = {"training": {"recipe": str(w["recipe"]), "rows": int(w["rows"]), "loss": [float(x) for x in w["loss"]],
                        "record_s": float(w["record_s"]), "train_s": float(w["train_s"]),
                        "weights": os.path.relpath(LEARNED_WEIGHTS, ROOT)},
           "config": f"held-out seeds {HELD_OUT_SEEDS} at {n}^3, {eval_steps} CFL steps from t = 0, "
                     f"steps {timed_from}..{eval_steps - 1} timed (L2 flushed)"}
    finals = {}
    modes = ("fp64", "fp64+learned", "fp32_ir", "fp32_ir+learned", "bf16tc_ir", "bf16tc_ir+learned")
    analysis = None
    for mode in modes:
        ms, its, used, preds, ratios = [], [], 0, 0, []
        for si, V in enumerate(Ve):
            c = Context(3, n, V, 3, 6, precision=mode.split("+")[0])
            if mode.endswith("learned"):
                learn_attach(c, net, 2)
            xs, vs, es = c.init_state()
            info = c.new_step_info(0.0, 1.0)
            for k in range(eval_steps):
                flush.fill_(7.0)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                c.rk2avg_step(xs, vs, es, 0.0, info)
                b.record(stream)
                b.synchronize()
                if k >= timed_from:
                    ms.append(a.elapsed_time(b))
                    its.append(sum(c.read_step_info(info).cg_iters))
            if mode.endswith("learned"):
                st = learn_stats(c)
                used += st["used"]
                preds += st["predictions"]
                ratios.append(st["mean_residual_ratio"])
            if si == 0:
                finals[mode] = [t.cpu().numpy() for t in (xs, vs, es)]
            if mode == "fp32_ir" and si == 0:
                # warm-start analysis on the state after the run: the next stage-1 right-hand
                # side solved from zero, then by the next step's stage-1 solve, which starts
                # from the last solution (the plain warm start) -- the same system
                rhs, sol = c.h1_vector(), c.h1_vector()
                c.update_qdata(xs, vs, es, None)
                c.force_mult(None, rhs)
                rhs.neg_()
                ci = c.new_cg_info()
                sol.zero_()
                c.mass_cg(rhs, sol, 1e-12, 1000, ci)
                it_zero = c.read_cg_info(ci).iters
                c.rk2avg_step(xs, vs, es, 0.0, info)
                it_prev = c.read_step_info(info).cg_iters[0]
                analysis = {"same_system_iters_from_zero": it_zero, "same_system_iters_from_previous": it_prev,
                            "note": "FP32-IR inner iterations of one stage-1 system of held-out seed 9 after "
                                    f"{eval_steps} steps, solved from a zero guess and from the previous solution"}
            c.close()
        out[mode] = {"ms_per_step": statistics.mean(ms), "cg_iters_per_step": statistics.mean(its)}
        if mode.endswith("learned"):
            out[mode]["learned_guess_used"] = used
            out[mode]["predictions"] = preds
            out[mode]["mean_initial_residual_ratio_learned_vs_previous"] = statistics.mean(ratios)
    base = finals["fp64"]
    for mode in modes[1:]:
        out[mode]["max_rel_field_diff_vs_fp64_gpu"] = max(
            float(_np.linalg.norm(a - b) / _np.linalg.norm(b)) for a, b in zip(finals[mode], base))
        out[mode]["speedup_vs_fp64"] = out["fp64"]["ms_per_step"] / out[mode]["ms_per_step"]
    for base_mode in ("fp64", "fp32_ir", "bf16tc_ir"):
        lm = out[base_mode + "+learned"]
        lm["gain_vs_" + base_mode] = out[base_mode]["ms_per_step"] / lm["ms_per_step"]
        lm["iters_saved_per_step"] = out[base_mode]["cg_iters_per_step"] - lm["cg_iters_per_step"]
    out["warm_start_analysis"] = analysis
    for prec, use_net in (("fp64", False), ("fp32_ir", False), ("fp32_ir", True), ("bf16tc_ir", True)):
        reduced_run("tg3d_6_q3_jit", prec, net if use_net else None)
    out["vs_oracle"] = "reduced case tg3d_6_q3_jit, filled in by the CPU-baseline leg (forms_vs_oracle)"
    net.close()
    return out


def remap_work(dim, p, q1, ne, nh1):
    """FP64 FLOPs of one remap element pass (one stage): gradients of x(tau) and of the
    stage input, interpolation of u, B^T of the advected gradients, the diagonal of
    M(tau), and the pointwise work (adjugate, adv, contraction) at every qpoint."""
    D, Q = p + 1, q1
    if dim == 3:
        interp = Q * D ** 3 + Q * Q * D * D + Q ** 3 * D
        grad = 2 * Q * D ** 3 + 3 * Q * Q * D * D + 3 * Q ** 3 * D
        point = 9 * 2 + 5 + dim * dim + dim * dim + 2   # adjugate, det, adv, contraction, weights
    else:
        interp = Q * D * D + Q * Q * D
        grad = 2 * Q * D * D + 2 * Q * Q * D
        point = 2 + dim * dim + dim * dim + 2
    nq = Q ** dim
    fma = ne * (2 * dim * grad + 2 * dim * interp + interp + nq * point)
    return dict(elem_flops=2 * fma,
                elem_bytes=8 * (3 * dim * nh1 + ne * nq + dim * ne * D ** dim + ne * D ** dim))


def _gll_min_spacing(p):
    """Smallest gap between the p+1 Gauss-Lobatto nodes on [0, 1] (endpoints and the
    roots of P_p'), i.e. the first interior node."""
    if p == 1:
        return 1.0
    r = np.real(np.polynomial.legendre.Legendre.basis(p).deriv().roots())
    return float(0.5 * (1.0 + np.min(r)))


def remap_report(flush, lagrange_steps=50, reps=5, wl_name="tg3d_24_q2"):
    """Velocity remap (Section 3.5) on the headline workload's mesh: after
    `lagrange_steps` CFL steps of 3D Taylor-Green (the paper's runs remap every 50
    cycles), remap v from the Lagrangian mesh back to the initial one. Pseudo-time
    steps: the fewest with the largest nodal displacement per step at most half the
    smallest GLL node spacing. Each timed remap restarts from the same v (restored
    and the L2 flushed outside the events)."""
    import torch
    from paper_2112_07075_b300 import inputs
    from paper_2112_07075_b300.lh import Context
    wl = WORKLOADS[wl_name]
    dim, n, p, q1 = wl["dim"], wl["n"], wl["order"], wl["q1"]
    V = inputs.box_vertices(dim, n, jitter=wl["jitter"], seed=3)
    ctx = Context(dim, n, V, p, q1, cfl=wl["cfl"])
    x, v, e = ctx.init_state("taylor_green")
    x_init = x.clone()
    info = ctx.new_step_info(0.0, wl["t_end"])
    for _ in range(lagrange_steps):
        ctx.rk2avg_step(x, v, e, 0.0, info)
    si = ctx.read_step_info(info)
    hmin = _gll_min_spacing(p) / n
    umax = float((x_init - x).abs().max().item())
    steps = max(1, int(np.ceil(umax / (0.5 * hmin))))
    v_lag = v.clone()
    rinfo = ctx.new_remap_info()
    stream = torch.cuda.current_stream()
    ts = []
    ctx.remap_velocity(x, x_init, v, steps, info=rinfo)      # warm-up
    ctx.timing_enable(True)
    ctx.timing_read()
    solver_ms, solves, iters = 0.0, 0, 0
    torch.cuda.nvtx.range_push("remap")   # lets a profiler select the timed remaps
    for _ in range(reps):
        v.copy_(v_lag)
        flush.fill_(5.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.remap_velocity(x, x_init, v, steps, info=rinfo)
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
        ms, ns = ctx.timing_read()
        solver_ms += ms
        solves += ns
        iters += ctx.read_remap_info(rinfo).cg_iters_total
    torch.cuda.nvtx.range_pop()
    ctx.timing_enable(False)
    ri = ctx.read_remap_info(rinfo)
    st = ctx.sync_status()
    sz = ctx.sizes
    # element pass alone (K(tau) v and the data of M(tau) at one tau), events around one launch
    W = work_model(dim, p, q1, sz.ne, sz.n_h1)
    RW = remap_work(dim, p, q1, sz.ne, sz.n_h1)
    kv = ctx.h1_vector()
    te = []
    for _ in range(reps):
        flush.fill_(6.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.remap_apply(x, x_init, 0.5, v, kv, None)
        b.record(stream)
        b.synchronize()
        te.append(a.elapsed_time(b))
    ms_remap = statistics.mean(ts)
    t_solver = solver_ms / max(1, solves)
    cg_flops = iters * W["cg_iter_flops"] + solves * W["mass_flops"]
    v64 = v.clone()
    # the same remap with the precision form's solver (FP32 inner PCG under FP64 refinement)
    c32 = Context(dim, n, V, p, q1, cfl=wl["cfl"], precision="fp32_ir")
    t32 = []
    for k in range(reps + 1):
        v.copy_(v_lag)
        flush.fill_(5.5)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        c32.remap_velocity(x, x_init, v, steps, info=rinfo)
        b.record(stream)
        b.synchronize()
        if k > 0:
            t32.append(a.elapsed_time(b))
    ri32 = c32.read_remap_info(rinfo)
    diff32 = float((v - v64).norm() / v64.norm())
    st32 = c32.sync_status()
    c32.close()
    ctx.close()
    return {
        "workload": f"{wl['desc']}; v remapped from the mesh after {lagrange_steps} Lagrange CFL steps "
                    f"(t = {si.t:.4g}) back to the initial mesh",
        "pseudo_steps": steps, "max_displacement": umax, "min_gll_spacing": hmin,
        "ms_per_remap": ms_remap, "ms_per_pseudo_step": ms_remap / steps,
        "mdofs": sz.nv / (ms_remap * 1e-3) / 1e6,
        "solves": ri.solves, "cg_iters_total": ri.cg_iters_total, "cg_iters_max": ri.cg_iters_max,
        "cg_rel_res_max": ri.cg_rel_res_max, "status": st,
        "solver_ms_per_solve": t_solver, "solver_share": solver_ms / max(1e-9, sum(ts)),
        "solver_tflops": cg_flops / (solver_ms * 1e-3) / 1e12 if solver_ms > 0 else None,
        "apply_ms": statistics.median(te),
        "apply_note": "lh_remap_apply (displacement, one element pass with K, node gather): events "
                      "around the call",
        "elem_gflop_per_pass": RW["elem_flops"] / 1e9,
        "apply_tflops": RW["elem_flops"] / (statistics.median(te) * 1e-3) / 1e12,
        "metric_note": "mdofs = H1 vector DOFs remapped per second (one whole remap call)",
        "fp32_ir": {"ms_per_remap": statistics.mean(t32), "speedup_vs_fp64": ms_remap / statistics.mean(t32),
                    "inner_iters_total": ri32.cg_iters_total, "cg_rel_res_max": ri32.cg_rel_res_max,
                    "rel_diff_vs_fp64": diff32, "status": st32},
    }


def stiffness_report(flush, lagrange_steps=50, reps=5, wl_name="tg3d_24_q2"):
    """Stiffness operator and discrete Laplacian (Sections 2.1, 3.3, 6) on the
    Lagrangian mesh of the headline workload after `lagrange_steps` CFL steps:
    PA setup on that mesh, the action S_x v, and the Laplacian -M_x^{-1} S_x v of the
    velocity (FP64 PCG to 1e-12 from a zero guess). L2 flushed before every timed call."""
    import torch
    from paper_2112_07075_b300 import inputs
    from paper_2112_07075_b300.lh import Context
    wl = WORKLOADS[wl_name]
    dim, n, p, q1 = wl["dim"], wl["n"], wl["order"], wl["q1"]
    V = inputs.box_vertices(dim, n, jitter=wl["jitter"], seed=3)
    ctx = Context(dim, n, V, p, q1, cfl=wl["cfl"])
    x, v, e = ctx.init_state("taylor_green")
    info = ctx.new_step_info(0.0, wl["t_end"])
    for _ in range(lagrange_steps):
        ctx.rk2avg_step(x, v, e, 0.0, info)
    stream = torch.cuda.current_stream()
    y, lap = ctx.h1_vector(), ctx.h1_vector()
    cinfo = ctx.new_cg_info()

    def timed(fn):
        ts = []
        for _ in range(reps + 1):
            flush.fill_(8.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts[1:])

    def lap_solve():
        lap.zero_()
        ctx.laplacian(v, lap, 1e-12, 1000, cinfo)
    t_setup = timed(lambda: ctx.stiffness_setup(x))
    t_mult = timed(lambda: ctx.stiffness_mult(v, y))
    t_lap = timed(lap_solve)
    ci = ctx.read_cg_info(cinfo)
    st = ctx.sync_status()
    sz = ctx.sizes
    D, Q = p + 1, q1
    grad = 2 * Q * D ** 3 + 3 * Q * Q * D * D + 3 * Q ** 3 * D if dim == 3 else 2 * Q * D * D + 2 * Q * Q * D
    nq = Q ** dim
    ns = dim * (dim + 1) // 2
    mult_flops = 2 * sz.ne * (2 * dim * grad + dim * nq * dim * dim)
    mult_bytes = 8 * (sz.ne * ns * nq + 2 * sz.nv + 2 * sz.ne * dim * D ** dim)
    W = work_model(dim, p, q1, sz.ne, sz.n_h1)
    ctx.close()
    return {
        "workload": f"{wl['desc']}; Lagrangian mesh after {lagrange_steps} CFL steps, velocity field",
        "setup_ms": t_setup, "mult_ms": t_mult, "laplacian_ms": t_lap,
        "laplacian_cg_iters": ci.iters, "laplacian_rel_res": ci.rel_res, "status": st,
        "mult_gflop": mult_flops / 1e9, "mult_tflops": mult_flops / (t_mult * 1e-3) / 1e12,
        "mult_algorithmic_mb": mult_bytes / 1e6,
        "laplacian_tflops": (mult_flops + ci.iters * W["cg_iter_flops"] + W["mass_flops"]) / (t_lap * 1e-3) / 1e12,
        "mult_mdofs": sz.nv / (t_mult * 1e-3) / 1e6,
        "note": "events around each call (setup: element pass + diagonal gather; mult: element pass + "
                "node gather; laplacian: mult + FP64 PCG on M_x from zero)",
    }


def tmop_report(flush, lagrange_steps=50, reps=5, wl_name="tg3d_24_q2"):
    """TMOP kernels (Section 2.2, Section 3.4 Eqs. 6-7, Jacobi diagonal) on the
    Lagrangian mesh of the headline workload after `lagrange_steps` CFL steps, with the
    initial mesh as x0 of the limiting term: target W = h I, h = 1/n, gamma = 0.1,
    d = h/2. Events around each call (element pass + gather), L2 flushed, median of 5."""
    import torch
    from paper_2112_07075_b300 import inputs
    from paper_2112_07075_b300.lh import Context
    wl = WORKLOADS[wl_name]
    dim, n, p, q1 = wl["dim"], wl["n"], wl["order"], wl["q1"]
    V = inputs.box_vertices(dim, n, jitter=wl["jitter"], seed=3)
    ctx = Context(dim, n, V, p, q1, cfl=wl["cfl"])
    x, v, e = ctx.init_state("taylor_green")
    x_init = x.clone()
    info = ctx.new_step_info(0.0, wl["t_end"])
    for _ in range(lagrange_steps):
        ctx.rk2avg_step(x, v, e, 0.0, info)
    stream = torch.cuda.current_stream()
    kw = dict(h=1.0 / n, gamma=0.1, dlim=0.5 / n)
    F = torch.zeros(1, dtype=torch.float64, device="cuda")
    g, y, dg = ctx.h1_vector(), ctx.h1_vector(), ctx.h1_vector()
    u = ctx.h1_vector()
    u.copy_(v)

    def timed(fn):
        ts = []
        for _ in range(reps + 1):
            flush.fill_(9.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts[1:])

    work = ctx.tmop_workspace()
    ypa = ctx.h1_vector()
    t = {"objective": timed(lambda: ctx.tmop_objective(x, x_init, F, **kw)),
         "gradient": timed(lambda: ctx.tmop_gradient(x, x_init, g, **kw)),
         "hessian_mult": timed(lambda: ctx.tmop_hessian_mult(x, u, y, **kw)),
         "hessian_diag": timed(lambda: ctx.tmop_hessian_diag(x, dg, **kw)),
         "hessian_setup_pa": timed(lambda: ctx.tmop_hessian_setup(x, work, **kw)),
         "hessian_mult_pa": timed(lambda: ctx.tmop_hessian_mult_pa(work, u, ypa, **kw))}
    pa_diff = float((ypa - y).norm() / y.norm())
    pa_mb = work.numel() * 8 / 1e6
    del work
    st = ctx.sync_status()
    sz = ctx.sizes
    D, Q = p + 1, q1
    grad = 2 * Q * D ** 3 + 3 * Q * Q * D * D + 3 * Q ** 3 * D if dim == 3 else 2 * Q * D * D + 2 * Q * Q * D
    interp = Q * D ** 3 + Q * Q * D * D + Q ** 3 * D if dim == 3 else Q * D * D + Q * Q * D
    npair = dim * (dim + 1) // 2
    # contraction FMAs per element (the pointwise metric work comes on top)
    nq_ = Q ** dim
    fma = {"objective": dim * (grad + interp), "gradient": dim * (2 * grad + 2 * interp),
           "hessian_mult": dim * (3 * grad + 2 * interp), "hessian_diag": dim * grad + (npair * dim + 1) * interp,
           "hessian_setup_pa": dim * grad,
           "hessian_mult_pa": dim * (2 * grad + 2 * interp) + nq_ * (dim * dim) ** 2}
    out = {"workload": f"{wl['desc']}; Lagrangian mesh after {lagrange_steps} CFL steps, x0 = the initial mesh",
           "params": kw, "objective_value": float(F.item()), "status": st,
           "pa_workspace_mb": pa_mb, "pa_vs_matrix_free_rel_diff": pa_diff,
           "pa_speedup_per_product": t["hessian_mult"] / t["hessian_mult_pa"]}
    for k, ms in t.items():
        out[k] = {"ms": ms, "contraction_gflop": 2 * sz.ne * fma[k] / 1e9,
                  "contraction_tflops": 2 * sz.ne * fma[k] / (ms * 1e-3) / 1e12}
    out["note"] = ("events around each call (fully matrix-free element pass with the metric and its "
                   "derivatives at every qpoint, plus the node gather for the vectors); contraction FLOPs "
                   "only, the pointwise metric work is extra")
    ctx.close()
    return out


def shock_report(flush, n=24, p=2, q1=4, t_end=0.05, max_attempts=2000):
    """Shock workload: 3D Sedov blast (E0 = 0.25 in the corner element, gamma = 1.4) on
    n^3 Q2 hexes, CFL 0.5 steps with the step control and rejection, from t = 0 to
    t_end. Every attempt (accepted or rejected) is timed with events (L2 flushed before
    it); value = vector DOFs x accepted steps / total time of all attempts."""
    import torch
    from paper_2112_07075_b300 import inputs
    from paper_2112_07075_b300.lh import Context
    dim = 3
    V = inputs.box_vertices(dim, n)
    ctx = Context(dim, n, V, p, q1, gamma=1.4, cfl=0.5)
    ctx.set_dt_control(True)
    x, v, e = ctx.init_state("sedov")
    info = ctx.new_step_info(0.0, t_end)
    stream = torch.cuda.current_stream()
    ev = []
    attempts, chunk = 0, 16
    while attempts < max_attempts:
        # chunks of 16 attempts; step by step near t_end so that no attempt runs past it
        for _ in range(chunk):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.fill_(10.0)
            a.record(stream)
            ctx.rk2avg_step(x, v, e, 0.0, info)
            b.record(stream)
            ev.append((a, b))
            attempts += 1
        si = ctx.read_step_info(info)
        left = t_end - si.t
        if left <= 1e-12 * t_end or si.status != 0:
            break
        chunk = 16 if left > 40.0 * si.dt else 1
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    si = ctx.read_step_info(info)
    st = ctx.sync_status()
    sz = ctx.sizes
    real = si.steps + si.rejections
    total = sum(ms)
    vm = v.norm(dim=0)
    gmax = int(torch.argmax(vm).item())
    r_peak = float(x[:, gmax].norm().item())
    out = {"workload": f"3D Sedov blast, {n}^3 hexes, Q{p}/Q{p - 1}, {q1}^3 Gauss points, gamma 1.4, CFL 0.5, "
                       f"step control with rejection, t = 0 -> {t_end}",
           "accepted_steps": si.steps, "rejected_attempts": si.rejections, "t_final": si.t, "status": st,
           "total_ms": total, "ms_per_attempt": total / max(1, real),
           "mdofs": sz.nv * si.steps / (total * 1e-3) / 1e6,
           "cg_iters_per_solve": si.cg_iters_total / max(1, 2 * real),
           "radius_of_max_speed": r_peak, "max_speed": float(vm.max().item())}
    ctx.close()
    return out


def stiffness_cpu_baseline(n=12):
    """The oracle's stiffness action (element matrices + global assembly + product) and
    Laplacian (LU of M_x) of a velocity-like field on an n^3 Q2 mesh with a smooth
    displacement: one of each, timed together."""
    from oracle.fem import Tables
    from oracle.mesh import Mesh
    from oracle.stiffness import Stiffness
    from paper_2112_07075_b300 import inputs
    m = Mesh(inputs.box_vertices(3, n), 3, n, 2)
    x = m.x0 + 0.01 * np.sin(3.0 * m.x0[::-1])
    v = inputs.uniform(8, (3, m.NH1), -1.0, 1.0)
    t0 = time.perf_counter()
    st = Stiffness(m, Tables(3, 2, 4), x)
    st.mult(v)
    t1 = time.perf_counter()
    st.laplacian(v)
    t2 = time.perf_counter()
    return {"value": 3 * m.NH1 / (t1 - t0) / 1e6, "unit": "MDOF/s (setup + action)", "cores": _cores(),
            "kind": "oracle", "laplacian_s": t2 - t1,
            "sample": f"{n}^3 Q2: assembly + one action {t1 - t0:.1f} s, Laplacian (LU) {t2 - t1:.1f} s"}


def tmop_cpu_baseline(n=24):
    """The oracle's TMOP objective and gradient (explicit sums) on the benchmark's
    24^3 Q2 mesh (jittered stand-in for the Lagrangian mesh) and its assembled Hessian
    action on an 8^3 sample (the dense element Hessians grow as NE x (3 x 27)^2)."""
    from oracle.fem import Tables
    from oracle.mesh import Mesh
    from oracle.tmop import Tmop
    from paper_2112_07075_b300 import inputs
    out = {}
    for nn, what in ((n, "grad"), (8, "hess")):
        m = Mesh(inputs.box_vertices(3, nn, jitter=0.1, seed=3), 3, nn, 2)
        x0 = Mesh(inputs.box_vertices(3, nn), 3, nn, 2).x0
        tm = Tmop(m, Tables(3, 2, 4), np.eye(3) / nn, x0, gamma=0.1, dlim=0.5 / nn)
        t0 = time.perf_counter()
        if what == "grad":
            tm.objective(m.x0)
            tm.gradient(m.x0)
        else:
            tm.hessian_mult(m.x0, m.x0)
        out[what] = (time.perf_counter() - t0, 3 * m.NH1)
    tg, ng = out["grad"]
    th, nh = out["hess"]
    return {"value": ng / tg / 1e6, "unit": "MDOF/s (objective + gradient)", "cores": _cores(), "kind": "oracle",
            "hessian_mult_mdofs_8cubed": nh / th / 1e6,
            "sample": f"objective + gradient at {n}^3 Q2 {tg:.1f} s; Hessian assembly + action at 8^3 {th:.1f} s"}


def shock_cpu_baseline(n=8, attempts=6):
    """The oracle's controlled steps of the 3D Sedov blast on an n^3 Q2 mesh."""
    from oracle.hydro import Hydro, Params, controlled_step
    from paper_2112_07075_b300 import inputs
    hy = Hydro(Params(dim=3, n=n, order=2, q1=4, vertices=inputs.box_vertices(3, n), gamma=1.4, cfl=0.5))
    x, v, e = hy.initial_state("sedov")
    t, c, acc = 0.0, 0.0, 0
    t0 = time.perf_counter()
    for _ in range(attempts):
        x, v, e, info = controlled_step(hy, x, v, e, t, 1.0, c)
        c = info.extra["c"]
        if not info.extra["rejected"]:
            t += info.dt
            acc += 1
    dt = time.perf_counter() - t0
    return {"value": 3 * hy.mesh.NH1 * acc / dt / 1e6, "unit": "MDOF/s", "cores": _cores(), "kind": "oracle",
            "sample": f"{attempts} controlled attempts ({acc} accepted) of 3D Sedov at {n}^3 Q2, {dt:.1f} s"}


def remap_cpu_baseline(n=12):
    """The oracle's remap (global assembly, direct solves) on one pseudo-time step of
    an n^3 Q2 mesh with a smooth displacement (a bounded sample: LU of the 3D mass
    matrix at 24^3 takes more than 15 minutes)."""
    from oracle.fem import Tables
    from oracle.mesh import Mesh
    from oracle.remap import Remap
    from paper_2112_07075_b300 import inputs
    m = Mesh(inputs.box_vertices(3, n), 3, n, 2)
    x1 = m.x0 + 0.005 * np.sin(3.0 * m.x0)
    R = Remap(m, Tables(3, 2, 4), x1, m.x0)
    v = inputs.uniform(8, (3, m.NH1), -1.0, 1.0)
    t0 = time.perf_counter()
    R.remap(v, 1)
    dt = time.perf_counter() - t0
    return {"value": 3 * m.NH1 / dt / 1e6, "unit": "MDOF/s (one pseudo-step)", "cores": _cores(),
            "kind": "oracle", "sample": f"1 pseudo-time step of a {n}^3 Q2 mesh, {dt:.1f} s"}


# ---------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def _cores():
    try:
        from threadpoolctl import threadpool_info
        n = max((i.get("num_threads", 1) for i in threadpool_info()), default=1)
        return int(n)
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(wl, V, steps=1):
    from oracle.hydro import Hydro, Params
    hy = Hydro(Params(dim=wl["dim"], n=wl["n"], order=wl["order"], q1=wl["q1"], vertices=V, cfl=wl["cfl"]))
    x, v, e = hy.initial_state("taylor_green")
    t0 = time.perf_counter()
    t = 0.0
    for _ in range(steps):
        x, v, e, info = hy.rk2avg_step(x, v, e, dt=None, t=t, t_end=wl["t_end"])
        t += info.dt
    dt = time.perf_counter() - t0
    nv = wl["dim"] * hy.mesh.NH1
    return {"value": nv * steps / dt / 1e6, "unit": "MDOF/s", "cores": _cores(), "kind": "oracle",
            "sample": f"{steps} RK2-average step(s) of the same workload from t=0 (setup excluded), "
                      f"{dt:.1f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2112_07075_b300 import inputs
    from oracle.hydro import Hydro, Params
    wl = WORKLOADS[args.workload]
    V = inputs.box_vertices(wl["dim"], wl["n"], jitter=wl["jitter"], seed=3)
    hy = Hydro(Params(dim=wl["dim"], n=wl["n"], order=wl["order"], q1=wl["q1"], vertices=V, cfl=wl["cfl"]))
    x, v, e = hy.initial_state("taylor_green")
    steps = max(1, min(args.steps, 2))
    t = 0.0
    x, v, e, info = hy.rk2avg_step(x, v, e, dt=None, t=t, t_end=wl["t_end"])   # warm-up
    t += info.dt
    t0 = time.perf_counter()
    for _ in range(steps):
        x, v, e, info = hy.rk2avg_step(x, v, e, dt=None, t=t, t_end=wl["t_end"])
        t += info.dt
    el = time.perf_counter() - t0
    nv = wl["dim"] * hy.mesh.NH1
    val = nv * steps / el / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "MDOF/s", "n_gpus": world,
            "steps": steps, "warmup": 1, "ms_per_step": 1e3 * el / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["desc"], "dim": wl["dim"], "n": wl["n"], "order": wl["order"],
                       "q1": wl["q1"]},
            "cpu_baseline": {"value": val, "unit": "MDOF/s", "cores": _cores(), "kind": "oracle",
                             "sample": f"{steps} timed RK2-average steps after 1 warm-up step "
                                       f"(bounded sample of the requested {args.steps})"},
            "e2e": {"value": val, "unit": "MDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20,
                    help="timed RK2 steps; 0 = the whole run from t = 0 to the workload's t_end")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tg3d_24_q2", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--forms", default="all",
                    choices=["all", "precision", "batching", "learned", "remap", "stiffness", "tmop", "shock"],
                    help="which form reports to add (default all; --no-forms for none)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32_ir", "bf16tc_ir"],
                    help="mass-solve precision of the main arm (the headline workload is FP64)")
    ap.add_argument("--remap-only", action="store_true",
                    help="print only the velocity-remap report (rank 0, one GPU)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.remap_only:
        run_remap_only(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
