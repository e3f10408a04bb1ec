#!/usr/bin/env python
"""Benchmark of the implicit Lagrangian hydrodynamics hot path on B300.

One step = one implicit midpoint Newton-GMRES step (residual, Jacobian actions inside
GMRES, preconditioner, Gram-Schmidt, line search, update) on the 3D point-blast
workload: [0,1]^3, 24^3 hexes, Q2-Q1, gamma 1.4, smooth viscosity, walls, state after a
few implicit steps from the corner deposit, dt = 2 x the explicit estimate.

value = unknowns x (residual + Jacobian-action evaluations) per second of step time
(GDoF/s of J.w & residual over the whole step), the chosen form = FP64 residual with
an FP32 Jacobian action.  Also reported: the plain FP64 step, standalone operator
throughputs, the roofline of the dominant kernel and the CPU oracle baseline.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = {"name": "blast3d_24_q2q1", "dim": 3, "n": (24, 24, 24), "k": 2, "gamma": 1.4, "energy": 0.25,
            "develop_steps": 3, "cfl": 2.0}
# Newton relative tolerance of the paper's defaults (Sec. 3.5); inexact Newton with GMRES to
# 1e-4 per linear solve.  (At 1e-8 the third Newton iterate of the workload sits at the
# threshold, 0.9-1.6e-8 depending on rounding, and the iteration count flips between forms.)
NEWTON = {"newton_rtol": 1e-5, "gmres_rtol": 1e-4, "gmres_maxit": 200, "restart": 30, "newton_maxit": 20}
L2_FLUSH_BYTES = 512 << 20


def _hbm_peak():
    """Measured copy bandwidth of this GPU pool (GB/s), else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6400.0, "fallback"


HBM_PEAK_GBS, HBM_PEAK_SOURCE = _hbm_peak()


def sf_macs(dim, k):
    """Multiply-adds of the sum-factorised contractions per element and field component."""
    D, Q = k + 1, 2 * k
    if dim == 3:
        grad = 2 * D ** 3 * Q + 3 * D ** 2 * Q ** 2 + 3 * D * Q ** 3
        valgrad = 2 * D ** 3 * Q + 3 * D ** 2 * Q ** 2 + 4 * D * Q ** 3

        def val(N):
            return N ** 3 * Q + N ** 2 * Q ** 2 + N * Q ** 3
    else:
        grad = 2 * D ** 2 * Q + 2 * D * Q ** 2
        valgrad = 2 * D ** 2 * Q + 3 * D * Q ** 2

        def val(N):
            return N ** 2 * Q + N * Q ** 2
    return grad, valgrad, val


def flops_per_element(dim, k, kind, visc=True):
    """Algorithmic FLOPs per element: contractions (2 per multiply-add, minimal factorised
    forms) + quadrature-point kernel (exact count of its code, lh_qp_flops) + per-point glue."""
    import ctypes as C
    import paper_2609_16424_b300 as lh
    grad, valgrad, val = sf_macs(dim, k)
    nq = (2 * k) ** dim
    qk = {"residual": 0, "jvp": 1, "jvp_rec": 3, "jtvp": 2}[kind]
    ops = C.c_longlong()
    lh.lib.lh_qp_flops(dim, qk, int(visc), C.byref(ops))
    if kind == "residual":
        macs = 2 * dim * grad + dim * val(k + 1) + 2 * val(k) + dim * valgrad + val(k)
        glue = dim + 2 + 3
    elif kind == "jvp":
        macs = 3 * dim * grad + dim * valgrad + 2 * val(k) + dim * valgrad + val(k)
        glue = 2 * dim * dim + 1 + dim + 2 + 3
    elif kind == "jvp_rec":   # linearised point map read from the record
        macs = dim * grad + dim * valgrad + val(k) + dim * valgrad + val(k)
        glue = 2 * dim * dim + 1 + dim + 2 + 2
    else:
        macs = 2 * dim * grad + dim * valgrad + 2 * val(k) + 2 * dim * valgrad + val(k)
        glue = 2 * dim * dim + dim + 3 + 3
    return 2 * macs + nq * (ops.value + glue)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms in the background; entering
    waits (up to 3 s) for the first sample so that the samples cover the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.perf_counter()
            while not self.rows and time.perf_counter() - t0 < 3.0:
                time.sleep(0.01)
            self.rows.clear()   # keep only the samples taken from here on
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace('.', '').isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace('.', '').isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 5 + i and r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows),
                "power_w_max": max(float(r[3]) for r in self.rows if r[3].replace('.', '').isdigit())
                if any(r[3].replace('.', '').isdigit() for r in self.rows) else None}


# ------------------------------------------------------------------------------------------
def setup_ours(device):
    import torch
    import paper_2609_16424_b300 as lh
    from paper_2609_16424_b300.states import blast_state
    W = WORKLOAD
    mesh = lh.Mesh(W["dim"], W["n"], (0.0,) * 3, (1.0,) * 3, W["k"], gamma=W["gamma"], visc=True,
                   device=device)
    u = blast_state(mesh, W["energy"])
    k = torch.zeros_like(u)
    for _ in range(W["develop_steps"]):
        dt = W["cfl"] * mesh.dt_estimate(u)
        mesh.newton_step(u, k, dt, jvp_prec="fp64", **NEWTON)
    dt = W["cfl"] * mesh.dt_estimate(u)
    return mesh, u, k, dt


def timed_steps(mesh, u_s, k_s, dt, steps, prec, flush, profile=False, arnoldi=1):
    """Per-step CUDA-event times (ms) and stats; the L2 flush between steps is not timed.
    profile: CUDA events around every element-kernel launch (the Arnoldi loop then runs on the
    host: events cannot be recorded inside the device-driven loop's graph)."""
    import torch
    import paper_2609_16424_b300 as lh
    u, k = u_s.clone(), k_s.clone()
    stream = torch.cuda.current_stream()
    times, stats = [], []
    if profile:
        mesh.profile(True)
    l0 = lh.launch_count()
    for _ in range(steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        u.copy_(u_s)
        k.copy_(k_s)
        st = mesh.newton_step(u, k, dt, jvp_prec=prec, arnoldi=0 if profile else arnoldi, **NEWTON)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        stats.append(st)
    launches = lh.launch_count() - l0
    prof = mesh.profile_read() if profile else None
    if profile:
        mesh.profile(False)
    return times, stats, launches, prof


# DRAM bytes (read + write) per launch of a kernel, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) of a launch inside the Newton steps of this
# workload (the event-instrumented repeat), with the digest of the CUDA sources it was built
# from.  The figure is
# reported only while the sources still have that digest (csrc_digest()).
NCU_TRAFFIC = {"k_jvp_rec_pipe<3,2,float>": {"bytes": 91842304 + 48640, "csrc": "063481fd900bc497"},
               "k_residual<3,2>": {"bytes": 13419008 + 40239104, "csrc": "063481fd900bc497"}}


def csrc_digest():
    """sha256 (16 hex digits) over the library's CUDA sources and the C header."""
    import glob
    import hashlib
    h = hashlib.sha256()
    files = sorted(glob.glob(os.path.join(ROOT, "paper_2609_16424_b300", "csrc", "*"))) + [
        os.path.join(ROOT, "include", "lh.h")]
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def fp32_ops_residual(dim, k, visc=True):
    """Float operations per element of the residual kernel as it runs: the sum-factorised
    contractions in double-float (a multiply-add costs 15 float operations: TwoProd with its
    cross terms 4, the accumulation TwoSum + FastTwoSum 11) and the point kernel in
    double-word arithmetic (lh_qp_flops kind 4), the per-point glue (dim + 4 products, one
    sum) weighed the same way (8 and 20 float operations)."""
    import ctypes as C
    import paper_2609_16424_b300 as lh
    grad, valgrad, val = sf_macs(dim, k)
    macs = 2 * dim * grad + dim * val(k + 1) + 2 * val(k) + dim * valgrad + val(k)
    ops = C.c_longlong()
    lh.lib.lh_qp_flops(dim, 4, int(visc), C.byref(ops))
    return 15 * macs + (2 * k) ** dim * (ops.value + 8 * (dim + 4) + 20)


def rec_kernel_name(dim, k):
    """The library's FP32 record J.w kernel for (dim, k): pipelined for elements of 64 points
    (3D Q2, 2D Q4), one point per thread for 3D Q1, else two points per thread."""
    if (dim, k) in ((3, 2), (2, 4)):
        return f"k_jvp_rec_pipe<{dim},{k},float>"
    if (dim, k) == (3, 1):
        return f"k_jvp_rec<{dim},{k},float>"
    return f"k_jvp_rec2<{dim},{k},float>"


def dominant_roofline(kind, launch_ms, ne, k, prec, fp64_peak, fp32_peak):
    """Roofline of the step's dominant element kernel (3D, order k).
    residual: float operations of its double-word arithmetic against the FP32 pipe's
    operation rate (half the FMA FLOP/s probe; an FMA is one operation), with the
    FP64-accurate algorithmic FLOP/s beside it against the FP64 FMA probe.
    FP32 record J.w: the larger of its FP32-FLOP fraction and its HBM fraction (algorithmic
    bytes: record, direction, element output)."""
    t = launch_ms * 1e-3
    name = {"residual": f"k_residual<3,{k}>", "jvp_fp64": f"k_jvp<3,{k},double,double>",
            "jvp_fp32": rec_kernel_name(3, k), "jvp_tc": f"k_jvp_tc<3,{k},{prec}>"}.get(kind, kind)
    out = {"kernel": name, "launch_ms": round(launch_ms, 5), "peak_source": "measured FMA probe (lh_probe_fma) "
           "this run" if kind != "jvp_fp32" else None}
    if kind == "residual":
        ops = fp32_ops_residual(3, k) * ne
        fl = flops_per_element(3, k, "residual") * ne
        out.update({"bound": "alu", "pipe": "fp32 (double-word arithmetic)", "unit": "Top/s",
                    "achieved": round(ops / t / 1e12, 4), "peak": round(fp32_peak / 2, 3),
                    "frac": round(ops / t / 1e12 / (fp32_peak / 2), 4), "fp32_ops_per_launch": ops,
                    "fp64_accurate_tflops": round(fl / t / 1e12, 4), "fp64_fma_peak_tflops": round(fp64_peak, 3),
                    "algorithmic_flops_per_launch": fl})
        return out
    if kind == "jvp_fp32":
        fl = flops_per_element(3, k, "jvp_rec") * ne
        by = record_bytes(3, k, ne)
        ff, fb = fl / t / 1e12 / fp32_peak, by / t / 1e9 / HBM_PEAK_GBS
        if fb >= ff:
            out.update({"bound": "hbm", "unit": "GB/s", "achieved": round(by / t / 1e9, 1), "peak": HBM_PEAK_GBS,
                        "frac": round(fb, 4), "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({HBM_PEAK_SOURCE})"})
        else:
            out.update({"bound": "alu", "pipe": "fp32", "unit": "TFLOP/s", "achieved": round(fl / t / 1e12, 4),
                        "peak": round(fp32_peak, 3), "frac": round(ff, 4),
                        "peak_source": "measured FMA probe (lh_probe_fma) this run"})
        out.update({"algorithmic_bytes_per_launch": by, "algorithmic_flops_per_launch": fl,
                    "hbm_frac": round(fb, 4), "fp32_flop_frac": round(ff, 4)})
        return out
    fl = flops_per_element(3, k, {"jvp_fp64": "jvp", "jvp_tc": "jvp_rec"}[kind]) * ne
    peak = fp64_peak if kind == "jvp_fp64" else fp32_peak
    out.update({"bound": "alu", "pipe": "fp64" if kind == "jvp_fp64" else "fp32", "unit": "TFLOP/s",
                "achieved": round(fl / t / 1e12, 4), "peak": round(peak, 3), "frac": round(fl / t / 1e12 / peak, 4),
                "algorithmic_flops_per_launch": fl})
    return out


def tc_mma_flops(dim, k, ne, kind):
    """Tensor-core flops one k_jvp_tc launch issues (dense, padded element operators:
    per batch of 16 elements one 128 x NF x KF forward MMA and 128 x NB x 64 backward MMAs
    over the padded quadrature points).  Not algorithmic work: reported for pipe usage."""
    rup = lambda x, m: (x + m - 1) // m * m
    nd, nl, nq = (k + 1) ** dim, k ** dim, (2 * k) ** dim
    nqp = rup(nq, 16)
    mk = 8 if kind == "tf32" else 16
    nf, kf, nb = 4 * nqp, rup(nd + nl, mk), rup(nd + nl, 16)
    batches = (ne + 15) // 16
    return batches * 2 * 128 * (nf * kf + nb * 4 * nqp)


def kernel_rate(mesh, fn, reps, flush):
    """Mean CUDA-event time (ms) of fn() over reps calls, L2 flushed before each."""
    import torch
    stream = torch.cuda.current_stream()
    ts = []
    for _ in range(reps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def e2e_steps(mesh, u_s, k_s, dt, steps, prec):
    """Same step through the public API with host buffers: pinned host -> device copy of
    (u, k_prev), the Newton step, device -> host copy of (u, k) inside the timed region."""
    import torch
    hu, hk = u_s.cpu().pin_memory(), k_s.cpu().pin_memory()
    ou, ok = torch.empty_like(hu).pin_memory(), torch.empty_like(hk).pin_memory()
    u, k = torch.empty_like(u_s), torch.empty_like(k_s)
    evals = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        u.copy_(hu, non_blocking=True)
        k.copy_(hk, non_blocking=True)
        st = mesh.newton_step(u, k, dt, jvp_prec=prec, **NEWTON)
        ou.copy_(u, non_blocking=True)
        ok.copy_(k, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        evals += st["residual_evals"] + st["jvp_evals"]
    t = time.perf_counter() - t0
    nbytes = 8 * mesh.n * 2
    return mesh.n * evals / t / 1e9, t / steps * 1e3, nbytes


def one_thread():
    """Limit BLAS pools to one thread when threadpoolctl is available (the oracle's
    einsum contractions run single-threaded either way)."""
    try:
        from threadpoolctl import threadpool_limits
        return threadpool_limits(limits=1)
    except ImportError:
        import contextlib
        return contextlib.nullcontext()


def oracle_residual_rate(u_np, k_np, tau, budget_s=15.0):
    """The CPU oracle's residual on the same workload state, single-threaded."""
    from oracle.fem import Mesh as OMesh
    from oracle.hydro import Hydro, Params
    W = WORKLOAD
    with one_thread():
        om = OMesh(W["n"], (0.0,) * 3, (1.0,) * 3, W["k"])
        hyd = Hydro(om, Params(om, gamma=W["gamma"], visc=True))
        t0 = time.perf_counter()
        reps = 0
        r = None
        while True:
            r = hyd.residual(u_np, k_np, tau)
            reps += 1
            if time.perf_counter() - t0 >= budget_s or reps >= 50:
                break
        t = (time.perf_counter() - t0) / reps
    return om.n_unknowns / t / 1e9, reps, t, r


def _oracle_worker(args):
    """One oracle process: residual evaluations of the bench state for about budget_s."""
    u_np, k_np, tau, budget_s = args
    with one_thread():
        from oracle.fem import Mesh as OMesh
        from oracle.hydro import Hydro, Params
        W = WORKLOAD
        om = OMesh(W["n"], (0.0,) * 3, (1.0,) * 3, W["k"])
        hyd = Hydro(om, Params(om, gamma=W["gamma"], visc=True))
        t0 = time.perf_counter()
        reps = 0
        while True:
            hyd.residual(u_np, k_np, tau)
            reps += 1
            if time.perf_counter() - t0 >= budget_s:
                break
        return reps, time.perf_counter() - t0, om.n_unknowns


def oracle_all_cores(u_np, k_np, tau, budget_s=8.0, max_procs=32, gb_per_proc=2.0):
    """The oracle on all host cores: one single-threaded process per core (spawned), each
    evaluating the residual of the full bench state; rate = all evaluations x n / the slowest
    process's time.  Processes are capped by max_procs and by available memory (~1.5 GB each)."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    procs = min(cores, max_procs)
    try:
        import psutil
        procs = max(1, min(procs, int(psutil.virtual_memory().available / (gb_per_proc * 2 ** 30))))
    except ImportError:
        pass
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        res = pool.map(_oracle_worker, [(u_np, k_np, tau, budget_s)] * procs)
    reps = sum(r[0] for r in res)
    t = max(r[1] for r in res)
    n = res[0][2]
    return n * reps / t / 1e9, procs, cores, reps, t


def aggregate_ranks(total_ms, units, device):
    """Whole-job timing over ranks: the slowest rank's time and the units of all ranks
    (weak scaling over independent replicas; no data-path collective)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_ms, float(units)], dtype=torch.float64, device=device)
    tmax, tsum = t.clone(), t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return tmax[0].item(), tsum[1].item()


# ------------------------------------------------------------------------------------------
def run_ours(args, rank, world, device):
    import numpy as np
    import torch
    import paper_2609_16424_b300 as lh
    torch.cuda.set_device(device)
    mesh, u_s, k_s, dt = setup_ours(device)
    n = mesh.n
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    prec = args.prec
    # warm-up (untimed)
    timed_steps(mesh, u_s, k_s, dt, args.warmup, prec, flush)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        wall0 = time.perf_counter()
        torch.cuda.nvtx.range_push("timed")
        times, stats, launches, _ = timed_steps(mesh, u_s, k_s, dt, args.steps, prec, flush)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        wall = time.perf_counter() - wall0
    # element-kernel durations: CUDA events around each launch in a repeat of the timed steps
    # (same state, kernels and inputs; the Arnoldi loop on the host, where events can be placed)
    torch.cuda.nvtx.range_push("kernel_timing")
    times_p, _, _, prof = timed_steps(mesh, u_s, k_s, dt, args.steps, prec, flush, profile=True)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if world > 1:
        torch.distributed.barrier()
    step_ms = sum(times) / len(times)
    evals = sum(s["residual_evals"] + s["jvp_evals"] for s in stats)
    total_ms = sum(times)
    units = n * evals
    if world > 1:
        total_ms, units = aggregate_ranks(total_ms, units, device)
    value = units / (total_ms * 1e-3) / 1e9
    if rank != 0:
        return None
    if args.quick:
        return {"metric": "quick", "value": round(value, 4), "ms_per_step": round(step_ms, 4),
                "step_kernel_ms": {k2: round(v[0], 3) for k2, v in prof.items()}, "gpu_launches": launches,
                "newton": [{k2: s[k2] for k2 in ("newton_its", "gmres_its_total", "residual_evals", "jvp_evals")}
                           for s in stats]}

    # plain FP64 form and the other reduced-precision J.w forms for comparison
    t64, s64, _, _ = timed_steps(mesh, u_s, k_s, dt, max(2, min(args.steps, 5)), "fp64", flush)
    other = {}
    for p2 in ("fp32", "tf32", "bf16"):
        if p2 == prec:
            continue
        tp, sp, _, _ = timed_steps(mesh, u_s, k_s, dt, max(2, min(args.steps, 5)), p2, flush)
        other[p2] = {"ms_per_step": round(sum(tp) / len(tp), 4),
                     "newton_its_per_step": statistics.mean(s["newton_its"] for s in sp),
                     "gmres_its_per_step": statistics.mean(s["gmres_its_total"] for s in sp)}
    # standalone operators on the bench state
    kd = k_s
    tau = 0.5 * dt
    r = torch.empty_like(u_s)
    dkd = torch.randn(n, dtype=torch.float64, device=device, generator=torch.Generator(device).manual_seed(0))
    dkf = dkd.float()
    of = torch.empty(n, dtype=torch.float32, device=device)
    od = torch.empty_like(u_s)
    reps = 10
    t_res = kernel_rate(mesh, lambda: mesh.residual(u_s, kd, tau, out=r), reps, flush)
    t_j64 = kernel_rate(mesh, lambda: mesh.jvp(u_s, kd, tau, dkd, out=od), reps, flush)
    t_j32 = kernel_rate(mesh, lambda: mesh.jvp(u_s, kd, tau, dkf, out=of), reps, flush)
    mesh.linearize(u_s, kd, tau)
    t_j32r = kernel_rate(mesh, lambda: mesh.jvp(u_s, kd, tau, dkf, out=of, lin=True), reps, flush)
    yv = torch.randn(n, dtype=torch.float64, device=device, generator=torch.Generator(device).manual_seed(5))
    yf = yv.float()
    t_jt64 = kernel_rate(mesh, lambda: mesh.jtvp(u_s, kd, tau, yv), reps, flush)
    t_jt32 = kernel_rate(mesh, lambda: mesh.jtvp(u_s, kd, tau, yf, lin=True), reps, flush)
    t_tc, kp_tc = {}, {}
    for kind in ("tf32", "bf16"):
        t_tc[kind] = kernel_rate(mesh, lambda: mesh.jvp(u_s, kd, tau, dkf, out=of, tc=kind), reps, flush)
        mesh.profile(True)
        for _ in range(reps):
            flush.fill_(1.0)
            mesh.jvp(u_s, kd, tau, dkf, out=of, tc=kind)
        kp_tc[kind] = mesh.profile_read()["jvp_tc"]
        mesh.profile(False)
    mesh.tc_status()
    # element-kernel-only times from the profiler (the roofline kernels)
    mesh.profile(True)
    for _ in range(reps):
        flush.fill_(1.0)
        mesh.residual(u_s, kd, tau, out=r)
        flush.fill_(1.0)
        mesh.jvp(u_s, kd, tau, dkd, out=od)
        flush.fill_(1.0)
        mesh.jvp(u_s, kd, tau, dkf, out=of)
    kp = mesh.profile_read()
    mesh.profile(True)
    for _ in range(reps):
        flush.fill_(1.0)
        mesh.jvp(u_s, kd, tau, dkf, out=of, lin=True)
    kpr = mesh.profile_read()
    mesh.profile(False)

    fp64_peak = lh.probe_fma("fp64")
    fp32_peak = lh.probe_fma("fp32")
    W = WORKLOAD
    ne = mesh.NE
    fl = {kind: flops_per_element(3, W["k"], kind) for kind in ("residual", "jvp", "jvp_rec")}
    # dominant kernel of the timed steps
    dom = max(prof.items(), key=lambda kv: kv[1][0])
    dom_kind, (dom_ms, dom_cnt) = dom[0], dom[1]
    roofline = dominant_roofline(dom_kind, dom_ms / dom_cnt, ne, W["k"], prec, fp64_peak, fp32_peak)
    roofline.update({"launches": dom_cnt, "share_of_step": round(dom_ms / sum(times_p), 4),
                     "timing": "CUDA events around each launch on the mesh stream, in a repeat of the timed "
                               "steps with the host-driven Arnoldi loop (the timed steps run it as one CUDA "
                               "graph per restart cycle, where events cannot be recorded)"})

    cap = NCU_TRAFFIC.get(roofline["kernel"])
    roofline["traffic"] = None
    if cap is not None and cap["csrc"] == csrc_digest():
        roofline["traffic"] = cap["bytes"]
        roofline["traffic_source"] = "ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch of this build"
    else:
        roofline["traffic_source"] = ("no ncu capture of this build of the kernel" if cap is None else
                                      "null: the kernel sources changed since the ncu capture")
    roofline["csrc_digest"] = csrc_digest()
    e2e_val, e2e_ms, e2e_bytes = e2e_steps(mesh, u_s, k_s, dt, max(2, min(args.steps, 5)), prec)
    out = {
        "metric": "GDoF/s of J.w & residual over the implicit step (FP64 residual, FP32 J.w)",
        "value": round(value, 4), "unit": "GDoF/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(step_ms, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic (corner point blast, developed 3 steps)",
        "config": {"workload": W["name"], "mesh": "24x24x24 hex, [0,1]^3", "order": "Q2-Q1", "n_unknowns": n,
                   "quad_points": mesh.NQ, "dt": dt, "cfl_multiple": W["cfl"], "newton": NEWTON,
                   "jvp_prec": prec, "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "wall_s_timed_region": round(wall, 3),
        "newton": {"its_per_step": statistics.mean(s["newton_its"] for s in stats),
                   "gmres_its_per_step": statistics.mean(s["gmres_its_total"] for s in stats),
                   "evals_per_step": evals / len(stats)},
        "other_jvp_forms_step": other,
        "plain_fp64_step": {"ms_per_step": round(sum(t64) / len(t64), 4),
                            "gmres_its_per_step": statistics.mean(s["gmres_its_total"] for s in s64),
                            "value": round(n * sum(s["residual_evals"] + s["jvp_evals"] for s in s64) / (sum(t64) * 1e-3) / 1e9, 4)},
        "kernels": {
            "residual_fp64": {"gdofs": round(n / (t_res * 1e-3) / 1e9, 4), "ms": round(t_res, 5),
                              "elem_kernel_ms": round(kp["residual"][0] / max(1, kp["residual"][1]), 5),
                              "tflops_elem": round(fl["residual"] * ne / (kp["residual"][0] / max(1, kp["residual"][1]) * 1e-3) / 1e12, 4)},
            "jvp_fp64": {"gdofs": round(n / (t_j64 * 1e-3) / 1e9, 4), "ms": round(t_j64, 5),
                         "elem_kernel_ms": round(kp["jvp_fp64"][0] / max(1, kp["jvp_fp64"][1]), 5),
                         "tflops_elem": round(fl["jvp"] * ne / (kp["jvp_fp64"][0] / max(1, kp["jvp_fp64"][1]) * 1e-3) / 1e12, 4)},
            "jvp_fp32": {"gdofs": round(n / (t_j32 * 1e-3) / 1e9, 4), "ms": round(t_j32, 5),
                         "elem_kernel_ms": round(kp["jvp_fp32"][0] / max(1, kp["jvp_fp32"][1]), 5),
                         "tflops_elem": round(fl["jvp"] * ne / (kp["jvp_fp32"][0] / max(1, kp["jvp_fp32"][1]) * 1e-3) / 1e12, 4)},
            "jvp_fp32_record": {"gdofs": round(n / (t_j32r * 1e-3) / 1e9, 4), "ms": round(t_j32r, 5),
                                "elem_kernel_ms": round(kpr["jvp_fp32"][0] / max(1, kpr["jvp_fp32"][1]), 5),
                                "tflops_elem": round(fl["jvp_rec"] * ne / (kpr["jvp_fp32"][0] / max(1, kpr["jvp_fp32"][1]) * 1e-3) / 1e12, 4)},
            "jtvp_fp64": {"gdofs": round(n / (t_jt64 * 1e-3) / 1e9, 4), "ms": round(t_jt64, 5)},
            "jtvp_fp32_record": {"gdofs": round(n / (t_jt32 * 1e-3) / 1e9, 4), "ms": round(t_jt32, 5)},
            **{f"jvp_{kind}_tensor_core": {
                "gdofs": round(n / (t_tc[kind] * 1e-3) / 1e9, 4), "ms": round(t_tc[kind], 5),
                "elem_kernel_ms": round(kp_tc[kind][0] / max(1, kp_tc[kind][1]), 5),
                "tflops_elem": round(fl["jvp_rec"] * ne / (kp_tc[kind][0] / max(1, kp_tc[kind][1]) * 1e-3) / 1e12, 4),
                "tensor_tflops": round(tc_mma_flops(3, W["k"], ne, kind) / (kp_tc[kind][0] / max(1, kp_tc[kind][1]) * 1e-3) / 1e12, 4)}
               for kind in ("tf32", "bf16")},
            "flops_per_element": fl, "fp64_peak_tflops": round(fp64_peak, 3), "fp32_peak_tflops": round(fp32_peak, 2)},
        "step_kernel_ms": {k2: round(v[0], 3) for k2, v in prof.items()},
        "roofline": roofline,
        "gpu_launches": launches,
        "e2e": {"value": round(e2e_val, 4), "unit": "GDoF/s", "ms_per_step": round(e2e_ms, 4),
                "h2d_bytes_per_step": e2e_bytes, "d2h_bytes_per_step": e2e_bytes},
        "clocks": clk.summary(),
    }
    if not args.headline_only and world == 1:
        w0 = time.perf_counter()
        out["config5_48cube"] = {
            "workload": "48^3 hex point blast / perturbed state, Q_k-Q_{k-1}, k = 1..4",
            "element_kernels": sweep_rows([1, 2, 3, 4], flush, fp64_peak, fp32_peak, device),
            "implicit_steps": config5_steps([1, 2, 3, 4], {1: 20, 2: 20, 3: 3, 4: 2}, 20, flush, device),
            "newton": NEWTON, "hbm_peak_gbs": HBM_PEAK_GBS, "hbm_peak_source": HBM_PEAK_SOURCE,
            "fp64_peak_tflops": round(fp64_peak, 3), "fp32_peak_tflops": round(fp32_peak, 2),
            "note": "element kernels on the seeded perturbed state, L2 flushed before each call; implicit "
                    "steps consecutive from the corner deposit at dt = 2 x explicit estimate; plain FP64 "
                    "steps 20 at k = 1, 2 and 3 / 2 at k = 3 / 4 (seconds per step)"}
        out["config3_interface"] = run_interface(args)
        out["config1_taylor_green"] = tg_fp64_steps()
        out["extras_wall_s"] = round(time.perf_counter() - w0, 1)
    if not args.no_cpu_baseline:
        import numpy as np
        u_np, k_np = u_s.cpu().numpy(), k_s.cpu().numpy()
        rate, reps_c, t_c, _ = oracle_residual_rate(u_np, k_np, tau)
        out["cpu_baseline"] = {"value": round(rate, 6), "unit": "GDoF/s", "cores": 1, "kind": "oracle",
                               "sample": f"oracle residual on the full bench state ({W['name']}, n={n}), "
                                         f"{reps_c} evaluations, {t_c:.2f} s each, 1 thread",
                               "jvp_fd_value": round(rate / 2, 6),
                               "jvp_fd_note": "directional finite-difference J.w = two oracle residuals"}
        if not args.headline_only:
            ra, procs, cores, reps_a, t_a = oracle_all_cores(u_np, k_np, tau)
            out["cpu_baseline_all_cores"] = {
                "value": round(ra, 6), "unit": "GDoF/s", "cores": procs, "host_cores": cores, "kind": "oracle",
                "sample": f"{procs} single-threaded oracle processes, each evaluating the residual of the full "
                          f"bench state; {reps_a} evaluations in {t_a:.1f} s"}
    return out


def run_cpu_config5(args):
    """The oracle's residual (and its two-residual finite-difference J.w) on the 48^3 Q2-Q1
    seeded perturbed state, one thread: one evaluation after the set-up (about a minute of
    host time, hence not part of the default run)."""
    import numpy as np
    import lh_synth
    from oracle.fem import Mesh as OMesh
    from oracle.hydro import Hydro, Params
    from oracle import problems
    with one_thread():
        t0 = time.perf_counter()
        om = OMesh((48, 48, 48), (0.0,) * 3, (1.0,) * 3, 2)
        hyd = Hydro(om, Params(om, gamma=1.4, visc=True))
        u = problems.perturbed_state(hyd, lh_synth.perturbed_draws((48, 48, 48), 2, 102))
        k = np.zeros_like(u)
        t_setup = time.perf_counter() - t0
        t1 = time.perf_counter()
        hyd.residual(u, k, 1e-4)
        t = time.perf_counter() - t1
    n = om.n_unknowns
    return {"metric": "oracle residual at 48^3 Q2-Q1 (config 5, k = 2), one thread", "value": round(n / t / 1e9, 6),
            "unit": "GDoF/s", "seconds_per_residual": round(t, 2), "setup_s": round(t_setup, 1), "n_unknowns": n,
            "jvp_fd_value": round(n / (2 * t) / 1e9, 6), "cores": 1, "kind": "oracle"}


def tg_fp64_steps():
    """2D Taylor-Green vortex, plain FP64 (8x8 Q2-Q1, p0 = 100, no viscosity, energy source):
    10 implicit midpoint steps at dt = 0.01, Newton-GMRES relative tolerance 1e-10."""
    import torch
    from paper_2609_16424_b300.states import taylor_green_problem
    mesh, u = taylor_green_problem(8, 2, p0=100.0, device="cuda:0")
    k = torch.zeros_like(u)
    times, its, gm = [], 0, 0
    for _ in range(10):
        ms, st = _ms(lambda: mesh.newton_step(u, k, 0.01, jvp_prec="fp64", newton_rtol=1e-10, gmres_rtol=1e-12,
                                              gmres_maxit=400, restart=60))
        times.append(ms)
        its += st["newton_its"]
        gm += st["gmres_its_total"]
    return {"workload": "tg2d_8x8_q2q1 (p0 = 100), FP64, dt 0.01, 10 steps", "n_unknowns": mesh.n,
            "ms_per_step": round(sum(times) / 10, 3), "newton_its_per_step": its / 10, "gmres_its_per_step": gm / 10,
            "l1_velocity_error": mesh.tg_velocity_error(u)}


def sweep_state(mesh, n, k, seed):
    """Synthetic perturbed state on the GPU from the seeded draws (walls on all faces)."""
    import torch
    import lh_synth
    d = lh_synth.perturbed_draws(n, k, seed)
    nv, dim = mesh.NV, len(n)
    x0 = mesh.initial_nodes()
    ids = torch.arange(nv, device=mesh.device)
    interior = torch.ones(nv, dtype=torch.bool, device=mesh.device)
    fixed = []
    stride = 1
    for c in range(dim):
        ext = k * n[c] + 1
        coord = (ids // stride) % ext
        stride *= ext
        on = (coord == 0) | (coord == ext - 1)
        interior &= ~on
        fixed.append(on)
    u = torch.zeros(mesh.n, dtype=torch.float64, device=mesh.device)
    h = 1.0 / n[0]
    u[:dim * nv] = x0 + (0.1 * h / k) * (torch.tensor(d["xi"], device=mesh.device) * interior).reshape(-1)
    v = torch.tensor(d["v"], device=mesh.device)
    for c in range(dim):
        v[c][fixed[c]] = 0.0
    u[dim * nv:2 * dim * nv] = v.reshape(-1)
    u[2 * dim * nv:] = torch.tensor(d["e"], device=mesh.device)
    return u


def run_sweep(args):
    """48^3 throughput sweep over orders k = 1..4: operator GDoF/s and the roofline of each
    element kernel (CUDA events around the element kernels, L2 flushed before each call)."""
    import torch
    import paper_2609_16424_b300 as lh
    dev = "cuda:0"
    torch.cuda.set_device(0)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    fp64 = lh.probe_fma("fp64")
    fp32 = lh.probe_fma("fp32")
    rows = sweep_rows(args.orders, flush, fp64, fp32, dev)
    return {"metric": "48^3 throughput sweep (element kernels, FP64 residual / FP64 J.w / FP32 record J.w / "
                      "TF32 and BF16 tensor-core record J.w)",
            "fp64_peak_tflops": round(fp64, 3), "fp32_peak_tflops": round(fp32, 2), "rows": rows,
            "data": "synthetic perturbed state (seeded), L2 flushed before each call"}


def record_bytes(dim, k, ne):
    """Algorithmic DRAM bytes of one record J.w element launch: the record (read once), the
    float direction (each element's dofs, lattice-shared nodes counted once) and the float
    element output (written once)."""
    import ctypes as C
    import paper_2609_16424_b300 as lh
    nr = C.c_int()
    lh.lib.lh_record_len(dim, C.byref(nr))
    nq = (2 * k) ** dim
    return ne * (4 * nr.value * nq + 4 * (dim * (k + 1) ** dim + k ** dim))


def sweep_rows(orders, flush, fp64, fp32, dev):
    """Element-kernel times and roofline fractions on the 48^3 perturbed state, per order."""
    import torch
    import paper_2609_16424_b300 as lh
    rows = []
    n = (48, 48, 48)
    for k in orders:
        mesh = lh.Mesh(3, n, (0, 0, 0), (1, 1, 1), k, gamma=1.4, h_coarse=1.0 / 24, device=dev)
        u = sweep_state(mesh, n, k, 100 + k)
        kk = torch.zeros_like(u)
        dk = torch.randn(mesh.n, dtype=torch.float64, device=dev, generator=torch.Generator(dev).manual_seed(k))
        dkf = dk.float()
        tau = 1e-4
        r = torch.empty_like(u)
        od = torch.empty_like(u)
        of = torch.empty(mesh.n, dtype=torch.float32, device=dev)
        mesh.linearize(u, kk, tau)
        tc_ok = k <= 2
        for _ in range(2):   # warm-up
            mesh.residual(u, kk, tau, out=r)
            mesh.jvp(u, kk, tau, dk, out=od)
            mesh.jvp(u, kk, tau, dkf, out=of, lin=True)
            if tc_ok:
                mesh.jvp(u, kk, tau, dkf, out=of, tc="bf16")
        torch.cuda.synchronize()
        reps = 5
        res = {}
        ops = [("residual", "residual", lambda: mesh.residual(u, kk, tau, out=r)),
               ("jvp_fp64", "jvp_fp64", lambda: mesh.jvp(u, kk, tau, dk, out=od)),
               ("jvp_fp32", "jvp_fp32", lambda: mesh.jvp(u, kk, tau, dkf, out=of, lin=True))]
        if tc_ok:
            ops += [("jvp_tf32_tc", "jvp_tc", lambda: mesh.jvp(u, kk, tau, dkf, out=of, tc="tf32")),
                    ("jvp_bf16_tc", "jvp_tc", lambda: mesh.jvp(u, kk, tau, dkf, out=of, tc="bf16"))]
        for name, pk, fn in ops:
            mesh.profile(True)
            for _ in range(reps):
                flush.fill_(1.0)
                fn()
            p = mesh.profile_read()
            mesh.profile(False)
            ms, cnt = p[pk]
            res[name] = ms / cnt
        if tc_ok:
            mesh.tc_status()
        fl = {kind: flops_per_element(3, k, kind) for kind in ("residual", "jvp", "jvp_rec")}
        ne = mesh.NE
        row = {"order": f"Q{k}-Q{k - 1}", "n_unknowns": mesh.n, "quad_points": mesh.NQ}
        for name, flk, peak, pipe in (("residual", "residual", fp64, "fp64"), ("jvp_fp64", "jvp", fp64, "fp64"),
                                      ("jvp_fp32", "jvp_rec", fp32, "fp32"), ("jvp_tf32_tc", "jvp_rec", fp32, "fp32"),
                                      ("jvp_bf16_tc", "jvp_rec", fp32, "fp32")):
            if name not in res:
                row[name] = "not supported at this order (dense element operator exceeds shared memory)"
                continue
            t = res[name]
            tf = fl[flk] * ne / (t * 1e-3) / 1e12
            row[name] = {"elem_kernel_ms": round(t, 4), "gdofs": round(mesh.n / (t * 1e-3) / 1e9, 3),
                         "tflops": round(tf, 3), "frac": round(tf / peak, 4), "pipe": pipe,
                         "flops_per_element": fl[flk]}
            if flk == "jvp_rec":
                by = record_bytes(3, k, ne)
                row[name]["hbm_gbs"] = round(by / (t * 1e-3) / 1e9, 1)
                row[name]["hbm_frac"] = round(by / (t * 1e-3) / 1e9 / HBM_PEAK_GBS, 4)
                row[name]["algorithmic_bytes"] = by
        rows.append(row)
        del mesh, u, kk, dk, dkf, r, od, of
        torch.cuda.empty_cache()
    return rows


def config5_steps(orders, fp64_steps, steps, flush, dev):
    """Implicit midpoint steps on the 48^3 point blast (Q_k-Q_{k-1}, gamma 1.4, smooth
    viscosity with h_coarse = 1/24, walls), consecutive from the corner deposit after one
    developing step, dt = 2 x the explicit estimate recomputed before each step (outside the
    timed region); per step CUDA-event time of the whole Newton-GMRES solve."""
    import torch
    import paper_2609_16424_b300 as lh
    from paper_2609_16424_b300.states import blast_state
    out = []
    n = (48, 48, 48)
    for k in orders:
        row = {"order": f"Q{k}-Q{k - 1}"}
        for prec, nsteps in (("fp32", steps), ("fp64", fp64_steps.get(k, 0))):
            if nsteps <= 0:
                continue
            mesh = lh.Mesh(3, n, (0, 0, 0), (1, 1, 1), k, gamma=1.4, h_coarse=1.0 / 24, device=dev)
            u = blast_state(mesh, 0.25)
            kk = torch.zeros_like(u)
            mesh.newton_step(u, kk, 2.0 * mesh.dt_estimate(u), jvp_prec=prec, **NEWTON)
            times, its, gm, ev = [], 0, 0, 0
            for _ in range(nsteps):
                dt = 2.0 * mesh.dt_estimate(u)
                flush.fill_(1.0)
                ms, st = _ms(lambda: mesh.newton_step(u, kk, dt, jvp_prec=prec, **NEWTON))
                times.append(ms)
                its += st["newton_its"]
                gm += st["gmres_its_total"]
                ev += st["residual_evals"] + st["jvp_evals"]
            row["n_unknowns"] = mesh.n
            row[prec] = {"steps": nsteps, "ms_per_step": round(sum(times) / nsteps, 3),
                         "newton_its_per_step": round(its / nsteps, 3), "gmres_its_per_step": round(gm / nsteps, 3),
                         "gdofs": round(mesh.n * ev / (sum(times) * 1e-3) / 1e9, 4)}
            del mesh, u, kk
            torch.cuda.empty_cache()
        if "fp32" in row and "fp64" in row:
            row["fp64_over_fp32"] = round(row["fp64"]["ms_per_step"] / row["fp32"]["ms_per_step"], 3)
        out.append(row)
    return out


def _ms(fn):
    import torch
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    out = fn()
    e1.record(s)
    e1.synchronize()
    return e0.elapsed_time(e1), out


def _mlp_family(make, nrun, ntrain, steps, dim, k, cfl, epochs, tols):
    """Train the learned proposal on seeded runs of a problem family, evaluate it on the
    held-out runs against plain extrapolation: per step, CUDA-event time of the whole
    Newton-GMRES solve (the proposal's features, forward pass and nodal averaging included),
    Newton and GMRES iterations, to one absolute tolerance tol x ||R(k^{n-1})|| for both."""
    import numpy as np
    import torch
    from paper_2609_16424_b300 import mlp
    import paper_2609_16424_b300 as lh
    t0 = time.perf_counter()
    runs, dropped = [], 0
    for i in range(nrun):
        m, u0 = make(i)
        try:
            runs.append((m, u0, mlp.trajectory(m, u0, steps, cfl=cfl, jvp_prec="fp32", **NEWTON)))
        except lh.LHError:   # a seed whose run fails at this step size is left out
            dropped += 1
    t_gen = time.perf_counter() - t0
    ntrain = min(ntrain, len(runs) - 1)
    m0 = runs[0][0]
    train = [tr for _, _, tr in runs[:ntrain]]
    fscale = torch.zeros(4, dtype=torch.float32, device="cuda")
    fscale[:3] = mlp.group_rms(m0, [k2 for tr in train for _, k2 in tr]).float()
    fscale[3] = float(np.mean([dt for tr in train for dt, _ in tr]))
    tscale = torch.ones(4, dtype=torch.float32, device="cuda")
    tscale[:3] = mlp.group_rms(m0, [tr[i][1] - tr[i - 1][1] for tr in train for i in range(1, len(tr))]).float()
    X, T = mlp.dataset(m0, train, fscale, tscale)
    n_in, n_out = mlp.feature_sizes(dim, k)
    net = mlp.MLP(n_in, 128, 3, n_out, seed=1)
    t0 = time.perf_counter()
    hist = mlp.train(net, X, T, epochs=epochs, batch=4096 if X.shape[0] >= 65536 else 1024)
    t_train = time.perf_counter() - t0
    out = {"training": {"runs": ntrain, "step_pairs": sum(len(tr) - 2 for tr in train), "element_samples":
                        int(X.shape[0]), "epochs": epochs, "loss_first": round(hist[0], 5),
                        "loss_last": round(hist[-1], 6), "train_s": round(t_train, 2), "datagen_s": round(t_gen, 2)},
           "heldout_runs": len(runs) - ntrain, "runs_dropped": dropped}
    opts = dict(NEWTON, newton_rtol=1e-30, jvp_prec="fp32")
    for tol in tols:
        rows = []
        for m, u0, tr in runs[ntrain:]:
            u = u0.clone()
            for i, (dt, kn) in enumerate(tr):
                tau = 0.5 * dt
                if i >= 2:
                    k1, k2 = tr[i - 1][1], tr[i - 2][1]
                    r1 = float(m.residual(u, k1, tau).norm())
                    atol = tol * r1
                    t_ex, st_ex = _ms(lambda: m.newton_step(u.clone(), k1.clone(), dt, newton_atol=atol, **opts))

                    def with_mlp():
                        k0 = mlp.apply(m, u, tau, k1, net.forward(mlp.features(m, k1, k2, dt, fscale)), tscale)
                        return k0, m.newton_step(u.clone(), k0, dt, newton_atol=atol, **opts)
                    t_ml, (k0, st_ml) = _ms(with_mlp)
                    rows.append([t_ex, st_ex["newton_its"], st_ex["gmres_its_total"], t_ml, st_ml["newton_its"],
                                 st_ml["gmres_its_total"], st_ml["r0"] / st_ex["r0"]])
                u = u + dt * kn
        a = np.array(rows).mean(axis=0)
        out[f"tol_{tol:g}"] = {
            "extrapolation": {"ms_per_step": round(a[0], 3), "newton_its": round(a[1], 3), "gmres_its": round(a[2], 2)},
            "learned": {"ms_per_step": round(a[3], 3), "newton_its": round(a[4], 3), "gmres_its": round(a[5], 2),
                        "initial_residual_ratio": round(a[6], 4)},
            "step_time_ratio": round(a[3] / a[0], 4), "heldout_steps": len(rows)}
    return out


def run_mlp(args):
    """Learned initial guess vs plain extrapolation on the two workload families of the
    proposal: the 2D Taylor-Green vortex on a 16 x 16 Q2-Q1 mesh (seeded velocity amplitude in
    [0.5, 1.5], pressure level p0 in [1, 10], FS-CFL 8) and the 3D point blast on 24^3 Q2-Q1
    (seeded gamma in [1.3, 1.7], deposit in [0.1, 0.5], FS-CFL 2); evaluated at the paper's
    Newton tolerance 1e-5 and at 1e-8 (relative to the fallback's initial residual)."""
    import numpy as np
    import torch
    import paper_2609_16424_b300 as lh
    from paper_2609_16424_b300.states import blast_state, taylor_green_problem
    torch.cuda.set_device(0)
    rng = np.random.default_rng(1)
    tgp = [(rng.uniform(0.5, 1.5), rng.uniform(1.0, 10.0)) for _ in range(args.mlp_tg_runs)]

    def tg(i):
        m, u = taylor_green_problem(16, 2, p0=tgp[i][1], device="cuda:0")
        u[2 * m.NV:4 * m.NV] *= tgp[i][0]
        return m, u
    rng = np.random.default_rng(0)
    bp = [(rng.uniform(1.3, 1.7), rng.uniform(0.1, 0.5)) for _ in range(6)]
    W = WORKLOAD

    def blast(i):
        m = lh.Mesh(3, W["n"], (0,) * 3, (1,) * 3, W["k"], gamma=bp[i][0], device="cuda:0")
        return m, blast_state(m, bp[i][1])
    ntg = args.mlp_tg_runs
    return {"metric": "implicit step with learned initial guess vs plain extrapolation (FP32 J.w)",
            "taylor_green_16x16_q2q1": _mlp_family(tg, ntg, ntg - min(40, max(4, ntg // 5)), 26, 2, 2, 8.0,
                                                   args.mlp_epochs, (1e-5, 1e-8)),
            "blast3d_24_q2q1": _mlp_family(blast, 6, 5, args.mlp_steps, 3, 2, W["cfl"], args.mlp_epochs,
                                           (1e-5, 1e-8)),
            "data": "synthetic seeded runs of each family; held-out runs for evaluation"}


def run_blast(args):
    """The 3D point blast (24^3 Q2-Q1, gamma 1.4, smooth viscosity, walls) from the corner
    deposit to t = t_end with the paper's implicit time step control (first step at FS-CFL 2
    of the explicit estimate, then driven by the Newton iteration count), Newton rtol 1e-5."""
    import torch
    import paper_2609_16424_b300 as lh
    from paper_2609_16424_b300.states import blast_state
    torch.cuda.set_device(0)
    W = WORKLOAD
    m = lh.Mesh(3, W["n"], (0,) * 3, (1,) * 3, W["k"], gamma=W["gamma"], device="cuda:0")
    u = blast_state(m, W["energy"])
    ke0, ie0 = m.energies(u)
    opts = dict(NEWTON, newton_rtol=1e-5)
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    steps, rejected, hist = m.advance(u, args.t_end, fs_cfl=W["cfl"], jvp_prec=args.prec, **opts)
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    ke, ie = m.energies(u)
    acc = [h for h in hist if h[3]]
    its = [h[2] for h in acc]
    return {"metric": "3D point blast 24^3 Q2-Q1 to t_end (implicit midpoint, FS-CFL 2 + Newton-count dt control)",
            "t_end": args.t_end, "steps": steps, "rejected": rejected, "wall_s": round(wall, 3),
            "ms_per_step": round(wall / max(steps, 1) * 1e3, 3), "newton_its_per_step": round(sum(its) / len(its), 3),
            "dt_first": acc[0][1], "dt_last": acc[-1][1], "jvp_prec": args.prec, "newton_rtol": 1e-5,
            "total_energy_start": ke0 + ie0, "total_energy_end": ke + ie,
            "relative_energy_drift": (ke + ie - ke0 - ie0) / (ke0 + ie0), "kinetic_end": ke}


def run_interface(args):
    """Three-state interface problem 56x24 Q3-Q2: 50 implicit midpoint steps at 10x the
    explicit time-step estimate, FP32 and TF32 J.w (the paper's Newton rtol 1e-5)."""
    import torch
    import paper_2609_16424_b300 as lh
    from paper_2609_16424_b300.states import interface_problem
    torch.cuda.set_device(0)
    out = {"metric": "three-state interface 56x24 Q3-Q2, 50 implicit steps at 10x explicit dt", "runs": {}}
    for prec in ("fp32", "tf32"):
        mesh, u = interface_problem(56, 24, 3, device="cuda:0")
        k = torch.zeros_like(u)
        ke0, ie0 = mesh.energies(u)
        times, its, gm, t = [], 0, 0, 0.0
        status = "ok"
        for step in range(50):
            dt = 10.0 * mesh.dt_estimate(u)
            try:
                ms, st = _ms(lambda: mesh.newton_step(u, k, dt, jvp_prec=prec, **NEWTON))
            except lh.LHError as err:
                status = f"step {step} failed: {err}"
                break
            times.append(ms)
            its += st["newton_its"]
            gm += st["gmres_its_total"]
            t += dt
        nsteps = max(1, len(times))
        ke1, ie1 = mesh.energies(u)
        out["runs"][prec] = {"status": status, "steps": len(times), "t_end": t,
                             "ms_per_step": round(statistics.mean(times), 3) if times else None,
                             "newton_its_per_step": its / nsteps, "gmres_its_per_step": gm / nsteps,
                             "relative_energy_drift": (ke1 + ie1 - ke0 - ie0) / (ke0 + ie0),
                             "n_unknowns": mesh.n}
    return out


# The paper's Taylor-Green table (Sec. 4.1, implicit columns; one MPI task on a laptop with
# an assembled Jacobian and a sparse direct solver): (k, FS-CFL, 1/h) -> (L1 error, steps, s).
# Its rows h = 1/16 .. 1/256 are the meshes of n = 1/(4 h) = 4 .. 64 elements per side: there
# the runs of this library take the printed step counts and reach the printed errors.
PAPER_TG_ELEMS = 4
PAPER_TG = {
    (2, 0.5, 16): (5.11e-02, 13, 0.2), (2, 2.0, 16): (5.75e-02, 4, 0.1), (2, 8.0, 16): (1.54e-01, 1, 0.1),
    (2, 0.5, 32): (9.42e-03, 26, 0.3), (2, 2.0, 32): (1.20e-02, 7, 0.2), (2, 8.0, 32): (1.05e-01, 2, 0.1),
    (2, 0.5, 64): (2.57e-03, 51, 1.4), (2, 2.0, 64): (3.55e-03, 12, 0.6), (2, 8.0, 64): (4.30e-02, 4, 0.4),
    (2, 0.5, 128): (6.66e-04, 102, 12), (2, 2.0, 128): (9.35e-04, 26, 3.6), (2, 8.0, 128): (9.46e-03, 7, 2.1),
    (2, 0.5, 256): (1.64e-04, 203, 126), (2, 2.0, 256): (2.35e-04, 51, 34), (2, 8.0, 256): (2.45e-03, 13, 16),
    (3, 0.5, 16): (1.24e-02, 20, 0.3), (3, 2.0, 16): (1.20e-02, 5, 0.2), (3, 8.0, 16): (2.09e-01, 2, 0.1),
    (3, 0.5, 32): (1.57e-03, 38, 1.3), (3, 2.0, 32): (1.64e-03, 10, 0.5), (3, 8.0, 32): (1.94e-02, 3, 0.3),
    (3, 0.5, 64): (1.80e-04, 76, 11), (3, 2.0, 64): (2.08e-04, 19, 3), (3, 8.0, 64): (3.39e-03, 5, 1.6),
    (3, 0.5, 128): (2.02e-05, 152, 106), (3, 2.0, 128): (2.42e-05, 38, 26), (3, 8.0, 128): (5.52e-04, 10, 7.7),
    (3, 0.5, 256): (2.32e-06, 304, 1150), (3, 2.0, 256): (3.66e-06, 76, 288), (3, 8.0, 256): (7.54e-05, 19, 71),
    (4, 0.5, 16): (5.25e-03, 26, 0.7), (4, 2.0, 16): (7.77e-03, 7, 0.4), (4, 8.0, 16): (7.62e+01, 2, 0.2),
    (4, 0.5, 32): (4.50e-04, 51, 4.3), (4, 2.0, 32): (9.63e-04, 13, 1.4), (4, 8.0, 32): (2.29e+02, 4, 1),
    (4, 0.5, 64): (1.49e-05, 102, 37), (4, 2.0, 64): (6.08e-05, 26, 9.5), (4, 8.0, 64): (5.45e-03, 7, 5.1),
    (4, 0.5, 128): (1.44e-06, 203, 360), (4, 2.0, 128): (4.34e-06, 51, 87), (4, 8.0, 128): (6.86e-04, 13, 28),
    (4, 0.5, 256): (8.36e-08, 405, 3613), (4, 2.0, 256): (2.66e-07, 102, 906), (4, 8.0, 256): (5.50e-05, 26, 242),
}


# The paper's explicit columns (ORIG-E, CFL 0.5, RK2-average / RK3 / RK4 for Q2 / Q3 / Q4):
# (k, 1/h) -> (L1 error, steps, s)
PAPER_TG_EXPLICIT = {
    (2, 16): (5.22e-02, 35, 0.1), (2, 32): (9.47e-03, 68, 0.3), (2, 64): (2.55e-03, 135, 1.3),
    (2, 128): (6.60e-04, 268, 8), (2, 256): (1.65e-04, 535, 57),
    (3, 16): (1.24e-02, 51, 0.2), (3, 32): (1.57e-03, 101, 0.6), (3, 64): (1.80e-04, 202, 3.8),
    (3, 128): (2.02e-05, 402, 26), (3, 256): (2.32e-06, 802, 200),
    (4, 16): (5.16e-03, 68, 0.3), (4, 32): (4.50e-04, 135, 1.5), (4, 64): (1.50e-05, 268, 10),
    (4, 128): (1.44e-06, 535, 76), (4, 256): (8.36e-08, 1069, 578),
}


# Taylor-Green runs: the paper solves each Newton system exactly (sparse direct solver), so
# one Newton iteration can meet the 1e-5 tolerance and let the controller grow dt; GMRES to
# 1e-6 keeps that possible (at 1e-4 every stage takes at least two iterations).
TG_NEWTON = dict(NEWTON, gmres_rtol=1e-6)


def run_tg_table(args):
    """2D Taylor-Green (p0 = 1) to t = 0.5 (Sec. 4.1): Q2-Q1 + SD2, Q3-Q2 + SD3, Q4-Q3 + SD4
    on h = 1/16 .. 1/256 at the given FS-CFL values, with the Newton-count time step control;
    L1 velocity error, its rate, accepted steps and wall time of each run.  Each run is also
    written to stderr when it ends."""
    import torch
    import paper_2609_16424_b300 as lh
    from paper_2609_16424_b300.states import taylor_green_problem
    torch.cuda.set_device(0)
    rows, t_start = [], time.perf_counter()
    for cfl in args.tg_cfl:
        for k in args.tg_orders:
            prev = None
            for inv_h in args.tg_h:
                if time.perf_counter() - t_start > args.tg_budget:
                    rows.append({"k": k, "fs_cfl": cfl, "inv_h": inv_h, "status": "skipped (time budget)"})
                    continue
                mesh, u = taylor_green_problem(inv_h, k, p0=1.0, device="cuda:0")
                torch.cuda.synchronize()
                w0 = time.perf_counter()
                steps, rejected, hist = mesh.advance(u, 0.5, fs_cfl=cfl, scheme=k, max_attempts=args.tg_attempts,
                                                     grow=not args.tg_fixed_dt, jvp_prec=args.prec,
                                                     **dict(TG_NEWTON, newton_rtol=args.tg_newton_rtol,
                                                            scaled_norm=int(args.tg_scaled_norm)))
                done = sum(h[1] for h in hist if h[3]) >= 0.5 - 1e-12
                torch.cuda.synchronize()
                wall = time.perf_counter() - w0
                err = mesh.tg_velocity_error(u)
                its = [h[2] for h in hist if h[3]]
                paper = PAPER_TG.get((k, cfl, PAPER_TG_ELEMS * inv_h))
                rows.append({"k": k, "scheme": f"SD{k}", "fs_cfl": cfl, "inv_h": inv_h, "n_unknowns": mesh.n,
                             "dt_first": hist[0][1] if hist else None,
                             "status": "ok" if done else f"stopped after {len(hist)} attempts",
                             "l1_error": err, "rate": (math.log2(prev / err) if prev else None), "steps": steps,
                             "rejected": rejected, "newton_its_max_mean": round(sum(its) / max(len(its), 1), 3),
                             "wall_s": round(wall, 3),
                             "paper": ({"l1_error": paper[0], "steps": paper[1], "time_s": paper[2]}
                                       if paper else None)})
                print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
                prev = err if done else None
                del mesh, u
    return {"metric": "2D Taylor-Green (p0 = 1) to t = 0.5, implicit SDIRK + Newton-count dt control",
            "dt_growth": not args.tg_fixed_dt, "jvp_prec": args.prec,
            "newton": dict(TG_NEWTON, newton_rtol=args.tg_newton_rtol, scaled_norm=int(args.tg_scaled_norm)),
            "runs": rows}


def run_accuracy_per_time(args):
    """Accuracy per unit run time on the 2D Taylor-Green vortex (p0 = 1, t = 0.5; the paper's
    Sec. 4.1 table): explicit RK2-average / SSP RK3 / RK4 at CFL args.xcfl of the explicit
    estimate (with the explicit step control) against the implicit SD2 / SD3 / SD4 at FS-CFL
    args.icfl with the Newton-count control, for Q2-Q1 / Q3-Q2 / Q4-Q3 on h = 1/16 .. 1/128.
    No viscosity (the paper sets it to zero for this problem).  L1 velocity error, steps and
    wall time of each run; both paths run on the GPU."""
    import torch
    from paper_2609_16424_b300.states import taylor_green_problem
    torch.cuda.set_device(0)
    rows, t_start = [], time.perf_counter()
    for k in args.tg_orders:
        for inv_h in args.tg_h:
            for path in ("explicit", "implicit"):
                if time.perf_counter() - t_start > args.tg_budget:
                    rows.append({"k": k, "inv_h": inv_h, "path": path, "status": "skipped (time budget)"})
                    continue
                mesh, u = taylor_green_problem(inv_h, k, p0=1.0, device="cuda:0")
                torch.cuda.synchronize()
                w0 = time.perf_counter()
                if path == "explicit":
                    st = mesh.explicit_advance(u, 0.5, cfl=args.xcfl, scheme=k, visc_model="imp")
                    steps, rejected = st["steps"], st["rejected"]
                else:
                    steps, rejected, _ = mesh.advance(u, 0.5, fs_cfl=args.icfl, scheme=k, jvp_prec=args.prec,
                                                      **dict(TG_NEWTON, newton_rtol=args.tg_newton_rtol))
                torch.cuda.synchronize()
                wall = time.perf_counter() - w0
                rows.append({"k": k, "inv_h": inv_h, "path": path,
                             "scheme": (f"RK{k}" if path == "explicit" else f"SD{k}"), "n_unknowns": mesh.n,
                             "l1_error": mesh.tg_velocity_error(u), "steps": steps, "rejected": rejected,
                             "wall_s": round(wall, 4),
                             "paper": (PAPER_TG.get((k, args.icfl, PAPER_TG_ELEMS * inv_h)) if path == "implicit"
                                       else PAPER_TG_EXPLICIT.get((k, PAPER_TG_ELEMS * inv_h)))})
                print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
                del mesh, u
    return {"metric": "Taylor-Green L1 error vs wall time, explicit RK vs implicit SDIRK (GPU)",
            "explicit_cfl": args.xcfl, "implicit_fs_cfl": args.icfl, "jvp_prec": args.prec,
            "newton": dict(TG_NEWTON, newton_rtol=args.tg_newton_rtol), "runs": rows}


def run_precond_compare(args):
    """Velocity-block preconditioners of the Newton-GMRES step (FP32 J.w, Newton rtol 1e-5,
    GMRES 1e-4): the exact mass inverse (kron, the benchmark's), the Jacobi of M_V alone
    (jacobi) and the Jacobi of the paper's block M_V + tau dF/dv (jvv_diag, Eq. (23)); median
    of 5 steps from the same state, on the point blast at the benchmark dt and at 4x it and
    on a Taylor-Green Q3 state at FS-CFL 8."""
    import torch
    import paper_2609_16424_b300 as lh
    from paper_2609_16424_b300.states import blast_state, taylor_green_problem
    torch.cuda.set_device(0)
    rows = []

    def probe(name, m, u, dt, kk, reps=5):
        for pc, extra in (("kron", {}), ("jvv_diag", {}), ("jacobi", {}), ("cheb", {"cheb_degree": 2}),
                          ("cheb", {"cheb_degree": 3}), ("cheb", {"cheb_degree": 5})):
            ts, st = [], None
            for _ in range(reps):
                ug, kg = u.clone(), kk.clone()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st = m.newton_step(ug, kg, dt, jvp_prec="fp32", precond=pc, **extra, **NEWTON)
                torch.cuda.synchronize()
                ts.append((time.perf_counter() - t0) * 1e3)
            rows.append({"case": name, "precond": pc + (f"{extra['cheb_degree']}" if extra else ""),
                         "ms": round(statistics.median(ts), 3), "newton": st["newton_its"],
                         "gmres": st["gmres_its_total"], "jvp_evals": st["jvp_evals"]})

    W = WORKLOAD
    m = lh.Mesh(3, W["n"], (0,) * 3, (1,) * 3, W["k"], gamma=W["gamma"], device="cuda:0")
    u = blast_state(m, W["energy"])
    kk = torch.zeros_like(u)
    dt = W["cfl"] * m.dt_estimate(u)
    for _ in range(W["develop_steps"]):
        m.newton_step(u, kk, dt, jvp_prec="fp32", **NEWTON)
    probe("blast3d 24^3 Q2-Q1, benchmark dt", m, u, dt, kk)
    probe("blast3d 24^3 Q2-Q1, 4x the benchmark dt", m, u, 4 * dt, kk)
    m2, u2 = taylor_green_problem(64, 3, device="cuda:0")
    k2 = torch.zeros_like(u2)
    dt2 = 8.0 * m2.dt_estimate(u2)
    m2.sdirk_step(u2, k2, dt2, scheme=3, jvp_prec="fp32", **NEWTON)
    probe("Taylor-Green 64^2 Q3-Q2, FS-CFL 8 (implicit midpoint step)", m2, u2, dt2, k2)
    return {"metric": "implicit step time by velocity-block preconditioner", "newton": NEWTON, "runs": rows}


def run_reference(args, rank):
    """The oracle (plain FP64 numpy, one thread) timed on this host: each step is one
    residual evaluation of the bench workload state."""
    if rank != 0:
        return None
    import numpy as np
    from oracle import problems  # noqa: F401
    from oracle.fem import Mesh as OMesh
    from oracle.hydro import Hydro, Params
    from oracle import solver
    W = WORKLOAD
    with one_thread():
        om = OMesh(W["n"], (0.0,) * 3, (1.0,) * 3, W["k"])
        hyd = Hydro(om, Params(om, gamma=W["gamma"], visc=True))
        # the same state construction as the GPU arm: deposit, then no developed steps
        # (the oracle cannot afford Newton steps at this size); dt-independent residual
        x0 = hyd.x0
        e = np.zeros((om.NE, om.NL))
        e[0, :] = W["energy"] * om.NE
        u = om.join(x0, np.zeros_like(x0), e)
        kk = np.zeros(om.n_unknowns)
        tau = 1e-3
        for _ in range(args.warmup):
            hyd.residual(u, kk, tau)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            hyd.residual(u, kk, tau)
        t = time.perf_counter() - t0
    value = om.n_unknowns * args.steps / t / 1e9
    return {"impl": "reference", "metric": "GDoF/s of J.w & residual over the implicit step (FP64 residual, FP32 J.w)",
            "value": round(value, 6), "unit": "GDoF/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(t / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (corner point blast)",
            "config": {"workload": W["name"], "n_unknowns": om.n_unknowns},
            "cpu_baseline": {"value": round(value, 6), "unit": "GDoF/s", "cores": 1, "kind": "oracle",
                             "sample": f"one oracle residual evaluation of the full {W['name']} state per step"},
            "e2e": {"value": round(value, 6), "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64", "tf32", "bf16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="timed steps only (profiling runs)")
    ap.add_argument("--headline-only", action="store_true",
                    help="skip the 48^3, interface and Taylor-Green extras and the all-cores oracle")
    ap.add_argument("--sweep", action="store_true", help="48^3 order sweep of the element kernels")
    ap.add_argument("--cpu-config5", action="store_true", help="the oracle residual at 48^3 Q2-Q1, one thread")
    ap.add_argument("--orders", type=int, nargs="+", default=[1, 2, 3, 4])
    ap.add_argument("--mlp", action="store_true", help="learned initial guess vs extrapolation")
    ap.add_argument("--mlp-steps", type=int, default=14)
    ap.add_argument("--mlp-epochs", type=int, default=30)
    ap.add_argument("--mlp-tg-runs", type=int, default=200,
                    help="seeded Taylor-Green runs (20%% held out, at most 40)")
    ap.add_argument("--blast-run", action="store_true", help="point blast to --t-end")
    ap.add_argument("--interface-run", action="store_true",
                    help="three-state interface problem, 50 steps at 10x explicit dt")
    ap.add_argument("--t-end", type=float, default=0.1)
    ap.add_argument("--precond-compare", action="store_true", help="velocity-block preconditioners")
    ap.add_argument("--accuracy-per-time", action="store_true",
                    help="Taylor-Green: explicit RK vs implicit SDIRK, error and wall time")
    ap.add_argument("--xcfl", type=float, default=0.5, help="explicit CFL (of the explicit estimate)")
    ap.add_argument("--icfl", type=float, default=2.0, help="implicit FS-CFL (of the explicit estimate)")
    ap.add_argument("--tg-table", action="store_true", help="Taylor-Green convergence table, SD2/SD3/SD4")
    ap.add_argument("--tg-orders", type=int, nargs="+", default=[2, 3, 4])
    ap.add_argument("--tg-cfl", type=float, nargs="+", default=[8.0, 2.0])
    ap.add_argument("--tg-h", type=int, nargs="+", default=[4, 8, 16, 32, 64],
                    help="elements per side (the paper's h = 1 / (4 n))")
    ap.add_argument("--tg-budget", type=float, default=240.0, help="seconds; later runs are skipped")
    ap.add_argument("--tg-attempts", type=int, default=600, help="step attempts per run at most")
    ap.add_argument("--tg-fixed-dt", action="store_true", help="never enlarge dt (rejections still shrink it)")
    ap.add_argument("--tg-newton-rtol", type=float, default=NEWTON["newton_rtol"])
    ap.add_argument("--tg-scaled-norm", action="store_true", help="row-weighted Newton/GMRES norm")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.cpu_config5:
        out = run_cpu_config5(args)
    elif args.sweep:
        out = run_sweep(args)
    elif args.mlp:
        out = run_mlp(args)
    elif args.interface_run:
        out = run_interface(args)
    elif args.blast_run:
        out = run_blast(args)
    elif args.tg_table:
        out = run_tg_table(args)
    elif args.precond_compare:
        out = run_precond_compare(args)
    elif args.accuracy_per_time:
        out = run_accuracy_per_time(args)
    elif args.impl == "reference":
        out = run_reference(args, rank)
    else:
        import torch
        if world > 1:
            torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
        out = run_ours(args, rank, world, f"cuda:{local}")
        if world > 1:
            torch.distributed.destroy_process_group()
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
