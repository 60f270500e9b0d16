#!/usr/bin/env python3
"""Benchmark: filtered-AIM Calderon TE-EFIE solves on GB300.

One step is one pass of the whole method for one scatterer: setup of every operator from the
contour (quadrature, grid, projections, kernel spectrum and its circular truncation, near
field, Gram inverse), the plane-wave excitation, and the GMRES solve of the filtered
Calderon system G^-1 S^alpha G^-1 N j = G^-1 S^alpha G^-1 E to a relative residual of 1e-5.
Workload: a seeded random smooth contour of perimeter 1000 wavelengths, 10 segments per
wavelength (N = 10000), a 2048 x 2048 grid (P = 4096), 4 x 4 stencils, alpha = 2k, one
right-hand side, FP64 grid arithmetic (double-float). Inputs are synthetic (no dataset exists
for this workload).

The default line also carries the other parts of the metric as sub-results, each timed on its
own: the same contour in mixed precision (complex64 grid, FP64 refinement to 1e-5), 64 plane
waves in every launch on the perimeter-400 contour, and a served Poisson stream with p50/p99
latency. The headline timed region runs the product path as shipped (no per-kernel events);
the per-kernel table and the roofline come from one more step run under kernel timing.

Under torchrun each rank solves its own contour (seed = rank): weak scaling, no collective in
the data path; value = all ranks' solves / max-over-ranks time.

--impl reference runs the CPU oracle (numpy/scipy FP64) on a bounded sample of the same
workload on the host cores, rank 0 only. --profile-case runs one operator of the single-solve
workload for kernel profilers.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "filtered AIM matvec HBM GB/s & solves/s at rel err<=1e-5; served p50/p99 latency"
UNIT = "solves/s"
SOLVE_TOL = 1e-5
RESTART = 3000
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
# FP32 pipe of GB300, the pipe double-float arithmetic runs on: 152 SMs x 128 FP32 lanes x 2 flop
# (FMA) x 2.07 GHz (the maximum SM clock) = 80.5 TFLOP/s; derived from unit counts and clocks
FP32_PIPE_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# FP64 pipe: 152 SMs x 2 FP64 FMA units x 2 flop x 2.07 GHz (nominal, derived)
FP64_PIPE_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
E2E_STEPS_MAX = 5

# DRAM traffic of k_col_conv per launch (dram__bytes_read.sum + dram__bytes_write.sum), the mean of
# the two launches of one filtered Calderon product (N: 3 channels, S^alpha: 1 channel), from one
# ncu capture of the current kernel and default schedule at the single-solve size; the capture and
# its command are in profiles/col_conv_*_single_solve_n10000.md. None where no capture of the
# current kernel exists.
COL_CONV_TRAFFIC = {"fp64": 533945856, "mixed": 201229440, "native": None}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--precision", choices=["fp64", "mixed", "native"], default="fp64",
                    help="fp64: FP64-accurate double-float grid arithmetic; mixed: complex64 grid with FP64 "
                         "refinement; native: IEEE binary64 grid arithmetic")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sub", action="store_true", help="skip the mixed / batching / serving sub-results")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--workload", choices=["single", "batching", "serving", "multi"], default="single",
                    help="single: one filtered Calderon solve per step (the default line, with sub-results); "
                         "batching / serving: that sub-result alone as its own line")
    ap.add_argument("--requests", type=int, default=40, help="serving: timed requests (after 10%% warm-up)")
    ap.add_argument("--policy", choices=["sjf", "fifo"], default="sjf", help="serving: admission order")
    ap.add_argument("--nrhs", type=int, default=64, help="batching: right-hand sides per solve (angles 2 pi r/nrhs)")
    ap.add_argument("--profile-case", action="store_true",
                    help="apply --op to a seeded vector of the single-solve workload --repeat times (for ncu)")
    ap.add_argument("--op", default="N", help="profile case: operator")
    ap.add_argument("--repeat", type=int, default=1, help="profile case: products")
    ap.add_argument("--time", action="store_true", help="profile case: print mean ms per launch of each kernel")
    ap.add_argument("--dft-stage", action="store_true",
                    help="time one radix-16 DFT pass on CUDA cores and on tensor cores (aim_dft_stage)")
    ap.add_argument("--stage-groups", type=int, default=152 * 32, help="dft stage: CTAs of 4096 complex64 values")
    ap.add_argument("--stage-passes", type=int, default=256, help="dft stage: passes per launch")
    ap.add_argument("--stage-variant", type=int, default=-1, help="dft stage: time only this variant (0, 1, 2)")
    return ap.parse_args()


def workload(seed):
    return synth.single_solve_scale(seed=seed)


def workload_config(wl, precision, world):
    return {"workload": "filtered Calderon TE-EFIE solve, perimeter 1000 wl, N=%d, grid %dx%d (P=%d), s=4, p=4, "
                        "alpha=2k, 1 rhs, GMRES(%d) rel. residual %.0e" % (wl.n, wl.m, wl.m, wl.fft_P, RESTART, SOLVE_TOL),
            "N": wl.n, "grid_m": wl.m, "fft_P": wl.fft_P, "alpha_over_k": wl.alpha / wl.k, "nrhs": 1,
            "precision": precision, "contour_seed": "rank", "ranks": world,
            "l2": "inputs larger than L2 (grid intermediate 3 x 1653 x 4096 complex per product > 129 MB)"}


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured (MEASURED_PEAKS.json)"
    except Exception:
        return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
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
        sms, maxs, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sms.append(float(parts[1]))
                    maxs.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sms:
            return None
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": max(maxs), "reasons": sorted(reasons),
                "samples": len(sms)}


# --------------------------------------------------------------------------------------
# roofline model of the dominant kernel (the column pass)
# --------------------------------------------------------------------------------------
def live_columns(wl, info, filtered):
    """Columns of the P x P spectrum the column pass transforms, and the stored half-columns
    (q' = 0..P/2) it reads. Filtered (Eq. 10): only columns with a bin inside the disc kappa <= alpha,
    kappa(0, q) = 2 pi min(q, P - q)/(P eps); the others need no transform, only zeros."""
    P = wl.fft_P
    H = P // 2
    live_half = H + 1
    if filtered:
        live_half = sum(1 for q in range(H + 1) if 2.0 * math.pi * q / (P * info["eps"]) <= info["alpha"])
    live = sum(1 for q in range(P) if min(q, P - q) < live_half)
    return live, live_half


def col_conv_algorithmic(wl, info, precision, channels, filtered=False):
    """Algorithmic bytes and flops of one column-pass launch.

    Bytes (the pass model of the method): each channel's m_rows x P intermediate read once and
    written once over the live columns (zeros written on the others), plus the stored
    (P/2+1)^2 spectrum read once per launch (all channels share it); b = 8 bytes per complex in
    mixed precision, 16 otherwise.
    Flops (the method's own count, the FFT convention 5 L log2 L per length-L transform): per live
    column and channel the pruned forward DFT of the m_rows nonzeros and the inverse DFT keeping
    m_rows outputs, each as two length-H transforms (4 x 5 H log2 H), plus the spectral product
    (6 flops per complex product at P points). The same count whatever the arithmetic.
    """
    P = wl.fft_P
    H = P // 2
    rows = info["row_hi"] - info["row_lo"] + 1
    b = 8 if precision == "mixed" else 16
    live, live_half = live_columns(wl, info, filtered)
    bytes_ = channels * (2 * rows * live * b + rows * (P - live) * b) + live_half * (H + 1) * b
    flops = channels * live * (4 * 5 * H * math.log2(H) + 6 * P)
    return bytes_, flops


def roofline(prof, wl, info, precision, peaks, src, kernel_stream_note):
    """Roofline of the column pass from one profiled step: achieved = algorithmic bytes per launch
    / mean CUDA-event launch time (the Calderon product alternates the N launch, 3 channels, and
    the S^alpha launch, 1 channel, so the per-launch model is the mean of the two)."""
    name = next((k for k in prof if k.startswith("col_conv")), None)
    if name is None:
        return None
    nl, tms = prof[name]
    avg_s = tms / nl / 1e3
    b3, f3 = col_conv_algorithmic(wl, info, precision, 3)
    b1, f1 = col_conv_algorithmic(wl, info, precision, 1, filtered=True)
    per_bytes = (b3 + b1) / 2
    per_flops = (f3 + f1) / 2
    ach = per_bytes / avg_s / 1e9
    alu_peak = FP64_PIPE_TFLOPS if precision == "native" else FP32_PIPE_TFLOPS
    return {"bound": "hbm", "kernel": name, "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": ach / peaks["hbm_gbs"], "traffic": COL_CONV_TRAFFIC.get(precision),
            "peak_source": src, "algorithmic_bytes_per_launch": per_bytes, "launches": nl,
            "avg_launch_ms": avg_s * 1e3, "timing": kernel_stream_note,
            "alu": {"method_flops_per_launch": per_flops, "achieved_tflops": per_flops / avg_s / 1e12,
                    "pipe": "FP64" if precision == "native" else "FP32",
                    "pipe_peak_tflops": alu_peak, "frac": per_flops / avg_s / 1e12 / alu_peak,
                    "note": "the method's flops (5 L log2 L per transform, 6 per complex product) in the "
                            "arithmetic of the mode; double-float runs each on ~8-20 FP32 instructions; pipe "
                            "peak derived from 152 SMs x lanes x 2 flop x 2.07 GHz"}}


def aggregate(elapsed: float, steps: int, world: int, device=None):
    """Max-over-ranks elapsed time and the whole-job rate (all ranks' steps / that time).

    Each rank works on its own problem (weak scaling), so the only exchange is this one
    reduction of a scalar; with world == 1 nothing is communicated.
    """
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([elapsed], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed = float(t.item())
    return elapsed, steps * world / elapsed


def _kernel_table(prof):
    return {k: {"launches": v[0], "total_ms": round(v[1], 3), "mean_ms": round(v[1] / max(v[0], 1), 5)}
            for k, v in prof.items()}


_STREAM = None


def solve_stream():
    """The stream every timed solve runs on. A solve on a stream of its own captures its Arnoldi
    step's operator product as a CUDA graph and replays it (the legacy default stream cannot be
    captured), as a user's solve on its own stream would; torch's events record on it too."""
    global _STREAM
    if _STREAM is None:
        import torch
        _STREAM = torch.cuda.Stream()
    return _STREAM


def _solve_once(aim, wl, prec, rhs, x, last=None):
    st = solve_stream()
    ctx = aim.Context(wl.nodes, wl.k, aim.TE, wl.m, fft_P=wl.fft_P, alpha=wl.alpha, stream=st)
    ctx.rhs_planewave(wl.angles, rhs, stream=st)
    x.zero_()
    info = ctx.solve("calderon_alpha", rhs, x, tol=SOLVE_TOL, restart=RESTART, max_iter=6000, precision=prec,
                     inner_tol=0.0, stream=st)
    if last is not None:
        last["info"] = info[0]
        last["ctx_info"] = ctx.info()
    ctx.close()


def single_solve_line(aim, wl, precision, steps, warmup, world, rank, dev, barrier, with_profile=True):
    """Times `steps` solves (setup + excitation + solve + destroy) after `warmup`, then one profiled
    step for the per-kernel table and the roofline. Returns the pieces of the JSON line."""
    import torch
    prec = {"fp64": aim.FP64, "mixed": aim.MIXED, "native": aim.FP64_NATIVE}[precision]
    st = solve_stream()
    with torch.cuda.stream(st):
        rhs = torch.empty((1, wl.n), dtype=torch.complex128, device=dev)
        x = torch.zeros_like(rhs)
    last = {}
    with torch.cuda.stream(st):
        for _ in range(warmup):
            _solve_once(aim, wl, prec, rhs, x, last)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(dev.index or 0)
    sampler.start()
    l0 = aim.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(st):
        e0.record()
        for _ in range(steps):
            _solve_once(aim, wl, prec, rhs, x, last)
        e1.record()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    elapsed = e0.elapsed_time(e1) / 1e3
    launches = aim.launch_count() - l0
    clocks = sampler.stop()
    prof = None
    if with_profile:
        # one more step with every launch bracketed by CUDA events on its own stream
        aim.profile_start()
        with torch.cuda.stream(st):
            _solve_once(aim, wl, prec, rhs, x)
        torch.cuda.synchronize()
        prof = aim.profile_stop()
    return elapsed, launches, clocks, prof, last


def gb300_arm(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_10784_gb300 import aim

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    wl = workload(args.seed + rank)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    warm = max(3, args.warmup)
    elapsed, launches, clocks, prof, last = single_solve_line(aim, wl, args.precision, args.steps, warm, world, rank,
                                                              dev, barrier)
    elapsed, value = aggregate(elapsed, args.steps, world, dev)

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    prec = {"fp64": aim.FP64, "mixed": aim.MIXED, "native": aim.FP64_NATIVE}[args.precision]
    rhs_h = torch.empty((1, wl.n), dtype=torch.complex128, pin_memory=True)
    x_h = torch.empty((1, wl.n), dtype=torch.complex128, pin_memory=True)
    with aim.Context(wl.nodes, wl.k, aim.TE, wl.m, fft_P=wl.fft_P, alpha=wl.alpha) as c0:
        c0.rhs_planewave(wl.angles, rhs_h)

    def step_e2e():
        st = solve_stream()
        ctx = aim.Context(wl.nodes, wl.k, aim.TE, wl.m, fft_P=wl.fft_P, alpha=wl.alpha, stream=st)
        ctx.solve("calderon_alpha", rhs_h, x_h, tol=SOLVE_TOL, restart=RESTART, max_iter=6000, precision=prec,
                  inner_tol=0.0, stream=st)
        ctx.close()

    e2e_steps = max(1, min(args.steps, E2E_STEPS_MAX))
    step_e2e()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        step_e2e()
    torch.cuda.synchronize()
    e2e_el, e2e_value = aggregate(time.perf_counter() - t0, e2e_steps, world, dev)
    e2e = {"value": e2e_value, "unit": UNIT, "steps": e2e_steps,
           "h2d_bytes_per_step": int(wl.nodes.nbytes + rhs_h.numel() * 16),
           "d2h_bytes_per_step": int(x_h.numel() * 16)}

    subs = {}
    if not args.no_sub and world == 1:
        subs["mixed_precision"] = mixed_sub(aim, wl, dev)
        subs["batching"] = batching_arm(args, aim, steps=1, warmup=1)
        subs["serving"] = serving_arm(args, aim)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank != 0:
        return None
    peaks, src = load_peaks()
    info = last["ctx_info"]
    roof = roofline(prof, wl, info, args.precision, peaks, src,
                    "CUDA events on the launching stream, one profiled solve after the timed region")
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": warm, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": {"fp64": "df64 (complex fp32-pair double-float grid and Gram-Schmidt products; c128 vectors)",
                     "mixed": "c64 grid + f64 refinement", "native": "c128"}[args.precision],
           "data": "synthetic (seeded random smooth contour family)",
           "config": workload_config(wl, args.precision, world), "e2e": e2e, "gpu_launches": launches,
           "roofline": roof, "clocks": clocks, "solve": last["info"],
           "setup_seconds_lib": info["setup_seconds"], "kernels": _kernel_table(prof)}
    out.update(subs)
    if not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline(wl, last["info"]["iters"])
    return out


def mixed_sub(aim, wl, dev, steps=3):
    """The same single-solve contour with the complex64 grid and FP64 refinement to 1e-5 (the
    precision configuration), timed alone; its column pass is the kernel the HBM roofline is about."""
    elapsed, launches, clocks, prof, last = single_solve_line(aim, wl, "mixed", steps, 1, 1, 0, dev, lambda: None)
    peaks, src = load_peaks()
    roof = roofline(prof, wl, last["ctx_info"], "mixed", peaks, src,
                    "CUDA events on the launching stream, one profiled solve after the timed region")
    return {"metric": "filtered Calderon solves/s at rel. residual 1e-5, complex64 grid + FP64 refinement",
            "value": steps / elapsed, "unit": UNIT, "steps": steps, "warmup": 1,
            "ms_per_step": elapsed / steps * 1e3, "gpu_launches": launches, "clocks": clocks,
            "solve": last["info"], "roofline": roof, "kernels": _kernel_table(prof),
            "config": "same contour and system as the headline; complex64 grid products and interpolation sums, "
                      "FP64 near-field sums, Gram inverse, Arnoldi and outer residual"}


# --------------------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# --------------------------------------------------------------------------------------
def oracle_sample(wl, iters, iters_source, n_near_rows=64, n_matvec=3):
    """Times the oracle on a bounded sample of one solve and extrapolates to solves/s.

    Sample: the oracle's grid kernel + spectrum and projections (full size); the near-pair search
    over the whole contour (full size, once); the exact near-field entries of `n_near_rows` rows,
    whose cost per row is scaled to N rows; `n_matvec` filtered Calderon products (mean).
    Solve time = setup + near field + iters x product time. The Arnoldi orthogonalisation of the
    oracle's GMRES is not counted (it would add to the oracle's time).
    """
    from oracle import aim as oaim
    t0 = time.perf_counter()
    op = oaim.TEOperators(wl.nodes, wl.k, wl.m, wl.fft_P, alpha=wl.alpha, near=False, direct_dft=False)
    t_grid = time.perf_counter() - t0
    t1 = time.perf_counter()
    oaim.near_pairs_te(wl.nodes, op.near_radius)
    t_pairs = time.perf_counter() - t1
    rows = np.arange(0, wl.n, max(1, wl.n // n_near_rows))[:n_near_rows]
    t2 = time.perf_counter()
    op._near_setup(rows=rows)               # its own pair search (t_pairs) + the entries of `rows`
    t_rows = max(0.0, time.perf_counter() - t2 - t_pairs)
    t_near = t_pairs + t_rows * wl.n / len(rows)
    x = synth.random_coeffs(wl.n, 1, 5)[0]
    op.calderon(x, filtered=True)           # first call factors G
    t3 = time.perf_counter()
    for _ in range(n_matvec):
        op.calderon(x, filtered=True)
    t_mv = (time.perf_counter() - t3) / n_matvec
    solve_s = t_grid + t_near + iters * t_mv
    return {"value": 1.0 / solve_s, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": "oracle setup (grid kernel, spectrum, projections) and near-pair search at full size; exact "
                      "near entries of %d of %d rows, per-row cost scaled; mean of %d filtered Calderon products; "
                      "solve = setup + near field + %d x product (%s)" %
                      (len(rows), wl.n, n_matvec, iters, iters_source),
            "seconds": {"grid_setup": t_grid, "near_pair_search": t_pairs, "near_entries_scaled": t_near - t_pairs,
                        "calderon_product": t_mv}}


# GMRES iterations of the filtered Calderon solve of this contour to 1e-5 (the GPU solve's count,
# FP64 mode; the oracle's GMRES on the same system takes the same count, which a GPU test checks on
# reduced contours). The reference arm has no GPU run to read it from.
SINGLE_SOLVE_ITERS = 1831


def cpu_baseline(wl, iters):
    return oracle_sample(wl, iters, "iterations: the GPU solve's count in this run, the same system and tolerance")


def reference_arm(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    wl = workload(args.seed)
    times = []
    res = None
    for i in range(max(3, args.warmup) + args.steps):
        res = oracle_sample(wl, SINGLE_SOLVE_ITERS, "iterations: %d, the GPU solve's count for this contour "
                                                    "and tolerance" % SINGLE_SOLVE_ITERS, n_near_rows=16, n_matvec=1)
        if i >= max(3, args.warmup):
            times.append(1.0 / res["value"])
    value = len(times) / sum(times)
    base = dict(res)
    base["value"] = value
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": 1e3 / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c128", "data": "synthetic (seeded random smooth contour family)",
            "config": workload_config(wl, "fp64", world), "cpu_baseline": base,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}


# --------------------------------------------------------------------------------------
# batching and serving workloads (sub-results of the default line, or lines of their own)
# --------------------------------------------------------------------------------------
def batching_arm(args, aim=None, steps=None, warmup=None):
    """nrhs plane waves (default 64, angles 2 pi r/nrhs) on one contour of perimeter 400 wl
    (N = 4000, 1024^2 grid), all right-hand sides in every grid launch, launch schedule from the
    autotuner. One step = setup + autotune + excitation + the batched filtered Calderon solve to 1e-5."""
    import torch
    if aim is None:
        import __graft_entry__
        __graft_entry__.build()
        from paper_2606_10784_gb300 import aim
    steps = args.steps if steps is None else steps
    warmup = max(1, args.warmup) if warmup is None else warmup
    precision = "mixed" if args.workload != "batching" else args.precision
    prec = {"fp64": aim.FP64, "mixed": aim.MIXED, "native": aim.FP64_NATIVE}[precision]
    wl = synth.batching_scale(args.seed, nrhs=args.nrhs)
    R = len(wl.angles)
    rhs = torch.empty((R, wl.n), dtype=torch.complex128, device="cuda")
    x = torch.zeros_like(rhs)
    last = {}

    sm = solve_stream()

    def step(solve=True):
        ctx = aim.Context(wl.nodes, wl.k, aim.TE, wl.m, fft_P=wl.fft_P, alpha=wl.alpha, stream=sm)
        last["schedule"] = ctx.autotune(nrhs=R, precision=prec, stream=sm)
        ctx.rhs_planewave(wl.angles, rhs, stream=sm)
        x.zero_()
        if solve:
            st, info = ctx.solve("calderon_alpha", rhs, x, tol=SOLVE_TOL, restart=RESTART, max_iter=6000,
                                 precision=prec, inner_tol=0.0, check=False, stream=sm)
            last["status"], last["info"] = st, info
        else:   # warm-up: setup, autotune and one batched product load every kernel
            ctx.matvec("calderon_alpha", rhs, x, precision=prec, stream=sm)
        ctx.close()

    with torch.cuda.stream(sm):
        for _ in range(warmup):
            step(solve=False)
    torch.cuda.synchronize()
    l0 = aim.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(sm):
        e0.record()
        for _ in range(steps):
            step()
        e1.record()
    torch.cuda.synchronize()
    el = e0.elapsed_time(e1) / 1e3
    its = [i["iters"] for i in last["info"]]
    return {"metric": "batched filtered Calderon solves (right-hand sides/s) at rel. residual 1e-5",
            "value": steps * R / el, "unit": "rhs-solves/s", "n_gpus": 1, "steps": steps,
            "warmup": "%d x (setup + autotune + one batched product)" % warmup, "ms_per_step": el / steps * 1e3,
            "higher_is_better": True, "dtype": precision, "data": "synthetic",
            "config": {"workload": "perimeter 400 wl, N=%d, grid %d^2 (P=%d), %d plane waves, alpha=2k, GMRES(%d)"
                                   % (wl.n, wl.m, wl.fft_P, R, RESTART), "schedule": last["schedule"]},
            "solve": {"status": last["status"], "iters_min": min(its), "iters_max": max(its),
                      "converged": sum(i["converged"] for i in last["info"])},
            "gpu_launches": aim.launch_count() - l0}


def serving_arm(args, aim=None):
    """Poisson stream (200 requests/s, seed 11): perimeter log-uniform in [5, 500] wavelengths at a
    wavenumber U[pi, 4pi], N = 10 per wavelength, grid 32^2..1024^2, 1..16 plane waves, filtered
    Calderon solves to 1e-5; admission by a device-memory budget, 4 concurrent slots."""
    import torch
    if aim is None:
        import __graft_entry__
        __graft_entry__.build()
        from paper_2606_10784_gb300 import aim
    from paper_2606_10784_gb300 import serving
    precision = "mixed" if args.workload != "serving" else args.precision
    n_warm = max(1, args.requests // 10)
    stream = synth.serving_stream(args.requests + n_warm, rate=200.0, seed=11)
    reqs = []
    for i, s in enumerate(stream):
        nodes = synth.StarContour.from_seed(s.seed % 100000).polygon(s.perimeter, s.n_seg)
        reqs.append(serving.SolveRequest(nodes=nodes, k=s.k, m=s.m, angles=synth.equispaced_angles(s.nrhs),
                                         alpha=s.alpha, precision={"fp64": aim.FP64, "mixed": aim.MIXED,
                                                                   "native": aim.FP64_NATIVE}[precision],
                                         tol=SOLVE_TOL, restart=RESTART, arrival=s.t_arrival, rid=i))
    free, total = torch.cuda.mem_get_info()
    budget = int(0.6 * free)
    import copy
    runs = {}
    for fused in (True, False):
        rs = copy.deepcopy(reqs)
        srv = serving.Server(memory_budget_bytes=budget, slots=4, policy=args.policy, fused=fused)
        serving.replay(srv, rs[:n_warm])
        l0 = aim.launch_count()
        t0 = time.perf_counter()
        res = serving.replay(srv, rs[n_warm:])
        el = time.perf_counter() - t0
        stats = srv.fusion_stats()
        srv.close()
        timed = [r for r in res if r.rid >= n_warm]
        runs[fused] = {"latency": serving.latency_summary(timed), "wall_s": el, "refused": srv.refused,
                       "gpu_launches": aim.launch_count() - l0, "fusion": stats}
    summ = runs[False]["latency"]
    return {"metric": "served filtered Calderon solves: p50/p99 latency and solves/s", "value": summ.get("solves_per_s"),
            "unit": "solves/s", "n_gpus": 1, "higher_is_better": True, "dtype": precision, "data": "synthetic",
            "latency": summ, "wall_s": runs[False]["wall_s"], "budget_bytes": budget, "refused": runs[False]["refused"],
            "gpu_launches": runs[False]["gpu_launches"],
            "fused": {"latency": runs[True]["latency"], "wall_s": runs[True]["wall_s"],
                      "gpu_launches": runs[True]["gpu_launches"], "fusion": runs[True]["fusion"]},
            "config": {"workload": "Poisson 200/s, perimeter log-U[5,500] wl, N=10/wl, grids 32^2..1024^2, "
                                   "1..16 rhs, %d timed requests after %d warm-up" % (len(reqs) - n_warm, n_warm),
                       "policy": args.policy, "slots": 4,
                       "fusion": "default: each slot launches its own products on its own stream; 'fused': the "
                                 "slots' solves share a batcher, products of concurrent requests of one size class "
                                 "run in one multi-context launch per stage"}}


def multi_arm(args, aim=None, rounds=20):
    """Several problems in one launch: filtered Calderon products of 8 contexts drawn from the serving
    stream (seed 11, each with its own nrhs plane-wave-sized random vectors), one round = one product
    of each. Timed both ways on one stream with CUDA events after one warm-up round: a separate
    aim_matvec per context, and aim_matvec_multi (every grid-pass stage of all eight in one
    persistent launch). Mixes: the first 8 requests with P <= 512, the first 8 with 512 <= P <= 1024,
    and the stream's first 8; in mixed precision and FP64."""
    import torch
    if aim is None:
        import __graft_entry__
        __graft_entry__.build()
        from paper_2606_10784_gb300 import aim
    stream = synth.serving_stream(200, rate=200.0, seed=11)
    mixes = {"P<=512": lambda P: P <= 512, "512<=P<=1024": lambda P: 512 <= P <= 1024, "first 8": lambda P: True}
    st = solve_stream()
    out = {"metric": "filtered Calderon products of 8 contexts per round: ms per round", "unit": "ms", "rounds": rounds,
           "mixes": {}}
    for name, keep in mixes.items():
        ctxs, xs, ys = [], [], []
        for s in stream:
            if len(ctxs) == 8:
                break
            if not keep(max(2 * s.m, 64)):   # the embedding side aim_setup selects for m (a power of two)
                continue
            nodes = synth.StarContour.from_seed(s.seed % 100000).polygon(s.perimeter, s.n_seg)
            ctxs.append(aim.Context(nodes, s.k, aim.TE, s.m, alpha=s.alpha, stream=st))
            x = torch.from_numpy(synth.random_coeffs(s.n_seg, s.nrhs, seed=len(ctxs))).cuda()
            xs.append(x)
            ys.append(torch.empty_like(x))
        row = {"fft_P": sorted({c.info()["fft_P"] for c in ctxs}), "nrhs": [int(x.shape[0]) for x in xs]}
        for pname, prec in (("mixed", aim.MIXED), ("fp64", aim.FP64)):
            def separate():
                for c, x, y in zip(ctxs, xs, ys):
                    c.matvec("calderon_alpha", x, y, precision=prec, stream=st)

            def fused():
                aim.matvec_multi(ctxs, ["calderon_alpha"] * len(ctxs), xs, ys, precision=prec, stream=st)

            for label, fn in (("separate", separate), ("multi", fused)):
                fn()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                for _ in range(rounds):
                    fn()
                e1.record(st)
                torch.cuda.synchronize()
                row["%s_%s_ms" % (pname, label)] = e0.elapsed_time(e1) / rounds
        out["mixes"][name] = row
        for c in ctxs:
            c.close()
    return out


# --------------------------------------------------------------------------------------
# profiling case (for ncu): one operator of the single-solve workload
# --------------------------------------------------------------------------------------
def profile_case(args):
    """Sets up the single-solve contour and applies --op --repeat times to a seeded random vector.
    The first k_col_conv launch is the operator's first column pass (3 channels for N, 1 for
    S_alpha), so `ncu -k regex:k_col_conv -c 1` captures one full-size launch. --time prints the mean
    device time per launch of each grid kernel (CUDA events on the launching stream, after one
    warm-up product)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_10784_gb300 import aim
    prec = {"fp64": aim.FP64, "mixed": aim.MIXED, "native": aim.FP64_NATIVE}[args.precision]
    wl = workload(args.seed)
    ctx = aim.Context(wl.nodes, wl.k, aim.TE, wl.m, fft_P=wl.fft_P, alpha=wl.alpha)
    x = torch.from_numpy(synth.random_coeffs(wl.n, 1, 0)).cuda()
    y = torch.empty_like(x)
    out = {"op": args.op, "precision": args.precision, "schedule": ctx.get_schedule(prec)}
    if args.time:
        ctx.matvec(args.op, x, y, precision=prec)
        torch.cuda.synchronize()
        aim.profile_start()
    for _ in range(max(1, args.repeat)):
        ctx.matvec(args.op, x, y, precision=prec)
    torch.cuda.synchronize()
    if args.time:
        prof = aim.profile_stop()
        out["ms_per_launch"] = {k: round(v[1] / max(v[0], 1), 4) for k, v in prof.items() if v[0]}
    ctx.close()
    return out


# --------------------------------------------------------------------------------------
# DFT stage on CUDA cores against tensor cores
# --------------------------------------------------------------------------------------
STAGE_VARIANTS = (("cuda_cores_fp32", 0), ("mma_tf32", 1), ("mma_tf32x3", 2), ("split_data_path_only", 3))
# the dense contraction of one DFT-16 column: 2 x 32 x 32 real flops
GEMM16_FLOPS = 2 * 32 * 32


def dft_stage_case(args):
    """Times aim_dft_stage: `--stage-passes` radix-16 passes over `--stage-groups` groups of 4096
    complex64 values held in shared memory, for each variant (the product's CUDA-core butterfly,
    mma.sync TF32, mma.sync split TF32). The rate is taken from the difference between launches of
    `--stage-passes` and half as many passes, so loads, stores and set-up cancel. Beside it: the tensor cores' TF32 rate measured by
    cuBLAS on a large GEMM, and the DFT-16 rate that rate would give a tcgen05 stage that spent
    nothing on data movement (2 x 32 x 32 flops per column, three products with the split).
    Accuracy: relative L2 error of one pass against the FP64 definition on two groups."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_10784_gb300 import aim
    G, passes = args.stage_groups, args.stage_passes
    gen = torch.Generator(device="cuda").manual_seed(0)
    x = torch.complex(torch.randn(G * 4096, device="cuda", generator=gen),
                      torch.randn(G * 4096, device="cuda", generator=gen))
    y = torch.empty_like(x)
    st = torch.cuda.current_stream()

    def timed(v, p, reps=7):
        for _ in range(3):
            aim.dft_stage(v, x, y, p, stream=st)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            aim.dft_stage(v, x, y, p, stream=st)
            e1.record(st)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    # FP64 reference of one pass on the first two groups (the definition in aim.h)
    x2 = x[:2 * 4096].cpu().numpy().astype(np.complex128)
    cols = x2.reshape(2, 16, 256).transpose(0, 2, 1)
    c, i = np.arange(256)[:, None], np.arange(16)[None, :]
    t = np.exp(-2j * np.pi * (c % 16) * i / 256) / 4
    F = np.exp(-2j * np.pi * np.outer(np.arange(16), np.arange(16)) / 16)
    ref = np.einsum("gci,ki->gck", cols * t[None], F).reshape(-1)
    out = {"case": "radix-16 DFT pass, %d groups x 4096 complex64 values in shared memory, %d passes per launch"
                   % (G, passes), "variants": {}}
    ref_split = (cols * t[None]).transpose(0, 2, 1).reshape(-1)   # variant 3: t(c, i) x_i(c) in place
    for name, v in STAGE_VARIANTS:
        if args.stage_variant >= 0 and v != args.stage_variant:
            continue
        half = passes // 2
        ms_p, ms_h = timed(v, passes), timed(v, half)
        rate = G * 256 * (passes - half) / ((ms_p - ms_h) * 1e-3)
        aim.dft_stage(v, x[:2 * 4096], y[:2 * 4096], 1, stream=st)
        torch.cuda.synchronize()
        want = ref_split if v == 3 else ref
        err = float(np.linalg.norm(y[:2 * 4096].cpu().numpy() - want) / np.linalg.norm(want))
        out["variants"][name] = {"ms_launch": round(ms_p, 4), "ms_launch_half_passes": round(ms_h, 4),
                                 "dft16_per_s": rate, "rel_err_one_pass": err}
    if "cuda_cores_fp32" not in out["variants"]:
        return out
    base = out["variants"]["cuda_cores_fp32"]["dft16_per_s"]
    for name in out["variants"]:
        out["variants"][name]["vs_cuda_cores"] = out["variants"][name]["dft16_per_s"] / base
    # tensor-core TF32 rate by cuBLAS (tcgen05 inside the library), burst
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    n = 8192
    a = torch.randn(n, n, device="cuda", generator=gen)
    b = torch.randn(n, n, device="cuda", generator=gen)
    for _ in range(3):
        torch.matmul(a, b)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(10):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    torch.backends.cuda.matmul.allow_tf32 = prev
    tf32 = 2.0 * n ** 3 / (best * 1e-3) / 1e12
    out["tensor_core_bound"] = {
        "tf32_gemm_tflops_cublas": tf32,
        "dft16_per_s_tf32": tf32 * 1e12 / GEMM16_FLOPS,
        "dft16_per_s_split_tf32": tf32 * 1e12 / (3 * GEMM16_FLOPS),
        "note": "a tcgen05 stage at the measured TF32 GEMM rate with no data movement, operand split or "
                "twiddle cost: the most any tensor-core DFT-16 stage could reach"}
    out["bound_vs_cuda_cores"] = {"tf32": out["tensor_core_bound"]["dft16_per_s_tf32"] / base,
                                  "split_tf32": out["tensor_core_bound"]["dft16_per_s_split_tf32"] / base}
    return out


def main():
    args = parse()
    if args.dft_stage:
        out = dft_stage_case(args)
    elif args.profile_case:
        out = profile_case(args)
    elif args.impl == "reference":
        out = reference_arm(args)
    elif args.workload == "batching":
        out = batching_arm(args)
    elif args.workload == "serving":
        out = serving_arm(args)
    elif args.workload == "multi":
        out = multi_arm(args)
    else:
        out = gb300_arm(args)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
