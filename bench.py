#!/usr/bin/env python3
"""Benchmark: filtered-AIM Calderon TE-EFIE solves on GB300.

One step is one pass of the whole method for one scatterer: setup of every operator from the
contour (quadrature, grid, projections, kernel spectrum and its circular truncation, near
field, Gram inverse), the plane-wave excitation, and the GMRES solve of the filtered
Calderon system G^-1 S^alpha G^-1 N j = G^-1 S^alpha G^-1 E to a relative residual of 1e-8.
Workload: a seeded random smooth contour of perimeter 1000 wavelengths, 10 segments per
wavelength (N = 10000), a 2048 x 2048 grid (P = 4096), 4 x 4 stencils, alpha = 2k, one
right-hand side. Inputs are synthetic (no dataset exists for this workload).

Under torchrun each rank solves its own contour (seed = rank): weak scaling, no collective in
the data path; value = all ranks' solves / max-over-ranks time.

--impl reference runs the CPU oracle (numpy/scipy FP64) on a bounded sample of the same
workload on the host cores, rank 0 only.
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
FP64_PEAK_TFLOPS = 1.25   # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (nominal GB300 FP64 rate)
FALLBACK_HBM_GBS = 6800.0


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
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--workload", choices=["single", "batching", "serving"], default="single",
                    help="single: one filtered Calderon solve per step (the default line); batching: 64 "
                         "right-hand sides per solve (perimeter 400 wl, 1024^2 grid); serving: a Poisson "
                         "stream of requests with p50/p99 latency")
    ap.add_argument("--requests", type=int, default=40, help="serving: timed requests (after 10%% warm-up)")
    ap.add_argument("--policy", choices=["sjf", "fifo"], default="sjf", help="serving: admission order")
    ap.add_argument("--nrhs", type=int, default=64, help="batching: right-hand sides per solve (angles 2 pi r/nrhs)")
    return ap.parse_args()


def workload(seed):
    return synth.single_solve_scale(seed=seed)


def workload_config(wl, precision, world):
    return {"workload": "filtered Calderon TE-EFIE solve, perimeter 1000 wl, N=%d, grid %dx%d (P=%d), s=4, p=4, "
                        "alpha=2k, 1 rhs, GMRES(%d) rel. residual %.0e" % (wl.n, wl.m, wl.m, wl.fft_P, RESTART, SOLVE_TOL),
            "N": wl.n, "grid_m": wl.m, "fft_P": wl.fft_P, "alpha_over_k": wl.alpha / wl.k, "nrhs": 1,
            "precision": precision, "contour_seed": "rank", "ranks": world,
            "l2": "inputs larger than L2 (grid intermediate 3 x 2048 x 4096 complex per product > 129 MB)"}


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
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


# Flop costs of one complex operation in the kernels' own arithmetic (FMA = 2 flops).
# Plain complex64/complex128: add 2, multiply 6. Double-float (each real an unevaluated sum of two
# floats): an add is TwoSum (6) + 2 adds + FastTwoSum (3) = 11 per real part, so 22 per complex
# add; a multiply's real part is two exact products (1 mul + 1 fma each = 6), TwoSum (6), 2 adds,
# 4 cross-term fmas (8) and FastTwoSum (3) = 25, so 50 per complex multiply.
CPLX_COST = {"plain": (2, 6), "df": (22, 50)}


def fft_flops(logh: int, kind: str) -> float:
    """Flops of one length-2^logh transform as the kernels run it: radix-16 passes (radix-2
    decimation in frequency inside, 10 non-trivial rotations per 16-point DFT) plus one radix-2^r
    pass; every pass but the first multiplies by R-1 twiddles, of which 11/4/1 (R = 16/8/4) are
    formed as products of table powers."""
    add, mul = CPLX_COST[kind]
    h = 1 << logh

    def dft(r):
        lg = int(math.log2(r))
        rot = {16: 10, 8: 2, 4: 0, 2: 0}[r]
        return (r // 2) * lg * 2 * add + rot * mul

    extra = {16: 11, 8: 4, 4: 1, 2: 0}
    radices = [16] * (logh // 4) + ([1 << (logh % 4)] if logh % 4 else [])
    total = 0.0
    for p, r in enumerate(radices):
        per = dft(r) + (0 if p == 0 else (r - 1 + extra[r]) * mul)
        total += (h // r) * per
    return total


def col_conv_algorithmic(wl, info, precision, channels, filtered=False):
    """Algorithmic work of one column-pass launch (the dominant kernel).

    Bytes: each channel's m_rows x P intermediate read once and written once, plus the stored
    (P/2+1)^2 spectrum read once per launch (all channels use the same spectrum). Flops: per column and channel four half-length
    transforms (fft_flops), the w^n twiddle of the odd half, the spectral product of P points
    and the recombination y = A + conj(w^n) B at every one of the H rows. For the filtered
    spectrum only the columns that the mask keeps count (2 pi min(q, P - q) / (P eps) <= alpha):
    the others need no transform, only a zero written per row.
    """
    P = wl.fft_P
    H = P // 2
    rows = info["row_hi"] - info["row_lo"] + 1
    kind = "df" if precision == "fp64" else "plain"
    add, mul = CPLX_COST[kind]
    b = 8 if precision == "mixed" else 16
    live_half = H + 1
    if filtered:
        live_half = sum(1 for q in range(H + 1) if 2.0 * math.pi * q / (P * info["eps"]) <= info["alpha"])
    live = sum(1 for q in range(P) if min(q, P - q) < live_half)
    bytes_ = channels * (2 * rows * live * b + rows * (P - live) * b) + live_half * (H + 1) * b
    per_col = 4 * fft_flops(int(math.log2(H)), kind) + H * mul + P * mul + H * (mul + add)
    flops = channels * live * per_col
    return bytes_, flops


FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # 152 SMs x 128 FP32 lanes x FMA x 2.07 GHz = 80.5

# DRAM traffic of k_col_conv per launch (dram__bytes_read.sum + dram__bytes_write.sum), the mean of
# the two launches of one filtered Calderon product (N: 3 channels, S^alpha: 1 channel), from one
# ncu capture of the default schedule at the single-solve size; the profiles directory gives the
# capture and its command. None where no capture matches the current kernel and schedule.
COL_CONV_TRAFFIC = {"fp64": 531852928, "mixed": 202739328, "native": None}


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
    prec = {"fp64": aim.FP64, "mixed": aim.MIXED, "native": aim.FP64_NATIVE}[args.precision]
    wl = workload(args.seed + rank)
    rhs = torch.empty((1, wl.n), dtype=torch.complex128, device=dev)
    x = torch.zeros_like(rhs)
    last = {}

    def step():
        ctx = aim.Context(wl.nodes, wl.k, aim.TE, wl.m, fft_P=wl.fft_P, alpha=wl.alpha)
        ctx.rhs_planewave(wl.angles, rhs)
        x.zero_()
        info = ctx.solve("calderon_alpha", rhs, x, tol=SOLVE_TOL, restart=RESTART, max_iter=6000, precision=prec,
                         inner_tol=0.0)
        last["info"] = info[0]
        last["ctx_info"] = ctx.info()
        ctx.close()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    aim.profile_start()
    l0 = aim.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    elapsed = e0.elapsed_time(e1) / 1e3
    launches = aim.launch_count() - l0
    prof = aim.profile_stop()
    clocks = sampler.stop()
    elapsed, value = aggregate(elapsed, args.steps, world, dev)

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    rhs_h = torch.empty((1, wl.n), dtype=torch.complex128, pin_memory=True)
    x_h = torch.empty((1, wl.n), dtype=torch.complex128, pin_memory=True)
    with aim.Context(wl.nodes, wl.k, aim.TE, wl.m, fft_P=wl.fft_P, alpha=wl.alpha) as c0:
        c0.rhs_planewave(wl.angles, rhs_h)

    def step_e2e():
        ctx = aim.Context(wl.nodes, wl.k, aim.TE, wl.m, fft_P=wl.fft_P, alpha=wl.alpha)
        ctx.solve("calderon_alpha", rhs_h, x_h, tol=SOLVE_TOL, restart=RESTART, max_iter=6000, precision=prec,
                  inner_tol=0.0)
        ctx.close()

    step_e2e()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_e2e()
    torch.cuda.synchronize()
    e2e_el, e2e_value = aggregate(time.perf_counter() - t0, args.steps, world, dev)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    e2e = {"value": e2e_value, "unit": UNIT,
           "h2d_bytes_per_step": int(wl.nodes.nbytes + rhs_h.numel() * 16),
           "d2h_bytes_per_step": int(x_h.numel() * 16)}

    if rank != 0:
        return None
    # roofline of the dominant kernel (largest total time in the timed region)
    traffic = COL_CONV_TRAFFIC.get(args.precision)
    peaks, src = load_peaks()
    top = max(prof.items(), key=lambda kv: kv[1][1])
    name, (nl, tms) = top
    avg_s = tms / nl / 1e3
    info = last["ctx_info"]
    roof = None
    if name.startswith("col_conv"):
        # the Calderon product runs 3 channels (N) and 1 channel (S^alpha) per application
        n_n = nl // 2
        b3, f3 = col_conv_algorithmic(wl, info, args.precision, 3)
        b1, f1 = col_conv_algorithmic(wl, info, args.precision, 1, filtered=True)
        per_launch_bytes = (b3 + b1) / 2
        per_launch_flops = (f3 + f1) / 2
        if args.precision in ("fp64", "native"):
            # FP64 mode runs double-float arithmetic on the FP32 pipe; native mode the FP64 pipe
            peak = FP32_PEAK_TFLOPS if args.precision == "fp64" else FP64_PEAK_TFLOPS
            ach = per_launch_flops / avg_s / 1e12
            roof = {"bound": "alu", "kernel": name, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": ach / peak, "traffic": traffic if name.startswith("col_conv") else None,
                    "peak_source": ("FP32 pipe nominal: 152 SMs x 128 lanes x 2 flop x 2.07 GHz (derived; "
                                    "MEASURED_PEAKS has no FP32 figure); flops counted in double-float arithmetic"
                                    if args.precision == "fp64" else
                                    "FP64 nominal: 152 SMs x 64 FP64 flop/clk x 2.07 GHz (derived)"),
                    "algorithmic_flops_per_launch": per_launch_flops,
                    "algorithmic_bytes_per_launch": per_launch_bytes,
                    "hbm_frac_of_measured": per_launch_bytes / avg_s / 1e9 / peaks["hbm_gbs"],
                    "launches": nl, "avg_launch_ms": avg_s * 1e3}
        else:
            ach = per_launch_bytes / avg_s / 1e9
            roof = {"bound": "hbm", "kernel": name, "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": ach / peaks["hbm_gbs"], "traffic": traffic, "peak_source": src,
                    "launches": nl, "avg_launch_ms": avg_s * 1e3}
    kernels = {k: {"launches": v[0], "total_ms": round(v[1], 3)} for k, v in prof.items()}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": max(3, args.warmup), "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "df64 (complex fp32-pair double-float grid and Gram-Schmidt products; c128 vectors)",
                                                   "mixed": "c64 grid + f64 refinement",
                                                   "native": "c128"}[args.precision],
           "data": "synthetic (seeded random smooth contour family)",
           "config": workload_config(wl, args.precision, world), "e2e": e2e, "gpu_launches": launches,
           "roofline": roof, "clocks": clocks, "solve": last["info"],
           "setup_seconds_lib": last["ctx_info"]["setup_seconds"], "kernels": kernels}
    if not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline(wl, last["info"]["iters"])
    return out


# --------------------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# --------------------------------------------------------------------------------------
def oracle_sample(wl, iters, n_near_rows=64, n_matvec=1):
    """Times the oracle on a bounded sample of one solve and extrapolates to solves/s.

    Sample: the oracle's grid kernel + spectrum (full size), projections (full size), the
    near-field correction for `n_near_rows` rows scaled to N rows, and `n_matvec` filtered
    Calderon products; solve time = setup + iters x product time, iters = the GPU solve's
    GMRES iteration count.
    """
    from oracle import aim as oaim
    t0 = time.perf_counter()
    op = oaim.TEOperators(wl.nodes, wl.k, wl.m, wl.fft_P, alpha=wl.alpha, near=False, direct_dft=False)
    t_grid = time.perf_counter() - t0
    rows = np.arange(0, wl.n, max(1, wl.n // n_near_rows))[:n_near_rows]
    t1 = time.perf_counter()
    op._near_setup(rows=rows)
    t_near = (time.perf_counter() - t1) * wl.n / len(rows)
    x = synth.random_coeffs(wl.n, 1, 5)[0]
    t2 = time.perf_counter()
    for _ in range(n_matvec):
        op.calderon(x, filtered=True)
    t_mv = (time.perf_counter() - t2) / n_matvec
    solve_s = t_grid + t_near + iters * t_mv
    return {"value": 1.0 / solve_s, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": "oracle setup (grid kernel, spectrum, projections) at full size + near field on %d of %d rows "
                      "scaled + %d filtered Calderon product(s); solve = setup + %d x product" %
                      (len(rows), wl.n, n_matvec, iters),
            "seconds": {"grid_setup": t_grid, "near_field_scaled": t_near, "calderon_product": t_mv}}


GPU_ITERS_HINT = 1831  # GMRES iterations of the GPU solve of this workload (used by the reference arm)


def cpu_baseline(wl, iters):
    return oracle_sample(wl, iters)


def reference_arm(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    wl = workload(args.seed)
    times = []
    res = None
    for i in range(max(3, args.warmup) + args.steps):
        t0 = time.perf_counter()
        res = oracle_sample(wl, GPU_ITERS_HINT, n_near_rows=16, n_matvec=1)
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
# batching and serving workloads (separate JSON lines; the default line is "single")
# --------------------------------------------------------------------------------------
def batching_arm(args):
    """nrhs plane waves (default 64, angles 2 pi r/nrhs) on one contour of perimeter 400 wl
    (N = 4000, 1024^2 grid), all right-hand sides in every grid launch, launch schedule from the
    autotuner. One step = setup + autotune + excitation + the batched filtered Calderon solve to 1e-5."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_10784_gb300 import aim
    prec = {"fp64": aim.FP64, "mixed": aim.MIXED, "native": aim.FP64_NATIVE}[args.precision]
    wl = synth.batching_scale(args.seed, nrhs=args.nrhs)
    R = len(wl.angles)
    rhs = torch.empty((R, wl.n), dtype=torch.complex128, device="cuda")
    x = torch.zeros_like(rhs)
    last = {}

    def step(solve=True):
        ctx = aim.Context(wl.nodes, wl.k, aim.TE, wl.m, fft_P=wl.fft_P, alpha=wl.alpha)
        last["schedule"] = ctx.autotune(nrhs=R, precision=prec)
        ctx.rhs_planewave(wl.angles, rhs)
        x.zero_()
        if solve:
            st, info = ctx.solve("calderon_alpha", rhs, x, tol=SOLVE_TOL, restart=RESTART, max_iter=6000,
                                 precision=prec, inner_tol=0.0, check=False)
            last["status"], last["info"] = st, info
        else:   # warm-up: setup, autotune and one batched product load every kernel
            ctx.matvec("calderon_alpha", rhs, x, precision=prec)
        ctx.close()

    for _ in range(max(1, args.warmup)):
        step(solve=False)
    torch.cuda.synchronize()
    aim.profile_start()
    l0 = aim.launch_count()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    prof = aim.profile_stop()
    its = [i["iters"] for i in last["info"]]
    return {"metric": "batched filtered Calderon solves (right-hand sides/s) at rel. residual 1e-5",
            "value": args.steps * R / el, "unit": "rhs-solves/s", "n_gpus": 1, "steps": args.steps,
            "warmup": "%d x (setup + autotune + one batched product)" % max(1, args.warmup), "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
            "dtype": args.precision, "data": "synthetic",
            "config": {"workload": "perimeter 400 wl, N=%d, grid %d^2 (P=%d), %d plane waves, alpha=2k, GMRES(%d)"
                                   % (wl.n, wl.m, wl.fft_P, R, RESTART), "schedule": last["schedule"]},
            "solve": {"status": last["status"], "iters_min": min(its), "iters_max": max(its),
                      "converged": sum(i["converged"] for i in last["info"])},
            "gpu_launches": aim.launch_count() - l0,
            "kernels": {k: {"launches": v[0], "total_ms": round(v[1], 3)} for k, v in prof.items()}}


def serving_arm(args):
    """Poisson stream (200 requests/s, seed 11): perimeter log-uniform in [5, 500] wavelengths at a
    wavenumber U[pi, 4pi], N = 10 per wavelength, grid 32^2..1024^2, 1..16 plane waves, filtered
    Calderon solves to 1e-5; admission by a device-memory budget, 4 concurrent slots."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_10784_gb300 import aim, serving
    n_warm = max(1, args.requests // 10)
    stream = synth.serving_stream(args.requests + n_warm, rate=200.0, seed=11)
    reqs = []
    for i, s in enumerate(stream):
        nodes = synth.StarContour.from_seed(s.seed % 100000).polygon(s.perimeter, s.n_seg)
        reqs.append(serving.SolveRequest(nodes=nodes, k=s.k, m=s.m, angles=synth.equispaced_angles(s.nrhs),
                                         alpha=s.alpha, precision={"fp64": aim.FP64, "mixed": aim.MIXED,
                                                                   "native": aim.FP64_NATIVE}[args.precision],
                                         tol=SOLVE_TOL, restart=RESTART, arrival=s.t_arrival, rid=i))
    free, total = torch.cuda.mem_get_info()
    budget = int(0.6 * free)
    srv = serving.Server(memory_budget_bytes=budget, slots=4, policy=args.policy)
    serving.replay(srv, reqs[:n_warm])
    t0 = time.perf_counter()
    res = serving.replay(srv, reqs[n_warm:])
    el = time.perf_counter() - t0
    srv.close()
    timed = [r for r in res if r.rid >= n_warm]
    summ = serving.latency_summary(timed)
    return {"metric": "served filtered Calderon solves: p50/p99 latency and solves/s", "value": summ.get("solves_per_s"),
            "unit": "solves/s", "n_gpus": 1, "higher_is_better": True, "dtype": args.precision, "data": "synthetic",
            "latency": summ, "wall_s": el, "budget_bytes": budget, "refused": srv.refused,
            "config": {"workload": "Poisson 200/s, perimeter log-U[5,500] wl, N=10/wl, grids 32^2..1024^2, "
                                   "1..16 rhs, %d timed requests after %d warm-up" % (len(reqs) - n_warm, n_warm),
                       "policy": args.policy, "slots": 4}}


def main():
    args = parse()
    if args.impl == "reference":
        out = reference_arm(args)
    elif args.workload == "batching":
        out = batching_arm(args)
    elif args.workload == "serving":
        out = serving_arm(args)
    else:
        out = gb300_arm(args)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
