"""Runs grid products on the single-solve workload, for kernel profilers and schedule sweeps.

    python -m paper_2606_10784_gb300.profile_case --precision fp64 --op N --repeat 1
    python -m paper_2606_10784_gb300.profile_case --precision fp64 --op N --repeat 20 --time --sweep

Sets up the perimeter-1000-wavelength contour (N = 10000 unknowns, 2048 x 2048 grid, P = 4096,
alpha = 2k) and applies the chosen operator `repeat` times to a seeded random vector. The first
k_col_conv launch is the operator's first column pass (3 channels for N, 1 for S_alpha), so
`ncu -k regex:k_col_conv -c 1` captures exactly one full-size launch.

--time prints the mean device time per launch of each grid kernel (CUDA events on the launching
stream, after one warm-up product). --sweep does that for every feasible launch schedule.
--schedule tpt,row_threads,col_cols[,elems_per_thread] fixes one schedule.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _timed(aim, ctx, op, x, y, prec, repeat):
    import torch
    ctx.matvec(op, x, y, precision=prec)
    torch.cuda.synchronize()
    aim.profile_start()
    for _ in range(repeat):
        ctx.matvec(op, x, y, precision=prec)
    torch.cuda.synchronize()
    prof = aim.profile_stop()
    return {k: round(v[1] / max(v[0], 1), 4) for k, v in prof.items() if v[0]}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--precision", choices=["fp64", "mixed", "native"], default="fp64")
    ap.add_argument("--op", default="N")
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--time", action="store_true")
    ap.add_argument("--sweep", action="store_true")
    ap.add_argument("--schedule", default="")
    args = ap.parse_args(argv)
    import torch

    import synth
    from paper_2606_10784_gb300 import aim
    prec = {"fp64": aim.FP64, "mixed": aim.MIXED, "native": aim.FP64_NATIVE}[args.precision]
    wl = synth.single_solve_scale(0)
    ctx = aim.Context(wl.nodes, wl.k, aim.TE, wl.m, fft_P=wl.fft_P, alpha=wl.alpha)
    x = torch.from_numpy(synth.random_coeffs(wl.n, args.nrhs, 0)).cuda()
    y = torch.empty_like(x)
    if args.schedule:
        vals = [int(v) for v in args.schedule.split(",")]
        ctx.set_schedule(prec, *vals)
    if args.sweep:
        for e in (16, 8):
            for t in (1, 2):
                for r in (128, 256, 1024):
                    for c in (0, 1, 2, 4, 8):
                        try:
                            ctx.set_schedule(prec, t, r, c, e)
                        except aim.AimError:
                            continue
                        ms = _timed(aim, ctx, args.op, x, y, prec, max(args.repeat, 1))
                        print(json.dumps({"schedule": ctx.get_schedule(prec), "ms_per_launch": ms}))
    elif args.time:
        ms = _timed(aim, ctx, args.op, x, y, prec, max(args.repeat, 1))
        print(json.dumps({"schedule": ctx.get_schedule(prec), "ms_per_launch": ms}))
    else:
        for _ in range(args.repeat):
            ctx.matvec(args.op, x, y, precision=prec)
    torch.cuda.synchronize()
    ctx.close()
    print("ok")


if __name__ == "__main__":
    main()
