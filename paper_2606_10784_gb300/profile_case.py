"""Runs one grid product on the single-solve workload, for kernel profilers.

    python -m paper_2606_10784_gb300.profile_case --precision fp64 --op N --repeat 1

Sets up the perimeter-1000-wavelength contour (N = 10000 unknowns, 2048 x 2048 grid, P = 4096,
alpha = 2k), applies the chosen operator `repeat` times to a seeded random vector and exits.
The first k_col_conv launch is the operator's first column pass (3 channels for N, 1 for
S_alpha), so `ncu -k regex:k_col_conv -c 1` captures exactly one full-size launch.
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--precision", choices=["fp64", "mixed", "native"], default="fp64")
    ap.add_argument("--op", default="N")
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--nrhs", type=int, default=1)
    args = ap.parse_args(argv)
    import torch

    import synth
    from paper_2606_10784_gb300 import aim
    prec = {"fp64": aim.FP64, "mixed": aim.MIXED, "native": aim.FP64_NATIVE}[args.precision]
    wl = synth.single_solve_scale(0)
    ctx = aim.Context(wl.nodes, wl.k, aim.TE, wl.m, fft_P=wl.fft_P, alpha=wl.alpha)
    x = torch.from_numpy(synth.random_coeffs(wl.n, args.nrhs, 0)).cuda()
    y = torch.empty_like(x)
    for _ in range(args.repeat):
        ctx.matvec(args.op, x, y, precision=prec)
    torch.cuda.synchronize()
    ctx.close()
    print("ok")


if __name__ == "__main__":
    main()
