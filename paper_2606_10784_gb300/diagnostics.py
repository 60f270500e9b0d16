"""Spectral diagnostics of the AIM operators (the singular-value studies of Sec. IV, Figs. 2-3).

An operator (S, S^alpha, N, N^alpha, the Calderon products, ...) is assembled column by column
through the library's batched product: `block` unit vectors per launch, so every column comes
from the same kernels a solve uses. Its singular values then come from a dense SVD, a library
routine applied to the assembled matrix. This is a diagnostic, not the hot path: assembly costs
n / block batched products and the SVD O(n^3), which suits contours of up to a few thousand
unknowns.

    python -m paper_2606_10784_gb300.diagnostics --perimeter 20 --op S_alpha
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

import numpy as np

from . import aim


def assemble(ctx: aim.Context, op: str, n: int, precision: int = aim.FP64, block: int = 64) -> np.ndarray:
    """The n x n matrix of `op` (complex128): column j is op applied to the j-th unit vector."""
    import torch
    A = np.empty((n, n), dtype=np.complex128)
    for j0 in range(0, n, block):
        nb = min(block, n - j0)
        x = torch.zeros((nb, n), dtype=torch.complex128, device="cuda")
        x[torch.arange(nb), torch.arange(j0, j0 + nb)] = 1.0
        y = torch.empty_like(x)
        ctx.matvec(op, x, y, precision=precision)
        A[:, j0:j0 + nb] = y.cpu().numpy().T
    return A


def singular_values(ctx: aim.Context, op: str, n: int, precision: int = aim.FP64, block: int = 64) -> np.ndarray:
    """Singular values of `op`, largest first."""
    return np.linalg.svd(assemble(ctx, op, n, precision, block), compute_uv=False)


def knee(sv: np.ndarray, drop: float = 1e-3) -> int:
    """Number of singular values above drop * the largest (where the filtered spectrum falls off)."""
    return int(np.count_nonzero(sv > drop * sv[0]))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--perimeter", type=float, default=20.0, help="circle perimeter in wavelengths")
    ap.add_argument("--seg-per-wl", type=float, default=10.0)
    ap.add_argument("--m", type=int, default=128)
    ap.add_argument("--alpha-over-k", type=float, default=2.0)
    ap.add_argument("--op", default="S_alpha")
    args = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import synth
    k = 2.0 * math.pi
    a = args.perimeter / (2.0 * math.pi)
    n = int(round(args.perimeter * args.seg_per_wl))
    ctx = aim.Context(synth.circle_polygon(a, n), k, aim.TE, args.m, alpha=args.alpha_over_k * k)
    sv = {op: singular_values(ctx, op, n) for op in dict.fromkeys([args.op, "S", "S_alpha"])}
    ctx.close()
    out = {"n": n, "radius_wl": a, "alpha_a": args.alpha_over_k * k * a,
           "modes_within_alpha": 2 * int(args.alpha_over_k * k * a) + 1,
           "knee_1e-3": {op: knee(s) for op, s in sv.items()},
           "sv_head": {op: [float(v) for v in s[:4]] for op, s in sv.items()},
           "sv_tail": {op: [float(v) for v in s[-4:]] for op, s in sv.items()}}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
