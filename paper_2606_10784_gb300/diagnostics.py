"""Spectral diagnostics of the AIM operators (the singular-value studies of Sec. IV, Figs. 2-3).

Singular values come from the library's Golub-Kahan-Lanczos bidiagonalisation on the GPU
(aim_lanczos_bidiag: every product through the grid product, both Lanczos bases reorthogonalised in
full in FP64). The k x k bidiagonal matrix it returns is small, and its SVD here gives the singular
values of the operator (all of them for k = n) and, with the Lanczos bases, its singular vectors
(one device GEMM).

Figs. 2-3 order the singular values "by the singular vectors of the Laplace-Beltrami operator on the
mesh". The reading taken here: the Laplace-Beltrami operator of the contour, discretised with the
same P1 hats (stiffness K_ij = int phi_i' phi_j', mass G of Eq. 3), has eigenvectors that run from
smooth to oscillating (Fourier modes of arc length on a smooth curve). Each singular vector of the
operator is matched to the Laplace-Beltrami eigenvector it overlaps most in the G inner product,
and the singular values are listed in the order of those eigenvalues. On a circle this is the
order of the mode number |n|, and the filtered spectrum then drops after |n| = alpha a.

The dense assembly of an operator (n batched products of unit vectors) is kept for small
cross-checks.

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


def start_vector(n: int, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


def lanczos_svd(ctx: aim.Context, op: str, n: int, k: int | None = None, precision: int = aim.FP64, seed: int = 0,
                vectors: bool = False):
    """Singular values (largest first) of `op` from k Lanczos steps on the GPU (k = n: all of them).
    With vectors=True also the right singular vectors, as an (n, k) complex128 numpy array."""
    import torch
    k = n if k is None else int(k)
    v0 = torch.from_numpy(start_vector(n, seed)).cuda()
    V = torch.empty((k + 1, n), dtype=torch.complex128, device="cuda") if vectors else None
    alpha, beta = ctx.lanczos_bidiag(op, k, v0, precision=precision, V=V)
    B = np.diag(alpha) + np.diag(beta[:k - 1], 1)
    if not vectors:
        return np.linalg.svd(B, compute_uv=False)
    _, s, Wh = np.linalg.svd(B)
    # A V_k = U_k B and B = Y diag(s) W^H: the right singular vectors of A are V_k W
    W = torch.from_numpy(np.ascontiguousarray(Wh.conj().T).astype(np.complex128)).cuda()
    vecs = (V[:k].transpose(0, 1) @ W).cpu().numpy()
    return s, vecs


def singular_values(ctx: aim.Context, op: str, n: int, precision: int = aim.FP64, seed: int = 0) -> np.ndarray:
    """All n singular values of `op`, largest first (n Lanczos steps)."""
    return lanczos_svd(ctx, op, n, None, precision, seed)


def laplace_beltrami(nodes: np.ndarray):
    """Eigenpairs of the contour's Laplace-Beltrami operator in the P1 hat basis: K x = lam G x with
    K_ii = 1/h_{i-1} + 1/h_i, K_{i,i+1} = -1/h_i (cyclic) and G the Gram matrix of Eq. 3. Returns
    eigenvalues ascending and G-orthonormal eigenvectors (columns). Dense: up to a few thousand hats."""
    from scipy.linalg import eigh
    nodes = np.asarray(nodes, dtype=np.float64)
    n = len(nodes)
    d = np.roll(nodes, -1, axis=0) - nodes
    h = np.hypot(d[:, 0], d[:, 1])
    K = np.zeros((n, n))
    G = np.zeros((n, n))
    for i in range(n):
        ip = (i + 1) % n
        K[i, i] += 1.0 / h[i]
        K[ip, ip] += 1.0 / h[i]
        K[i, ip] -= 1.0 / h[i]
        K[ip, i] -= 1.0 / h[i]
        G[i, i] += h[i] / 3.0
        G[ip, ip] += h[i] / 3.0
        G[i, ip] += h[i] / 6.0
        G[ip, i] += h[i] / 6.0
    lam, X = eigh(K, G)
    return lam, X, G


def lb_order(vecs: np.ndarray, lb_vecs: np.ndarray, G: np.ndarray) -> np.ndarray:
    """For each singular vector (column of vecs), the index of the Laplace-Beltrami eigenvector with
    the largest G-overlap |x^T G v|^2."""
    overlap = np.abs(lb_vecs.T @ (G @ vecs)) ** 2
    return np.argmax(overlap, axis=0)


def spectrum_by_lb(ctx: aim.Context, op: str, nodes: np.ndarray, k: int | None = None, precision: int = aim.FP64,
                   seed: int = 0):
    """Fig. 2/3 data: singular values of `op` listed in the order of their matched Laplace-Beltrami
    eigenvalues. Returns (lb_eigenvalue, lb_mode, sigma). lb_mode is the mode number of the matched
    eigenvector: a closed curve's Laplace-Beltrami eigenvalues are 0 and then pairs (a cosine-like and
    a sine-like mode), so eigenvector index i has mode number (i + 1) // 2, the |n| of e^{j n phi} on
    a circle."""
    n = len(nodes)
    s, vecs = lanczos_svd(ctx, op, n, k, precision, seed, vectors=True)
    lam, X, G = laplace_beltrami(nodes)
    idx = lb_order(vecs, X, G)
    order = np.argsort(idx, kind="stable")
    return lam[idx][order], (idx[order] + 1) // 2, s[order]


def knee(sv: np.ndarray, drop: float = 1e-3) -> int:
    """Number of singular values above drop * the largest (where the filtered spectrum falls off)."""
    return int(np.count_nonzero(sv > drop * np.max(sv)))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--perimeter", type=float, default=20.0, help="circle perimeter in wavelengths")
    ap.add_argument("--seg-per-wl", type=float, default=10.0)
    ap.add_argument("--m", type=int, default=128)
    ap.add_argument("--alpha-over-k", type=float, default=2.0)
    ap.add_argument("--op", default="S_alpha")
    ap.add_argument("--k", type=int, default=0, help="Lanczos steps (0: n)")
    args = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import synth
    k = 2.0 * math.pi
    a = args.perimeter / (2.0 * math.pi)
    n = int(round(args.perimeter * args.seg_per_wl))
    nodes = synth.circle_polygon(a, n)
    ctx = aim.Context(nodes, k, aim.TE, args.m, alpha=args.alpha_over_k * k)
    out = {"n": n, "radius_wl": a, "alpha_a": args.alpha_over_k * k * a,
           "modes_within_alpha": 2 * int(args.alpha_over_k * k * a) + 1}
    for op in dict.fromkeys([args.op, "S", "S_alpha"]):
        _, freq, s = spectrum_by_lb(ctx, op, nodes, args.k or None)
        out[op] = {"knee_1e-3": knee(s), "sv_head": [float(v) for v in s[:4]], "sv_tail": [float(v) for v in s[-4:]],
                   "last_lb_mode_above_1e-3": int(freq[s > 1e-3 * s.max()].max())}
    ctx.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
