"""Iterative and direct solves (oracle).

TEST INFRASTRUCTURE ONLY.

The paper applies filtering to operators that are then used by iterative solvers
(abstract, Sec. I) and studies the Calderon-preconditioned TE-EFIE
G^-1 S G^-1 N j = G^-1 S G^-1 E (Eq. 3). The solver itself is not specified; this is a
plain restarted GMRES (Saad & Schultz) with modified Gram-Schmidt and Givens rotations,
stopping on the relative residual of the system it is given.

Pins: GMRES against numpy.linalg.solve on random well-conditioned systems; the TM and TE
solutions against the cylinder series on circles.
"""
from __future__ import annotations

import numpy as np


def gmres(apply, b: np.ndarray, tol: float = 1e-10, restart: int = 50, max_iter: int = 2000, x0=None):
    """Restarted GMRES(restart). Returns (x, iterations, relative residual history)."""
    b = np.asarray(b, dtype=np.complex128)
    n = b.shape[0]
    x = np.zeros(n, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, [0.0]
    hist = []
    it = 0
    while it < max_iter:
        r = b - apply(x)
        beta = np.linalg.norm(r)
        hist.append(beta / bnorm)
        if beta / bnorm <= tol:
            break
        V = np.zeros((restart + 1, n), dtype=np.complex128)
        H = np.zeros((restart + 1, restart), dtype=np.complex128)
        cs = np.zeros(restart, dtype=np.complex128)
        sn = np.zeros(restart, dtype=np.complex128)
        g = np.zeros(restart + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(restart):
            w = apply(V[j])
            for i in range(j + 1):                       # modified Gram-Schmidt
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):                           # apply previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + np.conj(cs[i]) * H[i + 1, j]
                H[i, j] = t
            a, bb = H[j, j], H[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(bb) ** 2)
            cs[j] = np.conj(a) / den if den != 0 else 1.0
            sn[j] = np.conj(bb) / den if den != 0 else 0.0
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            j_done = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) / bnorm <= tol or it >= max_iter:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x = x + V[:j_done].T @ y
        if hist[-1] <= tol:
            r = b - apply(x)
            hist.append(np.linalg.norm(r) / bnorm)
            if hist[-1] <= tol * 10:
                break
    return x, it, hist


def dense_solve(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    return np.linalg.solve(A, b)


def assemble(apply, n: int) -> np.ndarray:
    """Dense matrix of a linear map, column by column (small n only)."""
    eye = np.eye(n, dtype=np.complex128)
    return np.stack([apply(eye[j]) for j in range(n)], axis=1)
