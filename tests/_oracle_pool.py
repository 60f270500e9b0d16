"""The oracle's near-field corrections at large N, computed in a spawn process pool.

TEST INFRASTRUCTURE. The oracle's exact near-field entries (singular quadrature for every close
hat pair, then the AIM entry of the same pair subtracted) cost ~15 ms per row on one core, which
is minutes at N = 10^4. Rows are independent, so the parity tests split them over worker
processes; each worker builds the oracle's own operators and runs its own `_near_setup` on a
chunk of rows, unchanged. The pool uses the spawn start method: a process forked after CUDA has
been initialised in the parent can hang.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np
import scipy.sparse as sp


def _near_chunk(args):
    nodes, k, m, P, alpha, L, s, rows = args
    from oracle import aim as oaim
    ref = oaim.TEOperators(nodes, k, m, P, s=s, alpha=alpha, L=L, near=False, direct_dft=False)
    ref._near_setup(rows=rows)
    cs, cn = ref.CS.tocoo(), ref.CN.tocoo()
    return cs.row, cs.col, cs.data, cn.row, cn.col, cn.data


def te_near_matrices(nodes, k, m, P, alpha, L, s=4, workers=None):
    """(CS, CN): the oracle's near-field corrections of S and N for every row, as n x n CSR."""
    n = len(nodes)
    workers = workers or max(1, min(16, os.cpu_count() or 1))
    chunks = [c for c in np.array_split(np.arange(n), workers) if len(c)]
    args = [(np.asarray(nodes), float(k), int(m), int(P), float(alpha), float(L), int(s), c) for c in chunks]
    if len(chunks) == 1:
        parts = [_near_chunk(args[0])]
    else:
        with mp.get_context("spawn").Pool(len(chunks)) as pool:
            parts = pool.map(_near_chunk, args)
    cat = lambda i: np.concatenate([p[i] for p in parts])
    CS = sp.csr_matrix((cat(2), (cat(0), cat(1))), shape=(n, n))
    CN = sp.csr_matrix((cat(5), (cat(3), cat(4))), shape=(n, n))
    return CS, CN


def te_reference(nodes, k, m, P, alpha, L, s=4, workers=None):
    """The oracle's TE operators with the near field of every row attached."""
    from oracle import aim as oaim
    ref = oaim.TEOperators(nodes, k, m, P, s=s, alpha=alpha, L=L, near=False, direct_dft=False)
    ref.CS, ref.CN = te_near_matrices(nodes, k, m, P, alpha, L, s=s, workers=workers)
    return ref


def check_rows(got, want, tol, what=""):
    """Row-by-row comparison: the largest error of any single output row, relative to the largest
    entry of the vector, and the normwise relative error, both within tol."""
    got = np.asarray(got)
    want = np.asarray(want)
    err = np.abs(got - want)
    scale = np.abs(want).max()
    worst = int(np.argmax(err))
    assert err.max() <= tol * scale, "%s: row %d off by %.3e of max|y| (tol %.0e)" % (what, worst, err.max() / scale, tol)
    rel = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert rel <= tol, "%s: relative L2 %.3e (tol %.0e)" % (what, rel, tol)
    return float(err.max() / scale), float(rel)
