"""Parity at the full single-solve size (perimeter 1000 wavelengths, N = 10000, 2048^2 grid,
P = 4096, alpha = 2k), in the launch configuration the benchmark times (one vector, default
schedule), in all three precisions.

The oracle applies every operator whole here: its FFT product (Eq. 8 / Eq. 10, a library FFT as
one step) at P = 4096 takes a fraction of a second, and the near-field correction of every row
is computed by the oracle's own `_near_setup`, spread over a spawn process pool. Every output
row is compared (row by row and normwise), so every band of grid rows is covered.
Tolerances: 1e-10 for FP64 (double-float) and native binary64, 1e-5 for mixed precision.
"""
import numpy as np
import pytest

import synth
from _oracle_pool import check_rows, te_reference

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 1e-5, 2: 1e-10}


@pytest.fixture(scope="module")
def fullsize():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2606_10784_gb300 import aim
    wl = synth.single_solve_scale(0)
    ctx = aim.Context(wl.nodes, wl.k, aim.TE, wl.m, fft_P=wl.fft_P, alpha=wl.alpha)
    ref = te_reference(wl.nodes, wl.k, wl.m, wl.fft_P, wl.alpha, ctx.info()["L"])
    x = synth.random_coeffs(wl.n, 1, seed=4)[0]
    yield wl, ctx, ref, x, aim
    ctx.close()


def gpu_apply(ctx, op, x, precision):
    xd = torch.from_numpy(x[None]).cuda()
    yd = torch.empty_like(xd)
    ctx.matvec(op, xd, yd, precision=precision)
    torch.cuda.synchronize()
    return yd.cpu().numpy()[0]


OPS = {
    "S_alpha": lambda ref, x: ref.S_alpha(x),
    "N": lambda ref, x: ref.N(x),
    "N_alpha": lambda ref, x: ref.N_alpha(x),
    "S": lambda ref, x: ref.S(x),
    "calderon_alpha": lambda ref, x: ref.calderon(x, filtered=True),
    "calderon": lambda ref, x: ref.calderon(x, filtered=False),
    "calderon_alpha2": lambda ref, x: ref.calderon_both(x),
}


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("op", list(OPS))
def test_fullsize_operator_every_row(fullsize, op, precision):
    wl, ctx, ref, x, aim = fullsize
    want = OPS[op](ref, x)
    got = gpu_apply(ctx, op, x, precision)
    check_rows(got, want, TOL[precision], "%s precision %d" % (op, precision))


def test_fullsize_near_field_pattern_matches_oracle(fullsize):
    wl, ctx, ref, x, aim = fullsize
    assert ctx.info()["nnz_near"] == ref.CN.nnz


def test_fullsize_gram_inverse(fullsize):
    wl, ctx, ref, x, aim = fullsize
    got = gpu_apply(ctx, "gram_inv", x, 0)
    check_rows(got, ref.gram_solve(x), 1e-12, "gram_inv")
