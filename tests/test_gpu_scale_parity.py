"""Operator parity at the sizes the batching and serving workloads run, which the small parity
cases do not reach: the batching contour (perimeter 400 wavelengths, N = 4000, 1024^2 grid,
P = 2048) with all 64 plane waves in one batched launch under the autotuned schedule, as the
benchmark runs it, and serving-sized grids (P = 512 and P = 1024) at wavenumbers other than 2 pi.

Every output row of each compared vector is checked against the oracle (FFT product, near field
of every row from a spawn process pool); 1e-10 in the FP64 modes, 1e-5 in mixed precision.
"""
import math

import numpy as np
import pytest

import synth
from _oracle_pool import check_rows, te_reference
from oracle import dense

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 1e-5, 2: 1e-10}


@pytest.fixture(scope="module")
def aimlib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2606_10784_gb300 import aim
    return aim


@pytest.fixture(scope="module")
def batching(aimlib):
    wl = synth.batching_scale(0, nrhs=64)
    ctx = aimlib.Context(wl.nodes, wl.k, aimlib.TE, wl.m, fft_P=wl.fft_P, alpha=wl.alpha)
    ref = te_reference(wl.nodes, wl.k, wl.m, wl.fft_P, wl.alpha, ctx.info()["L"])
    E = np.stack([dense.te_rhs(wl.nodes, wl.k, th) for th in wl.angles])
    yield wl, ctx, ref, E
    ctx.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("op", ["calderon_alpha", "N", "S_alpha"])
def test_batching_size_64_plane_waves_in_one_launch(aimlib, batching, op, precision):
    wl, ctx, ref, E = batching
    ctx.autotune(nrhs=64, precision=precision)
    xd = torch.from_numpy(E).cuda()
    yd = torch.empty_like(xd)
    ctx.matvec(op, xd, yd, precision=precision)
    torch.cuda.synchronize()
    got = yd.cpu().numpy()
    f = {"calderon_alpha": lambda v: ref.calderon(v, filtered=True), "N": ref.N, "S_alpha": ref.S_alpha}[op]
    for r in range(0, 64, 8):          # 8 of the 64 plane waves, spread over the batch
        check_rows(got[r], f(E[r]), TOL[precision], "%s rhs %d precision %d" % (op, r, precision))


SERVING = [
    # (perimeter in wavelengths, N, m, k): P = 2m
    ("p512_k3", 40.0, 400, 256, 3.0),
    ("p1024_k10", 150.0, 1500, 512, 10.0),
]


@pytest.fixture(scope="module", params=SERVING, ids=[c[0] for c in SERVING])
def serving_case(request, aimlib):
    _, per, n, m, k = request.param
    wl_len = 2.0 * math.pi / k
    nodes = synth.StarContour.from_seed(n).polygon(per * wl_len, n)
    eps_guess = 2.0 * np.abs(nodes).max() / (m - 7)
    alpha = max(1.05 * k, min(8.0 * k, (2.0 / 3.0) * math.pi / eps_guess))
    ctx = aimlib.Context(nodes, k, aimlib.TE, m, alpha=alpha)
    inf = ctx.info()
    assert inf["fft_P"] == 2 * m
    ref = te_reference(nodes, k, m, inf["fft_P"], alpha, inf["L"])
    yield nodes, k, ctx, ref
    ctx.close()


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_serving_sized_grids(aimlib, serving_case, precision):
    nodes, k, ctx, ref = serving_case
    x = synth.random_coeffs(len(nodes), 3, seed=31)
    xd = torch.from_numpy(x).cuda()
    for op, f in (("S", ref.S), ("S_alpha", ref.S_alpha), ("N", ref.N), ("N_alpha", ref.N_alpha),
                  ("calderon_alpha", lambda v: ref.calderon(v, filtered=True))):
        yd = torch.empty_like(xd)
        ctx.matvec(op, xd, yd, precision=precision)
        torch.cuda.synchronize()
        got = yd.cpu().numpy()
        for r in range(3):
            check_rows(got[r], f(x[r]), TOL[precision], "%s rhs %d precision %d" % (op, r, precision))
