"""Spectral diagnostics (the singular-value studies of Sec. IV): operators assembled through the
GPU product equal the oracle's, and so do their singular values. The filtered S^alpha keeps the
modes |n| <= alpha a of a circle and drops the rest by many orders of magnitude (Fig. 2's
statement), where the unfiltered S keeps all of them.
"""
import math

import numpy as np
import pytest

import synth
from oracle import aim as oaim

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K = 2.0 * math.pi


@pytest.fixture(scope="module", params=[(8.0, 80, 48, 128), (12.0, 120, 64, 128)], ids=["p8_n80", "p12_n120"])
def circle(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2606_10784_gb300 import aim, diagnostics
    per, n, m, P = request.param
    a = per / (2.0 * math.pi)
    nodes = synth.circle_polygon(a, n)
    ctx = aim.Context(nodes, K, aim.TE, m, fft_P=P, alpha=2.0 * K)
    ref = oaim.TEOperators(nodes, K, m, P, alpha=2.0 * K, L=ctx.info()["L"])
    yield ctx, ref, diagnostics, n, a
    ctx.close()


@pytest.mark.parametrize("op", ["S", "S_alpha", "N_alpha", "calderon_alpha"])
def test_assembled_operator_and_singular_values_match_oracle(circle, op):
    ctx, ref, diag, n, a = circle
    A = diag.assemble(ctx, op, n, block=32)
    f = {"S": ref.S, "S_alpha": ref.S_alpha, "N_alpha": ref.N_alpha,
         "calderon_alpha": lambda v: ref.calderon(v, True)}[op]
    I = np.eye(n, dtype=np.complex128)
    B = np.stack([f(I[j]) for j in range(n)], axis=1)
    assert np.linalg.norm(A - B) <= 1e-10 * np.linalg.norm(B)
    sa, sb = np.linalg.svd(A, compute_uv=False), np.linalg.svd(B, compute_uv=False)
    assert np.max(np.abs(sa - sb)) <= 1e-9 * sb[0]


def test_filtered_single_layer_truncates_beyond_alpha_a(circle):
    ctx, ref, diag, n, a = circle
    s = diag.singular_values(ctx, "S", n)
    sa = diag.singular_values(ctx, "S_alpha", n)
    within = 2 * int(2.0 * K * a) + 1          # modes |n| <= alpha a
    assert diag.knee(s) == n                   # S: no knee
    assert within <= diag.knee(sa) <= within + 8
    assert sa[-1] < 1e-6 * sa[0]
