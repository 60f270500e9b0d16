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


# --------------------------------------------------------------------------------------
# Golub-Kahan-Lanczos on the GPU (aim_lanczos_bidiag) against the SVD of the oracle's operators
# --------------------------------------------------------------------------------------
LZ_CASES = [
    ("circle_p8_n80", lambda: synth.circle_polygon(8.0 / (2 * math.pi), 80), 48, 128, 2.0),
    ("star_p20_n200", lambda: synth.StarContour.from_seed(3).polygon(20.0, 200), 96, 256, 2.0),
    ("star_p40_n400", lambda: synth.StarContour.from_seed(5).polygon(40.0, 400), 128, 256, 2.5),
]


@pytest.fixture(scope="module", params=LZ_CASES, ids=[c[0] for c in LZ_CASES])
def lz_case(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2606_10784_gb300 import aim, diagnostics
    _, mk, m, P, ak = request.param
    nodes = mk()
    ctx = aim.Context(nodes, K, aim.TE, m, fft_P=P, alpha=ak * K)
    ref = oaim.TEOperators(nodes, K, m, P, alpha=ak * K, L=ctx.info()["L"])
    n = len(nodes)
    I = np.eye(n, dtype=np.complex128)
    mats = {"S_alpha": np.stack([ref.S_alpha(I[j]) for j in range(n)], axis=1),
            "calderon_alpha": np.stack([ref.calderon(I[j], True) for j in range(n)], axis=1),
            "N": np.stack([ref.N(I[j]) for j in range(n)], axis=1)}
    svs = {op: np.linalg.svd(A, compute_uv=False) for op, A in mats.items()}
    yield ctx, nodes, svs, diagnostics, aim
    ctx.close()


@pytest.mark.parametrize("precision", [0, 2])
@pytest.mark.parametrize("op", ["S_alpha", "calderon_alpha", "N"])
def test_lanczos_gives_every_singular_value_of_the_oracle_operator(lz_case, op, precision):
    ctx, nodes, svs, diag, aim = lz_case
    s = diag.lanczos_svd(ctx, op, len(nodes), precision=precision)
    want = svs[op]
    assert np.max(np.abs(s - want)) <= 1e-9 * want[0], np.max(np.abs(s - want)) / want[0]


def test_lanczos_mixed_precision_singular_values(lz_case):
    ctx, nodes, svs, diag, aim = lz_case
    s = diag.lanczos_svd(ctx, "S_alpha", len(nodes), precision=aim.MIXED)
    want = svs["S_alpha"]
    assert np.max(np.abs(s - want)) <= 1e-5 * want[0]


def test_truncated_lanczos_converges_on_the_largest_singular_values(lz_case):
    ctx, nodes, svs, diag, aim = lz_case
    n = len(nodes)
    s = diag.lanczos_svd(ctx, "calderon_alpha", n, k=n // 2)
    want = svs["calderon_alpha"]
    assert np.max(np.abs(s[:8] - want[:8])) <= 1e-8 * want[0]


def test_spectrum_ordered_by_laplace_beltrami_drops_after_alpha_a():
    # Fig. 2: ordered by the Laplace-Beltrami eigenvectors (mode number |n| on a circle), the
    # singular values of S^alpha stay within a few decades up to |n| ~ alpha a and fall by many
    # orders of magnitude after it, while those of S do not fall
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2606_10784_gb300 import aim, diagnostics
    a = 20.0 / (2 * math.pi)
    n = 200
    nodes = synth.circle_polygon(a, n)
    ctx = aim.Context(nodes, K, aim.TE, 96, alpha=2.0 * K)
    na = 2.0 * K * a                          # alpha a = 40
    _, freq, s = diagnostics.spectrum_by_lb(ctx, "S_alpha", nodes)
    _, freq_u, su = diagnostics.spectrum_by_lb(ctx, "S", nodes)
    ctx.close()
    assert np.all(np.diff(freq) >= 0)
    top = s.max()
    assert np.all(s[freq <= na - 3] > 1e-3 * top)
    assert np.all(s[freq >= na + 8] < 1e-5 * top)
    assert np.all(su > 1e-3 * su.max())
