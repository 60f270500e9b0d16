"""The analytic filter of Eq. 6 on the grid (Sec. III-B, Fig. 1a) against the oracle.

The library samples g^alpha(eps sqrt(i^2+j^2)) in FP64 (pole subtracted, composite Gauss), the
oracle by QUADPACK's Cauchy-weight rule: the samples and their DFT must agree to 1e-10. A context
set up with AIM_FILTER_ANALYTIC uses that spectrum for its filtered operators, which must match the
oracle's analytic-filter operators (1e-10 in the FP64 modes, 1e-5 mixed). The unfiltered and the
numerically filtered spectra (Eq. 10) are read out and checked the same way, and Fig. 1's
comparison (circle, m = 50) is printed: the two filters agree inside the disc, and beyond alpha the
analytic spectrum keeps only the ringing of the finite grid window.
"""
import math

import numpy as np
import pytest

import synth
from oracle import aim as oaim

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K = 2.0 * math.pi
TOL = {0: 1e-10, 1: 1e-5, 2: 1e-10}

CASES = [
    # Fig. 1: a circle, m = 50 (P = 128), alpha = 8k as in the paper's experiments
    ("fig1_circle_m50", lambda: synth.circle_polygon(1.0, 200), 50, 0, 8.0),
    ("star_m32_P64", lambda: synth.StarContour.from_seed(0).polygon(6.0, 80), 32, 64, 3.0),
    ("star_m64_P256", lambda: synth.StarContour.from_seed(2).polygon(12.0, 150), 64, 256, 2.5),
    ("circle_m128_P256", lambda: synth.circle_polygon(1.0, 256), 128, 256, 4.0),
]


@pytest.fixture(scope="module")
def aimlib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2606_10784_gb300 import aim
    return aim


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def case(request, aimlib):
    name, mk, m, P, ak = request.param
    nodes = mk()
    an = aimlib.Context(nodes, K, aimlib.TE, m, fft_P=P, alpha=ak * K, filter_kind=aimlib.FILTER_ANALYTIC)
    nu = aimlib.Context(nodes, K, aimlib.TE, m, fft_P=P, alpha=ak * K)
    inf = an.info()
    assert inf["filter_kind"] == aimlib.FILTER_ANALYTIC and nu.info()["filter_kind"] == aimlib.FILTER_NUMERICAL
    ref = oaim.TEOperators(nodes, K, m, inf["fft_P"], alpha=ak * K, L=inf["L"], filter_kind="analytic")
    yield name, nodes, an, nu, ref, inf
    an.close()
    nu.close()


def table(ctx, which, H):
    out = torch.empty((H + 1, H + 1), dtype=torch.complex128, device="cuda")
    ctx.kernel_table(which, out)
    return out.cpu().numpy()


def test_analytic_samples_and_spectrum_match_oracle(aimlib, case):
    name, nodes, an, nu, ref, inf = case
    H = inf["fft_P"] // 2
    want = ref.c_an[:H + 1, :H + 1]
    got = table(an, aimlib.TABLE_ANALYTIC_SAMPLES, H)
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max(), np.abs(got - want).max()
    # the same table from a context without the analytic filter (computed on demand)
    assert np.array_equal(table(nu, aimlib.TABLE_ANALYTIC_SAMPLES, H), got)
    spec = ref.Chat_alpha[:H + 1, :H + 1]
    for ctx, which in ((an, aimlib.TABLE_SPECTRUM_FILTERED), (nu, aimlib.TABLE_ANALYTIC_SPECTRUM)):
        g = table(ctx, which, H)
        assert np.linalg.norm(g - spec) <= 1e-10 * np.linalg.norm(spec)


def test_unfiltered_and_numerical_spectra_match_oracle(aimlib, case):
    name, nodes, an, nu, ref, inf = case
    H = inf["fft_P"] // 2
    for which, want in ((aimlib.TABLE_SPECTRUM, ref.Chat), (aimlib.TABLE_SPECTRUM_FILTERED, ref.Chat * ref.mask)):
        w = want[:H + 1, :H + 1]
        g = table(nu, which, H)
        assert np.linalg.norm(g - w) <= 1e-10 * np.linalg.norm(w), which


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_analytic_filter_operators_match_oracle(aimlib, case, precision):
    name, nodes, an, nu, ref, inf = case
    x = synth.random_coeffs(len(nodes), 2, seed=13)
    xd = torch.from_numpy(x).cuda()
    for op, f in (("S_alpha", ref.S_alpha), ("N_alpha", ref.N_alpha),
                  ("calderon_alpha", lambda v: ref.calderon(v, filtered=True))):
        yd = torch.empty_like(xd)
        an.matvec(op, xd, yd, precision=precision)
        torch.cuda.synchronize()
        got = yd.cpu().numpy()
        for r in range(2):
            want = f(x[r])
            assert np.linalg.norm(got[r] - want) <= TOL[precision] * np.linalg.norm(want), (op, r)


def test_fig1_numerical_against_analytic_spectrum(aimlib, case):
    # Fig. 1: F(c_grid) with the analytic filter (a) and with the numerical truncation (b)
    name, nodes, an, nu, ref, inf = case
    if not name.startswith("fig1"):
        pytest.skip("Fig. 1 case only")
    H = inf["fft_P"] // 2
    A = table(nu, aimlib.TABLE_ANALYTIC_SPECTRUM, H)
    B = table(nu, aimlib.TABLE_SPECTRUM_FILTERED, H)
    P = inf["fft_P"]
    p = np.arange(H + 1)
    kap = (2 * math.pi / (P * inf["eps"])) * np.hypot(p[:, None], p[None, :])
    alpha = inf["alpha"]
    inside = (kap < 0.9 * alpha) & (np.abs(kap - K) > 0.3 * K)
    outside = kap > 1.1 * alpha
    pass_diff = np.linalg.norm((A - B)[inside]) / np.linalg.norm(B[inside])
    ring = np.abs(A[outside]).max() / np.abs(B[inside]).max()
    print("Fig. 1 (circle, m = 50, alpha = 8k): passband rel. difference %.3e, analytic ringing beyond "
          "1.1 alpha %.3e of the passband maximum, numerical beyond alpha: %s" %
          (pass_diff, ring, "zero" if np.all(B[kap > alpha * (1 + 1e-12)] == 0) else "nonzero"))
    assert np.all(B[kap > alpha * (1 + 1e-12)] == 0)
    assert pass_diff < 0.2 and ring < 0.05
