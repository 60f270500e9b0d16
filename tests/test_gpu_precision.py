"""Mixed precision at the single-solve size: the grid products in complex64, with FP64 kept for
the spectra, the near-field entries, Arnoldi and the outer residual, refined to 1e-5.

The contour is a circle of perimeter 1000 wavelengths (N = 10000, 2048^2 grid, P = 4096,
alpha = 2k), so the closed-form cylinder current (Jacobi-Anger expansion over the eigenvalues
mu_n of N, Eq. 2) is known. The filtered Calderon system (Eq. 3 with S^alpha of Eq. 10) is
solved three ways: FP64 (double-float grid), native binary64, and mixed. The FP64 operators equal
the oracle's to 1e-10 at this size (sampled rows). Each solution's residual is taken under the FP64
operator, and each is compared with the others and with the series. The figures are printed for
the record (`pytest -s`).

At 1000 wavelengths and 10 segments per wavelength the discretisation's phase (pollution) error
dominates the distance to the series: ~18 % for the unfiltered Calderon solution, which solves
its discrete system N x = E to ~3e-4, and ~13 % for the filtered one (the filter also leaves the
modes beyond alpha a loosely determined, Secs. III-B, IV). What precision must not do is change
that error: mixed, native and FP64 agree with the series to within 10 % of each other.
"""
import math

import numpy as np
import pytest

import synth
from oracle import special

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K = 2.0 * math.pi
PERIMETER = 1000.0
N = 10000
M_GRID, P_FFT = 2048, 4096
TOL = 1e-5
UNF_TOL = 1e-8


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def circle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2606_10784_gb300 import aim
    a = PERIMETER / (2.0 * math.pi)
    nodes = synth.circle_polygon(a, N)
    ctx = aim.Context(nodes, K, aim.TE, M_GRID, fft_P=P_FFT, alpha=2.0 * K)
    E = torch.empty((1, N), dtype=torch.complex128, device="cuda")
    ctx.rhs_planewave([0.0], E)
    series = special.te_cylinder_current(2.0 * math.pi * np.arange(N) / N, K * a, a)
    sols = {}
    for name, prec in (("fp64", aim.FP64), ("native", aim.FP64_NATIVE), ("mixed", aim.MIXED)):
        x = torch.zeros_like(E)
        info = ctx.solve("calderon_alpha", E, x, tol=TOL, restart=3000, max_iter=6000, precision=prec,
                         inner_tol=0.0)
        sols[name] = (x, info[0])
    # control: the filtered system solved again in FP64 from another starting guess (a small random
    # vector), to show how far apart two FP64 solutions at the same tolerance lie
    x0 = torch.from_numpy(synth.random_coeffs(N, 1, seed=17)).cuda()
    x0 *= 1e-2 * torch.linalg.norm(sols["fp64"][0]) / torch.linalg.norm(x0)
    info = ctx.solve("calderon_alpha", E, x0, tol=TOL, restart=3000, max_iter=6000, precision=aim.FP64,
                     x0_given=True)
    sols["fp64_x0"] = (x0, info[0])
    # the unfiltered Calderon system (lambda_n mu_n -> 1/4, well conditioned): solved to 1e-8 in
    # FP64 and in mixed precision, so that the distance between the two solutions shows the
    # precision, not the solver tolerance
    for name, prec in (("unfiltered", aim.FP64), ("unfiltered_mixed", aim.MIXED)):
        x = torch.zeros_like(E)
        info = ctx.solve("calderon", E, x, tol=UNF_TOL, restart=3000, max_iter=6000, precision=prec, inner_tol=0.0)
        sols[name] = (x, info[0])
    yield ctx, aim, E, series, sols
    ctx.close()


def apply(ctx, op, x):
    y = torch.empty_like(x)
    ctx.matvec(op, x, y, precision=0)
    torch.cuda.synchronize()
    return y


def test_all_precisions_converge_and_solve_the_fp64_system(circle):
    ctx, aim, E, series, sols = circle
    b = apply(ctx, "gram_inv", apply(ctx, "S_alpha", apply(ctx, "gram_inv", E)))
    bn = torch.linalg.norm(b).item()
    for name, (x, info) in sols.items():
        assert info["converged"] == 1, (name, info)
        if name.startswith("unfiltered"):
            continue
        r = torch.linalg.norm(b - apply(ctx, "calderon_alpha", x)).item() / bn
        print("precision %-6s: iters %5d outer %2d  residual under FP64 operator %.3e" %
              (name, info["iters"], info["outer_iters"], r))
        assert r <= 1.05 * TOL


def test_mixed_against_fp64_and_series(circle):
    ctx, aim, E, series, sols = circle
    xs = {k: v[0].cpu().numpy()[0] for k, v in sols.items()}
    en = np.linalg.norm(E.cpu().numpy())
    err = {}
    for name, x in xs.items():
        nres = np.linalg.norm(apply(ctx, "N", sols[name][0]).cpu().numpy()[0] - E.cpu().numpy()[0]) / en
        err[name] = rel(x, series)
        print("precision %-6s: rel L2 vs cylinder series %.3e   ||N x - E||/||E|| %.3e" % (name, err[name], nres))
    d_mixed = rel(xs["mixed"], xs["fp64"])
    d_native = rel(xs["native"], xs["fp64"])
    print("rel L2 mixed vs fp64 %.3e, native vs fp64 %.3e" % (d_mixed, d_native))
    # precision changes the series error by far less than the error itself
    for name in xs:
        assert err[name] < 0.3
    assert abs(err["mixed"] - err["fp64"]) < 0.1 * err["fp64"]
    assert abs(err["native"] - err["fp64"]) < 1e-3 * err["fp64"]
    assert d_mixed < 0.1


def test_mixed_equals_fp64_on_the_well_conditioned_system(circle):
    # the metric's "rel err <= 1e-5 after refinement", on a system whose solution is determined to
    # that accuracy by its residual: the unfiltered Calderon product
    ctx, aim, E, series, sols = circle
    x64 = sols["unfiltered"][0].cpu().numpy()[0]
    x32 = sols["unfiltered_mixed"][0].cpu().numpy()[0]
    d = rel(x32, x64)
    print("unfiltered Calderon, tol %.0e: mixed vs FP64 rel L2 %.3e (iters %d / %d, outer %d)" %
          (UNF_TOL, d, sols["unfiltered"][1]["iters"], sols["unfiltered_mixed"][1]["iters"],
           sols["unfiltered_mixed"][1]["outer_iters"]))
    assert d <= 1e-5


def test_filtered_solutions_agree_on_the_modes_the_filter_keeps(circle):
    # The filtered system compresses the circle's Fourier modes |n| > alpha a (Sec. III-B, Fig. 2), so
    # the distance between solutions is reported on the modes the filter keeps as well as whole. It
    # does not shrink there: two solutions with FP64 residuals below 1e-5 part where the system is
    # least determined, the modes around n = ka (ka = 1000 here), and a second FP64 solve from another
    # starting guess parts from the first in the same modes. The statement of accuracy at this size
    # is therefore the residual under the FP64 operator (test above) and the well-conditioned system
    # (unfiltered Calderon, test above); these figures are the record the precision study asks for.
    ctx, aim, E, series, sols = circle
    a = PERIMETER / (2.0 * math.pi)
    ka = K * a
    na = 2.0 * K * a                              # alpha a with alpha = 2k
    n_idx = np.abs(np.fft.fftfreq(N, 1.0 / N))
    spec = {k: np.fft.fft(v[0].cpu().numpy()[0]) for k, v in sols.items()}
    ref = spec["fp64"]
    bands = {"|n| <= alpha a": n_idx <= na, "|n| <= 0.9 ka": n_idx <= 0.9 * ka,
             "|n| <= 0.5 ka": n_idx <= 0.5 * ka}
    near_ka = (n_idx >= 0.9 * ka) & (n_idx <= 1.1 * ka)
    out = {}
    for name in ("mixed", "native", "fp64_x0"):
        d = np.abs(spec[name] - ref) ** 2
        out[name] = {b: float(np.sqrt(d[m].sum() / (np.abs(ref[m]) ** 2).sum())) for b, m in bands.items()}
        share = d[near_ka].sum() / d.sum()
        print("filtered, %-7s vs fp64: %s; whole vector %.3e; share of the difference in 0.9 ka <= |n| <= 1.1 ka: "
              "%.0f%%" % (name, ", ".join("%s %.2e" % kv for kv in out[name].items()), rel(spec[name], ref),
                           100 * share))
    # native and double-float FP64 follow the same Krylov path (the same arithmetic up to ~1e-14)
    assert out["native"]["|n| <= alpha a"] <= 1e-4
    assert out["mixed"]["|n| <= alpha a"] <= 5e-2
