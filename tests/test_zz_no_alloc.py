"""The no-allocation grid product (aim_grid_product_noalloc) against the allocating one.

Callers that cannot allocate device memory at call time (inside a CUDA graph capture, in
real-time loops with a fixed device footprint) use aim_grid_product_noalloc, whose scratch is a
fixed array inside the library. It must give what aim_grid_product gives, call after call (the
array keeps the previous call's contents, which must not leak into the next result), and it
must refuse batches whose intermediate grid does not fit the array.
"""
import math

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K = 2.0 * math.pi


@pytest.fixture(scope="module")
def aimlib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2606_10784_gb300 import aim
    return aim


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-6), (2, 1e-12)])
def test_noalloc_matches_allocating_product_on_consecutive_calls(aimlib, precision, tol):
    nodes = synth.StarContour.from_seed(7).polygon(12.0, 160)
    ctx = aimlib.Context(nodes, K, aimlib.TE, 64, fft_P=128, alpha=3.0 * K)
    inf = ctx.info()
    rows = slice(inf["row_lo"], inf["row_hi"] + 1)
    for call, seed in enumerate((1, 2)):          # two calls in a row, different inputs
        u = synth.random_grid(64, 2, seed=seed)
        u[:, :inf["row_lo"], :] = 0
        u[:, inf["row_hi"] + 1:, :] = 0
        ud = torch.from_numpy(u).cuda()
        for filtered in (False, True):
            want = torch.empty_like(ud)
            ctx.grid_product(ud, want, filtered, precision=precision)
            got = torch.full_like(ud, float("nan"))
            ctx.grid_product_noalloc(ud, got, filtered, precision=precision)
            torch.cuda.synchronize()
            w = want.cpu().numpy()[:, rows]
            g = got.cpu().numpy()[:, rows]
            assert np.all(np.isfinite(g)), (call, filtered)
            assert np.linalg.norm(g - w) <= tol * np.linalg.norm(w), (call, filtered)
    ctx.close()


def test_noalloc_rejects_batches_beyond_its_scratch(aimlib):
    nodes = synth.circle_polygon(20.0, 1200)
    ctx = aimlib.Context(nodes, K, aimlib.TE, 512, alpha=2.0 * K)
    inf = ctx.info()
    per_grid = inf["fft_P"] * (inf["row_hi"] - inf["row_lo"] + 1) * 16
    nrhs = (16 << 20) // per_grid + 1           # one grid more than the scratch holds
    u = torch.zeros((nrhs, 512, 512), dtype=torch.complex128, device="cuda")
    v = torch.empty_like(u)
    with pytest.raises(aimlib.AimError) as exc:
        ctx.grid_product_noalloc(u, v, True, precision=0)
    assert exc.value.status == aimlib.EINVAL
    assert "scratch" in str(exc.value)
    ctx.close()
