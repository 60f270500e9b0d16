"""The no-allocation grid product (aim_grid_product_noalloc) against the allocating one.

Some callers cannot allocate device memory when they need a product: real-time loops whose
device memory is fixed before they start, hosts that forbid cudaMalloc after start-up, and code
inside another runtime's memory pool. They use aim_grid_product_noalloc, whose scratch is a
fixed array inside the library. It runs the same kernels in the same order as aim_grid_product,
so it must give the same bits, call after call (the array keeps the previous call's contents,
which must not leak into the next result); it must leave the device's free memory unchanged; and
it must refuse batches whose intermediate grid does not fit the array.

This file is collected last, so a run that stops at its first failure has run every other test.
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


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_noalloc_matches_allocating_product_on_consecutive_calls(aimlib, precision):
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
            assert bool(torch.isfinite(got[:, rows]).all()), (call, filtered)
            assert torch.equal(got[:, rows], want[:, rows]), (call, filtered)
    ctx.close()


def test_noalloc_calls_leave_free_device_memory_unchanged(aimlib):
    nodes = synth.circle_polygon(5.0, 300)
    ctx = aimlib.Context(nodes, K, aimlib.TE, 96, alpha=3.0 * K)
    u = torch.from_numpy(synth.random_grid(96, 1, seed=3)).cuda()
    v = torch.empty_like(u)
    inf = ctx.info()
    u[:, :inf["row_lo"], :] = 0
    u[:, inf["row_hi"] + 1:, :] = 0
    # the first calls look up the array on this device and load each precision's kernels (lazy
    # module loading commits device memory for code once per process)
    for precision in (0, 1, 2):
        ctx.grid_product_noalloc(u, v, True, precision=precision)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for precision in (0, 1, 2, 0):
        ctx.grid_product_noalloc(u, v, True, precision=precision)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
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
