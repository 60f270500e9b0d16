"""Setup blobs through the device: a context imported from aim_export_setup's blob gives the same
bits as the context that wrote it (every operator, every precision, the kernel tables, a solve),
a blob of another problem or a corrupted one is refused, and the on-disk cache and the server
reload contexts after a restart.
"""
import math
import time

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K = 2.0 * math.pi

CASES = [
    # (id, contour, form, m, kwargs, operators)
    ("te_star_numerical", lambda: synth.StarContour.from_seed(6).polygon(30.0, 300), 1, 96,
     dict(alpha=2.0 * K), ["S", "S_alpha", "N", "N_alpha", "calderon", "calderon_alpha", "gram_inv"]),
    ("te_banded_gram", lambda: synth.StarContour.from_seed(7).polygon(60.0, 700), 1, 128,
     dict(alpha=3.0 * K, near_radius=0.4), ["S", "N", "calderon_alpha"]),
    ("te_analytic", lambda: synth.circle_polygon(2.0, 160), 1, 50,
     dict(alpha=4.0 * K, filter_kind=2), ["S_alpha", "calderon_alpha"]),
    ("tm_circle", lambda: synth.circle_polygon(3.0, 240), 0, 80,
     dict(alpha=2.5 * K, near_radius=0.3), ["S", "S_alpha", "efie", "efie_alpha"]),
    ("te_unfiltered", lambda: synth.circle_polygon(1.5, 128), 1, 40, dict(), ["S", "N", "calderon"]),
]


@pytest.fixture(scope="module")
def aim():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2606_10784_gb300 import aim
    return aim


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_imported_context_gives_the_same_bits(aim, case):
    _, mk, form, m, kw, ops = case
    nodes = mk()
    n = len(nodes)
    ctx = aim.Context(nodes, K, form, m, **kw)
    blob = ctx.export_setup()
    ctx2 = aim.Context(nodes, K, form, m, blob=blob, **kw)
    try:
        a, b = ctx.info(), ctx2.info()
        for f in ("n", "m", "fft_P", "s", "quad_p", "k", "L", "eps", "alpha", "n_active", "row_lo", "row_hi",
                  "nnz_near", "filter_kind"):
            assert a[f] == b[f], f
        assert b["device_bytes"] <= a["device_bytes"]
        # the blob of the imported context is the same blob
        assert np.array_equal(ctx2.export_setup(), blob)
        g = torch.Generator().manual_seed(11)
        x = torch.complex(torch.randn((2, n), generator=g, dtype=torch.float64),
                          torch.randn((2, n), generator=g, dtype=torch.float64)).cuda()
        for op in ops:
            for prec in (aim.FP64, aim.MIXED, aim.FP64_NATIVE):
                y1 = ctx.matvec(op, x, torch.empty_like(x), precision=prec)
                y2 = ctx2.matvec(op, x, torch.empty_like(x), precision=prec)
                torch.cuda.synchronize()
                assert torch.equal(y1, y2), (op, prec)
        H = a["fft_P"] // 2
        tables = [aim.TABLE_SPECTRUM, aim.TABLE_SPECTRUM_FILTERED]
        if kw.get("filter_kind") == aim.FILTER_ANALYTIC:
            tables.append(aim.TABLE_ANALYTIC_SAMPLES)
        for which in tables:
            t1 = ctx.kernel_table(which, torch.empty((H + 1, H + 1), dtype=torch.complex128, device="cuda"))
            t2 = ctx2.kernel_table(which, torch.empty((H + 1, H + 1), dtype=torch.complex128, device="cuda"))
            assert torch.equal(t1, t2), which
    finally:
        ctx.close()
        ctx2.close()


def test_solve_through_an_imported_context_is_identical(aim):
    nodes = synth.StarContour.from_seed(8).polygon(40.0, 400)
    ctx = aim.Context(nodes, K, aim.TE, 128, alpha=2.0 * K)
    ctx2 = aim.Context(nodes, K, aim.TE, 128, alpha=2.0 * K, blob=ctx.export_setup())
    try:
        rhs = torch.empty((2, 400), dtype=torch.complex128, device="cuda")
        ctx.rhs_planewave([0.0, 1.1], rhs)
        for prec in (aim.FP64, aim.MIXED):
            x1, x2 = torch.zeros_like(rhs), torch.zeros_like(rhs)
            i1 = ctx.solve("calderon_alpha", rhs, x1, tol=1e-8, restart=300, max_iter=600, precision=prec)
            i2 = ctx2.solve("calderon_alpha", rhs, x2, tol=1e-8, restart=300, max_iter=600, precision=prec)
            torch.cuda.synchronize()
            assert torch.equal(x1, x2)
            assert [i["iters"] for i in i1] == [i["iters"] for i in i2]
    finally:
        ctx.close()
        ctx2.close()


def test_import_refuses_another_problem_or_a_corrupted_blob(aim):
    nodes = synth.StarContour.from_seed(9).polygon(20.0, 200)
    ctx = aim.Context(nodes, K, aim.TE, 64, alpha=2.0 * K)
    blob = ctx.export_setup()
    ctx.close()

    def refused(fragment, b=blob, nd=nodes, k=K, **kw):
        args = dict(alpha=2.0 * K)
        args.update(kw)
        with pytest.raises(aim.AimError) as exc:
            aim.Context(nd, k, aim.TE, 64, blob=b, **args)
        assert exc.value.status == aim.EINVAL
        assert fragment in str(exc.value), str(exc.value)

    refused("k differs", k=K * 1.01)
    refused("filter radius alpha differs", alpha=2.5 * K)
    moved = nodes.copy()
    moved[5, 1] += 1e-9
    refused("vertices differ", nd=moved)
    refused("truncated", b=blob[:-16])
    bad = blob.copy()
    bad[len(bad) // 2] ^= 0x40
    refused("checksum", b=bad)
    # the untouched blob still imports
    aim.Context(nodes, K, aim.TE, 64, alpha=2.0 * K, blob=blob).close()


def test_export_needs_a_large_enough_buffer(aim):
    import ctypes
    nodes = synth.circle_polygon(1.0, 64)
    ctx = aim.Context(nodes, K, aim.TE, 32)
    try:
        size = ctypes.c_size_t(0)
        assert aim.lib().aim_export_setup(ctx._h, None, ctypes.byref(size), None) == aim.OK
        buf = np.empty(size.value - 1, dtype=np.uint8)
        small = ctypes.c_size_t(buf.size)
        assert aim.lib().aim_export_setup(ctx._h, buf.ctypes.data, ctypes.byref(small), None) == aim.EINVAL
        assert small.value == size.value - 1
    finally:
        ctx.close()


def test_disk_cache_reloads_and_rebuilds_a_damaged_file(aim, tmp_path):
    nodes = synth.StarContour.from_seed(10).polygon(25.0, 250)
    kw = dict(alpha=2.0 * K, fft_P=256)
    cache = aim.SetupCache(str(tmp_path))
    x = torch.ones((1, 250), dtype=torch.complex128, device="cuda")
    c1 = cache.context(nodes, K, aim.TE, 100, **kw)
    y1 = c1.matvec("calderon_alpha", x, torch.empty_like(x))
    c1.close()
    assert cache.stats() == {"hits": 0, "misses": 1, "rejected": 0}
    # a restarted process: a new cache object over the same directory
    cache2 = aim.SetupCache(str(tmp_path))
    c2 = cache2.context(nodes, K, aim.TE, 100, **kw)
    y2 = c2.matvec("calderon_alpha", x, torch.empty_like(x))
    c2.close()
    assert cache2.stats() == {"hits": 1, "misses": 0, "rejected": 0}
    assert torch.equal(y1, y2)
    # a damaged file is refused by the library, rebuilt and replaced
    path = cache2.path(aim.setup_key(nodes, K, aim.TE, 100, **kw))
    raw = np.fromfile(path, dtype=np.uint8)
    raw[-7] ^= 0xFF
    raw.tofile(path)
    c3 = cache2.context(nodes, K, aim.TE, 100, **kw)
    y3 = c3.matvec("calderon_alpha", x, torch.empty_like(x))
    c3.close()
    assert cache2.stats() == {"hits": 1, "misses": 1, "rejected": 1}
    assert torch.equal(y1, y3)
    c4 = cache2.context(nodes, K, aim.TE, 100, **kw)
    c4.close()
    assert cache2.stats()["hits"] == 2


def test_restarted_server_imports_its_contexts(aim, tmp_path):
    from paper_2606_10784_gb300 import serving
    reqs = []
    for i, (per, m) in enumerate([(10.0, 64), (30.0, 128)]):
        nodes = synth.StarContour.from_seed(20 + i).polygon(per, int(per * 10))
        reqs.append(serving.SolveRequest(nodes=nodes, k=K, m=m, angles=synth.equispaced_angles(2), alpha=2.0 * K,
                                         tol=1e-6, restart=300, rid=i))
    out = []
    for run in range(2):
        srv = serving.Server(memory_budget_bytes=8 << 30, slots=2, setup_cache_dir=str(tmp_path))
        for r in reqs:
            assert srv.submit(r)
        res = sorted(srv.drain(timeout=300), key=lambda r: r.rid)
        out.append((res, srv.setup_stats()))
        srv.close()
    (first, s1), (second, s2) = out
    assert s1 == {"hits": 0, "misses": 2, "rejected": 0}
    assert s2 == {"hits": 2, "misses": 0, "rejected": 0}
    for a, b in zip(first, second):
        assert a.status == aim.OK and b.status == aim.OK
        assert np.array_equal(a.x, b.x)


def test_import_is_faster_than_the_analytic_setup(aim):
    # the analytic filter samples a principal-value integral per grid offset: its setup is the
    # one a restart most wants to skip
    nodes = synth.circle_polygon(20.0, 1200)
    kw = dict(alpha=3.0 * K, filter_kind=aim.FILTER_ANALYTIC, fft_P=1024)
    t0 = time.perf_counter()
    ctx = aim.Context(nodes, K, aim.TE, 400, **kw)
    t_setup = time.perf_counter() - t0
    blob = ctx.export_setup()
    ctx.close()
    t0 = time.perf_counter()
    ctx2 = aim.Context(nodes, K, aim.TE, 400, blob=blob, **kw)
    t_import = time.perf_counter() - t0
    ctx2.close()
    print("analytic setup %.3f s, import %.3f s, blob %.1f MB" % (t_setup, t_import, blob.size / 1e6))
    assert t_import < t_setup
