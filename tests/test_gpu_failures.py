"""Failure paths of the C ABI, all made on the host side: a non-finite right-hand side, a time
limit that runs out, an iteration limit that is too small, a memory budget below the request's
bound, and a context used while another device is current. Each must come back as its status
code (never a trap), and the memory queries must bound what the device really commits.
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


@pytest.fixture(scope="module")
def star(aimlib):
    nodes = synth.StarContour.from_seed(4).polygon(60.0, 600)
    ctx = aimlib.Context(nodes, K, aimlib.TE, 128, fft_P=256, alpha=2.0 * K)
    rhs = torch.empty((2, 600), dtype=torch.complex128, device="cuda")
    ctx.rhs_planewave([0.0, 1.0], rhs)
    yield nodes, ctx, rhs
    ctx.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_nan_right_hand_side_is_a_numeric_error(aimlib, star, precision):
    nodes, ctx, rhs = star
    bad = rhs.clone()
    bad[1, 17] = float("nan")
    x = torch.zeros_like(bad)
    st, info = ctx.solve("calderon_alpha", bad, x, tol=1e-8, restart=100, max_iter=400, precision=precision,
                         check=False)
    assert st == aimlib.ENUMERIC
    assert "non-finite" in aimlib.lib().aim_last_error().decode()
    # the context stays usable: the next solve of a finite system converges
    x = torch.zeros_like(rhs)
    st, info = ctx.solve("calderon", rhs, x, tol=1e-8, restart=100, max_iter=400, precision=precision, check=False)
    assert st == aimlib.OK and all(i["converged"] == 1 for i in info)


@pytest.mark.parametrize("precision", [0, 1])
def test_time_limit_ends_the_solve_with_a_timeout(aimlib, star, precision):
    nodes, ctx, rhs = star
    x = torch.zeros_like(rhs)
    # a tolerance the nearly singular filtered system needs hundreds of iterations for, 1 ms allowed
    st, _ = ctx.solve("calderon_alpha", rhs, x, tol=1e-12, restart=1000, max_iter=4000, precision=precision,
                      timeout_ms=1, check=False)
    assert st == aimlib.ETIMEOUT
    assert "time limit" in aimlib.lib().aim_last_error().decode()


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_iteration_limit_reports_not_converged(aimlib, star, precision):
    nodes, ctx, rhs = star
    x = torch.zeros_like(rhs)
    st, info = ctx.solve("calderon_alpha", rhs, x, tol=1e-10, restart=100, max_iter=5, precision=precision,
                         check=False)
    assert st == aimlib.ENOCONV
    for i in info:
        assert i["converged"] == 0
        assert 0 < i["iters"] <= 5
        assert i["rel_res"] > 1e-10
    with pytest.raises(aimlib.AimError) as exc:
        ctx.solve("calderon_alpha", rhs, x, tol=1e-10, restart=100, max_iter=5, precision=precision)
    assert exc.value.status == aimlib.ENOCONV


def test_budget_below_the_request_bound_is_refused(aimlib):
    from paper_2606_10784_gb300 import serving
    nodes = synth.StarContour.from_seed(3).polygon(20.0, 200)
    req = serving.SolveRequest(nodes=nodes, k=K, m=64, angles=synth.equispaced_angles(2), alpha=3.0 * K,
                               tol=1e-6, restart=300, rid=0)
    need = serving.request_bytes(req)
    srv = serving.Server(memory_budget_bytes=need - 1, slots=1)
    assert srv.submit(req) is False
    assert srv.refused == [0]
    srv.close()
    srv = serving.Server(memory_budget_bytes=need, slots=1)
    assert srv.submit(req) is True
    res = srv.drain(timeout=120)
    srv.close()
    assert len(res) == 1 and res[0].status == aimlib.OK


CASES = [
    # (contour, form, m, P, near_radius, nrhs, restart, precision)
    ("star_te", lambda: synth.StarContour.from_seed(5).polygon(40.0, 400), 1, 128, 0, 0.0, 3, 200, 0),
    ("star_te_wide_near", lambda: synth.StarContour.from_seed(5).polygon(40.0, 400), 1, 128, 0, 2.5, 2, 150, 1),
    ("circle_tm", lambda: synth.circle_polygon(3.0, 300), 0, 96, 256, 0.0, 4, 100, 2),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_memory_queries_bound_what_the_device_commits(aimlib, case):
    _, mk, form, m, P, near_radius, nrhs, restart, precision = case
    nodes = mk()
    n = len(nodes)
    # warm-up: load the library's kernels once (module loading commits device memory of its own)
    warm = aimlib.Context(synth.circle_polygon(1.0, 64), K, form, 32, alpha=4.0 * K)
    w = torch.zeros((1, 64), dtype=torch.complex128, device="cuda")
    warm.rhs_planewave([0.0], w)
    wx = torch.zeros_like(w)
    warm.solve("efie" if form == 0 else "calderon", w, wx, tol=1e-6, restart=20, max_iter=40, precision=precision,
               check=False)
    warm.close()
    rhs = torch.zeros((nrhs, n), dtype=torch.complex128, device="cuda")
    x = torch.zeros_like(rhs)
    torch.cuda.synchronize()
    q_ctx = aimlib.query_bytes(nodes, form, m, fft_P=P, nrhs=nrhs, precision=precision, near_radius=near_radius)
    q_solve = aimlib.query_solve_bytes(nodes, form, m, fft_P=P, nrhs=nrhs, restart=restart, precision=precision,
                                       near_radius=near_radius)
    assert q_solve > q_ctx
    free0, _ = torch.cuda.mem_get_info()
    ctx = aimlib.Context(nodes, K, form, m, fft_P=P, near_radius=near_radius, alpha=3.0 * K)
    ctx.reserve(nrhs, precision)
    free1, _ = torch.cuda.mem_get_info()
    assert ctx.info()["device_bytes"] <= q_ctx
    assert free0 - free1 <= q_ctx
    ctx.rhs_planewave(synth.equispaced_angles(nrhs), rhs)
    ctx.solve("efie" if form == 0 else "calderon", rhs, x, tol=1e-9, restart=restart, max_iter=restart,
              precision=precision, check=False)
    torch.cuda.synchronize()
    free2, _ = torch.cuda.mem_get_info()
    assert ctx.info()["device_bytes"] <= q_solve
    assert free0 - free2 <= q_solve
    ctx.close()


def test_context_used_on_another_device_is_refused(aimlib):
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two GPUs: the context must live on a device that is not current")
    nodes = synth.circle_polygon(1.0, 64)
    torch.cuda.set_device(0)
    ctx = aimlib.Context(nodes, K, aimlib.TE, 32, alpha=4.0 * K)
    x = torch.zeros((1, 64), dtype=torch.complex128, device="cuda:1")
    y = torch.zeros_like(x)
    torch.cuda.set_device(1)
    try:
        for call in (lambda: ctx.matvec("S", x, y), lambda: ctx.rhs_planewave([0.0], y),
                     lambda: ctx.solve("calderon", x, y, tol=1e-6),
                     lambda: ctx.grid_product_noalloc(x.view(1, 8, 8), y.view(1, 8, 8), True)):
            with pytest.raises(aimlib.AimError) as exc:
                call()
            assert exc.value.status == aimlib.EINVAL
            assert "context's device" in str(exc.value)
    finally:
        torch.cuda.set_device(0)
        ctx.close()


def test_new_entry_points_report_misuse(aimlib):
    nodes = synth.circle_polygon(1.0, 64)
    tm = aimlib.Context(nodes, K, aimlib.TM, 32, alpha=4.0 * K)
    te = aimlib.Context(nodes, K, aimlib.TE, 32)            # no filter radius
    te2 = aimlib.Context(synth.circle_polygon(1.5, 96), K, aimlib.TE, 40, alpha=3.0 * K)
    try:
        v0 = torch.ones(64, dtype=torch.complex128, device="cuda")
        # Lanczos: TM collocation operators are not symmetric; k beyond n
        with pytest.raises(aimlib.AimError) as exc:
            tm.lanczos_bidiag("S", 8, v0)
        assert exc.value.status == aimlib.ESTATE
        with pytest.raises(aimlib.AimError) as exc:
            te.lanczos_bidiag("S", 65, v0)
        assert exc.value.status == aimlib.EINVAL
        # the analytic filter needs a filter radius
        out = torch.empty((33, 33), dtype=torch.complex128, device="cuda")
        with pytest.raises(aimlib.AimError) as exc:
            te.kernel_table(aimlib.TABLE_ANALYTIC_SAMPLES, out)
        assert exc.value.status == aimlib.ESTATE
        # one multi-context launch needs one pass geometry: change one context's schedule
        te2.set_schedule(aimlib.FP64, 2, 128, 0, 16)
        xs = [torch.ones((1, 64), dtype=torch.complex128, device="cuda"),
              torch.ones((1, 96), dtype=torch.complex128, device="cuda")]
        ys = [torch.empty_like(x) for x in xs]
        with pytest.raises(aimlib.AimError) as exc:
            aimlib.matvec_multi([te, te2], ["S", "S"], xs, ys, precision=aimlib.FP64)
        assert exc.value.status == aimlib.EINVAL
        assert "geometry" in str(exc.value)
    finally:
        for c in (tm, te, te2):
            c.close()
