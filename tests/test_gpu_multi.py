"""Several contexts of uneven size in one persistent launch (aim_matvec_multi): the batching pattern
of one fused launch over many problems. Each context's result must equal, bit for bit, the product
of the same context launched on its own (the work items run the same arithmetic in the same order),
and so match the oracle; every phase is covered (forward row passes with anterpolation, column
passes with the filtered spectrum's skipped columns, inverse row passes, gathers with near field).
"""
import math

import numpy as np
import pytest

import synth
from oracle import aim as oaim

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K = 2.0 * math.pi

# (perimeter in wavelengths, N, m, P): grids from 64 to 1024 points per FFT side
SIZES = [(3.0, 40, 24, 64), (8.0, 90, 40, 128), (12.0, 150, 64, 256), (30.0, 320, 160, 512), (60.0, 700, 400, 1024)]


@pytest.fixture(scope="module")
def mixed_sizes():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2606_10784_gb300 import aim
    ctxs, nodes = [], []
    for i, (per, n, m, P) in enumerate(SIZES):
        nd = synth.StarContour.from_seed(40 + i).polygon(per, n)
        nodes.append(nd)
        ctxs.append(aim.Context(nd, K, aim.TE, m, fft_P=P, alpha=(2.5 + 0.5 * i) * K))
    yield aim, ctxs, nodes
    for c in ctxs:
        c.close()


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_multi_context_launch_equals_separate_launches(mixed_sizes, precision):
    aim, ctxs, nodes = mixed_sizes
    ops = ["S_alpha", "N", "calderon_alpha", "calderon", "N_alpha"]
    xs = [torch.from_numpy(synth.random_coeffs(len(nd), 1 + (i % 3), seed=60 + i)).cuda() for i, nd in enumerate(nodes)]
    ys = [torch.full_like(x, float("nan")) for x in xs]
    aim.matvec_multi(ctxs, ops, xs, ys, precision=precision)
    for c, op, x, y in zip(ctxs, ops, xs, ys):
        want = torch.empty_like(x)
        c.matvec(op, x, want, precision=precision)
        torch.cuda.synchronize()
        assert torch.equal(y, want), (op, c.info()["fft_P"])


def test_multi_context_results_match_oracle(mixed_sizes):
    aim, ctxs, nodes = mixed_sizes
    xs = [torch.from_numpy(synth.random_coeffs(len(nd), 1, seed=80 + i)).cuda() for i, nd in enumerate(nodes)]
    ys = [torch.empty_like(x) for x in xs]
    aim.matvec_multi(ctxs, ["calderon_alpha"] * len(ctxs), xs, ys)
    for i, (c, nd) in enumerate(zip(ctxs, nodes)):
        inf = c.info()
        ref = oaim.TEOperators(nd, K, inf["m"], inf["fft_P"], alpha=inf["alpha"], L=inf["L"])
        want = ref.calderon(xs[i].cpu().numpy()[0], filtered=True)
        got = ys[i].cpu().numpy()[0]
        assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want)


def test_multi_context_tm_and_te_together(mixed_sizes):
    aim, ctxs, nodes = mixed_sizes
    circ = synth.circle_polygon(1.0, 256)
    tm = aim.Context(circ, K, aim.TM, 64, alpha=8.0 * K)
    try:
        pair = [tm, ctxs[2]]
        xs = [torch.from_numpy(synth.random_coeffs(256, 2, seed=5)).cuda(),
              torch.from_numpy(synth.random_coeffs(len(nodes[2]), 2, seed=6)).cuda()]
        ys = [torch.empty_like(x) for x in xs]
        aim.matvec_multi(pair, ["efie_alpha", "S"], xs, ys)
        for c, op, x, y in zip(pair, ["efie_alpha", "S"], xs, ys):
            want = torch.empty_like(x)
            c.matvec(op, x, want)
            torch.cuda.synchronize()
            assert torch.equal(y, want)
    finally:
        tm.close()


def test_multi_context_rejects_bad_calls(mixed_sizes):
    aim, ctxs, nodes = mixed_sizes
    x = torch.from_numpy(synth.random_coeffs(len(nodes[0]), 1, seed=1)).cuda()
    y = torch.empty_like(x)
    with pytest.raises(aim.AimError) as exc:
        aim.matvec_multi([ctxs[0], ctxs[0]], ["S", "S"], [x, x], [y, y])
    assert exc.value.status == aim.EINVAL
    with pytest.raises(aim.AimError) as exc:
        aim.matvec_multi([ctxs[0]], ["S"], [x.cpu()], [y])
    assert exc.value.status == aim.EINVAL


# --------------------------------------------------------------------------------------
# fused products of concurrent solves (aim_batcher, aim_solve_batched)
# --------------------------------------------------------------------------------------
@pytest.mark.parametrize("precision", [0, 1])
def test_concurrent_batched_solves_equal_solo_solves(mixed_sizes, precision):
    import threading
    aim, ctxs, nodes = mixed_sizes
    use = [1, 2, 3]                                   # P = 128, 256, 512: fusible size classes
    circ = synth.circle_polygon(2.0, 200)
    extra = aim.Context(circ, K, aim.TE, 96, fft_P=256, alpha=3.0 * K)   # a second P = 256 context
    pairs = [(ctxs[i], nodes[i]) for i in use] + [(extra, circ)]
    try:
        rhs = []
        for c, nd in pairs:
            r = torch.empty((2, len(nd)), dtype=torch.complex128, device="cuda")
            c.rhs_planewave([0.0, 1.0], r)
            rhs.append(r)
        torch.cuda.synchronize()
        kw = dict(tol=1e-8, restart=300, max_iter=2000, precision=precision, inner_tol=0.0)
        solo = []
        for (c, nd), r in zip(pairs, rhs):
            x = torch.zeros_like(r)
            info = c.solve("calderon_alpha", r, x, **kw)
            solo.append((x, info))
        batcher = aim.Batcher(max_wait_us=500)
        out = [None] * len(pairs)
        errors = []

        def work(i):
            try:
                c, nd = pairs[i]
                s = torch.cuda.Stream()
                x = torch.zeros_like(rhs[i])
                info = c.solve("calderon_alpha", rhs[i], x, stream=s, batcher=batcher, **kw)
                s.synchronize()
                out[i] = (x, info)
            except Exception as e:   # reported below
                errors.append(repr(e))

        threads = [threading.Thread(target=work, args=(i,)) for i in range(len(pairs))]
        for t in threads:
            t.start()
        for t in threads:
            t.join(timeout=300)
        assert not errors, errors
        stats = batcher.stats()
        batcher.close()
        for (xb, ib), (xs, is_) in zip(out, solo):
            assert ib == is_
            assert torch.equal(xb, xs)
        assert stats["fused_products"] > 0, stats
        print("batcher:", stats)
    finally:
        extra.close()
