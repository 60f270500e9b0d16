"""Serving: continuous batching of solves of different geometries and frequencies.

Each result must be the same whether the request ran alone or mixed with others on the
device (the kernels are deterministic, so the comparison is exact up to 1e-13), requests that
can never fit the memory budget are refused, and under a tight budget everything still
completes (admission waits for memory to free up).
"""
import math

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def serving():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2606_10784_gb300 import aim, serving as sv
    return aim, sv


def make_requests(sv, n=8, seed=3):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        per = float(rng.uniform(4.0, 14.0))
        k = float(rng.uniform(math.pi, 3 * math.pi))
        wl = 2 * math.pi / k
        nseg = max(48, int(10 * per))
        nodes = synth.StarContour.from_seed(100 + i).polygon(per * wl, nseg)
        m = 64 if per > 8 else 32
        alpha = 2.0 * k if i % 2 == 0 else None
        reqs.append(sv.SolveRequest(nodes=nodes, k=k, m=m, angles=synth.equispaced_angles(int(rng.integers(1, 5))),
                                    alpha=alpha, system="calderon_alpha" if alpha else "calderon",
                                    tol=1e-8, restart=600, rid=i))
    return reqs


@pytest.mark.parametrize("fused", [False, True])
def test_results_identical_alone_and_mixed(serving, fused):
    # fused: the slots' solves share a batcher, so products of concurrent requests run in
    # multi-context launches; every request's arithmetic is unchanged, so the results are too
    aim, sv = serving
    reqs = make_requests(sv)
    alone = {}
    srv = sv.Server(memory_budget_bytes=8 << 30, slots=1)
    for r in reqs:
        srv.submit(r)
        res = srv.drain(timeout=600)
    srv.close()
    for res_i in res:
        alone[res_i.rid] = res_i
    assert len(alone) == len(reqs)
    srv = sv.Server(memory_budget_bytes=8 << 30, slots=4, fused=fused)
    for r in make_requests(sv):
        srv.submit(r)
    mixed = {r.rid: r for r in srv.drain(timeout=600)}
    stats = srv.fusion_stats()
    srv.close()
    if fused:
        assert stats["products"] > 0
    for rid, a in alone.items():
        b = mixed[rid]
        assert a.status == 0 and b.status == 0
        assert all(i["converged"] for i in a.info)
        assert np.max(np.abs(a.x - b.x)) <= 1e-13 * np.max(np.abs(a.x))
    summ = sv.latency_summary(list(mixed.values()))
    assert summ["count"] == len(reqs) and summ["p99_s"] >= summ["p50_s"] > 0


def test_admission_refuses_and_waits(serving):
    aim, sv = serving
    reqs = make_requests(sv, n=6, seed=5)
    need = max(sv.request_bytes(r) for r in reqs)
    srv = sv.Server(memory_budget_bytes=need + (need // 2), slots=4, max_cached=1)
    huge = sv.SolveRequest(nodes=synth.circle_polygon(30.0, 2000), k=2 * math.pi, m=1024,
                           angles=synth.equispaced_angles(16), alpha=None, system="calderon", rid=99)
    assert not srv.submit(huge)
    for r in reqs:
        assert srv.submit(r)
    res = srv.drain(timeout=600)
    srv.close()
    assert srv.refused == [99]
    assert len(res) == len(reqs) and all(r.status == 0 for r in res)
