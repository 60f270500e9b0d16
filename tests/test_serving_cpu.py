"""Host logic of the solve server (no GPU): admission order under each policy."""
import collections
import time

import numpy as np
import pytest

pytest.importorskip("torch")


def _server(policy, max_wait_s=30.0):
    from paper_2606_10784_gb300 import serving
    srv = serving.Server.__new__(serving.Server)   # no worker threads: ordering logic only
    srv.policy = policy
    srv.max_wait_s = max_wait_s
    srv._queue = collections.deque()
    return srv


def _req(rid, n, m, nrhs, arrival):
    from paper_2606_10784_gb300 import serving
    return serving.SolveRequest(nodes=np.zeros((n, 2)), k=6.0, m=m, angles=np.zeros(nrhs), arrival=arrival, rid=rid)


def test_fifo_keeps_arrival_order():
    srv = _server("fifo")
    now = time.perf_counter()
    for rid, (n, m, r) in enumerate([(5000, 1024, 16), (50, 32, 1), (500, 128, 4)]):
        srv._queue.append((_req(rid, n, m, r, now), 0))
    assert srv._order() == [0, 1, 2]


def test_sjf_orders_by_estimated_work_and_ages_old_requests_first():
    srv = _server("sjf", max_wait_s=10.0)
    now = time.perf_counter()
    reqs = [(5000, 1024, 16, now), (50, 32, 1, now), (500, 128, 4, now), (4000, 1024, 2, now - 60.0),
            (60, 32, 1, now - 30.0)]
    for rid, (n, m, r, t) in enumerate(reqs):
        srv._queue.append((_req(rid, n, m, r, t), 0))
    # waited > 10 s: 3 and 4 first, in queue order; then the rest by work
    assert srv._order() == [3, 4, 1, 2, 0]


def test_unknown_policy_is_refused():
    from paper_2606_10784_gb300 import serving
    with pytest.raises(ValueError):
        serving.Server(1 << 20, policy="lifo")

