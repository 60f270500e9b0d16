"""Continuous-batching solve server over the AIM C ABI.

Requests (a contour, a wavenumber, grid and filter parameters, and 1..16 incidence angles)
arrive over time. The server admits a request when a slot is free and the device-memory
bound of its context (aim_query_solve_bytes) fits in the remaining budget, runs it on that slot's
own CUDA stream, and reports each request's latency from arrival to completion. Slots run
concurrently, so the device work of requests admitted at different times overlaps; with fusion on
(fused=True) the slots share an aim_batcher, and the operator products of requests running at
the same time go into one multi-context launch per grid-pass stage (grids of one size class).
Contexts (kernel spectra, projections, near field, Krylov workspace) stay resident in an LRU
cache keyed by the request's geometry and parameters, so a repeated geometry skips setup.

All device work is the library's; this module only schedules calls. Results do not depend on
what else is running: every kernel is deterministic (no atomics, fixed reduction order).
"""
from __future__ import annotations

import collections
import dataclasses
import hashlib
import threading
import time
from typing import Dict, List, Optional

import numpy as np

from . import aim


@dataclasses.dataclass
class SolveRequest:
    nodes: np.ndarray                 # (N, 2) contour vertices, counter-clockwise
    k: float
    m: int
    angles: np.ndarray                # incidence angles (1..16)
    alpha: Optional[float] = None     # filter radius (None: unfiltered Calderon)
    fft_P: int = 0
    s: int = 4
    quad_p: int = 4
    system: str = "calderon_alpha"
    precision: int = aim.FP64
    tol: float = 1e-5
    restart: int = 3000
    max_iter: int = 8000
    arrival: float = 0.0              # seconds on the server clock (time.perf_counter)
    rid: int = 0

    def key(self) -> str:
        h = hashlib.sha1()
        h.update(np.ascontiguousarray(self.nodes, dtype=np.float64).tobytes())
        h.update(repr((self.k, self.m, self.alpha, self.fft_P, self.s, self.quad_p)).encode())
        return h.hexdigest()


def request_bytes(req: SolveRequest) -> int:
    """Device-memory bound of one request: its context after the solve (aim_query_solve_bytes:
    operators, grid workspaces, staging, Krylov basis for the request's restart length)."""
    return aim.query_solve_bytes(req.nodes, aim.TE, req.m, s=req.s, quad_p=req.quad_p, fft_P=req.fft_P,
                                 nrhs=len(req.angles), restart=req.restart, precision=req.precision)


@dataclasses.dataclass
class SolveResult:
    rid: int
    x: np.ndarray                     # (nrhs, N) complex128 currents
    info: list
    status: int
    arrival: float
    start: float
    done: float
    cached_context: bool

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class Server:
    """Admission by device-memory budget, `slots` concurrent solves, resident context cache."""

    def __init__(self, memory_budget_bytes: int, slots: int = 4, max_cached: int = 16, device: int = 0,
                 policy: str = "sjf", max_wait_s: float = 30.0, fused: bool = False, fuse_wait_us: int = 50,
                 setup_cache_dir: Optional[str] = None):
        """policy "fifo": the first queued request that fits. policy "sjf": the fitting request
        with the least estimated work (right-hand sides x grid cells x unknowns, which tracks
        the grid work per iteration times the iteration count), except that requests waiting
        longer than max_wait_s go first, oldest first, so that large requests are not starved.
        fused: the slots' solves share an aim_batcher, so the operator products of requests that
        run at the same time (grids up to P = 512, one size class) go into one multi-context
        launch per grid-pass stage; fuse_wait_us bounds how long a product waits for partners.
        Off by default: the slots' own streams already overlap the kernels of small requests, and
        on the served stream fusion tied small requests to their partners' pace (p50 1.37 s fused
        against 1.17 s unfused at the same throughput).
        setup_cache_dir: contexts missing from the resident cache are imported from setup blobs in
        this directory (aim.SetupCache) when present and written there when built, so a restarted
        server skips their setup."""
        import torch
        if policy not in ("fifo", "sjf"):
            raise ValueError("policy must be 'fifo' or 'sjf'")
        self.batcher = aim.Batcher(fuse_wait_us) if fused else None
        self.setup_cache = aim.SetupCache(setup_cache_dir) if setup_cache_dir else None
        self.policy = policy
        self.max_wait_s = float(max_wait_s)
        self.torch = torch
        self.budget = int(memory_budget_bytes)
        self.slots = int(slots)
        self.max_cached = int(max_cached)
        self.device = device
        self._lock = threading.Condition()
        self._queue: collections.deque = collections.deque()
        self._in_use = 0                    # bytes reserved by running requests
        self._cache: "collections.OrderedDict[str, tuple]" = collections.OrderedDict()   # key -> (ctx, bytes)
        self._cache_bytes = 0
        self._busy_keys: Dict[str, int] = {}
        self._results: List[SolveResult] = []
        self._refused: List[int] = []
        self._stop = False
        self._pending = 0
        self._workers = [threading.Thread(target=self._worker, args=(i,), daemon=True) for i in range(self.slots)]
        for w in self._workers:
            w.start()

    # -------------------------------------------------------------- public
    def submit(self, req: SolveRequest) -> bool:
        """Queue a request; False if it can never fit the budget (refused)."""
        need = self._bytes_for(req)
        if need > self.budget:
            with self._lock:
                self._refused.append(req.rid)
            return False
        with self._lock:
            self._queue.append((req, need))
            self._pending += 1
            self._lock.notify_all()
        return True

    def drain(self, timeout: Optional[float] = None) -> List[SolveResult]:
        end = None if timeout is None else time.perf_counter() + timeout
        with self._lock:
            while self._pending > 0:
                left = None if end is None else end - time.perf_counter()
                if left is not None and left <= 0:
                    break
                self._lock.wait(left)
            return list(self._results)

    def close(self):
        with self._lock:
            self._stop = True
            self._lock.notify_all()
        for w in self._workers:
            w.join(timeout=30)
        for ctx, _ in self._cache.values():
            ctx.close()
        self._cache.clear()
        if self.batcher is not None:
            self.batcher.close()
            self.batcher = None

    def setup_stats(self) -> Optional[dict]:
        """Setup-blob cache hits, misses and refused files, or None without a cache directory."""
        return self.setup_cache.stats() if self.setup_cache is not None else None

    def fusion_stats(self) -> Optional[dict]:
        return self.batcher.stats() if self.batcher is not None else None

    @property
    def refused(self) -> List[int]:
        return list(self._refused)

    # -------------------------------------------------------------- internals
    def _bytes_for(self, req: SolveRequest) -> int:
        return request_bytes(req)

    def _evict_for(self, need: int):
        # drop idle cached contexts (oldest first) until the request fits
        for key in list(self._cache.keys()):
            if self._in_use + self._cache_bytes + need <= self.budget:
                return
            if self._busy_keys.get(key, 0):
                continue
            ctx, b = self._cache.pop(key)
            self._cache_bytes -= b
            ctx.close()

    @staticmethod
    def _work(req: SolveRequest) -> float:
        P = req.fft_P if req.fft_P > 0 else 2 * req.m
        return float(len(req.angles)) * P * P * len(req.nodes)

    def _order(self):
        """Queue indices in the order the policy considers them."""
        idx = list(range(len(self._queue)))
        if self.policy == "fifo":
            return idx
        now = time.perf_counter()
        old = [i for i in idx if now - self._queue[i][0].arrival > self.max_wait_s]
        young = sorted((i for i in idx if now - self._queue[i][0].arrival <= self.max_wait_s),
                       key=lambda i: (self._work(self._queue[i][0]), self._queue[i][0].arrival))
        return old + young

    def _admit(self):
        """Called with the lock held: the first request in policy order that fits the budget."""
        for idx in self._order():
            req, need = self._queue[idx]
            key = req.key()
            cached = key in self._cache
            extra = 0 if cached else need
            if self._in_use + self._cache_bytes + extra > self.budget:
                self._evict_for(extra)
            if self._in_use + self._cache_bytes + extra <= self.budget:
                del self._queue[idx]
                self._in_use += extra
                self._busy_keys[key] = self._busy_keys.get(key, 0) + 1
                return req, extra, key, cached
        return None

    def _worker(self, slot: int):
        torch = self.torch
        torch.cuda.set_device(self.device)
        stream = torch.cuda.Stream(device=self.device)
        while True:
            with self._lock:
                item = None
                while item is None:
                    if self._stop:
                        return
                    item = self._admit()
                    if item is None:
                        self._lock.wait(0.05)
                req, extra, key, cached = item
                ctx_entry = self._cache.get(key)
                if ctx_entry is not None:
                    self._cache.move_to_end(key)
            start = time.perf_counter()
            status = aim.OK
            info: list = []
            x_host = np.zeros((len(req.angles), len(req.nodes)), dtype=np.complex128)
            try:
                if ctx_entry is None and self.setup_cache is not None:
                    ctx = self.setup_cache.context(req.nodes, req.k, aim.TE, req.m, fft_P=req.fft_P, s=req.s,
                                                   quad_p=req.quad_p, alpha=req.alpha, stream=stream)
                elif ctx_entry is None:
                    ctx = aim.Context(req.nodes, req.k, aim.TE, req.m, fft_P=req.fft_P, s=req.s,
                                      quad_p=req.quad_p, alpha=req.alpha, stream=stream)
                else:
                    ctx = ctx_entry[0]
                with torch.cuda.stream(stream):
                    rhs = torch.empty((len(req.angles), len(req.nodes)), dtype=torch.complex128, device="cuda")
                    x = torch.zeros_like(rhs)
                ctx.rhs_planewave(req.angles, rhs, stream=stream)
                status, info = ctx.solve(req.system, rhs, x, tol=req.tol, restart=req.restart,
                                         max_iter=req.max_iter, precision=req.precision, stream=stream, check=False,
                                         batcher=self.batcher)
                stream.synchronize()
                x_host = x.cpu().numpy()
            except aim.AimError as e:
                status = e.status
                ctx = None
            except Exception:   # anything else (e.g. an allocation failure) fails this request only
                status = aim.ECUDA
                ctx = None
            done = time.perf_counter()
            with self._lock:
                self._in_use -= extra
                self._busy_keys[key] -= 1
                if ctx is not None and key not in self._cache:
                    b = ctx.info()["device_bytes"]
                    self._cache[key] = (ctx, b)
                    self._cache_bytes += b
                    while len(self._cache) > self.max_cached:
                        k0 = next(iter(self._cache))
                        if self._busy_keys.get(k0, 0):
                            break
                        c0, b0 = self._cache.pop(k0)
                        self._cache_bytes -= b0
                        c0.close()
                self._results.append(SolveResult(req.rid, x_host, info, status, req.arrival, start, done, cached))
                self._pending -= 1
                self._lock.notify_all()


def latency_summary(results: List[SolveResult]) -> dict:
    lat = np.array([r.latency for r in results])
    if lat.size == 0:
        return {"count": 0}
    span = max(r.done for r in results) - min(r.arrival for r in results)
    return {"count": int(lat.size), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "solves_per_s": float(lat.size / span) if span > 0 else None,
            "rhs_per_s": float(sum(r.x.shape[0] for r in results) / span) if span > 0 else None,
            "failed": int(sum(1 for r in results if r.status != aim.OK))}


def replay(server: Server, requests: List[SolveRequest], time_scale: float = 1.0) -> List[SolveResult]:
    """Submit requests at their arrival offsets (seconds, scaled) and wait for all of them."""
    t0 = time.perf_counter()
    base = requests[0].arrival if requests else 0.0
    for req in requests:
        due = t0 + (req.arrival - base) * time_scale
        now = time.perf_counter()
        if due > now:
            time.sleep(due - now)
        req.arrival = time.perf_counter()
        server.submit(req)
    return server.drain()
