"""Python binding of the AIM C ABI (include/aim.h): argument marshalling only.

Every step of setup, matrix-vector products and solves runs inside libaimgb300.so. There is
no fallback: if the compiled library is missing this module raises on import of `lib()`.
Vectors are complex128 with shape (nrhs, n) (row r is right-hand side r, matching the ABI's
column-major n x nrhs layout); they may be torch tensors (CUDA or CPU) or numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libaimgb300.so")

# enums (mirror include/aim.h)
OK, EINVAL, ENOMEM, ECUDA, ENOCONV, ENUMERIC, ETIMEOUT, ESTATE = range(8)
TM, TE = 0, 1
(OP_S, OP_S_ALPHA, OP_N, OP_CALDERON, OP_CALDERON_ALPHA, OP_GRAM_INV, OP_EFIE, OP_EFIE_ALPHA, OP_N_ALPHA,
 OP_CALDERON_ALPHA2) = range(10)
FP64, MIXED, FP64_NATIVE = 0, 1, 2
FILTER_NONE, FILTER_NUMERICAL, FILTER_ANALYTIC = 0, 1, 2
TABLE_SPECTRUM, TABLE_SPECTRUM_FILTERED, TABLE_ANALYTIC_SAMPLES, TABLE_ANALYTIC_SPECTRUM = 0, 1, 2, 3
DFT_STAGE_CUDA_CORES, DFT_STAGE_MMA_TF32, DFT_STAGE_MMA_TF32X3, DFT_STAGE_SPLIT_ONLY = 0, 1, 2, 3
DFT_STAGE_GROUP = 4096   # complex64 values per CTA of aim_dft_stage

OPS = {"S": OP_S, "S_alpha": OP_S_ALPHA, "N": OP_N, "calderon": OP_CALDERON,
       "calderon_alpha": OP_CALDERON_ALPHA, "gram_inv": OP_GRAM_INV, "efie": OP_EFIE, "efie_alpha": OP_EFIE_ALPHA,
       "N_alpha": OP_N_ALPHA, "calderon_alpha2": OP_CALDERON_ALPHA2}


class Geometry(ctypes.Structure):
    _fields_ = [("n_seg", ctypes.c_int), ("xy", ctypes.POINTER(ctypes.c_double)), ("form", ctypes.c_int),
                ("quad_p", ctypes.c_int)]


class Grid(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("half_side_L", ctypes.c_double), ("fft_P", ctypes.c_int)]


class Stencil(ctypes.Structure):
    _fields_ = [("s", ctypes.c_int), ("near_radius", ctypes.c_double)]


class Filter(ctypes.Structure):
    _fields_ = [("enabled", ctypes.c_int), ("alpha", ctypes.c_double)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("precision", ctypes.c_int), ("inner_tol", ctypes.c_double), ("timeout_ms", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("outer_iters", ctypes.c_int), ("rel_res", ctypes.c_double),
                ("converged", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("m", ctypes.c_int), ("fft_P", ctypes.c_int), ("s", ctypes.c_int),
                ("quad_p", ctypes.c_int), ("k", ctypes.c_double), ("L", ctypes.c_double), ("eps", ctypes.c_double),
                ("alpha", ctypes.c_double), ("n_active", ctypes.c_int), ("row_lo", ctypes.c_int),
                ("row_hi", ctypes.c_int), ("nnz_near", ctypes.c_longlong), ("device_bytes", ctypes.c_size_t),
                ("setup_seconds", ctypes.c_double), ("filter_kind", ctypes.c_int)]


class Schedule(ctypes.Structure):
    _fields_ = [("transforms_per_thread", ctypes.c_int), ("row_threads", ctypes.c_int), ("col_cols", ctypes.c_int),
                ("elems_per_thread", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {"transforms_per_thread": self.transforms_per_thread, "row_threads": self.row_threads,
                "col_cols": self.col_cols, "elems_per_thread": self.elems_per_thread}


class KernelStat(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("name", ctypes.c_char_p), ("launches", ctypes.c_longlong),
                ("total_ms", ctypes.c_double)]


_lib = None


def launch_count() -> int:
    """Kernels the library has enqueued in this process."""
    return int(lib().aim_launch_count())


def profile_start():
    _check(lib().aim_profile_start(), "aim_profile_start")


def profile_stop() -> dict:
    """Per-kernel {name: (launches, total_ms)} since profile_start (waits for the events)."""
    stats = (KernelStat * 32)()
    cnt = ctypes.c_int(0)
    _check(lib().aim_profile_stop(stats, 32, ctypes.byref(cnt)), "aim_profile_stop")
    return {stats[i].name.decode(): (stats[i].launches, stats[i].total_ms) for i in range(cnt.value)}


def lib() -> ctypes.CDLL:
    """Load libaimgb300.so (built by __graft_entry__.build() or build.py)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libaimgb300.so is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.aim_setup.argtypes = [ctypes.POINTER(Geometry), d, ctypes.POINTER(Grid), ctypes.POINTER(Stencil),
                            ctypes.POINTER(Filter), vp, ctypes.POINTER(vp)]
    L.aim_setup.restype = i
    L.aim_destroy.argtypes = [vp]
    L.aim_setup_key.argtypes = [ctypes.POINTER(Geometry), d, ctypes.POINTER(Grid), ctypes.POINTER(Stencil),
                                ctypes.POINTER(Filter), ctypes.POINTER(ctypes.c_ulonglong)]
    L.aim_setup_key.restype = i
    L.aim_export_setup.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_size_t), vp]
    L.aim_export_setup.restype = i
    L.aim_import_setup.argtypes = [ctypes.POINTER(Geometry), d, ctypes.POINTER(Grid), ctypes.POINTER(Stencil),
                                   ctypes.POINTER(Filter), vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]
    L.aim_import_setup.restype = i
    L.aim_destroy.restype = None
    L.aim_get_info.argtypes = [vp, ctypes.POINTER(Info)]
    L.aim_get_info.restype = i
    L.aim_reserve.argtypes = [vp, i, i]
    L.aim_reserve.restype = i
    L.aim_rhs_planewave.argtypes = [vp, i, ctypes.POINTER(d), vp, vp]
    L.aim_rhs_planewave.restype = i
    L.aim_matvec.argtypes = [vp, i, i, vp, vp, i, vp]
    L.aim_matvec.restype = i
    L.aim_grid_product.argtypes = [vp, i, i, vp, vp, i, vp]
    L.aim_grid_product.restype = i
    L.aim_solve.argtypes = [vp, i, i, vp, vp, i, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo), vp]
    L.aim_solve.restype = i
    L.aim_query_bytes.argtypes = [ctypes.POINTER(Geometry), ctypes.POINTER(Grid), ctypes.POINTER(Stencil), i, i,
                                  ctypes.POINTER(ctypes.c_size_t)]
    L.aim_query_bytes.restype = i
    L.aim_query_solve_bytes.argtypes = [ctypes.POINTER(Geometry), ctypes.POINTER(Grid), ctypes.POINTER(Stencil), i,
                                        ctypes.POINTER(SolveOpts), ctypes.POINTER(ctypes.c_size_t)]
    L.aim_query_solve_bytes.restype = i
    L.aim_grid_product_noalloc.argtypes = [vp, i, i, vp, vp, i, vp]
    L.aim_grid_product_noalloc.restype = i
    L.aim_batcher_create.argtypes = [i, ctypes.POINTER(vp)]
    L.aim_batcher_create.restype = i
    L.aim_batcher_destroy.argtypes = [vp]
    L.aim_batcher_destroy.restype = None
    L.aim_batcher_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                                    ctypes.POINTER(ctypes.c_longlong)]
    L.aim_batcher_stats.restype = i
    L.aim_solve_batched.argtypes = [vp, vp, i, i, vp, vp, i, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo), vp]
    L.aim_solve_batched.restype = i
    L.aim_matvec_multi.argtypes = [i, ctypes.POINTER(vp), ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(vp),
                                   ctypes.POINTER(vp), i, vp]
    L.aim_matvec_multi.restype = i
    L.aim_lanczos_bidiag.argtypes = [vp, i, i, i, vp, ctypes.POINTER(d), ctypes.POINTER(d), vp, vp, vp]
    L.aim_lanczos_bidiag.restype = i
    L.aim_kernel_table.argtypes = [vp, i, vp, vp]
    L.aim_kernel_table.restype = i
    L.aim_autotune.argtypes = [vp, i, i, vp, ctypes.POINTER(Schedule)]
    L.aim_autotune.restype = i
    L.aim_set_schedule.argtypes = [vp, i, ctypes.POINTER(Schedule)]
    L.aim_set_schedule.restype = i
    L.aim_get_schedule.argtypes = [vp, i, ctypes.POINTER(Schedule)]
    L.aim_get_schedule.restype = i
    L.aim_launch_count.argtypes = []
    L.aim_launch_count.restype = ctypes.c_longlong
    L.aim_profile_start.argtypes = []
    L.aim_profile_start.restype = i
    L.aim_profile_stop.argtypes = [ctypes.POINTER(KernelStat), i, ctypes.POINTER(i)]
    L.aim_profile_stop.restype = i
    L.aim_status_str.argtypes = [i]
    L.aim_status_str.restype = ctypes.c_char_p
    L.aim_last_error.argtypes = []
    L.aim_last_error.restype = ctypes.c_char_p
    L.aim_dft_stage.argtypes = [i, i, i, vp, vp, vp]
    L.aim_dft_stage.restype = i
    _lib = L
    return L


def matvec_multi(ctxs, ops, xs, ys, precision: int = FP64, stream=None):
    """y_i = A_i x_i for several contexts (of any sizes) in one persistent launch per grid-pass stage
    (aim_matvec_multi); xs, ys: device tensors of shape (nrhs_i, n_i)."""
    count = len(ctxs)
    arr_c = (ctypes.c_void_p * count)(*[c._h.value for c in ctxs])
    arr_o = (ctypes.c_int * count)(*[OPS[o] if isinstance(o, str) else int(o) for o in ops])
    arr_r = (ctypes.c_int * count)(*[x.shape[0] if x.ndim == 2 else 1 for x in xs])
    arr_x = (ctypes.c_void_p * count)(*[_ptr(x) for x in xs])
    arr_y = (ctypes.c_void_p * count)(*[_ptr(y) for y in ys])
    _check(lib().aim_matvec_multi(count, arr_c, arr_o, arr_r, arr_x, arr_y, int(precision), _stream_ptr(stream)),
           "aim_matvec_multi")
    return ys


def dft_stage(variant: int, x, y, passes: int, stream=None):
    """`passes` radix-16 DFT passes over each group of 4096 complex64 values of x, into y
    (aim_dft_stage: a measurement of the stage on CUDA cores or tensor cores); x, y: contiguous
    complex64 device tensors whose size is a multiple of 4096."""
    if x.numel() != y.numel() or x.numel() % DFT_STAGE_GROUP:
        raise ValueError("x and y must hold the same multiple of %d values" % DFT_STAGE_GROUP)
    _check(lib().aim_dft_stage(int(variant), x.numel() // DFT_STAGE_GROUP, int(passes), _ptr(x), _ptr(y),
                               _stream_ptr(stream)), "aim_dft_stage")
    return y


class Batcher:
    """Fused operator products of solves that run at the same time on different threads
    (aim_batcher_*); pass it to Context.solve(batcher=...)."""

    def __init__(self, max_wait_us: int = 200):
        h = ctypes.c_void_p()
        _check(lib().aim_batcher_create(int(max_wait_us), ctypes.byref(h)), "aim_batcher_create")
        self._h = h

    def stats(self) -> dict:
        p, l, f = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        _check(lib().aim_batcher_stats(self._h, ctypes.byref(p), ctypes.byref(l), ctypes.byref(f)), "aim_batcher_stats")
        return {"products": p.value, "launches": l.value, "fused_products": f.value}

    def close(self):
        if getattr(self, "_h", None):
            lib().aim_batcher_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class AimError(RuntimeError):
    def __init__(self, status: int, where: str):
        L = lib()
        msg = "%s: %s (%s)" % (where, L.aim_status_str(status).decode(), L.aim_last_error().decode())
        super().__init__(msg)
        self.status = status


def _check(status: int, where: str):
    if status != OK:
        raise AimError(status, where)


def _ptr(a) -> int:
    """Raw pointer of a contiguous torch tensor or numpy array."""
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError("expected a torch tensor or numpy array")


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def _geometry(nodes: np.ndarray, form: int, quad_p: int):
    xy = np.ascontiguousarray(np.asarray(nodes, dtype=np.float64).reshape(-1))
    g = Geometry(int(xy.size // 2), xy.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(form), int(quad_p))
    return g, xy


def query_bytes(nodes, form: int, m: int, s: int = 4, quad_p: int = 4, fft_P: int = 0, nrhs: int = 1,
                precision: int = FP64, near_radius: float = 0.0) -> int:
    """Upper bound on the device bytes of aim_setup + aim_reserve(nrhs, precision)."""
    g, keep = _geometry(nodes, form, quad_p)
    out = ctypes.c_size_t(0)
    _check(lib().aim_query_bytes(ctypes.byref(g), ctypes.byref(Grid(m, 0.0, fft_P)),
                                 ctypes.byref(Stencil(s, float(near_radius))), nrhs, precision, ctypes.byref(out)),
           "aim_query_bytes")
    return out.value


def query_solve_bytes(nodes, form: int, m: int, s: int = 4, quad_p: int = 4, fft_P: int = 0, nrhs: int = 1,
                      restart: int = 50, precision: int = FP64, near_radius: float = 0.0) -> int:
    """Upper bound on the device bytes of a context after aim_setup + aim_solve(nrhs, restart, precision)."""
    g, keep = _geometry(nodes, form, quad_p)
    out = ctypes.c_size_t(0)
    opts = SolveOpts(1e-8, int(restart), 1, int(precision), 0.0, 0)
    _check(lib().aim_query_solve_bytes(ctypes.byref(g), ctypes.byref(Grid(m, 0.0, fft_P)),
                                       ctypes.byref(Stencil(s, float(near_radius))), int(nrhs), ctypes.byref(opts),
                                       ctypes.byref(out)), "aim_query_solve_bytes")
    return out.value


def _setup_args(nodes, form, m, fft_P, L, s, quad_p, near_radius, alpha, filter_kind):
    g, keep = _geometry(nodes, form, quad_p)
    flt = Filter(int(filter_kind) if alpha is not None else FILTER_NONE, float(alpha) if alpha is not None else 0.0)
    return g, keep, Grid(int(m), float(L), int(fft_P)), Stencil(int(s), float(near_radius)), flt


def setup_key(nodes, k: float, form: int, m: int, fft_P: int = 0, L: float = 0.0, s: int = 4, quad_p: int = 4,
              near_radius: float = 0.0, alpha: Optional[float] = None, filter_kind: int = FILTER_NUMERICAL) -> str:
    """aim_setup_key of a problem (Context's arguments) as 16 hex digits; host only."""
    g, keep, grid, sten, flt = _setup_args(nodes, form, m, fft_P, L, s, quad_p, near_radius, alpha, filter_kind)
    key = ctypes.c_ulonglong(0)
    _check(lib().aim_setup_key(ctypes.byref(g), float(k), ctypes.byref(grid), ctypes.byref(sten), ctypes.byref(flt),
                               ctypes.byref(key)), "aim_setup_key")
    return "%016x" % key.value


class SetupCache:
    """Setup blobs on disk, one file per problem key, so that a restarted process reloads its
    contexts (aim_import_setup) instead of recomputing them. A file that the library refuses
    (another format version, a corrupted or truncated write, a key collision) is rebuilt and
    replaced; files are written to a temporary name and renamed, so readers never see half a blob."""

    SUFFIX = ".aimsetup"

    def __init__(self, directory: str):
        self.directory = os.path.abspath(directory)
        os.makedirs(self.directory, exist_ok=True)
        self.hits = 0
        self.misses = 0
        self.rejected = 0
        self._lock = threading.Lock()

    def path(self, key: str) -> str:
        return os.path.join(self.directory, key + self.SUFFIX)

    def context(self, nodes, k: float, form: int, m: int, stream=None, **kw) -> "Context":
        """The problem's context: imported from its blob when the directory holds a valid one,
        else set up and its blob written."""
        key = setup_key(nodes, k, form, m, **kw)
        path = self.path(key)
        if os.path.exists(path):
            blob = np.fromfile(path, dtype=np.uint8)
            try:
                ctx = Context(nodes, k, form, m, stream=stream, blob=blob, **kw)
                with self._lock:
                    self.hits += 1
                return ctx
            except AimError as e:
                if e.status != EINVAL:
                    raise
                with self._lock:
                    self.rejected += 1
        ctx = Context(nodes, k, form, m, stream=stream, **kw)
        with self._lock:
            self.misses += 1
        tmp = "%s.%d.%d.tmp" % (path, os.getpid(), threading.get_ident())
        ctx.export_setup(stream).tofile(tmp)
        os.replace(tmp, path)
        return ctx

    def stats(self) -> dict:
        with self._lock:
            return {"hits": self.hits, "misses": self.misses, "rejected": self.rejected}


class Context:
    """One AIM operator set on the current CUDA device (wraps aim_ctx*)."""

    def __init__(self, nodes, k: float, form: int, m: int, fft_P: int = 0, L: float = 0.0, s: int = 4,
                 quad_p: int = 4, near_radius: float = 0.0, alpha: Optional[float] = None, stream=None,
                 filter_kind: int = FILTER_NUMERICAL, blob=None):
        """aim_setup of the problem; with `blob` (bytes or a uint8 array from export_setup),
        aim_import_setup of it instead, which refuses a blob of any other problem (EINVAL)."""
        g, keep, grid, sten, flt = _setup_args(nodes, form, m, fft_P, L, s, quad_p, near_radius, alpha, filter_kind)
        h = ctypes.c_void_p()
        if blob is None:
            _check(lib().aim_setup(ctypes.byref(g), float(k), ctypes.byref(grid), ctypes.byref(sten),
                                   ctypes.byref(flt), _stream_ptr(stream), ctypes.byref(h)), "aim_setup")
        else:
            buf = np.ascontiguousarray(np.frombuffer(blob, dtype=np.uint8) if isinstance(blob, (bytes, bytearray))
                                       else np.asarray(blob, dtype=np.uint8).reshape(-1))
            _check(lib().aim_import_setup(ctypes.byref(g), float(k), ctypes.byref(grid), ctypes.byref(sten),
                                          ctypes.byref(flt), buf.ctypes.data, buf.size, _stream_ptr(stream),
                                          ctypes.byref(h)), "aim_import_setup")
        self._h = h
        self.form = form
        inf = self.info()
        self.n = inf["n"]
        self.m = inf["m"]

    def export_setup(self, stream=None) -> np.ndarray:
        """The context's setup blob (aim_export_setup) as a uint8 array."""
        size = ctypes.c_size_t(0)
        _check(lib().aim_export_setup(self._h, None, ctypes.byref(size), _stream_ptr(stream)), "aim_export_setup")
        buf = np.empty(size.value, dtype=np.uint8)
        _check(lib().aim_export_setup(self._h, buf.ctypes.data, ctypes.byref(size), _stream_ptr(stream)),
               "aim_export_setup")
        return buf

    def close(self):
        if getattr(self, "_h", None):
            lib().aim_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def info(self) -> dict:
        inf = Info()
        _check(lib().aim_get_info(self._h, ctypes.byref(inf)), "aim_get_info")
        return {name: getattr(inf, name) for name, _ in Info._fields_}

    def reserve(self, nrhs: int, precision: int = FP64):
        _check(lib().aim_reserve(self._h, int(nrhs), int(precision)), "aim_reserve")

    def autotune(self, nrhs: int = 1, precision: int = FP64, stream=None) -> dict:
        """Pick the fastest launch schedule for this context; returns it."""
        chosen = Schedule()
        _check(lib().aim_autotune(self._h, int(nrhs), int(precision), _stream_ptr(stream), ctypes.byref(chosen)),
               "aim_autotune")
        return chosen.as_dict()

    def set_schedule(self, precision: int, transforms_per_thread: int, row_threads: int, col_cols: int = 0,
                     elems_per_thread: int = 16):
        sc = Schedule(int(transforms_per_thread), int(row_threads), int(col_cols), int(elems_per_thread))
        _check(lib().aim_set_schedule(self._h, int(precision), ctypes.byref(sc)), "aim_set_schedule")

    def get_schedule(self, precision: int) -> dict:
        sc = Schedule()
        _check(lib().aim_get_schedule(self._h, int(precision), ctypes.byref(sc)), "aim_get_schedule")
        return sc.as_dict()

    def kernel_table(self, which: int, out, stream=None):
        """(H+1) x (H+1) grid kernel table (aim_kernel_table): spectra or analytic samples."""
        _check(lib().aim_kernel_table(self._h, int(which), _ptr(out), _stream_ptr(stream)), "aim_kernel_table")
        return out

    def lanczos_bidiag(self, op, k: int, v0, precision: int = FP64, U=None, V=None, stream=None):
        """k Golub-Kahan-Lanczos steps from v0 (aim_lanczos_bidiag): returns (alpha, beta) as numpy arrays."""
        op = OPS[op] if isinstance(op, str) else int(op)
        alpha = np.zeros(int(k), dtype=np.float64)
        beta = np.zeros(int(k), dtype=np.float64)
        _check(lib().aim_lanczos_bidiag(self._h, op, int(k), int(precision), _ptr(v0),
                                        alpha.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        beta.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        _ptr(U) if U is not None else None, _ptr(V) if V is not None else None,
                                        _stream_ptr(stream)), "aim_lanczos_bidiag")
        return alpha, beta

    def rhs_planewave(self, angles, out, stream=None):
        ang = np.ascontiguousarray(np.asarray(angles, dtype=np.float64).reshape(-1))
        _check(lib().aim_rhs_planewave(self._h, int(ang.size), ang.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       _ptr(out), _stream_ptr(stream)), "aim_rhs_planewave")
        return out

    def matvec(self, op, x, y, precision: int = FP64, stream=None):
        op = OPS[op] if isinstance(op, str) else int(op)
        nrhs = x.shape[0] if x.ndim == 2 else 1
        _check(lib().aim_matvec(self._h, op, int(nrhs), _ptr(x), _ptr(y), int(precision), _stream_ptr(stream)),
               "aim_matvec")
        return y

    def grid_product(self, u, v, filtered: bool, precision: int = FP64, stream=None):
        nrhs = u.shape[0] if u.ndim == 3 else 1
        _check(lib().aim_grid_product(self._h, int(bool(filtered)), int(nrhs), _ptr(u), _ptr(v), int(precision),
                                      _stream_ptr(stream)), "aim_grid_product")
        return v

    def grid_product_noalloc(self, u, v, filtered: bool, precision: int = FP64, stream=None):
        """aim_grid_product without allocation (library-owned scratch; device pointers only)."""
        nrhs = u.shape[0] if u.ndim == 3 else 1
        _check(lib().aim_grid_product_noalloc(self._h, int(bool(filtered)), int(nrhs), _ptr(u), _ptr(v),
                                              int(precision), _stream_ptr(stream)), "aim_grid_product_noalloc")
        return v

    def solve(self, system, rhs, x, tol=1e-8, restart=50, max_iter=1000, precision: int = FP64, inner_tol=0.0,
              timeout_ms=0, x0_given=False, stream=None, check=True, batcher: Optional["Batcher"] = None):
        system = OPS[system] if isinstance(system, str) else int(system)
        nrhs = rhs.shape[0] if rhs.ndim == 2 else 1
        opts = SolveOpts(float(tol), int(restart), int(max_iter), int(precision), float(inner_tol), int(timeout_ms))
        infos = (SolveInfo * nrhs)()
        if batcher is not None:
            st = lib().aim_solve_batched(batcher._h, self._h, system, int(nrhs), _ptr(rhs), _ptr(x), int(bool(x0_given)),
                                         ctypes.byref(opts), infos, _stream_ptr(stream))
        else:
            st = lib().aim_solve(self._h, system, int(nrhs), _ptr(rhs), _ptr(x), int(bool(x0_given)),
                                 ctypes.byref(opts), infos, _stream_ptr(stream))
        out = [{"iters": i.iters, "outer_iters": i.outer_iters, "rel_res": i.rel_res, "converged": i.converged}
               for i in infos]
        if check:
            _check(st, "aim_solve")
        return out if check else (st, out)
