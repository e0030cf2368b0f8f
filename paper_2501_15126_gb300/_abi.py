"""ctypes binding of libperm.so (include/perm.h): argument marshalling only.

Every permanent is computed by the library's CUDA kernels; this module only
converts numpy matrices to the C structs and back.  If libperm.so is missing
it raises: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libperm.so")

# perm_status_t
PERM_OK, PERM_ERR_ARG, PERM_ERR_SIZE, PERM_ERR_PATTERN, PERM_ERR_OVERFLOW, PERM_ERR_CUDA, PERM_ERR_NVRTC, \
    PERM_ERR_NOMEM, PERM_ERR_TIMEOUT, PERM_ERR_BUSY, PERM_ERR_NOT_READY, PERM_ERR_CANCELLED, PERM_ERR_INTERNAL = range(13)
PERM_F64, PERM_I64 = 0, 1
PERM_CSR, PERM_CSC = 0, 1
PERM_ORDER_AUTO, PERM_ORDER_NONE, PERM_ORDER_DEGREE, PERM_ORDER_PAPER, PERM_ORDER_SEARCH = 0, 1, 2, 3, 4
PERM_ENGINE_AUTO, PERM_ENGINE_GENERIC, PERM_ENGINE_CODEGEN, PERM_ENGINE_XSHARED = 0, 1, 2, 3
PERM_FLAG_NO_KERNEL_CACHE = 1
PERM_FLAG_NO_GRAPH = 2
PERM_FLAG_PAIRED_CHAIN = 4
PERM_FLAG_PURE_REG = 8
PERM_FLAG_ABS_SUM = 16
PERM_PREC_AUTO, PERM_PREC_F64, PERM_PREC_DD = 0, 1, 2
PERM_SITE_WAVE_LAUNCH, PERM_SITE_NVRTC, PERM_SITE_FINISH, PERM_SITE_UPLOAD, PERM_SITE_LAUNCH = 1, 2, 3, 4, 5

c_i32, c_i64, c_u64, c_dbl, c_vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p


class Matrix(ctypes.Structure):
    _fields_ = [("n", c_i32), ("nnz", c_i32), ("layout", c_i32), ("ptr", c_vp), ("idx", c_vp),
                ("vtype", c_i32), ("vals", c_vp)]


class Opts(ctypes.Structure):
    _fields_ = [("ordering", c_i32), ("engine", c_i32), ("reg_rows", c_i32), ("chunk_log2", c_i32),
                ("threads", c_i32), ("exact_words", c_i32), ("zero_skip", c_i32), ("flags", c_i32),
                ("gr_ratio", c_dbl), ("g_lo", c_u64), ("g_hi", c_u64), ("timeout_ms", c_i32), ("precision", c_i32),
                ("shared_rows", c_i32), ("reserved2", c_i32)]


class Result(ctypes.Structure):
    _fields_ = [("status", c_i32), ("vtype", c_i32), ("f64", c_dbl), ("f64_lo", c_dbl),
                ("i128_lo", c_u64), ("i128_hi", c_i64), ("partial", c_u64 * 3),
                ("exact_words", c_i32), ("engine", c_i32), ("ordering", c_i32), ("reg_rows", c_i32),
                ("reg_cols", c_i32), ("chunk_log2", c_i32), ("threads", c_i32), ("regs_per_thread", c_i32),
                ("steps", c_u64), ("ms_plan", c_dbl), ("ms_compile", c_dbl), ("ms_kernel", c_dbl),
                ("fp_ops_per_step", c_dbl), ("zero_skip_frac", c_dbl), ("abs_term_sum", c_dbl),
                ("precision", c_i32), ("shared_rows", c_i32)]

    @property
    def exact(self) -> int:
        v = (int(self.i128_hi) << 64) | int(self.i128_lo)
        return v

    @property
    def value(self):
        """The permanent: a Python int (exact path) or float (FP64 path)."""
        return self.exact if self.vtype == PERM_I64 else self.f64 + self.f64_lo

    @property
    def partial_int(self) -> int:
        return sum(int(self.partial[i]) << (64 * i) for i in range(max(self.exact_words, 1)))


class Inspect(ctypes.Structure):
    _fields_ = [("n", c_i32), ("structurally_zero", c_i32), ("ordering", c_i32),
                ("col_order", c_i32 * 64), ("row_order", c_i32 * 64), ("group_of_row", c_i32 * 64),
                ("group_size", c_i32 * 64), ("col_nnz", c_i32 * 64), ("reg_rows", c_i32), ("reg_cols", c_i32),
                ("exact_words", c_i32), ("bound_log2", c_dbl), ("ops_per_step", c_dbl),
                ("ops_per_step_paper", c_dbl), ("exact_limbs", c_i32), ("reserved0", c_i32),
                ("ops_per_step_walk", c_dbl), ("ring_ops_per_step", c_dbl),
                ("ops_per_step_four_state", c_dbl), ("ops_per_step_four_state_searched", c_dbl)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("max_inflight", c_i32), ("max_n", c_i32), ("step_budget", c_dbl), ("device", c_i32),
                ("timeout_ms", c_i32), ("precision", c_i32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", c_u64), ("rejected", c_u64), ("failed", c_u64), ("p50_ms", c_dbl),
                ("p99_ms", c_dbl), ("max_ms", c_dbl), ("perms_per_s", c_dbl)]


STRUCTS = [Matrix, Opts, Result, Inspect, ServerOpts, ServerStats]

# (name, restype, argtypes) of every entry point declared in include/perm.h
SIGNATURES = [
    ("perm_plan_create", c_i32, [ctypes.POINTER(Matrix), ctypes.POINTER(Opts), ctypes.POINTER(c_vp)]),
    ("perm_compute", c_i32, [c_vp, c_vp, ctypes.POINTER(Result)]),
    ("perm_plan_destroy", None, [c_vp]),
    ("perm_batch", c_i32, [ctypes.POINTER(Matrix), c_i32, ctypes.POINTER(Opts), c_vp, ctypes.POINTER(Result)]),
    ("perm_batch_sequential", c_i32, [ctypes.POINTER(Matrix), c_i32, ctypes.POINTER(Opts), c_vp,
                                      ctypes.POINTER(Result)]),
    ("perm_server_create", c_i32, [ctypes.POINTER(ServerOpts), ctypes.POINTER(c_vp)]),
    ("perm_submit", c_i32, [c_vp, ctypes.POINTER(Matrix), ctypes.POINTER(c_u64)]),
    ("perm_poll", c_i32, [c_vp, c_u64, c_i32, ctypes.POINTER(Result)]),
    ("perm_server_stats", c_i32, [c_vp, ctypes.POINTER(ServerStats)]),
    ("perm_server_destroy", None, [c_vp]),
    ("perm_inspect", c_i32, [ctypes.POINTER(Matrix), ctypes.POINTER(Opts), ctypes.POINTER(Inspect)]),
    ("perm_scbs", c_i32, [c_i32, ctypes.POINTER(c_i32)]),
    ("perm_alg2_launches", c_i32, [c_i64, c_i32, ctypes.POINTER(c_i64), ctypes.POINTER(c_i64),
                                   ctypes.POINTER(c_i64), c_i32, ctypes.POINTER(c_i32)]),
    ("perm_codegen_source", c_i32, [ctypes.POINTER(Matrix), ctypes.POINTER(Opts), ctypes.c_char_p, c_i64,
                                    ctypes.POINTER(c_i64)]),
    ("perm_generic_image", c_i32, [ctypes.POINTER(Matrix), ctypes.POINTER(Opts), c_vp, c_i64, ctypes.POINTER(c_i64),
                                   ctypes.POINTER(c_i32), ctypes.POINTER(c_i32), ctypes.POINTER(c_i32)]),
    ("perm_status_string", ctypes.c_char_p, [c_i32]),
    ("perm_last_error", ctypes.c_char_p, []),
    ("perm_device_available", c_i32, []),
    ("perm_version", ctypes.c_char_p, []),
    ("perm_sizeof", c_i64, [c_i32]),
    ("perm_issue_rates", c_i32, [c_vp, ctypes.POINTER(c_dbl), ctypes.POINTER(c_dbl)]),
    ("perm_compute_noalloc", c_i32, [ctypes.POINTER(Matrix), ctypes.POINTER(Opts), c_vp, ctypes.POINTER(Result)]),
    ("perm_debug_inject_failures", c_i32, [c_i32, c_i32]),
    ("perm_checkpoint_run", c_i32, [ctypes.POINTER(Matrix), ctypes.POINTER(Opts), ctypes.c_char_p, c_i32, c_i32, c_vp,
                                    ctypes.POINTER(Result)]),
]

_lib = None


def lib():
    """Loads libperm.so (built by paper_2501_15126_gb300.build); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libperm.so is not built (run __graft_entry__.build()); there is no fallback path")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class PermError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().perm_last_error().decode(errors="replace")
        super().__init__("%s: %s (%s)" % (where, lib().perm_status_string(status).decode(), msg))


def check(status: int, where: str):
    if status != PERM_OK:
        raise PermError(status, where)


class CSRMatrix:
    """Keeps the numpy buffers of a perm_matrix_t alive."""

    def __init__(self, a: np.ndarray | None = None, *, n=None, ptr=None, idx=None, vals=None, layout=PERM_CSR,
                 vtype=None):
        if a is not None:
            a = np.asarray(a)
            n = a.shape[0]
            nz = a != 0
            ptr = np.zeros(n + 1, dtype=np.int32)
            ptr[1:] = np.cumsum(nz.sum(axis=1))
            rows, cols = np.nonzero(nz)
            idx = cols.astype(np.int32)
            if vtype is None:
                vtype = PERM_I64 if np.issubdtype(a.dtype, np.integer) else PERM_F64
            vals = a[rows, cols]
        self.ptr = np.ascontiguousarray(ptr, dtype=np.int32)
        self.idx = np.ascontiguousarray(idx, dtype=np.int32)
        self.vals = np.ascontiguousarray(vals, dtype=np.int64 if vtype == PERM_I64 else np.float64)
        self.c = Matrix(int(n), int(len(self.idx)), int(layout), self.ptr.ctypes.data, self.idx.ctypes.data,
                        int(vtype), self.vals.ctypes.data)


def opts(**kw) -> Opts:
    o = Opts()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Plan:
    def __init__(self, a, **kw):
        self.m = a if isinstance(a, CSRMatrix) else CSRMatrix(a)
        self.o = opts(**kw)
        h = c_vp()
        check(lib().perm_plan_create(ctypes.byref(self.m.c), ctypes.byref(self.o), ctypes.byref(h)),
              "perm_plan_create")
        self.h = h

    def compute(self, stream: int = 0) -> Result:
        r = Result()
        check(lib().perm_compute(self.h, c_vp(stream), ctypes.byref(r)), "perm_compute")
        return r

    def close(self):
        if self.h:
            lib().perm_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def permanent(a, stream: int = 0, **kw) -> Result:
    """One permanent: plan, compute, destroy."""
    p = Plan(a, **kw)
    try:
        return p.compute(stream)
    finally:
        p.close()


def permanent_noalloc(a, stream: int = 0, **kw) -> Result:
    """perm_compute_noalloc: the same permanent without any allocation."""
    m = a if isinstance(a, CSRMatrix) else CSRMatrix(a)
    o = opts(**kw)
    r = Result()
    check(lib().perm_compute_noalloc(ctypes.byref(m.c), ctypes.byref(o), c_vp(stream), ctypes.byref(r)),
          "perm_compute_noalloc")
    return r


def checkpoint_run(a, path: str, slice_log2: int, max_slices: int = 0, stream: int = 0, **kw):
    """perm_checkpoint_run: (status, Result); status is PERM_OK or PERM_ERR_NOT_READY."""
    m = a if isinstance(a, CSRMatrix) else CSRMatrix(a)
    o = opts(**kw)
    r = Result()
    st = lib().perm_checkpoint_run(ctypes.byref(m.c), ctypes.byref(o), path.encode(), slice_log2, max_slices,
                                   c_vp(stream), ctypes.byref(r))
    if st not in (PERM_OK, PERM_ERR_NOT_READY):
        check(st, "perm_checkpoint_run")
    return st, r


def inspect(a, **kw) -> Inspect:
    m = a if isinstance(a, CSRMatrix) else CSRMatrix(a)
    o = opts(**kw)
    out = Inspect()
    check(lib().perm_inspect(ctypes.byref(m.c), ctypes.byref(o), ctypes.byref(out)), "perm_inspect")
    return out


def scbs(k: int) -> list[int]:
    out = (c_i32 * ((1 << k) - 1))()
    check(lib().perm_scbs(k, out), "perm_scbs")
    return list(out)


def alg2_launches(tau: int, n: int, cap: int = 64):
    s, d, e = (c_i64 * cap)(), (c_i64 * cap)(), (c_i64 * cap)()
    cnt = c_i32()
    check(lib().perm_alg2_launches(tau, n, s, d, e, cap, ctypes.byref(cnt)), "perm_alg2_launches")
    return [(s[i], d[i], e[i]) for i in range(min(cnt.value, cap))]


def codegen_source(a, **kw) -> str:
    m = a if isinstance(a, CSRMatrix) else CSRMatrix(a)
    o = opts(**kw)
    n = c_i64()
    check(lib().perm_codegen_source(ctypes.byref(m.c), ctypes.byref(o), None, 0, ctypes.byref(n)), "codegen")
    buf = ctypes.create_string_buffer(n.value + 1)
    check(lib().perm_codegen_source(ctypes.byref(m.c), ctypes.byref(o), buf, n.value + 1, ctypes.byref(n)),
          "codegen")
    return buf.value.decode()


def generic_image(a, **kw):
    """perm_generic_image: (image bytes, NMAX bucket, kernel family, abs_shift)."""
    m = a if isinstance(a, CSRMatrix) else CSRMatrix(a)
    o = opts(**kw)
    n, nmax, kind, shift = c_i64(), c_i32(), c_i32(), c_i32()
    check(lib().perm_generic_image(ctypes.byref(m.c), ctypes.byref(o), None, 0, ctypes.byref(n), ctypes.byref(nmax),
                                   ctypes.byref(kind), ctypes.byref(shift)), "perm_generic_image")
    buf = ctypes.create_string_buffer(n.value)
    check(lib().perm_generic_image(ctypes.byref(m.c), ctypes.byref(o), buf, n.value, ctypes.byref(n), None, None,
                                   None), "perm_generic_image")
    return buf.raw[: n.value], nmax.value, kind.value, shift.value


def issue_rates(stream: int = 0):
    """(FP64 ops/s, IMAD ops/s) measured on the current GPU."""
    f, i = c_dbl(), c_dbl()
    check(lib().perm_issue_rates(c_vp(stream), ctypes.byref(f), ctypes.byref(i)), "perm_issue_rates")
    return f.value, i.value


class Server:
    """perm_server_create / perm_submit / perm_poll / perm_server_destroy."""

    def __init__(self, max_inflight=0, max_n=0, step_budget=0.0, device=0, timeout_ms=0, precision=0):
        o = ServerOpts(max_inflight, max_n, step_budget, device, timeout_ms, precision)
        h = c_vp()
        check(lib().perm_server_create(ctypes.byref(o), ctypes.byref(h)), "perm_server_create")
        self.h = h
        self._keep = {}

    def submit(self, a) -> int:
        m = a if isinstance(a, CSRMatrix) else CSRMatrix(a)
        t = c_u64()
        st = lib().perm_submit(self.h, ctypes.byref(m.c), ctypes.byref(t))
        check(st, "perm_submit")
        return t.value

    def poll(self, ticket: int, timeout_ms: int = -1):
        """Result, or None when not ready within timeout_ms."""
        r = Result()
        st = lib().perm_poll(self.h, ticket, timeout_ms, ctypes.byref(r))
        if st == PERM_ERR_NOT_READY:
            return None
        check(st, "perm_poll")
        return r

    def stats(self) -> ServerStats:
        s = ServerStats()
        check(lib().perm_server_stats(self.h, ctypes.byref(s)), "perm_server_stats")
        return s

    def close(self):
        if self.h:
            lib().perm_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def inject_failures(site: int, count: int):
    """perm_debug_inject_failures: the next `count` calls at `site` take their error path."""
    check(lib().perm_debug_inject_failures(site, count), "perm_debug_inject_failures")


def batch(mats, sequential: bool = False, stream: int = 0, **kw):
    ms = [m if isinstance(m, CSRMatrix) else CSRMatrix(m) for m in mats]
    arr = (Matrix * len(ms))(*[m.c for m in ms])
    res = (Result * len(ms))()
    o = opts(**kw)
    fn = lib().perm_batch_sequential if sequential else lib().perm_batch
    check(fn(arr, len(ms), ctypes.byref(o), c_vp(stream), res), "perm_batch")
    return list(res)
