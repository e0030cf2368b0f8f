"""The CPU oracle for the sparse-permanent hot path (test infrastructure only).

Only the test-suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this package.  The product path never does.  It shares
no code with the CUDA path: the C source ``perm_oracle.c`` is compiled on its own
with gcc and loaded here with ctypes.

Functions take dense numpy matrices (float64 or int64, row-major) and follow the
paper's definitions:

* ``brute``            Eq. 1, the sum over all permutations (n <= 10).
* ``ryser``            Eq. 2, every column subset, exact modulo 2^128.
* ``ryser_gray``       Eq. 2 walked in Gray-code order (Sec. II), exact modulo 2^128.
* ``nw_range``         Algorithm 1 (Nijenhuis-Wilf) over a Gray-index range, long double,
                       with the start vector of Sec. II-A.
* ``nw_perm``          Algorithm 1 over the whole range times (4 (n mod 2) - 2).
* ``nw2_range``        Algorithm 1 with doubled x, in integers modulo 2^128.
* ``band_dp``          row-by-row dynamic program for banded matrices (independent of Ryser).
* ``rowdp``            Eq. 1 expanded row by row with equal subproblems merged: a permanent
                       for sparse matrices of any n <= 64 (independent of Ryser and of the walk).

Parity of every function is pinned in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "perm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MASK128 = (1 << 128) - 1


def build(force: bool = False) -> str:
    """Compiles perm_oracle.c into liboracle.so next to it (gcc, -ffp-contract=off)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def load(path: str):
    """Loads a compiled oracle library and declares its signatures."""
    L = ctypes.CDLL(path)
    i32, u64, p = ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p
    pld = ctypes.POINTER(ctypes.c_longdouble)
    pu64 = ctypes.POINTER(ctypes.c_uint64)
    L.oracle_brute_ld.argtypes = [i32, p, pld]
    L.oracle_brute_u128.argtypes = [i32, p, pu64, pu64]
    L.oracle_ryser_u128.argtypes = [i32, p, pu64, pu64]
    L.oracle_ryser_gray_range_u128.argtypes = [i32, p, u64, u64, pu64, pu64]
    L.oracle_nw_range_ld.argtypes = [i32, p, u64, u64, pld, pld]
    L.oracle_nw_perm_ld.argtypes = [i32, p, pld, pld]
    L.oracle_nw2_range_u128.argtypes = [i32, p, u64, u64, pu64, pu64]
    L.oracle_band_dp_ld.argtypes = [i32, i32, p, pld]
    L.oracle_band_dp_u128.argtypes = [i32, i32, p, pu64, pu64]
    L.oracle_rowdp_ld.argtypes = [i32, p, p, u64, pld]
    L.oracle_rowdp_u128.argtypes = [i32, p, p, u64, pu64, pu64]
    L.oracle_nw_range_ld_mt.argtypes = [i32, p, u64, u64, i32, pld, pld]
    L.oracle_nw2_range_u128_mt.argtypes = [i32, p, u64, u64, i32, pu64, pu64]
    L.oracle_ld_to_dd.argtypes = [pld, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    for name in ("oracle_brute_ld", "oracle_brute_u128", "oracle_ryser_u128",
                 "oracle_ryser_gray_range_u128", "oracle_nw_range_ld", "oracle_nw_perm_ld",
                 "oracle_nw2_range_u128", "oracle_band_dp_ld", "oracle_band_dp_u128",
                 "oracle_rowdp_ld", "oracle_rowdp_u128",
                 "oracle_nw_range_ld_mt", "oracle_nw2_range_u128_mt",
                 "oracle_long_double_bits", "oracle_long_double_mant_dig"):
        getattr(L, name).restype = ctypes.c_int
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load(build())
        return _lib


class using_library:
    """Context manager that swaps in another compiled copy of the oracle (the
    mutation tests use it to check that the pins catch planted mistakes)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        lib()
        self.saved = _lib
        _lib = load(self.path)
        return _lib

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


class LD:
    """A long double result held as an unevaluated double pair hi + lo."""

    __slots__ = ("hi", "lo")

    def __init__(self, v: ctypes.c_longdouble):
        hi, lo = ctypes.c_double(), ctypes.c_double()
        lib().oracle_ld_to_dd(ctypes.byref(v), ctypes.byref(hi), ctypes.byref(lo))
        self.hi, self.lo = hi.value, lo.value

    def __float__(self):
        return self.hi + self.lo

    def __repr__(self):
        return "LD(%r + %r)" % (self.hi, self.lo)


def _f64(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    assert a.ndim == 2 and a.shape[0] == a.shape[1]
    return a


def _i64(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.int64)
    assert a.ndim == 2 and a.shape[0] == a.shape[1]
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError("%s failed with code %d" % (what, rc))


def to_signed128(lo: int, hi: int) -> int:
    v = (hi << 64) | lo
    return v - (1 << 128) if v >> 127 else v


def _u128(fn, *args) -> int:
    lo, hi = ctypes.c_uint64(), ctypes.c_uint64()
    _check(fn(*args, ctypes.byref(lo), ctypes.byref(hi)), fn.__name__)
    return (hi.value << 64) | lo.value


def brute(a) -> LD:
    """Eq. 1 in long double (n <= 10 keeps it quick)."""
    a = _f64(a)
    out = ctypes.c_longdouble()
    _check(lib().oracle_brute_ld(a.shape[0], _ptr(a), ctypes.byref(out)), "brute")
    return LD(out)


def brute_int(a) -> int:
    """Eq. 1 in integers modulo 2^128, returned as a signed Python int."""
    a = _i64(a)
    v = _u128(lib().oracle_brute_u128, a.shape[0], _ptr(a))
    return to_signed128(v & ((1 << 64) - 1), v >> 64)


def ryser(a) -> int:
    """Eq. 2 written out over every subset, modulo 2^128, signed."""
    a = _i64(a)
    v = _u128(lib().oracle_ryser_u128, a.shape[0], _ptr(a))
    return to_signed128(v & ((1 << 64) - 1), v >> 64)


def ryser_gray(a, k_lo: int = 0, k_hi: int | None = None, signed_perm: bool = True) -> int:
    """Eq. 2 in Gray order.  Over the full range returns perm(A) (signed, mod 2^128);
    over a sub-range returns the raw partial sum modulo 2^128 (unsigned)."""
    a = _i64(a)
    n = a.shape[0]
    full = k_hi is None and k_lo == 0
    if k_hi is None:
        k_hi = 1 << n
    v = _u128(lib().oracle_ryser_gray_range_u128, n, _ptr(a), k_lo, k_hi)
    if full and signed_perm:
        if n & 1:
            v = (-v) & MASK128
        return to_signed128(v & ((1 << 64) - 1), v >> 64)
    return v


def nw_range(a, g_lo: int, g_hi: int, threads: int = 1):
    """Algorithm 1 partial sum over Gray indices [g_lo, g_hi): (sum, sum of |terms|)."""
    a = _f64(a)
    s, sa = ctypes.c_longdouble(), ctypes.c_longdouble()
    if threads > 1:
        rc = lib().oracle_nw_range_ld_mt(a.shape[0], _ptr(a), g_lo, g_hi, threads, ctypes.byref(s), ctypes.byref(sa))
    else:
        rc = lib().oracle_nw_range_ld(a.shape[0], _ptr(a), g_lo, g_hi, ctypes.byref(s), ctypes.byref(sa))
    _check(rc, "nw_range")
    return LD(s), LD(sa)


def nw_perm(a, threads: int = 1):
    """Algorithm 1 over the whole Gray range: (perm, sum of |terms| times |4(n mod 2)-2|)."""
    a = _f64(a)
    n = a.shape[0]
    if threads > 1:
        s, sa = nw_range(a, 0, 1 << (n - 1), threads)
        f = float(4 * (n % 2) - 2)
        res = LD.__new__(LD); res.hi, res.lo = s.hi * f, s.lo * f
        ab = LD.__new__(LD); ab.hi, ab.lo = sa.hi * 2.0, sa.lo * 2.0
        return res, ab
    p, sa = ctypes.c_longdouble(), ctypes.c_longdouble()
    _check(lib().oracle_nw_perm_ld(n, _ptr(a), ctypes.byref(p), ctypes.byref(sa)), "nw_perm")
    return LD(p), LD(sa)


def nw2_range(a, g_lo: int, g_hi: int, threads: int = 1) -> int:
    """Algorithm 1 with doubled x: sum_g (-1)^g prod_i 2x_i(g) modulo 2^128 (unsigned)."""
    a = _i64(a)
    n = a.shape[0]
    if threads > 1:
        return _u128(lib().oracle_nw2_range_u128_mt, n, _ptr(a), g_lo, g_hi, threads)
    return _u128(lib().oracle_nw2_range_u128, n, _ptr(a), g_lo, g_hi)


def band_dp(a, w: int) -> LD:
    a = _f64(a)
    out = ctypes.c_longdouble()
    _check(lib().oracle_band_dp_ld(a.shape[0], w, _ptr(a), ctypes.byref(out)), "band_dp")
    return LD(out)


def band_dp_int(a, w: int) -> int:
    a = _i64(a)
    v = _u128(lib().oracle_band_dp_u128, a.shape[0], w, _ptr(a))
    return to_signed128(v & ((1 << 64) - 1), v >> 64)


def rowdp_order(a) -> list[int]:
    """A row order that keeps rowdp's states few: each next row is the one
    whose nonzero columns add the fewest columns not yet touched (any order
    gives the same permanent; this one only keeps the state sets small)."""
    nz = np.asarray(a) != 0
    n = nz.shape[0]
    seen = np.zeros(n, dtype=bool)
    left = list(range(n))
    order = []
    while left:
        r = min(left, key=lambda i: (int((nz[i] & ~seen).sum()), i))
        left.remove(r)
        order.append(r)
        seen |= nz[r]
    return order


def _order_arg(order, n):
    o = np.ascontiguousarray(order if order is not None else range(n), dtype=np.int32)
    assert o.shape == (n,)
    return o


def rowdp(a, order=None, max_states: int = 1 << 22) -> LD:
    """perm(A) by rowdp in long double, rows in ``order`` (default: rowdp_order)."""
    a = _f64(a)
    o = _order_arg(rowdp_order(a) if order is None else order, a.shape[0])
    out = ctypes.c_longdouble()
    _check(lib().oracle_rowdp_ld(a.shape[0], _ptr(a), _ptr(o), max_states, ctypes.byref(out)), "rowdp")
    return LD(out)


def rowdp_int(a, order=None, max_states: int = 1 << 22) -> int:
    """perm(A) by rowdp in integers modulo 2^128, signed."""
    a = _i64(a)
    o = _order_arg(rowdp_order(a) if order is None else order, a.shape[0])
    v = _u128(lib().oracle_rowdp_u128, a.shape[0], _ptr(a), _ptr(o), max_states)
    return to_signed128(v & ((1 << 64) - 1), v >> 64)


def long_double_bits() -> int:
    return lib().oracle_long_double_mant_dig()
