"""Seeded synthetic workloads (inputs only; none of the permanent arithmetic).

Both the CUDA path (through the C ABI) and the CPU oracle are fed from these
generators, so the two sides see bit-identical matrices.  The random source is
numpy's PCG64 stream, whose output for a given seed is the same on every
platform.

Shapes follow the paper's synthetic set (Sec. VI-C: Erdos-Renyi nonzeros with
probability p, values drawn from the unit interval, matrices without a perfect
matching excluded) and the five workloads this library is measured on:

* ``single_er``     one ER matrix plus a forced nonzero diagonal (the diagonal
                    guarantees a perfect matching, i.e. perm != 0 for positive
                    values).  n=24/p=0.2 (0/1 values) and n=36/p=0.15 (real
                    values, columns shuffled) are the two single-matrix cases.
* ``band_plus``     a_ij != 0 iff |i-j| <= w, plus ``extra`` random off-band
                    nonzeros per row (n=48, w=3, extra=2); ``extra=0`` gives the
                    band-only sibling that a banded DP can check.
* ``batch``         many ER matrices of uneven n (n uniform in [12, 28], p
                    uniform in [0.2, 0.4], forced diagonal), alternating 0/1
                    and real values.
* ``serving_stream`` Poisson arrivals with n = 16 + m, P(m) proportional to
                    2^-m for m = 0..24, p uniform in [0.1, 0.3], forced
                    diagonal, value type a fair coin.
* ``table2_like``   six matrices with the shapes of the real-life set of
                    Table II (n, nnz, symmetric or not, diagonal or not) and
                    the value structure Sec. VI-E describes for them (mostly
                    distinct reals; all ones; over half +-1 with 40 distinct
                    values).  Patterns are random, not the real matrices.

Real values are (u + 1) * 2^-53 with u uniform on [0, 2^53): exactly
representable doubles in (0, 1].
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

TWO53 = 1 << 53


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def unit_values(g: np.random.Generator, size) -> np.ndarray:
    """Doubles (u + 1) * 2^-53, u uniform in [0, 2^53): every value lies in (0, 1]."""
    u = g.integers(0, TWO53, size=size, dtype=np.int64)
    return (u + 1).astype(np.float64) * (2.0 ** -53)


def fill_values(g: np.random.Generator, pattern: np.ndarray, values: str) -> np.ndarray:
    """Puts values on a boolean pattern: ``"01"`` -> int64 ones, ``"f64"`` -> (0, 1] doubles."""
    if values == "01":
        return pattern.astype(np.int64)
    if values == "f64":
        out = np.zeros(pattern.shape, dtype=np.float64)
        out[pattern] = unit_values(g, int(pattern.sum()))
        return out
    raise ValueError("values must be '01' or 'f64'")


def er_pattern(g: np.random.Generator, n: int, p: float, force_diag: bool = True) -> np.ndarray:
    pat = g.random((n, n)) < p
    if force_diag:
        np.fill_diagonal(pat, True)
    return pat


def single_er(n: int, p: float, seed: int, values: str = "f64", shuffle_cols: bool = False,
              force_diag: bool = True) -> np.ndarray:
    """One ER matrix (+ forced diagonal); optionally a seeded random column order."""
    g = rng(seed)
    pat = er_pattern(g, n, p, force_diag)
    a = fill_values(g, pat, values)
    if shuffle_cols:
        a = a[:, g.permutation(n)]
    return np.ascontiguousarray(a)


def single_er_pair(n: int, p: float, seed: int):
    """The same ER pattern twice: 0/1 values and (0, 1] values."""
    g = rng(seed)
    pat = er_pattern(g, n, p, True)
    return pat.astype(np.int64), fill_values(g, pat, "f64")


def band_plus(n: int = 48, w: int = 3, extra: int = 2, seed: int = 3, values: str = "01") -> np.ndarray:
    """Band |i-j| <= w plus ``extra`` distinct off-band columns per row."""
    g = rng(seed)
    idx = np.arange(n)
    pat = np.abs(idx[:, None] - idx[None, :]) <= w
    if extra:
        for i in range(n):
            off = np.flatnonzero(np.abs(idx - i) > w)
            pat[i, g.choice(off, size=extra, replace=False)] = True
    return np.ascontiguousarray(fill_values(g, pat, values))


@dataclass(frozen=True)
class Table2Shape:
    name: str              # the Table II matrix whose shape this copies
    n: int
    nnz: int
    symmetric: bool        # symmetric pattern (and values)
    diagonal: bool         # every diagonal entry present
    values: str            # "real": distinct (0,1] reals; "01": all ones; "pm1": > half +-1, 40 distinct


# Table II: name, n, nnz; the pattern kind and values follow Sec. VI-E's description of each matrix
# (stiffness, graph, mesh, power network, CFD, and d_ss's repeated +-1 values).
TABLE2_SHAPES = (
    Table2Shape("bcsstk01", 48, 400, True, True, "real"),
    Table2Shape("mycielskian6", 47, 472, True, False, "01"),
    Table2Shape("mesh1e1", 48, 306, True, True, "real"),
    Table2Shape("bcspwr02", 49, 167, True, True, "01"),
    Table2Shape("curtis54", 54, 291, False, True, "01"),
    Table2Shape("d_ss", 53, 144, False, True, "pm1"),
)


def table2_like(name: str, seed: int = 7) -> np.ndarray:
    """A random matrix with the shape of Table II's matrix ``name``: n, nnz,
    symmetry and diagonal as listed, values as Sec. VI-E describes them.  A
    pattern without a diagonal gets a random Hamiltonian cycle first, so it
    always has a perfect matching.  int64 for 0/1 values, float64 otherwise."""
    sh = next(t for t in TABLE2_SHAPES if t.name == name)
    g = rng(seed + 1000 * TABLE2_SHAPES.index(sh))
    n = sh.n
    pat = np.zeros((n, n), dtype=bool)
    if sh.diagonal:
        np.fill_diagonal(pat, True)
    else:
        cyc = g.permutation(n)
        for k in range(n):
            i, j = cyc[k], cyc[(k + 1) % n]
            pat[i, j] = pat[j, i] = True
    off = np.flatnonzero(~np.eye(n, dtype=bool).ravel())
    while int(pat.sum()) < sh.nnz:
        i, j = divmod(int(g.choice(off)), n)
        if pat[i, j]:
            continue
        if sh.symmetric:
            if int(pat.sum()) + 2 > sh.nnz:
                raise ValueError("a symmetric pattern needs an even off-diagonal count")
            pat[i, j] = pat[j, i] = True
        else:
            pat[i, j] = True
    if sh.values == "01":
        return pat.astype(np.int64)
    a = np.zeros((n, n), dtype=np.float64)
    if sh.values == "real":
        vals = unit_values(g, sh.nnz)
    else:   # "pm1": 55 % of the entries +1 or -1, the rest from 38 other distinct values
        pool = np.concatenate([[1.0, -1.0], np.round(g.uniform(-4.0, 4.0, 38), 3)])
        k1 = int(round(0.55 * sh.nnz))
        vals = np.concatenate([g.choice(pool[:2], k1), pool[2:], g.choice(pool[2:], sh.nnz - k1 - 38)])
        vals = vals[g.permutation(sh.nnz)]
    if sh.symmetric:
        iu = np.argwhere(np.triu(pat))
        for (i, j), v in zip(iu, vals):
            a[i, j] = a[j, i] = v
    else:
        a[pat] = vals
    return np.ascontiguousarray(a)


@dataclass
class BatchItem:
    a: np.ndarray          # dense; int64 for 0/1, float64 for real values
    values: str            # "01" or "f64"

    @property
    def n(self) -> int:
        return self.a.shape[0]


def batch(count: int = 10_000, n_lo: int = 12, n_hi: int = 28, p_lo: float = 0.2, p_hi: float = 0.4,
          seed: int = 4) -> list[BatchItem]:
    """``count`` ER matrices, n uniform in [n_lo, n_hi], p uniform in [p_lo, p_hi],
    forced diagonal, even items 0/1 and odd items real."""
    g = rng(seed)
    ns = g.integers(n_lo, n_hi + 1, size=count)
    ps = g.uniform(p_lo, p_hi, size=count)
    out = []
    for k in range(count):
        vals = "01" if k % 2 == 0 else "f64"
        pat = er_pattern(g, int(ns[k]), float(ps[k]), True)
        out.append(BatchItem(fill_values(g, pat, vals), vals))
    return out


@dataclass
class Request:
    t_arrival: float       # seconds since the stream started
    a: np.ndarray
    values: str


def serving_n(g: np.random.Generator, size: int, n_min: int = 16, n_max: int = 40) -> np.ndarray:
    """n = n_min + m with P(m) proportional to 2^-m, m = 0..n_max-n_min."""
    m = np.arange(n_max - n_min + 1)
    w = 0.5 ** m
    return n_min + g.choice(m, size=size, p=w / w.sum())


def serving_stream(rate: float = 2000.0, duration: float = 60.0, seed: int = 5, p_lo: float = 0.1,
                   p_hi: float = 0.3, n_min: int = 16, n_max: int = 40, limit: int | None = None) -> list[Request]:
    """Poisson arrivals at ``rate`` per second for ``duration`` seconds."""
    g = rng(seed)
    gaps = g.exponential(1.0 / rate, size=int(rate * duration * 1.5) + 16)
    t = np.cumsum(gaps)
    t = t[t < duration]
    if limit is not None:
        t = t[:limit]
    ns = serving_n(g, len(t), n_min, n_max)
    ps = g.uniform(p_lo, p_hi, size=len(t))
    coins = g.random(len(t)) < 0.5
    out = []
    for k in range(len(t)):
        vals = "01" if coins[k] else "f64"
        pat = er_pattern(g, int(ns[k]), float(ps[k]), True)
        out.append(Request(float(t[k]), fill_values(g, pat, vals), vals))
    return out


def to_csr(a: np.ndarray):
    """Dense -> CSR (int32 row pointers, int32 column ids, values in a's dtype)."""
    a = np.asarray(a)
    n = a.shape[0]
    nz = a != 0
    ptr = np.zeros(n + 1, dtype=np.int32)
    ptr[1:] = np.cumsum(nz.sum(axis=1))
    rows, cols = np.nonzero(nz)
    return ptr, cols.astype(np.int32), np.ascontiguousarray(a[rows, cols])


def to_csc(a: np.ndarray):
    """Dense -> CSC (the CSR of the transpose)."""
    return to_csr(np.asarray(a).T)


# Fixed special matrices used by tests (closed-form permanents).
def ones(n: int) -> np.ndarray:
    return np.ones((n, n), dtype=np.int64)


def ones_minus_identity(n: int) -> np.ndarray:
    return (np.ones((n, n), dtype=np.int64) - np.eye(n, dtype=np.int64))


def tridiagonal_ones(n: int) -> np.ndarray:
    idx = np.arange(n)
    return (np.abs(idx[:, None] - idx[None, :]) <= 1).astype(np.int64)


def permutation_matrix(n: int, seed: int) -> np.ndarray:
    g = rng(seed)
    a = np.zeros((n, n), dtype=np.int64)
    a[np.arange(n), g.permutation(n)] = 1
    return a
