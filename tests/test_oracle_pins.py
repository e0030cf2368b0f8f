"""Pins for the CPU oracle: each function is checked against something other
than itself -- brute force over permutations (Eq. 1), closed forms, invariants
of the permanent, and an independent banded dynamic program -- so that a dropped
term, a wrong sign, a wrong index or a transposed operand in any of them fails
here.  CPU only."""
import math

import numpy as np
import pytest

import oracle
from paper_2501_15126_gb300 import synth

MASK128 = (1 << 128) - 1


def derangements(n: int) -> int:
    d = [1, 0]
    for k in range(2, n + 1):
        d.append((k - 1) * (d[-1] + d[-2]))
    return d[n]


def fibonacci(k: int) -> int:
    a, b = 0, 1
    for _ in range(k):
        a, b = b, a + b
    return a


def rel(a, b):
    return abs(float(a) - float(b)) / max(abs(float(b)), 1e-300)


def rand_real(n, seed, density=1.0, signed=False):
    g = np.random.default_rng(seed)
    a = g.random((n, n)) * (g.random((n, n)) < density)
    if signed:
        a = a * np.where(g.random((n, n)) < 0.5, -1.0, 1.0)
    return a


def rand_int(n, seed, lo=-3, hi=4, density=1.0):
    g = np.random.default_rng(seed)
    a = g.integers(lo, hi, size=(n, n)) * (g.random((n, n)) < density)
    return a.astype(np.int64)


# --------------------------------------------------------------------------- Eq. 1

@pytest.mark.parametrize("n", range(1, 10))
def test_brute_closed_forms(n):
    assert float(oracle.brute(np.ones((n, n)))) == math.factorial(n)
    assert oracle.brute_int(synth.ones(n)) == math.factorial(n)
    assert oracle.brute_int(synth.ones_minus_identity(n)) == derangements(n)
    assert oracle.brute_int(synth.tridiagonal_ones(n)) == fibonacci(n + 1)
    assert oracle.brute_int(synth.permutation_matrix(n, n)) == 1


def test_brute_triangular_and_scaled_permutation():
    g = np.random.default_rng(7)
    for n in range(1, 9):
        d = g.integers(1, 9, size=n)
        u = np.triu(g.integers(-5, 6, size=(n, n)), 1) + np.diag(d)
        assert oracle.brute_int(u) == int(np.prod(d))
        assert oracle.brute_int(u.T.copy()) == int(np.prod(d))
        p = synth.permutation_matrix(n, 100 + n) * d[:, None]
        assert oracle.brute_int(p) == int(np.prod(d))
        assert rel(oracle.brute(p.astype(float)), float(np.prod(d))) < 1e-15


def test_brute_block_diagonal_is_product():
    a = rand_int(4, 1, 0, 5)
    b = rand_int(3, 2, 0, 5)
    m = np.zeros((7, 7), dtype=np.int64)
    m[:4, :4] = a
    m[4:, 4:] = b
    assert oracle.brute_int(m) == oracle.brute_int(a) * oracle.brute_int(b)


def test_brute_small_by_hand():
    # perm([[a, b], [c, d]]) = ad + bc
    assert oracle.brute_int(np.array([[2, 3], [5, 7]])) == 2 * 7 + 3 * 5
    # 3x3 written out: sum over the 6 permutations
    a = np.array([[1, 2, 3], [4, 5, 6], [7, 8, 10]])
    want = (1 * 5 * 10 + 1 * 6 * 8 + 2 * 4 * 10 + 2 * 6 * 7 + 3 * 4 * 8 + 3 * 5 * 7)
    assert oracle.brute_int(a) == want
    assert float(oracle.brute(a.astype(float))) == want


# --------------------------------------------------------------------------- Eq. 2

@pytest.mark.parametrize("n", range(1, 9))
def test_ryser_matches_brute_force(n):
    for seed in range(3):
        a = rand_int(n, 10 * n + seed)
        assert oracle.ryser(a) == oracle.brute_int(a)


@pytest.mark.parametrize("n", [10, 14, 18])
def test_ryser_closed_forms(n):
    assert oracle.ryser(synth.ones(n)) == math.factorial(n)
    assert oracle.ryser(synth.ones_minus_identity(n)) == derangements(n)
    assert oracle.ryser(synth.tridiagonal_ones(n)) == fibonacci(n + 1)
    assert oracle.ryser(synth.permutation_matrix(n, 3)) == 1


@pytest.mark.parametrize("n", range(1, 13))
def test_ryser_gray_matches_ryser(n):
    a = rand_int(n, 99 + n, -4, 5, 0.6)
    assert oracle.ryser_gray(a) == oracle.ryser(a)


def test_ryser_gray_closed_forms_large():
    n = 24
    assert oracle.ryser_gray(synth.ones(n)) == math.factorial(n)
    assert oracle.ryser_gray(synth.ones_minus_identity(n)) == derangements(n)
    # sub-ranges add up to the whole
    a = rand_int(14, 5, -2, 3, 0.5)
    whole = oracle.ryser_gray(a, 0, 1 << 14, signed_perm=False)
    parts = sum(oracle.ryser_gray(a, lo, lo + 1000, signed_perm=False) for lo in range(0, 16000, 1000))
    parts += oracle.ryser_gray(a, 16000, 1 << 14, signed_perm=False)
    assert parts & MASK128 == whole


# --------------------------------------------------------------------------- Algorithm 1

@pytest.mark.parametrize("n", range(1, 10))
def test_nw_matches_brute_force(n):
    for seed in range(3):
        a = rand_real(n, 1000 * n + seed, density=0.7, signed=(seed == 2))
        want = float(oracle.brute(a))
        got, absum = oracle.nw_perm(a)
        assert abs(float(got) - want) <= 1e-14 * max(float(absum), 1e-300)


def close_ld(result, want, n):
    """|got - want| within long-double rounding of the terms: each term carries
    about n roundings of u = 2^-(mantissa bits - 1), and the running sum adds
    rounding of the same order; 64 n u times the sum of |terms| covers both
    with margin while staying far below the 1e-9 relative scale."""
    got, absum = result
    u = 2.0 ** (1 - oracle.long_double_bits())
    return abs(float(got) - want) <= 64 * n * u * float(absum) + 1e-300


@pytest.mark.parametrize("n", [2, 5, 12, 17, 20])
def test_nw_closed_forms(n):
    assert close_ld(oracle.nw_perm(np.ones((n, n))), math.factorial(n), n)
    assert close_ld(oracle.nw_perm(synth.ones_minus_identity(n).astype(float)), derangements(n), n)
    assert close_ld(oracle.nw_perm(synth.tridiagonal_ones(n).astype(float)), fibonacci(n + 1), n)
    assert close_ld(oracle.nw_perm(synth.permutation_matrix(n, 8).astype(float)), 1.0, n)
    # and the error bound is not vacuous: it is far below the value itself
    got, absum = oracle.nw_perm(np.ones((n, n)))
    assert 64 * n * 2.0 ** (1 - oracle.long_double_bits()) * float(absum) < 1e-9 * math.factorial(n)


def test_nw_upper_triangular_and_block_diagonal():
    g = np.random.default_rng(3)
    n = 15
    d = g.random(n) + 0.5
    u = np.triu(g.random((n, n)), 1) + np.diag(d)
    assert rel(oracle.nw_perm(u)[0], float(np.prod(d))) < 1e-14
    assert rel(oracle.nw_perm(u.T.copy())[0], float(np.prod(d))) < 1e-14
    a, b = rand_real(6, 4), rand_real(7, 5)
    m = np.zeros((13, 13))
    m[:6, :6] = a
    m[6:, 6:] = b
    assert rel(oracle.nw_perm(m)[0], float(oracle.nw_perm(a)[0]) * float(oracle.nw_perm(b)[0])) < 1e-14


def test_nw_invariants():
    """perm(PAQ) = perm(A^T) = perm(A); scaling row i by c scales perm by c."""
    a = rand_real(14, 77, density=0.5)
    g = np.random.default_rng(0)
    base = float(oracle.nw_perm(a)[0])
    assert rel(oracle.nw_perm(a.T.copy())[0], base) < 1e-13
    for _ in range(3):
        pa = a[g.permutation(14)][:, g.permutation(14)]
        assert rel(oracle.nw_perm(np.ascontiguousarray(pa))[0], base) < 1e-13
    b = a.copy()
    b[5] *= 3.0
    assert rel(oracle.nw_perm(b)[0], 3.0 * base) < 1e-13


def test_nw_depends_on_the_last_column_entry():
    """The x-init takes a_{i,n-1}; a matrix whose last column is not the last
    stored entry of each row must still be right (row 0 has no entry in column n-1)."""
    a = np.array([[1.0, 2.0, 0.0], [0.0, 3.0, 4.0], [5.0, 0.0, 6.0]])
    assert rel(oracle.nw_perm(a)[0], float(oracle.brute(a))) < 1e-15


def test_nw_range_additivity_and_start_vector():
    """A range that starts mid-way builds its x from Gray(g_lo) (Sec. II-A); any
    split of [0, 2^(n-1)) must add up to the whole."""
    n = 13
    a = rand_real(n, 5, density=0.4) + np.eye(n)
    total = 1 << (n - 1)
    whole, whole_abs = oracle.nw_range(a, 0, total)
    cuts = [0, 1, 7, 512, 1000, 3071, total]
    s = sum(float(oracle.nw_range(a, lo, hi)[0]) for lo, hi in zip(cuts, cuts[1:]))
    assert abs(s - float(whole)) <= 1e-15 * float(whole_abs)


@pytest.mark.parametrize("threads", [1, 2, 5, 8])
def test_nw_range_threads_do_not_change_result(threads):
    n = 16
    a = rand_real(n, 6, density=0.3) + np.eye(n)
    one = oracle.nw_range(a, 0, 1 << (n - 1), threads=1)[0]
    many = oracle.nw_range(a, 0, 1 << (n - 1), threads=threads)[0]
    # chunking fixed by the range, so the thread count changes nothing; the
    # single-threaded call sums in one sweep, so allow rounding against it only
    assert abs(float(many) - float(one)) <= 1e-16 * abs(float(one)) * 64
    again = oracle.nw_range(a, 0, 1 << (n - 1), threads=3)[0]
    assert (many.hi, many.lo) == (again.hi, again.lo) or threads == 1


# --------------------------------------------------------------------------- doubled Algorithm 1, mod 2^128

@pytest.mark.parametrize("n", range(1, 12))
def test_nw2_full_range_is_scaled_permanent(n):
    a = rand_int(n, 300 + n, -3, 4, 0.6)
    perm = oracle.ryser(a)
    want = ((-1) ** (n - 1) * (1 << (n - 1)) * perm) & MASK128
    assert oracle.nw2_range(a, 0, 1 << (n - 1)) == want


def test_nw2_additivity_and_threads():
    n = 15
    a = rand_int(n, 3, 0, 2, 0.35) + np.eye(n, dtype=np.int64)
    total = 1 << (n - 1)
    whole = oracle.nw2_range(a, 0, total)
    parts = (oracle.nw2_range(a, 0, 777) + oracle.nw2_range(a, 777, 9000) + oracle.nw2_range(a, 9000, total))
    assert parts & MASK128 == whole
    assert oracle.nw2_range(a, 0, total, threads=4) == whole
    perm = oracle.ryser(a)
    assert whole == ((-1) ** (n - 1) * (1 << (n - 1)) * perm) & MASK128


# --------------------------------------------------------------------------- banded DP

def band(n, w, seed, ints=True):
    g = np.random.default_rng(seed)
    idx = np.arange(n)
    mask = np.abs(idx[:, None] - idx[None, :]) <= w
    if ints:
        return (g.integers(-3, 4, size=(n, n)) * mask).astype(np.int64)
    return g.random((n, n)) * mask


@pytest.mark.parametrize("w", [0, 1, 2, 3])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 9])
def test_band_dp_matches_brute_force(n, w):
    a = band(n, w, 10 * n + w)
    assert oracle.band_dp_int(a, w) == oracle.brute_int(a)
    af = band(n, w, 10 * n + w, ints=False)
    assert rel(oracle.band_dp(af, w), oracle.brute(af)) < 1e-15 or abs(float(oracle.brute(af))) < 1e-300


@pytest.mark.parametrize("n", [14, 18])
def test_band_dp_matches_ryser(n):
    a = band(n, 3, n)
    assert oracle.band_dp_int(a, 3) == oracle.ryser_gray(a)


def test_band_dp_fibonacci_and_rejects_offband():
    for n in (10, 30, 48):
        assert oracle.band_dp_int(synth.tridiagonal_ones(n), 1) == fibonacci(n + 1)
    assert rel(oracle.band_dp(synth.tridiagonal_ones(48).astype(float), 1), fibonacci(49)) < 1e-15
    with pytest.raises(ValueError):
        oracle.band_dp_int(synth.ones(6), 2)


def test_band_dp_matches_nw_on_band_sibling():
    a = synth.band_plus(n=20, w=3, extra=0, seed=11, values="f64")
    got, absum = oracle.nw_perm(a)
    assert abs(float(oracle.band_dp(a, 3)) - float(got)) <= 1e-15 * float(absum)


# --------------------------------------------------------------------------- row-expansion DP

def sparse_int(n, density, seed, lo=-3, hi=4):
    g = np.random.default_rng(seed)
    pat = g.random((n, n)) < density
    np.fill_diagonal(pat, True)
    return (g.integers(lo, hi, size=(n, n)) * pat).astype(np.int64)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 8])
def test_rowdp_matches_brute_force_in_any_row_order(n):
    """Eq. 1 by brute force, for every row order tried (signed integers and
    signed reals, with zeros)."""
    g = np.random.default_rng(n)
    a = sparse_int(n, 0.5, 70 + n)
    af = rand_real(n, 80 + n, density=0.6, signed=True)
    for _ in range(3):
        order = list(g.permutation(n))
        assert oracle.rowdp_int(a, order) == oracle.brute_int(a)
        assert rel(oracle.rowdp(af, order), oracle.brute(af)) < 1e-15 or abs(float(oracle.brute(af))) < 1e-300
    assert oracle.rowdp_int(a) == oracle.brute_int(a)


def test_rowdp_matches_ryser_and_band_dp():
    a = sparse_int(20, 0.15, 5)
    assert oracle.rowdp_int(a) == oracle.ryser_gray(a)
    b = synth.band_plus(n=40, w=3, extra=0, seed=2, values="01")
    assert oracle.rowdp_int(b) == oracle.band_dp_int(b, 3)
    assert oracle.rowdp_int(b, list(range(39, -1, -1))) == oracle.band_dp_int(b, 3)


def test_rowdp_closed_forms():
    """n! for the all-ones matrix, derangements for J - I, 1 for a permutation
    matrix, Fibonacci numbers for tridiagonal ones (n = 64: every column bit)."""
    for n in (6, 12):
        assert oracle.rowdp_int(synth.ones(n)) == math.factorial(n)
        assert oracle.rowdp_int(synth.ones_minus_identity(n)) == derangements(n)
    assert oracle.rowdp_int(synth.permutation_matrix(50, 3)) == 1
    assert oracle.rowdp_int(synth.tridiagonal_ones(64)) == fibonacci(65)
    assert rel(oracle.rowdp(synth.tridiagonal_ones(64).astype(float)), fibonacci(65)) < 1e-15


def test_rowdp_limits_and_bad_orders():
    with pytest.raises(ValueError):
        oracle.rowdp_int(synth.ones(14), max_states=100)
    with pytest.raises(ValueError):
        oracle.rowdp_int(synth.ones(4), [0, 1, 1, 3])


# --------------------------------------------------------------------------- cross-formula

def test_all_formulas_agree_on_integer_er():
    n = 11
    ai, af = synth.single_er_pair(n, 0.3, 42)
    r = oracle.ryser(ai)
    assert r == oracle.brute_int(ai) == oracle.ryser_gray(ai)
    assert rel(oracle.nw_perm(ai.astype(float))[0], r) < 1e-15
    n2 = (oracle.nw2_range(ai, 0, 1 << (n - 1)))
    assert n2 == ((-1) ** (n - 1) * (1 << (n - 1)) * r) & MASK128
