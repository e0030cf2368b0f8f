"""GPU parity on matrices with the shapes of the paper's real-life set
(Table II; values as Sec. VI-E describes them: mostly distinct reals, all
ones, or over half +-1).  On the binary and +-1 shapes almost every product
is zero, so the walks skip whole aligned spans of blocks.  Gray sub-ranges
anywhere in the walk are checked against the oracle's partial sums (exact: bit
for bit; FP64: within 64 n 2^-53 of the range's sum of |terms|), with the zero
skip on and off, on the generated kernels and, for n <= 48, the generic ones.
The reported skip fraction is checked against a count of the all-zero blocks."""
import numpy as np
import pytest

import oracle
from paper_2501_15126_gb300 import _abi as A
from paper_2501_15126_gb300 import synth

pytestmark = pytest.mark.gpu
MASK128 = (1 << 128) - 1
U = 2.0 ** -53
SPAN = 1 << 22


def in_plan_order(a):
    ins = A.inspect(a)
    return np.ascontiguousarray(a[:, list(ins.col_order)[: a.shape[0]]])


def starts(n):
    top = 1 << (n - 1)
    return (0, (1 << 33) + (3 << 25), top // 3 - (top // 3) % SPAN, top - SPAN)


@pytest.mark.parametrize("name", [t.name for t in synth.TABLE2_SHAPES])
def test_table2_shapes_subranges_against_the_oracle(name):
    a = synth.table2_like(name)
    n = a.shape[0]
    ao = in_plan_order(a)
    engines = [A.PERM_ENGINE_CODEGEN] + ([A.PERM_ENGINE_GENERIC] if n <= 48 else [])
    for lo in starts(n):
        hi = lo + SPAN
        if a.dtype == np.int64:
            want = oracle.nw2_range(ao, lo, hi, threads=16)
        else:
            s, sa = oracle.nw_range(ao, lo, hi, threads=16)
        for engine in engines:
            for zs in (0, 1):   # 0: skip on
                if a.dtype == np.int64:
                    r = A.permanent(a, g_lo=lo, g_hi=hi, engine=engine, zero_skip=zs)
                    assert r.partial_int & MASK128 == want, (lo, engine, zs)
                else:
                    r = A.permanent(a, g_lo=lo, g_hi=hi, engine=engine, zero_skip=zs, flags=A.PERM_FLAG_ABS_SUM)
                    assert abs(r.value - float(s)) <= 64 * n * U * float(sa), (lo, engine, zs)
                    assert abs(r.abs_term_sum - float(sa)) <= 1e-4 * float(sa)
                if zs:
                    assert r.zero_skip_frac == 0.0


def zero_block_fraction(ao, lo, hi, B):
    """Fraction of the 2^B-step blocks of [lo, hi) whose products are all zero,
    counted on the host from x(g) = x0 + the columns set in Gray(g)."""
    n = ao.shape[0]
    x0 = ao[:, n - 1] - 0.5 * ao.sum(axis=1)
    g = np.arange(lo, hi, dtype=np.uint64)
    gray = g ^ (g >> np.uint64(1))
    bits = ((gray[:, None] >> np.arange(n - 1, dtype=np.uint64)[None, :]) & np.uint64(1)).astype(np.float64)
    x = x0[None, :] + bits @ ao[:, : n - 1].T.astype(np.float64)
    zero = (x == 0).any(axis=1)
    return zero.reshape(-1, 1 << B).all(axis=1).mean()


@pytest.mark.parametrize("name", ["curtis54", "bcspwr02", "mycielskian6"])
def test_skip_fraction_is_bounded_by_the_all_zero_blocks(name):
    """Every skipped block has only zero products, so the skip fraction the
    library reports is at most the fraction of all-zero blocks.  Where zero
    rows of x are shared by the 32 chunks of a warp (the sparse shapes) the
    warp skips most of those blocks; in mycielskian6's denser pattern the
    chunks' columns K-1..K+4 touch nearly every row, so the lanes' zeros rarely
    coincide and only the bound holds."""
    a = synth.table2_like(name)
    ao = in_plan_order(a).astype(np.float64)
    lo, hi = 1 << 30, (1 << 30) + (1 << 18)
    r = A.permanent(a, g_lo=lo, g_hi=hi, engine=A.PERM_ENGINE_CODEGEN, chunk_log2=12)
    z = zero_block_fraction(ao, lo, hi, 5)
    assert 0.0 <= r.zero_skip_frac <= z + 1e-12, (r.zero_skip_frac, z)
    if name != "mycielskian6":
        assert r.zero_skip_frac > 0.5 * z, (r.zero_skip_frac, z)


def test_whole_walk_of_the_bcspwr02_shape_against_the_row_dp():
    """The whole 2^48-step walk of the bcspwr02 shape (n = 49, all ones; about
    a second, because the zero spans remove nearly all of it): exact, bit for
    bit against the oracle's row-expansion DP (Eq. 1); the same matrix with
    its columns permuted (perm(AQ) = perm(A)); and the FP64 walk."""
    a = synth.table2_like("bcspwr02")
    want = oracle.rowdp_int(a)
    r = A.permanent(a)
    assert r.value == want
    assert r.zero_skip_frac > 0.99
    q = np.random.default_rng(49).permutation(a.shape[0])
    assert A.permanent(np.ascontiguousarray(a[:, q])).value == want
    rf = A.permanent(a.astype(np.float64), flags=A.PERM_FLAG_ABS_SUM)
    assert abs(rf.value - want) <= max(1e-9 * want, 64 * 49 * U * rf.abs_term_sum)


@pytest.mark.parametrize("engine", [A.PERM_ENGINE_GENERIC, A.PERM_ENGINE_CODEGEN])
def test_two_state_walk_zero_spans_in_fp64(engine):
    """0/1 matrices walked in FP64 by the two-state walk (the generic kernel of
    the batch and serving FP64 path; a generated kernel with two-state chains
    and zero spans), where most terms are zero: whole walks at chunk lengths
    up to 2^16 (so spans reach whole chunks) equal the exact permanent,
    sub-ranges match the oracle's partial sums, the skip fraction shows the
    spans at work, and the batch path gives the same values."""
    mats = [synth.single_er(28, 0.1, s, values="01") for s in (3, 4)] + [synth.band_plus(30, 1, 1, seed=2)]
    for a in mats:
        n = a.shape[0]
        want = oracle.rowdp_int(a)
        af = a.astype(np.float64)
        for K in (8, 12, 16):
            r = A.permanent(af, engine=engine, chunk_log2=K)
            assert abs(r.value - want) <= 1e-9 * abs(want), (n, K, r.value, want)
        assert r.zero_skip_frac > 0.5, r.zero_skip_frac
        ao = in_plan_order(af)
        for lo in (0, 1 << 20, (1 << (n - 1)) - (1 << 18)):
            hi = lo + (1 << 18)
            s, sa = oracle.nw_range(ao, lo, hi, threads=16)
            rs = A.permanent(af, g_lo=lo, g_hi=hi, engine=engine, flags=A.PERM_FLAG_ABS_SUM)
            assert abs(rs.value - float(s)) <= 64 * n * U * float(sa) + 1e-300, (n, lo)
    if engine != A.PERM_ENGINE_GENERIC:
        return
    got = A.batch([m.astype(np.float64) for m in mats])
    for a, r in zip(mats, got):
        want = oracle.rowdp_int(a)
        assert abs(r.value - want) <= 1e-9 * abs(want)
