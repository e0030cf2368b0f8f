"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on
the same seeded inputs.  Exact (integer) results must be bit-identical; FP64
results of whole walks must agree within 1e-9 relative to |perm| (precision
AUTO reruns ill-conditioned walks in double-double to get there), and FP64
sub-range partial sums within 64 n 2^-53 of the range's sum of |terms|, the
rounding bound of an FP64 walk."""
import math

import numpy as np
import pytest

import oracle
from paper_2501_15126_gb300 import _abi as A
from paper_2501_15126_gb300 import synth

pytestmark = pytest.mark.gpu
MASK128 = (1 << 128) - 1
RTOL = 1e-9
U = 2.0 ** -53


def rel_err(got, want):
    return abs(got - want) / max(abs(want), 1e-300)


def fp_ok(res, a, threads=8):
    want, absum = oracle.nw_perm(a, threads=threads)
    err = abs(res.value - float(want))
    return err <= RTOL * abs(float(want)), err / max(abs(float(want)), 1e-300)


def rand_pattern(n, p, seed, values):
    g = np.random.default_rng(seed)
    pat = g.random((n, n)) < p
    np.fill_diagonal(pat, True)
    if values == "int":
        return (g.integers(-3, 4, size=(n, n)) * pat).astype(np.int64)
    if values == "01":
        return pat.astype(np.int64)
    return g.random((n, n)) * pat


@pytest.mark.parametrize("engine", [A.PERM_ENGINE_GENERIC, A.PERM_ENGINE_CODEGEN])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 9, 12, 15, 19])
def test_small_n_exact_matches_oracle(n, engine):
    if engine == A.PERM_ENGINE_CODEGEN and n <= 8:
        pytest.skip("n <= 8 runs the direct kernel")
    for seed, vals in ((n, "01"), (100 + n, "int")):
        a = rand_pattern(n, 0.4, seed, vals)
        want = oracle.ryser_gray(a)
        r = A.permanent(a, engine=engine)
        assert r.status == 0 and r.value == want, (n, vals, r.value, want)


@pytest.mark.parametrize("engine", [A.PERM_ENGINE_GENERIC, A.PERM_ENGINE_CODEGEN])
@pytest.mark.parametrize("n", [1, 2, 4, 7, 9, 13, 17, 20])
def test_small_n_f64_matches_oracle(n, engine):
    if engine == A.PERM_ENGINE_CODEGEN and n <= 8:
        pytest.skip("n <= 8 runs the direct kernel")
    a = rand_pattern(n, 0.5, 7 * n, "f64")
    if n <= 9:
        want = float(oracle.brute(a))
    else:
        want = float(oracle.nw_perm(a, threads=8)[0])
    r = A.permanent(a, engine=engine)
    assert rel_err(r.value, want) <= RTOL, (n, r.value, want)


def test_er24_exact_and_f64():
    """n=24, ER p=0.2 + diagonal, 0/1 values: bit-exact; the same pattern with
    (0,1] values: FP64 within 1e-9."""
    a01 = synth.single_er(24, 0.2, 1, values="01")
    want = oracle.ryser_gray(a01)
    for engine in (A.PERM_ENGINE_GENERIC, A.PERM_ENGINE_CODEGEN):
        r = A.permanent(a01, engine=engine)
        assert r.value == want
    pi, pf = synth.single_er_pair(24, 0.2, 1)
    for engine in (A.PERM_ENGINE_GENERIC, A.PERM_ENGINE_CODEGEN):
        ok, err = fp_ok(A.permanent(pf, engine=engine), pf)
        assert ok, err


def test_orderings_engines_and_words_agree_exactly():
    a = synth.single_er(22, 0.25, 9, values="01")
    want = oracle.ryser_gray(a)
    for ordering in (A.PERM_ORDER_NONE, A.PERM_ORDER_DEGREE, A.PERM_ORDER_PAPER, A.PERM_ORDER_AUTO):
        for words in (0, 2, 3):
            for engine in (A.PERM_ENGINE_GENERIC, A.PERM_ENGINE_CODEGEN):
                r = A.permanent(a, ordering=ordering, exact_words=words, engine=engine)
                assert r.value == want, (ordering, words, engine)


def test_zero_skip_and_chunking_do_not_change_exact_results():
    a = synth.band_plus(n=26, w=2, extra=1, seed=5, values="01")
    want = oracle.ryser_gray(a)
    for zs in (0, 1):
        for K in (0, 8, 12):
            for engine in (A.PERM_ENGINE_GENERIC, A.PERM_ENGINE_CODEGEN):
                r = A.permanent(a, zero_skip=zs, chunk_log2=K, engine=engine)
                assert r.value == want


def test_codegen_register_global_split():
    """Rows beyond k live in global memory (Algorithm 4 split); any k gives the same value."""
    a = synth.single_er(21, 0.2, 11, values="01")
    want = oracle.ryser_gray(a)
    af = synth.single_er(21, 0.2, 11, values="f64")
    wantf = float(oracle.nw_perm(af, threads=8)[0])
    for k in (0, 1, 6, 10, 14, 21):
        r = A.permanent(a, engine=A.PERM_ENGINE_CODEGEN, reg_rows=k)
        assert r.value == want, k
        rf = A.permanent(af, engine=A.PERM_ENGINE_CODEGEN, reg_rows=k)
        assert rel_err(rf.value, wantf) <= RTOL, k


def test_structurally_zero_and_edge_cases():
    a = np.eye(6, dtype=np.int64)
    a[2, 2] = 0
    assert A.permanent(a).value == 0                       # empty row
    b = np.zeros((5, 5), dtype=np.int64)
    b[:, 0] = 1
    b[0, :] = 1
    assert A.permanent(b).value == 0                       # no perfect matching
    assert A.permanent(np.array([[7]], dtype=np.int64)).value == 7
    assert A.permanent(np.array([[-2.5]])).value == -2.5
    n = 20
    assert A.permanent(synth.ones(n)).value == math.factorial(n)
    assert A.permanent(synth.permutation_matrix(30, 3)).value == 1


@pytest.mark.parametrize("engine", [A.PERM_ENGINE_GENERIC, A.PERM_ENGINE_CODEGEN])
def test_odd_limb_rings_give_closed_forms_exactly(engine):
    """Whole walks run in the narrowest ring of 32-bit limbs: J_21 and -J_15
    in 96 bits (-J_15 by its row-sum bound 15^15), J_30 in 160 bits.
    perm(J_n) = n!, perm(-J_n) = (-1)^n n!, and an explicit 64w-bit ring gives
    the same values."""
    for n, sign, limbs in ((21, 1, 3), (15, -1, 3), (30, 1, 5)):
        a = sign * synth.ones(n)
        assert A.inspect(a).exact_limbs == limbs
        want = sign ** n * math.factorial(n)
        assert A.permanent(a, engine=engine).value == want, (n, sign)
        assert A.permanent(a, engine=engine, exact_words=(limbs + 1) // 2).value == want, (n, sign)


@pytest.mark.parametrize("max_row", [127, 128, 900])
def test_folded_and_unfolded_exact_products(max_row):
    """Exact generic walks multiply slot quadruples in 32 bits first when every
    row's absolute sum is <= 127, and factor by factor otherwise; both sides of
    the boundary (and large entries) match the oracle bit for bit."""
    a = rand_pattern(17, 0.45, 21, "int")
    row = np.abs(a).sum(axis=1)
    i = int(np.argmax(row))
    a[i, i] += max_row - int(row[i]) if a[i, i] >= 0 else -(max_row - int(row[i]))
    assert int(np.abs(a).sum(axis=1).max()) == max_row
    want = oracle.ryser_gray(a)
    for K in (0, 5, 9):
        r = A.permanent(a, engine=A.PERM_ENGINE_GENERIC, chunk_log2=K)
        assert r.value == want, (max_row, K)


def test_ill_conditioned_f64_meets_1e9_on_every_engine_and_chunk_length():
    """A sparse (0,1] matrix whose permanent (9.7e-10) is 1.6e6 times smaller
    than the sum of its |Nijenhuis-Wilf terms|: the default precision reruns
    it in double-double, and the result is within 1e-9 of the permanent on
    every engine and chunk length; the reported sum of |terms| matches the
    oracle's."""
    a = synth.single_er(17, 0.1, 532, values="f64")
    want, absum = oracle.nw_perm(a, threads=8)
    want, absum = float(want), float(absum)
    assert absum / abs(want) > 1e6
    for engine in (A.PERM_ENGINE_GENERIC, A.PERM_ENGINE_CODEGEN):
        for K in (0, 5, 10):
            r = A.permanent(a, engine=engine, chunk_log2=K)
            assert rel_err(r.value, want) <= RTOL, (engine, K, r.value, want)
            assert abs(r.abs_term_sum - absum) <= 1e-4 * absum


def test_exact_negative_entries():
    a = rand_pattern(18, 0.35, 4, "int")
    assert A.permanent(a).value == oracle.ryser_gray(a)


def test_deterministic_repeat():
    a = synth.single_er(28, 0.2, 12, values="f64")
    p = A.Plan(a)
    r1, r2 = p.compute(), p.compute()
    assert (r1.f64, r1.f64_lo) == (r2.f64, r2.f64_lo)
    p.close()


# ------------------------------------------------------------------ sub-ranges at full size

def in_plan_order(a, **kw):
    """A partial sum over a Gray sub-range depends on the column order (the
    walk visits subsets of the ordered columns, and the last ordered column is
    the one never flipped), so the oracle gets the columns in the plan's order."""
    ins = A.inspect(a, ordering=kw.get("ordering", 0))
    order = list(ins.col_order)[: a.shape[0]]
    return np.ascontiguousarray(a[:, order])


def subrange_check_f64(a, lo, hi, **kw):
    r = A.permanent(a, g_lo=lo, g_hi=hi, flags=A.PERM_FLAG_ABS_SUM, **kw)
    s, sa = oracle.nw_range(in_plan_order(a, **kw), lo, hi, threads=16)
    n = a.shape[0]
    assert abs(r.value - float(s)) <= 64 * n * U * float(sa), (lo, hi, r.value, float(s), float(sa))
    assert abs(r.abs_term_sum - float(sa)) <= 1e-4 * float(sa)


def subrange_check_exact(a, lo, hi, **kw):
    r = A.permanent(a, g_lo=lo, g_hi=hi, **kw)
    want = oracle.nw2_range(in_plan_order(a, **kw), lo, hi, threads=16)
    assert r.partial_int & MASK128 == want, (lo, hi)


def test_subrange_sums_add_up_to_the_permanent():
    """Partial sums over a split of [0, 2^(n-1)) add up to the full walk."""
    a = synth.single_er(22, 0.3, 21, values="01")
    want = oracle.ryser_gray(a)
    n = 22
    cuts = [0, 1 << 10, 3 << 15, 1 << 20, 1 << 21]
    tot = sum(A.permanent(a, g_lo=lo, g_hi=hi).partial_int for lo, hi in zip(cuts, cuts[1:]))
    r = A.permanent(a)
    w = r.exact_words
    assert tot % (1 << (64 * w)) == ((-1) ** (n - 1) * (1 << (n - 1)) * want) % (1 << (64 * w))
    af = synth.single_er(22, 0.3, 21, values="f64")
    parts = sum(A.permanent(af, g_lo=lo, g_hi=hi).value for lo, hi in zip(cuts, cuts[1:]))
    assert rel_err(-2.0 * parts, A.permanent(af).value) < 1e-12


def test_empty_subrange_is_zero_and_launches_nothing():
    """[g, g) with g > 0 a multiple of 32 is the sum over no Gray index: 0, no
    steps (both ends 0 would mean the whole walk).  The exact path reports the
    ring width of any other sub-range of the matrix, so such a partial sum
    adds to the others (a rank with an empty shard)."""
    a = synth.single_er(22, 0.3, 21, values="01")
    af = synth.single_er(22, 0.3, 21, values="f64")
    w = A.permanent(a, g_lo=0, g_hi=1 << 10).exact_words
    for engine in (A.PERM_ENGINE_GENERIC, A.PERM_ENGINE_CODEGEN):
        for g in (32, 1 << 20):
            r = A.permanent(a, g_lo=g, g_hi=g, engine=engine)
            assert (r.steps, r.partial_int, r.exact_words) == (0, 0, w)
            rf = A.permanent(af, g_lo=g, g_hi=g, engine=engine)
            assert (rf.steps, rf.f64, rf.f64_lo) == (0, 0.0, 0.0)
    r = A.permanent_noalloc(a, g_lo=64, g_hi=64)
    assert (r.steps, r.partial_int, r.exact_words) == (0, 0, w)


def test_er36_subranges():
    """n=36, ER p=0.15 + diagonal, (0,1] values, shuffled columns: Gray sub-ranges
    anywhere in [0, 2^35), including ranges whose high bits are set."""
    a = synth.single_er(36, 0.15, 2, values="f64", shuffle_cols=True)
    span = 1 << 20
    for lo in (0, 1 << 25, (1 << 34) + (3 << 27), (1 << 35) - span):
        for engine in (A.PERM_ENGINE_GENERIC, A.PERM_ENGINE_CODEGEN):
            subrange_check_f64(a, lo, lo + span, engine=engine)


def test_band48_subranges_exact_and_f64():
    """n=48 band |i-j|<=3 + 2 off-band nonzeros per row, with the register/global split."""
    a01 = synth.band_plus(48, 3, 2, seed=3, values="01")
    af = synth.band_plus(48, 3, 2, seed=3, values="f64")
    span = 1 << 20
    for lo in (0, 1 << 30, (1 << 46) + (5 << 33), (1 << 47) - span):
        subrange_check_exact(a01, lo, lo + span, engine=A.PERM_ENGINE_CODEGEN)
        subrange_check_f64(af, lo, lo + span, engine=A.PERM_ENGINE_CODEGEN)
        subrange_check_exact(a01, lo, lo + span, engine=A.PERM_ENGINE_CODEGEN, reg_rows=20)
        subrange_check_f64(af, lo, lo + span, engine=A.PERM_ENGINE_CODEGEN, reg_rows=20)
    subrange_check_exact(a01, 1 << 30, (1 << 30) + span, engine=A.PERM_ENGINE_GENERIC)


@pytest.mark.parametrize("values", ["01", "f64"])
def test_largest_size_n64_subranges(values):
    """n = 64, the largest size the library takes (Gray indices up to
    2^63 - 1; above n = 48 only the generated kernels run): sub-ranges at the
    start, across bit 62 of the Gray index and at the very end of the walk,
    against the oracle."""
    a = synth.single_er(64, 0.08, 64, values=values)
    span, top = 1 << 20, 1 << 63
    for lo in (0, (top >> 1) - span // 2, top - span):
        if values == "01":
            subrange_check_exact(a, lo, lo + span)
        else:
            subrange_check_f64(a, lo, lo + span)


def test_three_level_placement_registers_shared_global():
    """The n=48 band workload with x in three tiers (Sec. V's split, carried to
    shared memory as Sec. VIII proposes): 20 rows in registers, 12 or 28 in
    shared memory, the rest in global memory; sub-ranges with high Gray bits
    set against the oracle, exact and FP64."""
    a01 = synth.band_plus(48, 3, 2, seed=3, values="01")
    af = synth.band_plus(48, 3, 2, seed=3, values="f64")
    span = 1 << 20
    for lo in (0, (1 << 46) + (5 << 33)):
        for k2 in (12, 28):
            kw = dict(engine=A.PERM_ENGINE_CODEGEN, reg_rows=20, shared_rows=k2)
            subrange_check_exact(a01, lo, lo + span, **kw)
            subrange_check_f64(af, lo, lo + span, **kw)
            assert A.permanent(a01, g_lo=lo, g_hi=lo + span, **kw).shared_rows == k2


@pytest.mark.parametrize("engine", [A.PERM_ENGINE_GENERIC, A.PERM_ENGINE_CODEGEN])
def test_band_only_sibling_full_walk_against_band_dp(engine):
    """Band-only matrices (|i-j| <= 3, no off-band entries) walked in full on the
    GPU and checked against the banded DP, an algorithm independent of Ryser:
    n=32 (2^31 Gray steps) exact and FP64, and n=36 exact through codegen."""
    a01 = synth.band_plus(32, 3, 0, seed=3, values="01")
    af = synth.band_plus(32, 3, 0, seed=3, values="f64")
    assert A.permanent(a01, engine=engine).value == oracle.band_dp_int(a01, 3)
    want = float(oracle.band_dp(af, 3))
    assert rel_err(A.permanent(af, engine=engine).value, want) <= RTOL
    if engine == A.PERM_ENGINE_CODEGEN:
        b01 = synth.band_plus(36, 3, 0, seed=13, values="01")
        assert A.permanent(b01, engine=engine).value == oracle.band_dp_int(b01, 3)


def test_er36_full_permanent_against_stored_oracle_value():
    """The n=36 workload at full size, in the launch configuration bench.py
    times, against the oracle's full-range value stored in tests/golden."""
    import os
    vals = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "er36_f64_perm.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()
        vals[k] = float(v)
    want = vals["perm_hi"] + vals["perm_lo"]
    a = synth.single_er(36, 0.15, 2, values="f64", shuffle_cols=True)
    r = A.permanent(a)
    assert r.engine == A.PERM_ENGINE_CODEGEN and r.precision == A.PERM_PREC_F64
    assert rel_err(r.value, want) <= RTOL, (r.value, want)
    ra = A.permanent(a, flags=A.PERM_FLAG_ABS_SUM)           # the same kernel keeping sum|terms|
    assert rel_err(ra.value, want) <= RTOL
    assert abs(ra.abs_term_sum - vals["abs_terms"]) <= 1e-4 * vals["abs_terms"]


def test_repeated_compute_replays_a_graph_with_identical_results():
    """From the second perm_compute on, a plan replays its launches as a CUDA
    graph; results stay bit-identical, with and without the graph."""
    for vals in ("f64", "01"):
        a = synth.single_er(24, 0.25, 61, values=vals)
        for engine in (A.PERM_ENGINE_GENERIC, A.PERM_ENGINE_CODEGEN):
            p = A.Plan(a, engine=engine)
            rs = [p.compute() for _ in range(4)]
            q = A.Plan(a, engine=engine, flags=A.PERM_FLAG_NO_GRAPH)
            ns = [q.compute() for _ in range(2)]
            for r in rs + ns:
                assert (r.f64, r.f64_lo, r.i128_lo, r.i128_hi) == (rs[0].f64, rs[0].f64_lo, rs[0].i128_lo, rs[0].i128_hi)
                assert r.ms_kernel > 0
            p.close()
            q.close()


def test_device_deadline_stops_a_long_walk_and_the_context_survives():
    """Failure detection without a fault: a 2^39-step walk with a 50 ms
    device-side deadline stops taking work and reports TIMEOUT; the next
    computes on the same context are correct."""
    import time
    big = synth.single_er(40, 0.1, 5, values="f64")
    for engine in (A.PERM_ENGINE_GENERIC, A.PERM_ENGINE_CODEGEN):
        t0 = time.time()
        with pytest.raises(A.PermError) as e:
            A.permanent(big, engine=engine, timeout_ms=50)
        assert e.value.status == A.PERM_ERR_TIMEOUT
        assert time.time() - t0 < 30
    small = synth.single_er(18, 0.3, 6, values="01")
    assert A.permanent(small).value == oracle.ryser_gray(small)
    res = A.batch([small, big], timeout_ms=50)
    assert res[1].status == A.PERM_ERR_TIMEOUT
    assert A.permanent(small, timeout_ms=60000).value == oracle.ryser_gray(small)


# ------------------------------------------------------------------ closed forms on every path

def _derangements(n):
    d = [1, 0]
    for k in range(2, n + 1):
        d.append((k - 1) * (d[-1] + d[-2]))
    return d[n]


def _fib(k):
    a, b = 0, 1
    for _ in range(k):
        a, b = b, a + b
    return a


def _closed_form_cases():
    g = np.random.default_rng(77)
    cases = [("J-I n=13", synth.ones_minus_identity(13), _derangements(13)),
             ("J-I n=20", synth.ones_minus_identity(20), _derangements(20)),
             ("tridiagonal n=30", synth.tridiagonal_ones(30), _fib(31))]
    d = g.integers(1, 4, size=24)
    p = synth.permutation_matrix(24, 5) * d[:, None]
    cases.append(("scaled permutation n=24", p.astype(np.int64), int(np.prod(d))))
    u = np.triu(g.integers(0, 3, size=(20, 20))).astype(np.int64)
    np.fill_diagonal(u, g.integers(1, 4, size=20))
    cases.append(("upper triangular n=20", u, int(np.prod(np.diag(u)))))
    blocks = [synth.ones(6), synth.ones_minus_identity(7), synth.tridiagonal_ones(8)]
    bd = np.zeros((21, 21), dtype=np.int64)
    o = 0
    for b in blocks:
        bd[o:o + b.shape[0], o:o + b.shape[0]] = b
        o += b.shape[0]
    cases.append(("block diagonal n=21", bd, 720 * _derangements(7) * _fib(9)))
    return cases


@pytest.mark.parametrize("engine", [A.PERM_ENGINE_GENERIC, A.PERM_ENGINE_CODEGEN, "batch"])
def test_closed_forms_exact_and_f64_on_every_path(engine):
    """Closed forms on the generic and generated kernels and the batch launch,
    in both arithmetics: D_n (J - I), Fibonacci (tridiagonal ones), a scaled
    permutation, a triangular matrix and a block-diagonal product.  FP64 is
    held to 1e-9 relative everywhere, including the triangular case whose
    alternating sum cancels by a factor 3.5e10 (precision AUTO reruns it in
    double-double)."""
    cases = _closed_form_cases()
    for name, a, want in cases:
        af = a.astype(np.float64)
        absum = float(oracle.nw_perm(af, threads=8)[1])
        if engine == "batch":
            r, rf = A.batch([a, af])
        else:
            r, rf = A.permanent(a, engine=engine), A.permanent(af, engine=engine)
        assert r.value == want, (name, engine)
        err = abs(rf.value - float(want))
        assert err <= RTOL * abs(float(want)), (name, engine, rf.value, want, absum)


def test_cross_path_01_matrix_f64_equals_exact():
    """A 0/1 matrix through the FP64 path agrees with the exact path within 1e-9."""
    a = synth.single_er(24, 0.2, 1, values="01")
    exact = A.permanent(a).value
    for engine in (A.PERM_ENGINE_GENERIC, A.PERM_ENGINE_CODEGEN):
        f = A.permanent(a.astype(np.float64), engine=engine).value
        assert rel_err(f, float(exact)) <= RTOL, (engine, f, exact)
