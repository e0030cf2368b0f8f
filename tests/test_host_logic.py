"""Host-side preprocessing checked against the paper: Theorem 1 / SCBS
(Sec. IV), the 5-thread chunk table, Lemma 1 and Lemma 2 counts, Algorithm 2
launch lists, Algorithm 3 ordering, Algorithm 4 partitioning, the structural
guard and the exact-width choice.  CPU only (inspection calls)."""
import os

import numpy as np
import pytest

from paper_2501_15126_gb300 import _abi as A
from paper_2501_15126_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, v = line.split(":", 1)
        out[k.strip()] = [int(t) for t in v.replace(",", " ").split()]
    return out


def signed(seq):
    return [s for s in seq]


def test_scbs_matches_the_paper():
    g = golden("scbs_sec4.txt")
    for k in (2, 3, 4):
        assert A.scbs(k) == g["scbs%d" % k]


def test_changed_bit_sequence_n5():
    g = golden("scbs_sec4.txt")
    assert [abs(v) - 1 for v in A.scbs(4)] == g["changed_bits_n5"]


def test_five_thread_chunk_table():
    """5 threads, chunks of 3 iterations of SCBS(4) (Sec. IV): the signed kernel
    calls per local iteration and the number of distinct ones."""
    g = golden("scbs_sec4.txt")
    seq = A.scbs(4)
    table = [[seq[t * 3 + l] for t in range(5)] for l in range(3)]
    assert table[0] == g["chunk3_row0"]
    assert table[1] == g["chunk3_row1"]
    assert table[2] == g["chunk3_row2"]
    assert [len(set(r)) for r in table] == g["chunk3_distinct"]


def test_theorem1_recursive_construction():
    """SCBS(k) = [SCBS(k-1), +(k-1), -SCBS(k-1)^R] (Sec. IV) against Theorem 1."""
    prev = A.scbs(1)
    assert prev == [1]
    for k in range(2, 15):
        rec = prev + [k] + [-v for v in reversed(prev)]
        assert A.scbs(k) == rec
        prev = rec


def test_lemma1_power_of_two_chunks():
    """Chunks of 2^k: all threads of a warp share the column at every local step
    except l = 2^(k-1) (same column, sign = parity of t) and l = 2^k."""
    seq = A.scbs(16)
    for k in (3, 5, 7):
        c = 1 << k
        for l in range(1, c + 1):
            vals = [seq[l + t * c - 1] for t in range(32) if l + t * c - 1 < len(seq)]
            cols = {abs(v) for v in vals}
            if l == c // 2:
                assert cols == {k} and {v > 0 for v in vals} == {True, False}
                assert all((v > 0) == (t % 2 == 0) for t, v in enumerate(vals))
            elif l == c:
                assert len(cols) > 1
            else:
                assert len(set(vals)) == 1


def test_lemma2_column_frequencies():
    for n in (6, 11, 17):
        seq = A.scbs(n - 1)
        for j in range(n - 1):
            assert sum(1 for v in seq if abs(v) - 1 == j) == 2 ** (n - j - 2)


def test_algorithm2_launch_lists():
    g = golden("alg2_launches.txt")
    assert A.alg2_launches(2, 12) == [tuple(g["tau2_n12"])]
    # every launch list covers [1, 2^(n-1)) with power-of-two chunks >= 1024 except possibly the last
    for tau, n in ((69120, 40), (55296, 45), (124416, 48), (1000, 30)):
        ls = A.alg2_launches(tau, n)
        start = 1
        for (s, d, e) in ls:
            assert s == start and e == 1 << (n - 1)
            assert d >= 1024 and d & (d - 1) == 0
            start = s + tau * d
        assert start >= 1 << (n - 1) or ls[-1][1] == 1024


def test_algorithm3_ordering_picks_min_unordered_degree():
    # a small matrix traced by hand: column degrees 3,1,2,3 ...
    a = np.array([[1, 0, 1, 0],
                  [1, 0, 0, 1],
                  [1, 1, 0, 1],
                  [0, 0, 1, 1]], dtype=np.int64)
    ins = A.inspect(a, ordering=A.PERM_ORDER_PAPER)
    # step 1: min cdeg is column 1 (1 nonzero) -> row 2 ordered; cdeg[0]=2, cdeg[3]=2, cdeg[2]=2
    # step 2: ties at 2 -> smallest index, column 0 -> rows 0, 1; cdeg[2]=1, cdeg[3]=1
    # round 3: column 2 (1) -> row 3; round 4: column 3
    assert list(ins.col_order)[:4] == [1, 0, 2, 3]
    assert list(ins.row_order)[:4] == [2, 0, 1, 3]
    assert list(ins.group_size)[:4] == [1, 2, 1, 0]


def test_orderings_and_cost_model():
    a = synth.single_er(36, 0.15, 2, values="f64", shuffle_cols=True)
    deg = A.inspect(a, ordering=A.PERM_ORDER_DEGREE)
    pap = A.inspect(a, ordering=A.PERM_ORDER_PAPER)
    auto = A.inspect(a)
    nnz = [int((a[:, j] != 0).sum()) for j in range(36)]
    assert [nnz[c] for c in list(deg.col_order)[:36]] == sorted(nnz)
    # AUTO starts from the cheaper of DEGREE and PAPER and searches column swaps
    # under the model of the scheme the walk runs
    assert auto.ordering in (A.PERM_ORDER_DEGREE, A.PERM_ORDER_PAPER, A.PERM_ORDER_SEARCH)
    assert auto.ops_per_step_walk <= min(deg.ops_per_step_walk, pap.ops_per_step_walk) + 1e-12
    assert sorted(list(auto.col_order)[:36]) == list(range(36))
    assert pap.ops_per_step < pap.ops_per_step_paper
    assert sum(list(pap.group_size)[:36]) == 36
    # every row's group is the first ordered column that touches it
    order = list(pap.col_order)[:36]
    for slot in range(36):
        r = pap.row_order[slot]
        first = min(p for p in range(36) if a[r, order[p]] != 0)
        assert pap.group_of_row[slot] == first


def test_algorithm4_partition_is_consistent():
    a = synth.band_plus(48, 3, 2, seed=3, values="01")
    ins = A.inspect(a, ordering=A.PERM_ORDER_PAPER)
    k, c = ins.reg_rows, ins.reg_cols
    assert 1 <= c <= 47 and 1 <= k <= 48
    assert k == sum(list(ins.group_size)[:c])   # k = rows touched by the first c columns


def test_structural_guard_and_exact_width():
    z = np.eye(5, dtype=np.int64)
    z[:, 0] = 1
    z[0, :] = 1
    z[1, 1] = 0
    z[2, 2] = 0      # rows 1, 2 only reach column 0 -> no perfect matching
    assert A.inspect(z).structurally_zero == 1
    assert A.inspect(np.eye(5, dtype=np.int64)).structurally_zero == 0
    a = synth.single_er(24, 0.2, 1, values="01")
    assert A.inspect(a).exact_words == 1
    b = synth.band_plus(48, 3, 2, seed=3, values="01")
    assert A.inspect(b).exact_words == 3
    ones = synth.ones(30)
    # Bregman: perm(J_30) = 30! ~ 2^107.7; the bound must cover it
    assert A.inspect(ones).bound_log2 >= np.log2(float(np.prod(np.arange(1, 31, dtype=float)))) - 1e-9


def test_ring_limbs_are_the_narrowest_that_hold_the_scaled_sum():
    """A whole exact walk holds (-1)^(n-1) 2^(n-1) perm: bound + (n-1) bits, a
    sign bit and a margin bit, in the fewest 32-bit limbs (at least 2), which
    fill the stored 64-bit words (2w-1 or 2w limbs)."""
    cases = [synth.single_er(24, 0.2, 1, values="01"), synth.band_plus(48, 3, 2, seed=3, values="01"),
             synth.ones(21), synth.ones(30), np.eye(12, dtype=np.int64)]
    cases += [synth.single_er(n, p, s, values="01") for n, p, s in ((28, 0.3, 2), (26, 0.4, 3), (16, 0.2, 4))]
    for a in cases:
        ins = A.inspect(a)
        need = ins.bound_log2 + a.shape[0] + 2
        assert 32 * ins.exact_limbs >= need and (ins.exact_limbs == 2 or 32 * (ins.exact_limbs - 1) < need)
        assert (ins.exact_limbs + 1) // 2 == ins.exact_words
    # 21! ~ 2^65.5: 65.5 + 23 bits -> three limbs (96-bit ring); 30! -> five (160-bit)
    assert A.inspect(synth.ones(21)).exact_limbs == 3
    assert A.inspect(synth.ones(30)).exact_limbs == 5
    # entries other than 0/1 take the row-sum bound: -J_15 -> 15^15 ~ 2^58.6 -> 58.6 + 17 bits
    assert A.inspect(-synth.ones(15)).exact_limbs == 3 and A.inspect(-synth.ones(15)).exact_words == 2
    assert A.inspect(synth.single_er(24, 0.2, 1, values="f64")).exact_limbs == 0


def test_codegen_source_bakes_the_matrix():
    a = synth.single_er(12, 0.3, 5, values="f64")
    src = A.codegen_source(a)
    assert "perm_walk" in src and "x[0]" in src and "0x1." in src
    srck = A.codegen_source(a, reg_rows=6)
    assert "xg[" in srck


def test_slot_layout_groups_and_column0_rows_by_next_column():
    """Slots are sorted by group (first ordered column touching the row), and
    group 0 (column 0's rows) by the next ordered column touching each row, so
    every group and every set S_m of the two-state chains is a contiguous slot
    range; column 0 touches exactly group 0."""
    cases = [synth.single_er(24, 0.2, 1, values="01"), synth.band_plus(48, 3, 2, seed=3, values="f64"),
             synth.single_er(28, 0.35, 7, values="f64"), synth.ones(9)]
    for a in cases:
        n = a.shape[0]
        for ordering in (A.PERM_ORDER_DEGREE, A.PERM_ORDER_PAPER, A.PERM_ORDER_NONE):
            ins = A.inspect(a, ordering=ordering)
            co, ro = list(ins.col_order[:n]), list(ins.row_order[:n])
            grp = list(ins.group_of_row[:n])
            assert grp == sorted(grp)
            r0 = list(ins.group_size[:n])[0]
            assert set(s for s in range(n) if a[ro[s], co[0]] != 0) == set(range(r0))
            nxt = [next((p for p in range(1, n - 1) if a[ro[s], co[p]] != 0), n - 1) for s in range(r0)]
            assert nxt == sorted(nxt), (ordering, nxt)
            for s in range(n):   # the group is the first touching position
                first = next((p for p in range(n) if a[ro[s], co[p]] != 0), n - 1)
                assert grp[s] == first


def test_generated_fp64_kernel_picks_the_cheaper_chain():
    """Generated FP64 kernels use two-state chains where the cost model says
    they take fewer operations per step than the paired chain (the n=48 band,
    the n=36 workload), and the paired chain where that is cheaper (a very
    sparse ER matrix, where column 0 touches one row); PERM_FLAG_PAIRED_CHAIN
    forces the paired chain; exact kernels keep one chain."""
    band = synth.band_plus(48, 3, 2, seed=3, values="f64")
    er36 = synth.single_er(36, 0.15, 2, values="f64")
    sparse = synth.single_er(32, 0.05, 3, values="f64")
    assert "kDual = true" in A.codegen_source(band)
    assert "kDual = false" in A.codegen_source(band, flags=A.PERM_FLAG_PAIRED_CHAIN)
    assert "kDual = true" in A.codegen_source(er36)
    assert "kDual = false" in A.codegen_source(sparse)
    assert "kDual = false" in A.codegen_source(synth.band_plus(48, 3, 2, seed=3, values="01"))   # exact: one chain


def test_generated_block_length_follows_arithmetic_and_zeros():
    """Generated kernels unroll 2^7-step blocks for FP64 walks and 2^5 for exact
    ones, and for FP64 walks where most terms have a zero factor (repeated
    values, Sec. VI-E), so that their zero skip starts at 2^5 steps; exact
    walks whose sampled terms are over 95 % zero but that get no zero spans
    skip single blocks only, and unroll 2^4.  The kernel's split keeps every
    row reached inside a block in registers (c >= B)."""
    import re

    def header(a, **kw):
        m = re.search(r"reg_cols\(c\)=(\d+) B=(\d+)", A.codegen_source(a, **kw))
        return int(m.group(1)), int(m.group(2))
    for a, B in [(synth.single_er(36, 0.15, 2, values="f64", shuffle_cols=True), 7),
                 (synth.table2_like("mesh1e1"), 7),
                 (synth.table2_like("d_ss"), 5),
                 (synth.table2_like("curtis54").astype(np.float64), 5),
                 (synth.table2_like("curtis54"), 5),
                 (synth.table2_like("mycielskian6"), 4),
                 (synth.single_er(24, 0.2, 1, values="01"), 4),
                 (synth.band_plus(48, 3, 2, seed=3, values="01"), 5)]:
        c, b = header(a)
        assert b == B and c >= B, (a.shape, a.dtype, b, c)


def test_zero_spans_only_where_a_warp_can_share_zero_rows():
    """Generated kernels widen zero skips into zero spans when most sampled
    terms are zero and the pattern is sparse enough (density below 1/6) for
    the six columns in which a warp's 32 chunks differ to leave rows
    untouched; otherwise the span code is left out."""
    def spans(a):
        return "kZeroSpans = true" in A.codegen_source(a)
    assert spans(synth.table2_like("curtis54")) and spans(synth.table2_like("bcspwr02"))
    assert spans(synth.table2_like("d_ss"))
    assert not spans(synth.table2_like("mycielskian6"))                                 # dense: lanes differ everywhere
    assert not spans(synth.band_plus(48, 3, 2, seed=3, values="01"))                    # density above 1/6
    assert not spans(synth.single_er(36, 0.15, 2, values="f64", shuffle_cols=True))     # distinct reals


def test_order_search_lowers_the_walk_cost_model():
    """The AUTO order search (FP64 walks of 2^30 steps and more) only accepts
    column swaps that lower the cost model of the scheme the walk runs; its
    result is a permutation of the columns and never costs more than the better
    of DEGREE and PAPER.  Shorter walks keep that better order."""
    cases = [(synth.single_er(36, 0.15, 2, values="f64", shuffle_cols=True), True),
             (synth.band_plus(48, 3, 2, seed=3, values="f64"), True),
             (synth.single_er(24, 0.2, 1, values="01"), False)]
    for a, fp64 in cases:
        n = a.shape[0]
        auto = A.inspect(a)
        base = min(A.inspect(a, ordering=o).ops_per_step_walk for o in (A.PERM_ORDER_DEGREE, A.PERM_ORDER_PAPER))
        assert sorted(list(auto.col_order)[:n]) == list(range(n))
        assert auto.ops_per_step_walk <= base + 1e-12
        if auto.ordering == A.PERM_ORDER_SEARCH:
            assert auto.ops_per_step_walk < base
        assert A.inspect(a, ordering=A.PERM_ORDER_SEARCH).ops_per_step_walk == auto.ops_per_step_walk
    # the n=36 workload: 8.23 -> about 6.5 counted FP64 operations per step
    er36 = A.inspect(cases[0][0])
    assert er36.ordering == A.PERM_ORDER_SEARCH and er36.ops_per_step_walk < 7.0
    short = synth.single_er(24, 0.2, 1, values="01")
    assert A.inspect(short).ordering in (A.PERM_ORDER_DEGREE, A.PERM_ORDER_PAPER)
    exact_long = synth.single_er(34, 0.2, 5, values="01")   # exact walks keep the start order
    assert A.inspect(exact_long).ordering in (A.PERM_ORDER_DEGREE, A.PERM_ORDER_PAPER)



def _schedule_counts(a, ins):
    """Per-step operation counts of the two chain schemes, by walking the Gray
    schedule step by step (column j = ctz(l) flips at step l) and counting what
    each step does, from the layout perm_inspect reports."""
    n = a.shape[0]
    co, ro = list(ins.col_order[:n]), list(ins.row_order[:n])
    R = list(ins.group_size[:n])
    nnz = [int(np.count_nonzero(a[:, c])) for c in co]
    S = [0] * (n + 1)
    for s in range(R[0]):
        nxt = next((p for p in range(1, n - 1) if a[ro[s], co[p]] != 0), n - 1)
        S[nxt] += 1
    steps = (1 << (n - 1)) - 1
    one_chain = two_state = 0.0
    for l in range(1, steps + 1):
        j = (l & -l).bit_length() - 1
        # one chain: flip column j, rebuild levels j..0 (|R_0| + ... + |R_j| products), accumulate
        one_chain += nnz[j] + sum(R[: j + 1]) + 1
        if j == 0:
            two_state += 2          # the odd step closes a pair: one difference, one accumulation
        else:
            two_state += nnz[j] + sum((R[m] + 1 if R[m] else 0) + 3 * S[m] for m in range(1, j + 1))
    return one_chain / steps, two_state / steps


def test_cost_models_match_a_step_by_step_count():
    """The closed-form step-cost models (Lemma 2 weights) equal a direct count
    over the Gray schedule: the one-chain model (perm_inspect ops_per_step) and
    the two-state-chain model of short FP64 walks (ops_per_step_walk)."""
    cases = [synth.single_er(12, 0.3, 1, values="f64"), synth.band_plus(14, 2, 1, seed=2, values="f64"),
             synth.single_er(16, 0.2, 7, values="f64"), synth.ones(9).astype(np.float64)]
    for a in cases:
        ins = A.inspect(a)
        one, two = _schedule_counts(a, ins)
        assert abs(ins.ops_per_step - one) < 1e-9 * one, (ins.ops_per_step, one)
        assert abs(ins.ops_per_step_walk - two) < 1e-9 * two, (ins.ops_per_step_walk, two)


def test_register_budget_of_generated_kernels():
    """FP64 walks of 2^30 steps and more are built for one 256-thread block
    per SM (up to 255 registers: x and both chains without spills), shorter
    FP64 walks, exact walks and CodeGen-PureReg for two (128 registers)."""
    import re

    def blocks(a, **kw):
        return int(re.search(r"__launch_bounds__\(256, (\d)\)", A.codegen_source(a, **kw)).group(1))
    a36 = synth.single_er(36, 0.15, 2, values="f64", shuffle_cols=True)
    assert blocks(a36) == 1
    assert blocks(a36, g_lo=0, g_hi=1 << 30) == 1
    assert blocks(a36, g_lo=0, g_hi=1 << 29) == 2
    assert blocks(a36, flags=A.PERM_FLAG_PURE_REG) == 2
    assert blocks(synth.single_er(28, 0.3, 6, values="f64")) == 2                   # 2^27 steps
    assert blocks(synth.band_plus(48, 3, 2, seed=3, values="01")) == 2                # exact
    assert blocks(synth.band_plus(48, 3, 2, seed=3, values="f64")) == 1


def _four_state_count(a, ins):
    """Per-step operations of four-state chains by walking the Gray schedule
    step by step: a flip of column j >= 2 updates its rows and rebuilds
    levels j..2 of the four chains; columns 0 and 1 never touch x; every
    fourth step closes a quad (four products combined and accumulated)."""
    n = a.shape[0]
    co = list(ins.col_order[:n])
    nz = a[:, co] != 0
    nnz = nz.sum(axis=0)
    first = [int(np.argmax(nz[i])) for i in range(n)]
    R = [first.count(m) for m in range(n)]
    S1, S2 = [0] * n, [0] * n
    for i in range(n):
        if nz[i, 0] or nz[i, 1]:
            nxt = next((p for p in range(2, n - 1) if nz[i, p]), None)
            if nxt is not None:
                (S2 if nz[i, 0] and nz[i, 1] else S1)[nxt] += 1
    steps = (1 << (n - 1)) - 1
    total = 0
    for l in range(1, steps + 1):
        j = (l & -l).bit_length() - 1
        if j >= 2:
            total += nnz[j] + sum((R[m] + 3 if R[m] else 0) + 5 * S1[m] + 7 * S2[m] for m in range(2, j + 1))
        if l % 4 == 3:
            total += 4
    return total / steps


def test_four_state_model_matches_a_step_by_step_count():
    """The four-state study model (perm_inspect ops_per_step_four_state) equals
    a direct count over the Gray schedule, and the order searched for it is
    never worse than the plan's order."""
    cases = [synth.single_er(12, 0.3, 1, values="f64"), synth.band_plus(14, 2, 1, seed=2, values="f64"),
             synth.single_er(16, 0.2, 7, values="f64"), synth.ones(9).astype(np.float64)]
    for a in cases:
        ins = A.inspect(a)
        want = _four_state_count(a, ins)
        assert abs(ins.ops_per_step_four_state - want) < 1e-9 * want, (ins.ops_per_step_four_state, want)
        assert ins.ops_per_step_four_state_searched <= ins.ops_per_step_four_state + 1e-12
    big = A.inspect(synth.single_er(36, 0.15, 2, values="f64", shuffle_cols=True))
    assert big.ops_per_step_four_state_searched < 0.8 * big.ops_per_step_walk
