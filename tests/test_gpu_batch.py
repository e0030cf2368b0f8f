"""GPU parity of perm_batch (one persistent launch per kernel family) against
the oracle and against one plan per matrix; results are identical alone and
in the mix."""
import numpy as np
import pytest

import oracle
from paper_2501_15126_gb300 import _abi as A
from paper_2501_15126_gb300 import synth

pytestmark = pytest.mark.gpu
MASK128 = (1 << 128) - 1


def oracle_value(item):
    a = item.a
    n = a.shape[0]
    if item.values == "01":
        if n <= 22:
            return oracle.ryser_gray(a)
        # doubled Algorithm 1 modulo 2^128 is (-1)^(n-1) 2^(n-1) perm; exact when |perm| < 2^(127-n)
        s = oracle.nw2_range(a, 0, 1 << (n - 1), threads=16)
        s = s - (1 << 128) if s >> 127 else s
        assert s % (1 << (n - 1)) == 0
        return (-1) ** (n - 1) * (s >> (n - 1))
    return float(oracle.nw_perm(a, threads=16)[0])


def check(item, r):
    want = oracle_value(item)
    if item.values == "01":
        assert r.value == want
    else:
        assert abs(r.value - want) <= 1e-9 * abs(want)


def test_small_mixed_batch_matches_oracle_and_sequential():
    items = synth.batch(count=80, n_lo=9, n_hi=22, seed=41)
    res = A.batch([it.a for it in items])
    seq = A.batch([it.a for it in items], sequential=True)
    for it, r, s in zip(items, res, seq):
        assert r.status == 0 and s.status == 0
        check(it, r)
        if it.values == "01":
            assert r.value == s.value
        else:
            assert abs(r.value - s.value) <= 1e-12 * abs(s.value)


def test_batch_edge_cases():
    z = np.eye(6, dtype=np.int64)
    z[3, 3] = 0
    mats = [np.array([[3]], dtype=np.int64), np.array([[0.5, 1.0], [2.0, 4.0]]), z, synth.ones(10)]
    res = A.batch(mats)
    assert res[0].value == 3
    assert abs(res[1].value - 4.0) < 1e-15
    assert res[2].value == 0
    assert res[3].value == 3628800
    bad = A.CSRMatrix(n=3, ptr=[0, 1, 2, 3], idx=[0, 7, 1], vals=[1.0, 1.0, 1.0], vtype=A.PERM_F64)
    res = A.batch([synth.ones(9), bad, synth.ones(11)])
    assert res[0].value == 362880 and res[1].status == A.PERM_ERR_PATTERN and res[2].value == 39916800


def test_full_size_batch_sampled_and_alone_vs_mix():
    """The 10,000-matrix workload (n in [12,28], p in [0.2,0.4] + diagonal,
    alternating 0/1 and real values): sampled matrices against the oracle, and
    every sampled matrix computed alone gives the same bits as in the batch."""
    items = synth.batch()
    res = A.batch([it.a for it in items])
    assert all(r.status == 0 for r in res)
    rng = np.random.default_rng(0)
    by_n = {}
    for i, it in enumerate(items):
        by_n.setdefault(it.n, []).append(i)
    sample = [by_n[28][0], by_n[28][1], by_n[27][0], by_n[27][1]]
    sample += list(rng.choice([i for i, it in enumerate(items) if it.n <= 24], size=24, replace=False))
    for i in sample:
        check(items[i], res[i])
        alone = A.batch([items[i].a])[0]
        if items[i].values == "01":
            assert alone.value == res[i].value
        else:
            assert (alone.f64, alone.f64_lo) == (res[i].f64, res[i].f64_lo)


def test_large_sparse_matrices_in_a_batch_match_the_row_dp():
    """The same large sparse matrices as the serving test (n = 26..40), in one
    batch with small ones, against the oracle's row-expansion DP."""
    from tests.test_gpu_serving import check_against_row_dp, large_sparse_requests
    mats = large_sparse_requests() + [it.a for it in synth.batch(count=40, seed=8) if it.n <= 20]
    res = A.batch(mats)
    for m, r in zip(mats, res):
        check_against_row_dp(m, r)
