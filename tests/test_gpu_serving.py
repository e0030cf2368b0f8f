"""GPU tests of the serving loop: results equal the oracle and are the same
alone and in a mix of concurrent requests; requests that arrive while others
run are admitted and overlap; timeouts and shutdown cancel cleanly."""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_2501_15126_gb300 import _abi as A
from paper_2501_15126_gb300 import synth

pytestmark = pytest.mark.gpu


def test_served_results_match_oracle_and_alone():
    reqs = synth.serving_stream(rate=2000.0, duration=0.05, seed=5)
    mats = [r.a for r in reqs][:60]
    with A.Server() as s:
        tickets = [s.submit(m) for m in mats]
        mixed = [s.poll(t, 60000) for t in tickets]
    alone = []
    for m in mats:
        with A.Server() as s:
            alone.append(s.poll(s.submit(m), 60000))
    for m, r, a in zip(mats, mixed, alone):
        assert r.status == 0 and a.status == 0
        if m.dtype == np.int64:
            assert r.value == a.value == oracle.ryser_gray(m) if m.shape[0] <= 22 else r.value == a.value
        else:
            assert (r.f64, r.f64_lo) == (a.f64, a.f64_lo)
            if m.shape[0] <= 24:
                want = float(oracle.nw_perm(m, threads=16)[0])
                assert abs(r.value - want) <= 1e-9 * abs(want)


def test_large_request_does_not_block_small_ones():
    """A 2^33-step request is sliced across waves; small requests submitted
    after it finish before it does, and everything matches the plan path."""
    big = synth.single_er(34, 0.12, 77, values="f64")
    small = [synth.single_er(18, 0.3, 100 + i, values="01") for i in range(20)]
    with A.Server() as s:
        tb = s.submit(big)
        time.sleep(0.005)
        ts = [s.submit(m) for m in small]
        done_small = [s.poll(t, 60000) for t in ts]
        t_small = time.time()
        rb = s.poll(tb, 120000)
        t_big = time.time()
        st = s.stats()
    assert t_small <= t_big
    for m, r in zip(small, done_small):
        assert r.value == oracle.ryser_gray(m)
    ref = A.permanent(big, engine=A.PERM_ENGINE_GENERIC)
    assert abs(rb.value - ref.value) <= 1e-9 * abs(ref.value)
    assert st.completed == 21 and st.p99_ms >= st.p50_ms > 0


def test_concurrent_submitters_and_poll_semantics():
    mats = [synth.single_er(20, 0.25, 300 + i, values="01") for i in range(40)]
    want = [oracle.ryser_gray(m) for m in mats]
    out = [None] * len(mats)
    with A.Server(max_inflight=8) as s:
        def worker(lo):
            for i in range(lo, len(mats), 4):
                out[i] = s.poll(s.submit(mats[i]), 60000)
        th = [threading.Thread(target=worker, args=(k,)) for k in range(4)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        with pytest.raises(A.PermError):
            s.poll(123456789, 0)          # unknown ticket
    assert [r.value for r in out] == want


def test_timeout_and_shutdown():
    big = synth.single_er(38, 0.1, 5, values="f64")
    s = A.Server(timeout_ms=50)
    t = s.submit(big)
    r = s.poll(t, 60000)
    assert r.status == A.PERM_ERR_TIMEOUT
    s.close()
    s2 = A.Server()
    t2 = s2.submit(synth.single_er(36, 0.1, 6, values="f64"))
    s2.close()      # cancels the unfinished request and frees everything


def large_sparse_requests():
    """Sparse requests of n = 26..40 (ER p = 0.06..0.1 + diagonal), 0/1 and
    (0,1] values, whose permanents the oracle's row-expansion DP (Eq. 1)
    gives at once."""
    out = []
    for k, (n, p) in enumerate([(26, 0.1), (30, 0.1), (34, 0.08), (36, 0.08), (40, 0.06)]):
        out.append(synth.single_er(n, p, 901 + k, values="01"))
        out.append(synth.single_er(n, p, 951 + k, values="f64"))
    return out


def check_against_row_dp(m, r):
    assert r.status == 0
    if m.dtype == np.int64:
        assert r.value == oracle.rowdp_int(m)
    else:
        want = float(oracle.rowdp(m))
        n = m.shape[0]
        assert abs(r.value - want) <= max(1e-9 * abs(want), 64 * n * 2.0 ** -53 * r.abs_term_sum), (n, r.value, want)


def test_large_sparse_requests_match_the_row_dp():
    """Served requests far beyond the oracle walk's reach on the CPU (up to 2^39
    Gray steps), mixed with small ones: exact results equal the oracle's
    row-expansion DP bit for bit, FP64 ones agree within 1e-9 or the rounding
    bound of their sum of |terms|."""
    big = large_sparse_requests()
    small = [r.a for r in synth.serving_stream(rate=2000.0, duration=0.01, seed=6) if r.a.shape[0] <= 22][:10]
    with A.Server() as s:
        tickets = [s.submit(m) for m in big + small]
        res = [s.poll(t, 120000) for t in tickets]
    for m, r in zip(big + small, res):
        check_against_row_dp(m, r)
