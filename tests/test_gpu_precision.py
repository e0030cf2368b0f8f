"""GPU checks of the FP64 accuracy contract (1e-9 relative to the permanent on
every path) and of the sum of |terms| that the walks report.

The Nijenhuis-Wilf sum alternates in sign (Sec. II, Eq. 2), so an FP64 walk
is good to about n 2^-53 sum|terms| -- far above 1e-9 |perm| when the terms
cancel heavily.  Precision AUTO reruns such walks in double-double
arithmetic; PERM_PREC_DD forces it; PERM_PREC_F64 keeps plain FP64.  The
oracle (Algorithm 1 in long double: 113-bit significand on the GPU machine) is
the reference throughout."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2501_15126_gb300 import _abi as A
from paper_2501_15126_gb300 import synth

pytestmark = pytest.mark.gpu
RTOL = 1e-9
U = 2.0 ** -53
GEN, CG = A.PERM_ENGINE_GENERIC, A.PERM_ENGINE_CODEGEN


def oracle_u():
    """Unit roundoff of the oracle's long double."""
    return 2.0 ** -oracle.long_double_bits()


def dd_err(r, want):
    """|(f64 + f64_lo) - (want.hi + want.lo)| without rounding the pairs first."""
    return abs((r.f64 - want.hi) + (r.f64_lo - want.lo))


def triangular20():
    """The upper-triangular closed form of the GPU parity tests (same stream)."""
    g = np.random.default_rng(77)
    g.integers(1, 4, size=24)
    u = np.triu(g.integers(0, 3, size=(20, 20))).astype(np.int64)
    np.fill_diagonal(u, g.integers(1, 4, size=20))
    return u.astype(np.float64), float(np.prod(np.diag(u)))


def ill17():
    return synth.single_er(17, 0.1, 532, values="f64")


@pytest.mark.parametrize("n", [3, 6, 9, 13, 18, 23])
def test_double_double_walk_matches_the_oracle_far_below_fp64(n):
    """PERM_PREC_DD on signed and (0,1] values: the error is within 64 n (2^-104 +
    u_oracle) sum|terms|, orders of magnitude below what FP64 can reach."""
    g = np.random.default_rng(1000 + n)
    pat = g.random((n, n)) < 0.45
    np.fill_diagonal(pat, True)
    signed = (g.random((n, n)) * 2.0 - 1.0) * pat
    for a in (signed, synth.single_er(n, 0.4, 2000 + n, values="f64")):
        want, absum = oracle.nw_perm(a, threads=8)
        tol = 64 * n * (2.0 ** -104 + oracle_u()) * float(absum)
        r = A.permanent(a, precision=A.PERM_PREC_DD)
        assert r.precision == A.PERM_PREC_DD
        assert dd_err(r, want) <= tol, (n, dd_err(r, want), tol)
        assert abs(r.abs_term_sum - float(absum)) <= 1e-4 * float(absum)


@pytest.mark.parametrize("engine", [GEN, CG, "batch", "noalloc", "server"])
def test_auto_precision_meets_1e9_on_ill_conditioned_inputs(engine):
    """The triangular closed form (perm = prod diag, sum|terms| / perm ~ 3.5e10)
    and a sparse n=17 matrix (kappa ~ 1.6e6): precision AUTO detects the
    cancellation from the FP64 walk's sum of |terms| and reruns in
    double-double; the result is within 1e-9 of the permanent, with no escape
    clause, on every path."""
    u, want_u = triangular20()
    a17 = ill17()
    want17 = float(oracle.nw_perm(a17, threads=8)[0])
    for a, want in ((u, want_u), (a17, want17)):
        absum = float(oracle.nw_perm(a, threads=8)[1])
        assert absum / abs(want) > 1e6
        if engine == "batch":
            r = A.batch([a])[0]
        elif engine == "noalloc":
            r = A.permanent_noalloc(a)
        elif engine == "server":
            with A.Server() as s:
                r = s.poll(s.submit(a), 60000)
        else:
            r = A.permanent(a, engine=engine)
        assert r.status == 0
        assert r.precision == A.PERM_PREC_DD, engine
        assert abs(r.value - want) <= RTOL * abs(want), (engine, r.value, want)


def test_forced_fp64_stays_within_its_rounding_bound_and_reports_the_terms():
    """PERM_PREC_F64 on the same ill-conditioned inputs: the error is within
    64 n 2^-53 sum|terms| (the FP64 bound), and abs_term_sum matches the
    oracle's sum of |terms| on every kernel (generic two-state and one-chain
    walks, generated paired and two-state walks, the direct kernel)."""
    for a in (ill17(), triangular20()[0]):
        n = a.shape[0]
        want, absum = oracle.nw_perm(a, threads=8)
        want, absum = float(want), float(absum)
        for engine in (GEN, CG):
            for flags in (0, A.PERM_FLAG_PAIRED_CHAIN):
                r = A.permanent(a, engine=engine, flags=flags | A.PERM_FLAG_ABS_SUM, precision=A.PERM_PREC_F64)
                assert r.precision == A.PERM_PREC_F64
                assert abs(r.value - want) <= 64 * n * U * absum
                assert abs(r.abs_term_sum - absum) <= 1e-4 * absum, (engine, flags)
    tiny = synth.single_er(7, 0.5, 3, values="f64")                  # the direct kernel
    w, sa = oracle.nw_perm(tiny)
    r = A.permanent(tiny, precision=A.PERM_PREC_F64)
    assert abs(r.abs_term_sum - float(sa)) <= 1e-4 * float(sa)
    big = synth.single_er(40, 0.12, 8, values="f64")                 # generic one-chain walk (48 slots)
    lo, hi = 1 << 30, (1 << 30) + (1 << 20)
    r = A.permanent(big, engine=GEN, g_lo=lo, g_hi=hi)
    ins = A.inspect(big)
    s, sa = oracle.nw_range(np.ascontiguousarray(big[:, list(ins.col_order)[:40]]), lo, hi, threads=16)
    assert abs(r.value - float(s)) <= 64 * 40 * U * float(sa)
    assert abs(r.abs_term_sum - float(sa)) <= 1e-4 * float(sa)


def test_well_conditioned_walks_stay_fp64_under_auto():
    """AUTO keeps plain FP64 where it meets the target: a well-conditioned
    n=22 matrix is not rerun, and agrees with the oracle within 1e-9."""
    a = synth.single_er(22, 0.3, 11, values="f64")
    want, absum = oracle.nw_perm(a, threads=8)
    assert 22 * U * float(absum) / abs(float(want)) < 1e-11
    r = A.permanent(a)
    assert r.precision == A.PERM_PREC_F64
    assert abs(r.value - float(want)) <= RTOL * abs(float(want))


def test_batch_and_server_mix_auto_reruns_with_plain_walks():
    """A batch and a server stream mixing ill-conditioned FP64 matrices,
    well-conditioned ones and 0/1 matrices: the ill-conditioned ones (only
    those) come back in double-double, and every FP64 result is within 1e-9 of
    the oracle; the exact ones are bit-exact."""
    mats = [ill17(), triangular20()[0], synth.single_er(20, 0.3, 5, values="f64"),
            synth.single_er(19, 0.3, 6, values="01"), synth.single_er(22, 0.3, 11, values="f64")]
    want = [oracle.ryser_gray(m) if m.dtype == np.int64 else float(oracle.nw_perm(m, threads=8)[0]) for m in mats]
    res = A.batch(mats)
    with A.Server() as s:
        served = [s.poll(t, 60000) for t in [s.submit(m) for m in mats]]
    for r_list in (res, served):
        for m, r, w in zip(mats, r_list, want):
            assert r.status == 0
            if m.dtype == np.int64:
                assert r.value == w
            else:
                assert abs(r.value - w) <= RTOL * abs(w)
        assert [r.precision for r in r_list] == [2, 2, 1, 0, 1]


def test_subrange_double_double_against_the_oracle():
    """A 2^20-step sub-range of the n=36 workload in double-double: within
    64 n (2^-104 + u_oracle) of the range's sum of |terms|."""
    a = synth.single_er(36, 0.15, 2, values="f64", shuffle_cols=True)
    lo, hi = (1 << 34) + (3 << 27), (1 << 34) + (3 << 27) + (1 << 20)
    r = A.permanent(a, g_lo=lo, g_hi=hi, precision=A.PERM_PREC_DD)
    ins = A.inspect(a)
    s, sa = oracle.nw_range(np.ascontiguousarray(a[:, list(ins.col_order)[:36]]), lo, hi, threads=16)
    assert dd_err(r, s) <= 64 * 36 * (2.0 ** -104 + oracle_u()) * float(sa)


# ------------------------------------------------------------------ failure paths (no GPU fault)

def test_injected_launch_and_nvrtc_failures_are_reported_and_the_next_call_works():
    """Host-side failure injection: a walk launch that 'fails' gives
    PERM_ERR_CUDA and the same plan then computes the right value; an NVRTC
    compile that 'fails' gives PERM_ERR_NVRTC and the next plan compiles."""
    a = synth.single_er(20, 0.3, 901, values="01")
    want = oracle.ryser_gray(a)
    try:
        p = A.Plan(a, engine=GEN)
        A.inject_failures(A.PERM_SITE_LAUNCH, 1)
        with pytest.raises(A.PermError) as e:
            p.compute()
        assert e.value.status == A.PERM_ERR_CUDA
        assert p.compute().value == want
        p.close()
        af = synth.single_er(21, 0.3, 902, values="f64")
        A.inject_failures(A.PERM_SITE_NVRTC, 1)
        with pytest.raises(A.PermError) as e:
            A.permanent(af, engine=CG, flags=A.PERM_FLAG_NO_KERNEL_CACHE)
        assert e.value.status == A.PERM_ERR_NVRTC
        wantf = float(oracle.nw_perm(af, threads=8)[0])
        r = A.permanent(af, engine=CG, flags=A.PERM_FLAG_NO_KERNEL_CACHE)
        assert abs(r.value - wantf) <= RTOL * abs(wantf)
    finally:
        for site in (A.PERM_SITE_LAUNCH, A.PERM_SITE_NVRTC):
            A.inject_failures(site, 0)


def test_server_fails_requests_of_a_failed_wave_then_serves_correct_results():
    """Serving with injected failures of a wave launch, a final reduction and an
    image upload: each affected request is published with PERM_ERR_CUDA (never
    with whatever its result range held), and the requests after it are
    served correctly."""
    mats = [synth.single_er(18, 0.3, 500 + i, values="01") for i in range(8)]
    want = [oracle.ryser_gray(m) for m in mats]
    try:
        with A.Server() as s:
            assert s.poll(s.submit(mats[0]), 60000).value == want[0]
            for k, site in enumerate((A.PERM_SITE_WAVE_LAUNCH, A.PERM_SITE_FINISH, A.PERM_SITE_UPLOAD)):
                A.inject_failures(site, 1)
                r = s.poll(s.submit(mats[1 + k]), 60000)
                assert r.status == A.PERM_ERR_CUDA, site
            got = [s.poll(t, 60000) for t in [s.submit(m) for m in mats]]
            assert [g.value for g in got] == want
            assert s.stats().failed == 3
    finally:
        for site in (A.PERM_SITE_WAVE_LAUNCH, A.PERM_SITE_FINISH, A.PERM_SITE_UPLOAD):
            A.inject_failures(site, 0)


def test_generated_exact_kernels_built_for_128_registers():
    """Exact generated kernels built for two resident blocks (128 registers),
    without the 255-register rebuild: -J_15 in a 128-bit ring (a kernel that
    once returned a wrong top limb when it spilled 1.4 KB) and J_30 / J_26 in a
    192-bit ring (hundreds of bytes of spills) give their closed forms."""
    os.environ["PERM_CODEGEN_MIN_BLOCKS"] = "2"
    try:
        for a, w, want in ((-synth.ones(15), 2, -math.factorial(15)), (synth.ones(30), 3, math.factorial(30)),
                           (synth.ones(26), 3, math.factorial(26))):
            r = A.permanent(a, engine=CG, exact_words=w, flags=A.PERM_FLAG_NO_KERNEL_CACHE)
            assert r.value == want, (a.shape, w)
    finally:
        del os.environ["PERM_CODEGEN_MIN_BLOCKS"]


def test_spilling_exact_kernels_are_checked_against_the_wide_build(monkeypatch):
    """At the default register budget an exact generated kernel whose
    128-register build spills is either rebuilt for 255 registers (frames above
    512 bytes: -J_15 with one ring product per row) or cross-checked against
    that build on probe chunks (J_30 in a 192-bit ring); both give their closed
    forms."""
    monkeypatch.delenv("PERM_CODEGEN_MIN_BLOCKS", raising=False)
    monkeypatch.setenv("PERM_CODEGEN_NO_FOLD", "1")
    r = A.permanent(-synth.ones(15), engine=CG, exact_words=2, flags=A.PERM_FLAG_NO_KERNEL_CACHE)
    assert r.value == -math.factorial(15)
    monkeypatch.delenv("PERM_CODEGEN_NO_FOLD")
    r = A.permanent(synth.ones(30), engine=CG, exact_words=3, flags=A.PERM_FLAG_NO_KERNEL_CACHE)
    assert r.value == math.factorial(30)
