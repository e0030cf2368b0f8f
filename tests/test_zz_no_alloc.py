"""perm_compute_noalloc: the permanent for callers that may not allocate
device memory (their memory pool belongs to someone else, or every byte of
HBM is reserved in advance, or they may not call cudaMalloc/cudaFree at all).
It keeps its scratch in a fixed 1 MiB device array inside the library instead
of allocating.  Each check calls it twice in a row on different matrices (the
array keeps the previous call's contents) and compares both results with the
CPU oracle -- bit-identical on the exact path, within 1e-9 relative on the
FP64 path -- and with perm_plan_create + perm_compute.  This file is collected
last on purpose."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2501_15126_gb300 import _abi as A
from paper_2501_15126_gb300 import synth

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


def oracle_value(a):
    if a.dtype == np.int64:
        return oracle.ryser_gray(a)
    return float(oracle.nw_perm(a, threads=16)[0])


def matches(r, want):
    if r.vtype == A.PERM_I64:
        return r.value == want
    return abs(r.value - want) <= 1e-9 * abs(want)


@pytest.mark.parametrize("values", ["01", "f64"])
def test_noalloc_matches_the_oracle_twice_in_a_row(values):
    m1 = synth.single_er(26, 0.22, 31, values=values)
    m2 = synth.single_er(19, 0.35, 32, values=values)
    w1, w2 = oracle_value(m1), oracle_value(m2)
    r1 = A.permanent_noalloc(m1)
    r2 = A.permanent_noalloc(m2)
    assert r1.status == 0 and r2.status == 0
    assert matches(r1, w1) and matches(r2, w2)
    assert matches(A.permanent(m1, engine=A.PERM_ENGINE_GENERIC), w1)
    assert not matches(r1, w2)


def test_noalloc_tiny_and_large_n():
    t = np.array([[2, 1, 0], [1, 3, 1], [0, 1, 4]], dtype=np.int64)
    assert A.permanent_noalloc(t).value == oracle.brute_int(t)
    b = synth.single_er(31, 0.15, 33, values="f64")
    r = A.permanent_noalloc(b)
    assert matches(r, float(A.permanent(b, engine=A.PERM_ENGINE_GENERIC).value))


@pytest.mark.parametrize("values", ["01", "f64"])
def test_noalloc_n40_subrange_against_the_oracle(values):
    """n = 40 (the 48-slot bucket, whose image is sized against the array's
    20480-byte region): a 2^28-step aligned sub-range, against the oracle's
    partial sum and against perm_plan_create + perm_compute."""
    a = synth.band_plus(40, 3, 2, seed=40, values=values)
    lo, hi = 0, 1 << 28
    r = A.permanent_noalloc(a, g_lo=lo, g_hi=hi)
    p = A.permanent(a, engine=A.PERM_ENGINE_GENERIC, g_lo=lo, g_hi=hi)
    ins = A.inspect(a)
    ao = np.ascontiguousarray(a[:, list(ins.col_order)[:40]])
    if values == "01":
        assert r.partial_int == p.partial_int
        bits = min(128, 64 * r.exact_words)
        mask = (1 << bits) - 1
        assert r.partial_int & mask == oracle.nw2_range(ao, lo, hi, threads=16) & mask
    else:
        s, sa = oracle.nw_range(ao, lo, hi, threads=16)
        assert abs(r.value - float(s)) <= 64 * 40 * U * float(sa)
        assert (r.f64, r.f64_lo) == (p.f64, p.f64_lo)


def test_noalloc_allocates_no_device_memory():
    """After a warm-up call, further calls leave the device's free memory
    exactly where it was."""
    import torch
    a = synth.single_er(24, 0.25, 35, values="f64")
    b = synth.single_er(22, 0.3, 36, values="01")
    A.permanent_noalloc(a)
    A.permanent_noalloc(b)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for m in (a, b, a, b):
        A.permanent_noalloc(m)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_what_does_not_fit_before_launching():
    """n > 48, and a sub-range whose ends are aligned only to 32 and too long
    for the array's task area, give PERM_ERR_SIZE with out.status set."""
    big = synth.single_er(49, 0.1, 34, values="01")
    with pytest.raises(A.PermError) as e:
        A.permanent_noalloc(big)
    assert e.value.status == A.PERM_ERR_SIZE
    a = synth.single_er(31, 0.15, 37, values="01")
    m = A.CSRMatrix(a)
    o = A.opts(g_lo=32, g_hi=1 << 30)
    r = A.Result()
    st = A.lib().perm_compute_noalloc(ctypes.byref(m.c), ctypes.byref(o), None, ctypes.byref(r))
    assert st == A.PERM_ERR_SIZE and r.status == A.PERM_ERR_SIZE


def test_noalloc_honours_the_device_deadline():
    """timeout_ms stops a long walk on the device (PERM_ERR_TIMEOUT, out.status
    set), and the next call is right."""
    big = synth.single_er(40, 0.1, 5, values="f64")
    with pytest.raises(A.PermError) as e:
        A.permanent_noalloc(big, timeout_ms=50)
    assert e.value.status == A.PERM_ERR_TIMEOUT
    small = synth.single_er(18, 0.3, 38, values="01")
    assert A.permanent_noalloc(small).value == oracle.ryser_gray(small)
