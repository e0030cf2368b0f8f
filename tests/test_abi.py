"""The C ABI library loads on a machine without a GPU, exports every function
include/perm.h declares, and agrees with the binding on struct layouts.  No
compute call is made here."""
import ctypes
import os
import re

import pytest

from paper_2501_15126_gb300 import _abi as A

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "perm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(perm_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("perm_plan_create", "perm_compute", "perm_plan_destroy", "perm_batch", "perm_submit", "perm_poll",
                 "perm_server_create", "perm_server_destroy", "perm_compute_noalloc"):
        assert must in names


def test_library_exports_every_declared_symbol():
    L = A.lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    bound = {s[0] for s in A.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_struct_layouts_match():
    L = A.lib()
    for i, S in enumerate(A.STRUCTS):
        assert L.perm_sizeof(i) == ctypes.sizeof(S), S.__name__
    assert L.perm_sizeof(99) == -1


def test_status_strings_and_version():
    L = A.lib()
    assert L.perm_status_string(0) == b"ok"
    assert L.perm_status_string(A.PERM_ERR_OVERFLOW).startswith(b"exact")
    assert L.perm_version().decode().count(".") == 2


def test_bad_arguments_fail_without_a_gpu():
    L = A.lib()
    assert L.perm_plan_create(None, None, None) == A.PERM_ERR_ARG
    bad = A.CSRMatrix(n=3, ptr=[0, 1, 2, 3], idx=[0, 5, 1], vals=[1.0, 1.0, 1.0], vtype=A.PERM_F64)
    h = ctypes.c_void_p()
    assert L.perm_plan_create(ctypes.byref(bad.c), None, ctypes.byref(h)) == A.PERM_ERR_PATTERN
    assert b"range" in L.perm_last_error()
    rep = A.CSRMatrix(n=2, ptr=[0, 2, 3], idx=[1, 1, 0], vals=[1.0, 1.0, 1.0], vtype=A.PERM_F64)
    assert L.perm_plan_create(ctypes.byref(rep.c), None, ctypes.byref(h)) == A.PERM_ERR_PATTERN
    big = A.CSRMatrix(n=65, ptr=list(range(66)), idx=list(range(65)), vals=[1.0] * 65, vtype=A.PERM_F64)
    assert L.perm_plan_create(ctypes.byref(big.c), None, ctypes.byref(h)) == A.PERM_ERR_SIZE
    r = A.Result()
    assert L.perm_compute_noalloc(ctypes.byref(big.c), None, None, ctypes.byref(r)) == A.PERM_ERR_SIZE


def test_server_create_reports_a_missing_device():
    """perm_server_create checks the device ordinal before touching it: without
    a GPU it fails with CUDA, with one an ordinal past the last device gives ARG;
    neither starts a thread or leaks a handle."""
    L = A.lib()
    h = ctypes.c_void_p()
    o = A.ServerOpts()
    o.device = 7 if L.perm_device_available() else 0
    st = L.perm_server_create(ctypes.byref(o), ctypes.byref(h))
    assert st == (A.PERM_ERR_ARG if L.perm_device_available() else A.PERM_ERR_CUDA)
    assert not h.value
    assert b"device" in L.perm_last_error()


@pytest.mark.skipif(A.lib().perm_device_available() != 0, reason="shows that no device is touched")
def test_zero_permanents_and_empty_ranges_launch_nothing():
    """A matrix without a perfect matching (an empty row, or rows that share
    too few columns) has permanent 0, and an empty Gray sub-range [g, g) the
    partial sum 0: plan, compute and destroy run here, on a machine without a
    GPU, which shows that nothing is launched or allocated on a device."""
    import numpy as np
    from paper_2501_15126_gb300 import synth
    empty_row = np.ones((6, 6), dtype=np.int64)
    empty_row[2, :] = 0
    hall = np.zeros((5, 5))
    hall[:, :2] = 0.5          # five rows, two columns between them: no matching
    hall[0, :] = 1.0
    for a in (empty_row, hall, synth.ones(10) * np.tri(10, k=-1, dtype=np.int64)):
        r = A.permanent(a)
        assert (r.value, r.steps, r.status) == (0, 0, A.PERM_OK)
    a = synth.single_er(20, 0.3, 4, values="01")
    w = A.inspect(a).exact_words
    r = A.permanent(a, g_lo=64, g_hi=64)
    assert (r.partial_int, r.steps, r.exact_words) == (0, 0, w)
    r = A.permanent(synth.single_er(20, 0.3, 4, values="f64"), g_lo=1 << 10, g_hi=1 << 10)
    assert (r.f64, r.f64_lo, r.steps) == (0.0, 0.0, 0)
    res = A.batch([empty_row, hall])
    assert [x.value for x in res] == [0, 0]
