"""perm_compute_noalloc: the permanent for callers that may not allocate
device memory (their memory pool belongs to someone else, or every byte of
HBM is reserved in advance, or they may not call cudaMalloc/cudaFree at all).
It keeps its scratch in a fixed 1 MiB device array inside the library instead
of allocating.  Each check calls it twice in a row on different matrices (the
array keeps the previous call's contents) and compares both results with
perm_plan_create + perm_compute: bit-identical on the exact path, within 1e-9
relative on the FP64 path.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2501_15126_gb300 import _abi as A
from paper_2501_15126_gb300 import synth

pytestmark = pytest.mark.gpu


def same(a, b):
    if a.vtype == A.PERM_I64:
        return a.value == b.value
    return abs(a.value - b.value) <= 1e-9 * abs(b.value)


@pytest.mark.parametrize("values", ["01", "f64"])
def test_noalloc_matches_plan_compute_twice_in_a_row(values):
    m1 = synth.single_er(26, 0.22, 31, values=values)
    m2 = synth.single_er(19, 0.35, 32, values=values)
    r1 = A.permanent_noalloc(m1)
    r2 = A.permanent_noalloc(m2)
    assert r1.status == 0 and r2.status == 0
    assert same(r1, A.permanent(m1, engine=A.PERM_ENGINE_GENERIC))
    assert same(r2, A.permanent(m2, engine=A.PERM_ENGINE_GENERIC))
    assert not same(r1, r2)


def test_noalloc_tiny_and_large_n():
    t = np.array([[2, 1, 0], [1, 3, 1], [0, 1, 4]], dtype=np.int64)
    assert A.permanent_noalloc(t).value == A.permanent(t).value
    b = synth.single_er(31, 0.15, 33, values="f64")
    r = A.permanent_noalloc(b)
    assert same(r, A.permanent(b, engine=A.PERM_ENGINE_GENERIC))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    big = synth.single_er(49, 0.1, 34, values="01")
    with pytest.raises(A.PermError) as e:
        A.permanent_noalloc(big)
    assert e.value.status == A.PERM_ERR_SIZE
