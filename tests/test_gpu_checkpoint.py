"""Resumable runs: a walk split across calls (and resumed from its file)
gives the same bits as one uninterrupted walk."""
import os

import pytest

import oracle
from paper_2501_15126_gb300 import _abi as A
from paper_2501_15126_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("values", ["01", "f64"])
def test_checkpointed_run_resumes_and_matches(values, tmp_path):
    a = synth.single_er(24, 0.25, 71, values=values)
    path = str(tmp_path / "run.ckpt")
    calls = 0
    while True:
        st, r = A.checkpoint_run(a, path, slice_log2=18, max_slices=7)
        calls += 1
        if st == A.PERM_OK:
            break
        assert st == A.PERM_ERR_NOT_READY and 0 < r.steps < 1 << 23
    assert calls == 5                                  # 32 slices, 7 per call
    whole = A.permanent(a)
    if values == "01":
        assert r.value == whole.value == oracle.ryser_gray(a)
    else:
        assert abs(r.value - whole.value) <= 1e-12 * abs(whole.value)
    st2, r2 = A.checkpoint_run(a, path, slice_log2=18)  # everything recorded: no new work
    assert st2 == A.PERM_OK and (r2.f64, r2.i128_lo) == (r.f64, r.i128_lo)
    other = synth.single_er(24, 0.25, 72, values=values)
    with pytest.raises(A.PermError) as e:
        A.checkpoint_run(other, path, slice_log2=18)
    assert e.value.status == A.PERM_ERR_ARG
