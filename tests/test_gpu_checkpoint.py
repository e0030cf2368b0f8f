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


@pytest.mark.parametrize("values", ["01", "f64"])
def test_torn_and_altered_records_are_recomputed(values, tmp_path):
    """A run stopped in the middle of writing leaves a torn last line; a later
    append must not glue onto it, and a record whose words were altered fails
    its check word.  Such records are recomputed, so the final value is the
    same bits as an uninterrupted run."""
    a = synth.single_er(22, 0.3, 73, values=values)
    path = str(tmp_path / "run.ckpt")
    st, r = A.checkpoint_run(a, path, slice_log2=16, max_slices=10)
    assert st == A.PERM_ERR_NOT_READY
    lines = open(path).read().splitlines(keepends=True)
    assert lines[0].startswith("perm-checkpoint v2") and len(lines) == 11
    # alter one word of slice record 3 (its check word no longer matches),
    # and cut the last record in the middle of a hex word (no newline)
    words = lines[3].split()
    words[2] = ("%016x" % (int(words[2], 16) ^ 1))
    lines[3] = " ".join(words) + "\n"
    lines[-1] = lines[-1][: len(lines[-1]) // 2]
    open(path, "w").write("".join(lines))
    st, r = A.checkpoint_run(a, path, slice_log2=16)
    assert st == A.PERM_OK
    whole_path = str(tmp_path / "whole.ckpt")
    st, w = A.checkpoint_run(a, whole_path, slice_log2=16)
    assert st == A.PERM_OK
    assert (r.f64, r.f64_lo, r.i128_lo, r.i128_hi) == (w.f64, w.f64_lo, w.i128_lo, w.i128_hi)
    if values == "01":
        assert r.value == oracle.ryser_gray(a)
    after = open(path).read().splitlines()
    assert after[10] == lines[-1]                      # the torn fragment stays on its own line
    assert all(line.startswith("slice ") for line in after[11:])
