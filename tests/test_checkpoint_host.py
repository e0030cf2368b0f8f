"""Checkpointed runs on the host (Sec. II-A: the Gray range splits into
independent slices whose partial sums add up to the whole).  A checkpoint
file whose slice records are all present needs no GPU: perm_checkpoint_run
only parses the records, combines them in slice order and finishes the sum.
Here the records are written from the oracle's partial sums, so the test pins
the record format and its check words, the combination (compensated FP64
additions, ring additions) and the finishing step against the oracle; and it
checks that a torn or altered record is not accepted (the call then tries to
recompute that slice, which without a GPU is a CUDA error)."""
import os
import struct
import tempfile

import numpy as np
import pytest

import oracle
from paper_2501_15126_gb300 import _abi as A
from paper_2501_15126_gb300 import synth

MASK64 = (1 << 64) - 1


def fnv1a(data: bytes) -> int:
    """FNV-1a, 64-bit (offset basis 14695981039346656037, prime 1099511628211)."""
    h = 14695981039346656037
    for b in data:
        h = ((h ^ b) * 1099511628211) & MASK64
    return h


def record(idx: int, words) -> str:
    check = fnv1a(struct.pack("<Q", idx) + b"".join(struct.pack("<Q", w) for w in words))
    return "slice %d %s %016x\n" % (idx, " ".join("%016x" % w for w in words), check)


def f64_word(v: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", v))[0]


def run(a, path, slice_log2):
    """perm_checkpoint_run: (status, Result or None)."""
    try:
        return A.checkpoint_run(a, path, slice_log2=slice_log2)
    except A.PermError as e:
        return e.status, None


def header_of(a, path, slice_log2):
    """The library writes the file's header before it computes anything; with
    no GPU the first slice then fails, which leaves the header behind."""
    st, _ = run(a, path, slice_log2)
    assert st == A.PERM_ERR_CUDA
    lines = open(path).read().splitlines()
    assert len(lines) == 1 and lines[0].startswith("perm-checkpoint v2 hash=")
    return lines[0] + "\n"


def plan_order(a):
    return np.ascontiguousarray(a[:, list(A.inspect(a).col_order)[: a.shape[0]]])


pytestmark = pytest.mark.skipif(A.lib().perm_device_available() != 0,
                                reason="the host-only form needs a machine without a GPU")


@pytest.mark.parametrize("n,seed", [(12, 1), (15, 2)])
def test_exact_records_from_the_oracle_give_the_permanent(n, seed):
    a = synth.single_er(n, 0.35, seed, values="01")
    ao = plan_order(a)
    words = A.inspect(a).exact_words
    assert words == 1   # the oracle's doubled walk is exact modulo 2^128
    slice_log2 = n - 4
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "run.ckpt")
        text = header_of(a, path, slice_log2)
        for i in range(8):
            part = oracle.nw2_range(ao, i << slice_log2, (i + 1) << slice_log2)
            text += record(i, [part & MASK64])
        open(path, "w").write(text)
        st, r = run(a, path, slice_log2)
        assert st == A.PERM_OK and r.value == oracle.ryser_gray(a)
        assert r.steps == 1 << (n - 1)
        # the same records in another order in the file: the same integer
        body = text.splitlines(keepends=True)
        open(path, "w").write(body[0] + "".join(reversed(body[1:])))
        st, r2 = run(a, path, slice_log2)
        assert st == A.PERM_OK and r2.value == r.value


def test_fp64_records_from_the_oracle_give_the_permanent():
    n = 14
    a = synth.single_er(n, 0.3, 3, values="f64")
    ao = plan_order(a)
    slice_log2 = n - 4
    want = float(oracle.nw_perm(a)[0])
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "run.ckpt")
        text = header_of(a, path, slice_log2)
        absum = 0.0
        for i in range(8):
            s, sa = oracle.nw_range(ao, i << slice_log2, (i + 1) << slice_log2)
            absum += float(sa)
            text += record(i, [f64_word(s.hi), f64_word(s.lo), f64_word(float(sa))])
        open(path, "w").write(text)
        st, r = run(a, path, slice_log2)
        assert st == A.PERM_OK
        assert abs(r.value - want) <= 1e-14 * abs(want)
        assert abs(r.abs_term_sum - 2.0 * absum) <= 1e-12 * absum


@pytest.mark.parametrize("damage", ["torn", "check", "word", "joined", "uppercase", "index"])
def test_damaged_records_are_not_accepted(damage):
    """Every record valid but one: a torn last line (no newline), a wrong check
    word, an altered sum, two records on one line, a word in upper-case hex,
    and an index beyond the last slice.  The damaged slice counts as missing,
    so the call goes on to compute it (a CUDA error here, without a GPU)."""
    n = 12
    a = synth.single_er(n, 0.35, 1, values="01")
    ao = plan_order(a)
    slice_log2 = n - 4
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "run.ckpt")
        text = header_of(a, path, slice_log2)
        recs = [record(i, [oracle.nw2_range(ao, i << slice_log2, (i + 1) << slice_log2) & MASK64]) for i in range(8)]
        if damage == "torn":
            recs[7] = recs[7][:-5]
        elif damage == "check":
            recs[3] = recs[3][:-2] + ("0" if recs[3][-2] != "0" else "1") + "\n"
        elif damage == "word":
            f = recs[5].split()
            f[2] = "%016x" % (int(f[2], 16) ^ 1)
            recs[5] = " ".join(f) + "\n"
        elif damage == "joined":
            recs[2] = recs[2][:-1] + " " + recs[3]
            recs[3] = ""
        elif damage == "uppercase":
            recs[4] = recs[4].upper().replace("SLICE", "slice")
        else:
            recs[6] = record(8, [0])   # slice 8 of 8 does not exist, and slice 6 is then missing
        open(path, "w").write(text + "".join(recs))
        st, _ = run(a, path, slice_log2)
        assert st == A.PERM_ERR_CUDA
        # the intact file gives the permanent
        open(path, "w").write(text + "".join(
            record(i, [oracle.nw2_range(ao, i << slice_log2, (i + 1) << slice_log2) & MASK64]) for i in range(8)))
        st, r = run(a, path, slice_log2)
        assert st == A.PERM_OK and r.value == oracle.ryser_gray(a)


def test_a_file_for_another_matrix_is_refused():
    n = 12
    a = synth.single_er(n, 0.35, 1, values="01")
    b = synth.single_er(n, 0.35, 2, values="01")
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "run.ckpt")
        header_of(a, path, n - 4)
        st, _ = run(b, path, n - 4)
        assert st == A.PERM_ERR_ARG
        st, _ = run(a, path, n - 5)
        assert st == A.PERM_ERR_ARG
