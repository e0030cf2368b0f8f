"""Host emulation of the precompiled generic kernels (the batch and serving
walks): the walk code of generic_impl.cuh and core.cuh is compiled as plain
host C++ under AddressSanitizer and UndefinedBehaviorSanitizer, with the
matrix image the library builds for the GPU (perm_generic_image) in a heap
buffer of exactly the image's size, so a read past the image is caught.
Each 2^K-step chunk of the Gray walk runs as one lane (warp votes and
shuffles reduce to the lane's own value) and its partial sum is compared
with the oracle's sum over the same Gray range: exact rings bit for bit
(modulo the ring, at most 2^128 for the oracle), FP64 within its rounding
bound, double-double within a bound FP64 could not meet.  Built twice, with
automatic variables initialised to zero and to a byte pattern.  Test
infrastructure; no GPU needed."""
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from paper_2501_15126_gb300 import _abi as A
from paper_2501_15126_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2501_15126_gb300", "csrc")
U = 2.0 ** -53

HARNESS = r'''
#include "shim.h"
#include "generic_impl.cuh"
#include <cstdio>
#include <cstdlib>
typedef pk::GenericPol<PERM_TEST_NMAX, PERM_TEST_ARITH> Pol;
int main(int argc, char **argv) {
    FILE *f = std::fopen(argv[1], "rb");
    if (!f) return 2;
    std::fseek(f, 0, SEEK_END);
    const long bytes = std::ftell(f);
    std::fseek(f, 0, SEEK_SET);
    void *img = std::aligned_alloc(16, (size_t)bytes);   // exactly the image: ASan sees any read past it
    if (std::fread(img, 1, (size_t)bytes, f) != (size_t)bytes) return 3;
    std::fclose(f);
    const int K = std::atoi(argv[2]);
    const int shift = std::atoi(argv[3]);
    const int zero_skip = std::atoi(argv[4]);
    unsigned long long q;
    while (std::scanf("%llu", &q) == 1) {
        Pol pol(reinterpret_cast<const Pol::M *>(img), shift);
        unsigned long long skipped = 0, w[6] = {0, 0, 0, 0, 0, 0};
        typename PERM_TEST_ARITH::Acc acc;
        if constexpr (Pol::kDual)
            acc = pk::walk_chunk_dual<Pol, PERM_TEST_ARITH, PERM_GENERIC_B>(pol, q, K, zero_skip, skipped);
        else
            acc = pk::walk_chunk_compact<PERM_TEST_NMAX, PERM_TEST_ARITH>(pol, q, K, zero_skip, skipped);
        PERM_TEST_ARITH::acc_store(w, acc);
        std::printf("%llu %llu", q, skipped);
        for (int i = 0; i < PERM_TEST_ARITH::ACC_WORDS; ++i) std::printf(" %016llx", w[i]);
        std::printf("\n");
    }
    std::free(img);
    return 0;
}
'''


def arith_of(kind):
    if kind == 0:
        return "pk::ArithF64"
    if kind == 1:
        return "pk::ArithDD"
    return "pk::ArithExact%s<%d>" % ("Fold" if kind & 1 else "", kind // 2)


def emulate(a, K, chunks, init, zero_skip=1, **kw):
    """Builds the harness for the matrix's kernel family and runs the chunks;
    returns ({q: [words]}, {q: skipped blocks}, kind, abs_shift)."""
    img, nmax, kind, shift = A.generic_image(a, **kw)
    with tempfile.TemporaryDirectory() as d:
        open(os.path.join(d, "image.bin"), "wb").write(img)
        open(os.path.join(d, "main.cpp"), "w").write(HARNESS)
        exe = os.path.join(d, "walk")
        subprocess.check_call(["g++", "-std=c++17", "-O1", "-g", "-fsanitize=address,undefined",
                               "-fno-sanitize-recover=all", "-ftrivial-auto-var-init=" + init,
                               "-DPERM_TEST_NMAX=%d" % nmax, "-DPERM_TEST_ARITH=" + arith_of(kind),
                               "-I", os.path.join(HERE, "host_emulation"), "-I", CSRC,
                               os.path.join(d, "main.cpp"), "-o", exe])
        out = subprocess.run([exe, os.path.join(d, "image.bin"), str(K), str(shift), str(zero_skip)],
                             input=" ".join(map(str, chunks)), capture_output=True, text=True, check=True).stdout
    res, skips = {}, {}
    for line in out.splitlines():
        f = line.split()
        res[int(f[0])] = [int(x, 16) for x in f[2:]]
        skips[int(f[0])] = int(f[1])
    return res, skips, kind, shift


def plan_order(a, **kw):
    ins = A.inspect(a, **{k: v for k, v in kw.items() if k == "ordering"})
    return np.ascontiguousarray(a[:, list(ins.col_order)[: a.shape[0]]])


def check(a, K, chunks, tol=None, zero_skip=1, **kw):
    """Every chunk against the oracle, in both builds (and their sums of
    |terms| within 1e-4 on the FP64 paths); returns (skip counts, kind)."""
    ao = plan_order(a, **kw)
    n = a.shape[0]
    got = {init: emulate(a, K, chunks, init, zero_skip, **kw) for init in ("zero", "pattern")}
    kind, shift = got["zero"][2], got["zero"][3]
    for q in chunks:
        if kind >= 2:
            mask = (1 << min(128, 32 * (kind // 2))) - 1   # the ring has kind // 2 limbs of 32 bits
            want = oracle.nw2_range(ao, q << K, (q + 1) << K) & mask
            for init in got:
                v = sum(w << (64 * i) for i, w in enumerate(got[init][0][q])) & mask
                assert v == want, (init, q)
        else:
            s, sa = oracle.nw_range(ao, q << K, (q + 1) << K)
            bound = (tol if tol is not None else 64 * n * U) * float(sa)
            for init in got:
                hi, lo, ab = np.array(got[init][0][q], dtype=np.uint64).view(np.float64)
                assert abs((hi + lo) - float(s)) <= bound, (init, q, hi + lo, float(s))
                assert abs(np.ldexp(ab, shift) - float(sa)) <= 1e-4 * float(sa), (init, q)
    assert got["zero"][0] == got["pattern"][0]
    return got["zero"][1], kind


def test_fp64_two_state_walk_at_16_and_32_slots():
    """FP64 batch-class matrices (ER p in [0.2, 0.4] + diagonal, (0,1]): n = 14
    (16 slots) and n = 27 (32 slots; the column order searched under the
    two-state model), both walked with two-state chains."""
    for n, p, seed, K in ((14, 0.35, 5, 8), (27, 0.3, 6, 10)):
        a = synth.single_er(n, p, seed, values="f64")
        top = (1 << (n - 1)) >> K
        _, kind = check(a, K, [0, 1, top // 3, top - 1])
        assert kind == 0


def test_fp64_single_chain_at_48_slots():
    """n = 40 FP64 (the 48-slot bucket keeps one chain): chunks with high Gray
    bits set."""
    a = synth.single_er(40, 0.12, 7, values="f64")
    K = 10
    top = (1 << 39) >> K
    _, kind = check(a, K, [0, 3, top // 2, top - 1])
    assert kind == 0


@pytest.mark.parametrize("values", ["01", "wide"])
def test_exact_rings_folded_and_unfolded(values):
    """Exact walks: a 0/1 matrix at 32 slots (row sums <= 127: slot quadruples
    folded in 32 bits) and one at 16 slots with entries up to +-40 and a
    diagonal of 100 (row sums above 127: no folding)."""
    if values == "01":
        a = synth.single_er(24, 0.3, 8, values="01")
    else:
        g = np.random.default_rng(9)
        a = synth.single_er(16, 0.3, 9, values="01") * g.integers(-40, 41, size=(16, 16))
        np.fill_diagonal(a, 100)
    K = 8
    top = (1 << (a.shape[0] - 1)) >> K
    _, kind = check(a, K, [0, 1, top // 5, top - 1])
    assert kind >= 2 and (kind & 1) == (1 if values == "01" else 0)


def test_exact_at_48_slots_with_zero_skips():
    """Exact walks at 48 slots: the n = 44 band |i-j| <= 2 plus one off-band
    nonzero per row, and a sparse 0/1 matrix (n = 40, p = 0.04) whose blocks
    are often all-zero, so the compact walk's single-block skip fires."""
    a = synth.band_plus(44, 2, 1, seed=4, values="01")
    K = 9
    top = (1 << 43) >> K
    check(a, K, [0, top // 3, top - 1])
    b = synth.single_er(40, 0.04, 11, values="01")
    top = (1 << 39) >> K
    skips, _ = check(b, K, [0, 1, top // 2, top - 1])
    assert sum(skips.values()) > 0


def test_double_double_meets_a_bound_fp64_cannot():
    """The upper-triangular closed form (perm = product of the diagonal) is
    ill-conditioned: sum|terms| / |perm| is about 10^10 at n = 24.  The
    double-double walk's chunk sums agree with the long-double oracle to
    2^-60 n sum|terms| (the oracle's own precision on x86 is 2^-64)."""
    n = 24
    g = np.random.default_rng(12)
    a = np.triu(g.random((n, n)) + 0.5)
    K = 10
    top = (1 << (n - 1)) >> K
    _, kind = check(a, K, [0, 1, top // 2, top - 1], tol=n * 2.0 ** -60, precision=A.PERM_PREC_DD)
    assert kind == 1


def test_zero_spans_of_the_two_state_walk():
    """A sparse 0/1 matrix walked in FP64 by the two-state generic walk, whose
    zero skips widen into zero spans: with the skip on and off the chunk sums
    agree with the oracle."""
    a = synth.single_er(28, 0.1, 3, values="01").astype(np.float64)
    K = 12
    top = (1 << 27) >> K
    chunks = [0, 1, 5, top // 3, top - 1]
    skips, kind = check(a, K, chunks)
    assert kind == 0 and sum(skips.values()) > 0
    skips, _ = check(a, K, chunks, zero_skip=0)
    assert sum(skips.values()) == 0
