"""Host emulation of generated kernels: the CUDA C++ that the code generator
emits for a matrix (with core.cuh) is compiled as plain host C++ under
AddressSanitizer and UndefinedBehaviorSanitizer, and each 2^K-step chunk of the
Gray walk is run as one lane (warp votes and shuffles reduce to the lane's own
value).  Every chunk's partial sum is compared with the oracle's sum over the
same Gray range (Algorithm 1 with doubled x, modulo the kernel's ring; or in
long double for FP64).  It is built twice, with automatic variables
initialised to zero and to a byte pattern: a read of an uninitialised value
that mattered would make the two disagree.  This pins the generated code's
logic and its freedom from undefined behaviour independently of any GPU
compiler (test infrastructure; no GPU needed)."""
import os
import re
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
alignas(16) unsigned char perm_xs[16];   // the kernel's dynamic shared memory (unused: the harness sets pol.xs)
#include "walk.cu"
#include <cstdio>
#include <cstdlib>
int main(int argc, char **argv) {
    const int K = std::atoi(argv[1]);
    static pk::GenPol::X xg[64], xs[64 * 256];
    pk::GenPol pol;
    pol.xg = xg;
    pol.stride = 1;
    pol.xs = xs;
    unsigned long long q;
    while (std::scanf("%llu", &q) == 1) {
        unsigned long long skipped = 0, w[6] = {0, 0, 0, 0, 0, 0};
        const auto acc = pk::walk_chunk<pk::GenPol, pk::A, PERM_TEST_B>(pol, q, K, 1, skipped);
        pk::A::acc_store(w, acc);
        std::printf("%llu", q);
        for (int i = 0; i < pk::A::ACC_WORDS; ++i) std::printf(" %016llx", w[i]);
        std::printf("\n");
    }
    return 0;
}
'''


def emulate(source, K, chunks, init):
    """Compiles the generated source with the harness (sanitizers on) and runs
    the given chunks; returns {q: [words]}."""
    with tempfile.TemporaryDirectory() as d:
        open(os.path.join(d, "walk.cu"), "w").write(source)
        open(os.path.join(d, "main.cpp"), "w").write(HARNESS)
        exe = os.path.join(d, "walk")
        B = int(re.search(r" B=(\d+)", source).group(1))   # the kernel's unrolled block, log2
        subprocess.check_call(["g++", "-std=c++17", "-O1", "-g", "-fsanitize=address,undefined",
                               "-fno-sanitize-recover=all", "-ftrivial-auto-var-init=" + init,
                               "-DPERM_TEST_B=%d" % B,
                               "-I", os.path.join(HERE, "host_emulation"), "-I", CSRC, "-I", d,
                               os.path.join(d, "main.cpp"), "-o", exe])
        out = subprocess.run([exe, str(K)], input=" ".join(map(str, chunks)), capture_output=True, text=True,
                             check=True).stdout
    res = {}
    for line in out.splitlines():
        f = line.split()
        res[int(f[0])] = [int(x, 16) for x in f[1:]]
    return res


def plan_order(a, **kw):
    ins = A.inspect(a, **{k: v for k, v in kw.items() if k == "ordering"})
    return np.ascontiguousarray(a[:, list(ins.col_order)[: a.shape[0]]])


def ring_limbs(source):
    m = re.search(r"typedef ArithExact<(\d+)> A;", source)
    return int(m.group(1)) if m else 0


def check_exact(a, K, chunks, **kw):
    src = A.codegen_source(a, engine=A.PERM_ENGINE_CODEGEN, **kw)
    limbs = ring_limbs(src)
    mask = (1 << min(128, 32 * limbs)) - 1   # the oracle is exact modulo 2^128
    ao = plan_order(a, **kw)
    got = {init: emulate(src, K, chunks, init) for init in ("zero", "pattern")}
    for q in chunks:
        want = oracle.nw2_range(ao, q << K, (q + 1) << K) & mask
        for init in got:
            v = sum(w << (64 * i) for i, w in enumerate(got[init][q])) & mask
            assert v == want, (init, q)


def check_f64(a, K, chunks, **kw):
    src = A.codegen_source(a, engine=A.PERM_ENGINE_CODEGEN, **kw)
    assert "typedef ArithF64 A;" in src
    ao = plan_order(a, **kw)
    n = a.shape[0]
    sh = int(re.search(r"static constexpr int abs_shift = (-?\d+);", src).group(1))
    got = {init: emulate(src, K, chunks, init) for init in ("zero", "pattern")}
    for q in chunks:
        s, sa = oracle.nw_range(ao, q << K, (q + 1) << K)
        for init in got:
            hi, lo, ab = (np.array(got[init][q], dtype=np.uint64).view(np.float64))
            assert abs(hi + lo - float(s)) <= 64 * n * U * float(sa), (init, q)
            assert abs(np.ldexp(ab, sh) - float(sa)) <= 1e-4 * float(sa), (init, q)


def test_negated_ones_in_a_128_bit_ring_with_and_without_folding(monkeypatch):
    """-J_15 with exact_words = 2 (a 128-bit ring): every chunk of the whole
    walk, with rows folded in 32 bits and with one ring product per row (the
    form that once returned a wrong top limb on the GPU when built for 128
    registers)."""
    a = -synth.ones(15)
    chunks = list(range(0, 1 << 14 >> 8))
    check_exact(a, 8, chunks, exact_words=2)
    monkeypatch.setenv("PERM_CODEGEN_NO_FOLD", "1")
    src = A.codegen_source(a, engine=A.PERM_ENGINE_CODEGEN, exact_words=2)
    assert "x[0] * x[1]" not in src
    check_exact(a, 8, chunks, exact_words=2)


def test_ones_in_a_192_bit_ring():
    """J_30 in a 192-bit ring (the kernel that spills most at 128 registers):
    chunks spread over the walk, including the last one."""
    a = synth.ones(30)
    K = 10
    last = (1 << 29 >> K) - 1
    check_exact(a, K, [0, 1, 7, 1000, 123457 % last, last // 2, last], exact_words=3)


def test_band_plus_off_band_exact_with_global_rows():
    """The n=48 band |i-j| <= 3 plus 2 off-band nonzeros per row, 0/1, with 20
    rows of x in registers and the rest in global memory (Algorithm 4's split):
    chunks with high Gray bits set."""
    a = synth.band_plus(48, 3, 2, seed=3, values="01")
    K = 9
    top = (1 << 47) >> K
    check_exact(a, K, [0, 5, top // 3, top - 1], reg_rows=20)
    check_exact(a, K, [0, top // 5, top - 1], reg_rows=20, shared_rows=12)   # three tiers


@pytest.mark.parametrize("flags", [0, 4])
def test_generated_f64_walks(flags):
    """FP64 generated kernels (two-state chains, and the paired chain with
    flags = PERM_FLAG_PAIRED_CHAIN): chunk sums within the FP64 rounding bound
    of the oracle's, and their sums of |terms| within 1e-4."""
    a = synth.single_er(24, 0.2, 1, values="f64")
    check_f64(a, 9, [0, 3, 1000, (1 << 23 >> 9) - 1], flags=flags)


@pytest.mark.parametrize("name", ["curtis54", "bcspwr02", "mycielskian6"])
def test_zero_spans_on_binary_table2_shapes(name):
    """Binary matrices with Table II's shapes, where almost every product is
    zero (Sec. VI-E): the walk skips whole aligned spans of blocks (up to a
    whole 2^12-step chunk) and applies each span's net flip (mycielskian6's
    kernel is built without spans and skips single blocks).  Every chunk's
    sum must still equal the oracle's over the same Gray range."""
    a = synth.table2_like(name)
    K = 12
    top = (1 << (a.shape[0] - 1)) >> K
    check_exact(a, K, [0, 1, 2, 3, top // 7, top // 3 + 1, top - 2, top - 1])


def test_zero_spans_on_the_d_ss_shape_in_fp64():
    """The d_ss shape (over half of the values +-1, 40 distinct): FP64 walk
    (with the sum of |terms|, which a walk of n > 32 keeps only on request),
    chunk sums within the rounding bound of the oracle's."""
    a = synth.table2_like("d_ss")
    K = 12
    top = (1 << (a.shape[0] - 1)) >> K
    check_f64(a, K, [0, 5, top // 3, top - 1], flags=A.PERM_FLAG_ABS_SUM)


def test_zero_spans_in_a_two_state_fp64_kernel():
    """A 0/1 ER matrix (n = 28, p = 0.1) walked in FP64: its generated kernel
    runs two-state chains and zero spans; chunk sums within the rounding bound
    of the oracle's."""
    a = synth.single_er(28, 0.1, 3, values="01").astype(np.float64)
    src = A.codegen_source(a, engine=A.PERM_ENGINE_CODEGEN)
    assert "kDual = true" in src and "kZeroSpans = true" in src
    K = 12
    top = (1 << 27) >> K
    check_f64(a, K, [0, 1, 5, top // 3, top - 1], flags=A.PERM_FLAG_ABS_SUM)


@pytest.mark.parametrize("values", ["01", "f64"])
def test_largest_size_n64(values):
    """n = 64, the largest size the library takes (Gray indices up to 2^63 - 1,
    a 192-bit ring on the exact path): an ER p = 0.08 + diagonal matrix, with
    chunks at the start, on both sides of bit 62 of the Gray index, and the
    very last chunk, against the oracle's sums over the same ranges."""
    a = synth.single_er(64, 0.08, 64, values=values)
    K = 12
    top = (1 << 63) >> K
    chunks = [0, 1, top // 2 - 1, top // 2, top - 2, top - 1]
    if values == "01":
        check_exact(a, K, chunks)
    else:
        check_f64(a, K, chunks, flags=A.PERM_FLAG_ABS_SUM)


def test_headline_matrix_with_x_in_three_tiers_and_pure_reg():
    """The n=36 workload (ER p = 0.15 + diagonal, (0,1], shuffled columns) in
    FP64: the two-state kernel with x split over registers, shared memory and
    global memory (18 + 8 + 10 rows: asking for 12 register rows gives the
    18 that the unrolled 2^7-step block reaches), and the CodeGen-PureReg kernel (every
    row in registers, a full product every step); chunks at the start, in the
    middle and at the end of the walk."""
    a = synth.single_er(36, 0.15, 2, values="f64", shuffle_cols=True)
    K = 12
    top = (1 << 35) >> K
    chunks = [0, 1, top // 2 + 3, top - 1]
    src = A.codegen_source(a, reg_rows=12, shared_rows=8, flags=A.PERM_FLAG_ABS_SUM)
    assert "reg_rows(k)=18 " in src and "xs[" in src and "xg[" in src
    check_f64(a, K, chunks, reg_rows=12, shared_rows=8, flags=A.PERM_FLAG_ABS_SUM)
    check_f64(a, K, chunks, flags=A.PERM_FLAG_PURE_REG | A.PERM_FLAG_ABS_SUM)
