"""GPU parity of the ablation baselines (Sec. VI-B, Table III): CodeGen-PureReg
(generated kernel, x in registers, the product of all n rows every step) and
GPU-SparsePerman (x in shared memory, CSC columns, zero tracking, a full
product every step), against the oracle.  They walk the same Gray chunks as the
fast path, so any difference is rounding: FP64 within 64 n 2^-53 of the sum
of |terms|, exact results bit-identical."""
import numpy as np
import pytest

import oracle
from paper_2501_15126_gb300 import _abi as A
from paper_2501_15126_gb300 import synth

pytestmark = pytest.mark.gpu
U = 2.0 ** -53
PURE = dict(engine=A.PERM_ENGINE_CODEGEN, flags=A.PERM_FLAG_PURE_REG | A.PERM_FLAG_ABS_SUM)
XSH = dict(engine=A.PERM_ENGINE_XSHARED)


@pytest.mark.parametrize("n", [2, 5, 9, 14, 19, 23])
def test_pure_reg_and_x_shared_match_the_oracle(n):
    a = synth.single_er(n, 0.35, 300 + n, values="f64")
    want, sa = oracle.nw_perm(a, threads=8)
    want, sa = float(want), float(sa)
    for kw in (PURE, XSH):
        r = A.permanent(a, precision=A.PERM_PREC_F64, **kw)
        assert r.engine == kw["engine"] or n <= 8          # tiny matrices take the direct kernel
        assert abs(r.value - want) <= 64 * n * U * sa, (kw, r.value, want)
        assert abs(r.abs_term_sum - sa) <= 1e-4 * sa
    if n >= 3:
        a01 = synth.single_er(n, 0.35, 400 + n, values="01")
        assert A.permanent(a01, **PURE).value == oracle.ryser_gray(a01)


def test_x_shared_zero_tracking_and_subranges_at_full_size():
    """The n=36 workload: 2^20-step sub-ranges with high Gray bits set, both
    baselines against the oracle's partial sums; a 0/1 matrix walked in FP64
    by the shared-memory kernel skips the steps whose x has a zero entry."""
    a = synth.single_er(36, 0.15, 2, values="f64", shuffle_cols=True)
    ins = A.inspect(a, ordering=A.PERM_ORDER_DEGREE)
    ao = np.ascontiguousarray(a[:, list(ins.col_order)[:36]])
    for lo in (0, (1 << 34) + (5 << 26)):
        hi = lo + (1 << 20)
        s, sa = oracle.nw_range(ao, lo, hi, threads=16)
        for kw in (PURE, XSH):
            r = A.permanent(a, g_lo=lo, g_hi=hi, ordering=A.PERM_ORDER_DEGREE, **kw)
            assert abs(r.value - float(s)) <= 64 * 36 * U * float(sa), kw
    b = synth.band_plus(20, 1, 0, seed=1, values="01").astype(np.float64)
    r = A.permanent(b, precision=A.PERM_PREC_F64, **XSH)
    assert r.value == float(oracle.band_dp_int(b.astype(np.int64), 1))
    assert r.zero_skip_frac > 0.5
