"""Reproducer: one generated exact kernel, three register budgets.

The 128-bit walk of -J_15 with one ring product per row (PERM_CODEGEN_NO_FOLD=1),
generated once and built by NVRTC for 3, 2 and 1 resident 256-thread blocks
per SM (80, 128 and 255 registers; PERM_CODEGEN_MIN_BLOCKS fixes the budget and
turns off the library's own guard).  perm(-J_15) = -15! = -1307674368000.  On
the GB300 with CUDA 13.0 the 128-register build (about 1.4 KB of spills) gives a
wrong top limb at every chunk length; the other two are right.  The same source
compiled as host C++ under ASan/UBSan matches the CPU oracle chunk by chunk
(tests/test_codegen_host_emulation.py).  The library's default budget never
runs that build (see the cross-check in csrc/codegen.cpp).

    python tests/reproducers/spilled_ring_walk.py        (needs a GPU)
"""
import math
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
os.environ["PERM_CODEGEN_NO_FOLD"] = "1"

from paper_2501_15126_gb300 import _abi as A  # noqa: E402
from paper_2501_15126_gb300 import synth  # noqa: E402


def main():
    a = -synth.ones(15)
    want = -math.factorial(15)
    for blocks in ("3", "2", "1"):
        os.environ["PERM_CODEGEN_MIN_BLOCKS"] = blocks
        for K in (0, 8, 10):
            r = A.permanent(a, engine=A.PERM_ENGINE_CODEGEN, exact_words=2, chunk_log2=K,
                            flags=A.PERM_FLAG_NO_KERNEL_CACHE)
            print("blocks/SM %s  registers %3d  K %2d  %s  %d" % (blocks, r.regs_per_thread, K,
                                                                 "ok   " if r.value == want else "WRONG", r.value))


if __name__ == "__main__":
    main()
