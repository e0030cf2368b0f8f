"""Writes the stored expected values under tests/golden/ by calling the CPU
oracle only (never the CUDA path).

    python tests/golden/make_golden.py [--threads T]

er36_f64_perm.txt: the n=36 ER (p=0.15, forced diagonal, (0,1] values, shuffled
columns, seed 2) matrix's permanent by Algorithm 1 in long double over the
full 2^35 Gray range, with the sum of |terms| (its conditioning).  Takes a few
minutes on 8 x86-64 cores (80-bit long double there; 64-bit significand).
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2501_15126_gb300 import synth  # noqa: E402


def main():
    threads = 8
    if "--threads" in sys.argv:
        threads = int(sys.argv[sys.argv.index("--threads") + 1])
    a = synth.single_er(36, 0.15, 2, values="f64", shuffle_cols=True)
    t0 = time.time()
    perm, absum = oracle.nw_perm(a, threads=threads)
    dt = time.time() - t0
    with open(os.path.join(HERE, "er36_f64_perm.txt"), "w") as f:
        f.write("# n=36 ER p=0.15 + diagonal, (0,1] values, shuffled columns, seed 2 (synth.single_er)\n")
        f.write("# oracle.nw_perm: Algorithm 1 in long double (%d-bit significand), %d threads, %.0f s\n"
                % (oracle.long_double_bits(), threads, dt))
        f.write("perm_hi %r\nperm_lo %r\nabs_terms %r\n" % (perm.hi, perm.lo, float(absum)))
    print(perm, absum, dt)


if __name__ == "__main__":
    main()
