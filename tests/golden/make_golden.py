"""Write the stored expected values used by the GPU parity tests.

Every value here comes from the CPU oracle (``oracle/``) alone, on inputs drawn by
``paper_2510_03421_gb300.inputs``; nothing is taken from the CUDA path.

    python tests/golden/make_golden.py
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2510_03421_gb300 import inputs  # noqa: E402


def write(name, lines):
    with open(os.path.join(HERE, name), "w") as f:
        f.write("\n".join(lines) + "\n")


def square26_01():
    A = inputs.square26_01().astype(np.int64)
    t0 = time.time()
    dp = oracle.subset_dp(A)
    t1 = time.time()
    gl = oracle.glynn(A)
    t2 = time.time()
    assert dp == gl, (dp, gl)
    write("square26_01.txt", [
        "# 26 x 26 0/1 matrix, Bernoulli(0.5) entries from inputs.square26_01() (seed %d)." % (inputs.SEED_BASE + 3),
        "# Exact permanent from the oracle's subset DP (%.1f s) and exact 128-bit Glynn (%.1f s), which agree." % (
            t1 - t0, t2 - t1),
        "seed %d" % (inputs.SEED_BASE + 3),
        "per %d" % dp,
    ])


def square16_f64():
    A = inputs.square16_f64()
    g = oracle.glynn(A, dd=True)
    r = oracle.ryser(A, dd=True)
    write("square16_f64.txt", [
        "# 16 x 16 float64 uniform[-1,1] from inputs.square16_f64() (seed %d)." % (inputs.SEED_BASE + 1),
        "# Oracle Glynn and Ryser in long double (LDBL_MANT_DIG = %d), as double-double hi lo." % oracle.ldbl_mant_dig(),
        "seed %d" % (inputs.SEED_BASE + 1),
        "glynn %r %r" % g,
        "ryser %r %r" % r,
    ])


if __name__ == "__main__":
    square16_f64()
    square26_01()
