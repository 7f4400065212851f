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


def rect20x40_f64():
    A = inputs.rect20x40_f64()
    t0 = time.time()
    g = oracle.glynn_rect_grouped(A, dd=True)
    t1 = time.time()
    s = oracle.glynn_rect_grouped_abs(A)
    g64 = oracle.glynn_rect_grouped(A, prec="f64")
    # the double-precision evaluation of the same sum must agree within its own
    # first-order rounding bound (n + 4 + 2^(m-1) (n-m+1)) u sum|t| / (2^(n-1) (n-m)!)
    m, n = A.shape
    norm = 2.0 ** (n - 1) * float(np.prod(np.arange(1, n - m + 1, dtype=np.float64)))
    bound = (n + 4 + 2.0 ** (m - 1) * (n - m + 1)) * 2.0 ** -53 * s / norm
    assert abs(g64 - (g[0] + g[1])) <= bound, (g64, g, bound)
    write("rect20x40_f64.txt", [
        "# 20 x 40 float64 uniform[0,1] from inputs.rect20x40_f64() (seed %d)." % (inputs.SEED_BASE + 3),
        "# Oracle Glynn with the 20 padding rows grouped by their number of -1 signs (Eq. glynn_rectangle),",
        "# long double (LDBL_MANT_DIG = %d), %.1f s; as double-double hi lo.  sum_abs is the sum of |term|" % (
            oracle.ldbl_mant_dig(), t1 - t0),
        "# over all 2^39 terms, unnormalised (the scale of any evaluation's rounding error).",
        "seed %d" % (inputs.SEED_BASE + 3),
        "glynn %r %r" % g,
        "sum_abs %r" % s,
    ])


if __name__ == "__main__":
    square16_f64()
    square26_01()
    rect20x40_f64()
