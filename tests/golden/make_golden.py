"""Write the stored expected values used by the GPU parity tests.

Every value here comes from the CPU oracle (``oracle/``) alone, on inputs drawn by
``paper_2510_03421_gb300.inputs``; nothing is taken from the CUDA path.

    python tests/golden/make_golden.py            # all but the Cauchy values
    python tests/golden/make_golden.py cauchy     # the Cauchy values (about 15 minutes)
"""
import os
import sys
import time
from fractions import Fraction

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
    # the same grouped sum in exact integers (oracle.exact): the long-double value
    # above is limited by its own rounding of a sum that cancels 10^7-fold
    from oracle import exact
    t2 = time.time()
    ex = exact.glynn_rect_grouped(A, workers=os.cpu_count() or 1)
    t3 = time.time()
    exd = float(ex)
    exlo = float(ex - Fraction(exd))
    assert abs(exd - (g[0] + g[1])) <= (n + 4) * 2.0 ** -(oracle.ldbl_mant_dig() - 1) * s / norm
    esym = oracle.glynn_esym_abs(A)
    write("rect20x40_f64.txt", [
        "# 20 x 40 float64 uniform[0,1] from inputs.rect20x40_f64() (seed %d)." % (inputs.SEED_BASE + 3),
        "# Oracle Glynn with the 20 padding rows grouped by their number of -1 signs (Eq. glynn_rectangle),",
        "# long double (LDBL_MANT_DIG = %d), %.1f s; as double-double hi lo.  sum_abs is the sum of |term|" % (
            oracle.ldbl_mant_dig(), t1 - t0),
        "# over all 2^39 terms, unnormalised (the scale of any evaluation's rounding error).",
        "# exact: the same sum in exact integers (oracle.exact, %.0f s), rounded to a double-double hi lo." % (t3 - t2),
        "# esym_abs: sum over the 2^19 real-row sign vectors of e_20(|c|) / 2^19, the scale of the closed-form",
        "# padding sum (oracle.glynn_esym_abs).",
        "seed %d" % (inputs.SEED_BASE + 3),
        "glynn %r %r" % g,
        "sum_abs %r" % s,
        "exact %r %r" % (exd, exlo),
        "esym_abs %r" % esym,
    ])


def cauchy_exact():
    # Cauchy matrices c_ij = 1 / (x_i - y_j) with the points of inputs.cauchy_points;
    # exact rational permanents by Borchardt's theorem (oracle.cauchy), rounded to double
    cases = [(24, 10, 1, [0]), (32, 11, 1, [0]), (40, 12, 1, [0]), (48, 13, 1, [0]), (64, 14, 1, [0]),
             (36, 15, 1216, [0, 1, 608, 1215])]
    lines = [
        "# Exact permanents of Cauchy matrices c_ij = 1 / (x_i - y_j), Eq. caucy_permanent, evaluated",
        "# in rationals by oracle.cauchy.permanent_borchardt and rounded to double.  Matrix `index` of",
        "# inputs.cauchy_points(n, seed, count=count): x ~ U[0.25, 0.75], y ~ U[-0.75, -0.25].",
    ]
    for n, off, count, idx in cases:
        seed = inputs.SEED_BASE + off
        x, y = inputs.cauchy_points(n, seed, count=count)
        for b in idx:
            t0 = time.time()
            v = oracle.cauchy.permanent_borchardt(x[b], y[b])
            lines.append("n %d seed %d count %d index %d per %r" % (n, seed, count, b, float(v)))
            print(lines[-1], "%.1f s" % (time.time() - t0), flush=True)
    write("cauchy_exact.txt", lines)


if __name__ == "__main__":
    if sys.argv[1:] == ["cauchy"]:
        cauchy_exact()
        sys.exit(0)
    if sys.argv[1:] == ["rect"]:
        rect20x40_f64()
        sys.exit(0)
    square16_f64()
    square26_01()
    rect20x40_f64()
