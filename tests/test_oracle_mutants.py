"""The oracle's pins catch plausible mistakes: each case plants one mistake in a
temporary copy of the oracle's C source -- a dropped term, a wrong sign, a wrong row
per Gray-code bit, a wrong binomial weight or normalisation, an off-by-one range, a
missing absolute value, a conjugated entry, a transposed matrix -- in the C source or
in the Python modules (scales, int128 decoding, the exact and rational oracles, the
cost model's reference perceptron),
builds the copy with gcc, and runs the pin tests (test_oracle_pins.py,
test_oracle_mlp.py) against it in a separate process.  Every mutant must make a pin fail; the unmodified copy must pass
them all.  Nothing outside the temporary directory is changed."""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")
PINS = [os.path.join(ROOT, "tests", f) for f in ("test_oracle_pins.py", "test_oracle_mlp.py")]
INC, C = "oracle_real.inc", "perm_oracle.c"
PY, EXACT, CAUCHY, MLP = "__init__.py", "exact.py", "cauchy.py", "mlp_ref.py"

# (name, file, text, replacement): the first occurrence of `text` is replaced
MUTANTS = [
    ("definition drops the maps with sigma(0) = n - 1", INC,
     "    if (used[j]) continue;\n    used[j] = 1;\n    sigma[i] = j;\n    SFX(def_rec_r)",
     "    if (used[j] || (i == 0 && j == n - 1)) continue;\n    used[j] = 1;\n    sigma[i] = j;\n    SFX(def_rec_r)"),
    ("definition with a determinant-like sign", INC, "    *acc += p;", "    *acc += (sigma[0] & 1) ? -p : p;"),
    ("Glynn sign not alternated", INC,
     "    sign = -sign;\n    delta[bound - pos] = -delta[bound - pos];\n    acc += sign * SFX(glynn_term_r)",
     "    sign = +sign;\n    delta[bound - pos] = -delta[bound - pos];\n    acc += sign * SFX(glynn_term_r)"),
    ("Glynn divided by 2^n", INC, "for (int i = 0; i < bound; ++i) norm *= 2;",
     "for (int i = 0; i <= bound; ++i) norm *= 2;"),
    ("Glynn padding rows without their signs", INC, "for (int k = m; k < n; ++k) sum += (REAL)delta[k];",
     "for (int k = m; k < n; ++k) sum += (REAL)1;"),
    ("Glynn without the (n - m)! normalisation", INC,
     "  for (int i = 2; i <= n - m; ++i) norm *= (REAL)i;\n  SFX(put_real)(acc / norm, out);",
     "  SFX(put_real)(acc / norm, out);"),
    ("Glynn partial sums: Gray bit b on row b", INC,
     "delta[i] = ((gray >> (n - 1 - i)) & 1u) ? -1 : 1;\n    REAL t = SFX(glynn_term_r)",
     "delta[i] = ((gray >> i) & 1u) ? -1 : 1;\n    REAL t = SFX(glynn_term_r)"),
    ("Glynn partial sums include their end", INC,
     "  for (uint64_t g = g0; g < g1; ++g) {\n    uint64_t gray = g ^ (g >> 1);\n    for (int i = 0; i < n; ++i) "
     "delta[i] = ((gray >> (n - 1 - i)) & 1u) ? -1 : 1;\n    REAL t = SFX(glynn_term_r)(m, n, A, ld, delta);\n"
     "    if (g & 1u)",
     "  for (uint64_t g = g0; g <= g1; ++g) {\n    uint64_t gray = g ^ (g >> 1);\n    for (int i = 0; i < n; ++i) "
     "delta[i] = ((gray >> (n - 1 - i)) & 1u) ? -1 : 1;\n    REAL t = SFX(glynn_term_r)(m, n, A, ld, delta);\n"
     "    if (g & 1u)"),
    ("sum of |term| without the absolute value", INC, "    acc += (t < 0) ? -t : t;", "    acc += t;"),
    ("grouped Glynn: padding shift k - t", INC, "prod *= colsum[j] + (REAL)(k - 2 * t);",
     "prod *= colsum[j] + (REAL)(k - t);"),
    ("grouped Glynn without the binomial weight", INC, "const REAL w = (REAL)binomial_u64(k, t);",
     "const REAL w = 1;"),
    ("e_m recurrence run upwards", INC, "for (int s = m; s >= 1; --s) e[s] += c * e[s - 1];",
     "for (int s = 1; s <= m; ++s) e[s] += c * e[s - 1];"),
    ("square Ryser without the final sign", INC, "  if (m & 1) acc = -acc;\n  SFX(put_real)(acc, out);",
     "  SFX(put_real)(acc, out);"),
    ("Ryser subset weight signed by n - s", INC, "if ((m - s) & 1) w = -w;", "if ((n - s) & 1) w = -w;"),
    ("Ryser subset weight C(n - m, m - s)", INC,
     "REAL w = (REAL)binomial_u64(n - s, m - s);\n    if ((m - s) & 1)",
     "REAL w = (REAL)binomial_u64(n - m, m - s);\n    if ((m - s) & 1)"),
    ("rectangular Ryser weight C(n - m + k, m - k)", INC, "REAL bin = (REAL)binomial_u64(n - m + k, k);",
     "REAL bin = (REAL)binomial_u64(n - m + k, m - k);"),
    ("rectangular Ryser sign not alternated", INC,
     "    acc += permsum;\n    sign = -sign;\n  }\n  SFX(put_real)(acc, out);",
     "    acc += permsum;\n  }\n  SFX(put_real)(acc, out);"),
    ("complex Glynn on conjugated entries", INC, "sum += SFX(elem_c)(A, ld, i, j) * (REAL)delta[i];",
     "sum += (creall(SFX(elem_c)(A, ld, i, j)) - cimagl(SFX(elem_c)(A, ld, i, j)) * (SFX(cplx_t))I) * "
     "(REAL)delta[i];"),
    ("exact Glynn padding rows without their signs", C, "for (int k = m; k < n; ++k) sum += delta[k];",
     "for (int k = m; k < n; ++k) sum += 1;"),
    ("exact Glynn without the (n - m)! normalisation", C,
     "  for (int i = 2; i <= n - m; ++i) norm *= i;\n  put_i128((u128)(v / norm), out);",
     "  put_i128((u128)(v / norm), out);"),
    ("Gaussian-integer product with a wrong sign", C, "r.re = a.re * b.re - a.im * b.im;",
     "r.re = a.re * b.re + a.im * b.im;"),
    ("exact square Ryser with the subset signs swapped", C,
     "if (__builtin_popcountll(k) & 1) acc -= rowsumprod; else acc += rowsumprod;",
     "if (__builtin_popcountll(k) & 1) acc += rowsumprod; else acc -= rowsumprod;"),
    ("subset DP stops one size short", C, "    if (r > m) continue;", "    if (r >= m) continue;"),
    ("exact definition drops the maps with sigma(0) = 0", C,
     "    if (used[j]) continue;\n    used[j] = 1;\n    sigma[i] = j;\n    def_rec_i(",
     "    if (used[j] || (i == 0 && j == 0)) continue;\n    used[j] = 1;\n    sigma[i] = j;\n    def_rec_i("),
    # the Python side: normalisations, the int128 decoding, the exact and rational oracles
    ("sum of |term| scale divided by 2^n", PY, "return s / (2.0 ** (n - 1)) /", "return s / (2.0 ** n) /"),
    ("closed-form scale divided by 2^m", PY, "/ 2.0 ** (m - 1)", "/ 2.0 ** m"),
    ("int128 results read without their sign", PY, "return v - (1 << 128) if v >> 127 else v", "return v"),
    ("per(|A|) of the real parts", PY, "A = np.abs(np.asarray(A)).astype(np.float64)",
     "A = np.real(np.asarray(A)).astype(np.float64)"),
    ("SBP selection matrix transposed", PY, "            P[j, k] = 1\n", "            P[k, j] = 1\n"),
    ("exact complex definition with a wrong product sign", EXACT,
     "pr, pi = pr * ar - pi * ai, pr * ai + pi * ar", "pr, pi = pr * ar + pi * ai, pr * ai + pi * ar"),
    ("exact grouped Glynn: padding shift off its scale", EXACT, "shift = (k - 2 * t) * one", "shift = (k - 2 * t)"),
    ("exact determinant ignores row swaps", CAUCHY, "            d = -d\n", ""),
    ("Borchardt without the Hadamard square", CAUCHY, "CC = [[c * c for c in row] for row in C]",
     "CC = [[c for c in row] for row in C]"),
    ("Cauchy determinant closed form with a flipped factor", CAUCHY, "num *= (X[j] - X[i]) * (Y[i] - Y[j])",
     "num *= (X[j] - X[i]) * (Y[j] - Y[i])"),
    # the reference perceptron of the cost model
    ("MLP gradient without the first ReLU mask", MLP, "d1 = (d2 @ W2.T) * (z1 > 0)", "d1 = d2 @ W2.T"),
    ("MLP weight gradient transposed", MLP, "gW2 = a1.T @ d2", "gW2 = d2.T @ a1"),
    ("MLP loss without the mask normalisation", MLP, "return float(np.sum(mask * (y - T) ** 2) / np.sum(mask))",
     "return float(np.sum(mask * (y - T) ** 2))"),
    ("MLP bias added after the activation", MLP, "    z1 = X @ W1 + b1\n    a1 = np.maximum(z1, 0.0)\n",
     "    z1 = X @ W1\n    a1 = np.maximum(z1, 0.0) + b1\n"),
]

RUNNER = """
import sys
sys.path.insert(0, sys.argv[1])
import oracle
assert oracle.__file__.startswith(sys.argv[1]), oracle.__file__
oracle.build(force=True)
print("BUILT", flush=True)
import pytest
sys.exit(int(pytest.main(["-x", "-q", "-p", "no:cacheprovider"] + sys.argv[2:])))
"""


def _copy_with(tmp, mutant):
    dst = os.path.join(tmp, "oracle")
    shutil.copytree(ORACLE, dst, ignore=shutil.ignore_patterns("*.so", "__pycache__", "*.tmp*"))
    if mutant is not None:
        _, fname, old, new = mutant
        path = os.path.join(dst, fname)
        with open(path) as f:
            src = f.read()
        assert old in src, mutant[0]
        with open(path, "w") as f:
            f.write(src.replace(old, new, 1))
    return tmp


def _run(tmp):
    p = subprocess.run([sys.executable, "-c", RUNNER, tmp] + PINS, cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    return p.returncode, p.stdout + p.stderr


def test_every_planted_mistake_fails_a_pin(tmp_path):
    dirs = []
    for k, mutant in enumerate([None] + MUTANTS):
        d = str(tmp_path / ("m%02d" % k))
        os.makedirs(d)
        dirs.append(_copy_with(d, mutant))
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        results = list(ex.map(_run, dirs))
    rc, log = results[0]
    assert rc == 0, "the unmodified copy fails its pins:\n" + log[-3000:]
    survivors = []
    for mutant, (rc, log) in zip(MUTANTS, results[1:]):
        assert "BUILT" in log, (mutant[0], log[-2000:])  # the mutant compiled and loaded
        if rc != 1:  # 1: tests failed; anything else (0 passed, 2+ errors) is not a kill
            survivors.append((mutant[0], rc))
    assert not survivors, survivors
