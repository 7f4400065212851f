"""The multi-limb arithmetic of the Cauchy path (``csrc/bigfloat.cuh``), compiled for
the host and checked against exact rationals: every multiplication, addition,
subtraction and reciprocal is within 2^(2 - 64 L) relative of the exact value, as the
header states, conversions from doubles are exact and conversions to doubles round
to nearest (ties to even).  Random operands plus the edge cases of the addition
(equal magnitudes of opposite sign, exponent gaps beyond the guard limbs, carries)."""
import os
import random
import shutil
import subprocess
import struct
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2510_03421_gb300", "csrc")
LS = (2, 4, 7, 16)


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("no nvcc")
    exe = str(tmp_path_factory.mktemp("bigfloat") / "bigfloat_check")
    subprocess.check_call([nvcc, "-std=c++17", "-O1", "-x", "cu", "-I", CSRC,
                           os.path.join(ROOT, "tests", "bigfloat_check.cu"), "-o", exe])
    return exe


def value(s, e, limbs):
    L = len(limbs)
    m = 0
    for v in limbs:
        m = (m << 64) | v
    q = Fraction(m, 1 << (64 * L)) * (Fraction(2) ** e)
    return -q if s else q


def rand_big(g, L, emin=-300, emax=300):
    limbs = [g.getrandbits(64) for _ in range(L)]
    limbs[0] |= 1 << 63
    return (g.getrandbits(1), g.randint(emin, emax), limbs)


def fmt(b):
    s, e, limbs = b
    return "%d %d %s" % (s, e, " ".join("%x" % v for v in limbs))


def run(exe, lines):
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    return out.stdout.strip().splitlines()


def parse(line):
    f = line.split()
    s, e, z = int(f[0]), int(f[1]), int(f[2])
    limbs = [int(v, 16) for v in f[3:]]
    return s, e, z, limbs


def check_result(line, exact, L):
    s, e, z, limbs = parse(line)
    if exact == 0:
        assert z == 1 and all(v == 0 for v in limbs)
        return
    assert z == 0 and limbs[0] >> 63 == 1  # normalised
    got = value(s, e, limbs)
    assert abs(got - exact) <= Fraction(4, 1 << (64 * L)) * abs(exact), (float(got), float(exact))


@pytest.mark.parametrize("L", LS)
def test_mul_add_sub_recip_within_the_stated_bound(checker, L):
    g = random.Random(4000 + L)
    cases = []
    for _ in range(150):
        a, b = rand_big(g, L), rand_big(g, L)
        cases += [("mul", a, b), ("add", a, b), ("sub", a, b), ("recip", a, None)]
    # addition edge cases: same exponent, opposite signs (deep cancellation); equal
    # magnitudes (zero); gaps up to and beyond the two guard limbs; carry out of the top
    for _ in range(60):
        a = rand_big(g, L)
        b = (1 - a[0], a[1], list(a[2]))
        b[2][-1] ^= 1 << g.randint(0, 63)
        cases.append(("add", a, b))
        cases.append(("add", a, (1 - a[0], a[1], list(a[2]))))
        gap = g.choice([1, 63, 64, 65, 64 * L, 64 * (L + 2) - 1, 64 * (L + 2), 64 * (L + 3)])
        cases.append(("add", a, (g.getrandbits(1), a[1] - gap, rand_big(g, L)[2])))
        cases.append(("add", (0, a[1], [(1 << 64) - 1] * L), (0, a[1], [(1 << 64) - 1] * L)))
    lines = ["%s %d %s%s" % (op, L, fmt(a), "" if b is None else " " + fmt(b)) for op, a, b in cases]
    for (op, a, b), line in zip(cases, run(checker, lines)):
        va = value(*a)
        vb = None if b is None else value(*b)
        exact = {"mul": lambda: va * vb, "add": lambda: va + vb, "sub": lambda: va - vb,
                 "recip": lambda: 1 / va}[op]()
        check_result(line, exact, L)


@pytest.mark.parametrize("L", LS)
def test_double_conversions(checker, L):
    g = random.Random(4100 + L)
    doubles = [0.0, 1.0, -1.0, 5e-324, -2.2250738585072014e-308, 1.7976931348623157e308, 0.1, -3.75]
    doubles += [struct.unpack("<d", struct.pack("<Q", g.getrandbits(63) & ~(0x7ff << 52) | (g.randint(1, 2046) << 52)))[0]
                for _ in range(100)]
    bits = [struct.unpack("<Q", struct.pack("<d", d))[0] for d in doubles]
    out = run(checker, ["d2b %d %x" % (L, b) for b in bits])
    for d, line in zip(doubles, out):
        s, e, z, limbs = parse(line)
        assert (z == 1 and d == 0.0) or value(s, e, limbs) == Fraction(d)
    # to the nearest double, ties to even: random values, and exact halfway cases
    bigs = [rand_big(g, L, -900, 900) for _ in range(100)]
    for _ in range(20):
        m = (g.getrandbits(52) | (1 << 52)) << 11 | (1 << 10)  # 53 bits, then exactly one half
        bigs.append((g.getrandbits(1), g.randint(-100, 100), [m] + [0] * (L - 1)))
    out = run(checker, ["b2d %d %s" % (L, fmt(b)) for b in bigs])
    for b, line in zip(bigs, out):
        got = struct.unpack("<d", struct.pack("<Q", int(line, 16)))[0]
        assert got == float(value(*b))
