"""Exact permanents of float64 matrices in Python integers -- TEST INFRASTRUCTURE ONLY.

A float64 entry is a dyadic rational, so a whole matrix becomes an integer matrix
times 2^-s for one s, and every sum below is carried out in exact integers; the result
is a ``fractions.Fraction``.  Slow (Python big integers); used to write stored
expected values (``tests/golden/make_golden.py``) where long-double accumulation of a
heavily cancelling sum would limit the truth itself.
"""
from __future__ import annotations

import math
from fractions import Fraction
from itertools import permutations

import numpy as np


def to_integer_matrix(A):
    """(Z, s) with A == Z * 2^-s exactly, Z a list of lists of Python ints."""
    A = np.asarray(A, dtype=np.float64)
    if not np.all(np.isfinite(A)):
        raise ValueError("non-finite entry")
    s = 0
    for x in A.ravel():
        num, den = float(x).as_integer_ratio()
        s = max(s, den.bit_length() - 1)  # den is a power of two
    Z = [[int(Fraction(float(x)) * (1 << s)) for x in row] for row in A]
    return Z, s


def definition(A):
    """Sum over the injective maps rows -> columns of the products (Eq.
    rectangular_permanent_definition), exactly; tiny matrices only.  Real input gives
    a Fraction, complex input a pair (re, im) of Fractions."""
    A = np.asarray(A)
    if A.shape[0] > A.shape[1]:
        A = A.T
    if A.dtype.kind == "c":
        m, n = A.shape
        R, s = to_integer_matrix(np.concatenate([A.real, A.imag], axis=0))
        re, im = R[:m], R[m:]
        tr, ti = 0, 0
        for sigma in permutations(range(n), m):
            pr, pi = 1, 0
            for i in range(m):
                ar, ai = re[i][sigma[i]], im[i][sigma[i]]
                pr, pi = pr * ar - pi * ai, pr * ai + pi * ar
            tr += pr
            ti += pi
        den = 1 << (s * m)
        return Fraction(tr, den), Fraction(ti, den)
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    Z, s = to_integer_matrix(A)
    total = 0
    for sigma in permutations(range(n), m):
        p = 1
        for i in range(m):
            p *= Z[i][sigma[i]]
        total += p
    return Fraction(total, 1 << (s * m))


def _grouped_range(Z, m, n, s, d0, d1) -> int:
    """Integer numerator of the grouped sum below over the sign vectors d0 <= d < d1."""
    k = n - m
    one = 1 << s  # the padding entries 1, on the scale of Z
    weights = [math.comb(k, t) for t in range(k + 1)]
    total = 0
    for d in range(d0, d1):
        signs = [1] + [(-1 if (d >> (m - 2 - i)) & 1 else 1) for i in range(m - 1)]
        c = [sum(signs[i] * Z[i][j] for i in range(m)) for j in range(n)]
        inner = 0
        for t in range(k + 1):
            shift = (k - 2 * t) * one
            p = 1
            for j in range(n):
                p *= c[j] + shift
            inner += -weights[t] * p if t & 1 else weights[t] * p
        if sum(1 for x in signs if x < 0) & 1:
            inner = -inner
        total += inner
    return total


def _grouped_task(args):
    return _grouped_range(*args)


def glynn_rect_grouped(A, workers: int = 1) -> Fraction:
    """Eq. glynn_rectangle with the n - m padding rows of ones grouped by their number t
    of -1 signs, in exact integers:
        per(A) = 1 / (2^(n-1) (n-m)!) sum over delta in {+-1}^m, delta_0 = +1, of
                 (prod_i delta_i) sum_t (-1)^t C(n-m, t) prod_j (c_j + (n-m-2t)),
    c_j = sum_i delta_i a_ij (the same grouping as the long-double oracle function of
    that name, with no rounding anywhere).  `workers` > 1 splits the sign vectors over
    that many processes (spawned)."""
    A = np.asarray(A, dtype=np.float64)
    if A.shape[0] > A.shape[1]:
        A = A.T
    m, n = A.shape
    if m == 0:
        return Fraction(1)
    Z, s = to_integer_matrix(A)
    D = 1 << (m - 1)
    if workers <= 1:
        total = _grouped_range(Z, m, n, s, 0, D)
    else:
        import multiprocessing
        parts = max(1, min(D, 8 * workers))
        cuts = [D * p // parts for p in range(parts + 1)]
        tasks = [(Z, m, n, s, cuts[p], cuts[p + 1]) for p in range(parts)]
        with multiprocessing.get_context("spawn").Pool(workers) as pool:
            total = sum(pool.map(_grouped_task, tasks))
    return Fraction(total, (1 << (s * n)) * (1 << (n - 1)) * math.factorial(n - m))
