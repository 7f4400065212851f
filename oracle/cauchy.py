"""Exact permanents of Cauchy matrices -- TEST INFRASTRUCTURE ONLY (part of ``oracle``).

A Cauchy matrix has c_ij = 1 / (x_i - y_j) (the paper's special-case paragraph on
Cauchy matrices, Eq. caucy_permanent).  Every double is a dyadic rational, so for
double inputs x and y the matrix, its determinant and its permanent are exact
rationals; this module computes them with :class:`fractions.Fraction` and nothing
else, so no rounding enters anywhere.

* :func:`cauchy_matrix` -- the exact matrix of the given doubles;
* :func:`det` -- Gaussian elimination in rationals (first nonzero pivot);
* :func:`cauchy_det_closed_form` -- Cauchy's determinant product formula, a
  textbook identity used to pin :func:`det`;
* :func:`permanent_definition` -- the definition, sum over permutations (n <= 8);
* :func:`permanent_borchardt` -- Borchardt's theorem, Eq. caucy_permanent:
  per(C) = det(C o C) / det(C), both determinants by :func:`det`.

Pins (``tests/test_oracle_pins.py``): the determinant against the closed form and
against integer matrices with known determinants; Borchardt's quotient against the
definition on small orders (the theorem itself, checked by brute force).
"""
from __future__ import annotations

import itertools
from fractions import Fraction


def _exact(v) -> Fraction:
    return Fraction(float(v))


def cauchy_matrix(x, y):
    """c_ij = 1 / (x_i - y_j) in exact rationals; x_i == y_j raises ZeroDivisionError."""
    X = [_exact(v) for v in x]
    Y = [_exact(v) for v in y]
    return [[1 / (xi - yj) for yj in Y] for xi in X]


def det(M) -> Fraction:
    """Determinant of a square matrix of rationals by Gaussian elimination, exact."""
    A = [[Fraction(v) for v in row] for row in M]
    n = len(A)
    d = Fraction(1)
    for c in range(n):
        p = next((r for r in range(c, n) if A[r][c] != 0), None)
        if p is None:
            return Fraction(0)
        if p != c:
            A[c], A[p] = A[p], A[c]
            d = -d
        d *= A[c][c]
        for r in range(c + 1, n):
            f = A[r][c] / A[c][c]
            if f:
                for k in range(c + 1, n):
                    A[r][k] -= f * A[c][k]
    return d


def cauchy_det_closed_form(x, y) -> Fraction:
    """det(C) = prod_{i<j} (x_j - x_i)(y_i - y_j) / prod_{i,j} (x_i - y_j) (Cauchy)."""
    X = [_exact(v) for v in x]
    Y = [_exact(v) for v in y]
    n = len(X)
    num = Fraction(1)
    for i in range(n):
        for j in range(i + 1, n):
            num *= (X[j] - X[i]) * (Y[i] - Y[j])
    den = Fraction(1)
    for xi in X:
        for yj in Y:
            den *= xi - yj
    return num / den


def permanent_definition(M) -> Fraction:
    """per(M) = sum over permutations s of prod_i M[i][s(i)], exact (small n only)."""
    n = len(M)
    if n > 8:
        raise ValueError("the definition is for n <= 8")
    total = Fraction(0)
    for s in itertools.permutations(range(n)):
        t = Fraction(1)
        for i in range(n):
            t *= M[i][s[i]]
        total += t
    return total


def permanent_borchardt(x, y) -> Fraction:
    """per(C) = det(C o C) / det(C) for c_ij = 1 / (x_i - y_j) (Eq. caucy_permanent),
    exact.  Needs distinct x_i, distinct y_j and x_i != y_j (det(C) != 0)."""
    C = cauchy_matrix(x, y)
    CC = [[c * c for c in row] for row in C]
    dC = det(C)
    if dC == 0:
        raise ZeroDivisionError("det(C) = 0: repeated points")
    return det(CC) / dC
