"""Pins for the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a value the
paper prints, a closed form, an invariant, or brute force on tiny inputs.  A
plausible slip anywhere in the oracle (a dropped term, a wrong sign, a wrong
Gray-code row, a transposed operand, a wrong binomial weight or normalisation)
fails at least one of them.
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2510_03421_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

INT_ALGOS = {
    "definition": oracle.definition,
    "glynn": oracle.glynn,
    "ryser": oracle.ryser,
    "ryser_rect": oracle.ryser_rect,
    "subset_dp": oracle.subset_dp,
}
FLOAT_ALGOS = {
    "definition": oracle.definition,
    "glynn": oracle.glynn,
    "ryser": oracle.ryser,
    "ryser_rect": oracle.ryser_rect,
    "glynn_rect_grouped": oracle.glynn_rect_grouped,
}


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def _read_worked_example():
    rows, per = [], None
    with open(os.path.join(GOLDEN, "worked_example_3x3.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("per"):
                per = int(line.split()[1])
            else:
                rows.append([int(x) for x in line.split()])
    return np.array(rows, dtype=np.int64), per


# ---------------------------------------------------------------- paper values
@pytest.mark.parametrize("name", sorted(INT_ALGOS))
def test_worked_example_int(name):
    A, per = _read_worked_example()
    assert INT_ALGOS[name](A) == per == 450


@pytest.mark.parametrize("name", sorted(FLOAT_ALGOS))
@pytest.mark.parametrize("prec", ["ld", "f64"])
def test_worked_example_float(name, prec):
    A, per = _read_worked_example()
    assert FLOAT_ALGOS[name](A.astype(np.float64), prec) == float(per)


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("n", range(1, 10))
@pytest.mark.parametrize("name", sorted(INT_ALGOS))
def test_all_ones_square_is_factorial(n, name):
    # precision section: the all-ones permanent is n!
    if name == "definition" and n > 8:
        pytest.skip("definition enumerates n! leaves")
    assert INT_ALGOS[name](np.ones((n, n), dtype=np.int64)) == math.factorial(n)


@pytest.mark.parametrize("m,n", [(1, 5), (2, 5), (3, 7), (4, 9), (5, 6), (2, 12), (6, 11)])
@pytest.mark.parametrize("name", sorted(INT_ALGOS))
def test_all_ones_rect(m, n, name):
    # precision section: the m x n all-ones permanent is n!/(n-m)!
    if name == "definition" and math.perm(n, m) > 2_000_000:
        pytest.skip("too many m-permutations")
    expect = math.factorial(n) // math.factorial(n - m)
    assert INT_ALGOS[name](np.ones((m, n), dtype=np.int64)) == expect
    got = FLOAT_ALGOS.get(name, oracle.glynn)(np.ones((m, n)))
    assert _rel(got, expect) < 1e-15


@pytest.mark.parametrize("m,n", [(3, 3), (4, 7), (6, 6), (5, 12), (9, 9)])
def test_identity_padded_with_zero_columns(m, n):
    # precision section: the identity (extra columns zero) has permanent 1
    A = np.zeros((m, n), dtype=np.int64)
    A[np.arange(m), np.arange(m)] = 1
    for name, f in INT_ALGOS.items():
        if name == "definition" and math.perm(n, m) > 2_000_000:
            continue
        assert f(A) == 1, name
    for name in ("glynn", "ryser", "ryser_rect"):
        assert _rel(FLOAT_ALGOS[name](A.astype(float)), 1.0) < 1e-14, name


def _derangements(n):
    d = [1, 0]
    for k in range(2, n + 1):
        d.append((k - 1) * (d[-1] + d[-2]))
    return d[n]


@pytest.mark.parametrize("n", range(1, 10))
def test_derangements(n):
    # per(J - I) counts the permutations without fixed points: D_n = (n-1)(D_{n-1} + D_{n-2})
    A = np.ones((n, n), dtype=np.int64) - np.eye(n, dtype=np.int64)
    for name, f in INT_ALGOS.items():
        if name == "definition" and n > 8:
            continue
        assert f(A) == _derangements(n), name


@pytest.mark.parametrize("n", range(1, 14))
def test_tridiagonal_ones_fibonacci(n):
    # permutations with |sigma(i) - i| <= 1 are counted by the Fibonacci number F_{n+1}
    A = np.zeros((n, n), dtype=np.int64)
    for i in range(n):
        for j in range(max(0, i - 1), min(n, i + 2)):
            A[i, j] = 1
    fib = [0, 1]
    while len(fib) < n + 3:
        fib.append(fib[-1] + fib[-2])
    for name in ("glynn", "ryser", "subset_dp"):
        assert INT_ALGOS[name](A) == fib[n + 1], name
    assert _rel(oracle.glynn(A.astype(float)), fib[n + 1]) < 1e-15


@pytest.mark.parametrize("n", [4, 7, 10])
def test_triangular_is_product_of_diagonal(n):
    g = inputs.rng(7 + n)
    A = np.triu(g.uniform(-1, 1, (n, n)))
    expect = float(np.prod(np.diag(A)))
    # the sums cancel down to prod(diag); bound the rounding by 2^n terms of size <= prod_i sum_j |a_ij|
    bound = 2.0 ** n * n * 1e-17 * float(np.prod(np.abs(A).sum(axis=1)))
    for name in ("glynn", "ryser", "ryser_rect"):
        assert abs(FLOAT_ALGOS[name](A) - expect) < max(bound, 1e-15 * abs(expect)), name
    if n <= 8:
        assert _rel(oracle.definition(A), expect) < 1e-15
    Ai = np.triu(g.integers(-5, 6, (n, n))).astype(np.int64)
    expect_i = int(np.prod([int(x) for x in np.diag(Ai)]))
    for name in ("glynn", "ryser", "subset_dp"):
        assert INT_ALGOS[name](Ai) == expect_i, name


def _elem_sym(v, m):
    # e_m(v) from the coefficients of prod (x - v_k) = sum (-1)^k e_k x^(n-k)
    c = np.poly(np.asarray(v, dtype=float))
    return (-1) ** m * c[m]


@pytest.mark.parametrize("m,n", [(3, 3), (5, 5), (3, 8), (6, 9), (10, 10)])
def test_rank_one_closed_form(m, n):
    # per(u v^T) = m! * prod(u) * e_m(v)
    g = inputs.rng(100 + 10 * m + n)
    u = g.uniform(0.5, 1.5, m)
    v = g.uniform(0.5, 1.5, n)
    A = np.outer(u, v)
    expect = math.factorial(m) * float(np.prod(u)) * _elem_sym(v, m)
    for name in ("glynn", "ryser", "glynn_rect_grouped"):
        assert _rel(FLOAT_ALGOS[name](A), expect) < 1e-12, name


def _det_fraction(M):
    M = [row[:] for row in M]
    n = len(M)
    det = Fraction(1)
    for c in range(n):
        p = next(r for r in range(c, n) if M[r][c] != 0)
        if p != c:
            M[c], M[p] = M[p], M[c]
            det = -det
        det *= M[c][c]
        for r in range(c + 1, n):
            f = M[r][c] / M[c][c]
            for k in range(c, n):
                M[r][k] -= f * M[c][k]
    return det


@pytest.mark.parametrize("n", [3, 5, 7])
def test_cauchy_borchardt_exact(n):
    # Eq. caucy_permanent: per(C) = det(C o C) / det(C) for c_ij = 1/(x_i - y_j),
    # evaluated exactly in rationals (x, y on a dyadic grid so C rounds once to double)
    g = inputs.rng(300 + n)
    x = [Fraction(int(k), 64) for k in g.choice(np.arange(16, 49), n, replace=False)]
    y = [Fraction(-int(k), 64) for k in g.choice(np.arange(16, 49), n, replace=False)]
    C = [[1 / (xi - yj) for yj in y] for xi in x]
    CC = [[c * c for c in row] for row in C]
    per_exact = _det_fraction(CC) / _det_fraction(C)
    Af = np.array([[float(c) for c in row] for row in C])
    # first-order effect of rounding C to double is bounded by n u per(|C|)
    tol = 4 * n * np.finfo(float).eps * oracle.glynn(np.abs(Af)) / abs(float(per_exact))
    for name in ("glynn", "ryser", "definition"):
        assert _rel(FLOAT_ALGOS[name](Af), float(per_exact)) < max(tol, 1e-15), name


@pytest.mark.parametrize("n", [4, 5, 6, 7])
def test_perfect_matching_count_brute_force(n):
    # the permanent of a 0/1 biadjacency matrix counts perfect matchings
    for trial in range(3):
        A = inputs.bernoulli01(n, n, 500 + 10 * n + trial, 0.6).astype(np.int64)
        count = sum(all(A[i, s[i]] for i in range(n)) for s in itertools.permutations(range(n)))
        for name, f in INT_ALGOS.items():
            assert f(A) == count, name


def test_small_closed_forms():
    a, b, c, d = 0.3, -1.7, 2.5, 0.9
    A = np.array([[a, b], [c, d]])
    for name, f in FLOAT_ALGOS.items():
        assert _rel(f(A), a * d + b * c) < 1e-15, name
    row = np.array([[0.5, -2.0, 3.25, 1.0]])
    for name, f in FLOAT_ALGOS.items():
        assert _rel(f(row), row.sum()) < 1e-15, name
    assert oracle.glynn(np.array([[4.0]])) == 4.0
    assert oracle.glynn(np.zeros((0, 3))) == 1.0


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("m,n", [(5, 5), (4, 7), (7, 7)])
def test_row_column_permutation_and_transpose(m, n):
    g = inputs.rng(40 + m + n)
    A = g.uniform(-1, 1, (m, n))
    ref = oracle.glynn(A)
    for _ in range(3):
        P = A[g.permutation(m)][:, g.permutation(n)]
        assert _rel(oracle.glynn(P), ref) < 1e-14
        assert _rel(oracle.ryser(P), ref) < 1e-14
    assert _rel(oracle.glynn(A.T), ref) < 1e-14  # m > n evaluated as per(A^T)
    assert _rel(oracle.ryser_rect(np.ascontiguousarray(A.T)), ref) < 1e-14


@pytest.mark.parametrize("m,n", [(5, 5), (4, 8)])
def test_multilinear_in_a_row_and_scaling(m, n):
    g = inputs.rng(60 + m + n)
    A = g.uniform(-1, 1, (m, n))
    x, y = g.uniform(-1, 1, n), g.uniform(-1, 1, n)
    al, be = 0.7, -1.3
    for f in (oracle.glynn, oracle.ryser):
        Ax, Ay, Am = A.copy(), A.copy(), A.copy()
        Ax[2], Ay[2], Am[2] = x, y, al * x + be * y
        lhs, rhs = f(Am), al * f(Ax) + be * f(Ay)
        assert abs(lhs - rhs) < 1e-13 * (abs(al * f(Ax)) + abs(be * f(Ay)) + 1e-300)
        assert _rel(f(2.5 * A), 2.5 ** m * f(A)) < 1e-14


@pytest.mark.parametrize("m,n", [(5, 5), (4, 7)])
def test_laplace_expansion_first_row(m, n):
    # per(A) = sum_j a_0j per(A with row 0 and column j removed)
    g = inputs.rng(80 + m + n)
    A = g.uniform(-1, 1, (m, n))
    rhs = sum(A[0, j] * oracle.glynn(np.delete(A[1:], j, axis=1)) for j in range(n))
    assert _rel(oracle.glynn(A), rhs) < 1e-13
    assert _rel(oracle.ryser(A), rhs) < 1e-13
    Ai = g.integers(-9, 10, (m, n)).astype(np.int64)
    rhs_i = sum(int(Ai[0, j]) * oracle.subset_dp(np.delete(Ai[1:], j, axis=1)) for j in range(n))
    assert oracle.glynn(Ai) == oracle.ryser(Ai) == rhs_i


@pytest.mark.parametrize("m,n", [(4, 4), (6, 6), (3, 7)])
def test_complex_identities(m, n):
    g = inputs.rng(90 + m + n)
    A = g.standard_normal((m, n)) + 1j * g.standard_normal((m, n))
    ref = oracle.glynn(A)
    for f in (oracle.ryser, oracle.definition, oracle.ryser_rect):
        assert _rel(f(A), ref) < 1e-13
    assert _rel(oracle.glynn(1j * A), (1j) ** m * ref) < 1e-13  # per(cA) = c^m per(A)
    assert _rel(oracle.glynn(np.conj(A)), np.conj(ref)) < 1e-13
    R = A.real.copy()
    assert _rel(oracle.glynn(R + 0j), oracle.glynn(R)) < 1e-15


# ---------------------------------------------------------------- Gray-code order
@pytest.mark.parametrize("n", range(2, 11))
def test_focus_pointer_is_reflected_gray_code(n):
    # the g-th flip of the reflected binary Gray code is at bit ctz(g); the
    # algorithm flips delta[bound - pos], i.e. row n-1-ctz(g)
    flips = oracle.glynn_flips(n)
    expect = [n - 1 - ((g & -g).bit_length() - 1) for g in range(1, 1 << (n - 1))]
    assert flips == expect
    if n == 3:
        assert flips == [2, 1, 2]
    if n == 4:
        assert flips == [3, 2, 3, 1, 3, 2, 3]


def test_single_terms_follow_the_focus_pointer_order():
    # term g of the partial sums is the g-th term of the algorithm: starting from all
    # +1, the flips of Algorithm "Glynn's Algorithm for Square Matrices" at n = 4 hit
    # rows 3, 2, 3, 1, 3, 2, 3, and term g carries the sign (-1)^g.  For a rank-one
    # A = u v^T every column sum of a term is (u . delta) v_j, so each single term is
    # (-1)^g (u . delta_g)^4 prod_j v_j: a wrong row per Gray bit or a wrong sign
    # changes the single terms even where the full sum is unchanged.
    u = np.array([1.0, 2.0, 5.0, 11.0])
    v = np.array([1.0, 3.0, -2.0, 7.0])
    A = np.outer(u, v)
    delta = np.ones(4)
    deltas = [delta.copy()]
    for row in [3, 2, 3, 1, 3, 2, 3]:
        delta[row] = -delta[row]
        deltas.append(delta.copy())
    for g, d in enumerate(deltas):
        term = (-1) ** g * float(u @ d) ** 4 * float(np.prod(v))
        assert oracle.glynn_partial(A, g, g + 1) == term, g
        assert oracle.glynn_partial(A.astype(np.int64), g, g + 1) == int(term), g
        assert oracle.glynn_partial(A * (1 + 1j), g, g + 1) == term * (1 + 1j) ** 4, g


@pytest.mark.parametrize("m,n,kind", [(5, 5, "real"), (4, 7, "real"), (6, 6, "complex"), (3, 8, "complex"),
                                      (7, 7, "int"), (4, 9, "int")])
def test_glynn_partial_sums_the_same_terms(m, n, kind):
    g = inputs.rng(120 + m + n)
    if kind == "real":
        A = g.uniform(-1, 1, (m, n))
    elif kind == "complex":
        A = g.standard_normal((m, n)) + 1j * g.standard_normal((m, n))
    else:
        A = g.integers(-7, 8, (m, n)).astype(np.int64)
    T = 1 << (n - 1)
    norm = T * math.factorial(n - m)
    full = oracle.glynn_partial(A, 0, T)
    if kind == "int":
        assert full % norm == 0 and full // norm == oracle.glynn(A) == oracle.subset_dp(A)
        cuts = sorted(set([0, T] + [int(c) for c in g.integers(0, T, 5)]))
        assert sum(oracle.glynn_partial(A, a, b) for a, b in zip(cuts, cuts[1:])) == full
    else:
        # the partial sum visits exactly the terms of the focus-pointer loop in the same
        # order, so the unnormalised totals agree to the last bit of the long double
        # (the rectangular normalisation by (n-m)! adds one long-double rounding)
        if kind == "real":
            F = sum(Fraction(x) for x in oracle.glynn_partial(A, 0, T, dd=True))
            R = sum(Fraction(x) for x in oracle.glynn(A, dd=True))
            if m == n:
                assert F == R * norm
            else:
                assert abs(F / norm - R) <= Fraction(1, 2 ** 60) * abs(R)
        assert _rel(full / norm, oracle.glynn(A)) < 1e-15
        assert _rel(full / norm, oracle.definition(A)) < 1e-13


def test_int_matches_long_double_and_f64():
    g = inputs.rng(777)
    for (m, n) in [(6, 6), (5, 9), (8, 8)]:
        A = g.integers(-20, 21, (m, n)).astype(np.int64)
        exact = oracle.subset_dp(A)
        assert oracle.glynn(A) == oracle.ryser(A) == exact
        assert abs(oracle.glynn(A.astype(float)) - exact) <= 1e-12 * abs(exact) + 1e-6
        assert abs(oracle.ryser(A.astype(float), "f64") - exact) <= 1e-10 * abs(exact) + 1e-6


def test_digits_lost_metric():
    # Eq. digits_lost: log10 of the relative error minus log10 of the machine epsilon
    eps = np.finfo(np.float64).eps
    assert abs(oracle.digits_lost(1.0 + 1000 * eps, 1.0) - 3.0) < 1e-9
    assert oracle.digits_lost(2.0, 2.0) == -np.inf


def test_long_double_width_is_reported():
    assert oracle.ldbl_mant_dig() in (53, 64, 106, 113)


@pytest.mark.parametrize("m,n", [(4, 4), (5, 5), (3, 7), (6, 9)])
def test_ryser_gray_partial_sums_to_the_permanent(m, n):
    # the Gray-ordered subset sum with the size weights of Eq. ryser_rectangle covers
    # every subset once, so the full range equals the permanent (definition)
    g = inputs.rng(150 + m + n)
    A = g.uniform(-1, 1, (m, n))
    full = oracle.ryser_partial(A, 0, 1 << n)
    assert _rel(full, oracle.definition(A)) < 1e-13
    cuts = sorted(set([0, 1 << n] + [int(c) for c in g.integers(0, 1 << n, 4)]))
    parts = sum(oracle.ryser_partial(A, a, b) for a, b in zip(cuts, cuts[1:]))
    assert _rel(parts, full) < 1e-13


# ------------------------------------------- Glynn with the padding rows grouped
@pytest.mark.parametrize("m,n", [(1, 1), (1, 7), (2, 6), (3, 8), (4, 10), (5, 9), (6, 6), (2, 13)])
def test_grouped_glynn_exact_on_small_integers(m, n):
    # integer entries in -3..3: every column sum, product and weighted sum is an integer
    # below 2^53, so the double evaluation is exact and must equal the exact definition
    g = inputs.rng(170 + 13 * m + n)
    A = g.integers(-3, 4, (m, n))
    assert oracle.glynn_rect_grouped(A.astype(np.float64), prec="f64") == float(oracle.definition(A))


@pytest.mark.parametrize("m,n", [(1, 5), (2, 5), (3, 7), (4, 9), (5, 6), (2, 12), (6, 11), (3, 30)])
def test_grouped_glynn_all_ones(m, n):
    # the alternating binomial sums cancel: allow the first-order long-double bound
    # (n + 4) eps sum|t| / (2^(n-1) (n-m)!) around the exact n! / (n-m)!
    A = np.ones((m, n))
    exact = math.factorial(n) // math.factorial(n - m)
    eps = 2.0 ** -(oracle.ldbl_mant_dig() - 1)
    bound = (n + 4) * eps * oracle.glynn_rect_grouped_abs(A) / (2.0 ** (n - 1) * math.factorial(n - m))
    assert abs(oracle.glynn_rect_grouped(A) - exact) <= bound
    if n <= 12:
        assert oracle.glynn_rect_grouped(A) == exact


@pytest.mark.parametrize("m,n", [(3, 9), (5, 11), (8, 12)])
def test_grouped_glynn_equals_ungrouped_sum(m, n):
    # same terms, grouped: the values agree and so do the sums of |term|
    g = inputs.rng(180 + m + n)
    A = g.uniform(-1, 1, (m, n))
    assert _rel(oracle.glynn_rect_grouped(A), oracle.glynn(A)) < 1e-14
    full_abs = oracle.glynn_partial_abs(A, 0, 1 << (n - 1))
    assert _rel(oracle.glynn_rect_grouped_abs(A), full_abs) < 1e-14


@pytest.mark.parametrize("m,n", [(4, 7), (6, 10)])
def test_grouped_glynn_invariants(m, n):
    # column permutation, multilinearity in a row and scaling (the definition's invariants)
    g = inputs.rng(190 + m + n)
    A = g.uniform(-1, 1, (m, n))
    p = oracle.glynn_rect_grouped(A)
    assert _rel(oracle.glynn_rect_grouped(A[:, g.permutation(n)]), p) < 1e-13
    B, C = A.copy(), A.copy()
    x, y = g.uniform(-1, 1, n), g.uniform(-1, 1, n)
    B[2], C[2] = x, y
    S = A.copy()
    S[2] = x + 3.0 * y
    lhs = oracle.glynn_rect_grouped(S)
    rhs = oracle.glynn_rect_grouped(B) + 3.0 * oracle.glynn_rect_grouped(C)
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0)


# ------------------------------------------- SBP coefficients (Eq. SBGpermanent)
@pytest.mark.parametrize("n,N", [(2, 5), (3, 7), (4, 8)])
def test_sbp_coefficients_sum_to_rectangular_permanent(n, N):
    # every injective map rows -> states has an image of n states, so summing per(C P)
    # over all n-subsets gives the rectangular permanent (Eq. rectangular_permanent_definition)
    g = inputs.rng(200 + n + N)
    C = g.integers(-3, 4, (n, N))
    total = 0
    for S in itertools.combinations(range(N), n):
        total += oracle.sbp_coefficient(C, sum(1 << j for j in S))
    assert total == oracle.definition(C)


def test_sbp_selection_matrix_and_closed_forms():
    P = oracle.sbp_selection_matrix(0b1011001, 7, 4)
    assert P.sum(axis=0).tolist() == [1, 1, 1, 1]  # one state per boson
    assert P.sum(axis=1).tolist() == [1, 0, 0, 1, 1, 0, 1]  # row sums are the occupations m_j
    assert [int(np.argmax(P[:, k])) for k in range(4)] == [0, 3, 4, 6]  # in increasing order
    with pytest.raises(ValueError):
        oracle.sbp_selection_matrix(0b111, 7, 4)
    # all-ones coefficients: every coefficient is n!
    assert oracle.sbp_coefficient(np.ones((5, 9), dtype=np.int64), 0b110110001) == math.factorial(5)
    # rank one C = u v^T: c_m = n! prod(u) prod_{j occupied} v_j
    g = inputs.rng(210)
    u, v = g.uniform(0.5, 1.5, 4), g.uniform(0.5, 1.5, 10)
    occ = 0b1001010010
    expect = math.factorial(4) * float(np.prod(u)) * float(np.prod([v[j] for j in range(10) if (occ >> j) & 1]))
    assert _rel(oracle.sbp_coefficient(np.outer(u, v), occ), expect) < 1e-13


# ------------------------------------------------ Gaussian integers (exact, 128-bit)
def _gaussian_brute(re, im):
    """Exact permanent of re + i im by enumerating the m-permutations, in Python ints."""
    m, n = re.shape
    sr = si = 0
    for perm in itertools.permutations(range(n), m):
        pr, pi = 1, 0
        for r, c in enumerate(perm):
            a, b = int(re[r, c]), int(im[r, c])
            pr, pi = pr * a - pi * b, pr * b + pi * a
        sr += pr
        si += pi
    return sr, si


@pytest.mark.parametrize("m,n", [(1, 3), (3, 3), (3, 5), (4, 6), (5, 5), (2, 7)])
def test_gaussian_glynn_and_definition_equal_brute_force(m, n):
    g = inputs.rng(220 + 10 * m + n)
    re, im = g.integers(-4, 5, (m, n)), g.integers(-4, 5, (m, n))
    sr, si = _gaussian_brute(re, im)
    assert oracle.definition_gaussian(re, im) == (sr, si)
    assert oracle.glynn_gaussian(re, im) == (sr, si)
    assert oracle.glynn_gaussian(re.T, im.T) == (sr, si)  # transpose rule


@pytest.mark.parametrize("n", [2, 5, 8])
def test_gaussian_closed_forms(n):
    # real-valued input: the real integer permanent; purely imaginary input:
    # per(i A) = i^n per(A); all entries 1 + i: (1 + i)^n n!
    g = inputs.rng(230 + n)
    A = g.integers(-5, 6, (n, n))
    p = oracle.glynn(A)
    Z = np.zeros_like(A)
    assert oracle.glynn_gaussian(A, Z) == (p, 0)
    ipow = [(1, 0), (0, 1), (-1, 0), (0, -1)][n % 4]
    assert oracle.glynn_gaussian(Z, A) == (ipow[0] * p, ipow[1] * p)
    w = (1 + 1j) ** n * math.factorial(n)
    assert oracle.glynn_gaussian(np.ones((n, n), int), np.ones((n, n), int)) == (int(w.real), int(w.imag))


# --- exact Cauchy permanents (oracle.cauchy), the truth for perm_cauchy


def test_exact_det_known_values():
    oc = oracle.cauchy
    # permutation matrices (every pivot search swaps rows): det = sign of the permutation
    for perm in itertools.permutations(range(4)):
        P = [[int(perm[i] == j) for j in range(4)] for i in range(4)]
        inv = sum(1 for i in range(4) for j in range(i + 1, 4) if perm[i] > perm[j])
        assert oc.det(P) == (-1) ** inv
    # Vandermonde on integer points: prod_{i<j} (t_j - t_i)
    t = [3, -1, 4, 10, -5, 9]
    V = [[ti ** k for k in range(len(t))] for ti in t]
    assert oc.det(V) == math.prod(t[j] - t[i] for i in range(len(t)) for j in range(i + 1, len(t)))
    # singular (two equal rows) and triangular
    assert oc.det([[1, 2, 3], [4, 5, 6], [1, 2, 3]]) == 0
    assert oc.det([[2, 7, 1], [0, -3, 5], [0, 0, Fraction(1, 7)]]) == Fraction(-6, 7)


@pytest.mark.parametrize("n", [1, 2, 4, 6, 9])
def test_exact_det_matches_cauchy_closed_form(n):
    # Cauchy's determinant formula is an identity independent of elimination
    x, y = inputs.cauchy_points(n, 700 + n)
    oc = oracle.cauchy
    assert oc.det(oc.cauchy_matrix(x[0], y[0])) == oc.cauchy_det_closed_form(x[0], y[0])


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7])
def test_borchardt_equals_definition_exactly(n):
    # Eq. caucy_permanent, checked by brute force in exact rationals: the paper's point
    # distribution, and interleaved points so that C has entries of both signs
    oc = oracle.cauchy
    x, y = inputs.cauchy_points(n, 710 + n)
    C = oc.cauchy_matrix(x[0], y[0])
    assert oc.permanent_borchardt(x[0], y[0]) == oc.permanent_definition(C)
    g = inputs.rng(720 + n)
    pts = g.permutation(g.uniform(-1.0, 1.0, 2 * n))
    xi, yi = pts[:n], pts[n:]
    C = oc.cauchy_matrix(xi, yi)
    assert oc.permanent_borchardt(xi, yi) == oc.permanent_definition(C)


def test_borchardt_small_closed_forms():
    oc = oracle.cauchy
    assert oc.permanent_borchardt([0.5], [-0.25]) == Fraction(4, 3)
    x, y = [0.5, 0.75], [-0.25, -0.5]
    c = [[Fraction(1) / (Fraction(a) - Fraction(b)) for b in y] for a in x]
    assert oc.permanent_borchardt(x, y) == c[0][0] * c[1][1] + c[0][1] * c[1][0]
    with pytest.raises(ZeroDivisionError):
        oc.permanent_borchardt([0.5, 0.5], [-0.25, -0.5])


def test_sbp_of_a_cauchy_matrix_equals_the_exact_cauchy_permanent():
    # Eq. SBGpermanent with a Cauchy coefficient matrix: the oracle's C P permanent (long
    # double, the selection matrix of the paper) against Borchardt's exact value for the
    # occupied points -- two independent oracle paths
    g = inputs.rng(760)
    n, N = 5, 9
    x = g.uniform(0.25, 0.75, n)
    y = g.uniform(-0.75, -0.25, N)
    C = 1.0 / (x[:, None] - y[None, :])
    for occ in (0b000011111, 0b110101001, 0b101010101, 0b111110000):
        ys = y[[j for j in range(N) if (occ >> j) & 1]]
        want = float(oracle.cauchy.permanent_borchardt(x, ys))
        got = oracle.sbp_coefficient(C, occ)
        # C rounded to double (two roundings per entry, all terms positive): n 2u, plus the sum
        assert abs(got - want) <= (2 * n + 4) * np.finfo(float).eps / 2 * want, (occ, got, want)


# ---------------------------------------------------------------------------
# Sums of |term| (the scales every float tolerance of the GPU tests is built on),
# pinned to closed forms that do not go through the oracle's term loops.
#
# Glynn on the all-ones m x n matrix (padded with rows of ones, Eq. glynn_rectangle):
# every column sum equals n - 2t, t = number of -1 signs among the n - 1 free rows,
# so sum|t| = sum_t C(n-1, t) |n - 2t|^n.  Scaling column j by v_j scales every term
# by v_j.  A diagonal matrix has |term| = prod_j |d_j| for each of the 2^(n-1) terms.
# Ryser on the all-ones m x n matrix: every row sum over S equals |S| = s, so
# sum|t| = sum_{s=1..m} C(n, s) C(n-s, m-s) s^m; scaling row i by r_i scales every
# term by r_i; a diagonal matrix has one nonzero term, the full set, prod_i |d_i|.

def _glynn_ones_abs(n):
    return sum(math.comb(n - 1, t) * abs(n - 2 * t) ** n for t in range(n))


def _ryser_ones_abs(m, n):
    return sum(math.comb(n, s) * math.comb(n - s, m - s) * s ** m for s in range(1, m + 1))


@pytest.mark.parametrize("n", [1, 2, 5, 9, 13])
def test_glynn_abs_all_ones_and_column_scaling(n):
    v = inputs.rng(600 + n).uniform(-2, 2, n)
    exact = _glynn_ones_abs(n) * float(np.prod(np.abs(v)))
    A = np.ones((n, n)) * v[None, :]
    assert _rel(oracle.glynn_partial_abs(A, 0, 1 << (n - 1)), exact) < 1e-15
    Ac = A * np.exp(1j * inputs.rng(610 + n).uniform(0, 6.3, n))[None, :]
    assert _rel(oracle.glynn_partial_abs(Ac, 0, 1 << (n - 1)), exact) < 1e-15
    assert _rel(oracle.glynn_abs(A), exact / 2.0 ** (n - 1)) < 1e-15


@pytest.mark.parametrize("m,n", [(1, 4), (2, 7), (3, 8), (5, 11), (4, 30), (2, 60)])
def test_glynn_abs_all_ones_rectangle(m, n):
    exact = float(_glynn_ones_abs(n))
    A = np.ones((m, n))
    assert _rel(oracle.glynn_rect_grouped_abs(A), exact) < 1e-15
    assert _rel(oracle.glynn_rect_grouped_abs(A.astype(complex)), exact) < 1e-15
    if n <= 14:
        assert _rel(oracle.glynn_partial_abs(A, 0, 1 << (n - 1)), exact) < 1e-15
        assert _rel(oracle.glynn_partial_abs(A.astype(complex), 0, 1 << (n - 1)), exact) < 1e-15
        norm = 2.0 ** (n - 1) * math.factorial(n - m)
        assert _rel(oracle.glynn_abs(A), exact / norm) < 1e-15


@pytest.mark.parametrize("n", [1, 3, 6, 10])
def test_glynn_abs_diagonal(n):
    d = inputs.rng(620 + n).uniform(0.5, 2, n) * np.where(np.arange(n) % 2, -1, 1)
    exact = 2.0 ** (n - 1) * float(np.prod(np.abs(d)))
    assert _rel(oracle.glynn_partial_abs(np.diag(d), 0, 1 << (n - 1)), exact) < 1e-15
    assert _rel(oracle.glynn_rect_grouped_abs(np.diag(d)), exact) < 1e-15
    dc = d * np.exp(1j * np.arange(n))
    assert _rel(oracle.glynn_partial_abs(np.diag(dc), 0, 1 << (n - 1)), exact) < 1e-15


@pytest.mark.parametrize("m,n", [(1, 1), (3, 3), (4, 9), (6, 6), (5, 12)])
def test_ryser_abs_all_ones_row_scaling_and_diagonal(m, n):
    r = inputs.rng(630 + m + n).uniform(-2, 2, m)
    exact = _ryser_ones_abs(m, n) * float(np.prod(np.abs(r)))
    A = r[:, None] * np.ones((m, n))
    assert _rel(oracle.ryser_abs(A), exact) < 1e-15
    Ac = A * np.exp(1j * inputs.rng(640 + m).uniform(0, 6.3, m))[:, None]
    assert _rel(oracle.ryser_abs(Ac), exact) < 1e-15
    d = np.abs(r) + 0.25
    assert _rel(oracle.ryser_abs(np.diag(d)), float(np.prod(d))) < 1e-15


@pytest.mark.parametrize("m,n,kind", [(5, 5, "real"), (4, 8, "real"), (5, 5, "complex"), (3, 7, "complex")])
def test_abs_sums_are_invariant_and_split_over_ranges(m, n, kind):
    # sum|t| of Glynn and of Ryser is unchanged by row and column permutations (Glynn:
    # flipping every sign leaves |term| unchanged, so the fixed first sign is no
    # restriction), scales by |c| with a column (square Glynn) or row (Ryser) scaled by
    # c, and partial ranges add up to the whole.
    g = inputs.rng(650 + m + n)
    A = g.uniform(-1, 1, (m, n))
    if kind == "complex":
        A = A + 1j * g.uniform(-1, 1, (m, n))
    ga, ra = oracle.glynn_abs(A), oracle.ryser_abs(A)
    P = A[g.permutation(m)][:, g.permutation(n)]
    assert _rel(oracle.glynn_abs(P), ga) < 1e-14
    assert _rel(oracle.ryser_abs(P), ra) < 1e-14
    c = 1.75 if kind == "real" else 1.0 - 1.5j
    if m == n:  # (the padding rows of a rectangle are not scaled with a column)
        B = A.copy()
        B[:, 1] *= c
        assert _rel(oracle.glynn_abs(B), abs(c) * ga) < 1e-14
    B = A.copy()
    B[1, :] *= c
    assert _rel(oracle.ryser_abs(B), abs(c) * ra) < 1e-14
    h = 1 << (n - 2)
    whole = oracle.glynn_partial_abs(A, 0, 1 << (n - 1))
    assert _rel(oracle.glynn_partial_abs(A, 0, h) + oracle.glynn_partial_abs(A, h, 1 << (n - 1)), whole) < 1e-15
    assert _rel(oracle.ryser_partial_abs(A, 0, 5) + oracle.ryser_partial_abs(A, 5, 1 << n), ra) < 1e-15
    # each sum|t| bounds the modulus of its (normalised) sum
    assert abs(oracle.glynn(A)) <= ga * (1 + 1e-14)
    assert abs(oracle.ryser(A)) <= ra * (1 + 1e-14)


@pytest.mark.parametrize("m,n", [(3, 3), (4, 6), (5, 5)])
def test_definition_abs_is_permanent_of_moduli(m, n):
    # per(|A|) by brute force over the injective maps; ones give n!/(n-m)!
    g = inputs.rng(670 + m + n)
    A = g.uniform(-1, 1, (m, n)) + 1j * g.uniform(-1, 1, (m, n))
    brute = sum(float(np.prod([abs(A[i, s[i]]) for i in range(m)])) for s in itertools.permutations(range(n), m))
    assert _rel(oracle.definition_abs(A), brute) < 1e-14
    assert oracle.definition_abs(np.ones((m, n))) == pytest.approx(math.factorial(n) / math.factorial(n - m), rel=1e-15)


# Scale of the closed-form padding sum: sum over the 2^(m-1) sign vectors of
# e_m(|c|) / 2^(m-1).  All-ones m x n: every column sum is m - 2t, so it is
# C(n, m) sum_t C(m-1, t) |m - 2t|^m / 2^(m-1); [D | 0] with D diagonal: only the
# first m columns are nonzero and e_m(|c|) = prod |d_j| for every sign vector; a
# square matrix gives Glynn's own sum of |term|.
@pytest.mark.parametrize("m,n", [(1, 1), (1, 6), (3, 3), (3, 9), (5, 11), (8, 20)])
def test_esym_abs_closed_forms(m, n):
    exact = math.comb(n, m) * sum(math.comb(m - 1, t) * abs(m - 2 * t) ** m for t in range(m)) / 2.0 ** (m - 1)
    assert _rel(oracle.glynn_esym_abs(np.ones((m, n))), exact) < 1e-15
    d = inputs.rng(700 + m + n).uniform(0.5, 2, m) * np.where(np.arange(m) % 2, -1, 1)
    Z = np.zeros((m, n))
    Z[np.arange(m), np.arange(m)] = d
    assert _rel(oracle.glynn_esym_abs(Z), float(np.prod(np.abs(d)))) < 1e-15
    ph = np.exp(1j * inputs.rng(705 + m).uniform(0, 6.3, m))
    assert _rel(oracle.glynn_esym_abs(Z * ph[:, None]), float(np.prod(np.abs(d)))) < 1e-15
    assert _rel(oracle.glynn_esym_abs(np.ones((m, n), complex)), exact) < 1e-15
    if m == n:
        A = inputs.rng(710 + n).uniform(-1, 1, (n, n))
        assert _rel(oracle.glynn_esym_abs(A), oracle.glynn_abs(A)) < 1e-14


@pytest.mark.parametrize("m,n", [(3, 7), (5, 9)])
def test_esym_abs_invariants_and_bound(m, n):
    # unchanged by row and column permutations, scaled by |c|^m with the matrix scaled
    # by c (every product in e_m has m factors), and it bounds |per(A)|
    g = inputs.rng(720 + m + n)
    A = g.uniform(-1, 1, (m, n))
    s = oracle.glynn_esym_abs(A)
    P = A[g.permutation(m)][:, g.permutation(n)]
    assert _rel(oracle.glynn_esym_abs(P), s) < 1e-14
    assert _rel(oracle.glynn_esym_abs(-2.5 * A), 2.5 ** m * s) < 1e-14
    assert abs(oracle.glynn(A)) <= s * (1 + 1e-14)


# ---------------------------------------------------------------------------
# Exact integer evaluation (oracle.exact): the definition on tiny inputs, closed forms
# and the long-double grouped sum on a well-conditioned shape.
def test_exact_grouped_glynn_pins():
    from oracle import exact
    for (m, n) in [(1, 3), (2, 5), (3, 6), (4, 4)]:
        A = inputs.rng(800 + m + n).uniform(-1, 1, (m, n))
        assert exact.glynn_rect_grouped(A) == exact.definition(A)
        assert exact.glynn_rect_grouped(A.T) == exact.definition(A)
    assert exact.glynn_rect_grouped(np.ones((3, 9))) == math.factorial(9) // math.factorial(6)
    assert exact.glynn_rect_grouped(np.eye(5)[:3]) == 1
    A = inputs.rng(811).uniform(0, 1, (6, 10))
    assert _rel(float(exact.glynn_rect_grouped(A)), oracle.glynn_rect_grouped(A)) < 1e-15
    Z, s = exact.to_integer_matrix(np.array([[0.5, -0.25], [3.0, 2.0 ** -40]]))
    assert s == 40 and Z[0][0] == 2 ** 39 and Z[1][1] == 1 and Z[0][1] == -(2 ** 38)


@pytest.mark.parametrize("m,n", [(2, 5), (3, 8), (5, 9)])
def test_ryser_abs_by_size_equals_gray_enumeration(m, n):
    # the combination enumeration and the Gray-ordered enumeration visit the same
    # weighted subsets (all-ones closed form pinned above)
    A = inputs.rng(740 + m + n).uniform(-1, 1, (m, n))
    assert _rel(oracle.ryser_abs(A), oracle.ryser_partial_abs(A, 0, 1 << n)) < 1e-14
    assert _rel(oracle.ryser_abs(np.ones((m, n))), _ryser_ones_abs(m, n)) < 1e-15


@pytest.mark.parametrize("m,n", [(2, 6), (4, 9), (6, 11)])
def test_complex_grouped_abs_equals_ungrouped(m, n):
    g = inputs.rng(760 + m + n)
    A = g.standard_normal((m, n)) + 1j * g.standard_normal((m, n))
    assert _rel(oracle.glynn_rect_grouped_abs(A), oracle.glynn_partial_abs(A, 0, 1 << (n - 1))) < 1e-14


def test_exact_complex_definition():
    from oracle import exact
    g = inputs.rng(820)
    A = g.uniform(-1, 1, (4, 5)) + 1j * g.uniform(-1, 1, (4, 5))
    re, im = exact.definition(A)
    ref = oracle.definition(A)
    assert _rel(complex(float(re), float(im)), ref) < 1e-15
    B = A.real.copy()
    re, im = exact.definition(B + 0j)
    assert im == 0 and re == exact.definition(B)
    # per(i I) = i^n
    re, im = exact.definition(1j * np.eye(3))
    assert (re, im) == (0, -1)
