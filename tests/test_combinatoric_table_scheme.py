"""The tail-table scheme of the combinatoric kernel (csrc/combinatoric.cu), run on the
CPU in exact integers: the colex ranks and unranking of column triples and
quadruples and quintuples, the tables of the last three, four and five rows built
from each other, the prefix unranking of the first `depth` rows, and the search's
branches with six rows left (six free columns), five (the direct path for five free
columns, and the general one), four or three.  Checked against the definition (Eq.
rectangular_permanent_definition) by brute force, for every prefix depth, with every
table index asserted in bounds.  This pins the indexing the kernel relies on; the
kernel itself is checked on the GPU (test_gpu_combinatoric.py)."""
from itertools import permutations
from math import comb, factorial, prod
import random

import pytest

TAIL_N = 16  # the kernel builds the tables for n <= 16


def bits(mask):
    out = []
    while mask:
        out.append((mask & -mask).bit_length() - 1)
        mask &= mask - 1
    return out


def unrank(idx, k, n):
    """Column set of colex rank idx among the k-subsets of range(n), ascending, found
    the kernel's way (largest top element first)."""
    cols = []
    rem, top = idx, n
    for j in range(k, 0, -1):
        c = j - 1
        while c + 1 < top and comb(c + 1, j) <= rem:
            c += 1
        rem -= comb(c, j)
        cols.append(c)
        top = c
    return tuple(reversed(cols))


def rank(cols):
    return sum(comb(c, j + 1) for j, c in enumerate(cols))


def tables(A, m, n, five):
    T3 = [None] * comb(TAIL_N, 3)
    T4 = [None] * comb(TAIL_N, 4)
    T5 = [None] * comb(TAIL_N, 5)
    r0, r1, r2 = A[m - 3], A[m - 2], A[m - 1]
    for idx in range(comb(n, 3)):
        x, y, z = unrank(idx, 3, n)
        assert 0 <= x < y < z < n and rank((x, y, z)) == idx
        T3[idx] = sum(r0[p[0]] * r1[p[1]] * r2[p[2]] for p in permutations((x, y, z)))
    if m >= 5:
        r = A[m - 4]
        for idx in range(comb(n, 4)):
            q = unrank(idx, 4, n)
            assert 0 <= q[0] < q[1] < q[2] < q[3] < n and rank(q) == idx
            v = 0
            for c in q:
                i = rank(tuple(d for d in q if d != c))
                assert 0 <= i < comb(n, 3)
                v += r[c] * T3[i]
            T4[idx] = v
    if five and m >= 6:
        r = A[m - 5]
        for idx in range(comb(n, 5)):
            q = unrank(idx, 5, n)
            assert all(0 <= a < b < n for a, b in zip(q, q[1:])) and rank(q) == idx
            v = 0
            for c in q:
                i = rank(tuple(d for d in q if d != c))
                assert 0 <= i < comb(n, 4)
                v += r[c] * T4[i]
            T5[idx] = v
    return T3, T4, T5


def table_sum(T, k, n, fm):
    s = 0
    cols = bits(fm)
    for sub in _subsets(cols, k):
        i = rank(sub)
        assert 0 <= i < comb(n, k)
        s += T[i]
    return s


def _subsets(cols, k):
    if k == 0:
        yield ()
        return
    for j in range(len(cols) - k + 1):
        for rest in _subsets(cols[j + 1:], k - 1):
            yield (cols[j],) + rest


def kernel_scheme(A, m, n, depth, five):
    tail = n <= TAIL_N and m >= 4
    tail4 = tail and m >= 5
    tail5 = tail and five and m >= 6  # the kernel builds the five-row table for real input
    T3, T4, T5 = tables(A, m, n, five) if tail else (None, None, None)
    allcols = (1 << n) - 1
    rowmask = [sum(1 << j for j in range(n) if A[i][j] != 0) for i in range(m)]

    def value(k, used):  # the search below row k with the columns `used` taken
        fm = allcols & ~used
        if tail5 and k == m - 6 and bin(fm).count("1") == 6:  # a square: one quintuple each
            c = bits(fm)
            s = 0
            for i in range(6):
                if (rowmask[k] >> c[i]) & 1:
                    r = rank(tuple(c[q] for q in range(6) if q != i))
                    assert 0 <= r < comb(n, 5)
                    s += A[k][c[i]] * T5[r]
            return s
        if tail4 and k == m - 5:
            if bin(fm).count("1") == 5:  # a square: the rest of each free column is one quadruple
                c = bits(fm)
                s = 0
                for i in range(5):
                    if (rowmask[k] >> c[i]) & 1:
                        r = rank(tuple(c[q] for q in range(5) if q != i))
                        assert 0 <= r < comb(n, 4)
                        s += A[k][c[i]] * T4[r]
                return s
            return sum(A[k][x] * table_sum(T4, 4, n, fm & ~(1 << x)) for x in bits(rowmask[k] & fm))
        if tail4 and k == m - 4:
            return table_sum(T4, 4, n, fm)
        if tail and k == m - 4:
            return sum(A[k][x] * table_sum(T3, 3, n, fm & ~(1 << x)) for x in bits(rowmask[k] & fm))
        if tail and k == m - 3:
            return table_sum(T3, 3, n, fm)
        if k == m - 1:
            return sum(A[k][c] for c in bits(rowmask[k] & fm))
        return sum(A[k][c] * value(k + 1, used | (1 << c)) for c in bits(rowmask[k] & fm))

    total = 0
    for r in range(factorial(n) // factorial(n - depth)):
        rem, used, pre = r, 0, 1
        for k in range(depth):  # mixed-radix digits: the digit-th free column
            digit = rem % (n - k)
            rem //= n - k
            c = bits(allcols & ~used)[digit]
            used |= 1 << c
            pre *= A[k][c]
        if pre:
            total += pre * (1 if depth == m else value(depth, used))
    return total


def definition(A, m, n):
    return sum(prod(A[i][p[i]] for i in range(m)) for p in permutations(range(n), m))


@pytest.mark.parametrize("m", range(1, 10))
def test_tail_tables_match_definition_at_every_depth(m):
    rnd = random.Random(4200 + m)
    for n in range(m, min(m + 4, 10)):
        A = [[rnd.choice([0, 0, 1, 2, -1, 3]) for _ in range(n)] for _ in range(m)]
        ref = definition(A, m, n)
        for depth in range(m + 1):
            if factorial(n) // factorial(n - depth) <= 20000:
                for five in (False, True):
                    assert kernel_scheme(A, m, n, depth, five) == ref, (m, n, depth, five)


def test_colex_unranking_is_a_bijection_up_to_16_columns():
    for k in (3, 4, 5):
        for n in range(k, TAIL_N + 1):
            got = [unrank(i, k, n) for i in range(comb(n, k))]
            assert len(set(got)) == comb(n, k)
            assert all(rank(s) == i for i, s in enumerate(got))
