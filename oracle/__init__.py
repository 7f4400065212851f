"""CPU oracle for the permanent -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library
(``paper_2510_03421_gb300``) and the library never imports it.

The arithmetic lives in ``perm_oracle.c`` (plain serial C, compiled with gcc by
:func:`build`); this module only marshals numpy arrays into it.  The exception is
:mod:`oracle.cauchy`: permanents of Cauchy matrices in exact rationals
(``fractions.Fraction``), by the definition and by Borchardt's theorem.

Conventions (the paper's rectangular definition, Eq. rectangular_permanent_definition):

* an ``m x n`` input with ``m > n`` is evaluated as ``per(A.T)``;
* ``per`` of a ``0 x n`` matrix is 1 (the empty product; the paper is silent);
* integer and boolean inputs are evaluated exactly in wrapping 128-bit integer
  arithmetic and returned as Python ``int`` (exact when the unnormalised sum fits
  in a signed 128-bit integer);
* float inputs are evaluated in ``long double`` (``prec="ld"``, the reference) or
  ``double`` (``prec="f64"``, the timed CPU baseline only); complex128 inputs in
  the corresponding complex type.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = [os.path.join(_HERE, "perm_oracle.c"), os.path.join(_HERE, "oracle_real.inc")]
_lib = None
_lock = threading.Lock()

MAX_N = 64


def build(force: bool = False) -> str:
    """Compile perm_oracle.c into liboracle.so next to this file (gcc, no GPU)."""
    newest = max(os.path.getmtime(p) for p in _SRC)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-o", tmp, _SRC[0], "-lm"],
                              cwd=_HERE)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            i, i64, u64, p = ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p
            for prec in ("ld", "f64"):
                for name in ("oracle_definition", "oracle_glynn", "oracle_ryser_rect"):
                    for c in ("", "_c"):
                        getattr(lib, "%s%s_%s" % (name, c, prec)).argtypes = [i, i, p, i64, p]
                for c in ("", "_c"):
                    getattr(lib, "oracle_ryser_square%s_%s" % (c, prec)).argtypes = [i, p, i64, p]
                    getattr(lib, "oracle_glynn_partial%s_%s" % (c, prec)).argtypes = [i, i, p, i64, u64, u64, p]
                getattr(lib, "oracle_glynn_partial_abs_%s" % prec).argtypes = [i, i, p, i64, u64, u64, p]
                getattr(lib, "oracle_glynn_partial_abs_c_%s" % prec).argtypes = [i, i, p, i64, u64, u64, p]
                getattr(lib, "oracle_ryser_partial_abs_%s" % prec).argtypes = [i, i, p, i64, u64, u64, p]
                getattr(lib, "oracle_ryser_partial_abs_c_%s" % prec).argtypes = [i, i, p, i64, u64, u64, p]
                getattr(lib, "oracle_ryser_partial_%s" % prec).argtypes = [i, i, p, i64, u64, u64, p]
                getattr(lib, "oracle_glynn_rect_grouped_%s" % prec).argtypes = [i, i, p, i64, p]
                getattr(lib, "oracle_glynn_rect_grouped_abs_%s" % prec).argtypes = [i, i, p, i64, p]
                getattr(lib, "oracle_glynn_esym_abs_%s" % prec).argtypes = [i, i, p, i64, p]
                getattr(lib, "oracle_glynn_esym_abs_c_%s" % prec).argtypes = [i, i, p, i64, p]
                getattr(lib, "oracle_glynn_rect_grouped_abs_c_%s" % prec).argtypes = [i, i, p, i64, p]
                getattr(lib, "oracle_ryser_rect_abs_%s" % prec).argtypes = [i, i, p, i64, p]
            for name in ("oracle_definition_i128", "oracle_glynn_i128", "oracle_ryser_rect_i128"):
                getattr(lib, name).argtypes = [i, i, p, i64, p]
            lib.oracle_ryser_square_i128.argtypes = [i, p, i64, p]
            lib.oracle_glynn_partial_i128.argtypes = [i, i, p, i64, u64, u64, p]
            for name in ("oracle_definition_ci128", "oracle_glynn_ci128"):
                getattr(lib, name).argtypes = [i, i, p, i64, p]
            lib.oracle_glynn_partial_ci128.argtypes = [i, i, p, i64, u64, u64, p]
            lib.oracle_subset_dp_i128.argtypes = [i, i, p, i64, p]
            lib.oracle_subset_dp_i128.restype = i
            lib.oracle_glynn_flips.argtypes = [i, p, i64]
            lib.oracle_glynn_flips.restype = i
            lib.oracle_ldbl_mant_dig.restype = i
            _lib = lib
    return _lib


def ldbl_mant_dig() -> int:
    """Mantissa bits of the C long double the oracle computes in (64 on x86-64, 113 on aarch64)."""
    return _load().oracle_ldbl_mant_dig()


def _kind(A: np.ndarray) -> str:
    if A.dtype.kind in "iub":
        return "int"
    if A.dtype.kind == "c":
        return "complex"
    if A.dtype.kind == "f":
        return "real"
    raise TypeError("unsupported dtype %s" % A.dtype)


def _prepare(A):
    A = np.asarray(A)
    if A.ndim != 2:
        raise ValueError("expected a 2-D matrix")
    if A.shape[0] > A.shape[1]:
        A = A.T  # per(A) = per(A^T) for m > n
    kind = _kind(A)
    if kind == "int":
        A = np.ascontiguousarray(A, dtype=np.int64)
    elif kind == "complex":
        A = np.ascontiguousarray(A, dtype=np.complex128)
    else:
        A = np.ascontiguousarray(A, dtype=np.float64)
    m, n = A.shape
    if n > MAX_N:
        raise ValueError("the oracle handles n <= %d (full sums are only practical for small n)" % MAX_N)
    return A, kind, m, n


def _i128(buf) -> int:
    v = int(buf[0]) | (int(buf[1]) << 64)
    return v - (1 << 128) if v >> 127 else v


def _real(buf, dd):
    return (float(buf[0]), float(buf[1])) if dd else float(buf[0]) + float(buf[1])


def _cplx(buf, dd):
    if dd:
        return (float(buf[0]), float(buf[1]), float(buf[2]), float(buf[3]))
    return complex(float(buf[0]) + float(buf[1]), float(buf[2]) + float(buf[3]))


def _call(base: str, A, prec: str = "ld", dd: bool = False, square_only: bool = False, extra=()):
    lib = _load()
    A, kind, m, n = _prepare(A)
    if m == 0:
        return 1 if kind == "int" else (1.0 if kind == "real" else 1 + 0j)
    if square_only and m != n:
        raise ValueError("%s needs a square matrix" % base)
    ptr = A.ctypes.data_as(ctypes.c_void_p)
    args = (m, ptr, n) if square_only else (m, n, ptr, n)
    if kind == "int":
        out = (ctypes.c_uint64 * 2)()
        getattr(lib, "%s_i128" % base)(*args, *extra, out)
        return _i128(out)
    if prec not in ("ld", "f64"):
        raise ValueError("prec must be 'ld' or 'f64'")
    if kind == "complex":
        out = (ctypes.c_double * 4)()
        getattr(lib, "%s_c_%s" % (base, prec))(*args, *extra, out)
        return _cplx(out, dd)
    out = (ctypes.c_double * 2)()
    getattr(lib, "%s_%s" % (base, prec))(*args, *extra, out)
    return _real(out, dd)


def definition(A, prec: str = "ld", dd: bool = False):
    """Sum over m-permutations of the products (Eq. rectangular_permanent_definition). Tiny n only."""
    return _call("oracle_definition", A, prec, dd)


def combinatoric(A, prec: str = "ld", dd: bool = False):
    """The combinatoric algorithm is the definition evaluated directly (cost O(m n!/(n-m)!))."""
    return definition(A, prec, dd)


def glynn(A, prec: str = "ld", dd: bool = False):
    """Glynn with the rectangular padding (Eq. glynn_rectangle; appendix Glynn algorithms)."""
    return _call("oracle_glynn", A, prec, dd)


def glynn_partial(A, g0: int, g1: int, prec: str = "ld", dd: bool = False):
    """Unnormalised sum of Glynn terms g0 <= g < g1 (term g uses delta from gray(g) = g ^ (g >> 1),
    bit b <-> row n-1-b, sign (-1)^g).  Integer input returns the sum modulo 2^128 as a signed int."""
    A_, kind, m, n = _prepare(A)
    if not (0 <= g0 <= g1 <= (1 << (n - 1))):
        raise ValueError("term range outside [0, 2^(n-1)]")
    return _call("oracle_glynn_partial", A_, prec, dd, extra=(g0, g1))


def glynn_partial_abs(A, g0: int, g1: int, prec: str = "ld") -> float:
    """Sum of |term| over the Glynn terms g0 <= g < g1 (real or complex input; complex
    terms by their modulus): the scale of the rounding error of any evaluation of that
    partial sum."""
    lib = _load()
    A, kind, m, n = _prepare(A)
    if kind == "int":
        raise TypeError("glynn_partial_abs takes a real or complex matrix")
    if not (0 <= g0 <= g1 <= (1 << (n - 1))):
        raise ValueError("term range outside [0, 2^(n-1)]")
    out = (ctypes.c_double * 2)()
    fn = "oracle_glynn_partial_abs_%s%s" % ("c_" if kind == "complex" else "", prec)
    getattr(lib, fn)(m, n, A.ctypes.data_as(ctypes.c_void_p), n, g0, g1, out)
    return float(out[0]) + float(out[1])


def glynn_abs(A, prec: str = "ld") -> float:
    """Sum of |term| over all 2^(n-1) terms of Eq. glynn_rectangle divided by the
    normalisation 2^(n-1) (n-m)!: the size, in units of per(A), of the terms Glynn's
    formula cancels (real or complex input; 1 for an empty matrix)."""
    A_, kind, m, n = _prepare(A)
    if m == 0:
        return 1.0
    s = glynn_partial_abs(A_, 0, 1 << (n - 1), prec)
    return s / (2.0 ** (n - 1)) / float(np.prod(np.arange(1, n - m + 1, dtype=np.float64)))


def glynn_rect_grouped(A, prec: str = "ld", dd: bool = False):
    """Glynn with the rectangular padding (Eq. glynn_rectangle), the padding sign vectors
    grouped by their number t of -1 signs (weight (-1)^t C(n-m, t)): 2^(m-1) (n-m+1)
    products instead of 2^(n-1).  Real input."""
    A, kind, m, n = _prepare(A)
    if kind != "real":
        raise TypeError("glynn_rect_grouped takes a real matrix")
    return _call("oracle_glynn_rect_grouped", A, prec, dd)


def glynn_rect_grouped_abs(A, prec: str = "ld") -> float:
    """Sum of |term| over all 2^(n-1) terms of Eq. glynn_rectangle (unnormalised), evaluated
    by the grouping of glynn_rect_grouped.  Real or complex input (complex by modulus)."""
    lib = _load()
    A, kind, m, n = _prepare(A)
    if kind == "int":
        raise TypeError("glynn_rect_grouped_abs takes a real or complex matrix")
    if m == 0:
        return 1.0
    out = (ctypes.c_double * 2)()
    fn = "oracle_glynn_rect_grouped_abs_%s%s" % ("c_" if kind == "complex" else "", prec)
    getattr(lib, fn)(m, n, A.ctypes.data_as(ctypes.c_void_p), n, out)
    return float(out[0]) + float(out[1])


def glynn_esym_abs(A, prec: str = "ld") -> float:
    """Scale of the rounding error of Eq. glynn_rectangle with the padding summed in
    closed form, per(A) = 2^-(m-1) sum_delta (prod delta) e_m(c(delta)): the sum over
    the 2^(m-1) sign vectors of e_m(|c|), divided by 2^(m-1) (real or complex input,
    |c| the modulus; equals glynn_abs for a square matrix)."""
    lib = _load()
    A, kind, m, n = _prepare(A)
    if kind == "int":
        raise TypeError("glynn_esym_abs takes a real or complex matrix")
    if m == 0:
        return 1.0
    out = (ctypes.c_double * 2)()
    fn = "oracle_glynn_esym_abs_%s%s" % ("c_" if kind == "complex" else "", prec)
    getattr(lib, fn)(m, n, A.ctypes.data_as(ctypes.c_void_p), n, out)
    return (float(out[0]) + float(out[1])) / 2.0 ** (m - 1)


def ryser_partial(A, g0: int, g1: int, prec: str = "ld") -> float:
    """Weighted Ryser sum over the Gray-ordered column subsets g0 <= g < g1 (real input)."""
    lib = _load()
    A, kind, m, n = _prepare(A)
    if kind != "real":
        raise TypeError("ryser_partial takes a real matrix")
    if not (0 <= g0 <= g1 <= (1 << n)):
        raise ValueError("subset range outside [0, 2^n]")
    out = (ctypes.c_double * 2)()
    getattr(lib, "oracle_ryser_partial_%s" % prec)(m, n, A.ctypes.data_as(ctypes.c_void_p), n, g0, g1, out)
    return float(out[0]) + float(out[1])


def ryser_partial_abs(A, g0: int, g1: int, prec: str = "ld") -> float:
    """Sum of |weight * prod_i rowsum_i| over the Gray-ordered column subsets g0 <= g < g1
    (the terms of ryser_partial; real or complex input, complex by modulus)."""
    lib = _load()
    A, kind, m, n = _prepare(A)
    if kind == "int":
        raise TypeError("ryser_partial_abs takes a real or complex matrix")
    if not (0 <= g0 <= g1 <= (1 << n)):
        raise ValueError("subset range outside [0, 2^n]")
    out = (ctypes.c_double * 2)()
    fn = "oracle_ryser_partial_abs_%s%s" % ("c_" if kind == "complex" else "", prec)
    getattr(lib, fn)(m, n, A.ctypes.data_as(ctypes.c_void_p), n, g0, g1, out)
    return float(out[0]) + float(out[1])


def ryser_abs(A, prec: str = "ld") -> float:
    """Sum of |term| over all terms of Ryser's formula (Eq. ryser_square; for m < n the
    subset-size form of Eq. ryser_rectangle with weights C(n-s, m-s)): the size of the
    terms Ryser's sum cancels (real or complex input; 1 for an empty matrix)."""
    A_, kind, m, n = _prepare(A)
    if m == 0:
        return 1.0
    if kind == "real" and m < n:
        # by subset size (combinations), as the rectangular appendix algorithm visits them
        out = (ctypes.c_double * 2)()
        getattr(_load(), "oracle_ryser_rect_abs_%s" % prec)(m, n, A_.ctypes.data_as(ctypes.c_void_p), n, out)
        return float(out[0]) + float(out[1])
    return ryser_partial_abs(A_, 0, 1 << n, prec)


def definition_abs(A, prec: str = "ld") -> float:
    """Sum of |term| over the terms of the definition (Eq.
    rectangular_permanent_definition), i.e. per(|A|) with |A| the entrywise modulus;
    every term of per(|A|) is nonnegative, so Glynn's sum of |A| evaluates it with
    little cancellation."""
    A = np.abs(np.asarray(A)).astype(np.float64)
    if min(A.shape) == 0:
        return 1.0
    return float(glynn(A, prec))


def ryser_square(A, prec: str = "ld", dd: bool = False):
    """Square Ryser over all 2^n column subsets (Eq. ryser_square; appendix algorithm)."""
    return _call("oracle_ryser_square", A, prec, dd, square_only=True)


def ryser_rect(A, prec: str = "ld", dd: bool = False):
    """Rectangular Ryser over column combinations with binomial weights (Eq. ryser_rectangle)."""
    return _call("oracle_ryser_rect", A, prec, dd)


def ryser(A, prec: str = "ld", dd: bool = False):
    A = np.asarray(A)
    return ryser_square(A, prec, dd) if A.shape[0] == A.shape[1] else ryser_rect(A, prec, dd)


def subset_dp(A) -> int:
    """Exact integer permanent by the column-subset dynamic programme (n <= 28)."""
    lib = _load()
    A, kind, m, n = _prepare(A)
    if kind != "int":
        raise TypeError("subset_dp is for integer matrices")
    if m == 0:
        return 1
    out = (ctypes.c_uint64 * 2)()
    rc = lib.oracle_subset_dp_i128(m, n, A.ctypes.data_as(ctypes.c_void_p), n, out)
    if rc != 0:
        raise MemoryError("subset DP table unavailable for n=%d" % n)
    return _i128(out)


def glynn_flips(n: int) -> list:
    """Rows flipped, step by step, by the focus-pointer generator of the Glynn algorithms."""
    lib = _load()
    cap = max(1, (1 << (n - 1)) - 1)
    buf = (ctypes.c_int * cap)()
    cnt = lib.oracle_glynn_flips(n, buf, cap)
    return [buf[i] for i in range(cnt)]


def digits_lost(evaluated, true, macheps: float = np.finfo(np.float64).eps) -> float:
    """Digits of precision lost (Eq. digits_lost): log10(|eval-true|/|true|) - log10(macheps)."""
    err = abs(evaluated - true)
    if err == 0:
        return -np.inf
    return float(np.log10(err / abs(true)) - np.log10(macheps))


def sbp_selection_matrix(occ: int, N: int, n: int) -> np.ndarray:
    """The N x n selection matrix P of an occupation bitstring (bit j of ``occ`` = m_j,
    state j occupied): P[j, k] = 1 when m_j = 1 and j is the k-th occupied state
    (Eq. SBGpermanent and the definition of p that precedes it).  Raises unless exactly
    n states are occupied."""
    P = np.zeros((N, n), dtype=np.int64)
    k = 0
    for j in range(N):
        if (occ >> j) & 1:
            if k == n:
                raise ValueError("more than n occupied states")
            P[j, k] = 1
            k += 1
    if k != n:
        raise ValueError("fewer than n occupied states")
    return P


def sbp_coefficient(C, occ: int, prec: str = "ld"):
    """Coefficient of the occupation bitstring ``occ`` in the symmetric product of
    bosons built from the n x N coefficient matrix C (Eq. SBP): c_m = per(C P), with P
    the selection matrix above (Eq. SBGpermanent).  C P is formed by a matrix product."""
    C = np.asarray(C)
    n, N = C.shape
    P = sbp_selection_matrix(int(occ), N, n)
    M = C @ P.astype(C.dtype)
    return glynn(M, prec)


def _gaussian(re, im):
    re = np.asarray(re, dtype=np.int64)
    im = np.asarray(im, dtype=np.int64)
    if re.shape != im.shape or re.ndim != 2:
        raise ValueError("real and imaginary parts must be equal-shaped matrices")
    if re.shape[0] > re.shape[1]:
        re, im = re.T, im.T
    A = np.ascontiguousarray(np.stack([re, im], axis=-1))
    return A, A.shape[0], A.shape[1]


def _call_gaussian(name, re, im, extra=()):
    lib = _load()
    A, m, n = _gaussian(re, im)
    if m == 0:
        return (1, 0)
    if n > MAX_N:
        raise ValueError("the oracle handles n <= %d" % MAX_N)
    out = (ctypes.c_uint64 * 4)()
    getattr(lib, name)(m, n, A.ctypes.data_as(ctypes.c_void_p), n, *extra, out)
    return (_i128(out[0:2]), _i128(out[2:4]))


def definition_gaussian(re, im):
    """Permanent of the Gaussian-integer matrix re + i im by the definition (Eq.
    rectangular_permanent_definition), exact in wrapping 128-bit integers: (re, im)."""
    return _call_gaussian("oracle_definition_ci128", re, im)


def glynn_gaussian(re, im):
    """Glynn (Eq. glynn_rectangle; the appendix algorithms) for the Gaussian-integer
    matrix re + i im, exact in wrapping 128-bit integers: (re, im) Python ints."""
    return _call_gaussian("oracle_glynn_ci128", re, im)


def glynn_partial_gaussian(re, im, g0: int, g1: int):
    """Unnormalised Glynn sum over terms g0 <= g < g1 of re + i im, modulo 2^128 (signed)."""
    return _call_gaussian("oracle_glynn_partial_ci128", re, im, extra=(g0, g1))


# Exact rational permanents of Cauchy matrices (Eq. caucy_permanent), pure Python.
from . import cauchy  # noqa: E402,F401
