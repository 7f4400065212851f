"""Helpers shared by the GPU parity tests (device, marshalling, tolerances).

Float tolerances.  A sum of terms t_g evaluated with a unit roundoff u per operation
has an error of at most about c u sum_g |t_g|, whatever order the terms are added in;
that sum of |term| is the scale the tolerance is built on, taken from the oracle for
the term set of the algorithm the kernel runs:

* ``scale(A, "glynn")``: Glynn's terms (Eq. glynn_rectangle, ungrouped), normalised by
  2^(n-1) (n-m)!;
* ``scale(A, "esym")``: the rectangular sum with the padding in closed form (the
  rectangles the integer pipes take, real and complex; see ``default_kind``);
* ``scale(A, "ryser")``: Ryser's weighted subset terms;
* ``scale(A, "definition")``: per(|A|), the terms of the combinatoric algorithm.

``close`` asserts |got - ref| <= max(rel |ref|, c (n + 2) u scale) and prints the
tolerance relative to |ref| on failure.  ``u`` is 2^-53 for the FP64 pipe and 2^-60 for
the integer-pipe arithmetic (its column sums are exact and its products keep at least
60 bits).  The truths are long-double oracle values: no test takes the double-precision
oracle (the timed CPU baseline) as its truth.  The scales need only a couple of correct
digits, so they are summed in double.
"""
import math
import os

import numpy as np

U = np.finfo(np.float64).eps / 2   # FP64 unit roundoff, 2^-53
U_FIX = 2.0 ** -60                 # integer-pipe arithmetic, per operation
U_CFIX = 2.0 ** -56                # complex integer-pipe arithmetic (four truncated products each)
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

_scale_cache = {}


def device():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch.device("cuda:0")


def to_dev(A, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(A)).to(dev)


def run(capi, fn, A, dev, opts=None):
    """Call capi.<fn> on a device copy of A and return the Python value."""
    import torch
    dA = to_dev(A, dev)
    out = getattr(capi, fn)(dA, opts=opts)
    torch.cuda.synchronize(dev)
    return capi.value(out, capi.dtype_code(dA))


def _shape(A):
    A = np.asarray(A)
    m, n = sorted(A.shape)
    return m, n


def scale(A, kind="glynn"):
    """Normalised sum of |term| of the algorithm `kind` on A (see the module docstring)."""
    import oracle
    A = np.asarray(A)
    if A.shape[0] > A.shape[1]:
        A = A.T
    A = np.ascontiguousarray(A)
    key = (kind, A.shape, A.dtype.str, hash(A.tobytes()))
    if key in _scale_cache:
        return _scale_cache[key]
    m, n = A.shape
    if m == 0:
        s = 1.0
    elif kind == "glynn":
        if m < n:
            # the grouped evaluation of the same sum of |term| (cheap for small m)
            s = oracle.glynn_rect_grouped_abs(A, prec="f64") / (2.0 ** (n - 1) * math.factorial(n - m))
        else:
            s = oracle.glynn_abs(A, prec="f64")
    elif kind == "esym":
        s = oracle.glynn_esym_abs(A, prec="f64") if m < n else oracle.glynn_abs(A, prec="f64")
    elif kind == "ryser":
        s = oracle.ryser_abs(A, prec="f64")
    elif kind == "definition":
        s = oracle.definition_abs(A, prec="f64")
    else:
        raise ValueError(kind)
    _scale_cache[key] = s
    return s


def default_kind(A, arith=0):
    """Term set perm_glynn evaluates for A with opts.arith = arith (0 AUTO, 1 FP64, 2
    FIXED, 3 MIXED): the integer pipes (FIXED, MIXED, or AUTO from n = 10) take the
    closed-form padding sum for the rectangles m <= 32 with n - m >= 3 or m <= 8 (real)
    and every complex rectangle m <= 32; everything else evaluates Glynn's terms."""
    A = np.asarray(A)
    m, n = _shape(A)
    if arith == 1 or not (arith in (2, 3) or n >= 10) or m >= n or m > 32:
        return "glynn"
    if A.dtype.kind == "c" or n - m >= 3 or m <= 8:
        return "esym"
    return "glynn"


def real_default_kind(A):
    """default_kind on the integer pipes (FIXED / MIXED / AUTO from n = 10)."""
    return default_kind(A, arith=2)


def auto_scale(capi, A, dev, exhaustive=False):
    """(scale, u) for perm_auto on A: the term set of the candidate perm_auto_choice
    names, or, when the choice is made by timing (exhaustive), the largest scale over
    the candidates."""
    A = np.asarray(A)
    cplx = A.dtype.kind == "c"
    kinds = {capi.PERM_CAND_COMBINATORIC: ("definition", U), capi.PERM_CAND_RYSER: ("ryser", U),
             capi.PERM_CAND_GLYNN: (default_kind(A, 0) if cplx else "glynn", U_CFIX if cplx else U),
             capi.PERM_CAND_GLYNN_FIXED: (default_kind(A, 3), U),
             capi.PERM_CAND_RYSER_FP64: ("ryser", U), capi.PERM_CAND_GLYNN_DMMA: ("glynn", U),
             capi.PERM_CAND_GLYNN_INT: (default_kind(A, 2), U),
             capi.PERM_CAND_GLYNN_SHORT: ("glynn" if cplx else default_kind(A, 3), U)}
    if exhaustive:
        return max(scale(A, k) for k, _ in kinds.values()), max(u for _, u in kinds.values())
    cand, _ = capi.perm_auto_choice(to_dev(A, dev))
    k, u = kinds.get(cand, ("glynn", U))
    return scale(A, k), u


def tolerance(ref, A, kind="glynn", rel=1e-12, c=8, u=U, s=None):
    m, n = _shape(A)
    if s is None:
        s = scale(A, kind)
    return max(rel * abs(ref), c * (n + 2) * u * s)


def close(got, ref, A, rel=1e-12, c=8, kind="glynn", u=U, s=None, what=""):
    """|got - ref| <= max(rel |ref|, c (n+2) u scale(A, kind)); the message gives the
    tolerance in units of |ref| (a tolerance near or above |ref| would make the check
    unable to fail)."""
    tol = tolerance(ref, A, kind, rel, c, u, s)
    err = abs(got - ref)
    assert err <= tol, "%s got %r ref %r |err| %.3g tol %.3g tol/|ref| %.3g err/|ref| %.3g" % (
        what, got, ref, err, tol, tol / abs(ref) if ref else float("inf"), err / abs(ref) if ref else float("inf"))
    return tol


def tol_ratio(ref, A, **kw):
    """The tolerance close() would use, in units of |ref|."""
    t = tolerance(ref, A, **kw)
    return t / abs(ref) if ref else float("inf")


def _oracle_call(args):
    import oracle
    name, A = args
    return getattr(oracle, name)(A)


def oracle_many(name, mats, workers=None):
    """oracle.<name>(A) for every A in mats, in long double, spread over a pool of
    spawned processes (the oracle is serial; large complex Glynn sums take seconds each
    where long double is software quad precision)."""
    import multiprocessing
    mats = [np.ascontiguousarray(A) for A in mats]
    if len(mats) <= 1:
        return [_oracle_call((name, A)) for A in mats]
    workers = workers or min(len(mats), os.cpu_count() or 1)
    with multiprocessing.get_context("spawn").Pool(workers) as pool:
        return pool.map(_oracle_call, [(name, A) for A in mats])


def read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, *v = line.split()
            vals[k] = v
    return vals
