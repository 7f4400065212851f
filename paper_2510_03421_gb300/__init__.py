"""GB300 permanent library: Glynn / Ryser Gray-code sweeps, the combinatoric
algorithm, a batched launcher, SBP coefficients, Cauchy permanents by Borchardt's
theorem and a learned dispatcher, behind the C ABI of ``include/perm.h``.  ``capi``
is the ctypes binding; ``inputs`` holds the seeded workload generators.

The functions of the paper's Python module (its usage section) are here under the
same names: ``combinatoric``, ``glynn``, ``ryser`` and ``opt`` (the cost-model
dispatcher), each with ``_square`` and ``_rectangular`` variants.  Each takes one 2-D
array (NumPy, or a torch tensor on the GPU or the host) and returns the permanent as
a Python number: ``float`` for real input, ``complex`` for complex input and an exact
``int`` for integer input (int128 arithmetic; an input whose exactness cannot be
guaranteed raises ``capi.PermError`` with status PERM_EOVERFLOW)."""

__all__ = ["capi", "inputs", "perm_glynn", "perm_ryser", "perm_combinatoric", "perm_auto", "perm_batched",
           "perm_glynn_partial", "perm_sbp", "perm_cauchy",
           "combinatoric", "glynn", "ryser", "opt",
           "combinatoric_square", "glynn_square", "ryser_square", "opt_square",
           "combinatoric_rectangular", "glynn_rectangular", "ryser_rectangular", "opt_rectangular"]

_CAPI_NAMES = ("perm_glynn", "perm_ryser", "perm_combinatoric", "perm_auto", "perm_batched", "perm_glynn_partial",
               "perm_sbp", "perm_cauchy")
_PAPER_NAMES = {"combinatoric": "perm_combinatoric", "glynn": "perm_glynn", "ryser": "perm_ryser",
                "opt": "perm_auto"}


def _scalar(fn_name, A, shape):
    from . import capi
    m, n = A.shape[0], A.shape[1]
    if shape == "square" and m != n:
        raise ValueError("%s_square: the matrix is %d x %d" % (fn_name, m, n))
    if shape == "rectangular" and m == n:
        raise ValueError("%s_rectangular: the matrix is square" % fn_name)
    out = getattr(capi, _PAPER_NAMES[fn_name])(A)
    if hasattr(out, "is_cuda") and out.is_cuda:
        import torch
        torch.cuda.synchronize(out.device)
    code = capi.dtype_code(A)
    v = capi.value(out, code)
    if code in (capi.PERM_U8, capi.PERM_I64):
        return int(v)
    return complex(v) if code == capi.PERM_C128 else float(v)


def _paper_function(fn_name, shape):
    def f(A):
        return _scalar(fn_name, A, shape)
    f.__name__ = fn_name + ("_" + shape if shape else "")
    f.__doc__ = "per(A) by %s%s, as a Python number." % (
        {"opt": "the cost-model dispatcher"}.get(fn_name, fn_name),
        "" if not shape else " (%s input only)" % shape)
    return f


def __getattr__(name):
    if name in _CAPI_NAMES:
        from . import capi
        return getattr(capi, name)
    for base in _PAPER_NAMES:
        for shape in ("", "square", "rectangular"):
            if name == base + ("_" + shape if shape else ""):
                return _paper_function(base, shape)
    raise AttributeError(name)
