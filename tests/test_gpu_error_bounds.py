"""The stated error bound (opts.err) holds where rounding is normwise, not termwise:
column sums that cancel (a column of ones and -(n-1), plus tiny noise), entries that
span 2^-30 .. 2^30 within one column (their rounding to fixed point is inexact), and
the identity padded with zero columns.  Every arithmetic that states a bound is
checked against the exact permanent (oracle.exact: the matrix as integers times a
power of two, summed without rounding; a long-double sum would itself be off on the
2^+-30 entries): |got - exact| <= err."""
import numpy as np
import pytest

from gpu_util import device, to_dev
from oracle import exact
from paper_2510_03421_gb300 import inputs

pytestmark = pytest.mark.gpu

GLYNN_ARITH = {"auto": dict(arith=0), "fp64": dict(arith=1), "fixed": dict(arith=2), "mixed": dict(arith=3),
               "fp64_tensor_core_start": dict(arith=1, start=2)}


@pytest.fixture(scope="module")
def dev():
    return device()


@pytest.fixture(scope="module")
def capi():
    from paper_2510_03421_gb300 import capi
    return capi


def cancelling(n, seed, m=None):
    """m x n uniform[-1,1] whose column 1 is (1, ..., 1, -(m-1)) + noise of 1e-12: its
    column sums cancel to about 1e-12 of the column's absolute sum for half the signs."""
    m = m or n
    g = inputs.rng(seed)
    A = g.uniform(-1, 1, (m, n))
    A[:, 1] = 1.0
    A[m - 1, 1] = -(m - 1.0)
    A[:, 1] += 1e-12 * g.uniform(-1, 1, m)
    return A


def wide_range(m, n, seed):
    g = inputs.rng(seed)
    return g.uniform(-1, 1, (m, n)) * np.exp2(g.integers(-30, 31, (m, n)))


def padded_identity(m, n):
    A = np.zeros((m, n))
    A[np.arange(m), np.arange(m)] = 1.0
    return A


def bounded(capi, dev, fn, A, opts):
    import torch
    err = torch.full((1,), -2.0, dtype=torch.float64, device=dev)
    out = getattr(capi, fn)(to_dev(A, dev), opts=dict(opts, err=err))
    torch.cuda.synchronize(dev)
    return capi.value(out, capi.PERM_F64), float(err.item())


_exact = {}


def truth(name, A):
    if name not in _exact:
        _exact[name] = float(exact.glynn_rect_grouped(A, workers=8 if min(A.shape) > 12 else 1))
    return _exact[name]


CASES = [("cancel 12", lambda: cancelling(12, 501)), ("cancel 18", lambda: cancelling(18, 502)),
         ("cancel 9x14", lambda: cancelling(14, 503, m=9)), ("wide 12", lambda: wide_range(12, 12, 504)),
         ("wide 16", lambda: wide_range(16, 16, 505)), ("wide 7x13", lambda: wide_range(7, 13, 506)),
         ("identity 6x13", lambda: padded_identity(6, 13)), ("identity 10x12", lambda: padded_identity(10, 12))]


@pytest.mark.parametrize("arith", sorted(GLYNN_ARITH))
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_glynn_bound_holds(capi, dev, arith, name, make):
    A = make()
    ref = truth(name, A)
    got, err = bounded(capi, dev, "perm_glynn", A, GLYNN_ARITH[arith])
    assert err >= 0.0, "no bound stated"
    assert abs(got - ref) <= err, (name, arith, got, ref, abs(got - ref), err)


@pytest.mark.parametrize("arith", [0, 1, 2])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_ryser_bound_holds(capi, dev, arith, name, make):
    A = make()
    ref = truth(name, A)
    got, err = bounded(capi, dev, "perm_ryser", A, dict(arith=arith))
    if err < 0.0:
        pytest.skip("this Ryser path states no bound")
    assert abs(got - ref) <= err, (name, arith, got, ref, abs(got - ref), err)


def test_bound_is_tight_on_well_conditioned_input(capi, dev):
    # on a random matrix the bound stays a small multiple of the rounding scale (the
    # FP64 sweep's includes the drift of its column sums over 2^8-term chunks)
    A = inputs.uniform_real(16, 16, 507)
    ref = truth("uniform 16", A)
    for arith, limit in ((0, 1e-10), (1, 1e-9), (2, 1e-10), (3, 1e-10)):
        got, err = bounded(capi, dev, "perm_glynn", A, dict(arith=arith))
        assert abs(got - ref) <= err <= limit * abs(ref), (arith, err / abs(ref))


def complex_cancelling(n, seed):
    g = inputs.rng(seed)
    A = g.uniform(-1, 1, (n, n)) + 1j * g.uniform(-1, 1, (n, n))
    A[:, 1] = 1.0 + 1.0j
    A[n - 1, 1] = -(n - 1.0) * (1.0 + 1.0j)
    A[:, 1] += 1e-12 * (g.uniform(-1, 1, n) + 1j * g.uniform(-1, 1, n))
    return A


def complex_wide(n, seed):
    g = inputs.rng(seed)
    return (g.uniform(-1, 1, (n, n)) + 1j * g.uniform(-1, 1, (n, n))) * np.exp2(g.integers(-30, 31, (n, n)))


@pytest.mark.parametrize("name,make", [("cancel c8", lambda: complex_cancelling(8, 511)),
                                       ("wide c7", lambda: complex_wide(7, 512)),
                                       ("identity c6x9", lambda: padded_identity(6, 9) + 0j)],
                         ids=["cancel c8", "wide c7", "identity c6x9"])
def test_complex_glynn_bound_holds(capi, dev, name, make):
    # a complex call that asks for a bound takes the FP64 sweep; the bound covers the
    # modulus of the error
    import torch
    A = make()
    re, im = exact.definition(A)
    ref = complex(float(re), float(im))
    err = torch.full((1,), -2.0, dtype=torch.float64, device=dev)
    out = capi.perm_glynn(to_dev(A, dev), opts=dict(err=err))
    torch.cuda.synchronize(dev)
    got = capi.value(out, capi.PERM_C128)
    e = float(err.item())
    assert e >= 0.0 and abs(got - ref) <= e, (name, got, ref, abs(got - ref), e)
