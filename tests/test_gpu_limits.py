"""Maximum sizes and limits through the C ABI: order-64 operands on every sweep (term
ranges at the start, the middle and the end of the 2^63-term index, against the
oracle's partial sums), the refusals past the limits, and the empty matrix."""
import numpy as np
import pytest

import oracle
from gpu_util import U, U_CFIX, close, default_kind, device, to_dev
from paper_2510_03421_gb300 import inputs

pytestmark = pytest.mark.gpu

T64 = 1 << 63


@pytest.fixture(scope="module")
def dev():
    return device()


@pytest.fixture(scope="module")
def capi():
    from paper_2510_03421_gb300 import capi
    return capi


def _ranges():
    return ((0, 2048), (T64 // 3, T64 // 3 + 1500), (T64 - 1777, T64))


@pytest.mark.parametrize("arith", [1, 2, 3])
def test_order_64_real_partials(capi, dev, arith):
    import torch
    A = inputs.uniform_real(64, 64, 8100)
    for a, b in _ranges():
        out = capi.perm_glynn_partial(to_dev(A, dev), a, b, opts=dict(arith=arith))
        torch.cuda.synchronize(dev)
        got = capi.dd_value(out)
        ref = oracle.glynn_partial(A, a, b)
        scale = oracle.glynn_partial_abs(A, a, b)
        # FP64 sweep: 2n + 4 roundings per term; the integer pipes are tighter
        assert abs(got - ref) <= max(1e-13 * abs(ref), 140 * 2.0 ** -53 * scale)


def test_order_64_complex_and_integer_partials(capi, dev):
    import torch
    C = inputs.complex_gaussian(64, 64, 8101)
    for a, b in _ranges():
        out = capi.perm_glynn_partial(to_dev(C, dev), a, b)
        torch.cuda.synchronize(dev)
        o = out.cpu().numpy()
        got = complex(o[0] + o[1], o[2] + o[3])
        ref = oracle.glynn_partial(C, a, b)
        assert abs(got - ref) <= 1e-11 * abs(ref)
    B = inputs.bernoulli01(64, 64, 8102)
    for a, b in _ranges():
        out = capi.perm_glynn_partial(to_dev(B, dev), a, b)
        torch.cuda.synchronize(dev)
        assert capi.value(out, capi.PERM_I64) == oracle.glynn_partial(B.astype(np.int64), a, b)


def test_limits_and_empty(capi, dev):
    import torch
    # more than 64 rows or columns
    with pytest.raises(capi.PermError) as e:
        capi.perm_glynn(np.ones((65, 65)))
    assert e.value.status == capi.PERM_ETOOBIG
    # 2^63 terms: above the default work cap, refused before any launch
    with pytest.raises(capi.PermError) as e:
        capi.perm_glynn(to_dev(inputs.uniform_real(64, 64, 8103), dev))
    assert e.value.status == capi.PERM_ETOOBIG
    # a term range past the end of the index
    with pytest.raises(capi.PermError) as e:
        capi.perm_glynn_partial(to_dev(inputs.uniform_real(10, 10, 8104), dev), 0, (1 << 9) + 1)
    assert e.value.status == capi.PERM_EINVAL
    # per(0 x n) = 1 on every entry point
    for fn in ("perm_glynn", "perm_ryser", "perm_combinatoric", "perm_auto"):
        out = getattr(capi, fn)(torch.zeros((0, 5), dtype=torch.float64, device=dev))
        torch.cuda.synchronize(dev)
        assert capi.value(out, capi.PERM_F64) == 1.0, fn


def test_leading_dimension_larger_than_n(capi, dev):
    # a column slice of a wider matrix: rows ld = 24 elements apart, read through the strides
    import torch
    g = inputs.rng(8110)
    for big, ref_of in ((g.uniform(-1, 1, (18, 24)), oracle.glynn),
                        (g.uniform(-1, 1, (11, 24)) + 1j * g.uniform(-1, 1, (11, 24)), oracle.glynn),
                        (g.integers(-3, 4, (12, 24)).astype(np.int64), oracle.subset_dp)):
        T = torch.from_numpy(big).to(dev)
        view = T[:, :17] if big.shape[0] <= 17 else T[:, :18]
        assert view.stride(0) == 24
        A = big[:, :view.shape[1]]
        out = capi.perm_glynn(view)
        torch.cuda.synchronize(dev)
        got = capi.value(out, capi.dtype_code(view))
        ref = ref_of(np.ascontiguousarray(A))
        if big.dtype == np.int64:
            assert got == ref
        else:
            cplx = big.dtype.kind == "c"
            close(got, ref, A, rel=1e-12, kind=default_kind(A), u=U_CFIX if cplx else U)
