"""Exact permanents of Gaussian-integer matrices (dtype PERM_CI64): bit-exact against
the oracle's 128-bit Glynn / definition, closed forms, partial sums modulo 2^128 at
full size, the overflow check and the entry points that refuse the dtype."""
import ctypes
import math

import numpy as np
import pytest

import oracle
from gpu_util import device
from paper_2510_03421_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return device()


@pytest.fixture(scope="module")
def capi():
    from paper_2510_03421_gb300 import capi
    return capi


def _run(capi, dev, re, im):
    import torch
    out = capi.perm_glynn_gaussian(torch.from_numpy(re).to(dev), torch.from_numpy(im).to(dev))
    torch.cuda.synchronize(dev)
    return capi.value(out, capi.PERM_CI64)


def _wrap(v):
    v &= (1 << 128) - 1
    return v - (1 << 128) if v >> 127 else v


@pytest.mark.parametrize("m,n", [(1, 1), (3, 3), (6, 6), (10, 10), (14, 14), (4, 9), (7, 12), (18, 18)])
def test_exact_against_oracle(capi, dev, m, n):
    g = inputs.rng(8300 + 10 * m + n)
    re, im = g.integers(-3, 4, (m, n)), g.integers(-3, 4, (m, n))
    ref = oracle.glynn_gaussian(re, im)
    assert _run(capi, dev, re, im) == ref
    assert _run(capi, dev, np.ascontiguousarray(re.T), np.ascontiguousarray(im.T)) == ref
    if n <= 7:
        assert oracle.definition_gaussian(re, im) == ref


def test_closed_forms_and_host_buffers(capi, dev):
    n = 12
    ones = np.ones((n, n), dtype=np.int64)
    w = (1 + 1j) ** n * math.factorial(n)
    assert _run(capi, dev, ones, ones) == (int(w.real), int(w.imag))
    g = inputs.rng(8310)
    A = g.integers(-4, 5, (9, 9))
    p = oracle.glynn(A)
    Z = np.zeros_like(A)
    assert _run(capi, dev, A, Z) == (p, 0)
    assert _run(capi, dev, Z, A) == (0, p)  # per(i A) = i^9 per(A) = i per(A)
    out = capi.perm_glynn_gaussian(A, Z)  # numpy in, numpy out
    assert isinstance(out, np.ndarray) and capi.value(out, capi.PERM_CI64) == (p, 0)


@pytest.mark.parametrize("n", [26, 32])
def test_partial_sums_modulo_2_128(capi, dev, n):
    import torch
    g = inputs.rng(8320 + n)
    re, im = g.integers(-2, 3, (n, n)), g.integers(-2, 3, (n, n))
    T = 1 << (n - 1)
    dre, dim = torch.from_numpy(re).to(dev), torch.from_numpy(im).to(dev)
    for a, b in ((0, 3000), (T // 3, T // 3 + 2500), (T - 2047, T)):
        out = capi.perm_glynn_partial_gaussian(dre, dim, a, b)
        torch.cuda.synchronize(dev)
        got = capi.value(out, capi.PERM_CI64)
        ref = oracle.glynn_partial_gaussian(re, im, a, b)
        assert got == (_wrap(ref[0]), _wrap(ref[1]))


def test_overflow_and_refusals(capi, dev):
    big = np.full((20, 20), 1 << 40, dtype=np.int64)
    with pytest.raises(capi.PermError) as e:
        capi.perm_glynn_gaussian(big, big, out=np.zeros(4, dtype=np.int64))
    assert e.value.status == capi.PERM_EOVERFLOW
    with pytest.raises(capi.PermError) as e:
        capi.perm_glynn_gaussian(np.ones((33, 33), np.int64), np.ones((33, 33), np.int64))
    assert e.value.status == capi.PERM_ETOOBIG
    G = np.ones((4, 4, 2), dtype=np.int64)
    out = np.zeros(4, dtype=np.int64)
    L = capi.lib()
    h = capi.handle(0)
    # perm_auto takes Glynn, the one algorithm for Gaussian integers: per(J_4 (1 + i)) = 24 (1 + i)^4
    assert L.perm_auto(h, G.ctypes.data, 4, 4, 4, capi.PERM_CI64, out.ctypes.data, None, None) == capi.PERM_OK
    assert capi.value(out, capi.PERM_CI64) == (-96, 0)


def test_gaussian_batch_exact_against_oracle(capi, dev):
    # perm_batched with PERM_CI64: one warp per matrix, two int128 parts per result
    import torch
    g = inputs.rng(9970)
    mats = []
    for k in range(120):
        m, n = int(g.integers(0, 10)), int(g.integers(1, 10))
        mats.append((g.integers(-2, 3, (m, n)), g.integers(-2, 3, (m, n))))
    mats.append((np.ones((16, 16), np.int64), np.zeros((16, 16), np.int64)))  # per = 16!
    offsets = np.zeros(len(mats), np.int64)
    offsets[1:] = np.cumsum([re.size for re, _ in mats])[:-1]
    packed = np.concatenate([np.stack([re, im], -1).reshape(-1) for re, im in mats] + [np.zeros(2, np.int64)])
    M = np.array([re.shape[0] for re, _ in mats], np.int32)
    N = np.array([re.shape[1] for re, _ in mats], np.int32)
    tp, to, tM, tN = (torch.from_numpy(a).to(dev) for a in (packed, offsets, M, N))
    out = capi.perm_batched_gaussian(tp, to, tM, tN)
    torch.cuda.synchronize(dev)
    for b, (re, im) in enumerate(mats):
        assert capi.value(out, capi.PERM_CI64, b) == oracle.glynn_gaussian(re, im), (b, re.shape)
    assert capi.value(out, capi.PERM_CI64, len(mats) - 1) == (math.factorial(16), 0)
    host = capi.perm_batched_gaussian(packed, offsets, M, N)
    assert all(capi.value(host, capi.PERM_CI64, b) == capi.value(out, capi.PERM_CI64, b) for b in range(len(mats)))


@pytest.mark.parametrize("m,n", [(1, 1), (3, 3), (5, 5), (4, 7), (7, 4), (9, 9), (6, 12), (12, 12)])
def test_gaussian_ryser_and_combinatoric_exact(capi, dev, m, n):
    # Ryser's formula (size weights in int128, complex products modulo 2^128) and the
    # combinatoric algorithm on Gaussian integers against the oracle in the same
    # arithmetic; a third of the entries zero, so the combinatoric search prunes
    g = inputs.rng(9980 + 13 * m + n)
    keep = g.random((m, n)) < 0.67
    re, im = g.integers(-3, 4, (m, n)) * keep, g.integers(-3, 4, (m, n)) * keep
    G = np.ascontiguousarray(np.stack([re, im], -1).astype(np.int64))
    want = oracle.glynn_gaussian(re, im)
    for name in ("perm_ryser", "perm_combinatoric"):
        if name == "perm_combinatoric" and max(m, n) > 9:
            continue
        out = np.zeros(4, dtype=np.int64)
        rc = getattr(capi.lib(), name)(capi.handle(0), G.ctypes.data, m, n, n, capi.PERM_CI64, out.ctypes.data,
                                       None, None)
        assert rc == capi.PERM_OK, name
        assert capi.value(out, capi.PERM_CI64) == want, name


def test_integer_combinatoric_range_check(capi, dev):
    # the combinatoric sum is exact while per(|A|) < 2^126.5: 6! (1e12)^6 is not
    big = np.full((6, 6), 10 ** 12, dtype=np.int64)
    out = np.zeros(2, dtype=np.int64)
    rc = capi.lib().perm_combinatoric(capi.handle(0), big.ctypes.data, 6, 6, 6, capi.PERM_I64, out.ctypes.data, None,
                                      None)
    assert rc == capi.PERM_EOVERFLOW
    ok = np.full((6, 6), 10 ** 5, dtype=np.int64)  # 6! 1e30 < 2^127
    rc = capi.lib().perm_combinatoric(capi.handle(0), ok.ctypes.data, 6, 6, 6, capi.PERM_I64, out.ctypes.data, None,
                                      None)
    assert rc == capi.PERM_OK and capi.value(out, capi.PERM_I64) == 720 * 10 ** 30
