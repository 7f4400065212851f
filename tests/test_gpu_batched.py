"""Parity of perm_batched (persistent size-class kernels in one CUDA graph) with the
long-double CPU oracle and with the single-matrix path.

Tolerance 8 (n + 2) u sum|t| (gpu_util.close; u = 2^-56 for the complex integer-pipe
classes).  The batched kernels evaluate a rectangle by the padded sum of Eq.
glynn_rectangle (Glynn's terms, scale "glynn"), which cancels far more than the
single-matrix closed form on signed rectangles; those checks use that scale."""
import numpy as np
import pytest

import oracle
from gpu_util import U_CFIX, close, device, oracle_many, tol_ratio
from paper_2510_03421_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return device()


@pytest.fixture(scope="module")
def capi():
    from paper_2510_03421_gb300 import capi
    return capi


def pack(mats, dtype):
    offsets = np.zeros(len(mats), dtype=np.int64)
    M = np.array([a.shape[0] for a in mats], dtype=np.int32)
    N = np.array([a.shape[1] for a in mats], dtype=np.int32)
    sizes = np.array([a.size for a in mats], dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)[:-1]
    packed = np.concatenate([np.ascontiguousarray(a, dtype=dtype).reshape(-1) for a in mats] + [np.zeros(1, dtype)])
    return packed, offsets, M, N


def to_torch(dev, *arrs):
    import torch
    return [torch.from_numpy(a).to(dev) for a in arrs]


def results(capi, out, code, count):
    return [capi.value(out, code, i) for i in range(count)]


def mixed_batch(kind, seed, count=160):
    g = inputs.rng(seed)
    mats = []
    for k in range(count):
        m, n = int(g.integers(0, 13)), int(g.integers(1, 13))
        if kind == "real":
            mats.append(g.uniform(-1, 1, (m, n)))
        else:
            mats.append((g.standard_normal((m, n)) + 1j * g.standard_normal((m, n))) / np.sqrt(2 * max(n, 1)))
    return mats


@pytest.mark.parametrize("kind", ["real", "complex"])
def test_mixed_shapes_vs_oracle(capi, dev, kind):
    import torch
    mats = mixed_batch(kind, 9500 if kind == "real" else 9501)
    dt = np.float64 if kind == "real" else np.complex128
    packed, offsets, M, N = pack(mats, dt)
    tp, to, tM, tN = to_torch(dev, packed, offsets, M, N)
    out = capi.perm_batched(tp, to, tM, tN)
    torch.cuda.synchronize(dev)
    code = capi.PERM_F64 if kind == "real" else capi.PERM_C128
    got = results(capi, out, code, len(mats))
    for A, x in zip(mats, got):
        close(x, oracle.glynn(A), A, u=U_CFIX if kind == "complex" else 2.0 ** -53)


def test_haar_blocks_split_items_and_host_buffers(capi, dev):
    import torch
    sizes, packed, offsets = inputs.batched_haar(96, 4, 20, 9601)
    M = sizes.astype(np.int32)
    N = sizes.astype(np.int32)
    tp, to, tM, tN = to_torch(dev, packed, offsets, M, N)
    out = capi.perm_batched(tp, to, tM, tN, opts=dict(chunk_log2=10))
    torch.cuda.synchronize(dev)
    got = results(capi, out, capi.PERM_C128, len(sizes))
    big = [b for b in range(len(sizes)) if sizes[b] > 13][::6]  # a sample of the split matrices
    mat = lambda b: packed[offsets[b]: offsets[b] + sizes[b] * sizes[b]].reshape(sizes[b], sizes[b])
    truth = dict(zip(big, oracle_many("glynn", [mat(b) for b in big])))
    for b, n in enumerate(sizes):
        A = mat(b)
        if n <= 13:
            close(got[b], oracle.glynn(A), A, u=U_CFIX)
        elif b in big:
            close(got[b], truth[b], A, u=U_CFIX)
            assert tol_ratio(truth[b], A, u=U_CFIX) <= 1e-9
    host_out = capi.perm_batched(packed, offsets, M, N)  # numpy in, numpy out: the same computation
    for b in range(len(sizes)):
        assert capi.value(host_out, capi.PERM_C128, b) == got[b]


_truths = {}


def _truth(key, A):
    """Long-double truth, computed once per matrix across the parametrised runs: Glynn
    for squares and near-squares, the by-combination rectangular Ryser otherwise (a
    padded Glynn sum over 2^(n-1) terms in software quad precision takes minutes)."""
    if key not in _truths:
        m, n = sorted(A.shape)
        B = A if A.shape[0] <= A.shape[1] else A.T
        if m == n:
            _truths[key] = oracle.glynn(A)
        elif A.dtype.kind == "f":
            _truths[key] = oracle.glynn_rect_grouped(B)
        else:
            _truths[key] = oracle.ryser_rect(B)
    return _truths[key]


@pytest.mark.parametrize("arith", [0, 1, 2, 3])
def test_complex_warp_classes_integer_pipes_and_fp64(capi, dev, arith):
    # padded orders 16..32 (n = 13..32) are warp items; by default they run on the integer
    # pipes (batched_fx.cu), with opts.arith = FP64 on the FP64 class kernels, with MIXED
    # a share of each product on the FP64 unit, with FIXED without it.  Square,
    # rectangular and transposed shapes, a matrix with a non-finite entry, an empty one.
    import torch
    g = inputs.rng(9650)
    shapes = [(13, 13), (14, 16), (16, 16), (17, 20), (20, 17), (19, 19), (18, 21), (6, 26), (20, 20), (0, 18),
              (12, 18)]
    mats = [(g.standard_normal(s) + 1j * g.standard_normal(s)) / np.sqrt(2 * max(s)) for s in shapes]
    mats[-1][3, 4] = np.nan
    packed, offsets, M, N = pack(mats, np.complex128)
    tp, to, tM, tN = to_torch(dev, packed, offsets, M, N)
    out = capi.perm_batched(tp, to, tM, tN, opts=dict(arith=arith))
    torch.cuda.synchronize(dev)
    got = results(capi, out, capi.PERM_C128, len(mats))
    for k, (A, x) in enumerate(zip(mats[:-1], got[:-1])):
        if min(A.shape) == 0:
            assert x == 1
            continue
        ref = _truth(("c", k), A)
        close(x, ref, A, u=U_CFIX)
        if A.shape[0] == A.shape[1]:
            assert tol_ratio(ref, A, u=U_CFIX) <= 1e-9
    assert np.isnan(got[-1].real) and np.isnan(got[-1].imag)


@pytest.mark.parametrize("arith", [0, 1, 2, 3])
def test_real_warp_classes_integer_pipes_and_fp64(capi, dev, arith):
    # real warp items of padded order 16..32 on the integer pipes (batched_fx.cu) by
    # default, on the FP64 class kernels with opts.arith = FP64; MIXED forces the FP64
    # share of each product, FIXED forbids it
    import torch
    g = inputs.rng(9670)
    shapes = [(13, 13), (14, 16), (16, 16), (17, 20), (20, 17), (19, 19), (21, 23), (6, 26), (22, 22), (0, 18),
              (6, 30), (12, 18)]
    mats = [g.uniform(-1, 1, s) for s in shapes]
    mats[-1][3, 4] = np.inf
    packed, offsets, M, N = pack(mats, np.float64)
    tp, to, tM, tN = to_torch(dev, packed, offsets, M, N)
    out = capi.perm_batched(tp, to, tM, tN, opts=dict(arith=arith))
    torch.cuda.synchronize(dev)
    got = results(capi, out, capi.PERM_F64, len(mats))
    for k, (A, x) in enumerate(zip(mats[:-1], got[:-1])):
        m, n = sorted(A.shape)
        if m == 0:
            assert x == 1.0
            continue
        ref = _truth(("r", k), A)
        close(x, ref, A)
        if m == n:
            assert tol_ratio(ref, A) <= 1e-9
    assert np.isnan(got[-1])


def test_graph_replay_sees_new_data(capi, dev):
    import torch
    mats = [inputs.uniform_real(n, n, 9700 + n) for n in (3, 7, 11, 15, 18)]
    packed, offsets, M, N = pack(mats, np.float64)
    tp, to, tM, tN = to_torch(dev, packed, offsets, M, N)
    out = torch.empty(len(mats), dtype=torch.float64, device=dev)
    capi.perm_batched(tp, to, tM, tN, out=out)
    first = out.cpu().numpy().copy()
    capi.perm_batched(tp, to, tM, tN, out=out)  # replay of the cached graph
    assert np.array_equal(first, out.cpu().numpy())
    tp.mul_(0.5)  # per(c A) = c^n per(A)
    capi.perm_batched(tp, to, tM, tN, out=out)
    torch.cuda.synchronize(dev)
    for k, A in enumerate(mats):
        close(float(out[k].item()), first[k] * 0.5 ** A.shape[0], A)


def test_limits(capi, dev):
    packed, offsets, M, N = pack([np.ones((33, 33))], np.float64)
    with pytest.raises(capi.PermError) as e:
        capi.perm_batched(packed, offsets, M, N)
    assert e.value.status == capi.PERM_ETOOBIG


def test_tuner_keeps_results(capi, dev):
    import torch
    sizes, packed, offsets = inputs.batched_haar(400, 4, 16, 9801)
    M = sizes.astype(np.int32)
    tp, to, tM = to_torch(dev, packed, offsets, M)
    tuned = capi.perm_batched(tp, to, tM, tM, opts=dict(exhaustive=1))  # times settings on a sample
    again = capi.perm_batched(tp, to, tM, tM)  # same sizes: the tuned setting is reused
    torch.cuda.synchronize(dev)
    for b in range(len(sizes)):
        n = int(sizes[b])
        A = packed[offsets[b]: offsets[b] + n * n].reshape(n, n)
        if n <= 12 or b % 10 == 0:
            close(capi.value(tuned, capi.PERM_C128, b), oracle.glynn(A), A, u=U_CFIX)
        # the replayed graph with the kept setting computes the same sums in the same order
        assert capi.value(again, capi.PERM_C128, b) == capi.value(tuned, capi.PERM_C128, b)


def test_bench_batch_full_size_sampled(capi, dev):
    # the bench's batched workload at its full size (100,000 complex Haar blocks, n in
    # 4..20, seed as in bench.py), tuned and then replayed from its CUDA graph as the
    # bench times it; two matrices of every order checked against the oracle one by one
    import torch
    count = 100000
    sizes, packed, offsets = inputs.batched_haar(count, 4, 20, inputs.SEED_BASE + 4)
    M = sizes.astype(np.int32)
    tp, to, tM = to_torch(dev, packed, offsets, M)
    out = torch.empty((count, 2), dtype=torch.float64, device=dev)
    capi.perm_batched(tp, to, tM, tM, out=out, opts=dict(exhaustive=1))
    out.fill_(float("nan"))
    capi.perm_batched(tp, to, tM, tM, out=out)  # graph replay with the tuned settings
    torch.cuda.synchronize(dev)
    got = out.cpu().numpy()
    assert np.all(np.isfinite(got))
    picks = []
    for n in range(4, 21):
        idx = np.nonzero(sizes == n)[0]
        picks += [(n, int(idx[0])), (n, int(idx[-1]))]
    mats = [packed[offsets[b]: offsets[b] + n * n].reshape(n, n) for n, b in picks]
    truths = oracle_many("glynn", mats)  # long double throughout, n = 17..20 included
    for (n, b), A, ref in zip(picks, mats, truths):
        close(complex(got[b, 0], got[b, 1]), ref, A, u=U_CFIX, what="n=%d b=%d" % (n, b))
        assert tol_ratio(ref, A, u=U_CFIX) <= 1e-9


# --- exact integer batches (one warp per matrix, int128)


def int_batch(seed, count, kind):
    g = inputs.rng(seed)
    mats = []
    for k in range(count):
        m, n = int(g.integers(0, 11)), int(g.integers(1, 11))
        if kind == "u8":
            mats.append((g.random((m, n)) < 0.6).astype(np.uint8))
        else:
            mats.append(g.integers(-3, 4, (m, n)).astype(np.int64))
    return mats


@pytest.mark.parametrize("kind", ["u8", "i64"])
def test_integer_batch_exact_against_oracle(capi, dev, kind):
    import torch
    mats = int_batch(9950 if kind == "u8" else 9951, 300, kind)
    dtype = np.uint8 if kind == "u8" else np.int64
    packed, offsets, M, N = pack(mats, dtype)
    tp, to, tM, tN = to_torch(dev, packed, offsets, M, N)
    out = capi.perm_batched(tp, to, tM, tN)
    torch.cuda.synchronize(dev)
    code = capi.PERM_U8 if kind == "u8" else capi.PERM_I64
    got = results(capi, out, code, len(mats))
    for b, A in enumerate(mats):
        want = oracle.glynn(A.astype(np.int64))
        assert got[b] == want, (b, A.shape, got[b], want)
    host = capi.perm_batched(packed, offsets, M, N)  # host buffers: same results
    assert results(capi, host, code, len(mats)) == got


def test_integer_batch_larger_orders_and_closed_forms(capi, dev):
    import math
    import torch
    g = inputs.rng(9960)
    mats = [np.ones((24, 24), np.uint8), np.ones((12, 20), np.uint8), np.ones((20, 12), np.uint8)]
    blocks = [(g.random((8, 8)) < 0.5).astype(np.uint8) for _ in range(2)]
    bd = np.zeros((16, 16), np.uint8)  # block diagonal: the product of the blocks' permanents
    bd[:8, :8], bd[8:, 8:] = blocks
    mats.append(bd)
    for n in (14, 18, 20):
        mats.append((g.random((n, n)) < 0.5).astype(np.uint8))
    packed, offsets, M, N = pack(mats, np.uint8)
    tp, to, tM, tN = to_torch(dev, packed, offsets, M, N)
    out = capi.perm_batched(tp, to, tM, tN)
    torch.cuda.synchronize(dev)
    got = results(capi, out, capi.PERM_U8, len(mats))
    assert got[0] == math.factorial(24)
    assert got[1] == math.factorial(20) // math.factorial(8) == got[2]
    assert got[3] == oracle.subset_dp(blocks[0].astype(np.int64)) * oracle.subset_dp(blocks[1].astype(np.int64))
    for b in range(4, len(mats)):
        assert got[b] == oracle.subset_dp(mats[b].astype(np.int64))


def test_integer_batch_range_check(capi, dev):
    import torch
    big = np.full((6, 6), 10 ** 12, dtype=np.int64)  # 2^5 6! 1e72 does not fit int128
    small = np.eye(3, dtype=np.int64)
    packed, offsets, M, N = pack([small, big], np.int64)
    with pytest.raises(capi.PermError) as e:
        capi.perm_batched(packed, offsets, M, N)  # host output: the status comes back
    assert e.value.status == capi.PERM_EOVERFLOW
    stream = torch.cuda.current_stream(dev).cuda_stream
    st = capi.ctypes.c_int(-1)
    assert capi.lib().perm_device_status(capi.handle(0), stream, capi.ctypes.byref(st)) == capi.PERM_OK
    tp, to, tM, tN = to_torch(dev, packed, offsets, M, N)
    out = capi.perm_batched(tp, to, tM, tN)
    assert capi.lib().perm_device_status(capi.handle(0), stream, capi.ctypes.byref(st)) == capi.PERM_OK
    assert st.value == capi.PERM_EOVERFLOW
    assert capi.value(out, capi.PERM_I64, 0) == 1
    g = np.zeros((1, 33), np.uint8)
    p2, o2, M2, N2 = pack([g], np.uint8)
    with pytest.raises(capi.PermError) as e:
        capi.perm_batched(p2, o2, M2, N2)
    assert e.value.status == capi.PERM_ETOOBIG
