"""Thin ctypes binding of ``libperm.so`` (declared in ``include/perm.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library.  The functions keep the C names (``perm_glynn``, ``perm_ryser``,
``perm_combinatoric``, ``perm_auto``, ``perm_batched``, ``perm_sbp``,
``perm_cauchy``, ``perm_cauchy_sbp``, ``perm_glynn_partial``; Gaussian integers
through ``perm_glynn_gaussian`` and ``perm_batched_gaussian``) and accept torch
tensors (CUDA or CPU) or numpy arrays; CPU / numpy buffers are passed as host
pointers and the library copies them itself.  If the shared library has not been
built this module raises -- there is no fallback.

Streams: a call given ``stream=`` launches on that stream, and an ``out`` tensor the
binding allocates belongs to that stream too.  The results are written asynchronously:
synchronise that stream (or make the reading stream wait on it) before reading ``out``
from another stream, e.g. with ``.item()`` or ``.cpu()`` on the current one.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libperm.so")

PERM_F64, PERM_C128, PERM_U8, PERM_I64, PERM_CI64 = 0, 1, 2, 3, 4
PERM_OK, PERM_EINVAL, PERM_ETOOBIG, PERM_EOVERFLOW, PERM_ECUDA, PERM_ENOMEM, PERM_EUNSUPPORTED = range(7)
PERM_ARITH_AUTO, PERM_ARITH_FP64, PERM_ARITH_FIXED, PERM_ARITH_MIXED = 0, 1, 2, 3
PERM_START_AUTO, PERM_START_SCALAR, PERM_START_DMMA = 0, 1, 2

EXPORTS = ("perm_create", "perm_destroy", "perm_glynn", "perm_ryser", "perm_combinatoric", "perm_auto",
           "perm_batched", "perm_glynn_partial", "perm_status_string", "perm_version", "perm_probe_rate", "perm_glynn_noalloc", "perm_device_status",
           "perm_auto_features", "perm_mlp_size", "perm_mlp_forward", "perm_mlp_grad", "perm_mlp_train",
           "perm_set_cost_model", "perm_auto_choice", "perm_ryser_partial", "perm_sbp", "perm_cauchy",
           "perm_cauchy_sbp")
(PERM_CAND_COMBINATORIC, PERM_CAND_RYSER, PERM_CAND_GLYNN, PERM_CAND_GLYNN_FIXED, PERM_CAND_RYSER_FP64,
 PERM_CAND_GLYNN_DMMA, PERM_CAND_GLYNN_INT, PERM_CAND_GLYNN_SHORT) = range(8)
PERM_NCAND = 8
PERM_CAND_CAUCHY = 8
PERM_NFEATURES = 12
PROBE_DFMA, PROBE_DMMA, PROBE_IMAD, PROBE_IADD, PROBE_FFMA = range(5)


class PermError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s failed: %s (status %d)" % (where, status_string(status), status))


class perm_opts(ctypes.Structure):
    _fields_ = [("chunk_log2", ctypes.c_int32), ("block", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("arith", ctypes.c_int32), ("start", ctypes.c_int32), ("exhaustive", ctypes.c_int32),
                ("max_terms", ctypes.c_uint64), ("err", ctypes.c_void_p)]


_lib = None
_lock = threading.Lock()
_handles: dict = {}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libperm.so is not built (run __graft_entry__.build() or "
                                   "python -m paper_2510_03421_gb300._build); no CPU fallback exists")
            L = ctypes.CDLL(LIB_PATH)
            vp, i64, i32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64
            L.perm_create.argtypes = [ctypes.POINTER(vp), i32]
            L.perm_destroy.argtypes = [vp]
            for name in ("perm_glynn", "perm_ryser", "perm_combinatoric", "perm_auto"):
                getattr(L, name).argtypes = [vp, vp, i64, i64, i64, i32, vp, vp, ctypes.POINTER(perm_opts)]
            L.perm_glynn_partial.argtypes = [vp, vp, i64, i64, i64, i32, u64, u64, vp, vp, ctypes.POINTER(perm_opts)]
            L.perm_ryser_partial.argtypes = [vp, vp, i64, i64, i64, i32, u64, u64, vp, vp, ctypes.POINTER(perm_opts)]
            L.perm_batched.argtypes = [vp, vp, vp, vp, vp, i64, i32, vp, vp, ctypes.POINTER(perm_opts)]
            L.perm_sbp.argtypes = [vp, vp, i64, i64, i64, i32, vp, i64, vp, vp, ctypes.POINTER(perm_opts)]
            L.perm_cauchy.argtypes = [vp, vp, vp, i64, i64, vp, vp, ctypes.POINTER(perm_opts)]
            L.perm_cauchy_sbp.argtypes = [vp, vp, i64, vp, i64, vp, i64, vp, vp, ctypes.POINTER(perm_opts)]
            L.perm_glynn_noalloc.argtypes = [vp, i64, i64, i64, vp, vp, ctypes.c_int32]
            L.perm_device_status.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int)]
            fp = ctypes.c_void_p
            L.perm_auto_features.argtypes = [i64, i64, ctypes.c_double, i32, fp]
            L.perm_mlp_size.argtypes = [i32, i32, i32, ctypes.POINTER(ctypes.c_int64)]
            L.perm_mlp_forward.argtypes = [fp, i32, i32, i32, fp, i64, fp, vp]
            L.perm_mlp_grad.argtypes = [fp, i32, i32, i32, fp, fp, fp, i64, fp, fp, vp]
            L.perm_mlp_train.argtypes = [fp, fp, fp, i64, i32, i32, i32, i32, i32, ctypes.c_float, u64, fp, fp, vp]
            L.perm_set_cost_model.argtypes = [vp, fp, i32, i32, i32]
            L.perm_auto_choice.argtypes = [vp, vp, i64, i64, i64, i32, ctypes.POINTER(perm_opts),
                                           ctypes.POINTER(ctypes.c_int), fp]
            L.perm_probe_rate.argtypes = [i32, i32, vp, ctypes.POINTER(ctypes.c_double)]
            L.perm_status_string.argtypes = [i32]
            L.perm_status_string.restype = ctypes.c_char_p
            for name in EXPORTS:
                if name != "perm_status_string":
                    getattr(L, name).restype = i32
            _lib = L
    return _lib


def status_string(status: int) -> str:
    return lib().perm_status_string(status).decode()


def handle(device: int = 0):
    with _lock:
        h = _handles.get(device)
    if h is None:
        hv = ctypes.c_void_p()
        rc = lib().perm_create(ctypes.byref(hv), device)
        if rc:
            raise PermError(rc, "perm_create")
        with _lock:
            h = _handles.setdefault(device, hv)
    return h


# ----------------------------------------------------------------------------- marshalling
def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def dtype_code(x) -> int:
    if _is_torch(x):
        import torch
        table = {torch.float64: PERM_F64, torch.complex128: PERM_C128, torch.uint8: PERM_U8,
                 torch.bool: PERM_U8, torch.int64: PERM_I64}
        if x.dtype not in table:
            raise TypeError("unsupported tensor dtype %s" % x.dtype)
        return table[x.dtype]
    kind = np.asarray(x).dtype
    if kind == np.float64:
        return PERM_F64
    if kind == np.complex128:
        return PERM_C128
    if kind in (np.uint8, np.bool_):
        return PERM_U8
    if kind == np.int64:
        return PERM_I64
    raise TypeError("unsupported array dtype %s" % kind)


def _matrix(A):
    """Returns (keepalive, pointer, m, n, ld, dtype code, torch device or None)."""
    if _is_torch(A):
        if A.dim() != 2:
            raise ValueError("expected a 2-D matrix")
        if A.numel() and A.stride(1) != 1:
            A = A.contiguous()
        m, n = A.shape
        ld = A.stride(0) if A.numel() else n
        return A, A.data_ptr(), m, n, max(ld, n), dtype_code(A), (A.device if A.is_cuda else None)
    A = np.asarray(A)
    if A.ndim != 2:
        raise ValueError("expected a 2-D matrix")
    if A.dtype == np.bool_:
        A = A.astype(np.uint8)
    A = np.ascontiguousarray(A)
    m, n = A.shape
    return A, A.ctypes.data, m, n, n, dtype_code(A), None


def _on_stream(device, stream):
    """Context in which torch allocates on the stream the call launches on, so that the
    caching allocator does not hand the block to other work while the call still runs."""
    import contextlib
    if device is None or stream is None:
        return contextlib.nullcontext()
    import torch
    s = stream if isinstance(stream, torch.cuda.Stream) else torch.cuda.ExternalStream(
        stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream), device=device)
    return torch.cuda.stream(s)


def _empty(shape, floating: bool, device, stream=None):
    if device is not None:
        import torch
        with _on_stream(device, stream):
            return torch.empty(shape, dtype=torch.float64 if floating else torch.int64, device=device)
    return np.empty(shape, dtype=np.float64 if floating else np.int64)


def _zeros(shape, device, stream=None):
    if device is not None:
        import torch
        with _on_stream(device, stream):
            return torch.zeros(shape, dtype=torch.int64, device=device)
    return np.zeros(shape, dtype=np.int64)


def _out_like(code: int, device, count: int = 1, stream=None):
    shape = (count,) if code == PERM_F64 else (count, 2)
    return _empty(shape, code in (PERM_F64, PERM_C128), device, stream)


def _ptr(x) -> int:
    return x.data_ptr() if _is_torch(x) else x.ctypes.data


def _stream(device, stream):
    if stream is not None:
        return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    if device is not None:
        import torch
        return torch.cuda.current_stream(device).cuda_stream
    return 0


def _opts(opts):
    if opts is None:
        return None
    if isinstance(opts, perm_opts):
        return ctypes.byref(opts)
    o = perm_opts()
    for k, v in dict(opts).items():
        if k == "err":
            v = _ptr(v) if v is not None else None
        setattr(o, k, v)
    return ctypes.byref(o)


def _device_index(device):
    return 0 if device is None else (device.index if device.index is not None else 0)


def _call(name, A, out, stream, opts):
    keep, p, m, n, ld, code, dev = _matrix(A)
    if out is None:
        out = _out_like(code, dev, stream=stream)
    rc = getattr(lib(), name)(handle(_device_index(dev)), p, m, n, ld, code, _ptr(out), _stream(dev, stream),
                              _opts(opts))
    if rc:
        raise PermError(rc, name)
    return out


def perm_glynn(A, out=None, stream=None, opts=None):
    """Glynn's formula with the rectangular extension; result written into ``out``."""
    return _call("perm_glynn", A, out, stream, opts)


def perm_ryser(A, out=None, stream=None, opts=None):
    """Ryser's formula (square: all subsets; rectangular: subsets of sizes 1..m)."""
    return _call("perm_ryser", A, out, stream, opts)


def perm_combinatoric(A, out=None, stream=None, opts=None):
    """The definition summed over all m-permutations."""
    return _call("perm_combinatoric", A, out, stream, opts)


def perm_auto(A, out=None, stream=None, opts=None):
    """Algorithm chosen by the library's cost model."""
    return _call("perm_auto", A, out, stream, opts)


def perm_glynn_partial(A, g_begin: int, g_end: int, out=None, stream=None, opts=None):
    """Unnormalised Glynn sum over terms [g_begin, g_end) (double-double / int128 modulo 2^128)."""
    keep, p, m, n, ld, code, dev = _matrix(A)
    if out is None:
        words = {PERM_F64: 2, PERM_C128: 4}.get(code, 2)
        out = _empty(words, code in (PERM_F64, PERM_C128), dev, stream)
    rc = lib().perm_glynn_partial(handle(_device_index(dev)), p, m, n, ld, code, g_begin, g_end, _ptr(out),
                                  _stream(dev, stream), _opts(opts))
    if rc:
        raise PermError(rc, "perm_glynn_partial")
    return out


def perm_ryser_partial(A, g_begin: int, g_end: int, out=None, stream=None, opts=None):
    """Weighted Ryser sum over the Gray-ordered subsets [g_begin, g_end) (double-double)."""
    keep, p, m, n, ld, code, dev = _matrix(A)
    if out is None:
        out = _empty(2, True, dev, stream)
    rc = lib().perm_ryser_partial(handle(_device_index(dev)), p, m, n, ld, code, g_begin, g_end, _ptr(out),
                                  _stream(dev, stream), _opts(opts))
    if rc:
        raise PermError(rc, "perm_ryser_partial")
    return out


def perm_batched(packed, offsets, M, N, out=None, stream=None, opts=None):
    """Permanents of many matrices; matrix b is M[b] x N[b] at packed[offsets[b]:] (row-major)."""
    code = dtype_code(packed)
    dev = packed.device if _is_torch(packed) and packed.is_cuda else None
    count = len(offsets)
    if out is None:
        out = _out_like(code, dev, count, stream)
    rc = lib().perm_batched(handle(_device_index(dev)), _ptr(packed), _ptr(offsets), _ptr(M), _ptr(N), count, code,
                            _ptr(out), _stream(dev, stream), _opts(opts))
    if rc:
        raise PermError(rc, "perm_batched")
    return out


def perm_sbp(C, occ, out=None, stream=None, opts=None):
    """SBP coefficients: out[k] = per of the n x n matrix of the occupied columns of the
    n x N matrix C (bit j of occ[k] = state j occupied); occ is a uint64 array/tensor."""
    keep, p, n, N, ld, code, dev = _matrix(C)
    count = len(occ)
    if out is None:
        out = _out_like(code, dev, count, stream)
    rc = lib().perm_sbp(handle(_device_index(dev)), p, n, N, ld, code, _ptr(occ), count, _ptr(out),
                        _stream(dev, stream), _opts(opts))
    if rc:
        raise PermError(rc, "perm_sbp")
    return out


def perm_cauchy(x, y, out=None, stream=None, opts=None):
    """Permanents of the Cauchy matrices c_ij = 1 / (x[b, i] - y[b, j]) by Borchardt's theorem;
    x and y are (count, n) or (n,) float64 arrays/tensors, contiguous; out gets count doubles."""
    if _is_torch(x):
        dev = x.device if x.is_cuda else None
        n = x.shape[-1]
        count = x.numel() // n if n else 0
        if y.shape != x.shape or not x.is_contiguous() or not y.is_contiguous():
            raise ValueError("x and y: contiguous, same shape")
    else:
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        if y.shape != x.shape:
            raise ValueError("x and y: same shape")
        dev = None
        n = x.shape[-1]
        count = x.size // n if n else 0
    if out is None:
        out = _out_like(PERM_F64, dev, count, stream)
    rc = lib().perm_cauchy(handle(_device_index(dev)), _ptr(x), _ptr(y), n, count, _ptr(out),
                           _stream(dev, stream), _opts(opts))
    if rc:
        raise PermError(rc, "perm_cauchy")
    return out


def perm_cauchy_sbp(x, y, occ, out=None, stream=None, opts=None):
    """SBP coefficients of the Cauchy coefficient matrix 1 / (x_i - y_j): out[k] = per of
    the Cauchy matrix of x and the y_j of the occupied states of occ[k] (uint64 bits)."""
    dev = x.device if _is_torch(x) and x.is_cuda else None
    if not _is_torch(x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.float64)
    count = len(occ)
    if out is None:
        out = _out_like(PERM_F64, dev, count, stream)
    rc = lib().perm_cauchy_sbp(handle(_device_index(dev)), _ptr(x), x.shape[-1], _ptr(y), y.shape[-1], _ptr(occ),
                               count, _ptr(out), _stream(dev, stream), _opts(opts))
    if rc:
        raise PermError(rc, "perm_cauchy_sbp")
    return out


def _gaussian(re, im):
    """(keepalive, pointer, m, n, ld, device) of the Gaussian-integer matrix re + i im as
    interleaved int64 pairs."""
    if _is_torch(re):
        import torch
        G = torch.stack([re.to(torch.int64), im.to(torch.int64)], dim=-1).contiguous()
        m, n = G.shape[0], G.shape[1]
        return G, G.data_ptr(), m, n, n, (G.device if G.is_cuda else None)
    G = np.ascontiguousarray(np.stack([np.asarray(re, np.int64), np.asarray(im, np.int64)], axis=-1))
    return G, G.ctypes.data, G.shape[0], G.shape[1], G.shape[1], None


def _gaussian_out(dev, stream=None):
    return _zeros(4, dev, stream)


def perm_batched_gaussian(packed, offsets, M, N, out=None, stream=None):
    """Exact permanents of many Gaussian-integer matrices: packed holds (re, im) int64
    pairs (matrix b's M[b] x N[b] entries from pair offsets[b] on); out gets two int128
    (real, imaginary) per matrix, read with value(out, PERM_CI64, b)."""
    dev = packed.device if _is_torch(packed) and packed.is_cuda else None
    count = len(offsets)
    if out is None:
        out = _zeros((count, 4), dev, stream)
    rc = lib().perm_batched(handle(_device_index(dev)), _ptr(packed), _ptr(offsets), _ptr(M), _ptr(N), count,
                            PERM_CI64, _ptr(out), _stream(dev, stream), None)
    if rc:
        raise PermError(rc, "perm_batched")
    return out


def perm_glynn_gaussian(re, im, out=None, stream=None, opts=None):
    """Exact permanent of the Gaussian-integer matrix re + i im (int64 parts): out holds
    two int128 (real, imaginary); read it with value(out, PERM_CI64)."""
    keep, p, m, n, ld, dev = _gaussian(re, im)
    if out is None:
        out = _gaussian_out(dev, stream)
    rc = lib().perm_glynn(handle(_device_index(dev)), p, m, n, ld, PERM_CI64, _ptr(out), _stream(dev, stream),
                          _opts(opts))
    if rc:
        raise PermError(rc, "perm_glynn")
    return out


def perm_glynn_partial_gaussian(re, im, g_begin: int, g_end: int, out=None, stream=None, opts=None):
    """Unnormalised Glynn sum of re + i im over terms [g_begin, g_end), modulo 2^128."""
    keep, p, m, n, ld, dev = _gaussian(re, im)
    if out is None:
        out = _gaussian_out(dev, stream)
    rc = lib().perm_glynn_partial(handle(_device_index(dev)), p, m, n, ld, PERM_CI64, g_begin, g_end, _ptr(out),
                                  _stream(dev, stream), _opts(opts))
    if rc:
        raise PermError(rc, "perm_glynn_partial")
    return out


def perm_glynn_noalloc(A, out=None, stream=None, grid: int = 0):
    """Real Glynn sweep that allocates nothing (scratch is a fixed device array in the
    library); A and out must be CUDA tensors on the current device."""
    keep, p, m, n, ld, code, dev = _matrix(A)
    if code != PERM_F64 or dev is None:
        raise TypeError("perm_glynn_noalloc takes a float64 CUDA tensor")
    if out is None:
        out = _out_like(code, dev, stream=stream)
    rc = lib().perm_glynn_noalloc(p, m, n, ld, _ptr(out), _stream(dev, stream), grid)
    if rc:
        raise PermError(rc, "perm_glynn_noalloc")
    return out


def _check(rc, name):
    if rc:
        raise PermError(rc, name)


def perm_auto_features(m: int, n: int, density: float, code: int):
    out = np.zeros(PERM_NFEATURES, dtype=np.float32)
    _check(lib().perm_auto_features(m, n, density, code, out.ctypes.data), "perm_auto_features")
    return out


def perm_mlp_size(in_dim: int, hidden: int, out_dim: int) -> int:
    c = ctypes.c_int64()
    _check(lib().perm_mlp_size(in_dim, hidden, out_dim, ctypes.byref(c)), "perm_mlp_size")
    return c.value


def perm_mlp_forward(weights, dims, X, Y=None, stream=None):
    """Y = MLP(X) on the GPU; weights, X, Y are float32 CUDA tensors."""
    import torch
    in_dim, hid, out_dim = dims
    if Y is None:
        with _on_stream(X.device, stream):
            Y = torch.empty((X.shape[0], out_dim), dtype=torch.float32, device=X.device)
    _check(lib().perm_mlp_forward(weights.data_ptr(), in_dim, hid, out_dim, X.data_ptr(), X.shape[0], Y.data_ptr(),
                                  _stream(X.device, stream)), "perm_mlp_forward")
    return Y


def perm_mlp_grad(weights, dims, X, T, mask, stream=None):
    """(gradient, loss) of the masked MSE with respect to the flat weights (CUDA tensors)."""
    import torch
    in_dim, hid, out_dim = dims
    with _on_stream(X.device, stream):
        grad = torch.empty_like(weights)
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
    _check(lib().perm_mlp_grad(weights.data_ptr(), in_dim, hid, out_dim, X.data_ptr(), T.data_ptr(), mask.data_ptr(),
                               X.shape[0], grad.data_ptr(), loss.data_ptr(), _stream(X.device, stream)),
           "perm_mlp_grad")
    return grad, loss


def perm_mlp_train(X, T, mask, dims, epochs: int, batch: int, lr: float, seed: int, stream=None):
    """Train on the GPU; returns (weights, per-epoch loss) as CUDA tensors."""
    import torch
    in_dim, hid, out_dim = dims
    with _on_stream(X.device, stream):
        weights = torch.empty(perm_mlp_size(in_dim, hid, out_dim), dtype=torch.float32, device=X.device)
        hist = torch.zeros(max(epochs, 1), dtype=torch.float32, device=X.device)
    _check(lib().perm_mlp_train(X.data_ptr(), T.data_ptr(), mask.data_ptr(), X.shape[0], in_dim, hid, out_dim, epochs,
                                batch, lr, seed, weights.data_ptr(), hist.data_ptr(), _stream(X.device, stream)),
           "perm_mlp_train")
    return weights, hist


def perm_set_cost_model(weights, dims, device: int = 0):
    """Install host float32 weights (numpy) as perm_auto's cost model; None removes it."""
    if weights is None:
        _check(lib().perm_set_cost_model(handle(device), None, 0, 0, 0), "perm_set_cost_model")
        return
    w = np.ascontiguousarray(weights, dtype=np.float32)
    _check(lib().perm_set_cost_model(handle(device), w.ctypes.data, *dims), "perm_set_cost_model")


def perm_auto_choice(A, opts=None):
    """(candidate, predicted log2 seconds per candidate) that perm_auto would use."""
    keep, p, m, n, ld, code, dev = _matrix(A)
    cand = ctypes.c_int(-1)
    pred = np.zeros(PERM_NCAND, dtype=np.float32)
    _check(lib().perm_auto_choice(handle(_device_index(dev)), p, m, n, ld, code, _opts(opts), ctypes.byref(cand),
                                  pred.ctypes.data), "perm_auto_choice")
    return cand.value, pred


def perm_probe_rate(kind: int, device: int = 0, stream=None) -> float:
    """Measured issue rate of one pipe (include/perm_probe.h)."""
    r = ctypes.c_double()
    rc = lib().perm_probe_rate(device, kind, _stream(None, stream), ctypes.byref(r))
    if rc:
        raise PermError(rc, "perm_probe_rate")
    return r.value


# ----------------------------------------------------------------------------- results
def _int128(lo, hi) -> int:
    v = (int(lo) & (2 ** 64 - 1)) | ((int(hi) & (2 ** 64 - 1)) << 64)
    return v - (1 << 128) if v >> 127 else v


def value(out, code: int, index: int = 0):
    """Python value of result `index` of `out` (float, complex, exact int, or a
    (real, imaginary) pair of exact ints for Gaussian integers)."""
    arr = out.detach().cpu().numpy() if _is_torch(out) else np.asarray(out)
    if code == PERM_F64:
        return float(arr.reshape(-1)[index])
    if code == PERM_CI64:
        q = arr.reshape(-1, 4)[index]
        return (_int128(q[0], q[1]), _int128(q[2], q[3]))
    row = arr.reshape(-1, 2)[index]
    if code == PERM_C128:
        return complex(float(row[0]), float(row[1]))
    lo, hi = int(row[0]) & (2 ** 64 - 1), int(row[1]) & (2 ** 64 - 1)
    v = lo | (hi << 64)
    return v - (1 << 128) if v >> 127 else v


def dd_value(out) -> float:
    """hi + lo of a double-double partial."""
    arr = out.detach().cpu().numpy() if _is_torch(out) else np.asarray(out)
    arr = arr.reshape(-1)
    return float(arr[0]) + float(arr[1])
