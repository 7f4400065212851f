"""Helpers shared by the GPU parity tests (device, marshalling, tolerances)."""
import math
import os

import numpy as np

U = np.finfo(np.float64).eps / 2
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


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


def term_bound(A):
    """prod_j sum_i |a'_ij| for the padded matrix a' (rows of ones appended): no Glynn or
    Ryser term (after normalisation by 2^(n-1)) exceeds it in modulus."""
    A = np.asarray(A)
    if A.shape[0] > A.shape[1]:
        A = A.T
    m, n = A.shape
    return float(np.prod(np.abs(A).sum(axis=0) + (n - m)))


def close(got, ref, A, rel=1e-12, mult=8):
    A = np.asarray(A)
    m, n = sorted(A.shape)
    tol = max(rel * abs(ref), mult * (n + 2) * U * term_bound(A) / math.factorial(n - m))
    assert abs(got - ref) <= tol, (got, ref, abs(got - ref), tol)


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
