"""perm_glynn_noalloc: the Glynn sweep for callers that cannot allocate device memory
(runtimes that hand out every buffer from a pool reserved up front, plugin hosts that
forbid cudaMalloc).  It uses a fixed scratch array in the library instead.

Checked here, on two consecutive calls that share that array: agreement with the
long-double oracle (tolerance 8 (n + 2) u sum|t| of the padded Glynn terms the FP64
sweep evaluates) and with perm_glynn within the sum of both calls' tolerances; the
two calls give identical bits.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import oracle
from gpu_util import U_FIX, close, default_kind, device, to_dev, tolerance
from paper_2510_03421_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return device()


@pytest.fixture(scope="module")
def capi():
    from paper_2510_03421_gb300 import capi
    return capi


@pytest.mark.parametrize("shape,seed", [((14, 14), 9001), ((9, 13), 9002), ((12, 7), 9003), ((21, 21), 9004)])
def test_noalloc_matches_oracle_and_perm_glynn_twice(capi, dev, shape, seed):
    import torch
    A = inputs.uniform_real(*shape, seed)
    dA = to_dev(A, dev)
    truth = oracle.glynn(A if A.shape[0] <= A.shape[1] else A.T)
    ref = capi.value(capi.perm_glynn(dA), capi.PERM_F64)
    kind = default_kind(A)
    close(ref, truth, A, kind=kind, u=U_FIX if kind == "esym" else 2.0 ** -53)
    both = tolerance(truth, A) + tolerance(truth, A, kind=kind)
    got = []
    for _ in range(2):  # the second call reuses the scratch the first one left behind
        out = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        capi.perm_glynn_noalloc(dA, out=out)
        torch.cuda.synchronize(dev)
        got.append(float(out.item()))
        close(got[-1], truth, A)
        assert abs(got[-1] - ref) <= both
    assert got[0] == got[1]


def test_noalloc_explicit_grid_and_limits(capi, dev):
    import torch
    A = inputs.uniform_real(16, 16, 9101)
    dA = to_dev(A, dev)
    truth = oracle.glynn(A)
    for grid in (1, 7, 2048):
        out = capi.perm_glynn_noalloc(dA, grid=grid)
        torch.cuda.synchronize(dev)
        close(float(out.item()), truth, A)
    with pytest.raises(capi.PermError) as e:
        capi.perm_glynn_noalloc(dA, grid=2049)
    assert e.value.status == capi.PERM_ETOOBIG
    host = np.ascontiguousarray(A)
    out = torch.empty(1, dtype=torch.float64, device=dev)
    rc = capi.lib().perm_glynn_noalloc(ctypes.c_void_p(host.ctypes.data), 16, 16, 16, ctypes.c_void_p(out.data_ptr()),
                                       None, 0)
    assert rc == capi.PERM_EINVAL


def test_noalloc_rejects_another_devices_memory(capi, dev):
    # refused on the host before any launch (needs a second GPU to run)
    import torch
    if torch.cuda.device_count() < 2:
        pytest.skip("one GPU")
    A = inputs.uniform_real(8, 8, 9201)
    other = torch.from_numpy(A).to("cuda:1")
    out = torch.empty(1, dtype=torch.float64, device=dev)
    with torch.cuda.device(0):
        rc = capi.lib().perm_glynn_noalloc(ctypes.c_void_p(other.data_ptr()), 8, 8, 8,
                                           ctypes.c_void_p(out.data_ptr()), None, 0)
    assert rc == capi.PERM_EINVAL
