"""perm_glynn_noalloc: the Glynn sweep for callers that cannot allocate device memory
(their device memory is owned by a pool or a host application).  It must agree with
perm_glynn within the tolerance of the other FP64 parity tests, on consecutive calls
that share its fixed scratch array.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from gpu_util import close, device, to_dev
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
def test_noalloc_matches_perm_glynn_twice(capi, dev, shape, seed):
    import torch
    A = inputs.uniform_real(*shape, seed)
    dA = to_dev(A, dev)
    ref = capi.value(capi.perm_glynn(dA), capi.PERM_F64)
    for _ in range(2):  # the second call reuses the scratch the first one left behind
        out = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        capi.perm_glynn_noalloc(dA, out=out)
        torch.cuda.synchronize(dev)
        close(float(out.item()), ref, A)


def test_noalloc_explicit_grid_and_limits(capi, dev):
    import torch
    A = inputs.uniform_real(16, 16, 9101)
    dA = to_dev(A, dev)
    ref = capi.value(capi.perm_glynn(dA), capi.PERM_F64)
    for grid in (1, 7, 2048):
        out = capi.perm_glynn_noalloc(dA, grid=grid)
        torch.cuda.synchronize(dev)
        close(float(out.item()), ref, A)
    with pytest.raises(capi.PermError) as e:
        capi.perm_glynn_noalloc(dA, grid=2049)
    assert e.value.status == capi.PERM_ETOOBIG
    host = np.ascontiguousarray(A)
    out = torch.empty(1, dtype=torch.float64, device=dev)
    rc = capi.lib().perm_glynn_noalloc(ctypes.c_void_p(host.ctypes.data), 16, 16, 16, ctypes.c_void_p(out.data_ptr()),
                                       None, 0)
    assert rc == capi.PERM_EINVAL
