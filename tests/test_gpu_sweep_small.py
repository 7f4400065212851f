"""Every entry point and arithmetic on many small random shapes (m <= n <= 9, both
orientations, dense and sparse, all dtypes) against the oracle's definition: a broad
parity net under the targeted tests."""
import numpy as np
import pytest

import oracle
from gpu_util import U, U_CFIX, device, run, scale
from paper_2510_03421_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return device()


@pytest.fixture(scope="module")
def capi():
    from paper_2510_03421_gb300 import capi
    return capi


def _matrix(g, kind, m, n, density):
    mask = g.random((m, n)) < density
    if kind == "f64":
        return np.where(mask, g.uniform(-1, 1, (m, n)), 0.0)
    if kind == "c128":
        return np.where(mask, g.uniform(-1, 1, (m, n)) + 1j * g.uniform(-1, 1, (m, n)), 0.0)
    if kind == "u8":
        return mask.astype(np.uint8)
    return np.where(mask, g.integers(-5, 6, (m, n)), 0).astype(np.int64)


@pytest.mark.parametrize("kind", ["f64", "c128", "u8", "i64"])
def test_random_small_shapes_all_entry_points(capi, dev, kind):
    g = inputs.rng(8400 + ["f64", "c128", "u8", "i64"].index(kind))
    entry = [("perm_glynn", None), ("perm_ryser", None), ("perm_combinatoric", None), ("perm_auto", None)]
    if kind in ("f64", "c128"):
        entry += [("perm_glynn", dict(arith=1)), ("perm_glynn", dict(arith=2)), ("perm_glynn", dict(arith=3))]
    for trial in range(24):
        m = int(g.integers(1, 10))
        n = int(g.integers(m, 10))
        A = _matrix(g, kind, m, n, float(g.choice([0.35, 1.0])))
        if trial % 2:
            A = np.ascontiguousarray(A.T)  # m > n: per(A^T)
        ref = oracle.definition(A)
        mm, nn = sorted(A.shape)
        # the largest sum of |term| over the term sets these entry points evaluate
        # (Glynn padded or in closed form, Ryser, the definition)
        if kind in ("f64", "c128"):
            s = max(scale(A, k) for k in ("glynn", "esym", "ryser", "definition"))
            tol = max(1e-12 * abs(ref), 8 * (nn + 2) * (U_CFIX if kind == "c128" else U) * s)
        for fn, opts in entry:
            got = run(capi, fn, A, dev, opts)
            if kind in ("u8", "i64"):
                assert got == ref, (fn, opts, A.shape)
            else:
                assert abs(got - ref) <= tol, (fn, opts, A.shape, got, ref, tol)
