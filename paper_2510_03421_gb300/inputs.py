"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random matrices; it holds none of the permanent
arithmetic, so both the CUDA path and the CPU oracle can be fed from it.

Distributions (benchmark section of the paper and the workload list of this
library):

* ``uniform_real``      i.i.d. uniform[lo, hi] float64 (the paper's real matrices use [-1, 1]);
* ``bernoulli01``       i.i.d. 0/1 entries (the paper's "random integer matrices");
* ``complex_gaussian``  i.i.d. standard complex Gaussian / sqrt(n) (boson-sampling-like);
* ``haar_unitary_block`` leading k x k block of a Haar-random unitary of order ``dim``
  (QR of a complex Gaussian with the phase fix Q diag(R_jj / |R_jj|));
* ``sparse_*``          entries kept with probability ``density``;
* ``cauchy``            c_ij = 1 / (x_i - y_j), x ~ U[0.25, 0.75], y ~ U[-0.75, -0.25], best
                        conditioned of ``draws`` samples (precision section of the paper).

Every generator takes an explicit integer seed (numpy PCG64).
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 20251001


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_real(m: int, n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    return rng(seed).uniform(lo, hi, size=(m, n))


def bernoulli01(m: int, n: int, seed: int, p: float = 0.5) -> np.ndarray:
    return (rng(seed).random(size=(m, n)) < p).astype(np.uint8)


def complex_gaussian(m: int, n: int, seed: int) -> np.ndarray:
    g = rng(seed)
    z = (g.standard_normal((m, n)) + 1j * g.standard_normal((m, n))) / np.sqrt(2.0)
    return z / np.sqrt(n)


def _haar_columns(dim: int, k: int, g: np.random.Generator, batch: int) -> np.ndarray:
    z = (g.standard_normal((batch, dim, k)) + 1j * g.standard_normal((batch, dim, k))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=1, axis2=2)
    ph = d / np.abs(d)
    return q * ph[:, None, :]


def haar_unitary_block(k: int, seed: int, dim: int = 64) -> np.ndarray:
    """Leading k x k block of a Haar unitary of order dim (the first k columns of Q only
    depend on the first k columns of the Gaussian, so a dim x k QR suffices)."""
    q = _haar_columns(dim, k, rng(seed), 1)[0]
    return np.ascontiguousarray(q[:k, :k])


def batched_haar(count: int, nmin: int, nmax: int, seed: int, dim: int = 64):
    """``count`` complex128 n_i x n_i blocks, n_i uniform in nmin..nmax, each from its own
    Haar unitary.  Returns (sizes int32[count], packed complex128 array, offsets int64[count])
    where matrix i occupies packed[offsets[i] : offsets[i] + n_i*n_i] row-major."""
    g = rng(seed)
    sizes = g.integers(nmin, nmax + 1, size=count).astype(np.int32)
    offsets = np.zeros(count, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes.astype(np.int64) ** 2)[:-1]
    total = int(offsets[-1] + int(sizes[-1]) ** 2) if count else 0
    packed = np.empty(total, dtype=np.complex128)
    for k in range(nmin, nmax + 1):
        idx = np.nonzero(sizes == k)[0]
        if idx.size == 0:
            continue
        q = _haar_columns(dim, k, g, idx.size)[:, :k, :k]
        for row, i in enumerate(idx):
            packed[offsets[i]: offsets[i] + k * k] = q[row].reshape(-1)
    return sizes, packed, offsets


def sparse_real(m: int, n: int, density: float, seed: int) -> np.ndarray:
    g = rng(seed)
    a = g.uniform(-1.0, 1.0, size=(m, n))
    return np.where(g.random(size=(m, n)) < density, a, 0.0)


def sparse_complex(m: int, n: int, density: float, seed: int) -> np.ndarray:
    g = rng(seed)
    a = g.uniform(-1.0, 1.0, size=(m, n)) + 1j * g.uniform(-1.0, 1.0, size=(m, n))
    return np.where(g.random(size=(m, n)) < density, a, 0.0)


def sparse01(m: int, n: int, density: float, seed: int) -> np.ndarray:
    return bernoulli01(m, n, seed, density)


def cauchy_points(n: int, seed: int, draws: int = 1, count: int = 1):
    """Points of `count` Cauchy matrices c_ij = 1 / (x_i - y_j), the recipe of the paper's
    accuracy tests: x ~ U[0.25, 0.75], y ~ U[-0.75, -0.25].  With draws > 1, each
    matrix keeps the draw whose C has the smallest 2-norm condition number.  Returns
    (x, y), each of shape (count, n)."""
    g = rng(seed)
    xs = np.empty((count, n))
    ys = np.empty((count, n))
    for b in range(count):
        best_cond = np.inf
        for _ in range(draws):
            x = g.uniform(0.25, 0.75, size=n)
            y = g.uniform(-0.75, -0.25, size=n)
            k = np.linalg.cond(1.0 / (x[:, None] - y[None, :])) if draws > 1 else 0.0
            if k < best_cond:
                xs[b], ys[b], best_cond = x, y, k
    return xs, ys


def cauchy(n: int, seed: int, draws: int = 1000) -> np.ndarray:
    x, y = cauchy_points(n, seed, draws)
    return 1.0 / (x[0][:, None] - y[0][None, :])


# The five workloads, by what they are.
def square16_f64(seed: int = SEED_BASE + 1) -> np.ndarray:
    return uniform_real(16, 16, seed)


def square36_f64(seed: int = SEED_BASE + 2) -> np.ndarray:
    return uniform_real(36, 36, seed)


def square32_c128(seed: int = SEED_BASE + 2) -> np.ndarray:
    return complex_gaussian(32, 32, seed)


def rect20x40_f64(seed: int = SEED_BASE + 3) -> np.ndarray:
    return uniform_real(20, 40, seed, 0.0, 1.0)


def square26_01(seed: int = SEED_BASE + 3) -> np.ndarray:
    return bernoulli01(26, 26, seed)
