"""Reference three-layer perceptron of the cost model, in float64 numpy -- TEST
INFRASTRUCTURE ONLY (the gradient check of the GPU training kernels).

    h1 = relu(x W1 + b1), h2 = relu(h1 W2 + b2), y = h2 W3 + b3
    L  = sum_{r,k} mask_rk (y_rk - t_rk)^2 / sum mask

The flat weight layout matches include/perm_mlp.h: W1 [in x hid], b1 [hid],
W2 [hid x hid], b2 [hid], W3 [hid x out], b3 [out].  The gradient is the chain
rule written out layer by layer; it is pinned in the tests against central
finite differences of `loss`.
"""
import numpy as np


def unpack(w, in_dim, hid, out_dim):
    w = np.asarray(w, dtype=np.float64)
    sizes = [in_dim * hid, hid, hid * hid, hid, hid * out_dim, out_dim]
    parts, k = [], 0
    for s in sizes:
        parts.append(w[k:k + s])
        k += s
    assert k == w.size
    W1, b1, W2, b2, W3, b3 = parts
    return W1.reshape(in_dim, hid), b1, W2.reshape(hid, hid), b2, W3.reshape(hid, out_dim), b3


def forward(w, dims, X):
    W1, b1, W2, b2, W3, b3 = unpack(w, *dims)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1 + b1
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ W2 + b2
    a2 = np.maximum(z2, 0.0)
    y = a2 @ W3 + b3
    return y, (X, z1, a1, z2, a2)


def loss(w, dims, X, T, mask):
    y, _ = forward(w, dims, X)
    mask = np.asarray(mask, dtype=np.float64)
    return float(np.sum(mask * (y - T) ** 2) / np.sum(mask))


def grad(w, dims, X, T, mask):
    W1, b1, W2, b2, W3, b3 = unpack(w, *dims)
    y, (X, z1, a1, z2, a2) = forward(w, dims, X)
    mask = np.asarray(mask, dtype=np.float64)
    dy = 2.0 * mask * (y - T) / np.sum(mask)
    gW3 = a2.T @ dy
    gb3 = dy.sum(axis=0)
    d2 = (dy @ W3.T) * (z2 > 0)
    gW2 = a1.T @ d2
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2.T) * (z1 > 0)
    gW1 = X.T @ d1
    gb1 = d1.sum(axis=0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
