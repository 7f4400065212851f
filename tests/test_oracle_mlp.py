"""Pin the float64 reference of the cost-model perceptron: its gradient must match
central finite differences of its loss (so the chain rule in it is right), and its
forward pass must match an independent layer-by-layer evaluation."""
import numpy as np

from oracle import mlp_ref


def test_gradient_matches_finite_differences():
    g = np.random.default_rng(3)
    dims = (5, 7, 3)
    n = 5 * 7 + 7 + 7 * 7 + 7 + 7 * 3 + 3
    w = g.normal(0, 0.5, n)
    X = g.normal(0, 1, (11, 5))
    T = g.normal(0, 1, (11, 3))
    mask = (g.random((11, 3)) < 0.7).astype(float)
    an = mlp_ref.grad(w, dims, X, T, mask)
    h = 1e-6
    for k in range(n):
        e = np.zeros(n)
        e[k] = h
        fd = (mlp_ref.loss(w + e, dims, X, T, mask) - mlp_ref.loss(w - e, dims, X, T, mask)) / (2 * h)
        assert abs(fd - an[k]) <= 1e-6 * (1 + abs(fd)), (k, fd, an[k])


def test_forward_layer_by_layer():
    g = np.random.default_rng(4)
    dims = (3, 4, 2)
    n = 3 * 4 + 4 + 16 + 4 + 8 + 2
    w = g.normal(0, 1, n)
    x = g.normal(0, 1, 3)
    W1 = w[:12].reshape(3, 4)
    b1 = w[12:16]
    W2 = w[16:32].reshape(4, 4)
    b2 = w[32:36]
    W3 = w[36:44].reshape(4, 2)
    b3 = w[44:46]
    h1 = [max(0.0, sum(x[i] * W1[i, o] for i in range(3)) + b1[o]) for o in range(4)]
    h2 = [max(0.0, sum(h1[i] * W2[i, o] for i in range(4)) + b2[o]) for o in range(4)]
    y = [sum(h2[i] * W3[i, o] for i in range(4)) + b3[o] for o in range(2)]
    got, _ = mlp_ref.forward(w, dims, x[None, :])
    assert np.allclose(got[0], y, rtol=1e-13, atol=1e-13)
