"""Pins for the cost-model network oracle: finite differences and a hand-computable case."""
import numpy as np

from oracle import mlp


def test_gradient_matches_central_finite_differences():
    rng = np.random.default_rng(0)
    in_dim = 7
    p = mlp.init(in_dim, seed=1)
    x = rng.normal(size=(40, in_dim))
    t = rng.normal(size=40)
    g = mlp.grad(p, x, t)
    idx = rng.choice(len(p), 300, replace=False)
    eps = 1e-6
    for i in idx:
        d = np.zeros_like(p)
        d[i] = eps
        fd = (mlp.loss(p + d, x, t) - mlp.loss(p - d, x, t)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 + 1e-4 * abs(fd), (i, fd, g[i])


def test_hand_case():
    # one input, all weights chosen so every unit is active: y = b3 + sum_j w3_j relu(...)
    in_dim = 1
    p = np.zeros(mlp.param_count(in_dim))
    W1, b1, W2, b2, w3, b3 = [a for a in mlp.split(p, in_dim)]
    o = 0
    p[0:64] = 1.0                 # W1: h1_j = relu(x)
    o = 64 + 64                   # skip b1
    p[o:o + 64 * 64] = np.eye(64).ravel()  # W2 = identity: h2 = h1
    o += 64 * 64 + 64             # skip b2
    p[o:o + 64] = 0.5             # w3
    p[o + 64] = 3.0               # b3
    y, h1, h2 = mlp.forward(p, np.array([[2.0]]))
    assert np.allclose(h1, 2.0) and np.allclose(h2, 2.0) and np.isclose(y[0], 3.0 + 64 * 0.5 * 2.0)
    y, _, _ = mlp.forward(p, np.array([[-2.0]]))  # ReLU cuts everything: y = b3
    assert np.isclose(y[0], 3.0)
