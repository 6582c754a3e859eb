"""Pins for the FP64 MLP restatement in oracle/mlp.py (no GPU): its analytic
gradient must match central finite differences of its loss, and a hand-built
network must give the hand-computed output."""
import numpy as np

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    dims = (5, 4, 3)
    n = 5 * 4 + 4 + 4 * 4 + 4 + 4 * 3 + 3
    p = rng.normal(size=n)
    X = rng.normal(size=(6, 5))
    T = rng.normal(size=(6, 3))
    g, _ = mlp.grad(p, dims, X, T)
    eps = 1e-6
    for i in range(n):
        d = np.zeros(n)
        d[i] = eps
        fd = (mlp.loss(p + d, dims, X, T) - mlp.loss(p - d, dims, X, T)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), i


def test_forward_hand_computed():
    # in=2, hidden=2, out=1: W1 = I, b1 = (0, -1), W2 = [[1,0],[1,1]], b2 = 0, W3 = (2, -1)^T, b3 = 0.5
    p = np.array([1, 0, 0, 1, 0, -1, 1, 0, 1, 1, 0, 0, 2, -1, 0.5], dtype=np.float64)
    y = mlp.forward(p, (2, 2, 1), np.array([[3.0, 2.0]]))
    # h1 = relu(3, 1) = (3, 1); h2 = relu(3*1+1*1, 0*3+1*1) = (4, 1); y = 8 - 1 + 0.5
    assert np.allclose(y, [[7.5]])
