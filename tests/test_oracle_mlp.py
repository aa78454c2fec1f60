"""Pins of the cost-model oracle (oracle/mlp.py): the analytic gradient
against central finite differences in float64, and the network without
hidden layers against the closed-form least-squares gradient."""
import numpy as np

from oracle import mlp as M


def _data(rng, B, n_in):
    X = rng.normal(size=(B, n_in))
    T = np.sin(X[:, 0]) + 0.5 * X[:, 1] ** 2 - X[:, 2]
    return X, T


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    dims = [5, 7, 6, 1]
    p = rng.normal(size=M.n_params(dims)) * 0.5
    X, T = _data(rng, 13, 5)
    _, g = M.loss_grad(p, dims, X, T)
    h = 1e-6
    for k in range(p.size):
        e = np.zeros_like(p)
        e[k] = h
        lp, _ = M.loss_grad(p + e, dims, X, T)
        lm, _ = M.loss_grad(p - e, dims, X, T)
        num = (lp - lm) / (2 * h)
        assert abs(num - g[k]) <= 1e-6 + 1e-5 * abs(num), k


def test_linear_network_closed_form():
    rng = np.random.default_rng(1)
    dims = [4, 1]
    p = rng.normal(size=M.n_params(dims))
    X, T = _data(rng, 50, 4)
    w, b = p[:4], p[4]
    loss, g = M.loss_grad(p, dims, X, T)
    r = X @ w + b - T
    assert np.isclose(loss, np.mean(r ** 2))
    assert np.allclose(g[:4], 2.0 / 50 * X.T @ r)
    assert np.isclose(g[4], 2.0 / 50 * r.sum())


def test_relu_blocks_gradient_of_dead_units():
    dims = [2, 3, 1]
    p = np.zeros(M.n_params(dims))
    p[6:9] = -1.0                    # every hidden bias negative: all units dead
    p[9:12] = 1.0
    X = np.array([[0.1, 0.2], [0.3, -0.1]])
    _, g = M.loss_grad(p, dims, X, np.array([1.0, 2.0]))
    assert np.all(g[:9] == 0) and np.all(g[9:12] == 0) and g[12] != 0
