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


def test_adam_two_steps_worked_by_hand():
    """theta0 = 1, gradients 0.5 then -0.25, lr 0.1 (betas 0.9, 0.999, eps
    1e-8), worked by hand: step 1 has m = 0.05, v = 0.00025, mhat = 0.5,
    vhat = 0.25, so theta moves by 0.1 * 0.5 / 0.50000001; step 2 has
    m = 0.045 - 0.025 = 0.02, v = 0.00024975 + 0.0000625 = 0.00031225,
    mhat = 0.02 / 0.19, vhat = 0.00031225 / 0.001999 = 0.1562031016, whose root
    is 0.3952253807, so theta moves by 0.0105263158 / 0.3952253907."""
    p, m, v = np.array([1.0]), np.zeros(1), np.zeros(1)
    p, m, v = M.adam_step(p, np.array([0.5]), m, v, 1, 0.1)
    assert np.isclose(m[0], 0.05, rtol=0, atol=1e-15) and np.isclose(v[0], 0.00025, rtol=0, atol=1e-15)
    assert abs(p[0] - 0.900000002) < 1e-12
    p, m, v = M.adam_step(p, np.array([-0.25]), m, v, 2, 0.1)
    assert abs(m[0] - 0.02) < 1e-15 and abs(v[0] - 0.00031225) < 1e-15
    assert abs(p[0] - 0.8733662987) < 1e-9


def test_adam_constant_gradient_closed_form():
    """Under a constant gradient g the bias corrections are exact: mhat = g and
    vhat = g^2 at every step, so each step moves a parameter by exactly
    lr * g / (|g| + eps), and a zero gradient does not move it."""
    rng = np.random.default_rng(2)
    g = np.concatenate([rng.normal(size=6) * 10.0 ** rng.integers(-4, 3, size=6), [0.0]])
    p0 = rng.normal(size=g.size)
    p, m, v = p0.copy(), np.zeros_like(g), np.zeros_like(g)
    lr = 3e-3
    for t in range(1, 6):
        p, m, v = M.adam_step(p, g, m, v, t, lr)
        assert np.allclose(p, p0 - t * lr * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-13)
    assert p[-1] == p0[-1]
