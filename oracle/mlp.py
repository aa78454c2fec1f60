"""CPU oracle of the cost-model network -- test infrastructure only.

A plain fully connected network in float64 numpy: layers of sizes
dims[0] -> dims[1] -> ... -> dims[-1], ReLU after every layer but the last,
mean squared error loss L = mean_b (y_b - t_b)^2.  The gradient is written out
by the chain rule (backpropagation); relu'(z) is taken as 1 for z > 0 and 0
otherwise.  Parameters use the same flat layout as the library: for each
layer, W[out][in] row-major, then b[out].

Pinned by tests/test_oracle_mlp.py against central finite differences and,
for a network without hidden layers, the closed-form least-squares gradient.
The Adam step is pinned by a two-step case worked by hand and by the closed
forms of bias-corrected Adam under a constant gradient.
"""
from __future__ import annotations

import numpy as np


def unpack(params: np.ndarray, dims: list[int]):
    Ws, bs, off = [], [], 0
    for I, O in zip(dims[:-1], dims[1:]):
        Ws.append(params[off:off + I * O].reshape(O, I))
        off += I * O
        bs.append(params[off:off + O])
        off += O
    assert off == params.size
    return Ws, bs


def n_params(dims: list[int]) -> int:
    return sum(I * O + O for I, O in zip(dims[:-1], dims[1:]))


def forward(params, dims, X):
    """Returns (output [B], list of pre-activations, list of activations)."""
    Ws, bs = unpack(np.asarray(params, dtype=np.float64), dims)
    a = np.asarray(X, dtype=np.float64)
    acts, pres = [a], []
    for l, (W, b) in enumerate(zip(Ws, bs)):
        z = a @ W.T + b
        pres.append(z)
        a = np.maximum(z, 0.0) if l + 1 < len(Ws) else z
        acts.append(a)
    return a[:, 0], pres, acts


def loss_grad(params, dims, X, T):
    """Mean squared error and its gradient with respect to the flat params."""
    params = np.asarray(params, dtype=np.float64)
    Ws, bs = unpack(params, dims)
    y, pres, acts = forward(params, dims, X)
    T = np.asarray(T, dtype=np.float64)
    B = y.size
    loss = float(np.mean((y - T) ** 2))
    dz = (2.0 * (y - T) / B)[:, None]           # dL/dz of the output layer
    grads = [None] * len(Ws)
    for l in range(len(Ws) - 1, -1, -1):
        gW = dz.T @ acts[l]                      # [O, I]
        gb = dz.sum(axis=0)
        grads[l] = (gW, gb)
        if l > 0:
            dz = (dz @ Ws[l]) * (pres[l - 1] > 0)
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat


def adam_step(params, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, "Adam: A Method for Stochastic
    Optimization", ICLR 2015, Algorithm 1) in float64, step number t >= 1:
    the moment estimates m <- b1 m + (1 - b1) g and v <- b2 v + (1 - b2) g^2,
    their bias corrections m / (1 - b1^t) and v / (1 - b2^t), and the move
    params <- params - lr * mhat / (sqrt(vhat) + eps).  Returns the new
    (params, m, v); the inputs are not modified."""
    g = np.asarray(grad, dtype=np.float64)
    m = b1 * np.asarray(m, dtype=np.float64) + (1.0 - b1) * g
    v = b2 * np.asarray(v, dtype=np.float64) + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    p = np.asarray(params, dtype=np.float64) - lr * mhat / (np.sqrt(vhat) + eps)
    return p, m, v
