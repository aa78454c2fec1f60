"""CPU oracle of the cost-model network -- test infrastructure only.

A plain fully connected network in float64 numpy: layers of sizes
dims[0] -> dims[1] -> ... -> dims[-1], ReLU after every layer but the last,
mean squared error loss L = mean_b (y_b - t_b)^2.  The gradient is written out
by the chain rule (backpropagation); relu'(z) is taken as 1 for z > 0 and 0
otherwise.  Parameters use the same flat layout as the library: for each
layer, W[out][in] row-major, then b[out].

Pinned by tests/test_oracle_mlp.py against central finite differences and,
for a network without hidden layers, the closed-form least-squares gradient.
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
