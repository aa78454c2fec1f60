"""The cost model's CUDA forward, backward and Adam kernels against the
float64 oracle (oracle/mlp.py).

Tolerance: every output and gradient entry is a sum of FP32 products; the
rounding error of a length-K sum is bounded by about K * 2^-24 times the sum
of the magnitudes of its terms.  With K <= 256 (batch) and 64 (hidden) the
bound is below 2e-5 of the largest term magnitude, so entries are compared
with atol = 1e-4 * (largest magnitude) and rtol = 1e-3."""
import numpy as np
import pytest
import torch

from oracle import mlp as M

pytestmark = pytest.mark.gpu


def _data(rng, B, n_in):
    X = rng.uniform(-1, 1, size=(B, n_in)).astype(np.float32)
    c = [X[:, k % n_in] for k in range(4)]
    T = (np.sin(3 * c[0]) + 0.5 * c[1] ** 2 - c[2] * c[3]).astype(np.float32)
    return X, T


@pytest.fixture(autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    global S
    from paper_2512_11112_b300 import spdz as S  # noqa: F401
    yield


@pytest.mark.parametrize("n_in,hidden,layers,B", [(12, 64, 3, 256), (5, 7, 2, 33), (3, 16, 1, 1)])
def test_forward_loss_grad_match_oracle(n_in, hidden, layers, B):
    rng = np.random.default_rng(n_in + B)
    m = S.spdz_mlp_create(n_in, hidden, layers, seed=9, stream=torch.cuda.current_stream().cuda_stream)
    try:
        dims = [n_in] + [hidden] * layers + [1]
        p = S.spdz_mlp_get_params(m)
        assert p.size == M.n_params(dims)
        # perturb the biases away from zero so ReLU boundaries are exercised
        p = p + rng.normal(scale=0.05, size=p.size).astype(np.float32)
        S.spdz_mlp_set_params(m, p)
        X, T = _data(rng, B, n_in)
        Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
        Y = torch.zeros(B, dtype=torch.float32, device="cuda")
        S.spdz_mlp_forward(m, Xd, Y, B)
        torch.cuda.synchronize()
        y_ref, _, _ = M.forward(p.astype(np.float64), dims, X.astype(np.float64))
        scale = max(1.0, float(np.abs(y_ref).max()))
        assert np.allclose(Y.cpu().numpy(), y_ref, rtol=1e-3, atol=1e-4 * scale)
        loss, g = S.spdz_mlp_loss_grad(m, Xd, Td, B)
        loss_ref, g_ref = M.loss_grad(p.astype(np.float64), dims, X.astype(np.float64), T.astype(np.float64))
        assert np.isclose(loss, loss_ref, rtol=1e-3)
        gs = float(np.abs(g_ref).max())
        assert np.allclose(g, g_ref, rtol=1e-3, atol=1e-4 * gs)
    finally:
        S.spdz_mlp_destroy(m)


def test_training_reduces_loss():
    rng = np.random.default_rng(3)
    n_in, B = 12, 2048
    X, T = _data(rng, B, n_in)
    m = S.spdz_mlp_create(n_in, 64, 3, seed=1, stream=torch.cuda.current_stream().cuda_stream)
    try:
        Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
        l0, _ = S.spdz_mlp_loss_grad(m, Xd, Td, B)
        l1 = S.spdz_mlp_train(m, Xd, Td, B, epochs=200, batch=256, lr=2e-3)
        assert l1 < 0.05 * l0, (l0, l1)
        # the trained parameters still agree with the oracle's loss
        p = S.spdz_mlp_get_params(m)
        loss_ref, _ = M.loss_grad(p.astype(np.float64), [n_in, 64, 64, 64, 1], X.astype(np.float64),
                                  T.astype(np.float64))
        assert np.isclose(l1, loss_ref, rtol=2e-3, atol=1e-6)
    finally:
        S.spdz_mlp_destroy(m)


def test_adam_step_matches_oracle():
    """Two Adam steps of the CUDA kernel (k_adam through spdz_mlp_adam_step)
    against the float64 oracle step on the same seeded gradients, element by
    element.  Gradients span magnitudes 1e-6 .. 1e2 and include exact zeros.
    Each FP32 step is a handful of correctly rounded operations, so the
    relative error of a move is a few units of 2^-24 and the stored parameter
    adds one rounding of its own magnitude: |p_gpu - p_ref| <= 1e-6 |p_ref| +
    1e-5 lr."""
    rng = np.random.default_rng(11)
    m = S.spdz_mlp_create(12, 64, 3, seed=5, stream=torch.cuda.current_stream().cuda_stream)
    try:
        p0 = S.spdz_mlp_get_params(m)
        npar = p0.size
        S.spdz_mlp_set_params(m, p0)                    # fresh moments, step counter 0
        lr = 1e-2
        ref_p, ref_m, ref_v = p0.astype(np.float64), np.zeros(npar), np.zeros(npar)
        for t in (1, 2):
            g = (rng.normal(size=npar) * 10.0 ** rng.uniform(-6, 2, size=npar)).astype(np.float32)
            g[rng.integers(0, npar, npar // 50)] = 0.0
            S.spdz_mlp_adam_step(m, torch.from_numpy(g).cuda(), lr)
            ref_p, ref_m, ref_v = M.adam_step(ref_p, g.astype(np.float64), ref_m, ref_v, t, lr)
            got = S.spdz_mlp_get_params(m).astype(np.float64)
            err = np.abs(got - ref_p)
            tol = 1e-6 * np.abs(ref_p) + 1e-5 * lr
            assert np.all(err <= tol), (t, int(np.argmax(err - tol)), float(np.max(err - tol)))
    finally:
        S.spdz_mlp_destroy(m)


def test_training_step_applies_bias_corrected_adam():
    """The first step of spdz_mlp_train (one mini-batch holding every row)
    moves each parameter by lr * g / (|g| + eps) of its full-batch gradient g,
    which is lr times the sign of g wherever the gradient is well above its
    FP32 rounding bound (1e-3 of the largest entry): checked against the
    float64 oracle's gradient and Adam step."""
    rng = np.random.default_rng(12)
    n_in, B, lr = 12, 256, 1e-3
    X, T = _data(rng, B, n_in)
    m = S.spdz_mlp_create(n_in, 64, 3, seed=2, stream=torch.cuda.current_stream().cuda_stream)
    try:
        p0 = S.spdz_mlp_get_params(m)
        p0 = p0 + rng.normal(scale=0.05, size=p0.size).astype(np.float32)
        S.spdz_mlp_set_params(m, p0)
        S.spdz_mlp_train(m, torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(), B, epochs=1, batch=B, lr=lr)
        got = S.spdz_mlp_get_params(m).astype(np.float64)
        dims = [n_in, 64, 64, 64, 1]
        _, g = M.loss_grad(p0.astype(np.float64), dims, X.astype(np.float64), T.astype(np.float64))
        ref, _, _ = M.adam_step(p0.astype(np.float64), g, np.zeros_like(g), np.zeros_like(g), 1, lr)
        sure = np.abs(g) > 1e-3 * np.abs(g).max()
        assert sure.sum() > 0.5 * g.size
        tol = 1e-6 * np.abs(ref) + 1e-5 * lr
        assert np.all(np.abs(got - ref)[sure] <= tol[sure])
        assert np.all(np.abs(got - p0) <= lr * (1 + 1e-5) + 1e-6 * np.abs(p0))
    finally:
        S.spdz_mlp_destroy(m)
