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
