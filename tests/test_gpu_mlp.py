"""Wake-surrogate kernels (through the C ABI) against the FP64 MLP oracle.

The parameters are rounded to BF16 values first, so the GPU's BF16 weight
copies equal its FP32 masters and both sides multiply the same weights; the
remaining difference is FP32 accumulation over 5 layers of <= 128 terms
(~1e-6 relative per layer), bounded here at 1e-4 of the largest gradient.
"""
import numpy as np
import pytest

from oracle import mlp_oracle as M

pytestmark = pytest.mark.gpu


def bf16_round(x):
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + (((u >> 16) & 1) + 0x7FFF)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32)


@pytest.fixture(scope="module")
def net():
    from paper_2402_13171_gb300 import build, surrogate
    build.build()
    n = surrogate.WakeMLP(seed=3)
    yield n
    n.destroy()


@pytest.mark.parametrize("B", [1, 300, 4099])
def test_forward_and_gradient_match_oracle(net, B):
    rng = np.random.default_rng(B)
    p = bf16_round(net.initial_params(5) * 2.0)
    net.set_params(p)
    assert np.array_equal(net.params(), p)
    X = rng.normal(0, 1, (B, 6)).astype(np.float32)
    T = rng.normal(0, 0.5, (B, 3)).astype(np.float32)
    dims = net.layer_dims()
    assert net.n_params == M.n_params(6, 128, 4, 3) == 50819
    Yo, _ = M.forward(p.astype(np.float64), X.astype(np.float64), dims)
    Yg = net.forward(X)
    np.testing.assert_allclose(Yg, Yo, rtol=0, atol=1e-5 * max(1.0, np.abs(Yo).max()))
    lo, go = M.loss_grad(p.astype(np.float64), X.astype(np.float64), T.astype(np.float64), dims)
    lg, gg = net.loss_grad(X, T)
    assert lg == pytest.approx(lo, rel=1e-5)
    np.testing.assert_allclose(gg, go, rtol=0, atol=1e-4 * np.abs(go).max())


def test_training_is_deterministic_and_learns(net):
    rng = np.random.default_rng(9)
    X = rng.uniform(-1, 1, (20000, 6)).astype(np.float32)
    T = np.stack([0.3 * np.sin(2 * X[:, 0]) * np.exp(-X[:, 1] ** 2), 0.1 * X[:, 2] * X[:, 3],
                  0.2 * np.cos(X[:, 4] + X[:, 5])], axis=1).astype(np.float32)
    p0 = net.initial_params(1)
    net.set_params(p0)
    l0, _ = net.loss_grad(X[:4096], T[:4096])
    net.set_data(X, T)
    net.train(400, batch=1024, lr=3e-3, seed=5)
    p1 = net.params()
    l1, _ = net.loss_grad(X[:4096], T[:4096])
    assert l1 < 0.1 * l0, (l0, l1)
    net.set_params(p0)
    net.train(400, batch=1024, lr=3e-3, seed=5)
    np.testing.assert_array_equal(net.params(), p1)
