"""Pins of the oracle's preconditioner network (oracle/mlp.py)."""
import numpy as np
import pytest

from oracle import mlp

torch = pytest.importorskip("torch")


def test_bf16_rounding_matches_torch():
    g = np.random.default_rng(0)
    x = np.concatenate([g.normal(size=10000) * 10.0 ** g.integers(-6, 6, size=10000),
                        [1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, np.pi, -2.5, 0.0]])
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), want)


def test_gelu_matches_torch_and_its_derivative():
    x = np.linspace(-6, 6, 2001)
    want = torch.nn.functional.gelu(torch.tensor(x), approximate="tanh").numpy()
    np.testing.assert_allclose(mlp.gelu(x), want, atol=1e-14)
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(x), fd, atol=1e-8)


def test_backprop_matches_central_differences():
    p = mlp.init_params(3)
    g = np.random.default_rng(4)
    X = g.normal(size=(40, 3))
    t = g.normal(size=40)
    L, grads = mlp.loss_and_grads(p, X, t, rounding=False)
    h = 1e-6
    for name in ("W1", "b1", "W2", "b2", "w3", "b3"):
        flat = p[name].ravel()
        for idx in g.choice(flat.size, size=min(6, flat.size), replace=False):
            q = {k: v.copy() for k, v in p.items()}
            q[name].ravel()[idx] += h
            Lp, _ = mlp.loss_and_grads(q, X, t, rounding=False)
            q[name].ravel()[idx] -= 2 * h
            Lm, _ = mlp.loss_and_grads(q, X, t, rounding=False)
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - grads[name].ravel()[idx]) <= 1e-6 * max(1.0, abs(fd))


def test_rounded_network_is_close_to_the_exact_one():
    p = mlp.init_params(5)
    X = np.random.default_rng(6).normal(size=(500, 3))
    y1, _ = mlp.forward(p, X, rounding=True)
    y0, _ = mlp.forward(p, X, rounding=False)
    assert np.linalg.norm(y1 - y0) <= 1e-2 * np.linalg.norm(y0)
