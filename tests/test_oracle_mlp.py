"""Pins of the FP64 reference of the correction network."""
import numpy as np
import pytest

from oracle import mlp
from workloads.water import init_mlp_params


def test_bf16_round_matches_library():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = (rng.normal(size=2000) * 10.0 ** rng.uniform(-5, 5, size=2000)).astype(np.float32)
    x = np.concatenate([x, np.float32([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 0.0])])
    ref = torch.tensor(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(x), ref)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    theta = init_mlp_params(3).astype(np.float64)
    theta[2048:2112] = rng.normal(size=64) * 0.1  # nonzero b1
    X = rng.normal(size=(20, 32))
    T = rng.normal(size=(20, 3))
    _, g = mlp.loss_and_grad(theta, X, T, bf16=False)
    h = 1e-6
    idx = rng.choice(mlp.N_PARAMS, size=120, replace=False)
    fd = np.empty(len(idx))
    for k, j in enumerate(idx):
        tp, tm = theta.copy(), theta.copy()
        tp[j] += h
        tm[j] -= h
        fd[k] = (mlp.loss_and_grad(tp, X, T, bf16=False)[0] - mlp.loss_and_grad(tm, X, T, bf16=False)[0]) / (2 * h)
    assert np.max(np.abs(fd - g[idx])) <= 1e-6 * max(1.0, np.max(np.abs(g[idx])))


def test_zero_weights_give_bias_and_linear_regime():
    p = {name: np.zeros(shape) for name, shape in mlp.SHAPES}
    p["b3"] = np.array([0.5, -1.0, 2.0])
    y, _ = mlp.forward(mlp.pack(p), np.ones((4, 32)), bf16=False)
    assert np.allclose(y, p["b3"])
    # small weights: tanh is the identity to third order, so y = W3 W2 W1 x
    rng = np.random.default_rng(2)
    for name, shape in mlp.SHAPES:
        p[name] = rng.normal(size=shape) * (1e-5 if name.startswith("W") else 0.0)
    x = rng.normal(size=(5, 32))
    y, _ = mlp.forward(mlp.pack(p), x, bf16=False)
    lin = x @ (p["W3"] @ p["W2"] @ p["W1"]).T
    assert np.max(np.abs(y - lin)) <= 1e-6 * np.max(np.abs(lin))
