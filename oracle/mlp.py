"""FP64 CPU reference of the coarse-mesh correction network (test infrastructure only).

The network maps per-site features (27 mesh-potential samples around the site
and a one-hot site type, padded to 32 inputs) to 3 outputs through two tanh
hidden layers of 64 units:

    h1 = tanh(W1 x + b1),  h2 = tanh(W2 h1 + b2),  y = W3 h2 + b3,
    loss = mean over sites of sum_c (y_c - t_c)^2.

Weights are rounded to BF16 before use (the GPU stores BF16 copies of FP32
master weights); everything else here is FP64.  The parameter vector is laid
out as [W1 (64x32, row-major), b1 (64), W2 (64x64), b2 (64), W3 (3x64), b3 (3)].

Only tests/, the smoke check and the benchmark's CPU-baseline leg may use this
module.
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT = 32, 64, 3
SHAPES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)),
          ("W3", (N_OUT, N_H)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round FP32 values to the nearest BF16 (ties to even) and return them as FP64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return (u.astype(np.uint32)).view(np.float32).astype(np.float64)


def unpack(theta: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + k], dtype=np.float64).reshape(shape)
        o += k
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def forward(theta: np.ndarray, X: np.ndarray, bf16: bool = True):
    """Outputs (n, 3) and the activations needed by backward."""
    t = bf16_round(theta) if bf16 else np.asarray(theta, dtype=np.float64)
    p = unpack(t)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.tanh(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.tanh(z2)
    y = h2 @ p["W3"].T + p["b3"]
    return y, (X, h1, h2, p)


def loss_and_grad(theta: np.ndarray, X: np.ndarray, T: np.ndarray, bf16: bool = True):
    """Mean-squared loss and its gradient with respect to the parameters used
    (the BF16-rounded ones when bf16 is set), by the chain rule."""
    y, (X, h1, h2, p) = forward(theta, X, bf16)
    n = X.shape[0]
    r = y - np.asarray(T, dtype=np.float64)
    loss = float(np.sum(r * r) / n)
    dy = 2.0 * r / n
    g = {}
    g["W3"] = dy.T @ h2
    g["b3"] = dy.sum(axis=0)
    dz2 = (dy @ p["W3"]) * (1.0 - h2 * h2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"]) * (1.0 - h1 * h1)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return loss, pack(g)
