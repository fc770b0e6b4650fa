"""FP64 CPU reference of the coarse-mesh correction network (test infrastructure only).

The network maps per-site features to 3 outputs through two tanh hidden
layers of 64 units.  Two feature sets exist:

* "stated": the 27 mesh-potential samples around the site and a one-hot site
  type, 30 inputs padded with two zeros to 32 (the learned-correction form as
  stated: local mesh-potential samples plus the site type);
* "cell" (the default): the same 30, then the site's position inside its mesh
  cell (sin, cos of 2 pi u per axis), padded with twelve zeros to 48.

The network, for either input width n_in:

    h1 = tanh(W1 x + b1),  h2 = tanh(W2 h1 + b2),  y = W3 h2 + b3,
    loss = mean over sites of sum_c (y_c - t_c)^2.

Weights are rounded to BF16 before use (the GPU stores BF16 copies of FP32
master weights); everything else here is FP64.  The parameter vector is laid
out as [W1 (64 x n_in, row-major), b1 (64), W2 (64x64), b2 (64), W3 (3x64),
b3 (3)]: 7,491 values at n_in = 48, 6,467 at n_in = 32; the width is read off
the vector's length.
With ``act_bf16`` the hidden activations are rounded to BF16 as well before
they enter the next layer: that is how tensor-core inference consumes them
(BF16 operands, FP32 accumulation); training keeps them unrounded.

Features (``features``): for each site, the coarse mesh potential phi
B-spline-interpolated at the 27 points r_i + h (a, b, c), a, b, c in
{-1, 0, 1} (h = box / mesh per axis), in the order 9 (a+1) + 3 (b+1) + (c+1),
times a scale s_in; then the one-hot site type (O, H, WC); then, "stated",
two zeros, or, "cell", sin(2 pi u_d), cos(2 pi u_d) for d = x, y, z with
u_d = x_d N_d / L_d the site's coordinate in mesh units (its offset inside
the mesh cell) and twelve zeros.  The interpolation is the oracle PPPM's own
(the same order-p stencil as its charge assignment), evaluated at the
shifted points: the definition itself.

``adam_step`` is the Adam update (Kingma and Ba, 2015) with bias correction.

Only tests/, the smoke check and the benchmark's CPU-baseline leg may use this
module.
"""
from __future__ import annotations

import numpy as np

N_H, N_OUT = 64, 3
N_PHI, N_TYPE, N_CELL = 27, 3, 6
FEATURE_WIDTH = {"stated": 32, "cell": 48}


def shapes(n_in: int) -> list:
    return [("W1", (N_H, n_in)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)),
            ("W3", (N_OUT, N_H)), ("b3", (N_OUT,))]


def n_params(n_in: int) -> int:
    return sum(int(np.prod(s)) for _, s in shapes(n_in))


def width_of(theta) -> int:
    """Input width n_in of a parameter vector, from its length."""
    rest = n_params(0)
    k = len(theta) - rest
    if k <= 0 or k % N_H:
        raise ValueError(f"{len(theta)} is not the parameter count of a network of this shape")
    return k // N_H


N_IN = FEATURE_WIDTH["cell"]
SHAPES = shapes(N_IN)
N_PARAMS = n_params(N_IN)


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round FP32 values to the nearest BF16 (ties to even) and return them as FP64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return (u.astype(np.uint32)).view(np.float32).astype(np.float64)


def unpack(theta: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in shapes(width_of(theta)):
        k = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + k], dtype=np.float64).reshape(shape)
        o += k
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel()
                           for name, _ in shapes(np.shape(p["W1"])[1])])


def forward(theta: np.ndarray, X: np.ndarray, bf16: bool = True, act_bf16: bool = False):
    """Outputs (n, 3) and the activations needed by backward."""
    t = bf16_round(theta) if bf16 else np.asarray(theta, dtype=np.float64)
    p = unpack(t)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.tanh(z1)
    if act_bf16:
        h1 = bf16_round(h1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.tanh(z2)
    if act_bf16:
        h2 = bf16_round(h2)
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


def adam_step(theta, m, v, g, step: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update at step number ``step`` (1-based); returns the new
    (theta, m, v).  m and v are the running first and second moments."""
    m = b1 * np.asarray(m, np.float64) + (1.0 - b1) * g
    v = b2 * np.asarray(v, np.float64) + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** step)
    vhat = v / (1.0 - b2 ** step)
    return np.asarray(theta, np.float64) - lr * mhat / (np.sqrt(vhat) + eps), m, v


def features(phi: np.ndarray, pos: np.ndarray, types: np.ndarray, box, mesh, p: int, s_in: float = 1.0,
             kind: str = "cell"):
    """Per-site network inputs (n, 32) for kind "stated" or (n, 48) for
    "cell", FP64, from the mesh potential phi."""
    from .pppm import interpolate
    pos = np.asarray(pos, dtype=np.float64)
    h = np.asarray(box, np.float64) / np.asarray(mesh, np.float64)
    n = pos.shape[0]
    X = np.zeros((n, FEATURE_WIDTH[kind]))
    k = 0
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            for c in (-1, 0, 1):
                shifted = pos + h * np.array([a, b, c], np.float64)
                X[:, k] = s_in * interpolate([phi], shifted, box, mesh, p)[:, 0]
                k += 1
    t = np.asarray(types).astype(np.int64)
    for j in range(3):
        X[:, 27 + j] = (t == j).astype(np.float64)
    if kind == "stated":
        return X
    for d in range(3):
        u = pos[:, d] / h[d]
        X[:, 30 + 2 * d] = np.sin(2.0 * np.pi * u)
        X[:, 31 + 2 * d] = np.cos(2.0 * np.pi * u)
    return X
