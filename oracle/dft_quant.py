"""Oracle (test infrastructure only): the DFT with int32-quantised partial sums.

In the paper's hardware-offloaded FFT (Section "Hardware-offloaded 3D FFT",
the data-quantisation panel of its ring-reduction figure, and the "Mixed-Int32"
runs of its evaluation), the DFT along one axis is a sum over nodes: each node
holds ``group`` consecutive mesh points of the line and contributes the partial
sum over its own points to every output; the partials are scaled by 10^7,
converted to int32 and added exactly by the network's integer reduction, and
the sum is scaled back.  This module writes that definition out:

    X_k = (1 / s) sum_n Q(s * sum_{t in node n} x_t e^{sign 2 pi i k t / L})

with Q rounding each of the real and imaginary parts to the nearest integer
(the paper does not say how it converts; round-to-nearest is the reading taken
here) and clamping it to the int32 range (a clamped value is reported as
saturated).  ``pppm_quantized`` is the FP64 PPPM of ``oracle.pppm`` with every
1D transform replaced by this one, in the axis order the library uses (forward
z, y, x; inverse x, y, z).  The fixed scale makes the error depend on what is
transformed, which the paper leaves open (it only says that most values lie
in [-1, 1]); the reading taken: the quantities the library transforms, i.e.
the charge per mesh point sum_i q_i W (not divided by h^3) forward, and the
field spectra already divided by N h^3 backward (so the inverse transforms
give the fields directly).
"""
from __future__ import annotations

import numpy as np

from .pppm import interpolate, spread, wavevectors

SCALE = 1.0e7
INT32_MAX = 2 ** 31 - 1


def quantize(v: np.ndarray, scale: float = SCALE):
    """Nearest integers of v * scale clamped to int32 (as int64), and whether
    any value was clamped."""
    r = np.rint(np.asarray(v, dtype=np.float64) * scale)
    sat = bool(np.any(np.abs(r) > INT32_MAX))
    return np.clip(r, -INT32_MAX - 1, INT32_MAX).astype(np.int64), sat


def dft_quantized(x: np.ndarray, axis: int, group: int, sign: int = -1, scale: float = SCALE):
    """The DFT of complex x along `axis` (unnormalised, e^{sign 2 pi i k t / L})
    with per-node partial sums of `group` points quantised to int32 at
    `scale` and added exactly.  Returns (result, saturated)."""
    x = np.asarray(x, dtype=np.complex128)
    L = x.shape[axis]
    if group < 1 or L % group:
        raise ValueError("group must divide the line length")
    k = np.arange(L)
    W = np.exp(sign * 2j * np.pi * np.outer(k, k) / L)  # W[k, t]
    xm = np.moveaxis(x, axis, -1)
    acc_re = np.zeros(xm.shape, dtype=np.int64)
    acc_im = np.zeros(xm.shape, dtype=np.int64)
    saturated = False
    for n in range(L // group):
        t = slice(n * group, (n + 1) * group)
        partial = xm[..., t] @ W[:, t].T  # [..., k]: this node's contribution to every output
        qr, sr = quantize(partial.real, scale)
        qi, si = quantize(partial.imag, scale)
        acc_re += qr
        acc_im += qi
        saturated = saturated or sr or si
    out = (acc_re.astype(np.float64) + 1j * acc_im.astype(np.float64)) / scale
    return np.moveaxis(out, -1, axis), saturated


def fftn_quantized(x, group, sign, axes, scale: float = SCALE):
    sat = False
    for ax in axes:
        x, s = dft_quantized(x, ax, group, sign, scale)
        sat = sat or s
    return x, sat


def pppm_quantized(o, pos, q, group: int, scale: float = SCALE):
    """Energy, forces and virial of the FP64 PPPM `o` (an oracle.pppm.OraclePPPM)
    with every transform quantised; also returns whether anything saturated."""
    box, mesh, p = o.box, o.mesh, o.p
    pos = np.asarray(pos, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    V = float(np.prod(box))
    N = int(np.prod(mesh))
    h3 = V / N
    charge = spread(pos, q, box, mesh, p) * h3  # sum_i q_i W per mesh point
    chat, s1 = fftn_quantized(charge, group, -1, (2, 1, 0), scale)
    rhohat = chat / h3
    kx, ky, kz = np.meshgrid(*wavevectors(box, mesh), indexing="ij")
    k2 = kx * kx + ky * ky + kz * kz
    e_k = V / (2.0 * N * N) * o.G * np.abs(rhohat) ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        c = np.where(k2 > 0.0, 2.0 * (1.0 + k2 / (4.0 * o.beta ** 2)) / k2, 0.0)
    virial = np.array([np.sum(e_k * (1.0 - c * kx * kx)), np.sum(e_k * (1.0 - c * ky * ky)),
                       np.sum(e_k * (1.0 - c * kz * kz)), np.sum(e_k * (-c * kx * ky)),
                       np.sum(e_k * (-c * kx * kz)), np.sum(e_k * (-c * ky * kz))])
    kd = []
    for d in range(3):
        kk = o.k[d].copy()
        if mesh[d] % 2 == 0:
            kk[mesh[d] // 2] = 0.0
        kd.append(kk)
    kdx, kdy, kdz = np.meshgrid(*kd, indexing="ij")
    phi_hat = o.G * rhohat
    fields, sat = [], s1
    for kk in (kdx, kdy, kdz):
        f, s = fftn_quantized(-1j * kk * phi_hat / N, group, +1, (0, 1, 2), scale)
        fields.append(np.real(f))
        sat = sat or s
    forces = q[:, None] * interpolate(fields, pos, box, mesh, p)
    pf = o.prefactor
    return dict(energy=pf * float(np.sum(e_k)), forces=pf * forces, virial=pf * virial, saturated=sat)
