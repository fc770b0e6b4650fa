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
saturated).  ``pppm_quantized`` is the FP64 PPPM of ``oracle.pppm`` with the
1D transforms along the chosen axes replaced by this one, in the axis order the
library uses (forward z, y, x; inverse x, y, z).  Readings where the paper is
silent:

* What is transformed.  The fixed scale makes the error depend on it and the
  paper only says that most values lie in [-1, 1].  Taken: the charge per mesh
  point sum_i q_i W (not divided by h^3) forward, and each field spectrum
  -i k_d phi_hat already divided by N h^3 backward (so the inverse transforms
  give the fields directly), each of the three formed before its first pass.
* Real or complex transforms.  In exact arithmetic a complex 3D FFT of the
  real mesh and the real-to-complex / complex-to-real pair agree; quantised,
  they do not, because a backward pass splits the FREQUENCY index into nodes
  and the mirror k -> -k maps that split onto a different one, so quantised
  backward passes of a Hermitian spectrum are not Hermitian.  Taken
  (``spectrum="half"``, the default): the pair that PPPM codes use for the real
  mesh -- forward, the z transform of each real line keeps kz <= Nz/2 and the
  y and x transforms act on that half; backward, x and y act on the half and
  the z transform takes each line's Hermitian extension (kz > Nz/2 from the
  conjugates) and keeps the real part.  ``spectrum="full"`` is the complex
  reading (every transform on all Nx Ny Nz points).
* Exact ties.  After the first quantised pass the values are integers over the
  scale, so with twiddles of +-1/2 a partial sum can be exactly half an integer;
  which way it rounds is then decided by the rounding of the partial sum
  itself (FP64 here).
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


def _transform(x, axis, group, sign, scale, quantised):
    """One axis: the quantised DFT, or the exact one (numpy) if not quantised."""
    if quantised:
        return dft_quantized(x, axis, group, sign, scale)
    if sign < 0:
        return np.fft.fft(x, axis=axis), False
    return np.fft.ifft(x, axis=axis) * x.shape[axis], False


def _ik_multipliers(o):
    """k_d per axis with the Nyquist component of an even mesh set to zero
    (the ik differentiation of Eq. 12)."""
    kd = []
    for d in range(3):
        kk = o.k[d].copy()
        if o.mesh[d] % 2 == 0:
            kk[o.mesh[d] // 2] = 0.0
        kd.append(kk)
    return kd


def pppm_quantized(o, pos, q, group: int, scale: float = SCALE, axes=(0, 1, 2), spectrum: str = "half"):
    """Energy, forces and virial of the FP64 PPPM `o` (an oracle.pppm.OraclePPPM)
    with the transforms along `axes` quantised at `scale` with nodes of `group`
    points (the other axes exact); also returns whether anything saturated.
    `spectrum`: "half" (real-to-complex pair, the default) or "full"."""
    box, mesh, p = o.box, tuple(int(m) for m in o.mesh), o.p
    for ax in axes:
        if mesh[ax] % group:
            raise ValueError("group must divide the quantised axes")
    if spectrum not in ("half", "full"):
        raise ValueError("spectrum is 'half' or 'full'")
    Nx, Ny, Nz = mesh
    Hz = Nz // 2 + 1 if spectrum == "half" else Nz
    pos = np.asarray(pos, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    V = float(np.prod(box))
    N = Nx * Ny * Nz
    h3 = V / N
    sat = False

    def step(x, ax, sign):
        nonlocal sat
        y, s = _transform(x, ax, group, sign, scale, ax in axes)
        sat = sat or s
        return y

    def hermitian_extension(x):
        """The full z extent of a half spectrum: kz > Nz/2 from conj(x[.., Nz - kz])."""
        if spectrum == "full":
            return x
        full = np.empty(x.shape[:2] + (Nz,), dtype=np.complex128)
        full[:, :, :Hz] = x
        for kz in range(Hz, Nz):
            full[:, :, kz] = np.conj(x[:, :, Nz - kz])
        return full

    # forward: the charge per mesh point, z (kept up to Hz), y, x
    charge = spread(pos, q, box, mesh, p) * h3
    x = step(charge.astype(np.complex128), 2, -1)[:, :, :Hz]
    x = step(step(x, 1, -1), 0, -1)
    chat = x / h3
    # energy and virial (Eqs. 7, 10) over the whole spectrum
    rhohat = chat
    if spectrum == "half":
        # kz > Nz/2 by the symmetry of the transform of a real mesh:
        # rho_hat(k) = conj(rho_hat(-k)), all three indices mirrored
        rhohat = np.empty((Nx, Ny, Nz), dtype=np.complex128)
        rhohat[:, :, :Hz] = chat
        mx, my = (-np.arange(Nx)) % Nx, (-np.arange(Ny)) % Ny
        for kz in range(Hz, Nz):
            rhohat[:, :, kz] = np.conj(chat[np.ix_(mx, my)][:, :, Nz - kz])
    kx, ky, kz = np.meshgrid(*wavevectors(box, mesh), indexing="ij")
    k2 = kx * kx + ky * ky + kz * kz
    e_k = V / (2.0 * N * N) * o.G * np.abs(rhohat) ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        c = np.where(k2 > 0.0, 2.0 * (1.0 + k2 / (4.0 * o.beta ** 2)) / k2, 0.0)
    virial = np.array([np.sum(e_k * (1.0 - c * kx * kx)), np.sum(e_k * (1.0 - c * ky * ky)),
                       np.sum(e_k * (1.0 - c * kz * kz)), np.sum(e_k * (-c * kx * ky)),
                       np.sum(e_k * (-c * kx * kz)), np.sum(e_k * (-c * ky * kz))])
    # backward: each -i k_d phi_hat / N through x, y, then z (real part)
    kdx, kdy, kdz = np.meshgrid(*_ik_multipliers(o), indexing="ij")
    phi_hat = o.G[:, :, :Hz] * chat
    fields = []
    for kk in (kdx, kdy, kdz):
        y = step(step(-1j * kk[:, :, :Hz] * phi_hat / N, 0, +1), 1, +1)
        fields.append(np.real(step(hermitian_extension(y), 2, +1)))
    forces = q[:, None] * interpolate(fields, pos, box, mesh, p)
    pf = o.prefactor
    return dict(energy=pf * float(np.sum(e_k)), forces=pf * forces, virial=pf * virial, saturated=sat)
