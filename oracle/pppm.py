"""Plain FP64 CPU PPPM (Poisson-ik) for Gaussian charges -- the oracle.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code,
table or constant generator with the CUDA implementation.

What it computes is the PPPM estimate of E_Gt (Eq. DPLR:EGt, Section 2.1) with
the Poisson-ik solver the paper names (Section 3.1: one forward and three
inverse 3D FFTs), step by step:

1. wrap each position into [0, L); u = x / h with h = L / N per axis;
2. order-p assignment: the p mesh points nearest to u get weights
   W = M_p(g + k - u), M_p the centred cardinal B-spline of order p, computed
   with the Cox-de Boor recursion;
3. rho_p = sum_i q_i Wx Wy Wz / (hx hy hz) (periodic);
4. rho_hat = DFT(rho) (``numpy.fft.fftn`` as the library step, full spectrum);
5. G(k): the Hockney-Eastwood optimal influence function for ik
   differentiation with the Gaussian reference force of Eq. DPLR:EGt;
6. E = V / (2 N^2) sum_{k != 0} G |rho_hat|^2 over the full spectrum;
7. Pi_ab = V / (2 N^2) sum_{k != 0} G |rho_hat|^2
          (delta_ab - 2 (1 + k^2 / (4 beta^2)) k_a k_b / k^2);
8. E_d = IDFT(-i k_d G rho_hat) (``numpy.fft.ifftn``, which carries the 1/N),
   with k_d set to 0 on the Nyquist index of an even axis;
9. F_i = q_i sum Wx Wy Wz (E_x, E_y, E_z) over the same stencil;
10. E, Pi and F are multiplied by ``prefactor``.

Readings where the paper is silent are those listed in the design notes:
beta is the Ewald splitting parameter (an inverse length), no k = 0 term, a
conducting (tin-foil) boundary, wavevector index m = i for i <= N/2 else i - N,
and alias range 2 in the numerator of G (the separable denominator summed to
|n| <= 20).
"""
from __future__ import annotations

import numpy as np


def bspline_N(p: int, t: np.ndarray) -> np.ndarray:
    """Uniform cardinal B-spline of order p with support [0, p) by the Cox-de Boor
    recursion N_1 = 1 on [0, 1); N_p(t) = (t N_{p-1}(t) + (p - t) N_{p-1}(t - 1)) / (p - 1)."""
    if p == 1:
        return ((t >= 0.0) & (t < 1.0)).astype(np.float64)
    return (t * bspline_N(p - 1, t) + (p - t) * bspline_N(p - 1, t - 1.0)) / (p - 1)


def bspline_M(p: int, x: np.ndarray) -> np.ndarray:
    """Centred cardinal B-spline of order p: M_p(x) = N_p(x + p/2)."""
    return bspline_N(p, np.asarray(x, dtype=np.float64) + 0.5 * p)


def stencil_offsets(p: int) -> np.ndarray:
    """Offsets k of the p stencil points relative to the base point g."""
    if p % 2 == 1:
        return np.arange(-(p - 1) // 2, (p - 1) // 2 + 1)
    return np.arange(-p // 2 + 1, p // 2 + 1)


def assign(pos: np.ndarray, box: np.ndarray, mesh, p: int):
    """Per axis: mesh indices (n, p) and B-spline weights (n, p) of every site."""
    pos = np.asarray(pos, dtype=np.float64)
    idx, wts = [], []
    ks = stencil_offsets(p)
    for d in range(3):
        L, N = float(box[d]), int(mesh[d])
        x = pos[:, d] - L * np.floor(pos[:, d] / L)
        x = np.where(x >= L, 0.0, x)
        h = L / N
        u = x / h
        g = np.floor(u + 0.5) if p % 2 == 1 else np.floor(u)
        pts = g[:, None] + ks[None, :]
        wts.append(bspline_M(p, pts - u[:, None]))
        idx.append(np.mod(pts.astype(np.int64), N))
    return idx, wts


def spread(pos, q, box, mesh, p):
    """Charge density rho on the mesh, shape mesh, (step 3)."""
    Nx, Ny, Nz = (int(m) for m in mesh)
    (ix, iy, iz), (wx, wy, wz) = assign(pos, box, mesh, p)
    rho = np.zeros(Nx * Ny * Nz)
    q = np.asarray(q, dtype=np.float64)
    for a in range(p):
        for b in range(p):
            for c in range(p):
                flat = (ix[:, a] * Ny + iy[:, b]) * Nz + iz[:, c]
                rho += np.bincount(flat, weights=q * wx[:, a] * wy[:, b] * wz[:, c],
                                   minlength=rho.size)
    h3 = np.prod(np.asarray(box, float) / np.asarray(mesh, float))
    return rho.reshape(Nx, Ny, Nz) / h3


def interpolate(fields, pos, box, mesh, p):
    """sum_stencil Wx Wy Wz f over the same stencil as the spread, for each field."""
    (ix, iy, iz), (wx, wy, wz) = assign(pos, box, mesh, p)
    out = np.zeros((pos.shape[0], len(fields)))
    for a in range(p):
        for b in range(p):
            for c in range(p):
                w = wx[:, a] * wy[:, b] * wz[:, c]
                for f, fld in enumerate(fields):
                    out[:, f] += w * fld[ix[:, a], iy[:, b], iz[:, c]]
    return out


def wavevectors(box, mesh):
    """k_d = 2 pi m_d / L_d with m = i for i <= N/2 else i - N, as 1D arrays."""
    ks = []
    for d in range(3):
        N = int(mesh[d])
        i = np.arange(N)
        m = np.where(i <= N // 2, i, i - N)
        ks.append(2.0 * np.pi * m / float(box[d]))
    return ks


def _sinc(x):
    """sin(x)/x with the value 1 at 0."""
    return np.sinc(np.asarray(x) / np.pi)


def influence(box, mesh, p, beta, alias: int = 2, denom_range: int = 20):
    """Hockney-Eastwood optimal influence function for ik differentiation.

    G(k) = sum_n (k . k_n / k_n^2) 4 pi exp(-k_n^2 / (4 beta^2)) U^2(k_n)
           / ( k^2 [ sum_n U^2(k_n) ]^2 ),
    k_n = k + 2 pi n / h (per axis), U(k) = prod_d sinc(k_d h_d / 2)^p.
    The numerator runs over n in [-alias, alias]^3; the denominator is separable
    and each axis factor runs over |n_d| <= denom_range.  G(0) = 0.
    """
    box = np.asarray(box, float)
    mesh = [int(m) for m in mesh]
    h = box / np.asarray(mesh, float)
    k1 = wavevectors(box, mesh)
    den = []
    for d in range(3):
        s = np.zeros(mesh[d])
        for nd in range(-denom_range, denom_range + 1):
            kn = k1[d] + 2.0 * np.pi * nd / h[d]
            s += _sinc(kn * h[d] / 2.0) ** (2 * p)
        den.append(s)
    kx, ky, kz = np.meshgrid(*k1, indexing="ij")
    k2 = kx * kx + ky * ky + kz * kz
    num = np.zeros(mesh)
    for nx in range(-alias, alias + 1):
        for ny in range(-alias, alias + 1):
            for nz in range(-alias, alias + 1):
                knx = kx + 2.0 * np.pi * nx / h[0]
                kny = ky + 2.0 * np.pi * ny / h[1]
                knz = kz + 2.0 * np.pi * nz / h[2]
                kn2 = knx * knx + kny * kny + knz * knz
                u2 = (_sinc(knx * h[0] / 2) * _sinc(kny * h[1] / 2) * _sinc(knz * h[2] / 2)) ** (2 * p)
                dot = kx * knx + ky * kny + kz * knz
                with np.errstate(divide="ignore", invalid="ignore"):
                    term = np.where(kn2 > 0.0, dot / kn2 * 4.0 * np.pi * np.exp(-kn2 / (4.0 * beta * beta)) * u2, 0.0)
                num += term
    dprod = den[0][:, None, None] * den[1][None, :, None] * den[2][None, None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        G = np.where(k2 > 0.0, num / (k2 * dprod * dprod), 0.0)
    return G


class OraclePPPM:
    """FP64 CPU PPPM for one box; G is computed once at construction (plan time)."""

    def __init__(self, box, mesh, order, beta, prefactor=1.0, alias=2):
        self.box = np.asarray(box, dtype=np.float64).reshape(3)
        self.mesh = tuple(int(m) for m in mesh)
        self.p = int(order)
        self.beta = float(beta)
        self.prefactor = float(prefactor)
        from . import native
        # plain C loops of the same formula as `influence` (agreement is tested)
        self.G = native.influence_ik(self.box, self.mesh, self.p, self.beta, alias=alias)
        self.k = wavevectors(self.box, self.mesh)

    def compute(self, pos, q, want_intermediates=False):
        box, mesh, p = self.box, self.mesh, self.p
        pos = np.asarray(pos, dtype=np.float64)
        q = np.asarray(q, dtype=np.float64)
        V = float(np.prod(box))
        N = int(np.prod(mesh))
        rho = spread(pos, q, box, mesh, p)
        rhohat = np.fft.fftn(rho)
        G = self.G
        kx, ky, kz = np.meshgrid(*self.k, indexing="ij")
        k2 = kx * kx + ky * ky + kz * kz
        e_k = V / (2.0 * N * N) * G * np.abs(rhohat) ** 2
        energy = float(np.sum(e_k))
        with np.errstate(divide="ignore", invalid="ignore"):
            c = np.where(k2 > 0.0, 2.0 * (1.0 + k2 / (4.0 * self.beta ** 2)) / k2, 0.0)
        virial = np.array([
            np.sum(e_k * (1.0 - c * kx * kx)),
            np.sum(e_k * (1.0 - c * ky * ky)),
            np.sum(e_k * (1.0 - c * kz * kz)),
            np.sum(e_k * (-c * kx * ky)),
            np.sum(e_k * (-c * kx * kz)),
            np.sum(e_k * (-c * ky * kz)),
        ])
        # ik differentiation; the derivative multiplier is 0 on a Nyquist index
        kd = []
        for d in range(3):
            kk = self.k[d].copy()
            if mesh[d] % 2 == 0:
                kk[mesh[d] // 2] = 0.0
            kd.append(kk)
        kdx, kdy, kdz = np.meshgrid(*kd, indexing="ij")
        phi_hat = G * rhohat
        fields = [np.real(np.fft.ifftn(-1j * kk * phi_hat)) for kk in (kdx, kdy, kdz)]
        forces = q[:, None] * interpolate(fields, pos, box, mesh, p)
        pf = self.prefactor
        out = dict(energy=pf * energy, forces=pf * forces, virial=pf * virial)
        if want_intermediates:
            out["rho"] = rho
            out["rhohat"] = rhohat
            out["fields"] = fields
            out["phi"] = np.real(np.fft.ifftn(phi_hat))
        return out

    def site_potential(self, pos, q):
        """phi(r_i) interpolated from the mesh potential IDFT(G rho_hat)."""
        r = self.compute(pos, q, want_intermediates=True)
        return interpolate([r["phi"]], np.asarray(pos, float), self.box, self.mesh, self.p)[:, 0]
