"""Seeded synthetic water boxes shaped like the systems of the DPLR paper.

This module only draws inputs: it holds none of the electrostatics. Both the
CPU oracle and the CUDA path consume what it returns, so it is the one piece
of code the two share.

A water molecule carries three charged sites, as in the DPLR model (the
Gaussian-charge picture of Section 2.1, Eqs. DPLR:Sm and DPLR:Wn): the oxygen
ion (+6), two hydrogen ions (+1 each) and one Wannier centroid (WC, -8) bound
to the oxygen.  The WC sits at W_n = R_O + Delta_n (Eq. DPLR:Wn); here Delta_n
is drawn, not predicted by a network: a displacement of 0.1-0.4 Angstrom along
the H-O-H bisector, towards the hydrogens.

Recipe (all lengths in Angstrom):

* oxygens on a jittered cubic lattice: ``ns = ceil(n_mol ** (1/3))`` points per
  side at spacing ``L / ns``; ``n_mol`` distinct lattice points are picked by a
  seeded permutation; each oxygen is jittered uniformly by up to
  ``min(0.2, (spacing - 2.3) / 2)`` per axis, so no two oxygens come closer
  than 2.3;
* each molecule gets a uniformly random orientation (Shoemake's quaternion
  recipe);
* rigid geometry: O-H 0.9572, H-O-H 104.52 degrees;
* site order is ``[all O, all H (H1, H2 of each molecule interleaved), all WC]``
  with type ids 0 = O, 1 = H, 2 = WC.

Hydrogens and WCs may lie slightly outside ``[0, L)``; a PPPM solver must wrap
positions itself.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

OH_BOND = 0.9572
HOH_ANGLE_DEG = 104.52
CHARGE_O = 6.0
CHARGE_H = 1.0
CHARGE_WC = -8.0
TYPE_O, TYPE_H, TYPE_WC = 0, 1, 2
VOLUME_PER_MOLECULE = 29.9  # Angstrom^3, liquid water density


@dataclass
class WaterBox:
    pos: np.ndarray      # (n, 3) float64
    q: np.ndarray        # (n,) float64
    types: np.ndarray    # (n,) int8
    box: np.ndarray      # (3,) float64, orthorhombic edge lengths
    n_mol: int

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def _shoemake_rotations(rng: np.random.Generator, m: int) -> np.ndarray:
    """m uniformly distributed rotation matrices, shape (m, 3, 3)."""
    u1, u2, u3 = rng.random(m), rng.random(m), rng.random(m)
    a = np.sqrt(1.0 - u1)
    b = np.sqrt(u1)
    x = a * np.sin(2 * np.pi * u2)
    y = a * np.cos(2 * np.pi * u2)
    z = b * np.sin(2 * np.pi * u3)
    w = b * np.cos(2 * np.pi * u3)
    r = np.empty((m, 3, 3))
    r[:, 0, 0] = 1 - 2 * (y * y + z * z)
    r[:, 0, 1] = 2 * (x * y - z * w)
    r[:, 0, 2] = 2 * (x * z + y * w)
    r[:, 1, 0] = 2 * (x * y + z * w)
    r[:, 1, 1] = 1 - 2 * (x * x + z * z)
    r[:, 1, 2] = 2 * (y * z - x * w)
    r[:, 2, 0] = 2 * (x * z - y * w)
    r[:, 2, 1] = 2 * (y * z + x * w)
    r[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return r


def make_water(n_mol: int, L: float, seed: int) -> WaterBox:
    """A cubic periodic box of edge L holding n_mol rigid waters plus one WC each."""
    if n_mol < 1:
        raise ValueError("n_mol must be >= 1")
    rng = np.random.default_rng(seed)
    ns = int(math.ceil(round(n_mol ** (1.0 / 3.0), 9)))
    while ns ** 3 < n_mol:
        ns += 1
    spacing = L / ns
    jitter = min(0.2, (spacing - 2.3) / 2.0)
    if jitter < 0.0:
        raise ValueError(f"box too dense: lattice spacing {spacing:.3f} < 2.3 Angstrom")
    pick = rng.permutation(ns ** 3)[:n_mol]
    ix, iy, iz = pick // (ns * ns), (pick // ns) % ns, pick % ns
    o = (np.stack([ix, iy, iz], axis=1) + 0.5) * spacing
    o = o + rng.uniform(-jitter, jitter, size=o.shape)

    half = math.radians(HOH_ANGLE_DEG) / 2.0
    body_h1 = np.array([math.sin(half), math.cos(half), 0.0]) * OH_BOND
    body_h2 = np.array([-math.sin(half), math.cos(half), 0.0]) * OH_BOND
    body_bis = np.array([0.0, 1.0, 0.0])
    rot = _shoemake_rotations(rng, n_mol)
    delta = rng.uniform(0.1, 0.4, size=n_mol)

    h1 = o + rot @ body_h1
    h2 = o + rot @ body_h2
    wc = o + (rot @ body_bis) * delta[:, None]
    h = np.empty((2 * n_mol, 3))
    h[0::2], h[1::2] = h1, h2

    pos = np.concatenate([o, h, wc], axis=0)
    q = np.concatenate([np.full(n_mol, CHARGE_O), np.full(2 * n_mol, CHARGE_H),
                        np.full(n_mol, CHARGE_WC)])
    types = np.concatenate([np.full(n_mol, TYPE_O), np.full(2 * n_mol, TYPE_H),
                            np.full(n_mol, TYPE_WC)]).astype(np.int8)
    return WaterBox(pos=pos, q=q, types=types, box=np.array([L, L, L], float), n_mol=n_mol)


def perturb(pos: np.ndarray, sigma: float, rng: np.random.Generator) -> np.ndarray:
    """One step of the random walk used for the 1,000-step workload: every
    coordinate gets independent N(0, sigma) noise (cumulative across steps)."""
    return pos + rng.normal(0.0, sigma, size=pos.shape)


def smooth_at_least(x: float) -> int:
    """Smallest 2^a 3^b 5^c that is >= x."""
    n = max(1, int(math.ceil(x - 1e-12)))
    while True:
        m = n
        for r in (2, 3, 5):
            while m % r == 0:
                m //= r
        if m == 1:
            return n
        n += 1


# ----------------------------------------------------------------- workloads
# Sizes of the paper's water systems: 64 waters in a ~12.4 A box (a small
# variant of the 128-water Table 1 box), 4,096 waters, and 72,192 waters =
# the 216,576-atom system of the 4,608-node weak-scaling point (Section 4.4).

WORKLOADS = {
    "water64": dict(n_mol=64, L=12.42, mesh=(32, 32, 32), order=5, beta=0.4, seed=1),
    # 128 waters in a ~16 A box, the system of the paper's accuracy table; its
    # int32 runs use the meshes 8x12x8, 10x15x10 and 12x18x12
    "water128": dict(n_mol=128, L=15.64, mesh=(12, 18, 12), order=5, beta=0.4, seed=4),
    "water4096": dict(n_mol=4096, L=49.7, mesh=(64, 64, 64), order=5, beta=0.4, seed=2),
    "water72192_m128": dict(n_mol=72192, L=129.3, mesh=(128, 128, 128), order=5, beta=0.4, seed=3),
    "water72192_m160": dict(n_mol=72192, L=129.3, mesh=(160, 160, 160), order=5, beta=0.4, seed=3),
    "water72192_m64": dict(n_mol=72192, L=129.3, mesh=(64, 64, 64), order=5, beta=0.4, seed=3),
}
NOISE_SEED_1000_STEPS = 30
NOISE_SIGMA_1000_STEPS = 0.01


def make_workload(name: str) -> tuple[WaterBox, dict]:
    w = WORKLOADS[name]
    return make_water(w["n_mol"], w["L"], w["seed"]), w


def batched_boxes(nbox: int = 96, seed: int = 5, lo: int = 64, hi: int = 8192,
                  spacing: float = 1.2) -> list[dict]:
    """Sizes of the many-small-boxes workload: molecule counts drawn
    log-uniformly in [lo, hi], cubic boxes at 29.9 A^3 per molecule, and a mesh
    per box with spacing <= `spacing` rounded up to a 2^a 3^b 5^c size."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(nbox):
        n_mol = int(math.floor(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        L = (VOLUME_PER_MOLECULE * n_mol) ** (1.0 / 3.0)
        m = smooth_at_least(L / spacing)
        out.append(dict(n_mol=n_mol, L=L, mesh=(m, m, m), seed=1000 + b))
    return out


def init_mlp_params(seed: int, n_in: int = 48, n_hidden: int = 64, n_out: int = 3) -> np.ndarray:
    """Seeded initial parameters of the correction network, as one float32
    vector [W1 (n_hidden x n_in), b1, W2 (n_hidden x n_hidden), b2,
    W3 (n_out x n_hidden), b3]: Glorot-uniform weights, zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in ((n_hidden, n_in), (n_hidden, n_hidden), (n_out, n_hidden)):
        lim = math.sqrt(6.0 / (fan_in + fan_out))
        parts.append(rng.uniform(-lim, lim, size=fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)


def dw_jacobian(wb: WaterBox, seed: int, scale: float = 0.02, dtype=np.float64, values: bool = True):
    """A synthetic Deep-Wannier Jacobian for the fold of Eq. DPLR:F_final, with
    the sparsity of a local model: the displacement Delta_n of the WC of
    molecule n depends on the three atoms of every molecule whose lattice
    point lies within one lattice step of n's (periodic; 27 molecules, 81
    atoms when all points are occupied).  Blocks are N(0, scale) 3 x 3.

    Atoms are the first 3 n_mol sites (O then H), WC n is hosted by O n.
    Returns compressed rows per atom: host_ptr (int32), host_wc (int32),
    jac_ptr (int64), jac_wc (int32), jac (nnz x 3 x 3, ``dtype``; None without
    ``values``, for callers that draw the blocks themselves)."""
    n_mol = wb.n_mol
    L = float(wb.box[0])
    ns = int(math.ceil(round(n_mol ** (1.0 / 3.0), 9)))
    while ns ** 3 < n_mol:
        ns += 1
    spacing = L / ns
    o = wb.pos[:n_mol]
    lat = np.floor(o / spacing).astype(np.int64) % ns
    grid = np.full((ns, ns, ns), -1, np.int64)
    grid[lat[:, 0], lat[:, 1], lat[:, 2]] = np.arange(n_mol)
    offs = np.array([(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)])
    cx = (lat[:, None, 0] + offs[None, :, 0]) % ns
    cy = (lat[:, None, 1] + offs[None, :, 1]) % ns
    cz = (lat[:, None, 2] + offs[None, :, 2]) % ns
    nb = grid.ravel()[(cx * ns + cy) * ns + cz]                      # (n_mol, 27) molecule or -1
    # the relation is symmetric: atom j of molecule m feeds the WCs of m's neighbours
    nbs = np.sort(nb, axis=1)
    valid = nbs >= 0
    cnt = valid.sum(axis=1)
    o_rows = nbs[valid]                                              # O atoms, molecule order
    h_rows = np.repeat(nbs, 2, axis=0)[np.repeat(valid, 2, axis=0)]  # H1, H2 of each molecule
    wcs = np.concatenate([o_rows, h_rows])
    n_atoms = 3 * n_mol
    jac_ptr = np.zeros(n_atoms + 1, np.int64)
    jac_ptr[1:] = np.cumsum(np.concatenate([cnt, np.repeat(cnt, 2)]))
    jac = None
    if values:
        rng = np.random.default_rng(seed)
        jac = (rng.standard_normal(size=(wcs.size, 3, 3), dtype=np.float32) * np.float32(scale)).astype(dtype)
    host_ptr = np.zeros(n_atoms + 1, np.int32)
    host_ptr[1:n_mol + 1] = np.arange(1, n_mol + 1)
    host_ptr[n_mol + 1:] = n_mol
    host_wc = np.arange(n_mol, dtype=np.int32)
    return host_ptr, host_wc, jac_ptr, wcs.astype(np.int32), jac
