"""Pins of the CPU oracle against facts the paper and the mathematics fix.

None of these compare the oracle with itself: each check uses a closed form,
a textbook constant, an exact identity, a finite difference, brute force on a
tiny box, or a library routine, chosen so that a dropped term, a wrong sign or
a transposed index in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

from oracle import native
from oracle.pppm import (OraclePPPM, assign, bspline_M, influence, interpolate, spread,
                         stencil_offsets, wavevectors)
from workloads.water import make_water, make_workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _nacl():
    na = [(0, 0, 0), (.5, .5, 0), (.5, 0, .5), (0, .5, .5)]
    cl = [(.5, 0, 0), (0, .5, 0), (0, 0, .5), (.5, .5, .5)]
    return np.array(na + cl, float), np.array([1.0] * 4 + [-1.0] * 4)


def _golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def _dipole_free_cell(seed=0):
    """Six charges, centrosymmetric about the box centre: neutral, zero dipole."""
    rng = np.random.default_rng(seed)
    L = np.array([3.0, 3.5, 4.0])
    c = L / 2
    d = rng.random((3, 3)) - 0.5
    pos = np.array([c + d[0], c - d[0], c + d[1], c - d[1], c + d[2], c - d[2]])
    q = np.array([1.0, 1.0, -1.5, -1.5, 0.5, 0.5])
    return pos, q, L


def _random_neutral(n, L, seed):
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 3)) * np.asarray(L)
    q = rng.normal(size=n)
    q -= q.mean()
    return pos, q


# ------------------------------------------------------------ direct E_Gt (C1)

def test_madelung_nacl():
    """Full point-charge Ewald built on the E_Gt sum reproduces the rock-salt
    Madelung constant (energy per ion pair = -M / r0, r0 = a / 2)."""
    g = _golden("madelung_nacl.txt")
    pos, q = _nacl()
    E = native.ewald_full(pos, q, 1.0, alpha=4.0)
    M = -E / 4 * 0.5
    assert abs(M - g["M"]) < g["tolerance"]


def test_ewald_alpha_invariance():
    """The split between the erfc sum and the E_Gt sum must not move the total:
    a wrong prefactor or exponent in Eq. DPLR:EGt breaks this."""
    pos, q = _nacl()
    Es = [native.ewald_full(pos, q, 1.0, alpha=a) for a in (2.0, 4.0, 6.0)]
    assert max(Es) - min(Es) < 1e-10 * abs(Es[0])
    pos, q = _random_neutral(10, [2.0, 2.5, 3.0], seed=4)
    Es = [native.ewald_full(pos, q, [2.0, 2.5, 3.0], alpha=a) for a in (2.5, 3.5, 5.0)]
    assert max(Es) - min(Es) < 1e-10 * max(abs(e) for e in Es)


def test_egt_equals_erf_image_sum():
    """E_Gt = 1/2 sum' q_i q_j erf(beta r)/r over image cells + (beta/sqrt(pi)) sum q^2
    for a neutral, dipole-free cell (no surface term), by brute force."""
    pos, q, L = _dipole_free_cell()
    beta = 0.8
    egt = native.egt_direct(pos, q, L, beta, cut=60.0, forces=False)["energy"]
    shell = native.erf_shell_sum(pos, q, L, beta, R=160.0)
    target = egt - beta / math.sqrt(math.pi) * float(np.sum(q * q))
    assert abs(shell - target) < 1e-6 * abs(target)


def test_egt_forces_finite_difference():
    pos, q = _random_neutral(7, [3.0, 3.5, 4.0], seed=1)
    L = np.array([3.0, 3.5, 4.0])
    beta = 1.1
    ref = native.egt_direct(pos, q, L, beta)
    h = 1e-5
    fd = np.zeros_like(pos)
    for j in range(pos.shape[0]):
        for d in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[j, d] += h
            pm[j, d] -= h
            fd[j, d] = -(native.egt_direct(pp, q, L, beta, forces=False)["energy"]
                         - native.egt_direct(pm, q, L, beta, forces=False)["energy"]) / (2 * h)
    assert np.linalg.norm(fd - ref["forces"]) < 1e-8 * np.linalg.norm(ref["forces"])


def test_egt_net_force_zero():
    wb, w = make_workload("water64")
    r = native.egt_direct(wb.pos, wb.q, wb.box, w["beta"])
    F = r["forces"]
    assert np.linalg.norm(F.sum(axis=0)) < 1e-12 * np.linalg.norm(F)


def _egt_general_cell(pos, q, H, beta, cut=40.0):
    """Eq. DPLR:EGt for a general cell (columns of H are the cell vectors),
    m = H^{-T} n; used only to differentiate under shear."""
    Hinv_T = np.linalg.inv(H).T
    V = abs(np.linalg.det(H))
    nmax = int(math.sqrt(cut) * beta * np.max(np.linalg.norm(H, axis=0)) / math.pi) + 3
    rng = np.arange(-nmax, nmax + 1)
    n = np.stack(np.meshgrid(rng, rng, rng, indexing="ij"), -1).reshape(-1, 3)
    n = n[np.any(n != 0, axis=1)]
    m = n @ Hinv_T.T
    m2 = np.sum(m * m, axis=1)
    keep = math.pi ** 2 * m2 / beta ** 2 <= cut
    m, m2 = m[keep], m2[keep]
    S = np.exp(-2j * math.pi * (m @ pos.T)) @ q
    return float(np.sum(np.exp(-math.pi ** 2 * m2 / beta ** 2) / m2 * np.abs(S) ** 2) / (2 * math.pi * V))


def test_egt_virial_strain_derivative():
    """Pi_ab = -dE/dF_ab under the affine deformation r -> F r, cell -> F cell,
    for all six components (off-diagonal ones through simple shear)."""
    pos, q = _random_neutral(6, [3.0, 3.5, 4.0], seed=2)
    L = np.array([3.0, 3.5, 4.0])
    beta = 1.0
    ref = native.egt_direct(pos, q, L, beta, cut=40.0, forces=False)
    H0 = np.diag(L)
    assert abs(_egt_general_cell(pos, q, H0, beta) - ref["energy"]) < 1e-12 * abs(ref["energy"])
    s = 1e-6
    comps = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    fd = []
    for a, b in comps:
        vals = []
        for sgn in (1, -1):
            F = np.eye(3)
            F[a, b] += sgn * s
            vals.append(_egt_general_cell(pos @ F.T, q, F @ H0, beta))
        fd.append(-(vals[0] - vals[1]) / (2 * s))
    fd = np.array(fd)
    assert np.linalg.norm(fd - ref["virial"]) < 1e-7 * np.linalg.norm(ref["virial"])


def test_water_is_neutral():
    for seed in (1, 2, 3):
        wb = make_water(64, 12.42, seed)
        assert abs(wb.q.sum()) < 1e-12
    for name in ("water4096", "water128"):
        wb, _ = make_workload(name)
        assert abs(wb.q.sum()) < 1e-12


@pytest.mark.parametrize("n_mol,L,seed", [(64, 12.42, 1), (128, 15.64, 4), (128, 15.64, 7)])
def test_water_geometry(n_mol, L, seed):
    wb = make_water(n_mol, L, seed)
    n = wb.n_mol
    o, h, wc = wb.pos[:n], wb.pos[n:3 * n], wb.pos[3 * n:]
    d1 = np.linalg.norm(h[0::2] - o, axis=1)
    d2 = np.linalg.norm(h[1::2] - o, axis=1)
    assert np.allclose(d1, 0.9572) and np.allclose(d2, 0.9572)
    cosang = np.sum((h[0::2] - o) * (h[1::2] - o), axis=1) / (d1 * d2)
    assert np.allclose(np.degrees(np.arccos(cosang)), 104.52)
    dw = np.linalg.norm(wc - o, axis=1)
    assert np.all((dw >= 0.1) & (dw <= 0.4))
    # minimum-image O-O distance
    dd = o[:, None, :] - o[None, :, :]
    dd -= wb.box * np.round(dd / wb.box)
    r = np.linalg.norm(dd, axis=-1) + np.eye(n) * 1e9
    assert r.min() >= 2.3


# ------------------------------------------------------------ B-spline weights

@pytest.mark.parametrize("p", [2, 3, 4, 5, 6, 7])
def test_bspline_moments(p):
    """Partition of unity and first moment: sum_k W_k = 1, sum_k (g + k) W_k = u."""
    rng = np.random.default_rng(p)
    pos = rng.random((500, 3)) * 7.3
    box = np.array([7.3, 7.3, 7.3])
    mesh = (11, 11, 11)
    idx, wts = assign(pos, box, mesh, p)
    for d in range(3):
        assert np.max(np.abs(wts[d].sum(axis=1) - 1.0)) < 1e-14
    # first moment, using unwrapped base points
    u = pos[:, 0] / (box[0] / mesh[0])
    g = np.floor(u + 0.5) if p % 2 else np.floor(u)
    pts = g[:, None] + stencil_offsets(p)[None, :]
    assert np.max(np.abs(np.sum(pts * wts[0], axis=1) - u)) < 1e-12


@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_bspline_truncated_power_definition(p):
    """M_p(x) = 1/(p-1)! sum_j (-1)^j C(p,j) (x + p/2 - j)_+^{p-1}."""
    x = np.linspace(-p / 2 - 0.3, p / 2 + 0.3, 1001)
    tp = np.zeros_like(x)
    for j in range(p + 1):
        tp += (-1) ** j * math.comb(p, j) * np.maximum(x + p / 2 - j, 0.0) ** (p - 1)
    tp /= math.factorial(p - 1)
    assert np.max(np.abs(bspline_M(p, x) - tp)) < 1e-11
    assert np.all(bspline_M(p, x[np.abs(x) >= p / 2]) == 0.0)


# ------------------------------------------------------------ influence function

def test_influence_numpy_equals_c():
    for box, mesh in (([12.42] * 3, (32, 32, 32)), ([9.0, 10.5, 12.0], (30, 36, 40)),
                      ([11.0, 9.0, 13.0], (15, 25, 27))):
        a = influence(box, mesh, 5, 0.4)
        b = native.influence_ik(box, mesh, 5, 0.4)
        assert np.max(np.abs(a - b)) <= 1e-14 * np.max(np.abs(a))


def test_influence_continuum_limit():
    """Where aliases are negligible (k h << 1, images damped by exp(-(2 pi/h)^2/(4 beta^2)))
    the optimal G is the continuum kernel of Eq. DPLR:EGt divided by the squared
    B-spline transform: G U^2(k) = 4 pi exp(-k^2/(4 beta^2)) / k^2."""
    box, mesh, beta, p = [40.0] * 3, (64, 64, 64), 0.4, 5
    h = 40.0 / 64
    G = native.influence_ik(box, mesh, p, beta)
    k = wavevectors(box, mesh)
    for (i, j, l) in ((1, 0, 0), (0, 2, 0), (1, 1, 1), (0, 0, 3), (2, 1, 0)):
        kv = (k[0][i], k[1][j], k[2][l])
        k2 = sum(c * c for c in kv)
        u2 = np.prod([np.sinc(c * h / 2 / np.pi) ** (2 * p) for c in kv])
        cont = 4 * math.pi * math.exp(-k2 / (4 * beta ** 2)) / k2
        assert abs(G[i, j, l] * u2 / cont - 1.0) < 1e-12


def test_influence_alias_range_converged():
    """Alias range 2 versus 3 in the numerator: no change at the coarsest mesh used."""
    box, mesh = [129.3 / 4] * 3, (16, 16, 16)  # same 2.02 A spacing as 64^3 on 129.3 A
    g2 = native.influence_ik(box, mesh, 5, 0.4, alias=2)
    g3 = native.influence_ik(box, mesh, 5, 0.4, alias=3)
    assert np.max(np.abs(g3 - g2)) <= 1e-12 * np.max(np.abs(g2))


# ------------------------------------------------------------ CPU PPPM (C2)

def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def test_pppm_vs_direct_water64():
    """PPPM 32^3, p = 5 against the direct sum on the 64-water box.
    Recorded errors: force 9.96e-6, energy 2.3e-6, virial 1.3e-5."""
    wb, w = make_workload("water64")
    ref = native.egt_direct(wb.pos, wb.q, wb.box, w["beta"])
    r = OraclePPPM(wb.box, w["mesh"], w["order"], w["beta"]).compute(wb.pos, wb.q)
    assert _rel(r["forces"], ref["forces"]) < 1.2e-5
    assert abs(r["energy"] - ref["energy"]) < 5e-6 * abs(ref["energy"])
    assert _rel(r["virial"], ref["virial"]) < 3e-5


def test_pppm_converges_with_mesh_and_order():
    wb, w = make_workload("water64")
    ref = native.egt_direct(wb.pos, wb.q, wb.box, w["beta"])
    errs_mesh = [_rel(OraclePPPM(wb.box, (m,) * 3, 5, 0.4).compute(wb.pos, wb.q)["forces"], ref["forces"])
                 for m in (24, 32, 48)]
    errs_p = [_rel(OraclePPPM(wb.box, (32,) * 3, p, 0.4).compute(wb.pos, wb.q)["forces"], ref["forces"])
              for p in (3, 5, 7)]
    assert errs_mesh[0] > errs_mesh[1] > errs_mesh[2]
    assert errs_p[0] > errs_p[1] > errs_p[2]
    assert errs_p[2] < 1e-6


def test_pppm_rectangular_radix235_vs_direct():
    """Non-cubic box, meshes with factors 2, 3, 5 and odd sizes, even order too."""
    pos, q = _random_neutral(40, [9.0, 10.5, 12.0], seed=7)
    box = np.array([9.0, 10.5, 12.0])
    ref = native.egt_direct(pos, q, box, 0.5)
    for mesh, p, tol in (((30, 36, 40), 5, 1e-5), ((27, 25, 45), 5, 1e-5), ((30, 36, 40), 4, 1e-4)):
        r = OraclePPPM(box, mesh, p, 0.5).compute(pos, q)
        assert _rel(r["forces"], ref["forces"]) < tol, (mesh, p)
        assert abs(r["energy"] - ref["energy"]) < tol * abs(ref["energy"]), (mesh, p)


def test_pppm_energy_equals_half_q_phi():
    """With the same G in the energy and the potential, 1/2 sum_i q_i phi(r_i) = E."""
    wb, w = make_workload("water64")
    o = OraclePPPM(wb.box, w["mesh"], w["order"], w["beta"])
    E = o.compute(wb.pos, wb.q)["energy"]
    phi = o.site_potential(wb.pos, wb.q)
    assert abs(0.5 * np.dot(wb.q, phi) - E) < 1e-13 * abs(E)


def test_pppm_translation_by_one_cell():
    wb, w = make_workload("water64")
    o = OraclePPPM(wb.box, w["mesh"], w["order"], w["beta"])
    r0 = o.compute(wb.pos, wb.q)
    shift = np.array([wb.box[0] / w["mesh"][0], 0.0, 2 * wb.box[2] / w["mesh"][2]])
    r1 = o.compute(wb.pos + shift, wb.q)
    assert abs(r1["energy"] - r0["energy"]) < 1e-13 * abs(r0["energy"])
    assert _rel(r1["forces"], r0["forces"]) < 1e-12
    assert _rel(r1["virial"], r0["virial"]) < 1e-12


def test_pppm_wrap_invariance():
    """Positions shifted by whole box vectors give the same result."""
    wb, w = make_workload("water64")
    o = OraclePPPM(wb.box, w["mesh"], w["order"], w["beta"])
    r0 = o.compute(wb.pos, wb.q)
    pos = wb.pos + wb.box * np.random.default_rng(0).integers(-2, 3, size=wb.pos.shape)
    r1 = o.compute(pos, wb.q)
    assert abs(r1["energy"] - r0["energy"]) < 1e-12 * abs(r0["energy"])
    assert _rel(r1["forces"], r0["forces"]) < 1e-12


def test_pppm_spread_conserves_charge_and_dipole():
    """sum_p rho_p h^3 = sum_i q_i, and (away from the wrap) the first moment of
    the mesh charge equals the dipole of the sites (B-spline moment identity)."""
    rng = np.random.default_rng(3)
    box = np.array([10.0, 10.0, 10.0])
    pos = 3.0 + 4.0 * rng.random((30, 3))
    q = rng.normal(size=30)
    mesh = (20, 20, 20)
    rho = spread(pos, q, box, mesh, 5)
    h = box / np.asarray(mesh)
    assert abs(rho.sum() * np.prod(h) - q.sum()) < 1e-12
    xs = np.arange(20) * h[0]
    dip = np.sum(rho.sum(axis=(1, 2)) * xs) * np.prod(h)
    assert abs(dip - np.dot(q, pos[:, 0])) < 1e-11


def test_pppm_interpolate_is_spread_transpose():
    """<rho(pos), f> h^3 = sum_i q_i (interp f)(r_i): the gather uses the same stencil."""
    rng = np.random.default_rng(5)
    box = np.array([8.0, 9.0, 7.0])
    mesh = (16, 18, 15)
    pos = rng.random((25, 3)) * box
    q = rng.normal(size=25)
    f = rng.normal(size=mesh)
    lhs = np.sum(spread(pos, q, box, mesh, 5) * f) * np.prod(box / np.asarray(mesh))
    rhs = np.dot(q, interpolate([f], pos, box, mesh, 5)[:, 0])
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)


def test_pppm_virial_vs_direct_rectangular():
    pos, q = _random_neutral(40, [9.0, 10.5, 12.0], seed=8)
    box = np.array([9.0, 10.5, 12.0])
    ref = native.egt_direct(pos, q, box, 0.5)
    r = OraclePPPM(box, (36, 40, 45), 7, 0.5).compute(pos, q)
    assert _rel(r["virial"], ref["virial"]) < 1e-6


@pytest.mark.slow
def test_pppm_vs_direct_water4096():
    """64^3 mesh, 16,384 sites: record the discretisation error (h = 0.78 A).
    Recorded: force 3.17e-4, energy 4.58e-4 relative."""
    wb, w = make_workload("water4096")
    ref = native.egt_direct(wb.pos, wb.q, wb.box, w["beta"])
    r = OraclePPPM(wb.box, w["mesh"], w["order"], w["beta"]).compute(wb.pos, wb.q)
    ferr = _rel(r["forces"], ref["forces"])
    eerr = abs(r["energy"] - ref["energy"]) / abs(ref["energy"])
    print(f"water4096 64^3: force rel err {ferr:.3e}, energy rel err {eerr:.3e}")
    assert ferr < 1e-3 and eerr < 1e-3  # recorded: 3.17e-4 and 4.58e-4
