"""Pins of the FP64 reference of the WC force fold (Eq. DPLR:F_final)."""
import numpy as np

from oracle import native
from oracle.wc_fold import fold


def _linear_model(n_atoms, n_wc, rng, deg=4):
    """Delta_n = sum_j A_nj (R_j - R_host(n)) over a few atoms j: a synthetic
    displacement model with an exact Jacobian (A_nj for j != host,
    -sum A_nj for the host)."""
    host = rng.permutation(n_atoms)[:n_wc]
    nb = [rng.choice([j for j in range(n_atoms) if j != host[n]], size=deg, replace=False) for n in range(n_wc)]
    A = rng.normal(size=(n_wc, deg, 3, 3)) * 0.05

    def wc_pos(R):
        W = R[host].copy()
        for n in range(n_wc):
            for k, j in enumerate(nb[n]):
                W[n] += A[n, k] @ (R[j] - R[host[n]])
        return W

    rows = [[] for _ in range(n_atoms)]
    for n in range(n_wc):
        for k, j in enumerate(nb[n]):
            rows[j].append((n, A[n, k]))
        rows[host[n]].append((n, -A[n].sum(axis=0)))
    jac_ptr = np.zeros(n_atoms + 1, np.int64)
    jac_wc, jac = [], []
    for j in range(n_atoms):
        for n, blk in rows[j]:
            jac_wc.append(n)
            jac.append(blk)
        jac_ptr[j + 1] = len(jac_wc)
    host_ptr = np.zeros(n_atoms + 1, np.int64)
    host_wc = []
    for j in range(n_atoms):
        for n in np.nonzero(host == j)[0]:
            host_wc.append(n)
        host_ptr[j + 1] = len(host_wc)
    return wc_pos, host_ptr, np.array(host_wc), jac_ptr, np.array(jac_wc), np.array(jac)


def test_fold_equals_finite_difference_of_the_total_energy():
    rng = np.random.default_rng(3)
    n_atoms, n_wc = 9, 4
    L = np.array([5.0, 5.5, 6.0])
    R = rng.random((n_atoms, 3)) * L
    qa = rng.normal(size=n_atoms)
    qw = rng.normal(size=n_wc)
    shift = (qa.sum() + qw.sum()) / n_atoms
    qa -= shift
    q = np.concatenate([qa, qw])
    beta = 0.9
    wc_pos, hp, hw, jp, jw, J = _linear_model(n_atoms, n_wc, rng)

    def energy(R):
        return native.egt_direct(np.vstack([R, wc_pos(R)]), q, L, beta, forces=False)["energy"]

    sites = np.vstack([R, wc_pos(R)])
    f_sites = native.egt_direct(sites, q, L, beta)["forces"]
    F = fold(f_sites, n_atoms, hp, hw, jp, jw, J)
    h = 1e-5
    fd = np.zeros_like(R)
    for j in range(n_atoms):
        for d in range(3):
            Rp, Rm = R.copy(), R.copy()
            Rp[j, d] += h
            Rm[j, d] -= h
            fd[j, d] = -(energy(Rp) - energy(Rm)) / (2 * h)
    assert np.linalg.norm(F - fd) <= 1e-7 * np.linalg.norm(fd)
    # without the Jacobian term the fold is visibly wrong (the pin has teeth)
    F0 = fold(f_sites, n_atoms, hp, hw)
    assert np.linalg.norm(F0 - fd) > 1e-3 * np.linalg.norm(fd)


def test_translation_invariant_model_conserves_total_force():
    # Delta depends on relative positions only, so the atoms' forces sum to the sites' forces
    rng = np.random.default_rng(4)
    n_atoms, n_wc = 20, 7
    _, hp, hw, jp, jw, J = _linear_model(n_atoms, n_wc, rng)
    f_sites = rng.normal(size=(n_atoms + n_wc, 3))
    F = fold(f_sites, n_atoms, hp, hw, jp, jw, J)
    assert np.allclose(F.sum(axis=0), f_sites.sum(axis=0), rtol=0, atol=1e-12)


def test_no_maps_and_host_only():
    rng = np.random.default_rng(5)
    f = rng.normal(size=(6, 3))
    assert np.array_equal(fold(f, 4), f[:4])
    F = fold(f, 4, host_ptr=[0, 1, 1, 2, 2], host_wc=[1, 0])
    assert np.allclose(F, f[:4] + np.array([f[5], [0, 0, 0], f[4], [0, 0, 0]]))
