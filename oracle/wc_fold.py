"""FP64 reference of the force fold of Eq. DPLR:F_final (test infrastructure only).

Only tests/, the smoke check and the benchmark's CPU-baseline leg may use this
module.

A Wannier centroid sits at W_n = R_host(n) + Delta_n(R) (Eq. DPLR:Wn), so by
the chain rule of Eq. DPLR:F_inter the long-range force on atom j is

    F_j = -dE_Gt/dR_j - sum_{n hosted by j} dE_Gt/dW_n
          - sum_n (dDelta_n/dR_j)^T dE_Gt/dW_n,

i.e. with F_site = -dE_Gt/d(site position) from the PPPM solve (atoms first,
then WCs):

    F_j = F_site[j] + sum_{n in host(j)} F_site[n_atoms + n]
          + sum_{(n, J) in row j} J^T F_site[n_atoms + n],

J = dDelta_n/dR_j as a 3 x 3 block (J[a, b] = dDelta_{n,a}/dR_{j,b}).
Both maps are given per atom in compressed rows: host_ptr/host_wc list the
WCs each atom hosts, jac_ptr/jac_wc/jac list the Jacobian blocks of the WCs
whose displacement depends on that atom.
"""
from __future__ import annotations

import numpy as np


def fold(f_sites, n_atoms, host_ptr=None, host_wc=None, jac_ptr=None, jac_wc=None, jac=None):
    f = np.asarray(f_sites, dtype=np.float64).reshape(-1, 3)
    out = f[:n_atoms].copy()
    fw = f[n_atoms:]
    if host_ptr is not None:
        host_ptr = np.asarray(host_ptr, dtype=np.int64)
        host_wc = np.asarray(host_wc, dtype=np.int64)
        for j in range(n_atoms):
            for k in range(host_ptr[j], host_ptr[j + 1]):
                out[j] += fw[host_wc[k]]
    if jac_ptr is not None:
        jac_ptr = np.asarray(jac_ptr, dtype=np.int64)
        jac_wc = np.asarray(jac_wc, dtype=np.int64)
        J = np.asarray(jac, dtype=np.float64).reshape(-1, 3, 3)
        # each block contributes J^T F_W(n) to its row's atom
        rows = np.repeat(np.arange(n_atoms), np.diff(jac_ptr))
        contrib = np.einsum("kab,ka->kb", J, fw[jac_wc])
        np.add.at(out, rows, contrib)
    return out
