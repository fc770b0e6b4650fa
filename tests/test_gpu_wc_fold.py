"""GPU parity of the WC force fold (Eq. DPLR:F_final) against the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle.wc_fold import fold
from workloads.water import dw_jacobian, make_workload

pytestmark = pytest.mark.gpu


def _dev(a, dt):
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def _maps(hp, hw, jp, jw, J, dt):
    return (_dev(hp, torch.int32), _dev(hw, torch.int32), _dev(jp, torch.int64), _dev(jw, torch.int32),
            _dev(J, dt))


@pytest.mark.parametrize("name", ["water64", "water4096"])
@pytest.mark.parametrize("dt,tol", [(torch.float64, 1e-14), (torch.float32, 1e-6)])
def test_fold_matches_oracle(cuda_device, name, dt, tol):
    from paper_2504_15508_gb300.pppm import wc_fold
    wb, _ = make_workload(name)
    hp, hw, jp, jw, J = dw_jacobian(wb, seed=7)
    rng = np.random.default_rng(1)
    f_sites = rng.normal(size=(wb.n, 3))
    n_atoms = 3 * wb.n_mol
    fs = _dev(f_sites, dt)
    maps = _maps(hp, hw, jp, jw, J, dt)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = wc_fold(fs, n_atoms, *maps, status=status)
    torch.cuda.synchronize()
    ref = fold(fs.double().cpu().numpy(), n_atoms, hp, hw, jp, jw, maps[4].double().cpu().numpy())
    err = np.linalg.norm(out.double().cpu().numpy() - ref) / np.linalg.norm(ref)
    print(f"wc_fold {name} {dt}: {err:.2e}")
    assert err <= tol and status.item() == 0
    again = wc_fold(fs, n_atoms, *maps)
    assert torch.equal(out, again)  # fixed summation order


def test_fold_of_pppm_forces_matches_oracle_chain(cuda_device):
    """End to end in FP64: GPU PPPM forces folded on the GPU vs oracle PPPM
    forces folded by the oracle."""
    from oracle.pppm import OraclePPPM
    from paper_2504_15508_gb300.pppm import Plan, wc_fold
    wb, w = make_workload("water64")
    plan = Plan(wb.box, w["mesh"], w["order"], w["beta"], precision="fp64")
    pos = _dev(wb.pos, torch.float64)
    q = _dev(wb.q, torch.float64)
    _, f, _ = plan.compute(pos, q)
    hp, hw, jp, jw, J = dw_jacobian(wb, seed=3)
    n_atoms = 3 * wb.n_mol
    out = wc_fold(f, n_atoms, *_maps(hp, hw, jp, jw, J, torch.float64))
    torch.cuda.synchronize()
    r = OraclePPPM(wb.box, w["mesh"], w["order"], w["beta"]).compute(wb.pos, wb.q)
    ref = fold(r["forces"], n_atoms, hp, hw, jp, jw, J)
    err = np.linalg.norm(out.cpu().numpy() - ref) / np.linalg.norm(ref)
    print(f"PPPM + fold vs oracle: {err:.2e}")
    assert err <= 1e-12


def test_fold_edge_cases(cuda_device):
    from paper_2504_15508_gb300.pppm import wc_fold
    rng = np.random.default_rng(2)
    f = _dev(rng.normal(size=(10, 3)), torch.float64)
    # no maps: the atoms' own forces
    assert torch.equal(wc_fold(f, 7), f[:7])
    # no WCs at all
    assert torch.equal(wc_fold(f, 10), f)
    # host map only, with empty rows
    hp = _dev([0, 1, 1, 1, 2, 2, 3, 3], torch.int32)
    hw = _dev([2, 0, 1], torch.int32)
    out = wc_fold(f, 7, hp, hw)
    ref = fold(f.cpu().numpy(), 7, hp.cpu().numpy(), hw.cpu().numpy())
    assert torch.allclose(out, torch.tensor(ref, device="cuda"), rtol=0, atol=1e-15)
    # an out-of-range WC index is skipped and flagged
    jp = _dev([0, 2, 2, 2, 2, 2, 2, 3], torch.int64)
    jw = _dev([1, 5, 0], torch.int32)
    J = _dev(rng.normal(size=(3, 3, 3)), torch.float64)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = wc_fold(f, 7, hp, hw, jp, jw, J, status=status)
    torch.cuda.synchronize()
    assert status.item() == 1
    keep = np.array([True, False, True])
    ref = fold(f.cpu().numpy(), 7, hp.cpu().numpy(), hw.cpu().numpy(), jp.cpu().numpy(),
               np.where(keep, jw.cpu().numpy(), 0), J.cpu().numpy() * keep[:, None, None])
    assert np.allclose(out.cpu().numpy(), ref, rtol=0, atol=1e-14)
    # zero atoms
    assert wc_fold(f[:0], 0).shape == (0, 3)
