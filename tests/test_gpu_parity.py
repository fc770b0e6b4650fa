"""GPU parity: every stage and the whole path of the CUDA library against the
FP64 CPU oracle on the same seeded inputs.

Tolerances (the spec contract): force RMS relative error
||F - F_ref|| / ||F_ref|| <= 1e-12 on the FP64 path and <= 1e-5 on the FP32
path; energy relative error <= 1e-6 on both.  The virial is reported and held
to the same bounds as the forces.  FP32 inputs are rounded once and the oracle
receives the rounded values.
"""
import numpy as np
import pytest
import torch

from oracle import native
from oracle.pppm import OraclePPPM, spread, wavevectors
from workloads.water import make_water, make_workload

pytestmark = pytest.mark.gpu

FTOL = {"fp64": 1e-12, "fp32": 1e-5}
ETOL = 1e-6


def _plan(*a, **k):
    from paper_2504_15508_gb300.pppm import Plan
    return Plan(*a, **k)


def _rel(a, b):
    a = np.asarray(a).astype(np.complex128 if np.iscomplexobj(a) else np.float64).ravel()
    b = np.asarray(b).astype(np.complex128 if np.iscomplexobj(b) else np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _dt(prec):
    return torch.float64 if prec == "fp64" else torch.float32


def _sites(pos, q, prec, dev):
    dt = _dt(prec)
    tp = torch.tensor(np.asarray(pos), dtype=dt, device=dev).contiguous()
    tq = torch.tensor(np.asarray(q), dtype=dt, device=dev).contiguous()
    return tp, tq, tp.double().cpu().numpy(), tq.double().cpu().numpy()


def _random_neutral(n, box, seed):
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 3)) * np.asarray(box)
    q = rng.normal(size=n)
    q -= q.mean()
    return pos, q


def _check(res, ref, prec, what="", etol=ETOL):
    e, f, v = res
    torch.cuda.synchronize()
    ferr = _rel(f.cpu().numpy(), ref["forces"])
    eerr = abs(e.item() - ref["energy"]) / abs(ref["energy"])
    verr = _rel(v.cpu().numpy(), ref["virial"])
    print(f"{what} {prec}: force {ferr:.3e} energy {eerr:.3e} virial {verr:.3e}")
    assert ferr <= FTOL[prec], (what, ferr)
    assert eerr <= etol, (what, eerr)
    assert verr <= max(FTOL[prec], 1e-10), (what, verr)


# ------------------------------------------------------------------ stages

@pytest.mark.parametrize("mesh", [(32, 32, 32), (30, 36, 40), (27, 25, 45), (12, 15, 16)])
def test_influence_table(cuda_device, pppm_lib, mesh):
    box = (9.0, 10.5, 12.0)
    plan = _plan(box, mesh, 5, 0.5, precision="fp64")
    G = plan.influence().cpu().numpy()
    ref = native.influence_ik(box, mesh, 5, 0.5)[:, :, : mesh[2] // 2 + 1]
    assert np.max(np.abs(G - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("mesh", [(32, 32, 32), (30, 36, 40), (27, 25, 45), (12, 15, 16), (160, 8, 6),
                                  (64, 128, 32), (128, 160, 64), (72, 96, 120), (48, 80, 90),
                                  (100, 108, 144), (192, 48, 256)])
def test_fft_r2c_c2r(cuda_device, pppm_lib, prec, mesh):
    plan = _plan((10.0, 11.0, 12.0), mesh, 5, 0.4, precision=prec)
    rng = np.random.default_rng(sum(mesh))
    x = rng.normal(size=mesh)
    xt = torch.tensor(x, dtype=_dt(prec), device=cuda_device)
    X = plan.fft_r2c(xt)
    ref = np.fft.rfftn(xt.double().cpu().numpy())
    tol = 1e-13 if prec == "fp64" else 2e-6
    assert _rel(X.cpu().numpy(), ref) <= tol
    # inverse of a Hermitian half spectrum (unnormalised)
    y = plan.fft_c2r(X)
    assert _rel(y.cpu().numpy() / np.prod(mesh), xt.double().cpu().numpy()) <= tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("order", [3, 4, 5, 7])
def test_spread(cuda_device, pppm_lib, prec, order):
    box = np.array([9.0, 10.5, 12.0])
    mesh = (30, 36, 40)
    pos, q = _random_neutral(500, box, seed=order)
    pos[:7] += np.array([[-9.0, 0, 0], [0, 21.0, 0], [0, 0, -36.0], [9.0, 10.5, 12.0], [1e-9, 0, 0],
                         [-1e-9, -1e-9, 0], [0, 0, 12.0 - 1e-12]])  # outside the box / on the edges
    tp, tq, pos_r, q_r = _sites(pos, q, prec, cuda_device)
    plan = _plan(box, mesh, order, 0.5, precision=prec)
    rho = plan.spread(tp, tq).double().cpu().numpy()
    ref = spread(pos_r, q_r, box, mesh, order)
    tol = 1e-13 if prec == "fp64" else 1e-6
    assert np.max(np.abs(rho - ref)) <= tol * np.max(np.abs(ref))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fields(cuda_device, pppm_lib, prec):
    wb, w = make_workload("water64")
    tp, tq, pos_r, q_r = _sites(wb.pos, wb.q, prec, cuda_device)
    plan = _plan(wb.box, w["mesh"], w["order"], w["beta"], precision=prec)
    fl = plan.fields(tp, tq).double().cpu().numpy()
    ref = OraclePPPM(wb.box, w["mesh"], w["order"], w["beta"]).compute(pos_r, q_r, want_intermediates=True)
    for d in range(3):
        assert _rel(fl[d], ref["fields"][d]) <= FTOL[prec], d


# ------------------------------------------------------------------ whole path

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_water64(cuda_device, pppm_lib, prec):
    wb, w = make_workload("water64")
    tp, tq, pos_r, q_r = _sites(wb.pos, wb.q, prec, cuda_device)
    plan = _plan(wb.box, w["mesh"], w["order"], w["beta"], precision=prec)
    ref = OraclePPPM(wb.box, w["mesh"], w["order"], w["beta"]).compute(pos_r, q_r)
    _check(plan.compute(tp, tq), ref, prec, "water64")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_water4096(cuda_device, pppm_lib, prec):
    wb, w = make_workload("water4096")
    tp, tq, pos_r, q_r = _sites(wb.pos, wb.q, prec, cuda_device)
    plan = _plan(wb.box, w["mesh"], w["order"], w["beta"], precision=prec)
    ref = OraclePPPM(wb.box, w["mesh"], w["order"], w["beta"]).compute(pos_r, q_r)
    _check(plan.compute(tp, tq), ref, prec, "water4096")


@pytest.mark.parametrize("mesh", [(72, 72, 72), (96, 90, 80), (120, 108, 100), (48, 144, 64)])
def test_water4096_fp32_meshes(cuda_device, pppm_lib, mesh):
    """The 4,096-water box on meshes whose lengths run the other compile-time
    FFT engines (and 64 beside them), FP32 against the FP64 oracle."""
    wb, w = make_workload("water4096")
    tp, tq, pos_r, q_r = _sites(wb.pos, wb.q, "fp32", cuda_device)
    plan = _plan(wb.box, mesh, w["order"], w["beta"], precision="fp32")
    ref = OraclePPPM(wb.box, mesh, w["order"], w["beta"]).compute(pos_r, q_r)
    _check(plan.compute(tp, tq), ref, "fp32", f"water4096 {mesh}")


@pytest.mark.parametrize("mesh", [128, 160])
def test_water72192_fp32(cuda_device, pppm_lib, mesh):
    """The 216,576-atom + 72,192-WC system at full size, FP32, as the bench runs it.
    Three calls in a row give bitwise the same result: the spread hands its
    4,096 (8,000) tiles to fewer resident warps by a ticket counter that the
    kernel itself must leave at zero for the next call."""
    wb, w = make_workload(f"water72192_m{mesh}")
    tp, tq, pos_r, q_r = _sites(wb.pos, wb.q, "fp32", cuda_device)
    plan = _plan(wb.box, w["mesh"], w["order"], w["beta"], precision="fp32")
    ref = OraclePPPM(wb.box, w["mesh"], w["order"], w["beta"]).compute(pos_r, q_r)
    first = [t.clone() for t in plan.compute(tp, tq)]
    _check(first, ref, "fp32", f"water72192 {mesh}^3")
    for _ in range(2):
        again = plan.compute(tp, tq)
        for a, b in zip(first, again):
            assert torch.equal(a, b)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["rect_odd", "order3", "order4", "order7", "tiny_mesh", "tile4", "coarse",
                                  "mixed_lengths", "box_beyond_mesh"])
def test_geometries(cuda_device, pppm_lib, prec, case):
    box = np.array([9.0, 10.5, 12.0])
    mesh, order, beta, n, tile = (30, 36, 40), 5, 0.5, 300, 0
    if case == "rect_odd":
        mesh = (27, 25, 45)
    elif case == "order3":
        order = 3
    elif case == "order4":
        order = 4
    elif case == "order7":
        order = 7
    elif case == "tiny_mesh":
        mesh, order = (6, 5, 8), 5
    elif case == "tile4":
        tile = 4
    elif case == "coarse":
        mesh, n = (8, 9, 10), 3000  # dense: many sites per tile
    elif case == "box_beyond_mesh":
        # 8-cell tiles on an 8^3 mesh: the padded z extent (12 points) is
        # shorter than the field box's odd z pitch (13)
        mesh, n, tile = (8, 8, 8), 100, 8
    elif case == "mixed_lengths":
        # three different compile-time FFT lengths: the x and y passes number
        # their lines over different outer counts (Ny Hz vs Nx Hz)
        mesh, n = (64, 128, 32), 2000
    pos, q = _random_neutral(n, box, seed=11)
    tp, tq, pos_r, q_r = _sites(pos, q, prec, cuda_device)
    plan = _plan(box, mesh, order, beta, precision=prec, tile=tile)
    ref = OraclePPPM(box, mesh, order, beta).compute(pos_r, q_r)
    _check(plan.compute(tp, tq), ref, prec, case)


# ------------------------------------------------------------------ edge cases

def test_empty_and_single_site(cuda_device, pppm_lib):
    plan = _plan((10.0, 10.0, 10.0), (16, 16, 16), 5, 0.5, precision="fp64")
    pos = torch.zeros((0, 3), dtype=torch.float64, device=cuda_device)
    q = torch.zeros(0, dtype=torch.float64, device=cuda_device)
    e, f, v = plan.compute(pos, q)
    torch.cuda.synchronize()
    assert e.item() == 0.0 and torch.all(v == 0)
    p1 = np.array([[1.0, 2.0, 3.0]])
    q1 = np.array([2.0])
    ref = OraclePPPM((10.0, 10.0, 10.0), (16, 16, 16), 5, 0.5).compute(p1, q1)
    e, f, v = plan.compute(torch.tensor(p1, device=cuda_device), torch.tensor(q1, device=cuda_device))
    torch.cuda.synchronize()
    assert abs(e.item() - ref["energy"]) <= 1e-12 * abs(ref["energy"])
    assert np.max(np.abs(f.cpu().numpy() - ref["forces"])) <= 1e-12 * max(1.0, np.max(np.abs(ref["forces"])))


def test_deterministic(cuda_device, pppm_lib):
    wb, w = make_workload("water4096")
    tp, tq, _, _ = _sites(wb.pos, wb.q, "fp32", cuda_device)
    plan = _plan(wb.box, w["mesh"], w["order"], w["beta"], precision="fp32")
    r1 = [t.clone() for t in plan.compute(tp, tq)]
    r2 = [t.clone() for t in plan.compute(tp, tq)]
    torch.cuda.synchronize()
    for a, b in zip(r1, r2):
        assert torch.equal(a, b)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("mesh,n,tile", [((8, 8, 8), 3000, 4), ((8, 9, 10), 3000, 4), ((6, 5, 8), 1000, 8)])
def test_dense_tiles_are_deterministic(cuda_device, pppm_lib, prec, mesh, n, tile):
    """Tiles holding more sites than the spread ranks in shared memory (256
    in the full-tile kernel: the first two cases, ~375 and up to ~270 a tile;
    512 in the generic kernel: the third, one tile of 1,000) are put in
    canonical order by ranks counted in global memory: two runs agree bitwise
    and both match the oracle."""
    box = (10.0, 11.0, 12.0)
    pos, q = _random_neutral(n, box, seed=21)
    tp, tq, pos_r, q_r = _sites(pos, q, prec, cuda_device)
    plan = _plan(box, mesh, 5, 0.4, precision=prec, tile=tile)
    r1 = [t.clone() for t in plan.compute(tp, tq)]
    r2 = [t.clone() for t in plan.compute(tp, tq)]
    torch.cuda.synchronize()
    for a, b in zip(r1, r2):
        assert torch.equal(a, b)
    ref = OraclePPPM(box, mesh, 5, 0.4).compute(pos_r, q_r)
    _check(r1, ref, prec, f"dense {mesh}")


def test_nonfinite_positions_flagged(cuda_device, pppm_lib):
    from paper_2504_15508_gb300 import _native as N
    wb, w = make_workload("water64")
    pos = wb.pos.copy()
    pos[5, 1] = np.nan
    pos[9, 0] = np.inf
    plan = _plan(wb.box, w["mesh"], w["order"], w["beta"], precision="fp32")
    tp, tq, _, _ = _sites(pos, wb.q, "fp32", cuda_device)
    plan.compute(tp, tq)
    assert plan.status() == N.PPPM_ERR_NONFINITE
    assert plan.status() == N.PPPM_OK  # cleared
    tp, tq, _, _ = _sites(wb.pos, wb.q, "fp32", cuda_device)
    plan.compute(tp, tq)
    assert plan.status() == N.PPPM_OK


def test_host_api_matches_device_api(cuda_device, pppm_lib):
    wb, w = make_workload("water64")
    plan = _plan(wb.box, w["mesh"], w["order"], w["beta"], precision="fp32")
    pos32 = wb.pos.astype(np.float32)
    q32 = wb.q.astype(np.float32)
    e_h, f_h, v_h = plan.compute_host(pos32, q32)
    e, f, v = plan.compute(torch.tensor(pos32, device=cuda_device), torch.tensor(q32, device=cuda_device))
    torch.cuda.synchronize()
    assert e_h == e.item()
    assert np.array_equal(f_h, f.cpu().numpy())
    assert np.array_equal(v_h, v.cpu().numpy())


def test_double_inputs_on_fp32_plan(cuda_device, pppm_lib):
    wb, w = make_workload("water4096")
    plan = _plan(wb.box, w["mesh"], w["order"], w["beta"], precision="fp32")
    ref = OraclePPPM(wb.box, w["mesh"], w["order"], w["beta"]).compute(wb.pos, wb.q)
    tp = torch.tensor(wb.pos, device=cuda_device)
    tq = torch.tensor(wb.q, device=cuda_device)
    _check(plan.compute(tp, tq), ref, "fp32", "double-in fp32 plan")


def test_prefactor(cuda_device, pppm_lib):
    wb, w = make_workload("water64")
    plan = _plan(wb.box, w["mesh"], w["order"], w["beta"], precision="fp64", prefactor=14.399645)
    ref = OraclePPPM(wb.box, w["mesh"], w["order"], w["beta"], prefactor=14.399645).compute(wb.pos, wb.q)
    tp, tq, _, _ = _sites(wb.pos, wb.q, "fp64", cuda_device)
    _check(plan.compute(tp, tq), ref, "fp64", "prefactor")


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("mesh", [(36, 36, 36), (30, 30, 30)])
def test_one_tile_holds_every_site(cuda_device, pppm_lib, prec, mesh):
    """60,000 charges inside one mesh tile (a clustered or corrupt frame): the
    canonical order of that tile comes from a radix sort whose cost grows
    linearly with the tile, so the call ends quickly (a pairwise ranking would
    take ~1e8 dependent loads a lane).  36^3 runs the full-tile kernels with
    tile edge 4, 30^3 the generic ones (30 is not a multiple of 4).  Two runs
    agree bitwise and match the oracle: forces at the path's tolerance; the
    FP32 energy to 1e-5, because here every mesh point of the cluster sums
    ~22,000 FP32 contributions (60,000 sites x 125 points over ~7^3 points)
    one after another, whose rounding grows like sqrt(22,000) x 2^-24 = 9e-6
    relative, far beyond the ~100 of a water tile."""
    import time
    box = np.array([12.0, 12.0, 12.0])
    rng = np.random.default_rng(77)
    n = 60000
    # u = x N / L stays in [0.5, 3.2) cells: base points 1..3, all in tile 0
    pos = 0.5 * box / mesh[0] + rng.random((n, 3)) * (2.7 * box / mesh[0])
    q = rng.normal(size=n)
    tp, tq, pos_r, q_r = _sites(pos, q, prec, cuda_device)
    plan = _plan(box, mesh, 5, 0.4, precision=prec)
    r1 = [t.clone() for t in plan.compute(tp, tq)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r2 = [t.clone() for t in plan.compute(tp, tq)]
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert dt < 2.0, dt
    for a, b in zip(r1, r2):
        assert torch.equal(a, b)
    ref = OraclePPPM(box, mesh, 5, 0.4).compute(pos_r, q_r)
    _check(r1, ref, prec, f"one tile {mesh}", etol=1e-5 if prec == "fp32" else ETOL)


def test_gather_wait_runs_out_cleanly(cuda_device, pppm_lib):
    """With a wait limit of 0 polls every tile's first wait for its field copy
    runs out: the call reports PPPM_ERR_TIMEOUT (after the block has waited
    for its copy once more, bounded), the device stays usable, and the next
    call with the default limit is correct."""
    from paper_2504_15508_gb300 import _native as N
    wb, w = make_workload("water4096")
    tp, tq, pos_r, q_r = _sites(wb.pos, wb.q, "fp32", cuda_device)
    plan = _plan(wb.box, w["mesh"], w["order"], w["beta"], precision="fp32")
    plan.set_wait_limit(0)
    plan.compute(tp, tq)
    assert plan.status() == N.PPPM_ERR_TIMEOUT
    assert plan.status() == N.PPPM_OK  # cleared
    plan.set_wait_limit(1 << 26)
    ref = OraclePPPM(wb.box, w["mesh"], w["order"], w["beta"]).compute(pos_r, q_r)
    _check(plan.compute(tp, tq), ref, "fp32", "after the timeout")
    assert plan.status() == N.PPPM_OK
