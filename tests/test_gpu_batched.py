"""The batched form: many independent water boxes in one persistent launch,
each equal to its own single-box evaluation within the FP32 tolerances
(force RMS relative <= 1e-5, energy relative <= 1e-6 against the FP64 oracle)."""
import numpy as np
import pytest
import torch

from oracle.pppm import OraclePPPM
from workloads.water import batched_boxes, make_water

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def _make_batch(nbox, seed, lo=64, hi=700):
    specs = batched_boxes(nbox=nbox, seed=seed, lo=lo, hi=hi)
    boxes = [make_water(s["n_mol"], s["L"], s["seed"]) for s in specs]
    pos = np.concatenate([b.pos for b in boxes]).astype(np.float32)
    q = np.concatenate([b.q for b in boxes]).astype(np.float32)
    offs = np.concatenate([[0], np.cumsum([b.n for b in boxes])]).astype(np.int64)
    return specs, boxes, pos, q, offs


@pytest.mark.parametrize("tile,dft", [(0, 18), (4, 18), (8, 18), (0, 0), (8, 0), (8, 12)])
def test_batched_matches_oracle_per_box(cuda_device, pppm_lib, tile, dft):
    """dft: lines up to this length take the tensor-core DFT (0: the FFT for all)."""
    from paper_2504_15508_gb300.pppm import BatchPlan
    specs, boxes, pos, q, offs = _make_batch(6, seed=5)
    bp = BatchPlan(np.array([[s["L"]] * 3 for s in specs]), None, order=5, beta=0.4, tile=tile)
    bp.set_dft(dft)
    tp = torch.tensor(pos, device=cuda_device)
    tq = torch.tensor(q, device=cuda_device)
    to = torch.tensor(offs, device=cuda_device)
    e, f, v = bp.compute(tp, tq, to)
    torch.cuda.synchronize()
    assert bp.status() == 0
    meshes = bp.meshes
    for b, wb in enumerate(boxes):
        sl = slice(offs[b], offs[b + 1])
        ref = OraclePPPM(wb.box, meshes[b], 5, 0.4).compute(pos[sl].astype(np.float64), q[sl].astype(np.float64))
        ferr = _rel(f[sl].cpu().numpy(), ref["forces"])
        eerr = abs(e[b].item() - ref["energy"]) / abs(ref["energy"])
        verr = _rel(v[b].cpu().numpy(), ref["virial"])
        assert ferr <= 1e-5 and eerr <= 1e-6 and verr <= 1e-5, (b, meshes[b], ferr, eerr, verr)


def test_staged_launch_agrees_with_persistent(cuda_device, pppm_lib):
    """The staged form runs the same stage code, compiled separately: each
    form is bitwise reproducible (first call and graph replay), and the two
    agree to rounding (1e-6 relative).  The autotuner's choice is one of the
    two forms."""
    from paper_2504_15508_gb300.pppm import BatchPlan
    specs, boxes, pos, q, offs = _make_batch(6, seed=11)
    tp, tq, to = (torch.tensor(pos, device=cuda_device), torch.tensor(q, device=cuda_device),
                  torch.tensor(offs, device=cuda_device))
    res = {}
    for form in ("persistent", "staged"):
        bp = BatchPlan(np.array([[s["L"]] * 3 for s in specs]), None, order=5, beta=0.4, tile=8)
        bp.set_launch(form)
        r1 = [t.clone() for t in bp.compute(tp, tq, to)]
        r2 = [t.clone() for t in bp.compute(tp, tq, to)]  # graph replay
        torch.cuda.synchronize()
        assert bp.status() == 0 and bp.launch == form
        for a, b in zip(r1, r2):
            assert torch.equal(a, b)
        res[form] = r1
    for a, b in zip(res["persistent"], res["staged"]):
        assert torch.linalg.norm((a - b).double()) <= 1e-6 * torch.linalg.norm(a.double())
    bp = BatchPlan(np.array([[s["L"]] * 3 for s in specs]), None, order=5, beta=0.4)
    bp.compute(tp, tq, to)
    torch.cuda.synchronize()
    assert bp.launch in ("persistent", "staged") and bp.tile in (4, 8)


def test_batched_graph_replay_and_single_box_equality(cuda_device, pppm_lib):
    from paper_2504_15508_gb300.pppm import BatchPlan, Plan
    specs, boxes, pos, q, offs = _make_batch(5, seed=7)
    bp = BatchPlan(np.array([[s["L"]] * 3 for s in specs]), None, order=5, beta=0.4)
    tp = torch.tensor(pos, device=cuda_device)
    tq = torch.tensor(q, device=cuda_device)
    to = torch.tensor(offs, device=cuda_device)
    out = (torch.empty(5, dtype=torch.float64, device=cuda_device),
           torch.empty((len(pos), 3), dtype=torch.float32, device=cuda_device),
           torch.empty((5, 6), dtype=torch.float64, device=cuda_device))
    r1 = [t.clone() for t in bp.compute(tp, tq, to, out=out)]   # tunes, then records the graph
    r2 = [t.clone() for t in bp.compute(tp, tq, to, out=out)]   # replays it
    torch.cuda.synchronize()
    for a, b in zip(r1, r2):
        assert torch.equal(a, b)
    assert bp.tile in (4, 8)
    meshes = bp.meshes
    for b, wb in enumerate(boxes):
        sl = slice(offs[b], offs[b + 1])
        plan = Plan(wb.box, meshes[b], 5, 0.4, precision="fp32", tile=bp.tile)
        e, f, v = plan.compute(tp[sl].contiguous(), tq[sl].contiguous())
        torch.cuda.synchronize()
        # the batched kernels evaluate the same arithmetic in a different order
        assert _rel(r2[1][sl].cpu().numpy(), f.cpu().numpy()) <= 1e-5
        assert abs(r2[0][b].item() - e.item()) <= 1e-6 * abs(e.item())


def test_batched_bounded_wait_times_out_cleanly(cuda_device, pppm_lib):
    """The wait probe makes box 0's scan wait for one binning item more than
    exist, so that bounded wait must run out: the launch still ends (every
    other stage's wait is satisfied or skipped), the status is
    PPPM_ERR_TIMEOUT, the other boxes are still correct, and the next run
    without the probe is correct for every box."""
    from paper_2504_15508_gb300 import _native as N
    from paper_2504_15508_gb300.pppm import BatchPlan
    specs, boxes, pos, q, offs = _make_batch(4, seed=9)
    bp = BatchPlan(np.array([[s["L"]] * 3 for s in specs]), None, order=5, beta=0.4, tile=8)
    tp = torch.tensor(pos, device=cuda_device)
    tq = torch.tensor(q, device=cuda_device)
    to = torch.tensor(offs, device=cuda_device)
    refs = [OraclePPPM(wb.box, bp.meshes[b], 5, 0.4).compute(pos[offs[b]:offs[b + 1]].astype(np.float64),
                                                              q[offs[b]:offs[b + 1]].astype(np.float64))
            for b, wb in enumerate(boxes)]
    bp.set_launch("persistent")  # the in-kernel waits belong to the persistent form
    bp.set(tile=8, spin_limit=1000)
    bp.set_wait_probe(True)
    e, f, v = bp.compute(tp, tq, to)
    torch.cuda.synchronize()
    assert bp.status() == N.PPPM_ERR_TIMEOUT
    assert bp.status() == N.PPPM_OK  # read and cleared
    for b in range(1, len(boxes)):
        sl = slice(offs[b], offs[b + 1])
        assert _rel(f[sl].cpu().numpy(), refs[b]["forces"]) <= 1e-5, b
    bp.set_wait_probe(False)
    bp.set(tile=8, spin_limit=1 << 24)
    e, f, v = bp.compute(tp, tq, to)
    torch.cuda.synchronize()
    assert bp.status() == N.PPPM_OK
    for b in range(len(boxes)):
        sl = slice(offs[b], offs[b + 1])
        assert _rel(f[sl].cpu().numpy(), refs[b]["forces"]) <= 1e-5, b
        assert abs(e[b].item() - refs[b]["energy"]) <= 1e-6 * abs(refs[b]["energy"]), b


@pytest.mark.parametrize("order,meshes", [
    (3, [(12, 15, 16), (16, 16, 16), (12, 16, 20), (16, 16, 16)]),
    (7, [(15, 16, 18), (16, 16, 16), (15, 16, 20), (16, 16, 16)]),
    (5, [(18, 75, 24), (16, 16, 16), (81, 20, 25), (16, 16, 16)]),
])
def test_batched_orders_rectangular_empty_and_single_site(cuda_device, pppm_lib, order, meshes):
    """Orders 3, 7 and 5; in one launch a water box, a box without sites, a
    rectangular box of random neutral charges on a mixed mesh and a box with
    one charge.  Every box equals the oracle; the empty one gives zeros.  The
    order-5 case mixes line lengths with compile-time FFT engines (16-25) and
    lengths without (75, 81), which take the run-time FFT in the same launch."""
    from paper_2504_15508_gb300.pppm import BatchPlan
    rng = np.random.default_rng(order)
    water = make_water(128, 15.64, 3)
    rect_box = np.array([14.0, 19.0, 23.5])
    rect_pos = rng.uniform(0, 1, (300, 3)) * rect_box
    rect_q = np.where(np.arange(300) % 2 == 0, 0.7, -0.7)
    one_box = np.array([10.0, 10.0, 10.0])
    one_pos = rng.uniform(0, 10, (1, 3))
    one_q = np.array([1.0])
    boxes = np.array([water.box, [20.0, 20.0, 20.0], rect_box, one_box])
    sites = [(water.pos, water.q), (np.zeros((0, 3)), np.zeros(0)), (rect_pos, rect_q), (one_pos, one_q)]
    pos = np.concatenate([p for p, _ in sites]).astype(np.float32)
    q = np.concatenate([c for _, c in sites]).astype(np.float32)
    offs = np.concatenate([[0], np.cumsum([len(c) for _, c in sites])]).astype(np.int64)
    bp = BatchPlan(boxes, np.array(meshes, dtype=np.int32), order=order, beta=0.4)
    e, f, v = bp.compute(torch.tensor(pos, device=cuda_device), torch.tensor(q, device=cuda_device),
                         torch.tensor(offs, device=cuda_device))
    torch.cuda.synchronize()
    assert bp.status() == 0
    e, f, v = e.cpu().numpy(), f.cpu().numpy(), v.cpu().numpy()
    assert e[1] == 0.0 and np.all(v[1] == 0.0)
    for b in (0, 2, 3):
        sl = slice(offs[b], offs[b + 1])
        ref = OraclePPPM(boxes[b], meshes[b], order, 0.4).compute(pos[sl].astype(np.float64),
                                                                  q[sl].astype(np.float64))
        assert abs(e[b] - ref["energy"]) <= 1e-6 * abs(ref["energy"]), (b, e[b], ref["energy"])
        assert _rel(v[b], ref["virial"]) <= 1e-5, b
        if b == 3:   # a lone charge feels (almost) no force from its own images
            assert np.max(np.abs(f[sl] - ref["forces"])) <= 1e-5 + 1e-5 * np.max(np.abs(ref["forces"]))
        else:
            assert _rel(f[sl], ref["forces"]) <= 1e-5, b


def test_batched_dense_tiles_are_deterministic(cuda_device, pppm_lib):
    """3,000 charges in a 10 A box on a 12^3 mesh with tile edge 8: ~890 sites
    a tile, past the 256 the spread ranks in shared memory; the canonical
    order then comes from ranks counted in global memory.  Two runs agree
    bitwise and match the oracle."""
    from paper_2504_15508_gb300.pppm import BatchPlan
    rng = np.random.default_rng(31)
    box = np.array([10.0, 10.0, 10.0])
    pos = (rng.random((3000, 3)) * box).astype(np.float32)
    q = rng.normal(size=3000)
    q = (q - q.mean()).astype(np.float32)
    offs = np.array([0, 3000], dtype=np.int64)
    bp = BatchPlan(box[None, :], np.array([[12, 12, 12]], dtype=np.int32), order=5, beta=0.4, tile=8)
    tp, tq, to = (torch.tensor(pos, device=cuda_device), torch.tensor(q, device=cuda_device),
                  torch.tensor(offs, device=cuda_device))
    r1 = [t.clone() for t in bp.compute(tp, tq, to)]
    r2 = [t.clone() for t in bp.compute(tp, tq, to)]
    torch.cuda.synchronize()
    assert bp.status() == 0 and bp.tile == 8
    for a, b in zip(r1, r2):
        assert torch.equal(a, b)
    ref = OraclePPPM(box, (12, 12, 12), 5, 0.4).compute(pos.astype(np.float64), q.astype(np.float64))
    assert _rel(r1[1].cpu().numpy(), ref["forces"]) <= 1e-5
    assert abs(r1[0].item() - ref["energy"]) <= 1e-6 * abs(ref["energy"])


_FULL = {}


def _full_batch():
    """The 96-box batch as the batched workload states it (seed 5, 64 to 8,192
    molecules log-uniformly, 29.9 A^3 a molecule, meshes at <= 1.2 A: 12^3 to
    54^3), with the oracle's result for every box, computed once."""
    if not _FULL:
        specs = batched_boxes(nbox=96, seed=5)
        boxes = [make_water(s["n_mol"], s["L"], s["seed"]) for s in specs]
        pos = np.concatenate([b.pos for b in boxes]).astype(np.float32)
        q = np.concatenate([b.q for b in boxes]).astype(np.float32)
        offs = np.concatenate([[0], np.cumsum([b.n for b in boxes])]).astype(np.int64)
        refs = []
        for b, (s, wb) in enumerate(zip(specs, boxes)):
            sl = slice(offs[b], offs[b + 1])
            refs.append(OraclePPPM(wb.box, s["mesh"], 5, 0.4).compute(pos[sl].astype(np.float64),
                                                                       q[sl].astype(np.float64)))
        _FULL.update(specs=specs, boxes=boxes, pos=pos, q=q, offs=offs, refs=refs)
    return _FULL


@pytest.mark.parametrize("tile,dft,staged", [(4, 0, False), (8, 0, False), (4, 18, False), (8, 18, False),
                                             (8, 0, True), (4, 18, True)])
def test_full_batched96_matches_oracle_per_box(cuda_device, pppm_lib, tile, dft, staged):
    """All 96 boxes in one launch, the largest (8,192-molecule class) on 54^3
    meshes, so that the shared-memory layout is sized by the 54-point lines;
    every box against the FP64 oracle: force RMS 1e-5, energy 1e-6, virial
    1e-5 relative, for both tile edges, with and without the tensor-core DFT
    of the short lines, in the persistent launch and in the staged one (one
    kernel per stage)."""
    from paper_2504_15508_gb300.pppm import BatchPlan
    F = _full_batch()
    specs, boxes, pos, q, offs, refs = F["specs"], F["boxes"], F["pos"], F["q"], F["offs"], F["refs"]
    assert max(s["mesh"][0] for s in specs) == 54 and min(s["mesh"][0] for s in specs) == 12
    bp = BatchPlan(np.array([[s["L"]] * 3 for s in specs]), None, order=5, beta=0.4, tile=tile)
    bp.set_dft(dft)
    bp.set_launch("staged" if staged else "persistent")
    assert [tuple(m) for m in bp.meshes] == [tuple(s["mesh"]) for s in specs]
    e, f, v = bp.compute(torch.tensor(pos, device=cuda_device), torch.tensor(q, device=cuda_device),
                         torch.tensor(offs, device=cuda_device))
    torch.cuda.synchronize()
    assert bp.status() == 0 and bp.tile == tile
    e, f, v = e.cpu().numpy(), f.cpu().numpy(), v.cpu().numpy()
    worst, bad = (0.0, 0.0, 0.0), []
    for b in range(len(boxes)):
        sl = slice(offs[b], offs[b + 1])
        ferr = _rel(f[sl], refs[b]["forces"])
        eerr = abs(e[b] - refs[b]["energy"]) / abs(refs[b]["energy"])
        verr = _rel(v[b], refs[b]["virial"])
        worst = tuple(max(a, c) for a, c in zip(worst, (ferr, eerr, verr)))
        if not (ferr <= 1e-5 and eerr <= 1e-6 and verr <= 1e-5):
            bad.append((b, specs[b]["n_mol"], specs[b]["mesh"][0], f"{ferr:.2e}", f"{eerr:.2e}", f"{verr:.2e}"))
    print(f"batched96 tile {tile} dft {dft} staged {staged}: worst force {worst[0]:.2e} energy {worst[1]:.2e} "
          f"virial {worst[2]:.2e}; over the bar: {bad}")
    assert not bad, bad
