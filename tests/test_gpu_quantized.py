"""The int32-quantised DFT of the paper's hardware-offloaded FFT (Section
"Hardware-offloaded 3D FFT", its quantisation panel; the "Mixed-Int32" runs of
its accuracy table) in the batched form, against the oracle of the same
definition (oracle.dft_quant) on the 128-water box of that table.

At the paper's scale 10^7 the quantisation changes the forces by about 3e-6
(relative), below the FP32 tolerance, so there the check is the FP32 bar
against both the quantised and the plain oracle.  At scale 10^4 it changes them
by about 3e-3, far above FP32 rounding: there the GPU must reproduce the
oracle's quantisation errors themselves (its distance to the quantised oracle
well below the quantisation effect), which a different rounding, scale, node
split or transform chain would not (independent errors of the same size give a
ratio near 1.4).  The oracle's reading is the real-to-complex one (half
spectrum, Hermitian extension before the z backward pass), as the kernels'."""
import numpy as np
import pytest
import torch

from oracle.dft_quant import pppm_quantized
from oracle.pppm import OraclePPPM
from workloads.water import make_water

pytestmark = pytest.mark.gpu

L128, MESH128 = 15.64, (12, 18, 12)


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def _boxes(seeds, extra=(), mesh=MESH128):
    boxes = [make_water(128, L128, s) for s in seeds] + [make_water(n, L, s) for (n, L, s) in extra]
    meshes = [mesh] * len(seeds) + [(24, 24, 24)] * len(extra)
    pos = np.concatenate([b.pos for b in boxes]).astype(np.float32)
    q = np.concatenate([b.q for b in boxes]).astype(np.float32)
    offs = np.concatenate([[0], np.cumsum([b.n for b in boxes])]).astype(np.int64)
    return boxes, np.array(meshes, dtype=np.int32), pos, q, offs


def _run(bp, dev, pos, q, offs):
    e, f, v = bp.compute(torch.tensor(pos, device=dev), torch.tensor(q, device=dev), torch.tensor(offs, device=dev))
    torch.cuda.synchronize()
    return e.cpu().numpy(), f.cpu().numpy(), v.cpu().numpy()


def _plan(boxes, meshes):
    from paper_2504_15508_gb300.pppm import BatchPlan
    return BatchPlan(np.array([b.box for b in boxes]), meshes, order=5, beta=0.4)


@pytest.mark.parametrize("mesh,group", [((8, 12, 8), 4), ((10, 15, 10), 5), (MESH128, 6), (MESH128, 3), (MESH128, 2)])
def test_quantized_paper_scale(cuda_device, pppm_lib, mesh, group):
    """The three meshes of the paper's int32 runs (the two coarser ones run
    with tile edge 4)."""
    boxes, meshes, pos, q, offs = _boxes([4, 5, 6], mesh=mesh)
    bp = _plan(boxes, meshes)
    _, f0, _ = _run(bp, cuda_device, pos, q, offs)   # switched on after a first run
    bp.set_quantized(group)
    e, f, v = _run(bp, cuda_device, pos, q, offs)
    assert bp.status() == 0
    assert not np.array_equal(f, f0)
    e2, f2, v2 = _run(bp, cuda_device, pos, q, offs)   # integer sums in a fixed order: reproducible
    assert np.array_equal(f, f2) and np.array_equal(e, e2) and np.array_equal(v, v2)
    for b, wb in enumerate(boxes):
        sl = slice(offs[b], offs[b + 1])
        p64, q64 = pos[sl].astype(np.float64), q[sl].astype(np.float64)
        o = OraclePPPM(wb.box, mesh, 5, 0.4)
        plain = o.compute(p64, q64)
        quant = pppm_quantized(o, p64, q64, group)
        assert not quant["saturated"]
        for ref in (quant, plain):
            assert _rel(f[sl], ref["forces"]) <= 1e-5
            assert abs(e[b] - ref["energy"]) <= 1e-6 * abs(ref["energy"])
            assert _rel(v[b], ref["virial"]) <= 1e-5


@pytest.mark.parametrize("mesh,group,axes", [(MESH128, 6, (0, 1, 2)), (MESH128, 2, (0, 1, 2)), (MESH128, 4, (0, 2)),
                                             (MESH128, 9, (1,)), ((8, 12, 8), 4, (0, 1, 2)),
                                             ((10, 15, 10), 5, (0, 1, 2))])
def test_quantized_coarse_scale_reproduces_oracle_errors(cuda_device, pppm_lib, mesh, group, axes):
    """The library quantises the lines of at most 18 points that the node size
    divides (group 4 on 12 x 18 x 12: x and z; group 9: y).  Left over after
    the match: exact ties (a partial sum of grid values times a twiddle of
    1/2), which FP32 and the oracle's FP64 may round either way."""
    scale = 1e4
    boxes, meshes, pos, q, offs = _boxes([4, 7], mesh=mesh)
    bp = _plan(boxes, meshes)
    e0, f0, v0 = _run(bp, cuda_device, pos, q, offs)          # unquantised, same kernels
    bp.set_quantized(group, scale)
    e, f, v = _run(bp, cuda_device, pos, q, offs)
    assert bp.status() == 0
    for b, wb in enumerate(boxes):
        sl = slice(offs[b], offs[b + 1])
        p64, q64 = pos[sl].astype(np.float64), q[sl].astype(np.float64)
        o = OraclePPPM(wb.box, mesh, 5, 0.4)
        plain = o.compute(p64, q64)
        quant = pppm_quantized(o, p64, q64, group, scale, axes=axes)
        d_f = _rel(quant["forces"], plain["forces"])
        d_e = abs(quant["energy"] - plain["energy"])
        d_v = float(np.linalg.norm(quant["virial"] - plain["virial"]))
        assert d_f > 5e-4                                    # the effect is far above FP32 rounding
        assert _rel(f[sl], quant["forces"]) <= 0.3 * d_f, (_rel(f[sl], quant["forces"]), d_f)
        # the energy's quantisation shift mostly cancels over the modes, so one
        # near-tie at a low-k mode that FP32 and FP64 round apart is as large
        # as the whole shift; hence a floor of 5e-6 (relative) besides 0.3
        assert abs(e[b] - quant["energy"]) <= 0.3 * d_e + 5e-6 * abs(plain["energy"]), (e[b] - quant["energy"], d_e)
        assert float(np.linalg.norm(v[b] - quant["virial"])) <= 0.3 * d_v + 5e-6 * np.linalg.norm(plain["virial"])
        # and the GPU's own quantised-minus-plain shift is the oracle's
        assert 0.7 <= _rel(f[sl], f0[sl]) / d_f <= 1.3


def test_quantized_leaves_long_lines_alone(cuda_device, pppm_lib):
    """A box whose lines are all longer than 18 points is not quantised."""
    boxes, meshes, pos, q, offs = _boxes([4], extra=[(512, 24.83, 11)])
    bp = _plan(boxes, meshes)
    bp.set_quantized(6, 1e3)
    e, f, v = _run(bp, cuda_device, pos, q, offs)
    assert bp.status() == 0
    sl = slice(offs[1], offs[2])
    ref = OraclePPPM(boxes[1].box, (24, 24, 24), 5, 0.4).compute(pos[sl].astype(np.float64), q[sl].astype(np.float64))
    assert _rel(f[sl], ref["forces"]) <= 1e-5
    assert abs(e[1] - ref["energy"]) <= 1e-6 * abs(ref["energy"])
    sl0 = slice(offs[0], offs[1])
    ref0 = OraclePPPM(boxes[0].box, MESH128, 5, 0.4).compute(pos[sl0].astype(np.float64), q[sl0].astype(np.float64))
    assert _rel(f[sl0], ref0["forces"]) > 1e-3                 # the short-line box is


def test_quantized_saturation_reported_then_recovers(cuda_device, pppm_lib):
    from paper_2504_15508_gb300 import _native as N
    boxes, meshes, pos, q, offs = _boxes([4])
    bp = _plan(boxes, meshes)
    bp.set_quantized(6, 1e12)                  # partial sums up to ~0.5 times 10^12 exceed int32
    _run(bp, cuda_device, pos, q, offs)
    assert bp.status() == N.PPPM_ERR_TOO_LARGE
    bp.set_quantized(6)
    e, f, v = _run(bp, cuda_device, pos, q, offs)
    assert bp.status() == 0
    ref = OraclePPPM(boxes[0].box, MESH128, 5, 0.4).compute(pos.astype(np.float64), q.astype(np.float64))
    assert _rel(f, ref["forces"]) <= 1e-5


def test_small_meshes_run_with_tile_edge_four(cuda_device, pppm_lib):
    """8 x 12 x 8 is below the 12 points tile edge 8 needs: the autotuner
    keeps 4, and forcing 8 is refused."""
    boxes, meshes, pos, q, offs = _boxes([4], mesh=(8, 12, 8))
    bp = _plan(boxes, meshes)
    _run(bp, cuda_device, pos, q, offs)
    assert bp.status() == 0 and bp.tile == 4
    bp.set(tile=8)
    tp, tq, to = (torch.tensor(pos, device=cuda_device), torch.tensor(q, device=cuda_device),
                  torch.tensor(offs, device=cuda_device))
    with pytest.raises(Exception):
        bp.compute(tp, tq, to)


def test_quantized_argument_checks(cuda_device, pppm_lib):
    from paper_2504_15508_gb300 import _native as N
    from paper_2504_15508_gb300.pppm import BatchPlan
    boxes, meshes, pos, q, offs = _boxes([4])
    bp3 = BatchPlan(np.array([boxes[0].box]), meshes, order=3, beta=0.4)
    assert pppm_lib.pppm_batch_set_quantized(bp3._h, 6, 1e7) == N.PPPM_ERR_INVALID_ARG   # order 5 only
    assert pppm_lib.pppm_batch_set_quantized(bp3._h, 0, 1e7) == N.PPPM_OK
    bp = _plan(boxes, meshes)
    for g, s in ((-1, 1e7), (19, 1e7), (6, 0.5), (6, float("nan")), (6, 1e16)):
        assert pppm_lib.pppm_batch_set_quantized(bp._h, g, s) == N.PPPM_ERR_INVALID_ARG
