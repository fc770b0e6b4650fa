"""The allocation-free spread entry point against the plan-based one.

pppm_spread_noalloc serves callers that cannot call cudaMalloc (host
callbacks, allocator hooks, processes whose device memory belongs to another
framework's pool): it works out of a fixed file-scope device array instead of a
plan's workspace.  Its output must equal pppm_spread's, call after call, even
though every call reuses the same scratch array.

This file sorts last so that, if it fails, a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _clustered(n_uniform, n_cluster, box, mesh, seed):
    """Uniform charges plus a cluster whose base points all fall in mesh cells
    5 and 6 of every axis: one tile of edge 8 (cells 0-7) or of edge 4
    (cells 4-7) then holds the whole cluster."""
    rng = np.random.default_rng(seed)
    box = np.asarray(box)
    h = box / np.asarray(mesh)
    pos = np.concatenate([rng.random((n_uniform, 3)) * box, (4.6 + 1.8 * rng.random((n_cluster, 3))) * h])
    q = rng.normal(size=len(pos))
    return pos, q - q.mean()


# (box, mesh, uniform sites, clustered sites): the tile edge and the spread
# kernel each case selects are in the comment
_CASES = [
    ((9.0, 10.5, 12.0), (30, 36, 40), 600, 0),       # edge 8, generic kernel, sparse
    ((9.0, 10.5, 12.0), (32, 40, 48), 300, 400),     # edge 8, full-tile kernel, one tile of ~400 (> 256)
    ((9.0, 10.5, 12.0), (30, 36, 40), 100, 700),     # edge 8, generic kernel, one tile of ~700 (> 512)
    ((9.0, 10.5, 12.0), (32, 36, 40), 20000, 400),   # edge 4 (dense box), full-tile kernel, one tile > 256
    ((9.0, 10.5, 12.0), (30, 36, 40), 257, 0),       # back to a small sparse input
]


def test_spread_noalloc_matches_spread(cuda_device, pppm_lib):
    """Consecutive calls on inputs of different sizes, tile edges and tile
    densities, each reusing the scratch array the previous call left behind:
    every output equals pppm_spread's bit for bit and matches the oracle's
    spread within the FP32 tolerance."""
    from oracle.pppm import spread as oracle_spread
    from paper_2504_15508_gb300 import _native as N
    from paper_2504_15508_gb300.pppm import Plan

    order = 5
    stream = torch.cuda.current_stream().cuda_stream
    for k, (box, mesh, n_uni, n_cl) in enumerate(_CASES):
        pos, q = _clustered(n_uni, n_cl, box, mesh, seed=k + 1)
        pos[:3] += np.asarray(box) * np.array([[-1, 0, 0], [0, 2, 0], [0, 0, -3]])  # outside the box
        n = len(pos)
        plan = Plan(box, mesh, order, 0.5, precision="fp32")
        b = (ctypes.c_double * 3)(*box)
        m = (ctypes.c_int * 3)(*mesh)
        tp = torch.tensor(pos, dtype=torch.float64, device=cuda_device)
        tq = torch.tensor(q, dtype=torch.float64, device=cuda_device)
        ref = plan.spread(tp, tq)
        for rep in range(2):
            out = torch.full(mesh, float("nan"), dtype=torch.float32, device=cuda_device)
            rc = pppm_lib.pppm_spread_noalloc(b, m, order, ctypes.c_void_p(stream), ctypes.c_void_p(tp.data_ptr()),
                                              ctypes.c_void_p(tq.data_ptr()), n, ctypes.c_void_p(out.data_ptr()))
            assert rc == N.PPPM_OK, N.strerror(rc)
            torch.cuda.synchronize()
            assert torch.equal(out, ref), (k, rep)
        rho_o = oracle_spread(pos, q, np.asarray(box), mesh, order)
        assert np.max(np.abs(out.double().cpu().numpy() - rho_o)) <= 1e-6 * np.max(np.abs(rho_o)), k
        plan.close()


def test_spread_noalloc_rejects_oversize(cuda_device, pppm_lib):
    from paper_2504_15508_gb300 import _native as N
    b = (ctypes.c_double * 3)(100.0, 100.0, 100.0)
    m = (ctypes.c_int * 3)(256, 256, 256)  # the tile patches alone exceed the 32 MiB scratch
    pos = torch.zeros((4, 3), dtype=torch.float64, device=cuda_device)
    q = torch.zeros(4, dtype=torch.float64, device=cuda_device)
    out = torch.empty((256, 256, 256), dtype=torch.float32, device=cuda_device)
    rc = pppm_lib.pppm_spread_noalloc(b, m, 5, None, ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(q.data_ptr()),
                                      4, ctypes.c_void_p(out.data_ptr()))
    assert rc == N.PPPM_ERR_TOO_LARGE
