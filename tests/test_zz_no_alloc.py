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


def _random_neutral(n, box, seed):
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 3)) * np.asarray(box)
    pos[:3] += np.asarray(box) * np.array([[-1, 0, 0], [0, 2, 0], [0, 0, -3]])  # outside the box
    q = rng.normal(size=n)
    return pos, q - q.mean()


def test_spread_noalloc_matches_spread(cuda_device, pppm_lib):
    from paper_2504_15508_gb300 import _native as N
    from paper_2504_15508_gb300.pppm import Plan

    box, mesh, order = (9.0, 10.5, 12.0), (30, 36, 40), 5
    plan = Plan(box, mesh, order, 0.5, precision="fp32")
    b = (ctypes.c_double * 3)(*box)
    m = (ctypes.c_int * 3)(*mesh)
    stream = torch.cuda.current_stream().cuda_stream
    # two calls in a row with different inputs and sizes: the second reuses the
    # scratch array the first left behind
    for seed, n in ((1, 600), (2, 257)):
        pos, q = _random_neutral(n, box, seed)
        tp = torch.tensor(pos, dtype=torch.float64, device=cuda_device)
        tq = torch.tensor(q, dtype=torch.float64, device=cuda_device)
        ref = plan.spread(tp, tq)
        out = torch.full(mesh, float("nan"), dtype=torch.float32, device=cuda_device)
        rc = pppm_lib.pppm_spread_noalloc(b, m, order, ctypes.c_void_p(stream), ctypes.c_void_p(tp.data_ptr()),
                                          ctypes.c_void_p(tq.data_ptr()), n, ctypes.c_void_p(out.data_ptr()))
        assert rc == N.PPPM_OK, N.strerror(rc)
        torch.cuda.synchronize()
        diff = (out.double() - ref.double()).abs().max().item()
        assert diff <= 1e-6 * ref.double().abs().max().item(), (seed, diff)


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
