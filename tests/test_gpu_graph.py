"""Captured steps: a replayed CUDA graph gives bitwise the results of the
ordinary call, for the captured sites and for new site pointers."""
import numpy as np
import pytest
import torch

from workloads.water import make_workload

pytestmark = pytest.mark.gpu


def _setup(name, prec):
    from paper_2504_15508_gb300.pppm import Plan
    wb, w = make_workload(name)
    dt = torch.float32 if prec == "fp32" else torch.float64
    plan = Plan(wb.box, w["mesh"], w["order"], w["beta"], precision=prec)
    pos = torch.tensor(wb.pos, dtype=dt, device="cuda")
    q = torch.tensor(wb.q, dtype=dt, device="cuda")
    return plan, pos, q


@pytest.mark.parametrize("name,prec", [("water4096", "fp32"), ("water64", "fp64"), ("water72192_m128", "fp32")])
def test_replay_matches_eager(cuda_device, name, prec):
    plan, pos, q = _setup(name, prec)
    g = plan.graph(pos, q)
    # a second frame at another address
    rng = np.random.default_rng(1)
    pos2 = (pos + torch.tensor(rng.normal(0, 0.05, size=tuple(pos.shape)), dtype=pos.dtype, device="cuda")).contiguous()
    for p in (pos, pos2, pos, pos2):
        e, f, v = (t.clone() for t in g.launch(p, q, stream=torch.cuda.current_stream()))
        e0, f0, v0 = plan.compute(p, q)
        torch.cuda.synchronize()
        assert torch.equal(f, f0) and torch.equal(e, e0) and torch.equal(v, v0)
    # no new pointers: the previous sites again
    e, f, v = (t.clone() for t in g.launch(stream=torch.cuda.current_stream()))
    torch.cuda.synchronize()
    assert torch.equal(f, f0)
    g.close()


def test_graph_rejects_bad_use(cuda_device):
    from paper_2504_15508_gb300 import _native as N
    plan, pos, q = _setup("water64", "fp32")
    with pytest.raises(N.PPPMError):
        plan.graph(pos, q, stream=torch.cuda.default_stream())   # legacy stream cannot be captured
    plan.profile(True)
    with pytest.raises(N.PPPMError):
        plan.graph(pos, q)
    plan.profile(False)
    g = plan.graph(pos, q)
    with pytest.raises(ValueError):
        g.launch(pos.double(), q.double())
    with pytest.raises(ValueError):
        g.launch(pos[:10].contiguous(), q[:10].contiguous())
    g.close()


def test_launch_refuses_a_changed_plan(cuda_device):
    from paper_2504_15508_gb300 import _native as N
    plan, pos, q = _setup("water64", "fp32")
    g = plan.graph(pos, q)
    g.launch(pos, q)
    plan.set_options(prefactor=2.0)          # options are baked into the capture
    with pytest.raises(N.PPPMError):
        g.launch(pos, q)
    g.close()
    g = plan.graph(pos, q)
    big = torch.cat([pos, pos + 0.5]).contiguous()
    plan.compute(big, torch.cat([q, q]).contiguous())   # more sites: the site buffers grow
    with pytest.raises(N.PPPMError):
        g.launch(pos, q)
    g.close()


def test_host_call_replays_its_graph_bitwise(cuda_device):
    """The host-pointer call captures its device part on the first call and
    replays it afterwards; every call must give the ordinary result."""
    plan, pos, q = _setup("water4096", "fp32")
    e0, f0, v0 = plan.compute(pos, q)
    torch.cuda.synchronize()
    hp, hq = pos.cpu().numpy(), q.cpu().numpy()
    out = (np.zeros(1), np.zeros(tuple(pos.shape), np.float32), np.zeros(6))
    for k in range(3):
        e, f, v = plan.compute_host(hp, hq, out=out)
        assert e == e0.item() and np.array_equal(f, f0.cpu().numpy()) and np.array_equal(v, v0.cpu().numpy())
    # a changed plan is recaptured, not replayed stale
    plan.set_options(prefactor=2.0)
    e, f, v = plan.compute_host(hp, hq, out=out)
    assert np.allclose(f, 2.0 * f0.cpu().numpy(), rtol=1e-6, atol=0)


def _pinned(a):
    t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    return t, t.numpy()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_host_call_pinned_and_pageable_inputs(cuda_device, prec):
    """Pinned host arrays are read in place by the device, pageable ones are
    copied first; either kind, at any address, through the same replayed
    graph, gives the device call's result bitwise."""
    plan, pos, q = _setup("water4096", prec)
    dt = np.float32 if prec == "fp32" else np.float64
    rng = np.random.default_rng(3)
    frames = [pos.cpu().numpy()]
    frames.append((frames[0] + rng.normal(0, 0.05, size=frames[0].shape)).astype(dt))
    hq = q.cpu().numpy()
    keep = []
    for k, (fr, pinned) in enumerate([(0, True), (1, True), (0, False), (1, True), (1, False)]):
        if pinned:
            tp, hp = _pinned(frames[fr])
            tq, hqq = _pinned(hq)
            keep += [tp, tq]  # distinct pinned buffers at new addresses every call
        else:
            hp, hqq = frames[fr].copy(), hq.copy()
        out = (np.zeros(1), np.zeros(frames[fr].shape, dt), np.zeros(6))
        e, f, v = plan.compute_host(hp, hqq, out=out)
        e0, f0, v0 = plan.compute(torch.tensor(frames[fr], device="cuda"), q)
        torch.cuda.synchronize()
        assert e == e0.item(), (k, pinned)
        assert np.array_equal(f, f0.cpu().numpy()) and np.array_equal(v, v0.cpu().numpy()), (k, pinned)


def test_host_call_site_count_changes(cuda_device):
    """Growing the site count reallocates the host-call staging and drops its
    graph; smaller and larger calls in any order stay exact."""
    plan, pos, q = _setup("water4096", "fp32")
    hp, hq = pos.cpu().numpy(), q.cpu().numpy()
    big_p = np.concatenate([hp, hp + 0.5]).astype(np.float32)
    big_q = np.concatenate([hq, hq]).astype(np.float32)
    for p_, q_ in [(hp, hq), (big_p, big_q), (hp, hq), (big_p, big_q)]:
        e, f, v = plan.compute_host(p_, q_)
        e0, f0, v0 = plan.compute(torch.tensor(p_, device="cuda"), torch.tensor(q_, device="cuda"))
        torch.cuda.synchronize()
        assert e == e0.item() and np.array_equal(f, f0.cpu().numpy()) and np.array_equal(v, v0.cpu().numpy())


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_dependent_launch_switch(cuda_device, prec):
    """Programmatic dependent launch between the kernels changes no result
    bit; switching it invalidates a graph captured before."""
    from paper_2504_15508_gb300 import _native as N
    plan, pos, q = _setup("water4096", prec)
    e1, f1, v1 = (t.clone() for t in plan.compute(pos, q))
    g = plan.graph(pos, q)
    plan.set_dependent_launch(False)
    e0, f0, v0 = (t.clone() for t in plan.compute(pos, q))
    torch.cuda.synchronize()
    assert torch.equal(f0, f1) and torch.equal(e0, e1) and torch.equal(v0, v1)
    with pytest.raises(N.PPPMError):
        g.launch(pos, q)
    g.close()
    g = plan.graph(pos, q)
    e2, f2, v2 = (t.clone() for t in g.launch(pos, q, stream=torch.cuda.current_stream()))
    torch.cuda.synchronize()
    assert torch.equal(f2, f1) and torch.equal(e2, e1)
    g.close()
    plan.set_dependent_launch(True)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_region_overflow_falls_back_inside_a_replay(cuda_device, prec):
    """4,000 charges in a 10 A box on a 32^3 mesh sort into fixed regions of
    256 slots per tile (edge 8, ~62 sites a tile).  A frame with every site
    inside one tile overflows its region: the fallback rebuilds the compact
    layout on the device, within the same captured graph.  Replays of the
    spread-out frame, the clustered frame and the spread-out one again each
    equal the eager call bitwise and the oracle within the path's tolerance."""
    from oracle.pppm import OraclePPPM
    from paper_2504_15508_gb300.pppm import Plan
    dt = torch.float32 if prec == "fp32" else torch.float64
    box, mesh, n = (10.0, 10.0, 10.0), (32, 32, 32), 4000
    rng = np.random.default_rng(44)
    spread_out = rng.random((n, 3)) * 10.0
    clustered = 0.2 + rng.random((n, 3)) * 2.0   # base points in cells 1-7: tile 0
    q = rng.normal(size=n)
    q -= q.mean()
    plan = Plan(box, mesh, 5, 0.4, precision=prec)
    tq = torch.tensor(q, dtype=dt, device="cuda")
    frames = [torch.tensor(p, dtype=dt, device="cuda") for p in (spread_out, clustered, spread_out)]
    g = plan.graph(frames[0], tq)
    ftol = 1e-5 if prec == "fp32" else 1e-12
    for k, p in enumerate(frames):
        e, f, v = (t.clone() for t in g.launch(p, tq, stream=torch.cuda.current_stream()))
        e0, f0, v0 = plan.compute(p, tq)
        torch.cuda.synchronize()
        assert torch.equal(f, f0) and torch.equal(e, e0) and torch.equal(v, v0), k
        ref = OraclePPPM(box, mesh, 5, 0.4).compute(p.double().cpu().numpy(), tq.double().cpu().numpy())
        ferr = np.linalg.norm(f.double().cpu().numpy() - ref["forces"]) / np.linalg.norm(ref["forces"])
        assert ferr <= ftol, (k, ferr)
        # FP32 energy of the clustered frame: ~4,000 x 125 / 7^3 = 1,500 sequential
        # additions a point, rounding sqrt(1500) x 2^-24 = 2.3e-6
        etol = 1e-6 if (prec == "fp64" or k != 1) else 5e-6
        assert abs(e.item() - ref["energy"]) <= etol * abs(ref["energy"]), k
    g.close()
