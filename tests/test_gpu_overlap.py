"""Running the force evaluation concurrently with other work on another
stream (the long/short-range overlap) leaves its results bitwise unchanged,
and those results match the FP64 oracle within the FP32 tolerances."""
import numpy as np
import pytest
import torch

from oracle.pppm import OraclePPPM
from workloads.water import make_workload

pytestmark = pytest.mark.gpu


def test_concurrent_streams_give_identical_results(cuda_device):
    from paper_2504_15508_gb300.pppm import Plan
    wb, w = make_workload("water4096")
    plan = Plan(wb.box, w["mesh"], w["order"], w["beta"], precision="fp32")
    pos = torch.tensor(wb.pos, dtype=torch.float32, device="cuda")
    q = torch.tensor(wb.q, dtype=torch.float32, device="cuda")
    e0, f0, v0 = (t.clone() for t in plan.compute(pos, q))
    torch.cuda.synchronize()
    hi = torch.cuda.Stream(priority=-1)
    lo = torch.cuda.Stream(priority=0)
    x = torch.randn((4096, 4096), device="cuda", dtype=torch.bfloat16)
    g = plan.graph(pos, q)
    for _ in range(5):
        g.launch(pos, q, stream=hi)
        with torch.cuda.stream(lo):
            y = torch.tanh(x @ x)        # unrelated load in flight at the same time
        out = plan.compute(pos, q, stream=hi)
    torch.cuda.synchronize()
    assert torch.equal(out[1], f0) and torch.equal(out[0], e0) and torch.equal(g.out[1], f0)
    assert torch.isfinite(y).all()
    g.close()
    # the overlapped result itself against the oracle (force RMS 1e-5, energy and virial)
    ref = OraclePPPM(wb.box, w["mesh"], w["order"], w["beta"]).compute(pos.double().cpu().numpy(),
                                                                      q.double().cpu().numpy())
    f = out[1].double().cpu().numpy()
    assert np.linalg.norm(f - ref["forces"]) <= 1e-5 * np.linalg.norm(ref["forces"])
    assert abs(out[0].item() - ref["energy"]) <= 1e-6 * abs(ref["energy"])
    assert np.linalg.norm(out[2].cpu().numpy() - ref["virial"]) <= 1e-5 * np.linalg.norm(ref["virial"])
