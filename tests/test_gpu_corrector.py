"""GPU parity of the learned coarse-mesh correction against the FP64 oracle,
and a held-out test of what the trained network gains.

Precision of the comparisons:
* features are BF16 on both sides (the oracle rounds its FP64 values through
  FP32 to BF16); they must agree to one BF16 unit in the last place, and most
  of them exactly;
* the tensor-core forward takes weights and hidden activations as BF16 and
  accumulates in FP32; the oracle runs the same roundings in FP64
  (act_bf16=True), so only rounding order and tanh differ;
* training (gradients) is FP32 with BF16-rounded weights; the oracle's
  gradient of the same loss in FP64 bounds it to 1e-4 relative;
* Adam is compared one step at a time, the oracle fed the GPU's gradient.
"""
import os

import numpy as np
import pytest
import torch

from oracle import mlp
from oracle.pppm import OraclePPPM
from workloads.water import init_mlp_params, make_water

pytestmark = pytest.mark.gpu


def _mods():
    from paper_2504_15508_gb300 import learned
    from paper_2504_15508_gb300.pppm import Corrector, Plan
    return Plan, Corrector, learned


KINDS = ["cell", "stated"]


def _theta(seed, bias_scale=0.1, kind="cell"):
    n_in = mlp.FEATURE_WIDTH[kind]
    rng = np.random.default_rng(seed)
    t = init_mlp_params(seed, n_in=n_in).astype(np.float64)
    o = 0
    for name, shape in mlp.shapes(n_in):
        k = int(np.prod(shape))
        if name.startswith("b"):
            t[o:o + k] = rng.normal(size=k) * bias_scale
        o += k
    return t.astype(np.float32)


def _sites(w, dev="cuda"):
    pos = torch.tensor(w.pos, dtype=torch.float32, device=dev).contiguous()
    q = torch.tensor(w.q, dtype=torch.float32, device=dev).contiguous()
    types = torch.tensor(w.types, dtype=torch.int8, device=dev).contiguous()
    return pos, q, types


def _bf16_ulp(v):
    a = np.maximum(np.abs(v), 1e-30)
    return 2.0 ** (np.floor(np.log2(a)) - 7)


CASES = [  # n_mol, L, mesh, order, seed
    (64, 12.42, 16, 5, 1),
    (64, 12.42, 16, 4, 11),
    (64, 12.42, 15, 7, 12),
    (64, 12.42, 18, 3, 13),
    (4096, 49.7, 24, 5, 2),
]


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("n_mol,L,m,p,seed", CASES)
def test_features_match_oracle(cuda_device, n_mol, L, m, p, seed, kind):
    Plan, Corrector, _ = _mods()
    w = make_water(n_mol, L, seed)
    coarse = Plan((L,) * 3, (m,) * 3, order=p, beta=0.4)
    corr = Corrector(coarse, params=_theta(0, kind=kind), s_in=0.37, s_out=1.0, features=kind)
    pos, q, types = _sites(w)
    feat, fc = corr.features(pos, q, types)
    torch.cuda.synchronize()
    g = feat.float().cpu().numpy().astype(np.float64)
    posf, qf = pos.double().cpu().numpy(), q.double().cpu().numpy()
    orc = OraclePPPM((L,) * 3, (m,) * 3, p, 0.4)
    phi = orc.compute(posf, qf, want_intermediates=True)["phi"]
    X = mlp.features(phi, posf, w.types, (L,) * 3, (m,) * 3, p, s_in=0.37, kind=kind)
    ref = mlp.bf16_round(X.astype(np.float32))
    assert g.shape == X.shape == (w.n, mlp.FEATURE_WIDTH[kind])
    d = np.abs(g - ref)
    ulp = _bf16_ulp(np.maximum(np.abs(g), np.abs(ref)))
    exact = float(np.mean(d == 0))
    print(f"features N={m} p={p}: exact {exact:.4f}, max |d|/ulp {np.max(d / _bf16_ulp(np.abs(ref))):.2f}")
    # potential samples: one BF16 step, or the FP32 mesh error near zero
    assert np.all(d[:, :27] <= ulp[:, :27] + 1e-5 * np.max(np.abs(ref[:, :27])))
    # one-hot type and padding exactly; cell-offset terms to one step (+ FP32 location error)
    if kind == "cell":
        assert np.array_equal(g[:, 27:30], X[:, 27:30]) and not g[:, 36:].any()
        assert np.all(d[:, 30:36] <= ulp[:, 30:36] + 2e-6)
    else:
        assert np.array_equal(g[:, 27:30], X[:, 27:30]) and not g[:, 30:].any()
    assert exact >= 0.95


def test_potential_output_leaves_the_forces_unchanged(cuda_device):
    Plan, Corrector, _ = _mods()
    w = make_water(4096, 49.7, 2)
    P = Plan((49.7,) * 3, (32,) * 3, order=5, beta=0.4)
    pos, q, types = _sites(w)
    e0, f0, v0 = (t.clone() for t in P.compute(pos, q))
    corr = Corrector(P, params=_theta(1))  # switches the potential output on
    e1, f1, v1 = P.compute(pos, q)
    torch.cuda.synchronize()
    assert torch.equal(f0, f1) and torch.equal(e0, e1) and torch.equal(v0, v1)
    del corr


FORWARDS = ["tcgen05", "mma_sync"]


@pytest.mark.parametrize("fwd", FORWARDS)
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("n", [1, 7, 16, 37, 127, 128, 129, 1000, 16384])
def test_forward_matches_oracle(cuda_device, n, kind, fwd):
    Plan, Corrector, _ = _mods()
    w = make_water(4096, 49.7, 2)
    P = Plan((49.7,) * 3, (24,) * 3, order=5, beta=0.4)
    theta = _theta(3, kind=kind)
    corr = Corrector(P, params=theta, s_in=0.5, s_out=1.0, features=kind)
    corr.set_forward(fwd)
    pos, q, types = _sites(w)
    feat, _ = corr.features(pos, q, types)
    feat = feat[:n].contiguous()
    y = corr.forward(feat)
    torch.cuda.synchronize()
    X = feat.float().cpu().numpy().astype(np.float64)
    yr, _ = mlp.forward(theta, X, bf16=True, act_bf16=True)
    yg = y.cpu().numpy()
    err = np.abs(yg - yr)
    scale = np.max(np.abs(yr))
    print(f"forward {fwd} n={n}: max {np.max(err) / scale:.2e} "
          f"rms {np.sqrt(np.mean(err ** 2)) / np.sqrt(np.mean(yr ** 2)):.2e}")
    assert np.max(err) <= 4e-3 * scale
    assert np.sqrt(np.mean(err ** 2)) <= 1e-3 * np.sqrt(np.mean(yr ** 2))
    assert P.status() == 0


@pytest.mark.parametrize("kind", KINDS)
def test_forward_kernels_agree(cuda_device, kind):
    """The tcgen05 and mma.sync forwards take the same BF16 operands and
    accumulate in FP32 in different orders: they agree to the rounding of the
    BF16 activations, and each is reproducible run to run; a feature pointer
    off the 16-byte grid runs the mma.sync kernel and gives its result."""
    Plan, Corrector, _ = _mods()
    w = make_water(4096, 49.7, 2)
    P = Plan((49.7,) * 3, (24,) * 3, order=5, beta=0.4)
    corr = Corrector(P, params=_theta(5, kind=kind), s_in=0.5, s_out=1.0, features=kind)
    pos, q, types = _sites(w)
    feat, _ = corr.features(pos, q, types)
    ys = {}
    for fwd in FORWARDS:
        corr.set_forward(fwd)
        a = corr.forward(feat)
        b = corr.forward(feat)
        torch.cuda.synchronize()
        assert torch.equal(a, b), fwd
        ys[fwd] = a
    d = (ys["tcgen05"] - ys["mma_sync"]).abs()
    assert float(d.max()) <= 4e-3 * float(ys["mma_sync"].abs().max())
    # rows 1.. of a copy whose row 1 starts 4 bytes off the 16-byte grid
    n_in = corr.n_in
    flat = torch.zeros(feat.numel() + 8, dtype=feat.dtype, device=feat.device)
    flat[2:2 + feat.numel()] = feat.reshape(-1)
    shifted = flat[2 + n_in:2 + feat.numel()].view(-1, n_in)
    assert shifted.data_ptr() % 16 == 4
    corr.set_forward("tcgen05")
    y_shift = corr.forward(shifted)
    corr.set_forward("mma_sync")
    y_ref = corr.forward(feat[1:].contiguous())
    torch.cuda.synchronize()
    assert torch.equal(y_shift, y_ref)
    # a pointer off the 4-byte grid is refused on the host, for either kernel
    odd = flat[1 + n_in:1 + n_in + 4 * n_in].view(-1, n_in)
    assert odd.data_ptr() % 4 == 2
    for fwd in FORWARDS:
        corr.set_forward(fwd)
        with pytest.raises(RuntimeError):
            corr.forward(odd)
    assert P.status() == 0


def test_tcgen05_forward_wait_times_out_cleanly(cuda_device):
    """A completion wait limited to zero polls runs out in every CTA: the plan's
    status reports PPPM_ERR_TIMEOUT, and the next call with the normal limit
    (tensor memory freed, nothing left in flight) is correct."""
    from paper_2504_15508_gb300 import _native as N
    Plan, Corrector, _ = _mods()
    w = make_water(4096, 49.7, 2)
    P = Plan((49.7,) * 3, (24,) * 3, order=5, beta=0.4)
    corr = Corrector(P, params=_theta(7), s_in=0.5, s_out=1.0)
    pos, q, types = _sites(w)
    feat, _ = corr.features(pos, q, types)
    corr.set_forward("mma_sync")
    y_ref = corr.forward(feat)
    corr.set_forward("tcgen05")
    corr.set_wait_limit(0)
    corr.forward(feat)
    torch.cuda.synchronize()
    assert P.status() == N.PPPM_ERR_TIMEOUT
    assert P.status() == 0  # read and cleared
    corr.set_wait_limit(1 << 26)
    y = corr.forward(feat)
    torch.cuda.synchronize()
    assert P.status() == 0
    assert torch.equal(y, y_ref)
    with pytest.raises(RuntimeError):
        corr.set_wait_limit(-1)


@pytest.mark.parametrize("kind", KINDS)
def test_apply_is_coarse_plus_correction(cuda_device, kind):
    Plan, Corrector, _ = _mods()
    w = make_water(4096, 49.7, 2)
    P = Plan((49.7,) * 3, (24,) * 3, order=5, beta=0.4)
    theta = _theta(4, kind=kind)
    corr = Corrector(P, params=theta, s_in=0.4, s_out=0.05, features=kind)
    pos, q, types = _sites(w)
    feat, fc = corr.features(pos, q, types)
    y = corr.forward(feat)
    e, f, v = corr.apply(pos, q, types)
    torch.cuda.synchronize()
    expect = fc + (q[:, None] * 0.05) * y
    assert torch.allclose(f, expect, rtol=1e-6, atol=1e-6 * float(expect.abs().max()))
    # against the oracle end to end: coarse FP64 PPPM + q s_out network(features)
    posf, qf = pos.double().cpu().numpy(), q.double().cpu().numpy()
    orc = OraclePPPM((49.7,) * 3, (24,) * 3, 5, 0.4)
    r = orc.compute(posf, qf, want_intermediates=True)
    X = mlp.bf16_round(mlp.features(r["phi"], posf, w.types, (49.7,) * 3, (24,) * 3, 5, 0.4,
                                    kind=kind).astype(np.float32))
    yr, _ = mlp.forward(theta, X, bf16=True, act_bf16=True)
    fr = r["forces"] + qf[:, None] * 0.05 * yr
    corr_part = qf[:, None] * 0.05 * yr
    err = np.linalg.norm(f.cpu().numpy() - fr) / np.linalg.norm(corr_part)
    print(f"apply vs oracle: |dF| / |correction| = {err:.2e}")
    assert err <= 5e-3


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("nb,use_idx", [(1000, True), (128, False), (4099, True)])
def test_gradient_matches_oracle(cuda_device, nb, use_idx, kind):
    Plan, Corrector, _ = _mods()
    w = make_water(4096, 49.7, 2)
    P = Plan((49.7,) * 3, (24,) * 3, order=5, beta=0.4)
    theta = _theta(5, kind=kind)
    corr = Corrector(P, params=theta, s_in=0.5, s_out=1.0, features=kind)
    pos, q, types = _sites(w)
    feat, _ = corr.features(pos, q, types)
    rng = np.random.default_rng(nb)
    n = feat.shape[0]
    T = rng.normal(size=(n, 3)).astype(np.float32) * 0.3
    target = torch.tensor(T, device="cuda")
    idx_np = rng.integers(0, n, size=nb).astype(np.int32) if use_idx else np.arange(nb, dtype=np.int32)
    idx = torch.tensor(idx_np, device="cuda") if use_idx else None
    loss, g = corr.grad(feat, target, idx=idx, nb=nb)
    torch.cuda.synchronize()
    X = feat.float().cpu().numpy().astype(np.float64)[idx_np]
    lr_, gr = mlp.loss_and_grad(theta, X, T[idx_np].astype(np.float64), bf16=True)
    gg = g.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(gg - gr) / np.linalg.norm(gr)
    cos = float(gg @ gr / (np.linalg.norm(gg) * np.linalg.norm(gr)))
    print(f"grad nb={nb}: rel {rel:.2e} cos {cos:.8f} loss {loss.item():.6e} vs {lr_:.6e}")
    assert rel <= 1e-4 and cos >= 1 - 1e-8
    assert abs(loss.item() - lr_) <= 1e-5 * lr_
    # per block of parameters too (no block may hide behind the others)
    o = 0
    for name, shape in mlp.shapes(mlp.FEATURE_WIDTH[kind]):
        k = int(np.prod(shape))
        assert np.linalg.norm(gg[o:o + k] - gr[o:o + k]) <= 1e-4 * np.linalg.norm(gr[o:o + k]) + 1e-9, name
        o += k


@pytest.mark.parametrize("kind", KINDS)
def test_adam_steps_match_oracle(cuda_device, kind):
    Plan, Corrector, _ = _mods()
    w = make_water(4096, 49.7, 2)
    P = Plan((49.7,) * 3, (24,) * 3, order=5, beta=0.4)
    theta = _theta(6, kind=kind)
    corr = Corrector(P, params=theta, s_in=0.5, s_out=1.0, features=kind)
    pos, q, types = _sites(w)
    feat, _ = corr.features(pos, q, types)
    rng = np.random.default_rng(0)
    target = torch.tensor(rng.normal(size=(feat.shape[0], 3)).astype(np.float32) * 0.3, device="cuda")
    th = theta.astype(np.float64)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    lr = 1e-3
    for step in range(1, 4):
        idx = torch.tensor(rng.integers(0, feat.shape[0], size=2048).astype(np.int32), device="cuda")
        _, g = corr.grad(feat, target, idx=idx)
        corr.train_step(feat, target, idx, lr)
        gg = g.cpu().numpy().astype(np.float64)
        th, m, v = mlp.adam_step(th, m, v, gg, step, lr)
        got = corr.get_weights()[0].astype(np.float64)
        assert np.max(np.abs(got - th)) <= 1e-6 * max(1.0, np.max(np.abs(th))) + 1e-3 * lr, step
        th = got  # continue from the GPU's FP32 master values


@pytest.mark.parametrize("kind", KINDS)
def test_training_is_deterministic_and_resumes_bitwise(cuda_device, tmp_path, kind):
    Plan, Corrector, learned = _mods()
    w = make_water(4096, 49.7, 2)
    P = Plan((49.7,) * 3, (24,) * 3, order=5, beta=0.4)
    pos, q, types = _sites(w)
    theta = _theta(7, kind=kind)
    rng = np.random.default_rng(1)

    def run(c, steps, seed):
        feat, _ = c.features(pos, q, types)
        tgt = torch.tensor(np.random.default_rng(2).normal(size=(feat.shape[0], 3)).astype(np.float32),
                           device="cuda")
        gen = torch.Generator(device="cuda")
        gen.manual_seed(seed)
        for _ in range(steps):
            idx = torch.randint(0, feat.shape[0], (1024,), generator=gen, device="cuda", dtype=torch.int32)
            c.train_step(feat, tgt, idx, 1e-3)
        return c.get_weights()[0]

    a = Corrector(P, params=theta, s_in=0.5, s_out=1.0, features=kind)
    run(a, 5, 10)
    ck = str(tmp_path / "corr.bin")
    a.save(ck)
    wa = run(a, 5, 11)
    b = Corrector(P, params=_theta(8, kind=kind), s_in=2.0, s_out=3.0, features=kind)
    b.load(ck)
    assert b.scales == (0.5, 1.0)
    wb = run(b, 5, 11)
    assert np.array_equal(wa, wb)
    # a fresh run from the same start is bit-identical as well
    c = Corrector(P, params=theta, s_in=0.5, s_out=1.0, features=kind)
    run(c, 5, 10)
    assert np.array_equal(run(c, 5, 11), wa)
    del rng


def test_checkpoint_rejects_garbage_and_bad_arguments(cuda_device, tmp_path):
    Plan, Corrector, _ = _mods()
    from paper_2504_15508_gb300 import _native as N
    P = Plan((20.0,) * 3, (16,) * 3, order=5, beta=0.4)
    corr = Corrector(P, params=_theta(0))
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"not a checkpoint at all")
    with pytest.raises(N.PPPMError):
        corr.load(str(bad))
    with pytest.raises(N.PPPMError):
        corr.load(str(tmp_path / "missing.bin"))
    with pytest.raises(ValueError):
        corr.set_weights(np.zeros(10, np.float32), 1.0, 1.0)
    with pytest.raises(N.PPPMError):
        corr.set_weights(np.zeros(corr.nparams, np.float32), 0.0, 1.0)
    with pytest.raises(ValueError):
        Corrector(Plan((20.0,) * 3, (16,) * 3, order=5, beta=0.4, precision="fp64"))
    # a checkpoint of one feature set does not load into the other
    ck = tmp_path / "cell.bin"
    corr.save(str(ck))
    other = Corrector(P, params=_theta(0, kind="stated"), features="stated")
    assert other.nparams == 6467 and other.n_in == 32 and corr.nparams == 7491 and corr.n_in == 48
    with pytest.raises(N.PPPMError):
        other.load(str(ck))
    # no sites: the corrected call is the (empty) coarse call
    z = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    e, f, v = corr.apply(z, torch.zeros(0, device="cuda"), torch.zeros(0, dtype=torch.int8, device="cuda"))
    torch.cuda.synchronize()
    assert f.shape == (0, 3) and e.item() == 0.0


@pytest.mark.parametrize("kind", KINDS)
def test_trained_network_gains_on_held_out_frames(cuda_device, kind):
    """Train on frames of 8 base configurations, evaluate on 2 others.  With
    the cell set the corrected coarse mesh must be clearly closer to the fine
    mesh than the coarse mesh alone; the stated set (samples and type alone)
    carries almost nothing of the coarse-mesh error, which depends on where a
    site sits inside its cell, so for it the test asserts only that the
    correction does not make the forces worse, and prints the gain."""
    Plan, Corrector, learned = _mods()
    n_mol, L = 4096, 49.7
    coarse = Plan((L,) * 3, (24,) * 3, order=5, beta=0.4)
    fine = Plan((L,) * 3, (60,) * 3, order=5, beta=0.4)
    corr = Corrector(coarse, features=kind)
    spec = learned.FrameSpec(n_mol=n_mol, L=L, base_seeds=tuple(range(100, 108)), frames_per_base=8, sigma=0.05)
    ds = learned.build_dataset(corr, fine, spec)
    log = learned.train(corr, ds, steps=3000, batch=4096, lr=2e-3, seed=0, init_seed=0)
    held = learned.FrameSpec(n_mol=n_mol, L=L, base_seeds=(200, 201), frames_per_base=2, sigma=0.05, noise_seed=9)
    res = learned.evaluate(corr, fine, held)
    print(f"held-out force RMS vs fine ({kind}): coarse {res['coarse']:.4e} corrected {res['corrected']:.4e} "
          f"gain {res['coarse'] / res['corrected']:.2f}x; loss {log.loss[0][1]:.3e} -> {log.loss[-1][1]:.3e} "
          f"in {log.seconds:.2f} s")
    if kind == "cell":
        assert res["corrected"] < 0.8 * res["coarse"]
    else:
        assert res["corrected"] <= 1.02 * res["coarse"]
