"""Training and evaluation of the learned coarse-mesh correction.

The data come from the method itself: each frame is a seeded synthetic water
configuration; its labels are the forces of a fine-mesh FP32 PPPM; its inputs
are the features of the coarse plan (``Corrector.features``).  Every step of
the arithmetic (both PPPM solves, features, targets, forward, backward, Adam)
runs in the CUDA library; this module only allocates device buffers, draws
minibatch indices and loops.

Frames: a base configuration ``make_water(n_mol, L, seed)`` plus independent
N(0, sigma) noise on every coordinate, drawn on the device by a seeded torch
generator (one per base configuration), so the positions are reproducible for
a given seed and device.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch  # evaluation sums and minibatch indices only

from workloads.water import make_water, init_mlp_params

from .pppm import Corrector, Plan


@dataclass
class FrameSpec:
    n_mol: int
    L: float
    base_seeds: tuple
    frames_per_base: int
    sigma: float = 0.05
    noise_seed: int = 0


@dataclass
class Dataset:
    feat: torch.Tensor     # (frames * n, n_in) bf16, n_in = 48 or 32
    target: torch.Tensor   # (frames * n, 3) f32
    n_sites: int
    n_frames: int


@dataclass
class TrainLog:
    steps: int = 0
    loss: list = field(default_factory=list)   # (step, loss) samples
    seconds: float = 0.0


def frames(spec: FrameSpec, device="cuda"):
    """Yield (pos f32 (n,3), q f32 (n,), types int8 (n,)) device tensors."""
    for b in spec.base_seeds:
        w = make_water(spec.n_mol, spec.L, int(b))
        base = torch.tensor(w.pos, dtype=torch.float64, device=device)
        q = torch.tensor(w.q, dtype=torch.float32, device=device)
        types = torch.tensor(w.types, dtype=torch.int8, device=device)
        gen = torch.Generator(device=device)
        gen.manual_seed(int(spec.noise_seed) * 1_000_003 + int(b))
        for _ in range(spec.frames_per_base):
            noise = torch.randn(base.shape, generator=gen, dtype=torch.float64, device=device)
            yield (base + spec.sigma * noise).to(torch.float32).contiguous(), q, types


def build_dataset(corr: Corrector, fine: Plan, spec: FrameSpec, calibrate: bool = True) -> Dataset:
    """Features and targets of every frame, resident on the device.  With
    ``calibrate`` the scales are chosen on the first frame."""
    n = 4 * spec.n_mol
    F = len(spec.base_seeds) * spec.frames_per_base
    dev = torch.device("cuda")
    feat = torch.empty((F * n, corr.n_in), dtype=torch.bfloat16, device=dev)
    target = torch.empty((F * n, 3), dtype=torch.float32, device=dev)
    fc = torch.empty((n, 3), dtype=torch.float32, device=dev)
    for k, (pos, q, types) in enumerate(frames(spec)):
        _, ff, _ = fine.compute(pos, q)
        if k == 0 and calibrate:
            corr.calibrate(pos, q, types, ff)
        corr.features(pos, q, types, feat=feat[k * n:(k + 1) * n], forces=fc)
        corr.targets(ff, fc, q, out=target[k * n:(k + 1) * n])
    return Dataset(feat=feat, target=target, n_sites=n, n_frames=F)


def train(corr: Corrector, ds: Dataset, steps: int, batch: int = 4096, lr: float = 2e-3,
          seed: int = 0, log_every: int = 100, init_seed: int | None = None) -> TrainLog:
    """Adam on random minibatches with a cosine learning-rate decay."""
    if init_seed is not None:
        s_in, s_out = corr.scales
        corr.set_weights(init_mlp_params(init_seed, n_in=corr.n_in), s_in, s_out)
    dev = ds.feat.device
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed))
    total = ds.feat.shape[0]
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    log = TrainLog()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for k in range(steps):
        idx = torch.randint(0, total, (batch,), generator=gen, device=dev, dtype=torch.int32)
        lr_k = lr * 0.5 * (1.0 + math.cos(math.pi * k / max(1, steps)))
        corr.train_step(ds.feat, ds.target, idx, lr_k, loss=loss)
        if log_every and (k % log_every == 0 or k == steps - 1):
            log.loss.append((k, float(loss.item())))
    e1.record()
    torch.cuda.synchronize()
    log.steps = steps
    log.seconds = e0.elapsed_time(e1) / 1e3
    return log


def rms_rel(f: torch.Tensor, ref: torch.Tensor) -> float:
    """sqrt(sum |f - ref|^2 / sum |ref|^2) over all sites, summed in FP64."""
    a = f.double()
    b = ref.double()
    return float(torch.sqrt(torch.sum((a - b) ** 2) / torch.sum(b * b)).item())


def evaluate(corr: Corrector, fine: Plan, spec: FrameSpec, plain=()) -> dict:
    """Force RMS error against the fine mesh on the frames of ``spec``: the
    coarse plan alone, corrected, and any extra plain plans given."""
    out = {"coarse": [], "corrected": []}
    for P in plain:
        out[f"plain_{P.mesh[0]}"] = []
    for pos, q, types in frames(spec):
        _, ff, _ = fine.compute(pos, q)
        _, fc, _ = corr.coarse.compute(pos, q)
        _, fx, _ = corr.apply(pos, q, types)
        out["coarse"].append(rms_rel(fc, ff))
        out["corrected"].append(rms_rel(fx, ff))
        for P in plain:
            _, fp, _ = P.compute(pos, q)
            out[f"plain_{P.mesh[0]}"].append(rms_rel(fp, ff))
    return {k: float(np.sqrt(np.mean(np.square(v)))) for k, v in out.items()}
