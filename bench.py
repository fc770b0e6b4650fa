#!/usr/bin/env python
"""Benchmark: PPPM force evaluations per second on the 216,576-atom + 72,192-WC
water system (72,192 molecules, cubic 129.3 A box, order 5, beta 0.4 1/A,
FP32), over a 1,000-step random walk of the positions (0.01 A Gaussian noise
per coordinate and step, cumulative).

One step = one full force evaluation (bin/sort, spread, forward FFT,
influence with energy/virial, three ik inverse FFTs, gather) on that step's
positions.  Inputs of all 1,000 frames are resident in HBM before timing; L2
is flushed (256 MiB write) between timed steps, outside the timed events.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--mesh 128|160] [--impl ours|reference]

Rank 0 prints one JSON line.  With N > 1 (torchrun) every rank runs an
independent replica (the single-box path does not shard): weak scaling.
--impl reference times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "PPPM force evals/sec at 216,576 atoms+WCs"
UNIT = "evals/s"
N_FRAMES = 1000
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--mesh", type=int, default=128, choices=[128, 160])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--profile-steps", type=int, default=200)
    ap.add_argument("--frames", type=int, default=N_FRAMES, help="random-walk frames held on the device")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-wc-fold", action="store_true", help="skip the WC force fold measurement")
    ap.add_argument("--no-cufft", action="store_true", help="skip the cuFFT comparison leg")
    ap.add_argument("--workload", default="water72192", choices=["water72192", "batched96", "learned64", "overlap"],
                    help="water72192: the 216,576-atom system (default); batched96: 96 independent boxes; "
                         "learned64: the same system on a 64^3 mesh with the learned correction; "
                         "overlap: the 128^3 step concurrent with a short-range stand-in on a second stream")
    ap.add_argument("--train-frames", type=int, default=2000, help="learned64: training frames (20 bases)")
    ap.add_argument("--train-steps", type=int, default=20000, help="learned64: Adam steps")
    ap.add_argument("--train-batch", type=int, default=8192, help="learned64: sites per Adam step")
    ap.add_argument("--held-frames", type=int, default=100, help="learned64: held-out frames per base (2 bases)")
    ap.add_argument("--forward-only", action="store_true",
                    help="learned64: time only the network forward kernels (mma.sync and tcgen05) on the "
                         "system's features, seeded random weights, no training")
    return ap.parse_args()


def workload_name(mesh):
    return f"water72192_m{mesh}"


def workload_config(mesh, n):
    return {
        "workload": f"water72192: 216,576 atoms + 72,192 WCs = {n} sites, cubic 129.3 A, mesh {mesh}^3, "
                    f"order 5, beta 0.4/A, FP32, {N_FRAMES}-step 0.01 A random walk",
        "n_sites": n,
        "mesh": [mesh, mesh, mesh],
        "order": 5,
        "beta": 0.4,
        "frames": N_FRAMES,
        "l2": "flushed between timed steps (256 MiB write, outside the events)",
        "launch": "one CUDA graph of the step, replayed with each frame's site pointers",
    }


# --------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "20",
                 "-i", str(gpu_index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_index_for(local_rank: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v for v in vis.split(",") if v.strip()]
        if local_rank < len(ids) and ids[local_rank].strip().isdigit():
            return int(ids[local_rank])
    return local_rank


# --------------------------------------------------------------------- bytes
def algorithmic_bytes(n: int, mesh: int) -> dict:
    """Bytes each kernel must move at minimum (FP32): inputs read once, outputs
    written once.  Sites are 16 B in (position + charge), forces 12 B out."""
    N = mesh ** 3
    NH = mesh * mesh * (mesh // 2 + 1)
    return {
        "spread": 16 * n + 4 * N,
        "gather": 12 * N + 16 * n + 12 * n,
        "fft_z_r2c": 4 * N + 8 * NH,
        "fft_y": 16 * NH,
        "fft_x_influence": 8 * NH + 4 * NH + 16 * NH,
        "fft_y_inverse3": 16 * NH + 24 * NH,
        "fft_z_c2r": 24 * NH + 12 * N,
        # the one-pass sort into fixed tile regions: positions and charges in;
        # record (16 B: B-spline arguments, charge), cell, original index,
        # tile and rank out
        "bin": 16 * n + 32 * n,
        "scatter": 0,  # the region sort's fallback: idle unless a region overflows
        "tiles_init": 8 * ((mesh + 7) // 8) ** 3,
        "fold": 8 * N,
        "scan": 0,
    }


def step_algorithmic_bytes(n: int, mesh: int) -> int:
    """The whole step as the method needs it: spread, one forward FFT pass,
    influence, three inverse FFT passes, gather."""
    N = mesh ** 3
    NH = mesh * mesh * (mesh // 2 + 1)
    return (16 * n + 4 * N) + (4 * N + 8 * NH) + (8 * NH + 4 * NH) + 3 * (8 * NH + 4 * N) + (12 * N + 28 * n)


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch from
# one ncu --set full capture of the kernel as it stands, on this workload; an
# entry is removed whenever its kernel changes.
NCU_TRAFFIC = {
    ("gather", 128): 44.61e6,
    ("spread", 128): 7.73e6,
    ("bin", 128): 4.87e6,
    ("fft_z_r2c", 128): 30.71e6,
    ("fft_y", 128): 8.54e6,
    ("fft_x_influence", 128): 12.86e6,
    ("fft_y_inverse3", 128): 17.08e6,
    ("fft_z_c2r", 128): 25.75e6,
    ("fft_x_influence", 160): 24.98e6,
    ("gather", 160): 82.63e6,
}


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# --------------------------------------------------------------------- oracle (CPU)
# The oracle on every host core: a spawn-started process pool (started after
# the GPU work has begun, so fork is not an option), one plan per worker built
# once (plan-time influence function excluded), one thread a worker.
_POOL_ORACLE = None


def _pool_init(box, mesh, order, beta, q):
    global _POOL_ORACLE
    os.environ["OMP_NUM_THREADS"] = "1"
    from oracle.pppm import OraclePPPM
    _POOL_ORACLE = (OraclePPPM(box, mesh, order, beta), q)


def _pool_eval(pos):
    o, q = _POOL_ORACLE
    r = o.compute(pos, q)
    return r["energy"]


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_all_cores(wb, w, frames_fn, rounds: int, workers: int | None = None):
    """Throughput of the FP64 oracle with one evaluation per host core at a
    time: `rounds` rounds of `workers` evaluations of successive frames, each
    round timed by the wall clock (one warm-up round first).  Returns (median
    evals/s, per-round evals/s, workers)."""
    import multiprocessing as mp
    workers = workers or host_cores()
    old = os.environ.get("OMP_NUM_THREADS")
    os.environ["OMP_NUM_THREADS"] = "1"  # inherited by the spawned workers
    ctx = mp.get_context("spawn")
    rates = []
    try:
        with ctx.Pool(workers, initializer=_pool_init,
                      initargs=(wb.box, w["mesh"], w["order"], w["beta"], wb.q)) as pool:
            k = 0
            for rnd in range(rounds + 1):
                batch = [frames_fn(k + j) for j in range(workers)]
                k += workers
                t0 = time.perf_counter()
                pool.map(_pool_eval, batch, chunksize=1)
                dt = time.perf_counter() - t0
                if rnd > 0:
                    rates.append(workers / dt)
    finally:
        if old is None:
            os.environ.pop("OMP_NUM_THREADS", None)
        else:
            os.environ["OMP_NUM_THREADS"] = old
    return statistics.median(rates), rates, workers


def oracle_single(wb, w, frames_fn, evals: int):
    """Median time of `evals` single-threaded FP64 oracle evaluations."""
    from oracle.pppm import OraclePPPM
    o = OraclePPPM(wb.box, w["mesh"], w["order"], w["beta"])
    ts, first = [], None
    for k in range(evals):
        pos = frames_fn(k)
        t0 = time.perf_counter()
        r = o.compute(pos, wb.q)
        ts.append(time.perf_counter() - t0)
        if first is None:
            first = r
    return 1.0 / statistics.median(ts), ts, first


def direct_ewald_times():
    """The direct E_Gt sum (energy, forces, virial) on the two small water
    boxes, on all host cores (its loops are OpenMP) and, for the 64-water box,
    on one core."""
    import ctypes

    from oracle import native
    from workloads.water import make_workload
    gomp = None
    try:
        gomp = ctypes.CDLL("libgomp.so.1")
    except OSError:
        pass
    out = {}
    cores = host_cores()
    for name, single in (("water64", True), ("water4096", False)):
        wb, w = make_workload(name)
        res = {"sites": wb.n}
        for label, nt in (("all_cores", cores), ("single_thread", 1)):
            if label == "single_thread" and (not single or gomp is None):
                continue
            if gomp is not None:
                gomp.omp_set_num_threads(nt)
            ts = []
            for _ in range(3 if name == "water64" else 1):
                t0 = time.perf_counter()
                native.egt_direct(wb.pos, wb.q, wb.box, w["beta"])
                ts.append(time.perf_counter() - t0)
            res[label] = {"evals_per_s": 1.0 / statistics.median(ts), "seconds": statistics.median(ts),
                          "threads": nt, "evals": len(ts)}
        out[name] = res
    if gomp is not None:
        gomp.omp_set_num_threads(cores)
    return out


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part", "hardware")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def run_reference(args):
    from workloads.water import NOISE_SEED_1000_STEPS, NOISE_SIGMA_1000_STEPS, make_workload
    wb, w = make_workload(workload_name(args.mesh))
    rng = np.random.default_rng(NOISE_SEED_1000_STEPS)
    cur = [wb.pos.astype(np.float32).astype(np.float64)]

    def frame(k):
        if k > 0:
            cur[0] = (cur[0] + rng.normal(0.0, NOISE_SIGMA_1000_STEPS, size=cur[0].shape)).astype(np.float32).astype(np.float64)
        return cur[0]

    # one round of evaluations per step, one evaluation per host core in a
    # round; the warm-up round is untimed; at most 3 timed rounds (each a few
    # seconds), so that any K ends within about a minute
    frames = {}

    def frame_at(k):
        while len(frames) <= k:
            frames[len(frames)] = frame(len(frames))
        return frames[k]

    rounds = max(1, min(args.steps, 3))
    val, rates, cores = oracle_all_cores(wb, w, frame_at, rounds)
    done = rounds
    sample = (f"{rounds} round(s) of {cores} concurrent full FP64 evaluations (one per host core, spawned "
              f"worker processes, one thread each) of successive frames of the workload, after one untimed "
              f"round; median round throughput; plan-time influence function excluded; K = {args.steps} "
              f"requested, capped at 3 rounds")
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": done, "warmup": min(args.warmup, 1), "ms_per_step": 1e3 / val, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {k: v for k, v in workload_config(args.mesh, wb.n).items() if k != "launch"},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                         "cpu": cpu_model(), "rounds_evals_per_s": rates},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------- WC fold
def run_wc_fold(args, wb, forces, flush, stream, peak):
    """Time the fold of the WC forces onto the atoms with a synthetic
    Deep-Wannier Jacobian of local sparsity (each WC depends on the 81 atoms of
    the 27 molecules around it): one launch streams the Jacobian once."""
    import torch

    from paper_2504_15508_gb300.pppm import wc_fold
    from workloads.water import dw_jacobian

    dev = forces.device
    hp, hw, jp, jw, _ = dw_jacobian(wb, seed=11, values=False)
    n_atoms, n_wc = 3 * wb.n_mol, wb.n_mol
    nnz = int(jp[-1])
    gen = torch.Generator(device=dev)
    gen.manual_seed(11)
    jac = 0.02 * torch.randn((nnz, 3, 3), generator=gen, dtype=torch.float32, device=dev)
    maps = (torch.tensor(hp, device=dev), torch.tensor(hw, device=dev), torch.tensor(jp, device=dev),
            torch.tensor(jw, device=dev), jac)
    out = torch.empty((n_atoms, 3), dtype=torch.float32, device=dev)
    for _ in range(3):
        wc_fold(forces, n_atoms, *maps, out=out, stream=stream)
    K = min(args.steps, 200)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    torch.cuda.synchronize()
    for k in range(K):
        flush.fill_(float(k))
        evs[k][0].record(stream)
        wc_fold(forces, n_atoms, *maps, out=out, stream=stream)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs) / K
    # Jacobian blocks + WC indices, row offsets, host map, site forces in, atom forces out
    alg = nnz * (36 + 4) + (n_atoms + 1) * (8 + 4) + n_wc * 4 + (n_atoms + n_wc) * 12 + n_atoms * 12
    achieved = alg / (ms * 1e-3) / 1e9
    return {"kernel": "wc_fold", "n_atoms": n_atoms, "n_wc": n_wc, "jacobian_blocks": nnz,
            "us_per_launch": ms * 1e3, "launches": K,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "algorithmic_bytes": alg, "traffic": None}}


# --------------------------------------------------------------------- cuFFT comparison
FFT_PASSES = ("fft_z_r2c", "fft_y", "fft_x_influence", "fft_y_inverse3", "fft_z_c2r")


def cufft_comparison(plan, mesh, dev, stream, flush, kernels, reps=50):
    """cuFFT (through torch.fft) timed as a comparison only, never on the
    product path: the R2C transform of the charge mesh and the C2R transforms
    of three field spectra (one batched call), CUDA events on the compute
    stream, L2 flushed before every call.  Set against the sum of this
    library's FFT passes, which also fold the spread's tile patches (z
    forward), apply the influence function with the energy/virial sums and
    form the three ik spectra (x pass), and write the padded interleaved field
    meshes (z inverse).  The own forward transform is also compared with
    cuFFT's output."""
    import torch
    N = mesh
    gen = torch.Generator(device=dev)
    gen.manual_seed(5)
    x = torch.randn((N, N, N), generator=gen, device=dev, dtype=torch.float32)
    spec3 = torch.randn((3, N, N, N // 2 + 1), generator=gen, device=dev, dtype=torch.complex64)
    with torch.cuda.stream(stream):
        for _ in range(3):
            torch.fft.rfftn(x)
            torch.fft.irfftn(spec3, s=(N, N, N), dim=(-3, -2, -1))

        def timed(fn):
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
            for k in range(reps):
                flush.fill_(float(k))
                evs[k][0].record(stream)
                fn()
                evs[k][1].record(stream)
            torch.cuda.synchronize()
            return statistics.median(a.elapsed_time(b) for a, b in evs)

        r2c = timed(lambda: torch.fft.rfftn(x))
        c2r3 = timed(lambda: torch.fft.irfftn(spec3, s=(N, N, N), dim=(-3, -2, -1)))
        ref = torch.fft.rfftn(x.double())
    own = plan.fft_r2c(x, stream=stream)
    torch.cuda.synchronize()
    diff = float((own.to(torch.complex128) - ref).norm() / ref.norm())
    cufft_ms = r2c + c2r3
    own_ms = sum(kernels[k]["ms_per_launch"] for k in FFT_PASSES if kernels.get(k, {}).get("ms_per_launch"))
    return {"what": "cuFFT via torch.fft: rfftn of the real mesh + irfftn of 3 spectra (batched), FP32; "
                    "comparison only", "mesh": [N, N, N], "cufft_r2c_us": r2c * 1e3, "cufft_c2r3_us": c2r3 * 1e3,
            "cufft_total_us": cufft_ms * 1e3, "own_fft_passes_us": own_ms * 1e3,
            "own_over_cufft": own_ms / cufft_ms if cufft_ms > 0 else None,
            "own_r2c_vs_cufft_fp64_rel": diff, "reps": reps, "timing": "median of CUDA-event pairs, L2 flushed"}


# --------------------------------------------------------------------- ours
def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2504_15508_gb300.pppm import Plan
    from workloads.water import NOISE_SEED_1000_STEPS, NOISE_SIGMA_1000_STEPS, make_workload

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    wb, w = make_workload(workload_name(args.mesh))
    n = wb.n
    # frames: cumulative Gaussian random walk, generated on the device once (seeded)
    gen = torch.Generator(device=dev)
    gen.manual_seed(NOISE_SEED_1000_STEPS)
    base = torch.tensor(wb.pos, dtype=torch.float64, device=dev)
    nf = max(1, min(args.frames, N_FRAMES))
    frames = torch.empty((nf, n, 3), dtype=torch.float32, device=dev)
    cur = base.clone()
    for k in range(nf):
        if k > 0:
            cur += NOISE_SIGMA_1000_STEPS * torch.randn(cur.shape, generator=gen, dtype=torch.float64, device=dev)
        frames[k] = cur.float()
    del cur, base
    q = torch.tensor(wb.q, dtype=torch.float32, device=dev)

    plan = Plan(wb.box, w["mesh"], w["order"], w["beta"], precision="fp32")
    plan.reserve(n)
    energy = torch.empty(1, dtype=torch.float64, device=dev)
    forces = torch.empty((n, 3), dtype=torch.float32, device=dev)
    virial = torch.empty(6, dtype=torch.float64, device=dev)
    out = (energy, forces, virial)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def eager_step(k):
        plan.compute(frames[k % nf], q, out=out, stream=stream)

    for k in range(args.warmup):
        flush.fill_(float(k))
        eager_step(k)
    torch.cuda.synchronize()
    # the timed steps replay one captured graph of the step, each on its own frame
    graph = plan.graph(frames[0], q, out=out)

    def step(k):
        graph.launch(frames[k % nf], q, stream=stream)

    for k in range(args.warmup):
        flush.fill_(float(k))
        step(k)
    torch.cuda.synchronize()

    K = args.steps
    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    sampler = ClockSampler(gpu_index_for(local))
    time.sleep(0.05)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for k in range(K):
        flush.fill_(float(k))
        ev_s[k].record(stream)
        step(k)
        ev_e[k].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    step_ms = [ev_s[k].elapsed_time(ev_e[k]) for k in range(K)]
    total_ms = float(sum(step_ms))
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * K / (total_ms * 1e-3)

    graph.close()
    # per-kernel breakdown: a second timed loop with event brackets around each launch
    P = min(K, args.profile_steps)
    plan.profile(True)
    for k in range(P):
        flush.fill_(float(k))
        eager_step(k)
    torch.cuda.synchronize()
    prof = plan.profile_read()
    plan.profile(False)
    kernels = {name: {"ms_per_launch": ms / c if c else None, "launches": c} for name, (ms, c) in prof.items()}
    launches_per_step = sum(1 for name, (ms, c) in prof.items() if c)

    peak, peak_kind = read_peaks()
    alg = algorithmic_bytes(n, args.mesh)
    dom = max((nm for nm in prof if prof[nm][1]), key=lambda nm: prof[nm][0])
    dom_ms = prof[dom][0] / prof[dom][1]
    achieved = alg[dom] / (dom_ms * 1e-3) / 1e9
    roofline = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_kind": peak_kind, "traffic": NCU_TRAFFIC.get((dom, args.mesh)),
                "algorithmic_bytes": alg[dom]}
    per_kernel_frac = {nm: (alg[nm] / (kernels[nm]["ms_per_launch"] * 1e-3) / 1e9) / peak
                       for nm in kernels if kernels[nm]["launches"] and alg.get(nm)}
    step_bytes = step_algorithmic_bytes(n, args.mesh)
    ms_per_step = total_ms / K

    # end to end through the host-pointer C ABI call (copies inside the timed region)
    E = min(args.e2e_steps, nf)
    host_frames = frames[:E].cpu().pin_memory()
    host_q = q.cpu().pin_memory()
    hq = host_q.numpy()
    # results land in pinned host buffers owned by the caller
    h_out = (torch.zeros(1, dtype=torch.float64).pin_memory().numpy(),
             torch.zeros((n, 3), dtype=torch.float32).pin_memory().numpy(),
             torch.zeros(6, dtype=torch.float64).pin_memory().numpy())
    for k in range(min(3, E)):
        plan.compute_host(host_frames[k].numpy(), hq, out=h_out)
    # each step timed on the host clock around the blocking call (copies in,
    # the step, copies out); the median step, so that a host-side stall of
    # another process on the machine does not stand for the path
    step_s = []
    t0 = time.perf_counter()
    for k in range(E):
        t1 = time.perf_counter()
        e_h, f_h, v_h = plan.compute_host(host_frames[k].numpy(), hq, out=h_out)
        step_s.append(time.perf_counter() - t1)
    e2e_s = time.perf_counter() - t0
    med = statistics.median(step_s)
    e2e_val = world / med
    e2e = {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 16 * n, "d2h_bytes_per_step": 12 * n + 56,
           "steps": E, "host_memory": "pinned inputs and outputs", "statistic": "median step",
           "mean_step_value": world * E / e2e_s}

    # the WC force fold (Eq. DPLR:F_final) on this step's forces, timed on its own
    wc_fold_line = run_wc_fold(args, wb, forces, flush, stream, peak) if not args.no_wc_fold else None
    cufft = cufft_comparison(plan, args.mesh, dev, stream, flush, kernels) if not args.no_cufft else None

    # parity of frame 0 and the CPU baseline (rank 0, N = 1 only)
    parity, cpu = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        host_fr = {}

        def hframe(k):
            if k not in host_fr:
                host_fr[k] = frames[k % nf].double().cpu().numpy()
            return host_fr[k]

        e_g, f_g, v_g = plan.compute(frames[0], q)
        torch.cuda.synchronize()
        single_val, single_ts, ref = oracle_single(wb, w, hframe, 3)
        all_val, all_rates, cores = oracle_all_cores(wb, w, hframe, 3)
        ewald = direct_ewald_times()
        fg = f_g.double().cpu().numpy()
        parity = {"force_rms_rel_err": float(np.linalg.norm(fg - ref["forces"]) / np.linalg.norm(ref["forces"])),
                  "energy_rel_err": abs(e_g.item() - ref["energy"]) / abs(ref["energy"]),
                  "virial_rel_err": float(np.linalg.norm(v_g.cpu().numpy() - ref["virial"]) /
                                          np.linalg.norm(ref["virial"])),
                  "vs": "FP64 CPU oracle, frame 0"}
        cpu = {"value": all_val, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": (f"all cores: 3 rounds of {cores} concurrent full FP64 evaluations (spawned worker "
                          f"processes, one thread each) of frames of the random walk after one untimed round, "
                          f"median round; single thread: median of 3 evaluations of frames 0-2; plan-time "
                          f"influence function excluded"),
               "cpu": cpu_model(),
               "all_cores": {"evals_per_s": all_val, "rounds_evals_per_s": all_rates, "workers": cores},
               "single_thread": {"evals_per_s": single_val, "seconds": single_ts},
               "direct_ewald": ewald}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic", "config": workload_config(args.mesh, n),
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
        "gpu_launches": launches_per_step * K,
        "kernels": kernels, "kernel_hbm_frac": per_kernel_frac,
        "step_roofline": {"algorithmic_bytes": step_bytes,
                          "achieved_gbs": step_bytes / (ms_per_step * 1e-3) / 1e9,
                          "frac": step_bytes / (ms_per_step * 1e-3) / 1e9 / peak},
        "parity": parity, "wall_s_timed_loop": wall,
        "wc_fold": wc_fold_line,
        "cufft_comparison": cufft,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()


# --------------------------------------------------------------------- batched form
def run_batched(args):
    """96 independent water boxes per GPU (64 to 8,192 molecules, log-uniform,
    29.9 A^3 per molecule, meshes at <= 1.2 A spacing) in one persistent launch
    replayed from a CUDA graph.  On one GPU it is compared with the same boxes
    as 96 single-box calls, issued one by one and captured into one CUDA graph
    (one stream, or four); with N GPUs (torchrun) 96 N boxes are split across
    the ranks by cost (weak scaling, no collective in the data path)."""
    import torch
    import torch.distributed as dist

    from paper_2504_15508_gb300.pppm import BatchPlan, Plan
    from paper_2504_15508_gb300.shard import box_costs, gather_by_box, partition, slowest
    from workloads.water import batched_boxes, make_water

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    all_specs = batched_boxes(nbox=96 * world, seed=5)
    mine = partition(box_costs([4 * s["n_mol"] for s in all_specs], [s["mesh"] for s in all_specs]), world)[rank]
    specs = [all_specs[b] for b in mine]
    nb = len(specs)
    boxes = [make_water(s["n_mol"], s["L"], s["seed"]) for s in specs]
    pos = np.concatenate([b.pos for b in boxes]).astype(np.float32)
    q = np.concatenate([b.q for b in boxes]).astype(np.float32)
    offs = np.concatenate([[0], np.cumsum([b.n for b in boxes])]).astype(np.int64)
    n = int(offs[-1])
    tp = torch.tensor(pos, device=dev)
    tq = torch.tensor(q, device=dev)
    to = torch.tensor(offs, device=dev)
    bp = BatchPlan(np.array([[s["L"]] * 3 for s in specs]), None, order=5, beta=0.4)
    out = (torch.empty(nb, dtype=torch.float64, device=dev), torch.empty((n, 3), dtype=torch.float32, device=dev),
           torch.empty((nb, 6), dtype=torch.float64, device=dev))
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for k in range(max(3, args.warmup)):
        bp.compute(tp, tq, to, out=out, stream=stream)
    torch.cuda.synchronize()
    K = args.steps

    def timed(fn):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        for k in range(K):
            flush.fill_(float(k))
            evs[k][0].record(stream)
            fn()
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs) / K

    ms_batched = slowest(timed(lambda: bp.compute(tp, tq, to, out=out, stream=stream)))
    # the launch form the autotuner chose, then each form forced
    auto_form = bp.launch
    ms_form = {}
    for form in ("persistent", "staged"):
        bp.set_launch(form)
        for k in range(3):
            bp.compute(tp, tq, to, out=out, stream=stream)
        torch.cuda.synchronize()
        ms_form[form] = slowest(timed(lambda: bp.compute(tp, tq, to, out=out, stream=stream)))
    bp.set_launch("auto")
    for k in range(3):
        bp.compute(tp, tq, to, out=out, stream=stream)
    torch.cuda.synchronize()
    energies = gather_by_box(len(all_specs), mine, out[0].cpu().numpy())
    line = {
        "metric": "batched PPPM evals/s, 96 water boxes of 64-8,192 molecules", "value": world * 1e3 / ms_batched,
        "unit": "batch-evals/s", "n_gpus": world, "steps": K, "warmup": args.warmup, "ms_per_step": ms_batched,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batched96: 96 cubic water boxes per GPU ({len(all_specs)} in all, split by cost), "
                               f"meshes at <= 1.2 A, order 5; this rank: {nb} boxes, "
                               f"{int(sum(s['n_mol'] for s in specs))} molecules, {n} sites",
                   "tile": bp.tile, "l2": "flushed between timed steps"},
        "energy_sum_all_boxes": float(np.sum(energies)),
        "launch_form": auto_form, "ms_by_launch_form": ms_form,
        "staged_speedup_vs_persistent": ms_form["persistent"] / ms_form["staged"],
    }
    if world == 1:
        # the same batch with lines of length <= 18 as a DFT on the tensor cores
        f_fft = out[1].clone()
        bp.set_dft(18)
        for k in range(3):
            bp.compute(tp, tq, to, out=out, stream=stream)
        ms_dft = timed(lambda: bp.compute(tp, tq, to, out=out, stream=stream))
        torch.cuda.synchronize()
        dft_vs_fft = float(torch.linalg.norm(out[1].double() - f_fft.double()) / torch.linalg.norm(f_fft.double()))
        bp.set_dft(0)
        for k in range(3):
            bp.compute(tp, tq, to, out=out, stream=stream)
        meshes = bp.meshes
        plans = [Plan(b.box, meshes[i], 5, 0.4, precision="fp32") for i, b in enumerate(boxes)]
        sl = [slice(int(offs[i]), int(offs[i + 1])) for i in range(nb)]
        pv = [(tp[x].contiguous(), tq[x].contiguous()) for x in sl]
        outs = [(torch.empty(1, dtype=torch.float64, device=dev), torch.empty((x.stop - x.start, 3),
                 dtype=torch.float32, device=dev), torch.empty(6, dtype=torch.float64, device=dev)) for x in sl]

        def singles():
            for i in range(nb):
                plans[i].compute(pv[i][0], pv[i][1], out=outs[i], stream=stream)

        for _ in range(3):
            singles()
        Ks, K = K, min(K, 50)
        ms_single = timed(singles)
        K = Ks

        # the fair baseline: the same 96 single-box calls captured into one
        # CUDA graph (no host launch cost per kernel), on one stream and spread
        # over four streams (the plans own separate workspaces)
        def singles_graph(nstreams):
            side = torch.cuda.Stream()
            side.wait_stream(stream)
            with torch.cuda.stream(side):
                for i in range(nb):
                    plans[i].compute(pv[i][0], pv[i][1], out=outs[i], stream=side)
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            subs = [torch.cuda.Stream() for _ in range(nstreams)]
            with torch.cuda.graph(g, stream=side):
                if nstreams == 1:
                    for i in range(nb):
                        plans[i].compute(pv[i][0], pv[i][1], out=outs[i], stream=side)
                else:
                    for st in subs:
                        st.wait_stream(side)
                    for i in range(nb):
                        plans[i].compute(pv[i][0], pv[i][1], out=outs[i], stream=subs[i % nstreams])
                    for st in subs:
                        side.wait_stream(st)
            return g

        ms_graph = {}
        for ns in (1, 4):
            g = singles_graph(ns)
            for _ in range(3):
                g.replay()
            torch.cuda.synchronize()
            ms_graph[ns] = timed(g.replay)
            del g
        bp.compute(tp, tq, to, out=out, stream=stream)
        torch.cuda.synchronize()
        diff = max(float(torch.linalg.norm(out[1][sl[i]].double() - outs[i][1].double()) /
                         torch.linalg.norm(outs[i][1].double())) for i in range(nb))
        ediff = max(abs(out[0][i].item() - outs[i][0].item()) / abs(outs[i][0].item()) for i in range(nb))
        line.update({
            "single_box_calls_ms": ms_single, "speedup_vs_single_box_calls": ms_single / ms_batched,
            "single_box_graph_ms": {"1_stream": ms_graph[1], "4_streams": ms_graph[4]},
            "speedup_vs_single_box_graph": min(ms_graph.values()) / ms_batched,
            "tensor_core_dft_ms": ms_dft, "tensor_core_dft_speedup": ms_batched / ms_dft,
            "force_rel_diff_dft_vs_fft": dft_vs_fft,
            "max_force_rel_diff_vs_single": diff, "max_energy_rel_diff_vs_single": ediff,
        })
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# --------------------------------------------------------------------- learned form
def run_forward(args):
    """The learned correction's network forward alone: the 288,768 sites'
    features on the 64^3 coarse mesh (both feature sets), seeded random
    weights, each kernel (warp-level mma.sync, tcgen05 with tensor-memory
    accumulators) timed as replays of a CUDA graph of the call, L2 flushed
    before each; the two kernels' outputs are compared."""
    import torch

    from paper_2504_15508_gb300.pppm import Corrector, Plan
    from workloads.water import init_mlp_params, make_workload

    dev = torch.device("cuda", 0)
    wb, w = make_workload("water72192_m64")
    n = wb.n
    coarse = Plan(wb.box, (64,) * 3, 5, 0.4, precision="fp32")
    pos = torch.tensor(wb.pos, dtype=torch.float32, device=dev)
    q = torch.tensor(wb.q, dtype=torch.float32, device=dev)
    types = torch.tensor(wb.types, dtype=torch.int8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    K = args.steps

    def graph_timed(fn):
        side = torch.cuda.Stream()
        with torch.cuda.stream(side):
            for _ in range(max(3, args.warmup)):
                fn(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            fn(side)
        torch.cuda.synchronize()
        cur = torch.cuda.current_stream()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        for k in range(K):
            flush.fill_(float(k))
            evs[k][0].record(cur)
            g.replay()
            evs[k][1].record(cur)
        torch.cuda.synchronize()
        return statistics.median(a.elapsed_time(b) for a, b in evs)

    sampler = ClockSampler(gpu_index_for(0))
    kinds = {}
    for kind in ("stated", "cell"):
        n_in = Corrector.WIDTH[kind]
        corr = Corrector(coarse, params=init_mlp_params(3, n_in=n_in).astype(np.float32), s_in=0.5, s_out=1.0,
                         features=kind)
        feat, _ = corr.features(pos, q, types)
        flop = 2.0 * n * (n_in * 64 + 64 * 64 + 64 * 3)
        res, ys = {}, {}
        for fwd in ("mma_sync", "tcgen05"):
            corr.set_forward(fwd)
            y = torch.empty((n, 3), dtype=torch.float32, device=dev)
            ms = graph_timed(lambda st: corr.forward(feat, out=y, stream=st))
            res[fwd] = {"us": ms * 1e3, "tflops": flop / (ms * 1e-3) / 1e12}
            ys[fwd] = y
        if coarse.status() != 0:
            raise RuntimeError("forward kernel status set")
        res["max_abs_diff"] = float((ys["tcgen05"] - ys["mma_sync"]).abs().max())
        res["inputs"] = n_in
        kinds[kind] = res
        corr.close()
    clocks = sampler.stop()
    main = kinds["stated"]["mma_sync"]["us"]
    line = {
        "metric": "learned-correction network forward, sites/s", "value": n / (main * 1e-6), "unit": "sites/s",
        "n_gpus": 1, "steps": K, "warmup": args.warmup, "ms_per_step": main * 1e-3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": f"water72192 features on the 64^3 mesh ({n} sites), n_in-64-64-3 tanh network, "
                               f"seeded random weights; the line's value: stated set, mma.sync kernel",
                   "l2": "flushed between timed steps"},
        "kernels": kinds, "clocks": clocks, "gpu_launches": K,
    }
    print(json.dumps(line), flush=True)


def run_learned(args):
    """The 216,576-atom system on a coarse 64^3 mesh plus the learned
    correction, trained here on fine-mesh (160^3) forces of seeded perturbed
    frames, evaluated on held-out frames against the fine mesh; timed against
    the plain FP32 PPPM on the smallest mesh reaching the same force error.
    Both feature sets run: the stated one (27 potential samples + site type)
    and the cell one (the same + the site's offset inside its mesh cell).
    Every timed evaluation, corrected or plain, is a replay of a CUDA graph of
    the whole call."""
    import torch

    from paper_2504_15508_gb300 import learned
    from paper_2504_15508_gb300.pppm import Corrector, Plan
    from workloads.water import make_workload

    dev = torch.device("cuda", 0)
    wb, w = make_workload("water72192_m64")
    L, n_mol, n = float(wb.box[0]), wb.n_mol, wb.n
    box = (L, L, L)
    coarse = Plan(box, (64,) * 3, 5, 0.4, precision="fp32")
    fine = Plan(box, (160,) * 3, 5, 0.4, precision="fp32")
    nbase = 20
    fpb = max(1, args.train_frames // nbase)
    spec = learned.FrameSpec(n_mol=n_mol, L=L, base_seeds=tuple(range(100, 100 + nbase)), frames_per_base=fpb,
                             sigma=0.05, noise_seed=0)
    held = learned.FrameSpec(n_mol=n_mol, L=L, base_seeds=(200, 201), frames_per_base=args.held_frames, sigma=0.05,
                             noise_seed=7)
    meshes = [64, 72, 80, 90, 96, 100, 108, 120, 128]
    plain = [Plan(box, (m,) * 3, 5, 0.4, precision="fp32") for m in meshes[1:]]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    pos, q, types = next(learned.frames(held))
    K = args.steps
    o_c = (torch.empty(1, dtype=torch.float64, device=dev), torch.empty((n, 3), dtype=torch.float32, device=dev),
           torch.empty(6, dtype=torch.float64, device=dev))

    def graph_timed(fn):
        """Capture fn (stream-ordered library calls) once as a CUDA graph after
        warm-up calls, then time K replays, L2 flushed before each."""
        side = torch.cuda.Stream()
        with torch.cuda.stream(side):
            for _ in range(max(3, args.warmup)):
                fn(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            fn(side)
        for _ in range(3):
            g.replay()
        torch.cuda.synchronize()
        cur = torch.cuda.current_stream()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        for k in range(K):
            flush.fill_(float(k))
            evs[k][0].record(cur)
            g.replay()
            evs[k][1].record(cur)
        torch.cuda.synchronize()
        del g
        return statistics.median(a.elapsed_time(b) for a, b in evs)

    ms_plain = {64: graph_timed(lambda st: coarse.compute(pos, q, out=o_c, stream=st))}
    for P in plain + [fine]:
        ms_plain[P.mesh[0]] = graph_timed(lambda st, P=P: P.compute(pos, q, out=o_c, stream=st))

    sampler = ClockSampler(gpu_index_for(0))
    modes = {}
    for kind in ("stated", "cell"):
        corr = Corrector(coarse, features=kind)
        t0 = time.perf_counter()
        ds = learned.build_dataset(corr, fine, spec)
        torch.cuda.synchronize()
        t_data = time.perf_counter() - t0
        log = learned.train(corr, ds, steps=args.train_steps, batch=args.train_batch, lr=2e-3, seed=0, init_seed=0,
                            log_every=max(1, args.train_steps // 20))
        data_bytes = ds.feat.numel() * 2 + ds.target.numel() * 4
        del ds
        torch.cuda.empty_cache()
        err = learned.evaluate(corr, fine, held, plain=plain)
        err["plain_64"] = err["coarse"]
        eq = next((m for m in meshes if err[f"plain_{m}"] <= err["corrected"]), None)
        feat = torch.empty((n, corr.n_in), dtype=torch.bfloat16, device=dev)
        y = torch.empty((n, 3), dtype=torch.float32, device=dev)
        ms_corr = graph_timed(lambda st: corr.apply(pos, q, types, out=o_c, stream=st))
        ms_feat = graph_timed(lambda st: corr.features(pos, q, types, feat=feat, forces=o_c[1], stream=st))
        ms_mlp = graph_timed(lambda st: corr.forward(feat, out=y, stream=st))
        # the same forward on the tcgen05 kernel, for comparison
        corr.set_forward("tcgen05")
        ms_mlp_tc = graph_timed(lambda st: corr.forward(feat, out=y, stream=st))
        corr.set_forward("mma_sync")
        mlp_flop = 2.0 * n * (corr.n_in * 64 + 64 * 64 + 64 * 3)
        speedup = ms_plain[eq] / ms_corr if eq is not None else None
        # the plain mesh of exactly the corrected error, by interpolating
        # log(error) and time linearly between the two neighbouring meshes
        interp = None
        for m0, m1 in zip(meshes, meshes[1:]):
            e0, e1 = err[f"plain_{m0}"], err[f"plain_{m1}"]
            if e1 <= err["corrected"] <= e0:
                f = math.log(e0 / err["corrected"]) / math.log(e0 / e1)
                t = ms_plain[m0] + f * (ms_plain[m1] - ms_plain[m0])
                interp = {"mesh": m0 + f * (m1 - m0), "ms": t, "speedup": t / ms_corr}
                break
        modes[kind] = {
            "inputs": corr.n_in, "params": corr.nparams,
            "force_rms_rel_err_vs_fine160": err,
            "equal_error_plain_mesh": eq,
            "speedup_vs_plain_at_equal_error": speedup,
            "equal_error_interpolated": interp,
            "gain_in_error_vs_coarse": err["coarse"] / err["corrected"],
            "ms": {"corrected": ms_corr, "coarse_plus_features": ms_feat, "mlp_forward": ms_mlp,
                   "mlp_forward_tcgen05": ms_mlp_tc},
            "mlp_forward_tflops": {"mma_sync": mlp_flop / (ms_mlp * 1e-3) / 1e12,
                                   "tcgen05": mlp_flop / (ms_mlp_tc * 1e-3) / 1e12},
            "train": {"steps": log.steps, "batch": args.train_batch, "seconds": log.seconds,
                      "data_seconds": t_data, "data_gb": data_bytes / 1e9, "loss": log.loss[::4] + log.loss[-1:]},
        }
        corr.close()
        torch.cuda.empty_cache()
    clocks = sampler.stop()
    main = modes["stated"]
    line = {
        "metric": "learned coarse-mesh PPPM force evals/s at 216,576 atoms+WCs", "value": 1e3 / main["ms"]["corrected"],
        "unit": UNIT, "n_gpus": 1, "steps": K, "warmup": args.warmup, "ms_per_step": main["ms"]["corrected"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16", "data": "synthetic",
        "config": {"workload": f"learned64: water72192 ({n} sites, cubic {L} A) on a 64^3 mesh, order 5, beta 0.4/A, "
                               f"plus the learned correction (the line's value: the stated feature set, 27 "
                               f"potential samples + site type); labels from the 160^3 FP32 PPPM",
                   "train_frames": len(spec.base_seeds) * fpb, "train_bases": nbase, "frame_sigma_A": 0.05,
                   "held_out": f"2 other base configurations (seeds 200, 201) x {args.held_frames} frames",
                   "l2": "flushed between timed steps",
                   "launch": "every timed call (corrected and plain) is a replay of one CUDA graph of the call"},
        "modes": modes,
        "ms_plain": {f"plain_{m}": v for m, v in ms_plain.items()},
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------- long/short-range overlap
class ShortRangeStandIn:
    """A stand-in for the short-range model's per-atom cost: the fitting-net
    shape of the paper's DP model (three hidden layers of 240, tanh) applied
    to a synthetic 128-wide descriptor per atom, in BF16 through torch's
    cuBLAS matmuls.  It is load, not part of the method: its only role is to
    occupy the GPU the way short-range inference would."""

    def __init__(self, n_atoms, device, seed=17, width=240, d_in=128):
        import torch
        g = torch.Generator(device=device)
        g.manual_seed(seed)
        self.x = torch.randn((n_atoms, d_in), generator=g, device=device).to(torch.bfloat16)
        dims = [d_in, width, width, width, 1]
        self.w = [(torch.randn((dims[i], dims[i + 1]), generator=g, device=device) / dims[i] ** 0.5)
                  .to(torch.bfloat16) for i in range(4)]
        self.flops = 2 * n_atoms * sum(dims[i] * dims[i + 1] for i in range(4))
        self.out = None

    def __call__(self):
        import torch
        h = self.x
        for w in self.w[:-1]:
            h = torch.tanh(h @ w)
        self.out = h @ self.w[-1]
        return self.out


def run_overlap(args):
    """The 128^3 force evaluation (one captured graph) and the short-range
    stand-in, alone, back to back on one stream, and concurrently on two
    streams (long range at high or at equal priority; PPPM kernels with and
    without programmatic dependent launch), as in the paper's overlap of long-
    and short-range forces (Section "Long-range and Short-range Force
    Overlap")."""
    import torch

    from paper_2504_15508_gb300.pppm import Plan
    from workloads.water import make_workload

    dev = torch.device("cuda", 0)
    wb, w = make_workload("water72192_m128")
    n = wb.n
    pos = torch.tensor(wb.pos, dtype=torch.float32, device=dev)
    q = torch.tensor(wb.q, dtype=torch.float32, device=dev)
    plan = Plan(wb.box, w["mesh"], w["order"], w["beta"], precision="fp32")
    plan.reserve(n)
    lo = torch.cuda.Stream(device=dev, priority=0)
    hi = torch.cuda.Stream(device=dev, priority=-1)
    lo2 = torch.cuda.Stream(device=dev, priority=0)
    sr = ShortRangeStandIn(3 * wb.n_mol, dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    main = torch.cuda.current_stream()
    K = args.steps

    def timed(body):
        for k in range(max(3, args.warmup)):
            body()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        for k in range(K):
            flush.fill_(float(k))
            evs[k][0].record(main)
            body()
            evs[k][1].record(main)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs) / K

    def concurrent(g, lr_stream, sr_stream):
        def body():
            start = torch.cuda.Event()
            start.record(main)
            lr_stream.wait_event(start)
            sr_stream.wait_event(start)
            g.launch(pos, q, stream=lr_stream)
            with torch.cuda.stream(sr_stream):
                sr()
            done_lr, done_sr = torch.cuda.Event(), torch.cuda.Event()
            done_lr.record(lr_stream)
            done_sr.record(sr_stream)
            main.wait_event(done_lr)
            main.wait_event(done_sr)
        return body

    t_sr = timed(lambda: sr())
    # with and without programmatic dependent launch between the PPPM kernels:
    # its early-scheduled blocks hold SM resources the concurrent work could use
    runs = {}
    f_ref = None
    same = True
    for pdl in (True, False):
        plan.set_dependent_launch(pdl)
        g = plan.graph(pos, q)
        r = {"long_range_alone": timed(lambda: g.launch(pos, q, stream=main))}

        def sequential():
            g.launch(pos, q, stream=main)
            sr()

        r["sequential"] = timed(sequential)
        r["concurrent"] = timed(concurrent(g, hi, lo))  # long range on the high-priority stream
        r["concurrent_equal_priority"] = timed(concurrent(g, lo2, lo))
        # results under overlap are those of the step alone, with either launch mode
        g.launch(pos, q, stream=main)
        torch.cuda.synchronize()
        if f_ref is None:
            f_ref = g.out[1].clone()
        same = same and bool(torch.equal(g.out[1], f_ref))
        g.close()
        runs["dependent_launch_on" if pdl else "dependent_launch_off"] = r
    plan.set_dependent_launch(True)
    # the headline: the best concurrent configuration, against the best back-to-back one
    best_key, best_mode = min(((m, k) for k in runs for m in ("concurrent", "concurrent_equal_priority")),
                              key=lambda mk: runs[mk[1]][mk[0]])
    t_par = runs[best_mode][best_key]
    t_seq = min(r["sequential"] for r in runs.values())
    t_lr = min(r["long_range_alone"] for r in runs.values())
    line = {
        "metric": "long-range step concurrent with a short-range load", "value": 1e3 / t_par,
        "unit": "steps/s", "n_gpus": 1, "steps": K, "warmup": args.warmup, "ms_per_step": t_par,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16", "data": "synthetic",
        "config": {"workload": f"overlap: water72192 ({n} sites) PPPM on 128^3 (captured graph) with a "
                               f"{3 * wb.n_mol}-atom 128-240-240-240-1 BF16 MLP stand-in "
                               f"({sr.flops / 1e9:.1f} GFLOP) on a second stream",
                   "best": {"streams": "long range at high priority" if best_key == "concurrent"
                            else "equal priorities", "pppm_launch": best_mode},
                   "l2": "flushed between timed steps"},
        "ms": {"short_range_alone": t_sr, **{k: v for k, v in runs.items()}},
        "speedup_vs_sequential": t_seq / t_par,
        "hidden_fraction_of_shorter": (t_lr + t_sr - t_par) / min(t_lr, t_sr),
        "short_range_tflops_alone": sr.flops / (t_sr * 1e-3) / 1e12,
        "pppm_results_unchanged": same,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "ours" and args.workload == "overlap":
        run_overlap(args)
        return
    if args.impl == "ours" and args.workload == "batched96":
        run_batched(args)
        return
    if args.impl == "ours" and args.workload == "learned64":
        if args.forward_only:
            run_forward(args)
        else:
            run_learned(args)
        return
    if args.impl == "reference":
        if int(os.environ.get("RANK", "0")) == 0:
            run_reference(args)
        return
    run_ours(args)


if __name__ == "__main__":
    main()
