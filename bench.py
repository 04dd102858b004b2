"""Throughput of the cryoSplat splatting path on B300: fwd+bwd particle images/s.

Workload (default): D = 256 pixels, N = 100,000 Gaussians, a batch of 128 particles with
their own poses and defocus (the D = 256 / N = 100k volume of the mixed-batch
configuration), seeded synthetic inputs shaped like the paper's data.  One step =
project -> bin/sort -> render -> CTF -> loss -> CTF adjoint -> render backward -> Adam over
the whole batch.

Printed (rank 0, one JSON line): the batched, fused form's images/s as ``value``; the plain
form (one particle per launch sequence, batch size 1 as in the paper) on the same GPU; an
end-to-end figure through the public API with host buffers; the roofline of the dominant
kernel against the SFU ex2 peak; the FP64 oracle timed on the host cores as a CPU
baseline; SM clocks sampled during the timed region.

``--impl reference`` times the FP64 oracle itself on the host cores (the slow reference
arm), on the same config and metric.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2508_04929_b300 import synth  # noqa: E402

METRIC = "fwd+bwd particle images/s at D=256,N=100k vs plain form; % of SFU-exp roofline"
UNIT = "images/s"
SM_MAX_MHZ = 2032.0
CTF_SNR = 0.05
# DRAM bytes (ncu dram__bytes_read.sum + dram__bytes_write.sum) per tile pair of one launch of
# each render kernel, from the capture summarised in profiles/render_kernels_d256_n100k_b64.md
# (B = 64; the kernels read each pair's index and record once, so traffic scales with the pair
# count).  Valid only for the gs_render.cu whose SHA-256 is recorded: otherwise null.
RENDER_TRAFFIC = {"sha256": "1744410d1f3913910f5752efe7e142735fa7b1a6823497ea13f3f1da30fb616d",
                  "bytes_per_pair": {"fwd": (306.636544e6 + 16.469504e6) / 25319264,
                                     "bwd": (320.559616e6 + 3.130112e6) / 25319264}}


# libgs kernels launched by one graph-captured training step (cuFFT's and torch's gradient
# zeroing are library kernels and not counted)
def step_kernels(D, tile):
    """The library's kernels that one graph-captured training step launches, once each (cuFFT's
    2-D transforms at sizes other than 256 and torch's zeroing of the gradient are not ours)."""
    r = "8" if tile == 8 else "16"  # tiles 16 and 32 share the region kernels
    ctf = ("k_rows_r2c2", "k_ctf_cols", "k_rows_c2r") if D == 256 else ("k_ctf_loss",)
    return ("k_activate", "k_project", "k_bin_count", "k_bin_scan", "k_bin_tiles", "k_bin_base", "k_bin_scatter",
            "k_render_fwd" + r, *ctf, "k_render_bwd" + r, "k_bwd_finalize", "k_adam", "k_count_step")


class _NoDist:
    """Single-process stand-in for torch.distributed in the dry run."""

    @staticmethod
    def all_reduce(t):
        return t


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--D", type=int, default=256)
    p.add_argument("--N", type=int, default=100_000)
    p.add_argument("--B", type=int, default=128)
    p.add_argument("--tile", type=int, default=0, help="0 = autotune")
    p.add_argument("--chunk", type=int, default=0, help="0 = autotune")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--mixed", type=int, default=1, help="also time the mixed-size batch (1/0)")
    p.add_argument("--cpu-sample", type=int, default=0, help="images in the CPU sample (0 = one per core, max 16)")
    p.add_argument("--dp", action="store_true",
                   help="time the data-parallel training step (all-reduce of dL/dTheta before Adam); the default "
                        "when several ranks run")
    p.add_argument("--replicas", action="store_true",
                   help="with several ranks, time independent replicas (no collective) instead of the "
                        "data-parallel step")
    p.add_argument("--dry-run", action="store_true",
                   help="exercise only the rank launch, the collective and the JSON line on the host (gloo, "
                        "no GPU work); the line carries no measurement")
    p.add_argument("--no-config2", action="store_true", help="skip the D=128, N=20k, B=64 batched-vs-plain line")
    return p.parse_args()


def spawn_ranks(args):
    """bench.py --gpus N (N > 1) started without a launcher: re-run it as N ranks under
    torch.distributed.run on this node (127.0.0.1, a free port) and return the exit code."""
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
           "--master-addr=127.0.0.1", f"--master-port={port}", os.path.abspath(__file__), *sys.argv[1:]]
    return subprocess.call(cmd)


def run_dry(args, rank, world, dist):
    """The multi-rank plumbing without GPU work: each rank 'renders' its own particles (a host
    array standing in for its part of dL/dTheta), the ranks all-reduce it as the data-parallel
    step does, and rank 0 prints the JSON line with no measured value."""
    import torch
    g = torch.full((args.N, 11), float(rank + 1), dtype=torch.float32)
    dist.all_reduce(g)
    expect = world * (world + 1) / 2
    ok = bool(torch.all(g == expect))
    if rank == 0:
        par = "replicas" if args.replicas else "dp"
        print(json.dumps({"metric": METRIC, "value": None, "unit": UNIT, "n_gpus": world, "steps": 0,
                          "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f32", "data": "dry run: no GPU work, nothing measured",
                          "config": dict(workload(args), parallelism=par), "dry_run": {"allreduce_ok": ok}}),
              flush=True)


def workload(args):
    return {"workload": f"D={args.D},N={args.N},B={args.B} synthetic particles (uniform-ball centres, "
                        f"log-uniform 0.5-3 px scales, random rotations/poses, defocus 1-3 um)",
            "D": args.D, "N": args.N, "batch": args.B, "seed": 0,
            "l2": "inputs larger than L2 (records and gradient partials ~0.8 GB per step)"}


def render_traffic(kind, pairs):
    """DRAM bytes of one render launch over ``pairs`` tile pairs, or None when the kernel
    source differs from the profiled one."""
    import hashlib
    src = os.path.join(ROOT, "paper_2508_04929_b300", "csrc", "gs_render.cu")
    try:
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    per = RENDER_TRAFFIC["bytes_per_pair"].get(kind)
    if RENDER_TRAFFIC["sha256"] != sha or per is None:
        return None
    return per * pairs


def max_over_ranks(x, dist=None, device="cpu"):
    """The maximum of x over all ranks (x itself without a process group): the job's time
    is that of its slowest rank."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measure_h2d(torch, host, dev, reps=5):
    """Pinned host -> device bandwidth of this machine (GB/s) for one step's images, copied in four
    chunks on four streams as the feeders do; the end-to-end rate cannot exceed B images per
    step's copy time."""
    streams = [torch.cuda.Stream() for _ in range(4)]
    cur = torch.cuda.current_stream()

    def once():
        for s, d, h in zip(streams, dev.chunk(4), host.chunk(4)):
            s.wait_stream(cur)
            with torch.cuda.stream(s):
                d.copy_(h, non_blocking=True)
        for s in streams:
            cur.wait_stream(s)

    once()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        once()
    e1.record()
    torch.cuda.synchronize()
    return reps * host.numel() * host.element_size() / (e0.elapsed_time(e1) * 1e-3) / 1e9


def measure_ex2_peak(torch, L, reps=5):
    """ex2.approx throughput of this GPU (ex2/s), measured with the library's probe
    (gs_probe_ex2: 8 independent ex2 chains per thread, 8 CTAs of 256 threads per SM): the
    SFU-exp peak that the render kernels' roofline is quoted against."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    sink = torch.zeros(1, dtype=torch.float32, device="cuda")
    blocks, iters = 8 * sms, 4096
    L.gs_probe_ex2(blocks, iters, sink)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    cnt = 0.0
    for _ in range(reps):
        cnt += L.gs_probe_ex2(blocks, iters, sink)
    e1.record()
    torch.cuda.synchronize()
    return cnt / (e0.elapsed_time(e1) * 1e-3), sms


def make_inputs(args, seed=0):
    rng = synth.rng_for(seed)
    th = synth.random_gaussians(args.N, args.D, rng)
    Ws = synth.random_poses(args.B, rng).reshape(args.B, 9)
    ctf = synth.random_ctf(args.B, rng)
    th_gt = synth.random_gaussians(args.N, args.D, rng)
    return th, Ws, ctf, th_gt, rng


# ---------------------------------------------------------------------------------------
# CPU baseline: the FP64 oracle, one particle per process (spawned before CUDA starts)
# ---------------------------------------------------------------------------------------
def _oracle_image(payload):
    import oracle as O
    th, W, ctf_row, Y, D = payload
    t0 = time.perf_counter()
    O.forward_backward(th, W[None].reshape(1, 3, 3), D, Y[None], ctf_row[None])
    return time.perf_counter() - t0


def start_cpu_pool(n):
    import concurrent.futures as cf
    import multiprocessing as mp
    return cf.ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn"))


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_cpu_sample(pool, th, Ws, ctf, Y, D, n):
    payloads = [(th, Ws[b], ctf[b], Y[b], D) for b in range(n)]
    t0 = time.perf_counter()
    per = list(pool.map(_oracle_image, payloads))
    wall = time.perf_counter() - t0
    return wall, per


# ---------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            time.sleep(0.25)
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        sm, mx, reasons = [], SM_MAX_MHZ, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------------------
# the plain form: one particle per launch sequence (batch size 1, as in the paper), Adam per image
# ---------------------------------------------------------------------------------------
def best_plain(plain):
    """The faster of the plain form's two measured variants (None if neither has a number): the
    speedups divide by it, so that the baseline is the best the per-image form achieved."""
    vals = [v for v in (plain or {}).values() if v]
    return max(vals) if vals else None


def run_plain(args, L, torch, Splatter, t, W, C, Y, tile, chunk, dev, pairs_hint, nimg=None):
    """Images/s of the plain per-image form, two ways: with the pair buffer sized up front
    from the batch's mean pair count (x 2, no host sync per image), and with the buffer grown
    on demand (gs_bin_sort's count read back to the host after every image)."""
    nimg = min(args.B if nimg is None else nimg, 64)
    out = {}
    # each form twice, alternating, best of the two: the launch-bound plain form is sensitive to
    # whatever else the host is doing
    for name, grow in (("presized", False), ("grow_sync", True), ("presized", False), ("grow_sync", True)):
        p1 = Splatter(Y.shape[-1], t.shape[0], 1, tile=tile, chunk=chunk, device=dev,
                      pair_capacity=None if grow else 2 * pairs_hint + 4096)
        th1 = t.clone()
        m1, v1, g1 = torch.zeros_like(t), torch.zeros_like(t), torch.zeros_like(t)
        for b in range(2):
            g1.zero_()
            p1.forward_backward(th1, W[b:b + 1], C[b:b + 1], Y[b:b + 1], g1, grow=grow, fused=True)
        torch.cuda.synchronize()
        s0 = time.perf_counter()
        for b in range(nimg):
            g1.zero_()
            p1.forward_backward(th1, W[b:b + 1], C[b:b + 1], Y[b:b + 1], g1, grow=grow, fused=True)
            L.gs_step(th1, g1, m1, v1, b + 1)
        torch.cuda.synchronize()
        rate = nimg / (time.perf_counter() - s0)
        status = p1.status()
        p1.close()
        if not grow and status & L.GS_STATUS_OVERFLOW:
            rate = None  # the pre-sized buffer was too small: no valid number
        if rate is None or out.get(name, 0.0) is None:
            out[name] = None
        else:
            out[name] = max(out.get(name, 0.0), rate)
    return out


# ---------------------------------------------------------------------------------------
# the batched step against the plain form at D = 128, N = 20k, B = 64
# ---------------------------------------------------------------------------------------
def run_config2(args, L, torch, Splatter, dev, steps=10):
    """The D = 128, N = 20,000, B = 64 configuration: the graph-captured batched step (tile and
    chunk autotuned) against the plain per-image form on the same GPU."""
    from paper_2508_04929_b300 import autotune
    from paper_2508_04929_b300.batched import GraphStep, Problem
    D, N, B = 128, 20_000, 64
    rng = synth.rng_for(7)
    t = torch.from_numpy(synth.random_gaussians(N, D, rng)).to(dev)
    W = torch.from_numpy(synth.random_poses(B, rng).reshape(B, 9)).to(dev)
    C = torch.from_numpy(synth.random_ctf(B, rng)).to(dev)
    tg = torch.from_numpy(synth.random_gaussians(N, D, rng)).to(dev)
    gt = Splatter(D, N, B, tile=16, chunk=128, device=dev)
    _, X = gt.forward(tg, W, C)
    sig = math.sqrt(float(X.double().var()) / 0.1)
    gen = torch.Generator(device=dev).manual_seed(77)
    Y = (X + sig * torch.randn(X.shape, device=dev, generator=gen)).contiguous()
    gt.close()
    tune = autotune.tune(D, N, B, t, W, C, Y, device=dev, tiles=(8, 16, 32), chunks=(64, 128))
    prob = Problem(D=D, theta=t.clone(), W=W, ctf=C, Y=Y, tile=tune["tile"], chunk=tune["chunk"])
    gs = GraphStep([prob], adam=True)
    for _ in range(3):
        gs.replay()
    torch.cuda.synchronize()
    st = gs.check()
    n_pairs = int(prob.sp.n_pairs.item()) & 0xFFFFFFFF
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        gs.replay()
    e1.record()
    torch.cuda.synchronize()
    st |= gs.check()
    ms = e0.elapsed_time(e1) / steps
    gs.close()

    class _A:  # the plain form's arguments at this size
        pass
    a = _A()
    a.B = B
    plain = run_plain(a, L, torch, Splatter, t, W, C, Y, tune["tile"], tune["chunk"], dev,
                      pairs_hint=n_pairs // B)
    batched = B / (ms * 1e-3)
    return {"workload": f"D={D},N={N},B={B} synthetic particles, SNR 0.1", "tile": tune["tile"],
            "chunk": tune["chunk"], "batched": batched, "batched_ms_per_step": ms, "plain": plain,
            "speedup_vs_plain": batched / best_plain(plain) if best_plain(plain) else None,
            "status": st, "unit": UNIT}


# ---------------------------------------------------------------------------------------
# mixed-size batch: 4 volumes (N = 10k/30k/60k/100k at D = 96/128/192/256), 128 particles
# each, SNR 0.05, one CUDA graph; tile size and chunk depth autotuned per volume
# ---------------------------------------------------------------------------------------
MIXED = ((96, 10_000), (128, 30_000), (192, 60_000), (256, 100_000))


def run_mixed(args, dev, torch, B=128, steps=10):
    from paper_2508_04929_b300.batched import GraphStep, Problem
    from paper_2508_04929_b300.splat import Splatter
    probs = []
    for i, (D, N) in enumerate(MIXED):
        rng = synth.rng_for(100 + i)
        th = torch.from_numpy(synth.random_gaussians(N, D, rng)).to(dev)
        W = torch.from_numpy(synth.random_poses(B, rng).reshape(B, 9)).to(dev)
        C = torch.from_numpy(synth.random_ctf(B, rng)).to(dev)
        tg = torch.from_numpy(synth.random_gaussians(N, D, rng)).to(dev)
        gt = Splatter(D, N, B, tile=16, chunk=128, device=dev)
        _, X = gt.forward(tg, W, C)
        sig = math.sqrt(float(X.double().var()) / CTF_SNR)
        gen = torch.Generator(device=dev).manual_seed(4321 + i)
        Y = (X + sig * torch.randn(X.shape, device=dev, generator=gen)).contiguous()
        gt.close()
        probs.append(Problem(D=D, theta=th, W=W, ctf=C, Y=Y))
    gs = GraphStep(probs, adam=True, autotune_chunks=(64, 128))
    for _ in range(3):
        gs.replay()
    torch.cuda.synchronize()
    st = gs.check()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        gs.replay()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    out = {"workload": "4 volumes N=10k/30k/60k/100k at D=96/128/192/256, 128 particles each, one CUDA graph",
           "value": 4 * B / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "status": st,
           "launch_shapes": [{"D": p.D, "N": p.N, "tile": p.tile, "chunk": p.chunk} for p in gs.problems]}
    gs.close()
    return out


# ---------------------------------------------------------------------------------------
# evaluation: GMM voxelization (D^3) and FSC against the ground truth
# ---------------------------------------------------------------------------------------
def run_evaluation(args, dev, torch, theta, theta_gt, reps=5):
    from paper_2508_04929_b300 import volume
    D = args.D
    for _ in range(2):
        v1 = volume.voxelize(theta, D)
        v2 = volume.voxelize(theta_gt, D)
        curve = volume.fsc(v1, v2)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    tv, tf = [], []
    for _ in range(reps):
        e[0].record()
        v1 = volume.voxelize(theta, D)
        e[1].record()
        curve = volume.fsc(v1, v2)
        e[2].record()
        torch.cuda.synchronize()
        tv.append(e[0].elapsed_time(e[1]))
        tf.append(e[1].elapsed_time(e[2]))
    # voxel evaluations: the per-axis 3-sigma boxes of the Gaussians (FP32, as in the kernel)
    import numpy as np
    from paper_2508_04929_b300 import synth as _s  # noqa: F401
    th = theta.detach().cpu().numpy().astype(np.float64)
    s = np.log1p(np.exp(th[:, 3:6]))
    q = th[:, 6:10] / np.linalg.norm(th[:, 6:10], axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.stack([np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
                  np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
                  np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], -2)
    half = 3.0 * np.sqrt(np.einsum("nam,nm->na", R * R, s * s)) * D
    evals = float(np.prod(np.floor(2 * half) + 1, axis=1).sum())
    tv_m, tf_m = statistics.median(tv), statistics.median(tf)
    return {"workload": f"voxelize N={theta.shape[0]} Gaussians on {D}^3, FSC of two {D}^3 volumes",
            "voxelize_ms": tv_m, "fsc_ms": tf_m, "voxel_evals": evals,
            "voxel_evals_per_s": evals / (tv_m * 1e-3),
            "fsc_vs_ground_truth_shells_1_4_16_64": [float(curve[i]) for i in (1, 4, 16, 64) if i < curve.numel()]}


# ---------------------------------------------------------------------------------------
# the reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------------------
def run_reference(args, rank):
    if rank != 0:
        return
    th, Ws, ctf, th_gt, rng = make_inputs(args)
    Y = synth.smooth_field(args.B, args.D, rng, scale=1.0)  # stand-in observed images (cost is data independent)
    cores = cpu_cores()
    n = args.cpu_sample or min(cores, 16)
    pool = start_cpu_pool(min(n, cores))
    for _ in range(args.warmup if args.warmup < 1 else 1):
        run_cpu_sample(pool, th, Ws, ctf, Y, args.D, min(n, args.B))
    times = []
    for _ in range(args.steps):
        wall, _ = run_cpu_sample(pool, th, Ws, ctf, Y, args.D, min(n, args.B))
        times.append(wall)
    pool.shutdown()
    tot = sum(times)
    imgs = min(n, args.B) * args.steps
    v = imgs / tot
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload(args),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": min(n, cores), "kind": "oracle",
                             "sample": f"{min(n, args.B)} of the {args.B} particles per step, one per process"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------
def main():
    args = parse()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(spawn_ranks(args))
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.dry_run:
        import torch.distributed as dist
        if world > 1:
            dist.init_process_group("gloo")
        run_dry(args, rank, world, dist if world > 1 else _NoDist())
        if world > 1:
            dist.destroy_process_group()
        return
    # several ranks train one model by default: one all-reduce of dL/dTheta per step (DataParallelStep)
    args.dp = args.dp or (world > 1 and not args.replicas)
    cores = cpu_cores()
    want_cpu = rank == 0 and world == 1 and not args.no_cpu_baseline
    n_cpu = args.cpu_sample or min(cores, 16)
    pool = start_cpu_pool(min(n_cpu, cores)) if want_cpu else None  # before the first CUDA call

    import torch
    from paper_2508_04929_b300 import build
    build.build()
    from paper_2508_04929_b300 import _lib as L
    from paper_2508_04929_b300.splat import Splatter
    from paper_2508_04929_b300 import autotune

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)

    th, Ws, ctf, th_gt, rng = make_inputs(args, seed=rank)
    t = torch.from_numpy(th).to(dev)
    W = torch.from_numpy(Ws).to(dev)
    C = torch.from_numpy(ctf).to(dev)

    # observed images: clean CTF images of a ground-truth GMM (rendered by this path) + noise
    gt = Splatter(args.D, args.N, args.B, tile=16, chunk=128, device=dev)
    tg = torch.from_numpy(th_gt).to(dev)
    _, Xgt = gt.forward(tg, W, C)
    sig = math.sqrt(float(Xgt.double().var()) / CTF_SNR)
    gen = torch.Generator(device=dev).manual_seed(1234 + rank)
    Y = (Xgt + sig * torch.randn(Xgt.shape, device=dev, generator=gen)).contiguous()
    gt.close()
    del gt, tg, Xgt

    tile, chunk = args.tile, args.chunk
    tune = None
    if tile == 0 or chunk == 0:
        tune = autotune.tune(args.D, args.N, args.B, t, W, C, Y, device=dev,
                             tiles=(tile,) if tile else (8, 16, 32), chunks=(chunk,) if chunk else (64, 128, 256))
        tile, chunk = tune["tile"], tune["chunk"]

    # --- batched, fused form: the whole step as one CUDA graph (autotuned launch shape) ---
    from paper_2508_04929_b300.batched import GraphStep, Problem
    prob = Problem(D=args.D, theta=t.clone(), W=W.clone(), ctf=C.clone(), Y=Y, tile=tile, chunk=chunk)
    gs = GraphStep([prob], adam=not args.dp)
    sp = prob.sp
    stream = torch.cuda.current_stream()
    step = gs.replay
    if args.dp:  # replicated Theta, one all-reduce of dL/dTheta per step, replicated Adam
        from paper_2508_04929_b300 import distributed as DPm
        dps = DPm.DataParallelStep(prob.theta, *DPm.graph_step_parts(gs))
        step = dps
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    st = gs.check()
    # algorithmic work: Gaussian-pixel evaluations inside the support boxes of this batch
    box = sp.proj[: args.B * args.N * 32].view(torch.int16).view(args.B, args.N, 16)[:, :, 12:16].to(torch.int64)
    area = ((box[..., 1] - box[..., 0] + 1).clamp(min=0) * (box[..., 3] - box[..., 2] + 1).clamp(min=0))
    e_alg = int(area.sum())
    n_pairs = int(sp.n_pairs.item()) & 0xFFFFFFFF

    # the timed steps, the per-kernel timings and the end-to-end steps all start from this state
    # (Adam moves Theta, and with it the number of tile pairs, from step to step)
    snap = [x.clone() for x in (prob.theta, prob.m, prob.v, prob.t)]

    def restore():
        for x, y in zip((prob.theta, prob.m, prob.v, prob.t), snap):
            x.copy_(y)

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms_total = e0.elapsed_time(e1)
        st_timed = gs.check()  # an overflow inside the timed steps would have dropped pairs
        restore()
        # the same kernels once more, eagerly, with CUDA events around the two render calls
        ev = {k: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for k in ("proj", "bin", "fwd", "bwd", "fft")}
        kt = {k: [] for k in ev}
        dth = torch.zeros_like(t)
        for _ in range(min(args.steps, 5)):
            dth.zero_()
            torch.cuda._sleep(2_000_000)  # keeps the GPU busy while the host queues the parts below
            ev["proj"][0].record(stream)
            sp.project(prob.theta, W)
            ev["proj"][1].record(stream)
            ev["bin"][0].record(stream)
            sp.bin_sort(grow=False)
            ev["bin"][1].record(stream)
            ev["fwd"][0].record(stream)
            sp.render()
            ev["fwd"][1].record(stream)
            ev["fft"][0].record(stream)
            sp.ctf_loss_grad(sp.Q, C, Y)
            ev["fft"][1].record(stream)
            ev["bwd"][0].record(stream)
            sp.backward(prob.theta, W, sp.dQ, dth)
            ev["bwd"][1].record(stream)
            torch.cuda.synchronize()
            for k in kt:
                kt[k].append(ev[k][0].elapsed_time(ev[k][1]))
    ms_total = max_over_ranks(ms_total, dist, dev)
    ms_step = ms_total / args.steps
    value = world * args.B / (ms_step * 1e-3)
    t_fwd = statistics.median(kt["fwd"])
    t_bwd = statistics.median(kt["bwd"])
    t_ctf = statistics.median(kt["fft"])
    t_proj = statistics.median(kt["proj"])
    t_bin = statistics.median(kt["bin"])

    # --- plain form: one particle per launch sequence, batch size 1, Adam per image ---
    plain = None
    if not args.no_plain:
        plain = run_plain(args, L, torch, Splatter, t, W, C, Y, tile, chunk, dev,
                          pairs_hint=n_pairs // max(args.B, 1))

    # --- end to end through the public API with host buffers: copy in, replay, loss out ---
    Yh = Y.cpu().pin_memory()
    Wh = W.cpu().pin_memory()
    Ch = C.cpu().pin_memory()
    # Each step's inputs are copied from pinned host memory into one of three input slots of the
    # graph-captured step while earlier steps run, and the step replays that slot's graphs: the
    # front half (projection, binning, render) waits only for the poses, so on the first step it
    # starts while the images are still being copied in.  Each step's losses come back to pinned
    # host memory; the host reads them two steps later, after enqueueing the steps in between, so
    # that neither a slow host nor a late copy leaves the GPU waiting.  (The data-parallel step is
    # fed through the static buffers, one step behind.)
    depth = 1 if args.dp else 2  # steps the host runs ahead of the losses it reads
    lossh = [torch.empty(args.B, dtype=torch.float32).pin_memory() for _ in range(depth + 1)]
    h2d = Yh.numel() * 4 + Wh.numel() * 4 + Ch.numel() * 4
    d2h = lossh[0].numel() * 4
    from paper_2508_04929_b300.batched import HostFeeder, SlotFeeder
    if not args.dp:
        gs.record_slots(depth + 1)
    feeder = HostFeeder(gs) if args.dp else SlotFeeder(gs)
    if not args.dp:  # two untimed fed steps: the slot graphs' first launches are not part of the rate
        for _ in range(2):
            feeder.prefetch(Wh, Ch, Yh)
            feeder.step()
        torch.cuda.synchronize()
    restore()
    done = [torch.cuda.Event() for _ in range(depth + 1)]
    host_losses = 0.0
    torch.cuda.synchronize()
    s0 = time.perf_counter()
    ahead = 1 if args.dp else min(depth, args.steps)  # steps whose inputs are in flight before the first replay
    for _ in range(ahead):
        feeder.prefetch(Wh, Ch, Yh)
    read = 0
    for i in range(args.steps):
        if args.dp:
            feeder.load()
        if i + ahead < args.steps:
            feeder.prefetch(Wh, Ch, Yh)
        if args.dp:
            step()
        else:
            feeder.step()
        lossh[i % (depth + 1)].copy_(prob.sp.loss[: args.B], non_blocking=True)
        done[i % (depth + 1)].record()
        if i - read >= depth:  # the host reads the losses of the step `depth` steps back
            done[read % (depth + 1)].synchronize()
            host_losses += float(lossh[read % (depth + 1)].sum())
            read += 1
    while read < args.steps:
        done[read % (depth + 1)].synchronize()
        host_losses += float(lossh[read % (depth + 1)].sum())
        read += 1
    e2e = world * args.B * args.steps / (time.perf_counter() - s0)
    st_e2e = gs.check()
    h2d_gbps = measure_h2d(torch, Yh, prob.Y)
    torch.cuda.synchronize()
    gs.close()

    # --- evaluation: voxelize the fitted and ground-truth GMMs (D^3) and their FSC ---
    evaluation = run_evaluation(args, dev, torch, prob.theta, torch.from_numpy(th_gt).to(dev))

    # --- mixed batch: four volumes of different D and N in one graph (autotuned each) ---
    mixed = None
    if args.mixed:
        mixed = run_mixed(args, dev, torch)

    # --- the D = 128, N = 20k, B = 64 configuration: batched step against the plain form ---
    config2 = None
    if not args.no_config2 and not args.no_plain and rank == 0:
        config2 = run_config2(args, L, torch, Splatter, dev)

    # --- the SFU-exp peak of this GPU, measured by the library's ex2 probe ---
    peak_exp, sms = measure_ex2_peak(torch, L)

    cpu = None
    if pool is not None:
        Ynp = Y.cpu().numpy()
        n = min(n_cpu, args.B)
        wall, per = run_cpu_sample(pool, th, Ws, ctf, Ynp, args.D, n)
        pool.shutdown()
        cpu = {"value": n / wall, "unit": UNIT, "cores": min(n_cpu, cores), "kind": "oracle",
               "sample": f"{n} of the {args.B} particles (same inputs), one particle per process, "
                         f"median {statistics.median(per):.1f} s per particle"}

    dom = "bwd" if t_bwd >= t_fwd else "fwd"
    t_dom = max(t_bwd, t_fwd)
    achieved = e_alg / (t_dom * 1e-3)
    clocks = clk.summary()
    mhz = clocks["sm_mhz"] or SM_MAX_MHZ
    ex2_per_clk = peak_exp / (sms * mhz * 1e6)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(workload(args), tile=tile, chunk=chunk,
                           parallelism=("dp" if args.dp else "replicas") if world > 1 else ("dp1" if args.dp else "single")),
            "plain_form": None if plain is None else {
                "value": best_plain(plain), "presized": plain["presized"], "value_with_host_sync": plain["grow_sync"],
                "unit": UNIT,
                "form": "one particle per launch sequence, Adam per image; presized: pair buffer sized up front "
                        "(no host sync per image); value_with_host_sync: pair count read back after every image; "
                        "value: the faster of the two"},
            "speedup_vs_plain": (value / world / best_plain(plain)) if plain and best_plain(plain) else None,
            "config2": config2,
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "h2d_GBps": h2d_gbps, "h2d_bound": world * args.B / (h2d / (h2d_gbps * 1e9)),
                    "pipelining": "each step's host->device copy (into one of three input slots of the captured step) runs while earlier steps do; a step's render starts before its images have arrived; every step's losses are copied back and read by the host two steps later"},
            "gpu_launches": len(step_kernels(args.D, tile)) * args.steps,
            "roofline": {"bound": "alu", "kernel": f"k_render_{dom}", "achieved": achieved / 1e9,
                         "peak": peak_exp / 1e9, "unit": "Gex2/s", "frac": achieved / peak_exp,
                         "traffic": render_traffic(dom, n_pairs),
                         "peak_source": f"measured on this GPU by gs_probe_ex2: {ex2_per_clk:.2f} ex2/clk/SM x {sms} SMs "
                                        f"at {mhz:.0f} MHz"},
            "fwd_bwd_splat": {"ms_project": t_proj, "ms_bin_sort": t_bin, "ms_fwd": t_fwd, "ms_bwd": t_bwd,
                              "ms_ctf_loss_adjoint": t_ctf, "alg_evals_per_step": e_alg,
                              "pairs_per_step": n_pairs,
                              "frac_of_sfu_roofline": (2 * e_alg / ((t_fwd + t_bwd) * 1e-3)) / peak_exp},
            "cpu_baseline": cpu, "clocks": clocks,
            "status": st | st_timed | st_e2e,
            "status_read": "after the warm-up, after the timed steps and after the end-to-end steps",
            "autotune": tune,
            "mixed_batch": mixed,
            "evaluation": evaluation,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
