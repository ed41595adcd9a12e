#!/usr/bin/env python3
"""Benchmark of the dual-quaternion Julia isosurface renderer on GB300.

Workload (one step): the five seeded 1920x1080 frames (c ~ U[-0.8,0.8]^8 with
numpy default_rng(seed), seeds 0..4), max_iter 16, 512 march steps, 10 bisection
steps, central-difference normals (h = 1e-4), ambient+diffuse shading to RGBA8,
FP32 throughout.  Inputs (parameter blocks) and output planes (24 B/pixel) stay
resident on the device; a 256 MiB buffer is written between steps to flush L2.

Metric: DQ iterations/s (algorithmic iterations: escape count, or max_iter for an
inside sample, plus the n* steps of each normal evaluation, counted by the
kernels) with frames/s beside it; roofline of the march kernel against the FP32
FMA peak (152 SMs x 128 lanes x 2 flop x 2070 MHz), 52 flops per DQ iteration.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl dqj|reference]

With --impl reference the FP64 CPU oracle is timed on the host cores on a bounded
pixel sample of the same frames (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DQ iterations/s and 1080p frames/s (fraction of FP32 FMA peak); served p50/p99 latency"
UNIT = "DQ iterations/s"
SEEDS = (0, 1, 2, 3, 4)
FLOPS_PER_ITER = 52          # specialised square + c + EUCLID8 modulus test, FMA = 2 flops
SM_MAX_MHZ = 2070.0
FP32_LANES_PER_SM = 128
WORKLOAD = "dq-julia 1920x1080, c~U[-0.8,0.8]^8 seeds 0-4, max_iter 16, 512 march + 10 bisect, FP32"
KERNEL_SOURCES = ("paper_2303_14827_gb300/csrc/render.cu", "paper_2303_14827_gb300/csrc/dq_math.cuh",
                  "paper_2303_14827_gb300/csrc/dqj_internal.h")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "march_kernel_1080p.md")


def kernel_sha() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes per march launch from the committed ncu summary, if it was
    taken on the current kernel sources."""
    try:
        text = open(TRAFFIC_FILE).read()
    except OSError:
        return None
    m = re.search(r"kernel_sha256_16:\s*([0-9a-f]+)", text)
    t = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m or not t or m.group(1) != kernel_sha():
        return None
    return float(t.group(1))


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sms, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sms:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sms)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def max_over_ranks(v: float, world: int) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def workload_scenes(precision: int):
    from paper_2303_14827_gb300 import scenes
    return [scenes.full_hd_scene(s, precision=precision) for s in SEEDS]


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline leg and --impl reference)
# ---------------------------------------------------------------------------
def oracle_sample_rate(target_s: float, seed: int = 11):
    """Time the FP64 oracle on a random pixel sample of the workload frames,
    growing the sample until it takes about target_s.  Returns (iters/s, frames/s
    equivalent, cores, description, seconds)."""
    import oracle
    from paper_2303_14827_gb300 import scenes
    frames = workload_scenes(scenes.PRECISION_FP32)
    W, H = frames[0]["width"], frames[0]["height"]
    n = 256
    while True:
        t0 = time.perf_counter()
        iters = 0
        threads = 0
        for k, s in enumerate(frames):
            pix = scenes.sample_pixels(W, H, n, seed=seed + k)
            r = oracle.render(s, pixels=pix)
            iters += r["class_iters"] + r["normal_iters"]
            threads = r["threads"]
        dt = time.perf_counter() - t0
        if dt >= 0.4 * target_s or n >= W * H:
            px_per_s = n * len(frames) / dt
            desc = (f"{n} random pixels from each of the 5 workload frames ({n * len(frames)} pixels, "
                    f"{dt:.1f} s, FP64 oracle, {threads} threads)")
            return iters / dt, px_per_s / (W * H), threads, desc, dt
        n = int(min(W * H, n * max(2.0, 1.2 * target_s / max(dt, 1e-3))))


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    steps, warm = args.steps, args.warmup
    per_step = max(1.0, args.ref_seconds / max(steps + warm, 1))
    rate, fps, cores, desc, _ = oracle_sample_rate(per_step)
    # bounded samples of the same size, timed step by step; n from the measured pixel rate
    import oracle
    from paper_2303_14827_gb300 import scenes
    frames = workload_scenes(scenes.PRECISION_FP32)
    W, H = frames[0]["width"], frames[0]["height"]
    n = max(64, int(fps * W * H * per_step / len(frames)))
    times, iters = [], []
    for st in range(warm + steps):
        t0 = time.perf_counter()
        it = 0
        for k, s in enumerate(frames):
            r = oracle.render(s, pixels=scenes.sample_pixels(W, H, n, seed=100 + st * 7 + k))
            it += r["class_iters"] + r["normal_iters"]
            cores = r["threads"]
        dt = time.perf_counter() - t0
        if st >= warm:
            times.append(dt)
            iters.append(it)
    value = sum(iters) / sum(times)
    sample = f"{n} random pixels from each of the 5 workload frames per step ({5 * n} pixels, FP64 oracle)"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "impl": "reference",
        "n_gpus": args.gpus, "steps": steps, "warmup": warm,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args, world, rank, local):
    import torch

    from paper_2303_14827_gb300 import binding, scenes

    torch.cuda.set_device(local)
    binding.load()
    frames = workload_scenes(args.precision)
    nf = len(frames)
    W, H = frames[0]["width"], frames[0]["height"]
    ctx = binding.dqj_create(local)
    ring = nf * (args.steps + 1)
    binding.dqj_set_profiling(ctx, min(ring, 4096))
    outs = [binding.alloc_outputs(W, H, device=f"cuda:{local}") for _ in frames]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{local}")
    stream = torch.cuda.current_stream(local)
    sh = stream.cuda_stream

    def step(i: int):
        flush.fill_(i & 0xFF)
        for s, o in zip(frames, outs):
            binding.dqj_render(ctx, s, binding.outputs_of(o), sh)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    st = [binding.stats_dict(o["stats"]) for o in outs]
    iters_per_step = sum(x["class_iters"] + x["normal_iters"] for x in st)
    march_iters = [x["march_iters"] for x in st]

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0.record(stream)
        for i in range(args.steps):
            step(args.warmup + i)
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms, world)
    pass_ms = binding.dqj_pass_ms(ctx, nf * args.steps)
    st2 = [binding.stats_dict(o["stats"]) for o in outs]
    assert st2 == st, "iteration counts changed between steps"

    total_iters = iters_per_step * args.steps * world
    value = total_iters / (ms_max * 1e-3)
    fps = nf * args.steps * world / (ms_max * 1e-3)

    # roofline of the dominant kernel (the march), over every launch of the region
    march_ms = [p[0] for p in pass_ms]
    march_flops = sum(FLOPS_PER_ITER * march_iters[i % nf] for i in range(len(march_ms)))
    achieved = march_flops / (sum(march_ms) * 1e-3) / 1e12
    num_sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak = num_sms * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    clocks = clk.summary()
    roof = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "TFLOP/s",
            "frac": round(achieved / peak, 4), "traffic": recorded_traffic(),
            "kernel": "march_kernel<float,ALGEBRAIC,EUCLID8>", "launches": len(march_ms),
            "avg_launch_ms": round(sum(march_ms) / len(march_ms), 4),
            "flops_per_iter": FLOPS_PER_ITER,
            "peak_basis": f"{num_sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {SM_MAX_MHZ:.0f} MHz (max clock)"}
    if clocks.get("sm_mhz"):
        roof["frac_at_sampled_clock"] = round(achieved / (peak * clocks["sm_mhz"] / SM_MAX_MHZ), 4)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == 0 else
        ("f32+f64-recheck" if args.precision == 1 else "f64"), "data": "synthetic",
        "config": {"workload": WORKLOAD, "frames_per_step": nf, "width": W, "height": H, "max_iter": 16,
                   "march_steps": 512, "bisect_steps": 10, "precision": args.precision,
                   "l2": "256 MiB buffer written between steps", "parallelism": f"replica x{world}"},
        "frames_per_s": fps,
        "iters_per_frame": [x["class_iters"] + x["normal_iters"] for x in st],
        "hits_per_frame": [x["hits"] for x in st],
        "pass_ms_mean": [round(sum(p[i] for p in pass_ms) / len(pass_ms), 4) for i in range(4)],
        "roofline": roof,
        "clocks": clocks,
        "gpu_launches": (2 if args.precision != 1 else 4) * nf * args.steps,
    }

    # end to end through the public API with host buffers
    if not args.no_e2e:
        host = []
        for _ in frames:
            host.append({
                "iter": torch.empty((H, W), dtype=torch.int32).pin_memory(),
                "depth": torch.empty((H, W), dtype=torch.float32).pin_memory(),
                "normal": torch.empty((H, W, 3), dtype=torch.float32).pin_memory(),
                "rgba": torch.empty((H, W, 4), dtype=torch.uint8).pin_memory(),
                "stats": torch.zeros(binding.DQJ_NSTATS, dtype=torch.int64).pin_memory(),
                "pitch_px": W})
        for s, o in zip(frames, host):  # warm-up of the host path
            binding.dqj_render_host(ctx, s, binding.outputs_of(o))
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            for s, o in zip(frames, host):
                binding.dqj_render_host(ctx, s, binding.outputs_of(o))
        dt = max_over_ranks(time.perf_counter() - t0, world)
        e2e_iters = sum(int(o["stats"][0]) + int(o["stats"][1]) for o in host)
        line["e2e"] = {"value": e2e_iters * args.steps * world / dt, "unit": UNIT,
                       "h2d_bytes_per_step": nf * binding.ctypes.sizeof(binding.dqj_params),
                       "d2h_bytes_per_step": nf * (W * H * 24 + 8 * binding.DQJ_NSTATS),
                       "frames_per_s": nf * args.steps * world / dt}

    if rank == 0 and not args.no_cpu_baseline:
        rate, _, cores, desc, _ = oracle_sample_rate(args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}

    binding.dqj_destroy(ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("dqj", "reference"), default="dqj")
    ap.add_argument("--precision", type=int, default=0, choices=(0, 1, 2))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=60.0)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "dqj":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    world, rank, local = dist_init()
    if args.impl == "reference":
        rc = run_reference(args, world, rank)
    else:
        rc = run_gpu(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
