#!/usr/bin/env python3
"""Benchmark of the dual-quaternion Julia isosurface renderer on GB300.

Workload (one step): the five seeded 1920x1080 frames (c ~ U[-0.8,0.8]^8 with
numpy default_rng(seed), seeds 0..4), max_iter 16, 512 march steps, 10 bisection
steps, central-difference normals (h = 1e-4), ambient+diffuse shading to RGBA8,
in the contract-accurate mode: FP32 with an FP64 recheck of every sample whose
escape test came within 1e-3 relative of R^2 (FP32 + FP64 recheck), the mode
held to the parity contract on whole frames.  Inputs (parameter blocks) and
output planes (24 B/pixel) stay resident on the device; a 256 MiB buffer is
written between steps to flush L2.

Metric: DQ iterations/s (algorithmic iterations: escape count, or max_iter for an
inside sample, plus the n* steps of each normal evaluation, counted by the
kernels) with frames/s beside it; roofline of the march kernel against the FP32
FMA peak (152 SMs x 128 lanes x 2 flop x 2070 MHz), 52 flops per DQ iteration.
Beside it: plain FP32 (outside the parity contract, with its measured
differences from the all-FP64 render), the precision report, a general slice
frame, the served form (10,000 Poisson requests), the 64-frame batch, the
256x256 frame and the CPU oracle.

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
WORKLOAD = "dq-julia 1920x1080, c~U[-0.8,0.8]^8 seeds 0-4, max_iter 16, 512 march + 10 bisect"
MODE_NAMES = {0: "FP32", 1: "FP32 + FP64 recheck (margin 1e-3)", 2: "FP64"}
DTYPES = {0: "f32", 1: "f32+f64-recheck", 2: "f64"}
KERNEL_SOURCES = ("paper_2303_14827_gb300/csrc/render.cu", "paper_2303_14827_gb300/csrc/render_common.cuh",
                  "paper_2303_14827_gb300/csrc/dq_math.cuh", "paper_2303_14827_gb300/csrc/dqj_internal.h")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "march4_kernel_1080p.md")


def kernel_sha() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(tag: str):
    """DRAM bytes per march launch (`tag`: recheck, plain or general) from the
    committed ncu summary, if it was taken on the current kernel sources."""
    try:
        text = open(TRAFFIC_FILE).read()
    except OSError:
        return None
    m = re.search(r"kernel_sha256_16:\s*([0-9a-f]+)", text)
    t = re.search(r"traffic_bytes_per_launch\[%s\]:\s*([0-9.eE+]+)" % re.escape(tag), text)
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
                 "-lms", "25"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            t0 = time.time()  # sampling must be running when the timed region starts
            while not self.lines and time.time() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.01)
            self.lines.clear()
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


def oracle_full_frames():
    """The FP64 oracle on whole frames: the 256x256 single-frame scene on all
    host cores and on one core, and one 1920x1080 workload frame (seed 0) on
    all cores."""
    import oracle
    from paper_2303_14827_gb300 import scenes
    out = {}
    for name, s, threads in (("256x256_all_cores", scenes.default_scene(), 0),
                             ("256x256_one_core", scenes.default_scene(), 1),
                             ("1920x1080_seed0_all_cores", scenes.full_hd_scene(0), 0)):
        t0 = time.perf_counter()
        r = oracle.render(s, threads=threads)
        dt = time.perf_counter() - t0
        out[name] = {"seconds": round(dt, 3), "threads": r["threads"],
                     "iters_per_s": (r["class_iters"] + r["normal_iters"]) / dt}
    return out


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
def fp32_peak_tflops(local) -> tuple:
    import torch
    num_sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak = num_sms * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    return peak, f"{num_sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {SM_MAX_MHZ:.0f} MHz (max clock)"


def timed_frames(ctx, frames, outs, steps, warmup, local, world, flush):
    """Render `frames` once per step as one dqj_render_batch (W warm-up steps,
    then K timed steps between barriers, the L2 flushed before each step).  Returns (max-over-ranks ms,
    per-frame stats, per-launch pass times of the timed renders, clocks)."""
    import torch

    from paper_2303_14827_gb300 import binding
    stream = torch.cuda.current_stream(local)
    sh = stream.cuda_stream
    douts = [binding.outputs_of(o) for o in outs]

    def step(i: int):  # one batch of frames, pipelined by the library
        flush.fill_(i & 0xFF)
        binding.dqj_render_batch(ctx, frames, douts, sh)

    for i in range(warmup):
        step(i)
    torch.cuda.synchronize()
    st = [binding.stats_dict(o["stats"]) for o in outs]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0.record(stream)
        for i in range(steps):
            step(warmup + i)
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    pass_ms = binding.dqj_pass_ms(ctx, len(frames) * steps)
    st2 = [binding.stats_dict(o["stats"]) for o in outs]
    assert [x["march_iters"] for x in st2] == [x["march_iters"] for x in st], "iteration counts changed between steps"
    return ms, st, pass_ms, clk.summary()


def march_roofline(pass_ms, stats, peak, peak_basis, kernel, traffic, clocks=None):
    """Algorithmic FP32 flops of the march kernel (52 per DQ iteration it
    performed) over its CUDA-event time, every launch of the timed region."""
    nf = len(stats)
    march_ms = [p[0] for p in pass_ms]
    flops = sum(FLOPS_PER_ITER * stats[i % nf]["march_iters"] for i in range(len(march_ms)))
    achieved = flops / (sum(march_ms) * 1e-3) / 1e12
    roof = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "TFLOP/s",
            "frac": round(achieved / peak, 4), "traffic": traffic, "kernel": kernel, "launches": len(march_ms),
            "avg_launch_ms": round(sum(march_ms) / len(march_ms), 4), "flops_per_iter": FLOPS_PER_ITER,
            "peak_basis": peak_basis}
    if clocks and clocks.get("sm_mhz"):
        roof["frac_at_sampled_clock"] = round(achieved / (peak * clocks["sm_mhz"] / SM_MAX_MHZ), 4)
    return roof


def mode_section(ctx, frames, outs, steps, warmup, local, world, flush, peak, basis, kernel, tag):
    """One precision mode on `frames`: ms per frame, DQ iterations/s, frames/s,
    mean per-pass times and the march roofline."""
    ms, st, pass_ms, clocks = timed_frames(ctx, frames, outs, steps, warmup, local, world, flush)
    nf = len(frames)
    it = sum(x["class_iters"] + x["normal_iters"] for x in st)
    return {"ms_per_frame": round(ms / (steps * nf), 4), "iters_per_s": it * steps * world / (ms * 1e-3),
            "frames_per_s": nf * steps * world / (ms * 1e-3),
            "pass_ms_mean": [round(sum(p[i] for p in pass_ms) / len(pass_ms), 4) for i in range(4)],
            "rechecks_per_frame": [x["rechecks"] for x in st], "fixups_per_frame": [x["fixups"] for x in st],
            "roofline": march_roofline(pass_ms, st, peak, basis, kernel, recorded_traffic(tag), clocks),
            "clocks": clocks}, ms, st, pass_ms, clocks


def run_gpu(args, world, rank, local):
    import numpy as np
    import torch

    from paper_2303_14827_gb300 import binding, scenes

    torch.cuda.set_device(local)
    binding.load()
    prec = args.precision
    frames = workload_scenes(prec)
    nf = len(frames)
    W, H = frames[0]["width"], frames[0]["height"]
    ctx = binding.dqj_create(local)
    binding.dqj_set_profiling(ctx, min(nf * (args.steps + 1), 4096))
    outs = [binding.alloc_outputs(W, H, device=f"cuda:{local}") for _ in frames]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{local}")
    peak, basis = fp32_peak_tflops(local)
    # the paired march: two samples of each ray per round unless DQJ_MARCH_SAMPLES=1
    k2 = "march2_kernel" if os.environ.get("DQJ_MARCH_SAMPLES", "").strip() == "1" else "march4_kernel"
    kname = {0: f"{k2}<ALGEBRAIC,EUCLID8,plain,axis>", 1: f"{k2}<ALGEBRAIC,EUCLID8,recheck,axis>",
             2: "march_kernel<double,ALGEBRAIC,EUCLID8>"}

    # the headline: the workload frames in the requested mode (default: FP32 + FP64 recheck)
    ms, st, pass_ms, clocks = timed_frames(ctx, frames, outs, args.steps, args.warmup, local, world, flush)
    iters_per_step = sum(x["class_iters"] + x["normal_iters"] for x in st)
    value = iters_per_step * args.steps * world / (ms * 1e-3)
    fps = nf * args.steps * world / (ms * 1e-3)
    roof = march_roofline(pass_ms, st, peak, basis, kname[prec],
                          recorded_traffic({0: "plain", 1: "recheck"}.get(prec, "fp64")), clocks)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[prec], "data": "synthetic",
        "config": {"workload": WORKLOAD + ", " + MODE_NAMES[prec], "frames_per_step": nf, "width": W, "height": H,
                   "max_iter": 16, "march_steps": 512, "bisect_steps": 10, "precision": prec,
                   "recheck_margin": 1e-3, "l2": "256 MiB buffer written between steps",
                   "parallelism": f"replica x{world}"},
        "frames_per_s": fps,
        "iters_per_frame": [x["class_iters"] + x["normal_iters"] for x in st],
        "hits_per_frame": [x["hits"] for x in st],
        "rechecks_per_frame": [x["rechecks"] for x in st],
        "fixups_per_frame": [x["fixups"] for x in st],
        "pass_ms_mean": [round(sum(p[i] for p in pass_ms) / len(pass_ms), 4) for i in range(4)],
        "pass_names": ["march", "bisect+normal+shade", "fp64 recheck", "fp64 re-render"],
        "roofline": roof,
        "clocks": clocks,
        "gpu_launches": (4 if prec == 1 else 2) * nf * args.steps,
    }

    # plain FP32 beside it: faster, outside the parity contract (see its differences below)
    if prec != 0:
        f0 = workload_scenes(0)
        sec, _, _, _, _ = mode_section(ctx, f0, outs, args.steps, args.warmup, local, world, flush, peak, basis,
                                       kname[0], "plain")
        sec["parity"] = ("outside the parity contract: escape decisions within FP32 rounding of R^2 are not "
                         "rechecked; see precision_report for its differences from the all-FP64 render")
        line["plain_fp32"] = sec

    # a general slice frame: random orthonormal slice frame in R^8 (first-iterate form)
    rng = np.random.default_rng(7)
    gen = [scenes.full_hd_scene(k, precision=p, slice_basis=scenes.random_slice_frame(rng))
           for k, p in ((0, 0), (1, 0), (2, 0))]
    gsec = {"workload": "1920x1080, c~U[-0.8,0.8]^8 seeds 0-2, slice frame = QR of an 8x3 Gaussian "
                        "(default_rng(7)), max_iter 16, 512 march + 10 bisect"}
    for p, tag in ((1, "recheck"), (0, "plain")):
        fr = [dict(g, precision=p) for g in gen]
        sec, _, _, _, _ = mode_section(ctx, fr, outs[:3], max(3, args.steps // 3), args.warmup, local, world,
                                       flush, peak, basis, f"{k2}<ALGEBRAIC,EUCLID8,{tag},general>",
                                       "general_" + tag)
        gsec[tag] = sec
    line["general_slice"] = gsec

    # end to end through the public API with host buffers, in the headline mode
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
        host_outs = [binding.outputs_of(o) for o in host]
        binding.dqj_render_host_batch(ctx, frames, host_outs)  # warm-up of the host path
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(args.steps):  # one step: the five frames, copies back overlapped with the next render
            binding.dqj_render_host_batch(ctx, frames, host_outs)
        dt = max_over_ranks(time.perf_counter() - t0, world)
        e2e_iters = sum(int(o["stats"][0]) + int(o["stats"][1]) for o in host)
        line["e2e"] = {"value": e2e_iters * args.steps * world / dt, "unit": UNIT,
                       "h2d_bytes_per_step": nf * binding.ctypes.sizeof(binding.dqj_params),
                       "d2h_bytes_per_step": nf * (W * H * 24 + 8 * binding.DQJ_NSTATS),
                       "frames_per_s": nf * args.steps * world / dt}
    binding.dqj_destroy(ctx)
    del outs, flush
    torch.cuda.empty_cache()

    if not args.no_precision_report:
        line["precision_report"] = precision_section(local)
    if not args.no_serve:
        line["served"] = serving_section(local, n_sat=512, n_stream=args.requests, rates=(0.8, 1.0))
        rq = serving_section(local, n_sat=512, n_stream=0, rates=(), policies=(), precision=1)
        line["served_recheck"] = {k: rq[k] for k in ("requests_burst", "served_frames_per_s",
                                                     "plain_back_to_back_frames_per_s", "served_over_plain",
                                                     "burst_scheduler")}
        line["served_recheck"]["mode"] = MODE_NAMES[1]
        line["batch64"] = batch_section(local)

    line["c1"] = c1_section(local)
    if rank == 0 and not args.no_cpu_baseline:
        rate, _, cores, desc, _ = oracle_sample_rate(args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
                                "full_frames": oracle_full_frames()}

    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0



def gather_parts(planes, gathered, owner, world):
    """The gather of the frame split: every rank's output planes (dict of
    (H, pitch, ...) tensors, each rank's own tiles rendered) are all-gathered
    into `gathered` (dict of (world, H, pitch, ...) tensors), and each pixel is
    taken from the rank that owns its tile (`owner`, (H, pitch) int64)."""
    import torch
    import torch.distributed as dist
    for k, o in planes.items():
        g = gathered[k]
        dist.all_gather_into_tensor(g.view((-1,) + tuple(g.shape[2:])), o.contiguous())  # parts along dim 0
        m = owner[(...,) + (None,) * (o.dim() - 2)]
        o.copy_(torch.gather(gathered[k], 0, m.expand_as(o).unsqueeze(0)).squeeze(0))


def run_split(args, world, rank, local):
    """The frame split across ranks (one GPU each): every rank renders the
    tiles t with t mod N == rank of the five workload frames
    (dqj_render_tiles), the output planes are gathered to every rank
    (all_gather) and put together by tile owner, all inside the timed region.
    Strong scaling: the whole frames' DQ iterations over the max-over-ranks
    time."""
    import torch

    from paper_2303_14827_gb300 import binding
    torch.cuda.set_device(local)
    binding.load()
    frames = workload_scenes(args.precision)
    nf = len(frames)
    W, H = frames[0]["width"], frames[0]["height"]
    dev = f"cuda:{local}"
    ctx = binding.dqj_create(local)
    outs = [binding.alloc_outputs(W, H, device=dev) for _ in frames]
    owners = [torch.as_tensor(binding.tile_parts_of_pixels(ctx, s, world), device=dev) for s in frames]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(local)
    planes = ("iter", "depth", "normal", "rgba")
    gath = {k: torch.empty((world,) + tuple(outs[0][k].shape), dtype=outs[0][k].dtype, device=dev) for k in planes}
    def step(i):
        flush.fill_(i & 0xFF)
        for s, o, own in zip(frames, outs, owners):
            binding.dqj_render_tiles(ctx, s, binding.outputs_of(o), stream.cuda_stream, rank, world)
            if world > 1:  # gather every part, put each pixel from its tile's owner
                gather_parts({k: o[k] for k in planes}, gath, own, world)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for i in range(args.steps):
            step(args.warmup + i)
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    ctx2 = binding.dqj_create(local)  # the whole frames' algorithmic iterations
    it = 0
    for s, o in zip(frames, outs):
        ref = binding.alloc_outputs(W, H, device=dev)
        binding.dqj_render(ctx2, s, binding.outputs_of(ref), stream.cuda_stream)
        torch.cuda.synchronize()
        st = binding.stats_dict(ref["stats"])
        it += st["class_iters"] + st["normal_iters"]
    binding.dqj_destroy(ctx2)
    binding.dqj_destroy(ctx)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": it * args.steps / (ms * 1e-3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": DTYPES[args.precision], "data": "synthetic",
            "config": {"workload": WORKLOAD + ", " + MODE_NAMES[args.precision], "frames_per_step": nf,
                       "l2": "256 MiB buffer written between steps", "parallelism": f"frame split x{world}",
                       "gather": "all_gather of the output planes, put together by tile owner, in the timed region"},
            "frames_per_s": nf * args.steps / (ms * 1e-3), "clocks": clk.summary(),
            "gpu_launches": (4 if args.precision == 1 else 2) * nf * args.steps}), flush=True)
    return 0


# ---------------------------------------------------------------------------
# served form: saturation, Poisson latency, and the mixed 64-frame batch
# ---------------------------------------------------------------------------
class OutputPool:
    """Reusable device output planes per resolution (caller-owned outputs must
    stay valid until the request completes).  Planes are allocated up front by
    prefill; `misses` counts allocations made later.  After an allocation only
    torch's own stream is synchronized (the library writes outputs from its own
    streams): a device-wide synchronize would wait for the persistent launch."""

    def __init__(self, device):
        self.device = device
        self.free = {}
        self.misses = 0

    def _alloc(self, w, h):
        from paper_2303_14827_gb300 import binding
        return binding.alloc_outputs(w, h, device=self.device)

    def prefill(self, reqs):
        import collections

        import torch
        need = collections.Counter((s["width"], s["height"]) for s in reqs)
        for key, n in need.items():
            lst = self.free.setdefault(key, [])
            while len(lst) < n:
                lst.append(self._alloc(*key))
        torch.cuda.synchronize(self.device)  # the library writes outputs from its own streams

    def get(self, w, h):
        import torch
        lst = self.free.setdefault((w, h), [])
        if lst:
            return lst.pop()
        self.misses += 1
        o = self._alloc(w, h)
        torch.cuda.current_stream(self.device).synchronize()
        return o

    def put(self, w, h, o):
        self.free.setdefault((w, h), []).append(o)


def served_run(ctx, reqs, arrivals, pool):
    """Submit reqs[i] at time arrivals[i] (seconds from start, sorted), poll until
    all are done.  Returns (latencies in s, makespan s).  Python's cyclic garbage
    collector is paused meanwhile, so that none of its pauses lands inside a
    measured latency."""
    import gc
    gc.collect()
    gc.disable()
    try:
        return _served_run(ctx, reqs, arrivals, pool)
    finally:
        gc.enable()


def _served_run(ctx, reqs, arrivals, pool):
    from paper_2303_14827_gb300 import binding
    n = len(reqs)
    lat = [None] * n
    inflight = {}
    nxt = 0
    t0 = time.perf_counter()
    last_done = t0
    while nxt < n or inflight:
        now = time.perf_counter() - t0
        while nxt < n and arrivals[nxt] <= now:
            s = reqs[nxt]
            o = pool.get(s["width"], s["height"])
            try:
                t = binding.dqj_submit(ctx, s, binding.outputs_of(o))
            except binding.DqjError as e:
                if e.status != binding.DQJ_ERR_BUSY:
                    raise
                pool.put(s["width"], s["height"], o)
                break
            inflight[t] = (nxt, o, t0 + arrivals[nxt])
            nxt += 1
        for t in list(inflight):
            done, st = binding.dqj_poll(ctx, t)
            if done:
                i, o, ta = inflight.pop(t)
                assert st == binding.DQJ_OK, st
                tn = time.perf_counter()
                lat[i] = tn - ta
                last_done = tn
                s = reqs[i]
                pool.put(s["width"], s["height"], o)
    return lat, last_done - t0


def plain_back_to_back(ctx, reqs, pool, stream):
    """The same requests rendered one after another with dqj_render on one stream."""
    import torch

    from paper_2303_14827_gb300 import binding
    outs = [pool.get(s["width"], s["height"]) for s in reqs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s, o in zip(reqs, outs):
        binding.dqj_render(ctx, s, binding.outputs_of(o), stream.cuda_stream)
    stream.synchronize()
    dt = time.perf_counter() - t0
    for s, o in zip(reqs, outs):
        pool.put(s["width"], s["height"], o)
    return dt


def pct(v, q):
    v = sorted(v)
    return v[min(len(v) - 1, int(round(q * (len(v) - 1))))]


POLICY_NAMES = {0: "fifo", 1: "shortest"}


def serving_section(local, n_sat=256, n_stream=600, rates=(0.8, 1.0), policies=(0, 1), precision=0):
    """Served vs back-to-back frames/s on a burst of the serving mix, then Poisson
    arrivals at the given fractions of the measured saturation rate, under each
    serving policy (arrival order; earliest estimated finish), with latency
    percentiles (and their sample counts) overall and per request size.  All
    requests in the given precision mode."""
    import numpy as np
    import torch

    from paper_2303_14827_gb300 import binding, scenes
    stream_reqs = [s for _, s in scenes.serving_stream(seed=2, n=max(n_sat, n_stream), precision=precision)]
    pool = OutputPool(f"cuda:{local}")
    ctx = binding.dqj_create(local)
    try:
        warm = stream_reqs[:32]
        burst = stream_reqs[:n_sat]
        pool.prefill(burst)
        served_run(ctx, warm, [0.0] * len(warm), pool)
        plain_back_to_back(ctx, warm, pool, torch.cuda.current_stream(local))
        s0 = binding.dqj_serve_stats(ctx)
        _, t_served = served_run(ctx, burst, [0.0] * len(burst), pool)
        s1 = binding.dqj_serve_stats(ctx)
        t_plain = plain_back_to_back(ctx, burst, pool, torch.cuda.current_stream(local))
        sat = len(burst) / t_served
        out = {"requests_burst": len(burst), "served_frames_per_s": sat,
               "plain_back_to_back_frames_per_s": len(burst) / t_plain,
               "served_over_plain": t_plain / t_served,
               "burst_scheduler": {k: s1[k] - s0[k] for k in s1}, "poisson": []}
        rng = np.random.default_rng(2)
        gaps = rng.exponential(1.0, n_stream)
        reqs = stream_reqs[:n_stream]
        sizes = [(s["width"], s["height"]) for s in reqs]
        for policy in policies:
            binding.dqj_serve_policy(ctx, policy)
            for f in rates:
                arr = np.cumsum(gaps / (f * sat)).tolist()
                lat, span = served_run(ctx, reqs, arr, pool)
                by_size = {}
                for wh in sorted(set(sizes), key=lambda v: v[0] * v[1]):
                    ls = [x for x, z in zip(lat, sizes) if z == wh]
                    by_size["%dx%d" % wh] = {"n": len(ls), "p50_ms": round(1e3 * pct(ls, 0.50), 3),
                                             "p99_ms": round(1e3 * pct(ls, 0.99), 3)}
                out["poisson"].append({"policy": POLICY_NAMES[policy], "offered_fraction_of_saturation": f,
                                       "requests": len(reqs), "latency_samples": len(lat),
                                       "p50_ms": 1e3 * pct(lat, 0.50),
                                       "p99_ms": 1e3 * pct(lat, 0.99), "achieved_frames_per_s": len(reqs) / span,
                                       "by_size": by_size})
        binding.dqj_serve_policy(ctx, binding.DQJ_SERVE_FIFO)
        out["output_pool_misses"] = pool.misses
        out["scheduler"] = binding.dqj_serve_stats(ctx)
        return out
    finally:
        binding.dqj_destroy(ctx)


def batch_section(local, n=64):
    """The 64 mixed frames (random slices, resolutions, max_iter) as one served
    batch in the persistent launch vs back to back, with autotuned tiles."""
    import torch

    from paper_2303_14827_gb300 import binding, scenes
    reqs = scenes.batch_scenes(seed=1, n=n)
    pool = OutputPool(f"cuda:{local}")
    ctx = binding.dqj_create(local)
    try:
        binding.dqj_autotune(ctx, 0)
        pool.prefill(reqs)
        served_run(ctx, reqs[:8], [0.0] * 8, pool)
        _, t_served = served_run(ctx, reqs, [0.0] * n, pool)
        t_plain = plain_back_to_back(ctx, reqs, pool, torch.cuda.current_stream(local))
        return {"frames": n, "served_frames_per_s": n / t_served, "plain_back_to_back_frames_per_s": n / t_plain,
                "served_over_plain": t_plain / t_served}
    finally:
        binding.dqj_destroy(ctx)


def c1_section(local, reps=40):
    """The 256x256 single-frame scene (max_iter 12, 256 march + 8 bisection
    steps) on the GPU: ms per frame (CUDA events, mean over reps after a
    warm-up), frames/s and DQ iterations/s."""
    import torch

    from paper_2303_14827_gb300 import binding, scenes
    s = scenes.default_scene()
    ctx = binding.dqj_create(local)
    stream = torch.cuda.current_stream(local)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    o = binding.alloc_outputs(s["width"], s["height"], device=f"cuda:{local}")
    try:
        for _ in range(3):
            binding.dqj_render(ctx, s, binding.outputs_of(o), stream.cuda_stream)
        e0.record(stream)
        for _ in range(reps):
            binding.dqj_render(ctx, s, binding.outputs_of(o), stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        st = binding.stats_dict(o["stats"])
        # the same frames launched from a CUDA graph of 8 captured renders
        cap = torch.cuda.Stream(local)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cap):
            for _ in range(8):
                binding.dqj_render(ctx, s, binding.outputs_of(o), cap.cuda_stream)
        g.replay()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(max(1, reps // 8)):
            g.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        ms_graph = e0.elapsed_time(e1) / (8 * max(1, reps // 8))
        del g  # a graph holding renders goes before its context
        torch.cuda.synchronize()
        # the same frames as batches of 8 (dqj_render_batch: a frame's bisection
        # runs beside the next frame's march), into 8 output sets
        bo = [binding.alloc_outputs(s["width"], s["height"], device=f"cuda:{local}") for _ in range(8)]
        bdo = [binding.outputs_of(x) for x in bo]
        binding.dqj_render_batch(ctx, [s] * 8, bdo, stream.cuda_stream)
        e0.record(stream)
        for _ in range(max(1, reps // 8)):
            binding.dqj_render_batch(ctx, [s] * 8, bdo, stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_batch = e0.elapsed_time(e1) / (8 * max(1, reps // 8))
    finally:
        binding.dqj_destroy(ctx)
    it = st["class_iters"] + st["normal_iters"]
    return {"workload": "256x256, c = (-0.2,0.6,0.2,0.2 | 0.1,0,0,0.05), max_iter 12, 256 march + 8 bisect, FP32",
            "ms_per_frame": round(ms, 4), "frames_per_s": 1e3 / ms, "iters_per_frame": it,
            "iters_per_s": it / (ms * 1e-3), "hits": st["hits"],
            "graph_ms_per_frame": round(ms_graph, 4), "graph_frames_per_s": 1e3 / ms_graph,
            "batch8_ms_per_frame": round(ms_batch, 4), "batch8_frames_per_s": 1e3 / ms_batch}


def precision_section(local, reps=3):
    """FP32, FP32 + FP64 recheck and all-FP64 renders of the workload frames (and
    of the default c at 1920x1080, which has many hits): time per frame, recheck
    rate, and the FP32 / FP32+recheck images against the all-FP64 GPU image
    (hit/miss flips, iteration mismatches on agreeing pixels, depth error on
    agreeing hits).  The FP64 render is itself held to the oracle by the tests."""
    import torch

    from paper_2303_14827_gb300 import binding, scenes
    rows = [("seed%d" % k, scenes.full_hd_scene(k)) for k in SEEDS]
    rows.append(("default_c_1080p", scenes.default_scene(width=1920, height=1080, max_iter=16, march_steps=512,
                                                        bisect_steps=10)))
    ctx = binding.dqj_create(local)
    stream = torch.cuda.current_stream(local)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = []
    try:
        for name, base in rows:
            W, H = base["width"], base["height"]
            res = {}
            for prec in (scenes.PRECISION_FP32, scenes.PRECISION_FP32_RECHECK, scenes.PRECISION_FP64):
                s = dict(base, precision=prec)
                o = binding.alloc_outputs(W, H, device=f"cuda:{local}")
                binding.dqj_render(ctx, s, binding.outputs_of(o), stream.cuda_stream)  # warm-up
                best = 1e30
                for _ in range(reps):
                    e0.record(stream)
                    binding.dqj_render(ctx, s, binding.outputs_of(o), stream.cuda_stream)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    best = min(best, e0.elapsed_time(e1))
                res[prec] = (o, best, binding.stats_dict(o["stats"]))
            ref, ref_ms, _ = res[scenes.PRECISION_FP64]
            rd = ref["depth"][:, :W]
            rh = torch.isfinite(rd)
            row = {"frame": name, "fp64_ms": round(ref_ms, 3), "hits_fp64": int(rh.sum())}
            for prec, tag in ((scenes.PRECISION_FP32, "fp32"), (scenes.PRECISION_FP32_RECHECK, "recheck")):
                o, ms, st = res[prec]
                d = o["depth"][:, :W]
                h = torch.isfinite(d)
                agree = h == rh
                both = h & rh
                err = (d[both].double() - rd[both].double()).abs()
                row[tag] = {
                    "ms": round(ms, 3), "speedup_vs_fp64": round(ref_ms / ms, 2),
                    "flip_frac": float((~agree).sum()) / (W * H),
                    "iter_mismatch_agreeing": int(((o["iter"][:, :W] != ref["iter"][:, :W]) & agree).sum()),
                    "depth_err_max": float(err.max()) if err.numel() else 0.0,
                    "depth_err_median": float(err.median()) if err.numel() else 0.0,
                }
                if prec == scenes.PRECISION_FP32_RECHECK:
                    row[tag]["recheck_rate"] = st["rechecks"] / max(st["samples"], 1)
                    row[tag]["rechecks"] = st["rechecks"]
                    row[tag]["fixups"] = st["fixups"]
            out.append(row)
    finally:
        binding.dqj_destroy(ctx)
    return out


def run_precision_only(args, world, rank, local):
    """C4: precision modes on the 1080p workload frames (one JSON line)."""
    import torch
    torch.cuda.set_device(local)
    from paper_2303_14827_gb300 import binding
    binding.load()
    rows = precision_section(local)
    line = {"metric": "FP32 / FP32+FP64-recheck vs all-FP64: flips, depth error, recheck rate, speedup",
            "value": statistics.median(r["recheck"]["speedup_vs_fp64"] for r in rows),
            "unit": "x speedup of FP32+recheck over all-FP64 (median over frames)", "n_gpus": 1,
            "higher_is_better": True, "data": "synthetic",
            "config": {"workload": WORKLOAD + "; plus the default c at 1920x1080", "recheck_margin": 1e-3},
            "frames": rows}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def sweep_section(local, reps=3):
    """Level of detail against cost (the paper's Fig. detail): sample points N
    and iteration limit n swept on two 1920x1080 scenes with visible sets (the
    default c and the Fig. highres2 constant), FP32: ms per frame (best of
    reps), DQ iterations/s and the fraction of hit pixels."""
    import torch

    from paper_2303_14827_gb300 import binding, scenes
    bases = {"default_c": scenes.default_scene(width=1920, height=1080, bisect_steps=10),
             "highres2": scenes.default_scene(c=list(scenes.PAPER_C_VALUES["highres2"]), width=1920, height=1080,
                                              bisect_steps=10)}
    ctx = binding.dqj_create(local)
    stream = torch.cuda.current_stream(local)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    o = binding.alloc_outputs(1920, 1080, device=f"cuda:{local}")
    rows = []
    try:
        for name, base in bases.items():
            for n_steps in (128, 256, 512, 1024):
                for mi in (6, 10, 15, 24):
                    sc = dict(base, march_steps=n_steps, max_iter=mi)
                    binding.dqj_render(ctx, sc, binding.outputs_of(o), stream.cuda_stream)
                    best = 1e30
                    for _ in range(reps):
                        e0.record(stream)
                        binding.dqj_render(ctx, sc, binding.outputs_of(o), stream.cuda_stream)
                        e1.record(stream)
                        torch.cuda.synchronize()
                        best = min(best, e0.elapsed_time(e1))
                    st = binding.stats_dict(o["stats"])
                    it = st["class_iters"] + st["normal_iters"]
                    rows.append({"scene": name, "march_steps": n_steps, "max_iter": mi, "ms": round(best, 3),
                                 "iters_per_s": it / (best * 1e-3), "hit_frac": st["hits"] / (1920 * 1080)})
    finally:
        binding.dqj_destroy(ctx)
    return rows


def voxel_section(local, reps=5):
    """Voxel occupancy grids (the paper's Fig. voxels prototype) of the default c:
    the paper's 50^3 and 100^3 and the largest 1024^3, FP32 (and FP32+recheck at
    1024^3): ms per grid (best of reps), cells/s, DQ iterations/s and the
    fraction of the FP32 FMA peak."""
    import torch

    from paper_2303_14827_gb300 import binding, scenes
    ctx = binding.dqj_create(local)
    stream = torch.cuda.current_stream(local)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    num_sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak = num_sms * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6
    rows = []
    try:
        for g, prec in ((50, 0), (100, 0), (1024, 0), (1024, 1)):
            s = scenes.default_scene(max_iter=16, precision=prec)
            occ = torch.empty(g ** 3, dtype=torch.uint8, device=f"cuda:{local}")
            st = torch.zeros(binding.DQJ_NSTATS, dtype=torch.int64, device=f"cuda:{local}")
            binding.dqj_voxelize(ctx, s, g, occ, None, st, stream.cuda_stream)
            best = 1e30
            for _ in range(reps):
                e0.record(stream)
                binding.dqj_voxelize(ctx, s, g, occ, None, st, stream.cuda_stream)
                e1.record(stream)
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            sd = binding.stats_dict(st)
            rate = sd["class_iters"] / (best * 1e-3)
            rows.append({"grid": g, "precision": prec, "ms": round(best, 4), "cells_per_s": g ** 3 / (best * 1e-3),
                         "iters_per_s": rate, "frac_fp32_peak": round(rate * FLOPS_PER_ITER / peak, 4),
                         "inside_frac": sd["hits"] / g ** 3, "rechecks": sd["rechecks"], "fixups": sd["fixups"]})
            del occ
    finally:
        binding.dqj_destroy(ctx)
    return rows


def voxel_image_section(local, reps=5):
    """Fig. voxels: the ray-traced 1920x1080 image of the default c beside
    images of its voxel grids (50^3 and 100^3 as in the paper, then finer), all
    FP32 + FP64 recheck.  Per grid: ms to voxelize and to render the grid's
    image (best of reps, CUDA events), cells the rays crossed per second, and
    the comparison with the traced image: the fraction of pixels whose hit/miss
    differs, the hit masks' intersection over union, and the median and 90th
    percentile depth difference on common hits in cell widths."""
    import numpy as np
    import torch

    from paper_2303_14827_gb300 import binding, scenes
    W, H = 1920, 1080
    s = scenes.default_scene(width=W, height=H, max_iter=16, march_steps=512, bisect_steps=10,
                             precision=scenes.PRECISION_FP32_RECHECK)
    ctx = binding.dqj_create(local)
    stream = torch.cuda.current_stream(local)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dev = f"cuda:{local}"

    def best_of(fn):
        fn()
        best = 1e30
        for _ in range(reps):
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    traced = binding.alloc_outputs(W, H, device=dev)
    img = binding.alloc_outputs(W, H, device=dev, stats=False)
    rows = []
    try:
        t_ms = best_of(lambda: binding.dqj_render(ctx, s, binding.outputs_of(traced), stream.cuda_stream))
        td = traced["depth"].cpu().numpy().astype(np.float64)
        hit_t = np.isfinite(td)
        for g in (50, 100, 200, 400, 1024):
            occ = torch.empty(g ** 3, dtype=torch.uint8, device=dev)
            v_ms = best_of(lambda: binding.dqj_voxelize(ctx, s, g, occ, None, None, stream.cuda_stream))
            r_ms = best_of(lambda: binding.dqj_render_voxels(ctx, s, g, occ, binding.outputs_of(img),
                                                             stream.cuda_stream))
            vd = img["depth"].cpu().numpy().astype(np.float64)
            cells = int(img["iter"].sum(dtype=torch.int64))
            hit_v = np.isfinite(vd)
            both = hit_v & hit_t
            dz = np.abs(vd[both] - td[both]) / (4.0 / g)
            rows.append({"grid": g, "voxelize_ms": round(v_ms, 4), "render_ms": round(r_ms, 4),
                         "cells_crossed_per_s": cells / (r_ms * 1e-3),
                         "hit_mask_differs_frac": round(float((hit_v != hit_t).mean()), 6),
                         "hit_mask_iou": round(float(both.sum() / max(1, (hit_v | hit_t).sum())), 5),
                         "depth_diff_cells_p50": round(float(np.median(dz)), 4) if dz.size else None,
                         "depth_diff_cells_p90": round(float(np.percentile(dz, 90)), 4) if dz.size else None})
            del occ
    finally:
        binding.dqj_destroy(ctx)
    return {"traced_ms": round(t_ms, 4), "traced_hits": int(hit_t.sum()), "grids": rows}


def run_voxel_only(args, world, rank, local):
    import torch
    torch.cuda.set_device(local)
    from paper_2303_14827_gb300 import binding
    binding.load()
    rows = voxel_section(local)
    big = next(r for r in rows if r["grid"] == 1024 and r["precision"] == 0)
    line = {"metric": "voxel occupancy grid: cells/s and DQ iterations/s (fraction of FP32 FMA peak)",
            "value": big["iters_per_s"], "unit": "DQ iterations/s (1024^3, FP32)", "n_gpus": 1,
            "higher_is_better": True, "data": "synthetic",
            "config": {"workload": "default c, default slice, max_iter 16, grids 50^3 / 100^3 / 1024^3 over the box"},
            "rows": rows, "vs_raytraced": voxel_image_section(local)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def de_section(local, reps=5):
    """The paper's own traversal (distance-estimate sphere tracing, Eq.
    distfract2) against the fixed-step march on the same 1920x1080 scenes:
    the five workload frames and the default c.  FP32, and both traversals in
    the contract-accurate FP32 + FP64 recheck mode; ms per frame (best of reps,
    CUDA events), DQ iterations, samples, hit pixels and FP64 re-renders."""
    import torch

    from paper_2303_14827_gb300 import binding, scenes
    frames = [("seed%d" % k, scenes.full_hd_scene(k)) for k in SEEDS]
    frames.append(("default_c", scenes.default_scene(width=1920, height=1080, max_iter=16, march_steps=512,
                                                     bisect_steps=10)))
    ctx = binding.dqj_create(local)
    stream = torch.cuda.current_stream(local)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    o = binding.alloc_outputs(1920, 1080, device=f"cuda:{local}")
    rows = []
    try:
        for name, base in frames:
            row = {"frame": name}
            rc = dict(base, precision=scenes.PRECISION_FP32_RECHECK)
            for tag, sc in (("march", base), ("de", dict(base, traversal=scenes.TRAVERSAL_DE)),
                            ("march_recheck", rc), ("de_recheck", dict(rc, traversal=scenes.TRAVERSAL_DE))):
                binding.dqj_render(ctx, sc, binding.outputs_of(o), stream.cuda_stream)
                best = 1e30
                for _ in range(reps):
                    e0.record(stream)
                    binding.dqj_render(ctx, sc, binding.outputs_of(o), stream.cuda_stream)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    best = min(best, e0.elapsed_time(e1))
                st = binding.stats_dict(o["stats"])
                row[tag] = {"ms": round(best, 4), "iters": st["class_iters"] + st["normal_iters"],
                            "samples": st["samples"], "hits": st["hits"], "fixups": st["fixups"]}
            row["de_speedup"] = round(row["march"]["ms"] / row["de"]["ms"], 2)
            row["de_recheck_speedup"] = round(row["march_recheck"]["ms"] / row["de_recheck"]["ms"], 2)
            rows.append(row)
    finally:
        binding.dqj_destroy(ctx)
    return rows


def run_de_only(args, world, rank, local):
    import torch
    torch.cuda.set_device(local)
    from paper_2303_14827_gb300 import binding
    binding.load()
    rows = de_section(local)
    fps = len(rows) / (sum(r["de"]["ms"] for r in rows) * 1e-3)
    line = {"metric": "1080p frames/s with distance-estimate sphere tracing (vs the fixed-step march)",
            "value": fps, "unit": "frames/s", "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": WORKLOAD + "; plus the default c; de_epsilon 1e-3, 512 steps at most"},
            "rows": rows}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_sweep_only(args, world, rank, local):
    import torch
    torch.cuda.set_device(local)
    from paper_2303_14827_gb300 import binding
    binding.load()
    rows = sweep_section(local)
    line = {"metric": "level of detail vs cost: ms per 1080p frame over march steps x max_iter",
            "value": statistics.median(r["iters_per_s"] for r in rows), "unit": "DQ iterations/s (median)",
            "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": "1920x1080, default c and Fig. highres2 c, N in {128,256,512,1024}, "
                                   "max_iter in {6,10,15,24}, 10 bisect, FP32"},
            "rows": rows}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_serve_only(args, world, rank, local):
    """C5: Poisson stream of render requests at offered rates relative to the
    measured saturation throughput (one JSON line)."""
    import torch
    torch.cuda.set_device(local)
    from paper_2303_14827_gb300 import binding
    binding.load()
    res = serving_section(local, n_sat=min(512, args.requests), n_stream=args.requests,
                          rates=(0.5, 0.8, 1.0, 1.2))
    one = next(p for p in res["poisson"] if p["offered_fraction_of_saturation"] == 1.0)
    line = {"metric": "served p50/p99 latency (ms) and frames/s", "value": one["achieved_frames_per_s"],
            "unit": "frames/s", "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": "Poisson stream: 256^2/512^2/1024^2/1920x1080 at 0.4/0.3/0.2/0.1, max_iter 8..32, "
                                   "c random walk (sigma 0.01) from the default c, 512 march + 10 bisect, FP32, "
                                   "16 GiB budget"},
            "served": res}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0

def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("dqj", "reference"), default="dqj")
    ap.add_argument("--precision", type=int, default=1, choices=(0, 1, 2),
                    help="headline mode: 0 FP32, 1 FP32 + FP64 recheck (default), 2 FP64")
    ap.add_argument("--no-precision-report", action="store_true")
    ap.add_argument("--split", action="store_true",
                    help="frame split across the ranks (tile subsets + gather, strong scaling) instead of replicas")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=60.0)
    ap.add_argument("--no-serve", action="store_true", help="skip the served/batch sections")
    ap.add_argument("--serve", action="store_true", help="only the Poisson serving benchmark")
    ap.add_argument("--requests", type=int, default=10000)
    ap.add_argument("--sweep", action="store_true", help="only the march steps x max_iter detail sweep")
    ap.add_argument("--voxel", action="store_true", help="only the voxel occupancy grid benchmark")
    ap.add_argument("--de", action="store_true", help="only the sphere-tracing vs march comparison")
    ap.add_argument("--precision-report", action="store_true",
                    help="only the FP32 / recheck / FP64 comparison on the workload frames")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "dqj":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    world, rank, local = dist_init()
    if args.impl == "reference":
        rc = run_reference(args, world, rank)
    elif args.serve:
        rc = run_serve_only(args, world, rank, local)
    elif args.precision_report:
        rc = run_precision_only(args, world, rank, local)
    elif args.sweep:
        rc = run_sweep_only(args, world, rank, local)
    elif args.voxel:
        rc = run_voxel_only(args, world, rank, local)
    elif args.de:
        rc = run_de_only(args, world, rank, local)
    elif args.split:
        rc = run_split(args, world, rank, local)
    else:
        rc = run_gpu(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
