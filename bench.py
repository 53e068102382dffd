#!/usr/bin/env python3
"""Benchmark: Range-Doppler compression of the 4096 x 4096 complex64 scene.

One step = one pass of the whole hot path over the scene through
sar_rda_process_oop: fused range compression with the corner turn folded into
its store (raw -> image), then the fused azimuth compression in place on
image -- two kernel launches through the C-ABI (three, raw -> work -> image,
on a plan that does not fold the corner turn).  The raw echo is never
modified, so every step does identical work; steps rotate over four raw
buffers, so each step's inputs and outputs (128 MiB read of raw, 128 MiB
image) exceed the 129 MB L2 and no step is served from L2.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
the host cores instead (the reference arm: a bounded sample of lines per step,
scaled to a whole scene).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (N > 1, torchrun): independent replicas, one scene stream per GPU.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

# 32 hardware work queues instead of 8, set before CUDA starts: the serving
# section runs one stream per in-flight request and size class, and stream
# priorities only order work on different queues (with 8, a small request can
# wait behind a large one queued ahead of it on a shared queue)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "4096² scene compress ms & HBM roofline fraction; p99 latency under mixed-size load"
WORKLOAD = "rda_4096x4096_c64_5targets_seed2"
N_AZ = N_RANGE = 4096
N_RAW_BUFFERS = 4


EXTRAS = ("passes", "scene_256", "pipelined", "az_major", "unfused", "precision", "rda_full", "long_lines",
          "any_length", "ragged_batch", "serving")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--e2e-scenes", type=int, default=16, help="scenes per sar_rda_process_host_n call (e2e)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--range-schedule", default=None, help="schedule of the range pass (default: autotuned)")
    ap.add_argument("--azimuth-schedule", default=None, help="schedule of the azimuth pass (default: autotuned)")
    ap.add_argument("--no-autotune", action="store_true", help="use the compiled-in preferred schedules")
    ap.add_argument("--no-extras", action="store_true", help="skip the ragged-batch and serving measurements")
    ap.add_argument("--ragged-strips", type=int, default=64,
                    help="strips of the ragged-batch section (64: the configuration; fewer for a small ncu case)")
    ap.add_argument("--extras", default=",".join(EXTRAS),
                    help="comma-separated extra measurements to run after the headline step")
    args = ap.parse_args()
    unknown = {x.strip() for x in args.extras.split(",") if x.strip()} - set(EXTRAS)
    if unknown:
        ap.error(f"unknown --extras {sorted(unknown)}; choose from {', '.join(EXTRAS)}")
    return args


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def hbm_peak():
    p = measured_peaks()
    if "hbm_gbs" in p:
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
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
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(init: bool = True):
    """Rank, world size and local rank from the torchrun environment; with
    more than one rank, join the process group (NCCL, or gloo when
    BENCH_BACKEND=gloo).  Replicas only: the group carries the start barrier
    and the max-over-ranks of the timings, never scene data."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and init:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend())
    return rank, world, local


def backend() -> str:
    return "gloo" if os.environ.get("BENCH_BACKEND", "nccl") == "gloo" else "nccl"


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(ms_step_max: float, world: int) -> float:
    """Whole-job time per scene: every rank finishes one scene per step, so
    `world` scenes complete every (max over ranks) step time."""
    return ms_step_max / world


# ---------------------------------------------------------------------------
# the oracle on the host cores (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

def oracle_scene_ms(raw, Hr, Ha, lines: int, nthreads: int) -> float:
    """Time the oracle on `lines` range lines + `lines` azimuth lines of the
    scene (plus the corner turn of that share) and scale to one whole scene."""
    import numpy as np
    import oracle
    o = oracle.default()
    rows = raw[:lines].astype(np.complex128)
    t0 = time.perf_counter()
    rc = o.compress_lines(rows, Hr, nthreads=nthreads)
    t1 = time.perf_counter()
    ct = o.corner_turn(rc)                              # lines x 4096 -> 4096 x lines
    t2 = time.perf_counter()
    az_in = np.zeros((lines, N_AZ), np.complex128)
    az_in[:, :lines] = ct[:lines]
    t3 = time.perf_counter()
    o.compress_lines(az_in, Ha, nthreads=nthreads)
    t4 = time.perf_counter()
    scale = N_AZ / lines
    return ((t1 - t0) + (t2 - t1) + (t4 - t3)) * scale * 1e3


def cpu_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def reference_arm(args, rank, world):
    if rank != 0:
        return
    import numpy as np
    import sarsim
    import oracle
    spec = sarsim.scene_4096()
    raw = sarsim.echo(spec)
    o = oracle.default()
    Hr = o.matched_filter(N_RANGE, sarsim.lfm_chirp(*spec.range_chirp))
    Ha = o.matched_filter(N_AZ, sarsim.lfm_chirp(*spec.az_chirp))
    nth = cpu_threads()
    # size the per-step sample so the whole run stays within ~3 minutes
    probe = oracle_scene_ms(raw, Hr, Ha, nth, nth) / (N_AZ / nth)       # ms per line-pair
    budget_ms = 150e3 / max(1, args.steps + args.warmup)
    lines = int(max(1, min(N_AZ, budget_ms / max(probe, 1e-6))))
    if lines >= nth:
        lines = (lines // nth) * nth
    for _ in range(args.warmup):
        oracle_scene_ms(raw, Hr, Ha, lines, nth)
    per = [oracle_scene_ms(raw, Hr, Ha, lines, nth) for _ in range(args.steps)]
    v = statistics.mean(per)
    sample = (f"{lines} range lines + {lines} azimuth lines of 4096 per step (FP64 C oracle), "
              f"scaled x{N_AZ / lines:g} to one 4096x4096 scene")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n_az": N_AZ, "n_range": N_RANGE, "parallelism": "host threads"},
           "cpu_baseline": {"value": v, "unit": "ms", "cores": nth, "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# the 4096^2 scene's three passes timed separately (corner turn not folded)
# ---------------------------------------------------------------------------

def _median_ms(stream, fn, reps: int = 20, warm: int = 3) -> float:
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t = []
    for i in range(reps + warm):
        e0.record(stream)
        fn(i)
        e1.record(stream)
        e1.synchronize()
        if i >= warm:
            t.append(e0.elapsed_time(e1))
    t.sort()
    return t[len(t) // 2]


def passes_bench(sar, Hr, Ha, raws, work, image, stream) -> dict:
    """Range pass, corner turn and azimuth pass of the 4096^2 scene as three
    separate kernels (an unfolded plan), each the median of 20 launches over
    rotating inputs larger than L2; GB/s over 16 B per sample each."""
    plan = sar.sar_plan_create(N_RANGE, N_AZ, Hr, Ha, flags=sar.SAR_PLAN_UNFOLDED_CORNER_TURN)
    ms_r = _median_ms(stream, lambda i: sar.sar_range_compress_oop(plan, raws[i % len(raws)], work, stream))
    ms_c = _median_ms(stream, lambda i: sar.sar_corner_turn(plan, raws[i % len(raws)], image, stream))
    ms_a = _median_ms(stream, lambda i: sar.sar_azimuth_compress(plan, image, stream))
    plan.destroy()
    b = 16.0 * N_RANGE * N_AZ
    return {"range_pass_ms": ms_r, "corner_turn_ms": ms_c, "azimuth_pass_ms": ms_a,
            "range_pass_GBps": b / (ms_r * 1e-3) / 1e9, "corner_turn_GBps": b / (ms_c * 1e-3) / 1e9,
            "azimuth_pass_GBps": b / (ms_a * 1e-3) / 1e9, "sum_ms": ms_r + ms_c + ms_a}


# ---------------------------------------------------------------------------
# the 256 x 256 scene: per pass, end to end as one CUDA-graph launch, oracle
# ---------------------------------------------------------------------------

def scene_256_bench(sar, dev, stream, host_threads: int, graph_reps: int = 1000) -> dict:
    import numpy as np
    import torch
    import sarsim
    spec = sarsim.scene_256()
    n = 256
    raw_np = sarsim.echo(spec)
    raw = torch.from_numpy(raw_np).to(dev)
    Hr = torch.empty(n, dtype=torch.complex64, device=dev)
    Ha = torch.empty(n, dtype=torch.complex64, device=dev)
    sar.sar_make_lfm_spectrum(n, *spec.range_chirp, Hr, stream)
    sar.sar_make_lfm_spectrum(n, *spec.az_chirp, Ha, stream)
    stream.synchronize()
    work, image = torch.empty_like(raw), torch.empty_like(raw)
    plan = sar.sar_plan_create(n, n, Hr, Ha)
    flat = sar.sar_plan_create(n, n, Hr, Ha, flags=sar.SAR_PLAN_UNFOLDED_CORNER_TURN)
    out = {"folded": sar.sar_plan_folds_corner_turn(plan)}
    us = lambda fn: 1e3 * _median_ms(stream, fn)
    if out["folded"]:
        out["range_pass_with_corner_turn_us"] = us(lambda i: sar.sar_range_compress_ct(plan, raw, image, stream))
    out["range_pass_us"] = us(lambda i: sar.sar_range_compress_oop(flat, raw, work, stream))
    out["corner_turn_us"] = us(lambda i: sar.sar_corner_turn(flat, work, image, stream))
    out["azimuth_pass_us"] = us(lambda i: sar.sar_azimuth_compress(flat, image, stream))
    # end to end: the whole scene as one CUDA-graph launch
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        sar.sar_rda_process_oop(plan, raw, work, image, stream)      # warm (tables, attributes)
        stream.synchronize()
        with torch.cuda.graph(g, stream=stream, capture_error_mode="relaxed"):
            sar.sar_rda_process_oop(plan, raw, work, image, stream)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(10):
        g.replay()
    e0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(graph_reps):
            g.replay()
    e1.record(stream)
    e1.synchronize()
    out["graph_us_per_scene"] = 1e3 * e0.elapsed_time(e1) / graph_reps
    plan.destroy()
    flat.destroy()
    if host_threads:
        import oracle
        o = oracle.default()
        Hr64 = o.matched_filter(n, sarsim.lfm_chirp(*spec.range_chirp))
        Ha64 = o.matched_filter(n, sarsim.lfm_chirp(*spec.az_chirp))
        for label, nth in (("oracle_ms_1_thread", 1), ("oracle_ms_all_threads", host_threads)):
            t = []
            for _ in range(5):
                t0 = time.perf_counter()
                o.rda(raw_np, Hr64, Ha64, nthreads=nth)
                t.append((time.perf_counter() - t0) * 1e3)
            out[label] = sorted(t)[2]
        out["oracle_threads"] = host_threads
    return out


# ---------------------------------------------------------------------------
# two scenes in flight: the range pass of scene k+1 beside the azimuth pass of k
# ---------------------------------------------------------------------------

def pipelined_bench(sar, plan, raws, image, dev, sequential_ms: float, scenes: int = 400) -> dict:
    """Throughput with consecutive scenes overlapped on two streams: the folded
    range pass of scene k+1 (stream A) runs beside the azimuth pass of scene k
    (stream B); two image buffers, events order each buffer's reuse.  Both
    passes are issue- or latency-bound rather than HBM-bound, so running them
    side by side fills issue slots each leaves idle.  Amortised time per
    scene; the headline value is one scene's latency."""
    import torch
    sa, sb = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    images = [image, torch.empty_like(image)]
    done = [torch.cuda.Event(), torch.cuda.Event()]     # azimuth pass finished with images[i]
    ready = [torch.cuda.Event(), torch.cuda.Event()]    # range pass filled images[i]
    for d in done:
        d.record(sb)

    def run(k):
        i = k % 2
        sa.wait_event(done[i])
        sar.sar_range_compress_ct(plan, raws[k % len(raws)], images[i], sa)
        ready[i].record(sa)
        sb.wait_event(ready[i])
        sar.sar_azimuth_compress(plan, images[i], sb)
        done[i].record(sb)

    for k in range(8):
        run(k)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(sa)
    sb.wait_event(t0)
    for k in range(scenes):
        run(k)
    sa.wait_stream(sb)
    t1.record(sa)
    t1.synchronize()
    ms = t0.elapsed_time(t1) / scenes
    return {"ms_per_scene": ms, "scenes": scenes, "sequential_ms_per_scene": sequential_ms,
            "speedup": sequential_ms / ms, "path_GBps_folded": 536870912 / (ms * 1e-3) / 1e9,
            "note": "amortised over consecutive scenes, two in flight on two streams (range pass of k+1 beside "
                    "the azimuth pass of k); inputs larger than L2 (rotating raw buffers)"}


# ---------------------------------------------------------------------------
# azimuth-major output: the fourth pass, timed separately
# ---------------------------------------------------------------------------

def az_major_bench(sar, Hr, Ha, raw, work, image, stream, reps: int = 50) -> dict:
    """The scene through sar_rda_process_oop with and without
    SAR_PLAN_OUT_AZ_MAJOR (the transpose back to [n_az][n_range]), and the
    transpose alone; medians of `reps`."""
    import torch
    out = torch.empty_like(work)

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t = []
        for i in range(reps + 3):
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            if i >= 3:
                t.append(e0.elapsed_time(e1))
        t.sort()
        return t[len(t) // 2]

    std = sar.sar_plan_create(N_RANGE, N_AZ, Hr, Ha)
    maj = sar.sar_plan_create(N_RANGE, N_AZ, Hr, Ha, flags=sar.SAR_PLAN_OUT_AZ_MAJOR)
    ms_std = timed(lambda: sar.sar_rda_process_oop(std, raw, work, image, stream))
    ms_maj = timed(lambda: sar.sar_rda_process_oop(maj, raw, work, out, stream))
    ms_t = timed(lambda: sar.sar_transpose(N_RANGE, N_AZ, image, out, stream))
    std.destroy()
    maj.destroy()
    return {"ms_per_scene_range_major": ms_std, "ms_per_scene_az_major": ms_maj, "fourth_pass_ms": ms_t,
            "fourth_pass_GBps": 2 * 8 * N_RANGE * N_AZ / (ms_t * 1e-3) / 1e9}


# ---------------------------------------------------------------------------
# the unfused comparison pipeline (paper Table II's baseline, on the GPU)
# ---------------------------------------------------------------------------

def unfused_bench(sar, plan, raw, work, image, stream, fused_ms: float, reps: int = 50) -> dict:
    import torch
    times = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for i in range(reps + 3):
        work.copy_(raw)                     # the unfused path compresses raw in place: restore it (untimed)
        e0.record(stream)
        sar.sar_rda_process_unfused(plan, work, image, stream)
        e1.record(stream)
        e1.synchronize()
        if i >= 3:
            times.append(e0.elapsed_time(e1))
    times.sort()
    ms = times[len(times) // 2]
    return {"ms_per_scene": ms, "kernels_per_scene": 7, "fusion_speedup": ms / fused_ms,
            "note": "per pass: FFT kernel, spectrum-multiply kernel, IFFT kernel (6 transfers per line), plus "
                    "the corner turn; median of 50 scenes, raw restored outside the timed events"}


# ---------------------------------------------------------------------------
# split-precision tensor-core variants on the same scene
# ---------------------------------------------------------------------------

def precision_bench(sar, Hr, Ha, raw, work, image, stream, reps: int = 50) -> dict:
    """Time the 4096^2 scene with each split-precision plan (three kernels:
    range pass, corner turn, azimuth pass) on both tensor-core engines
    (tcgen05.mma with TMEM accumulators, the default; warp-level mma.sync),
    and the FP32 plan through the same unfolded path; the images are compared
    with the FP32 image here and with the FP64 oracle in
    tests/test_gpu_parity.py."""
    import torch
    out = {}
    ref = None
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(plan):
        times = []
        for i in range(reps + 3):
            e0.record(stream)
            sar.sar_rda_process_oop(plan, raw, work, image, stream)
            e1.record(stream)
            e1.synchronize()
            if i >= 3:
                times.append(e0.elapsed_time(e1))
        times.sort()
        return times[len(times) // 2]

    for name in ("FP32", "FP16X2", "BF16X2", "BF16X3"):
        code = getattr(sar, "SAR_PREC_" + name)
        plan = sar.sar_plan_create(N_RANGE, N_AZ, Hr, Ha, precision=code, flags=sar.SAR_PLAN_UNFOLDED_CORNER_TURN)
        engines = (("tcgen05_tmem_a", 0), ("tcgen05_smem_a", 2), ("mma_sync", 1)) if name != "FP32" else (("fp32", 0),)
        row = {}
        for ename, eng in engines:
            sar.sar_set_split_engine(eng)
            try:
                ms = timed(plan)
                sar.sar_plan_status(plan, stream)
            finally:
                sar.sar_set_split_engine(0)
            img = image.clone()
            if ref is None:
                ref = img
            diff = float(torch.linalg.vector_norm(img - ref) / torch.linalg.vector_norm(ref))
            row[ename] = {"ms_per_scene": ms, "rel_l2_vs_fp32_path": diff}
        out[name] = row if name != "FP32" else row["fp32"]
        plan.destroy()
    out["note"] = ("unfolded three-kernel path for every precision; the error against the FP64 oracle "
                   "is checked by the parity tests")
    return out


# ---------------------------------------------------------------------------
# lines longer than one block's shared memory (thread-block clusters)
# ---------------------------------------------------------------------------

def long_lines_bench(sar, stream, peak, reps: int = 10) -> dict:
    """Fused pass (FFT, x H, IFFT per line) over 384 MiB of lines of 32768,
    65536 and 131072 samples, every cluster schedule timed by the native
    autotuner (median of `reps` launches); GB/s over 16 B per sample."""
    out = {}
    for n in (32768, 65536, 131072):
        n_lines = (384 << 20) // (8 * n)
        best, best_ms, all_ms = sar.sar_autotune(n, n_lines, reps=reps, stream=stream)
        gbs = {k: 16.0 * n * n_lines / (ms * 1e-3) / 1e9 for k, ms in all_ms.items()}
        out[str(n)] = {"lines": n_lines, "best": best["name"], "ms": best_ms,
                       "gb_s": gbs[best["name"]], "frac_hbm": gbs[best["name"]] / peak,
                       "all_gb_s": {k: round(v, 1) for k, v in sorted(gbs.items(), key=lambda x: -x[1])}}
    return out


# ---------------------------------------------------------------------------
# line lengths that are not powers of two (zero-padded linear convolution)
# ---------------------------------------------------------------------------

def any_length_bench(sar, dev, stream, peak, reps: int = 20) -> dict:
    """The fused range pass over about 384 MiB of lines of n samples for
    lengths that are not powers of two -- the mixed-radix engine at n itself
    where n's prime factors are 2, 3, 5, 7 (1000, 3000, 5000, 8000), the
    zero-padded convolution at L = next pow2 >= 2n - 1 otherwise (1009,
    3001) -- beside the power-of-two lengths around them; GB/s over 16 B per
    sample of n (one read and one write)."""
    import torch
    out = {}
    for n in (1000, 1009, 1024, 3000, 3001, 4096, 5000, 8000, 8192):
        n_lines = 1 << max(8, ((384 << 20) // (8 * n) - 1).bit_length())
        data = torch.zeros((n_lines, n), dtype=torch.complex64, device=dev)
        Hr = torch.ones(n, dtype=torch.complex64, device=dev)
        Ha = torch.ones(n_lines, dtype=torch.complex64, device=dev)
        plan = sar.sar_plan_create(n, n_lines, Hr, Ha)
        sched = sar.sar_plan_get_schedules(plan)[0]
        L = sched["n"]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        times = []
        for i in range(reps + 3):
            e0.record(stream)
            sar.sar_range_compress(plan, data, stream)
            e1.record(stream)
            e1.synchronize()
            if i >= 3:
                times.append(e0.elapsed_time(e1))
        times.sort()
        ms = times[len(times) // 2]
        gbs = 16.0 * n * n_lines / (ms * 1e-3) / 1e9
        out[str(n)] = {"engine_length": L, "schedule": sched["name"], "lines": n_lines, "ms": ms, "gb_s": gbs,
                       "frac_hbm": gbs / peak}
        plan.destroy()
        # the DFT alone at the same length (mixed radix at 7-smooth n, Bluestein at other non-powers of two)
        times = []
        for i in range(reps + 3):
            e0.record(stream)
            sar.sar_fft_lines(n, n_lines, data, data, False, stream)
            e1.record(stream)
            e1.synchronize()
            if i >= 3:
                times.append(e0.elapsed_time(e1))
        times.sort()
        out[str(n)]["fft_gb_s"] = 16.0 * n * n_lines / (times[len(times) // 2] * 1e-3) / 1e9
        del data
    # whole scenes at 7-smooth range lengths: the range pass with the corner
    # turn folded in (mixed radix) and the azimuth pass, against the three
    # separate kernels; two rotating raw buffers, ms per scene over 20 scenes
    scenes = {}
    for n_range, n_az in ((3000, 3000), (5000, 5000), (1000, 16384)):
        Hr = torch.ones(n_range, dtype=torch.complex64, device=dev)
        Ha = torch.ones(n_az, dtype=torch.complex64, device=dev)
        raws = [torch.randn(n_az, n_range, dtype=torch.complex64, device=dev) for _ in range(2)]
        work = torch.empty(n_az, n_range, dtype=torch.complex64, device=dev)
        img = torch.empty(n_range, n_az, dtype=torch.complex64, device=dev)
        torch.cuda.synchronize()
        row = {}
        for key, flags in (("folded", 0), ("unfolded", sar.SAR_PLAN_UNFOLDED_CORNER_TURN)):
            plan = sar.sar_plan_create(n_range, n_az, Hr, Ha, flags=flags)
            for i in range(3):
                sar.sar_rda_process_oop(plan, raws[i % 2], work, img, stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for i in range(20):
                sar.sar_rda_process_oop(plan, raws[i % 2], work, img, stream)
            e1.record(stream)
            e1.synchronize()
            row[key + "_ms"] = e0.elapsed_time(e1) / 20
            row[key + "_plan_folds"] = bool(sar.sar_plan_folds_corner_turn(plan))
            plan.destroy()
        gbs = 32.0 * n_range * n_az / (row["folded_ms"] * 1e-3) / 1e9
        row.update({"folded_gb_s_32B": gbs, "folded_frac_hbm_32B": gbs / peak})
        scenes[f"{n_range}x{n_az}"] = row
        del raws, work, img
    out["scenes"] = scenes
    out["scenes_note"] = ("range x azimuth; GB/s over 32 B per sample (the folded range pass and the azimuth pass); "
                          "unfolded: range pass, corner turn, azimuth pass")
    return out


# ---------------------------------------------------------------------------
# full Range-Doppler processing with RCMC on a migration scene
# ---------------------------------------------------------------------------

def rda_full_bench(sar, dev, stream, work, image, reps: int = 50) -> dict:
    import torch
    import sarsim
    tg, rc, ap, geo, snr, seed = sarsim.migration_scene_4096()
    raw = torch.from_numpy(sarsim.echo_migration(N_AZ, N_RANGE, tg, rc, ap, geo, snr, seed)).to(dev)
    Hr = torch.empty(N_RANGE, dtype=torch.complex64, device=dev)
    sar.sar_make_lfm_spectrum(N_RANGE, *rc, Hr, stream)
    stream.synchronize()
    plan = sar.sar_plan_create(N_RANGE, N_AZ, Hr, Hr)
    sar.sar_plan_set_geometry(plan, *geo.as_tuple(), 16)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    for i in range(reps + 3):
        e0.record(stream)
        sar.sar_rda_full(plan, raw, work, image, stream)
        e1.record(stream)
        e1.synchronize()
        if i >= 3:
            times.append(e0.elapsed_time(e1))
    times.sort()
    ms = times[len(times) // 2]
    # RCMC alone on the range-Doppler image the azimuth FFT left in `image`
    # (the input and output, 2 x 134 MB, exceed L2)
    rc = []
    for i in range(reps + 3):
        e0.record(stream)
        sar.sar_rcmc(plan, image, work, stream)
        e1.record(stream)
        e1.synchronize()
        if i >= 3:
            rc.append(e0.elapsed_time(e1))
    rc.sort()
    rc_ms = rc[len(rc) // 2]
    plan.destroy()
    return {"ms_per_scene": ms, "rcmc_ms": rc_ms, "rcmc_GBps": 2 * 8 * N_AZ * N_RANGE / rc_ms / 1e6,
            "kernels_per_scene": 4 if sar.sar_plan_folds_corner_turn else 5,
            "steps": "range compression + corner turn, azimuth FFT, RCMC (16-tap Hann sinc), "
                     "range-dependent azimuth filter + IFFT",
            "geometry": {"kappa": geo.kappa, "v_s": geo.v_s, "r_near": geo.r_near, "aperture_lines": ap}}


# ---------------------------------------------------------------------------
# ragged batch: 64 strips of mixed sizes in one CUDA-graph launch
# ---------------------------------------------------------------------------

def ragged_batch_bench(sar, roofline, dev, stream, peak, reps: int = 10, strips_n: int = 64) -> dict:
    import torch
    import sarsim
    specs = sarsim.ragged_batch_specs(4, strips_n)
    hr, ha, strips, keep = {}, {}, [], []
    with torch.cuda.stream(stream):
        for sp in specs:
            if sp.n_range not in hr:
                hr[sp.n_range] = torch.empty(sp.n_range, dtype=torch.complex64, device=dev)
                sar.sar_make_lfm_spectrum(sp.n_range, *sp.range_chirp, hr[sp.n_range], stream)
            if sp.l_az not in ha:
                ha[sp.l_az] = torch.empty(sp.l_az, dtype=torch.complex64, device=dev)
                sar.sar_make_lfm_spectrum(sp.l_az, *sp.az_chirp, ha[sp.l_az], stream)
            raw = torch.empty((sp.n_az, sp.n_range), dtype=torch.complex64, device=dev)
            sar.sar_simulate_echo(sp.n_az, sp.n_range, sp.targets, sp.range_chirp, sp.az_chirp, sp.snr_db, sp.seed,
                                  raw, stream)
            img = torch.empty((sp.n_range, sp.n_az), dtype=torch.complex64, device=dev)
            strips.append(dict(n_range=sp.n_range, n_az=sp.n_az, raw=raw, image=img, range_spectrum=hr[sp.n_range],
                               az_spectrum=ha[sp.l_az]))
            keep.append((raw, img))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(batch):
        for _ in range(2):
            sar.sar_batch_run(batch, stream)
        torch.cuda.synchronize()
        times = []
        for _ in range(reps):
            e0.record(stream)
            sar.sar_batch_run(batch, stream)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        times.sort()
        return times[len(times) // 2]

    # the default: one persistent kernel, corner turn folded into the range items
    batch = sar.sar_batch_create(strips)
    info = sar.sar_batch_info(batch)
    ms = timed(batch)
    sar.sar_batch_status(batch, stream)
    batch.destroy()
    alg = sum(roofline.rda_bytes_folded(sp.n_az, sp.n_range) for sp in specs)   # 32 B per sample
    alg48 = sum(roofline.rda_bytes(sp.n_az, sp.n_range) for sp in specs)
    gbs = alg / (ms * 1e-3) / 1e9
    # the multi-kernel graph (one launch per class, batched corner turn)
    mbatch = sar.sar_batch_create(strips, flags=sar.SAR_BATCH_MULTI_KERNEL)
    minfo = sar.sar_batch_info(mbatch)
    mms = timed(mbatch)
    mbatch.destroy()
    # the same strips with their azimuth lines compressed at exactly n_az
    # (SAR_BATCH_EXACT_AZIMUTH; azimuth spectra of n_az values)
    hx = {}
    with torch.cuda.stream(stream):
        for st, sp in zip(strips, specs):
            key = (sp.n_az, sp.az_chirp)
            if key not in hx:
                hx[key] = torch.empty(sp.n_az, dtype=torch.complex64, device=dev)
                sar.sar_make_lfm_spectrum(sp.n_az, min(sp.az_chirp[0], sp.n_az), sp.az_chirp[1], hx[key], stream)
            st["az_spectrum"] = hx[key]
    torch.cuda.synchronize()
    xbatch = sar.sar_batch_create(strips, flags=sar.SAR_BATCH_EXACT_AZIMUTH)
    xinfo = sar.sar_batch_info(xbatch)
    for _ in range(2):
        sar.sar_batch_run(xbatch, stream)
    xt = []
    for _ in range(reps):
        e0.record(stream)
        sar.sar_batch_run(xbatch, stream)
        e1.record(stream)
        e1.synchronize()
        xt.append(e0.elapsed_time(e1))
    xt.sort()
    xms = xt[len(xt) // 2]
    xbatch.destroy()
    return {"strips": info["strips"], "samples": info["samples"], "ms_per_graph_launch": ms,
            "kernels_per_graph": info["kernels_per_run"], "range_classes": info["range_classes"],
            "azimuth_classes": info["azimuth_classes"], "algorithmic_bytes": alg,
            "achieved_GBps": gbs, "frac_of_hbm_peak": gbs / peak,
            "bytes_note": "32 B per unpadded sample (range pass with the corner turn folded in, azimuth pass)",
            "inputs": f"{len(specs)} seeded strips (sarsim.ragged_batch_specs(4, {len(specs)})), echoes by the device simulator",
            "multi_kernel": {"ms_per_graph_launch": mms, "kernels_per_graph": minfo["kernels_per_run"],
                             "algorithmic_bytes": alg48, "achieved_GBps": alg48 / (mms * 1e-3) / 1e9,
                             "frac_of_hbm_peak": alg48 / (mms * 1e-3) / 1e9 / peak,
                             "note": "SAR_BATCH_MULTI_KERNEL: one launch per class and a batched corner turn, "
                                     "48 B per unpadded sample"},
            "exact_azimuth": {"ms_per_graph_launch": xms, "kernels_per_graph": xinfo["kernels_per_run"],
                              "azimuth_classes": xinfo["azimuth_classes"],
                              "achieved_GBps": alg48 / (xms * 1e-3) / 1e9,
                              "note": "SAR_BATCH_EXACT_AZIMUTH: circular correlation at each strip's n_az"}}


# ---------------------------------------------------------------------------
# serving: Poisson stream of mixed-size scenes through the request loop
# ---------------------------------------------------------------------------

def serving_bench(sar, dev, stream, n_requests: int = 2000, budget_gib: int = 120, max_inflight: int = 32) -> dict:
    import numpy as np
    import torch
    import sarsim
    variants = 2
    classes = []
    with torch.cuda.stream(stream):
        for size in sarsim.SERVING_SIZES:
            for v in range(variants):
                sp = sarsim.serving_scene(size, v)
                pool = torch.empty((size, size), dtype=torch.complex64, device=dev)
                sar.sar_simulate_echo(size, size, sp.targets, sp.range_chirp, sp.az_chirp, sp.snr_db, sp.seed, pool,
                                      stream)
                hr = torch.empty(size, dtype=torch.complex64, device=dev)
                ha = torch.empty(size, dtype=torch.complex64, device=dev)
                sar.sar_make_lfm_spectrum(size, *sp.range_chirp, hr, stream)
                sar.sar_make_lfm_spectrum(size, *sp.az_chirp, ha, stream)
                classes.append(dict(n_range=size, n_az=size, pool=pool, range_spectrum=hr, az_spectrum=ha))
    torch.cuda.synchronize()
    draws = sarsim.serving_requests(5, n_requests, variants)
    cls = [k * variants + v for k, v in draws]
    size_of = [classes[c]["n_range"] for c in cls]

    def loads(srv, sat) -> dict:
        res_out = {}
        for load in (0.5, 0.9):
            arrivals = sarsim.poisson_arrivals(5 + int(load * 10), n_requests, load * sat)
            res = sar.sar_server_run(srv, [(float(t), c) for t, c in zip(arrivals, cls)],
                                     mode=sar.SAR_SERVE_OPEN_LOOP)
            if any(r["status"] != 0 for r in res):
                raise RuntimeError("a served request failed")
            lat = np.array([r["latency_s"] for r in res]) * 1e3
            span = max(r["done_s"] for r in res) - float(arrivals[0])
            by_size = {f"{n}^2": float(np.percentile([x for x, m in zip(lat, size_of) if m == n], 99))
                       for n in sarsim.SERVING_SIZES if n in size_of}
            res_out[f"load_{int(load * 100)}pct"] = {
                "offered_scenes_per_s": load * sat, "achieved_scenes_per_s": n_requests / span,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "max_ms": float(lat.max()), "p99_ms_by_size": by_size}
        return res_out

    # the served configuration: smaller scenes on higher-priority streams
    out_env = {"CUDA_DEVICE_MAX_CONNECTIONS": os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS")}
    srv = sar.sar_server_create(classes, hbm_budget_bytes=budget_gib << 30, max_inflight=max_inflight,
                                size_priority=True)
    sar.sar_server_run(srv, [(0.0, c) for c in cls[:64]], mode=sar.SAR_SERVE_CLOSED_LOOP)     # warm-up
    res = sar.sar_server_run(srv, [(0.0, c) for c in cls], mode=sar.SAR_SERVE_CLOSED_LOOP)
    makespan = max(r["done_s"] for r in res)
    sat = n_requests / makespan
    mean_bytes = float(np.mean([classes[c]["n_range"] * classes[c]["n_az"] * 8 for c in cls]))
    # each size class served alone (closed loop, same slots and budget): its
    # ms per scene, and the throughput the mix would reach if its scenes ran
    # one class after another at those rates (no cross-class overlap)
    alone = {}
    for k, size in enumerate(sarsim.SERVING_SIZES):
        reps = max(4, int(64 * (2048 / size) ** 2))
        r1 = sar.sar_server_run(srv, [(0.0, k * variants)] * reps, mode=sar.SAR_SERVE_CLOSED_LOOP)
        alone[f"{size}^2"] = 1e3 * max(r["done_s"] for r in r1) / reps
    serial_ms = sum(p * alone[f"{n}^2"] for n, p in zip(sarsim.SERVING_SIZES, sarsim.SERVING_MIX))
    out = {"requests": n_requests, "size_mix": dict(zip([f"{n}^2" for n in sarsim.SERVING_SIZES],
                                                        sarsim.SERVING_MIX)),
           "hbm_budget_GiB": budget_gib, "max_inflight": max_inflight, "mean_scene_MiB": mean_bytes / 2 ** 20,
           "size_priority": True, "aging_s": 0.0, "env": out_env,
           "saturation_scenes_per_s": sat,
           "alone_ms_per_scene": alone,
           "mix_of_alone_rates_scenes_per_s": 1e3 / serial_ms,
           "traffic_note": "per scene 48 B per sample: the ingest copy (16) and the folded two-pass compression (32)",
           "saturation_latency_ms": {"p50": float(np.percentile([r["latency_s"] for r in res], 50) * 1e3),
                                     "p99": float(np.percentile([r["latency_s"] for r in res], 99) * 1e3)}}
    out.update(loads(srv, sat))
    srv.destroy()
    # the same offered loads with every request at one stream priority
    srv = sar.sar_server_create(classes, hbm_budget_bytes=budget_gib << 30, max_inflight=max_inflight)
    sar.sar_server_run(srv, [(0.0, c) for c in cls[:64]], mode=sar.SAR_SERVE_CLOSED_LOOP)
    out["one_priority"] = loads(srv, sat)
    srv.destroy()
    out["inputs"] = ("pool scenes by the device simulator (sarsim.serving_scene, 2 variants per size), "
                     "requests sarsim.serving_requests(5, n), Poisson arrivals sarsim.poisson_arrivals")
    return out


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def main():
    args = parse()
    if args.impl == "reference":
        # the oracle runs on the host of rank 0 only; other ranks exit at once
        rank, world, _ = dist_setup(init=False)
        reference_arm(args, rank, world)
        return
    rank, world, local = dist_setup()
    assert args.warmup >= 3, "at least 3 warm-up steps"
    import numpy as np
    import torch
    import sarsim
    import paper_2604_03585_gb300 as sar
    from paper_2604_03585_gb300 import roofline

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    spec = sarsim.scene_4096()
    raw_h = torch.from_numpy(sarsim.echo(spec)).pin_memory()
    with torch.cuda.stream(stream):
        Hr = torch.empty(N_RANGE, dtype=torch.complex64, device=dev)
        Ha = torch.empty(N_AZ, dtype=torch.complex64, device=dev)
        sar.sar_make_lfm_spectrum(N_RANGE, *spec.range_chirp, Hr, stream)
        sar.sar_make_lfm_spectrum(N_AZ, *spec.az_chirp, Ha, stream)
        stream.synchronize()
        if not args.no_autotune and (args.range_schedule is None or args.azimuth_schedule is None):
            # what each pass will run: the azimuth lines through the fused
            # kernel, the range lines through the folded range + corner turn
            sar.sar_autotune(N_AZ, N_RANGE * 3, reps=5, stream=stream)    # 384 MiB per timed launch
            sar.sar_autotune(N_RANGE, N_AZ, reps=5, stream=stream, kind=sar.SAR_TUNE_RANGE_CT)
        plan = sar.sar_plan_create_ex(N_RANGE, N_AZ, Hr, Ha, range_schedule=args.range_schedule,
                                      az_schedule=args.azimuth_schedule)
        sched_r, sched_a = sar.sar_plan_get_schedules(plan)
        raws = [raw_h.to(dev, non_blocking=False) for _ in range(N_RAW_BUFFERS)]
        work = torch.empty((N_AZ, N_RANGE), dtype=torch.complex64, device=dev)
        image = torch.empty((N_RANGE, N_AZ), dtype=torch.complex64, device=dev)
    torch.cuda.synchronize()

    folded = sar.sar_plan_folds_corner_turn(plan)

    def step(i, ev=None):
        r = raws[i % N_RAW_BUFFERS]
        if ev is not None:
            ev[0].record(stream)
        if folded:      # range compression writes the corner-turned image itself
            sar.sar_range_compress_ct(plan, r, image, stream)
            if ev is not None:
                ev[1].record(stream)
        else:
            sar.sar_range_compress_oop(plan, r, work, stream)
            if ev is not None:
                ev[1].record(stream)
            sar.sar_corner_turn(plan, work, image, stream)
            if ev is not None:
                ev[2].record(stream)
        sar.sar_azimuth_compress(plan, image, stream)
        if ev is not None:
            ev[3].record(stream)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()

    K = args.steps
    # per-kernel CUDA events on every EV_EVERY-th step of the timed region
    # only: an event between two kernels delays the second by about a
    # microsecond, so events on every step would inflate the step time
    EV_EVERY = 16
    evs = {i: [torch.cuda.Event(enable_timing=True) for _ in range(4)] for i in range(0, K, EV_EVERY)}
    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.05)
    for i in range(2):   # the GPU idled through the sleep: back to speed before the timed region
        step(i)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for i in range(K):
        step(i, evs.get(i))
    t_end.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(world)
    total_ms = t_start.elapsed_time(t_end)
    total_ms = allmax(total_ms, world)
    ms_step = total_ms / K
    per = {"range_pass": [], "corner_turn": [], "azimuth_pass": []}
    for e in evs.values():
        per["range_pass"].append(e[0].elapsed_time(e[1]))
        if folded:
            per["azimuth_pass"].append(e[1].elapsed_time(e[3]))
        else:
            per["corner_turn"].append(e[1].elapsed_time(e[2]))
            per["azimuth_pass"].append(e[2].elapsed_time(e[3]))
    kern_ms = {k: statistics.mean(v) for k, v in per.items() if v}
    if folded:
        kern_ms["range_pass+corner_turn"] = kern_ms.pop("range_pass")

    # e2e: the host-buffer entry point, copies inside the timed region
    img_h = torch.empty((N_RANGE, N_AZ), dtype=torch.complex64).pin_memory()
    for _ in range(3):                                        # staging buffers, streams, events: once
        sar.sar_rda_process_host(plan, raw_h, img_h, stream)
    barrier(world)
    KE = max(3, args.e2e_steps)
    e2e_calls = []
    for _ in range(KE):
        t0 = time.perf_counter()
        sar.sar_rda_process_host(plan, raw_h, img_h, stream)   # returns with the image in host memory
        e2e_calls.append((time.perf_counter() - t0) * 1e3)
    single_ms = allmax(statistics.median(e2e_calls), world)
    # a stream of scenes through one call: the echo of scene q + 1 travels in
    # while the image of scene q travels out (two echoes, the second the first
    # at half amplitude, and two images, alternating, all pinned; every
    # scene's copies inside the timed region)
    SN = max(2, args.e2e_scenes)
    raw_h2 = (raw_h * 0.5).pin_memory()
    img_h2 = torch.empty_like(img_h).pin_memory()
    raws_n = [raw_h if q % 2 == 0 else raw_h2 for q in range(SN)]
    imgs_n = [img_h if q % 2 == 0 else img_h2 for q in range(SN)]
    sar.sar_rda_process_host_n(plan, raws_n, imgs_n, stream)
    barrier(world)
    stream_calls = []
    for _ in range(max(3, KE // 4)):
        t0 = time.perf_counter()
        sar.sar_rda_process_host_n(plan, raws_n, imgs_n, stream)   # returns with every image in host memory
        stream_calls.append((time.perf_counter() - t0) * 1e3 / SN)
    e2e_ms = allmax(statistics.median(stream_calls), world)
    # the copies alone on this machine (pinned, one cudaMemcpyAsync each way), one
    # direction at a time (the floor of a single call) and both at once (the
    # floor of the stream)
    scratch = torch.empty_like(raw_h, device=dev)
    scratch2 = torch.empty_like(raw_h, device=dev)
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    copy_ms = {"h2d": [], "d2h": [], "both": []}
    for _ in range(5):
        t0 = time.perf_counter()
        scratch.copy_(raw_h, non_blocking=True)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        img_h.copy_(scratch, non_blocking=True)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        with torch.cuda.stream(s_in):
            scratch.copy_(raw_h, non_blocking=True)
        with torch.cuda.stream(s_out):
            img_h2.copy_(scratch2, non_blocking=True)
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        copy_ms["h2d"].append((t1 - t0) * 1e3)
        copy_ms["d2h"].append((t2 - t1) * 1e3)
        copy_ms["both"].append((t3 - t2) * 1e3)
    del scratch, scratch2
    floor = statistics.median(copy_ms["h2d"]) + statistics.median(copy_ms["d2h"])
    e2e_stats = {"scenes_per_call": SN, "calls": len(stream_calls),
                 "statistic": "median over calls of host wall time per call / scenes per call",
                 "copies_both_directions_ms": statistics.median(copy_ms["both"]),
                 "single_call": {"api": "sar_rda_process_host, one scene per call", "median_ms": single_ms,
                                 "mean_ms": statistics.mean(e2e_calls), "min_ms": min(e2e_calls),
                                 "max_ms": max(e2e_calls), "calls": KE,
                                 "copies_alone_ms": floor},
                 "h2d_GBps": raw_h.numel() * 8 / (statistics.median(copy_ms["h2d"]) * 1e-3) / 1e9,
                 "d2h_GBps": img_h.numel() * 8 / (statistics.median(copy_ms["d2h"]) * 1e-3) / 1e9}

    peak, peak_kind = hbm_peak()
    bytes_pass = roofline.fused_pass_bytes(N_AZ, N_RANGE)
    dominant = max(kern_ms, key=kern_ms.get)
    dom_ms = kern_ms[dominant]
    if dominant == "range_pass+corner_turn":
        traffic_key = "range_ct " + sched_r["name"]
    elif dominant == "range_pass":
        traffic_key = "fused " + sched_r["name"]
    elif dominant == "azimuth_pass":
        traffic_key = "fused " + sched_a["name"]
    else:
        traffic_key = None
    traffic = roofline.recorded_traffic(traffic_key, os.path.join(ROOT, "profiles")) if traffic_key else None
    achieved = bytes_pass / (dom_ms * 1e-3) / 1e9
    path_bytes = roofline.rda_bytes(N_AZ, N_RANGE)            # three passes, 48 B/sample
    path_gbs = path_bytes / (ms_step * 1e-3) / 1e9
    min_bytes = roofline.rda_bytes_folded(N_AZ, N_RANGE)     # corner turn folded, 32 B/sample

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        nth = cpu_threads()
        raw_np = raw_h.numpy()
        import oracle
        o = oracle.default()
        Hr64 = o.matched_filter(N_RANGE, sarsim.lfm_chirp(*spec.range_chirp))
        Ha64 = o.matched_filter(N_AZ, sarsim.lfm_chirp(*spec.az_chirp))
        lines = 512
        v = oracle_scene_ms(raw_np, Hr64, Ha64, lines, nth)
        v1 = oracle_scene_ms(raw_np, Hr64, Ha64, 64, 1)
        cpu = {"value": v, "unit": "ms", "cores": nth, "kind": "oracle",
               "sample": f"{lines} range + {lines} azimuth lines of the 4096x4096 scene (FP64 C oracle, "
                         f"{nth} threads), scaled x{N_AZ // lines} to one scene",
               "single_thread_ms": v1, "single_thread_sample": "64 + 64 lines, one thread, scaled x64",
               "nproc": os.cpu_count()}

    extras = {}
    wanted = set() if args.no_extras else {x.strip() for x in args.extras.split(",") if x.strip()}
    if "passes" in wanted:
        extras["passes"] = passes_bench(sar, Hr, Ha, raws, work, image, stream)
    if "scene_256" in wanted:
        extras["scene_256"] = scene_256_bench(sar, dev, stream, cpu_threads() if rank == 0 else 0)
    if "pipelined" in wanted and folded:
        extras["pipelined"] = pipelined_bench(sar, plan, raws, image, dev, ms_step)
    if "az_major" in wanted:
        extras["az_major"] = az_major_bench(sar, Hr, Ha, raws[0], work, image, stream)
    if "unfused" in wanted:
        extras["unfused"] = unfused_bench(sar, plan, raws[0], work, image, stream, ms_step)
    if "precision" in wanted:
        extras["precision"] = precision_bench(sar, Hr, Ha, raws[0], work, image, stream)
    if "rda_full" in wanted:
        extras["rda_full"] = rda_full_bench(sar, dev, stream, work, image)
    if "long_lines" in wanted:
        extras["long_lines"] = long_lines_bench(sar, stream, peak)
    if "any_length" in wanted:
        extras["any_length"] = any_length_bench(sar, dev, stream, peak)
    if "ragged_batch" in wanted:
        extras["ragged_batch"] = ragged_batch_bench(sar, roofline, dev, stream, peak, strips_n=args.ragged_strips)
    if "serving" in wanted:
        extras["serving"] = serving_bench(sar, dev, stream)

    value = job_value(ms_step, world)
    out = {
        "metric": METRIC, "value": value, "unit": "ms", "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_az": N_AZ, "n_range": N_RANGE, "parallelism": f"replicas{world}",
                   "l2": "inputs larger than L2: 4 rotating 128 MiB raw buffers; a step reads one (128 MiB) and writes and rereads the 128 MiB image",
                   "range_schedule": sched_r["name"], "azimuth_schedule": sched_a["name"]},
        "roofline": {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
                     "bytes_per_launch": bytes_pass,
                     "traffic_note": "ncu dram read+write per launch (profiles/ncu_traffic.json); writes still in "
                                     "L2 when the kernel ends are not counted"},
        "path_roofline": {"bytes_per_step": path_bytes, "achieved": path_gbs, "peak": peak, "unit": "GB/s",
                          "frac": path_gbs / peak, "bytes_note": "three passes at 16 B/sample each"},
        "path_roofline_folded": {"bytes_per_step": min_bytes,
                                 "achieved": min_bytes / (ms_step * 1e-3) / 1e9,
                                 "frac": min_bytes / (ms_step * 1e-3) / 1e9 / peak,
                                 "bytes_note": "corner turn folded into the range pass: 32 B/sample"},
        "corner_turn_folded": bool(folded),
        "kernels_ms": kern_ms,
        "gflops_convention": roofline.rda_flops(N_AZ, N_RANGE) / (ms_step * 1e-3) / 1e9,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": raw_h.numel() * 8,
                "d2h_bytes_per_step": img_h.numel() * 8,
                "api": "sar_rda_process_host_n, pinned host buffers: ms per scene of a stream of scenes",
                **e2e_stats},
        "gpu_launches": (2 if folded else 3) * K,
        **extras,
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    plan.destroy()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
