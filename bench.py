#!/usr/bin/env python3
"""Throughput benchmark of the analyzer hot path; prints one JSON line on rank 0.

Workload: 3840x2160 8-bit 4:2:0 synthetic video (seeded: 30% flat block-aligned area,
sinusoid texture of period 2-8 px, global pan), block size 32 with the low-pass option --
the all-optimisations mode of the paper's speed test (Section 3).  One step is one
vca_push_frames call over a batch of frames already resident in HBM (all seven features
of every frame, the h state update and the feature read-back).  The batch (64 frames,
796 MB) is larger than L2, so no step reads its inputs from cache.

`e2e` is the same metric through the same public call with pinned HOST frames: the
host-to-device copies and the device-to-host feature copy are inside the timed region.

Multi-GPU: the path shards by video (each channel keeps its own h state), so N ranks run
N independent analyzers on N batches (weak scaling, no collective on the data path);
the timing is the max over ranks.

--impl reference times the CPU oracle (the plain FP64 statement of the method) on the
host cores, on a bounded sample of the same workload.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "2160p 8-bit frames/sec (7 features), % of HBM roofline; p99 per-frame latency"
PAPER_FPS = 292.68  # paper, Section 3: VCA v2.0 with all optimisations on 8 CPU threads, UHD 8-bit
W, H = 3840, 2160
FRAME_BYTES = W * H + 2 * (W // 2) * (H // 2)  # 12,441,600 B per 8-bit 4:2:0 frame
KERNEL_SOURCES = ("paper_2304_12384_gb300/csrc/vca_tc.cu", "paper_2304_12384_gb300/csrc/vca_plain.cu",
                  "paper_2304_12384_gb300/csrc/vca_plain.cuh", "paper_2304_12384_gb300/csrc/vca_ptx.cuh",
                  "paper_2304_12384_gb300/csrc/vca_fixed.cuh")


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="vca", choices=["vca", "reference"])
    p.add_argument("--frames", type=int, default=64, help="frames per step (one push)")
    p.add_argument("--distinct", type=int, default=16, help="distinct synthetic frames tiled into the batch")
    p.add_argument("--kernel", default="auto", choices=["auto", "plain", "tc"])
    p.add_argument("--block-size", type=int, default=32)
    p.add_argument("--full", action="store_true", help="all coefficients instead of the low-pass subset")
    p.add_argument("--no-extras", action="store_true", help="skip variants, latency, e2e and cpu baseline")
    p.add_argument("--extras", default="all",
                   help="comma-separated subset of latency,e2e,variants,tune,siti,ladder,serving,cpu (default all)")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# CPU legs (oracle)
# ---------------------------------------------------------------------------

def oracle_fps(frames, cfg, budget_s):
    """Frames/s of the oracle on the host cores over a bounded sample; returns (fps, n)."""
    from oracle import frame_block_values, frame_features

    prev = None
    n = 0
    t0 = time.perf_counter()
    while True:
        y, u, v = frames[n % len(frames)]
        vals = frame_block_values(y, u, v, cfg)
        frame_features(vals, prev, cfg)
        prev = vals["H_Y"]
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s or n >= 200:
            return n / el, n


# Worker side of the all-cores oracle timing (a spawned process pool: the parent has used the GPU).
_POOL_FRAMES = None


def _pool_init(spec_args, cfg):
    global _POOL_FRAMES, _POOL_CFG
    from synth import frames_list, uhd_spec

    _POOL_FRAMES = frames_list(uhd_spec(*spec_args[:1], bit_depth=spec_args[1]), 0, spec_args[2])
    _POOL_CFG = cfg


def _pool_block_values(i):
    from oracle import frame_block_values

    y, u, v = _POOL_FRAMES[i % len(_POOL_FRAMES)]
    return frame_block_values(y, u, v, _POOL_CFG)


def oracle_fps_all_cores(cfg, budget_s, workers, distinct=2):
    """Frames/s of the oracle on `workers` processes: per-frame block values in parallel (the
    frames are generated in each worker, not sent), frame features in order in this process.
    Returns (fps, frames)."""
    import multiprocessing as mp

    from oracle import frame_features

    ctx = mp.get_context("spawn")
    with ctx.Pool(workers, initializer=_pool_init, initargs=((3, 8, distinct), cfg)) as pool:
        pool.map(_pool_block_values, range(workers))  # warm: imports and frame generation
        prev = None
        n = 0
        t0 = time.perf_counter()
        while True:
            for vals in pool.map(_pool_block_values, range(n, n + workers)):
                frame_features(vals, prev, cfg)
                prev = vals["H_Y"]
            n += workers
            el = time.perf_counter() - t0
            if el >= budget_s or n >= 400:
                return n / el, n


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import Config
    from synth import frames_list, uhd_spec

    lp = not args.full
    cfg = Config(W, H, 8, args.block_size, lp)
    cores = os.cpu_count() or 1
    per_step = max(1.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    times = []
    total_frames = 0
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        _, n = oracle_fps_all_cores(cfg, per_step if i >= args.warmup else 0.0, cores)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
            total_frames += n
    value = total_frames / sum(times)
    sample = (f"{total_frames} frames of 3840x2160 8-bit (2 distinct synthetic frames), w={args.block_size}, "
              f"low_pass={lp}, oracle frame_block_values on {cores} processes + frame_features in order")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": value / PAPER_FPS, "dtype": "int64",
        "data": "synthetic", "config": workload_config(args),
        "cpu_baseline": {"value": value, "unit": "frames/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------------------
# GPU legs
# ---------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, power, reasons = [], None, [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
                power.append(float(f[3]))
            except ValueError:
                continue
            for n, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


def workload_config(args):
    lp = not args.full
    return {"workload": f"3840x2160 8-bit 4:2:0 synthetic, block {args.block_size}, "
                        f"{'low-pass quarter' if lp else 'all coefficients'}, {args.frames} frames per push",
            "width": W, "height": H, "bit_depth": 8, "block_size": args.block_size, "low_pass": lp,
            "frames_per_step": args.frames,
            "l2": f"inputs larger than L2 ({args.frames * FRAME_BYTES / 1e6:.0f} MB per step, 129 MB L2)"}


def kernel_source_hash():
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel_name, block_size, low_pass):
    """DRAM bytes per frame of the analysis kernel from the committed ncu summary, if it was
    captured from the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "traffic_summary.txt")
    if not os.path.exists(path):
        return None
    want = kernel_source_hash()
    key = f"{kernel_name} w{block_size} lp{int(low_pass)}"
    with open(path) as f:
        for line in f:
            if line.startswith(key + " "):
                parts = dict(p.split("=", 1) for p in line.split()[3:] if "=" in p)
                if parts.get("source_hash") == want:
                    return float(parts["dram_bytes_per_frame"])
    return None


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def make_device_frames(args, device, bit_depth=8):
    import numpy as np
    import torch

    from synth import frames_list, pack_planes, uhd_spec

    frames = frames_list(uhd_spec(3, bit_depth=bit_depth), 0, args.distinct)
    pk = pack_planes(frames)
    tens = []
    for k in ("y", "u", "v"):
        a = pk[k]
        if a.dtype == np.uint16:
            a = a.view(np.int16)
        src = torch.from_numpy(np.ascontiguousarray(a))
        dst = torch.empty((args.frames,) + tuple(src.shape[1:]), dtype=src.dtype, device=device)
        for i in range(args.frames):
            dst[i].copy_(src[i % args.distinct])
        tens.append(dst)
    return frames, tens


def time_pushes(an, y, u, v, steps, warmup, stream, barrier):
    import torch

    from paper_2304_12384_gb300 import vca

    for _ in range(warmup):
        an.push(y, u, v)
    an.sync()
    barrier()
    torch.cuda.synchronize()
    vca.vca_set_kernel_timing(an.handle, 1)
    ms0, n0 = vca.vca_read_kernel_timing(an.handle)
    l0 = an.launches
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(steps):
        an.push(y, u, v)
    vca.vca_stream_join(an.handle)  # the last push's reduction and read-back run on a second stream
    end.record(stream)
    end.synchronize()
    torch.cuda.synchronize()
    barrier()
    ms = start.elapsed_time(end)
    ms1, n1 = vca.vca_read_kernel_timing(an.handle)
    vca.vca_set_kernel_timing(an.handle, 0)
    launches = an.launches - l0
    kernel_ms = (ms1 - ms0) / max(1, n1 - n0)
    return ms, kernel_ms, launches


def rank_reducers(world, backend="nccl", device=None):
    """(barrier, max_over_ranks) for world ranks: process-group collectives when world > 1 (the
    group is created here if needed), no-ops for one rank."""
    if world <= 1:
        return (lambda: None), (lambda x: x)
    import torch
    import torch.distributed as dist

    if not dist.is_initialized():
        if backend == "nccl":
            dist.init_process_group(backend, device_id=device)
        else:
            dist.init_process_group(backend)
    where = device if backend == "nccl" else "cpu"

    def max_over_ranks(x):
        t = torch.tensor([x], dtype=torch.float64, device=where)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    return dist.barrier, max_over_ranks


def whole_job_rate(ms_local, steps, frames_per_step, world, max_over_ranks):
    """Frames/s of the whole job: every rank's frames over the slowest rank's time (ms), and the
    milliseconds per step of that rank."""
    ms_max = max_over_ranks(ms_local)
    return steps * frames_per_step * world / (ms_max / 1000.0), ms_max / steps


def run_vca(args):
    import torch

    from paper_2304_12384_gb300 import build as vbuild
    from paper_2304_12384_gb300 import vca

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    barrier, max_over_ranks = rank_reducers(world, "nccl", device)

    vbuild.build()
    kern = {"auto": vca.VCA_KERNEL_AUTO, "plain": vca.VCA_KERNEL_PLAIN, "tc": vca.VCA_KERNEL_TC}[args.kernel]
    lp = not args.full
    stream = torch.cuda.current_stream(device)
    frames, (y, u, v) = make_device_frames(args, device)
    torch.cuda.synchronize()

    an = vca.Analyzer(W, H, 8, args.block_size, lp, kernel=kern, max_batch=args.frames, stream=stream.cuda_stream)
    kernel_name = {1: "plain", 2: "tc"}[an.kernel]
    sampler = ClockSampler(local)
    sampler.start()
    ms, kernel_ms, launches = time_pushes(an, y, u, v, args.steps, args.warmup, stream, barrier)
    clocks = sampler.stop()
    value, ms_per_step = whole_job_rate(ms, args.steps, args.frames, world, max_over_ranks)

    peak, peak_kind = load_peaks()
    kernel_frames_per_launch = args.frames
    achieved = kernel_frames_per_launch * FRAME_BYTES / (kernel_ms / 1000.0) / 1e9
    traffic_pf = measured_traffic(kernel_name, args.block_size, lp)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic_pf * kernel_frames_per_launch if traffic_pf else None,
                "peak_kind": peak_kind, "kernel": f"vca analysis ({kernel_name})",
                "algorithmic_bytes_per_launch": kernel_frames_per_launch * FRAME_BYTES,
                "kernel_ms_per_launch": kernel_ms}

    extras = {}
    if not args.no_extras and rank == 0:
        extras = run_extras(args, an, y, u, v, frames, stream, kern, lp, device)
    an.close()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": value / PAPER_FPS, "dtype": "int32", "data": "synthetic",
            "config": workload_config(args), "kernel": kernel_name, "roofline": roofline,
            "gpu_launches": launches, "clocks": clocks,
            "hbm_roofline_fps": peak * 1e9 / FRAME_BYTES,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


EXTRAS = ("latency", "e2e", "variants", "tune", "siti", "ladder", "serving", "cpu")


def extras_selector(spec):
    """The predicate `name -> wanted?` of a comma-separated --extras value ("all" selects every
    extra).  The set lives in this function's scope, so no name bound later in the caller can
    change what is selected."""
    wanted = frozenset(x.strip() for x in spec.split(",") if x.strip())
    unknown = wanted - set(EXTRAS) - {"all"}
    if unknown:
        raise ValueError(f"unknown extras: {sorted(unknown)} (choose from {', '.join(EXTRAS)}, all)")
    return lambda name: "all" in wanted or name in wanted


def run_extras(args, an, y, u, v, frames, stream, kern, lp, device):
    import numpy as np
    import torch

    from oracle import Config
    from paper_2304_12384_gb300 import vca

    out = {}
    want = extras_selector(args.extras)

    if want("latency"):
        # Per-frame latency: one device-resident frame per push, features read back (blocking).
        lat = []
        for i in range(20 + 200):
            t0 = time.perf_counter()
            an.push(y[i % args.frames], u[i % args.frames], v[i % args.frames])
            last = vca.vca_read_frame_features(an.handle, an.frames_pushed - 1, 1)
            t1 = time.perf_counter()
            if i >= 20:
                lat.append((t1 - t0) * 1000.0)
        assert last.frame >= 0
        out["latency_ms"] = {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                             "frames": len(lat), "mode": "one 2160p frame per push, blocking feature read"}

    if want("e2e"):
        # End to end: pinned host frames through the same call, copies inside the timed region.
        hy = y.cpu().pin_memory()
        hu = u.cpu().pin_memory()
        hv = v.cpu().pin_memory()
        for _ in range(2):
            an.push(hy, hu, hv)
        an.sync()
        steps = max(3, min(args.steps, 10))
        t0 = time.perf_counter()
        for _ in range(steps):
            an.push(hy, hu, hv)
            vca.vca_read_frame_features(an.handle, an.frames_pushed - 1, 1)
        an.sync()
        el = time.perf_counter() - t0
        out["e2e"] = {"value": steps * args.frames / el, "unit": "frames/s",
                      "h2d_bytes_per_step": args.frames * FRAME_BYTES, "d2h_bytes_per_step": args.frames * 8 * 8}
        del hy, hu, hv

    if want("variants"):
        # Other block-size / low-pass variants and the plain CUDA-core form, same frames.
        variants = {}
        lp_name = {False: "full", True: "lowpass", "downsample": "downsample"}
        for (bs, vlp, vk) in ((32, True, vca.VCA_KERNEL_PLAIN), (32, False, kern), (16, True, kern), (16, False, kern),
                              (16, True, vca.VCA_KERNEL_PLAIN), (16, False, vca.VCA_KERNEL_PLAIN),
                              (32, False, vca.VCA_KERNEL_PLAIN), (32, "downsample", vca.VCA_KERNEL_AUTO)):
            try:
                a2 = vca.Analyzer(W, H, 8, bs, vlp, kernel=vk, max_batch=args.frames, stream=stream.cuda_stream)
            except vca.VcaError as e:
                variants[f"w{bs}_{lp_name[vlp]}_{vk}"] = f"unsupported: {e}"
                continue
            name = f"w{bs}_{lp_name[vlp]}_{ {1: 'plain', 2: 'tc'}[a2.kernel] }"
            ms, kms, _ = time_pushes(a2, y, u, v, max(3, args.steps // 3), 2, stream, lambda: None)
            n = max(3, args.steps // 3) * args.frames
            gbs = args.frames * FRAME_BYTES / (kms / 1000.0) / 1e9
            variants[name] = {"fps": n / (ms / 1000.0), "kernel_ms_per_launch": kms,
                              "hbm_frac_of_measured": gbs / load_peaks()[0]}
            a2.close()
        # 10-bit 2160p (16-bit words): tensor-core and CUDA-core forms on the same frames.
        _, (y10, u10, v10) = make_device_frames(args, device, bit_depth=10)
        for vk in (vca.VCA_KERNEL_TC, vca.VCA_KERNEL_PLAIN):
            a2 = vca.Analyzer(W, H, 10, 32, True, kernel=vk, max_batch=args.frames, stream=stream.cuda_stream)
            name = f"w32_lowpass_10bit_{ {1: 'plain', 2: 'tc'}[a2.kernel] }"
            ms, kms, _ = time_pushes(a2, y10, u10, v10, max(3, args.steps // 3), 2, stream, lambda: None)
            n = max(3, args.steps // 3) * args.frames
            gbs = args.frames * 2 * FRAME_BYTES / (kms / 1000.0) / 1e9
            variants[name] = {"fps": n / (ms / 1000.0), "kernel_ms_per_launch": kms,
                              "hbm_frac_of_measured": gbs / load_peaks()[0]}
            a2.close()
        del y10, u10, v10
        # 4:2:2 (CUDA cores): half-width, full-height chroma planes -- the two halves of the luma
        # planes serve as U and V, so a frame reads 2 W H bytes.
        a2 = vca.Analyzer(W, H, 8, 32, True, kernel=vca.VCA_KERNEL_AUTO, max_batch=args.frames,
                          stream=stream.cuda_stream, chroma_format=vca.VCA_CHROMA_422)
        ms, kms, _ = time_pushes(a2, y, y[:, :, : W // 2], y[:, :, W // 2:], max(3, args.steps // 3), 2, stream,
                                 lambda: None)
        n = max(3, args.steps // 3) * args.frames
        gbs = args.frames * 2 * W * H / (kms / 1000.0) / 1e9
        variants[f"w32_lowpass_422_{ {1: 'plain', 2: 'tc'}[a2.kernel] }"] = {
            "fps": n / (ms / 1000.0), "kernel_ms_per_launch": kms, "hbm_frac_of_measured": gbs / load_peaks()[0]}
        a2.close()
        # 4:4:4: full-size chroma planes (the luma planes serve as U and V), 3 W H bytes per frame, on
        # both kernels.
        for vk in (vca.VCA_KERNEL_AUTO, vca.VCA_KERNEL_PLAIN):
            a2 = vca.Analyzer(W, H, 8, 32, True, kernel=vk, max_batch=args.frames, stream=stream.cuda_stream,
                              chroma_format=vca.VCA_CHROMA_444)
            ms, kms, _ = time_pushes(a2, y, y, y, max(3, args.steps // 3), 2, stream, lambda: None)
            n = max(3, args.steps // 3) * args.frames
            gbs = args.frames * 3 * W * H / (kms / 1000.0) / 1e9
            variants[f"w32_lowpass_444_{ {1: 'plain', 2: 'tc'}[a2.kernel] }"] = {
                "fps": n / (ms / 1000.0), "kernel_ms_per_launch": kms, "hbm_frac_of_measured": gbs / load_peaks()[0]}
            a2.close()
        out["variants"] = variants

    if want("tune"):
        # Launch-shape tuning of the benchmark's configuration on its own frames (16 of them): every
        # candidate's analysis time per frame, the chosen shape and its gain over the default one.
        vca.vca_tune_clear()
        cfg = vca._config(W, H, 8, args.block_size, lp)
        best, cands = vca.vca_autotune(cfg, y[:16], u[:16], v[:16], reps=5, stream=stream.cuda_stream)
        default = [c for c in cands if c["kernel"] == 2 and c["tc_ctas"] == 0] or \
                  [c for c in cands if c["kernel"] == 1 and c["plain_warps"] == 4]
        out["tune"] = {"chosen": best, "candidates": cands,
                       "gain_over_default": default[0]["ms_per_frame"] / best["ms_per_frame"],
                       "note": "vca_autotune on 16 of the step's frames; the bench step itself runs the default shape"}
        vca.vca_tune_clear()

    if want("siti"):
        # SI / TI of the same 2160p frames (the paper's comparison features; its CPU reference runs
        # at 8.55 fps on an i7-11370H, Section 3 -- another machine, context only).
        s = vca.Siti(W, H, 8, max_batch=args.frames, stream=stream.cuda_stream)
        s.push(y)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = 5
        for _ in range(reps):
            s.push(y)
        el = time.perf_counter() - t0
        out["siti"] = {"fps": reps * args.frames / el, "frames_per_push": args.frames, "launches_per_push": 2,
                       "hbm_frac_of_measured": reps * args.frames * W * H / el / 1e9 / load_peaks()[0],
                       "timing": "host wall clock per synchronous push (luma read once, 3x3 neighbourhood from cache)"}
        s.close()

    if want("ladder"):
        out["ladder"] = run_ladder(args, stream)

    if want("serving"):
        out["serving"] = run_serving(args, policy=0)
        out["serving_ticks"] = run_serving(args, policy=1)

    if want("cpu"):
        # CPU oracle on the host cores (all of them, and one), bounded samples of the same workload;
        # its features of the first frames also give the per-feature error of the GPU path.
        from oracle import analyze_sequence

        cfg = Config(W, H, 8, args.block_size, lp)
        cores = os.cpu_count() or 1
        fps1, n1 = oracle_fps(frames[:2], cfg, args.cpu_seconds / 3)
        fps, n = oracle_fps_all_cores(cfg, args.cpu_seconds, cores)
        out["cpu_baseline"] = {"value": fps, "unit": "frames/s", "cores": cores, "kind": "oracle",
                               "sample": f"{n} frames of the same 3840x2160 workload through the FP64/int64 oracle "
                                         f"(numpy; per-frame block values on {cores} processes)",
                               "single_core": {"value": fps1, "frames": n1}}
        nerr = min(4, len(frames))
        a2 = vca.Analyzer(W, H, 8, args.block_size, lp, kernel=kern, max_batch=nerr, stream=stream.cuda_stream)
        a2.push(y[:nerr], u[:nerr], v[:nerr])
        exp = analyze_sequence(frames[:nerr], cfg)
        errs = {}
        for t in range(nerr):
            got = a2.frame_features(t)
            for k, e in exp[t].items():
                if e != 0.0:
                    errs[k] = max(errs.get(k, 0.0), abs(got[k] - e) / abs(e))
            errs["h_vs_max(h,E_Y)"] = max(errs.get("h_vs_max(h,E_Y)", 0.0),
                                          abs(got["h"] - exp[t]["h"]) / max(abs(exp[t]["h"]), exp[t]["E_Y"]))
        a2.close()
        out["feature_error"] = {"max_rel": errs, "frames": nerr,
                                "against": "FP64 oracle, same synthetic frames, first frames of the step"}
    return out


def run_ladder(args, stream, distinct=2, ticks=200):
    """24-channel ladder tick (4 channels at each of 640x360 .. 3840x2160, half 10-bit, block 32,
    low-pass): the batched path (one graph per tick: a tensor-core launch per sample size, each
    ending with the reduction of its channels' frames) against one push per channel per tick
    through the single-analyzer path."""
    import numpy as np
    import torch

    from paper_2304_12384_gb300 import vca
    from synth import frames_list, ladder_specs, pack_planes

    specs = ladder_specs(4, n_frames=distinct)
    dev = []
    tick_bytes = 0
    for sp in specs:
        pk = pack_planes(frames_list(sp, 0, distinct))
        planes = []
        for k in ("y", "u", "v"):
            a = pk[k]
            if a.dtype == np.uint16:
                a = a.view(np.int16)
            planes.append(torch.from_numpy(np.ascontiguousarray(a)).cuda())
        dev.append(planes)
        tick_bytes += sp.width * sp.height * 3 // 2 * (2 if sp.bit_depth > 8 else 1)
    torch.cuda.synchronize()
    ans = [vca.Analyzer(sp.width, sp.height, sp.bit_depth, 32, True, max_batch=1, stream=stream.cuda_stream)
           for sp in specs]

    # Each tick's frame references (views of the resident frames), made once: a tick then costs
    # what the library does, not the slicing of 72 tensors.  The batched path takes them as tick
    # arguments built once per resident frame (Batch.frame_refs), as a caller ticking from a ring
    # of frame buffers would.
    tick_refs = [[(y[t], u[t], v[t]) for (y, u, v) in dev] for t in range(distinct)]

    def refs(t):
        return tick_refs[t % distinct]

    batch = vca.Batch(ans)
    batch_refs = [batch.frame_refs(r) for r in tick_refs]
    warm = 10

    def timed_ticks():
        for t in range(warm):
            batch.tick(batch_refs[t % distinct])
        batch.sync()
        t0 = time.perf_counter()
        for t in range(ticks):
            batch.tick(batch_refs[t % distinct])
        batch.sync()
        return time.perf_counter() - t0

    el_default = timed_ticks()  # SM split weight at creation (1.15)
    weight, _ = batch.autotune(batch_refs[0], reps=40)
    l0 = batch.launches()
    el_b = timed_ticks()
    launches = batch.launches() - l0
    batch.close()

    for t in range(3):
        for a, r in zip(ans, refs(t)):
            a.push(*r)
    for a in ans:
        a.sync()
    t0 = time.perf_counter()
    for t in range(ticks):
        for a, r in zip(ans, refs(t)):
            a.push(*r)
    for a in ans:
        vca.vca_read_frame_features(a.handle, a.frames_pushed - 1, 1)
    el_s = time.perf_counter() - t0
    for a in ans:
        a.close()
    peak = load_peaks()[0]
    tb = ticks / el_b
    return {"channels": len(specs), "tick_bytes": tick_bytes, "ticks": ticks,
            "batched_ticks_per_s": tb, "batched_gbs": tb * tick_bytes / 1e9,
            "batched_hbm_frac_of_measured": tb * tick_bytes / 1e9 / peak,
            "batched_launches_per_tick": launches / (ticks + warm),
            "split_weight_tuned": weight, "batched_ticks_per_s_untuned": ticks / el_default,
            "per_channel_push_ticks_per_s": ticks / el_s,
            "hbm_roofline_ticks_per_s": peak * 1e9 / tick_bytes,
            "timing": "host wall clock around queued ticks, synchronized at both ends; frames device-resident"}


def run_serving(args, n_channels=64, distinct=4, capacity_s=3.0, poisson_s=6.0, seed=5, policy=0):
    """Serving loop: 64 live channels (frame size uniform over the six ladder resolutions, 8/10-bit
    mix, 2-second segments at 30 or 60 fps = 60 or 120 frames), segments copied from device
    buffers into the server's rings (standing in for a decoder) and analysed under the server's
    policy (0: each landed segment one multi-frame work item; 1: frame-interleaved batched ticks).
    First the capacity (segments/s with every channel submitting back to back), then Poisson
    arrivals per channel at 0.8 x capacity in total; latency = features ready - arrival."""
    import numpy as np
    import torch

    from paper_2304_12384_gb300 import vca
    from synth import LADDER_RESOLUTIONS, SequenceSpec, frames_list, pack_planes

    rng = np.random.default_rng(seed)
    chans = []
    for i in range(n_channels):
        w, h = LADDER_RESOLUTIONS[int(rng.integers(len(LADDER_RESOLUTIONS)))]
        chans.append((w, h, int(rng.choice([8, 10])), int(rng.choice([60, 120]))))
    # One 120-frame source segment per (size, depth) class, shared by that class's channels.
    src = {}
    for (w, h, bd, _) in chans:
        if (w, h, bd) in src:
            continue
        pk = pack_planes(frames_list(SequenceSpec(w, h, distinct, 9000 + w + bd, bit_depth=bd), 0, distinct))
        planes = []
        for k in ("y", "u", "v"):
            a = pk[k]
            if a.dtype == np.uint16:
                a = a.view(np.int16)
            t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
            planes.append(t[torch.arange(120, device="cuda") % distinct].contiguous())
        src[(w, h, bd)] = planes
    torch.cuda.synchronize()
    srv = vca.Server(policy=policy)
    ids = [srv.add_channel(w, h, bd, 32, True, max_segment_frames=seg) for (w, h, bd, seg) in chans]
    stats0 = srv.stats()

    def submit(i, tag):
        w, h, bd, seg = chans[i]
        y, u, v = src[(w, h, bd)]
        return srv.submit_frames(ids[i], y[:seg], u[:seg], v[:seg], tag=tag)

    # Capacity: keep every channel's two slots busy.
    done = []
    t_end = time.monotonic() + capacity_s
    tag = 0
    t0 = time.monotonic()
    while time.monotonic() < t_end:
        sent = 0
        for i in range(n_channels):
            if submit(i, tag) == vca.VCA_OK:
                tag += 1
                sent += 1
        done += srv.poll(1024)
        if not sent:
            time.sleep(0.0002)
    while len(done) < tag:
        done += srv.poll(1024)
        time.sleep(0.0005)
    el = time.monotonic() - t0
    capacity = len(done) / el
    frames_cap = sum(d["n_frames"] for d in done) / el

    # Poisson arrivals at 0.8 x capacity, each channel an independent stream of rate/n_channels.
    rate = 0.8 * capacity / n_channels
    arrivals = []
    for i in range(n_channels):
        t = rng.exponential(1.0 / rate)
        while t < poisson_s:
            arrivals.append((t, i))
            t += rng.exponential(1.0 / rate)
    arrivals.sort()
    backlog = [[] for _ in range(n_channels)]
    arrival_ns = {}
    lat = []
    base = time.monotonic_ns()
    k = 0
    tag0 = 1 << 32
    n_arr = len(arrivals)
    while len(lat) < n_arr:
        now = time.monotonic_ns()
        while k < n_arr and base + int(arrivals[k][0] * 1e9) <= now:
            t_arr, i = arrivals[k]
            backlog[i].append((tag0 + k, base + int(t_arr * 1e9)))
            k += 1
        for i in range(n_channels):
            while backlog[i]:
                tg, ta = backlog[i][0]
                if submit(i, tg) != vca.VCA_OK:
                    break
                arrival_ns[tg] = ta
                backlog[i].pop(0)
        for d in srv.poll(1024):
            if d["tag"] in arrival_ns:
                lat.append((d["ready_ns"] - arrival_ns.pop(d["tag"])) / 1e6)
        time.sleep(0.0002)
    st = srv.stats()
    srv.close()
    lat = np.array(lat)
    return {"channels": n_channels, "segments_capacity_per_s": capacity, "frames_capacity_per_s": frames_cap,
            "poisson_rate_segments_per_s": 0.8 * capacity, "segments": int(lat.size),
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "max": float(lat.max()), "mean": float(lat.mean())},
            "device_budget_bytes": st["budget_bytes"], "device_used_bytes": st["used_bytes"],
            "launches": st["launches"] - stats0["launches"], "ticks": st["ticks"],
            "policy": "segments (one multi-frame push per landed segment)" if policy == 0
            else "ticks (one frame of every channel per batched tick)",
            "mix": "frame size uniform over 640x360..3840x2160, 8/10-bit, 60/120-frame segments; "
                   "segments copied device-to-device into the server's rings inside the measured latency"}


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_vca(args)


if __name__ == "__main__":
    main()
