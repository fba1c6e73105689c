#!/usr/bin/env python3
"""Throughput of the FastBlend hot path (arXiv 2311.09265) on B300.

Default workload: Eq. 2 all-pairs sliding-window blend of a 60-frame 512x512 RGB clip,
patch 5x5, window 15, 6 patch-match iterations (784 NNFs per step), synthetic guides
under smooth random affine motion and LUT+noise style frames.  One step = one
fb_blend_window call over the whole clip (pair set-up, NNF init, all iterations,
remap, blend, normalise).

Prints ONE JSON line (rank 0):
  value      blended frames/s, device-resident inputs, CUDA events, max over ranks
  e2e        the same through the C ABI with pinned HOST buffers (copies inside)
  roofline   dominant kernel (the Alg. 1 Jacobi iteration) against the dp4a ALU bound
  cpu_baseline  the CPU oracle on a bounded sample of the same workload

--impl reference times the CPU oracle (the only reference: the paper ships no code).
Multi-GPU (torchrun), no data-path collective; a gloo barrier and a max-reduce bracket the
timed region.  --shard frames (default): one clip of N x 60 frames is split by output
frame (fb_shard_plan), each rank blending its range from its frames plus the window's
halo (fb_blend_window_range) -- weak scaling, 60 output frames per GPU; modes whose NNFs
couple frames across the clip (fast, tracking) and the learned and interpolation
workloads fall back to replicas.  --shard replicas: every rank blends its own clip.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "blended frames/s at 512² w=15; NNF candidate-evals/s vs integer/HBM roofline"
L2_BYTES = 126 * 1024 * 1024
FLUSH_BYTES = 512 * 1024 * 1024
SM_COUNT_NOMINAL = 148
SM_MAX_MHZ_NOMINAL = 2032.0
DP4A_PER_CLK_SM = 64        # integer dot-product (dp4a) issue rate per SM per clock
# Guide weight of the improved loss (Sec. 3.4) in the balanced workload.
BALANCED_ALPHA = 10
# What the ncu captures of the iteration kernels show bounds them (see profiles/): the dp4a
# ALU peak above is the arithmetic roofline, not the limit these gathers reach.
LIMITER = {"k5": "L1TEX pipe 84-88 % of peak on scattered candidate loads (ncu); DRAM 2-4 %",
           "k7": "L1TEX pipe 90-92 % of peak on scattered candidate loads (ncu); DRAM 2 %"}
# dram__bytes_read.sum + dram__bytes_write.sum of one launch of the workload's iteration
# kernel, from an ncu capture of the current kernel on a smaller case scaled by the pairs
# per launch (see profiles/); None when not captured or when the workload is overridden.
TRAFFIC_PER_LAUNCH = {"blend_512": 5.71e9, "tracking_512": 4.08e9, "balanced_512": 9.11e9,
                      "aligned_1024x576": 7.41e9, "interp_1024x576": 2.47e9}
# 32-byte L1 sectors the plain iteration kernel loads per pixel of each pair and launch:
# ncu l1tex__t_sectors_pipe_lsu_mem_global_op_ld.sum of the captured launch divided by its
# pairs x pixels (k = 5: 1185.3 M / (168 x 512 x 512); k = 7: 729.1 M / (20 x 576 x 1024);
# see profiles/).  A CPU replay of the k = 5 load sequence (slot order, early exit) gives
# 26.5.  The L1 data pipe moves one such sector per wavefront, so sectors per second
# against a live probe of scattered 32-byte loads is the gather roofline of these kernels.
SECTORS_PER_PIXEL_ITER = {5: 26.92, 7: 61.81}
GATHER_PROBE_BYTES = {"l1_resident": 64 * 1024, "l2_resident": 4 * 1024 * 1024}


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("fastblend", "reference"), default="fastblend")
    ap.add_argument("--workload", default="blend_512",
                    choices=sorted(synth.WORKLOADS) + ["batch_32", "batch_small", "learned_512", "initnet_512",
                                                       "balanced_512", "fast_512", "accurate_512",
                                                       "tracking_1024x576", "tracking_512",
                                                       "aligned_1024x576"])
    ap.add_argument("--window", type=int, default=0,
                    help="override the blend window of the headline-clip workloads (odd)")
    ap.add_argument("--batch-clips", default="",
                    help="batch_32: submit only these manifest clips, e.g. 12,13 (small profiling "
                         "cases)")
    ap.add_argument("--frames", type=int, default=0,
                    help="interpolation workloads: keep the clip's first F frames, keys 0 and "
                         "F - 1 styled with the clip's two key styles (small profiling cases)")
    ap.add_argument("--learned-iters", type=int, default=2,
                    help="Alg. 1 iterations after the learned initialiser (learned_512)")
    ap.add_argument("--shard", choices=("frames", "replicas"), default="frames",
                    help="N > 1: split one clip by output frame (frames) or give every rank "
                         "its own clip (replicas)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-sample-frames", type=int, default=5)
    return ap.parse_args(argv)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_device(local: int) -> int:
    """The GPU of local rank `local`: one per rank; ranks beyond the visible devices share
    them round-robin (a functional run of the multi-rank path on fewer GPUs -- its kernels
    never wait on another rank's, so sharing is safe, but its timings are not scaling
    numbers)."""
    import torch
    n = torch.cuda.device_count()
    return local % n if n else local


class RankGroup:
    """The ranks of one bench run.  With more than one rank a gloo group carries the
    barriers around the timed region and the max-over-ranks reduction of the timings;
    the data path itself never communicates (each rank blends its own clips)."""

    def __init__(self):
        self.rank, self.world, self.local = dist_env()
        if self.world > 1:
            import torch.distributed as dist
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group("gloo", rank=self.rank, world_size=self.world)

    def barrier(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()

    def max(self, x: float) -> float:
        if self.world == 1:
            return x
        import torch
        import torch.distributed as dist
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def sum(self, x: float) -> float:
        if self.world == 1:
            return x
        import torch
        import torch.distributed as dist
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


def shard_seed(workload_seed: int, rank: int) -> int:
    """Rank r blends its own clip; rank 0 blends the named workload itself."""
    return workload_seed + 7919 * rank


def aggregate(n_frames_per_rank: int, steps: int, world: int, max_total_ms: float) -> float:
    """Whole-job frames/s: every rank's frames over the slowest rank's time."""
    return world * n_frames_per_rank * steps / (max_total_ms / 1e3)


def truncate_interpolation(w: synth.Workload, g, s, frames: int):
    """The first `frames` frames of a two-key interpolation clip, keys 0 and frames - 1
    (the key styles unchanged)."""
    import dataclasses
    if not frames or w.mode != "interpolate":
        return w, g, s
    if len(w.keys) != 2 or not 2 <= frames <= w.N:
        raise ValueError("--frames needs a two-key interpolation workload and 2 <= F <= N")
    return dataclasses.replace(w, N=frames, keys=(0, frames - 1)), g[:frames].copy(), s


def make_inputs(w: synth.Workload, seed: int):
    if seed == w.seed:
        # the named workload's own clip (a window override keeps the clip)
        return synth.make_clip(next(k for k, v in synth.WORKLOADS.items() if v.name == w.name))
    if w.motion == "shift":
        g, _ = synth.shift_clip(w.N, w.H, w.W, seed)
        s = synth.colour_matrix_styles(g, seed)
    else:
        g, _ = synth.affine_clip(w.N, w.H, w.W, seed)
        s = synth.lut_styles(g, seed)
    if w.mode == "interpolate":
        s = s[list(w.keys)].copy()
    return g, s


# ----------------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_median": statistics.median(power) if power else None}


# ----------------------------------------------------------------------------------
# CPU oracle (cpu_baseline and the reference arm)
# ----------------------------------------------------------------------------------
TRACKING_BLEND_SAMPLE_FRAMES = 5


def tracking_sample(w: synth.Workload, g, s, aligned=False):
    """A bounded oracle sample of a tracking workload: the oracle couples every NNF of a
    chain, so one output frame costs the whole clip.  Interpolation: the clip's first 4
    frames of the same size with keys 0 and 3 (2 interpolated frames, 4 tracked NNFs in
    two chains of 2).  Blend: the clip's first 5 frames (all 20 pairs of the window)."""
    import numpy as np
    if w.mode == "blend":
        n = TRACKING_BLEND_SAMPLE_FRAMES
        return np.ascontiguousarray(g[:n]), np.ascontiguousarray(s[:n]), None
    return (np.ascontiguousarray(g[:4]),
            np.ascontiguousarray(np.stack([s[0], s[1 if aligned else 0]])), [0, 3])


def tracking_sample_outputs(w: synth.Workload) -> int:
    return TRACKING_BLEND_SAMPLE_FRAMES if w.mode == "blend" else 2


def oracle_frame_seconds(w: synth.Workload, g, s, frames, alpha=None, fast=False, accurate=False,
                         tracking=False, aligned=False):
    import oracle
    t0 = time.perf_counter()
    if tracking:
        g4, k4, keys = tracking_sample(w, g, s, aligned)
        if aligned:
            oracle.interpolate_aligned(g4, keys, k4, w.patch, w.iters, alpha, tracking=True,
                                       seed=w.seed)
        elif w.mode == "blend":
            oracle.blend_window_tracking(g4, k4, w.window, w.patch, w.iters, seed=w.seed)
        else:
            oracle.interpolate_tracking(g4, keys, k4, w.patch, w.iters, seed=w.seed)
        return time.perf_counter() - t0
    for i in frames:
        if w.mode == "blend" and accurate:
            oracle.blend_frame_accurate(g, s, w.window, i, w.patch, w.iters, alpha, seed=w.seed)
        elif w.mode == "blend" and fast:
            oracle.blend_frame_fast(g, s, w.window, i, w.patch, w.iters, seed=w.seed)
        elif w.mode == "blend" and alpha is not None:
            oracle.blend_frame_balanced(g, s, w.window, i, w.patch, w.iters, alpha, seed=w.seed)
        elif w.mode == "blend":
            oracle.blend_frame(g, s, w.window, i, w.patch, w.iters, seed=w.seed)
        else:
            oracle.interpolate_frame(g, list(w.keys), s, i, w.patch, w.iters, seed=w.seed)
    return time.perf_counter() - t0


def sample_frames(w: synth.Workload, n: int):
    """Interior frames whose window is full (the typical, not the cheapest, frames)."""
    mid = w.N // 2
    return [mid + d for d in range(n)]


def cpu_baseline(w: synth.Workload, g, s, n_frames: int, alpha=None, fast=False, accurate=False,
                 tracking=False, aligned=False):
    import oracle
    if tracking:
        secs = oracle_frame_seconds(w, g, s, [], alpha, tracking=True, aligned=aligned)
        return {"value": tracking_sample_outputs(w) / secs, "unit": "frames/s",
                "cores": oracle.num_threads(), "kind": "oracle",
                "sample": (f"the clip's first {TRACKING_BLEND_SAMPLE_FRAMES} frames ({w.H}x{w.W}), "
                           f"window {w.window}: all {TRACKING_BLEND_SAMPLE_FRAMES} output frames, "
                           f"{TRACKING_BLEND_SAMPLE_FRAMES * (TRACKING_BLEND_SAMPLE_FRAMES - 1)} "
                           f"tracked NNFs (windows truncated by the sample's length)"
                           if w.mode == "blend" else
                           f"the clip's first 4 frames ({w.H}x{w.W}) with keys 0 and 3: 2 "
                           f"interpolated frames, 4 tracked NNFs"
                           + (" coupled by the Eq. 10 alignment loss (the two keys styled with "
                              "the clip's two key styles)" if aligned else ""))
                          + f"; C oracle, OpenMP, {secs:.1f} s"}
    frames = sample_frames(w, n_frames)
    secs = oracle_frame_seconds(w, g, s, frames, alpha, fast, accurate)
    return {"value": len(frames) / secs, "unit": "frames/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{len(frames)} of {w.N} output frames ({frames}) of the same clip, each "
                      f"with its full window of NNFs; C oracle, OpenMP, {secs:.1f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    if args.workload in BATCH_MANIFESTS:
        N, H, W, window, patch = batch_manifest(args.workload, BATCH_SEED)[0]
        g, s = synth.batch_clip(N, H, W, seed=BATCH_SEED)
        w = synth.Workload(f"batched submission of the {args.workload} manifest (sample: clip 0)",
                           "blend", N, H, W, patch=patch, iters=BATCH_ITERS, window=window,
                           seed=BATCH_SEED)
    else:
        w = synth.WORKLOADS[base_workload(args.workload)]
        if args.window and w.mode == "blend":
            import dataclasses
            w = dataclasses.replace(w, window=args.window)
        g, s = make_inputs(w, w.seed)
        w, g, s = truncate_interpolation(w, g, s, args.frames)
    alpha = (BALANCED_ALPHA if args.workload in ("balanced_512", "accurate_512", "aligned_1024x576")
             else None)
    fast = args.workload == "fast_512"
    accurate = args.workload == "accurate_512"
    aligned = args.workload == "aligned_1024x576"
    tracking = args.workload in ("tracking_1024x576", "tracking_512") or aligned
    frames = sample_frames(w, 1)
    for _ in range(args.warmup):
        oracle_frame_seconds(w, g, s, frames, alpha, fast, accurate, tracking, aligned)
    total = 0.0
    for _ in range(args.steps):
        total += oracle_frame_seconds(w, g, s, frames, alpha, fast, accurate, tracking, aligned)
    n_out = tracking_sample_outputs(w) if tracking else len(frames)
    value = args.steps * n_out / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": workload_label(args.workload, w, args.learned_iters),
                   "frames": w.N, "height": w.H, "width": w.W,
                   "patch": w.patch, "window": w.window, "iters": w.iters,
                   "step": "one output frame of the clip (bounded CPU sample)"},
        "cpu_baseline": {"value": value, "unit": "frames/s", "cores": oracle.num_threads(),
                         "kind": "oracle",
                         "sample": ("each step interpolates frames 1-2 of the clip's first 4 "
                                    "frames with keys 0 and 3 (tracking couples whole chains"
                                    + (", alignment couples the two keys' NNFs)" if aligned else ")")
                                    if tracking and w.mode != "blend" else
                                    f"each step blends the clip's first {TRACKING_BLEND_SAMPLE_FRAMES} "
                                    "frames (tracking couples whole chains)" if tracking else
                                    f"each step blends output frame {frames[0]} of {w.N}")},
        "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------------
def iter_ops_per_launch(w: synth.Workload, pairs=None) -> int:
    """Algorithmic byte-pair ops of one Jacobi-iteration launch (levels = 1): every
    pair (all of the workload's, or `pairs`), every pixel, 4 propagation + R
    random-search candidates, 3k^2 byte pairs."""
    n = w.pairs() if pairs is None else pairs
    return n * w.H * w.W * (4 + w.random_search_radii()) * 3 * w.patch * w.patch


def shard_inputs(w: synth.Workload, n_total: int, first: int, last: int):
    """Frames [first, last) of the n_total-frame clip that a frame-sharded run splits:
    the workload's motion model drawn for the whole clip (same seed on every rank), and
    styles drawn per frame index, so every rank sees the same clip wherever it is cut."""
    import numpy as np
    if w.motion == "shift":   # small clips: draw the whole clip, keep the range
        g, _ = synth.shift_clip(n_total, w.H, w.W, w.seed)
        s = synth.colour_matrix_styles(g, w.seed)
        return np.ascontiguousarray(g[first:last]), np.ascontiguousarray(s[first:last])
    g, _ = synth.affine_clip(n_total, w.H, w.W, w.seed, frames=(first, last))
    return g, synth.lut_styles_indexed(g, w.seed, first)


def workload_label(name: str, w: synth.Workload, learned_iters: int = 2) -> str:
    """config.workload: what one step computes, with the sizes it runs at."""
    dims = f"{w.N}x{w.H}x{w.W} k{w.patch}"
    dims += f" w{w.window}" if w.mode == "blend" else " keys " + ",".join(map(str, w.keys))
    it = f" n{w.iters}"
    labels = {
        "learned_512": f"learned-init blend all-pairs {dims}: BF16 conv initialiser (tcgen05) + "
                       f"{learned_iters} Alg. 1 iteration(s)",
        "balanced_512": f"balanced blend all-pairs {dims}{it}: Sec. 3.4 improved loss, "
                        f"alpha {BALANCED_ALPHA}",
        "fast_512": f"fast-mode blend {dims}{it}: Sec. 3.4 remapping / blending tables and "
                    "interval queries (Algs. 3-5)",
        "accurate_512": f"accurate blend all-pairs {dims}{it}: Sec. 3.4 mean-remap alignment "
                        f"loss, alpha {BALANCED_ALPHA}",
        "tracking_512": f"tracking blend all-pairs {dims}{it}: Sec. 3.5.1 chain-neighbour candidates",
        "tracking_1024x576": f"tracking interpolation {dims}{it}: Sec. 3.5.1 chain-neighbour "
                             "candidates",
        "aligned_1024x576": f"aligned + tracking interpolation {dims}{it}: Eq. 10 alignment loss "
                            f"(alpha {BALANCED_ALPHA}) and Sec. 3.5.1 tracking",
    }
    if name in labels:
        return labels[name]
    if name in synth.WORKLOADS and w != synth.WORKLOADS[name]:
        return f"{w.name}, run at {dims}{it}"
    return w.name


def base_workload(name: str) -> str:
    """The synthetic clip a mode workload runs on."""
    if name in ("balanced_512", "learned_512", "initnet_512", "fast_512", "accurate_512",
                "tracking_512"):
        return "blend_512"
    if name in ("tracking_1024x576", "aligned_1024x576"):
        return "interp_1024x576"
    return name


def tracking_neighbour_refs(w: synth.Workload) -> int:
    """Chain-neighbour candidates per pixel summed over the pairs of a call with tracking:
    a chain of n consecutive target frames from one source has 2 (n - 1)."""
    if w.mode == "blend":
        M, refs = w.window // 2, 0
        for j in range(w.N):
            for lo, hi in ((max(0, j - M), j - 1), (j + 1, min(w.N - 1, j + M))):
                refs += 2 * max(hi - lo, 0)
        return refs
    keys = list(w.keys)
    bounds = [-1] + keys + [w.N]
    refs = 0
    for a, b in zip(bounds[:-1], bounds[1:]):
        n = b - a - 1                              # frames strictly between two keys
        chains = (a >= 0) + (b < w.N)              # served from the left and / or right key
        refs += chains * 2 * max(n - 1, 0)
    return refs


def aligned_pairs(w: synth.Workload) -> int:
    """Pairs that carry the Eq. 10 coupled loss: both pairs of every frame strictly
    between two keys."""
    keys = list(w.keys)
    return 2 * sum(b - a - 1 for a, b in zip(keys[:-1], keys[1:]))


def run_gpu(args):
    import torch

    import paper_2311_09265_b300 as fbp

    grp = RankGroup()
    rank, world, local = grp.rank, grp.world, grp.local
    local = rank_device(local)
    torch.cuda.set_device(local)
    fbp.build()
    learned = args.workload == "learned_512"
    balanced = args.workload == "balanced_512"
    fast = args.workload == "fast_512"
    accurate = args.workload == "accurate_512"
    aligned = args.workload == "aligned_1024x576"
    tracking = args.workload in ("tracking_1024x576", "tracking_512") or aligned
    w = synth.WORKLOADS[base_workload(args.workload)]
    if args.window and w.mode == "blend":
        import dataclasses
        w = dataclasses.replace(w, window=args.window)
    # --shard frames: one clip of world x N frames split by output frame; each rank holds
    # its range plus the window's halo and blends the range with fb_blend_window_range.
    shard = None
    if (world > 1 and args.shard == "frames" and w.mode == "blend"
            and not (fast or tracking or learned)):
        import dataclasses
        n_total = w.N * world
        shard = fbp.fb_shard_plan(n_total, w.window, world, rank)
        shard["n_total"] = n_total
        shard["pairs"] = len(fbp.fb_pair_plan_range(n_total, shard["out_first"], shard["n_out"],
                                                    window=w.window))
        g, s = shard_inputs(w, n_total, shard["frame_base"], shard["frame_base"] + shard["n_in"])
        w_job = dataclasses.replace(w, N=n_total)       # what the whole job computes
    else:
        g, s = make_inputs(w, shard_seed(w.seed, rank))
        w, g, s = truncate_interpolation(w, g, s, args.frames)
        w_job = None
    n_out = shard["n_out"] if shard else w.N
    ctx = fbp.Context(local)
    params = fbp.Params.make(w.patch, w.iters, w.levels, 0, w.seed)
    if balanced:
        params = fbp.Params.make(w.patch, w.iters, 1, 0, w.seed, flags=fbp.FB_FLAG_BALANCED,
                                 alpha=BALANCED_ALPHA)
    if accurate:
        params = fbp.Params.make(w.patch, w.iters, 1, 0, w.seed, flags=fbp.FB_FLAG_ACCURATE,
                                 alpha=BALANCED_ALPHA)
    if tracking:
        params = fbp.Params.make(w.patch, w.iters, 1, 0, w.seed,
                                 flags=fbp.FB_FLAG_TRACKING | (fbp.FB_FLAG_ALIGN if aligned else 0),
                                 alpha=BALANCED_ALPHA if aligned else 0)
    fast_info = None
    if fast:
        params = fbp.Params.make(w.patch, w.iters, 1, 0, w.seed, flags=fbp.FB_FLAG_FAST)
        n_nnfs, n_entries, n_pieces = fbp.fb_fast_plan(w.N, w.window)
        fast_info = {"nnfs": n_nnfs, "direct_nnfs": w.pairs(), "table_entries": n_entries,
                     "query_pieces": n_pieces}
    learned_info = None
    if learned:
        # The learned initialiser: trained here, on the method's own NNFs of seeded clips
        # that differ from the evaluated clip, by the library's forward/backward kernels.
        from paper_2311_09265_b300 import initnet_train
        net, hist, t_data, t_train = initnet_train.train_default(ctx, w.H, w.W, max_pairs=256)
        ctx.set_initnet(net)
        params = fbp.Params.make(w.patch, args.learned_iters, 1, 0, w.seed)
        params.flags = fbp.FB_FLAG_LEARNED_INIT
        learned_info = {"timing": "the initialiser is trained once before the timed region "
                                  "(training_set_s + training_s, not in ms_per_step); each timed "
                                  "step runs its forward pass and the refinement iterations",
                        "training_set_s": t_data, "training_s": t_train,
                        "training_steps": hist[-1][0] + 1, "loss_first": hist[0][1],
                        "loss_last": hist[-1][1], "refinement_iters": args.learned_iters,
                        "net_params": net.n_params, "downscale": net.ds}
    g_d = torch.tensor(g, device="cuda")
    s_d = torch.tensor(s, device="cuda")
    out = torch.empty((n_out, w.H, w.W, 3), dtype=torch.float32, device="cuda")
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def step(gg, ss, oo):
        if shard:
            return fbp.fb_blend_window_range(ctx, gg, ss, w.window, params, shard["n_total"],
                                             shard["frame_base"], shard["out_first"], n_out, out=oo)
        if w.mode == "blend":
            return fbp.fb_blend_window(ctx, gg, ss, w.window, params, out=oo)
        return fbp.fb_interpolate(ctx, gg, list(w.keys), ss, params, out=oo)

    for _ in range(max(args.warmup, 0)):
        step(g_d, s_d, out)
    torch.cuda.synchronize()

    # ---- timed region: device-resident inputs ----
    grp.barrier()
    torch.cuda.synchronize()
    ctx.profile(True)
    launches0 = ctx.launches
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()                       # evict L2 between steps
            starts[k].record()
            step(g_d, s_d, out)
            ends[k].record()
        torch.cuda.synchronize()
    grp.barrier()
    launches = ctx.launches - launches0
    prof = ctx.profile_read()
    ctx.profile(False)
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    total_ms = grp.max(sum(step_ms))
    # whole-job frames/s: every rank's output frames over the slowest rank's time (a
    # frame-sharded job outputs its world x N-frame clip once per step)
    value = aggregate(w.N, args.steps, world, total_ms)
    clocks = clk.summary()

    # ---- end to end through the C ABI with pinned host buffers ----
    e2e = None
    if not args.no_e2e:
        g_h = torch.tensor(g).pin_memory()
        s_h = torch.tensor(s).pin_memory()
        o_h = torch.empty((n_out, w.H, w.W, 3), dtype=torch.float32).pin_memory()
        step(g_h, s_h, o_h)                     # warm (staging buffers)
        grp.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step(g_h, s_h, o_h)                 # synchronous: returns with o_h filled
        t_e2e = grp.max(time.perf_counter() - t0)
        # copies of the whole job: every rank's inputs in and its output frames out
        e2e = {"value": world * w.N * args.steps / t_e2e, "unit": "frames/s",
               "h2d_bytes_per_step": int(grp.sum(g_h.numel() + s_h.numel())),
               "d2h_bytes_per_step": int(grp.sum(o_h.numel() * 4))}

    if learned:
        # NNF energy (mean Eq. 1 error of all 784 final fields) against the plain search.
        def energy_and_ms(pp):
            pp.flags |= fbp.FB_FLAG_REPORT_ENERGY
            fbp.fb_blend_window(ctx, g_d, s_d, w.window, pp, out=out)
            e, c = ctx.energy()
            pp.flags &= ~fbp.FB_FLAG_REPORT_ENERGY
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            fbp.fb_blend_window(ctx, g_d, s_d, w.window, pp, out=out)
            torch.cuda.synchronize()
            a.record()
            fbp.fb_blend_window(ctx, g_d, s_d, w.window, pp, out=out)
            b.record()
            torch.cuda.synchronize()
            return e / c, a.elapsed_time(b)
        plain = fbp.Params.make(w.patch, w.iters, 1, 0, w.seed)
        e_plain, ms_plain = energy_and_ms(plain)
        lp = fbp.Params.make(w.patch, args.learned_iters, 1, 0, w.seed)
        lp.flags = fbp.FB_FLAG_LEARNED_INIT
        e_learn, ms_learn = energy_and_ms(lp)
        learned_info.update({"energy_learned": e_learn, "energy_plain_6_iters": e_plain,
                             "energy_ratio": e_learn / e_plain, "ms_learned": ms_learn,
                             "ms_plain_6_iters": ms_plain, "speedup_vs_plain": ms_plain / ms_learn})

    # ---- roofline of the dominant kernel ----
    rate, _ = ctx.probe_dp4a()
    # the ALU roofline of the instruction sequence the kernels actually issue (live probe)
    mix_rate = ctx.probe_ssd_mix(w.patch)[0] if w.patch in (5, 7) else None
    plain_iter = not (balanced or accurate or tracking or aligned or fast or learned)
    gather_rates = ({k: ctx.probe_gather(b)[0] for k, b in GATHER_PROBE_BYTES.items()}
                    if plain_iter and w.patch in SECTORS_PER_PIXEL_ITER else None)
    iter_ms, iter_n = prof["iter"]
    kernel_total_ms = sum(v[0] for v in prof.values())
    # per launch of this rank (a frame shard launches its own range's pairs)
    ops = (iter_ops_per_launch(w, shard["pairs"] if shard else None)
           if w.levels == 1 else None)  # same per launch with learned init
    if ops and (balanced or accurate):
        ops *= 2   # each candidate compares a guide patch and a style patch
    if ops and fast:
        ops = ops * fast_info["nnfs"] // w.pairs()   # the fast mode computes fewer NNFs
    if ops and tracking:
        ops += tracking_neighbour_refs(w) * w.H * w.W * 3 * w.patch * w.patch
    if ops and aligned:
        ops = ops * (2 * aligned_pairs(w) + (w.pairs() - aligned_pairs(w))) // w.pairs()
    if fast:
        # context: the direct window sum of the same clip and window, one untimed-by-the-
        # contract measurement with CUDA events
        direct = fbp.Params.make(w.patch, w.iters, 1, 0, w.seed)
        fbp.fb_blend_window(ctx, g_d, s_d, w.window, direct, out=out)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fbp.fb_blend_window(ctx, g_d, s_d, w.window, direct, out=out)
        b.record()
        torch.cuda.synchronize()
        fast_info["direct_ms_per_step"] = a.elapsed_time(b)
    roof = None
    if iter_n and ops:
        avg_s = iter_ms / iter_n / 1e3
        achieved = ops / avg_s / 1e12
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        probe_per_clk = rate / (sms * clocks["sm_mhz"] * 1e6) if clocks.get("sm_mhz") else None
        peak = DP4A_PER_CLK_SM * 4 * SM_COUNT_NOMINAL * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12
        roof = {"bound": "alu", "kernel": ("nnf_iter_balanced (Alg. 1 Jacobi iteration, Sec. 3.4 "
                                           "improved loss)" if balanced else
                                           "nnf_iter_balanced (Alg. 1 Jacobi iteration, Sec. 3.4 "
                                           "mean-remap loss)" if accurate else
                                           "nnf_iter_align (Alg. 1 Jacobi iteration, Eq. 10 "
                                           "alignment loss + Sec. 3.5.1 tracking)" if aligned else
                                           "nnf_iter_track (Alg. 1 Jacobi iteration with the "
                                           "tracking of Sec. 3.5.1)" if tracking else
                                           "nnf_iter (Alg. 1 Jacobi iteration)"),
                "achieved": achieved, "peak": peak, "unit": "T byte-pair ops/s",
                "frac": achieved / peak, "traffic": (None if args.window or args.frames
                                                      else TRAFFIC_PER_LAUNCH.get(args.workload)),
                "observed_limiter": LIMITER.get("k7" if w.patch == 7 else "k5"),
                "peak_basis": (f"{DP4A_PER_CLK_SM} dp4a/clk/SM x {SM_COUNT_NOMINAL} SMs x "
                               f"{SM_MAX_MHZ_NOMINAL:.0f} MHz x 4 byte pairs (derived; the live "
                               f"register-only probe measured {probe_per_clk:.1f} dp4a/clk/SM)"
                               if probe_per_clk else "derived"),
                "peak_chosen_mix": mix_rate / 1e12 if mix_rate else None,
                "frac_chosen_mix": achieved / (mix_rate / 1e12) if mix_rate else None,
                "chosen_mix_basis": (f"register-only probe of the k = {w.patch} kernels' Eq. 1 "
                                     "sequence (3 dp4a per word, " + ("20" if w.patch == 5 else "42") +
                                     " words" +
                                     " per candidate, accumulate + early-exit compare per slot), "
                                     "measured live" if mix_rate else None),
                "avg_launch_ms": iter_ms / iter_n, "launches": iter_n,
                "share_of_kernel_time": iter_ms / kernel_total_ms if kernel_total_ms else None,
                "candidate_evals_per_s": (w_job.candidate_evals() / world if shard else
                                          w.candidate_evals() * (fast_info["nnfs"] / w.pairs() if fast else 1)
                                          + (tracking_neighbour_refs(w) * w.H * w.W * w.iters
                                             if tracking else 0)
                                          if not learned else
                                          w.pairs() * w.H * w.W * (1 + args.learned_iters *
                                                                   (4 + w.random_search_radii())))
                * args.steps * world / (total_ms / 1e3),
                "probe_dp4a_per_s": rate}
        if roof["traffic"]:
            # The other side of the roofline: the launch's DRAM bytes (ncu) at the measured
            # copy bandwidth, against the ops at the measured rate of the kernel's own
            # instruction sequence; the fraction is the slower of the two over the launch.
            hbm_peak, hbm_basis = measured_peak("hbm_gbs", 6400.0)
            t_hbm = roof["traffic"] / (hbm_peak * 1e9)
            roof["hbm"] = {"traffic_bytes_per_launch": roof["traffic"],
                           "achieved_gbs": roof["traffic"] / avg_s / 1e9, "peak_gbs": hbm_peak,
                           "peak_basis": hbm_basis, "frac": roof["traffic"] / avg_s / 1e9 / hbm_peak,
                           "t_hbm_ms": t_hbm * 1e3}
            if mix_rate:
                t_int = ops / mix_rate
                roof["t_int_ms"] = t_int * 1e3
                roof["slower_bound"] = "alu" if t_int >= t_hbm else "hbm"
                roof["frac_max_bound"] = max(t_int, t_hbm) / avg_s
        if gather_rates and w.levels == 1:
            pairs_launch = shard["pairs"] if shard else w.pairs()
            sectors = SECTORS_PER_PIXEL_ITER[w.patch] * pairs_launch * w.H * w.W
            got = sectors / avg_s
            roof["gather"] = {
                "sectors_per_pixel_iter": SECTORS_PER_PIXEL_ITER[w.patch],
                "achieved_sectors_per_s": got,
                "peak_l1_resident": gather_rates["l1_resident"],
                "frac_l1_resident": got / gather_rates["l1_resident"],
                "peak_l2_resident": gather_rates["l2_resident"],
                "frac_l2_resident": got / gather_rates["l2_resident"],
                "basis": ("32-byte L1 sectors per launch (ncu count of the captured launch, per pair "
                          "and pixel) / the live launch time, against fb_probe_gather: independent "
                          "scattered 256-bit loads at the kernel's occupancy over a 64 KiB "
                          "(L1-resident) and a 4 MiB (L2-resident) buffer, measured live")}

    line = {
        "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": workload_label(args.workload, w, args.learned_iters),
                   "frames": w_job.N if shard else w.N, "height": w.H, "width": w.W,
                   "patch": w.patch, "window": w.window,
                   "iters": w.iters if not learned else args.learned_iters, "levels": w.levels,
                   "nnfs_per_step": (w_job.pairs() if shard else
                                     fast_info["nnfs"] if fast else w.pairs()),
                   "candidate_evals_per_step": (w_job.candidate_evals() if shard else
                                                w.candidate_evals()
                                                + (tracking_neighbour_refs(w) * w.H * w.W * w.iters
                                                   if tracking else 0) if not learned else
                                                w.pairs() * w.H * w.W * (1 + args.learned_iters *
                                                                         (4 + w.random_search_radii()))),
                   "learned_init": learned_info,
                   "fast_mode": fast_info,
                   "l2": f"flushed between steps ({FLUSH_BYTES >> 20} MiB write)",
                   "parallelism": (f"one {w_job.N}-frame clip split by output frame over {world} "
                                   f"GPUs ({w.N} per GPU, {w.window // 2}-frame input halo, "
                                   "fb_blend_window_range; no data-path collective)" if shard
                                   else f"{world} independent clip(s), one per GPU")},
        "roofline": roof,
        "e2e": e2e,
        "gpu_launches": launches,
        "kernel_ms": {k: v[0] / args.steps for k, v in prof.items() if v[1]},
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, g, s, args.cpu_sample_frames,
                                            BALANCED_ALPHA if balanced or accurate or aligned else None,
                                            fast, accurate, tracking, aligned)
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    grp.close()
    return 0


# ----------------------------------------------------------------------------------
# Batched submission: 32 clips of uneven size, length, window and patch
# ----------------------------------------------------------------------------------
BATCH_SEED = synth.clip_seed(3)
BATCH_ITERS = 6
# The batched workloads' manifests: 32 uneven clips of 256-1024 px (per-clip launches
# already fill the GPU), and 512 small clips of 64-128 px (a serving mix of thumbnails:
# one clip's launches fill a fraction of the SMs, and launches are many).
BATCH_MANIFESTS = {
    "batch_32": dict(n_clips=32, sizes=(256, 1024), frames=(16, 120), windows=(5, 31)),
    "batch_small": dict(n_clips=512, sizes=(64, 128), frames=(6, 12), windows=(3, 5)),
}
BATCH_DESCRIPTIONS = {
    "batch_32": "32 uneven clips (256-1024 px, 16-120 frames, windows 5-31, patch 5/7, n=6)",
    "batch_small": "512 small clips (64-128 px, 6-12 frames, windows 3-5, patch 5/7, n=6)",
}


def batch_manifest(workload: str, seed: int):
    return synth.batch_manifest(seed=seed, **BATCH_MANIFESTS[workload])


def batch_iter_ops(manifest) -> int:
    """Algorithmic byte-pair ops of all Jacobi-iteration launches of one submission."""
    tot = 0
    for N, H, W, window, patch in manifest:
        M = (window - 1) // 2
        pairs = sum(min(N - 1, i + M) - max(0, i - M) for i in range(N))
        R = int(math.floor(math.log2(max(H, W)))) + 1
        tot += pairs * H * W * (4 + R) * 3 * patch * patch
    return tot * BATCH_ITERS


def batch_candidate_evals(manifest) -> int:
    tot = 0
    for N, H, W, window, patch in manifest:
        M = (window - 1) // 2
        pairs = sum(min(N - 1, i + M) - max(0, i - M) for i in range(N))
        R = int(math.floor(math.log2(max(H, W)))) + 1
        tot += pairs * H * W * (1 + BATCH_ITERS * (4 + R))
    return tot


def run_gpu_batch(args):
    import torch

    import paper_2311_09265_b300 as fbp

    grp = RankGroup()
    rank, world, local = grp.rank, grp.world, grp.local
    local = rank_device(local)
    torch.cuda.set_device(local)
    fbp.build()
    manifest = batch_manifest(args.workload, shard_seed(BATCH_SEED, rank))
    picked = ([int(i) for i in args.batch_clips.split(",")] if args.batch_clips
              else list(range(len(manifest))))
    manifest = [manifest[i] for i in picked]
    clips, host = [], []
    for n, (N, H, W, window, patch) in zip(picked, manifest):
        g, s = synth.batch_clip(N, H, W, seed=shard_seed(BATCH_SEED, rank) + n)
        host.append((g, s))
        clips.append((torch.tensor(g, device="cuda"), torch.tensor(s, device="cuda"), window, patch,
                      torch.empty((N, H, W, 3), dtype=torch.float32, device="cuda")))
    frames = sum(m[0] for m in manifest)
    ctx = fbp.Context(local)
    params = fbp.Params.make(5, BATCH_ITERS, 1, 0, BATCH_SEED)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    t_build = time.perf_counter()
    fbp.fb_blend_batch(ctx, clips, params)        # the first call tunes, captures and runs
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t_build
    for _ in range(max(args.warmup, 1) - 1):
        fbp.fb_blend_batch(ctx, clips, params)
    torch.cuda.synchronize()
    grp.barrier()
    torch.cuda.synchronize()
    launches0 = ctx.launches
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            starts[k].record()
            fbp.fb_blend_batch(ctx, clips, params)   # graph replay
            ends[k].record()
        torch.cuda.synchronize()
    launches = ctx.launches - launches0
    grp.barrier()
    total_ms = grp.max(sum(a.elapsed_time(b) for a, b in zip(starts, ends)))
    value = aggregate(frames, args.steps, world, total_ms)
    clocks = clk.summary()

    modes = {k: ("per-clip launches" if fbp.fb_ctx_batch_mode(ctx, k) == 1 else "persistent")
             for k in (5, 7)}
    # Kernel breakdown: one untimed submission with direct launches and event timing.
    ctx.profile(True)
    fbp.fb_blend_batch(ctx, clips, params, flags=fbp.FB_BATCH_NO_GRAPH)
    prof = ctx.profile_read()
    ctx.profile(False)
    iter_ms, iter_n = prof["iter"]
    kernel_total_ms = sum(v[0] for v in prof.values())
    peak = DP4A_PER_CLK_SM * 4 * SM_COUNT_NOMINAL * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12
    achieved = batch_iter_ops(manifest) / (iter_ms / 1e3) / 1e12 if iter_ms else None
    roof = {"bound": "alu", "kernel": ("Alg. 1 Jacobi iterations of the batch: "
                                       + ", ".join(f"k={k} {'nnf_iter per clip' if m != 'persistent' else 'persistent batch_iter'}"
                                                   for k, m in modes.items())),
            "achieved": achieved, "peak": peak, "unit": "T byte-pair ops/s",
            "frac": achieved / peak if achieved else None, "traffic": None,
            "peak_basis": f"{DP4A_PER_CLK_SM} dp4a/clk/SM x {SM_COUNT_NOMINAL} SMs x "
                          f"{SM_MAX_MHZ_NOMINAL:.0f} MHz x 4 byte pairs (derived)",
            "avg_launch_ms": iter_ms / iter_n if iter_n else None, "launches": iter_n,
            "share_of_kernel_time": iter_ms / kernel_total_ms if kernel_total_ms else None,
            "candidate_evals_per_s": batch_candidate_evals(manifest) * args.steps * world
            / (total_ms / 1e3)}
    variants = {k: fbp.batch_variant_name(fbp.fb_ctx_batch_variant(ctx, k)) for k in (5, 7)}
    claims = {k: fbp.fb_ctx_batch_claim(ctx, k) for k in (5, 7)}

    # The same clips through one fb_blend_window call each, in the same run (one warm-up
    # loop so the per-call scratch exists, then one timed loop, L2 flushed first).
    def per_clip_loop():
        for g, s, window, patch, o in clips:
            fbp.fb_blend_window(ctx, g, s, window, fbp.Params.make(patch, BATCH_ITERS, 1, 0, BATCH_SEED), out=o)
    per_clip_loop()
    torch.cuda.synchronize()
    flush.zero_()
    la, lb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    la.record()
    per_clip_loop()
    lb.record()
    torch.cuda.synchronize()
    loop_ms = la.elapsed_time(lb)

    e2e = None
    if not args.no_e2e:
        # End to end: pinned host inputs copied in, outputs copied out, every step.
        hg = [torch.tensor(g).pin_memory() for g, _ in host]
        hs = [torch.tensor(s).pin_memory() for _, s in host]
        ho = [torch.empty(c[4].shape, dtype=torch.float32).pin_memory() for c in clips]
        grp.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            for (g, s, _, _, _), a, b in zip(clips, hg, hs):
                g.copy_(a, non_blocking=True)
                s.copy_(b, non_blocking=True)
            fbp.fb_blend_batch(ctx, clips, params)
            for c, o in zip(clips, ho):
                o.copy_(c[4], non_blocking=True)
            torch.cuda.synchronize()
        t_e2e = grp.max(time.perf_counter() - t0)
        e2e = {"value": world * frames * args.steps / t_e2e, "unit": "frames/s",
               "h2d_bytes_per_step": int(sum(a.numel() + b.numel() for a, b in zip(hg, hs))),
               "d2h_bytes_per_step": int(sum(o.numel() * 4 for o in ho))}

    line = {
        "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": (f"batched persistent submission of {BATCH_DESCRIPTIONS[args.workload]}"
                                + (f", manifest clips {args.batch_clips}" if args.batch_clips else "")),
                   "frames_per_step": frames, "clips": len(manifest),
                   "nnfs_per_step": sum(sum(min(N - 1, i + (w - 1) // 2) - max(0, i - (w - 1) // 2)
                                            for i in range(N)) for N, H, W, w, k in manifest),
                   "candidate_evals_per_step": batch_candidate_evals(manifest),
                   "tuned_modes": modes, "tuned_variants": variants, "tuned_tiles_per_claim": claims,
                   "first_call_s": t_build,
                   "per_clip_loop_ms": loop_ms,
                   "speedup_vs_per_clip_loop": loop_ms / (total_ms / args.steps),
                   "l2": f"flushed between steps ({FLUSH_BYTES >> 20} MiB write)",
                   "parallelism": f"{world} independent batch(es), one per GPU"},
        "roofline": roof, "e2e": e2e, "gpu_launches": launches,
        "kernel_ms": {k: v[0] for k, v in prof.items() if v[1]}, "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        N, H, W, window, patch = manifest[0]
        g, s = host[0]
        t0 = time.perf_counter()
        oracle.blend_frame(g, s, window, N // 2, patch, BATCH_ITERS, seed=BATCH_SEED)
        secs = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": 1.0 / secs, "unit": "frames/s",
                                "cores": oracle.num_threads(), "kind": "oracle",
                                "sample": f"output frame {N // 2} of clip 0 ({N}x{H}x{W}, window "
                                          f"{window}, patch {patch}); {secs:.1f} s"}
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    grp.close()
    return 0


# ----------------------------------------------------------------------------------
# learned initialiser alone: the forward pass of its convolution pyramid
# ----------------------------------------------------------------------------------
INITNET_PAIRS = 256
INITNET_DIVISORS = [1, 1, 2, 2, 4, 4, 8, 8, 4, 2, 1, 1]  # grid of each layer: (H/ds)/divisor


def initnet_flops_per_pair(H: int, W: int, ds: int) -> int:
    """2 * outputs * Cout * 9 * Cin summed over the twelve 3x3 convolutions."""
    from paper_2311_09265_b300.initnet_layout import LAYERS
    hq, wq = H // ds, W // ds
    return sum(2 * (hq // d) * (wq // d) * cout * 9 * cin
               for (cin, cout), d in zip(LAYERS, INITNET_DIVISORS))


def measured_peak(key: str, fallback: float):
    """A peak from MEASURED_PEAKS.json (copy bandwidth and cuBLAS bf16 throughput measured on
    this machine's GPUs), else the given fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key]), "measured"
    except (OSError, KeyError, ValueError):
        return fallback, "fallback"


def run_gpu_initnet(args):
    """One step = the initialiser's forward (input box means, 12 convolutions on the
    tensor cores, head) over 256 ordered pairs of the headline clip's 512x512 guides, with
    He-initialised weights (the time does not depend on the weight values)."""
    import numpy as np
    import torch

    import paper_2311_09265_b300 as fbp
    from paper_2311_09265_b300 import initnet_train

    grp = RankGroup()
    rank, world, local = grp.rank, grp.world, grp.local
    local = rank_device(local)
    torch.cuda.set_device(local)
    fbp.build()
    w = synth.WORKLOADS["blend_512"]
    g, _ = make_inputs(w, shard_seed(w.seed, rank))
    rng = np.random.default_rng(shard_seed(w.seed, rank))
    tgt_i = rng.integers(0, w.N, INITNET_PAIRS)
    src_j = np.clip(tgt_i + rng.choice([-3, -2, -1, 1, 2, 3], INITNET_PAIRS), 0, w.N - 1)
    g_d = torch.tensor(g, device="cuda")
    src, tgt = g_d[torch.tensor(src_j)].contiguous(), g_d[torch.tensor(tgt_i)].contiguous()
    ctx = fbp.Context(local)
    net = fbp.InitNet(ctx, INITNET_PAIRS, w.H, w.W, downscale=8)
    net.set_params(initnet_train.initial_params(net.n_params, 1))
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    for _ in range(max(args.warmup, 0)):
        net.forward(src, tgt)
    torch.cuda.synchronize()
    grp.barrier()
    launches0 = ctx.launches
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            starts[k].record()
            net.forward(src, tgt)
            ends[k].record()
        torch.cuda.synchronize()
    grp.barrier()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    total_ms = grp.max(sum(step_ms))
    flops = initnet_flops_per_pair(w.H, w.W, 8) * INITNET_PAIRS
    peak, basis = measured_peak("bf16_tflops", 1800.0)
    achieved = flops / (statistics.median(step_ms) / 1e3) / 1e12

    # One training step on the same pairs (forward, smooth-L1 loss, backward, Adam): the
    # twelve weight gradients and the input gradients of layers 1-11 cost a forward each,
    # 3 F - F(layer 0) FLOPs in all.  Context for the forward line, timed the same way.
    target = torch.zeros((INITNET_PAIRS, w.H // 8, w.W // 8, 2), dtype=torch.float32, device="cuda")
    for _ in range(max(args.warmup, 1)):
        net.train_step(src, tgt, target, lr=1e-6)
    torch.cuda.synchronize()
    from paper_2311_09265_b300.initnet_layout import LAYERS
    f0 = 2 * (w.H // 8) * (w.W // 8) * LAYERS[0][1] * 9 * LAYERS[0][0] * INITNET_PAIRS
    train_flops = 3 * flops - f0
    tms = []
    for _ in range(max(args.steps, 1)):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        net.train_step(src, tgt, target, lr=1e-6)
        b.record()
        torch.cuda.synchronize()
        tms.append(a.elapsed_time(b))
    assert net.status() == fbp.FB_OK
    train_ms = statistics.median(tms)
    train_tflops = train_flops / (train_ms / 1e3) / 1e12
    line = {
        "metric": "learned-initialiser forward: NNF pairs/s at 512x512 (64x64 grid)",
        "value": world * INITNET_PAIRS * args.steps / (total_ms / 1e3), "unit": "pairs/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": "learned-initialiser forward, 256 pairs of 512x512 guides, "
                               "downscale 8, 12 conv layers (779,592 parameters)",
                   "pairs_per_step": INITNET_PAIRS, "flops_per_pair": flops // INITNET_PAIRS,
                   "l2": f"flushed between steps ({FLUSH_BYTES >> 20} MiB write)",
                   "parallelism": f"{world} independent replica(s), one per GPU"},
        "roofline": {"bound": "tensor", "kernel": "whole forward (12 TMA-fed tcgen05 convolutions + "
                     "input, concatenation and head kernels)", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                     "peak_basis": f"bf16 dense, {basis} (cuBLAS burst)",
                     "train_step": {"ms": train_ms, "flops": train_flops, "achieved": train_tflops,
                                    "frac": train_tflops / peak,
                                    "what": "forward + loss + backward (12 weight gradients, input "
                                            "gradients of layers 1-11) + Adam, 256 pairs, median of "
                                            f"{len(tms)}"}},
        "e2e": None, "gpu_launches": ctx.launches - launches0, "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line))
    net.close()
    ctx.close()
    grp.close()
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in BATCH_MANIFESTS:
        return run_gpu_batch(args)
    if args.workload == "initnet_512":
        return run_gpu_initnet(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
