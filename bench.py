#!/usr/bin/env python
"""Benchmark of the skew-Gaussian rasterizer on one GB300 (or N replicas).

Workload (default ``unbounded_1m``): 1M skew Gaussians (60% in a ball of
radius 2, 40% on a shell of radius 20-50), SH degree 3, one 1920x1080 view
on a radius-6 orbit, upstream image gradient ~ N(0,1).  A step is one pass
of the hot path: sr_preprocess, sr_bin_sort, sr_render_fwd, sr_render_bwd
(which includes the projection backward).  Inputs are resident in HBM when
the timed region starts; L2 is flushed (a 256 MiB memset) before every
timed step, outside the step's CUDA events.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the same workload instead, one full forward + backward frame per
step.
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
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd / fwd+bwd frames/s, 1M skew Gaussians at 1080p: batched+BF16 vs plain FP32"
UNIT = "frames/s"
HBM_FALLBACK = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1_000_000, help="Gaussians (default: the 1M workload)")
    ap.add_argument("--no-variants", action="store_true", help="only the headline FP32 fwd+bwd form")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end (host buffers) measurement")
    ap.add_argument("--oracle-threads", type=int, default=0,
                    help="threads of the FP64 oracle (CPU baseline and reference arm; 0: all cores)")
    ap.add_argument("--workload", default="unbounded_1m", choices=["unbounded_1m", "mixed_5m"])
    ap.add_argument("--fwd-px", type=int, default=0, choices=[0, 1, 2, 4],
                    help="forward pixels per thread (0: autotune)")
    ap.add_argument("--bwd-px", type=int, default=0, choices=[0, 1, 2, 4],
                    help="backward pixels per thread (0: autotune)")
    ap.add_argument("--fwd-batch", type=int, default=256, choices=[128, 256, 512],
                    help="forward records per staged batch when the launch shape is fixed")
    ap.add_argument("--bwd-batch", type=int, default=128, choices=[128, 256],
                    help="backward records per staged batch when the launch shape is fixed")
    ap.add_argument("--fwd-blocks", type=int, default=0, help="forward blocks per SM cap when the shape is fixed")
    ap.add_argument("--bwd-blocks", type=int, default=0, help="backward blocks per SM cap when the shape is fixed")
    ap.add_argument("--persistent", type=int, default=0, choices=[0, 1, 2, 3],
                    help="persistent composites (bit 0 forward, bit 1 backward) when the shape is fixed")
    return ap.parse_args()


COUNTERS = os.path.join(ROOT, "profiles", "render_counters_unbounded_500k_1080p.json")
KERNEL_SOURCES = ("render.cu", "common.cuh")


def render_counters():
    """ncu counters of the two composites from a capture of a smaller frame
    (instruction counts per pair, DRAM bytes per launch) and whether the
    kernel sources are still the ones the capture was taken with."""
    import hashlib

    try:
        d = json.load(open(COUNTERS))
    except Exception:
        return None, False
    src = b"".join(open(os.path.join(ROOT, "paper_2605_18334_gb300", "csrc", f), "rb").read() for f in KERNEL_SOURCES)
    return d, hashlib.sha256(src).hexdigest() == d.get("source_sha256")


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------

def workload(n):
    from paper_2605_18334_gb300 import scenes

    sc = scenes.unbounded(seed=2, n=n)
    cam = scenes.orbit_camera(0.0, 1920, 1080)
    up = scenes.upstream_grad(2, 1080, 1920)
    return sc, cam, up


def config_dict(n):
    return {"workload": "unbounded_1m" if n == 1_000_000 else f"unbounded_{n}", "gaussians": n,
            "resolution": "1920x1080", "views": 1, "sh_degree": 3, "skew": "N(0,1.5^2) local frame",
            "step": "preprocess+bin_sort+render_fwd+render_bwd", "l2": "flushed (256 MiB memset) before each step"}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id=None):
        self.bus_id = bus_id
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.bus_id:
                cmd += ["-i", self.bus_id]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# distributed helpers (one process per GPU; no data-path collective)
# ---------------------------------------------------------------------------

def dist_setup(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    """The largest of the ranks' values (timing only; no data-path collective)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------

def run_ours(args):
    import torch

    from paper_2605_18334_gb300 import native as N
    from paper_2605_18334_gb300.rasterizer import Config, Gaussians, Rasterizer

    rank, world = dist_setup(args)
    dev = torch.device("cuda", torch.cuda.current_device())
    sc, cam, up = workload(args.n)
    g = Gaussians.from_scene(sc, device=dev)
    cfg = Config()
    r = Rasterizer(g, [cam], cfg, key_capacity=int(12 * args.n))
    d_img = torch.as_tensor(up, device=dev).reshape(-1).contiguous()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step(gs, rr, dimg, backward=True):
        rr.forward(gs)
        if backward:
            return rr.backward(gs, dimg)
        return None

    if args.fwd_px and args.bwd_px:  # fixed launch shapes (e.g. for a profiler run)
        r.set_pixels_per_thread(args.fwd_px, args.bwd_px)
        r.set_batch(args.fwd_batch, args.bwd_batch)
        r.set_blocks_per_sm(args.fwd_blocks, args.bwd_blocks)
        r.set_persistent(bool(args.persistent & 1), bool(args.persistent & 2))
        tune = {"fwd_pixels_per_thread": args.fwd_px, "bwd_pixels_per_thread": args.bwd_px, "fwd_ms": {},
                "bwd_ms": {}, "fixed": True}
    else:
        tune = r.autotune(g, d_img)
    for _ in range(max(3, args.warmup)):
        step(g, r, d_img)
    torch.cuda.synchronize()

    K = args.steps
    NS = 5
    names = ["preprocess", "bin_sort", "render_fwd", "render_bwd_composite", "render_bwd_project"]
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(NS + 1)] for _ in range(K)]
    props = torch.cuda.get_device_properties(dev)
    bus = getattr(props, "pci_bus_id", None)
    launches0 = N.sr_kernel_launches()
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(bus if isinstance(bus, str) else None) as clk:
        for k in range(K):
            flush.zero_()
            e = ev[k]
            e[0].record(stream)
            r.preprocess(g)
            e[1].record(stream)
            r.keys = r.bin_sort()
            e[2].record(stream)
            r.render_fwd()
            e[3].record(stream)
            r.backward_composite(d_img)
            e[4].record(stream)
            r.backward_project(g)
            e[5].record(stream)
        torch.cuda.synchronize()
        launches = N.sr_kernel_launches() - launches0
        # the composites' arithmetic roofs, measured at the clock of this run
        alu = N.sr_measure_alu_peaks(flush.data_ptr(), stream.cuda_stream)
    barrier(world)
    stage_ms = np.array([[ev[k][i].elapsed_time(ev[k][i + 1]) for i in range(NS)] for k in range(K)])
    step_ms = stage_ms.sum(1)
    total_ms = max_over_ranks(float(step_ms.sum()), world)
    ms_per_step = total_ms / K
    value = world * K / (total_ms / 1e3)
    tested, blended = N.sr_frame_counters(r.plan, r.ws.data_ptr(), stream.cuda_stream)
    replayed = int(r.n_contrib.to(torch.int64).sum().item())
    clocks = clk.summary()

    cfgd = config_dict(args.n)
    cfgd["launch"] = {"fwd_pixels_per_thread": tune["fwd_pixels_per_thread"],
                      "bwd_pixels_per_thread": tune["bwd_pixels_per_thread"],
                      "fwd_batch": r.config.fwd_batch or 256, "bwd_batch": r.config.bwd_batch or 128,
                      "fwd_blocks_per_sm": r.config.fwd_blocks_per_sm, "bwd_blocks_per_sm": r.config.bwd_blocks_per_sm,
                      "persistent": r.config.persistent, "autotuned": not tune.get("fixed")}
    out = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": K,
           "warmup": max(3, args.warmup), "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfgd,
           "gpu_launches": int(launches)}
    fwd_ms = stage_ms[:, :3].sum(1).mean()
    stage_mean = stage_ms.mean(0)
    out["stages_ms"] = {k: round(float(v), 4) for k, v in zip(names, stage_mean)}
    out["fwd_frames_per_s"] = round(1e3 / fwd_ms, 2)
    out["keys"] = int(r.keys)
    out["pairs_tested"] = tested
    out["pairs_replayed_bwd"] = replayed
    out["pairs_blended"] = blended
    out["blends_per_s"] = round(blended / (stage_mean[2] / 1e3), 1)
    out["pairs_tested_per_s"] = round(tested / (stage_mean[2] / 1e3), 1)
    out["clocks"] = clocks
    out["autotune_ms"] = {"fwd": {str(k): round(v, 4) for k, v in tune["fwd_ms"].items()},
                          "bwd": {str(k): round(v, 4) for k, v in tune["bwd_ms"].items()},
                          "fwd_batch": {str(k): round(v, 4) for k, v in tune.get("fwd_batch_ms", {}).items()},
                          "bwd_batch": {str(k): round(v, 4) for k, v in tune.get("bwd_batch_ms", {}).items()},
                          "fwd_blocks_per_sm": {str(k): round(v, 4) for k, v in
                                                tune.get("fwd_blocks_per_sm_ms", {}).items()},
                          "bwd_blocks_per_sm": {str(k): round(v, 4) for k, v in
                                                tune.get("bwd_blocks_per_sm_ms", {}).items()},
                          "fwd_persistent": {str(k): round(v, 4) for k, v in tune.get("fwd_persistent_ms", {}).items()},
                          "bwd_persistent": {str(k): round(v, 4) for k, v in tune.get("bwd_persistent_ms", {}).items()}}

    # roofline of the dominant stage (measured live with the events above)
    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", HBM_FALLBACK))
    sms = props.multi_processor_count
    # FP32 lane results per second: the faster of scalar and packed FP32x2
    # FMA, as measured by sr_measure_alu_peaks in this run
    alu_peak = max(alu["fma_lane_ops_per_s"], alu["ffma2_lane_ops_per_s"]) / 1e12
    # work per launch of the composites: FP32 lane results (FADD, FMUL and FFMA
    # thread instructions, the packed FP32x2 forms counted twice) per tested
    # (forward) or replayed (backward) pair from the ncu capture of the
    # smaller frame, times this frame's pairs; nominal counts (25 per tested
    # pair, 25 per replayed + 60 per blended pair) when the kernels changed
    cnt, fresh = render_counters()
    nominal = {2: tested * 25, 3: replayed * 25 + blended * 60}
    units = {2: (tested, "pairs_tested"), 3: (replayed, "pairs_replayed_bwd")}
    ops, ops_source, issue = {}, {}, {}
    for k, kname in ((2, "render_fwd"), (3, "render_bwd_composite")):
        kc = cnt["kernels"].get(kname) if cnt else None
        if kc and fresh:
            scale = units[k][0] / cnt[units[k][1]]
            ops[k] = kc["fp32_lane_results"] * scale
            ops_source[k] = (f"ncu counters of a {cnt['keys']}-key frame, scaled by {units[k][1]} "
                             f"({cnt[units[k][1]]} -> {units[k][0]})")
            issue[k] = kc["warp_instructions"] * scale / (sms * 4 * (clocks.get("sm_mhz") or 2070.0) * 1e6 *
                                                          stage_mean[k] / 1e3)
        else:
            ops[k] = nominal[k]
            ops_source[k] = "nominal (25 FP32 operations per tested pair; 25 per replayed + 60 per blended pair)"
    pre_bytes = args.n * 248 + args.n * 20 + int((r.tile_counts() > 0).sum()) * 64
    nrec = int((r.tile_counts() > 0).sum())
    proj_bytes = args.n * (248 + 4) + nrec * 64 + args.n * 248
    bytes_ = {0: pre_bytes, 4: proj_bytes}
    dom = int(np.argmax(stage_mean))
    traffic = None
    if cnt and fresh and args.n == 1_000_000:
        kc = cnt["kernels"].get(names[dom], {})
        traffic = kc.get("dram_bytes_unbounded_1m")  # captured on this frame itself
    if dom in ops:
        achieved = ops[dom] / (stage_mean[dom] / 1e3) / 1e12
        out["roofline"] = {"kernel": names[dom], "bound": "alu", "achieved": round(achieved, 3),
                           "peak": round(alu_peak, 3), "unit": "TFLOP/s", "frac": round(achieved / alu_peak, 4),
                           "traffic": traffic,
                           "peak_source": "measured in this run (sr_measure_alu_peaks: FP32 lane results/s)",
                           "work_source": ops_source[dom]}
        if dom in issue:
            out["roofline"]["issue_slot_utilisation"] = round(issue[dom], 4)
    else:
        b = bytes_.get(dom, 0)
        achieved = b / (stage_mean[dom] / 1e3) / 1e9
        out["roofline"] = {"kernel": names[dom], "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm,
                           "unit": "GB/s", "frac": round(achieved / hbm, 4), "traffic": None}
    out["other_stages"] = {
        "render_fwd_TFLOPs": round(ops[2] / (stage_mean[2] / 1e3) / 1e12, 3),
        "render_fwd_work_source": ops_source[2],
        "issue_slot_utilisation": {names[k]: round(v, 4) for k, v in issue.items()},
        "render_bwd_composite_TFLOPs": round(ops[3] / (stage_mean[3] / 1e3) / 1e12, 3),
        "alu_peak_TFLOPs": round(alu_peak, 3),
        "alu_peaks_measured_per_s": {k: (round(v / 1e12, 3) if k != "seconds" else round(v, 4))
                                     for k, v in alu.items()},
        "preprocess_GBps": round(pre_bytes / (stage_mean[0] / 1e3) / 1e9, 1),
        "render_bwd_project_GBps": round(proj_bytes / (stage_mean[4] / 1e3) / 1e9, 1),
        "bin_sort_GBps": round((args.n * 4 * 16 + int(r.keys) * (8 + 16 * r.plan.sort_passes + 8)) /
                               (stage_mean[1] / 1e3) / 1e9, 1),
        "hbm_peak_GBps": hbm}

    if not args.no_variants:
        out["variants"] = variants(args, sc, cam, up, dev, flush)
        out["variants"]["trajectory_64"] = trajectory(args, sc, dev, flush)
        out["variants"]["train_step"] = train_step(args, sc, cam, dev, flush)
        out["variants"]["densify"] = densify_step(args, sc, dev, flush)
    if not args.no_e2e:
        out["e2e"] = e2e(args, sc, cam, up, dev, world)
        if not args.no_variants:
            # the same end-to-end step with BF16 storage of SH, log-scales and
            # skew: the host-to-device bytes shrink, the gradients stay FP32
            out["variants"]["bf16_storage_e2e"] = e2e(args, sc, cam, up, dev, world, storage=torch.bfloat16)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(sc, cam, up, args.oracle_threads)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def timed(fn, K, flush, stream):
    import torch

    ts = []
    for _ in range(K):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        ts.append((a, b))
    torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in ts]))


def variants(args, sc, cam, up, dev, flush):
    import torch

    from paper_2605_18334_gb300.rasterizer import Config, Gaussians, Rasterizer

    K = max(5, args.steps // 2)
    stream = torch.cuda.current_stream()
    res = {}
    d_img = torch.as_tensor(up, device=dev).reshape(-1).contiguous()
    for name, dt in (("fp32", torch.float32), ("bf16_storage", torch.bfloat16)):
        g = Gaussians.from_scene(sc, device=dev, sh_dtype=dt, scale_dtype=dt, skew_dtype=dt)
        r = Rasterizer(g, [cam], Config(), key_capacity=int(12 * args.n))
        r.autotune(g, d_img)
        for _ in range(3):
            r.forward(g)
            r.backward(g, d_img)
        fwd = timed(lambda: r.forward(g), K, flush, stream)
        fb = timed(lambda: (r.forward(g), r.backward(g, d_img)), K, flush, stream)
        res[name] = {"fwd_frames_per_s": round(1e3 / fwd, 2), "fwdbwd_frames_per_s": round(1e3 / fb, 2)}
        if name == "fp32":
            # a render-only plan (no blend masks, no backward state): what a viewer uses
            rf = Rasterizer(g, [cam], Config(forward_only=True), key_capacity=int(12 * args.n))
            rf.autotune(g)
            for _ in range(3):
                rf.forward(g)
            res["fp32_forward_only_plan"] = {"fwd_frames_per_s": round(1e3 / timed(lambda: rf.forward(g), K, flush,
                                                                                     stream), 2)}
            del rf
        del r, g
        torch.cuda.empty_cache()
    # batched + BF16: 8 views of the orbit at 1080p in one plan, BF16 SH,
    # log-scale and skew storage, forward and forward+backward
    from paper_2605_18334_gb300 import scenes

    cams8 = scenes.trajectory_cameras(8, resolutions=((1920, 1080),))
    g = Gaussians.from_scene(sc, device=dev, sh_dtype=torch.bfloat16, scale_dtype=torch.bfloat16,
                             skew_dtype=torch.bfloat16)
    r = Rasterizer(g, cams8, Config(), key_capacity=int(12 * args.n * 8))
    up8 = torch.cat([torch.as_tensor(scenes.upstream_grad(70 + v, 1080, 1920), device=dev).reshape(-1)
                     for v in range(8)]).contiguous()
    r.autotune(g, up8)
    for _ in range(3):
        r.forward(g)
        r.backward(g, up8)
    fwd = timed(lambda: r.forward(g), K, flush, stream)
    fb = timed(lambda: (r.forward(g), r.backward(g, up8)), K, flush, stream)
    res["batched8_bf16"] = {"views": 8, "fwd_frames_per_s": round(8e3 / fwd, 2),
                            "fwdbwd_frames_per_s": round(8e3 / fb, 2), "keys": int(r.keys)}
    del r, g
    torch.cuda.empty_cache()
    return res


def train_step(args, sc, cam, dev, flush):
    """Training step at the headline frame: render, photometric loss (L1 +
    D-SSIM) and its gradient, backward to every attribute, one Adam update of
    all 62 FP32 values per Gaussian; per-stage CUDA events, L2 flushed before
    each step.  The target is a fixed synthetic image (uniform noise)."""
    import numpy as np
    import torch

    from paper_2605_18334_gb300.rasterizer import Gaussians
    from paper_2605_18334_gb300.train import Trainer

    K = max(5, args.steps // 2)
    stream = torch.cuda.current_stream()
    g = Gaussians.from_scene(sc, device=dev)
    target = torch.as_tensor(np.random.default_rng(3).uniform(0, 1, 3 * 1080 * 1920).astype(np.float32),
                             device=dev).contiguous()
    tr = Trainer(g, [cam], target, key_capacity=int(12 * args.n))
    tr.rast.autotune(g, target)
    for _ in range(3):
        tr.step()
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(K)]
    for k in range(K):
        flush.zero_()
        e = ev[k]
        e[0].record(stream)
        tr.rast.forward(g)
        e[1].record(stream)
        tr.loss(target)
        e[2].record(stream)
        tr.grads = tr.rast.backward(g, tr.loss.d_images, out=tr.grads)
        e[3].record(stream)
        tr.adam.step(tr.grads)
        e[4].record(stream)
    torch.cuda.synchronize()
    ms = np.array([[ev[k][i].elapsed_time(ev[k][i + 1]) for i in range(4)] for k in range(K)]).mean(0)
    n_vals = sum(getattr(g, f).numel() for f in ("means", "log_scales", "quats", "opacity_logits", "skew", "sh"))
    adam_bytes = n_vals * 28  # read param, grad, m, v; write param, m, v (FP32)
    out = {"steps_per_s": round(1e3 / ms.sum(), 2),
           "stages_ms": {"forward": round(ms[0], 4), "loss": round(ms[1], 4), "backward": round(ms[2], 4),
                         "adam": round(ms[3], 4)},
           "adam_GBps": round(adam_bytes / (ms[3] / 1e3) / 1e9, 1), "loss": round(float(tr.loss.loss.item()), 6)}
    del tr, g
    torch.cuda.empty_cache()
    return out


def densify_step(args, sc, dev, flush):
    """One densification of the 1M scene (remove / keep / clone / split from
    seeded synthetic statistics, thresholds that densify about a fifth of
    the Gaussians), device time of sr_densify with the L2 flushed before
    each call; algorithmic bytes: every input Gaussian and its statistics
    read once, every output Gaussian and its map entry written once."""
    import numpy as np
    import torch

    from paper_2605_18334_gb300 import native as N
    from paper_2605_18334_gb300.densify import densify
    from paper_2605_18334_gb300.rasterizer import Gaussians, _stream_ptr

    g = Gaussians.from_scene(sc, device=dev)
    n = g.n
    rng = np.random.default_rng(11)
    uv = torch.as_tensor(rng.exponential(0.1, n).astype(np.float32), device=dev)
    seen = torch.as_tensor(rng.integers(1, 8, n).astype(np.int32), device=dev)
    zm = torch.as_tensor(rng.exponential(0.05, n).astype(np.float32), device=dev)
    cfg = dict(grad_uv=0.04, grad_z=0.2, log_scale_split=-3.5, logit_prune=-2.5)
    res = densify(g, uv, seen, zm, **cfg)  # sizes, and the output arrays the timed calls rewrite
    cap = 2 * n
    outs = [torch.empty(cap, 3, device=dev), torch.empty(cap, 3, device=dev), torch.empty(cap, 4, device=dev),
            torch.empty(cap, device=dev), torch.empty(cap, 3, device=dev), torch.empty(cap, g.sh[0].numel(), device=dev)]
    arrays = N.sr_scene_arrays(*[t.data_ptr() for t in outs[:5]], None, outs[5].data_ptr())
    src_map = torch.empty(cap, dtype=torch.int32, device=dev)
    counts = torch.zeros(4, dtype=torch.int64, device=dev)
    scratch = torch.empty(N.sr_densify_scratch_size(n), dtype=torch.uint8, device=dev)
    c_cfg = N.sr_densify_config(cfg["grad_uv"], cfg["grad_z"], cfg["log_scale_split"], cfg["logit_prune"])
    gc = g.to_c()
    stream = torch.cuda.current_stream()

    def call():
        N.sr_densify(gc, uv.data_ptr(), seen.data_ptr(), zm.data_ptr(), c_cfg, arrays, src_map.data_ptr(),
                     counts.data_ptr(), scratch.data_ptr(), _stream_ptr(stream))

    for _ in range(3):
        call()
    ts = []
    for _ in range(10):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        call()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    ms = float(np.median(ts))
    per_g = 4 * (3 + 3 + 4 + 1 + 3 + g.sh[0].numel())
    nbytes = n * (per_g + 12) + res.counts["total"] * (per_g + 4)
    out = {"ms": round(ms, 4), "counts": res.counts, "GBps": round(nbytes / (ms / 1e3) / 1e9, 1),
           "input_gaussians_per_s": round(n / (ms / 1e3), 1)}
    del g, res, outs
    torch.cuda.empty_cache()
    return out


def trajectory(args, sc, dev, flush, n_views=64):
    """Batched camera trajectory: n_views cameras on the closed spline orbit,
    resolutions cycling 640x360 / 1280x720 / 1920x1080, forward only.  One
    plan over all views (shared key pool, one composite launch over every
    tile), captured once in a CUDA graph and replayed, against the same views
    rendered one by one with single-view plans."""
    import torch

    from paper_2605_18334_gb300 import scenes
    from paper_2605_18334_gb300.rasterizer import Config, Gaussians, Rasterizer

    cams = scenes.trajectory_cameras(n_views)
    g = Gaussians.from_scene(sc, device=dev)
    stream = torch.cuda.current_stream()
    r = Rasterizer(g, cams, Config(forward_only=True))
    r.forward(g)  # sizes the key pool (grows the plan once)
    r.autotune(g)
    r.forward(g)
    keys = int(r.keys)
    s = torch.cuda.Stream()
    s.wait_stream(stream)
    with torch.cuda.stream(s):
        r.preprocess(g, s)
        r.bin_sort(s, sync=False)
        r.render_fwd(s)
    stream.wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        r.preprocess(g, s)
        r.bin_sort(s, sync=False)
        r.render_fwd(s)
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    K = max(3, args.steps // 4)
    ms_graph = timed(graph.replay, K, flush, stream)
    # the composite alone, one block per tile against a persistent grid
    composite = {}
    chosen = r.config.persistent
    for pers in (0, 1):
        r.set_persistent(fwd=bool(pers))
        for _ in range(3):
            r.render_fwd()
        composite["persistent" if pers else "block_per_tile"] = round(timed(lambda: r.render_fwd(), K, flush,
                                                                            stream), 4)
    r.config.persistent = chosen
    r.cfg_c = r.config.to_c()
    # the same views one by one, each with its own plan (sized beforehand)
    singles = []
    for c in cams:
        rs = Rasterizer(g, [c], Config(forward_only=True))
        rs.forward(g)
        singles.append(rs)
    torch.cuda.synchronize()

    def sequential():
        for rs in singles:
            rs.forward(g)

    for _ in range(3):
        sequential()
    ms_seq = timed(sequential, K, flush, stream)
    res = {"views": n_views, "resolutions": "640x360/1280x720/1920x1080 cycling", "keys": keys,
           "batched_graph_fwd_views_per_s": round(n_views / (ms_graph / 1e3), 2),
           "sequential_fwd_views_per_s": round(n_views / (ms_seq / 1e3), 2),
           "batched_ms": round(ms_graph, 3), "sequential_ms": round(ms_seq, 3),
           "composite_ms": composite,
           "launch": {"fwd_pixels_per_thread": r.config.fwd_pixels_per_thread, "fwd_batch": r.config.fwd_batch,
                      "fwd_blocks_per_sm": r.config.fwd_blocks_per_sm, "persistent": r.config.persistent}}
    del singles, r, graph
    torch.cuda.empty_cache()
    return res


def _layout(specs):
    """Byte offsets of (name, shape, dtype) fields packed into one flat buffer,
    each on a 256-byte boundary, and the buffer's size."""
    import torch

    offs, off = [], 0
    for _, shape, dt in specs:
        off = (off + 255) & ~255
        n = math.prod(shape) * torch.empty((), dtype=dt).element_size()
        offs.append((off, n))
        off += n
    return offs, off


def _carve(buf, specs):
    """Views of the flat uint8 buffer ``buf`` laid out by ``_layout``."""
    offs, _ = _layout(specs)
    return {name: buf[o:o + n].view(dt).view(shape) for (name, shape, dt), (o, n) in zip(specs, offs)}


def e2e(args, sc, cam, up, dev, world, storage=None):
    """Same metric through the C ABI with host buffers: every step copies the
    scene and the upstream gradient from pinned host memory, renders forward
    and backward, and reads the image and all gradients back into pinned host
    memory.  Inputs and results each live in one flat buffer per side (the
    attribute, image and gradient tensors are views of it), so a step is one
    host-to-device and one device-to-host copy.  The copies run on their own
    streams (one per direction) into and out of double buffers, so step k's
    transfers overlap the compute of its neighbours; the timed region covers
    all K steps' copies and compute.  ``storage``: dtype of the SH, log-scale
    and skew arrays on the host and the device (their gradients stay FP32)."""
    import torch

    from paper_2605_18334_gb300.rasterizer import Config, Gaussians, Rasterizer

    fields = ("means", "log_scales", "quats", "opacity_logits", "skew", "sh")
    st = storage or torch.float32
    src = Gaussians.from_scene(sc, device="cpu", sh_dtype=st, scale_dtype=st, skew_dtype=st)
    up_t = torch.as_tensor(up).reshape(-1).contiguous()
    in_specs = [(k, tuple(getattr(src, k).shape), getattr(src, k).dtype) for k in fields]
    in_specs.append(("upstream", tuple(up_t.shape), torch.float32))
    _, in_bytes = _layout(in_specs)

    def gaussians(v):
        return Gaussians(*(v[k] for k in fields), src.sh_degree)

    host_in = torch.empty(in_bytes, dtype=torch.uint8).pin_memory()
    hv = _carve(host_in, in_specs)
    for k in fields:
        hv[k].copy_(getattr(src, k))
    hv["upstream"].copy_(up_t)
    dev_in = [torch.empty(in_bytes, dtype=torch.uint8, device=dev) for _ in range(2)]
    dv = [_carve(b, in_specs) for b in dev_in]
    for b in range(2):  # both buffers hold a real frame before anything runs on them
        dev_in[b].copy_(host_in)
    r = Rasterizer(gaussians(dv[0]), [cam], Config(), key_capacity=int(12 * args.n))
    r.autotune(gaussians(dv[0]), dv[0]["upstream"])
    out_specs = [("image", tuple(r.images.shape), torch.float32)]
    out_specs += [(k, tuple(getattr(src, k).shape), torch.float32) for k in fields]
    _, out_bytes = _layout(out_specs)
    dev_out = [torch.empty(out_bytes, dtype=torch.uint8, device=dev) for _ in range(2)]
    ov = [_carve(b, out_specs) for b in dev_out]
    gout = [{k: ov[i][k] for k in fields} | {"split_dir": None} for i in range(2)]
    host_out = [torch.empty(out_bytes, dtype=torch.uint8).pin_memory() for _ in range(2)]
    h2d, d2h = in_bytes, out_bytes
    comp = torch.cuda.current_stream()
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(2)]    # inputs of buffer i landed
    ev_done = [torch.cuda.Event() for _ in range(2)]  # compute on buffer i finished
    ev_out = [torch.cuda.Event() for _ in range(2)]   # results of buffer i read back
    for e in ev_done + ev_out:
        e.record(comp)

    def copy_in(i):
        with torch.cuda.stream(s_in):
            s_in.wait_event(ev_done[i])
            dev_in[i].copy_(host_in, non_blocking=True)
            ev_in[i].record(s_in)

    def compute(i):
        comp.wait_event(ev_in[i])
        comp.wait_event(ev_out[i])
        g = gaussians(dv[i])
        r.forward(g, out=ov[i]["image"], sync=False)  # no host stall per frame; capacity checked after the run
        r.backward(g, dv[i]["upstream"], out=gout[i])
        ev_done[i].record(comp)

    def copy_out(i):
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_done[i])
            host_out[i].copy_(dev_out[i], non_blocking=True)
            ev_out[i].record(s_out)

    def run(steps):
        copy_in(0)
        for k in range(steps):
            if k + 1 < steps:
                copy_in((k + 1) % 2)
            compute(k % 2)
            copy_out(k % 2)
        torch.cuda.synchronize()

    run(max(3, args.warmup))
    # three timed runs of K steps, the median reported: the host link is
    # shared with the node's other GPUs, and one short run can catch a
    # neighbour's transfer
    K = max(10, args.steps)
    rates = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run(K)
        dt = max_over_ranks(time.perf_counter() - t0, world)
        rates.append(world * K / dt)
    r.check()  # the frames (all of the same scene) fitted the key capacity; raises otherwise
    return {"value": round(statistics.median(rates), 3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "runs": [round(x, 3) for x in rates], "steps_per_run": K,
            "copies": "one flat buffer per direction and step, double-buffered, overlapped with compute"}


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# ---------------------------------------------------------------------------

def oracle_frame(sc, cam, up):
    """One full frame of the FP64 oracle, timed on the host cores: the
    projection of every Gaussian, the composite of every pixel (mode B: each
    pixel's list of the Gaussians whose footprint reaches it, in depth order;
    the same result as brute force over every Gaussian), and the backward of
    the dense upstream gradient at every pixel through the projection.
    Returns (forward seconds, forward + backward seconds)."""
    import oracle

    oracle.build()
    oc = oracle.camera_from_gl(cam)
    ocfg = oracle.config()
    t0 = time.perf_counter()
    pre = oracle.preprocess(sc, oc, ocfg)
    oracle.render_frame(sc, oc, ocfg, pre=pre)
    t1 = time.perf_counter()
    oracle.render_backward(sc, oc, ocfg, up, pre=pre, frame=True)
    t2 = time.perf_counter()
    return t1 - t0, t2 - t0


def _oracle_sample(sc, cam):
    return (f"one full {cam['width']}x{cam['height']} frame of all {sc.n} Gaussians: projection, composite of every "
            f"pixel and backward of an upstream gradient at every pixel (FP64, per-pixel footprint lists)")


def cpu_baseline(sc, cam, up, threads=0):
    import oracle

    oracle.build()
    if threads:
        oracle.set_num_threads(threads)
    fwd_s, frame_s = oracle_frame(sc, cam, up)
    return {"value": round(1.0 / frame_s, 6), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": _oracle_sample(sc, cam), "fwd_frames_per_s": round(1.0 / fwd_s, 6),
            "seconds": round(frame_s, 2)}


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands on the host cores, one
    full forward + backward frame of the workload per step."""
    import oracle

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    oracle.build()
    if args.oracle_threads:
        oracle.set_num_threads(args.oracle_threads)
    sc, cam, up = workload(args.n)
    for _ in range(args.warmup):
        oracle_frame(sc, cam, up)
    t0 = time.perf_counter()
    frames = [oracle_frame(sc, cam, up) for _ in range(args.steps)]
    wall = time.perf_counter() - t0
    ms = 1e3 * float(np.mean([f[1] for f in frames]))
    value = 1e3 / ms
    out = {"metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_dict(args.n),
           "impl": "reference",
           "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                            "sample": _oracle_sample(sc, cam),
                            "fwd_frames_per_s": round(1e3 / (1e3 * float(np.mean([f[0] for f in frames]))), 6)},
           "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "gpu_launches": 0, "wall_s": round(wall, 1)}
    print(json.dumps(out), flush=True)


def run_mixed_5m(args):
    """5M Gaussians (config-3 geometry, half with skew exactly 0, the rest
    skew ~ N(0, 2^2)), SH degree 3 stored in BF16:
      A. a 32-view 3840x2160 trajectory, forward only, 8 views per plan;
      B. an 8-view 1920x1080 forward+backward step, as one batched plan and
         with the tile key lists rebuilt for the backward (one workspace)."""
    import torch

    from paper_2605_18334_gb300 import scenes
    from paper_2605_18334_gb300.rasterizer import Config, Gaussians, Rasterizer, render_views_recompute

    rank, world = dist_setup(args)
    dev = torch.device("cuda", torch.cuda.current_device())
    sc = scenes.mixed_5m()
    g = Gaussians.from_scene(sc, device=dev, sh_dtype=torch.bfloat16)
    del sc
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    K = max(3, args.steps // 5)
    W = max(3, args.warmup)  # untimed calls before each timed section
    # A: 32 views at 4K, forward only, 4 groups of 8 views through one plan
    cams4k = scenes.trajectory_cameras(32, resolutions=((3840, 2160),))
    groups = [cams4k[i:i + 8] for i in range(0, 32, 8)]
    ra = Rasterizer(g, groups[0], Config(forward_only=True), key_capacity=1 << 28)
    keys_a = []
    for grp in groups:  # size the key pool for every group
        ra.set_cameras(grp)
        ra.forward(g)
        keys_a.append(int(ra.keys))
    ra.autotune(g)

    def traj():
        for grp in groups:
            ra.set_cameras(grp)
            ra.forward(g)

    for _ in range(W):
        traj()
    ms_a = timed(traj, K, flush, stream)
    cap_a = ra.key_capacity
    del ra
    torch.cuda.empty_cache()
    # B: 8 views at 1080p, forward + backward
    cams = scenes.trajectory_cameras(8, resolutions=((1920, 1080),))
    ups = [torch.as_tensor(scenes.upstream_grad(60 + v, 1080, 1920), device=dev) for v in range(8)]
    flat = torch.cat([u.reshape(-1) for u in ups]).contiguous()
    rb = Rasterizer(g, cams, Config(), key_capacity=1 << 27)
    rb.forward(g)
    rb.autotune(g, flat)
    fb = lambda: (rb.forward(g), rb.backward(g, flat))
    for _ in range(W):
        fb()
    ms_batched = timed(fb, K, flush, stream)
    ws_batched = int(rb.plan.ws_bytes)
    keys_b = int(rb.keys)
    del rb
    torch.cuda.empty_cache()
    plans = {}
    for _ in range(W):
        render_views_recompute(g, cams, ups, Config(), plans)
    ms_recompute = timed(lambda: render_views_recompute(g, cams, ups, Config(), plans), K, flush, stream)
    ws_recompute = sum(int(r.plan.ws_bytes) for r in plans.values())
    value = 8 / (ms_batched / 1e3)
    out = {"metric": METRIC, "value": round(value, 3), "unit": "views/s", "n_gpus": world, "steps": K,
           "warmup": W, "ms_per_step": round(ms_batched, 3), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32 (SH stored bf16)", "data": "synthetic",
           "config": {"workload": "mixed_5m", "gaussians": 5_000_000, "zero_skew_fraction": 0.5,
                      "l2": "flushed (256 MiB memset) before each step"},
           "trajectory_4k": {"views": 32, "resolution": "3840x2160", "views_per_plan": 8,
                             "fwd_views_per_s": round(32 / (ms_a / 1e3), 2), "ms": round(ms_a, 2),
                             "keys_per_group": keys_a, "key_capacity": cap_a},
           "fwdbwd_8x1080p": {"batched_views_per_s": round(8 / (ms_batched / 1e3), 2),
                              "recompute_keys_views_per_s": round(8 / (ms_recompute / 1e3), 2),
                              "batched_ms": round(ms_batched, 2), "recompute_ms": round(ms_recompute, 2),
                              "workspace_bytes_batched": ws_batched, "workspace_bytes_recompute": ws_recompute,
                              "keys": keys_b}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_mixed_5m(cams4k[0], cams[0], ups[0].cpu().numpy(), args.oracle_threads)
    if rank == 0:
        print(json.dumps(out), flush=True)


def cpu_baseline_mixed_5m(cam4k, cam1080, up, threads=0):
    """The FP64 oracle on the 5M scene, one view of each part: the first 4K
    view of the trajectory, forward only (its rate stands for the 32-view
    trajectory's views/s), and the first 1080p view forward + backward (its
    rate stands for the 8-view step's views/s).  The oracle reads the FP32
    SH coefficients the BF16 copies were rounded from: the same arithmetic."""
    import oracle

    from paper_2605_18334_gb300 import scenes

    oracle.build()
    if threads:
        oracle.set_num_threads(threads)
    sc = scenes.mixed_5m()
    oc = oracle.camera_from_gl(cam4k)
    ocfg = oracle.config()
    t0 = time.perf_counter()
    pre = oracle.preprocess(sc, oc, ocfg)
    oracle.render_frame(sc, oc, ocfg, pre=pre)
    fwd4k = time.perf_counter() - t0
    del pre
    _, fb = oracle_frame(sc, cam1080, up)
    return {"value": round(1.0 / fb, 6), "unit": "views/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": (f"one 1920x1080 view of the 8-view step, forward + backward, and one 3840x2160 view of the "
                       f"32-view trajectory, forward only, of all {sc.n} Gaussians (FP64, per-pixel footprint lists); "
                       f"each view's rate stands for its part's views/s"),
            "fwdbwd_1080p_seconds": round(fb, 2), "fwd_4k_views_per_s": round(1.0 / fwd4k, 6),
            "fwd_4k_seconds": round(fwd4k, 2)}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "mixed_5m":
        run_mixed_5m(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
