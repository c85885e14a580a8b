"""Benchmark of the scale-aware Gaussian rasterizer (GSASR, arXiv 2501.06838).

A step is one pass of the whole hot path over one batch of synthetic input:
footprint pass, prefix sum, pair emission, radix sort, tile ranges, tile
raster (forward), and, for workloads with an adjoint, the raster adjoint and
the parameter chain rule. Default workload: LR 256x256, one Gaussian per LR
pixel (N = 65,536), x4 -> 1024x1024, forward + adjoint, FP32 parameters.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...     the FP64 CPU oracle on the same workload

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events on
the launching stream; L2 is flushed (256 MiB write) before every step, outside
the events. Under torchrun the job is split over the ranks (shard_workload):
images over ranks with no collective, or one image in row bands with an
all-reduce of the gradients; the time is the max over ranks and rank 0 prints
one JSON line.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import gs_synthetic as S  # noqa: E402

METRIC = "HR Mpix/s fwd and fwd+bwd at ×4/×12 vs FP64 oracle error; % FP32/SFU peak"
UNIT = "HR Mpix/s"

# ALU roofline of the raster kernels. Measured on
# GB300 with a probe: an SM issues 4 warp-instructions per clock; MUFU.EX2 runs
# at 32 lanes/clk/SM and holds its scheduler for 4 issue cycles per warp
# instruction; the FP32 pipe does 32 lane-operations per clock per scheduler,
# packed two-wide (FFMA2/FADD2/FMUL2) or not, so packing halves issue slots but
# not FP32 pipe time. Per (Gaussian, pixel) pair the method needs 1 exp2 and
#   forward: 5 FP32 ops (exponent 2, colour 3):
#            max(FP32 pipe 5, issue 4 + 5/2)  = 6.5 cycles per warp of pairs
#   adjoint: 12 FP32 ops (exponent 2, g.c 3, G w Y 2, Y moments 2, colour 3):
#            max(FP32 pipe 12, issue 4 + 12/2) = 12 cycles per warp of pairs
# so peak pairs/clk/SM = 4 * 32 / cycles.
SMS = 152
WARP_ISSUE_PER_SM_CLK = 4
PAIR_CYCLES = {"raster_fwd": 6.5, "raster_bwd": 12.0, "raster_bwd_gw": 12.0}

# DRAM bytes (read + write) of one launch of the dominant kernel, from one ncu
# capture per workload (summaries under profiles/), valid only for the kernel
# source they were taken on: reported as null once that source file changes.
TRAFFIC = {
    ("c2", "raster_bwd"): ("gs_adjoint_tile.cu",
                           "d329f4b6381f0a3278e01aa6c5f2dc462ed321c7207134b08b7a6235270e4c31",
                           21309184 + 0, "profiles/raster_bwd_c2_1024x1024.md"),
    ("c4x12-bf16", "raster_bwd"): ("gs_adjoint_tile.cu",
                                   "d329f4b6381f0a3278e01aa6c5f2dc462ed321c7207134b08b7a6235270e4c31",
                                   349436928 + 20665088,
                                   "profiles/raster_bwd_c4x12_bf16_5760x3240.md"),
    ("c4x12-bf16", "raster_fwd"): ("gs_raster.cu",
                                   "a1d3fc604d7d88dbb6ddcab89fd2d676a52d2fe9dd3e9fb2e164cfe5074db27f",
                                   37752320 + 233056512,
                                   "profiles/raster_fwd_c4x12_bf16_5760x3240.md"),
}


def measured_traffic(workload_name, kernel, args):
    import hashlib
    key = (workload_name, kernel)
    default_flags = args.norm is None and args.align is None and args.ratio is None and \
        not args.tile and not args.batch and getattr(args, "adjoint", None) is None and \
        getattr(args, "binning", None) is None and getattr(args, "raster", None) is None
    if key not in TRAFFIC or not default_flags:
        return None, None
    src_name, sha_ok, nbytes, where = TRAFFIC[key]
    src = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2501_06838_gb300",
                       "csrc", src_name)
    with open(src, "rb") as f:
        if hashlib.sha256(f.read()).hexdigest() != sha_ok:
            return None, None
    return nbytes, where


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# --------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------
WORKLOADS = {
    "c2": "LR 256x256, m=1 (N=65,536), x4 -> 1024x1024, forward + adjoint, FP32 params",
    "c1": "LR 48x48, m=1 (N=2,304), x4 -> 192x192, forward, FP32 params",
    "c4x8-bf16": "LR 480x270, m=4 (N=518,400), x8 -> 3840x2160, forward + adjoint, BF16 params",
    "c4x12-bf16": "LR 480x270, m=4 (N=518,400), x12 -> 5760x3240, forward + adjoint, BF16 params",
    "c4x12-f16": "LR 480x270, m=4 (N=518,400), x12 -> 5760x3240, forward + adjoint, FP16 params",
    "c4x12-f32": "LR 480x270, m=4 (N=518,400), x12 -> 5760x3240, forward + adjoint, FP32 params",
    "c3": "16 images, LR 64..480 x 64..360, m=1, s ~ U[1.5, 12], batched forward, FP32 params",
    "c3eq": "16 equal images (config 3's mean LR size and mean scale), batched forward, FP32",
    "c5": "training step: batch 16 of 48x48 LR crops, s ~ U[1, 4], 8-block 64-ch conv encoder + "
          "1x1 Gaussian head, BF16 params, batched render fwd+bwd, L1 loss, Adam",
    "rab4": "r-ablation shape: LR 180x180, m=16 (N=518,400), x4 -> 720x720, Algorithm 1 ratio "
            "window (--ratio, default 0.1), forward, FP32 params",
    "rab8": "r-ablation shape: LR 90x90, m=16 (N=129,600), x8 -> 720x720, Algorithm 1 ratio "
            "window (--ratio, default 0.1), forward, FP32 params",
}
# The whole GSASR inference pipeline with random weights (EDSR-baseline encoder,
# Gaussian decoder with k = 12, m = 16, d = 180, L = 6, five heads, render with
# r = 0.1) on the computational-cost table's shape: a 720x720 output from an LR
# image of 720 / s pixels a side.
PIPELINE_SCALES = {"gsasr-x2": 2, "gsasr-x3": 3, "gsasr-x4": 4, "gsasr-x6": 6, "gsasr-x8": 8,
                   "gsasr-x12": 12}
for _k, _s in PIPELINE_SCALES.items():
    WORKLOADS[_k] = (f"whole GSASR inference, random weights: LR {720 // _s}x{720 // _s} -> "
                     f"720x720 (x{_s}); EDSR-baseline encoder, Gaussian decoder (k=12, m=16, "
                     f"d=180, L=6), five heads, render with r=0.1; network BF16 in PyTorch, "
                     f"render in this library")
# The paper's whole-pipeline inference times (EDSR backbone, one A100, 720x720
# ground truth; computational-cost table), ms per image.
PAPER_PIPELINE_MS = {2: 1573.0, 3: 806.0, 4: 543.0, 6: 265.0, 8: 195.0, 12: 91.0}


def workload(name, args):
    """-> (list of GaussianSet, list of View, with_adjoint, dtype name)."""
    if name == "c2":
        g, v = S.config2()
        return g, v, True, "f32"
    if name == "c1":
        g, v = S.config1()
        return g, v, False, "f32"
    if name.startswith("c4x"):
        sc, dt = name[3:].split("-")
        g, v = S.config4(float(sc), dt)
        return g, v, True, dt
    if name == "c3":
        g, v = S.config3()
        return g, v, False, "f32"
    if name == "c3eq":
        g, v = S.config3_equal()
        return g, v, False, "f32"
    if name in ("rab4", "rab8"):
        g, v = S.ratio_ablation(float(name[3:]), args.ratio if args.ratio is not None else 0.1)
        return g, v, False, "f32"
    raise SystemExit(f"unknown workload {name}")


# The paper's own render-only timings (its CUDA rasterizer on one A100, FP32,
# supplementary "computational burden" table): 168 ms at x4 and 71 ms at x8 for
# a 720x720 output, i.e. HR Mpix/s on the r-ablation shape with r = 0.1.
PAPER_RENDER_MPIX_S = {"rab4": 720 * 720 / 0.168 / 1e6, "rab8": 720 * 720 / 0.071 / 1e6}


def paper_ratio(args, value):
    """value / the paper's number for exactly this workload, else None."""
    if args.workload not in PAPER_RENDER_MPIX_S:
        return None
    if args.norm is not None or args.align is not None or args.ratio not in (None, 0.1):
        return None
    return round(value / PAPER_RENDER_MPIX_S[args.workload], 3)


def binning_desc(code, gsets, views):
    grid_ok = all(g.ref_grid_m > 0 for g in gsets) and \
        all(v.out_w <= 32767 and v.out_h <= 32767 for v in views)
    grid = code == 2 or (code == 0 and grid_ok)
    return "grid-implicit" if grid else "sorted pairs"


def view_desc(v):
    win = (f"ratio r={v.trunc_k:g}" if v.window == S.WINDOW_RATIO else f"{v.trunc_k:g}-sigma box") \
        if v.trunc_k > 0 else "untruncated"
    return {"norm": "peak" if v.norm == S.NORM_PEAK else "density", "window": win,
            "align": "half-pixel" if v.align == S.ALIGN_HALF else "x/s (Eq. 4)"}


def apply_view_flags(views, args):
    """--norm / --align / --ratio overrides of every view of a workload."""
    out = []
    for v in views:
        d = dict(v.__dict__)
        if args.norm is not None:
            d["norm"] = {"density": S.NORM_DENSITY, "peak": S.NORM_PEAK}[args.norm]
        if args.align is not None:
            d["align"] = {"eq4": S.ALIGN_EQ4, "half": S.ALIGN_HALF}[args.align]
        if args.ratio is not None:
            d["window"], d["trunc_k"] = S.WINDOW_RATIO, args.ratio
        d.pop("adjoint", None)
        d.pop("binning", None)
        d.pop("raster", None)
        nv = S.View(**d)
        if getattr(args, "adjoint", None) is not None:
            nv.adjoint = {"auto": 0, "tile": 1, "gaussian": 2, "quadrant": 3}[args.adjoint]
        if getattr(args, "binning", None) is not None:
            nv.binning = {"auto": 0, "sort": 1, "grid": 2}[args.binning]
        if getattr(args, "raster", None) is not None:
            nv.raster = {"auto": 0, "tile": 1, "pair": 2}[args.raster]
        out.append(nv)
    return out


# --------------------------------------------------------------------------
# Clock sampling during the timed region
# --------------------------------------------------------------------------
# NVML clock sampler run as its own process (read-only queries), so that the
# benchmark's launch loop, which holds the Python interpreter lock, cannot
# delay the samples: one line "time sm_mhz max_mhz reason_bits" per sample.
_NVML_LOOP = r"""
import ctypes, sys, time
lib = ctypes.CDLL("libnvidia-ml.so.1")
if lib.nvmlInit_v2() != 0:
    sys.exit(1)
h = ctypes.c_void_p()
bus, idx, iv = sys.argv[1].encode(), int(sys.argv[2]), float(sys.argv[3])
if not bus or lib.nvmlDeviceGetHandleByPciBusId_v2(ctypes.c_char_p(bus), ctypes.byref(h)) != 0:
    if lib.nvmlDeviceGetHandleByIndex_v2(idx, ctypes.byref(h)) != 0:
        sys.exit(2)
clk, mx, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx))
get = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
    lib.nvmlDeviceGetCurrentClocksThrottleReasons
while True:
    if lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0 and get(h, ctypes.byref(rs)) == 0:
        sys.stdout.write(f"{time.time():.6f} {clk.value} {mx.value} {rs.value}\n")
        sys.stdout.flush()
    time.sleep(iv)
"""


class ClockSampler:
    """SM clock and clock-event reasons of one GPU, sampled every 2 ms by a
    separate process through NVML (read-only; nvidia-smi every 200 ms if that
    fails), timestamped, from before the timed region to the end of a
    clock-sampled repeat of it."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, interval_s: float = 0.002):
        self.gpu = gpu_index
        self.interval = interval_s
        self.samples = []   # (host time, sm_mhz, max_mhz, reason names)
        self.proc = None
        self.src = None
        self.t0 = self.t1 = None
        self._first = threading.Event()

    def _bus_id(self):
        try:
            import torch
            p = torch.cuda.get_device_properties(self.gpu)
            return f"{p.pci_domain_id:08x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
        except Exception:
            return ""

    def start(self):
        try:
            self.proc = subprocess.Popen(
                [sys.executable, "-c", _NVML_LOOP, self._bus_id(), str(self.gpu), str(self.interval)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.src = f"nvml every {self.interval * 1e3:g} ms"
            threading.Thread(target=self._read_nvml, daemon=True).start()
            if self._first.wait(10.0):
                return
            self.proc.kill()
        except Exception:
            pass
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.src = "nvidia-smi every 200 ms"
            threading.Thread(target=self._read_smi, daemon=True).start()
        except Exception:
            self.proc = None

    def _read_nvml(self):
        for line in self.proc.stdout:
            parts = line.split()
            if len(parts) == 4:
                bits = int(parts[3])
                self.samples.append((float(parts[0]), float(parts[1]), float(parts[2]),
                                     {n for b, n in self.REASONS.items() if bits & b}))
                self._first.set()

    def _read_smi(self):
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                try:
                    sm, mx = float(parts[1]), float(parts[2])
                except ValueError:
                    continue
                self.samples.append((time.time(), sm, mx, {n for n, v in zip(names, parts[5:9])
                                                           if "Active" in v and "Not" not in v}))

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock sampling unavailable"]}
        time.sleep(max(0.01, 2 * self.interval))
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        t0 = self.t0 if self.t0 is not None else float("-inf")
        t1 = self.t1 if self.t1 is not None else float("inf")
        load = [x for x in self.samples if x[0] >= t0]   # the timed region and the repeat after it
        timed = [x for x in load if x[0] <= t1]
        sm = [x[1] for x in load]
        reasons = set()
        for x in load:
            reasons |= x[3]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(x[2] for x in load) if load else None,
                "reasons": sorted(reasons), "samples": len(load),
                "samples_timed_region": len(timed),
                "sm_mhz_timed_region": statistics.median([x[1] for x in timed]) if timed else None,
                "source": self.src}


# --------------------------------------------------------------------------
# The GPU arm
# --------------------------------------------------------------------------
# Algorithmic DRAM bytes of the memory-bound passes (per launch): the footprint
# pass reads each Gaussian's parameters and writes its 64-byte record (and, with
# grid binning, its 8-byte compact window); the chain rule reads parameters and
# the 32 bytes of record-space moments and writes 36 bytes of gradients and
# the 32 bytes of cleared moments (the footprint pass clears them too); with
# sorted binning the emit pass writes 8 bytes
# per (tile, Gaussian) pair (reading 16 bytes of each record), a radix histogram
# pass reads the 4-byte keys, a scatter pass reads and writes keys and values
# (16 bytes per pair) and the ranges pass reads the keys.
def hbm_stage_rates(stage_raw, steps, stats, dtname, grid):
    n, pairs = stats["n_gaussians"], stats["tile_pairs"]
    pb = {"f32": 36, "bf16": 18, "f16": 18}[dtname]
    per_launch = {"preprocess": n * (pb + 64 + 32 + (8 if grid else 0)),
                  "preprocess_bwd": n * (pb + 32 + 36 + 32),
                  "emit": pairs * 8 + n * 16, "radix_hist": pairs * 4,
                  "radix_scatter": pairs * 16, "ranges": pairs * 4}
    peak = float(load_peaks()[0].get("hbm_gbs", 6800.0))
    out = {}
    for k, b in per_launch.items():
        if k not in stage_raw or b == 0:
            continue
        ms, cnt = stage_raw[k]
        if cnt == 0 or ms <= 0:
            continue
        gbs = b * cnt / (ms * 1e-3) / 1e9
        out[k] = {"bytes_per_launch": int(b), "launches_per_step": cnt // steps,
                  "ms_per_launch": round(ms / cnt, 5), "achieved_gbs": round(gbs, 1),
                  "frac_of_measured_hbm": round(gbs / peak, 4)}
    return out


# The parameter draws of each single-image workload, so that a rank can render
# another image of the same shape (seed = its index in the batch; index 0 is
# the workload's own image).
SIGMA_RANGE = {"c1": (0.3, 2.0), "c2": (0.3, 2.0), "rab4": (0.2, 3.0), "rab8": (0.2, 3.0)}


def batch_member(name, g, index):
    """Image `index` of a batch of images shaped like `g` (the workload's)."""
    if index == 0:
        return g
    rng = SIGMA_RANGE.get(name, (0.2, 3.0) if name.startswith("c4x") else (0.3, 2.0))
    return S.draw_gaussians(index, g.lr_h, g.lr_w, g.ref_grid_m, rng, dtype=g.dtype)


def shard_workload(args, gsets, views, rank, world):
    """The part of the job that rank `rank` of `world` renders, and how the
    job is split (host logic only; no GPU):
      images: a multi-image workload's images partitioned over the ranks,
              longest first (shard.shard_images), no collective: a fixed batch
              (strong scaling); a single-image workload becomes a batch of
              `world` images of its shape, one per rank (weak scaling);
      bands:  the rows of a single image split into one band per rank
              (shard.band_rows / band_view); the forward needs no exchange and
              the adjoint's per-band gradients are summed over the ranks with
              one all-reduce of N x 9 floats (strong scaling).
    Returns (gsets, views, info)."""
    from paper_2501_06838_gb300 import shard
    job_pix = sum(v.out_h * v.out_w for v in views)
    if world == 1:
        return gsets, views, {"mode": "none", "scaling": "weak", "job_hr_pixels": job_pix,
                              "parallelism": "one GPU"}
    mode = args.shard
    if mode == "bands":
        if len(views) != 1:
            raise SystemExit("--shard bands splits one image: use it with a single-image workload")
        tile = args.tile or 16
        r0, rows = shard.band_rows(views[0].out_h, world, tile)[rank]
        if rows < 1:
            raise SystemExit(f"{views[0].out_h} rows give rank {rank} an empty band")
        return gsets, [shard.band_view(views[0], r0, rows)], {
            "mode": "bands", "scaling": "strong", "job_hr_pixels": job_pix, "band": [r0, rows],
            "parallelism": f"row bands of one image over {world} ranks (rows {r0}..{r0 + rows - 1} "
                           f"on rank {rank}), all-reduce of the N x 9 gradients"}
    if len(views) > 1:
        parts = shard.shard_images(shard.image_costs(views), world)
        mine = parts[rank]
        return [gsets[i] for i in mine], [views[i] for i in mine], {
            "mode": "images", "scaling": "strong", "job_hr_pixels": job_pix, "rank_images": mine,
            "parallelism": f"{len(views)} images partitioned over {world} ranks (longest first, "
                           f"images {mine} on rank {rank}), no collective"}
    return [batch_member(args.workload, gsets[0], rank)], views, {
        "mode": "images", "scaling": "weak", "job_hr_pixels": world * job_pix,
        "parallelism": f"a batch of {world} images of this shape, one per rank, no collective"}


def run_gpu(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    import paper_2501_06838_gb300 as gs
    from paper_2501_06838_gb300 import shard

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    gsets, views, with_adj, dtname = workload(args.workload, args)
    views = apply_view_flags(views, args)
    gsets, views, shard_info = shard_workload(args, gsets, views, rank, world)
    band_allreduce = shard_info["mode"] == "bands" and with_adj
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[dtname]

    def dev_g(g):
        arrs = g.storage()
        ts = []
        for a in arrs:
            t = torch.from_numpy(np.ascontiguousarray(a).view(np.int16)).view(torch.bfloat16) \
                if dtname == "bf16" else torch.from_numpy(np.ascontiguousarray(a))
            ts.append(t.to(dev).contiguous())
        return gs.Gaussians(*ts, ref_grid_m=g.ref_grid_m)

    dgs = [dev_g(g) for g in gsets]
    tuned = None
    if args.tune or (args.tune is None and args.workload in ("c3",) and not args.tile):
        # the launch parameters the library's autotuner picks for this workload
        import importlib
        T = importlib.import_module("paper_2501_06838_gb300.tune")
        tuned = T.tune(dgs, views, with_grads=with_adj, reps=3)
        args.tile, args.batch = tuned["tile"], tuned["batch"]
        for v in views:
            v.binning, v.raster, v.adjoint = tuned["binning_code"], tuned["raster"], tuned["adjoint"]
    plan = gs.Plan(dgs, views, tile=args.tile, batch=args.batch, with_grads=with_adj)
    if with_adj:
        for i, v in enumerate(views):
            plan.grad_outs[i].copy_(torch.from_numpy(S.grad_out(1, v.out_h, v.out_w)))
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    hr_pix = sum(v.out_h * v.out_w for v in views)

    def step():
        plan.fwd(stream)
        if with_adj:
            plan.bwd(stream)
            if band_allreduce:
                shard.allreduce_band_grads(plan.grads[0])

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    plan.status()
    stats = plan.stats()
    gs.timing_read()

    # ---- timed region (device-resident inputs) ----
    # Events inside a step cost the GPU about 2 us each, so the timed region
    # brackets each step and the dominant kernel only; the forward-only rate
    # and the stage breakdown come from the passes after it.
    timed_kernels = ["raster_bwd", "raster_bwd_gw"] if with_adj else ["raster_fwd"]
    clocks = ClockSampler(local_rank)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.mark_start()
    launches0 = gs.launch_count()
    # the dominant kernel is bracketed on every `kernel_every`-th timed step
    # (by default every step; sparser: never the first, which follows the host
    # synchronisation, and always the last). Events between the chained kernels
    # stop the next launch from overlapping the previous one's drain.
    every = max(1, args.kernel_every)
    use_graph = args.graph if args.graph is not None else args.workload in ("c3", "c3eq")
    if use_graph:
        # the whole step as one CUDA graph (captured once, replayed per step);
        # the dominant kernel's events are the graph's event-record nodes, read
        # after each replay
        cap = torch.cuda.Stream()
        cap.wait_stream(stream)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        l0 = gs.launch_count()
        gs.timing_enable(timed_kernels)
        with torch.cuda.graph(graph, stream=cap):
            plan.fwd(torch.cuda.current_stream())
            if with_adj:
                plan.bwd(torch.cuda.current_stream())
        gs.timing_enable([])
        launches_per_step = gs.launch_count() - l0
        for _ in range(2):
            flush.zero_()
            graph.replay()
        torch.cuda.synchronize()
        gs.timing_read()
        ktimes = {}
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            graph.replay()
            ev[k][1].record(stream)
            ev[k][1].synchronize()
            for kk, (ms, cnt) in gs.timing_read().items():
                a0, c0 = ktimes.get(kk, (0.0, 0))
                ktimes[kk] = (a0 + ms, c0 + cnt)
        torch.cuda.synchronize()
        gs.timing_release()
        del graph
        launches = launches_per_step * args.steps
    else:
        for k in range(args.steps):
            flush.zero_()
            gs.timing_enable(timed_kernels if k % every == every - 1 or k == args.steps - 1 else [])
            ev[k][0].record(stream)
            plan.fwd(stream)
            if with_adj:
                plan.bwd(stream)
                if band_allreduce:
                    shard.allreduce_band_grads(plan.grads[0])
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        launches = gs.launch_count() - launches0
        gs.timing_enable([])
        ktimes = gs.timing_read()
    clocks.mark_end()
    timed_ktimes = dict(ktimes)
    if world > 1:
        dist.barrier()
    # a clock-sampled repeat of the same steps right after the timed region,
    # so that a short timed region still gets enough clock samples under load
    n_timed_samples = len(clocks.samples)
    t_rep = time.time()
    while len(clocks.samples) < n_timed_samples + 25 and time.time() - t_rep < 2.0:
        for _ in range(args.steps):
            flush.zero_()
            step()
        torch.cuda.synchronize()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)

    # ---- forward-only rate (same steps, forward bracketed) ----
    fwd_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
    gs.timing_enable(["raster_fwd"])
    for k in range(args.steps):
        flush.zero_()
        fwd_ev[k][0].record(stream)
        plan.fwd(stream)
        fwd_ev[k][1].record(stream)
        if with_adj:
            plan.bwd(stream)
    torch.cuda.synchronize()
    gs.timing_enable([])
    for k2, v2 in gs.timing_read().items():
        ktimes.setdefault(k2, v2)
    fwd_ms = [a.elapsed_time(b) for a, b in fwd_ev]
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    plan.status()

    # ---- per-stage breakdown (after the timed region, every kernel timed) ----
    gs.timing_enable(None)
    for _ in range(3):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    gs.timing_enable([])
    stage_raw = gs.timing_read()
    stage = {k: round(v[0] / 3, 5) for k, v in stage_raw.items()}
    hbm_stages = hbm_stage_rates(stage_raw, 3, stats, dtname,
                                 binning_desc(plan.V[0].binning, gsets, views) == "grid-implicit")

    # ---- measured unit throughputs (the ALU roofline's inputs) ----
    unit_rates = None
    if rank == 0 and not args.no_probe:
        pk = gs.render.probe_peaks() if hasattr(gs, "render") and hasattr(gs.render, "probe_peaks") \
            else None
        if pk is None:
            import importlib
            pk = importlib.import_module("paper_2501_06838_gb300.render").probe_peaks()
        f_max = float(load_peaks()[0].get("sm_max_mhz", 2070.0)) * 1e6
        per = lambda v: round(v / pk["sm_count"] / f_max, 2)
        unit_rates = {"ffma_per_sm_clk": per(pk["ffma_per_s"]),
                      "ffma2_lane_ops_per_sm_clk": per(pk["ffma2_lane_ops_per_s"]),
                      "ex2_per_sm_clk": per(pk["ex2_per_s"]),
                      "fwd_pairs_scalar_per_sm_clk": per(pk["fwd_pairs_scalar_per_s"]),
                      "fwd_pairs_packed_per_sm_clk": per(pk["fwd_pairs_packed_per_s"]),
                      "clock_basis_mhz": f_max / 1e6}

    # ---- roofline of the dominant kernel ----
    peaks, peak_src = load_peaks()
    f_clk = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    dom = max(timed_ktimes.items(), key=lambda kv: kv[1][0])[0] if timed_ktimes else None
    roof = None
    if dom:
        ms, cnt = ktimes[dom]
        per_launch_s = ms / cnt * 1e-3
        pairs = stats["pixel_pairs"]
        achieved = pairs / per_launch_s / 1e9
        peak = SMS * f_clk * WARP_ISSUE_PER_SM_CLK * 32 / PAIR_CYCLES[dom] / 1e9
        traffic, traffic_src = measured_traffic(args.workload, dom, args)
        roof = {"bound": "alu", "kernel": dom, "achieved": round(achieved, 2),
                "peak": round(peak, 2), "unit": "Gpair/s", "frac": round(achieved / peak, 4),
                "traffic": traffic, "traffic_unit": "bytes per launch (ncu dram read + write)",
                "traffic_source": traffic_src,
                "peak_basis": (f"{SMS} SMs x {WARP_ISSUE_PER_SM_CLK} warp-issue/clk x 32 x "
                               f"{f_clk / 1e6:.0f} MHz / {PAIR_CYCLES[dom]} cycles per warp of pairs "
                               f"({peak_src} sm_max_mhz)"),
                "pairs_per_launch": pairs, "ms_per_launch": round(ms / cnt, 5)}

    res = {
        "metric": METRIC,
        "value": round(shard_info["job_hr_pixels"] * args.steps / (total_ms * 1e-3) / 1e6, 2),
        "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(total_ms / args.steps, 5), "higher_is_better": True,
        "scaling": shard_info["scaling"], "vs_baseline": None, "dtype": dtname,
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}",
                   "view": view_desc(views[0]),
                   "l2": "flushed before every step (256 MiB write, outside the timed events)",
                   "tile": plan.V[0].tile or 16,
                   "smem_batch": plan.V[0].batch or (64 if plan.V[0].tile == 32 else 32),
                   "binning": binning_desc(plan.V[0].binning, gsets, views),
                   "autotuned": None if tuned is None else {k: tuned[k] for k in
                                                           ("tile", "batch", "binning", "raster",
                                                            "adjoint", "ms",
                                                            "from_cache", "n_timed")},
                   "adjoint": {2: "gaussian-warp", 3: "tile quadrants"}.get(stats.get("adjoint"), "tile")
                   if with_adj else None,
                   "raster": "pair of tiles" if stats.get("raster") == 2 else "tile",
                   "cuda_graph": bool(use_graph),
                   "hr_pixels_per_step": shard_info["job_hr_pixels"],
                   "gaussians": sum(g.n for g in dgs),
                   "parallelism": shard_info["parallelism"]},
        "fwd_mpix_s": round(hr_pix * args.steps / (sum(fwd_ms) * 1e-3) / 1e6, 2),
        "kernel_ms": {k: round(v[0] / v[1], 5) for k, v in ktimes.items()},
        "kernel_ms_note": (f"the dominant kernel timed by CUDA events inside the timed region"
                           f"{'' if every == 1 else f', on every {every}th step'}; raster_fwd (with "
                           f"an adjoint) in a second pass of the same steps"),
        "stage_ms_per_step": stage,
        "pairs": {"pixel_pairs": stats["pixel_pairs"], "tile_pairs": stats["tile_pairs"]},
        "hbm_stages": hbm_stages,
        "roofline": roof, "gpu_launches": int(launches), "clocks": clk,
        "unit_rates": unit_rates,
    }

    vb = paper_ratio(args, res["value"])
    if vb is not None:
        res["vs_baseline"] = vb
        res["baseline_note"] = (f"paper's render-only time on one A100, FP32 (computational-burden "
                                f"table): {PAPER_RENDER_MPIX_S[args.workload]:.2f} HR Mpix/s")

    # ---- end to end through the public API with host buffers ----
    if not args.no_e2e:
        e2e = run_e2e(args, plan, gsets, views, with_adj, dtname, dev, stream, flush)
        tot = e2e.pop("total_ms")
        if world > 1:
            t = torch.tensor([tot], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            tot = float(t.item())
        e2e["value"] = round(shard_info["job_hr_pixels"] * args.steps / (tot * 1e-3) / 1e6, 2)
        e2e["ms_per_step"] = round(tot / args.steps, 5)
        pt = e2e.pop("pipelined_total_ms")
        if world > 1:
            t = torch.tensor([pt], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            pt = float(t.item())
        e2e["pipelined"] = {"value": round(shard_info["job_hr_pixels"] * args.steps /
                                          (pt * 1e-3) / 1e6, 2),
                            "ms_per_step": round(pt / args.steps, 5),
                            "l2": "not flushed between the overlapping steps; every step copies "
                                  "all its inputs in and all its results out"}
        res["e2e"] = e2e

    # ---- CPU baseline: the FP64 oracle on the host cores, bounded sample ----
    if rank == 0 and world == 1 and not args.no_cpu:
        cb, err = run_cpu_baseline(gsets, views, with_adj, plan, args.cpu_seconds)
        res["cpu_baseline"] = cb
        if err:
            res["error_vs_oracle"] = err
    return res


def run_x12(args, rank, world, local_rank):
    """The x12 half of the metric beside the default x4 line: config 4 at x12
    (LR 480x270, m = 4, N = 518,400 -> 5760x3240, BF16 parameters), forward +
    adjoint, with the same steps and warm-up, its own clock record and
    roofline."""
    a = argparse.Namespace(**vars(args))
    a.workload, a.no_e2e, a.no_cpu, a.no_probe, a.tune, a.graph = \
        "c4x12-bf16", True, True, True, False, None
    r = run_gpu(a, rank, world, local_rank)
    keep = ("value", "unit", "ms_per_step", "steps", "warmup", "dtype", "fwd_mpix_s", "kernel_ms",
            "stage_ms_per_step", "pairs", "roofline", "clocks", "gpu_launches")
    out = {"workload": r["config"]["workload"]}
    out.update({k: r[k] for k in keep if k in r})
    return out


def run_train(args, rank, world, local_rank):
    """Config 5: end-to-end training steps (encoder + head + render + loss +
    backward + Adam); reports rendered HR Mpix/s, step time and the share of
    the step spent in the library's kernels."""
    import torch
    import torch.distributed as dist

    import paper_2501_06838_gb300 as gs
    from paper_2501_06838_gb300.train_step import TrainStep
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    step = TrainStep(device=dev)
    lr, hrs, scales = S.config5_batch(rank)
    lr_t = torch.from_numpy(lr).to(dev)
    hr_t = [torch.from_numpy(h).to(dev) for h in hrs]
    hr_pix = sum(h.shape[1] * h.shape[2] for h in hrs)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        step(lr_t, hr_t, scales)
    torch.cuda.synchronize()
    gs.timing_read()
    clocks = ClockSampler(local_rank)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = gs.launch_count()
    gs.timing_enable(None)
    tot = 0.0
    loss = None
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        loss = step(lr_t, hr_t, scales)
        b.record()
        b.synchronize()
        tot += a.elapsed_time(b)
    gs.timing_enable([])
    kt = gs.timing_read()
    launches = gs.launch_count() - launches0
    clk = clocks.stop()
    if world > 1:
        t = torch.tensor([tot], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot = float(t.item())
    render_ms = sum(v[0] for v in kt.values())
    return {"metric": METRIC, "value": round(world * hr_pix * args.steps / (tot * 1e-3) / 1e6, 2),
            "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(tot / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": f"c5: {WORKLOADS['c5']}", "hr_pixels_per_step": hr_pix,
                       "scales": [round(s, 3) for s in scales],
                       "l2": "flushed before every step (256 MiB write, outside the timed events)"},
            "render_share": round(render_ms / tot, 4),
            "render_ms_per_step": round(render_ms / args.steps, 4),
            "kernel_ms_per_step": {k: round(v[0] / args.steps, 5) for k, v in kt.items()},
            "final_loss": float(loss), "gpu_launches": int(launches), "clocks": clk}


def pipeline_flops(cfg, h, w):
    """Multiply-adds x 2 of one GSASR inference at LR h x w (the model's own
    arithmetic: head width d / heads, no padding)."""
    k, m, d, heads, c = cfg.k, cfg.m, cfg.d, cfg.heads, cfg.n_feats
    hp, wp = -(-h // k) * k, -(-w // k) * k
    ntok, nwin, t = m * hp * wp, (hp // k) * (wp // k), m * k * k
    hid = cfg.mlp_ratio * d
    conv = 2 * h * w * 9 * (3 * c + (2 * cfg.n_resblocks + 1) * c * c)
    mlp = 2 * ntok * 2 * d * hid
    inject = (2 * hp * wp * c * 2 * d + 4 * nwin * t * k * k * d + 2 * ntok * d * d + mlp)
    wsa = 2 * ntok * 4 * d * d + 4 * nwin * t * t * d + mlp
    sca = 2 * ntok * 2 * d * d + 4 * ntok * cfg.scale_tokens * d + mlp
    head = 2 * ntok * (5 * 2 * d * d + 9 * d)
    return {"encoder": conv, "decoder": inject + cfg.blocks * (2 * wsa + sca) + head}


def run_pipeline(args, rank, world, local_rank):
    """The whole GSASR inference (encoder, Gaussian decoder, heads, render) on
    the computational-cost table's shape, timed per stage with CUDA events."""
    import torch

    import paper_2501_06838_gb300 as gs
    from paper_2501_06838_gb300.gsasr import GSASR, GSASRConfig
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    scale = PIPELINE_SCALES[args.workload]
    lr_img = S.pipeline_input(scale)
    h, w = lr_img.shape[1:]
    torch.backends.cudnn.benchmark = True    # fixed shapes: let cuDNN pick its conv kernels
    torch.manual_seed(0)
    cfg = GSASRConfig(pad_width=getattr(args, "pipeline_width", "padded") == "padded")
    net = GSASR(cfg).to(dev, dtype=torch.bfloat16).eval()   # BF16 weights and activations
    lr_t = torch.from_numpy(lr_img)[None].to(dev)
    scales = torch.full((1,), float(scale), device=dev)
    hr_pix = S.out_size(h, scale) * S.out_size(w, scale)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def run(evs=None):
        with torch.no_grad():
            if evs:
                evs[0].record()
            f = net.encode(lr_t)
            if evs:
                evs[1].record()
            raw = net.decode(f, scales, h, w)
            if evs:
                evs[2].record()
        out = net.render(raw, h, w, scale)
        if evs:
            evs[3].record()
        return out

    for _ in range(args.warmup):
        flush.zero_()
        run()
    torch.cuda.synchronize()
    gs.timing_read()
    clocks = ClockSampler(local_rank)
    clocks.start()
    torch.cuda.synchronize()
    launches0 = gs.launch_count()
    gs.timing_enable(["raster_fwd"])
    stages = np.zeros(3)
    tot = 0.0
    for _ in range(args.steps):
        flush.zero_()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        out = run(evs)
        evs[3].synchronize()
        st = [evs[i].elapsed_time(evs[i + 1]) for i in range(3)]
        stages += st
        tot += sum(st)
    gs.timing_enable([])
    kt = gs.timing_read()
    launches = gs.launch_count() - launches0
    clk = clocks.stop()
    assert out[0].shape == (3, S.out_size(h, scale), S.out_size(w, scale))
    assert bool(torch.isfinite(out[0]).all())
    ms = tot / args.steps
    fl = pipeline_flops(net.cfg, h, w)
    peaks, peak_src = load_peaks()
    bf16_peak = float(peaks.get("bf16_tflops_sustained", 1700.0))   # a long step: sustained
    net_ms = (stages[0] + stages[1]) / args.steps
    achieved = (fl["encoder"] + fl["decoder"]) / (net_ms * 1e-3) / 1e12
    value = hr_pix / (ms * 1e-3) / 1e6
    paper_value = hr_pix / (PAPER_PIPELINE_MS[scale] * 1e-3) / 1e6
    raster = kt.get("raster_fwd", (0.0, 1))
    return {"metric": "HR Mpix/s, whole GSASR inference (encoder + Gaussian decoder + render)",
            "value": round(value, 3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": round(value / paper_value, 2),
            "baseline_note": (f"the paper's whole-pipeline time on one A100 (EDSR backbone, "
                              f"computational-cost table): {PAPER_PIPELINE_MS[scale]:.0f} ms per "
                              f"720x720 image"),
            "dtype": "bf16 network, render from bf16 raw outputs in f32", "data": "synthetic (random weights)",
            "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}",
                       "lr": [h, w], "gaussians": net.cfg.m * h * w, "hr_pixels_per_step": hr_pix,
                       "d": net.cfg.d, "d_stored": net.cfg.d_store,
                       "l2": "flushed before every step; the decoder's activations are GBs"},
            "stage_ms": {"encoder": round(stages[0] / args.steps, 3),
                         "decoder": round(stages[1] / args.steps, 3),
                         "head_and_render": round(stages[2] / args.steps, 3)},
            "render_share": round(stages[2] / tot, 4),
            "raster_fwd_ms": round(raster[0] / max(raster[1], 1), 4),
            "roofline": {"bound": "tensor", "kernel": "encoder + decoder (PyTorch: cuBLAS GEMMs, "
                                                      "fused attention)",
                         "achieved": round(achieved, 1), "peak": bf16_peak, "unit": "TFLOP/s",
                         "frac": round(achieved / bf16_peak, 4), "traffic": None,
                         "flops_per_step": fl, "peak_source": f"{peak_src} bf16_tflops_sustained"},
            "gpu_launches": int(launches), "clocks": clk,
            "cpu_baseline": None,
            "cpu_baseline_note": "the oracle covers the render only, not the network"}


def _packed(specs, device):
    """One pinned host buffer and one device buffer holding tensors of the given
    (shape, dtype), each slice 256-byte aligned: a step's inputs (or results)
    move in one copy."""
    import torch
    offs, o = [], 0
    for shape, dt in specs:
        nb = math.prod(shape) * torch.empty((), dtype=dt).element_size()
        offs.append((o, nb))
        o = (o + nb + 255) // 256 * 256
    host = torch.empty(max(o, 256), dtype=torch.uint8, pin_memory=True)
    devb = torch.empty(max(o, 256), dtype=torch.uint8, device=device)
    hv = [host[a:a + nb].view(dt).view(shape) for (a, nb), (shape, dt) in zip(offs, specs)]
    dv = [devb[a:a + nb].view(dt).view(shape) for (a, nb), (shape, dt) in zip(offs, specs)]
    return host, devb, hv, dv


def _e2e_set(plan, with_adj, dev):
    """A packed input/output buffer set and a Plan rendering from / into it."""
    import torch
    import importlib
    R = importlib.import_module("paper_2501_06838_gb300.render")
    in_specs = [(tuple(t.shape), t.dtype) for dg in plan.gs for t in dg.tensors()]
    if with_adj:
        in_specs += [(tuple(go.shape), go.dtype) for go in plan.grad_outs]
    hin, din, hiv, div = _packed(in_specs, dev)
    src = [t for dg in plan.gs for t in dg.tensors()] + (list(plan.grad_outs) if with_adj else [])
    for h, t in zip(hiv, src):
        h.copy_(t.cpu())
    din.copy_(hin)   # the Plan sizes its workspace from the device parameters
    out_specs = [(tuple(o.shape), o.dtype) for o in plan.outs]
    if with_adj:
        out_specs += [(tuple(g.shape), g.dtype) for g in plan.grads]
    hout, dout, hov, dov = _packed(out_specs, dev)
    gsd, k = [], 0
    for dg in plan.gs:
        gsd.append(R.Gaussians(*div[k:k + 5], ref_grid_m=dg.ref_grid_m, head=dg.head))
        k += 5
    nimg = len(plan.outs)
    p = R.Plan(gsd, plan.views, tile=plan.V[0].tile, batch=plan.V[0].batch, with_grads=with_adj,
               outs=dov[:nimg], grad_outs=div[k:] if with_adj else None,
               grads=dov[nimg:] if with_adj else None)
    return {"hin": hin, "din": din, "hout": hout, "dout": dout, "plan": p}


def run_e2e(args, plan, gsets, views, with_adj, dtname, dev, stream, flush):
    """Same metric through the public API with HOST buffers: every step copies
    its inputs (parameters and upstream gradient, one packed pinned buffer) to
    the device, renders (and runs the adjoint), and copies the image and the
    gradients back (one packed buffer); copies inside the timed region.
    value: serial steps (copy in, compute, copy out), L2 flushed before each.
    pipelined: a stream of steps over two buffer sets, the copies of one step
    overlapping the compute of its neighbours (copy-in, compute and copy-out
    streams ordered by events; every step still moves all its bytes)."""
    import torch
    sets = [_e2e_set(plan, with_adj, dev) for _ in range(2)]
    h2d = sets[0]["hin"].numel()
    d2h = sets[0]["hout"].numel()

    def serial(S):
        S["din"].copy_(S["hin"], non_blocking=True)
        S["plan"].fwd(stream)
        if with_adj:
            S["plan"].bwd(stream)
        S["hout"].copy_(S["dout"], non_blocking=True)

    with torch.cuda.stream(stream):
        for _ in range(max(1, args.warmup)):
            flush.zero_()
            serial(sets[0])
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            serial(sets[0])
            b.record(stream)
            b.synchronize()
            tot += a.elapsed_time(b)

    s_in, s_cmp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ev = {(k, i): torch.cuda.Event() for k in ("in", "cmp", "out") for i in (0, 1)}

    def pipelined(steps):
        for k in range(steps):
            i = k & 1
            S = sets[i]
            if k >= 2:
                s_in.wait_event(ev[("cmp", i)])      # inputs of step k - 2 consumed
            with torch.cuda.stream(s_in):
                S["din"].copy_(S["hin"], non_blocking=True)
            ev[("in", i)].record(s_in)
            s_cmp.wait_event(ev[("in", i)])
            if k >= 2:
                s_cmp.wait_event(ev[("out", i)])     # results of step k - 2 copied out
            S["plan"].fwd(s_cmp)
            if with_adj:
                S["plan"].bwd(s_cmp)
            ev[("cmp", i)].record(s_cmp)
            s_out.wait_event(ev[("cmp", i)])
            with torch.cuda.stream(s_out):
                S["hout"].copy_(S["dout"], non_blocking=True)
            ev[("out", i)].record(s_out)

    pipelined(max(3, args.warmup))
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s_in)
    pipelined(args.steps)
    s_in.wait_stream(s_out)
    b.record(s_in)
    b.synchronize()
    piped = a.elapsed_time(b)
    for S in sets:
        S["plan"].status()
    return {"unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "total_ms": tot, "pipelined_total_ms": piped,
            "copies_per_step": {"h2d": 1, "d2h": 1}}


def oracle_step(gsets, views, with_adj, band=None, threads=0, grad_outs=None):
    """One oracle step: render (and adjoint) of every image, or of the top
    `band` rows of every image. Returns (images, grads, HR pixels done)."""
    import oracle
    outs, grads, px = [], [], 0
    for i, (g, v) in enumerate(zip(gsets, views)):
        vv = v if band is None else dataclasses.replace(v, out_h=min(band, v.out_h))
        outs.append(oracle.render(g, vv, threads=threads))
        if with_adj:
            go = grad_outs[i] if grad_outs is not None else S.grad_out(1, v.out_h, v.out_w)
            grads.append(oracle.adjoint(g, vv, go[:, :vv.out_h], threads=threads))
        px += vv.out_h * vv.out_w
    return outs, grads, px


def sample_band(gsets, views, with_adj, seconds):
    """None if one oracle step of the whole workload fits in `seconds`, else
    the number of top rows per image that does (probed on 32 rows)."""
    probe = min(32, max(v.out_h for v in views))
    t0 = time.time()
    oracle_step(gsets, views, with_adj, band=probe)
    t = time.time() - t0
    full = t * max(v.out_h for v in views) / probe
    if full <= seconds:
        return None
    return max(16, int(probe * seconds / max(t, 1e-9)))


def run_cpu_baseline(gsets, views, with_adj, plan, seconds):
    """Times the FP64 oracle (fwd + adjoint when the workload has one) on all
    host cores, on a bounded sample: whole images when a step fits in a few
    seconds, else the top rows of each image. Also returns this run's GPU error
    against it (normwise per channel / per field)."""
    import oracle
    oracle.build()
    cores = oracle.hardware_threads()
    use_band = sample_band(gsets, views, with_adj, seconds / 2)
    reps, px, t = 0, 0, 0.0
    outs = grads = None
    while t < seconds or reps == 0:
        t1 = time.time()
        outs, grads, npx = oracle_step(gsets, views, with_adj, band=use_band)
        t += time.time() - t1
        px += npx
        reps += 1
    sample = (f"{reps} oracle step(s) of the full workload" if use_band is None else
              f"{reps} oracle step(s) on the top {use_band} rows of every image")
    cb = {"value": round(px / t / 1e6, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
          "sample": sample + (" (fwd + adjoint)" if with_adj else " (fwd)"),
          "seconds": round(t, 2)}
    # the same oracle on one core, on a sample of about a tenth of that time
    band1 = sample_band(gsets, views, with_adj, seconds / 10 / max(cores, 1))
    t1 = time.time()
    _, _, px1 = oracle_step(gsets, views, with_adj, band=band1, threads=1)
    t1 = time.time() - t1
    cb["single_core"] = {"value": round(px1 / t1 / 1e6, 4), "cores": 1,
                         "sample": ("one oracle step of the full workload" if band1 is None else
                                    f"one oracle step on the top {band1} rows of every image"),
                         "seconds": round(t1, 2)}
    # error of this run's GPU result against the oracle (on the same sample)
    err = {}
    try:
        img_err = []
        for o, ref in zip(plan.outs, outs):
            a = o[:, :ref.shape[1]].cpu().double().numpy()
            img_err.append(float((np.abs(a - ref).max(axis=(1, 2)) / np.abs(ref).max(axis=(1, 2))).max()))
        err["image_normwise"] = max(img_err)
        if with_adj and use_band is None:
            ge = []
            for gr, ref in zip(plan.grads, grads):
                a = gr.cpu().double().numpy()
                ge.append(float((np.abs(a - ref).max(axis=0) / np.abs(ref).max(axis=0)).max()))
            err["grad_normwise"] = max(ge)
    except Exception as e:  # keep the bench line even if the comparison fails
        err["error"] = repr(e)
    return cb, err


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle itself, timed per step on the host."""
    if rank != 0:
        return None
    import oracle
    oracle.build()
    gsets, views, with_adj, dtname = workload(args.workload, args)
    views = apply_view_flags(views, args)
    band = sample_band(gsets, views, with_adj, max(1.0, args.ref_step_seconds))
    for _ in range(args.warmup):
        oracle_step(gsets, views, with_adj, band=band)
    tot, px = 0.0, 0
    for _ in range(args.steps):
        t1 = time.time()
        _, _, npx = oracle_step(gsets, views, with_adj, band=band)
        tot += time.time() - t1
        px += npx
    val = round(px / tot / 1e6, 4)
    sample = ("the full workload per step" if band is None else
              f"the top {band} rows of every image per step")
    cores = oracle.hardware_threads()
    return {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(tot / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}",
                       "view": view_desc(views[0])},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample + (" (fwd + adjoint)" if with_adj else " (fwd)")},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=sorted(WORKLOADS))
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--batch", type=int, default=0)
    ap.add_argument("--norm", choices=["density", "peak"], default=None,
                    help="normalisation of Eq. 2 (default: the workload's, density)")
    ap.add_argument("--align", choices=["eq4", "half"], default=None,
                    help="pixel sampling: x/s (Eq. 4) or (x + 1/2)/s - 1/2")
    ap.add_argument("--ratio", type=float, default=None,
                    help="use Algorithm 1's ratio window with this r instead of the 3-sigma box")
    ap.add_argument("--adjoint", choices=["auto", "tile", "gaussian", "quadrant"], default=None,
                    help="adjoint kernel: per-tile with atomics, per 8 x 8 quadrant of 16 x 16 "
                         "tiles with atomics, or one warp per Gaussian")
    ap.add_argument("--binning", choices=["auto", "sort", "grid"], default=None,
                    help="per-tile Gaussian lists: radix-sorted pairs or grid-implicit")
    ap.add_argument("--raster", choices=["auto", "tile", "pair"], default=None,
                    help="forward raster layout: one warp per tile or per pair of tiles")
    ap.add_argument("--tune", dest="tune", action="store_true", default=None,
                    help="pick tile / batch / binning with the library's autotuner "
                         "(default for the c3 workload)")
    ap.add_argument("--no-tune", dest="tune", action="store_false")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-probe", action="store_true", help="skip the unit-throughput probe")
    ap.add_argument("--shard", choices=["auto", "images", "bands"], default="auto",
                    help="with several GPUs: partition images over the ranks (a single image "
                         "becomes a batch of one image per rank), or split one image into row "
                         "bands with an all-reduce of the gradients")
    ap.add_argument("--no-x12", action="store_true",
                    help="c2 only: skip the x12 measurement (config 4, BF16) added to the line")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--graph", dest="graph", action="store_true", default=None,
                    help="time each step as one CUDA-graph replay (default for c3 / c3eq)")
    ap.add_argument("--no-graph", dest="graph", action="store_false")
    ap.add_argument("--kernel-every", type=int, default=1,
                    help="bracket the dominant kernel with CUDA events on every k-th timed step "
                         "(1: every step; sparser brackets leave more steps with overlapped "
                         "launches, but the bracketed launches then measured ~5%% longer)")
    ap.add_argument("--ref-step-seconds", type=float, default=3.0)
    ap.add_argument("--pipeline-width", choices=["padded", "real"], default="padded",
                    help="gsasr-x*: hold the decoder's d = 180 at 184 (aligned GEMM rows) or not")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res), flush=True)
        return
    import torch
    import torch.distributed as dist
    if world > 1:
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    import __graft_entry__
    __graft_entry__.build()
    if args.workload in PIPELINE_SCALES:
        if world > 1:
            raise SystemExit("the whole-pipeline workloads run on one GPU")
        res = run_pipeline(args, rank, world, local_rank)
    elif args.workload == "c5":
        res = run_train(args, rank, world, local_rank)
    else:
        res = run_gpu(args, rank, world, local_rank)
        if args.workload == "c2" and not args.no_x12:
            res["x12"] = run_x12(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
