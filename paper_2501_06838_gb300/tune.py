"""Autotuner for the launch parameters of the render: screen tile edge
(8, 16, 32 HR px) and Gaussians per shared-memory batch (32 or 64 per warp
group). Each candidate is timed on the caller's own workload with CUDA events
(median of `reps` calls after a warm-up), the fastest is returned and cached
in a JSON file keyed by the device, the parameter dtype, whether the adjoint is
included, and the workload's size class (log2 of HR pixels, of images and of
tile pairs per HR pixel).
"""
from __future__ import annotations

import json
import math
import os
import threading

import torch

from .render import Plan, count_pairs

CANDIDATES = ((16, 32), (16, 64), (8, 32), (8, 64), (32, 64), (32, 128))
_lock = threading.Lock()


def default_cache() -> str:
    return os.environ.get("GS_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "gs_tune.json"))


def signature(gs, views, with_grads: bool) -> str:
    px = sum(v.out_h * v.out_w for v in views)
    pairs = count_pairs(gs, views, tile=16)
    dev = torch.cuda.get_device_name(gs[0].rho.device)
    dt = str(gs[0].offset.dtype).replace("torch.", "")
    return (f"{dev}|{dt}|{'fwdbwd' if with_grads else 'fwd'}|px{round(math.log2(max(px, 1)))}"
            f"|img{round(math.log2(len(views)))}|ppp{round(math.log2(max(pairs, 1) / px * 256))}")


def _time(plan: Plan, with_grads: bool, reps: int) -> float:
    for _ in range(2):
        plan.fwd()
        if with_grads:
            plan.bwd()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        plan.fwd()
        if with_grads:
            plan.bwd()
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b))
    plan.status()
    return sorted(ts)[len(ts) // 2]


def tune(gs, views, with_grads: bool = True, candidates=CANDIDATES, reps: int = 5,
         cache: str | None = None, refresh: bool = False) -> dict:
    """-> {"tile": t, "batch": b, "ms": median ms, "table": {..}} for this
    workload; reads and updates the JSON cache."""
    cache = cache or default_cache()
    key = signature(gs, views, with_grads)
    with _lock:
        table = {}
        if os.path.exists(cache):
            try:
                with open(cache) as f:
                    table = json.load(f)
            except (OSError, ValueError):
                table = {}
        if key in table and not refresh:
            return table[key]
    results = {}
    for tile, batch in candidates:
        plan = Plan(gs, views, tile=tile, batch=batch, with_grads=with_grads)
        if with_grads:
            for go in plan.grad_outs:
                go.normal_()
        results[f"{tile}x{batch}"] = _time(plan, with_grads, reps)
        del plan
    best = min(results, key=results.get)
    tile, batch = (int(x) for x in best.split("x"))
    entry = {"tile": tile, "batch": batch, "ms": results[best], "table": results}
    with _lock:
        os.makedirs(os.path.dirname(cache) or ".", exist_ok=True)
        table = {}
        if os.path.exists(cache):
            try:
                with open(cache) as f:
                    table = json.load(f)
            except (OSError, ValueError):
                table = {}
        table[key] = entry
        tmp = cache + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1)
        os.replace(tmp, cache)
    return entry
