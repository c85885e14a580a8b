"""Autotuner for the launch parameters of the render (screen tile edge,
Gaussians per shared-memory batch, binning, raster layout, adjoint kernel): a
thin binding of the library's
gs_tune, which times every candidate on the caller's own workload with CUDA
events (median of `reps` calls after two warm-up calls), returns the fastest
and keeps it in a JSON-lines cache keyed by the workload's signature (device, dtype,
fwd or fwd+bwd, and the log2 size classes of HR pixels, images and pairs per
pixel).
"""
from __future__ import annotations

import ctypes
import os

from . import _abi
from .render import Plan, _stream

_BINNING = {_abi.GS_BINNING_SORT: "sort", _abi.GS_BINNING_GRID: "grid"}


def default_cache() -> str:
    return os.environ.get("GS_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "gs_tune.jsonl"))


def tune(gs, views, with_grads: bool = True, reps: int = 5, cache: str | None = None,
         stream=None) -> dict:
    """-> {"tile", "batch", "binning", "adjoint", "raster", "ms", "from_cache", "n_timed"}
    for this workload (the launch parameters to put in its views)."""
    cache = cache or default_cache()
    os.makedirs(os.path.dirname(cache) or ".", exist_ok=True)
    # tile 8 with the sorted pair list needs the most workspace: it fits every
    # candidate
    saved = [getattr(v, "binning", 0) for v in views]
    for v in views:
        v.binning = _abi.GS_BINNING_SORT
    try:
        plan = Plan(gs, views, tile=8, batch=32, with_grads=with_grads, stream=stream)
    finally:
        for v, b in zip(views, saved):
            v.binning = b
    if with_grads:
        for go in plan.grad_outs:
            go.normal_()
    t = _abi.GsTuning()
    lib = _abi.load()
    st = lib.gs_tune(plan.n, plan.G, plan.V, plan.P_out, plan.P_go if with_grads else None,
                     plan.P_gr if with_grads else None, plan.ws.ptr, plan.ws.nbytes,
                     _stream(stream), int(reps), cache.encode(), ctypes.byref(t))
    _abi.check(st, "gs_tune")
    return {"tile": t.tile, "batch": t.batch, "binning": _BINNING.get(t.binning, t.binning),
            "binning_code": t.binning, "adjoint": t.adjoint, "raster": t.raster,
            "ms": float(t.ms),
            "from_cache": bool(t.from_cache), "n_timed": t.n_timed}
