"""Sharding for several GPUs: one process per GPU.

Batches: images are independent (own Gaussians, size and scale), so a
multi-GPU render partitions the images across ranks and needs no collective on
the data path; the only communication is the host-side max of the timings.
Images are assigned longest-first (by HR pixels) to the least-loaded rank,
which keeps uneven batches balanced.

One large image: its HR rows are split into horizontal bands, one per rank
(`gs_view.row0`). Each rank renders its band from all the Gaussians: the
forward needs no exchange (the bands are the image's rows, bit for bit when
each band starts on a tile row). The adjoint of a band is the gradient of the
loss restricted to its rows, so the image's gradient is the sum of the bands':
one all-reduce of the N x 9 gradients (`allreduce_band_grads`).
"""
from __future__ import annotations

from typing import Sequence


def shard_images(costs: Sequence[float], world: int) -> list[list[int]]:
    """Partition image indices over `world` ranks, longest processing time
    first. Returns, per rank, its image indices in ascending order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    loads = [0.0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda k: (-costs[k], k)):
        r = min(range(world), key=lambda q: (loads[q], q))
        parts[r].append(i)
        loads[r] += costs[i]
    return [sorted(p) for p in parts]


def image_costs(views) -> list[float]:
    """Cost proxy of each image: its HR pixel count (the render's work grows
    with HR pixels at a fixed Gaussian density)."""
    return [float(v.out_h * v.out_w) for v in views]


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over the ranks of the default process group (the
    job-level time of a step); identity without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def band_rows(out_h: int, parts: int, tile: int = 16) -> list[tuple[int, int]]:
    """Split out_h rows into `parts` bands (row0, rows) starting on tile rows
    (so that every band renders its rows exactly as the whole image does),
    as even as the tile rows allow; bands may be empty when there are fewer
    tile rows than parts."""
    if parts < 1 or tile < 1 or out_h < 0:
        raise ValueError("need parts >= 1, tile >= 1, out_h >= 0")
    trows = -(-out_h // tile)
    bands = []
    for p in range(parts):
        t0, t1 = (trows * p) // parts, (trows * (p + 1)) // parts
        r0, r1 = min(out_h, t0 * tile), min(out_h, t1 * tile)
        bands.append((r0, r1 - r0))
    return bands


def band_view(view, row0: int, rows: int):
    """A copy of `view` restricted to image rows row0 .. row0 + rows - 1.
    rows must be >= 1: a rank whose band from band_rows() is empty renders
    nothing and passes zero gradients to allreduce_band_grads()."""
    import copy
    if rows < 1 or row0 < 0:
        raise ValueError(f"band of {rows} rows at row {row0}: an empty band renders nothing")
    v = copy.copy(view)
    v.out_h = rows
    v.row0 = row0
    return v


def allreduce_band_grads(grads):
    """Sum a band's parameter gradients over the ranks of the default process
    group (in place; the image's gradient on every rank). Identity without a
    process group."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(grads, op=dist.ReduceOp.SUM)
    return grads
