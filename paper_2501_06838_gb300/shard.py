"""Image-level sharding for several GPUs: one process per GPU.

Images of a batch are independent (own Gaussians, size and scale), so a
multi-GPU render partitions the images across ranks and needs no collective on
the data path; the only communication is the host-side max of the timings.
Images are assigned longest-first (by HR pixels x mean footprint proxy) to the
least-loaded rank, which keeps uneven batches balanced.
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
