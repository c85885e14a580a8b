"""GB300 (sm_103a) scale-aware differentiable 2D Gaussian rasterizer.

The hot path of GSASR (arXiv 2501.06838): Gaussians predicted on an LR grid
are rendered into a super-resolved image at any scale factor (Eq. 4 with the
Algorithm-1 window) and differentiated. The computation runs in the CUDA
library libgs.so behind the C-ABI in include/gs.h; this package is its thin
PyTorch binding.
"""
from ._abi import GsError, load as load_library  # noqa: F401
from .render import (Gaussians, GSRender, GSRenderBatched, Plan, View, Workspace, count_pairs,  # noqa: F401
                     launch_count, timing_enable, timing_read, timing_release, make_workspace, read_stats, render, render_batched,
                     render_batched_bwd, render_bwd, render_single_bwd, render_single_fwd,
                     out_size, sync_status, workspace_bytes)

__all__ = ["Gaussians", "GSRender", "GSRenderBatched", "Plan", "View", "Workspace", "timing_enable",
           "timing_read", "timing_release", "GsError", "count_pairs",
           "launch_count", "load_library", "make_workspace", "read_stats", "render",
           "render_batched", "render_batched_bwd", "render_bwd", "render_single_bwd",
           "render_single_fwd", "out_size", "sync_status", "workspace_bytes"]
