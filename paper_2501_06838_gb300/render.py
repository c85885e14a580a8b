"""PyTorch-facing binding of the GSASR scale-aware rasterizer (libgs.so).

PyTorch provides device memory and streams; all arithmetic of the render and
its adjoint runs in the library's CUDA kernels (include/gs.h). Functions:

  count_pairs(gs, views)                    exact (tile, Gaussian) pair count (syncs)
  render(g, view) / render_batched(gs, views)          forward (Eq. 4, Algorithm 1)
  render_bwd(...) / render_batched_bwd(...)            adjoint with frozen windows
  GSRender.apply(offset, sigma, rho, rgb, alpha, view)  autograd, one image
  GSRenderBatched.apply(views, m, sizes, offset, ...)   autograd, uneven batch

Parameters are physical (post-activation): offset o (or absolute centre when
ref_grid_m == 0), sigma, rho, rgb, alpha, all in LR pixels (GSASR, arXiv
2501.06838, Sec. 3.1-3.2), stored as float32, bfloat16 or float16 -- or raw
outputs of the Gaussian primary head when `Gaussians.head` is set (the
library applies the head's activations and returns gradients for the raw
values).
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
from typing import Sequence

import torch

from . import _abi

_DTYPES = {torch.float32: _abi.GS_F32, torch.bfloat16: _abi.GS_BF16, torch.float16: _abi.GS_F16}

WINDOW_SIGMA, WINDOW_RATIO = _abi.GS_WINDOW_SIGMA, _abi.GS_WINDOW_RATIO
NORM_DENSITY, NORM_PEAK = _abi.GS_NORM_DENSITY, _abi.GS_NORM_PEAK
ALIGN_EQ4, ALIGN_HALF = _abi.GS_ALIGN_EQ4, _abi.GS_ALIGN_HALF


@dataclasses.dataclass
class View:
    """Output request (a gs_view): an out_h x out_w HR image of an lr_h x lr_w
    LR grid at scale s (Eq. 4). window: WINDOW_SIGMA (|x/s - mu| <= k sigma,
    k = trunc_k) or WINDOW_RATIO (Algorithm 1, ratio r = trunc_k); norm:
    NORM_DENSITY (Eq. 2) or NORM_PEAK; align: ALIGN_EQ4 (x samples x / s) or
    ALIGN_HALF ((x + 1/2) / s - 1/2). row0: the first image row the output
    holds (a horizontal band of out_h rows; 0 for the whole image)."""
    lr_h: int
    lr_w: int
    out_h: int
    out_w: int
    scale: float
    trunc_k: float = 3.0
    norm: int = 0
    window: int = 0
    align: int = 0
    row0: int = 0


def out_size(lr: int, scale: float) -> int:
    """floor(s * lr) with s rounded to float32 (the product is exact in double)."""
    return int(math.floor(float(ctypes.c_float(scale).value) * lr))


@dataclasses.dataclass
class Gaussians:
    """Device parameters of one image's Gaussians (contiguous tensors)."""
    offset: torch.Tensor  # [N, 2]
    sigma: torch.Tensor   # [N, 2]
    rho: torch.Tensor     # [N]
    rgb: torch.Tensor     # [N, 3]
    alpha: torch.Tensor   # [N]
    ref_grid_m: int = 1
    head: object = None   # fused head (sigma_lo, sigma_span, rho_scale, offset_scale, offset_tanh)

    @property
    def n(self) -> int:
        return int(self.rho.shape[0])

    def tensors(self):
        return (self.offset, self.sigma, self.rho, self.rgb, self.alpha)

    @staticmethod
    def from_arrays(arrays, ref_grid_m: int, device="cuda", dtype=torch.float32):
        """From host arrays (numpy or tensors) of (offset, sigma, rho, rgb, alpha)."""
        ts = [torch.as_tensor(a).to(device=device, dtype=dtype).contiguous() for a in arrays]
        return Gaussians(*ts, ref_grid_m=ref_grid_m)


def _need(t: torch.Tensor, shape, dtype, device: torch.device, what: str) -> torch.Tensor:
    """Host-side check of a caller-supplied buffer before its pointer reaches
    the library: the library trusts every pointer and size it is given."""
    if t.device != device:
        raise ValueError(f"{what} is on {t.device}, the parameters on {device}")
    if t.dtype != dtype:
        raise TypeError(f"{what} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous() or tuple(t.shape) != tuple(shape):
        raise ValueError(f"{what} must be contiguous with shape {tuple(shape)}, "
                         f"got {tuple(t.shape)}")
    return t


def _device(gs: Sequence[Gaussians], stream=None) -> torch.device:
    """The one CUDA device all images' parameters are on. It must be the
    current device, whose stream the library launches on (or the device of
    the stream passed)."""
    dev = gs[0].rho.device
    if dev.type != "cuda":
        raise ValueError("parameter tensors must be CUDA tensors")
    for g in gs:
        for t in g.tensors():
            if t.device != dev:
                raise ValueError(f"all parameter tensors must be on one device ({dev}, {t.device})")
    sdev = stream.device if stream is not None else torch.device("cuda", torch.cuda.current_device())
    if sdev != dev:
        raise ValueError(f"parameters are on {dev} but the launch stream is on {sdev}; "
                         f"use torch.cuda.device({dev}) or pass a stream of that device")
    return dev


def _struct_g(g: Gaussians) -> _abi.GsGaussians:
    ts = g.tensors()
    dt = ts[0].dtype
    if dt not in _DTYPES:
        raise TypeError(f"unsupported parameter dtype {dt}")
    n = g.n
    shapes = ((n, 2), (n, 2), (n,), (n, 3), (n,))
    for t, shp in zip(ts, shapes):
        if t.dtype != dt:
            raise TypeError("all parameter tensors must share one dtype")
        if not t.is_cuda:
            raise ValueError("parameter tensors must be CUDA tensors")
        if t.device != ts[0].device:
            raise ValueError("all parameter tensors must be on one device")
        if not t.is_contiguous() or tuple(t.shape) != shp:
            raise ValueError(f"parameter tensor must be contiguous with shape {shp}, got {tuple(t.shape)}")
    hp = None
    if g.head is not None:
        h = g.head
        hp = ctypes.pointer(_abi.GsHead(float(h.sigma_lo), float(h.sigma_span), float(h.rho_scale),
                                        float(h.offset_scale), int(h.offset_tanh)))
    G = _abi.GsGaussians(ts[0].data_ptr(), ts[1].data_ptr(), ts[2].data_ptr(),
                         ts[3].data_ptr(), ts[4].data_ptr(), n, _DTYPES[dt], int(g.ref_grid_m), hp)
    G._head_keep = hp   # the C struct points into this object during the call
    return G


def _struct_v(v, tile: int = 0, batch: int = 0, adjoint: int = 0) -> _abi.GsView:
    tile = tile or getattr(v, "tile", 0) or 0
    batch = batch or getattr(v, "batch", 0) or 0
    adjoint = adjoint or getattr(v, "adjoint", 0) or 0
    return _abi.GsView(int(v.lr_h), int(v.lr_w), int(v.out_h), int(v.out_w), float(v.scale),
                       float(getattr(v, "trunc_k", 3.0)), int(getattr(v, "norm", 0)),
                       int(tile), int(batch), int(getattr(v, "window", 0)),
                       int(getattr(v, "align", 0)), int(adjoint), int(getattr(v, "binning", 0)),
                       int(getattr(v, "row0", 0)), int(getattr(v, "raster", 0)))


def _arrays(gs: Sequence[Gaussians], views, tile=0, batch=0):
    n = len(gs)
    if n != len(views) or n == 0:
        raise ValueError("need one view per image and at least one image")
    structs = [_struct_g(g) for g in gs]
    G = (_abi.GsGaussians * n)(*structs)
    G._head_keep = [st._head_keep for st in structs]   # head structs the array points to
    V = (_abi.GsView * n)(*[_struct_v(v, tile, batch) for v in views])
    return n, G, V


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class Workspace:
    """Caller-owned device scratch for one render (and its adjoint)."""

    def __init__(self, nbytes: int, device=None):
        self.buf = torch.empty(int(nbytes), dtype=torch.uint8, device=device or "cuda")
        self.device = self.buf.device
        if self.buf.data_ptr() % 256:
            raise RuntimeError("workspace allocation is not 256-byte aligned")

    @property
    def ptr(self) -> int:
        return self.buf.data_ptr()

    @property
    def nbytes(self) -> int:
        return self.buf.numel()


def workspace_bytes(gs, views, capacity: int, tile=0, batch=0) -> int:
    n, G, V = _arrays(gs, views, tile, batch)
    b = _abi.load().gs_workspace_size(n, G, V, int(capacity))
    if b == 0:
        raise _abi.GsError(_abi.GS_ERR_INVALID, "gs_workspace_size", _abi.last_error())
    return int(b)


def _check_ws(ws: Workspace, dev: torch.device):
    if ws.device != dev:
        raise ValueError(f"workspace is on {ws.device}, the parameters on {dev}")


def count_pairs(gs, views, tile=0, batch=0, stream=None) -> int:
    """Exact number of (tile, Gaussian) pairs; synchronises the stream."""
    n, G, V = _arrays(gs, views, tile, batch)
    dev = _device(gs, stream)
    ws = Workspace(workspace_bytes(gs, views, 0, tile, batch), dev)
    out = ctypes.c_int64(0)
    _abi.check(_abi.load().gs_count_pairs(n, G, V, ws.ptr, ws.nbytes, _stream(stream),
                                          ctypes.byref(out)), "gs_count_pairs")
    return int(out.value)


def make_workspace(gs, views, capacity=None, tile=0, batch=0, slack: float = 0.0,
                   stream=None) -> Workspace:
    if capacity is None:
        capacity = count_pairs(gs, views, tile, batch, stream)
    capacity = int(capacity * (1.0 + slack)) + (1 if slack else 0)
    return Workspace(workspace_bytes(gs, views, capacity, tile, batch), gs[0].rho.device)


def render_batched(gs, views, outs=None, ws: Workspace | None = None, tile=0, batch=0,
                   stream=None, check: bool = False):
    """Forward render of several images in one launch chain. Returns (outs, ws)."""
    n, G, V = _arrays(gs, views, tile, batch)
    dev = _device(gs, stream)
    if outs is None:
        outs = [torch.empty((3, v.out_h, v.out_w), dtype=torch.float32, device=dev) for v in views]
    if len(outs) != n:
        raise ValueError("need one output per image")
    for o, v in zip(outs, views):
        _need(o, (3, v.out_h, v.out_w), torch.float32, dev, "output")
    if ws is None:
        ws = make_workspace(gs, views, None, tile, batch, stream=stream)
    _check_ws(ws, dev)
    P = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
    _abi.check(_abi.load().gs_render_batched(n, G, V, P, ws.ptr, ws.nbytes, _stream(stream)),
               "gs_render_batched")
    if check:
        sync_status(ws, stream)
    return outs, ws


def render_batched_bwd(gs, views, grad_outs, ws: Workspace, grads=None, tile=0, batch=0,
                       stream=None, check: bool = False):
    """Adjoint of the last render_batched on ws. Returns a list of [N_i, 9] float32."""
    n, G, V = _arrays(gs, views, tile, batch)
    dev = _device(gs, stream)
    _check_ws(ws, dev)
    if len(grad_outs) != n:
        raise ValueError("need one upstream gradient per image")
    grad_outs = [g.contiguous().float() for g in grad_outs]
    for go, v in zip(grad_outs, views):
        _need(go, (3, v.out_h, v.out_w), torch.float32, dev, "grad_out")
    if grads is None:
        grads = [torch.empty((g.n, 9), dtype=torch.float32, device=dev) for g in gs]
    if len(grads) != n:
        raise ValueError("need one gradient buffer per image")
    for gr, g in zip(grads, gs):
        _need(gr, (g.n, 9), torch.float32, dev, "gradient buffer")
    GO = (ctypes.c_void_p * n)(*[g.data_ptr() for g in grad_outs])
    GR = (ctypes.c_void_p * n)(*[g.data_ptr() for g in grads])
    _abi.check(_abi.load().gs_render_batched_bwd(n, G, V, GO, GR, ws.ptr, ws.nbytes,
                                                 _stream(stream)), "gs_render_batched_bwd")
    if check:
        sync_status(ws, stream)
    return grads


def render(g: Gaussians, view, out=None, ws=None, tile=0, batch=0, stream=None, check=False):
    outs, ws = render_batched([g], [view], None if out is None else [out], ws, tile, batch,
                              stream, check)
    return outs[0], ws


def render_bwd(g: Gaussians, view, grad_out, ws, grads=None, tile=0, batch=0, stream=None,
               check=False):
    return render_batched_bwd([g], [view], [grad_out], ws, None if grads is None else [grads],
                              tile, batch, stream, check)[0]


def render_single_fwd(g: Gaussians, view, out, ws: Workspace, tile=0, batch=0, stream=None):
    """Forward through the single-image entry point gs_render_fwd."""
    G = _struct_g(g)
    V = _struct_v(view, tile, batch)
    dev = _device([g], stream)
    _check_ws(ws, dev)
    _need(out, (3, view.out_h, view.out_w), torch.float32, dev, "output")
    _abi.check(_abi.load().gs_render_fwd(ctypes.byref(G), ctypes.byref(V), out.data_ptr(),
                                         ws.ptr, ws.nbytes, _stream(stream)), "gs_render_fwd")
    return out


def render_single_bwd(g: Gaussians, view, grad_out, grads, ws: Workspace, tile=0, batch=0,
                      stream=None):
    """Adjoint through the single-image entry point gs_render_bwd."""
    G = _struct_g(g)
    V = _struct_v(view, tile, batch)
    dev = _device([g], stream)
    _check_ws(ws, dev)
    _need(grad_out, (3, view.out_h, view.out_w), torch.float32, dev, "grad_out")
    _need(grads, (g.n, 9), torch.float32, dev, "gradient buffer")
    _abi.check(_abi.load().gs_render_bwd(ctypes.byref(G), ctypes.byref(V), grad_out.data_ptr(),
                                         grads.data_ptr(), ws.ptr, ws.nbytes, _stream(stream)),
               "gs_render_bwd")
    return grads


def sync_status(ws: Workspace, stream=None):
    """Raise GsError if the kernels flagged a device-side problem (resets it)."""
    _abi.check(_abi.load().gs_sync_status(ws.ptr, _stream(stream)), "device status")


def read_stats(ws: Workspace, stream=None) -> dict:
    st = _abi.GsStats()
    _abi.check(_abi.load().gs_read_stats(ws.ptr, _stream(stream), ctypes.byref(st)), "gs_read_stats")
    return {f: getattr(st, f) for f, _ in _abi.GsStats._fields_}


def launch_count() -> int:
    return int(_abi.load().gs_launch_count())


# --------------------------------------------------------------------------
# Autograd (differentiable rendering, Sec. 3.1 "Fast Rasterization" and
# Sec. 3.2 "Rendering": the L1 loss is back-propagated through the render).
# Per-pixel weights are recomputed in the backward, never stored.
# --------------------------------------------------------------------------
def _split_grads(gr: torch.Tensor, dtype):
    return (gr[:, 0:2].to(dtype), gr[:, 2:4].to(dtype), gr[:, 4].to(dtype),
            gr[:, 5:8].to(dtype), gr[:, 8].to(dtype))


class GSRender(torch.autograd.Function):
    """apply(offset, sigma, rho, rgb, alpha, view[, ref_grid_m[, head]]): with a
    head the five tensors are raw head outputs and their gradients are too."""

    @staticmethod
    def forward(ctx, offset, sigma, rho, rgb, alpha, view, ref_grid_m: int = 1, head=None):
        g = Gaussians(offset.contiguous(), sigma.contiguous(), rho.contiguous(), rgb.contiguous(),
                      alpha.contiguous(), ref_grid_m, head)
        out, ws = render(g, view)
        ctx.g, ctx.view, ctx.ws = g, view, ws
        return out

    @staticmethod
    def backward(ctx, grad_out):
        gr = render_bwd(ctx.g, ctx.view, grad_out, ctx.ws)
        return (*_split_grads(gr, ctx.g.offset.dtype), None, None, None)


class GSRenderBatched(torch.autograd.Function):
    """Images of uneven sizes and scales in one launch chain. Parameters are
    concatenated over images; sizes[i] Gaussians belong to image i. With a
    head (a fused Gaussian primary head for every image) they are raw head
    outputs: apply(views, ref_grid_m, sizes, head, offset, sigma, rho, rgb,
    alpha); pass head=None for physical parameters."""

    @staticmethod
    def forward(ctx, views, ref_grid_m, sizes, head, offset, sigma, rho, rgb, alpha):
        gs, o = [], 0
        ts = [t.contiguous() for t in (offset, sigma, rho, rgb, alpha)]
        for n in sizes:
            gs.append(Gaussians(*[t[o:o + n] for t in ts], ref_grid_m=ref_grid_m, head=head))
            o += n
        outs, ws = render_batched(gs, views)
        ctx.gs, ctx.views, ctx.ws, ctx.dtype = gs, views, ws, offset.dtype
        return tuple(outs)

    @staticmethod
    def backward(ctx, *grad_outs):
        go = [torch.zeros((3, v.out_h, v.out_w), device=ctx.gs[0].rho.device) if g is None else g
              for g, v in zip(grad_outs, ctx.views)]
        grads = render_batched_bwd(ctx.gs, ctx.views, go, ctx.ws)
        gr = torch.cat(grads, 0)
        return (None, None, None, None, *_split_grads(gr, ctx.dtype))


class Plan:
    """A prepared render of fixed images: the ctypes arguments, the workspace
    and the output / gradient buffers are built once, so each call costs one
    C-ABI call. Fill `grad_outs` (or pass your own) before calling bwd().
    The calls are asynchronous and can be captured in a CUDA graph."""

    def __init__(self, gs, views, tile=0, batch=0, capacity=None, slack: float = 0.0,
                 with_grads: bool = True, stream=None, outs=None, grad_outs=None, grads=None):
        """outs / grad_outs / grads: optional caller-allocated device tensors
        ([3, out_h, out_w] float32 per image; [N_i, 9] float32 per image)."""
        self.gs, self.views = list(gs), list(views)
        self.n, self.G, self.V = _arrays(self.gs, self.views, tile, batch)
        dev = _device(self.gs, stream)
        self.ws = make_workspace(self.gs, self.views, capacity, tile, batch, slack, stream)
        self.outs = list(outs) if outs is not None else \
            [torch.empty((3, v.out_h, v.out_w), dtype=torch.float32, device=dev) for v in self.views]
        if len(self.outs) != self.n:
            raise ValueError("need one output per image")
        for o, v in zip(self.outs, self.views):
            _need(o, (3, v.out_h, v.out_w), torch.float32, dev, "output")
        self.P_out = (ctypes.c_void_p * self.n)(*[o.data_ptr() for o in self.outs])
        self.lib = _abi.load()
        if with_grads:
            self.grad_outs = list(grad_outs) if grad_outs is not None else \
                [torch.zeros_like(o) for o in self.outs]
            self.grads = list(grads) if grads is not None else \
                [torch.empty((g.n, 9), dtype=torch.float32, device=dev) for g in self.gs]
            if len(self.grad_outs) != self.n or len(self.grads) != self.n:
                raise ValueError("need one upstream gradient and one gradient buffer per image")
            for go, gr, v, g in zip(self.grad_outs, self.grads, self.views, self.gs):
                _need(go, (3, v.out_h, v.out_w), torch.float32, dev, "grad_out")
                _need(gr, (g.n, 9), torch.float32, dev, "gradient buffer")
            self.P_go = (ctypes.c_void_p * self.n)(*[g.data_ptr() for g in self.grad_outs])
            self.P_gr = (ctypes.c_void_p * self.n)(*[g.data_ptr() for g in self.grads])

    def fwd(self, stream=None):
        st = self.lib.gs_render_batched(self.n, self.G, self.V, self.P_out, self.ws.ptr,
                                        self.ws.nbytes, _stream(stream))
        if st:
            _abi.check(st, "gs_render_batched")
        return self.outs

    def bwd(self, stream=None):
        st = self.lib.gs_render_batched_bwd(self.n, self.G, self.V, self.P_go, self.P_gr,
                                            self.ws.ptr, self.ws.nbytes, _stream(stream))
        if st:
            _abi.check(st, "gs_render_batched_bwd")
        return self.grads

    def status(self, stream=None):
        sync_status(self.ws, stream)

    def stats(self, stream=None) -> dict:
        return read_stats(self.ws, stream)


def timing_enable(kernel_names=None):
    """Per-kernel CUDA-event timing of the named kernels (None: all; []: off)."""
    lib = _abi.load()
    if kernel_names is None:
        mask = -1
    else:
        ids = {lib.gs_kernel_name(i).decode(): i for i in range(32) if lib.gs_kernel_name(i)}
        mask = 0
        for k in kernel_names:
            if k not in ids:
                raise ValueError(f"unknown kernel {k!r}; known: {sorted(ids)}")
            mask |= 1 << ids[k]
    _abi.check(lib.gs_timing_enable(mask), "gs_timing_enable")


def timing_read() -> dict:
    """{kernel name: (total ms, launches)} since the last read (synchronises)."""
    lib = _abi.load()
    ms = (ctypes.c_double * 32)()
    cnt = (ctypes.c_int64 * 32)()
    n = lib.gs_timing_read(ms, cnt, 32)
    return {lib.gs_kernel_name(i).decode(): (ms[i], cnt[i]) for i in range(n) if cnt[i]}


def timing_release():
    """Drop the timed launches recorded under stream capture (before the graph goes)."""
    _abi.check(_abi.load().gs_timing_release(), "gs_timing_release")


def probe_peaks() -> dict:
    """Measured FFMA / FFMA2 / MUFU.EX2 rates and the forward pair mix (per
    second and per SM per clock at the device's maximum clock)."""
    lib = _abi.load()
    dev = torch.cuda.current_device()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    buf = torch.empty(sms * 6 * 256, dtype=torch.float32, device="cuda")
    pk = _abi.GsPeaks()
    _abi.check(lib.gs_probe_peaks(buf.data_ptr(), buf.numel() * 4, _stream(), ctypes.byref(pk)),
               "gs_probe_peaks")
    return {f: getattr(pk, f) for f, _ in _abi.GsPeaks._fields_ if f != "reserved"}
