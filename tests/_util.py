"""Shared helpers of the GPU tests: device copies of synthetic inputs and the
error metrics (normwise per channel / per gradient field)."""
import numpy as np

import gs_synthetic as S


def device_gaussians(g: S.GaussianSet, device="cuda"):
    """Copy the stored parameter arrays of `g` to the device in their dtype."""
    import torch
    import paper_2501_06838_gb300 as gs
    ts = []
    for arr in g.storage():
        if g.dtype == "bf16":
            t = torch.from_numpy(np.ascontiguousarray(arr).view(np.int16)).view(torch.bfloat16)
        else:
            t = torch.from_numpy(np.ascontiguousarray(arr))
        ts.append(t.to(device).contiguous())
    return gs.Gaussians(*ts, ref_grid_m=g.ref_grid_m, head=getattr(g, "head", None))


def normwise(a, ref, axis=None):
    """max |a - ref| / max |ref| (per channel of a [3,H,W] image when axis=(1,2))."""
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.abs(ref).max(axis=axis)
    num = np.abs(a - ref).max(axis=axis)
    return num / np.where(den > 0, den, 1.0)


def psnr(a, ref):
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    mse = np.mean((a - ref) ** 2)
    peak = np.abs(ref).max()
    return float("inf") if mse == 0 else 10 * np.log10(peak * peak / mse)


def view_with(v: S.View, **kw):
    d = dict(lr_h=v.lr_h, lr_w=v.lr_w, out_h=v.out_h, out_w=v.out_w, scale=v.scale,
             trunc_k=v.trunc_k, norm=v.norm, window=v.window, align=v.align)
    d.update(kw)
    return S.View(**d)


def absolute(mu, sigma, rho, rgb, alpha, lr_h, lr_w):
    f32 = lambda a: np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)
    return S.GaussianSet(f32(mu), f32(sigma), f32(rho), f32(rgb), f32(alpha), lr_h=lr_h, lr_w=lr_w,
                         ref_grid_m=0)
