"""FP64 CPU oracle of the scale-aware Gaussian rasterizer (GSASR, Sec. 3.1).

TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this package. It shares no code with the CUDA
library and never imports it.

The numerics live in `gs_oracle.cpp` (plain C++, FP64, std::thread); this file
compiles it with g++ (no FMA contraction, so the float32 window decisions are
reproducible) and wraps it with ctypes/numpy.

Functions (all citations are to GSASR, arXiv 2501.06838):
  render(g, view, mode="rect"|"allpairs")   Eq. 1-4 with the Algorithm-1 window
                                             (sigma box or ratio box; Eq. 4 or
                                             half-pixel alignment)
  adjoint(g, view, grad_out)                 d(sum grad_out*I)/d params, frozen windows
  complex_step(g, view, grad_out, gids)      same derivative by complex step
  rects(g, view)                             the integer windows R_i
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


class OView(ctypes.Structure):
    _fields_ = [("lr_h", ctypes.c_int32), ("lr_w", ctypes.c_int32),
                ("out_h", ctypes.c_int32), ("out_w", ctypes.c_int32),
                ("scale", ctypes.c_float), ("trunc_k", ctypes.c_float),
                ("norm", ctypes.c_int32), ("ref_grid_m", ctypes.c_int32),
                ("window", ctypes.c_int32), ("align", ctypes.c_int32)]


class OHead(ctypes.Structure):
    _fields_ = [("sigma_lo", ctypes.c_float), ("sigma_span", ctypes.c_float),
                ("rho_scale", ctypes.c_float), ("offset_scale", ctypes.c_float),
                ("offset_tanh", ctypes.c_int32), ("pad", ctypes.c_int32 * 3)]


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (idempotent)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread",
               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        lp = ctypes.POINTER(ctypes.c_int64)
        hp = ctypes.POINTER(OHead)
        fp = ctypes.POINTER(ctypes.c_float)
        common = [dp, dp, dp, dp, dp, ctypes.c_int64, ctypes.POINTER(OView), hp]
        lib.gso_rects.argtypes = common + [ip]
        lib.gso_render.argtypes = common + [ctypes.c_int, ctypes.c_int, ip, dp]
        lib.gso_adjoint.argtypes = common + [dp, ctypes.c_int, ip, dp]
        lib.gso_complex_step.argtypes = common + [dp, lp, ctypes.c_int64, ctypes.c_double, dp]
        lib.gso_hardware_threads.argtypes = []
        lib.gso_gaussian_loss.argtypes = common + [dp, ctypes.c_int64, dp]
        lib.gso_gaussian_loss.restype = ctypes.c_double
        lib.gso_centre.argtypes = [dp, ctypes.c_int64, ctypes.POINTER(OView), hp, ctypes.c_int64, dp]
        lib.gso_head_f32.argtypes = [fp, ctypes.c_int64, ctypes.c_int, fp]
        for f in (lib.gso_rects, lib.gso_render, lib.gso_adjoint, lib.gso_complex_step,
                  lib.gso_hardware_threads, lib.gso_centre, lib.gso_head_f32):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def hardware_threads() -> int:
    return int(_load().gso_hardware_threads())


def _f64(a, shape):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64)).reshape(shape)
    return a


def _ptr(a, t=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _args(g, view, ref_grid_m=None):
    n = int(g.rho.shape[0])
    arrs = [_f64(g.offset, (n, 2)), _f64(g.sigma, (n, 2)), _f64(g.rho, (n,)),
            _f64(g.rgb, (n, 3)), _f64(g.alpha, (n,))]
    m = g.ref_grid_m if ref_grid_m is None else ref_grid_m
    ov = OView(view.lr_h, view.lr_w, view.out_h, view.out_w, view.scale,
               view.trunc_k, view.norm, m, getattr(view, "window", 0), getattr(view, "align", 0))
    h = getattr(g, "head", None)
    hd = None if h is None else ctypes.pointer(
        OHead(h.sigma_lo, h.sigma_span, h.rho_scale, h.offset_scale, int(h.offset_tanh)))
    return n, arrs, ov, hd


def rects(g, view) -> np.ndarray:
    n, arrs, ov, hd = _args(g, view)
    out = np.zeros((n, 4), dtype=np.int32)
    rc = _load().gso_rects(*[_ptr(a) for a in arrs], n, ctypes.byref(ov), hd,
                           _ptr(out, ctypes.c_int32))
    if rc:
        raise ValueError(f"oracle: invalid view ({rc})")
    return out


def _rect_arg(r, n):
    if r is None:
        return None, None
    r = np.ascontiguousarray(np.asarray(r, dtype=np.int32).reshape(n, 4))
    return r, _ptr(r, ctypes.c_int32)


def render(g, view, mode: str = "rect", threads: int = 0, frozen_rects=None) -> np.ndarray:
    """I_SR as float64 [3, out_h, out_w]."""
    n, arrs, ov, hd = _args(g, view)
    out = np.empty((3, view.out_h, view.out_w), dtype=np.float64)
    keep, rp = _rect_arg(frozen_rects, n)
    rc = _load().gso_render(*[_ptr(a) for a in arrs], n, ctypes.byref(ov), hd,
                            {"rect": 0, "allpairs": 1}[mode], threads, rp, _ptr(out))
    if rc:
        raise ValueError(f"oracle: invalid view ({rc})")
    return out


def adjoint(g, view, grad_out, threads: int = 0, frozen_rects=None) -> np.ndarray:
    """[N, 9] gradients (o_x, o_y, sigma_x, sigma_y, rho, r, g, b, alpha); with a
    head, with respect to the raw head outputs."""
    n, arrs, ov, hd = _args(g, view)
    go = _f64(grad_out, (3, view.out_h, view.out_w))
    out = np.empty((n, 9), dtype=np.float64)
    keep, rp = _rect_arg(frozen_rects, n)
    rc = _load().gso_adjoint(*[_ptr(a) for a in arrs], n, ctypes.byref(ov), hd, _ptr(go), threads,
                             rp, _ptr(out))
    if rc:
        raise ValueError(f"oracle: invalid view ({rc})")
    return out


def complex_step(g, view, grad_out, gids, h: float = 1e-30) -> np.ndarray:
    n, arrs, ov, hd = _args(g, view)
    go = _f64(grad_out, (3, view.out_h, view.out_w))
    ids = np.ascontiguousarray(np.asarray(gids, dtype=np.int64))
    out = np.empty((len(ids), 9), dtype=np.float64)
    rc = _load().gso_complex_step(*[_ptr(a) for a in arrs], n, ctypes.byref(ov), hd, _ptr(go),
                                  _ptr(ids, ctypes.c_int64), len(ids), h, _ptr(out))
    if rc:
        raise ValueError(f"oracle: bad arguments ({rc})")
    return out


def centre(g, view, gid: int) -> np.ndarray:
    """FP64 centre mu = p + o of Gaussian `gid` (LR pixels)."""
    n, arrs, ov, hd = _args(g, view)
    mu = np.zeros(2, dtype=np.float64)
    rc = _load().gso_centre(_ptr(arrs[0]), n, ctypes.byref(ov), hd, int(gid), _ptr(mu))
    if rc:
        raise ValueError("oracle: bad arguments")
    return mu


def gaussian_loss(g, view, grad_out, gid: int, theta) -> float:
    """sum over the frozen window R_gid of grad_out . G_gid with parameters theta
    = (mu_x, mu_y, sigma_x, sigma_y, rho, r, g, b, alpha)."""
    n, arrs, ov, hd = _args(g, view)
    go = _f64(grad_out, (3, view.out_h, view.out_w))
    th = _f64(theta, (9,))
    return float(_load().gso_gaussian_loss(*[_ptr(a) for a in arrs], n, ctypes.byref(ov), hd,
                                           _ptr(go), int(gid), _ptr(th)))


def theta_of(g, view, gid: int) -> np.ndarray:
    if getattr(g, "head", None) is not None:   # the raw head outputs themselves
        return np.array([g.offset[gid, 0], g.offset[gid, 1], g.sigma[gid, 0], g.sigma[gid, 1],
                         g.rho[gid], g.rgb[gid, 0], g.rgb[gid, 1], g.rgb[gid, 2], g.alpha[gid]],
                        dtype=np.float64)
    mu = centre(g, view, gid)
    return np.array([mu[0], mu[1], g.sigma[gid, 0], g.sigma[gid, 1], g.rho[gid],
                     g.rgb[gid, 0], g.rgb[gid, 1], g.rgb[gid, 2], g.alpha[gid]], dtype=np.float64)


def central_difference(g, view, grad_out, gids, h: float = 1e-4) -> np.ndarray:
    """[k, 9] central differences of the frozen-window loss (step h per parameter)."""
    n, arrs, ov, hd = _args(g, view)
    go = _f64(grad_out, (3, view.out_h, view.out_w))
    ptrs = [_ptr(a) for a in arrs]
    lib = _load()
    out = np.zeros((len(gids), 9))
    for t, gid in enumerate(gids):
        th = theta_of(g, view, gid)
        for p in range(9):
            tp, tm = th.copy(), th.copy()
            tp[p] += h
            tm[p] -= h
            lp = lib.gso_gaussian_loss(*ptrs, n, ctypes.byref(ov), hd, _ptr(go), int(gid), _ptr(tp))
            lm = lib.gso_gaussian_loss(*ptrs, n, ctypes.byref(ov), hd, _ptr(go), int(gid), _ptr(tm))
            out[t, p] = (lp - lm) / (2 * h)
    return out


def head_f32(x, kind: str) -> np.ndarray:
    """The fixed float32 sequences the window uses with a fused head:
    kind 'sigmoid', 'tanh' or 'exp' of float32 inputs."""
    xs = np.ascontiguousarray(np.asarray(x, dtype=np.float32).ravel())
    y = np.empty_like(xs)
    _load().gso_head_f32(_ptr(xs, ctypes.c_float), xs.size, {"sigmoid": 0, "tanh": 1, "exp": 2}[kind],
                         _ptr(y, ctypes.c_float))
    return y
