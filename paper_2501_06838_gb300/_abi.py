"""ctypes mirror of include/gs.h and loader of the in-tree libgs.so.

Argument marshalling only: every step of the render runs in the CUDA kernels
of libgs.so. There is no fallback: if the library is missing, loading fails
with an error that says how to build it.
"""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgs.so")

GS_OK, GS_ERR_INVALID, GS_ERR_CAPACITY, GS_ERR_CUDA, GS_ERR_UNSUPPORTED, GS_ERR_TIMEOUT, \
    GS_ERR_INTERNAL = range(7)
GS_F32, GS_BF16, GS_F16 = 0, 1, 2
GS_NORM_DENSITY, GS_NORM_PEAK = 0, 1
GS_WINDOW_SIGMA, GS_WINDOW_RATIO = 0, 1
GS_ALIGN_EQ4, GS_ALIGN_HALF = 0, 1
GS_ADJOINT_AUTO, GS_ADJOINT_TILE, GS_ADJOINT_GAUSSIAN, GS_ADJOINT_QUADRANT = 0, 1, 2, 3
GS_BINNING_AUTO, GS_BINNING_SORT, GS_BINNING_GRID = 0, 1, 2
GS_RASTER_AUTO, GS_RASTER_TILE, GS_RASTER_PAIR = 0, 1, 2

EXPORTS = ("gs_workspace_size", "gs_count_pairs", "gs_render_fwd", "gs_render_bwd",
           "gs_render_batched", "gs_render_batched_bwd", "gs_sync_status", "gs_read_stats",
           "gs_last_error", "gs_status_string", "gs_launch_count", "gs_timing_enable",
           "gs_timing_read", "gs_timing_release", "gs_kernel_name", "gs_version",
           "gs_render_fwd_noalloc", "gs_noalloc_sync_status", "gs_probe_peaks", "gs_tune")


class GsHead(ctypes.Structure):
    _fields_ = [("sigma_lo", ctypes.c_float), ("sigma_span", ctypes.c_float),
                ("rho_scale", ctypes.c_float), ("offset_scale", ctypes.c_float),
                ("offset_tanh", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class GsGaussians(ctypes.Structure):
    _fields_ = [("offset", ctypes.c_void_p), ("sigma", ctypes.c_void_p),
                ("rho", ctypes.c_void_p), ("rgb", ctypes.c_void_p),
                ("alpha", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("dtype", ctypes.c_int32), ("ref_grid_m", ctypes.c_int32),
                ("head", ctypes.POINTER(GsHead))]


class GsView(ctypes.Structure):
    _fields_ = [("lr_h", ctypes.c_int32), ("lr_w", ctypes.c_int32),
                ("out_h", ctypes.c_int32), ("out_w", ctypes.c_int32),
                ("scale", ctypes.c_float), ("trunc_k", ctypes.c_float),
                ("norm", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("batch", ctypes.c_int32), ("window", ctypes.c_int32),
                ("align", ctypes.c_int32), ("adjoint", ctypes.c_int32),
                ("binning", ctypes.c_int32), ("row0", ctypes.c_int32),
                ("raster", ctypes.c_int32)]


class GsStats(ctypes.Structure):
    _fields_ = [("tile_pairs", ctypes.c_int64), ("pixel_pairs", ctypes.c_int64),
                ("capacity", ctypes.c_int64), ("n_gaussians", ctypes.c_int64),
                ("n_tiles", ctypes.c_int32), ("status", ctypes.c_int32),
                ("raster", ctypes.c_int32), ("adjoint", ctypes.c_int32)]


class GsPeaks(ctypes.Structure):
    _fields_ = [("ffma_per_s", ctypes.c_double), ("ffma2_lane_ops_per_s", ctypes.c_double),
                ("ex2_per_s", ctypes.c_double), ("fwd_pairs_scalar_per_s", ctypes.c_double),
                ("fwd_pairs_packed_per_s", ctypes.c_double), ("sm_count", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class GsTuning(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32), ("batch", ctypes.c_int32), ("binning", ctypes.c_int32),
                ("adjoint", ctypes.c_int32), ("ms", ctypes.c_float), ("from_cache", ctypes.c_int32),
                ("n_timed", ctypes.c_int32), ("raster", ctypes.c_int32)]


class GsError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        super().__init__(f"{where}: {_STATUS_NAMES.get(status, status)}: {msg}")


_STATUS_NAMES = {0: "GS_OK", 1: "GS_ERR_INVALID", 2: "GS_ERR_CAPACITY", 3: "GS_ERR_CUDA",
                 4: "GS_ERR_UNSUPPORTED", 5: "GS_ERR_TIMEOUT", 6: "GS_ERR_INTERNAL"}

_lib = None
_lock = threading.Lock()


def load(path: str | None = None):
    """Load libgs.so (built by paper_2501_06838_gb300.build.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: build it first with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(p)
        G, V = ctypes.POINTER(GsGaussians), ctypes.POINTER(GsView)
        vp, sz, i32, i64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32, ctypes.c_int64
        fpp = ctypes.POINTER(ctypes.c_void_p)
        sig = {
            "gs_workspace_size": (sz, [i32, G, V, i64]),
            "gs_count_pairs": (i32, [i32, G, V, vp, sz, vp, ctypes.POINTER(i64)]),
            "gs_render_fwd": (i32, [G, V, vp, vp, sz, vp]),
            "gs_render_bwd": (i32, [G, V, vp, vp, vp, sz, vp]),
            "gs_render_batched": (i32, [i32, G, V, fpp, vp, sz, vp]),
            "gs_render_batched_bwd": (i32, [i32, G, V, fpp, fpp, vp, sz, vp]),
            "gs_sync_status": (i32, [vp, vp]),
            "gs_read_stats": (i32, [vp, vp, ctypes.POINTER(GsStats)]),
            "gs_last_error": (ctypes.c_char_p, []),
            "gs_status_string": (ctypes.c_char_p, [i32]),
            "gs_launch_count": (i64, []),
            "gs_timing_enable": (i32, [i32]),
            "gs_timing_read": (i32, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64), i32]),
            "gs_timing_release": (i32, []),
            "gs_kernel_name": (ctypes.c_char_p, [i32]),
            "gs_version": (ctypes.c_char_p, []),
            "gs_render_fwd_noalloc": (i32, [G, V, vp, vp]),
            "gs_noalloc_sync_status": (i32, [vp]),
            "gs_probe_peaks": (i32, [vp, sz, vp, ctypes.POINTER(GsPeaks)]),
            "gs_tune": (i32, [i32, G, V, fpp, fpp, fpp, vp, sz, vp, i32, ctypes.c_char_p,
                              ctypes.POINTER(GsTuning)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def last_error() -> str:
    return load().gs_last_error().decode()


def check(status: int, where: str):
    if status != GS_OK:
        raise GsError(status, where, last_error())
