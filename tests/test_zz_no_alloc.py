"""gs_render_fwd_noalloc: the forward render for callers that cannot allocate
device memory (a plugin whose host framework owns all device memory, a
real-time loop that must not call cudaMalloc). Its scratch is a fixed static
array in device memory instead of a caller workspace.

Checked through the C-ABI on calls in a row with different inputs, so that each
call after the first sees the scratch the previous one left behind: every
output must match gs_render_fwd (own workspace) and the FP64 oracle within the
forward parity tolerance (1e-5 normwise per channel), and the device status
the kernels leave in the static array (gs_noalloc_sync_status) must be GS_OK.
The cases cover grid binning (Gaussians on the reference grid) and the sorted
pair list (absolute centres), which lays out four pair arrays, the radix
histograms and the ranges in the same array. Requests too large for the array
are refused, both on the fixed per-Gaussian part and, after the pair count, on
the pairs. This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import gs_synthetic as S
import oracle
from _util import absolute, device_gaussians, normwise

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _structs(dg, v):
    import importlib
    R = importlib.import_module("paper_2501_06838_gb300.render")
    return R._struct_g(dg), R._struct_v(v)


def _reference(dg, v):
    import torch
    import paper_2501_06838_gb300 as gs
    ws = gs.make_workspace([dg], [v])
    out = torch.empty((3, v.out_h, v.out_w), device="cuda")
    gs.render_single_fwd(dg, v, out, ws)
    gs.sync_status(ws)
    return out


def _noalloc(lib, dg, v, stream):
    import torch
    G, V = _structs(dg, v)
    out = torch.full((3, v.out_h, v.out_w), float("nan"), device="cuda")
    st = lib.gs_render_fwd_noalloc(ctypes.byref(G), ctypes.byref(V), out.data_ptr(), stream)
    return st, out


def _absolute_set(seed, lr_h, lr_w, n):
    rng = np.random.default_rng(seed)
    return absolute(np.stack([rng.uniform(-0.5, lr_w - 0.5, n), rng.uniform(-0.5, lr_h - 0.5, n)], 1),
                    np.exp(rng.uniform(np.log(0.3), np.log(2.0), (n, 2))), rng.uniform(-0.9, 0.9, n),
                    rng.uniform(0, 1, (n, 3)), rng.uniform(0, 1, n), lr_h, lr_w)


def test_noalloc_matches_workspace_render_in_a_row():
    import torch
    from paper_2501_06838_gb300 import _abi, build
    build.build()
    lib = _abi.load()
    stream = torch.cuda.current_stream().cuda_stream
    g1, v1 = S.config1()[0][0], S.config1()[1][0]
    g2 = S.draw_gaussians(3, 37, 53, 1, (0.3, 2.0))
    v2 = S.View(37, 53, S.out_size(37, 2.7), S.out_size(53, 2.7), 2.7)
    g3 = _absolute_set(5, 29, 41, 1500)   # absolute centres: the sorted pair list
    v3 = S.View(29, 41, S.out_size(29, 3.4), S.out_size(41, 3.4), 3.4)
    for g, v in ((g1, v1), (g2, v2), (g3, v3), (g2, v2)):
        dg = device_gaussians(g)
        st, out = _noalloc(lib, dg, v, stream)
        assert st == 0, lib.gs_last_error()
        st = lib.gs_noalloc_sync_status(stream)
        assert st == 0, lib.gs_last_error()
        got = out.cpu().double().numpy()
        ref = _reference(dg, v)
        err = normwise(got, ref.cpu().double().numpy(), axis=(1, 2))
        assert np.all(err < TOL), err
        err = normwise(got, oracle.render(g, v), axis=(1, 2))
        assert np.all(err < TOL), err


def test_noalloc_rejects_oversized_request():
    import torch
    from paper_2501_06838_gb300 import _abi
    lib = _abi.load()
    stream = torch.cuda.current_stream().cuda_stream
    # the per-Gaussian part alone is larger than the static array
    g, v = S.config4(8.0, "f32")
    dg = device_gaussians(g[0])
    st, out = _noalloc(lib, dg, v[0], stream)
    assert st == _abi.GS_ERR_UNSUPPORTED
    assert b"before any pair" in lib.gs_last_error()
    # the per-Gaussian part fits, the (tile, Gaussian) pairs do not: untruncated
    # windows put each of 2304 Gaussians into all 8100 tiles of a 1440^2 output
    g = S.config1()[0][0]
    v = S.View(48, 48, 1440, 1440, 30.0, trunc_k=0.0)
    st, out = _noalloc(lib, device_gaussians(g), v, stream)
    assert st == _abi.GS_ERR_UNSUPPORTED
    assert b"pairs need" in lib.gs_last_error()
    assert lib.gs_noalloc_sync_status(stream) == 0, lib.gs_last_error()
    # the array is still usable after a refusal
    g1, v1 = S.config1()[0][0], S.config1()[1][0]
    dg = device_gaussians(g1)
    st, out = _noalloc(lib, dg, v1, stream)
    assert st == 0 and lib.gs_noalloc_sync_status(stream) == 0, lib.gs_last_error()
    err = normwise(out.cpu().double().numpy(), oracle.render(g1, v1), axis=(1, 2))
    assert np.all(err < TOL), err
