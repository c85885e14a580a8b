"""gs_render_fwd_noalloc: the forward render for callers that cannot allocate
device memory (a plugin whose host framework owns all device memory, a
real-time loop that must not call cudaMalloc). Its scratch is a fixed static
array in device memory instead of a caller workspace.

Checked through the C-ABI on two calls in a row with different inputs, so the
second call sees the scratch the first call left behind; each output must
match gs_render_fwd (own workspace) within the forward parity tolerance
(1e-5 normwise per channel). This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import gs_synthetic as S
from _util import device_gaussians, normwise

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


def test_noalloc_matches_workspace_render_twice():
    import torch
    from paper_2501_06838_gb300 import _abi, build
    build.build()
    lib = _abi.load()
    stream = torch.cuda.current_stream().cuda_stream
    g1, v1 = S.config1()[0][0], S.config1()[1][0]
    g2 = S.draw_gaussians(3, 37, 53, 1, (0.3, 2.0))
    v2 = S.View(37, 53, S.out_size(37, 2.7), S.out_size(53, 2.7), 2.7)
    for g, v in ((g1, v1), (g2, v2)):
        dg = device_gaussians(g)
        st, out = _noalloc(lib, dg, v, stream)
        assert st == 0, lib.gs_last_error()
        torch.cuda.synchronize()
        ref = _reference(dg, v)
        err = normwise(out.cpu().double().numpy(), ref.cpu().double().numpy(), axis=(1, 2))
        assert np.all(err < TOL), err


def test_noalloc_rejects_oversized_request():
    import torch
    from paper_2501_06838_gb300 import _abi
    lib = _abi.load()
    stream = torch.cuda.current_stream().cuda_stream
    g, v = S.config4(8.0, "f32")
    dg = device_gaussians(g[0])
    st, out = _noalloc(lib, dg, v[0], stream)
    assert st == _abi.GS_ERR_UNSUPPORTED
    assert b"static scratch holds" in lib.gs_last_error()
