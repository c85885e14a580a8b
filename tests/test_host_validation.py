"""Every host-side argument rule of the C-ABI, through the host-only entry
point gs_workspace_size (no GPU, no CUDA call): a valid request sizes a
workspace; each single violation returns 0 and leaves a message naming it."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_2501_06838_gb300 import build, _abi
    build.build()
    return _abi.load()


def _request(n_images=1):
    from paper_2501_06838_gb300 import _abi
    G = (_abi.GsGaussians * n_images)(*[_abi.GsGaussians(1, 1, 1, 1, 1, 2304, 0, 1, None)
                                        for _ in range(n_images)])
    V = (_abi.GsView * n_images)(*[_abi.GsView(48, 48, 192, 192, 4.0, 3.0, 0, 16, 64, 0, 0, 0, 0, 0)
                                   for _ in range(n_images)])
    return G, V


def _head(**kw):
    from paper_2501_06838_gb300 import _abi
    h = dict(sigma_lo=0.0, sigma_span=1.0, rho_scale=1.0, offset_scale=1.0, offset_tanh=0)
    h.update(kw)
    hd = _abi.GsHead(h["sigma_lo"], h["sigma_span"], h["rho_scale"], h["offset_scale"],
                     h["offset_tanh"])
    return hd


# (what to change, message fragment)
SINGLE = [
    (lambda G, V: setattr(G[0], "n", -1), b"n < 0"),
    (lambda G, V: setattr(G[0], "dtype", 3), b"unknown dtype"),
    (lambda G, V: setattr(G[0], "ref_grid_m", 2), b"ref_grid_m"),
    (lambda G, V: setattr(V[0], "lr_h", 0), b"sizes must be >= 1"),
    (lambda G, V: setattr(V[0], "out_w", 0), b"sizes must be >= 1"),
    (lambda G, V: setattr(V[0], "scale", 0.0), b"scale"),
    (lambda G, V: setattr(V[0], "scale", -2.0), b"scale"),
    (lambda G, V: setattr(V[0], "scale", float("inf")), b"scale"),
    (lambda G, V: setattr(V[0], "trunc_k", float("nan")), b"trunc_k"),
    (lambda G, V: setattr(V[0], "norm", 2), b"unknown norm"),
    (lambda G, V: setattr(V[0], "window", 2), b"unknown window"),
    (lambda G, V: setattr(V[0], "align", 2), b"unknown align"),
    (lambda G, V: setattr(V[0], "adjoint", 4), b"unknown adjoint"),
    (lambda G, V: setattr(V[0], "adjoint", -1), b"unknown adjoint"),
    (lambda G, V: (setattr(V[0], "adjoint", 3), setattr(V[0], "tile", 8),
                   setattr(V[0], "batch", 0)), b"adjoint QUADRANT needs tile 16"),
    (lambda G, V: (setattr(V[0], "adjoint", 3), setattr(V[0], "tile", 32),
                   setattr(V[0], "batch", 0)), b"adjoint QUADRANT needs tile 16"),
    (lambda G, V: setattr(V[0], "binning", 3), b"unknown binning"),
    (lambda G, V: setattr(V[0], "row0", -4), b"row0"),
    (lambda G, V: setattr(V[0], "out_w", 194), b"larger than"),
    (lambda G, V: setattr(V[0], "tile", 24), b"tile must be"),
    (lambda G, V: setattr(V[0], "batch", 16), b"batch must be"),
    (lambda G, V: setattr(V[0], "batch", 1024), b"batch must be"),
    (lambda G, V: setattr(V[0], "batch", 128), b"batch must be"),
    (lambda G, V: (setattr(V[0], "tile", 32), setattr(V[0], "batch", 32)), b"batch must be"),
    (lambda G, V: (setattr(V[0], "tile", 8), setattr(V[0], "batch", 512)), b"batch must be"),
    (lambda G, V: setattr(V[0], "raster", 3), b"unknown raster"),
    (lambda G, V: (setattr(V[0], "raster", 2), setattr(V[0], "binning", 1)), b"raster PAIR needs"),
    (lambda G, V: (setattr(V[0], "raster", 2), setattr(V[0], "tile", 8),
                   setattr(V[0], "batch", 0)), b"raster PAIR needs"),
    (lambda G, V: setattr(G[0], "n", 2305), b"m * lr_h"),
    (lambda G, V: setattr(G[0], "rgb", None), b"null parameter pointer"),
]


@pytest.mark.parametrize("k", range(len(SINGLE)))
def test_single_rule(lib, k):
    G, V = _request()
    assert lib.gs_workspace_size(1, G, V, 0) > 0
    change, msg = SINGLE[k]
    change(G, V)
    assert lib.gs_workspace_size(1, G, V, 0) == 0
    assert msg in lib.gs_last_error(), lib.gs_last_error()


def test_pair_capacity_range(lib):
    G, V = _request()
    assert lib.gs_workspace_size(1, G, V, (1 << 31) - 1) > 0
    assert lib.gs_workspace_size(1, G, V, 1 << 31) == 0
    assert b"pair_capacity" in lib.gs_last_error()
    assert lib.gs_workspace_size(1, G, V, -1) == 0


def test_call_level_rules(lib):
    G, V = _request()
    assert lib.gs_workspace_size(0, G, V, 0) == 0
    assert b"n_images" in lib.gs_last_error()
    assert lib.gs_workspace_size(1, None, V, 0) == 0
    assert b"null" in lib.gs_last_error()


@pytest.mark.parametrize("field,value", [("tile", 8), ("batch", 32), ("adjoint", 2),
                                         ("binning", 1), ("raster", 1)])
def test_batch_members_must_agree(lib, field, value):
    G, V = _request(2)
    assert lib.gs_workspace_size(2, G, V, 0) > 0
    setattr(V[1], field, value)
    assert lib.gs_workspace_size(2, G, V, 0) == 0
    assert b"image 1" in lib.gs_last_error() and b"differ" in lib.gs_last_error()


def test_uneven_batch_is_valid(lib):
    """Images of different sizes, scales, windows and alignments share one call."""
    G, V = _request(2)
    V[1].lr_h, V[1].lr_w, V[1].scale = 30, 70, 2.5
    V[1].out_h, V[1].out_w = 75, 175
    V[1].window, V[1].trunc_k, V[1].align, V[1].norm = 1, 0.1, 1, 1
    G[1].n, G[1].ref_grid_m = 4 * 30 * 70, 4
    assert lib.gs_workspace_size(2, G, V, 0) > 0


@pytest.mark.parametrize("kw", [dict(sigma_lo=-0.1), dict(sigma_span=0.0),
                                dict(sigma_span=float("inf")), dict(rho_scale=1.5),
                                dict(offset_scale=float("nan")), dict(offset_tanh=2)])
def test_head_rules(lib, kw):
    G, V = _request()
    good = _head()
    G[0].head = ctypes.pointer(good)
    assert lib.gs_workspace_size(1, G, V, 0) > 0
    bad = _head(**kw)
    G[0].head = ctypes.pointer(bad)
    assert lib.gs_workspace_size(1, G, V, 0) == 0
    assert b"invalid head" in lib.gs_last_error()
    bad2 = _head()
    bad2.reserved[1] = 7
    G[0].head = ctypes.pointer(bad2)
    assert lib.gs_workspace_size(1, G, V, 0) == 0
    assert b"reserved 0" in lib.gs_last_error()


def test_grid_binning_needs_a_reference_grid(lib):
    from paper_2501_06838_gb300 import _abi
    G, V = _request()
    V[0].binning = _abi.GS_BINNING_GRID
    assert lib.gs_workspace_size(1, G, V, 0) > 0
    G[0].ref_grid_m = 0          # absolute centres: no grid to enumerate from
    assert lib.gs_workspace_size(1, G, V, 0) == 0
    assert b"grid binning" in lib.gs_last_error()
    V[0].binning = _abi.GS_BINNING_AUTO   # AUTO falls back to the sorted pair list
    assert lib.gs_workspace_size(1, G, V, 0) > 0


def test_half_pixel_scale_limit(lib):
    G, V = _request()
    V[0].align = 1
    V[0].lr_h = V[0].lr_w = 1
    G[0].n = 1
    V[0].out_h = V[0].out_w = 1
    V[0].scale = 2.0 ** 23
    assert lib.gs_workspace_size(1, G, V, 0) == 0
    assert b"2^23" in lib.gs_last_error()
    V[0].scale = 2.0 ** 22
    assert lib.gs_workspace_size(1, G, V, 0) > 0


def test_output_bound_matches_out_size(lib):
    """The library's output bound floor(s * lr) + 1 (s as float32, the product
    exact in double) agrees with the binding's and the generators' out_size for
    drawn scales and sizes: out_size + 1 is accepted, out_size + 2 is not."""
    import importlib

    import numpy as np

    import gs_synthetic as S
    R = importlib.import_module("paper_2501_06838_gb300.render")
    rng = np.random.default_rng(3)
    for _ in range(200):
        lr_h, lr_w = int(rng.integers(1, 400)), int(rng.integers(1, 400))
        s = float(np.float32(rng.uniform(0.05, 30.0)))
        oh, ow = R.out_size(lr_h, s), R.out_size(lr_w, s)
        assert (oh, ow) == (S.out_size(lr_h, s), S.out_size(lr_w, s))
        G, V = _request()
        G[0].n, V[0].lr_h, V[0].lr_w, V[0].scale = lr_h * lr_w, lr_h, lr_w, s
        V[0].out_h, V[0].out_w = oh + 1, ow + 1
        assert lib.gs_workspace_size(1, G, V, 0) > 0, (lr_h, lr_w, s)
        V[0].out_h = oh + 2
        assert lib.gs_workspace_size(1, G, V, 0) == 0, (lr_h, lr_w, s)
