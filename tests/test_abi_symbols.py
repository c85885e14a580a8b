"""The C-ABI library builds, loads without a GPU and exports every function
include/gs.h declares; host-only entry points behave (no CUDA call made)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(gs_[a-z_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2501_06838_gb300 import build, _abi
    build.build()
    return _abi.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    from paper_2501_06838_gb300 import _abi
    assert set(_abi.EXPORTS) == set(names)


def test_host_only_entry_points(lib):
    from paper_2501_06838_gb300 import _abi
    assert lib.gs_status_string(2) == b"GS_ERR_CAPACITY"
    assert lib.gs_version().startswith(b"gs ")
    assert lib.gs_kernel_name(9) == b"raster_fwd"
    G = (_abi.GsGaussians * 1)(_abi.GsGaussians(1, 1, 1, 1, 1, 2304, 0, 1, None))
    V = (_abi.GsView * 1)(_abi.GsView(48, 48, 192, 192, 4.0, 3.0, 0, 16, 64, 0, 0, 0,
                                      _abi.GS_BINNING_SORT, 0))
    a = lib.gs_workspace_size(1, G, V, 0)
    b = lib.gs_workspace_size(1, G, V, 100000)
    assert 0 < a < b
    # 4 u32 arrays per pair plus the radix histograms
    assert b - a >= 16 * 100000
    # grid binning keeps one pair array (the per-tile lists) and no sort buffers
    V[0].binning = _abi.GS_BINNING_GRID
    ga, gb = lib.gs_workspace_size(1, G, V, 0), lib.gs_workspace_size(1, G, V, 100000)
    assert 4 * 100000 <= gb - ga < b - a
    V[0].binning = _abi.GS_BINNING_SORT
    # invalid requests return 0 with a message
    V[0].tile = 12
    assert lib.gs_workspace_size(1, G, V, 0) == 0
    assert b"tile" in lib.gs_last_error()
    V[0].tile = 16
    G[0].n = 2303
    assert lib.gs_workspace_size(1, G, V, 0) == 0
    assert b"m * lr_h" in lib.gs_last_error()
    G[0].n = 2304
    V[0].out_h = 194
    assert lib.gs_workspace_size(1, G, V, 0) == 0
    V[0].out_h = 193
    assert lib.gs_workspace_size(1, G, V, 0) > 0
    # a row band: rows row0 .. row0 + out_h - 1 must lie within floor(s * lr_h) + 1
    V[0].out_h, V[0].row0 = 64, 100
    assert lib.gs_workspace_size(1, G, V, 0) > 0
    V[0].row0 = 130
    assert lib.gs_workspace_size(1, G, V, 0) == 0
    assert b"larger than" in lib.gs_last_error()
    V[0].row0 = -1
    assert lib.gs_workspace_size(1, G, V, 0) == 0
    assert b"row0" in lib.gs_last_error()
    V[0].out_h, V[0].row0 = 192, 0
    V[0].scale = float("nan")
    assert lib.gs_workspace_size(1, G, V, 0) == 0
    assert lib.gs_launch_count() == 0
