"""The sorted pair list (scan, emit, stable radix sort, tile ranges) at full
size, against the FP64 oracle.

The sorted path is the only binning for absolute centres (ref_grid_m = 0) and
for outputs wider or taller than 32767 px, so it is checked on the full
configurations, not only on the small cases where both binnings run:
  - config 2 (LR 256^2, x4 -> 1024^2, FP32), forward and adjoint, and its image
    bit for bit against grid binning (each tile gets the same Gaussians in the
    same order);
  - config 4 at x8 (LR 480x270, m = 4, N = 518,400, 3840x2160) with BF16
    parameter storage, against the oracle on the same rounded values;
  - a render with more than 2^18 tiles, whose 19-bit tile keys take three radix
    passes of at most 9 bits (tile 8, a 2,097,600 x 8 output).
Tolerance: 1e-5 normwise per channel (image) and per field (adjoint), the
parity bar of the FP32 arithmetic.
"""
import numpy as np
import pytest

import gs_synthetic as S
import oracle
from _util import device_gaussians, normwise

pytestmark = pytest.mark.gpu
TOL = 1e-5
SORT, GRID = 1, 2
FIELDS = ("o_x", "o_y", "sigma_x", "sigma_y", "rho", "r", "g", "b", "alpha")


def _run(g, v, binning, go, tile=0):
    import torch
    import paper_2501_06838_gb300 as gs
    v.binning = binning
    dg = device_gaussians(g)
    out, ws = gs.render(dg, v, tile=tile, check=True)
    stats = gs.read_stats(ws)
    gr = gs.render_bwd(dg, v, torch.from_numpy(go.astype(np.float32)).cuda(), ws, tile=tile,
                       check=True)
    return out.cpu().numpy(), stats, gr.cpu().double().numpy()


def _check(g, v, out, gr, go):
    err = normwise(out.astype(np.float64), oracle.render(g, v), axis=(1, 2))
    assert np.all(err < TOL), err
    err = normwise(gr, oracle.adjoint(g, v, go), axis=0)
    assert np.all(err < TOL), dict(zip(FIELDS, err))


def test_sorted_config2_full():
    gset, views = S.config2()
    g, v = gset[0], views[0]
    go = S.grad_out(1, v.out_h, v.out_w)
    out, st, gr = _run(g, v, SORT, go)
    _check(g, v, out, gr, go)
    out_grid, st_grid, _ = _run(g, v, GRID, go)
    assert np.array_equal(out, out_grid)
    assert st["tile_pairs"] == st_grid["tile_pairs"]
    assert st["pixel_pairs"] == st_grid["pixel_pairs"]


def test_sorted_config4_x8_bf16():
    gset, views = S.config4(8.0, "bf16")
    g, v = gset[0], views[0]
    go = S.grad_out(1, v.out_h, v.out_w)
    out, st, gr = _run(g, v, SORT, go)
    _check(g, v, out, gr, go)


def test_sorted_three_radix_passes():
    import paper_2501_06838_gb300 as gs
    lr_w, s = 262200, 8.0
    g = S.draw_gaussians(41, 1, lr_w, 1, (0.3, 2.0))
    v = S.View(1, lr_w, 8, int(s) * lr_w, s)
    go = S.grad_out(42, v.out_h, v.out_w)
    out, st, gr = _run(g, v, 0, go, tile=8)   # AUTO: wider than 32767 px -> sorted
    tiles = (v.out_w // 8) * 1
    assert st["n_tiles"] == tiles and tiles > 2 ** 18
    assert int(tiles - 1).bit_length() == 19   # three passes of at most 9 bits
    _check(g, v, out, gr, go)
