"""Grid-implicit binning against the sorted pair list.

With centres on the reference grid (mu = p + o, Sec. 3.2) a tile can find its
Gaussians by enumerating LR cells within the per-image reach of the windows
and testing each window; the sorted list finds them by a radix sort of every
(tile, Gaussian) pair. Both must hand each tile the same Gaussians in the same
order: the forward is compared bit for bit, the adjoint against the oracle,
the pair counts exactly.
"""
import numpy as np
import pytest

import gs_synthetic as S
import oracle
from _util import absolute, device_gaussians, normwise

pytestmark = pytest.mark.gpu
SORT, GRID = 1, 2
FIELDS = ("o_x", "o_y", "sigma_x", "sigma_y", "rho", "r", "g", "b", "alpha")


def _run(g, v, binning, tile=0, batch=0, go=None):
    import torch
    import paper_2501_06838_gb300 as gs
    v.binning = binning
    dg = device_gaussians(g)
    out, ws = gs.render(dg, v, tile=tile, batch=batch, check=True)
    st = gs.read_stats(ws)
    gr = None
    if go is not None:
        gr = gs.render_bwd(dg, v, torch.from_numpy(go.astype(np.float32)).cuda(), ws, tile=tile,
                           batch=batch, check=True).cpu().double().numpy()
    return out.cpu().numpy(), st, gr


CASES = {
    "c1": lambda: (S.config1()[0][0], S.config1()[1][0]),
    "ragged": lambda: (S.draw_gaussians(3, 37, 53, 1, (0.3, 2.0)),
                       S.View(37, 53, S.out_size(37, 2.7), S.out_size(53, 2.7), 2.7)),
    "m4_wide": lambda: (S.draw_gaussians(8, 16, 20, 4, (0.2, 3.0)),
                        S.View(16, 20, S.out_size(16, 9.5), S.out_size(20, 9.5), 9.5)),
    "m9": lambda: (S.draw_gaussians(4, 20, 24, 9, (0.2, 1.5)), S.View(20, 24, 61, 73, 3.05)),
    "m16_ratio": lambda: (S.draw_gaussians(6, 12, 14, 16, (0.2, 3.0)),
                          S.View(12, 14, 48, 56, 4.0, trunc_k=0.1, window=S.WINDOW_RATIO)),
    "half_pixel": lambda: (S.draw_gaussians(7, 18, 22, 1, (0.3, 2.0)),
                           S.View(18, 22, 59, 72, 3.3, align=S.ALIGN_HALF)),
    "untruncated": lambda: (S.draw_gaussians(5, 12, 10, 1, (0.3, 2.0)),
                            S.View(12, 10, 42, 35, 3.5, trunc_k=0.0)),
    "scale_below_one": lambda: (S.draw_gaussians(9, 40, 30, 1, (0.3, 2.0)),
                                S.View(40, 30, S.out_size(40, 0.6), S.out_size(30, 0.6), 0.6)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_grid_equals_sort(case):
    g, v = CASES[case]()
    go = S.grad_out(13, v.out_h, v.out_w)
    a, sa, ga = _run(g, v, SORT, go=go)
    b, sb, gb = _run(g, v, GRID, go=go)
    assert np.array_equal(a, b)
    assert sa["tile_pairs"] == sb["tile_pairs"] and sa["pixel_pairs"] == sb["pixel_pairs"]
    ref = oracle.adjoint(g, v, go)
    for gr in (ga, gb):
        err = normwise(gr, ref, axis=0)
        assert np.all(err < 1e-5), dict(zip(FIELDS, err))


@pytest.mark.parametrize("tile,batch", [(8, 32), (8, 64), (16, 64), (32, 64), (32, 128)])
def test_grid_launch_shapes(tile, batch):
    g, v = CASES["ragged"]()
    go = S.grad_out(14, v.out_h, v.out_w)
    a, _, _ = _run(g, v, SORT, tile, batch)
    b, _, gb = _run(g, v, GRID, tile, batch, go=go)
    assert np.array_equal(a, b)
    err = normwise(gb, oracle.adjoint(g, v, go), axis=0)
    assert np.all(err < 1e-5), dict(zip(FIELDS, err))


def test_grid_batched_uneven():
    import torch
    import paper_2501_06838_gb300 as gs
    gsets, views = [], []
    for i, (h, w, s, m) in enumerate([(20, 26, 2.7, 1), (17, 23, 3.1, 4), (24, 16, 1.5, 1),
                                      (9, 31, 6.25, 16), (5, 5, 11.0, 1)]):
        gsets.append(S.draw_gaussians(80 + i, h, w, m, (0.3, 2.0)))
        views.append(S.View(h, w, S.out_size(h, s), S.out_size(w, s), s))
    dgs = [device_gaussians(g) for g in gsets]
    outs = {}
    for mode in (SORT, GRID):
        for v in views:
            v.binning = mode
        o, ws = gs.render_batched(dgs, views, check=True)
        outs[mode] = [x.cpu().numpy() for x in o]
    for a, b, g, v in zip(outs[SORT], outs[GRID], gsets, views):
        assert np.array_equal(a, b)
        assert np.all(normwise(b.astype(np.float64), oracle.render(g, v), axis=(1, 2)) < 1e-5)


def test_grid_needs_reference_grid():
    import paper_2501_06838_gb300 as gs
    from paper_2501_06838_gb300 import _abi
    rng = np.random.default_rng(3)
    n = 50
    g = absolute(rng.uniform(0, 10, (n, 2)), rng.uniform(0.3, 2, (n, 2)), rng.uniform(-0.9, 0.9, n),
                 rng.uniform(0, 1, (n, 3)), rng.uniform(0, 1, n), 10, 10)
    v = S.View(10, 10, 30, 30, 3.0)
    v.binning = GRID
    with pytest.raises(_abi.GsError) as e:
        gs.render(device_gaussians(g), v, check=True)
    assert "grid binning needs every image on a reference grid" in str(e.value)
    v.binning = 0   # AUTO falls back to the sorted list
    out, _ = gs.render(device_gaussians(g), v, check=True)
    assert np.all(normwise(out.cpu().double().numpy(), oracle.render(g, v), axis=(1, 2)) < 1e-5)


def test_grid_cuda_graph_replay():
    import torch
    import importlib
    R = importlib.import_module("paper_2501_06838_gb300.render")
    gset, views = S.config2()
    v = views[0]
    v.binning = GRID
    plan = R.Plan([device_gaussians(gset[0])], [v])
    plan.grad_outs[0].copy_(torch.from_numpy(S.grad_out(1, v.out_h, v.out_w).astype(np.float32)))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.fwd(s)
        plan.bwd(s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    ref_out, ref_gr = plan.outs[0].clone(), plan.grads[0].clone()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        plan.fwd(s)
        plan.bwd(s)
    plan.outs[0].zero_()
    graph.replay()
    torch.cuda.synchronize()
    plan.status()
    assert torch.equal(plan.outs[0], ref_out)
    assert torch.allclose(plan.grads[0], ref_gr, rtol=1e-5, atol=1e-6 * ref_gr.abs().max().item())


RASTER_TILE, RASTER_PAIR = 1, 2


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("batch", [0, 64])
def test_pair_raster_equals_tile_raster(case, batch):
    """One warp per horizontal pair of 16 x 16 tiles (grid binning) renders
    each tile with exactly the Gaussians and arithmetic of one warp per tile:
    the images are bit for bit the same, the per-tile lists it leaves give the
    adjoint the oracle's gradients, and the stats report the layout that ran."""
    import torch
    import paper_2501_06838_gb300 as gs
    g, v = CASES[case]()
    go = S.grad_out(15, v.out_h, v.out_w)
    outs = {}
    for raster in (RASTER_TILE, RASTER_PAIR):
        v.binning, v.raster = GRID, raster
        dg = device_gaussians(g)
        out, ws = gs.render(dg, v, tile=16, batch=batch, check=True)
        assert gs.read_stats(ws)["raster"] == raster
        gr = gs.render_bwd(dg, v, torch.from_numpy(go).cuda(), ws, tile=16, batch=batch,
                           check=True).cpu().double().numpy()
        outs[raster] = out.cpu().numpy()
        err = normwise(gr, oracle.adjoint(g, v, go), axis=0)
        assert np.all(err < 1e-5), (raster, dict(zip(FIELDS, err)))
    assert np.array_equal(outs[RASTER_TILE], outs[RASTER_PAIR])


def test_pair_raster_batched_bands_and_auto():
    """Pairs over an uneven batch (odd tile columns leave a last tile alone in
    its pair), row bands of one image, and the AUTO choice (pairs only for
    3-sigma windows at scale >= 6)."""
    import paper_2501_06838_gb300 as gs
    gsets, views = [], []
    for i, (h, w, s) in enumerate([(20, 26, 2.7), (17, 23, 6.5), (9, 31, 12.0), (5, 5, 11.0)]):
        gsets.append(S.draw_gaussians(90 + i, h, w, 1, (0.3, 2.0)))
        views.append(S.View(h, w, S.out_size(h, s), S.out_size(w, s), s))
    dgs = [device_gaussians(g) for g in gsets]
    res = {}
    for raster in (RASTER_TILE, RASTER_PAIR, 0):
        for v in views:
            v.binning, v.raster = GRID, raster
        o, ws = gs.render_batched(dgs, views, check=True)
        res[raster] = ([x.cpu().numpy() for x in o], gs.read_stats(ws)["raster"])
    assert res[0][1] == RASTER_PAIR   # a scale >= 6 with 3-sigma windows
    for a, b, c in zip(res[RASTER_TILE][0], res[RASTER_PAIR][0], res[0][0]):
        assert np.array_equal(a, b) and np.array_equal(a, c)
    for x, g, v in zip(res[RASTER_PAIR][0], gsets, views):
        assert np.all(normwise(x.astype(np.float64), oracle.render(g, v), axis=(1, 2)) < 1e-5)
    # a band of one image, rows 32 .. 79, against the whole image's rows
    g, v = gsets[2], views[2]
    v.raster = RASTER_PAIR
    whole, _ = gs.render(dgs[2], v, check=True)
    band = S.View(v.lr_h, v.lr_w, 48, v.out_w, v.scale)
    band.row0, band.binning, band.raster = 32, GRID, RASTER_PAIR
    ob, _ = gs.render(dgs[2], band, check=True)
    assert np.array_equal(ob.cpu().numpy(), whole.cpu().numpy()[:, 32:80])
    # AUTO keeps one warp per tile at small scales
    v0 = views[0]
    v0.raster = 0
    _, ws = gs.render(dgs[0], v0, check=True)
    assert gs.read_stats(ws)["raster"] == RASTER_TILE
