"""The three adjoint kernels against the FP64 oracle and each other.

TILE sums each Gaussian's moments per screen tile and adds them with atomics;
QUADRANT does the same per 8 x 8 quadrant of 16 x 16 tiles, each quadrant
keeping the Gaussians of its tile's list whose window meets it; GAUSSIAN gives
each Gaussian one warp that walks its own window (Eq. 4's sum over R_i) in a
fixed order, so its gradients are bitwise reproducible. All must meet the
adjoint bar (1e-5 normwise per gradient field, FP32 parameters) on even and
odd output widths (the GAUSSIAN walk loads column pairs as float2 only when
rows are 8-byte aligned; quadrants past the right and bottom edges), narrow
and wide windows, and batches.
"""
import numpy as np
import pytest

import gs_synthetic as S
import oracle
from _util import absolute, device_gaussians, normwise

pytestmark = pytest.mark.gpu
TOL = 1e-5
FIELDS = ("o_x", "o_y", "sigma_x", "sigma_y", "rho", "r", "g", "b", "alpha")
TILE, GAUSSIAN, QUADRANT = 1, 2, 3


def _grads(g, v, go, mode, tile=0):
    import torch
    import paper_2501_06838_gb300 as gs
    v.adjoint = mode
    dg = device_gaussians(g)
    _, ws = gs.render(dg, v, tile=tile, check=True)
    gr = gs.render_bwd(dg, v, torch.from_numpy(go.astype(np.float32)).cuda(), ws, tile=tile,
                       check=True)
    return gr.cpu().double().numpy()


def _check(gr, ref):
    err = normwise(gr, ref, axis=0)
    assert np.all(err < TOL), dict(zip(FIELDS, err))


CASES = {
    "c1": lambda: (S.config1()[0][0], S.config1()[1][0]),
    "ragged_odd_width": lambda: (S.draw_gaussians(3, 37, 53, 1, (0.3, 2.0)),
                                 S.View(37, 53, S.out_size(37, 2.7), S.out_size(53, 2.7), 2.7)),
    "grid_m4_wide": lambda: (S.draw_gaussians(8, 16, 20, 4, (0.2, 3.0)),
                             S.View(16, 20, S.out_size(16, 9.5), S.out_size(20, 9.5), 9.5)),
    "untruncated": lambda: (S.draw_gaussians(5, 12, 10, 1, (0.3, 2.0)),
                            S.View(12, 10, 42, 35, 3.5, trunc_k=0.0)),
    "ratio_window": lambda: (S.draw_gaussians(6, 20, 26, 1, (0.3, 2.0)),
                             S.View(20, 26, 54, 70, 2.7, trunc_k=0.1, window=S.WINDOW_RATIO)),
    "half_pixel_peak": lambda: (S.draw_gaussians(7, 18, 22, 1, (0.3, 2.0)),
                                S.View(18, 22, 59, 72, 3.3, norm=S.NORM_PEAK, align=S.ALIGN_HALF)),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("mode", [TILE, GAUSSIAN, QUADRANT])
def test_modes_vs_oracle(case, mode):
    g, v = CASES[case]()
    go = S.grad_out(11, v.out_h, v.out_w)
    _check(_grads(g, v, go, mode), oracle.adjoint(g, v, go))


@pytest.mark.parametrize("mode", [GAUSSIAN, QUADRANT])
def test_off_image_and_tiny_windows(mode):
    """Absolute centres partly or wholly outside the image, sigmas down to 0.05
    LR px (one- and two-pixel windows: the narrowest lane layouts; 50 rows
    leave the bottom quadrants of the last tile row past the output)."""
    rng = np.random.default_rng(19)
    n = 600
    mu = np.stack([rng.uniform(-6, 36, n), rng.uniform(-6, 26, n)], 1)
    mu[:10] += 1000.0
    g = absolute(mu, rng.uniform(0.05, 2.5, (n, 2)), rng.uniform(-0.95, 0.95, n),
                 rng.uniform(0, 1, (n, 3)), rng.uniform(0, 1, n), 20, 30)
    for W in (75, 76):
        v = S.View(20, 30, 50, W, 2.5)
        go = S.grad_out(12, v.out_h, v.out_w)
        _check(_grads(g, v, go, mode), oracle.adjoint(g, v, go))


def test_gaussian_mode_bitwise_deterministic_and_tile_close():
    gset, views = S.config2()
    g, v = gset[0], views[0]
    go = S.grad_out(1, v.out_h, v.out_w)
    a = _grads(g, v, go, GAUSSIAN)
    b = _grads(g, v, go, GAUSSIAN)
    assert np.array_equal(a, b)
    t = _grads(g, v, go, TILE)
    q = _grads(g, v, go, QUADRANT)
    ref = oracle.adjoint(g, v, go)
    _check(a, ref)
    _check(t, ref)
    _check(q, ref)


@pytest.mark.parametrize("mode", [GAUSSIAN, QUADRANT])
def test_batched_mixed_widths(mode):
    import torch
    import paper_2501_06838_gb300 as gs
    gsets, views = [], []
    for i, (h, w, s) in enumerate([(20, 26, 2.7), (17, 23, 3.1), (24, 16, 1.5), (9, 31, 6.25)]):
        gsets.append(S.draw_gaussians(60 + i, h, w, 1, (0.3, 2.0)))
        v = S.View(h, w, S.out_size(h, s), S.out_size(w, s), s)
        v.adjoint = mode
        views.append(v)
    dgs = [device_gaussians(g) for g in gsets]
    outs, ws = gs.render_batched(dgs, views, check=True)
    gos = [S.grad_out(70 + i, v.out_h, v.out_w) for i, v in enumerate(views)]
    grads = gs.render_batched_bwd(dgs, views, [torch.from_numpy(x.astype(np.float32)).cuda()
                                               for x in gos], ws, check=True)
    for g, v, go, gr in zip(gsets, views, gos, grads):
        _check(gr.cpu().double().numpy(), oracle.adjoint(g, v, go))


def test_mixed_adjoint_modes_rejected():
    import paper_2501_06838_gb300 as gs
    from paper_2501_06838_gb300 import _abi
    g = S.draw_gaussians(1, 8, 8, 1, (0.3, 2.0))
    v1, v2 = S.View(8, 8, 16, 16, 2.0), S.View(8, 8, 16, 16, 2.0)
    v1.adjoint, v2.adjoint = TILE, GAUSSIAN
    dg = device_gaussians(g)
    with pytest.raises(_abi.GsError) as e:
        gs.render_batched([dg, dg], [v1, v2], check=True)
    assert e.value.status == _abi.GS_ERR_INVALID


@pytest.mark.parametrize("tile", [8, 32])
def test_quadrant_needs_tile16(tile):
    import paper_2501_06838_gb300 as gs
    from paper_2501_06838_gb300 import _abi
    g = S.draw_gaussians(1, 8, 8, 1, (0.3, 2.0))
    v = S.View(8, 8, 16, 16, 2.0)
    v.adjoint = QUADRANT
    with pytest.raises(_abi.GsError, match="QUADRANT needs tile 16"):
        gs.render(device_gaussians(g), v, tile=tile, check=True)


def test_quadrant_long_lists_partial_hits():
    """Tiles whose lists run to hundreds of Gaussians, of which each quadrant
    keeps a varying part (the queue refills across many list chunks), and
    the resolved adjoint the forward reports."""
    import paper_2501_06838_gb300 as gs
    g = S.draw_gaussians(23, 24, 30, 4, (0.2, 3.0))
    v = S.View(24, 30, S.out_size(24, 6.5), S.out_size(30, 6.5), 6.5)
    go = S.grad_out(24, v.out_h, v.out_w)
    _check(_grads(g, v, go, QUADRANT), oracle.adjoint(g, v, go))
    v.adjoint = QUADRANT
    _, ws = gs.render(device_gaussians(g), v, check=True)
    st = gs.read_stats(ws)
    assert st["adjoint"] == QUADRANT and st["tile_pairs"] > 64 * st["n_tiles"]


def test_gaussian_mode_blocks_mixed_grids_and_partial_blocks():
    """The Gaussian-warp adjoint in blocks of 8 x 8 LR cells: one batch with
    m = 1, 4 and 9 images whose LR sizes are not multiples of 8 (partial
    blocks at the right and bottom edges), output widths with and without
    16-byte rows; and a batch with an absolute-centre image (m = 0), which
    runs the one-warp-per-Gaussian launch for every image."""
    import torch
    import paper_2501_06838_gb300 as gs
    for ms in ((1, 4, 9), (1, 0)):
        gsets, views = [], []
        for i, m in enumerate(ms):
            h, w, s = 13 + 5 * i, 19 + 3 * i, 3.25 - 0.5 * i
            if m == 0:
                rng = np.random.default_rng(80 + i)
                n = h * w
                mu = np.stack([rng.uniform(0, w, n), rng.uniform(0, h, n)], 1)
                gsets.append(absolute(mu, rng.uniform(0.2, 2.0, (n, 2)), rng.uniform(-0.9, 0.9, n),
                                      rng.uniform(0, 1, (n, 3)), rng.uniform(0, 1, n), h, w))
            else:
                gsets.append(S.draw_gaussians(80 + i, h, w, m, (0.2, 2.0)))
            v = S.View(h, w, S.out_size(h, s), S.out_size(w, s), s)
            v.adjoint = GAUSSIAN
            views.append(v)
        dgs = [device_gaussians(g) for g in gsets]
        _, ws = gs.render_batched(dgs, views, check=True)
        gos = [S.grad_out(90 + i, v.out_h, v.out_w) for i, v in enumerate(views)]
        grads = gs.render_batched_bwd(dgs, views, [torch.from_numpy(x.astype(np.float32)).cuda()
                                                   for x in gos], ws, check=True)
        for g, v, go, gr in zip(gsets, views, gos, grads):
            _check(gr.cpu().double().numpy(), oracle.adjoint(g, v, go))
