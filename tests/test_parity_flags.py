"""GPU vs the FP64 oracle for the window and alignment variants of the render:
Algorithm 1's ratio window (|x - s mu| < s r W per axis, rasterization ratio r,
Sec. 3.1 "Fast Rasterization") and the half-pixel sampling (x + 1/2)/s - 1/2
of Eq. 4. Same tolerances as the default path: 1e-5 normwise per channel or
per gradient field; windows and pair counts bit-exact.
"""
import numpy as np
import pytest

import gs_synthetic as S
import oracle
from _util import absolute, device_gaussians, normwise

pytestmark = pytest.mark.gpu
TOL = 1e-5
FIELDS = ("o_x", "o_y", "sigma_x", "sigma_y", "rho", "r", "g", "b", "alpha")


def _ragged(window, k, align, norm=S.NORM_DENSITY):
    g = S.draw_gaussians(3, 37, 53, 1, (0.3, 2.0))
    s = 2.7
    v = S.View(37, 53, S.out_size(37, s), S.out_size(53, s), s, trunc_k=k, norm=norm,
               window=window, align=align)
    return g, v


CASES = [(S.WINDOW_RATIO, 0.02, S.ALIGN_EQ4), (S.WINDOW_RATIO, 0.1, S.ALIGN_EQ4),
         (S.WINDOW_RATIO, 0.05, S.ALIGN_HALF), (S.WINDOW_SIGMA, 3.0, S.ALIGN_HALF),
         (S.WINDOW_SIGMA, 0.0, S.ALIGN_HALF)]


@pytest.mark.parametrize("tile", [8, 16, 32])
@pytest.mark.parametrize("window,k,align", CASES)
def test_forward(window, k, align, tile):
    import paper_2501_06838_gb300 as gs
    g, v = _ragged(window, k, align)
    out, ws = gs.render(device_gaussians(g), v, tile=tile, check=True)
    ref = oracle.render(g, v)
    assert np.all(normwise(out.cpu().double().numpy(), ref, axis=(1, 2)) < TOL)
    r = oracle.rects(g, v)
    area = ((r[:, 1] - r[:, 0] + 1).clip(0) * (r[:, 3] - r[:, 2] + 1).clip(0))
    assert gs.read_stats(ws)["pixel_pairs"] == int(area.sum())


@pytest.mark.parametrize("window,k,align", CASES[1:4])
@pytest.mark.parametrize("norm", [S.NORM_DENSITY, S.NORM_PEAK])
def test_adjoint(window, k, align, norm):
    import torch
    import paper_2501_06838_gb300 as gs
    g, v = _ragged(window, k, align, norm)
    go = S.grad_out(4, v.out_h, v.out_w)
    dg = device_gaussians(g)
    _, ws = gs.render(dg, v, check=True)
    gr = gs.render_bwd(dg, v, torch.from_numpy(go.astype(np.float32)).cuda(), ws, check=True)
    err = normwise(gr.cpu().double().numpy(), oracle.adjoint(g, v, go), axis=0)
    assert np.all(err < TOL), dict(zip(FIELDS, err))


@pytest.mark.parametrize("window,k", [(S.WINDOW_RATIO, 0.07), (S.WINDOW_SIGMA, 3.0)])
@pytest.mark.parametrize("align", [S.ALIGN_EQ4, S.ALIGN_HALF])
def test_windows_bit_exact(window, k, align):
    """A lone Gaussian lights exactly the pixels of the oracle's integer window."""
    import paper_2501_06838_gb300 as gs
    rng = np.random.default_rng(22 + align)
    for _ in range(30):
        s = float(np.float32(rng.uniform(1.0, 12.0)))
        mu = rng.uniform(0, 8, (1, 2))
        g = absolute(mu, rng.uniform(0.2, 2.0, (1, 2)), rng.uniform(-0.9, 0.9, 1), np.ones((1, 3)),
                     np.ones(1), 8, 8)
        v = S.View(8, 8, S.out_size(8, s), S.out_size(8, s), s, trunc_k=k, norm=S.NORM_PEAK,
                   window=window, align=align)
        out, ws = gs.render(device_gaussians(g), v, check=True)
        r = oracle.rects(g, v)[0]
        lit = out.cpu().numpy()[0] > 0
        mask = np.zeros_like(lit)
        if r[0] <= r[1] and r[2] <= r[3]:
            mask[r[2]:r[3] + 1, r[0]:r[1] + 1] = True
        assert not np.any(lit & ~mask)
        area = max(0, r[1] - r[0] + 1) * max(0, r[3] - r[2] + 1)
        assert gs.read_stats(ws)["pixel_pairs"] == area


def test_batched_mixed_flags():
    """One batched launch chain over images that each pick their own window,
    alignment and normalisation."""
    import torch
    import paper_2501_06838_gb300 as gs
    specs = [(S.WINDOW_SIGMA, 3.0, S.ALIGN_EQ4, S.NORM_DENSITY, 2.7),
             (S.WINDOW_RATIO, 0.06, S.ALIGN_HALF, S.NORM_PEAK, 3.5),
             (S.WINDOW_SIGMA, 3.0, S.ALIGN_HALF, S.NORM_DENSITY, 1.5),
             (S.WINDOW_RATIO, 0.03, S.ALIGN_EQ4, S.NORM_DENSITY, 4.0)]
    gsets, views = [], []
    for i, (w, k, a, nm, s) in enumerate(specs):
        h, wd = 20 + 3 * i, 26 - 2 * i
        gsets.append(S.draw_gaussians(40 + i, h, wd, 1, (0.3, 2.0)))
        views.append(S.View(h, wd, S.out_size(h, s), S.out_size(wd, s), s, trunc_k=k, norm=nm,
                            window=w, align=a))
    dgs = [device_gaussians(g) for g in gsets]
    ws = gs.make_workspace(dgs, views)
    outs = [torch.empty((3, v.out_h, v.out_w), device="cuda") for v in views]
    gs.render_batched(dgs, views, outs, ws)
    gos = [S.grad_out(50 + i, v.out_h, v.out_w) for i, v in enumerate(views)]
    grads = [torch.empty((g.n, 9), device="cuda") for g in gsets]
    gs.render_batched_bwd(dgs, views, [torch.from_numpy(x.astype(np.float32)).cuda() for x in gos],
                          ws, grads=grads)
    gs.sync_status(ws)
    for g, v, o, go, gr in zip(gsets, views, outs, gos, grads):
        assert np.all(normwise(o.cpu().double().numpy(), oracle.render(g, v), axis=(1, 2)) < TOL)
        err = normwise(gr.cpu().double().numpy(), oracle.adjoint(g, v, go), axis=0)
        assert np.all(err < TOL), dict(zip(FIELDS, err))
