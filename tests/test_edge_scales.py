"""Edge cases of the scale factor and of the output size, against the FP64
oracle: the paper's out-of-distribution scales (x16, x24, x30, Sec. 4.2), the
identity scale s = 1 (Eq. 4 reduces to Eq. 3 on the LR grid), Algorithm 1's
ratio window wide enough that every Gaussian reaches every pixel of a small
image (r = 2: s r W = 33 HR pixels against a 16-pixel-wide output),
and the largest width grid binning takes (32767 HR pixels: windows are kept
as 16-bit integers) next to one pixel more, where AUTO binning falls back to
the sorted list and an explicit GRID request is refused.
"""
import numpy as np
import pytest

import gs_synthetic as S
import oracle
from _util import device_gaussians, normwise

pytestmark = pytest.mark.gpu
TOL = 1e-5
FIELDS = ("o_x", "o_y", "sigma_x", "sigma_y", "rho", "r", "g", "b", "alpha")


def _fwd_bwd(g, v, go, binning=0):
    import torch
    import paper_2501_06838_gb300 as gs
    v.binning = binning
    dg = device_gaussians(g)
    out, ws = gs.render(dg, v, check=True)
    gr = gs.render_bwd(dg, v, torch.from_numpy(go.astype(np.float32)).cuda(), ws, check=True)
    return out.cpu().double().numpy(), gr.cpu().double().numpy()


@pytest.mark.parametrize("scale", [16.0, 24.0, 30.0])
@pytest.mark.parametrize("window", [S.WINDOW_SIGMA, S.WINDOW_RATIO])
def test_out_of_distribution_scales(scale, window):
    g = S.draw_gaussians(31, 10, 12, 4, (0.2, 3.0))
    k = 3.0 if window == S.WINDOW_SIGMA else 0.1
    v = S.View(10, 12, S.out_size(10, scale), S.out_size(12, scale), scale, trunc_k=k,
               window=window)
    go = S.grad_out(32, v.out_h, v.out_w)
    out, gr = _fwd_bwd(g, v, go)
    assert np.all(normwise(out, oracle.render(g, v), axis=(1, 2)) < TOL)
    err = normwise(gr, oracle.adjoint(g, v, go), axis=0)
    assert np.all(err < TOL), dict(zip(FIELDS, err))


def test_identity_scale():
    g = S.draw_gaussians(33, 23, 31, 1, (0.3, 2.0))
    v = S.View(23, 31, 23, 31, 1.0)
    go = S.grad_out(34, 23, 31)
    out, gr = _fwd_bwd(g, v, go)
    assert np.all(normwise(out, oracle.render(g, v), axis=(1, 2)) < TOL)
    err = normwise(gr, oracle.adjoint(g, v, go), axis=0)
    assert np.all(err < TOL), dict(zip(FIELDS, err))


@pytest.mark.parametrize("binning", [1, 2])
def test_ratio_window_covering_everything(binning):
    g = S.draw_gaussians(35, 6, 5, 4, (0.2, 3.0))
    v = S.View(6, 5, S.out_size(6, 3.3), S.out_size(5, 3.3), 3.3, trunc_k=2.0,
               window=S.WINDOW_RATIO)
    go = S.grad_out(36, v.out_h, v.out_w)
    out, gr = _fwd_bwd(g, v, go, binning)
    r = oracle.rects(g, v)
    # every window is the whole image (clamped)
    assert np.all(r[:, 0] == 0) and np.all(r[:, 1] == v.out_w - 1)
    assert np.all(r[:, 2] == 0) and np.all(r[:, 3] == v.out_h - 1)
    assert np.all(normwise(out, oracle.render(g, v), axis=(1, 2)) < TOL)
    err = normwise(gr, oracle.adjoint(g, v, go), axis=0)
    assert np.all(err < TOL), dict(zip(FIELDS, err))


def test_grid_binning_width_limit():
    import paper_2501_06838_gb300 as gs
    from paper_2501_06838_gb300 import _abi
    g = S.draw_gaussians(37, 2, 8192, 1, (0.3, 0.8))
    s_max = 3.99995    # floor(fl32(s) * 8192) = 32767
    v = S.View(2, 8192, S.out_size(2, s_max), S.out_size(8192, s_max), s_max)
    assert v.out_w == 32767
    go = S.grad_out(38, v.out_h, v.out_w)
    out, gr = _fwd_bwd(g, v, go, binning=2)
    ref = oracle.render(g, v)
    assert np.all(normwise(out, ref, axis=(1, 2)) < TOL)
    err = normwise(gr, oracle.adjoint(g, v, go), axis=0)
    assert np.all(err < TOL), dict(zip(FIELDS, err))
    # the sorted list gives the same image bit for bit
    out_sort, _ = _fwd_bwd(g, v, go, binning=1)
    assert np.array_equal(out, out_sort)
    # one pixel wider: grid binning refused, AUTO takes the sorted list
    v2 = S.View(2, 8192, S.out_size(2, 4.0), S.out_size(8192, 4.0), 4.0)
    assert v2.out_w == 32768
    v2.binning = 2
    with pytest.raises(_abi.GsError):
        gs.render(device_gaussians(g), v2, check=True)
    v2.binning = 0
    out2, _ = gs.render(device_gaussians(g), v2, check=True)
    assert np.all(normwise(out2.cpu().double().numpy(), oracle.render(g, v2), axis=(1, 2)) < TOL)
