"""GPU forward vs the FP64 oracle (Eq. 4 with the Algorithm-1 window).

Tolerance: 1e-5 normwise per channel, max|gpu - oracle| / max|oracle| (FP32
parameters; the forward sums non-negative terms, so the float32 error is a few
ulp of the pixel value times the number of contributors, far below 1e-5).
"""
import numpy as np
import pytest

import gs_synthetic as S
import oracle
from _util import absolute, device_gaussians, normwise, view_with

pytestmark = pytest.mark.gpu
TOL = 1e-5


def gpu_render(g, v, tile=0, batch=0):
    import paper_2501_06838_gb300 as gs
    out, ws = gs.render(device_gaussians(g), v, tile=tile, batch=batch, check=True)
    return out.cpu().double().numpy(), ws


@pytest.mark.parametrize("tile", [8, 16, 32])
@pytest.mark.parametrize("norm", [S.NORM_DENSITY, S.NORM_PEAK])
def test_config1(tile, norm):
    gset, views = S.config1()
    g, v = gset[0], view_with(views[0], norm=norm)
    out, _ = gpu_render(g, v, tile=tile)
    ref = oracle.render(g, v)
    assert np.all(normwise(out, ref, axis=(1, 2)) < TOL)


@pytest.mark.parametrize("tile,batch", [(8, 32), (8, 64), (16, 32), (16, 64), (32, 64), (32, 128)])
def test_ragged_noninteger_scale(tile, batch):
    """LR 37x53 at s = 2.7: partial tiles on both edges, several smem batches."""
    g = S.draw_gaussians(3, 37, 53, 1, (0.3, 2.0))
    s = 2.7
    v = S.View(37, 53, S.out_size(37, s), S.out_size(53, s), s)
    out, _ = gpu_render(g, v, tile=tile, batch=batch)
    ref = oracle.render(g, v)
    assert np.all(normwise(out, ref, axis=(1, 2)) < TOL)


@pytest.mark.parametrize("m", [4, 9, 16])
def test_reference_grids(m):
    g = S.draw_gaussians(4, 20, 24, m, (0.2, 1.5))
    v = S.View(20, 24, 61, 73, 3.05)
    out, _ = gpu_render(g, v)
    ref = oracle.render(g, v)
    assert np.all(normwise(out, ref, axis=(1, 2)) < TOL)


def test_absolute_centres_off_image():
    """Absolute centres, some outside the image, some so far out their window is empty."""
    rng = np.random.default_rng(9)
    n = 500
    mu = np.stack([rng.uniform(-6, 36, n), rng.uniform(-6, 26, n)], 1)
    mu[:10] += 1000.0
    g = absolute(mu, rng.uniform(0.3, 2.5, (n, 2)), rng.uniform(-0.95, 0.95, n),
                 rng.uniform(0, 1, (n, 3)), rng.uniform(0, 1, n), 20, 30)
    v = S.View(20, 30, 50, 75, 2.5)
    out, _ = gpu_render(g, v)
    ref = oracle.render(g, v)
    assert np.all(normwise(out, ref, axis=(1, 2)) < TOL)


def test_untruncated():
    g = S.draw_gaussians(5, 12, 10, 1, (0.3, 2.0))
    v = S.View(12, 10, 42, 35, 3.5, trunc_k=0.0)
    out, _ = gpu_render(g, v)
    ref = oracle.render(g, v)
    assert np.all(normwise(out, ref, axis=(1, 2)) < TOL)


def test_high_correlation_and_tiny_sigma():
    rng = np.random.default_rng(12)
    n = 300
    mu = np.stack([rng.uniform(0, 16, n), rng.uniform(0, 16, n)], 1)
    sig = rng.uniform(0.05, 3.0, (n, 2))
    rho = rng.choice([-0.999, -0.99, 0.0, 0.99, 0.999], n)
    g = absolute(mu, sig, rho, rng.uniform(0, 1, (n, 3)), rng.uniform(0, 1, n), 16, 16)
    v = S.View(16, 16, 64, 64, 4.0)
    out, _ = gpu_render(g, v)
    ref = oracle.render(g, v)
    assert np.all(normwise(out, ref, axis=(1, 2)) < TOL)


def test_empty_and_single_pixel():
    import paper_2501_06838_gb300 as gs
    # no Gaussians at all -> zeros
    e = S.GaussianSet(np.zeros((0, 2)), np.ones((0, 2)), np.zeros(0), np.zeros((0, 3)),
                      np.zeros(0), 4, 4, 0)
    out, ws = gpu_render(e, S.View(4, 4, 9, 7, 2.0))
    assert out.shape == (3, 9, 7) and np.all(out == 0)
    assert gs.read_stats(ws)["tile_pairs"] == 0
    # a 1x1 output
    g = S.draw_gaussians(6, 1, 1, 1, (0.3, 2.0))
    v = S.View(1, 1, 1, 1, 1.0)
    out, _ = gpu_render(g, v)
    np.testing.assert_allclose(out, oracle.render(g, v), rtol=TOL, atol=0)
    # every Gaussian off-image -> zeros, zero pairs
    rng = np.random.default_rng(1)
    far = absolute(rng.uniform(100, 200, (50, 2)), np.ones((50, 2)), np.zeros(50),
                   np.ones((50, 3)), np.ones(50), 8, 8)
    out, ws = gpu_render(far, S.View(8, 8, 16, 16, 2.0))
    assert np.all(out == 0) and gs.read_stats(ws)["tile_pairs"] == 0


def test_config2_forward_and_stats():
    import paper_2501_06838_gb300 as gs
    gset, views = S.config2()
    g, v = gset[0], views[0]
    out, ws = gpu_render(g, v)
    ref = oracle.render(g, v)
    assert np.all(normwise(out, ref, axis=(1, 2)) < TOL)
    st = gs.read_stats(ws)
    rects = oracle.rects(g, v)
    area = ((rects[:, 1] - rects[:, 0] + 1).clip(0) * (rects[:, 3] - rects[:, 2] + 1).clip(0))
    assert st["pixel_pairs"] == int(area.sum())          # integer windows: bit-exact
    assert st["status"] == 0


def test_windows_bit_exact():
    """Every Gaussian's integer window equals the oracle's, seen through the
    pixels a lone Gaussian lights up (exact integer decision, Algorithm 1)."""
    import paper_2501_06838_gb300 as gs
    rng = np.random.default_rng(21)
    for trial in range(30):
        s = float(np.float32(rng.uniform(1.0, 12.0)))
        mu = rng.uniform(0, 8, (1, 2))
        g = absolute(mu, rng.uniform(0.2, 2.0, (1, 2)), rng.uniform(-0.9, 0.9, 1), np.ones((1, 3)),
                     np.ones(1), 8, 8)
        v = S.View(8, 8, S.out_size(8, s), S.out_size(8, s), s, norm=S.NORM_PEAK)
        out, _ = gpu_render(g, v)
        r = oracle.rects(g, v)[0]
        lit = out[0] > 0
        mask = np.zeros_like(lit)
        if r[0] <= r[1] and r[2] <= r[3]:
            mask[r[2]:r[3] + 1, r[0]:r[1] + 1] = True
        # pixels inside the window can underflow to 0 only far out in the tails
        assert not np.any(lit & ~mask)
        ref = oracle.render(g, v)
        assert np.array_equal(ref[0] > 0, mask) or np.all(ref[0][mask & ~lit] < 1e-30)
