"""The seeded synthetic inputs follow their stated recipe (no GPU): shapes,
sizes and Gaussian counts of every workload, parameter ranges and
distributions (log-uniform sigma, uniform offsets, rho, colour and opacity),
float32 (or BF16) representability, determinism per seed, and the expected
algorithmic work: (2k)^2 m E[sigma_x] E[sigma_y] window pixels per HR pixel,
independent of the scale."""
import math

import numpy as np
import pytest

import gs_synthetic as S


def _f32_exact(a):
    return np.array_equal(np.asarray(a, np.float64).astype(np.float32).astype(np.float64), a)


def _check_ranges(g, sig_lo, sig_hi, m):
    half = 0.5 / math.sqrt(m)
    assert np.all(np.abs(g.offset) <= half + 1e-7)
    assert np.all((g.sigma >= sig_lo * (1 - 1e-6)) & (g.sigma <= sig_hi * (1 + 1e-6)))
    assert np.all(np.abs(g.rho) < 0.9 + 1e-6)
    assert np.all((g.rgb >= 0) & (g.rgb <= 1)) and np.all((g.alpha >= 0) & (g.alpha <= 1))
    for a in g.fields():
        assert _f32_exact(a)


def test_config1_and_2_shapes_and_distributions():
    (g1,), (v1,) = S.config1()
    assert (g1.n, v1.out_h, v1.out_w, v1.scale, g1.ref_grid_m) == (2304, 192, 192, 4.0, 1)
    (g2,), (v2,) = S.config2()
    assert (g2.n, v2.lr_h, v2.out_h, v2.out_w) == (65536, 256, 1024, 1024)
    for g in (g1, g2):
        _check_ranges(g, 0.3, 2.0, 1)
    # log-uniform sigma: log sigma has the mean and variance of U[log 0.3, log 2]
    lo, hi = math.log(0.3), math.log(2.0)
    ls = np.log(g2.sigma).ravel()
    n = ls.size
    assert abs(ls.mean() - (lo + hi) / 2) < 4 * (hi - lo) / math.sqrt(12 * n)
    assert abs(ls.var() / ((hi - lo) ** 2 / 12) - 1) < 0.02
    # uniform offsets, rho, colour, opacity: means at the centres of their ranges
    for a, c, w in ((g2.offset, 0.0, 1.0), (g2.rho, 0.0, 1.8), (g2.rgb, 0.5, 1.0),
                    (g2.alpha, 0.5, 1.0)):
        assert abs(a.mean() - c) < 4 * w / math.sqrt(12 * a.size)


def test_config2_expected_work():
    """Window pixels per HR pixel = (2 k s sigma_x)(2 k s sigma_y) summed over the
    Gaussians / HR pixels; its expectation (2k)^2 m E[sigma]^2 with E[sigma] =
    (b - a) / ln(b / a) for log-uniform sigma is 28.9 at k = 3."""
    (g,), (v,) = S.config2()
    k, s = 3.0, v.scale
    per_px = np.sum((2 * k * s * g.sigma[:, 0]) * (2 * k * s * g.sigma[:, 1])) / (v.out_h * v.out_w)
    e_sig = (2.0 - 0.3) / math.log(2.0 / 0.3)
    expect = (2 * k) ** 2 * 1 * e_sig ** 2
    assert abs(expect - 28.9) < 0.05
    assert abs(per_px / expect - 1) < 0.02
    # config 4 (m = 4, sigma in [0.2, 3]): 153.9 per HR pixel at x8 and at x12 alike
    e4 = (2 * k) ** 2 * 4 * ((3.0 - 0.2) / math.log(3.0 / 0.2)) ** 2
    assert abs(e4 - 153.9) < 0.1
    for sc in (8.0, 12.0):
        (g4,), (v4,) = S.config4(sc, "bf16")
        o = g4.originals
        p4 = np.sum((2 * k * sc * o.sigma[:, 0]) * (2 * k * sc * o.sigma[:, 1])) / (v4.out_h * v4.out_w)
        assert abs(p4 / e4 - 1) < 0.01


def test_config3_sizes_and_scales():
    sz = S.config3_sizes()
    assert len(sz) == 16
    for h, w, s in sz:
        assert h % 4 == 0 and w % 4 == 0 and 64 <= w <= 480 and 64 <= h <= 360
        assert 1.5 <= s <= 12.0 and float(np.float32(s)) == s
    gs, vs = S.config3()
    for g, v, (h, w, s) in zip(gs, vs, sz):
        assert g.n == h * w and (v.lr_h, v.lr_w, v.scale) == (h, w, s)
        assert (v.out_h, v.out_w) == (math.floor(s * h), math.floor(s * w))
        _check_ranges(g, 0.3, 2.0, 1)
    assert len({(v.lr_h, v.lr_w) for v in vs}) > 8      # uneven sizes
    hr = sum(v.out_h * v.out_w for v in vs)
    assert 5e6 < hr < 5e8


def test_config3_equal_matches_means():
    sz = S.config3_sizes()
    gs, vs = S.config3_equal()
    assert len({(v.lr_h, v.lr_w, v.scale) for v in vs}) == 1
    v = vs[0]
    assert abs(v.lr_h - np.mean([a for a, _, _ in sz])) <= 2
    assert abs(v.lr_w - np.mean([b for _, b, _ in sz])) <= 2
    assert abs(v.scale - np.mean([c for _, _, c in sz])) < 1e-5


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_config4_low_precision(dtype):
    (g,), (v,) = S.config4(12.0, dtype)
    assert (g.n, v.lr_h, v.lr_w, v.out_h, v.out_w, g.ref_grid_m) == (518400, 270, 480, 3240, 5760, 4)
    assert g.dtype == dtype and g.originals is not None
    o = g.originals
    _check_ranges(o, 0.2, 3.0, 4)
    # the stored values are the originals rounded to the storage type
    for a, b in zip(g.fields(), o.fields()):
        np.testing.assert_array_equal(a, S.storage_round(b, dtype))
    rel = np.abs(g.sigma - o.sigma) / o.sigma
    # unit roundoff: 2^-8 (8 significand bits) and 2^-11 (11)
    assert rel.max() <= (2.0 ** -8 if dtype == "bf16" else 2.0 ** -11) * (1 + 1e-9)
    (g8,), (v8,) = S.config4(8.0, dtype)
    assert (v8.out_h, v8.out_w) == (2160, 3840)


def test_ratio_ablation_and_pipeline_shapes():
    for s, lr, n in ((4.0, 180, 518400), (8.0, 90, 129600)):
        (g,), (v,) = S.ratio_ablation(s, 0.1)
        assert (v.lr_h, v.out_h, g.n, g.ref_grid_m) == (lr, 720, n, 16)
        assert v.window == S.WINDOW_RATIO and abs(v.trunc_k - 0.1) < 1e-7
    for s, lr in ((2, 360), (3, 240), (4, 180), (6, 120), (8, 90), (12, 60)):
        img = S.pipeline_input(s)
        assert img.shape == (3, lr, lr) and img.dtype == np.float32
        assert img.min() >= 0 and img.max() <= 1 and img.std() > 0.02


def test_seeded_and_deterministic():
    a, b = S.draw_gaussians(5, 20, 30, 4), S.draw_gaussians(5, 20, 30, 4)
    c = S.draw_gaussians(6, 20, 30, 4)
    for x, y in zip(a.fields(), b.fields()):
        np.testing.assert_array_equal(x, y)
    assert not np.array_equal(a.sigma, c.sigma)
    np.testing.assert_array_equal(S.grad_out(1, 8, 9), S.grad_out(1, 8, 9))
    x5, h5, s5 = S.config5_batch(3, batch=2)
    y5, k5, t5 = S.config5_batch(3, batch=2)
    assert s5 == t5 and np.array_equal(x5, y5) and all(np.array_equal(p, q) for p, q in zip(h5, k5))
    assert all(h.shape == (3, S.out_size(48, s), S.out_size(48, s)) for h, s in zip(h5, s5))


def test_bf16_rounding_matches_torch():
    """The generators' float32 -> bfloat16 rounding (round to nearest even, on
    the bit pattern) equals torch's conversion on CPU, ties and subnormals
    included; float16 storage is numpy's IEEE conversion."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(8)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-6, 6, 20000),
                        np.float32(1.0) + np.arange(-64, 64) * np.float32(2.0 ** -16),  # ties
                        np.array([0.0, -0.0, 1e-40, -3e-39, 3.0e38, -1.7e38])]).astype(np.float32)
    ours = S.bf16_bits_to_f32(S.round_bf16_bits(x))
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(ours.view(np.uint32), ref.view(np.uint32))
    h = x[np.abs(x) < 65504]   # within float16's range
    np.testing.assert_array_equal(S.storage_round(h.astype(np.float64), "f16"),
                                  h.astype(np.float16).astype(np.float64))
