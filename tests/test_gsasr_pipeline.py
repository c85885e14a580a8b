"""The whole-pipeline timing model (encoder, Gaussian decoder, heads, render;
Sec. 3.2). Host-side index logic on the CPU: the decoder's token grid maps to
the render's Gaussian order with the oracle's reference positions (m points
per LR pixel at equal intervals, Sec. 3.2), window partition and cyclic shift
invert, the relative position indices depend on the offset alone, and the
padded attention heads and the padded embedding width compute what unpadded
ones do. On the GPU: the
decoder's raw head outputs, rendered by the library with the fused head and
Algorithm 1's ratio window, match the FP64 oracle on the same rounded values.
"""
import math

import numpy as np
import pytest
import torch

import gs_synthetic as S
import oracle

TINY = dict(n_feats=8, n_resblocks=1, k=4, m=16, d=24, heads=2, head_pad=16, blocks=1,
            scale_tokens=2, window_chunk=3)


def test_token_grid_order_matches_reference_positions():
    from paper_2501_06838_gb300.gsasr import gaussian_order
    h, w, m = 5, 7, 16
    r = math.isqrt(m)
    gh, gw = r * h + 4, r * w + 8      # padded grid: the crop must drop the extra tokens
    ty, tx = torch.meshgrid(torch.arange(gh, dtype=torch.float64),
                            torch.arange(gw, dtype=torch.float64), indexing="ij")
    grid = torch.stack([(tx + 0.5) / r - 0.5, (ty + 0.5) / r - 0.5], -1)[None]
    pos = gaussian_order(grid, h, w, m)[0].numpy()
    n = m * h * w
    g = S.GaussianSet(np.zeros((n, 2)), np.ones((n, 2)), np.zeros(n), np.zeros((n, 3)),
                      np.zeros(n), h, w, ref_grid_m=m)
    v = S.View(h, w, 2 * h, 2 * w, 2.0)
    ref = np.stack([oracle.centre(g, v, i) for i in range(n)])
    assert np.array_equal(pos, ref)


def test_window_partition_and_shift_invert():
    from paper_2501_06838_gb300.gsasr import window_partition, window_reverse
    x = torch.randn(2, 12, 18, 5)
    wp = window_partition(x, 6)
    assert wp.shape == (2 * 2 * 3, 36, 5)
    assert torch.equal(window_reverse(wp, 6, 2, 12, 18), x)
    # window (b, wy, wx) holds the rows wy*6.. and columns wx*6.. of image b
    assert torch.equal(wp[1 * 3 + 2].view(6, 6, 5), x[0, 6:12, 12:18])
    sh = torch.roll(x, shifts=(-3, -3), dims=(1, 2))
    back = torch.roll(window_reverse(window_partition(sh, 6), 6, 2, 12, 18), (3, 3), (1, 2))
    assert torch.equal(back, x)


def test_relative_indices_depend_on_offset_only():
    from paper_2501_06838_gb300.gsasr import relative_index_cross, relative_index_self
    w = 6
    idx = relative_index_self(w)
    ys, xs = np.divmod(np.arange(w * w), w)
    off = {}
    for i in range(w * w):
        for j in range(w * w):
            key = (ys[i] - ys[j], xs[i] - xs[j])
            assert off.setdefault(key, int(idx[i, j])) == int(idx[i, j])
    assert len(set(off.values())) == len(off) == (2 * w - 1) ** 2
    assert int(idx.min()) == 0 and int(idx.max()) == (2 * w - 1) ** 2 - 1
    k, r = 3, 4
    ci = relative_index_cross(k, r)
    assert ci.shape == ((r * k) ** 2, k * k)
    ty, tx = np.divmod(np.arange((r * k) ** 2), r * k)
    py, px = np.divmod(np.arange(k * k), k)
    off = {}
    for i in range(ci.shape[0]):
        for j in range(ci.shape[1]):
            # geometric offset (LR pixels) of the Gaussian's reference point from the pixel
            key = ((ty[i] + 0.5) / r - 0.5 - py[j], (tx[i] + 0.5) / r - 0.5 - px[j])
            assert off.setdefault(key, int(ci[i, j])) == int(ci[i, j])
    assert len(set(off.values())) == len(off)
    assert 0 <= int(ci.min()) and int(ci.max()) < (2 * r * k) ** 2


def test_padded_heads_equal_unpadded():
    from paper_2501_06838_gb300.gsasr import _Attention
    torch.manual_seed(3)
    d, heads, hd = 12, 2, 6
    a = _Attention(d, 10, heads, hd)
    b = _Attention(d, 10, heads, 8)
    with torch.no_grad():
        b.q.weight.view(heads, 8, d)[:, :hd] = a.q.weight.view(heads, hd, d)
        b.q.bias.view(heads, 8)[:, :hd] = a.q.bias.view(heads, hd)
        b.kv.weight.view(2 * heads, 8, 10)[:, :hd] = a.kv.weight.view(2 * heads, hd, 10)
        b.kv.bias.view(2 * heads, 8)[:, :hd] = a.kv.bias.view(2 * heads, hd)
        b.proj.weight.view(d, heads, 8)[:, :, :hd] = a.proj.weight.view(d, heads, hd)
        b.proj.bias.copy_(a.proj.bias)
    q, ctx = torch.randn(3, 7, d), torch.randn(3, 5, 10)
    bias = torch.randn(heads, 7, 5)
    assert torch.allclose(a(q, ctx, bias), b(q, ctx, bias), atol=1e-6)
    # and the padded columns stay zero after construction
    assert torch.all(b.q.weight.view(heads, 8, d)[:, hd:] == 0)


def test_tiny_pipeline_cpu_shapes():
    from paper_2501_06838_gb300.gsasr import GSASR, GSASRConfig
    torch.manual_seed(0)
    net = GSASR(GSASRConfig(**TINY))
    lr = torch.rand(2, 3, 6, 10)       # not whole windows: padded to 8 x 12
    with torch.no_grad():
        raw = net(lr, torch.tensor([2.0, 3.5]))
        raw2 = net(lr, torch.tensor([2.0, 3.5]))
    assert raw.shape == (2, 16 * 6 * 10, 9)
    assert torch.isfinite(raw).all() and torch.equal(raw, raw2)
    with pytest.raises(ValueError):
        GSASR(GSASRConfig(m=12))


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 2e-5)])
def test_padded_width_equals_unpadded(dtype, tol):
    """d = 20 held at 24: the extra channels of the residual stream carry the
    mean of the real ones, so the width-24 layer norms (eps and weights scaled)
    equal the width-20 ones; every other extra channel is ignored. The padded
    model, loaded from the unpadded one, computes the same raw outputs."""
    from paper_2501_06838_gb300.gsasr import GSASR, GSASRConfig
    cfg = dict(TINY, d=20, heads=2, head_pad=16)
    torch.manual_seed(4)
    a = GSASR(GSASRConfig(**cfg, pad_width=False)).to(dtype)
    b = GSASR(GSASRConfig(**cfg, pad_width=True)).to(dtype)
    assert a.cfg.d_store == 20 and b.cfg.d_store == 24
    with torch.no_grad():    # random, non-trivial layer-norm weights and biases
        for mod in a.modules():
            if isinstance(mod, torch.nn.LayerNorm):
                mod.weight.uniform_(0.5, 1.5)
                mod.bias.uniform_(-0.3, 0.3)
    b.load_unpadded(a.state_dict())
    lr = torch.rand(2, 3, 6, 10, dtype=dtype)
    sc = torch.tensor([2.0, 3.5])
    with torch.no_grad():
        ra, rb = a(lr, sc), b(lr, sc)
        # the residual stream's extra channels hold the real channels' mean
        x = b.inject(b.e_base, b.encode(lr), 2, 32, 48)
    assert ra.shape == rb.shape
    assert float((ra - rb).abs().max() / ra.abs().max()) < tol
    assert torch.allclose(x[..., 20:], x[..., :20].mean(-1, keepdim=True).expand(-1, -1, -1, 4),
                          atol=tol * float(x.abs().max()) * 10)
    with pytest.raises(ValueError):
        b.load_unpadded({k: v for k, v in list(a.state_dict().items())[1:]})


@pytest.mark.gpu
def test_pipeline_render_matches_oracle():
    """The decoder's BF16 raw outputs through the fused head and the ratio
    window (r = 0.1) against the FP64 oracle on the same values."""
    from _util import normwise
    from paper_2501_06838_gb300.gsasr import GSASR, GSASRConfig, PipelineHead
    torch.manual_seed(1)
    net = GSASR(GSASRConfig(**TINY)).cuda().eval()
    h, w, s = 8, 12, 3.0
    f = S.image_function(5, 12)
    ys, xs = np.mgrid[0:h, 0:w]
    lr = torch.from_numpy(f(xs, ys).astype(np.float32))[None].cuda()
    with torch.no_grad(), torch.autocast("cuda", dtype=torch.bfloat16):
        raw = net(lr, torch.tensor([s], device="cuda"))
    out = net.render(raw, h, w, s)[0]
    assert raw.dtype == torch.bfloat16 and out.shape == (3, 24, 36)
    r = raw[0].float().cpu().numpy().astype(np.float64)
    hd = PipelineHead()
    g = S.GaussianSet(r[:, 0:2], r[:, 2:4], r[:, 4], r[:, 5:8], r[:, 8], h, w, ref_grid_m=16,
                      dtype="bf16", head=S.Head(hd.sigma_lo, hd.sigma_span, hd.rho_scale,
                                                hd.offset_scale, hd.offset_tanh))
    v = S.View(h, w, 24, 36, s, trunc_k=0.1, window=S.WINDOW_RATIO)
    ref = oracle.render(g, v)
    assert np.all(normwise(out.cpu().double().numpy(), ref, axis=(1, 2)) < 1e-5)
