"""The whole GSASR inference pipeline with random weights, for timing.

LR image -> EDSR-baseline encoder -> Gaussian decoder -> Gaussian primary
heads -> this library's scale-aware render (GSASR, arXiv 2501.06838, Sec. 3.2
and Fig. 2; the computational-cost table times this chain on 720 x 720
outputs):

  encoder      EDSR-baseline without its upsampler: 16 residual blocks of
               64-channel 3x3 convolutions -> features F [B, 64, H, W];
  embeddings   one learnable block E_base of m k^2 embeddings of width d per
               k x k window of F, duplicated over the windows (Sec. 3.2,
               Gaussian Embedding), N = m H W Gaussians in all;
  injection    window cross-attention, queries from the embeddings, keys and
               values from the window's features, plus a learnable relative
               position bias B (the condition injection block);
  interaction  L blocks of window self-attention, shifted-window
               self-attention and a cross-attention to scale tokens, each
               followed by an MLP (the Gaussian interaction block);
  heads        five decoupled MLPs of three linear layers with two ReLUs ->
               raw offset, sigma, rho, colour and opacity (Gaussian primary
               head); their activations run fused in the render (gs_head);
  render       Eq. 4 with Algorithm 1's ratio window, in the library's
               kernels (forward only at inference).

Hyper-parameters follow Sec. 4.1: k = 12, m = 16, d = 180, L = 6. Where the
paper leaves a detail open (heads, MLP width, the scale tokens, the padding of
F to whole windows, the shifted windows' boundary mask) this module takes a
stated reading, chosen so the arithmetic has the paper's shape; the weights
are random, so only the timing means anything. The network runs in PyTorch
(cuBLAS GEMMs and PyTorch's fused attention kernels); only the render is this
library's own code.

Storage width. The width-d stream is held at d_store = 184 channels (d rounded
up to a multiple of 8) so that every GEMM has 16-byte aligned BF16 rows. The
extra channels of the residual stream each carry the mean of the d real ones
(every layer adding into the stream has its extra output rows set to the mean
of its real rows), which lets one fused LayerNorm of width d_store compute the
width-d one exactly (_PLayerNorm); all other extra channels are zero and
ignored. load_unpadded() maps the state of the width-d model.

Token layout. The decoder keeps its tokens on the sub-pixel grid
[B, sqrt(m) Hp, sqrt(m) Wp, d]: token (ty, tx) is the Gaussian whose reference
position is (x, y) = ((tx + 1/2) / sqrt(m) - 1/2, (ty + 1/2) / sqrt(m) - 1/2)
in LR pixels, i.e. LR pixel (i, j) = (ty // sqrt(m), tx // sqrt(m)) and
sub-grid point (b, a) = (ty % sqrt(m), tx % sqrt(m)). gaussian_order() maps the
grid to the render's index order gid = ((i W + j) m + b sqrt(m) + a), whose
reference positions are the same points (m equally spaced points per LR pixel,
Sec. 3.2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch
import torch.nn as nn
import torch.nn.functional as F
from torch.nn.attention import SDPBackend, sdpa_kernel

from .render import WINDOW_RATIO, Gaussians, View, out_size, render_batched


@dataclass
class GSASRConfig:
    """Sec. 4.1 values by default; small values serve the CPU tests."""
    n_feats: int = 64          # EDSR-baseline width
    n_resblocks: int = 16      # EDSR-baseline depth
    k: int = 12                # window size (LR pixels)
    m: int = 16                # Gaussians per LR pixel (a square number)
    d: int = 180               # embedding width
    heads: int = 6             # attention heads (head width d / heads = 30)
    head_pad: int = 32         # head width as computed (zero-padded; fused kernels want 8 | width)
    blocks: int = 6            # L, Gaussian interaction blocks
    mlp_ratio: int = 2         # MLP hidden width / d
    scale_tokens: int = 8      # tokens the scale cross-attention attends to
    window_chunk: int = 32     # windows per attention call (bounds temporaries)
    pad_width: bool = True     # hold the width-d stream at a multiple of 8

    @property
    def d_store(self) -> int:
        """Width the embeddings are held at: d rounded up to a multiple of 8, so
        that every GEMM of the decoder has 16-byte aligned rows in BF16; d itself
        with pad_width off. The extra channels of the residual stream carry the
        mean of the real ones, which makes the layer norms exact (_PLayerNorm);
        every other extra channel is zero and every layer ignores them."""
        return -(-self.d // 8) * 8 if self.pad_width else self.d


@dataclass
class PipelineHead:
    """Activations of the Gaussian primary head (Sec. 3.2): sigmoid for sigma
    (in LR pixels, span 1), colour and opacity; tanh for rho, scaled by 0.99
    so that |rho| < 1 holds in float32 (the render's domain); no activation on
    the offset."""
    sigma_lo: float = 0.0
    sigma_span: float = 1.0
    rho_scale: float = 0.99
    offset_scale: float = 1.0
    offset_tanh: int = 0


# --------------------------------------------------------------------------
# Geometry of the token grid (index logic only; tested on the CPU).
# --------------------------------------------------------------------------
def window_partition(x: torch.Tensor, w: int) -> torch.Tensor:
    """[B, Gh, Gw, C] -> [B * (Gh / w) * (Gw / w), w * w, C], windows row-major."""
    b, gh, gw, c = x.shape
    x = x.view(b, gh // w, w, gw // w, w, c).permute(0, 1, 3, 2, 4, 5)
    return x.reshape(-1, w * w, c)


def window_reverse(x: torch.Tensor, w: int, b: int, gh: int, gw: int) -> torch.Tensor:
    """Inverse of window_partition."""
    c = x.shape[-1]
    x = x.view(b, gh // w, gw // w, w, w, c).permute(0, 1, 3, 2, 4, 5)
    return x.reshape(b, gh, gw, c)


def relative_index_self(w: int) -> torch.Tensor:
    """[w^2, w^2] index into a (2w - 1)^2 table of the offset between two
    tokens of a w x w window (Swin's relative position bias)."""
    ys, xs = torch.meshgrid(torch.arange(w), torch.arange(w), indexing="ij")
    ys, xs = ys.reshape(-1), xs.reshape(-1)
    dy = ys[:, None] - ys[None, :] + (w - 1)
    dx = xs[:, None] - xs[None, :] + (w - 1)
    return dy * (2 * w - 1) + dx


def relative_index_cross(k: int, r: int) -> torch.Tensor:
    """[(r k)^2, k^2] index into a (2 r k)^2 table of the offset, in 1/r LR
    pixel steps, between a Gaussian token of a window (sub-grid r x r per
    pixel) and a feature pixel of the same window: r * (its pixel offset)
    taken at the sub-grid point, shifted to be non-negative."""
    w = r * k
    ty, tx = torch.meshgrid(torch.arange(w), torch.arange(w), indexing="ij")
    py, px = torch.meshgrid(torch.arange(k), torch.arange(k), indexing="ij")
    dy = ty.reshape(-1)[:, None] - r * py.reshape(-1)[None, :] + (w - r)
    dx = tx.reshape(-1)[:, None] - r * px.reshape(-1)[None, :] + (w - r)
    return dy * (2 * w) + dx


def gaussian_order(grid: torch.Tensor, h: int, w: int, m: int) -> torch.Tensor:
    """Token grid [B, >= r h, >= r w, C] (r = sqrt(m)) -> [B, m h w, C] in the
    render's order gid = ((i w + j) m + b r + a), cropping the padding."""
    r = math.isqrt(m)
    b, c = grid.shape[0], grid.shape[-1]
    g = grid[:, :r * h, :r * w]
    g = g.reshape(b, h, r, w, r, c).permute(0, 1, 3, 2, 4, 5)
    return g.reshape(b, m * h * w, c)


# --------------------------------------------------------------------------
# Network (random weights; plain PyTorch layers).
# --------------------------------------------------------------------------
def _compute_dtype(x: torch.Tensor) -> torch.dtype:
    """The dtype the attention runs in: autocast's when it is on."""
    if x.is_cuda and torch.is_autocast_enabled("cuda"):
        return torch.get_autocast_dtype("cuda")
    return x.dtype


def _sdpa(Q, K, V, mask, scale):
    """Scaled dot-product attention, on the GPU through cuDNN's fused kernel
    when it takes the case: with a bias it runs about 3x faster there than in
    PyTorch's default choice (the memory-efficient kernel)."""
    if Q.is_cuda:
        try:
            with sdpa_kernel([SDPBackend.CUDNN_ATTENTION]):
                return F.scaled_dot_product_attention(Q, K, V, attn_mask=mask, scale=scale)
        except RuntimeError:
            pass
    return F.scaled_dot_product_attention(Q, K, V, attn_mask=mask, scale=scale)


def _bias(owner: nn.Module, dtype) -> torch.Tensor:
    """Relative position bias [heads, T, S] of a layer, gathered from its
    table once per call; outside autograd (inference) kept until the table
    changes, since it is a function of the weights alone."""
    table, index = owner.table, owner.index
    if torch.is_grad_enabled():
        return table[index].permute(2, 0, 1).to(dtype).contiguous()
    key = (dtype, table.device, table._version, table.data_ptr())
    cached = getattr(owner, "_bias_cache", None)
    if cached is None or cached[0] != key:
        cached = (key, table[index].permute(2, 0, 1).to(dtype).contiguous())
        owner._bias_cache = cached
    return cached[1]


class _ResBlock(nn.Module):
    def __init__(self, c: int):
        super().__init__()
        self.c1 = nn.Conv2d(c, c, 3, padding=1)
        self.c2 = nn.Conv2d(c, c, 3, padding=1)

    def forward(self, x):
        return x + self.c2(torch.relu(self.c1(x)))


class EDSRBaseline(nn.Module):
    """EDSR-baseline feature extractor (no upsampler): conv, residual blocks,
    conv, global skip."""

    def __init__(self, n_feats: int = 64, n_resblocks: int = 16):
        super().__init__()
        self.head = nn.Conv2d(3, n_feats, 3, padding=1)
        self.body = nn.Sequential(*[_ResBlock(n_feats) for _ in range(n_resblocks)])
        self.tail = nn.Conv2d(n_feats, n_feats, 3, padding=1)

    def forward(self, x):
        h = self.head(x)
        return h + self.tail(self.body(h))


class _PLinear(nn.Linear):
    """nn.Linear(in_real -> out_real) held at widths (in_store, out_store).
    The extra input columns are zero, so extra input channels are ignored.
    The extra output rows are zero (pad="zero"), or each is the mean of the
    real rows (pad="mean"), so that every extra output equals the mean of the
    real outputs. Initialised as the real layer."""

    def __init__(self, in_real: int, out_real: int, in_store: int = 0, out_store: int = 0,
                 pad: str = "zero"):
        super().__init__(in_store or in_real, out_store or out_real)
        self.in_real, self.out_real, self.pad = in_real, out_real, pad
        if (self.in_features, self.out_features) != (in_real, out_real):
            ref = nn.Linear(in_real, out_real)
            with torch.no_grad():
                self.weight.zero_()
                self.bias.zero_()
                self.weight[:out_real, :in_real] = ref.weight
                self.bias[:out_real] = ref.bias
            self.sync_pads()

    @torch.no_grad()
    def sync_pads(self):
        """Re-derive the extra rows and columns from the real block."""
        r, c = self.out_real, self.in_real
        self.weight[:, c:] = 0
        fill_w = self.weight[:r].mean(0) if self.pad == "mean" else 0
        fill_b = self.bias[:r].mean() if self.pad == "mean" else 0
        self.weight[r:] = fill_w
        self.bias[r:] = fill_b


class _PLayerNorm(nn.LayerNorm):
    """LayerNorm over d_real channels held at d_store, for an input whose extra
    channels each carry the mean m of the real ones (the residual stream of
    this model, whose producers are pad="mean" layers). Then the d_store-wide
    statistics are m and (d_real / d_store) var, so a LayerNorm of width d_store
    with eps and the real weights both scaled by d_real / d_store (the weights
    by its square root) gives the d_real-wide LayerNorm on the real channels,
    exactly; its extra outputs are zero (zero weight and bias there)."""

    def __init__(self, d_real: int, d_store: int = 0, eps: float = 1e-5):
        c = d_real / float(d_store or d_real)
        super().__init__(d_store or d_real, eps=eps * c)
        self.d_real, self.gain = d_real, math.sqrt(c)
        with torch.no_grad():
            self.weight[:d_real] = self.gain
            self.weight[d_real:] = 0
            self.bias[d_real:] = 0


class _Attention(nn.Module):
    """Multi-head attention with queries from x and keys / values from ctx,
    heads padded from d / heads to head_pad columns (zero weights; the scale
    stays 1 / sqrt(d / heads))."""

    def __init__(self, d: int, ctx_dim: int, heads: int, head_pad: int, d_store: int = 0,
                 ctx_store: int = 0):
        super().__init__()
        self.heads, self.hd, self.hp = heads, d // heads, head_pad
        self.q = _PLinear(d, heads * head_pad, d_store)
        self.kv = _PLinear(ctx_dim, 2 * heads * head_pad, ctx_store)
        self.proj = _PLinear(heads * head_pad, d, 0, d_store, pad="mean")
        with torch.no_grad():   # padded columns carry zeros
            for lin, rows in ((self.q, 1), (self.kv, 2)):
                wv = lin.weight.view(rows * heads, head_pad, -1)
                wv[:, self.hd:] = 0
                lin.bias.view(rows * heads, head_pad)[:, self.hd:] = 0
            self.proj.weight.view(-1, heads, head_pad)[:, :, self.hd:] = 0

    def split(self, t, n):
        return t.view(t.shape[0], n, self.heads, self.hp).transpose(1, 2)

    def forward(self, q, ctx, bias=None):
        """q: [Bq, T, d] (Bq = 1 broadcasts); ctx: [Bw, S, ctx_dim];
        bias: [heads, T, S] or None."""
        bw, t, s = ctx.shape[0], q.shape[1], ctx.shape[1]
        Q = self.split(self.q(q), t).expand(bw, -1, -1, -1)
        K, V = self.kv(ctx).chunk(2, dim=-1)
        K, V = self.split(K.contiguous(), s), self.split(V.contiguous(), s)
        mask = None if bias is None else bias[None].expand(bw, -1, -1, -1)
        o = _sdpa(Q, K, V, mask, 1.0 / math.sqrt(self.hd))
        return self.proj(o.transpose(1, 2).reshape(bw, t, self.heads * self.hp))


class _MLP(nn.Module):
    def __init__(self, d: int, ratio: int, d_store: int = 0):
        super().__init__()
        self.fc1 = _PLinear(d, ratio * d, d_store)
        self.fc2 = _PLinear(ratio * d, d, 0, d_store, pad="mean")

    def forward(self, x):
        return self.fc2(F.gelu(self.fc1(x)))


class ConditionInjection(nn.Module):
    """Window cross-attention from the Gaussian embeddings to the window's
    LR features, with a relative position bias, then an MLP."""

    def __init__(self, cfg: GSASRConfig):
        super().__init__()
        r = math.isqrt(cfg.m)
        self.cfg = cfg
        dp = cfg.d_store
        self.ln_q, self.ln_f, self.ln_m = _PLayerNorm(cfg.d, dp), nn.LayerNorm(cfg.n_feats), \
            _PLayerNorm(cfg.d, dp)
        self.att = _Attention(cfg.d, cfg.n_feats, cfg.heads, cfg.head_pad, dp)
        self.table = nn.Parameter(0.02 * torch.randn((2 * r * cfg.k) ** 2, cfg.heads))
        self.register_buffer("index", relative_index_cross(cfg.k, r), persistent=False)
        self.mlp = _MLP(cfg.d, cfg.mlp_ratio, dp)

    def forward(self, e_base, feats, b, gh, gw):
        """e_base: [T, d]; feats: [B, Hp, Wp, C] -> token grid [B, gh, gw, d]."""
        cfg = self.cfg
        f = self.ln_f(feats)
        fw = window_partition(f.to(_compute_dtype(f)), cfg.k)        # [nW, k^2, C]
        q = self.ln_q(e_base)[None]
        bias = _bias(self, _compute_dtype(fw))       # [heads, T, k^2]
        outs = [self.att(q, fw[i:i + cfg.window_chunk], bias)
                for i in range(0, fw.shape[0], cfg.window_chunk)]
        x = e_base[None] + torch.cat(outs, 0)                        # [nW, T, d]
        x = window_reverse(x, math.isqrt(cfg.m) * cfg.k, b, gh, gw)
        return x + self.mlp(self.ln_m(x))


class _WindowSelfAttention(nn.Module):
    def __init__(self, cfg: GSASRConfig, shift: bool):
        super().__init__()
        self.cfg, self.shift = cfg, shift
        self.w = math.isqrt(cfg.m) * cfg.k
        dp = cfg.d_store
        self.ln, self.ln_m = _PLayerNorm(cfg.d, dp), _PLayerNorm(cfg.d, dp)
        self.att = _Attention(cfg.d, cfg.d, cfg.heads, cfg.head_pad, dp, dp)
        self.table = nn.Parameter(0.02 * torch.randn((2 * self.w - 1) ** 2, cfg.heads))
        self.register_buffer("index", relative_index_self(self.w), persistent=False)
        self.mlp = _MLP(cfg.d, cfg.mlp_ratio, dp)

    def forward(self, x):
        b, gh, gw, _ = x.shape
        h = self.ln(x)
        h = h.to(_compute_dtype(h))       # move the windows in the compute dtype
        sh = self.w // 2 if self.shift else 0
        if sh:
            h = torch.roll(h, shifts=(-sh, -sh), dims=(1, 2))
        hw = window_partition(h, self.w)
        bias = _bias(self, _compute_dtype(hw))     # [heads, T, T]
        c = self.cfg.window_chunk
        o = torch.cat([self.att(hw[i:i + c], hw[i:i + c], bias) for i in range(0, hw.shape[0], c)], 0)
        o = window_reverse(o, self.w, b, gh, gw)
        if sh:
            o = torch.roll(o, shifts=(sh, sh), dims=(1, 2))
        x = x + o
        return x + self.mlp(self.ln_m(x))


class _ScaleAttention(nn.Module):
    """Cross-attention of every embedding to a few tokens made from the scale
    factor (sinusoidal features of log s through an MLP)."""

    def __init__(self, cfg: GSASRConfig):
        super().__init__()
        self.cfg = cfg
        dp = cfg.d_store
        self.embed = nn.Sequential(nn.Linear(32, cfg.d), nn.GELU(),
                                   nn.Linear(cfg.d, cfg.scale_tokens * cfg.d))
        self.ln, self.ln_m = _PLayerNorm(cfg.d, dp), _PLayerNorm(cfg.d, dp)
        self.att = _Attention(cfg.d, cfg.d, cfg.heads, cfg.head_pad, dp)
        self.mlp = _MLP(cfg.d, cfg.mlp_ratio, dp)

    def forward(self, x, scale_feat):
        b, gh, gw, d = x.shape
        tok = self.embed(scale_feat).view(b, self.cfg.scale_tokens, self.cfg.d)
        o = self.att(self.ln(x).view(b, gh * gw, d), tok).view(b, gh, gw, d)
        x = x + o
        return x + self.mlp(self.ln_m(x))


class GaussianInteraction(nn.Module):
    """One Gaussian interaction block: window and shifted-window self-attention
    among the embeddings, then the scale cross-attention."""

    def __init__(self, cfg: GSASRConfig):
        super().__init__()
        self.wsa = _WindowSelfAttention(cfg, shift=False)
        self.swsa = _WindowSelfAttention(cfg, shift=True)
        self.sca = _ScaleAttention(cfg)

    def forward(self, x, scale_feat):
        return self.sca(self.swsa(self.wsa(x)), scale_feat)


class GaussianPrimaryHead(nn.Module):
    """Five decoupled MLPs (three linear layers, two ReLUs) -> raw
    (offset 2, sigma 2, rho 1, colour 3, opacity 1)."""
    OUTS = (2, 2, 1, 3, 1)

    def __init__(self, d: int, d_store: int = 0):
        super().__init__()
        dp = d_store or d
        self.mlps = nn.ModuleList([nn.Sequential(_PLinear(d, d, dp, dp), nn.ReLU(),
                                                 _PLinear(d, d, dp, dp), nn.ReLU(),
                                                 _PLinear(d, o, dp)) for o in self.OUTS])

    def forward(self, x):
        return torch.cat([f(x) for f in self.mlps], -1)


def scale_features(s: torch.Tensor) -> torch.Tensor:
    """[B] scale factors -> [B, 32] sinusoidal features of log s."""
    f = (2.0 ** torch.arange(16, device=s.device, dtype=torch.float32))
    a = torch.log(s.float())[:, None] * f[None]
    return torch.cat([torch.sin(a), torch.cos(a)], -1)


class GSASR(nn.Module):
    """LR image -> raw Gaussian head outputs in the render's order (decode),
    and -> SR image through the library's render (__call__ / sr)."""

    def __init__(self, cfg: GSASRConfig | None = None):
        super().__init__()
        self.cfg = cfg = cfg or GSASRConfig()
        r = math.isqrt(cfg.m)
        if r * r != cfg.m or cfg.d % cfg.heads or cfg.head_pad < cfg.d // cfg.heads:
            raise ValueError("m must be a square, heads must divide d, head_pad >= d / heads")
        self.encoder = EDSRBaseline(cfg.n_feats, cfg.n_resblocks)
        e = torch.zeros((r * cfg.k) ** 2, cfg.d_store)
        e[:, :cfg.d] = 0.02 * torch.randn((r * cfg.k) ** 2, cfg.d)
        e[:, cfg.d:] = e[:, :cfg.d].mean(1, keepdim=True)
        self.e_base = nn.Parameter(e)
        self.inject = ConditionInjection(cfg)
        self.blocks = nn.ModuleList([GaussianInteraction(cfg) for _ in range(cfg.blocks)])
        self.ln = _PLayerNorm(cfg.d, cfg.d_store)
        self.head = GaussianPrimaryHead(cfg.d, cfg.d_store)

    @torch.no_grad()
    def sync_pads(self):
        """Restore the extra channels of the width-d_store layers from the real
        ones (needed after the real weights change)."""
        d = self.cfg.d
        self.e_base[:, d:] = self.e_base[:, :d].mean(1, keepdim=True)
        for mod in self.modules():
            if isinstance(mod, _PLinear):
                mod.sync_pads()
            elif isinstance(mod, _PLayerNorm):
                mod.weight[mod.d_real:] = 0
                mod.bias[mod.d_real:] = 0

    @torch.no_grad()
    def load_unpadded(self, state: dict):
        """Load the state of the same model held at width d (pad_width=False):
        each tensor into its leading block, the layer norms' weights times
        sqrt(d / d_store), then sync_pads()."""
        own = self.state_dict()
        if set(own) != set(state):
            raise ValueError("state of a different model")
        for name, t in own.items():
            src = state[name]
            if src.dim() != t.dim() or any(a > b for a, b in zip(src.shape, t.shape)):
                raise ValueError(f"{name}: {tuple(src.shape)} does not fit {tuple(t.shape)}")
            t.zero_()
            t[tuple(slice(0, n) for n in src.shape)] = src
        for mod in self.modules():
            if isinstance(mod, _PLayerNorm):
                mod.weight[:mod.d_real] *= mod.gain
        self.sync_pads()

    def encode(self, lr):
        """[B, 3, H, W] -> features [B, Hp, Wp, C] padded (reflect) to whole windows."""
        k = self.cfg.k
        f = self.encoder(lr.to(self.encoder.head.weight.dtype))
        h, w = f.shape[-2:]
        ph, pw = (-h) % k, (-w) % k
        if ph or pw:
            f = F.pad(f, (0, pw, 0, ph), mode="reflect" if ph < h and pw < w else "replicate")
        return f.permute(0, 2, 3, 1).contiguous()

    def decode(self, feats, scales, h, w):
        """features [B, Hp, Wp, C], scales [B] -> raw [B, m h w, 9] (render order)."""
        cfg = self.cfg
        r = math.isqrt(cfg.m)
        b, hp, wp, _ = feats.shape
        x = self.inject(self.e_base, feats, b, r * hp, r * wp)
        sf = scale_features(scales).to(self.e_base.dtype)
        for blk in self.blocks:
            x = blk(x, sf)
        raw = self.head(self.ln(x))
        return gaussian_order(raw, h, w, cfg.m)

    def forward(self, lr, scales):
        h, w = lr.shape[-2:]
        return self.decode(self.encode(lr), scales, h, w)

    def gaussians(self, raw_b: torch.Tensor, head=None) -> Gaussians:
        """One image's raw outputs [N, 9] -> the render's SoA parameter tensors
        with the fused head."""
        t = raw_b
        return Gaussians(t[:, 0:2].contiguous(), t[:, 2:4].contiguous(), t[:, 4].contiguous(),
                         t[:, 5:8].contiguous(), t[:, 8].contiguous(), ref_grid_m=self.cfg.m,
                         head=head or PipelineHead())

    def render(self, raw, h: int, w: int, scale: float, ratio: float = 0.1, out_hw=None,
               norm: int = 0, head=None):
        """Raw outputs [B, m h w, 9] -> list of [3, oh, ow] SR images: the
        fused head and Algorithm 1's ratio window (r = 0.1, Sec. 3.1) at out_hw
        (default floor(s h) x floor(s w))."""
        oh, ow = out_hw or (out_size(h, scale), out_size(w, scale))
        gs = [self.gaussians(raw[i], head) for i in range(raw.shape[0])]
        views = [View(h, w, oh, ow, float(scale), trunc_k=ratio, window=WINDOW_RATIO, norm=norm)
                 for _ in gs]
        outs, _ = render_batched(gs, views)
        return outs

    def sr(self, lr, scale: float, ratio: float = 0.1, out_hw=None, norm: int = 0):
        """Super-resolve [B, 3, H, W] at scale s (decode, then render)."""
        b, _, h, w = lr.shape
        raw = self(lr, torch.full((b,), float(scale), device=lr.device))
        return self.render(raw, h, w, scale, ratio, out_hw, norm)
