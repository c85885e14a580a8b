"""Seeded synthetic inputs for the scale-aware Gaussian rasterizer.

This module is shared by the CUDA path (tests, bench) and by the FP64 oracle's
tests. It only draws random numbers and rounds them to a storage dtype: it holds
none of the renderer's arithmetic (no reference grid, no footprint, no density).

Workload recipes (GSASR, arXiv 2501.06838):
  * N = m * H * W Gaussians per LR image (Sec. 3.2, "Gaussian Embedding"), each a
    jittered offset o around its reference position (mu = p + o, Sec. 3.2,
    "Gaussian Primary Head");
  * per Gaussian, drawn in this order from one PCG64 stream: offset x, offset y,
    log sigma_x, log sigma_y, rho, r, g, b, alpha;
  * offsets ~ U[-0.5, 0.5] / sqrt(m) (jitter inside the Gaussian's reference
    cell), sigma ~ log-uniform in LR pixels, rho ~ U(-0.9, 0.9), RGB and alpha
    ~ U[0, 1];
  * float64 draws are rounded to float32 (the "FP32 originals"), then to the
    storage dtype (bf16 / f16) when one is asked for.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

DTYPES = ("f32", "bf16", "f16")
NORM_DENSITY = 0
NORM_PEAK = 1
WINDOW_SIGMA = 0   # |x - s mu| <= s k sigma (k = 3)
WINDOW_RATIO = 1   # |x - s mu| < s r W, |y - s mu| < s r H (Algorithm 1, ratio r)
ALIGN_EQ4 = 0      # HR pixel x samples LR x / s (Eq. 4 as printed)
ALIGN_HALF = 1     # HR pixel x samples LR (x + 1/2) / s - 1/2


def round_f32(x: np.ndarray) -> np.ndarray:
    return np.asarray(x, dtype=np.float64).astype(np.float32)


def round_bf16_bits(x32: np.ndarray) -> np.ndarray:
    """float32 -> bfloat16 bit patterns (uint16), round to nearest even."""
    x32 = np.ascontiguousarray(x32, dtype=np.float32)
    bits = x32.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    rounded = ((bits + 0x7FFF + lsb) >> 16).astype(np.uint16)
    nan = np.isnan(x32)
    if nan.any():
        rounded[nan] = 0x7FC0
    return rounded


def bf16_bits_to_f32(bits: np.ndarray) -> np.ndarray:
    return (np.asarray(bits, dtype=np.uint32) << 16).view(np.float32)


def storage_round(x64: np.ndarray, dtype: str) -> np.ndarray:
    """Value actually stored for `dtype`, returned exactly widened to float64."""
    x32 = round_f32(x64)
    if dtype == "f32":
        return x32.astype(np.float64)
    if dtype == "bf16":
        return bf16_bits_to_f32(round_bf16_bits(x32)).astype(np.float64)
    if dtype == "f16":
        return x32.astype(np.float16).astype(np.float64)
    raise ValueError(f"unknown dtype {dtype}")


def storage_array(x64: np.ndarray, dtype: str) -> np.ndarray:
    """The raw storage array (float32, uint16 bf16 bits, or float16)."""
    x32 = round_f32(x64)
    if dtype == "f32":
        return x32
    if dtype == "bf16":
        return round_bf16_bits(x32)
    if dtype == "f16":
        return x32.astype(np.float16)
    raise ValueError(f"unknown dtype {dtype}")


@dataclasses.dataclass
class Head:
    """The Gaussian primary head's activations (Sec. 3.2), fused into the
    renderer: sigma = sigma_lo + sigma_span * sigmoid(raw), rho = rho_scale *
    tanh(raw), c = sigmoid(raw), alpha = sigmoid(raw), o = offset_scale * raw
    (or offset_scale * tanh(raw) with offset_tanh). The paper's own head is
    sigma_lo = 0, sigma_span = 1, rho_scale = 1, offset_scale = 1, no tanh."""
    sigma_lo: float = 0.0
    sigma_span: float = 1.0
    rho_scale: float = 1.0
    offset_scale: float = 1.0
    offset_tanh: int = 0


@dataclasses.dataclass
class GaussianSet:
    """Gaussian parameters of one image: physical (post-activation) values, or
    raw head outputs when `head` is set.

    Arrays hold the STORED values widened exactly to float64: what the renderer
    reads. `originals` keeps the float32 originals when `dtype` is reduced.
    ref_grid_m > 0: `offset` is o and the centre is mu = p(index) + o.
    ref_grid_m == 0: `offset` holds the absolute centre mu (LR pixels).
    """
    offset: np.ndarray  # [N, 2]
    sigma: np.ndarray   # [N, 2]
    rho: np.ndarray     # [N]
    rgb: np.ndarray     # [N, 3]
    alpha: np.ndarray   # [N]
    lr_h: int
    lr_w: int
    ref_grid_m: int = 1
    dtype: str = "f32"
    originals: "GaussianSet | None" = None
    head: "Head | None" = None

    @property
    def n(self) -> int:
        return int(self.rho.shape[0])

    def fields(self):
        return (self.offset, self.sigma, self.rho, self.rgb, self.alpha)

    def storage(self):
        """Raw storage arrays (what a device copy of the parameters holds)."""
        return tuple(storage_array(a, self.dtype) for a in self.fields())

    def with_dtype(self, dtype: str) -> "GaussianSet":
        base = self.originals if self.originals is not None else self
        vals = [storage_round(a, dtype) for a in base.fields()]
        return GaussianSet(*vals, lr_h=base.lr_h, lr_w=base.lr_w,
                           ref_grid_m=base.ref_grid_m, dtype=dtype,
                           originals=None if dtype == "f32" else base, head=base.head)

    def subset(self, idx) -> "GaussianSet":
        idx = np.asarray(idx)
        return GaussianSet(self.offset[idx], self.sigma[idx], self.rho[idx],
                           self.rgb[idx], self.alpha[idx], self.lr_h, self.lr_w,
                           0, self.dtype, None)


@dataclasses.dataclass
class View:
    """Output request: HR image of out_h x out_w sampled at scale s (Eq. 4)."""
    lr_h: int
    lr_w: int
    out_h: int
    out_w: int
    scale: float          # a float32 value
    trunc_k: float = 3.0  # window parameter: k (sigma box) or r (ratio box); <= 0: untruncated
    norm: int = NORM_DENSITY
    window: int = 0       # 0: |x - s mu| <= s k sigma; 1: |x - s mu| < s r W (Algorithm 1)
    align: int = 0        # 0: HR pixel x samples x / s (Eq. 4); 1: (x + 1/2) / s - 1/2

    def __post_init__(self):
        self.scale = float(np.float32(self.scale))
        self.trunc_k = float(np.float32(self.trunc_k))


def out_size(lr: int, scale: float) -> int:
    """floor(s * lr) with s the float32 scale (the product is exact in f64)."""
    return int(math.floor(float(np.float32(scale)) * lr))


def draw_gaussians(seed: int, lr_h: int, lr_w: int, m: int = 1,
                   sigma_range=(0.3, 2.0), dtype: str = "f32",
                   offset_half=0.5) -> GaussianSet:
    rng = np.random.Generator(np.random.PCG64(seed))
    n = m * lr_h * lr_w
    u = rng.random((n, 9))
    cell = 1.0 / math.sqrt(m)
    lo, hi = math.log(sigma_range[0]), math.log(sigma_range[1])
    offset = (u[:, 0:2] * 2.0 - 1.0) * offset_half * cell
    sigma = np.exp(lo + u[:, 2:4] * (hi - lo))
    rho = -0.9 + 1.8 * u[:, 4]
    rgb = u[:, 5:8].copy()
    alpha = u[:, 8].copy()
    f32 = GaussianSet(*(storage_round(a, "f32") for a in (offset, sigma, rho, rgb, alpha)),
                      lr_h=lr_h, lr_w=lr_w, ref_grid_m=m, dtype="f32")
    return f32 if dtype == "f32" else f32.with_dtype(dtype)


def draw_raw_head(seed: int, lr_h: int, lr_w: int, m: int = 1, head: Head | None = None,
                  dtype: str = "f32", spread: float = 1.5) -> GaussianSet:
    """Raw head outputs ~ N(0, spread^2) per value (offsets ~ N(0, (0.25/sqrt m)^2)),
    for the fused-head render: the set's `head` maps them to physical values."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = m * lr_h * lr_w
    z = rng.standard_normal((n, 9))
    offset = z[:, 0:2] * (0.25 / math.sqrt(m))
    sigma, rho = z[:, 2:4] * spread, z[:, 4] * spread
    rgb, alpha = z[:, 5:8] * spread, z[:, 8] * spread
    f32 = GaussianSet(*(storage_round(a, "f32") for a in (offset, sigma, rho, rgb, alpha)),
                      lr_h=lr_h, lr_w=lr_w, ref_grid_m=m, dtype="f32", head=head or Head())
    return f32 if dtype == "f32" else f32.with_dtype(dtype)


def grad_out(seed: int, out_h: int, out_w: int) -> np.ndarray:
    """Upstream gradient ~ N(0, 1) per output element, float32 [3, H, W]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((3, out_h, out_w)).astype(np.float32)


def sample_indices(seed: int, n: int, k: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.sort(rng.choice(n, size=min(k, n), replace=False))


# --------------------------------------------------------------------------
# The five workloads. Each returns (list of GaussianSet, list of View).
# --------------------------------------------------------------------------

def config1():
    """Forward-only FP32: LR 48x48, m=1 (N=2,304), x4 -> 192x192, seed 0."""
    g = draw_gaussians(0, 48, 48, 1, (0.3, 2.0))
    return [g], [View(48, 48, 192, 192, 4.0)]


def config2():
    """Forward + adjoint FP32: LR 256x256, m=1 (N=65,536), x4 -> 1024x1024."""
    g = draw_gaussians(0, 256, 256, 1, (0.3, 2.0))
    return [g], [View(256, 256, 1024, 1024, 4.0)]


def config3_sizes(seed: int = 0, n_images: int = 16):
    """LR sizes (multiples of 4, W in 64..480, H in 64..360) and s ~ U[1.5, 12]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ws = rng.integers(16, 121, size=n_images) * 4
    hs = rng.integers(16, 91, size=n_images) * 4
    ss = rng.uniform(1.5, 12.0, size=n_images).astype(np.float32)
    return [(int(h), int(w), float(s)) for h, w, s in zip(hs, ws, ss)]


def config3(n_images: int = 16):
    """Batched uneven FP32: 16 images, m=1, non-integer scales in [1.5, 12]."""
    gs, vs = [], []
    for i, (h, w, s) in enumerate(config3_sizes(0, n_images)):
        gs.append(draw_gaussians(100 + i, h, w, 1, (0.3, 2.0)))
        vs.append(View(h, w, out_size(h, s), out_size(w, s), s))
    return gs, vs


def config3_equal(n_images: int = 16):
    """16 images of one size: the mean LR size (rounded to a multiple of 4) and
    the mean scale of config 3; the equal-size reference for its throughput."""
    sz = config3_sizes(0, n_images)
    h = int(round(np.mean([a for a, _, _ in sz]) / 4)) * 4
    w = int(round(np.mean([b for _, b, _ in sz]) / 4)) * 4
    s = float(np.float32(np.mean([c for _, _, c in sz])))
    gs = [draw_gaussians(200 + i, h, w, 1, (0.3, 2.0)) for i in range(n_images)]
    return gs, [View(h, w, out_size(h, s), out_size(w, s), s) for _ in range(n_images)]


def config4(scale: float = 12.0, dtype: str = "bf16"):
    """Reduced precision: LR 480x270 (W x H), m=4 (N=518,400), sigma in [0.2, 3]."""
    g = draw_gaussians(0, 270, 480, 4, (0.2, 3.0), dtype=dtype)
    return [g], [View(270, 480, out_size(270, scale), out_size(480, scale), scale)]


def ratio_ablation(scale: float = 4.0, r: float = 0.1, hr: int = 720):
    """The shape of the rasterization-ratio ablation (Sec. 3.1, r-ablation table):
    a square hr x hr output from an LR image of hr / s pixels a side, m = 16
    Gaussians per LR pixel, Algorithm 1's ratio window with ratio r."""
    lr = int(round(hr / scale))
    g = draw_gaussians(0, lr, lr, 16, (0.2, 3.0))
    return [g], [View(lr, lr, out_size(lr, scale), out_size(lr, scale), scale, trunc_k=r,
                      window=WINDOW_RATIO)]


def pipeline_input(scale: float, hr: int = 720, seed: int = 7) -> np.ndarray:
    """LR image [3, lr, lr] float32 of the computational-cost table's shape
    (a 720x720 crop down-scaled by s): the seeded image function sampled at
    the LR pixel centres, lr = round(hr / s)."""
    lr = int(round(hr / scale))
    f = image_function(seed, lr)
    ys, xs = np.mgrid[0:lr, 0:lr]
    return f(xs, ys).astype(np.float32)


def config5_scales(seed: int = 0, batch: int = 16):
    rng = np.random.Generator(np.random.PCG64(seed))
    return [float(np.float32(s)) for s in rng.uniform(1.0, 4.0, size=batch)]


# --------------------------------------------------------------------------
# Config 5: a seeded continuous image function, sampled at the LR pixel
# centres for the input crop and at (x/s, y/s) for the HR target (the sampling
# convention of Eq. 4), so every scale factor has an exact target.
# --------------------------------------------------------------------------
@dataclasses.dataclass
class ImageFunction:
    freqs: np.ndarray    # [K, 2] cycles per LR pixel
    phases: np.ndarray   # [K]
    amps: np.ndarray     # [K, 3]
    normals: np.ndarray  # [E, 2] unit edge normals
    offsets: np.ndarray  # [E]
    steps: np.ndarray    # [E, 3] colour jump across each edge
    base: np.ndarray     # [3]

    def __call__(self, x, y):
        """x, y: arrays of LR coordinates; returns [3, *x.shape] in ~[0, 1]."""
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        out = np.zeros((3,) + x.shape)
        for (fx, fy), ph, a in zip(self.freqs, self.phases, self.amps):
            out += a[:, None, None] * np.cos(2 * np.pi * (fx * x + fy * y) + ph)[None]
        for (nx, ny), d, st in zip(self.normals, self.offsets, self.steps):
            ramp = 0.5 * (1 + np.tanh((nx * x + ny * y - d) / 0.5))
            out += st[:, None, None] * ramp[None]
        return np.clip(out + self.base[:, None, None], 0.0, 1.0)


def image_function(seed: int, size: int = 48) -> ImageFunction:
    rng = np.random.Generator(np.random.PCG64(seed))
    k, e = 12, 3
    ang = rng.uniform(0, 2 * np.pi, k)
    rad = rng.uniform(0.01, 0.15, k)
    theta = rng.uniform(0, 2 * np.pi, e)
    return ImageFunction(
        freqs=np.stack([rad * np.cos(ang), rad * np.sin(ang)], 1),
        phases=rng.uniform(0, 2 * np.pi, k),
        amps=rng.normal(0, 0.08, (k, 3)),
        normals=np.stack([np.cos(theta), np.sin(theta)], 1),
        offsets=rng.uniform(0.3, 0.7, e) * size * (np.abs(np.cos(theta)) + np.abs(np.sin(theta))),
        steps=rng.normal(0, 0.25, (e, 3)),
        base=rng.uniform(0.3, 0.7, 3))


def config5_batch(step: int, batch: int = 16, size: int = 48):
    """(lr images [B, 3, 48, 48] float32, HR targets list of [3, floor(48 s)]^2,
    scales) for training step `step` (seed 1000 * step + i per sample)."""
    scales = config5_scales(10_000 + step, batch)
    lrs, hrs = [], []
    ys, xs = np.mgrid[0:size, 0:size]
    for i, s in enumerate(scales):
        f = image_function(1000 * step + i, size)
        lrs.append(f(xs, ys).astype(np.float32))
        n = out_size(size, s)
        Y, X = np.mgrid[0:n, 0:n] / np.float64(np.float32(s))
        hrs.append(f(X, Y).astype(np.float32))
    return np.stack(lrs), hrs, scales
