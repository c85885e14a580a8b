"""Config 5: one end-to-end training step through the renderer.

A random-init 8-block, 64-channel 3x3 convolutional encoder on 48x48 LR crops
and a 1x1-convolution Gaussian head predict, per LR pixel, one Gaussian's
offset, sigma, rho, colour and opacity (the head's activations follow GSASR
Sec. 3.2, Gaussian Primary Head: tanh for rho, sigmoid for sigma, colour and
opacity, mu = p + o; by default they run fused inside the renderer's footprint
pass, with their derivatives in its chain-rule pass). The raw outputs are
stored in BF16 and rendered by the library's batched autograd Function at a per-sample scale s ~ U[1, 4]
(training-time scales of Sec. 4.1); the L1 loss against the HR target
(Sec. 3.2, Rendering) is back-propagated through the render's adjoint into the
encoder. The encoder and head are plain PyTorch layers: they stand in for the
paper's learned backbone and decoder, which this library does not implement.
"""
from __future__ import annotations

import torch
import torch.nn as nn

from .render import GSRenderBatched, View, out_size


class ResBlock(nn.Module):
    def __init__(self, c: int):
        super().__init__()
        self.c1 = nn.Conv2d(c, c, 3, padding=1)
        self.c2 = nn.Conv2d(c, c, 3, padding=1)

    def forward(self, x):
        return x + self.c2(torch.relu(self.c1(x)))


class HeadSpec:
    """The head's activations: o = tanh (|o| < 1 LR px), sigma = 0.2 + 2.8 sigmoid
    (LR px), rho = 0.9 tanh, colour and opacity sigmoid (a gs_head)."""
    sigma_lo, sigma_span, rho_scale, offset_scale, offset_tanh = 0.2, 2.8, 0.9, 1.0, 1


class ToyGaussianSR(nn.Module):
    """LR image [B, 3, H, W] -> per-pixel Gaussian parameters (m = 1): raw head
    outputs (activated inside the renderer), or with activate=True the physical
    parameters through PyTorch's own activations."""

    def __init__(self, channels: int = 64, blocks: int = 8):
        super().__init__()
        self.inp = nn.Conv2d(3, channels, 3, padding=1)
        self.body = nn.Sequential(*[ResBlock(channels) for _ in range(blocks)])
        self.head = nn.Conv2d(channels, 9, 1)

    def forward(self, lr, activate: bool = False):
        h = self.head(self.body(self.inp(lr)))           # [B, 9, H, W]
        h = h.permute(0, 2, 3, 1).reshape(lr.shape[0], -1, 9)
        if not activate:
            return h[..., 0:2], h[..., 2:4], h[..., 4], h[..., 5:8], h[..., 8]
        H = HeadSpec
        offset = H.offset_scale * torch.tanh(h[..., 0:2])
        sigma = H.sigma_lo + H.sigma_span * torch.sigmoid(h[..., 2:4])
        rho = H.rho_scale * torch.tanh(h[..., 4])
        rgb = torch.sigmoid(h[..., 5:8])
        alpha = torch.sigmoid(h[..., 8])
        return offset, sigma, rho, rgb, alpha


class TrainStep:
    """Holds the model, optimiser and views; call(lr, targets, scales) runs one
    optimisation step and returns the loss (a device tensor)."""

    def __init__(self, size: int = 48, device="cuda", param_dtype=torch.bfloat16, lr=2e-4,
                 norm: int = 0, fused_head: bool = True):
        torch.manual_seed(0)
        self.model = ToyGaussianSR().to(device)
        self.opt = torch.optim.Adam(self.model.parameters(), lr=lr)
        self.size = size
        self.dtype = param_dtype
        self.norm = norm
        self.device = device
        self.fused_head = fused_head

    def views(self, scales):
        return [View(self.size, self.size, out_size(self.size, s), out_size(self.size, s), s,
                     norm=self.norm) for s in scales]

    def __call__(self, lr_images, targets, scales):
        views = self.views(scales)
        b = lr_images.shape[0]
        offset, sigma, rho, rgb, alpha = self.model(lr_images, activate=not self.fused_head)
        n = self.size * self.size
        cast = lambda t: t.reshape((b * n,) + t.shape[2:]).to(self.dtype).contiguous()
        outs = GSRenderBatched.apply(views, 1, [n] * b, HeadSpec if self.fused_head else None,
                                     cast(offset), cast(sigma), cast(rho), cast(rgb), cast(alpha))
        loss = sum((o - t).abs().mean() for o, t in zip(outs, targets)) / b
        self.opt.zero_grad(set_to_none=True)
        loss.backward()
        self.opt.step()
        return loss.detach()
