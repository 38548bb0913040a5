"""Batched GPU generator of surgical-like stereo pairs (training data).

The same recipe as stereo.make_cfg2, vectorised over a batch with PyTorch
on the device so that tens of thousands of training pairs cost seconds:
smoothed-noise texture with an x-ramp, textureless rectangles, dark
ellipses, a plane-plus-bumps disparity field, a linear backward warp for the
right view, right-only saturated highlights, uint8 rounding, and the
ground truth on the left grid by fixed-point iteration. It draws from a
seeded torch.Generator, so a seed gives the same batch on the same device
and PyTorch version; evaluation pairs come from the numpy generator with
other seeds. No part of the matcher's arithmetic is here.
"""
from __future__ import annotations

import math

import torch
import torch.nn.functional as F


def _gauss1d(sigma, device):
    r = int(math.ceil(3 * sigma))
    x = torch.arange(-r, r + 1, device=device, dtype=torch.float32)
    k = torch.exp(-x * x / (2 * sigma * sigma))
    return k / k.sum(), r


def _interp_rows(img, xs):
    """Linear interpolation of each row of img (B, H, W) at xs (B, H, W), clamped."""
    W = img.shape[-1]
    xs = xs.clamp(0.0, W - 1.0)
    i0 = torch.floor(xs).clamp(max=W - 2).long()
    t = xs - i0
    v0 = torch.gather(img, 2, i0)
    v1 = torch.gather(img, 2, i0 + 1)
    return (1 - t) * v0 + t * v1


class TorchCfg2Generator:
    def __init__(self, h=480, w=640, dmax=64.0, device="cuda"):
        self.h, self.w, self.dmax = h, w, float(dmax)
        self.device = torch.device(device)
        self.k, self.r = _gauss1d(2.0, self.device)
        yy, xx = torch.meshgrid(torch.arange(h, device=self.device, dtype=torch.float32),
                                torch.arange(w, device=self.device, dtype=torch.float32),
                                indexing="ij")
        self.yy, self.xx = yy, xx

    def _u(self, g, *shape, lo=0.0, hi=1.0):
        return torch.rand(*shape, generator=g, device=self.device) * (hi - lo) + lo

    def batch(self, seed: int, n: int):
        """n pairs: (left u8 (n,H,W), right u8, disparity f32 with NaN where occluded)."""
        g = torch.Generator(device=self.device)
        g.manual_seed(int(seed))
        H, W, dmax = self.h, self.w, self.dmax
        xx, yy = self.xx, self.yy
        # texture: smoothed uniform noise, stretched, plus a 0 -> 40 ramp
        s = self._u(g, n, 1, H, W, hi=255.0)
        s = F.pad(s, (self.r, self.r, 0, 0), mode="reflect")
        s = F.conv2d(s, self.k.view(1, 1, 1, -1))
        s = F.pad(s, (0, 0, self.r, self.r), mode="reflect")
        s = F.conv2d(s, self.k.view(1, 1, -1, 1))[:, 0]
        mu = s.mean(dim=(1, 2), keepdim=True)
        sd = s.std(dim=(1, 2), keepdim=True).clamp_min(1e-6)
        scene = (s - mu) / sd * 40.0 + 128.0 + xx / max(W - 1, 1) * 40.0
        # textureless rectangles (about 20% of the area)
        flat = torch.zeros(n, H, W, dtype=torch.bool, device=self.device)
        for _ in range(8):
            rw = self._u(g, n, 1, 1, lo=0.06, hi=0.20) * W
            rh = self._u(g, n, 1, 1, lo=0.06, hi=0.20) * H
            x0 = self._u(g, n, 1, 1) * (W - rw)
            y0 = self._u(g, n, 1, 1) * (H - rh)
            val = self._u(g, n, 1, 1, lo=60.0, hi=200.0)
            inside = (xx >= x0) & (xx < x0 + rw) & (yy >= y0) & (yy < y0 + rh)
            inside &= flat.float().mean(dim=(1, 2), keepdim=True) < 0.20
            scene = torch.where(inside, val, scene)
            flat |= inside
        # dark ellipses
        dark = torch.zeros_like(flat)
        for i in range(3):
            cx, cy = self._u(g, n, 1, 1) * W, self._u(g, n, 1, 1) * H
            ax = self._u(g, n, 1, 1, lo=0.10, hi=0.22) * W
            ay = self._u(g, n, 1, 1, lo=0.10, hi=0.22) * H
            use = self._u(g, n, 1, 1) < (1.0 if i < 2 else 0.5)
            dark |= use & (((xx - cx) / ax) ** 2 + ((yy - cy) / ay) ** 2 <= 1.0)
        scene = torch.where(dark, scene * 0.2, scene)
        # disparity: plane plus six bumps in [0, dmax]
        p0 = self._u(g, n, 1, 1, lo=0.10, hi=0.30) * dmax
        p1 = self._u(g, n, 1, 1, lo=0.45, hi=0.65) * dmax
        ty = self._u(g, n, 1, 1, lo=-0.10, hi=0.10) * dmax
        d = p0 + (p1 - p0) * xx / max(W - 1, 1) + ty * (yy / max(H - 1, 1) - 0.5)
        for _ in range(6):
            cx, cy = self._u(g, n, 1, 1) * W, self._u(g, n, 1, 1) * H
            a = self._u(g, n, 1, 1, lo=-0.2, hi=0.2) * dmax
            sg = self._u(g, n, 1, 1, lo=0.05, hi=0.12) * W
            d = d + a * torch.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * sg * sg))
        d = d.clamp(0.0, dmax)
        # views
        xr = xx.expand(n, H, W)
        right = _interp_rows(scene, xr + d)
        flat_r = _interp_rows(flat.float(), xr + d) > 0.5
        left = scene + torch.randn(n, H, W, generator=g, device=self.device) * flat
        right = right + torch.randn(n, H, W, generator=g, device=self.device) * flat_r
        right = right + torch.randn(n, H, W, generator=g, device=self.device) * 2.0
        for _ in range(10):
            cx, cy = self._u(g, n, 1, 1) * W, self._u(g, n, 1, 1) * H
            rad = self._u(g, n, 1, 1, lo=5.0, hi=20.0)
            right = right + 400.0 * torch.exp(-((xx - cx) ** 2 + (yy - cy) ** 2)
                                              / (2 * (rad / 1.5) ** 2))
        # ground truth on the left grid: D_l(x) = D_r(x - D_l(x))
        dl = d.clone()
        for _ in range(10):
            dl = _interp_rows(d, xr - dl)
        dl = torch.where(xr - dl < 0, torch.full_like(dl, float("nan")), dl)
        to_u8 = lambda v: v.round().clamp(0, 255).to(torch.uint8)  # noqa: E731
        return to_u8(left), to_u8(right), dl
