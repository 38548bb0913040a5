"""Seeded synthetic rectified stereo pairs.

Convention: disparity D >= 0 with I_l(x, y) ~= I_r(x - D, y) on aligned rows
(the paper's pairs are rectified and vertically aligned, Sec. 3).

The generators stand in for the paper's Unity3D colon phantom and Hamlyn
in-vivo videos (Sec. 3), neither of which exists here. They reproduce the
properties the paper's method is about: textured tissue, textureless patches,
dark regions and non-Lambertian highlights seen by one camera only.

Every function takes an explicit seed and draws from numpy's PCG64, so the
same pair is produced on every machine.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy.ndimage import gaussian_filter

SEED_BASE = 2106_07136


@dataclass
class StereoPair:
    left: np.ndarray   # (H, W) uint8, or float32 for the exact sub-pixel fixtures
    right: np.ndarray  # same shape and dtype as left
    disp: np.ndarray   # (H, W) float64 ground truth on the left grid; NaN = unknown/occluded
    name: str = ""

    @property
    def shape(self):
        return self.left.shape


def pair_seed(config: int, index: int) -> int:
    """Seed of pair `index` of workload `config` (1-based config numbers)."""
    return SEED_BASE + 1000 * config + index


def _texture(rng, h, w, sigma=2.0, mean=128.0, std=40.0, ramp=40.0):
    """Uniform noise smoothed by a Gaussian, stretched to (mean, std), plus an x-ramp."""
    n = rng.uniform(0.0, 255.0, size=(h, w))
    s = gaussian_filter(n, sigma, mode="reflect")
    s = (s - s.mean()) / max(s.std(), 1e-12) * std + mean
    s = s + np.linspace(0.0, ramp, w)[None, :]
    return s


def _bumps(rng, h, w, count, amp, sig_lo, sig_hi):
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    f = np.zeros((h, w))
    for _ in range(count):
        cx = rng.uniform(0, w)
        cy = rng.uniform(0, h)
        a = rng.uniform(-amp, amp)
        s = rng.uniform(sig_lo, sig_hi)
        f += a * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2.0 * s * s))
    return f


def _interp_rows(img, xs):
    """Linear interpolation of each row of `img` at positions xs (same shape), clamped."""
    h, w = img.shape
    xs = np.clip(xs, 0.0, w - 1.0)
    i0 = np.floor(xs).astype(np.int64)
    i0 = np.minimum(i0, w - 2)
    t = xs - i0
    rows = np.arange(h)[:, None]
    return (1.0 - t) * img[rows, i0] + t * img[rows, i0 + 1]


def _warp_right(scene, d_right):
    """Right view: R(x_r, y) = scene(x_r + D(x_r, y), y), linear along x."""
    h, w = scene.shape
    xr = np.arange(w, dtype=np.float64)[None, :].repeat(h, axis=0)
    return _interp_rows(scene, xr + d_right)


def _left_ground_truth(d_right, iters=10):
    """Disparity on the left grid: solve D_l(x) = D_r(x - D_l(x)) by fixed point.

    Pixels whose match falls left of the right image (x - D_l < 0) are occluded
    in the right view and have no ground truth (NaN).
    """
    h, w = d_right.shape
    x = np.arange(w, dtype=np.float64)[None, :].repeat(h, axis=0)
    dl = d_right.copy()
    for _ in range(iters):
        dl = _interp_rows(d_right, x - dl)
    dl[(x - dl) < 0.0] = np.nan
    return dl


def _to_u8(img):
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


def _disparity_field(rng, h, w, dmax, n_bumps):
    """Plane plus Gaussian bumps, clamped to [0, dmax]."""
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    p0 = rng.uniform(0.10, 0.30) * dmax
    p1 = rng.uniform(0.45, 0.65) * dmax
    ty = rng.uniform(-0.10, 0.10) * dmax
    plane = p0 + (p1 - p0) * xx / max(w - 1, 1) + ty * (yy / max(h - 1, 1) - 0.5)
    sig_lo, sig_hi = 0.05 * w, 0.12 * w
    d = plane + _bumps(rng, h, w, n_bumps, 0.20 * dmax, sig_lo, sig_hi)
    return np.clip(d, 0.0, dmax)


def make_cfg1(seed: int = pair_seed(1, 0), h: int = 120, w: int = 160) -> StereoPair:
    """Small textured pair: 160x120, disparity 0..8 px (plane + 3 bumps).

    Left: uniform noise smoothed by sigma=2 px, stretched to mean 128 / std 40,
    plus a 0->40 gray x-ramp. Right: left warped by the field with linear
    interpolation, plus N(0, 2^2) gray noise. Both rounded to uint8.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    scene = _texture(rng, h, w)
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    d = 4.0 * xx / max(w - 1, 1) + _bumps(rng, h, w, 3, 2.0, 15.0, 30.0)
    d = np.clip(d, 0.0, 8.0)
    right = _warp_right(scene, d) + rng.normal(0.0, 2.0, size=(h, w))
    return StereoPair(_to_u8(scene), _to_u8(right), _left_ground_truth(d), f"cfg1/{seed}")


def make_cfg2(seed: int = pair_seed(2, 0), h: int = 480, w: int = 640,
              dmax: float | None = None) -> StereoPair:
    """Surgical-like pair: 640x480, disparity 0..64 px (plane + 6 bumps).

    - 20% of the scene area is textureless: rectangles of constant gray with
      independent N(0, 1) noise in each view;
    - dark regions: 2-3 ellipses covering about 15% of the area, scaled by 0.2
      in both views;
    - specular highlights in the right view only: 10 Gaussian blobs of radius
      5-20 px driven past 255 and clipped (saturated cores);
    - right view noise N(0, 2^2); both views rounded to uint8.
    `dmax` defaults to 64 at 640 px and scales as width/10 otherwise.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    if dmax is None:
        dmax = 64.0 if w == 640 else w / 10.0
    scene = _texture(rng, h, w)
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)

    flat = np.zeros((h, w), dtype=bool)
    while flat.mean() < 0.20:
        rw = int(rng.uniform(0.06, 0.20) * w)
        rh = int(rng.uniform(0.06, 0.20) * h)
        x0 = int(rng.integers(0, w - rw))
        y0 = int(rng.integers(0, h - rh))
        scene[y0:y0 + rh, x0:x0 + rw] = rng.uniform(60.0, 200.0)
        flat[y0:y0 + rh, x0:x0 + rw] = True

    dark = np.zeros((h, w), dtype=bool)
    n_dark = int(rng.integers(2, 4))
    for _ in range(n_dark):
        cx, cy = rng.uniform(0, w), rng.uniform(0, h)
        ax = rng.uniform(0.10, 0.22) * w
        ay = rng.uniform(0.10, 0.22) * h
        dark |= ((xx - cx) / ax) ** 2 + ((yy - cy) / ay) ** 2 <= 1.0
    scene = np.where(dark, scene * 0.2, scene)

    d = _disparity_field(rng, h, w, dmax, 6)
    right = _warp_right(scene, d)
    flat_r = _warp_right(flat.astype(np.float64), d) > 0.5
    left = scene + rng.normal(0.0, 1.0, size=(h, w)) * flat
    right = right + rng.normal(0.0, 1.0, size=(h, w)) * flat_r
    right = right + rng.normal(0.0, 2.0, size=(h, w))
    for _ in range(10):
        cx, cy = rng.uniform(0, w), rng.uniform(0, h)
        rad = rng.uniform(5.0, 20.0)
        right = right + 400.0 * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2.0 * (rad / 1.5) ** 2))
    return StereoPair(_to_u8(left), _to_u8(right), _left_ground_truth(d), f"cfg2/{seed}")


def make_pair(config: int, index: int = 0, **kw) -> StereoPair:
    seed = pair_seed(config, index)
    if config == 1:
        return make_cfg1(seed, **kw)
    if config == 2:
        return make_cfg2(seed, **kw)
    raise ValueError(f"no generator for workload {config}")


def make_batch(config: int, count: int, first_index: int = 0, **kw):
    """Stack `count` seeded pairs: returns (left[B,H,W] u8, right[B,H,W] u8, disp[B,H,W] f64)."""
    pairs = [make_pair(config, first_index + i, **kw) for i in range(count)]
    return (np.stack([p.left for p in pairs]), np.stack([p.right for p in pairs]),
            np.stack([p.disp for p in pairs]))


def make_linear_texture_pair(h, w, d, a0=0.5, a1=0.05, seed=SEED_BASE,
                             dtype=np.float32) -> StereoPair:
    """Float32 pair whose warp is exact under linear interpolation.

    L(x, y) = a(y) * x + b(y) with a(y) = a0 + a1 * y (linear in y, so the
    binomial pyramid and Sobel-x keep the form exactly away from the border)
    and random b(y). R(x, y) = L(x + d, y) analytically, so D = d everywhere.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    b = rng.uniform(0.0, 100.0, size=(h, 1))
    a = a0 + a1 * yy
    left = a * xx + b
    right = a * (xx + d) + b
    disp = np.full((h, w), float(d))
    return StereoPair(left.astype(dtype), right.astype(dtype), disp, f"linear/{d}")


def make_integer_shift_pair(h, w, k, seed=SEED_BASE) -> StereoPair:
    """uint8 pair with R(x) = L(x + k) exactly (no interpolation).

    The last k columns of R see texture outside the left image and are drawn
    from a wider smoothed-noise strip.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    wide = _to_u8(_texture(rng, h, w + k, ramp=0.0))
    left = wide[:, :w].copy()
    right = wide[:, k:k + w].copy()
    disp = np.full((h, w), float(k))
    disp[:, :k] = np.nan
    return StereoPair(left, right, disp, f"shift/{k}")


def make_flat_pair(h, w, value=100) -> StereoPair:
    """Constant images: no texture, every disparity explains the pair equally."""
    left = np.full((h, w), value, dtype=np.uint8)
    return StereoPair(left, left.copy(), np.full((h, w), np.nan), "flat")


class VideoStream:
    """Seeded synthetic stereo video (a stream of the serving workload).

    One textured scene (as in make_cfg2: textureless rectangles, dark
    regions, right-view highlights) wider than the frame; each frame pans the
    view by up to 2 px and moves each disparity bump centre by 1-3 px in its
    own direction, so consecutive disparity fields drift smoothly.
    """

    def __init__(self, seed, h, w, dmax=None, margin=64):
        self.rng = np.random.Generator(np.random.PCG64(seed))
        self.h, self.w, self.margin = h, w, margin
        self.dmax = dmax if dmax is not None else w / 10.0
        base = make_cfg2(seed=seed, h=h, w=w + margin, dmax=self.dmax)
        self.scene = base.left.astype(np.float64)
        rng = self.rng
        self.bumps = [dict(cx=rng.uniform(0, w), cy=rng.uniform(0, h),
                           a=rng.uniform(-0.2, 0.2) * self.dmax,
                           s=rng.uniform(0.05, 0.12) * w,
                           dx=rng.uniform(-1, 1), dy=rng.uniform(-1, 1))
                      for _ in range(6)]
        self.p0 = rng.uniform(0.10, 0.30) * self.dmax
        self.p1 = rng.uniform(0.45, 0.65) * self.dmax
        self.offset = margin // 2
        self.frame_index = 0

    def _field(self):
        yy, xx = np.mgrid[0:self.h, 0:self.w].astype(np.float64)
        d = self.p0 + (self.p1 - self.p0) * xx / max(self.w - 1, 1)
        for b in self.bumps:
            d += b["a"] * np.exp(-((xx - b["cx"]) ** 2 + (yy - b["cy"]) ** 2) / (2 * b["s"] ** 2))
        return np.clip(d, 0.0, self.dmax)

    def next(self) -> StereoPair:
        rng = self.rng
        if self.frame_index > 0:
            self.offset = int(np.clip(self.offset + rng.integers(-2, 3), 0, self.margin))
            for b in self.bumps:
                step = rng.uniform(1.0, 3.0)
                norm = max(np.hypot(b["dx"], b["dy"]), 1e-9)
                b["cx"] += step * b["dx"] / norm
                b["cy"] += step * b["dy"] / norm
        scene = self.scene[:, self.offset:self.offset + self.w]
        d = self._field()
        right = _warp_right(scene, d) + rng.normal(0.0, 2.0, size=(self.h, self.w))
        self.frame_index += 1
        return StereoPair(_to_u8(scene), _to_u8(right), _left_ground_truth(d),
                          f"video/{self.frame_index}")
