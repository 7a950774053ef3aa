"""Seeded synthetic CCD frame sets shaped like the paper's workloads.

The paper reduces MITSuME frames: 16-bit CCD images, 60 s exposures, nine-point
dithering so that point sources move between exposures (Sec. 2.1), reduced by
bias, dark and flat calibration followed by alignment and co-adding (Sec. 2.2).
Its data are not available, so frame sets are synthesised here with the same
structure.  This module only *creates inputs*: it holds none of the reduction's
arithmetic, and both the CUDA path and the oracle consume what it returns.

Recipe (one frame set of ``n`` frames of ``W x H`` pixels):

* bias master  = 1000 ADU + N(0, 10) fixed pattern (FP32)
* dark master  = 0.05 ADU/s * (1 + 0.2 N(0,1)), clipped at 0 (FP32 rate)
* flat master  = (1 + 0.02 N(0,1)) * (1 - 0.05 (r / r_max)^2) (FP32)
* exposure     = 60 s for every frame
* sky          = Poisson, mean 300 e-, gain 1 e-/ADU
* stars        = 200 Gaussian PSFs (FWHM 3 px), lognormal flux with median
                 5e3 e- and sigma_ln = 1, fixed sky positions; frame k sees the
                 scene translated by its dither offset o_k
* read noise   = N(0, 10) ADU per pixel and frame
* cosmic rays  = 20 single pixels per frame of U(5e3, 3e4) ADU
* raw          = clip(round(bias + dark*t + flat*(sky + stars) + noise + CR),
                 0, 65535) as uint16

The returned offsets satisfy the sampling convention of the reduction: output
pixel (x, y) samples frame k at (x + dx_k, y + dy_k), so passing dx_k = o_k
lines the stars up again.
"""
from __future__ import annotations

import dataclasses

import numpy as np

FWHM_TO_SIGMA = 1.0 / 2.3548200450309493


@dataclasses.dataclass
class FrameSet:
    raw: np.ndarray        # [n, H, W] uint16
    bias: np.ndarray       # [H, W] float32, ADU
    dark: np.ndarray       # [H, W] float32, ADU/s
    flat: np.ndarray       # [H, W] float32, dimensionless
    exptime: np.ndarray    # [n] float32, s
    dx: np.ndarray         # [n] float64, px
    dy: np.ndarray         # [n] float64, px

    @property
    def n(self) -> int:
        return int(self.raw.shape[0])

    @property
    def H(self) -> int:
        return int(self.raw.shape[1])

    @property
    def W(self) -> int:
        return int(self.raw.shape[2])


def make_masters(W: int, H: int, rng: np.random.Generator):
    bias = (1000.0 + rng.normal(0.0, 10.0, size=(H, W))).astype(np.float32)
    dark = np.clip(0.05 * (1.0 + 0.2 * rng.normal(size=(H, W))), 0.0, None).astype(np.float32)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    cx, cy = 0.5 * (W - 1), 0.5 * (H - 1)
    r2 = (xx - cx) ** 2 + (yy - cy) ** 2
    r2max = max(cx * cx + cy * cy, 1.0)
    vignette = 1.0 - 0.05 * r2 / r2max
    flat = ((1.0 + 0.02 * rng.normal(size=(H, W))) * vignette).astype(np.float32)
    return bias, dark, flat


def _render_stars(img: np.ndarray, xs: np.ndarray, ys: np.ndarray, flux: np.ndarray,
                  sigma: float) -> None:
    """Adds point-sampled Gaussian PSFs to ``img`` (in electrons)."""
    H, W = img.shape
    rad = int(np.ceil(5.0 * sigma))
    norm = 1.0 / (2.0 * np.pi * sigma * sigma)
    for x0, y0, f in zip(xs, ys, flux):
        ix, iy = int(np.floor(x0)), int(np.floor(y0))
        xa, xb = max(ix - rad, 0), min(ix + rad + 2, W)
        ya, yb = max(iy - rad, 0), min(iy + rad + 2, H)
        if xa >= xb or ya >= yb:
            continue
        gx = np.arange(xa, xb, dtype=np.float64) - x0
        gy = np.arange(ya, yb, dtype=np.float64) - y0
        psf = np.exp(-0.5 * (gy[:, None] ** 2 + gx[None, :] ** 2) / (sigma * sigma))
        img[ya:yb, xa:xb] += f * norm * psf


def make_set(W: int, H: int, n: int, offset_range: float, seed: int, *,
             n_stars: int = 200, n_cr: int = 20, sky: float = 300.0,
             exptime: float = 60.0, fwhm: float = 3.0, read_noise: float = 10.0,
             masters=None) -> FrameSet:
    """One frame set (all frames share the masters), deterministic in ``seed``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if masters is None:
        bias, dark, flat = make_masters(W, H, rng)
    else:
        bias, dark, flat = masters
    sigma = fwhm * FWHM_TO_SIGMA
    # Scene: fixed star positions on the reference grid (a margin keeps most of
    # each PSF inside every dithered frame).
    sx = rng.uniform(0.0, W - 1.0, size=n_stars)
    sy = rng.uniform(0.0, H - 1.0, size=n_stars)
    sflux = rng.lognormal(mean=np.log(5e3), sigma=1.0, size=n_stars)
    dx = rng.uniform(-offset_range, offset_range, size=n) if offset_range > 0 else np.zeros(n)
    dy = rng.uniform(-offset_range, offset_range, size=n) if offset_range > 0 else np.zeros(n)
    t = np.full(n, exptime, dtype=np.float32)
    raw = np.empty((n, H, W), dtype=np.uint16)
    for k in range(n):
        e = rng.poisson(sky, size=(H, W)).astype(np.float64)
        # frame k shows the scene point p at detector position p + o_k
        _render_stars(e, sx + dx[k], sy + dy[k], sflux, sigma)
        adu = bias.astype(np.float64) + dark.astype(np.float64) * float(t[k]) \
            + flat.astype(np.float64) * e + rng.normal(0.0, read_noise, size=(H, W))
        cx = rng.integers(0, W, size=n_cr)
        cy = rng.integers(0, H, size=n_cr)
        adu[cy, cx] += rng.uniform(5e3, 3e4, size=n_cr)
        raw[k] = np.clip(np.rint(adu), 0, 65535).astype(np.uint16)
    return FrameSet(raw=raw, bias=bias, dark=dark, flat=flat, exptime=t,
                    dx=dx.astype(np.float64), dy=dy.astype(np.float64))


def make_const_set(W: int, H: int, n: int, raw_value: int, bias: float, dark: float,
                   flat: float, exptime: float, dx=None, dy=None) -> FrameSet:
    """Constant frames and masters (closed-form cases)."""
    dx = np.zeros(n) if dx is None else np.asarray(dx, dtype=np.float64)
    dy = np.zeros(n) if dy is None else np.asarray(dy, dtype=np.float64)
    return FrameSet(raw=np.full((n, H, W), raw_value, dtype=np.uint16),
                    bias=np.full((H, W), bias, dtype=np.float32),
                    dark=np.full((H, W), dark, dtype=np.float32),
                    flat=np.full((H, W), flat, dtype=np.float32),
                    exptime=np.full(n, exptime, dtype=np.float32), dx=dx, dy=dy)


# Named workloads: sizes follow the paper's frame geometry and the benchmark
# configurations of this library.
def workload_small(seed: int = 11486000) -> FrameSet:
    """5 frames of 512x512, offsets in +-5 px (bilinear case)."""
    return make_set(512, 512, 5, 5.0, seed)


def workload_bands(seed: int = 11486001, W: int = 1024, H: int = 1024, n: int = 10,
                   bands: int = 3, offset_range: float = 10.0) -> list[FrameSet]:
    """3 bands x 10 frames of 1024x1024, one master set per band (spline case)."""
    return [make_set(W, H, n, offset_range, seed + 7919 * b) for b in range(bands)]


def batch_shapes(seed: int = 11486003, nsets: int = 64):
    """Frame counts U{3..40} and sizes from {512^2, 1024^2, 2048^2, 4096^2}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = rng.integers(3, 41, size=nsets)
    sides = rng.choice(np.array([512, 1024, 2048, 4096]), size=nsets)
    return [(int(n), int(s), int(s)) for n, s in zip(ns, sides)]


# ---------------------------------------------------------------------------
# Device-side generator for the large benchmark workloads.  Same recipe, drawn
# with torch's generator on the GPU (a different random stream than numpy's),
# so multi-GB sets are created in milliseconds instead of minutes.
# ---------------------------------------------------------------------------
def make_set_torch(W: int, H: int, n: int, offset_range: float, seed: int, device,
                   n_stars: int = 200, n_cr: int = 20, sky: float = 300.0,
                   exptime: float = 60.0, fwhm: float = 3.0, read_noise: float = 10.0,
                   masters=None, raw_out=None):
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    gh = np.random.Generator(np.random.PCG64(seed))
    f32 = torch.float32
    if masters is None:
        bias = 1000.0 + 10.0 * torch.randn((H, W), generator=g, device=device, dtype=f32)
        dark = torch.clamp(0.05 * (1.0 + 0.2 * torch.randn((H, W), generator=g, device=device,
                                                             dtype=f32)), min=0.0)
        yy = torch.arange(H, device=device, dtype=f32)[:, None]
        xx = torch.arange(W, device=device, dtype=f32)[None, :]
        cx, cy = 0.5 * (W - 1), 0.5 * (H - 1)
        r2 = (xx - cx) ** 2 + (yy - cy) ** 2
        vign = 1.0 - 0.05 * r2 / max(cx * cx + cy * cy, 1.0)
        flat = (1.0 + 0.02 * torch.randn((H, W), generator=g, device=device, dtype=f32)) * vign
    else:
        bias, dark, flat = masters
    sigma = fwhm * FWHM_TO_SIGMA
    sx = gh.uniform(0.0, W - 1.0, size=n_stars)
    sy = gh.uniform(0.0, H - 1.0, size=n_stars)
    sflux = gh.lognormal(mean=np.log(5e3), sigma=1.0, size=n_stars)
    dx = gh.uniform(-offset_range, offset_range, size=n) if offset_range > 0 else np.zeros(n)
    dy = gh.uniform(-offset_range, offset_range, size=n) if offset_range > 0 else np.zeros(n)
    t = np.full(n, exptime, dtype=np.float32)
    raw = raw_out if raw_out is not None else torch.empty((n, H, W), dtype=torch.uint16,
                                                          device=device)
    rad = int(np.ceil(5.0 * sigma))
    off = torch.arange(-rad, rad + 2, device=device, dtype=f32)
    norm = 1.0 / (2.0 * np.pi * sigma * sigma)
    for k in range(n):
        e = torch.poisson(torch.full((H, W), sky, device=device, dtype=f32), generator=g)
        px = torch.tensor(sx + dx[k], device=device, dtype=f32)
        py = torch.tensor(sy + dy[k], device=device, dtype=f32)
        fl = torch.tensor(sflux, device=device, dtype=f32)
        gx = torch.floor(px)[:, None] + off[None, :]          # [S, B]
        gy = torch.floor(py)[:, None] + off[None, :]
        wx = torch.exp(-0.5 * ((gx - px[:, None]) / sigma) ** 2)
        wy = torch.exp(-0.5 * ((gy - py[:, None]) / sigma) ** 2)
        vals = (fl * norm)[:, None, None] * wy[:, :, None] * wx[:, None, :]
        ix = gx.long()[:, None, :].expand_as(vals)
        iy = gy.long()[:, :, None].expand_as(vals)
        ok = (ix >= 0) & (ix < W) & (iy >= 0) & (iy < H)
        e.view(-1).index_add_(0, (iy * W + ix)[ok], vals[ok])
        adu = bias + dark * float(t[k]) + flat * e \
            + read_noise * torch.randn((H, W), generator=g, device=device, dtype=f32)
        cxs = torch.randint(0, W, (n_cr,), generator=g, device=device)
        cys = torch.randint(0, H, (n_cr,), generator=g, device=device)
        adu[cys, cxs] += 5e3 + 2.5e4 * torch.rand((n_cr,), generator=g, device=device)
        raw[k] = torch.clamp(torch.round(adu), 0, 65535).to(torch.int32).to(torch.uint16)
    return dict(raw=raw, bias=bias.contiguous(), dark=dark.contiguous(),
                flat=flat.contiguous(), exptime=t, dx=dx.astype(np.float64),
                dy=dy.astype(np.float64))
