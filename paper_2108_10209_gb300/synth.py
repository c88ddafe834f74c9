"""Seeded synthetic inputs (stand-ins for the paper's BSD68 / Set12 / FMD-Confocal images).

This module holds only input generation -- no step of the denoising method. Both the CUDA
path and the CPU oracle are fed the arrays it returns. Every generator takes an explicit
integer seed and uses numpy's PCG64, so an image is reproducible from (recipe, seed).

Recipes (the paper's datasets are not available; these mimic their shapes and noise models):
  blobs     32x32-style "cells": 6 Gaussian blobs (sigma 2-6 px, amplitude U(0.3, 0.9)) on 0.1.
  ellipses  microscopy-like cells: filled ellipses (semi-axes U(4, 20), angle U(0, pi),
            intensity U(0.2, 1.0), painter's order) on 0.05, blurred with a Gaussian of
            sigma 1.5 (reflect boundary, truncated at 4 sigma). 200 ellipses per 512x512,
            the count scaled with the area for other sizes.
  noise     Gaussian:          y = clean + N(0, sigma^2), not clipped (Methods: inputs are not
                               clipped).
            Poisson-Gaussian:  y = Poisson(peak * clean) / peak + N(0, read^2)  (FMD-Confocal-like
                               shot + read noise, renormalised by the photon peak).
  u16       quantisation of a noisy image to 16-bit integers, then /65535 (microscope output).
  volume    a live-cell-like Z-stack: ellipsoid "cells" (xy semi-axes U(4, 20), z semi-axis
            U(1.5, 6) slices, angle U(0, pi), intensity U(0.2, 1.0), painter's order) on 0.05,
            each slice blurred like `ellipses`, Poisson-Gaussian noise per slice (seeded per
            slice). 200 cells per 512x512 of slice area, times Z / 20.
"""
from __future__ import annotations

import numpy as np

try:  # scipy is present on both machines; the blur falls back to a separable numpy filter
    from scipy.ndimage import gaussian_filter as _gf
except Exception:  # pragma: no cover
    _gf = None


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def blobs(h: int = 32, w: int = 32, seed: int = 0, n: int = 6) -> np.ndarray:
    r = rng(seed)
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    img = np.full((h, w), 0.1)
    for _ in range(n):
        cy, cx = r.uniform(0, h), r.uniform(0, w)
        s = r.uniform(2.0, 6.0)
        a = r.uniform(0.3, 0.9)
        img += a * np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2 * s * s))
    return np.clip(img, 0.0, 1.0)


def _blur(img: np.ndarray, sigma: float) -> np.ndarray:
    if _gf is not None:
        return _gf(img, sigma, mode="reflect", truncate=4.0)
    rad = int(4.0 * sigma + 0.5)
    k = np.exp(-0.5 * (np.arange(-rad, rad + 1) / sigma) ** 2)
    k /= k.sum()
    p = np.pad(img, rad, mode="symmetric")
    p = np.apply_along_axis(lambda v: np.convolve(v, k, mode="valid"), 0, p)
    return np.apply_along_axis(lambda v: np.convolve(v, k, mode="valid"), 1, p)


def ellipses(h: int = 512, w: int = 512, seed: int = 0, n: int | None = None,
             blur: float = 1.5) -> np.ndarray:
    r = rng(seed)
    if n is None:
        n = max(1, int(round(200 * h * w / (512 * 512))))
    img = np.full((h, w), 0.05)
    for _ in range(n):
        cy, cx = r.uniform(0, h), r.uniform(0, w)
        a, b = r.uniform(4, 20), r.uniform(4, 20)
        th = r.uniform(0, np.pi)
        inten = r.uniform(0.2, 1.0)
        R = int(np.ceil(max(a, b))) + 1
        y0, y1 = max(0, int(cy) - R), min(h, int(cy) + R + 1)
        x0, x1 = max(0, int(cx) - R), min(w, int(cx) + R + 1)
        if y0 >= y1 or x0 >= x1:
            continue
        yy, xx = np.mgrid[y0:y1, x0:x1].astype(np.float64)
        dy, dx = yy - cy, xx - cx
        u = (dx * np.cos(th) + dy * np.sin(th)) / a
        v = (-dx * np.sin(th) + dy * np.cos(th)) / b
        m = u * u + v * v <= 1.0
        img[y0:y1, x0:x1][m] = inten
    if blur and blur > 0:
        img = _blur(img, blur)
    return np.clip(img, 0.0, 1.0)


def gaussian_noise(clean: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    return clean + rng(seed).normal(0.0, sigma, clean.shape)


def poisson_gaussian(clean: np.ndarray, peak: float, read: float, seed: int) -> np.ndarray:
    r = rng(seed)
    return r.poisson(peak * np.clip(clean, 0, None)) / peak + r.normal(0.0, read, clean.shape)


def to_u16(noisy: np.ndarray) -> np.ndarray:
    return np.clip(np.rint(noisy * 65535.0), 0, 65535).astype(np.uint16)


def from_u16(q: np.ndarray) -> np.ndarray:
    return q.astype(np.float64) / 65535.0


def psnr(a: np.ndarray, ref: np.ndarray, peak: float = 1.0) -> float:
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(ref, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10.0 * np.log10(peak * peak / mse)


# ---- the workloads -------------------------------------------------------------------------

def image_small(seed: int = 0):
    """32x32 blobs + Gaussian noise sigma 25/255 (the fixed 10-step parity case).
    Returns (clean, noisy) as float64; the noisy image is rounded to float32 so that both
    sides start from identical values."""
    clean = blobs(32, 32, seed=seed)
    noisy = gaussian_noise(clean, 25.0 / 255.0, seed=seed + 1000003)
    return clean, noisy.astype(np.float32).astype(np.float64)


def image_cells(h: int = 512, w: int = 512, sigma: float = 25.0 / 255.0, seed: int = 0):
    """Ellipse cells + Gaussian noise (the 512x512 plain FP32 workload and its relatives)."""
    clean = ellipses(h, w, seed=seed)
    noisy = gaussian_noise(clean, sigma, seed=seed + 1000003)
    return clean, noisy.astype(np.float32).astype(np.float64)


def image_cells_pg(h: int = 512, w: int = 512, peak: float = 30.0, read: float = 0.02,
                   seed: int = 0):
    """Ellipse cells + Poisson-Gaussian noise (photon peak, read-noise sigma)."""
    clean = ellipses(h, w, seed=seed)
    noisy = poisson_gaussian(clean, peak, read, seed=seed + 2000003)
    return clean, noisy.astype(np.float32).astype(np.float64)


def volume_cells(Z: int = 41, h: int = 1024, w: int = 1024, seed: int = 0, peak: float = 30.0,
                 read: float = 0.02, n: int | None = None):
    """(clean, noisy) Z-stacks of shape (Z, h, w); noisy is float32-representable."""
    r = rng(seed)
    if n is None:
        n = max(1, int(round(200 * h * w / (512 * 512) * Z / 20)))
    vol = np.full((Z, h, w), 0.05)
    for _ in range(n):
        cz, cy, cx = r.uniform(0, Z), r.uniform(0, h), r.uniform(0, w)
        a, b, c = r.uniform(4, 20), r.uniform(4, 20), r.uniform(1.5, 6)
        th = r.uniform(0, np.pi)
        inten = r.uniform(0.2, 1.0)
        R = int(np.ceil(max(a, b))) + 1
        y0, y1 = max(0, int(cy) - R), min(h, int(cy) + R + 1)
        x0, x1 = max(0, int(cx) - R), min(w, int(cx) + R + 1)
        if y0 >= y1 or x0 >= x1:
            continue
        yy, xx = np.mgrid[y0:y1, x0:x1].astype(np.float64)
        dy, dx = yy - cy, xx - cx
        u = (dx * np.cos(th) + dy * np.sin(th)) / a
        v = (-dx * np.sin(th) + dy * np.cos(th)) / b
        q = u * u + v * v
        for z in range(max(0, int(np.floor(cz - c))), min(Z, int(np.ceil(cz + c)) + 1)):
            t = 1.0 - ((z + 0.5 - cz) / c) ** 2
            if t > 0:
                vol[z, y0:y1, x0:x1][q <= t] = inten
    clean = np.stack([np.clip(_blur(vol[z], 1.5), 0.0, 1.0) for z in range(Z)])
    noisy = np.stack([poisson_gaussian(clean[z], peak, read, seed=seed + 7000003 + z)
                      for z in range(Z)])
    return clean, noisy.astype(np.float32).astype(np.float64)


BATCH_SIZES = ((256, 256), (512, 512), (768, 512), (1024, 768))


def batch_jobs(n: int = 64, seed: int = 3_000_000):
    """n independent jobs: sizes uniform over BATCH_SIZES (H, W), sigma U[15, 50]/255."""
    r = rng(seed)
    jobs = []
    for i in range(n):
        h, w = BATCH_SIZES[int(r.integers(0, len(BATCH_SIZES)))]
        sigma = float(r.uniform(15.0, 50.0)) / 255.0
        jobs.append(dict(h=h, w=w, sigma=sigma, seed=seed + 1 + i))
    return jobs


def serving_stream(n: int = 1000, rate: float = 10.0, seed: int = 4_000_000,
                   smin: int = 256, smax: int = 2048):
    """Poisson arrivals: side log-uniform in [smin, smax] rounded to even, square images;
    noise Gaussian sigma U[10, 50]/255 or Poisson-Gaussian with peak U(10, 100)."""
    r = rng(seed)
    t = np.cumsum(r.exponential(1.0 / rate, n))
    out = []
    for i in range(n):
        s = int(round(np.exp(r.uniform(np.log(smin), np.log(smax)))))
        s = max(2, s - (s % 2))
        if r.uniform() < 0.5:
            noise = dict(kind="gauss", sigma=float(r.uniform(10, 50)) / 255.0)
        else:
            noise = dict(kind="pg", peak=float(r.uniform(10, 100)), read=0.02)
        out.append(dict(t=float(t[i]), side=s, noise=noise, seed=seed + 1 + i))
    return out


def make_serving_image(req: dict) -> np.ndarray:
    """The u16-normalised noisy image of one serving request."""
    s = req["side"]
    clean = ellipses(s, s, seed=req["seed"])
    nz = req["noise"]
    if nz["kind"] == "gauss":
        noisy = gaussian_noise(clean, nz["sigma"], req["seed"] + 1000003)
    else:
        noisy = poisson_gaussian(clean, nz["peak"], nz["read"], req["seed"] + 2000003)
    return from_u16(to_u16(noisy)), clean
