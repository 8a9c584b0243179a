"""Synthetic serial-crystallography frames.

The paper's datasets (lysozyme on a JUNGFRAU 4M, Se-SAD streptavidin on a
CSPAD) are not available, so seeded frames with the same detector shapes stand
in for them:

* CSPAD-like: 32 panels x 185 x 388 (§4.2 timing notes, 2-megapixel CSPAD);
* epix10k-like: 16 panels x 352 x 384;
* JUNGFRAU-like: 8 panels x 512 x 1024 (§4.2 timing notes).

Each frame: a Gaussian background N(mean, sd) clamped at 0, optional hot
pixels set to a fixed value, and Gaussian Bragg spots
A * exp(-r^2 / (2 sigma^2)) with A ~ U[amp_lo, amp_hi], sigma ~ U[sig_lo, sig_hi]
and a centre uniform over the panel (continuous).  All arithmetic is float64;
the frame is cast to float32 at the end.  Frame k of a recipe with seed s draws
from PCG64(SeedSequence([s, k])), so any frame can be regenerated alone.
"""
from __future__ import annotations

import concurrent.futures as cf
import dataclasses
import os

import numpy as np

GEOMETRIES = {
    "cspad": (32, 185, 388),
    "epix10k": (16, 352, 384),
    "jungfrau": (8, 512, 1024),
}


@dataclasses.dataclass(frozen=True)
class FrameRecipe:
    geometry: tuple
    bg_mean: float = 20.0
    bg_sd: float = 5.0
    peaks: tuple = ("fixed", 50)      # ("fixed", n) | ("uniform", lo, hi) | ("loguniform", hi)
    amp: tuple = (200.0, 2000.0)
    sigma: tuple = (1.0, 1.5)
    hot_fraction: float = 0.0
    hot_value: float = 5000.0
    seed: int = 1


RECIPES = {
    # one CSPAD-like frame, 50 peaks (the single-frame case)
    "cspad_single": FrameRecipe(GEOMETRIES["cspad"], peaks=("fixed", 50), seed=1),
    # 1,000 CSPAD-like frames with 20..100 peaks each (the batched workload)
    "cspad_batch": FrameRecipe(GEOMETRIES["cspad"], peaks=("uniform", 20, 100), seed=2),
    # epix10k-like frames: mean 30 sd 8, 1% hot pixels at 5,000, 0..300 peaks
    # with a heavy tail: n = floor(301^U) - 1
    "epix_hot": FrameRecipe(GEOMETRIES["epix10k"], bg_mean=30.0, bg_sd=8.0,
                            peaks=("loguniform", 300), hot_fraction=0.01, seed=3),
    # large-panel frames for mixed streams, 0..500 peaks
    "jungfrau_mixed": FrameRecipe(GEOMETRIES["jungfrau"], peaks=("uniform", 0, 500), seed=4),
    "cspad_mixed": FrameRecipe(GEOMETRIES["cspad"], peaks=("uniform", 0, 500), seed=5),
    "epix_mixed": FrameRecipe(GEOMETRIES["epix10k"], bg_mean=30.0, bg_sd=8.0,
                              peaks=("uniform", 0, 500), hot_fraction=0.01, seed=6),
}

_STAMP = 7  # spots are drawn over +-7 px (beyond 7 sigma of the widest spot)


def _n_peaks(rng: np.random.Generator, spec) -> int:
    kind = spec[0]
    if kind == "fixed":
        return int(spec[1])
    if kind == "uniform":
        return int(rng.integers(spec[1], spec[2] + 1))
    if kind == "loguniform":
        return int(np.floor((spec[1] + 1) ** rng.random())) - 1
    raise ValueError(f"unknown peak-count spec {spec!r}")


def make_frame(recipe: FrameRecipe, index: int, out: np.ndarray | None = None,
               return_truth: bool = False):
    """Frame `index` of `recipe` as float32[P][H][W] (written into `out` if given)."""
    P, H, W = recipe.geometry
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([recipe.seed, index])))
    img = rng.normal(recipe.bg_mean, recipe.bg_sd, size=(P, H, W))
    np.maximum(img, 0.0, out=img)
    if recipe.hot_fraction > 0:
        n_hot = int(round(recipe.hot_fraction * P * H * W))
        flat = img.reshape(-1)
        flat[rng.integers(0, flat.size, n_hot)] = recipe.hot_value
    n = _n_peaks(rng, recipe.peaks)
    panel = rng.integers(0, P, n)
    cy = rng.uniform(0, H, n)
    cx = rng.uniform(0, W, n)
    amp = rng.uniform(recipe.amp[0], recipe.amp[1], n)
    sig = rng.uniform(recipe.sigma[0], recipe.sigma[1], n)
    for k in range(n):
        y0, y1 = max(int(cy[k]) - _STAMP, 0), min(int(cy[k]) + _STAMP + 1, H)
        x0, x1 = max(int(cx[k]) - _STAMP, 0), min(int(cx[k]) + _STAMP + 1, W)
        yy = np.arange(y0, y1)[:, None] + 0.5 - cy[k]
        xx = np.arange(x0, x1)[None, :] + 0.5 - cx[k]
        img[panel[k], y0:y1, x0:x1] += amp[k] * np.exp(-(yy * yy + xx * xx) / (2 * sig[k] ** 2))
    if out is None:
        out = np.empty((P, H, W), np.float32)
    out[...] = img
    if return_truth:
        return out, dict(panel=panel, y=cy, x=cx, amp=amp, sigma=sig)
    return out


def make_batch(recipe: FrameRecipe, n_frames: int, first: int = 0) -> np.ndarray:
    P, H, W = recipe.geometry
    out = np.empty((n_frames, P, H, W), np.float32)
    for k in range(n_frames):
        make_frame(recipe, first + k, out=out[k])
    return out


def make_batch_threaded(recipe: FrameRecipe, n_frames: int, first: int = 0,
                        out: np.ndarray | None = None, workers: int | None = None) -> np.ndarray:
    """Same frames as make_batch; numpy releases the GIL while it draws."""
    P, H, W = recipe.geometry
    if out is None:
        out = np.empty((n_frames, P, H, W), np.float32)
    workers = workers or min(32, os.cpu_count() or 1)
    with cf.ThreadPoolExecutor(workers) as ex:
        list(ex.map(lambda k: make_frame(recipe, first + k, out=out[k]), range(n_frames)))
    return out
