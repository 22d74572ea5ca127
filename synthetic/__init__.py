"""Seeded synthetic targets that stand in for the paper's test images.

The paper's error study (Section 5.2, Fig. 4) uses six 8-bit grayscale 256x256 images
from the USC-SIPI database. Those images are not available here and are not recreated.
These generators make target amplitudes of the same shape and range instead:

  * ``blob_target``: a sum of 16 Gaussian blobs, centres uniform over the raster (no
    wrap), sigma uniform in [4, 32] pixels scaled by min(H, W)/256, weights uniform in
    [0.25, 1], normalised to a maximum of 1.
  * ``noise_target``: band-limited noise, a complex Gaussian spectrum kept for
    |k| <= min(H, W)/16, transformed back with numpy's library FFT, real part, min-max
    scaled to [0, 1].

This module holds input generation only, none of the hologram method's arithmetic, so
both the oracle tests and the CUDA path may use it. Every output is float32 [H, W] and a
pure function of (H, W, seed).
"""

import numpy as np

BLOB_SEED_BASE = 1000
NOISE_SEED_BASE = 2000


def blob_target(H, W, seed, n_blobs=16):
    rng = np.random.Generator(np.random.PCG64(seed))
    scale = min(H, W) / 256.0
    cy = rng.uniform(0.0, H, n_blobs)
    cx = rng.uniform(0.0, W, n_blobs)
    sigma = rng.uniform(4.0, 32.0, n_blobs) * scale
    weight = rng.uniform(0.25, 1.0, n_blobs)
    y = np.arange(H, dtype=np.float64)[:, None]
    x = np.arange(W, dtype=np.float64)[None, :]
    t = np.zeros((H, W), dtype=np.float64)
    for b in range(n_blobs):
        d2 = (y - cy[b]) ** 2 + (x - cx[b]) ** 2
        t += weight[b] * np.exp(-d2 / (2.0 * sigma[b] ** 2))
    t /= t.max()
    return t.astype(np.float32)


def noise_target(H, W, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    spec = rng.standard_normal((H, W)) + 1j * rng.standard_normal((H, W))
    ky = np.fft.fftfreq(H) * H
    kx = np.fft.fftfreq(W) * W
    keep = (ky[:, None] ** 2 + kx[None, :] ** 2) <= (min(H, W) / 16.0) ** 2
    field = np.fft.ifft2(spec * keep).real
    field -= field.min()
    field /= field.max()
    return field.astype(np.float32)


def target(kind, H, W, index=0):
    """Target number ``index`` of a kind ('blob' or 'noise') with its standard seed."""
    if kind == "blob":
        return blob_target(H, W, BLOB_SEED_BASE + index)
    if kind == "noise":
        return noise_target(H, W, NOISE_SEED_BASE + index)
    raise ValueError(f"unknown target kind {kind!r}")


def random_field(H, W, seed):
    """Complex float64 Gaussian test field (for transform tests), a pure function of seed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((H, W)) + 1j * rng.standard_normal((H, W))
