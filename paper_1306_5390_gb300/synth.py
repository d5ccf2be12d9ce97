"""Seeded synthetic greyscale images with salt-and-pepper noise.

The paper evaluates on photographs from the Berkeley Segmentation Dataset
(Section 3), which is not available here.  These generators stand in for it:
smooth content (a sum of Gaussian bumps plus a linear gradient), optionally a
fine random texture and bounded uniform noise, then impulse ("salt and
pepper") corruption at a chosen density.

This module holds none of the denoiser's arithmetic.  It is the one piece of
code that both the CPU oracle tests and the CUDA path use, and it only draws
random numbers and builds images.  All draws come from numpy's PCG64 seeded
with ``seed_for(config, image)``; rows are generated in fixed blocks so that
even the 8192 x 8192 images need little temporary memory and the stream of
draws does not depend on available memory.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 1306539
_BLOCK_ROWS = 1024


def seed_for(config_index: int, image_index: int = 0) -> int:
    """Seed of image ``image_index`` in workload ``config_index``."""
    return SEED_BASE + config_index * 1_000_000 + image_index


def smooth_field(rows: int, cols: int, rng: np.random.Generator,
                 n_bumps: int = 8) -> np.ndarray:
    """Unscaled float64 field: ``n_bumps`` isotropic Gaussians + a gradient.

    Each bump has its centre uniform over the image, sigma uniform in
    [0.05, 0.3] * min(rows, cols) and amplitude uniform in [-1, 1].  The
    gradient has a uniform random direction and amplitude uniform in [0, 1]
    across the longer side.
    """
    m = float(min(rows, cols))
    cy = rng.uniform(0, rows, n_bumps)
    cx = rng.uniform(0, cols, n_bumps)
    sig = rng.uniform(0.05, 0.3, n_bumps) * m
    amp = rng.uniform(-1.0, 1.0, n_bumps)
    theta = rng.uniform(0.0, 2.0 * np.pi)
    gamp = rng.uniform(0.0, 1.0)
    span = float(max(rows, cols, 2) - 1)
    x = np.arange(cols, dtype=np.float64)
    y = np.arange(rows, dtype=np.float64)
    gx = np.exp(-((x[None, :] - cx[:, None]) ** 2) / (2.0 * sig[:, None] ** 2))
    gy = np.exp(-((y[None, :] - cy[:, None]) ** 2) / (2.0 * sig[:, None] ** 2))
    gy = gy * amp[:, None]
    out = np.empty((rows, cols), dtype=np.float64)
    grad_x = gamp * np.cos(theta) * x / span
    grad_y = gamp * np.sin(theta) * y / span
    for r0 in range(0, rows, _BLOCK_ROWS):
        r1 = min(rows, r0 + _BLOCK_ROWS)
        blk = gy[:, r0:r1].T @ gx  # sum over bumps of amp*gy*gx
        blk += grad_y[r0:r1, None]
        blk += grad_x[None, :]
        out[r0:r1] = blk
    return out


def texture_field(rows: int, cols: int, rng: np.random.Generator,
                  n_waves: int = 4, total_amp: float = 6.0) -> np.ndarray:
    """Sum of ``n_waves`` plane sinusoids, period uniform in [4, 32] px,
    random direction and phase; peak total amplitude ``total_amp`` grey levels."""
    out = np.zeros((rows, cols), dtype=np.float64)
    per = rng.uniform(4.0, 32.0, n_waves)
    ang = rng.uniform(0.0, 2.0 * np.pi, n_waves)
    ph = rng.uniform(0.0, 2.0 * np.pi, n_waves)
    x = np.arange(cols, dtype=np.float64)[None, :]
    y = np.arange(rows, dtype=np.float64)[:, None]
    a = total_amp / n_waves
    for i in range(n_waves):
        kx = 2.0 * np.pi * np.cos(ang[i]) / per[i]
        ky = 2.0 * np.pi * np.sin(ang[i]) / per[i]
        out += a * np.sin(kx * x + ky * y + ph[i])
    return out


def scale_to_u8(field: np.ndarray, lo: float, hi: float) -> np.ndarray:
    """Min-max scale a float field to [lo, hi] (float64, not yet rounded)."""
    fmin = float(field.min())
    fmax = float(field.max())
    if fmax <= fmin:
        return np.full(field.shape, 0.5 * (lo + hi))
    out = field - fmin
    out *= (hi - lo) / (fmax - fmin)
    out += lo
    return out


def clean_image(rows: int, cols: int, seed: int, texture: bool = False,
                uniform_noise: int = 0) -> np.ndarray:
    """The noise-free uint8 image.

    Plain content is scaled to [20, 235].  With ``texture`` the smooth part is
    scaled to [26, 229] and a +/-6 grey-level texture is added (so the sum
    stays in [20, 235]).  With ``uniform_noise`` = u > 0, i.i.d. integers
    uniform in [-u, u] are added and the result clamped to [0, 255].
    Rounding is half-to-even.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    f = smooth_field(rows, cols, rng)
    if texture:
        v = scale_to_u8(f, 26.0, 229.0)
        v += texture_field(rows, cols, rng)
    else:
        v = scale_to_u8(f, 20.0, 235.0)
    img = np.rint(v)
    if uniform_noise > 0:
        for r0 in range(0, rows, _BLOCK_ROWS):
            r1 = min(rows, r0 + _BLOCK_ROWS)
            img[r0:r1] += rng.integers(-uniform_noise, uniform_noise + 1,
                                       size=(r1 - r0, cols))
    np.clip(img, 0, 255, out=img)
    return img.astype(np.uint8)


def add_salt_pepper(img: np.ndarray, density: float, seed: int) -> np.ndarray:
    """Impulse noise: each pixel independently, with probability ``density``,
    becomes 0 or 255 (each with probability 1/2).  Returns a new array."""
    rng = np.random.Generator(np.random.PCG64(seed ^ 0x5A5A5A5A))
    out = img.copy()
    rows, cols = img.shape
    for r0 in range(0, rows, _BLOCK_ROWS):
        r1 = min(rows, r0 + _BLOCK_ROWS)
        u = rng.random((r1 - r0, cols), dtype=np.float32)
        s = rng.random((r1 - r0, cols), dtype=np.float32)
        hit = u < density
        blk = out[r0:r1]
        blk[hit & (s < 0.5)] = 0
        blk[hit & (s >= 0.5)] = 255
    return out


def noisy_image(rows: int, cols: int, density: float, seed: int,
                texture: bool = False, uniform_noise: int = 0):
    """(clean, noisy) pair of uint8 arrays of shape (rows, cols)."""
    clean = clean_image(rows, cols, seed, texture=texture,
                        uniform_noise=uniform_noise)
    return clean, add_salt_pepper(clean, density, seed)


def random_image(rows: int, cols: int, seed: int, levels=None) -> np.ndarray:
    """Unstructured test image: i.i.d. uniform bytes, or i.i.d. draws from
    ``levels`` (a small palette) when given.  Used for fuzzing."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if levels is None:
        return rng.integers(0, 256, size=(rows, cols), dtype=np.uint8)
    lv = np.asarray(levels, dtype=np.uint8)
    return lv[rng.integers(0, len(lv), size=(rows, cols))]


# ---------------------------------------------------------------------------
# Workload descriptions (sizes and settings of the benchmark configurations).

def workload_256():
    """One 256 x 256 image, 10 % impulse noise, alpha 10, beta 1, max_k 32."""
    seed = seed_for(0, 0)
    clean, noisy = noisy_image(256, 256, 0.10, seed)
    return dict(name="256x256 sp10 a10 b1", clean=clean, noisy=noisy,
                alpha=10, beta=1, max_k=32, seed=seed)


def workload_bsds_like(n_images: int = 64, first: int = 0, last: int = None):
    """64 images, half 481 x 321 and half 321 x 481 (the BSDS shapes), with
    texture and +/-8 uniform noise; swept over impulse density
    {10,30,50,70,90} %, alpha {5,10,20} and beta {1,2}.  Yields one dict per
    (image, setting), for images first .. last - 1 (default all; each image
    comes from its own seed, so a slice holds the same images as the whole)."""
    dens = (0.10, 0.30, 0.50, 0.70, 0.90)
    for i in range(first, n_images if last is None else min(last, n_images)):
        rows, cols = (321, 481) if i % 2 == 0 else (481, 321)
        seed = seed_for(1, i)
        clean = clean_image(rows, cols, seed, texture=True, uniform_noise=8)
        for di, d in enumerate(dens):
            noisy = add_salt_pepper(clean, d, seed + 7919 * (di + 1))
            for a in (5, 10, 20):
                for b in (1, 2):
                    yield dict(name=f"{rows}x{cols} sp{int(d*100)} a{a} b{b}",
                               clean=clean, noisy=noisy, alpha=a, beta=b,
                               max_k=32, seed=seed, density=d, image=i)


def workload_8192(beta: int = 1, size: int = 8192):
    """One 8192 x 8192 image, 30 % impulse noise, alpha 10 (beta 1, 2 or 3)."""
    seed = seed_for(2, 0)
    clean, noisy = noisy_image(size, size, 0.30, seed)
    return dict(name=f"{size}x{size} sp30 a10 b{beta}", clean=clean,
                noisy=noisy, alpha=10, beta=beta, max_k=32, seed=seed)


def batch_shapes(n_images: int = 512, min_side: int = 128, max_side: int = 2048, seed: int = None):
    """Side lengths of the uneven batch: each side uniform in
    [min_side, max_side] (independently, so the aspect ratio is random)."""
    rng = np.random.Generator(np.random.PCG64(seed_for(3, 0) if seed is None else seed))
    return [(int(r), int(c)) for r, c in rng.integers(min_side, max_side + 1, size=(n_images, 2))]


def workload_batch(n_images: int = 512, min_side: int = 128, max_side: int = 2048, first: int = 0,
                   last: int = None):
    """The uneven batch: images with sides uniform in 128..2048, impulse
    density uniform in 5..70 %, alpha 10, beta 1, max_k 32.  Yields one dict
    per image (images first .. last - 1, default all; each is generated from
    its own seed, so a slice is the same images as in the whole batch)."""
    shapes = batch_shapes(n_images, min_side, max_side)
    for i in range(first, n_images if last is None else min(last, n_images)):
        rows, cols = shapes[i]
        seed = seed_for(3, 1 + i)
        rng = np.random.Generator(np.random.PCG64(seed))
        density = float(rng.uniform(0.05, 0.70))
        clean, noisy = noisy_image(rows, cols, density, seed)
        yield dict(name=f"{rows}x{cols} sp{density * 100:.1f} a10 b1", clean=clean, noisy=noisy,
                   alpha=10, beta=1, max_k=32, seed=seed, density=density, image=i)
