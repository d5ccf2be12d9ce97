"""The CPU oracle spread over all host cores (TEST INFRASTRUCTURE ONLY).

The oracle is plain single-threaded C; the full-size parity tests need it on
images of up to 67 M pixels, so these helpers run it in worker processes
(started with ``spawn``, so that no worker inherits a CUDA context).  Nothing
here does any of the method's arithmetic: every pass is ``oracle.one_pass``
or ``oracle.denoise``.

``banded_denoise`` - one large image, cut into horizontal bands.
    Band b owns rows [r0, r1).  It runs on a crop of rows [r0 - M, r1 + M)
    (clipped to the image), M = max_k * beta + beta.  One pass reads only the
    (2 beta + 1)^2 window of each pixel (Algorithms 1-2), so after t passes
    only the crop rows within t * beta of a cut crop edge can differ from the
    same rows of the whole image; the owned rows are exact after every pass up
    to max_k.  Each band reports, for every pass t = 1..max_k, how many of its
    owned pixels pass t changed.  The sums over the bands are the whole
    image's per-pass change counts, which fix k and the converged flag by the
    stopping rule of Section 2: the loop stops after the first pass that
    changes no pixel (converged, k = passes before it) or once max_k passes
    changed pixels.  A pass that changes nothing leaves a fixed point, so the
    owned rows after max_k passes are the whole image's final result in both
    cases, and every band can simply run max_k passes.

``window_denoise`` - one rectangular window of an image too large for the
    oracle (the same margin argument in both directions): the crop is the
    window grown by M pixels on every side (clipped to the image: a crop
    edge that is an image edge is exact as it is), its centre is exact after
    every pass up to max_k, and the per-pass change counts inside the window
    are lower bounds of the whole image's (a pass that changed a window
    pixel changed the image).

``batch_denoise`` / ``bsds_denoise`` - independent images of a workload, one
    task per image.  The worker regenerates the image from the workload's
    seed (synth), runs ``oracle.denoise`` and returns the result (with the
    noisy input for the uneven batch).
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np


def workers() -> int:
    return max(1, min(os.cpu_count() or 1, 64))


def _band(job):
    import oracle
    crop, own0, own1, alpha, beta, max_k = job
    img = crop
    counts = []
    for _ in range(max_k):
        nxt, _ = oracle.one_pass(img, alpha, beta)
        counts.append(int((nxt[own0:own1] != img[own0:own1]).sum()))
        img = nxt
    return img[own0:own1].copy(), counts


def banded_denoise(img: np.ndarray, alpha: int, beta: int, max_k: int, bands: int = 0):
    """The oracle's (out, k, converged, per-pass change counts) for a large
    image, computed band by band in parallel (see the module docstring)."""
    img = np.ascontiguousarray(img, dtype=np.uint8)
    rows = img.shape[0]
    if max_k == 0:
        return img.copy(), 0, False, []
    n = bands or workers()
    n = max(1, min(n, rows))
    edges = [rows * i // n for i in range(n + 1)]
    m = max_k * beta + beta
    jobs = []
    for i in range(n):
        r0, r1 = edges[i], edges[i + 1]
        c0, c1 = max(0, r0 - m), min(rows, r1 + m)
        jobs.append((img[c0:c1].copy(), r0 - c0, r1 - c0, alpha, beta, max_k))
    with mp.get_context("spawn").Pool(min(n, workers())) as pool:
        res = pool.map(_band, jobs, chunksize=1)
    out = np.concatenate([r[0] for r in res], axis=0)
    per_pass = [sum(r[1][t] for r in res) for t in range(max_k)]
    k, conv = max_k, False
    for t, c in enumerate(per_pass):
        if c == 0:
            k, conv = t, True
            break
    return out, k, conv, per_pass[:k + (1 if conv else 0)]


def _batch_image(job):
    import oracle
    from paper_1306_5390_gb300 import synth
    n_images, i, alpha, beta, max_k = job
    w = next(synth.workload_batch(n_images, first=i, last=i + 1))
    ref, k, conv = oracle.denoise(w["noisy"], alpha, beta, max_k)
    return w["noisy"], ref, k, conv


def batch_denoise(n_images: int, alpha: int = 10, beta: int = 1, max_k: int = 32):
    """[(noisy, oracle output, k, converged)] for every image of the uneven
    batch workload (synth.workload_batch), in image order."""
    jobs = [(n_images, i, alpha, beta, max_k) for i in range(n_images)]
    # Largest images first, so that the pool's tail is short.
    from paper_1306_5390_gb300 import synth
    shapes = synth.batch_shapes(n_images)
    order = sorted(range(n_images), key=lambda i: -shapes[i][0] * shapes[i][1])
    with mp.get_context("spawn").Pool(workers()) as pool:
        res = pool.map(_batch_image, [jobs[i] for i in order], chunksize=1)
    out = [None] * n_images
    for i, r in zip(order, res):
        out[i] = r
    return out


def _bsds_image(job):
    import oracle
    from paper_1306_5390_gb300 import synth
    n_images, i = job
    out = {}
    for w in synth.workload_bsds_like(n_images, first=i, last=i + 1):
        out[(w["density"], w["alpha"], w["beta"])] = oracle.denoise(w["noisy"], w["alpha"], w["beta"], w["max_k"])
    return out


def bsds_denoise(n_images: int = 64):
    """{(density, alpha, beta): [(oracle output, k, converged) per image]}
    for every run of the 481x321 / 321x481 sweep (synth.workload_bsds_like)."""
    with mp.get_context("spawn").Pool(workers()) as pool:
        res = pool.map(_bsds_image, [(n_images, i) for i in range(n_images)], chunksize=1)
    out = {}
    for per_image in res:
        for key, r in per_image.items():
            out.setdefault(key, []).append(r)
    return out


def window_denoise(img: np.ndarray, y0: int, x0: int, h: int, w: int, alpha: int, beta: int, max_k: int):
    """The oracle's bytes of img[y0:y0+h, x0:x0+w] after max_k passes and the
    number of that window's pixels each pass t = 1..max_k changed (see the
    module docstring), from a crop with a margin of max_k * beta + beta."""
    import oracle
    rows, cols = img.shape
    m = max_k * beta + beta
    cy0, cx0 = max(0, y0 - m), max(0, x0 - m)
    cy1, cx1 = min(rows, y0 + h + m), min(cols, x0 + w + m)
    cur = np.ascontiguousarray(img[cy0:cy1, cx0:cx1], dtype=np.uint8)
    sy, sx = y0 - cy0, x0 - cx0
    counts = []
    for _ in range(max_k):
        nxt, _ = oracle.one_pass(cur, alpha, beta)
        counts.append(int((nxt[sy:sy + h, sx:sx + w] != cur[sy:sy + h, sx:sx + w]).sum()))
        cur = nxt
    return cur[sy:sy + h, sx:sx + w].copy(), counts
