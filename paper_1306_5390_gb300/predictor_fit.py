"""Fit the k-predictor's network (needs a CUDA device).

    python -m paper_1306_5390_gb300.predictor_fit --beta 1 --out predictor_b1.npy

Training pairs: seeded synthetic images (sides log-uniform in 64..2048,
random aspect, impulse density uniform in 0..80 %, alpha 10) and their k, computed
by the library's exact denoiser (max_k 32; bit-identical to the method's
definition).  The labels are written beside the weights (<out>_labels.npz:
k, n and the generator seed) so that a sample of them can be checked against
the CPU oracle without a GPU (tests/test_predictor_labels.py).  Features (64 x 64 area means, 16-bin histogram) come from the
library's own feature kernel, so training sees exactly what inference sees.
The network of hgrms_predictor_load (four 3 x 3 convolutions of 16 channels
with ReLU, channel means, a linear head on [means, histogram]) is fitted on
the device by hgrms_predictor_train (tensor-core forward and backward
convolutions, mean squared error on k, Adam) and written as float32 in the
order hgrms_predictor_load documents.  Prints the mean absolute k
error on held-out images and on the first images of the uneven
128..2048 workload.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
if os.path.dirname(HERE) not in sys.path:
    sys.path.insert(0, os.path.dirname(HERE))


def training_specs(n: int, seed: int):
    """(rows, cols, density, image seed) of the n training images."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        r, c = (int(round(np.exp(v))) for v in rng.uniform(np.log(64), np.log(2048), size=2))
        density = float(rng.uniform(0.0, 0.8))
        out.append((r, c, density, seed * 100003 + i))
    return out


def training_images(n: int, seed: int):
    from paper_1306_5390_gb300 import synth
    for r, c, density, s in training_specs(n, seed):
        yield synth.noisy_image(r, c, density, s)[1]


def _image(spec):
    from paper_1306_5390_gb300 import synth
    r, c, density, s = spec
    return synth.noisy_image(r, c, density, s)[1]


def labels_and_features(d, beta, specs, torch, pool, chunk=500):
    """k (exact denoiser) and features (x0, hist) of every image; the images
    are synthesised chunk by chunk in the process pool and dropped after
    use."""
    ks, x0s, hists = [], [], []
    for s0 in range(0, len(specs), chunk):
        part = pool.map(_image, specs[s0:s0 + chunk], chunksize=8)
        dev = [torch.from_numpy(im).cuda() for im in part]
        _, x0, hist, _ = d.predict_k(beta, dev, features=True)
        ks.extend(d.denoise_batch(dev, 10, beta, 32))
        x0s.append(x0)
        hists.append(hist)
    return np.array(ks, dtype=np.float32), np.concatenate(x0s), np.concatenate(hists)


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--beta", type=int, default=1)
    p.add_argument("--n", type=int, default=20000)
    p.add_argument("--epochs", type=int, default=40)
    p.add_argument("--seed", type=int, default=5)
    p.add_argument("--out", default=os.path.join(HERE, "predictor_b1.npy"))
    args = p.parse_args(argv)
    import multiprocessing as mp
    import torch  # device memory for the training images
    from paper_1306_5390_gb300 import build, hgrms, synth
    build.build()
    pool = mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1)))
    d = hgrms.Denoiser(0)
    d.load_predictor(args.beta, np.zeros(hgrms.PREDICTOR_WEIGHTS, dtype=np.float32))
    specs = training_specs(args.n, args.seed)
    k, x0, hist = labels_and_features(d, args.beta, specs, torch, pool)
    n_train = int(0.9 * len(specs))
    # Initial weights: He-normal convolutions, zero biases, a head that
    # starts at the mean k.
    rng = np.random.Generator(np.random.PCG64(args.seed))
    w0 = np.zeros(hgrms.PREDICTOR_WEIGHTS, dtype=np.float32)
    off = 0
    for cin in (1, 16, 16, 16):
        w0[off:off + 9 * cin * 16] = rng.normal(0.0, np.sqrt(2.0 / (9 * cin)), size=9 * cin * 16)
        off += 9 * cin * 16
    w0[-1] = float(k[:n_train].mean())
    # The fit runs on the device: forward, input and weight gradients of
    # every convolution on the tensor cores, Adam on CUDA cores.
    w, loss = d.train_predictor(w0, x0[:n_train], hist[:n_train], k[:n_train], epochs=args.epochs, batch=256,
                                lr=3e-3, seed=args.seed)
    assert w.size == hgrms.PREDICTOR_WEIGHTS
    np.save(args.out, w)
    np.savez_compressed(args.out.replace(".npy", "_labels.npz"), k=k.astype(np.int16), n=np.int64(args.n),
                        seed=np.int64(args.seed), beta=np.int64(args.beta), alpha=np.int64(10), max_k=np.int64(32))
    # Held-out error, with the library's own (BF16 tensor-core) inference.
    d.load_predictor(args.beta, w)
    kh = []
    for s0 in range(n_train, len(specs), 500):
        part = pool.map(_image, specs[s0:s0 + 500], chunksize=8)
        kh.append(d.predict_k(args.beta, [torch.from_numpy(im).cuda() for im in part]))
    kh = np.concatenate(kh)
    uneven = [w_["noisy"] for w_ in synth.workload_batch(512, last=64)]
    dev_u = [torch.from_numpy(im).cuda() for im in uneven]
    ku = np.array(d.denoise_batch(dev_u, 10, args.beta, 32), dtype=np.float32)
    khu = d.predict_k(args.beta, dev_u)
    pool.close()
    print(json.dumps({"beta": args.beta, "n": args.n, "held_out": len(kh),
                      "held_out_mae": round(float(np.mean(np.abs(kh - k[n_train:]))), 3),
                      "held_out_k_at_max_frac": round(float(np.mean(k[n_train:] >= 32)), 3),
                      "uneven64_mae": round(float(np.mean(np.abs(khu - ku))), 3),
                      "k_mean_train": round(float(k.mean()), 3), "final_train_loss": round(float(loss), 3),
                      "out": args.out}))
    d.close()


if __name__ == "__main__":
    main()
