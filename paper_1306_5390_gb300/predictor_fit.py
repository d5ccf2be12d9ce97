"""Fit the k-predictor's network (needs a CUDA device).

    python -m paper_1306_5390_gb300.predictor_fit --beta 1 --out predictor_b1.npy

Training pairs: seeded synthetic images (sides log-uniform in 64..2048,
random aspect, impulse density uniform in 0..80 %, alpha 10) and their k, computed
by the library's exact denoiser (max_k 32; bit-identical to the method's
definition).  Features (64 x 64 area means, 16-bin histogram) come from the
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


def training_images(n: int, seed: int):
    from paper_1306_5390_gb300 import synth
    rng = np.random.Generator(np.random.PCG64(seed))
    for i in range(n):
        r, c = (int(round(np.exp(v))) for v in rng.uniform(np.log(64), np.log(2048), size=2))
        density = float(rng.uniform(0.0, 0.8))
        yield synth.noisy_image(r, c, density, seed * 100003 + i)[1]


def labels_and_features(d, beta, imgs, torch, chunk=250):
    """k (exact denoiser) and features (x0, hist) of every image."""
    ks, x0s, hists = [], [], []
    for s0 in range(0, len(imgs), chunk):
        part = imgs[s0:s0 + chunk]
        dev = [torch.from_numpy(im).cuda() for im in part]
        _, x0, hist, _ = d.predict_k(beta, dev, features=True)
        ks.extend(d.denoise_batch(dev, 10, beta, 32))
        x0s.append(x0)
        hists.append(hist)
    return np.array(ks, dtype=np.float32), np.concatenate(x0s), np.concatenate(hists)


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--beta", type=int, default=1)
    p.add_argument("--n", type=int, default=8000)
    p.add_argument("--epochs", type=int, default=40)
    p.add_argument("--seed", type=int, default=5)
    p.add_argument("--out", default=os.path.join(HERE, "predictor_b1.npy"))
    args = p.parse_args(argv)
    import torch  # device memory for the training images
    from paper_1306_5390_gb300 import build, hgrms, synth
    build.build()
    d = hgrms.Denoiser(0)
    d.load_predictor(args.beta, np.zeros(hgrms.PREDICTOR_WEIGHTS, dtype=np.float32))
    imgs = list(training_images(args.n, args.seed))
    k, x0, hist = labels_and_features(d, args.beta, imgs, torch)
    n_train = int(0.9 * len(imgs))
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
    # Held-out error, with the library's own (BF16 tensor-core) inference.
    d.load_predictor(args.beta, w)
    held = imgs[n_train:]
    kh = np.concatenate([d.predict_k(args.beta, [torch.from_numpy(im).cuda() for im in held[s:s + 1000]])
                         for s in range(0, len(held), 1000)])
    uneven = [w_["noisy"] for w_ in synth.workload_batch(512, last=64)]
    dev_u = [torch.from_numpy(im).cuda() for im in uneven]
    ku = np.array(d.denoise_batch(dev_u, 10, args.beta, 32), dtype=np.float32)
    khu = d.predict_k(args.beta, dev_u)
    print(json.dumps({"beta": args.beta, "n": args.n, "held_out": len(held),
                      "held_out_mae": round(float(np.mean(np.abs(kh - k[n_train:]))), 3),
                      "uneven64_mae": round(float(np.mean(np.abs(khu - ku))), 3),
                      "k_mean_train": round(float(k.mean()), 3), "final_train_loss": round(float(loss), 3),
                      "out": args.out}))
    d.close()


if __name__ == "__main__":
    main()
