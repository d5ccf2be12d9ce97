"""The k-predictor's training labels against the oracle (no GPU).

predictor_fit labels its training images with the library's exact denoiser
and stores the labels beside the fitted weights.  Here a fixed random sample
of those images is regenerated from the stored seed and denoised by the CPU
oracle (Algorithms 1-2 iterated as in Section 2, max_k 32): every sampled
label must equal the oracle's k.  Images up to 512 x 512 are sampled so the
check stays quick."""
import os

import numpy as np
import pytest

from paper_1306_5390_gb300 import synth

LABELS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1306_5390_gb300",
                      "predictor_b1_labels.npz")


@pytest.mark.skipif(not os.path.exists(LABELS), reason="no stored training labels")
def test_sampled_training_labels_equal_oracle_k(oracle_mod):
    from paper_1306_5390_gb300 import predictor_fit
    z = np.load(LABELS)
    n, seed = int(z["n"]), int(z["seed"])
    assert z["k"].shape == (n,) and n >= 20000
    specs = predictor_fit.training_specs(n, seed)
    small = [i for i, (r, c, _, _) in enumerate(specs) if r * c <= 512 * 512]
    rng = np.random.Generator(np.random.PCG64(12345))
    pick = sorted(rng.choice(small, size=40, replace=False).tolist())
    for i in pick:
        r, c, density, s = specs[i]
        noisy = synth.noisy_image(r, c, density, s)[1]
        _, k, _ = oracle_mod.denoise(noisy, int(z["alpha"]), int(z["beta"]), int(z["max_k"]))
        assert k == int(z["k"][i]), (i, r, c, density, k, int(z["k"][i]))
