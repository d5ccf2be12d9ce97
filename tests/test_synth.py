"""CPU checks of the seeded synthetic inputs (the stand-ins for the paper's
BSDS photographs): value ranges, impulse density and values, determinism,
the workload shapes and settings.  These are the properties the input
recipe states; none of the denoiser's arithmetic is involved."""
import math

import numpy as np

from paper_1306_5390_gb300 import synth


def test_seeds():
    assert synth.seed_for(0) == 1306539
    assert synth.seed_for(3, 7) == 1306539 + 3 * 1_000_000 + 7


def test_clean_image_range_and_determinism():
    a = synth.clean_image(200, 311, 12345)
    b = synth.clean_image(200, 311, 12345)
    c = synth.clean_image(200, 311, 12346)
    assert a.dtype == np.uint8 and a.shape == (200, 311)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.min() == 20 and a.max() == 235  # min-max scaled to [20, 235], rounded
    t = synth.clean_image(200, 311, 12345, texture=True)
    assert 20 <= t.min() and t.max() <= 235
    u = synth.clean_image(200, 311, 12345, texture=True, uniform_noise=8)
    d = u.astype(int) - t.astype(int)
    assert np.abs(d).max() <= 8 and 0 <= u.min() and u.max() <= 255


def test_smooth_content_has_few_alpha_edges():
    """The smooth content changes slowly: neighbouring clean pixels differ by
    less than alpha = 10 almost everywhere (what makes salt and pepper the
    only isolated values)."""
    a = synth.clean_image(256, 256, synth.seed_for(0, 0)).astype(int)
    dx = np.abs(np.diff(a, axis=1))
    dy = np.abs(np.diff(a, axis=0))
    assert (dx < 10).mean() > 0.99 and (dy < 10).mean() > 0.99


def test_salt_and_pepper_density_and_values():
    clean = synth.clean_image(512, 512, 999)
    for dens in (0.05, 0.3, 0.7, 0.9):
        noisy = synth.add_salt_pepper(clean, dens, 4242)
        hit = noisy != clean  # (clean values are in [20, 235], never 0 or 255)
        n = hit.size
        # binomial: within 5 standard deviations
        assert abs(hit.mean() - dens) < 5 * math.sqrt(dens * (1 - dens) / n)
        vals = noisy[hit]
        assert set(np.unique(vals).tolist()) <= {0, 255}
        salt = (vals == 255).mean()
        assert abs(salt - 0.5) < 5 * math.sqrt(0.25 / vals.size)
        assert np.array_equal(synth.add_salt_pepper(clean, dens, 4242), noisy)  # seeded


def test_workload_settings():
    w = synth.workload_256()
    assert w["noisy"].shape == (256, 256) and (w["alpha"], w["beta"], w["max_k"]) == (10, 1, 32)
    assert abs((w["noisy"] != w["clean"]).mean() - 0.10) < 0.01
    w = synth.workload_8192(2, size=1024)  # the 8192 recipe at a smaller size
    assert w["noisy"].shape == (1024, 1024) and (w["alpha"], w["beta"]) == (10, 2)
    assert abs((w["noisy"] != w["clean"]).mean() - 0.30) < 0.005
    it = synth.workload_bsds_like(2)
    first = [next(it) for _ in range(30)]
    assert {x["noisy"].shape for x in first} == {(321, 481)}
    assert {(x["density"], x["alpha"], x["beta"]) for x in first} == {
        (d, a, b) for d in (0.1, 0.3, 0.5, 0.7, 0.9) for a in (5, 10, 20) for b in (1, 2)}
    assert next(it)["noisy"].shape == (481, 321)


def test_uneven_batch():
    shapes = synth.batch_shapes(512)
    assert len(shapes) == 512
    sides = np.array(shapes)
    assert sides.min() >= 128 and sides.max() <= 2048
    assert sides.mean() > 900 and sides.mean() < 1250  # uniform in 128..2048: mean 1088
    ws = list(synth.workload_batch(512, last=3))
    assert [w["noisy"].shape for w in ws] == shapes[:3]
    for w in ws:
        assert 0.05 <= w["density"] <= 0.70 and (w["alpha"], w["beta"], w["max_k"]) == (10, 1, 32)
    # a slice gives the same images as the whole batch
    again = list(synth.workload_batch(512, first=1, last=2))
    assert np.array_equal(again[0]["noisy"], ws[1]["noisy"])
