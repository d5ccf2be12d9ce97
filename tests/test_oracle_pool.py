"""The banded, multi-process oracle driver used by the full-size parity tests
must give exactly what the single-process oracle gives on the whole image:
the output bytes, k, the converged flag and the per-pass change counts.  The
cases put band edges inside every window, converge before max_k (so that
bands run passes past convergence), stop at max_k, and use more bands than
workers and one row per band.  The window form (used where even the banded
oracle would take minutes) is pinned the same way: windows that tile the
image, with edges inside every window position and at the image's edges,
give the whole image's bytes, and their per-pass change counts sum to the
whole image's."""
import numpy as np
import pytest

from paper_1306_5390_gb300 import synth


@pytest.mark.parametrize("rows,cols,density,beta,max_k,bands", [
    (300, 257, 0.30, 1, 32, 7),
    (301, 190, 0.50, 2, 6, 5),
    (160, 150, 0.30, 3, 32, 4),
    (97, 120, 0.70, 1, 3, 97),
    (90, 64, 0.20, 2, 0, 3),
])
def test_banded_equals_whole_image(oracle_mod, rows, cols, density, beta, max_k, bands):
    import oracle_pool
    _, noisy = synth.noisy_image(rows, cols, density, synth.seed_for(60, rows + beta))
    ref, k_ref, c_ref, ch_ref = oracle_mod.denoise(noisy, 10, beta, max_k, return_changes=True)
    out, k, conv, ch = oracle_pool.banded_denoise(noisy, 10, beta, max_k, bands=bands)
    assert (k, conv) == (k_ref, c_ref)
    assert ch == ch_ref
    assert np.array_equal(out, ref)


def test_batch_driver_matches_single_images(oracle_mod):
    import oracle_pool
    res = oracle_pool.batch_denoise(3)
    for i, w in enumerate(synth.workload_batch(3)):
        noisy, ref, k, conv = res[i]
        assert np.array_equal(noisy, w["noisy"])
        r2, k2, c2 = oracle_mod.denoise(w["noisy"], 10, 1, 32)
        assert (k, conv) == (k2, c2) and np.array_equal(ref, r2)


def test_bsds_driver_matches_single_images(oracle_mod):
    import oracle_pool
    res = oracle_pool.bsds_denoise(2)
    n = 0
    for w in synth.workload_bsds_like(2):
        key = (w["density"], w["alpha"], w["beta"])
        ref, k, conv = res[key][w["image"]]
        r2, k2, c2 = oracle_mod.denoise(w["noisy"], w["alpha"], w["beta"], w["max_k"])
        assert (k, conv) == (k2, c2) and np.array_equal(ref, r2)
        n += 1
    assert n == 60 and all(len(v) == 2 for v in res.values())


@pytest.mark.parametrize("rows,cols,density,alpha,beta,max_k,wh,ww,si", [
    (200, 230, 0.30, 10, 1, 12, 37, 50, 201),
    (150, 161, 0.30, 10, 2, 6, 64, 29, 152),
    (120, 97, 0.05, 10, 1, 40, 23, 31, 500),   # converges at k = 3
    (90, 100, 0.50, 10, 3, 4, 90, 13, 93),
    (90, 100, 0.30, 0, 2, 6, 30, 33, 91),      # alpha 0: changes spread beta pixels per pass
])
def test_windows_tile_the_whole_image(oracle_mod, rows, cols, density, alpha, beta, max_k, wh, ww, si):
    import oracle_pool
    _, noisy = synth.noisy_image(rows, cols, density, synth.seed_for(61, si))
    ref, k_ref, c_ref, ch_ref = oracle_mod.denoise(noisy, alpha, beta, max_k, return_changes=True)
    out = np.zeros_like(noisy)
    per_pass = np.zeros(max_k, dtype=np.int64)
    for y0 in range(0, rows, wh):
        for x0 in range(0, cols, ww):
            h, w = min(wh, rows - y0), min(ww, cols - x0)
            win, counts = oracle_pool.window_denoise(noisy, y0, x0, h, w, alpha, beta, max_k)
            out[y0:y0 + h, x0:x0 + w] = win
            per_pass += np.asarray(counts, dtype=np.int64)
    assert np.array_equal(out, ref)
    runs = len(ch_ref)
    assert per_pass[:runs].tolist() == ch_ref
    assert not per_pass[runs:].any()  # passes past convergence change nothing
    if si == 500:
        assert c_ref and k_ref < max_k
