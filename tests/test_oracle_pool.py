"""The banded, multi-process oracle driver used by the full-size parity tests
must give exactly what the single-process oracle gives on the whole image:
the output bytes, k, the converged flag and the per-pass change counts.  The
cases put band edges inside every window, converge before max_k (so that
bands run passes past convergence), stop at max_k, and use more bands than
workers and one row per band."""
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
