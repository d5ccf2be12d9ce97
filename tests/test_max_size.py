"""The largest image the C ABI accepts: 65536 x 65536 (2^32 pixels, both
sides at the header's limit), denoised in place on the device by
hgrms_denoise.

At this size the canvas offsets pass 2^31 and 2^32 bytes, the change-list
entries use every bit of their 16-bit row and column fields, and the
128-row fused tiles, the list-pass loop (two CTAs per SM) and the copy-out
all run.  Nothing here is faster than the oracle on 2^32 pixels, so the
oracle checks windows (tests/oracle_pool.window_denoise: a pixel's value
after t passes depends only on the image within t * beta of it, by
Algorithm 2's window and Section 2's iteration): twelve 128 x 128 windows,
among them the four corners, the rows whose canvas offsets straddle 2^31
and 2^32 bytes, and a tile seam, compared byte for byte.  A pass that
changed a window pixel changed the image, so changes in the windows at
every pass 1..max_k fix k = max_k and "not converged" exactly.  Over the
whole image, the border band (closer than beta to an edge) must be
unchanged.  The image tiles a 4096 x 4096 synthetic one (30 % impulses),
each 4096-row band shifted by its own column offset.
"""
import numpy as np
import pytest

from paper_1306_5390_gb300 import synth

pytestmark = pytest.mark.gpu

N = 65536
WIN = 128


def max_size_image():
    _, base = synth.noisy_image(4096, 4096, 0.30, synth.seed_for(70, 0))
    img = np.empty((N, N), dtype=np.uint8)
    for b in range(N // 4096):
        img[4096 * b:4096 * (b + 1)] = np.tile(np.roll(base, 331 * b + 17, axis=1), (1, N // 4096))
    return img


def windows(pitch_rows_2_31, pitch_rows_2_32):
    rng = np.random.Generator(np.random.PCG64(1306))
    w = [(0, 0), (0, N - WIN), (N - WIN, 0), (N - WIN, N - WIN),
         (pitch_rows_2_31 - WIN // 2, 30000), (pitch_rows_2_32 - WIN // 2, 12345),
         (pitch_rows_2_32 - WIN // 2, N - WIN), (114 * 287 - WIN // 2, 240 * 137 - WIN // 2)]
    for _ in range(4):
        w.append((int(rng.integers(0, N - WIN)), int(rng.integers(0, N - WIN))))
    return w


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_largest_image_windows_k_and_border(oracle_mod, torch_cuda):
    import oracle_pool
    from paper_1306_5390_gb300 import build, hgrms
    torch = torch_cuda
    build.build()
    img = max_size_image()
    # Canvas rows of about 65792 bytes (the width in whole 240-column tiles
    # plus padding, rounded to 128): the image rows near byte offsets 2^31
    # and 2^32 of the canvas.
    pitch = (16 + 274 * 240 + 16 + 127) // 128 * 128
    wins = windows((1 << 31) // pitch - 16, (1 << 32) // pitch - 16)
    with hgrms.Denoiser(0) as d:
        for beta, max_k in ((1, 12), (2, 6)):
            dev = torch.from_numpy(img).cuda()
            k = d.denoise(dev, 10, beta, max_k)
            torch.cuda.synchronize()
            out = dev.cpu().numpy()
            del dev
            assert d.stats()["tile_rows"] == 128 - 2 * (hgrms.hgrms_default_passes(beta) - 1) * beta
            per_pass = np.zeros(max_k, dtype=np.int64)
            for (y0, x0) in wins:
                ref, counts = oracle_pool.window_denoise(img, y0, x0, WIN, WIN, 10, beta, max_k)
                got = out[y0:y0 + WIN, x0:x0 + WIN]
                assert np.array_equal(got, ref), (beta, y0, x0, int((got != ref).sum()))
                per_pass += np.asarray(counts, dtype=np.int64)
            assert per_pass.min() > 0, per_pass.tolist()
            assert k == max_k and not d.converged()
            b = beta
            assert np.array_equal(out[:b], img[:b]) and np.array_equal(out[-b:], img[-b:])
            assert np.array_equal(out[:, :b], img[:, :b]) and np.array_equal(out[:, -b:], img[:, -b:])
            assert int((out[4096:4352] != img[4096:4352]).sum()) > 0
