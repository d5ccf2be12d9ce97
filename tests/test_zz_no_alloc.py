"""hgrms_denoise_noalloc, the allocation-free entry point.

Callers whose device memory belongs to a pool or a host application they
cannot bypass, or whose latency-critical path cannot risk an allocation,
use hgrms_denoise_noalloc: its scratch lives in a fixed device array, so a
call allocates nothing.  A series of calls in a row, through the C ABI, must
each return exactly what the oracle computes for the same image, and what
hgrms_denoise returns for it (every pixel and k; the denoiser is integer
arithmetic, so the tolerance of all parity tests here is zero).  The series
shares the array: a large image followed by a small one (whose extent lies
inside the bytes the large call left behind), every window size with its own
fused kernel (beta 1, 2, 3, 7), an image at the documented 2048 x 2048 bound,
and a max_k far beyond convergence (the launches stop once the device reports
convergence).
"""
import numpy as np
import pytest

from paper_1306_5390_gb300 import synth

pytestmark = pytest.mark.gpu

# (rows, cols, density, alpha, beta, max_k, seed index)
CALLS = [
    (481, 321, 0.30, 10, 1, 32, 0),
    (700, 1000, 0.20, 10, 2, 32, 1),
    (481, 321, 0.30, 10, 1, 32, 0),     # the first image again, after a larger one
    (173, 95, 0.50, 10, 1, 32, 2),      # smaller still
    (400, 500, 0.30, 10, 3, 32, 3),
    (200, 300, 0.20, 10, 7, 32, 4),
    (2048, 2048, 0.30, 10, 1, 32, 5),   # the size that always fits
    (300, 301, 0.10, 10, 1, 100000, 6),  # converges long before max_k
    (96, 64, 0.30, 0, 1, 3, 7),         # alpha 0: every interior pixel takes the exact path
]


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _oracle(oracle_mod, noisy, alpha, beta, max_k):
    if noisy.size >= 1 << 22:
        import oracle_pool
        out, k, conv, _ = oracle_pool.banded_denoise(noisy, alpha, beta, max_k)
        return out, k, conv
    return oracle_mod.denoise(noisy, alpha, beta, max_k)


def test_noalloc_calls_in_a_row_match_oracle_and_denoise(oracle_mod, torch_cuda):
    torch = torch_cuda
    from paper_1306_5390_gb300 import build, hgrms
    build.build()
    with hgrms.Denoiser(0) as d:
        for i, (rows, cols, density, alpha, beta, max_k, si) in enumerate(CALLS):
            _, noisy = synth.noisy_image(rows, cols, density, synth.seed_for(40, si))
            ref, k_ref, conv_ref = _oracle(oracle_mod, noisy, alpha, beta, max_k)
            dev = torch.from_numpy(noisy).cuda()
            k_den = d.denoise(dev, alpha, beta, max_k)
            img = torch.from_numpy(noisy).cuda()
            torch.cuda.synchronize()
            k = hgrms.hgrms_denoise_noalloc(img.data_ptr(), rows, cols, alpha, beta, max_k, None)
            out = img.cpu().numpy()
            bad = int((out != ref).sum())
            assert k == k_ref and bad == 0, f"call {i}: k={k} vs oracle {k_ref}, {bad} pixels differ"
            assert (k < max_k) == conv_ref, f"call {i}: converged flag"
            assert k == k_den and torch.equal(img, dev), f"call {i}: differs from hgrms_denoise"


def test_noalloc_rejects_what_it_cannot_hold(torch_cuda):
    torch = torch_cuda
    from paper_1306_5390_gb300 import hgrms
    big = torch.zeros((4096, 4096), dtype=torch.uint8, device="cuda")
    assert hgrms.hgrms_denoise_noalloc(big.data_ptr(), 4096, 4096, 10, 1, 5, None) == hgrms.HGRMS_ETOOBIG
    host = np.zeros((16, 16), dtype=np.uint8)
    assert hgrms.hgrms_denoise_noalloc(host.ctypes.data, 16, 16, 10, 1, 5, None) == hgrms.HGRMS_EINVAL
    small = torch.zeros((16, 16), dtype=torch.uint8, device="cuda")
    assert hgrms.hgrms_denoise_noalloc(small.data_ptr(), 16, 16, 10, 0, 5, None) == hgrms.HGRMS_EINVAL
