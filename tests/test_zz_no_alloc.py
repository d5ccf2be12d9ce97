"""hgrms_denoise_noalloc, the allocation-free entry point, against hgrms_denoise.

Callers whose device memory belongs to a pool or a host application they
cannot bypass, or whose latency-critical path cannot risk an allocation,
use hgrms_denoise_noalloc: its scratch lives in a fixed device array, so a
call allocates nothing.  Two calls in a row, through the C ABI, must each
return exactly what hgrms_denoise returns for the same image (every pixel
and k; the denoiser is integer arithmetic, so the tolerance of all parity
tests here is zero).  The second call also shows that the contents the first
call leaves in the shared array do not leak into the next result.
"""
import numpy as np
import pytest

from paper_1306_5390_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_noalloc_matches_denoise_on_two_calls(torch_cuda):
    torch = torch_cuda
    from paper_1306_5390_gb300 import build, hgrms
    build.build()
    cases = [(481, 321, 0.30, 10, 1, 32), (700, 1000, 0.20, 10, 2, 32)]
    with hgrms.Denoiser(0) as d:
        for i, (rows, cols, density, alpha, beta, max_k) in enumerate(cases):
            _, noisy = synth.noisy_image(rows, cols, density, synth.seed_for(40, i))
            ref = torch.from_numpy(noisy).cuda()
            k_ref = d.denoise(ref, alpha, beta, max_k)
            img = torch.from_numpy(noisy).cuda()
            torch.cuda.synchronize()
            k = hgrms.hgrms_denoise_noalloc(img.data_ptr(), rows, cols, alpha, beta, max_k, None)
            assert k == k_ref, (i, k, k_ref)
            assert torch.equal(img, ref), f"call {i}: {int((img != ref).sum())} pixels differ"


def test_noalloc_rejects_what_it_cannot_hold(torch_cuda):
    torch = torch_cuda
    from paper_1306_5390_gb300 import hgrms
    big = torch.zeros((4096, 4096), dtype=torch.uint8, device="cuda")
    assert hgrms.hgrms_denoise_noalloc(big.data_ptr(), 4096, 4096, 10, 1, 5, None) == hgrms.HGRMS_ETOOBIG
    host = np.zeros((16, 16), dtype=np.uint8)
    assert hgrms.hgrms_denoise_noalloc(host.ctypes.data, 16, 16, 10, 1, 5, None) == hgrms.HGRMS_EINVAL
    small = torch.zeros((16, 16), dtype=torch.uint8, device="cuda")
    assert hgrms.hgrms_denoise_noalloc(small.data_ptr(), 16, 16, 10, 0, 5, None) == hgrms.HGRMS_EINVAL
