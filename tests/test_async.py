"""GPU tests of the asynchronous entry point (hgrms_denoise_async /
hgrms_wait): the same bytes, k and converged flag as the synchronous call
and the oracle, several handles queued on one stream, and the one-call
limit per handle."""
import numpy as np
import pytest

from paper_1306_5390_gb300 import synth

pytestmark = pytest.mark.gpu


def noisy(rows, cols, density, seed):
    return synth.noisy_image(rows, cols, density, seed)[1]


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1306_5390_gb300 import build
    build.build()
    return torch


CASES = [((300, 517), 0.3, 10, 1, 32), ((257, 301), 0.5, 5, 2, 32), ((190, 250), 0.3, 20, 3, 9),
         ((64, 40), 0.1, 10, 4, 3), ((1, 300), 0.3, 10, 1, 5), ((6, 6), 0.9, 0, 2, 4)]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_async_matches_oracle_and_sync(oracle_mod, torch_cuda, case):
    from paper_1306_5390_gb300 import hgrms
    torch = torch_cuda
    (rows, cols), dens, alpha, beta, max_k = CASES[case]
    img = noisy(rows, cols, dens, 7000 + case)
    ref, k_ref, c_ref = oracle_mod.denoise(img, alpha, beta, max_k)
    with hgrms.Denoiser(0) as d:
        t = torch.from_numpy(img.copy()).cuda()
        d.denoise_async(t, alpha, beta, max_k)
        k = d.wait()
        assert k == k_ref and d.converged() == c_ref
        assert np.array_equal(t.cpu().numpy(), ref)
        # the synchronous call on the same handle afterwards agrees
        t2 = torch.from_numpy(img.copy()).cuda()
        assert d.denoise(t2, alpha, beta, max_k) == k_ref
        assert np.array_equal(t2.cpu().numpy(), ref)


def test_handles_queued_on_one_stream(oracle_mod, torch_cuda):
    """Three handles on the default stream, three calls queued before any
    wait (different beta, so different kernels and list-pass launches)."""
    from paper_1306_5390_gb300 import hgrms
    torch = torch_cuda
    imgs = [noisy(400, 333, 0.3, 7100 + i) for i in range(3)]
    refs = [oracle_mod.denoise(im, 10, b, 32) for im, b in zip(imgs, (1, 2, 3))]
    ds = [hgrms.Denoiser(0, timing=True) for _ in range(3)]
    try:
        for rep in range(2):
            ts = [torch.from_numpy(im.copy()).cuda() for im in imgs]
            for d, t, b in zip(ds, ts, (1, 2, 3)):
                d.denoise_async(t, 10, b, 32)
            ks = [d.wait() for d in ds]
            for t, k, d, (ref, k_ref, c_ref) in zip(ts, ks, ds, refs):
                assert k == k_ref and d.converged() == c_ref
                assert np.array_equal(t.cpu().numpy(), ref)
                st = d.stats()
                assert st["kernel_ms"] > 0 and st["passes"] >= k
    finally:
        for d in ds:
            d.close()


def test_one_outstanding_call_per_handle(torch_cuda):
    from paper_1306_5390_gb300 import hgrms
    torch = torch_cuda
    img = noisy(128, 128, 0.3, 7200)
    with hgrms.Denoiser(0) as d:
        assert hgrms.hgrms_wait(d.h) == hgrms.HGRMS_EINVAL  # nothing queued
        t = torch.from_numpy(img.copy()).cuda()
        u = torch.from_numpy(img.copy()).cuda()
        d.denoise_async(t, 10, 1, 32)
        assert hgrms.hgrms_denoise_async(d.h, u.data_ptr(), 128, 128, 10, 1, 32) == hgrms.HGRMS_EBUSY
        assert hgrms.hgrms_denoise(d.h, u.data_ptr(), 128, 128, 10, 1, 32) == hgrms.HGRMS_EBUSY
        k = d.wait()
        assert k >= 1
        assert hgrms.hgrms_wait(d.h) == hgrms.HGRMS_EINVAL  # already finished
        assert d.denoise(u, 10, 1, 32) == k
        assert torch.equal(t, u)


def test_async_host_memory(oracle_mod, torch_cuda):
    """Pageable host memory is rejected; page-locked host memory the device
    reads directly is accepted and gets the result."""
    from paper_1306_5390_gb300 import hgrms
    torch = torch_cuda
    img = noisy(200, 160, 0.3, 7300)
    ref, k_ref, _ = oracle_mod.denoise(img, 10, 1, 32)
    with hgrms.Denoiser(0) as d:
        pageable = img.copy()
        assert hgrms.hgrms_denoise_async(d.h, pageable.ctypes.data, 200, 160, 10, 1, 32) == hgrms.HGRMS_EINVAL
        pinned = torch.from_numpy(img.copy()).pin_memory()
        d.denoise_async(pinned, 10, 1, 32)
        assert d.wait() == k_ref
        assert np.array_equal(pinned.numpy(), ref)


def test_async_with_autotune_runs_synchronously(oracle_mod, torch_cuda):
    from paper_1306_5390_gb300 import hgrms
    torch = torch_cuda
    img = noisy(300, 300, 0.3, 7400)
    ref, k_ref, _ = oracle_mod.denoise(img, 10, 2, 32)
    with hgrms.Denoiser(0, autotune=True) as d:
        t = torch.from_numpy(img.copy()).cuda()
        d.denoise_async(t, 10, 2, 32)
        assert d.wait() == k_ref
        assert np.array_equal(t.cpu().numpy(), ref)
