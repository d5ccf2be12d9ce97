"""Handles on different streams whose calls overlap on the device.

Each call ends with one cooperative list-pass launch whose CTAs wait for one
another at every pass.  Two such launches running at the same time could
each hold SM slots that the other's CTAs need; the library therefore runs
the cooperative launches of all handles of a device one after another, in
the order they are issued, while the rest of the calls' work overlaps.  Here
two handles, each on its own stream, queue list-pass-heavy calls
(hgrms_denoise_async) before either is waited for, and a third handle runs
synchronous calls on the default stream meanwhile: every call must finish
(no HGRMS_ETIMEOUT) with the oracle's bytes, k and converged flag."""
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


def test_overlapping_calls_on_two_streams(oracle_mod, torch_cuda):
    import oracle_pool
    from paper_1306_5390_gb300 import build, hgrms
    torch = torch_cuda
    build.build()
    cases = [(2048, 2048, 0.30, 1, 0), (2048, 1536, 0.30, 2, 1), (1024, 1024, 0.5, 1, 2)]
    imgs, refs = [], []
    for rows, cols, dens, beta, si in cases:
        _, noisy = synth.noisy_image(rows, cols, dens, synth.seed_for(62, si))
        imgs.append(noisy)
        out, k, conv, _ = oracle_pool.banded_denoise(noisy, 10, beta, 32)
        refs.append((out, k, conv))
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    ds = [hgrms.Denoiser(0, cuda_stream=st.cuda_stream) for st in streams]
    dsync = hgrms.Denoiser(0)
    try:
        for rep in range(3):
            ts = [torch.from_numpy(im).cuda() for im in imgs]
            torch.cuda.synchronize()
            for d, t, (r, c, dens, beta, si) in zip(ds, ts, cases):
                d.denoise_async(t, 10, beta, 32)
            # meanwhile, synchronous calls of a third handle on the default stream
            k3 = dsync.denoise(ts[2], 10, cases[2][3], 32)
            ks = [d.wait() for d in ds]
            torch.cuda.synchronize()
            for i, (d, k) in enumerate(zip(ds, ks)):
                out, k_ref, c_ref = refs[i]
                assert k == k_ref and d.converged() == c_ref, (rep, i, k, k_ref)
                assert np.array_equal(ts[i].cpu().numpy(), out), (rep, i)
            assert k3 == refs[2][1] and np.array_equal(ts[2].cpu().numpy(), refs[2][0])
    finally:
        for d in ds:
            d.close()
        dsync.close()
