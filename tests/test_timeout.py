"""The bounded device wait gives up cleanly (HGRMS_ETIMEOUT).

The list-pass launch separates passes with a grid-wide barrier whose wait
is bounded: after its poll limit a CTA records an error and returns instead
of waiting forever.  HGRMS_OPT_WAIT_TEST makes every barrier wait for one
arrival more than the launch has CTAs - an arrival that never comes - with a
short poll limit, so the wait runs out on purpose.  No CTA is left waiting
and nothing in flight is abandoned (a CTA has no outstanding asynchronous
work at the barrier), so the call returns HGRMS_ETIMEOUT and the handle and
the device stay usable: the next call on the same handle, with the option
off, must give the oracle's bytes and k.  The paper's Algorithms 1-2 have no
such wait; this checks the boundary's error contract.
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


@pytest.mark.parametrize("beta", [1, 2])
def test_barrier_wait_runs_out_then_handle_recovers(oracle_mod, torch_cuda, beta):
    from paper_1306_5390_gb300 import build, hgrms
    torch = torch_cuda
    build.build()
    _, noisy = synth.noisy_image(481, 321, 0.30, synth.seed_for(50, beta))
    ref, k_ref, c_ref = oracle_mod.denoise(noisy, 10, beta, 32)
    assert k_ref > hgrms.hgrms_default_passes(beta)  # list passes run after the first fused launch
    with hgrms.Denoiser(0) as d:
        t = torch.from_numpy(noisy).cuda()
        d.set_option(hgrms.HGRMS_OPT_WAIT_TEST, 2000)
        rc = hgrms.hgrms_denoise(d.h, t.data_ptr(), 481, 321, 10, beta, 32)
        assert rc == hgrms.HGRMS_ETIMEOUT, hgrms.strerror(rc)
        assert hgrms.hgrms_last_cuda_error(d.h) == 0
        torch.cuda.synchronize()  # the context is healthy
        # host image, the synchronous path with its copies: same error
        h = noisy.copy()
        assert hgrms.hgrms_denoise(d.h, h.ctypes.data, 481, 321, 10, beta, 32) == hgrms.HGRMS_ETIMEOUT
        d.set_option(hgrms.HGRMS_OPT_WAIT_TEST, 0)
        for _ in range(2):
            t = torch.from_numpy(noisy).cuda()
            k = d.denoise(t, 10, beta, 32)
            assert k == k_ref and d.converged() == c_ref
            assert np.array_equal(t.cpu().numpy(), ref)


def test_wait_test_option_range(torch_cuda):
    from paper_1306_5390_gb300 import hgrms
    with hgrms.Denoiser(0) as d:
        assert hgrms.hgrms_set_option(d.h, hgrms.HGRMS_OPT_WAIT_TEST, -1) == hgrms.HGRMS_EINVAL
        assert hgrms.hgrms_set_option(d.h, hgrms.HGRMS_OPT_WAIT_TEST, (1 << 22) + 1) == hgrms.HGRMS_EINVAL
        assert hgrms.hgrms_set_option(d.h, hgrms.HGRMS_OPT_WAIT_TEST, 0) == hgrms.HGRMS_OK
