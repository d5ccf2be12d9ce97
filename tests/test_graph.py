"""GPU tests of graph replay (HGRMS_OPT_GRAPH): a call whose arguments
match an earlier one replays the CUDA graph recorded for it, and the result
stays bit-identical to the oracle across repeated calls, parameter changes,
batches, asynchronous calls and calls the graph does not cover."""
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


def test_replay_matches_oracle(oracle_mod, torch_cuda):
    from paper_1306_5390_gb300 import hgrms
    torch = torch_cuda
    img = noisy(300, 411, 0.3, 8000)
    src = torch.from_numpy(img).cuda()
    t = torch.empty_like(src)
    with hgrms.Denoiser(0, timing=True) as d:
        d.set_option(hgrms.HGRMS_OPT_GRAPH, 1)
        for beta in (1, 2, 3):
            ref, k_ref, c_ref = oracle_mod.denoise(img, 10, beta, 32)
            for rep in range(3):
                t.copy_(src)
                k = d.denoise(t, 10, beta, 32)
                st = d.stats()
                assert st["graph"] == (2 if rep == 0 else 1)
                assert k == k_ref and d.converged() == c_ref
                assert np.array_equal(t.cpu().numpy(), ref)
                assert st["kernel_ms"] > 0  # launch times recorded inside the graph
        # another alpha: another graph, then replays again
        ref, k_ref, _ = oracle_mod.denoise(img, 20, 1, 32)
        for rep in range(2):
            t.copy_(src)
            assert d.denoise(t, 20, 1, 32) == k_ref
            assert d.stats()["graph"] == (2 if rep == 0 else 1)
            assert np.array_equal(t.cpu().numpy(), ref)


def test_replay_other_buffer_and_small_max_k(oracle_mod, torch_cuda):
    from paper_1306_5390_gb300 import hgrms
    torch = torch_cuda
    img = noisy(128, 200, 0.5, 8100)
    with hgrms.Denoiser(0) as d:
        d.set_option(hgrms.HGRMS_OPT_GRAPH, 1)
        for max_k in (0, 1, 3, 9):
            ref, k_ref, c_ref = oracle_mod.denoise(img, 10, 1, max_k)
            for rep in range(2):
                t = torch.from_numpy(img.copy()).cuda()  # a new buffer: a new graph unless the address repeats
                assert d.denoise(t, 10, 1, max_k) == k_ref and d.converged() == c_ref
                assert np.array_equal(t.cpu().numpy(), ref)


def test_replay_batch_and_async(oracle_mod, torch_cuda):
    from paper_1306_5390_gb300 import hgrms
    torch = torch_cuda
    imgs = [noisy(r, c, 0.3, 8200 + i) for i, (r, c) in enumerate([(100, 90), (33, 250), (200, 200), (5, 5)])]
    refs = [oracle_mod.denoise(im, 10, 2, 32) for im in imgs]
    srcs = [torch.from_numpy(im).cuda() for im in imgs]
    ts = [torch.empty_like(s) for s in srcs]
    with hgrms.Denoiser(0) as d:
        d.set_option(hgrms.HGRMS_OPT_GRAPH, 1)
        for rep in range(3):
            for t, s in zip(ts, srcs):
                t.copy_(s)
            ks = d.denoise_batch(ts, 10, 2, 32)
            assert d.stats()["graph"] == (2 if rep == 0 else 1)
            for t, k, (ref, k_ref, _) in zip(ts, ks, refs):
                assert k == k_ref and np.array_equal(t.cpu().numpy(), ref)
        for rep in range(3):
            ts[2].copy_(srcs[2])
            d.denoise_async(ts[2], 10, 2, 32)
            assert d.wait() == refs[2][1]
            assert d.stats()["graph"] == (2 if rep == 0 else 1)
            assert np.array_equal(ts[2].cpu().numpy(), refs[2][0])


def test_host_image_runs_without_graph(oracle_mod, torch_cuda):
    from paper_1306_5390_gb300 import hgrms
    img = noisy(150, 150, 0.3, 8300)
    ref, k_ref, _ = oracle_mod.denoise(img, 10, 1, 32)
    with hgrms.Denoiser(0) as d:
        d.set_option(hgrms.HGRMS_OPT_GRAPH, 1)
        for rep in range(2):
            out = img.copy()  # pageable host memory: staged by copies, no graph
            assert d.denoise(out, 10, 1, 32) == k_ref
            assert d.stats()["graph"] == 0
            assert np.array_equal(out, ref)


def test_graph_cache_keeps_eight(oracle_mod, torch_cuda):
    from paper_1306_5390_gb300 import hgrms
    torch = torch_cuda
    img = noisy(64, 64, 0.3, 8400)
    src = torch.from_numpy(img).cuda()
    t = torch.empty_like(src)
    with hgrms.Denoiser(0) as d:
        d.set_option(hgrms.HGRMS_OPT_GRAPH, 1)
        for alpha in range(1, 11):  # ten keys: the first two are dropped
            t.copy_(src)
            d.denoise(t, alpha, 1, 32)
            assert d.stats()["graph"] == 2
        for alpha, expect in ((10, 1), (3, 1), (1, 2)):
            ref, k_ref, _ = oracle_mod.denoise(img, alpha, 1, 32)
            t.copy_(src)
            assert d.denoise(t, alpha, 1, 32) == k_ref
            assert d.stats()["graph"] == expect
            assert np.array_equal(t.cpu().numpy(), ref)


def test_predicted_schedule_as_graph(oracle_mod, torch_cuda):
    """The predicted-k schedule recorded as a graph and replayed: the graph
    holds the predicted number of fused launches and then the list passes,
    which continue exactly where the device's convergence state says; bytes
    and k equal the oracle's for every call, and a repeated call replays."""
    from paper_1306_5390_gb300 import hgrms
    torch = torch_cuda
    imgs = [noisy(r, c, dens, 8500 + i) for i, (r, c, dens) in enumerate([(333, 250, 0.3), (129, 700, 0.6)])]
    refs = [oracle_mod.denoise(im, 10, 1, 32) for im in imgs]
    srcs = [torch.from_numpy(im).cuda() for im in imgs]
    ts = [torch.empty_like(s) for s in srcs]
    with hgrms.Denoiser(0) as d:
        try:
            d.load_predictor(1)
        except FileNotFoundError:
            pytest.skip("no fitted predictor weights")
        d.set_option(hgrms.HGRMS_OPT_PREDICT_K, 1)
        d.set_option(hgrms.HGRMS_OPT_GRAPH, 1)
        # (a call that grows the handle's buffers makes earlier graphs stale,
        # so each image is recorded and then replayed)
        for t, s, (ref, k_ref, _) in zip(ts, srcs, refs):
            for rep in range(2):
                t.copy_(s)
                assert d.denoise(t, 10, 1, 32) == k_ref
                st = d.stats()
                assert st["k_pred"] >= 0, st
                assert st["graph"] == (2 if rep == 0 else 1), st
                assert np.array_equal(t.cpu().numpy(), ref)
