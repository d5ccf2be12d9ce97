"""GPU parity of the batched schedule (hgrms_denoise_batch) against the oracle.

A batch runs every image through one fused launch and one persistent
list-pass launch; each image's output and k must equal what the oracle
computes for that image alone (integer arithmetic: tolerance zero), and
image i converged exactly when k_i < max_k.  Covers uneven sizes with
degenerate images in the same batch, every beta with a compiled default
kernel, alpha and max_k edge values, chunking by memory budget and by the
32-bit change-list packing, list overflow, host pointers, and all 512 images of the uneven
128..2048 workload at full size.
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


@pytest.fixture(scope="module")
def den(torch_cuda):
    from paper_1306_5390_gb300 import build, hgrms
    build.build()
    d = hgrms.Denoiser(0)
    yield d
    d.close()


def mixed_batch(n, seed, max_side=400):
    """Uneven sizes (including 1 x 1, thin and tiny images) and impulse
    densities from 5 to 90 %."""
    rng = np.random.Generator(np.random.PCG64(seed))
    fixed = [(1, 1), (2, 9), (3, 3), (5, 5), (1, 300), (300, 2), (17, 241), (241, 17)]
    imgs = []
    for i in range(n):
        if i < len(fixed):
            r, c = fixed[i]
        else:
            r, c = (int(v) for v in rng.integers(6, max_side + 1, size=2))
        density = float(rng.uniform(0.05, 0.90))
        imgs.append(synth.noisy_image(r, c, density, seed * 1000 + i)[1])
    return imgs


def run_batch(den, torch, imgs, alpha, beta, max_k, host=False, **opts):
    from paper_1306_5390_gb300 import hgrms
    den.set_option(hgrms.HGRMS_OPT_KERNEL, 0)
    den.set_option(hgrms.HGRMS_OPT_PASSES, opts.get("passes", 0))
    den.set_option(hgrms.HGRMS_OPT_LIST_CAP, opts.get("list_cap", 0))
    den.set_option(hgrms.HGRMS_OPT_BATCH_MB, opts.get("batch_mb", 0))
    den.set_option(hgrms.HGRMS_OPT_RELAUNCH_PPM, opts.get("relaunch_ppm", 0))
    if host:
        work = [np.ascontiguousarray(im).copy() for im in imgs]
        ks = den.denoise_batch(work, alpha, beta, max_k)
        outs = work
    else:
        work = [torch.from_numpy(np.ascontiguousarray(im).copy()).cuda() for im in imgs]
        ks = den.denoise_batch(work, alpha, beta, max_k)
        outs = [t.cpu().numpy() for t in work]
    conv = den.converged()
    for opt in (hgrms.HGRMS_OPT_PASSES, hgrms.HGRMS_OPT_LIST_CAP, hgrms.HGRMS_OPT_BATCH_MB,
                hgrms.HGRMS_OPT_RELAUNCH_PPM):
        den.set_option(opt, 0)
    return outs, ks, conv


def check(oracle_mod, imgs, outs, ks, conv, alpha, beta, max_k, label=""):
    all_conv = True
    for i, (im, out, k) in enumerate(zip(imgs, outs, ks)):
        ref, k_ref, c_ref = oracle_mod.denoise(im, alpha, beta, max_k)
        bad = int((out != ref).sum())
        assert bad == 0 and k == k_ref, (
            f"{label} image {i} {im.shape} a={alpha} b={beta} max_k={max_k}: {bad} pixels differ, k={k} vs {k_ref}")
        assert (k < max_k) == bool(c_ref), (label, i, k, max_k, c_ref)
        all_conv &= bool(c_ref)
    assert conv == all_conv


@pytest.mark.parametrize("beta", [1, 2, 3, 4, 5, 6, 7])
def test_mixed_batch_every_beta(oracle_mod, den, torch_cuda, beta):
    imgs = mixed_batch(24, 100 + beta)
    outs, ks, conv = run_batch(den, torch_cuda, imgs, 10, beta, 32)
    check(oracle_mod, imgs, outs, ks, conv, 10, beta, 32, "mixed")


@pytest.mark.parametrize("alpha,max_k", [(0, 32), (1, 32), (255, 32), (10, 0), (10, 1), (10, 3), (10, 8),
                                         (10, 9), (20, 200)])
def test_alpha_and_max_k_edges(oracle_mod, den, torch_cuda, alpha, max_k):
    imgs = mixed_batch(16, 200 + alpha + max_k)
    outs, ks, conv = run_batch(den, torch_cuda, imgs, alpha, 1, max_k)
    check(oracle_mod, imgs, outs, ks, conv, alpha, 1, max_k, "edges")


@pytest.mark.parametrize("beta,passes", [(1, 1), (1, 3), (1, 6), (2, 2), (3, 1)])
def test_other_passes_per_launch(oracle_mod, den, torch_cuda, beta, passes):
    imgs = mixed_batch(12, 300 + 10 * beta + passes)
    outs, ks, conv = run_batch(den, torch_cuda, imgs, 10, beta, 32, passes=passes)
    check(oracle_mod, imgs, outs, ks, conv, 10, beta, 32, f"T={passes}")


def test_chunked_by_memory_budget(oracle_mod, den, torch_cuda):
    """A 1 MiB budget splits the batch into many chunks (one image each for
    the larger images); results are unchanged."""
    imgs = mixed_batch(20, 400)
    outs, ks, conv = run_batch(den, torch_cuda, imgs, 10, 1, 32, batch_mb=1)
    check(oracle_mod, imgs, outs, ks, conv, 10, 1, 32, "budget")


def test_chunked_by_entry_packing(oracle_mod, den, torch_cuda):
    """A 3 x 40000 image needs 16 column bits, so with 9 row bits at most 128
    images share a launch: 150 images run as two chunks."""
    rng = np.random.Generator(np.random.PCG64(7))
    imgs = [synth.noisy_image(3, 40000, 0.3, 77)[1], synth.noisy_image(300, 40, 0.3, 78)[1]]
    for i in range(148):
        r, c = (int(v) for v in rng.integers(5, 40, size=2))
        imgs.append(synth.noisy_image(r, c, float(rng.uniform(0.05, 0.6)), 500 + i)[1])
    outs, ks, conv = run_batch(den, torch_cuda, imgs, 10, 1, 32)
    check(oracle_mod, imgs, outs, ks, conv, 10, 1, 32, "packing")


@pytest.mark.parametrize("list_cap", [1, 50, 2000])
def test_list_overflow_in_batch(oracle_mod, den, torch_cuda, list_cap):
    imgs = mixed_batch(10, 500 + list_cap)
    outs, ks, conv = run_batch(den, torch_cuda, imgs, 10, 1, 32, list_cap=list_cap)
    check(oracle_mod, imgs, outs, ks, conv, 10, 1, 32, f"cap={list_cap}")


def test_host_pointer_batch(oracle_mod, den, torch_cuda):
    imgs = mixed_batch(12, 600)
    outs, ks, conv = run_batch(den, torch_cuda, imgs, 10, 2, 32, host=True)
    check(oracle_mod, imgs, outs, ks, conv, 10, 2, 32, "host")


def test_unaligned_device_images(oracle_mod, den, torch_cuda):
    """Images at odd byte offsets of one device buffer, in a batch: the
    batched copies read and write exactly the images' bytes."""
    torch = torch_cuda
    imgs = mixed_batch(9, 700, max_side=90)
    sizes = [im.size for im in imgs]
    buf = torch.full((sum(sizes) + 3 * len(imgs) + 8,), 7, dtype=torch.uint8, device="cuda")
    views, off = [], 1
    for im in imgs:
        v = buf[off:off + im.size].view(im.shape)
        v.copy_(torch.from_numpy(im))
        views.append(v)
        off += im.size + 3
    ks = den.denoise_batch(views, 10, 1, 32)
    outs = [v.cpu().numpy() for v in views]
    check(oracle_mod, imgs, outs, ks, den.converged(), 10, 1, 32, "unaligned")
    # the gap bytes are untouched
    host = buf.cpu().numpy()
    off = 1
    assert host[0] == 7
    for im in imgs:
        off += im.size
        assert (host[off:off + 3] == 7).all()
        off += 3


def test_empty_batch(den, torch_cuda):
    assert den.denoise_batch([], 10, 1, 32) == []


def test_batch_equals_single_calls(den, torch_cuda):
    """The batch and the single-image path give the same bytes and k."""
    torch = torch_cuda
    imgs = mixed_batch(10, 800)
    outs, ks, _ = run_batch(den, torch, imgs, 10, 1, 32)
    for im, out, k in zip(imgs, outs, ks):
        t = torch.from_numpy(im.copy()).cuda()
        assert den.denoise(t, 10, 1, 32) == k
        assert np.array_equal(t.cpu().numpy(), out)


def test_uneven_workload_all_512_images(oracle_mod, torch_cuda):
    """The whole uneven workload (512 images, sides uniform in 128..2048,
    density 5..70 %, 629 M pixels) as the benchmark runs it: the images one
    after another in one device buffer, one hgrms_denoise_batch call on an
    autotuned handle (the first call tunes, the second reuses the choice),
    and with the learned k-predictor choosing the schedule.  Every image's
    bytes, k and converged flag (k < max_k) against the oracle, which runs
    image by image on all host cores."""
    import oracle_pool
    from paper_1306_5390_gb300 import hgrms
    torch = torch_cuda
    n = 512
    res = oracle_pool.batch_denoise(n)
    shapes = [r[0].shape for r in res]
    sizes = [a * b for a, b in shapes]
    offs = np.cumsum([0] + sizes)
    pristine = torch.from_numpy(np.concatenate([r[0].ravel() for r in res])).cuda()
    work = torch.empty_like(pristine)
    views = [work[int(offs[i]):int(offs[i + 1])].view(shapes[i]) for i in range(n)]
    d = hgrms.Denoiser(0, autotune=True)
    try:
        runs = []
        for call in range(2):
            work.copy_(pristine)
            runs.append((d.denoise_batch(views, 10, 1, 32), work.cpu().numpy()))
        try:
            d.load_predictor(1)
            d.set_option(hgrms.HGRMS_OPT_PREDICT_K, 1)
            work.copy_(pristine)
            runs.append((d.denoise_batch(views, 10, 1, 32), work.cpu().numpy()))
        except FileNotFoundError:
            pass
    finally:
        d.close()
    for ri, (ks, flat) in enumerate(runs):
        bad = []
        for i, (noisy, ref, k_ref, c_ref) in enumerate(res):
            out = flat[int(offs[i]):int(offs[i + 1])].reshape(shapes[i])
            if k_ref != ks[i] or c_ref != (ks[i] < 32) or not np.array_equal(out, ref):
                bad.append((i, shapes[i], ks[i], k_ref, int((out != ref).sum())))
        assert not bad, f"run {ri}: {len(bad)} images differ, first {bad[:5]}"


@pytest.mark.parametrize("beta,passes,max_k,list_cap", [(1, 0, 32, 0), (1, 3, 32, 0), (2, 0, 32, 0), (3, 0, 13, 0),
                                                      (1, 0, 32, 40), (2, 2, 32, 40), (1, 1, 20, 0)])
def test_fused_relaunches_in_batch(oracle_mod, den, torch_cuda, beta, passes, max_k, list_cap):
    """A threshold of 1 pixel per million makes every fused launch after the
    first run while anything changed (up to 8 of them), with list passes for
    what is left; with a small list capacity some change sets overflow, so
    the next fused launch starts with a dense pass."""
    imgs = mixed_batch(14, 900 + 10 * beta + passes + list_cap)
    outs, ks, conv = run_batch(den, torch_cuda, imgs, 10, beta, max_k, passes=passes, list_cap=list_cap,
                               relaunch_ppm=1)
    check(oracle_mod, imgs, outs, ks, conv, 10, beta, max_k, f"relaunch b={beta} T={passes} cap={list_cap}")


def test_autotuner_single_and_batch(oracle_mod, den, torch_cuda):
    """The autotuner's first call of a class times the candidates without
    writing the images, then denoises with the fastest; results match the
    oracle and the second call of the class reuses the choice."""
    from paper_1306_5390_gb300 import hgrms
    torch = torch_cuda
    d = hgrms.Denoiser(0, autotune=True)
    try:
        _, noisy = synth.noisy_image(333, 517, 0.35, synth.seed_for(33, 0))
        ref, k_ref, c_ref = oracle_mod.denoise(noisy, 10, 1, 32)
        for call in range(2):
            t = torch.from_numpy(noisy.copy()).cuda()
            k = d.denoise(t, 10, 1, 32)
            st = d.stats()
            assert k == k_ref and d.converged() == bool(c_ref)
            assert np.array_equal(t.cpu().numpy(), ref)
            assert st["autotuned"] == 1
            assert (st["tune_ms"] > 0) == (call == 0)
            assert hgrms.hgrms_has_kernel(1, st["passes_per_launch"]) == 1
            assert st["tile_eval_max"] in (1024, 2048, 4096, 8192)
        imgs = mixed_batch(12, 1000)
        work = [torch.from_numpy(im.copy()).cuda() for im in imgs]
        ks = d.denoise_batch(work, 10, 2, 32)
        assert d.stats()["autotuned"] == 1
        check(oracle_mod, imgs, [w.cpu().numpy() for w in work], ks, d.converged(), 10, 2, 32, "autotune")
    finally:
        d.close()


def test_batch_mixing_device_pinned_and_pageable(oracle_mod, den, torch_cuda):
    """One batch with device images, page-locked host images (read and
    written by the kernels) and pageable host images (staged by copies)."""
    torch = torch_cuda
    imgs = mixed_batch(12, 1100)
    work, outs_get = [], []
    for i, im in enumerate(imgs):
        if i % 3 == 0:
            t = torch.from_numpy(im.copy()).cuda()
            work.append(t)
            outs_get.append(lambda t=t: t.cpu().numpy())
        elif i % 3 == 1:
            p = torch.from_numpy(im.copy()).pin_memory()
            arr = p.numpy()
            work.append(arr)
            outs_get.append(lambda arr=arr, p=p: arr.copy())
        else:
            arr = im.copy()
            work.append(arr)
            outs_get.append(lambda arr=arr: arr.copy())
    ks = den.denoise_batch(work, 10, 1, 32)
    check(oracle_mod, imgs, [g() for g in outs_get], ks, den.converged(), 10, 1, 32, "mixed memory")
