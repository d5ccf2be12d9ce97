"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bit-exact comparison of every output pixel, of k and of the converged flag
(the method is integer arithmetic, so the tolerance is zero).  Covers every
compiled (beta, passes-per-launch) kernel, tile-straddling and ragged
shapes, degenerate sizes, alpha edge values, max_k edge values, host and
device pointers, the batch entry point, the 256x256 and 481x321 workloads
in full, and the 8192x8192 workload in full (every byte, k and the converged
flag, with the oracle run band by band on all host cores).
"""
import numpy as np
import pytest

from paper_1306_5390_gb300 import synth

pytestmark = pytest.mark.gpu

ALL_KERNELS = [(1, 1), (1, 2), (1, 3), (1, 4), (1, 6), (1, 8), (2, 1), (2, 2), (2, 3), (2, 4),
               (3, 1), (3, 2), (4, 1), (4, 2), (5, 1), (6, 1), (7, 1)]


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


def gpu_denoise(d, torch, img, alpha, beta, max_k, passes=0, kernel=0, host=False, list_cap=0, relaunch_ppm=0):
    from paper_1306_5390_gb300 import hgrms
    d.set_option(hgrms.HGRMS_OPT_PASSES, passes)
    d.set_option(hgrms.HGRMS_OPT_KERNEL, kernel)
    d.set_option(hgrms.HGRMS_OPT_LIST_CAP, list_cap)
    d.set_option(hgrms.HGRMS_OPT_RELAUNCH_PPM, relaunch_ppm)
    if host:
        out = np.ascontiguousarray(img).copy()
        k = d.denoise(out, alpha, beta, max_k)
    else:
        t = torch.from_numpy(np.ascontiguousarray(img).copy()).cuda()
        k = d.denoise(t, alpha, beta, max_k)
        out = t.cpu().numpy()
    return out, k, d.converged()


def assert_same(oracle_mod, d, torch, img, alpha, beta, max_k, **kw):
    ref, k_ref, c_ref = oracle_mod.denoise(img, alpha, beta, max_k)
    out, k, c = gpu_denoise(d, torch, img, alpha, beta, max_k, **kw)
    bad = int((out != ref).sum())
    assert bad == 0 and k == k_ref and c == c_ref, (
        f"shape={img.shape} a={alpha} b={beta} max_k={max_k} {kw}: {bad} pixels differ, "
        f"k={k} vs {k_ref}, converged={c} vs {c_ref}")
    return k


def test_workload_256(oracle_mod, den, torch_cuda):
    w = synth.workload_256()
    k = assert_same(oracle_mod, den, torch_cuda, w["noisy"], w["alpha"], w["beta"], w["max_k"])
    assert k >= 1
    assert_same(oracle_mod, den, torch_cuda, w["noisy"], w["alpha"], w["beta"], w["max_k"], host=True)


@pytest.mark.parametrize("beta,passes", ALL_KERNELS)
def test_every_kernel_on_tile_straddling_shapes(oracle_mod, den, torch_cuda, beta, passes):
    th = 64 - 2 * (passes - 1) * beta
    shapes = [(th + 1, 241), (2 * th - 1, 239), (th, 480), (3 * th + 5, 97)]
    for i, (r, c) in enumerate(shapes):
        _, noisy = synth.noisy_image(r, c, 0.3, synth.seed_for(20, 100 * beta + 10 * passes + i))
        mk = 32 if beta <= 2 else 12
        assert_same(oracle_mod, den, torch_cuda, noisy, 10, beta, mk, passes=passes)
    img = synth.random_image(th + 3, 250, 5000 + beta, levels=[0, 20, 25, 30, 35, 255])
    assert_same(oracle_mod, den, torch_cuda, img, 6, beta, 9, passes=passes)


@pytest.mark.parametrize("beta", [1, 2, 3])
def test_degenerate_and_ragged_shapes(oracle_mod, den, torch_cuda, beta):
    shapes = [(1, 1), (1, 300), (300, 1), (2, 2), (2 * beta, 70), (70, 2 * beta),
              (2 * beta + 1, 2 * beta + 1), (5, 7), (17, 255), (33, 17), (100, 1000), (481, 321)]
    for i, (r, c) in enumerate(shapes):
        _, noisy = synth.noisy_image(r, c, 0.25, synth.seed_for(21, 10 * beta + i))
        assert_same(oracle_mod, den, torch_cuda, noisy, 10, beta, 32)
        assert_same(oracle_mod, den, torch_cuda, noisy, 10, beta, 32, kernel=1)


@pytest.mark.parametrize("alpha", [0, 1, 2, 128, 254, 255])
def test_alpha_edges(oracle_mod, den, torch_cuda, alpha):
    img = synth.random_image(90, 300, 900 + alpha)
    for beta in (1, 2):
        assert_same(oracle_mod, den, torch_cuda, img, alpha, beta, 6)
    _, noisy = synth.noisy_image(90, 300, 0.2, synth.seed_for(22, alpha))
    assert_same(oracle_mod, den, torch_cuda, noisy, alpha, 1, 32)


@pytest.mark.parametrize("max_k", [0, 1, 2, 3, 4, 5, 7, 9, 33])
def test_max_k_not_multiple_of_passes(oracle_mod, den, torch_cuda, max_k):
    _, noisy = synth.noisy_image(200, 333, 0.5, synth.seed_for(23, max_k))
    for passes in (1, 4, 8):
        assert_same(oracle_mod, den, torch_cuda, noisy, 10, 1, max_k, passes=passes)


@pytest.mark.parametrize("beta,passes", [(1, 1), (1, 4), (1, 8), (2, 2), (2, 4), (3, 1), (3, 2), (5, 1)])
def test_fused_only_schedule(oracle_mod, den, torch_cuda, beta, passes):
    """Repeated fused launches, whose first pass learns the previous launch's
    changes from the per-pixel change bitmap."""
    for i, (r, c) in enumerate(((200, 481), (131, 250), (64, 700))):
        _, noisy = synth.noisy_image(r, c, 0.3, synth.seed_for(30, 10 * beta + i))
        assert_same(oracle_mod, den, torch_cuda, noisy, 10, beta, 32 if beta < 3 else 12, passes=passes, kernel=2)


@pytest.mark.parametrize("list_cap", [1, 7, 100, 1000])
def test_list_overflow_falls_back_to_full_pass(oracle_mod, den, torch_cuda, list_cap):
    """Change lists far smaller than the changes: list passes must switch to
    evaluating every pixel and stay exact."""
    for beta in (1, 2):
        _, noisy = synth.noisy_image(150, 333, 0.4, synth.seed_for(31, beta))
        for passes in (1, 2):
            assert_same(oracle_mod, den, torch_cuda, noisy, 10, beta, 32, passes=passes, list_cap=list_cap)


@pytest.mark.parametrize("beta,passes", [(1, 8), (1, 2), (2, 4), (3, 2), (4, 1)])
@pytest.mark.parametrize("ppm", [1, 5000])
def test_fused_relaunches(oracle_mod, den, torch_cuda, beta, passes, ppm):
    """Relaunch thresholds that make later fused launches run (every one
    while pixels change, or while more than 0.5 % would be evaluated)."""
    for i, (r, c) in enumerate([(301, 517), (64, 1000), (530, 250)]):
        _, noisy = synth.noisy_image(r, c, 0.45, synth.seed_for(31, 10 * beta + i))
        assert_same(oracle_mod, den, torch_cuda, noisy, 10, beta, 32, passes=passes, relaunch_ppm=ppm)
    _, noisy = synth.noisy_image(200, 300, 0.6, synth.seed_for(32, beta))
    assert_same(oracle_mod, den, torch_cuda, noisy, 10, beta, 32, passes=passes, relaunch_ppm=1, list_cap=30)


def test_unfused_kernel_every_beta(oracle_mod, den, torch_cuda):
    for beta in range(1, 8):
        _, noisy = synth.noisy_image(120, 250, 0.3, synth.seed_for(24, beta))
        assert_same(oracle_mod, den, torch_cuda, noisy, 10, beta, 10, kernel=1)


def test_host_pointer_path(oracle_mod, den, torch_cuda):
    for beta in (1, 2):
        _, noisy = synth.noisy_image(333, 517, 0.3, synth.seed_for(25, beta))
        assert_same(oracle_mod, den, torch_cuda, noisy, 10, beta, 32, host=True)


def test_pinned_host_pointer_path(oracle_mod, den, torch_cuda):
    """Page-locked host images are read and written by the copy kernels
    directly (no staging copy); odd shapes and an odd byte offset."""
    torch = torch_cuda
    for i, (r, c) in enumerate([(200, 333), (8193 // 8, 1000), (17, 255)]):
        _, noisy = synth.noisy_image(r, c, 0.3, synth.seed_for(34, i))
        buf = torch.empty(r * c + 1, dtype=torch.uint8).pin_memory()
        host = buf.numpy()[1:].reshape(r, c)
        host[...] = noisy
        ref, k_ref, c_ref = oracle_mod.denoise(noisy, 10, 1 + i % 2, 32)
        k = den.denoise(host, 10, 1 + i % 2, 32)
        assert k == k_ref and den.converged() == bool(c_ref)
        assert np.array_equal(host, ref), (r, c)


@pytest.mark.parametrize("max_k", [9, 10, 13, 20, 31, 32, 40])
def test_list_pass_endings_device_and_pinned(oracle_mod, den, torch_cuda, max_k):
    """Runs that end by max_k after a few list passes, by convergence, or
    after many passes, for device and pinned host images (which the kernels
    read and write directly), must all give the oracle's bytes and k."""
    torch = torch_cuda
    for i, (r, c, dens) in enumerate([(301, 517, 0.3), (200, 200, 0.02), (57, 1000, 0.5)]):
        _, noisy = synth.noisy_image(r, c, dens, synth.seed_for(35, 10 * i + max_k))
        assert_same(oracle_mod, den, torch_cuda, noisy, 10, 1, max_k)
        ref, k_ref, c_ref = oracle_mod.denoise(noisy, 10, 1, max_k)
        buf = torch.from_numpy(noisy.copy()).pin_memory()
        host = buf.numpy()
        den.set_option(1, 0)
        k = den.denoise(host, 10, 1, max_k)
        assert k == k_ref and np.array_equal(host, ref), (r, c, max_k)


def test_unaligned_device_pointer(oracle_mod, den, torch_cuda):
    torch = torch_cuda
    _, noisy = synth.noisy_image(150, 160, 0.3, synth.seed_for(26, 0))
    ref, k_ref, c_ref = oracle_mod.denoise(noisy, 10, 1, 32)
    buf = torch.zeros(150 * 160 + 3, dtype=torch.uint8, device="cuda")
    view = buf[3:].view(150, 160)
    view.copy_(torch.from_numpy(noisy))
    k = den.denoise(view, 10, 1, 32)
    assert k == k_ref
    assert np.array_equal(view.cpu().numpy(), ref)
    assert int(buf[:3].sum()) == 0


def test_batch_matches_per_image(oracle_mod, den, torch_cuda):
    torch = torch_cuda
    shapes = [(128, 128), (321, 481), (481, 321), (200, 2048), (7, 9), (1, 1)]
    imgs, refs = [], []
    for i, (r, c) in enumerate(shapes):
        _, noisy = synth.noisy_image(r, c, 0.05 + 0.1 * i, synth.seed_for(27, i))
        imgs.append(torch.from_numpy(noisy).cuda())
        refs.append(oracle_mod.denoise(noisy, 10, 1, 32))
    ks = den.denoise_batch(imgs, 10, 1, 32)
    for t, (ref, k_ref, _), k in zip(imgs, refs, ks):
        assert k == k_ref
        assert np.array_equal(t.cpu().numpy(), ref)
    host = [synth.noisy_image(r, c, 0.2, synth.seed_for(28, i))[1] for i, (r, c) in enumerate(shapes)]
    hrefs = [oracle_mod.denoise(h, 10, 2, 32) for h in host]
    ks = den.denoise_batch(host, 10, 2, 32)
    for h, (ref, k_ref, _), k in zip(host, hrefs, ks):
        assert k == k_ref and np.array_equal(h, ref)


def test_bsds_like_workload_all_runs(oracle_mod, den, torch_cuda):
    """The 481x321 / 321x481 sweep in full, as the benchmark runs it: for each
    of the 30 settings (density 10..90 %, alpha 5/10/20, beta 1/2), the 64
    images in one hgrms_denoise_batch call; all 1920 outputs, k and converged
    flags against the oracle (run image by image on all host cores).  Two
    images also go through the single-image call for every setting."""
    import oracle_pool
    torch = torch_cuda
    refs = oracle_pool.bsds_denoise(64)
    settings = {}
    for w in synth.workload_bsds_like(64):
        settings.setdefault((w["density"], w["alpha"], w["beta"]), []).append(w)
    assert len(settings) == 30
    gpu_denoise(den, torch, settings[(0.3, 10, 1)][0]["noisy"], 10, 1, 32)  # options back to defaults
    for key, items in sorted(settings.items()):
        dens, a, b = key
        work = [torch.from_numpy(w["noisy"]).cuda() for w in items]
        ks = den.denoise_batch(work, a, b, 32)
        bad = []
        for i, (w, t, k, (ref, k_ref, c_ref)) in enumerate(zip(items, work, ks, refs[key])):
            out = t.cpu().numpy()
            if k != k_ref or c_ref != (k < 32) or not np.array_equal(out, ref):
                bad.append((i, k, k_ref, int((out != ref).sum())))
        assert not bad, f"setting {key}: {len(bad)} images differ, first {bad[:4]}"
        for i in range(2):
            out, k, c = gpu_denoise(den, torch, items[i]["noisy"], a, b, 32)
            ref, k_ref, c_ref = refs[key][i]
            assert k == k_ref and c == c_ref and np.array_equal(out, ref), (key, i)


def test_tall_and_wide_extremes(oracle_mod, den, torch_cuda):
    for (r, c) in ((65536, 20), (12, 65536)):
        _, noisy = synth.noisy_image(r, c, 0.3, synth.seed_for(29, r))
        assert_same(oracle_mod, den, torch_cuda, noisy, 10, 1, 8)


@pytest.mark.parametrize("beta", [1, 2])
def test_tall_tiles_on_a_ragged_large_image(torch_cuda, beta):
    """Single images of at least 32 Mi pixels run the 128-row fused tiles;
    a 5803 x 5795 image (33.6 M pixels, neither side a multiple of the
    tile) at 40 % impulses against the oracle run band by band on all host
    cores: every byte, k and the converged flag."""
    import oracle_pool
    from paper_1306_5390_gb300 import build, hgrms
    build.build()
    rows, cols, max_k = 5803, 5795, 16
    _, noisy = synth.noisy_image(rows, cols, 0.40, synth.seed_for(30, beta))
    ref, k_ref, c_ref, _ = oracle_pool.banded_denoise(noisy, 10, beta, max_k)
    with hgrms.Denoiser(0) as d:
        t = torch_cuda.from_numpy(noisy).cuda()
        k = d.denoise(t, 10, beta, max_k)
        assert d.stats()["tile_rows"] == 128 - 2 * (hgrms.hgrms_default_passes(beta) - 1) * beta
        out = t.cpu().numpy()
        assert k == k_ref and d.converged() == c_ref and int((out != ref).sum()) == 0


def test_argument_errors_leave_image_untouched(den, torch_cuda):
    from paper_1306_5390_gb300 import hgrms
    torch = torch_cuda
    t = torch.full((10, 10), 7, dtype=torch.uint8, device="cuda")
    for args in ((10, 10, -1, 1, 5), (10, 10, 256, 1, 5), (10, 10, 10, 0, 5), (10, 10, 10, 8, 5),
                 (10, 10, 10, 1, -1), (0, 10, 10, 1, 5), (10, 0, 10, 1, 5), (70000, 1, 10, 1, 5)):
        assert hgrms.hgrms_denoise(den.h, t.data_ptr(), *args) == hgrms.HGRMS_EINVAL
    assert hgrms.hgrms_denoise(den.h, 0, 10, 10, 10, 1, 5) == hgrms.HGRMS_EINVAL
    den.set_option(hgrms.HGRMS_OPT_PASSES, 4)
    assert hgrms.hgrms_denoise(den.h, t.data_ptr(), 10, 10, 10, 3, 5) == hgrms.HGRMS_EINVAL
    den.set_option(hgrms.HGRMS_OPT_PASSES, 0)
    assert int((t != 7).sum()) == 0


@pytest.fixture(scope="module")
def bench_step_8192(torch_cuda):
    """The benchmark's step on the 8192x8192 workload, exactly as bench.py
    times it: one handle per beta (1, 2, 3) on one stream, launch timing on,
    the three calls queued with hgrms_denoise_async and then waited for; once
    with max_k 32 (to convergence) and once with the paper's fixed k = 5.
    Returns {(beta, max_k): (output, k, converged)}."""
    from paper_1306_5390_gb300 import build, hgrms
    torch = torch_cuda
    build.build()
    betas = (1, 2, 3)
    got = {}
    ds = [hgrms.Denoiser(0, timing=True) for _ in betas]
    try:
        for max_k in (32, 5):
            ws = [synth.workload_8192(b) for b in betas]
            ts = [torch.from_numpy(w["noisy"]).cuda() for w in ws]
            for d, t, w, b in zip(ds, ts, ws, betas):
                d.denoise_async(t, w["alpha"], b, max_k)
            for d, t, b in zip(ds, ts, betas):
                k = d.wait()
                got[(b, max_k)] = (t.cpu().numpy(), k, d.converged())
            del ts
    finally:
        for d in ds:
            d.close()
    return got


@pytest.mark.parametrize("max_k", [32, 5])
@pytest.mark.parametrize("beta", [1, 2, 3])
def test_8192_full_size_every_pixel(oracle_mod, bench_step_8192, beta, max_k):
    """8192x8192, 30 % impulse noise, alpha 10: every one of the 67.1 M output
    bytes, k and the converged flag of the benchmark's own calls against the
    oracle, which runs band by band on all host cores (tests/oracle_pool:
    exact per-pass change counts, so k and the flag are the whole image's).
    This size alone runs the list-pass loop with two CTAs per SM and the
    fused relaunch slots."""
    import oracle_pool
    w = synth.workload_8192(beta)
    out, k, conv = bench_step_8192[(beta, max_k)]
    ref, k_ref, c_ref, changes = oracle_pool.banded_denoise(w["noisy"], w["alpha"], beta, max_k)
    bad = int((out != ref).sum())
    assert bad == 0 and k == k_ref and conv == c_ref, (
        f"beta={beta} max_k={max_k}: {bad} of {out.size} pixels differ, k={k} vs {k_ref}, "
        f"converged={conv} vs {c_ref}, oracle changes per pass {changes}")


def test_rms_arithmetic_exhaustive(torch_cuda):
    """The kernels' integer root mean square, floor(sqrt(floor(sum / flag))),
    against exact integer math for every flag 1..225 and every quotient
    0..255^2, at both ends of the quotient's range of sums (q * flag and
    q * flag + flag - 1), through the C ABI."""
    import math
    from paper_1306_5390_gb300 import hgrms
    torch = torch_cuda
    lib = hgrms.load_library()
    isq = np.array([math.isqrt(q) for q in range(255 * 255 + 1)], dtype=np.int32)
    q = torch.arange(0, 255 * 255 + 1, dtype=torch.int32, device="cuda")
    for flag in range(1, 226):
        for r in (0, flag - 1):
            s = q * flag + r
            keep = s <= flag * 255 * 255
            s = s[keep].contiguous()
            f = torch.full_like(s, flag)
            out = torch.empty_like(s)
            assert lib.hgrms_rms(s.data_ptr(), f.data_ptr(), out.data_ptr(), s.numel(), None) == 0
            expect = isq[(s.cpu().numpy() // flag)]
            assert np.array_equal(out.cpu().numpy(), expect), (flag, r)


def _golden_files():
    import os
    d = os.path.join(os.path.dirname(__file__), "golden")
    return sorted(f for f in os.listdir(d) if f.endswith(".txt"))


@pytest.mark.parametrize("name", _golden_files())
def test_golden_worked_examples_on_gpu(den, torch_cuda, name):
    """The hand-derived worked examples (tests/golden, each citing its
    passage of the paper) through the CUDA path: bytes, k and the converged
    flag equal the values derived from the paper, with no oracle in
    between."""
    import os
    from test_oracle import load_golden
    g = load_golden(os.path.join(os.path.dirname(__file__), "golden", name))
    for kernel in (0, 1):  # the default schedule and the unfused kernel
        out, k, conv = gpu_denoise(den, torch_cuda, g["input"], g["alpha"], g["beta"], g["max_k"], kernel=kernel)
        assert k == g["k"] and conv == bool(g["converged"]), (name, kernel, k, conv)
        np.testing.assert_array_equal(out, g["output"], err_msg=f"{name} kernel {kernel}")


@pytest.mark.parametrize("beta", [1, 2, 3, 4, 5])
def test_tma_staging_on_and_off_identical(oracle_mod, den, torch_cuda, beta):
    """Tiles staged by TMA (HGRMS_OPT_TMA 1, the default) and by ordinary
    loads (0) give the oracle's bytes and k: device images whose width is a
    multiple of 16 (the first launch loads them by TMA too), widths that are
    not (the first launch falls back to ordinary loads), host images (copied
    into the canvas, then TMA), and beta 5 (no staging buffer fits)."""
    from paper_1306_5390_gb300 import hgrms
    torch = torch_cuda
    shapes = [(300, 512), (257, 333), (64, 16)]
    try:
        for i, (r, c) in enumerate(shapes):
            _, noisy = synth.noisy_image(r, c, 0.3, synth.seed_for(61, 10 * beta + i))
            ref, k_ref, c_ref = oracle_mod.denoise(noisy, 10, beta, 12)
            for tma in (1, 0):
                den.set_option(hgrms.HGRMS_OPT_TMA, tma)
                for host in (False, True):
                    out, k, conv = gpu_denoise(den, torch, noisy, 10, beta, 12, host=host)
                    assert k == k_ref and conv == c_ref and np.array_equal(out, ref), (r, c, tma, host)
    finally:
        den.set_option(hgrms.HGRMS_OPT_TMA, 1)
