"""The learned k-predictor on the GPU (BF16 tensor-core convolutions).

The features (64 x 64 area means, 16-bin histogram) are checked against
their definition computed here; the network's outputs against a NumPy
forward pass of the same weights from the same features, with the BF16
rounding of weights and activations the kernels apply (FP32 accumulation,
so the tolerance covers accumulation order and the occasional one-ulp BF16
rounding difference it causes).  A call whose schedule follows the
predicted k must still give the oracle's bytes and k.
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
    from paper_1306_5390_gb300 import build
    build.build()
    return torch


def bf16(x):
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32)


def ref_features(img):
    rows, cols = img.shape
    x0 = np.zeros((64, 64))
    for i in range(64):
        r0 = i * rows // 64
        r1 = max(r0 + 1, (i + 1) * rows // 64)
        for j in range(64):
            c0 = j * cols // 64
            c1 = max(c0 + 1, (j + 1) * cols // 64)
            x0[i, j] = img[r0:r1, c0:c1].astype(np.float64).mean() / 255.0
    hist = np.bincount((img >> 4).ravel(), minlength=16) / img.size
    return x0, hist


def ref_network(w, x0, hist):
    """NumPy forward pass: weights in hgrms_predictor_load's order."""
    off = 0
    convs = []
    for cin in (1, 16, 16, 16):
        convs.append(bf16(w[off:off + 9 * cin * 16]).reshape(9, cin, 16).astype(np.float64))
        off += 9 * cin * 16
    biases = w[off:off + 64].reshape(4, 16).astype(np.float64)
    off += 64
    head = w[off:off + 33].astype(np.float64)
    x = bf16(x0).astype(np.float64)[:, :, None]
    for l in range(4):
        pad = np.pad(x, ((1, 1), (1, 1), (0, 0)))
        acc = np.zeros((64, 64, 16))
        for t in range(9):
            dy, dx = t // 3 - 1, t % 3 - 1
            acc += pad[1 + dy:65 + dy, 1 + dx:65 + dx, :] @ convs[l][t]
        x = bf16(np.maximum(acc + biases[l], 0.0).astype(np.float32)).astype(np.float64)
    gap = x.reshape(-1, 16).mean(axis=0)
    k = max(0.0, head[32] + head[:16] @ gap + head[16:32] @ hist)
    return gap, k


def random_weights(seed, scale=0.25):
    from paper_1306_5390_gb300 import hgrms
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.normal(0.0, scale, size=hgrms.PREDICTOR_WEIGHTS).astype(np.float32)
    w[-33:] = rng.uniform(0.0, 2.0, size=33)  # positive head: k_hat > 0
    return w


def test_features_match_definition(torch_cuda):
    torch = torch_cuda
    from paper_1306_5390_gb300 import hgrms
    shapes = [(1, 1), (3, 200), (64, 64), (65, 63), (100, 37), (481, 321), (1000, 700)]
    imgs = [synth.noisy_image(r, c, 0.3, 600 + i)[1] for i, (r, c) in enumerate(shapes)]
    with hgrms.Denoiser(0) as d:
        d.load_predictor(1, random_weights(1))
        _, x0, hist, _ = d.predict_k(1, [torch.from_numpy(im).cuda() for im in imgs], features=True)
    for i, im in enumerate(imgs):
        rx, rh = ref_features(im)
        np.testing.assert_allclose(x0[i], rx, rtol=0, atol=2e-6, err_msg=str(im.shape))
        np.testing.assert_allclose(hist[i], rh, rtol=1e-6, atol=1e-7, err_msg=str(im.shape))


@pytest.mark.parametrize("seed", [2, 3])
def test_network_matches_numpy(torch_cuda, seed):
    torch = torch_cuda
    from paper_1306_5390_gb300 import hgrms
    w = random_weights(seed)
    shapes = [(64, 64), (300, 500), (97, 1000), (2048, 128)]
    imgs = [synth.noisy_image(r, c, 0.05 + 0.2 * i, 700 + 10 * seed + i)[1] for i, (r, c) in enumerate(shapes)]
    with hgrms.Denoiser(0) as d:
        d.load_predictor(1, w)
        kh, x0, hist, gap = d.predict_k(1, [torch.from_numpy(im).cuda() for im in imgs], features=True)
    for i in range(len(imgs)):
        g_ref, k_ref = ref_network(w, x0[i], hist[i])
        np.testing.assert_allclose(gap[i], g_ref, rtol=2e-2, atol=2e-3, err_msg=f"image {i}")
        assert abs(kh[i] - k_ref) <= 2e-2 * max(1.0, abs(k_ref)), (i, kh[i], k_ref)


def test_predicted_schedule_is_exact(oracle_mod, torch_cuda):
    """With the predicted-k schedule (fitted weights, or random ones that
    over- or under-estimate), bytes and k equal the oracle's."""
    torch = torch_cuda
    from paper_1306_5390_gb300 import hgrms
    imgs = [synth.noisy_image(r, c, dens, 800 + i)[1]
            for i, (r, c, dens) in enumerate([(200, 300, 0.05), (333, 250, 0.3), (129, 700, 0.6), (40, 40, 0.2)])]
    refs = [oracle_mod.denoise(im, 10, 1, 32) for im in imgs]
    for w in (None, random_weights(9, scale=0.5), np.zeros(hgrms.PREDICTOR_WEIGHTS, dtype=np.float32)):
        with hgrms.Denoiser(0) as d:
            try:
                d.load_predictor(1, w)
            except FileNotFoundError:
                continue
            d.set_option(hgrms.HGRMS_OPT_PREDICT_K, 1)
            for im, (ref, k_ref, _) in zip(imgs, refs):
                t = torch.from_numpy(im.copy()).cuda()
                assert d.denoise(t, 10, 1, 32) == k_ref
                assert np.array_equal(t.cpu().numpy(), ref)
                assert d.stats()["k_pred"] >= 0
            work = [torch.from_numpy(im.copy()).cuda() for im in imgs]
            ks = d.denoise_batch(work, 10, 1, 32)
            for t, (ref, k_ref, _), k in zip(work, refs, ks):
                assert k == k_ref and np.array_equal(t.cpu().numpy(), ref)


def test_predictor_argument_errors(torch_cuda):
    torch = torch_cuda
    from paper_1306_5390_gb300 import hgrms
    with hgrms.Denoiser(0) as d:
        t = torch.zeros((8, 8), dtype=torch.uint8, device="cuda")
        with pytest.raises(hgrms.HgrmsError):
            d.predict_k(1, [t])  # nothing loaded
        with pytest.raises(hgrms.HgrmsError):
            d.load_predictor(1, np.zeros(10, dtype=np.float32))
        d.load_predictor(2, random_weights(4))
        with pytest.raises(hgrms.HgrmsError):
            d.predict_k(2, [np.zeros((8, 8), dtype=np.uint8)])  # pageable host memory
        assert d.predict_k(2, [t]).shape == (1,)


def torch_reference_grad(torch, w, x0, hist, k):
    """Gradient of mean((y - k)^2) in float64 with autograd, from the
    BF16-rounded weights and inputs the device uses."""
    nconv = 144 + 3 * 2304  # conv weights are BF16 on the device; biases and head stay FP32
    wt = torch.tensor(np.concatenate([bf16(w[:nconv]), w[nconv:]]).astype(np.float64), requires_grad=True)
    x = torch.tensor(bf16(x0).astype(np.float64)).unsqueeze(1)
    off = 0
    h = x
    for l, cin in enumerate((1, 16, 16, 16)):
        wl = wt[off:off + 9 * cin * 16].view(3, 3, cin, 16).permute(3, 2, 0, 1)  # [co][ci][ky][kx]
        off += 9 * cin * 16
        bl = wt[144 + 3 * 2304 + 16 * l: 144 + 3 * 2304 + 16 * (l + 1)]
        h = torch.relu(torch.nn.functional.conv2d(h, wl, bl, padding=1))
    head = wt[144 + 3 * 2304 + 64:]
    g = h.mean(dim=(2, 3))
    y = head[32] + g @ head[:16] + torch.tensor(hist.astype(np.float64)) @ head[16:32]
    loss = torch.mean((y - torch.tensor(k.astype(np.float64))) ** 2)
    loss.backward()
    return wt.grad.numpy(), float(loss.detach())


def test_training_gradient_matches_autograd(torch_cuda):
    """The device gradient (tensor-core forward, input gradients and weight
    gradients) against float64 autograd; BF16 activations and gradients on
    the device bound the agreement to about a percent."""
    torch = torch_cuda
    from paper_1306_5390_gb300 import hgrms
    rng = np.random.Generator(np.random.PCG64(21))
    n = 12
    x0 = rng.uniform(0.0, 1.0, size=(n, 64, 64)).astype(np.float32)
    hist = rng.dirichlet(np.ones(16), size=n).astype(np.float32)
    k = rng.uniform(0.0, 32.0, size=n).astype(np.float32)
    w = random_weights(22, scale=0.2)
    with hgrms.Denoiser(0) as d:
        g, loss = d.predictor_grad(w, x0, hist, k)
    g_ref, loss_ref = torch_reference_grad(torch, w, x0, hist, k)
    assert abs(loss - loss_ref) <= 2e-2 * loss_ref
    groups = [(0, 144), (144, 2448), (2448, 4752), (4752, 7056), (7056, 7120), (7120, 7153)]
    for a, b in groups:
        err = np.linalg.norm(g[a:b] - g_ref[a:b]) / max(np.linalg.norm(g_ref[a:b]), 1e-12)
        assert err < 5e-2, (a, b, err)


def test_training_reduces_loss(torch_cuda):
    """A learnable target (k grows with the fraction of pixels in the two
    extreme bins): the device fit cuts the loss several-fold."""
    torch = torch_cuda
    from paper_1306_5390_gb300 import hgrms
    rng = np.random.Generator(np.random.PCG64(23))
    n = 512
    x0 = rng.uniform(0.0, 1.0, size=(n, 64, 64)).astype(np.float32)
    hist = rng.dirichlet(np.ones(16), size=n).astype(np.float32)
    k = (40.0 * (hist[:, 0] + hist[:, 15]) + 2.0).astype(np.float32)
    w0 = random_weights(24, scale=0.1)
    w0[-33:] = 0.0
    with hgrms.Denoiser(0) as d:
        _, loss0 = d.predictor_grad(w0, x0, hist, k)
        w, loss = d.train_predictor(w0, x0, hist, k, epochs=30, batch=64, lr=1e-2, seed=3)
        _, loss1 = d.predictor_grad(w, x0, hist, k)
    assert np.isfinite(loss1) and loss1 < 0.2 * loss0, (loss0, loss, loss1)
