"""The request server (hgrms_server_*): continuous batching on one GPU.

Each request's output and k must be the same when it is served alone and
when it is served in a mix of concurrent requests of other sizes and
settings (integer arithmetic: tolerance zero), and equal to the oracle's.
"""
import threading
import time

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


def requests_mix(n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        r, c = (int(v) for v in rng.integers(3, 500, size=2))
        density = float(rng.uniform(0.05, 0.8))
        alpha = int(rng.choice([10, 20]))
        beta = int(rng.choice([1, 2]))
        max_k = int(rng.choice([32, 5]))
        out.append((synth.noisy_image(r, c, density, seed * 1000 + i)[1], alpha, beta, max_k))
    return out


def test_same_alone_and_in_the_mix(oracle_mod, torch_cuda):
    from paper_1306_5390_gb300 import hgrms
    reqs = requests_mix(36, 11)
    alone = []
    with hgrms.Server(0, hbm_budget_bytes=1 << 30, slots=1) as srv:
        for img, a, b, mk in reqs:
            out = np.empty_like(img)
            k, info = srv.wait(srv.submit(img, a, b, mk, out=out))
            assert info["batch_size"] == 1
            alone.append((out, k))
    # The mix: three slots, requests submitted from two threads with gaps,
    # host images written to separate outputs.
    mixed = [None] * len(reqs)
    with hgrms.Server(0, hbm_budget_bytes=1 << 30, slots=3) as srv:
        ids = [None] * len(reqs)
        outs = [np.empty_like(img) for img, *_ in reqs]

        def submit(idx):
            for i in idx:
                img, a, b, mk = reqs[i]
                ids[i] = srv.submit(img, a, b, mk, out=outs[i])
                if i % 5 == 0:
                    time.sleep(0.002)

        th = [threading.Thread(target=submit, args=(list(range(j, len(reqs), 2)),)) for j in range(2)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        sizes = []
        for i in range(len(reqs)):
            k, info = srv.wait(ids[i])
            mixed[i] = (outs[i], k)
            sizes.append(info["batch_size"])
        st = srv.stats()
        assert st["served"] == len(reqs) and st["error"] == 0
    assert max(sizes) > 1, "no request shared a batch"
    for i, ((o1, k1), (o2, k2)) in enumerate(zip(alone, mixed)):
        assert k1 == k2 and np.array_equal(o1, o2), i
    for i in range(0, len(reqs), 4):
        img, a, b, mk = reqs[i]
        ref, k_ref, _ = oracle_mod.denoise(img, a, b, mk)
        assert alone[i][1] == k_ref and np.array_equal(alone[i][0], ref), i


def test_device_images_in_place(oracle_mod, torch_cuda):
    torch = torch_cuda
    from paper_1306_5390_gb300 import hgrms
    reqs = requests_mix(12, 12)
    with hgrms.Server(0, hbm_budget_bytes=1 << 30, slots=2) as srv:
        ts = [torch.from_numpy(img.copy()).cuda() for img, *_ in reqs]
        ids = [srv.submit(t, a, b, mk) for t, (_, a, b, mk) in zip(ts, reqs)]
        for t, rid, (img, a, b, mk) in zip(ts, ids, reqs):
            k, _ = srv.wait(rid)
            ref, k_ref, _ = oracle_mod.denoise(img, a, b, mk)
            assert k == k_ref and np.array_equal(t.cpu().numpy(), ref)


def test_tiny_budget_serves_large_requests_alone(oracle_mod, torch_cuda):
    """With a 64 MiB budget over 4 slots a 1500 x 1500 request exceeds a
    slot's share: it is served alone; the results are unchanged."""
    from paper_1306_5390_gb300 import hgrms
    big = synth.noisy_image(1500, 1500, 0.3, 1234)[1]
    small = [synth.noisy_image(40, 50, 0.3, 1300 + i)[1] for i in range(6)]
    with hgrms.Server(0, hbm_budget_bytes=64 << 20, slots=4) as srv:
        ob = np.empty_like(big)
        rb = srv.submit(big, 10, 1, 32, out=ob)
        rs = [srv.submit(s, 10, 1, 32) for s in small]
        k, info = srv.wait(rb)
        ref, k_ref, _ = oracle_mod.denoise(big, 10, 1, 32)
        assert k == k_ref and np.array_equal(ob, ref) and info["batch_size"] == 1
        for s, rid in zip(small, rs):
            srv.wait(rid)


def test_injected_allocation_failure_then_recovery(oracle_mod, torch_cuda):
    """A failure made on the host, with no GPU fault: the slot's buffer
    allocation for host images is made to fail.  A device image needs no
    such buffer and is served; the next host request completes with
    HGRMS_ENOMEM, its output untouched, and the server reports that error;
    a pending count can be withdrawn; the requests after it are served with
    the oracle's bytes and k."""
    from paper_1306_5390_gb300 import hgrms
    torch = torch_cuda
    imgs = [synth.noisy_image(300 + 7 * i, 200 + 5 * i, 0.3, 1500 + i)[1] for i in range(3)]
    refs = [oracle_mod.denoise(img, 10, 1, 32) for img in imgs]
    with hgrms.Server(0, hbm_budget_bytes=1 << 30, slots=1) as srv:
        srv.fail_allocations(1)
        dev = torch.from_numpy(imgs[0].copy()).cuda()
        k, _ = srv.wait(srv.submit(dev, 10, 1, 32))
        assert k == refs[0][1] and np.array_equal(dev.cpu().numpy(), refs[0][0])
        out = np.zeros_like(imgs[1])
        with pytest.raises(hgrms.HgrmsError) as err:
            srv.wait(srv.submit(imgs[1], 10, 1, 32, out=out))
        assert err.value.code == hgrms.HGRMS_ENOMEM
        assert not out.any()
        assert srv.stats()["error"] == hgrms.HGRMS_ENOMEM
        srv.fail_allocations(2)
        srv.fail_allocations(0)
        for img, (ref, k_ref, _) in zip(imgs, refs):
            out = np.empty_like(img)
            k, _ = srv.wait(srv.submit(img, 10, 1, 32, out=out))
            assert k == k_ref and np.array_equal(out, ref)


def test_argument_errors(torch_cuda):
    from paper_1306_5390_gb300 import hgrms
    lib = hgrms.load_library()
    import ctypes
    h = ctypes.c_void_p()
    assert lib.hgrms_server_create(ctypes.byref(h), 0, 1 << 20, 2) == hgrms.HGRMS_EINVAL  # budget too small
    assert lib.hgrms_server_create(ctypes.byref(h), 0, 1 << 30, 0) == hgrms.HGRMS_EINVAL
    with hgrms.Server(0, hbm_budget_bytes=1 << 30, slots=1) as srv:
        img = np.zeros((8, 8), dtype=np.uint8)
        rid = ctypes.c_ulonglong()
        assert lib.hgrms_server_submit(srv.h, img.ctypes.data, None, 8, 8, 10, 1, 5, ctypes.byref(rid)) \
            == hgrms.HGRMS_EINVAL  # a host image needs an output
        assert lib.hgrms_server_submit(srv.h, img.ctypes.data, img.ctypes.data, 8, 8, 10, 0, 5,
                                       ctypes.byref(rid)) == hgrms.HGRMS_EINVAL
        assert lib.hgrms_server_wait(srv.h, 987654321, 0.0, None) == hgrms.HGRMS_EINVAL
        k, _ = srv.wait(srv.submit(img, 10, 1, 5))
        assert k == 0
