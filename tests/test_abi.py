"""CPU-side checks of the C ABI: the library builds, loads and exports every
function include/hgrms.h declares; argument errors are reported without any
device work; the binding fails loudly when the library is absent."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hgrms.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1306_5390_gb300 import build, hgrms
    build.build()
    return hgrms.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hgrms_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("hgrms_create", "hgrms_denoise", "hgrms_denoise_batch", "hgrms_destroy"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1306_5390_gb300 import hgrms
    out = subprocess.run(["nm", "-D", "--defined-only", hgrms.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (hgrms_\w+)", out))
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)
    assert set(hgrms.EXPORTED) == set(declared_functions())
    # Nothing but the ABI leaks out of the library.
    assert not [s for s in re.findall(r"\bT (\w+)", out) if s.startswith("_ZN2hg")]


def test_strerror(lib):
    from paper_1306_5390_gb300 import hgrms
    assert hgrms.strerror(0) == "success"
    for code in (-1, -2, -3, -4, -5, -6, -7, -8):
        assert hgrms.strerror(code) not in ("success", "unknown error")
    assert hgrms.strerror(-99) == "unknown error"


def test_null_handle_errors_without_device_work(lib):
    from paper_1306_5390_gb300 import hgrms
    buf = (ctypes.c_uint8 * 16)()
    assert lib.hgrms_denoise(None, ctypes.addressof(buf), 4, 4, 10, 1, 5) == hgrms.HGRMS_EINVAL
    assert lib.hgrms_converged(None) == hgrms.HGRMS_EINVAL
    assert lib.hgrms_set_option(None, 1, 0) == hgrms.HGRMS_EINVAL
    assert lib.hgrms_last_cuda_error(None) == hgrms.HGRMS_EINVAL
    st = hgrms.hgrms_stats_t()
    assert lib.hgrms_stats(None, ctypes.byref(st)) == hgrms.HGRMS_EINVAL
    assert lib.hgrms_create(None, 0, None) == hgrms.HGRMS_EINVAL
    lib.hgrms_destroy(None)  # accepted
    ks = [0]
    assert hgrms.hgrms_denoise_batch(None, [ctypes.addressof(buf)], [4], [4], 10, 1, 5, ks) == hgrms.HGRMS_EINVAL
    assert lib.hgrms_denoise_async(None, ctypes.addressof(buf), 4, 4, 10, 1, 5) == hgrms.HGRMS_EINVAL
    assert lib.hgrms_wait(None) == hgrms.HGRMS_EINVAL


def test_kernel_table(lib):
    from paper_1306_5390_gb300 import hgrms
    for beta in range(1, 8):
        t = hgrms.hgrms_default_passes(beta)
        assert t >= 1 and hgrms.hgrms_has_kernel(beta, t) == 1
        assert hgrms.hgrms_has_kernel(beta, 1) == 1
    assert hgrms.hgrms_default_passes(0) == hgrms.HGRMS_EINVAL
    assert hgrms.hgrms_default_passes(8) == hgrms.HGRMS_EINVAL
    assert hgrms.hgrms_has_kernel(8, 1) == 0
    assert hgrms.hgrms_has_kernel(3, 4) == 0  # halo T*beta = 12 exceeds the tile margin


def test_no_gpu_is_reported_not_hidden(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1306_5390_gb300 import hgrms
    h = ctypes.c_void_p()
    assert lib.hgrms_create(ctypes.byref(h), 0, None) == hgrms.HGRMS_ENODEV
    assert h.value is None
    with pytest.raises(hgrms.HgrmsError):
        hgrms.Denoiser(0)


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_1306_5390_gb300 import hgrms
    monkeypatch.setattr(hgrms, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        hgrms.load_library(str(tmp_path / "nope.so"))


def test_server_without_device(lib):
    """Creating a server needs a CUDA device (ENODEV here); bad arguments
    are rejected first."""
    import ctypes
    from paper_1306_5390_gb300 import hgrms
    h = ctypes.c_void_p()
    assert lib.hgrms_server_create(None, 0, 1 << 30, 2) == hgrms.HGRMS_EINVAL
    assert lib.hgrms_server_create(ctypes.byref(h), 0, 1 << 30, 0) == hgrms.HGRMS_EINVAL
    rc = lib.hgrms_server_create(ctypes.byref(h), 0, 1 << 30, 2)
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except ImportError:
        has_gpu = False
    if not has_gpu:
        assert rc == hgrms.HGRMS_ENODEV and not h.value
    else:
        assert rc == hgrms.HGRMS_OK
        lib.hgrms_server_destroy(h)
    lib.hgrms_server_destroy(None)  # accepted
    assert lib.hgrms_server_wait(None, 1, 0.0, None) == hgrms.HGRMS_EINVAL
    assert lib.hgrms_server_fail_allocations(None, 1) == hgrms.HGRMS_EINVAL


def test_header_constants_match_the_binding():
    """Every #define HGRMS_* integer constant of the header has the same value
    in the Python binding."""
    from paper_1306_5390_gb300 import hgrms
    text = open(HEADER).read()
    found = 0
    for name, val in re.findall(r"#define\s+(HGRMS_[A-Z0-9_]+)\s+\(?(-?\d+)\)?\s", text):
        assert getattr(hgrms, name) == int(val), name
        found += 1
    m = re.search(r"#define\s+HGRMS_NOALLOC_SCRATCH_BYTES\s+\((\d+)u << (\d+)\)", text)
    assert m and hgrms.HGRMS_NOALLOC_SCRATCH_BYTES == int(m.group(1)) << int(m.group(2))
    assert found >= 20
