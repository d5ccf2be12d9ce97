"""ctypes binding of the C ABI in ``include/hgrms.h`` (argument marshalling only).

Every step of the method runs in the CUDA library ``_lib/libhgrms.so``.  The
functions below have the C names; ``denoise`` / ``denoise_batch`` are thin
conveniences that accept numpy arrays (host memory) or CUDA torch tensors
(device memory, denoised in place).  If the library is missing or cannot be
loaded, every call raises ``RuntimeError``: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libhgrms.so")

HGRMS_OK = 0
HGRMS_EINVAL = -1
HGRMS_ENOMEM = -2
HGRMS_ECUDA = -3
HGRMS_ETIMEOUT = -4
HGRMS_ENODEV = -5
HGRMS_ETOOBIG = -6
HGRMS_EAGAIN = -7
HGRMS_EBUSY = -8
HGRMS_NOALLOC_SCRATCH_BYTES = 16 << 20

HGRMS_OPT_KERNEL = 1
HGRMS_OPT_PASSES = 2
HGRMS_OPT_TIMING = 3
HGRMS_OPT_LIST_CAP = 4
HGRMS_OPT_BATCH_MB = 5
HGRMS_OPT_RELAUNCH_PPM = 6
HGRMS_OPT_TILE_EVAL_MAX = 7
HGRMS_OPT_AUTOTUNE = 8
HGRMS_OPT_PREDICT_K = 9
HGRMS_OPT_LIST_CTAS = 10
HGRMS_OPT_GRAPH = 11
HGRMS_OPT_WAIT_TEST = 12
HGRMS_OPT_TMA = 13

# Every symbol the header declares (the CPU tests check the library exports them).
EXPORTED = (
    "hgrms_create", "hgrms_destroy", "hgrms_denoise", "hgrms_denoise_batch", "hgrms_denoise_async", "hgrms_wait",
    "hgrms_converged", "hgrms_strerror", "hgrms_last_cuda_error", "hgrms_set_option",
    "hgrms_stats", "hgrms_launch_times", "hgrms_default_passes", "hgrms_has_kernel",
    "hgrms_denoise_noalloc", "hgrms_server_create", "hgrms_server_submit", "hgrms_server_wait",
    "hgrms_server_stats", "hgrms_server_fail_allocations", "hgrms_server_destroy", "hgrms_predictor_load",
    "hgrms_predict_k",
    "hgrms_predictor_train", "hgrms_predictor_grad", "hgrms_rms",
)

PREDICTOR_WEIGHTS = 9 * 16 + 3 * 9 * 16 * 16 + 4 * 16 + 33  # floats per network


class hgrms_request_info_t(ctypes.Structure):
    _fields_ = [
        ("k", ctypes.c_int),
        ("latency_ms", ctypes.c_double),
        ("queue_ms", ctypes.c_double),
        ("batch_size", ctypes.c_int),
        ("slot", ctypes.c_int),
    ]


class hgrms_stats_t(ctypes.Structure):
    _fields_ = [
        ("launches", ctypes.c_int),
        ("work_launches", ctypes.c_int),
        ("passes", ctypes.c_int),
        ("passes_executed", ctypes.c_int),
        ("passes_per_launch", ctypes.c_int),
        ("tile_rows", ctypes.c_int),
        ("tile_cols", ctypes.c_int),
        ("ctas_per_launch", ctypes.c_longlong),
        ("kernel_ms", ctypes.c_double),
        ("idle_kernel_ms", ctypes.c_double),
        ("evals_fused", ctypes.c_longlong),
        ("evals_list", ctypes.c_longlong),
        ("tile_eval_max", ctypes.c_int),
        ("autotuned", ctypes.c_int),
        ("tune_ms", ctypes.c_double),
        ("k_pred", ctypes.c_double),
        ("graph", ctypes.c_int),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class HgrmsError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})" if what else f"{strerror(code)} ({code})")


_lib = None
_lock = threading.Lock()


def load_library(path: str | None = None):
    """Load (once) and return the ctypes library; raises RuntimeError if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(
                f"CUDA library not built: {p} is missing (run __graft_entry__.build() "
                "or python -m paper_1306_5390_gb300.build)")
        lib = ctypes.CDLL(p)
        vp = ctypes.c_void_p
        ip = ctypes.POINTER(ctypes.c_int)
        lib.hgrms_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp]
        lib.hgrms_create.restype = ctypes.c_int
        lib.hgrms_destroy.argtypes = [vp]
        lib.hgrms_destroy.restype = None
        lib.hgrms_denoise.argtypes = [vp, vp] + [ctypes.c_int] * 5
        lib.hgrms_denoise.restype = ctypes.c_int
        lib.hgrms_denoise_async.argtypes = [vp, vp] + [ctypes.c_int] * 5
        lib.hgrms_denoise_async.restype = ctypes.c_int
        lib.hgrms_wait.argtypes = [vp]
        lib.hgrms_wait.restype = ctypes.c_int
        lib.hgrms_denoise_batch.argtypes = [vp, ctypes.POINTER(vp), ip, ip] + [ctypes.c_int] * 4 + [ip]
        lib.hgrms_denoise_batch.restype = ctypes.c_int
        lib.hgrms_converged.argtypes = [vp]
        lib.hgrms_converged.restype = ctypes.c_int
        lib.hgrms_strerror.argtypes = [ctypes.c_int]
        lib.hgrms_strerror.restype = ctypes.c_char_p
        lib.hgrms_last_cuda_error.argtypes = [vp]
        lib.hgrms_last_cuda_error.restype = ctypes.c_int
        lib.hgrms_set_option.argtypes = [vp, ctypes.c_int, ctypes.c_int]
        lib.hgrms_set_option.restype = ctypes.c_int
        lib.hgrms_stats.argtypes = [vp, ctypes.POINTER(hgrms_stats_t)]
        lib.hgrms_stats.restype = ctypes.c_int
        lib.hgrms_launch_times.argtypes = [vp, ctypes.POINTER(ctypes.c_float), ip, ctypes.c_int]
        lib.hgrms_launch_times.restype = ctypes.c_int
        lib.hgrms_denoise_noalloc.argtypes = [vp] + [ctypes.c_int] * 5 + [vp]
        lib.hgrms_denoise_noalloc.restype = ctypes.c_int
        lib.hgrms_rms.argtypes = [vp, vp, vp, ctypes.c_int, vp]
        lib.hgrms_rms.restype = ctypes.c_int
        lib.hgrms_default_passes.argtypes = [ctypes.c_int]
        lib.hgrms_default_passes.restype = ctypes.c_int
        lib.hgrms_has_kernel.argtypes = [ctypes.c_int, ctypes.c_int]
        lib.hgrms_has_kernel.restype = ctypes.c_int
        llp = ctypes.POINTER(ctypes.c_longlong)
        lib.hgrms_server_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_longlong, ctypes.c_int]
        lib.hgrms_server_create.restype = ctypes.c_int
        lib.hgrms_server_submit.argtypes = [vp, vp, vp] + [ctypes.c_int] * 5 + [ctypes.POINTER(ctypes.c_ulonglong)]
        lib.hgrms_server_submit.restype = ctypes.c_int
        lib.hgrms_server_wait.argtypes = [vp, ctypes.c_ulonglong, ctypes.c_double,
                                          ctypes.POINTER(hgrms_request_info_t)]
        lib.hgrms_server_wait.restype = ctypes.c_int
        lib.hgrms_server_stats.argtypes = [vp, llp, llp, llp, llp]
        lib.hgrms_server_stats.restype = ctypes.c_int
        lib.hgrms_server_fail_allocations.argtypes = [vp, ctypes.c_int]
        lib.hgrms_server_fail_allocations.restype = ctypes.c_int
        lib.hgrms_server_destroy.argtypes = [vp]
        lib.hgrms_server_destroy.restype = None
        fp = ctypes.POINTER(ctypes.c_float)
        lib.hgrms_predictor_load.argtypes = [vp, ctypes.c_int, fp, ctypes.c_int]
        lib.hgrms_predictor_load.restype = ctypes.c_int
        lib.hgrms_predict_k.argtypes = [vp, ctypes.c_int, ctypes.POINTER(vp), ip, ip, ctypes.c_int, fp, fp, fp, fp]
        lib.hgrms_predict_k.restype = ctypes.c_int
        lib.hgrms_predictor_train.argtypes = [vp, fp, fp, fp, fp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_float, ctypes.c_ulonglong, fp]
        lib.hgrms_predictor_train.restype = ctypes.c_int
        lib.hgrms_predictor_grad.argtypes = [vp, fp, fp, fp, fp, ctypes.c_int, fp, fp]
        lib.hgrms_predictor_grad.restype = ctypes.c_int
        _lib = lib
        return lib


# ---- C-named functions -----------------------------------------------------

def hgrms_create(device: int = 0, cuda_stream: int | None = None) -> int:
    h = ctypes.c_void_p()
    rc = load_library().hgrms_create(ctypes.byref(h), int(device), cuda_stream)
    if rc != HGRMS_OK:
        raise HgrmsError(rc, "hgrms_create")
    return h.value


def hgrms_destroy(h) -> None:
    load_library().hgrms_destroy(h)


def hgrms_denoise(h, img_ptr: int, rows: int, cols: int, alpha: int, beta: int, max_k: int) -> int:
    """Raw call: returns k or a negative code (not raised)."""
    return load_library().hgrms_denoise(h, img_ptr, rows, cols, alpha, beta, max_k)


def hgrms_denoise_async(h, img_ptr: int, rows: int, cols: int, alpha: int, beta: int, max_k: int) -> int:
    """Raw call: queues the call; returns 0 or a negative code (not raised)."""
    return load_library().hgrms_denoise_async(h, img_ptr, rows, cols, alpha, beta, max_k)


def hgrms_wait(h) -> int:
    """Raw call: k of the queued call, or a negative code (not raised)."""
    return load_library().hgrms_wait(h)


def hgrms_denoise_batch(h, ptrs, rows, cols, alpha: int, beta: int, max_k: int, k_out) -> int:
    n = len(ptrs)
    P = (ctypes.c_void_p * max(n, 1))(*ptrs)
    R = (ctypes.c_int * max(n, 1))(*rows)
    C = (ctypes.c_int * max(n, 1))(*cols)
    K = (ctypes.c_int * max(n, 1))()
    rc = load_library().hgrms_denoise_batch(h, P, R, C, n, alpha, beta, max_k, K)
    for i in range(n):
        k_out[i] = K[i]
    return rc


def hgrms_denoise_noalloc(img_ptr: int, rows: int, cols: int, alpha: int, beta: int, max_k: int,
                          cuda_stream: int | None = None) -> int:
    """Raw call of the allocation-free entry point: returns k or a negative code."""
    return load_library().hgrms_denoise_noalloc(img_ptr, rows, cols, alpha, beta, max_k, cuda_stream)


def hgrms_converged(h) -> int:
    return load_library().hgrms_converged(h)


def strerror(code: int) -> str:
    return load_library().hgrms_strerror(int(code)).decode()


hgrms_strerror = strerror


def hgrms_last_cuda_error(h) -> int:
    return load_library().hgrms_last_cuda_error(h)


def hgrms_set_option(h, option: int, value: int) -> int:
    return load_library().hgrms_set_option(h, option, value)


def hgrms_stats(h) -> dict:
    st = hgrms_stats_t()
    rc = load_library().hgrms_stats(h, ctypes.byref(st))
    if rc != HGRMS_OK:
        raise HgrmsError(rc, "hgrms_stats")
    return st.as_dict()


def hgrms_launch_times(h):
    """[(ms, kind)] per launch of the last call (kind 0 fused, 1 list, 2 unfused, 3 ran no pass)."""
    lib = load_library()
    n = lib.hgrms_launch_times(h, None, None, 0)
    if n < 0:
        raise HgrmsError(n, "hgrms_launch_times")
    ms = (ctypes.c_float * max(n, 1))()
    kd = (ctypes.c_int * max(n, 1))()
    lib.hgrms_launch_times(h, ms, kd, n)
    return [(float(ms[i]), int(kd[i])) for i in range(n)]


def hgrms_default_passes(beta: int) -> int:
    return load_library().hgrms_default_passes(beta)


def hgrms_has_kernel(beta: int, passes: int) -> int:
    return load_library().hgrms_has_kernel(beta, passes)


# ---- Conveniences --------------------------------------------------------

class Denoiser:
    """Owns one library handle (one device, one stream)."""

    def __init__(self, device: int = 0, cuda_stream: int | None = None, kernel: int = 0,
                 passes: int = 0, timing: bool = False, autotune: bool = False):
        self.h = hgrms_create(device, cuda_stream)
        self.device = device
        self.set_option(HGRMS_OPT_KERNEL, kernel)
        self.set_option(HGRMS_OPT_PASSES, passes)
        self.set_option(HGRMS_OPT_AUTOTUNE, int(bool(autotune)))
        self.set_option(HGRMS_OPT_TIMING, int(bool(timing)))

    def set_option(self, opt: int, value: int) -> None:
        rc = hgrms_set_option(self.h, opt, value)
        if rc != HGRMS_OK:
            raise HgrmsError(rc, "hgrms_set_option")

    def close(self) -> None:
        if self.h:
            hgrms_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _ptr_shape(img):
        if isinstance(img, np.ndarray):
            if img.dtype != np.uint8 or img.ndim != 2 or not img.flags.c_contiguous:
                raise ValueError("image must be a C-contiguous 2-D uint8 array")
            return img.ctypes.data, img.shape[0], img.shape[1]
        # torch tensor (duck-typed: no import of torch here)
        if img.dim() != 2 or not img.is_contiguous() or str(img.dtype) != "torch.uint8":
            raise ValueError("image must be a contiguous 2-D uint8 tensor")
        return img.data_ptr(), img.shape[0], img.shape[1]

    def denoise(self, img, alpha: int, beta: int, max_k: int) -> int:
        """Denoise ``img`` in place; returns k.  ``img``: numpy (host) or CUDA tensor."""
        ptr, rows, cols = self._ptr_shape(img)
        k = hgrms_denoise(self.h, ptr, rows, cols, alpha, beta, max_k)
        if k < 0:
            raise HgrmsError(k, "hgrms_denoise")
        return k

    def denoise_async(self, img, alpha: int, beta: int, max_k: int) -> None:
        """Queue the in-place denoising of ``img`` (a CUDA tensor, or page-locked
        host memory the device can read) on the handle's stream; ``wait()``
        returns k."""
        ptr, rows, cols = self._ptr_shape(img)
        rc = hgrms_denoise_async(self.h, ptr, rows, cols, alpha, beta, max_k)
        if rc < 0:
            raise HgrmsError(rc, "hgrms_denoise_async")

    def wait(self) -> int:
        """Finish the call queued by ``denoise_async``; returns its k."""
        k = hgrms_wait(self.h)
        if k < 0:
            raise HgrmsError(k, "hgrms_wait")
        return k

    def denoise_batch(self, imgs, alpha: int, beta: int, max_k: int):
        ps = [self._ptr_shape(im) for im in imgs]
        ks = [0] * len(ps)
        rc = hgrms_denoise_batch(self.h, [p[0] for p in ps], [p[1] for p in ps], [p[2] for p in ps],
                                 alpha, beta, max_k, ks)
        if rc != HGRMS_OK:
            raise HgrmsError(rc, "hgrms_denoise_batch")
        return ks

    def converged(self) -> bool:
        return hgrms_converged(self.h) == 1

    def load_predictor(self, beta: int, weights=None) -> None:
        """Load the k-predictor network for beta (float32 weights in the
        order hgrms_predictor_load documents; default: the fitted weights
        shipped with the package, predictor_b<beta>.npy)."""
        if weights is None:
            weights = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), f"predictor_b{beta}.npy"))
        w = np.ascontiguousarray(weights, dtype=np.float32).ravel()
        rc = load_library().hgrms_predictor_load(self.h, int(beta), w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                 int(w.size))
        if rc != HGRMS_OK:
            raise HgrmsError(rc, "hgrms_predictor_load")

    def train_predictor(self, weights, x0, hist, k, epochs: int, batch: int = 256, lr: float = 3e-3,
                        seed: int = 1):
        """Fit the predictor on the device; returns (fitted weights, last
        epoch's mean loss)."""
        fp = ctypes.POINTER(ctypes.c_float)
        w = np.ascontiguousarray(weights, dtype=np.float32).ravel().copy()
        x0 = np.ascontiguousarray(x0, dtype=np.float32)
        hist = np.ascontiguousarray(hist, dtype=np.float32)
        k = np.ascontiguousarray(k, dtype=np.float32)
        loss = ctypes.c_float()
        rc = load_library().hgrms_predictor_train(self.h, w.ctypes.data_as(fp), x0.ctypes.data_as(fp),
                                                  hist.ctypes.data_as(fp), k.ctypes.data_as(fp), int(len(k)),
                                                  int(epochs), int(batch), float(lr), int(seed), ctypes.byref(loss))
        if rc != HGRMS_OK:
            raise HgrmsError(rc, "hgrms_predictor_train")
        return w, loss.value

    def predictor_grad(self, weights, x0, hist, k):
        """(gradient, loss) of the mean squared k error over all images."""
        fp = ctypes.POINTER(ctypes.c_float)
        w = np.ascontiguousarray(weights, dtype=np.float32).ravel()
        x0 = np.ascontiguousarray(x0, dtype=np.float32)
        hist = np.ascontiguousarray(hist, dtype=np.float32)
        k = np.ascontiguousarray(k, dtype=np.float32)
        g = np.zeros(PREDICTOR_WEIGHTS, dtype=np.float32)
        loss = ctypes.c_float()
        rc = load_library().hgrms_predictor_grad(self.h, w.ctypes.data_as(fp), x0.ctypes.data_as(fp),
                                                 hist.ctypes.data_as(fp), k.ctypes.data_as(fp), int(len(k)),
                                                 g.ctypes.data_as(fp), ctypes.byref(loss))
        if rc != HGRMS_OK:
            raise HgrmsError(rc, "hgrms_predictor_grad")
        return g, loss.value

    def predict_k(self, beta: int, imgs, features: bool = False):
        """Predicted k per image (device-readable images); with features=True
        also (x0 [n,64,64], hist [n,16], gap [n,16])."""
        ps = [self._ptr_shape(im) for im in imgs]
        n = len(ps)
        kh = np.zeros(n, dtype=np.float32)
        fp = ctypes.POINTER(ctypes.c_float)
        x0 = np.zeros((n, 64, 64), dtype=np.float32) if features else None
        hist = np.zeros((n, 16), dtype=np.float32) if features else None
        gap = np.zeros((n, 16), dtype=np.float32) if features else None
        arr = (ctypes.c_void_p * max(1, n))(*[p[0] for p in ps])
        rows = (ctypes.c_int * max(1, n))(*[p[1] for p in ps])
        cols = (ctypes.c_int * max(1, n))(*[p[2] for p in ps])

        def ptr(a):
            return a.ctypes.data_as(fp) if a is not None else None
        rc = load_library().hgrms_predict_k(self.h, int(beta), arr, rows, cols, n, ptr(kh), ptr(x0), ptr(hist), ptr(gap))
        if rc != HGRMS_OK:
            raise HgrmsError(rc, "hgrms_predict_k")
        return (kh, x0, hist, gap) if features else kh

    def stats(self) -> dict:
        return hgrms_stats(self.h)

    def launch_times(self):
        return hgrms_launch_times(self.h)


def denoise(img, alpha: int, beta: int, max_k: int, device: int = 0) -> int:
    """One-shot in-place denoise (creates and frees a handle)."""
    with Denoiser(device) as d:
        return d.denoise(img, alpha, beta, max_k)


class Server:
    """Continuous-batching request server (hgrms_server_*): submit images
    (host numpy arrays, or CUDA tensors denoised in place), wait for results.

        with Server(0, hbm_budget_bytes=40 << 30, slots=4) as srv:
            rid = srv.submit(img, alpha=10, beta=1, max_k=32)
            k, info = srv.wait(rid)
    """

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 40 << 30, slots: int = 4):
        lib = load_library()
        h = ctypes.c_void_p()
        rc = lib.hgrms_server_create(ctypes.byref(h), int(device), int(hbm_budget_bytes), int(slots))
        if rc != HGRMS_OK:
            raise HgrmsError(rc, "hgrms_server_create")
        self.h = h.value
        self._keep = {}  # request id -> the buffers the request uses

    def submit(self, img, alpha: int, beta: int, max_k: int, out=None) -> int:
        """Queue `img` (2-D uint8 numpy array or CUDA tensor).  A host image's
        result goes to `out` (default: in place); returns the request id."""
        if hasattr(img, "data_ptr"):
            if not img.is_contiguous():
                raise ValueError("image must be contiguous")
            src = img.data_ptr()
            dst = None
            rows, cols = img.shape
        else:
            if not img.flags["C_CONTIGUOUS"] or img.dtype.itemsize != 1:
                raise ValueError("image must be a C-contiguous uint8 array")
            if out is None:
                out = img
            src = img.ctypes.data
            dst = out.ctypes.data
            rows, cols = img.shape
        rid = ctypes.c_ulonglong()
        rc = load_library().hgrms_server_submit(self.h, src, dst, int(rows), int(cols), int(alpha), int(beta),
                                                int(max_k), ctypes.byref(rid))
        if rc != HGRMS_OK:
            raise HgrmsError(rc, "hgrms_server_submit")
        self._keep[rid.value] = (img, out)
        return rid.value

    def wait(self, rid: int, timeout_s: float = -1.0):
        """(k, info dict) of request `rid` once served."""
        info = hgrms_request_info_t()
        rc = load_library().hgrms_server_wait(self.h, ctypes.c_ulonglong(rid), float(timeout_s), ctypes.byref(info))
        if rc == HGRMS_EAGAIN:
            raise TimeoutError(f"request {rid} not finished")
        self._keep.pop(rid, None)
        if rc < 0:
            raise HgrmsError(rc, "hgrms_server_wait")
        return rc, {f: getattr(info, f) for f, _ in info._fields_}

    def stats(self) -> dict:
        v = [ctypes.c_longlong() for _ in range(4)]
        err = load_library().hgrms_server_stats(self.h, *[ctypes.byref(x) for x in v])
        return dict(served=v[0].value, batches=v[1].value, queued=v[2].value, max_in_flight=v[3].value,
                    error=err)

    def fail_allocations(self, n: int) -> None:
        """Tests of the failure path: the next n buffer allocations of the
        slots fail (hgrms_server_fail_allocations)."""
        rc = load_library().hgrms_server_fail_allocations(self.h, int(n))
        if rc < 0:
            raise HgrmsError(rc, "hgrms_server_fail_allocations")

    def close(self) -> None:
        if self.h:
            load_library().hgrms_server_destroy(self.h)
            self.h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
