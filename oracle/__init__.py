"""CPU oracle for the P-HGRMS denoiser (TEST INFRASTRUCTURE ONLY).

Python access to ``hgrms_oracle.c``: a plain, slow, single-threaded C
implementation of Algorithms 1 and 2 of the paper and of the Section 2
iteration.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may use it.  The CUDA library does not depend on it and
shares no code with it.

``build()`` compiles the C file with gcc into ``oracle/_build/liboracle.so``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hgrms_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no architecture-specific flags)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    os.makedirs(_LIB_DIR, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    u8p = ctypes.POINTER(ctypes.c_uint8)
    i32p = ctypes.POINTER(ctypes.c_int32)
    lib.hgo_isqrt.argtypes = [ctypes.c_uint32]
    lib.hgo_isqrt.restype = ctypes.c_uint32
    lib.hgo_literal_find_isolated.argtypes = [u8p, i32p] + [ctypes.c_int] * 4
    lib.hgo_literal_find_isolated.restype = None
    lib.hgo_literal_remove_noise.argtypes = [u8p, u8p, i32p] + [ctypes.c_int] * 4
    lib.hgo_literal_remove_noise.restype = ctypes.c_long
    lib.hgo_literal_denoise.argtypes = [u8p] + [ctypes.c_int] * 5 + [
        ctypes.POINTER(ctypes.c_int)]
    lib.hgo_literal_denoise.restype = ctypes.c_int
    lib.hgo_card.argtypes = [u8p, i32p] + [ctypes.c_int] * 4
    lib.hgo_card.restype = None
    lib.hgo_pass.argtypes = [u8p, u8p] + [ctypes.c_int] * 4
    lib.hgo_pass.restype = ctypes.c_long
    lib.hgo_denoise.argtypes = [u8p] + [ctypes.c_int] * 5 + [
        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_long)]
    lib.hgo_denoise.restype = ctypes.c_int
    lib.hgo_psnr.argtypes = [u8p, u8p, ctypes.c_long]
    lib.hgo_psnr.restype = ctypes.c_double
    _lib = lib
    return lib


def _u8(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _i32(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _img(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.uint8)
    if a.ndim != 2:
        raise ValueError("image must be 2-D (rows, cols)")
    return a


def isqrt(x: int) -> int:
    return int(_load().hgo_isqrt(int(x)))


def card(img, alpha: int, beta: int) -> np.ndarray:
    """Cardinality matrix C (gather form of Algorithm 1), int32."""
    img = _img(img)
    out = np.zeros(img.shape, dtype=np.int32)
    _load().hgo_card(_u8(img), _i32(out), img.shape[0], img.shape[1], alpha, beta)
    return out


def literal_card(img, alpha: int, beta: int) -> np.ndarray:
    """Cardinality matrix C built by scattered increments (Algorithm 1)."""
    img = _img(img)
    out = np.zeros(img.shape, dtype=np.int32)
    _load().hgo_literal_find_isolated(_u8(img), _i32(out), img.shape[0],
                                      img.shape[1], alpha, beta)
    return out


def literal_remove_noise(img, card_m, alpha: int, beta: int):
    """Algorithm 2 as printed, into a copy of img.  Returns (I', changed)."""
    img = _img(img)
    card_m = np.ascontiguousarray(card_m, dtype=np.int32)
    temp = img.copy()
    ch = _load().hgo_literal_remove_noise(_u8(img), _u8(temp), _i32(card_m),
                                          img.shape[0], img.shape[1], alpha, beta)
    return temp, int(ch)


def one_pass(img, alpha: int, beta: int):
    """One pass (Algorithm 1 then 2).  Returns (out, changed_pixel_count)."""
    img = _img(img)
    out = np.empty_like(img)
    ch = _load().hgo_pass(_u8(img), _u8(out), img.shape[0], img.shape[1],
                          alpha, beta)
    return out, int(ch)


def denoise(img, alpha: int, beta: int, max_k: int, return_changes: bool = False):
    """Iterate passes to a fixed point or max_k changing passes.

    Returns (out, k, converged) or, with ``return_changes``, also the list of
    changed-pixel counts per pass run."""
    out = _img(img).copy()
    conv = ctypes.c_int(0)
    changes = (ctypes.c_long * (max_k + 1))()
    k = _load().hgo_denoise(_u8(out), out.shape[0], out.shape[1], alpha, beta,
                            max_k, ctypes.byref(conv), changes)
    if k < 0:
        raise MemoryError("oracle: out of host memory")
    if return_changes:
        npass = k + (1 if conv.value else 0)
        return out, k, bool(conv.value), [int(changes[i]) for i in range(npass)]
    return out, k, bool(conv.value)


def literal_denoise(img, alpha: int, beta: int, max_k: int):
    """The literal Algorithm 1 / Algorithm 2 / copy-back loop."""
    out = _img(img).copy()
    conv = ctypes.c_int(0)
    k = _load().hgo_literal_denoise(_u8(out), out.shape[0], out.shape[1], alpha,
                                    beta, max_k, ctypes.byref(conv))
    if k < 0:
        raise MemoryError("oracle: out of host memory")
    return out, k, bool(conv.value)


def psnr(ref, img) -> float:
    ref = np.ascontiguousarray(ref, dtype=np.uint8)
    img = np.ascontiguousarray(img, dtype=np.uint8)
    if ref.shape != img.shape:
        raise ValueError("shape mismatch")
    return float(_load().hgo_psnr(_u8(ref), _u8(img), ref.size))
