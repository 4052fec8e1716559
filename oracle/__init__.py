"""CPU oracle for the JPEG decode back-end (test infrastructure only).

The oracle is the plain statement of what the GPU back-end computes
(dequantisation, the Eq. 1/Eq. 2 fixed-point IDCT with range-limit clamp,
Alg. 1 upsampling and its 4:2:0 reading, Alg. 2 colour conversion in fixed
point) plus a baseline Huffman decoder.  It is plain C (``orc_*.c``) compiled
with gcc and called through ctypes.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path
and never calls it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = ["orc_idct.c", "orc_idct_aan.c", "orc_color.c", "orc_upsample.c", "orc_backend.c", "orc_huffman.c"]
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liborc.so`` (gcc, -O2 -fwrapv)."""
    srcs = [os.path.join(_HERE, s) for s in _SRC] + [os.path.join(_HERE, "orc.h")]
    if not force and os.path.exists(_LIB):
        t = os.path.getmtime(_LIB)
        if all(os.path.getmtime(s) <= t for s in srcs):
            return _LIB
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fwrapv", "-fno-strict-aliasing", "-fPIC", "-shared",
           "-Wall", "-Wno-unused-function", "-o", tmp] + [os.path.join(_HERE, s) for s in _SRC] + ["-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class OrcImage(ctypes.Structure):
    _fields_ = [
        ("width", ctypes.c_int32), ("height", ctypes.c_int32),
        ("h_samp", ctypes.c_int32 * 3), ("v_samp", ctypes.c_int32 * 3),
        ("coef", ctypes.c_void_p * 3),
        ("blocks_w", ctypes.c_int32 * 3), ("blocks_h", ctypes.c_int32 * 3),
        ("qtab", ctypes.c_void_p * 3),
        ("fancy", ctypes.c_int32),
        ("idct", ctypes.c_int32),
    ]


class OrcJpegInfo(ctypes.Structure):
    _fields_ = [
        ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("ncomp", ctypes.c_int32),
        ("h_samp", ctypes.c_int32 * 3), ("v_samp", ctypes.c_int32 * 3),
        ("blocks_w", ctypes.c_int32 * 3), ("blocks_h", ctypes.c_int32 * 3),
        ("qtab", (ctypes.c_uint16 * 64) * 3),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            _lib.orc_idct_block.argtypes = [P, P, P]
            _lib.orc_idct_core.argtypes = [P, P, P]
            _lib.orc_idct_blocks.argtypes = [P, P, P, ctypes.c_int64]
            _lib.orc_idct_core_blocks.argtypes = [P, P, P, ctypes.c_int64]
            _lib.orc_idct_constants.argtypes = [P]
            _lib.orc_idct_aan_blocks.argtypes = [P, P, P, ctypes.c_int64]
            _lib.orc_idct_aan_core_blocks.argtypes = [P, P, P, ctypes.c_int64]
            _lib.orc_idct_aan_constants.argtypes = [P, P]
            _lib.orc_ycc_to_rgb.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P]
            _lib.orc_ycc_to_rgb_all.argtypes = [P]
            _lib.orc_upsample.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                          ctypes.c_int, ctypes.c_int, ctypes.c_int, P, ctypes.c_int64]
            _lib.orc_backend_decode.argtypes = [ctypes.POINTER(OrcImage), P, ctypes.c_int64]
            _lib.orc_backend_decode.restype = ctypes.c_int
            _lib.orc_backend_decode_gray.argtypes = [ctypes.c_int32, ctypes.c_int32, P, ctypes.c_int32, ctypes.c_int32,
                                                     P, P, ctypes.c_int64, ctypes.c_int32]
            _lib.orc_backend_decode_gray.restype = ctypes.c_int
            _lib.orc_backend_decode_mt.argtypes = [ctypes.POINTER(OrcImage), P, ctypes.c_int64, ctypes.c_int]
            _lib.orc_backend_decode_mt.restype = ctypes.c_int
            _lib.orc_jpeg_decode_coefs.argtypes = [P, ctypes.c_int64, ctypes.POINTER(OrcJpegInfo),
                                                   ctypes.POINTER(ctypes.c_void_p * 3)]
            _lib.orc_jpeg_decode_coefs.restype = ctypes.c_int
        return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


# ---- IDCT ------------------------------------------------------------------

def idct_constants() -> np.ndarray:
    k = np.zeros(12, np.int32)
    lib().orc_idct_constants(_ptr(k))
    return k


def idct_blocks(coef: np.ndarray, q: np.ndarray, aan: bool = False) -> np.ndarray:
    """coef (n, 64) int16 natural order, q (64,) -> (n, 64) uint8 samples
    (the LLM IDCT, or the AAN one with ``aan``)."""
    coef = np.ascontiguousarray(coef, np.int16).reshape(-1, 64)
    q = np.ascontiguousarray(q, np.uint16).reshape(64)
    out = np.zeros((coef.shape[0], 64), np.uint8)
    fn = lib().orc_idct_aan_blocks if aan else lib().orc_idct_blocks
    fn(_ptr(coef), _ptr(q), _ptr(out), coef.shape[0])
    return out


def idct_core_blocks(coef: np.ndarray, q: np.ndarray | None = None, aan: bool = False) -> np.ndarray:
    """Rounded 2-D IDCT without level shift / clamp, (n, 64) int32."""
    coef = np.ascontiguousarray(coef, np.int16).reshape(-1, 64)
    q = np.ones(64, np.uint16) if q is None else np.ascontiguousarray(q, np.uint16).reshape(64)
    out = np.zeros((coef.shape[0], 64), np.int32)
    fn = lib().orc_idct_aan_core_blocks if aan else lib().orc_idct_core_blocks
    fn(_ptr(coef), _ptr(q), _ptr(out), coef.shape[0])
    return out


def idct_aan_constants():
    """(S (8, 8) int32 scale table [v, u], (K1, K2, K3, K4)) of the AAN IDCT."""
    s = np.zeros(64, np.int32)
    k = np.zeros(4, np.int32)
    lib().orc_idct_aan_constants(_ptr(s), _ptr(k))
    return s.reshape(8, 8), tuple(int(v) for v in k)


# ---- colour conversion ----------------------------------------------------

def ycc_to_rgb_all() -> np.ndarray:
    """(256, 256, 256, 3) uint8 indexed [Y, Cb, Cr]."""
    out = np.zeros((256, 256, 256, 3), np.uint8)
    lib().orc_ycc_to_rgb_all(_ptr(out))
    return out


def ycc_to_rgb(y: int, cb: int, cr: int) -> tuple[int, int, int]:
    out = np.zeros(3, np.uint8)
    lib().orc_ycc_to_rgb(int(y), int(cb), int(cr), _ptr(out))
    return tuple(int(v) for v in out)


# ---- upsampling -------------------------------------------------------------

def upsample(plane: np.ndarray, sx: int, sy: int, fancy: bool) -> np.ndarray:
    plane = np.ascontiguousarray(plane, np.uint8)
    ch, cw = plane.shape
    out = np.zeros((ch * sy, cw * sx), np.uint8)
    lib().orc_upsample(_ptr(plane), cw, ch, cw, sx, sy, int(bool(fancy)), _ptr(out), cw * sx)
    return out


# ---- whole back-end -----------------------------------------------------------

def _orc_image(width, height, h_samp, v_samp, planes, qtabs, fancy, keep, aan=False):
    img = OrcImage()
    img.width, img.height = int(width), int(height)
    for c in range(3):
        p = np.ascontiguousarray(planes[c], np.int16)
        q = np.ascontiguousarray(qtabs[c], np.uint16).reshape(64)
        keep += [p, q]
        img.h_samp[c], img.v_samp[c] = int(h_samp[c]), int(v_samp[c])
        img.coef[c] = _ptr(p)
        img.blocks_h[c], img.blocks_w[c] = int(p.shape[0]), int(p.shape[1])
        img.qtab[c] = _ptr(q)
    img.fancy = int(bool(fancy))
    img.idct = int(bool(aan))
    return img


def backend_decode(width, height, h_samp, v_samp, planes, qtabs, fancy, threads: int = 1,
                   aan: bool = False) -> np.ndarray:
    """planes[c]: (blocks_h, blocks_w, 64) int16; returns (H, W, 3) uint8.
    ``aan`` selects the AAN IDCT instead of the LLM one."""
    keep = []
    img = _orc_image(width, height, h_samp, v_samp, planes, qtabs, fancy, keep, aan)
    out = np.zeros((height, width, 3), np.uint8)
    if threads <= 1:
        rc = lib().orc_backend_decode(ctypes.byref(img), _ptr(out), 3 * width)
    else:
        rc = lib().orc_backend_decode_mt(ctypes.byref(img), _ptr(out), 3 * width, int(threads))
        rc = 0 if rc > 0 else rc
    if rc != 0:
        raise ValueError("oracle: inconsistent image description")
    return out


def backend_decode_gray(width, height, plane, qtab, aan: bool = False) -> np.ndarray:
    """Single-component image: plane (blocks_h, blocks_w, 64) int16; returns
    (H, W, 3) uint8 with R = G = B = Y."""
    p = np.ascontiguousarray(plane, np.int16)
    q = np.ascontiguousarray(qtab, np.uint16).reshape(64)
    out = np.zeros((height, width, 3), np.uint8)
    rc = lib().orc_backend_decode_gray(int(width), int(height), _ptr(p), int(p.shape[1]), int(p.shape[0]), _ptr(q),
                                       _ptr(out), 3 * width, int(bool(aan)))
    if rc != 0:
        raise ValueError("oracle: inconsistent grayscale description")
    return out


# ---- entropy decoding -----------------------------------------------------------

def jpeg_decode_coefs(data: bytes):
    """Parse a baseline JFIF stream and Huffman-decode it.

    Returns (info dict, [plane0, plane1, plane2]) with planes shaped
    (blocks_h, blocks_w, 64) int16 in natural order."""
    buf = np.frombuffer(data, np.uint8).copy()
    info = OrcJpegInfo()
    rc = lib().orc_jpeg_decode_coefs(_ptr(buf), buf.size, ctypes.byref(info), None)
    if rc != 0:
        raise ValueError(f"oracle: malformed JPEG stream ({rc})")
    planes = [np.zeros((info.blocks_h[c], info.blocks_w[c], 64), np.int16) for c in range(3)]
    arr = (ctypes.c_void_p * 3)(*[_ptr(p) for p in planes])
    rc = lib().orc_jpeg_decode_coefs(_ptr(buf), buf.size, ctypes.byref(info), ctypes.byref(arr))
    if rc != 0:
        raise ValueError(f"oracle: malformed JPEG stream ({rc})")
    d = dict(width=info.width, height=info.height,
             h_samp=tuple(info.h_samp), v_samp=tuple(info.v_samp),
             qtabs=[np.array(info.qtab[c][:], np.uint16) for c in range(3)])
    return d, planes
