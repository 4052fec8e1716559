"""Python binding of the GB300 JPEG back-end (``libjdec.so``, C ABI in
``include/jdec.h``).

Argument marshalling only: every step of the decode runs in the library's
CUDA kernels.  Device buffers are torch CUDA tensors (PyTorch provides device
memory and streams); host buffers are numpy arrays.  If the library cannot be
loaded the import of the context fails loudly -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, ECUDA, EUNSUPPORTED, EBUSY, ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
UPSAMPLE_FANCY, UPSAMPLE_REPLICATE = 0, 1
IDCT_AAN = 2   # the AAN scaled IDCT instead of the default LLM form
TEST_WITHHOLD_LOADS = 0x80000000   # testing aid: the kernel's bounded waits run out (JDEC_ETIMEOUT)
SAMPLINGS = {"444": ((1, 1, 1), (1, 1, 1)), "422": ((2, 1, 1), (1, 1, 1)), "420": ((2, 1, 1), (2, 1, 1)),
             "440": ((1, 1, 1), (2, 1, 1))}


class JdecError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_str(status)} ({status})")


class JpegInfo(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("ncomp", ctypes.c_int32),
                ("h_samp", ctypes.c_uint8 * 3), ("v_samp", ctypes.c_uint8 * 3),
                ("blocks_w", ctypes.c_int32 * 3), ("blocks_h", ctypes.c_int32 * 3),
                ("qtab", (ctypes.c_uint16 * 64) * 3), ("restart_interval", ctypes.c_int32),
                ("scan_offset", ctypes.c_int64), ("scan_bytes", ctypes.c_int64)]


class Options(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_size_t), ("max_batch", ctypes.c_int),
                ("autotune", ctypes.c_int), ("tune_file", ctypes.c_char_p), ("jpeg_chunk_rows", ctypes.c_int)]


class Image(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("ncomp", ctypes.c_int32),
                ("h_samp", ctypes.c_uint8 * 3), ("v_samp", ctypes.c_uint8 * 3),
                ("coef", ctypes.c_void_p * 3),
                ("blocks_w", ctypes.c_int32 * 3), ("blocks_h", ctypes.c_int32 * 3),
                ("qtab", ctypes.c_void_p * 3),
                ("rgb", ctypes.c_void_p), ("rgb_pitch", ctypes.c_int64), ("flags", ctypes.c_uint32)]


def library_path() -> str:
    return os.path.join(_HERE, "_build", "libjdec.so")


def load(build_if_missing: bool = True, path: str | None = None):
    """Loads ``libjdec.so`` (building it first when it is missing or stale and
    nvcc is available), or the library at ``path``.  Raises if the library
    cannot be loaded."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if path is not None:
            build_if_missing = False
        path = path or library_path()
        if build_if_missing:
            try:
                from . import build as _b
                path = _b.build()
            except RuntimeError:
                if not os.path.exists(path):
                    raise
        if not os.path.exists(path):
            raise RuntimeError(f"GB300 back-end library missing: {path} (run the build first)")
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        lib.jdec_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(Options)]
        lib.jdec_create.restype = ctypes.c_int
        lib.jdec_decode_coeffs.argtypes = [P, ctypes.POINTER(Image), P]
        lib.jdec_decode_coeffs.restype = ctypes.c_int
        lib.jdec_decode_batch.argtypes = [P, ctypes.POINTER(Image), ctypes.c_int32, P]
        lib.jdec_decode_batch.restype = ctypes.c_int
        lib.jdec_decode_host.argtypes = [P, ctypes.POINTER(Image), P]
        lib.jdec_decode_host.restype = ctypes.c_int
        lib.jdec_decode_host_batch.argtypes = [P, ctypes.POINTER(Image), ctypes.c_int32, P]
        lib.jdec_decode_host_batch.restype = ctypes.c_int
        lib.jdec_sync_status.argtypes = [P, P]
        lib.jdec_sync_status.restype = ctypes.c_int
        lib.jdec_destroy.argtypes = [P]
        lib.jdec_destroy.restype = ctypes.c_int
        lib.jdec_status_str.argtypes = [ctypes.c_int]
        lib.jdec_status_str.restype = ctypes.c_char_p
        lib.jdec_decode_batch_static.argtypes = [ctypes.POINTER(Image), ctypes.c_int32, P]
        lib.jdec_decode_batch_static.restype = ctypes.c_int
        lib.jdec_batch_static_status.argtypes = [P]
        lib.jdec_batch_static_status.restype = ctypes.c_int
        lib.jdec_jpeg_parse.argtypes = [P, ctypes.c_size_t, ctypes.POINTER(JpegInfo)]
        lib.jdec_jpeg_parse.restype = ctypes.c_int
        lib.jdec_entropy_decode.argtypes = [P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p * 3)]
        lib.jdec_entropy_decode.restype = ctypes.c_int
        lib.jdec_entropy_decode_mt.argtypes = [P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p * 3),
                                               ctypes.c_int32]
        lib.jdec_entropy_decode_mt.restype = ctypes.c_int
        lib.jdec_decode_jpeg.argtypes = [P, P, ctypes.c_size_t, P, ctypes.c_int64, ctypes.c_uint32, ctypes.c_int32, P]
        lib.jdec_decode_jpeg.restype = ctypes.c_int
        _lib = lib
        return lib


def status_str(status: int) -> str:
    return load().jdec_status_str(int(status)).decode()


def exported_symbols() -> list[str]:
    return ["jdec_create", "jdec_decode_coeffs", "jdec_decode_batch", "jdec_decode_host",
            "jdec_sync_status", "jdec_destroy", "jdec_status_str", "jdec_jpeg_parse", "jdec_entropy_decode",
            "jdec_decode_batch_static", "jdec_decode_jpeg", "jdec_entropy_decode_mt", "jdec_decode_host_batch",
            "jdec_batch_static_status"]


def decode_batch_static(imgs, stream=None, check=True) -> int:
    """Allocation-free batched decode on the current device (see
    jdec_decode_batch_static in include/jdec.h)."""
    arr = (Image * len(imgs))(*imgs)
    st = load().jdec_decode_batch_static(arr, len(imgs), ctypes.c_void_p(_stream_ptr(stream)))
    if check and st != OK:
        raise JdecError(st, "jdec_decode_batch_static")
    return st


def batch_static_status(stream=None) -> int:
    """Waits for the stream and returns (and clears) the device-side status of
    the last allocation-free batch call (see jdec_batch_static_status)."""
    return load().jdec_batch_static_status(ctypes.c_void_p(_stream_ptr(stream)))


def jpeg_parse(data) -> JpegInfo:
    """Headers of a baseline JPEG stream (host only)."""
    buf = data if isinstance(data, (bytes, bytearray)) else bytes(data)
    info = JpegInfo()
    st = load().jdec_jpeg_parse(ctypes.c_char_p(bytes(buf)), len(buf), ctypes.byref(info))
    if st != OK:
        raise JdecError(st, "jdec_jpeg_parse")
    return info


def entropy_decode(data, planes, threads: int = 1) -> None:
    """Huffman-decodes `data` into host int16 planes (numpy arrays or pinned
    torch CPU tensors) shaped (blocks_h, blocks_w, 64) -- 3, or 1 for a
    grayscale stream -- on up to `threads` host threads when the stream has
    restart intervals.  Releases the GIL."""
    ptrs = (ctypes.c_void_p * 3)(*[(p.ctypes.data if isinstance(p, np.ndarray) else p.data_ptr()) for p in planes])
    buf = data if isinstance(data, bytes) else bytes(data)
    if threads > 1:
        st = load().jdec_entropy_decode_mt(ctypes.c_char_p(buf), len(buf), ctypes.byref(ptrs), int(threads))
    else:
        st = load().jdec_entropy_decode(ctypes.c_char_p(buf), len(buf), ctypes.byref(ptrs))
    if st != OK:
        raise JdecError(st, "jdec_entropy_decode")


def _stream_ptr(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _flags(fancy, aan):
    return (UPSAMPLE_FANCY if fancy else UPSAMPLE_REPLICATE) | (IDCT_AAN if aan else 0)


def make_image(width, height, sampling, planes, qtabs, rgb, rgb_pitch=None, fancy=True,
               keep=None, host=False, aan=False) -> Image:
    """Fills a ``jdec_image``.  planes: 3 int16 arrays/tensors shaped
    (blocks_h, blocks_w, 64), or 1 for a grayscale image (sampling "gray");
    qtabs: one host uint16 array of 64 per plane; rgb: uint8 buffer (device
    tensor, or host numpy array with ``host=True``); ``aan`` selects the AAN
    IDCT."""
    ncomp = len(planes)
    hs, vs = ((1, 1, 1), (1, 1, 1)) if ncomp == 1 else (SAMPLINGS[sampling] if isinstance(sampling, str) else sampling)
    im = Image()
    im.width, im.height, im.ncomp = int(width), int(height), ncomp
    keep = keep if keep is not None else []
    for c in range(3):
        im.h_samp[c], im.v_samp[c] = int(hs[c]), int(vs[c])
    for c in range(ncomp):
        p = planes[c]
        if host:
            p = np.ascontiguousarray(p, np.int16)
            im.coef[c] = p.ctypes.data
        else:
            assert p.is_cuda and p.dtype.itemsize == 2 and p.is_contiguous()
            im.coef[c] = p.data_ptr()
        keep.append(p)
        im.blocks_h[c], im.blocks_w[c] = int(p.shape[0]), int(p.shape[1])
        q = np.ascontiguousarray(np.asarray(qtabs[c]).reshape(64), np.uint16)
        keep.append(q)
        im.qtab[c] = q.ctypes.data
    if host:
        im.rgb = rgb.ctypes.data
        im.rgb_pitch = int(rgb_pitch if rgb_pitch is not None else rgb.strides[0])
    else:
        im.rgb = rgb.data_ptr()
        im.rgb_pitch = int(rgb_pitch if rgb_pitch is not None else rgb.stride(0))
    keep.append(rgb)
    im.flags = _flags(fancy, aan)
    return im


def make_image_flat(width, height, sampling, base_ptr: int, shapes, qtabs, rgb_ptr: int, rgb_pitch: int,
                    fancy=True, keep=None, aan=False) -> Image:
    """Fills a ``jdec_image`` whose planes lie one after another in one device
    buffer starting at ``base_ptr`` (shapes: (blocks_h, blocks_w) per plane;
    3 planes, or 1 for grayscale); ``rgb_ptr``: device RGB buffer."""
    ncomp = len(shapes)
    hs, vs = ((1, 1, 1), (1, 1, 1)) if ncomp == 1 else (SAMPLINGS[sampling] if isinstance(sampling, str) else sampling)
    im = Image()
    im.width, im.height, im.ncomp = int(width), int(height), ncomp
    keep = keep if keep is not None else []
    off = 0
    for c in range(3):
        im.h_samp[c], im.v_samp[c] = int(hs[c]), int(vs[c])
    for c in range(ncomp):
        bh, bw = int(shapes[c][0]), int(shapes[c][1])
        im.coef[c] = base_ptr + off
        off += bh * bw * 128
        im.blocks_h[c], im.blocks_w[c] = bh, bw
        q = np.ascontiguousarray(np.asarray(qtabs[c]).reshape(64), np.uint16)
        keep.append(q)
        im.qtab[c] = q.ctypes.data
    im.rgb = int(rgb_ptr)
    im.rgb_pitch = int(rgb_pitch)
    im.flags = _flags(fancy, aan)
    return im


class Context:
    """One ``jdec_ctx`` (not thread-safe: one per host thread)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, max_batch: int = 0,
                 autotune: bool = False, tune_file: str | None = None, jpeg_chunk_rows: int = 0):
        self._lib = load()
        self._opt = Options(int(device), int(hbm_budget_bytes), int(max_batch), int(bool(autotune)),
                            tune_file.encode() if tune_file else None, int(jpeg_chunk_rows))
        h = ctypes.c_void_p()
        st = self._lib.jdec_create(ctypes.byref(h), ctypes.byref(self._opt))
        if st != OK:
            raise JdecError(st, "jdec_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.jdec_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self) -> int:
        return self._h.value

    def decode_coeffs(self, img: Image, stream=None, check=True) -> int:
        st = self._lib.jdec_decode_coeffs(self._h, ctypes.byref(img), ctypes.c_void_p(_stream_ptr(stream)))
        if check and st != OK:
            raise JdecError(st, "jdec_decode_coeffs")
        return st

    def decode_batch(self, imgs, stream=None, check=True) -> int:
        arr = (Image * len(imgs))(*imgs)
        st = self._lib.jdec_decode_batch(self._h, arr, len(imgs), ctypes.c_void_p(_stream_ptr(stream)))
        if check and st != OK:
            raise JdecError(st, "jdec_decode_batch")
        return st

    def decode_jpeg(self, data: bytes, rgb, fancy: bool = True, threads: int = 1, stream=None,
                    check=True, aan: bool = False) -> int:
        """Baseline JPEG bytes (host) -> device RGB tensor (H, W, 3) or (H, pitch)
        uint8; host entropy decoding overlaps the device back-end."""
        buf = bytes(data)
        st = self._lib.jdec_decode_jpeg(self._h, ctypes.c_char_p(buf), len(buf), ctypes.c_void_p(rgb.data_ptr()),
                                        int(rgb.stride(0)), _flags(fancy, aan),
                                        int(threads), ctypes.c_void_p(_stream_ptr(stream)))
        if check and st != OK:
            raise JdecError(st, "jdec_decode_jpeg")
        return st

    def decode_host(self, img: Image, stream=None, check=True) -> int:
        st = self._lib.jdec_decode_host(self._h, ctypes.byref(img), ctypes.c_void_p(_stream_ptr(stream)))
        if check and st != OK:
            raise JdecError(st, "jdec_decode_host")
        return st

    def decode_host_batch(self, imgs, stream=None, check=True) -> int:
        """Host-buffer images in one call; consecutive images' copies and
        decoding overlap (jdec_decode_host_batch)."""
        arr = (Image * len(imgs))(*imgs)
        st = self._lib.jdec_decode_host_batch(self._h, arr, len(imgs), ctypes.c_void_p(_stream_ptr(stream)))
        if check and st != OK:
            raise JdecError(st, "jdec_decode_host_batch")
        return st

    def sync(self, stream=None, check=True) -> int:
        st = self._lib.jdec_sync_status(self._h, ctypes.c_void_p(_stream_ptr(stream)))
        if check and st != OK:
            raise JdecError(st, "jdec_sync_status")
        return st


def decode(ctx: Context, img, device_planes=None, rgb=None, stream=None, aan=False):
    """Convenience: decode a ``synth.CoefImage`` whose planes are uploaded to
    the current CUDA device; returns the (H, W, 3) uint8 device tensor
    (``aan``: with the AAN IDCT)."""
    import torch
    if device_planes is None:
        device_planes = [torch.from_numpy(np.ascontiguousarray(p)).cuda() for p in img.planes]
    if rgb is None:
        rgb = torch.empty((img.height, img.width, 3), dtype=torch.uint8, device="cuda")
    keep = []
    im = make_image(img.width, img.height, (img.h_samp, img.v_samp), device_planes, img.qtabs, rgb,
                    fancy=img.fancy, keep=keep, aan=aan)
    ctx.decode_coeffs(im, stream)
    return rgb
