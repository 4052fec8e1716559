"""External pin: NVIDIA's nvJPEG library (run only, through its public C API)
decodes the encoder's baseline JFIF streams to exactly the same RGB bytes as
the oracle with replicated chroma upsampling, for 4:4:4, 4:2:2, 4:2:0 and 4:4:0 --
an independent implementation of the same integer IDCT (13-bit constants,
column pass then row pass, the same rounding), replication and 16-bit
fixed-point colour conversion.  The GPU path, which equals the oracle, then
equals nvJPEG too.  (nvJPEG replicates chroma; the triangular mode is pinned
by Alg. 1 and the oracle's own tests.)"""
import ctypes
import ctypes.util

import numpy as np
import pytest

from paper_1311_5304_gb300 import jdec, synth
from gpu_util import assert_same, oracle_rgb

pytestmark = pytest.mark.gpu


def _nvjpeg():
    for cand in ("libnvjpeg.so", "libnvjpeg.so.13", ctypes.util.find_library("nvjpeg"),
                 "/usr/local/cuda/lib64/libnvjpeg.so"):
        if not cand:
            continue
        try:
            return ctypes.CDLL(cand)
        except OSError:
            continue
    return None


class _Image(ctypes.Structure):
    _fields_ = [("channel", ctypes.c_void_p * 4), ("pitch", ctypes.c_size_t * 4)]


RGBI = 5   # nvjpegOutputFormat_t: interleaved RGB


@pytest.fixture(scope="module")
def nvj():
    lib = _nvjpeg()
    if lib is None:
        pytest.skip("nvJPEG not available")
    return lib


def nvjpeg_decode(lib, data, w, h):
    import torch
    handle, state = ctypes.c_void_p(), ctypes.c_void_p()
    assert lib.nvjpegCreateSimple(ctypes.byref(handle)) == 0
    try:
        assert lib.nvjpegJpegStateCreate(handle, ctypes.byref(state)) == 0
        out = torch.zeros((h, 3 * w), dtype=torch.uint8, device="cuda")
        img = _Image()
        img.channel[0] = out.data_ptr()
        img.pitch[0] = 3 * w
        buf = ctypes.create_string_buffer(data, len(data))
        st = lib.nvjpegDecode(handle, state, buf, ctypes.c_size_t(len(data)), RGBI, ctypes.byref(img),
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        torch.cuda.synchronize()
        lib.nvjpegJpegStateDestroy(state)
        assert st == 0, f"nvjpegDecode status {st}"
        return out.cpu().numpy().reshape(h, w, 3)
    finally:
        lib.nvjpegDestroy(handle)


@pytest.mark.parametrize("sampling", ["444", "422", "420", "440"])
@pytest.mark.parametrize("quality,sigma", [(50, 8.0), (90, 4.0), (98, 16.0)])
def test_oracle_equals_nvjpeg(orc, nvj, sampling, quality, sigma):
    img = synth.make_image(733, 517, sampling, quality, seed=41 + quality, kind="texture", sigma=sigma,
                           fancy=False)
    data = synth.encode_jfif(img)
    assert_same(oracle_rgb(orc, img), nvjpeg_decode(nvj, data, img.width, img.height),
                f"oracle vs nvJPEG {sampling} q{quality}")


@pytest.mark.parametrize("sampling", ["444", "422", "420", "440"])
def test_gpu_path_equals_nvjpeg(nvj, sampling):
    import torch
    img = synth.make_image(1031, 769, sampling, 85, seed=7, kind="texture", sigma=4, fancy=False)
    data = synth.encode_jfif(img)
    with jdec.Context() as ctx:
        out = torch.zeros((img.height, img.width, 3), dtype=torch.uint8, device="cuda")
        ctx.decode_jpeg(data, out, fancy=False, threads=1)
        ctx.sync()
        got = out.cpu().numpy()
    assert_same(got, nvjpeg_decode(nvj, data, img.width, img.height), f"GPU path vs nvJPEG {sampling}")


def test_grayscale_equals_nvjpeg(orc, nvj):
    src = synth.make_image(733, 517, "444", 90, seed=43, kind="texture", sigma=4)
    img = synth.gray_image(src)
    data = synth.encode_jfif(img)
    want = orc.backend_decode_gray(img.width, img.height, img.planes[0], img.qtabs[0])
    assert_same(want, nvjpeg_decode(nvj, data, img.width, img.height), "gray oracle vs nvJPEG")
