"""GPU parity of the AAN scaled IDCT (JDEC_IDCT_AAN; the algorithm Sec. 2
names) through the C ABI: every sampling and upsampling mode, tiny, ragged
and multi-strip images, 16-bit tables (whose prescaled products wrap int32),
the 8192x8192 4:2:0 workload, mixed AAN/LLM batches, host buffers, JPEG
streams and grayscale.  Tolerance 0: the integer result is bit-exact with the
oracle's AAN back-end."""
import zlib

import numpy as np
import pytest

from paper_1311_5304_gb300 import jdec, synth
from gpu_util import assert_same, gpu_rgb, oracle_rgb, upload

pytestmark = pytest.mark.gpu

MODES = [("444", True), ("422", False), ("422", True), ("420", False), ("420", True), ("440", False), ("440", True)]
SIZES = [(1, 1), (8, 8), (17, 9), (33, 31), (161, 97), (1283, 901)]


@pytest.fixture(scope="module")
def ctx():
    with jdec.Context() as c:
        yield c


@pytest.mark.parametrize("sampling,fancy", MODES)
def test_every_mode_and_size(ctx, orc, sampling, fancy):
    rng = np.random.default_rng(zlib.crc32(f"aan{sampling}{fancy}".encode()))
    for (w, h) in SIZES:
        img = synth.random_image(rng, w, h, sampling, fancy=fancy)
        got, _, _ = gpu_rgb(ctx, img, aan=True)
        assert_same(got, oracle_rgb(orc, img, aan=True), f"AAN {sampling} fancy={fancy} {w}x{h}")


def test_sixteen_bit_tables_wrap_identically(ctx, orc):
    rng = np.random.default_rng(77)
    for sampling in ("444", "420"):
        img = synth.random_image(rng, 203, 151, sampling, dense=True, qmax=65535)
        got, _, _ = gpu_rgb(ctx, img, aan=True)
        assert_same(got, oracle_rgb(orc, img, aan=True), f"AAN 16-bit tables {sampling}")


def test_full_size_8192_420(ctx, orc):
    img = synth.make_image(8192, 8192, "420", 90, seed=13115304 + 2000, kind="texture", sigma=4.0,
                           cover=0.85, fancy=True)
    got, _, _ = gpu_rgb(ctx, img, aan=True)
    assert_same(got, oracle_rgb(orc, img, aan=True), "AAN 8192x8192 4:2:0")
    # the two IDCTs' samples agree within one level on ordinary content; Alg. 2
    # turns one level of Y, Cb and Cr into at most 1 + 1.772 + rounding of RGB
    llm, _, _ = gpu_rgb(ctx, img)
    d = np.abs(llm.astype(np.int16) - got.astype(np.int16))
    assert int(d.max()) <= 4
    assert float(d.mean()) < 0.1


def test_mixed_batch_of_both_idcts(ctx, orc):
    import torch
    rng = np.random.default_rng(91)
    imgs, flags = [], []
    for i in range(24):
        s = ["420", "422", "444", "440"][i % 4]
        imgs.append(synth.random_image(rng, int(rng.integers(1, 600)), int(rng.integers(1, 400)), s,
                                       fancy=bool(i % 3), qmax=255 if i % 5 else 65535))
        flags.append(bool(i % 2))
    keep, outs, descs = [], [], []
    for im, aan in zip(imgs, flags):
        out = torch.full((im.height, im.width, 3), 0xCD, dtype=torch.uint8, device="cuda")
        outs.append(out)
        descs.append(jdec.make_image(im.width, im.height, (im.h_samp, im.v_samp), upload(im), im.qtabs, out,
                                     fancy=im.fancy, keep=keep, aan=aan))
    ctx.decode_batch(descs)
    ctx.sync()
    for i, (im, aan) in enumerate(zip(imgs, flags)):
        assert_same(outs[i].cpu().numpy(), oracle_rgb(orc, im, aan=aan), f"batch image {i} aan={aan}")


def test_host_buffers(ctx, orc):
    img = synth.make_image(1283, 901, "422", 85, seed=12, kind="texture", sigma=4.0, fancy=True)
    out = np.full((img.height, img.width, 3), 0xCD, np.uint8)
    keep = []
    d = jdec.make_image(img.width, img.height, (img.h_samp, img.v_samp), img.planes, img.qtabs, out,
                        fancy=True, keep=keep, host=True, aan=True)
    ctx.decode_host(d)
    ctx.sync()
    assert_same(out, oracle_rgb(orc, img, aan=True), "AAN host buffers")


@pytest.mark.parametrize("sampling", ["444", "420"])
def test_jpeg_stream(ctx, orc, sampling):
    import torch
    img = synth.make_image(733, 517, sampling, 87, seed=17, kind="texture", sigma=4, fancy=True)
    data = synth.encode_jfif(img, 5)
    for threads in (1, 8):
        out = torch.full((img.height, img.width, 3), 0xCD, dtype=torch.uint8, device="cuda")
        ctx.decode_jpeg(data, out, fancy=True, threads=threads, aan=True)
        ctx.sync()
        assert_same(out.cpu().numpy(), oracle_rgb(orc, img, aan=True), f"AAN JPEG {sampling} threads={threads}")


def test_grayscale(ctx, orc):
    import torch
    img = synth.gray_image(synth.make_image(517, 333, "444", 90, seed=3, kind="texture", sigma=4))
    out = torch.full((img.height, img.width, 3), 0xCD, dtype=torch.uint8, device="cuda")
    keep = []
    d = jdec.make_image(img.width, img.height, "gray", upload(img), img.qtabs, out, keep=keep, aan=True)
    ctx.decode_coeffs(d)
    ctx.sync()
    want = orc.backend_decode_gray(img.width, img.height, img.planes[0], img.qtabs[0], aan=True)
    assert_same(out.cpu().numpy(), want, "AAN grayscale")
