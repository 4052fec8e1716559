"""jdec_decode_jpeg: JPEG bytes in host memory -> device RGB, with host
entropy decoding in chunks overlapped with the back-end (and decoded by
several threads when restart intervals allow).  The result must be exactly
the oracle's back-end applied to the encoder's coefficients, whatever the
chunking, thread count or restart layout."""
import numpy as np
import pytest

from paper_1311_5304_gb300 import jdec, synth
from gpu_util import POISON, assert_same, oracle_rgb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = jdec.Context()
    yield c
    c.close()


def _rgb(h, w, pad=0):
    import torch
    return torch.full((h, 3 * w + pad), POISON, dtype=torch.uint8, device="cuda")


@pytest.mark.parametrize("sampling,fancy", [("444", True), ("422", True), ("422", False), ("420", True),
                                            ("420", False), ("440", True), ("440", False)])
@pytest.mark.parametrize("restart", ["none", "row", "odd"])
def test_matches_oracle(ctx, orc, sampling, fancy, restart):
    import torch
    img = synth.make_image(733, 517, sampling, 87, seed=17, kind="texture", sigma=4, fancy=fancy)
    mx = img.planes[0].shape[1] // img.h_samp[0]
    ri = {"none": 0, "row": mx, "odd": 5}[restart]
    data = synth.encode_jfif(img, ri)
    want = oracle_rgb(orc, img)
    for threads in (1, 8):
        buf = _rgb(img.height, img.width, pad=5)
        ctx.decode_jpeg(data, buf, fancy=fancy, threads=threads)
        ctx.sync()
        torch.cuda.synchronize()
        host = buf.cpu().numpy()
        assert_same(host[:, :3 * img.width].reshape(img.height, img.width, 3), want,
                    f"{sampling} fancy={fancy} restart={restart} threads={threads}")
        assert np.all(host[:, 3 * img.width:] == POISON)


def test_large_image_many_chunks(ctx, orc):
    import torch
    img = synth.make_image(4001, 2999, "420", 90, seed=23, kind="texture", sigma=4, fancy=True)
    data = synth.encode_jfif(img, img.planes[0].shape[1] // 2)
    buf = _rgb(img.height, img.width)
    ctx.decode_jpeg(data, buf, threads=16)
    ctx.sync()
    got = buf.cpu().numpy().reshape(img.height, img.width, 3)
    assert_same(got, oracle_rgb(orc, img), "4001x2999 4:2:0")
    # the same context decodes again (staging reuse) and gives the same bytes
    buf2 = _rgb(img.height, img.width)
    ctx.decode_jpeg(data, buf2, threads=1)
    ctx.sync()
    assert torch.equal(buf, buf2)


def test_malformed_stream_is_rejected(ctx):
    img = synth.make_image(320, 240, "420", 80, seed=3)
    data = synth.encode_jfif(img, 20)
    buf = _rgb(img.height, img.width)
    assert ctx.decode_jpeg(data[: len(data) // 3], buf, threads=4, check=False) == jdec.EINVAL
    assert ctx.decode_jpeg(data[:40], buf, check=False) == jdec.EINVAL
    ctx.sync()
    # still usable
    ctx.decode_jpeg(data, buf)
    ctx.sync()


@pytest.mark.parametrize("restart", [0, 1])
def test_grayscale_stream(ctx, orc, restart):
    src = synth.make_image(777, 515, "444", 88, seed=29, kind="texture", sigma=4)
    img = synth.gray_image(src)
    mx = img.planes[0].shape[1]
    data = synth.encode_jfif(img, mx * restart)
    want = orc.backend_decode_gray(img.width, img.height, img.planes[0], img.qtabs[0])
    for threads in (1, 8):
        buf = _rgb(img.height, img.width, pad=3)
        ctx.decode_jpeg(data, buf, threads=threads)
        ctx.sync()
        host = buf.cpu().numpy()
        assert_same(host[:, :3 * img.width].reshape(img.height, img.width, 3), want,
                    f"gray restart={restart} threads={threads}")
        assert np.all(host[:, 3 * img.width:] == POISON)


@pytest.mark.parametrize("chunk_rows", [1, 2, 7, 1000])
@pytest.mark.parametrize("sampling", ["420", "422"])
def test_chunk_size_option(orc, sampling, chunk_rows):
    # the context's chunk size (Sec. 4.5's profiled parameter) changes only
    # the pipelining, never the bytes: 1-thread chunks of any height, and
    # restart-aligned parallel chunks (rounded up to whole intervals of 3 rows)
    img = synth.make_image(613, 407, sampling, 85, seed=41, kind="texture", sigma=4, fancy=True)
    mx = img.planes[0].shape[1] // img.h_samp[0]
    data = synth.encode_jfif(img, 3 * mx)
    want = oracle_rgb(orc, img)
    with jdec.Context(jpeg_chunk_rows=chunk_rows) as c:
        for threads in (1, 6):
            buf = _rgb(img.height, img.width)
            c.decode_jpeg(data, buf, threads=threads)
            c.sync()
            got = buf.cpu().numpy().reshape(img.height, img.width, 3)
            assert_same(got, want, f"{sampling} chunk_rows={chunk_rows} threads={threads}")
