"""Host entropy decoder of the library (serving path) against the oracle's
Huffman decoder and the encoder's input planes: identical coefficients."""
import numpy as np
import pytest

from paper_1311_5304_gb300 import jdec, synth


def _decode(data):
    info = jdec.jpeg_parse(data)
    planes = [np.zeros((info.blocks_h[c], info.blocks_w[c], 64), np.int16) for c in range(3)]
    jdec.entropy_decode(data, planes)
    return info, planes


@pytest.mark.parametrize("sampling", ["444", "422", "420", "440"])
@pytest.mark.parametrize("restart", [0, 1, 5])
def test_matches_encoder_and_oracle(orc, sampling, restart):
    img = synth.make_image(121, 67, sampling, 88, seed=restart + 3, kind="texture", sigma=5)
    data = synth.encode_jfif(img, restart)
    info, planes = _decode(data)
    assert (info.width, info.height) == (121, 67)
    assert tuple(info.h_samp) == tuple(img.h_samp) and tuple(info.v_samp) == tuple(img.v_samp)
    assert info.restart_interval == restart
    oinfo, oplanes = orc.jpeg_decode_coefs(data)
    for c in range(3):
        assert np.array_equal(planes[c], img.planes[c])
        assert np.array_equal(planes[c], oplanes[c])
        assert np.array_equal(np.array(info.qtab[c][:], np.uint16), img.qtabs[c])


def test_dense_coefficients_long_codes_and_stuffing():
    rng = np.random.default_rng(12)
    img = synth.random_image(rng, 96, 80, "420")
    for p in img.planes:
        p[..., 1:] = rng.integers(-1023, 1024, size=p[..., 1:].shape)
        p[..., 0] = rng.integers(-1000, 1001, size=p[..., 0].shape)
    for restart in (0, 3):
        data = synth.encode_jfif(img, restart)
        _, planes = _decode(data)
        for c in range(3):
            assert np.array_equal(planes[c], img.planes[c])


def test_every_run_length_size_and_large_dc_steps(orc):
    # Sparse coefficients at random positions (zero runs of every length,
    # ZRL codes for runs of 16 or more, end of block anywhere), magnitudes of
    # every size 1..10 and DC steps of size 11: codes and magnitude bits that
    # fit the decoder's 11-bit combined table, ones that do not, and codes
    # longer than its 9-bit lookahead, mixed in one stream.
    rng = np.random.default_rng(5304)
    img = synth.random_image(rng, 152, 104, "420")
    for p in img.planes:
        ac = np.zeros(p[..., 1:].shape, np.int16)
        n = ac.shape[-1]
        nnz = rng.integers(0, 12, size=ac.shape[:-1])
        for idx in np.ndindex(*ac.shape[:-1]):
            pos = rng.choice(n, size=int(nnz[idx]), replace=False)
            size = rng.integers(1, 11, size=pos.size)
            mag = rng.integers(1 << (size - 1), 1 << size)
            ac[idx + (pos,)] = np.where(rng.integers(0, 2, size=pos.size) == 1, mag, -mag)
        p[..., 1:] = ac
        # alternate the DC between the extremes: differences of size 11
        dc = np.where(rng.integers(0, 2, size=p[..., 0].shape) == 1, 1020, -1020)
        p[..., 0] = dc + rng.integers(-3, 4, size=dc.shape)
    for restart in (0, 2):
        data = synth.encode_jfif(img, restart)
        _, planes = _decode(data)
        _, oplanes = orc.jpeg_decode_coefs(data)
        for c in range(3):
            assert np.array_equal(planes[c], img.planes[c])
            assert np.array_equal(planes[c], oplanes[c])


def test_rejects_malformed_and_unsupported():
    img = synth.make_image(32, 32, "420", 75)
    data = synth.encode_jfif(img)
    with pytest.raises(jdec.JdecError):
        jdec.jpeg_parse(data[:50])
    with pytest.raises(jdec.JdecError) as e:
        jdec.jpeg_parse(data.replace(b"\xff\xc0", b"\xff\xc2", 1))   # progressive
    assert e.value.status == jdec.EUNSUPPORTED
    info = jdec.jpeg_parse(data)
    planes = [np.zeros((info.blocks_h[c], info.blocks_w[c], 64), np.int16) for c in range(3)]
    with pytest.raises(jdec.JdecError):
        jdec.entropy_decode(data[:200], planes)


def test_large_image_throughput_sane():
    img = synth.make_image(1920, 1080, "420", 85, kind="texture", sigma=4, cover=0.85)
    data = synth.encode_jfif(img)
    import time
    t = time.perf_counter()
    _, planes = _decode(data)
    dt = time.perf_counter() - t
    for c in range(3):
        assert np.array_equal(planes[c], img.planes[c])
    assert dt < 2.0


def _decode_mt(data, threads):
    info = jdec.jpeg_parse(data)
    planes = [np.full((info.blocks_h[c], info.blocks_w[c], 64), 0x5A5A, np.int16) for c in range(3)]
    jdec.entropy_decode(data, planes, threads=threads)
    return planes


@pytest.mark.parametrize("sampling", ["444", "422", "420", "440"])
@pytest.mark.parametrize("restart_rows", [None, 1, 3])
def test_threaded_decode_equals_sequential(sampling, restart_rows):
    # restart intervals of whole MCU rows (chunks start at rows), of a
    # fraction of a row that lines up every few rows, or none (one thread)
    img = synth.make_image(509, 389, sampling, 85, seed=31, kind="texture", sigma=4)
    mx = img.planes[0].shape[1] // img.h_samp[0]
    restart = 0 if restart_rows is None else (mx * restart_rows if restart_rows != 3 else 7)
    data = synth.encode_jfif(img, restart)
    for threads in (2, 5, 16):
        planes = _decode_mt(data, threads)
        for c in range(3):
            assert np.array_equal(planes[c], img.planes[c]), (threads, c)


def test_threaded_decode_rejects_truncated_stream():
    img = synth.make_image(256, 256, "420", 80, seed=5, kind="texture", sigma=4)
    mx = img.planes[0].shape[1] // 2
    data = synth.encode_jfif(img, mx)
    info = jdec.jpeg_parse(data)
    planes = [np.zeros((info.blocks_h[c], info.blocks_w[c], 64), np.int16) for c in range(3)]
    with pytest.raises(jdec.JdecError):
        jdec.entropy_decode(data[: len(data) // 2], planes, threads=4)


@pytest.mark.parametrize("restart", [0, 1, 9])
def test_grayscale_streams(restart):
    src = synth.make_image(301, 203, "444", 85, seed=19, kind="texture", sigma=4)
    img = synth.gray_image(src)
    data = synth.encode_jfif(img, restart)
    info = jdec.jpeg_parse(data)
    assert info.ncomp == 1 and (info.width, info.height) == (301, 203)
    assert (info.blocks_w[0], info.blocks_h[0]) == img.planes[0].shape[1::-1]
    for threads in (1, 4):
        plane = np.zeros((info.blocks_h[0], info.blocks_w[0], 64), np.int16)
        jdec.entropy_decode(data, [plane], threads=threads)
        assert np.array_equal(plane, img.planes[0])


def test_fill_bytes_before_restart_markers():
    # T.81 B.1.1.2: any marker may be preceded by fill bytes 0xFF; the one-
    # thread and the restart-parallel decoders both accept them
    img = synth.make_image(64, 48, "420", 80, seed=6, kind="texture", sigma=4)
    mx = img.planes[0].shape[1] // 2
    data = synth.encode_jfif(img, mx)
    filled = bytearray()
    i = 0
    while i < len(data):
        if data[i] == 0xFF and i + 1 < len(data) and 0xD0 <= data[i + 1] <= 0xD7:
            filled += b"\xff\xff\xff"
        filled.append(data[i])
        i += 1
    info = jdec.jpeg_parse(bytes(filled))
    for threads in (1, 4):
        planes = [np.zeros((info.blocks_h[c], info.blocks_w[c], 64), np.int16) for c in range(3)]
        jdec.entropy_decode(bytes(filled), planes, threads=threads)
        for c in range(3):
            assert np.array_equal(planes[c], img.planes[c])
