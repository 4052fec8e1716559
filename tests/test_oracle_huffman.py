"""Pins for the oracle's entropy decoder: streams written by the input-side
JFIF encoder (a separate implementation of T.81's coding procedures) must
decode to exactly the coefficient planes, tables and geometry they encode."""
import numpy as np
import pytest

from paper_1311_5304_gb300 import synth


def _check(orc, img, restart=0):
    data = synth.encode_jfif(img, restart)
    info, planes = orc.jpeg_decode_coefs(data)
    assert (info["width"], info["height"]) == (img.width, img.height)
    assert info["h_samp"] == tuple(img.h_samp) and info["v_samp"] == tuple(img.v_samp)
    for c in range(3):
        assert np.array_equal(planes[c], img.planes[c]), c
        assert np.array_equal(info["qtabs"][c], img.qtabs[c])
    return data


@pytest.mark.parametrize("sampling", ["444", "422", "420", "440"])
@pytest.mark.parametrize("restart", [0, 1, 7])
def test_round_trip_synthetic(orc, sampling, restart):
    img = synth.make_image(72, 40, sampling, 85, seed=5 + restart, kind="texture", sigma=6)
    _check(orc, img, restart)


def test_round_trip_high_entropy_and_stuffing(orc):
    # dense random coefficients: long codes, many 0xFF bytes to stuff
    rng = np.random.default_rng(4)
    img = synth.random_image(rng, 64, 64, "420")
    for p in img.planes:
        p[..., 1:] = rng.integers(-1023, 1024, size=p[..., 1:].shape)
        p[..., 0] = rng.integers(-1000, 1001, size=p[..., 0].shape)
    data = _check(orc, img, 3)
    assert data.count(b"\xff\x00") > 10


def test_round_trip_all_zero_and_tiny(orc):
    rng = np.random.default_rng(8)
    for (w, h) in [(1, 1), (9, 3), (16, 16)]:
        img = synth.random_image(rng, w, h, "420")
        for p in img.planes:
            p[...] = 0
        _check(orc, img)


def test_malformed_stream_is_rejected(orc):
    img = synth.make_image(32, 32, "420", 75)
    data = synth.encode_jfif(img)
    with pytest.raises(ValueError):
        orc.jpeg_decode_coefs(data[:100])
    with pytest.raises(ValueError):
        orc.jpeg_decode_coefs(b"\x00\x01" + data[2:])


def test_decoded_image_psnr(orc):
    img = synth.make_image(128, 96, "420", 80, kind="gradient", sigma=2)
    info, planes = orc.jpeg_decode_coefs(synth.encode_jfif(img))
    rgb = orc.backend_decode(128, 96, info["h_samp"], info["v_samp"], planes, info["qtabs"], True).astype(float)
    src = np.clip(np.rint(synth.render_rgb(128, 96, img.meta["seed"], "gradient", 2)), 0, 255)
    assert 10 * np.log10(255 ** 2 / np.mean((rgb - src) ** 2)) > 30
