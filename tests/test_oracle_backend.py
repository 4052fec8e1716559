"""Pins for the oracle's whole back-end: a second, naive per-output-pixel
implementation (direct index arithmetic, no planes or tiling) must equal the
oracle on tiny images of every sampling and upsampling mode, and the MCU
geometry must follow Sec. 2."""
import zlib

import numpy as np
import pytest

from paper_1311_5304_gb300 import synth

SIZES = [(1, 1), (8, 8), (15, 17), (16, 16), (17, 9), (33, 31), (7, 40)]


def naive_decode(orc, img, aan=False):
    hs, vs = img.h_samp, img.v_samp
    hmax, vmax = max(hs), max(vs)
    W, H = img.width, img.height
    cache = {}

    def sample(c, i, j):
        # sample (column i, row j) of component c from its block's IDCT
        bx, by = i // 8, j // 8
        key = (c, bx, by)
        if key not in cache:
            cache[key] = orc.idct_blocks(img.planes[c][by, bx][None], img.qtabs[c], aan=aan)[0]
        return int(cache[key][(j % 8) * 8 + (i % 8)])

    def comp_value(c, x, y):
        sx, sy = hmax // hs[c], vmax // vs[c]
        cw = -(-W * hs[c] // hmax)
        ch = -(-H * vs[c] // vmax)
        cl = lambda v, n: min(max(v, 0), n - 1)
        if sx == 1 and sy == 1:
            return sample(c, x, y)
        if not img.fancy:
            return sample(c, x // sx, y // sy)
        if sx == 1:
            # h1v2: the Alg. 1 weights along the column
            j = y // 2
            nb = j - 1 if y % 2 == 0 else j + 1
            bias = 1 if y % 2 == 0 else 2
            return (3 * sample(c, x, j) + sample(c, x, cl(nb, ch)) + bias) >> 2
        i = x // 2
        nb = i - 1 if x % 2 == 0 else i + 1
        if sy == 1:
            bias = 1 if x % 2 == 0 else 2
            return (3 * sample(c, i, y) + sample(c, cl(nb, cw), y) + bias) >> 2
        j = y // 2
        far = cl(j - 1 if y % 2 == 0 else j + 1, ch)
        S = lambda ii: 3 * sample(c, ii, j) + sample(c, ii, far)
        bias = 8 if x % 2 == 0 else 7
        return (3 * S(i) + S(cl(nb, cw)) + bias) >> 4

    out = np.zeros((H, W, 3), np.uint8)
    for y in range(H):
        for x in range(W):
            Y, Cb, Cr = (comp_value(c, x, y) for c in range(3))
            cb, cr = Cb - 128, Cr - 128
            r = Y + ((91881 * cr + 32768) >> 16)
            g = Y + ((-22554 * cb - 46802 * cr + 32768) >> 16)
            b = Y + ((116130 * cb + 32768) >> 16)
            out[y, x] = [min(max(v, 0), 255) for v in (r, g, b)]
    return out


@pytest.mark.parametrize("sampling", ["444", "422", "420", "440"])
@pytest.mark.parametrize("fancy", [False, True])
def test_backend_equals_naive_per_pixel(orc, sampling, fancy):
    rng = np.random.default_rng(zlib.crc32(f"{sampling}{fancy}".encode()))
    for (w, h) in SIZES:
        img = synth.random_image(rng, w, h, sampling, fancy=fancy)
        got = orc.backend_decode(w, h, img.h_samp, img.v_samp, img.planes, img.qtabs, fancy)
        assert np.array_equal(got, naive_decode(orc, img)), (w, h)


@pytest.mark.parametrize("sampling", ["444", "420"])
def test_backend_with_aan_idct_equals_naive_per_pixel(orc, sampling):
    rng = np.random.default_rng(zlib.crc32(f"aan{sampling}".encode()))
    for (w, h) in SIZES:
        img = synth.random_image(rng, w, h, sampling, fancy=True)
        got = orc.backend_decode(w, h, img.h_samp, img.v_samp, img.planes, img.qtabs, True, aan=True)
        assert np.array_equal(got, naive_decode(orc, img, aan=True)), (w, h)
        got_mt = orc.backend_decode(w, h, img.h_samp, img.v_samp, img.planes, img.qtabs, True, threads=3, aan=True)
        assert np.array_equal(got_mt, got)


def test_mcu_geometry_follows_sec2():
    # 4:4:4 MCU is 8x8 px, 4:2:2 is 16x8 px, 4:2:0 is 16x16 px, 4:4:0 is 8x16 px
    for s, (mw, mh) in {"444": (8, 8), "422": (16, 8), "420": (16, 16), "440": (8, 16)}.items():
        hs, vs, mx, my = synth.geometry(mw, mh, s)
        assert (mx, my) == (1, 1)
        hs, vs, mx, my = synth.geometry(mw + 1, mh + 1, s)
        assert (mx, my) == (2, 2)


def test_multithreaded_equals_single(orc):
    rng = np.random.default_rng(99)
    for s in ("444", "422", "420", "440"):
        img = synth.random_image(rng, 203, 77, s)
        a = orc.backend_decode(203, 77, img.h_samp, img.v_samp, img.planes, img.qtabs, True)
        b = orc.backend_decode(203, 77, img.h_samp, img.v_samp, img.planes, img.qtabs, True, threads=5)
        assert np.array_equal(a, b)


def test_synthetic_image_decodes_near_source(orc):
    # End-to-end sanity of the generator + oracle: q90 4:4:4 decodes close to
    # the source content (chroma subsampling and noise excluded).
    img = synth.make_image(64, 48, "444", 90, kind="gradient", sigma=0.0)
    rgb = orc.backend_decode(64, 48, img.h_samp, img.v_samp, img.planes, img.qtabs, True).astype(float)
    src = np.clip(np.rint(synth.render_rgb(64, 48, img.meta["seed"], "gradient", 0.0)), 0, 255)
    psnr = 10 * np.log10(255 ** 2 / np.mean((rgb - src) ** 2))
    assert psnr > 35


# ---- single-component (grayscale) images ------------------------------------

@pytest.mark.parametrize("w,h", [(1, 1), (8, 8), (15, 17), (33, 31), (640, 481)])
def test_gray_equals_444_with_neutral_chroma(orc, w, h):
    # Alg. 2 maps (Y, 128, 128) to (Y, Y, Y) (grey axis, pinned exhaustively
    # in the colour tests) and an all-zero block decodes to 128 (DC-only
    # closed form), so a grayscale image must decode like a 4:4:4 image with
    # all-zero chroma planes, whatever their tables.
    rng = np.random.default_rng(w * 1000 + h)
    img = synth.random_image(rng, w, h, "444")
    got = orc.backend_decode_gray(w, h, img.planes[0], img.qtabs[0])
    zero = np.zeros_like(img.planes[1])
    want = orc.backend_decode(w, h, img.h_samp, img.v_samp, [img.planes[0], zero, zero],
                              [img.qtabs[0], img.qtabs[1], img.qtabs[2]], True)
    assert np.array_equal(got, want)


def test_gray_is_the_idct_of_each_block(orc):
    # naive per-pixel statement: pixel (x, y) = IDCT of block (x/8, y/8) at
    # (x%8, y%8), in all three channels
    rng = np.random.default_rng(5)
    w, h = 37, 29
    img = synth.random_image(rng, w, h, "444")
    plane, q = img.planes[0], img.qtabs[0]
    blocks = orc.idct_blocks(plane.reshape(-1, 64), q).reshape(plane.shape[0], plane.shape[1], 8, 8)
    got = orc.backend_decode_gray(w, h, plane, q)
    for y in range(h):
        for x in range(w):
            assert got[y, x].tolist() == [int(blocks[y // 8, x // 8, y % 8, x % 8])] * 3
