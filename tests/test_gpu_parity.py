"""GPU parity: the fused sm_103a kernel, called through the C ABI, must give
exactly the oracle's RGB bytes (integer path: bit-exact, tolerance 0) on
every sampling and upsampling mode, ragged sizes, several strips and chunks,
adversarial coefficients, odd pitches, and the full-size workloads."""
import json
import zlib
import os

import numpy as np
import pytest

from paper_1311_5304_gb300 import jdec, synth
from gpu_util import assert_padding_untouched, assert_same, gpu_rgb, oracle_rgb, upload

pytestmark = pytest.mark.gpu

MODES = [("444", True), ("422", False), ("422", True), ("420", False), ("420", True), ("440", False), ("440", True)]


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    c = jdec.Context()
    yield c
    c.close()


def test_config1_512_420_q75_replicate(ctx, orc):
    img = synth.make_image(512, 512, "420", 75, seed=13115304 + 1000, kind="gradient", sigma=8.0, fancy=False)
    got, _, _ = gpu_rgb(ctx, img)
    assert_same(got, oracle_rgb(orc, img), "config 1")


@pytest.mark.parametrize("sampling,fancy", MODES)
def test_tiny_and_ragged_sizes(ctx, orc, sampling, fancy):
    rng = np.random.default_rng(zlib.crc32(f"{sampling}{fancy}".encode()))
    for (w, h) in [(1, 1), (2, 2), (7, 9), (8, 8), (15, 17), (16, 16), (17, 33), (33, 31), (40, 7), (129, 65)]:
        img = synth.random_image(rng, w, h, sampling, fancy=fancy)
        got, _, _ = gpu_rgb(ctx, img)
        assert_same(got, oracle_rgb(orc, img, 1), f"{sampling} fancy={fancy} {w}x{h}")


@pytest.mark.parametrize("sampling,fancy", MODES)
def test_multi_strip_multi_chunk(ctx, orc, sampling, fancy):
    rng = np.random.default_rng(7 + len(sampling) + int(fancy))
    for (w, h) in [(1000, 700), (333, 517), (2049, 1025)]:
        img = synth.random_image(rng, w, h, sampling, fancy=fancy)
        got, _, _ = gpu_rgb(ctx, img)
        assert_same(got, oracle_rgb(orc, img), f"{sampling} fancy={fancy} {w}x{h}")


@pytest.mark.parametrize("sampling,fancy", [("420", True), ("444", True), ("422", False), ("440", True)])
def test_maximum_width_and_height(ctx, orc, sampling, fancy):
    # the largest dimension the boundary accepts (65535), thin and wide: a
    # ragged last MCU column / row, thousands of strips, one strip of many rows
    rng = np.random.default_rng(zlib.crc32(f"max{sampling}{fancy}".encode()))
    for (w, h) in [(65535, 37), (23, 65535), (65535, 1031)]:
        img = synth.random_image(rng, w, h, sampling, fancy=fancy)
        got, _, _ = gpu_rgb(ctx, img)
        assert_same(got, oracle_rgb(orc, img), f"{sampling} fancy={fancy} {w}x{h}")


@pytest.mark.parametrize("sampling,fancy", MODES)
def test_synthetic_content(ctx, orc, sampling, fancy):
    img = synth.make_image(1920, 1080, sampling, 85, seed=99, kind="texture", sigma=4.0, fancy=fancy)
    got, _, _ = gpu_rgb(ctx, img)
    assert_same(got, oracle_rgb(orc, img), f"{sampling} fancy={fancy}")


def test_adversarial_coefficients_wrap_identically(ctx, orc):
    # int16 extremes with 16-bit quantisation steps overflow int32 inside the
    # transform; both sides wrap mod 2^32 and must still agree bit for bit.
    rng = np.random.default_rng(2 ** 31 - 1)
    for sampling, fancy in MODES:
        img = synth.random_image(rng, 77, 45, sampling, fancy=fancy, dense=True)
        for p in img.planes:
            p[...] = rng.choice(np.array([-32768, 32767, -1, 0, 1, 12345, -23456], np.int16), size=p.shape)
        img.qtabs = [rng.integers(1, 65536, size=64).astype(np.uint16) for _ in range(3)]
        got, _, _ = gpu_rgb(ctx, img)
        assert_same(got, oracle_rgb(orc, img, 1), f"adversarial {sampling} fancy={fancy}")


@pytest.mark.parametrize("pitch_extra,offset", [(0, 0), (5, 0), (13, 1), (64, 3), (8, 8)])
def test_pitch_and_alignment(ctx, orc, pitch_extra, offset):
    rng = np.random.default_rng(pitch_extra * 31 + offset)
    for sampling, fancy in MODES:
        img = synth.random_image(rng, 53, 37, sampling, fancy=fancy)
        pitch = 3 * img.width + pitch_extra
        got, host, _ = gpu_rgb(ctx, img, pitch=pitch, offset=offset)
        assert_same(got, oracle_rgb(orc, img, 1), f"pitch {pitch} offset {offset}")
        assert_padding_untouched(host, img, pitch, offset)


@pytest.mark.parametrize("wt", [1, 2, 3, 5, 8, 13, 17, 32, 42, 64])
def test_every_strip_width(orc, tmp_path, wt):
    # pin the strip width for every variant and size class through a tune file
    entries = [[v, sc, wt] for v in range(5) for sc in range(20)]
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    path = tmp_path / "tune.json"
    path.write_text(json.dumps({"gpu": "x", "sms": sms, "entries": entries}))
    rng = np.random.default_rng(wt)
    with jdec.Context(tune_file=str(path)) as c:
        for sampling, fancy in MODES:
            img = synth.random_image(rng, 301, 129, sampling, fancy=fancy)
            got, _, _ = gpu_rgb(c, img)
            assert_same(got, oracle_rgb(orc, img), f"wt={wt} {sampling} fancy={fancy}")


@pytest.mark.parametrize("wt,nidct", [(3, 32), (17, 32), (5, 96), (32, 96)])
def test_every_warp_split(orc, tmp_path, wt, nidct):
    # one, two or three IDCT warps (the rest convert colour), forced through a tune file
    entries = [[v, sc, wt, nidct] for v in range(5) for sc in range(20)]
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    path = tmp_path / "tune.json"
    path.write_text(json.dumps({"gpu": "x", "sms": sms, "entries": entries}))
    rng = np.random.default_rng(1000 * wt + nidct)
    with jdec.Context(tune_file=str(path)) as c:
        for sampling, fancy in MODES:
            img = synth.random_image(rng, 517, 263, sampling, fancy=fancy)
            got, _, _ = gpu_rgb(c, img)
            assert_same(got, oracle_rgb(orc, img), f"wt={wt} nidct={nidct} {sampling} fancy={fancy}")


def test_invalid_descriptions_launch_nothing(ctx):
    import torch
    rng = np.random.default_rng(3)
    img = synth.random_image(rng, 40, 24, "420")
    planes = upload(img)
    raw = torch.full((3 * 40 * 24,), 0xCD, dtype=torch.uint8, device="cuda")

    def status(**kw):
        keep = []
        im = jdec.make_image(40, 24, "420", planes, img.qtabs, raw, rgb_pitch=120, keep=keep)
        for k, v in kw.items():
            if k in ("blocks_w", "h_samp", "v_samp"):
                getattr(im, k)[v[0]] = v[1]
            else:
                setattr(im, k, v)
        return ctx.decode_coeffs(im, check=False)

    assert status() == jdec.OK
    torch.cuda.synchronize()
    raw.fill_(0xCD)
    assert status(blocks_w=(0, 7)) == jdec.EINVAL
    assert status(rgb_pitch=119) == jdec.EINVAL
    assert status(width=0) == jdec.EINVAL
    assert status(height=70000) == jdec.EINVAL
    assert status(ncomp=1) == jdec.EUNSUPPORTED
    assert status(h_samp=(1, 2)) == jdec.EUNSUPPORTED
    assert status(h_samp=(0, 3)) == jdec.EUNSUPPORTED
    assert status(flags=7) == jdec.EINVAL
    assert status(rgb=None) == jdec.EINVAL
    keep = []
    im = jdec.make_image(40, 24, "420", planes, img.qtabs, raw, rgb_pitch=120, keep=keep)
    im.coef[1] = im.coef[1] + 2   # misaligned plane pointer
    assert ctx.decode_coeffs(im, check=False) == jdec.EINVAL
    torch.cuda.synchronize()
    assert int((raw != 0xCD).sum()) == 0
    assert ctx.sync(check=False) == jdec.OK


@pytest.mark.parametrize("sampling", ["444", "422", "420", "440"])
def test_config2_full_size_8192(ctx, orc, sampling):
    img = synth.make_image(8192, 8192, sampling, 90, seed=13115304 + 2000, kind="texture", sigma=4.0,
                           cover=0.85, fancy=True)
    got, _, _ = gpu_rgb(ctx, img)
    assert_same(got, oracle_rgb(orc, img), f"8192x8192 {sampling}")


@pytest.mark.parametrize("q,sigma", [(30, 2), (50, 4), (75, 8), (90, 16), (98, 32)])
def test_config3_sparsity_sweep(ctx, orc, q, sigma):
    for (w, h) in [(4000, 3000), (4001, 2999)]:
        img = synth.make_image(w, h, "420", q, seed=13115304 + 3000 + q, kind="gradient", sigma=sigma,
                               fancy=True)
        got, _, _ = gpu_rgb(ctx, img)
        assert_same(got, oracle_rgb(orc, img), f"{w}x{h} q{q}")


def test_repeat_launches_are_deterministic(ctx, orc):
    img = synth.make_image(777, 555, "420", 80, seed=5, kind="texture", sigma=3.0)
    planes = upload(img)
    a, _, _ = gpu_rgb(ctx, img, planes=planes)
    for _ in range(3):
        b, _, _ = gpu_rgb(ctx, img, planes=planes)
        assert np.array_equal(a, b)
    assert_same(a, oracle_rgb(orc, img), "repeat")


@pytest.mark.parametrize("sampling,w,h", [("420", 1912, 9725), ("420", 8184, 4097), ("444", 1272, 2001),
                                          ("444", 8184, 1031)])
def test_fixed_width_path_edges(ctx, orc, sampling, w, h):
    # Large images with 8-byte aligned rows and a width that is a multiple of
    # 8 take the compile-time-width code (4:4:4 strips of 32 MCUs, 4:2:0 of
    # 20): a right-edge MCU half outside the image, a padded last strip
    # (8184 = 511.5 MCUs wide), ragged heights; a forced width (general code)
    # must give the same bytes, both equal to the oracle
    img = synth.make_image(w, h, sampling, 88, seed=w * 7 + h, kind="texture", sigma=3.0, fancy=True)
    planes = upload(img)
    got, host, _ = gpu_rgb(ctx, img, planes=planes, pitch=3 * w + 8)
    assert_padding_untouched(host, img, 3 * w + 8, 0)
    want = oracle_rgb(orc, img)
    assert_same(got, want, f"fixed width {sampling} {w}x{h}")
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    v = 0 if sampling == "444" else 4
    forced = os.path.join(os.environ.get("TMPDIR", "/tmp"), f"jdec_force_{os.getpid()}.json")
    with open(forced, "w") as f:
        json.dump({"gpu": "x", "sms": sms, "entries": [[v, sc, 12] for sc in range(20)]}, f)
    try:
        with jdec.Context(tune_file=forced) as c2:
            got2, _, _ = gpu_rgb(c2, img, planes=planes)
    finally:
        os.unlink(forced)
    assert np.array_equal(got2, got)
