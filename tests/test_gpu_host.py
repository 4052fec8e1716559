"""jdec_decode_host and jdec_decode_host_batch: host coefficient planes and
host RGB, copied in row bands through device staging (two alternating slots
for consecutive images of one batch call).  Pageable and page-locked buffers,
odd pitches: exactly the oracle's bytes inside W x H, row padding untouched."""
import numpy as np
import pytest

from paper_1311_5304_gb300 import jdec, synth
from gpu_util import POISON, assert_same, oracle_rgb

pytestmark = pytest.mark.gpu

CASES = [("444", True, 1000, 301), ("422", True, 777, 520), ("420", True, 1283, 901), ("420", False, 333, 257)]


@pytest.fixture(scope="module")
def ctx():
    c = jdec.Context()
    yield c
    c.close()


def _decode(ctx, img, out, pitch, pinned_planes):
    import torch
    planes = img.planes
    if pinned_planes:
        planes = [torch.from_numpy(np.ascontiguousarray(p)).pin_memory().numpy() for p in img.planes]
    keep = [planes]
    d = jdec.make_image(img.width, img.height, (img.h_samp, img.v_samp), planes, img.qtabs, out,
                        rgb_pitch=pitch, fancy=img.fancy, keep=keep, host=True)
    ctx.decode_host(d)
    ctx.sync()
    return out[:, :3 * img.width].reshape(img.height, img.width, 3)


@pytest.mark.parametrize("sampling,fancy,w,h", CASES)
def test_pageable_buffers(ctx, orc, sampling, fancy, w, h):
    rng = np.random.default_rng(w * h)
    img = synth.random_image(rng, w, h, sampling, fancy=fancy)
    pitch = 3 * w + 5
    out = np.full((h, pitch), POISON, np.uint8)
    got = _decode(ctx, img, out, pitch, pinned_planes=False)
    assert_same(got, oracle_rgb(orc, img), f"pageable {sampling} {w}x{h}")
    assert np.all(out[:, 3 * w:] == POISON)


@pytest.mark.parametrize("sampling,fancy,w,h", CASES)
def test_pinned_buffers(ctx, orc, sampling, fancy, w, h):
    import torch
    rng = np.random.default_rng(w * h + 1)
    img = synth.random_image(rng, w, h, sampling, fancy=fancy)
    pitch = 3 * w + 7
    buf = torch.full((h, pitch), POISON, dtype=torch.uint8).pin_memory()
    out = buf.numpy()
    got = _decode(ctx, img, out, pitch, pinned_planes=True)
    assert_same(got, oracle_rgb(orc, img), f"pinned {sampling} {w}x{h}")
    assert np.all(out[:, 3 * w:] == POISON)


def test_host_batch_equals_oracle_in_order(ctx, orc):
    import torch
    rng = np.random.default_rng(2024)
    imgs, aans = [], []
    for i in range(7):
        s = ["420", "444", "422", "440"][i % 4]
        imgs.append(synth.random_image(rng, int(rng.integers(1, 900)), int(rng.integers(1, 700)), s,
                                       fancy=bool(i % 3), qmax=255 if i % 4 else 65535))
        aans.append(i % 3 == 2)
    gray = synth.gray_image(synth.random_image(rng, 301, 203, "444"))
    outs, descs, keep = [], [], []
    for i, im in enumerate(imgs + [gray]):
        pitch = 3 * im.width + (i % 5)
        out = torch.full((im.height, pitch), POISON, dtype=torch.uint8).pin_memory().numpy()
        planes = [torch.from_numpy(np.ascontiguousarray(p)).pin_memory().numpy() for p in im.planes]
        keep += [planes, out]
        aan = aans[i] if i < len(imgs) else True
        descs.append(jdec.make_image(im.width, im.height, "gray" if len(im.planes) == 1 else (im.h_samp, im.v_samp),
                                     planes, im.qtabs, out, rgb_pitch=pitch, fancy=im.fancy, keep=keep, host=True,
                                     aan=aan))
        outs.append((im, out, aan))
    ctx.decode_host_batch(descs)
    ctx.sync()
    for i, (im, out, aan) in enumerate(outs):
        got = out[:, :3 * im.width].reshape(im.height, im.width, 3)
        if len(im.planes) == 1:
            want = orc.backend_decode_gray(im.width, im.height, im.planes[0], im.qtabs[0], aan=aan)
        else:
            want = oracle_rgb(orc, im, aan=aan)
        assert_same(got, want, f"host batch image {i}")
        assert np.all(out[:, 3 * im.width:] == POISON)


def test_host_batch_rejects_before_enqueueing(ctx):
    rng = np.random.default_rng(5)
    imgs = [synth.random_image(rng, 64, 48, "420") for _ in range(3)]
    outs = [np.full((48, 3 * 64), POISON, np.uint8) for _ in imgs]
    keep = []
    descs = [jdec.make_image(64, 48, "420", im.planes, im.qtabs, outs[i], fancy=True, keep=keep, host=True)
             for i, im in enumerate(imgs)]
    descs[2].rgb_pitch = 10   # invalid: the whole call is refused
    assert ctx.decode_host_batch(descs, check=False) == jdec.EINVAL
    ctx.sync()
    assert all(np.all(o == POISON) for o in outs)
    assert ctx.decode_host_batch([], check=False) == jdec.OK
