"""jdec_decode_host: host coefficient planes and host RGB, copied in row
bands through device staging.  Pageable and page-locked buffers, odd pitches:
exactly the oracle's bytes inside W x H, row padding untouched."""
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
