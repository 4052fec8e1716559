"""Single-component (grayscale) images through every entry point: bit-exact
R = G = B = Y against the oracle's grayscale back-end, alone and mixed with
colour images in batches, from device and host buffers."""
import numpy as np
import pytest

from paper_1311_5304_gb300 import jdec, synth
from gpu_util import POISON, assert_same, oracle_rgb

pytestmark = pytest.mark.gpu


def gray_image(rng, w, h, qmax=255):
    img = synth.random_image(rng, w, h, "444", qmax=qmax)
    return img.planes[0], img.qtabs[0]


@pytest.fixture(scope="module")
def ctx():
    c = jdec.Context()
    yield c
    c.close()


def _decode(ctx, w, h, plane, q, pitch=None):
    import torch
    pitch = pitch or 3 * w
    out = torch.full((h, pitch), POISON, dtype=torch.uint8, device="cuda")
    keep = []
    d = jdec.make_image(w, h, "gray", [torch.from_numpy(np.ascontiguousarray(plane)).cuda()], [q], out,
                        rgb_pitch=pitch, keep=keep)
    ctx.decode_coeffs(d)
    ctx.sync()
    host = out.cpu().numpy()
    return host[:, :3 * w].reshape(h, w, 3), host


@pytest.mark.parametrize("w,h", [(1, 1), (7, 9), (8, 8), (33, 31), (640, 481), (2049, 1025), (4096, 3072)])
def test_matches_oracle(ctx, orc, w, h):
    rng = np.random.default_rng(w * 7 + h)
    plane, q = gray_image(rng, w, h, qmax=255 if w % 2 else 65535)
    got, host = _decode(ctx, w, h, plane, q, pitch=3 * w + 5)
    assert_same(got, orc.backend_decode_gray(w, h, plane, q), f"gray {w}x{h}")
    assert np.all(host[:, 3 * w:] == POISON)


def test_batch_mixed_with_colour(ctx, orc):
    import torch
    rng = np.random.default_rng(77)
    keep, descs, outs, wants = [], [], [], []
    for i in range(12):
        w, h = int(rng.integers(1, 900)), int(rng.integers(1, 600))
        out = torch.full((h, 3 * w), POISON, dtype=torch.uint8, device="cuda")
        if i % 3 == 0:
            plane, q = gray_image(rng, w, h)
            descs.append(jdec.make_image(w, h, "gray", [torch.from_numpy(plane).cuda()], [q], out, keep=keep))
            wants.append(orc.backend_decode_gray(w, h, plane, q))
        else:
            img = synth.random_image(rng, w, h, ["444", "422", "420"][i % 3], fancy=bool(i % 2))
            planes = [torch.from_numpy(np.ascontiguousarray(p)).cuda() for p in img.planes]
            descs.append(jdec.make_image(w, h, (img.h_samp, img.v_samp), planes, img.qtabs, out,
                                         fancy=img.fancy, keep=keep))
            wants.append(oracle_rgb(orc, img))
        outs.append(out)
    ctx.decode_batch(descs)
    ctx.sync()
    for i, (o, want) in enumerate(zip(outs, wants)):
        h, w = want.shape[:2]
        assert_same(o.cpu().numpy().reshape(h, w, 3), want, f"batch item {i}")
    # the allocation-free entry point as well
    outs2 = []
    for i, d in enumerate(descs):
        h, w = wants[i].shape[:2]
        o = torch.full((h, 3 * w), POISON, dtype=torch.uint8, device="cuda")
        d.rgb = o.data_ptr()
        outs2.append(o)
    assert jdec.decode_batch_static(descs) == jdec.OK
    torch.cuda.synchronize()
    for i, (o, want) in enumerate(zip(outs2, wants)):
        h, w = want.shape[:2]
        assert_same(o.cpu().numpy().reshape(h, w, 3), want, f"static batch item {i}")


def test_host_buffers(ctx, orc):
    rng = np.random.default_rng(9)
    w, h = 1283, 901
    plane, q = gray_image(rng, w, h)
    out = np.full((h, 3 * w + 3), POISON, np.uint8)
    keep = []
    d = jdec.make_image(w, h, "gray", [plane], [q], out, keep=keep, host=True)
    ctx.decode_host(d)
    ctx.sync()
    assert_same(out[:, :3 * w].reshape(h, w, 3), orc.backend_decode_gray(w, h, plane, q), "gray host")
    assert np.all(out[:, 3 * w:] == POISON)


def test_unsupported_single_component_sampling(ctx):
    import torch
    rng = np.random.default_rng(1)
    plane, q = gray_image(rng, 64, 64)
    out = torch.empty((64, 192), dtype=torch.uint8, device="cuda")
    keep = []
    d = jdec.make_image(64, 64, "gray", [torch.from_numpy(plane).cuda()], [q], out, keep=keep)
    d.h_samp[0] = 2
    assert ctx.decode_coeffs(d, check=False) == jdec.EUNSUPPORTED
