"""Batched decoding (one persistent launch over a flattened MCU work list,
recorded as a CUDA graph): every image must come out bit-identical to the
oracle and to its own single-image launch, whatever the mix of sizes,
samplings, upsampling modes and quantisation tables in the batch."""
import numpy as np
import pytest

from paper_1311_5304_gb300 import jdec, synth
from gpu_util import assert_same, oracle_rgb, upload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = jdec.Context()
    yield c
    c.close()


def _rgb_buffers(imgs):
    import torch
    return [torch.full((im.height, im.width, 3), 0xCD, dtype=torch.uint8, device="cuda") for im in imgs]


def _descs(imgs, planes, rgbs, keep):
    return [jdec.make_image(im.width, im.height, (im.h_samp, im.v_samp), planes[i], im.qtabs, rgbs[i],
                            fancy=im.fancy, keep=keep) for i, im in enumerate(imgs)]


def _mixed(rng, n, wmax=700, hmax=500):
    imgs = []
    for i in range(n):
        s = ["420", "422", "444", "440"][i % 4]
        w, h = int(rng.integers(1, wmax)), int(rng.integers(1, hmax))
        im = synth.random_image(rng, w, h, s, fancy=bool(i % 4 != 1), qmax=255 if i % 5 else 65535)
        imgs.append(im)
    return imgs


def test_mixed_batch_matches_oracle_and_plain(ctx, orc):
    import torch
    rng = np.random.default_rng(4)
    imgs = _mixed(rng, 40)
    planes = [upload(im) for im in imgs]
    keep = []
    rgb_b = _rgb_buffers(imgs)
    ctx.decode_batch(_descs(imgs, planes, rgb_b, keep))
    rgb_p = _rgb_buffers(imgs)
    for d in _descs(imgs, planes, rgb_p, keep):
        ctx.decode_coeffs(d)
    ctx.sync()
    for i, im in enumerate(imgs):
        got = rgb_b[i].cpu().numpy()
        assert np.array_equal(got, rgb_p[i].cpu().numpy()), i
        assert_same(got, oracle_rgb(orc, im, 1), f"batch image {i} {im.width}x{im.height} {im.sampling}")


def test_graph_replay_with_new_contents(ctx, orc):
    # same shape twice (the recorded graph is replayed), different coefficients
    rng = np.random.default_rng(9)
    a = _mixed(rng, 12, 300, 200)
    b = [synth.random_image(rng, im.width, im.height, im.sampling, fancy=im.fancy) for im in a]
    for imgs in (a, b, a):
        planes = [upload(im) for im in imgs]
        keep = []
        rgbs = _rgb_buffers(imgs)
        ctx.decode_batch(_descs(imgs, planes, rgbs, keep))
        ctx.sync()
        for i, im in enumerate(imgs):
            assert_same(rgbs[i].cpu().numpy(), oracle_rgb(orc, im, 1), f"replay image {i}")


def test_batch_of_one_and_tiny_images(ctx, orc):
    rng = np.random.default_rng(17)
    for n in (1, 2, 7):
        imgs = [synth.random_image(rng, int(rng.integers(1, 40)), int(rng.integers(1, 40)),
                                   ["420", "422", "444"][k % 3]) for k in range(n)]
        planes = [upload(im) for im in imgs]
        keep = []
        rgbs = _rgb_buffers(imgs)
        ctx.decode_batch(_descs(imgs, planes, rgbs, keep))
        ctx.sync()
        for i, im in enumerate(imgs):
            assert_same(rgbs[i].cpu().numpy(), oracle_rgb(orc, im, 1), f"n={n} image {i}")


def test_invalid_batch_launches_nothing(ctx):
    import torch
    rng = np.random.default_rng(1)
    imgs = _mixed(rng, 3, 60, 60)
    planes = [upload(im) for im in imgs]
    keep = []
    rgbs = _rgb_buffers(imgs)
    ds = _descs(imgs, planes, rgbs, keep)
    ds[1].rgb_pitch = 1
    assert ctx.decode_batch(ds, check=False) == jdec.EINVAL
    torch.cuda.synchronize()
    assert all(int((r != 0xCD).sum()) == 0 for r in rgbs)
    assert jdec.load().jdec_decode_batch(ctx._h, None, 1, None) == jdec.EINVAL


def test_config4_full_batch_matches_oracle(ctx, orc):
    # 1024 images, W ~ U[160, 4096], H ~ U[120, 3072], 40/30/30 % 4:2:0/4:2:2/4:4:4,
    # quality ~ U{50..95}: crops of per-sampling coefficient atlases.  Every
    # image is compared with the oracle (and with its own plain launch).
    import torch
    seed = 13115304 + 4000
    specs = synth.batch_specs(1024, seed)
    atl = {s: synth.atlas(s, seed=seed + k) for k, s in enumerate(("420", "422", "444"))}
    offs = synth.crop_offsets(specs, atl, seed)
    dev_atl = {s: [torch.from_numpy(p).cuda() for p in a.planes] for s, a in atl.items()}
    planes, rgbs, descs, keep = [], [], [], []
    for i, (w, h, s, q) in enumerate(specs):
        pl = [p.contiguous() for p in synth.crop_planes(dev_atl[s], s, w, h, offs[i])]
        planes.append(pl)
        rgb = torch.empty((h, w, 3), dtype=torch.uint8, device="cuda")
        rgbs.append(rgb)
        qt = [synth.quality_table(q, False), synth.quality_table(q, True), synth.quality_table(q, True)]
        descs.append(jdec.make_image(w, h, s, pl, qt, rgb, keep=keep))
    ctx.decode_batch(descs)
    ctx.sync()
    for i in range(1024):
        w, h, s, q = specs[i]
        ref = torch.empty_like(rgbs[i])
        keep2 = []
        qt = [synth.quality_table(q, False), synth.quality_table(q, True), synth.quality_table(q, True)]
        ctx.decode_coeffs(jdec.make_image(w, h, s, planes[i], qt, ref, keep=keep2))
        ctx.sync()
        got = rgbs[i].cpu().numpy()
        assert np.array_equal(ref.cpu().numpy(), got), i
        im = synth.batch_image(specs, atl, offs, i)
        assert_same(got, oracle_rgb(orc, im), f"config-4 image {i} {im.width}x{im.height} {s}")


def test_back_to_back_batches_without_waiting(ctx, orc):
    # Calls issued back to back prepare their work lists in alternating
    # staging buffers while earlier batches still run; each batch must still
    # decode its own images (same and different shapes, no host wait between)
    rng = np.random.default_rng(23)
    batches = [_mixed(rng, 9, 260, 200), None, _mixed(rng, 14, 180, 120), None, _mixed(rng, 5, 400, 300)]
    batches[1] = [synth.random_image(rng, im.width, im.height, im.sampling, fancy=im.fancy) for im in batches[0]]
    batches[3] = [synth.random_image(rng, im.width, im.height, im.sampling, fancy=im.fancy) for im in batches[2]]
    keep, outs = [], []
    for imgs in batches:
        planes = [upload(im) for im in imgs]
        rgbs = _rgb_buffers(imgs)
        keep.append(planes)
        ctx.decode_batch(_descs(imgs, planes, rgbs, keep))
        outs.append(rgbs)
    ctx.sync()
    for b, imgs in enumerate(batches):
        for i, im in enumerate(imgs):
            assert_same(outs[b][i].cpu().numpy(), oracle_rgb(orc, im, 1), f"batch {b} image {i}")
