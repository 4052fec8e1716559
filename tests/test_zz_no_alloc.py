"""jdec_decode_batch_static: the batched decode for callers that cannot
allocate device memory -- processes whose HBM is all held by another
allocator (a framework's caching pool), and latency-critical paths that cannot
take the device-wide synchronisation of cudaMalloc/cudaFree.  It keeps its
descriptors and work list in a static device array instead of context-owned
buffers.

Called through the C ABI, two calls in a row with different batches must
each give exactly the oracle's bytes and those of the context-owned
jdec_decode_batch (every stage is integer: tolerance 0), also on a
non-default stream and with CTAs whose items mix variant classes.  Oversized
requests (more than 128 images, or a work list above 16384 items) return
JDEC_EINVAL and write nothing.  Collected last so that a failure here leaves
every other test already run."""
import numpy as np
import pytest

from paper_1311_5304_gb300 import jdec, synth
from gpu_util import assert_same, oracle_rgb

pytestmark = pytest.mark.gpu


def _batch(rng, n, wmax, hmax):
    import torch
    imgs, planes = [], []
    for i in range(n):
        s = ["420", "422", "444", "440"][i % 4]
        im = synth.random_image(rng, int(rng.integers(1, wmax)), int(rng.integers(1, hmax)), s,
                                fancy=bool(i % 4 != 2), qmax=255 if i % 5 else 65535)
        imgs.append(im)
        planes.append([torch.from_numpy(np.ascontiguousarray(p)).cuda() for p in im.planes])
    return imgs, planes


def _descs(imgs, planes, keep, aan):
    import torch
    rgbs = [torch.full((im.height, im.width, 3), 0xCD, dtype=torch.uint8, device="cuda") for im in imgs]
    ds = [jdec.make_image(im.width, im.height, (im.h_samp, im.v_samp), planes[i], im.qtabs, rgbs[i],
                          fancy=im.fancy, keep=keep, aan=aan[i]) for i, im in enumerate(imgs)]
    return ds, rgbs


@pytest.mark.parametrize("side_stream", [False, True])
def test_static_scratch_batch_matches_oracle_and_context_batch_twice(orc, side_stream):
    import torch
    torch.cuda.set_device(0)
    rng = np.random.default_rng(20261204 + int(side_stream))
    stream = torch.cuda.Stream() if side_stream else None
    with jdec.Context() as ctx:
        # the second batch has many small images of every class, so that one
        # CTA runs items of several classes in the shared layout
        for call, (n, wmax, hmax) in enumerate([(24, 900, 700), (97, 120, 90)]):
            imgs, planes = _batch(rng, n, wmax, hmax)
            aan = [i % 3 == 0 for i in range(n)]
            keep = []
            ds_static, rgb_static = _descs(imgs, planes, keep, aan)
            ds_ctx, rgb_ctx = _descs(imgs, planes, keep, aan)
            torch.cuda.synchronize()
            assert jdec.decode_batch_static(ds_static, stream=stream, check=False) == jdec.OK
            ctx.decode_batch(ds_ctx)
            torch.cuda.synchronize()
            ctx.sync()
            for i, im in enumerate(imgs):
                got = rgb_static[i].cpu().numpy()
                assert np.array_equal(got, rgb_ctx[i].cpu().numpy()), (call, i)
                assert_same(got, oracle_rgb(orc, im, 1, aan=aan[i]),
                            f"call {call} image {i} {im.width}x{im.height} {im.sampling}")


def test_static_scratch_rejects_too_many_images():
    import torch
    torch.cuda.set_device(0)
    rng = np.random.default_rng(3)
    imgs, planes = _batch(rng, 129, 20, 20)
    ds, rgbs = _descs(imgs, planes, [], [False] * 129)
    assert jdec.decode_batch_static(ds, check=False) == jdec.EINVAL
    torch.cuda.synchronize()
    assert all(int((r != 0xCD).sum()) == 0 for r in rgbs)


def test_static_scratch_rejects_a_work_list_beyond_its_limit(orc):
    # 128 images (within the image limit) of 65535 x 8 pixels, 4:4:4: each has
    # 256 strips of one MCU row, so the work list needs about 32768 items,
    # twice the static array's 16384.  The planes are shared by every image.
    import torch
    torch.cuda.set_device(0)
    w, h = 65535, 8
    im = synth.random_image(np.random.default_rng(5), w, h, "444")
    planes = [torch.from_numpy(np.ascontiguousarray(p)).cuda() for p in im.planes]
    keep = []
    rgbs = [torch.full((h, w, 3), 0xCD, dtype=torch.uint8, device="cuda") for _ in range(2)]
    ds = [jdec.make_image(w, h, (im.h_samp, im.v_samp), planes, im.qtabs, rgbs[k % 2], keep=keep)
          for k in range(128)]
    assert jdec.decode_batch_static(ds, check=False) == jdec.EINVAL
    torch.cuda.synchronize()
    assert all(int((r != 0xCD).sum()) == 0 for r in rgbs)
    # two of the same images, a batch the array holds, decode normally
    assert jdec.decode_batch_static(ds[:2], check=False) == jdec.OK
    torch.cuda.synchronize()
    want = oracle_rgb(orc, im)
    for r in rgbs:
        assert_same(r.cpu().numpy(), want, "65535x8 4:4:4")


def test_static_scratch_reports_a_device_timeout_and_stays_usable(orc):
    # The withheld-load testing aid arms the load barriers and issues no copy:
    # every CTA's bounded wait gives up, the CTA stops without writing, the
    # error word in the static array is set and jdec_batch_static_status
    # reports JDEC_ETIMEOUT (then clears it); the next call decodes exactly.
    import time
    import torch
    torch.cuda.set_device(0)
    rng = np.random.default_rng(11)
    imgs, planes = _batch(rng, 3, 300, 200)
    keep = []
    ds, rgbs = _descs(imgs, planes, keep, [False] * 3)
    for d in ds:
        d.flags |= jdec.TEST_WITHHOLD_LOADS
    t0 = time.time()
    assert jdec.decode_batch_static(ds, check=False) == jdec.OK
    assert jdec.batch_static_status() == jdec.ETIMEOUT
    assert 1.5 < time.time() - t0 < 30.0
    assert all(int((r != 0xCD).sum()) == 0 for r in rgbs)
    assert jdec.batch_static_status() == jdec.OK
    ds, rgbs = _descs(imgs, planes, keep, [False] * 3)
    assert jdec.decode_batch_static(ds, check=False) == jdec.OK
    assert jdec.batch_static_status() == jdec.OK
    for i, im in enumerate(imgs):
        assert_same(rgbs[i].cpu().numpy(), oracle_rgb(orc, im, 1), f"after timeout, image {i}")
