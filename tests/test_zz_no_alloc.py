"""jdec_decode_batch_static: the batched decode for callers that cannot
allocate device memory (code running under CUDA-graph stream capture,
processes whose HBM is all held by another allocator, paths that cannot take
the device synchronisation of cudaMalloc/cudaFree).  It keeps its work list in
a static device array instead of context-owned buffers.

Called through the C ABI, two calls in a row with different batches must
each give exactly the bytes of the context-owned jdec_decode_batch (the
integer path is bit-exact, tolerance 0).  Collected last so that a failure
here leaves every other test already run."""
import numpy as np
import pytest

from paper_1311_5304_gb300 import jdec, synth

pytestmark = pytest.mark.gpu


def _batch(rng, n, wmax, hmax):
    import torch
    imgs, planes, keep = [], [], []
    for i in range(n):
        s = ["420", "422", "444", "440"][i % 4]
        im = synth.random_image(rng, int(rng.integers(1, wmax)), int(rng.integers(1, hmax)), s,
                                fancy=bool(i % 4 != 2), qmax=255 if i % 5 else 65535)
        imgs.append(im)
        planes.append([torch.from_numpy(np.ascontiguousarray(p)).cuda() for p in im.planes])
    return imgs, planes, keep


def _descs(imgs, planes, keep):
    import torch
    rgbs = [torch.full((im.height, im.width, 3), 0xCD, dtype=torch.uint8, device="cuda") for im in imgs]
    ds = [jdec.make_image(im.width, im.height, (im.h_samp, im.v_samp), planes[i], im.qtabs, rgbs[i],
                          fancy=im.fancy, keep=keep, aan=(i % 3 == 0)) for i, im in enumerate(imgs)]
    return ds, rgbs


def test_static_scratch_batch_matches_context_batch_twice():
    import torch
    torch.cuda.set_device(0)
    rng = np.random.default_rng(20261204)
    with jdec.Context() as ctx:
        for call, (n, wmax, hmax) in enumerate([(24, 900, 700), (37, 400, 300)]):
            imgs, planes, keep = _batch(rng, n, wmax, hmax)
            ds_static, rgb_static = _descs(imgs, planes, keep)
            ds_ctx, rgb_ctx = _descs(imgs, planes, keep)
            assert jdec.decode_batch_static(ds_static, check=False) == jdec.OK
            ctx.decode_batch(ds_ctx)
            torch.cuda.synchronize()
            ctx.sync()
            for i in range(n):
                assert torch.equal(rgb_static[i], rgb_ctx[i]), (call, i)


def test_static_scratch_rejects_oversized_batches():
    import torch
    torch.cuda.set_device(0)
    rng = np.random.default_rng(3)
    imgs, planes, keep = _batch(rng, 129, 20, 20)
    ds, rgbs = _descs(imgs, planes, keep)
    assert jdec.decode_batch_static(ds, check=False) == jdec.EINVAL
    torch.cuda.synchronize()
    assert all(int((r != 0xCD).sum()) == 0 for r in rgbs)
