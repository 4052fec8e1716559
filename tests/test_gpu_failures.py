"""Failure detection without a GPU fault.

* A launch whose coefficient loads are withheld (JDEC_TEST_WITHHOLD_LOADS:
  the load barriers are armed but no copy is issued) must end by itself: each
  CTA's bounded wait gives up after its limit, the CTA stops without writing a
  pixel, jdec_sync_status reports JDEC_ETIMEOUT, and the same context then
  decodes normally, bit-exact.  Both warp-role kinds are exercised (split
  roles for 4:4:4, unified roles for full-width triangular 4:2:0 strips).
* An injected device-buffer allocation failure (JDEC_TEST_FAIL_ALLOCS=1, read
  at context creation) returns JDEC_ENOMEM from the call that needed the
  buffer, and the next call on the same context succeeds."""
import json
import time

import numpy as np
import pytest

from paper_1311_5304_gb300 import jdec, synth
from gpu_util import POISON, assert_same, gpu_rgb, oracle_rgb, upload

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("sampling,wt", [("444", 8), ("420", 20)])
def test_withheld_loads_time_out_and_context_stays_usable(orc, tmp_path, sampling, wt):
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    tune = tmp_path / "tune.json"
    # full-width strips: unified roles for 4:2:0 triangular, split roles for 4:4:4
    tune.write_text(json.dumps({"gpu": "x", "sms": sms, "entries": [[v, sc, wt] for v in range(5) for sc in range(20)]}))
    rng = np.random.default_rng(7 if sampling == "444" else 8)
    img = synth.random_image(rng, 640, 96, sampling, fancy=True)
    planes = upload(img)
    with jdec.Context(tune_file=str(tune)) as ctx:
        rgb = torch.full((img.height, img.width, 3), POISON, dtype=torch.uint8, device="cuda")
        keep = []
        d = jdec.make_image(img.width, img.height, (img.h_samp, img.v_samp), planes, img.qtabs, rgb,
                            fancy=img.fancy, keep=keep)
        d.flags |= jdec.TEST_WITHHOLD_LOADS
        t0 = time.time()
        assert ctx.decode_coeffs(d, check=False) == jdec.OK
        assert ctx.sync(check=False) == jdec.ETIMEOUT
        waited = time.time() - t0
        assert 1.5 < waited < 30.0
        assert int((rgb != POISON).sum()) == 0
        # the error word was cleared and the context still decodes
        assert ctx.sync(check=False) == jdec.OK
        got, _, _ = gpu_rgb(ctx, img, planes=planes)
        assert_same(got, oracle_rgb(orc, img), f"after timeout {sampling}")


def test_withhold_flag_rejected_by_batch_and_host_calls():
    rng = np.random.default_rng(9)
    img = synth.random_image(rng, 64, 48, "420")
    with jdec.Context() as ctx:
        import torch
        planes = upload(img)
        rgb = torch.empty((img.height, img.width, 3), dtype=torch.uint8, device="cuda")
        keep = []
        d = jdec.make_image(img.width, img.height, (img.h_samp, img.v_samp), planes, img.qtabs, rgb, keep=keep)
        d.flags |= jdec.TEST_WITHHOLD_LOADS
        assert ctx.decode_batch([d], check=False) == jdec.EINVAL
        hd = jdec.make_image(img.width, img.height, (img.h_samp, img.v_samp), img.planes, img.qtabs,
                             np.empty((img.height, img.width, 3), np.uint8), keep=keep, host=True)
        hd.flags |= jdec.TEST_WITHHOLD_LOADS
        assert ctx.decode_host(hd, check=False) == jdec.EINVAL


def test_injected_allocation_failure_leaves_context_usable(orc, monkeypatch):
    rng = np.random.default_rng(10)
    img = synth.random_image(rng, 301, 203, "422", fancy=True)
    monkeypatch.setenv("JDEC_TEST_FAIL_ALLOCS", "1")
    ctx = jdec.Context()
    monkeypatch.delenv("JDEC_TEST_FAIL_ALLOCS")
    try:
        keep = []
        out = np.full((img.height, img.width, 3), POISON, np.uint8)
        hd = jdec.make_image(img.width, img.height, (img.h_samp, img.v_samp), img.planes, img.qtabs, out,
                             fancy=img.fancy, keep=keep, host=True)
        assert ctx.decode_host(hd, check=False) == jdec.ENOMEM
        assert ctx.decode_host(hd, check=False) == jdec.OK
        assert ctx.sync(check=False) == jdec.OK
        assert_same(out, oracle_rgb(orc, img), "after injected allocation failure")
    finally:
        ctx.close()
