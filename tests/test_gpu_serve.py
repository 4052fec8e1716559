"""Continuous-batching server: every request's RGB equals its standalone
decode (bit for bit) whatever else shares its batches, the HBM budget is never
exceeded, and a malformed request fails alone."""
import numpy as np
import pytest

from paper_1311_5304_gb300 import jdec, serve, synth

pytestmark = pytest.mark.gpu

MIX = ((48, 40, 0.6), (320, 240, 0.3), (1000, 700, 0.1))


@pytest.fixture(scope="module")
def ctx():
    c = jdec.Context()
    yield c
    c.close()


def _standalone(ctx, data):
    import torch
    info = jdec.jpeg_parse(data)
    planes = [np.zeros((info.blocks_h[c], info.blocks_w[c], 64), np.int16) for c in range(3)]
    jdec.entropy_decode(data, planes)
    dp = [torch.from_numpy(p).cuda() for p in planes]
    rgb = torch.empty((info.height, info.width, 3), dtype=torch.uint8, device="cuda")
    keep = []
    qt = [np.array(info.qtab[c][:], np.uint16) for c in range(3)]
    ctx.decode_coeffs(jdec.make_image(info.width, info.height, (tuple(info.h_samp), tuple(info.v_samp)), dp, qt, rgb,
                                      keep=keep))
    ctx.sync()
    return rgb.cpu().numpy(), planes, qt, info


def test_results_identical_alone_and_in_the_mix(ctx, orc):
    pool = serve.request_pool(77, per_class=(6, 4, 2), mix=MIX)
    srv = serve.Server(ctx, hbm_budget_bytes=64 << 20, keep_results=True)
    try:
        stats = serve.run_load(srv, pool, rate=3000.0, n=300, seed=5, mix=MIX, timeout=60)
    finally:
        srv.close()
    assert stats["drained"] and stats["completed"] == 300 and stats["errors"] == 0
    assert srv.peak_used <= 64 << 20
    alone = {}
    for r in srv.finished:
        key = id(r.data)
        if key not in alone:
            alone[key] = _standalone(ctx, r.data)
        assert np.array_equal(r.rgb.cpu().numpy(), alone[key][0]), r.rid
    # and the standalone decodes equal the oracle
    for (rgb, planes, qt, info) in list(alone.values())[:4]:
        want = orc.backend_decode(info.width, info.height, tuple(info.h_samp), tuple(info.v_samp), planes, qt, True)
        assert np.array_equal(rgb, want)


def test_budget_limits_admission(ctx):
    pool = serve.request_pool(78, per_class=(2, 2, 2), mix=MIX)
    big = serve.Server(ctx, hbm_budget_bytes=10 << 20, keep_results=False)   # two 1000x700 requests (4.2 MB each)
    try:
        stats = serve.run_load(big, pool, rate=20000.0, n=120, seed=9, mix=MIX, timeout=60)
    finally:
        big.close()
    assert stats["completed"] == 120
    assert big.peak_used <= 10 << 20


def test_malformed_request_fails_alone(ctx):
    pool = serve.request_pool(79, per_class=(3, 1, 1), mix=MIX)
    srv = serve.Server(ctx, hbm_budget_bytes=64 << 20, keep_results=True)
    try:
        import time
        now = time.perf_counter()
        good = [serve.Request(i, now, data=pool[0][i % 3]) for i in range(10)]
        bad = serve.Request(99, now, data=pool[1][0][:300])
        for r in good[:5] + [bad] + good[5:]:
            srv.submit(r)
        assert srv.drain(60)
    finally:
        srv.close()
    errs = [r for r in srv.finished if r.error]
    assert [r.rid for r in errs] == [99]
    assert sum(1 for r in srv.finished if r.error is None) == 10


def test_coefficient_mode(ctx):
    pool = serve.request_pool(80, per_class=(3, 2, 1), mode="coef", mix=MIX)
    srv = serve.Server(ctx, hbm_budget_bytes=64 << 20, keep_results=True)
    try:
        stats = serve.run_load(srv, pool, rate=5000.0, n=100, seed=3, mode="coef", mix=MIX, timeout=60)
    finally:
        srv.close()
    assert stats["completed"] == 100


def test_request_larger_than_budget_is_rejected(ctx):
    pool = serve.request_pool(81, per_class=(1, 1, 1), mix=MIX)
    srv = serve.Server(ctx, hbm_budget_bytes=1 << 20, keep_results=False)
    try:
        import time
        now = time.perf_counter()
        srv.submit(serve.Request(1, now, data=pool[0][0]))   # 48x40: fits
        srv.submit(serve.Request(2, now, data=pool[2][0]))   # 1000x700: 4.2 MB, never fits
        assert srv.drain(60)
    finally:
        srv.close()
    by = {r.rid: r for r in srv.finished}
    assert by[1].error is None and by[2].error is not None


def test_grayscale_requests_in_the_mix(ctx, orc):
    # grayscale and colour JPEG requests share batches; each equals the oracle
    import time
    grays = []
    for k in range(3):
        src = synth.make_image(200 + 37 * k, 150 + 11 * k, "444", 85, seed=90 + k, kind="texture", sigma=4)
        g = synth.gray_image(src)
        grays.append((synth.encode_jfif(g), g))
    colour = serve.request_pool(82, per_class=(2, 2, 0), mix=MIX)
    srv = serve.Server(ctx, hbm_budget_bytes=64 << 20, keep_results=True)
    try:
        now = time.perf_counter()
        rid = 0
        for data, _ in grays:
            srv.submit(serve.Request(rid, now, data=data))
            rid += 1
        for cls in colour[:2]:
            for data in cls:
                srv.submit(serve.Request(rid, now, data=data))
                rid += 1
        assert srv.drain(60)
    finally:
        srv.close()
    by = {r.rid: r for r in srv.finished}
    assert all(r.error is None for r in by.values())
    for i, (_, g) in enumerate(grays):
        want = orc.backend_decode_gray(g.width, g.height, g.planes[0], g.qtabs[0])
        assert np.array_equal(by[i].rgb.cpu().numpy(), want), i


def test_plain_mode_gives_the_batched_results(ctx):
    # the per-request launch mode (one jdec_decode_coeffs per request) decodes
    # every request to the same bytes as its standalone decode
    pool = serve.request_pool(83, per_class=(4, 3, 1), mix=MIX)
    srv = serve.Server(ctx, hbm_budget_bytes=64 << 20, keep_results=True, plain=True)
    try:
        stats = serve.run_load(srv, pool, rate=4000.0, n=120, seed=6, mix=MIX, timeout=60)
    finally:
        srv.close()
    assert stats["drained"] and stats["completed"] == 120 and stats["errors"] == 0
    assert srv.peak_used <= 64 << 20
    alone = {}
    for r in srv.finished:
        key = id(r.data)
        if key not in alone:
            alone[key] = _standalone(ctx, r.data)[0]
        assert np.array_equal(r.rgb.cpu().numpy(), alone[key]), r.rid
