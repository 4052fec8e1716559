"""The seeded input generator (shared by the tests and the benchmark; no
decode arithmetic): every image is a pure function of its seed and recipe,
whatever the thread count, and different seeds give different content."""
import numpy as np
import pytest

from paper_1311_5304_gb300 import synth


@pytest.mark.parametrize("sampling,kind", [("420", "texture"), ("444", "gradient"), ("440", "texture")])
def test_same_seed_same_planes_for_any_thread_count(sampling, kind):
    imgs = [synth.make_image(333, 217, sampling, 85, seed=77, kind=kind, sigma=4.0, threads=t)
            for t in (1, 3, 8)]
    for im in imgs[1:]:
        for a, b in zip(imgs[0].planes, im.planes):
            assert np.array_equal(a, b)
        for a, b in zip(imgs[0].qtabs, im.qtabs):
            assert np.array_equal(a, b)


def test_seeds_and_qualities_change_the_content():
    a = synth.make_image(128, 96, "420", 85, seed=1, kind="texture", sigma=4.0)
    b = synth.make_image(128, 96, "420", 85, seed=2, kind="texture", sigma=4.0)
    c = synth.make_image(128, 96, "420", 50, seed=1, kind="texture", sigma=4.0)
    assert not np.array_equal(a.planes[0], b.planes[0])
    assert not np.array_equal(a.qtabs[0], c.qtabs[0])


def test_quality_scaling_follows_the_ijg_rule():
    # Q = clamp((t * s + 50) / 100, 1, 255), s = 5000 / q below 50, else 200 - 2q,
    # applied to the same base table: q = 50 returns the base table itself
    base = synth.make_image(16, 16, "444", 50, seed=1).qtabs[0].astype(np.int64)
    for q in (10, 75, 90, 100):
        s = 5000 // q if q < 50 else 200 - 2 * q
        want = np.clip((base * s + 50) // 100, 1, 255)
        assert np.array_equal(synth.make_image(16, 16, "444", q, seed=1).qtabs[0], want), q


@pytest.mark.parametrize("sampling", ["444", "422", "420"])
def test_large_image_content_has_its_nonzero_ac_band(sampling):
    # The 8192x8192 q90 texture images (cover 0.85, grain 4) have 30-60 % of
    # their AC coefficients nonzero over all planes, chroma included, with the
    # fraction falling along zig-zag order.  The statistics are local (texture
    # cells of at most 192 px), so a 1024x1024 crop of the same recipe shows them.
    img = synth.make_image(1024, 1024, sampling, 90, seed=13115304 + 2000, kind="texture", sigma=4.0, cover=0.85)
    assert 0.30 <= synth.nonzero_ac_fraction(img) <= 0.60
    for p in img.planes[1:]:
        assert np.count_nonzero(p[..., 1:]) / p[..., 1:].size >= 0.25
    nz = sum(np.count_nonzero(p, axis=(0, 1)) for p in img.planes)
    assert nz[1] > nz[20] > nz[63]
