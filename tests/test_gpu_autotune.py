"""Strip-width autotuner: the first image of each (variant, size class) is
timed at the candidate widths and the fastest is kept and saved; results stay
bit-exact, the table is written as JSON for this GPU, and a new context
loading it decodes the same bytes with the tuned width."""
import json

import numpy as np
import pytest

from paper_1311_5304_gb300 import jdec, synth
from gpu_util import assert_same, gpu_rgb, oracle_rgb

pytestmark = pytest.mark.gpu

CANDIDATES = {4, 6, 8, 10, 12, 16, 20, 21, 24, 31, 32, 42}


def test_autotune_writes_table_and_stays_exact(orc, tmp_path):
    path = tmp_path / "tune.json"
    imgs = [synth.make_image(2048, 1536, s, 85, seed=61, kind="texture", sigma=4, fancy=True)
            for s in ("444", "422", "420")]
    with jdec.Context(autotune=True, tune_file=str(path)) as ctx:
        for img in imgs:
            got, _, _ = gpu_rgb(ctx, img)
            assert_same(got, oracle_rgb(orc, img), f"autotuned {img.sampling}")
    table = json.loads(path.read_text())
    import torch
    assert table["sms"] == torch.cuda.get_device_properties(0).multi_processor_count
    entries = table["entries"]
    assert {e[0] for e in entries} == {0, 2, 4}   # 4:4:4, 4:2:2 and 4:2:0 triangular
    assert all(e[2] in CANDIDATES for e in entries)
    # a second context loads the table (no tuning) and decodes the same bytes
    with jdec.Context(tune_file=str(path)) as ctx2:
        for img in imgs:
            got, _, _ = gpu_rgb(ctx2, img)
            assert_same(got, oracle_rgb(orc, img), f"loaded table {img.sampling}")


def test_table_of_another_gpu_is_ignored(orc, tmp_path):
    path = tmp_path / "tune.json"
    path.write_text(json.dumps({"gpu": "other", "sms": 7, "entries": [[v, sc, 1] for v in range(5) for sc in range(20)]}))
    img = synth.make_image(640, 480, "420", 80, seed=3, kind="texture", sigma=4, fancy=True)
    with jdec.Context(tune_file=str(path)) as ctx:
        got, _, _ = gpu_rgb(ctx, img)
    assert_same(got, oracle_rgb(orc, img), "foreign table")


@pytest.mark.parametrize("text", ['{"sms"', '{"sms": }', '{"gpu": "x", "sms": 152, "entries": [[4, 5', "", "\x00\xff"])
def test_malformed_table_is_ignored(orc, tmp_path, text):
    path = tmp_path / "tune.json"
    path.write_bytes(text.encode("latin-1"))
    img = synth.make_image(640, 480, "420", 80, seed=3, kind="texture", sigma=4, fancy=True)
    with jdec.Context(tune_file=str(path)) as ctx:
        got, _, _ = gpu_rgb(ctx, img)
    assert_same(got, oracle_rgb(orc, img), "malformed table")


def test_batch_autotune_picks_a_shape_per_class_and_stays_exact(orc, tmp_path):
    # jdec_decode_batch with autotune times strip width x IDCT-thread split per
    # (batch class, size class), keeps the fastest, saves it as a kind-1 entry,
    # and every image stays bit-exact; a context loading the table reuses it
    import torch
    path = tmp_path / "tune.json"
    rng = np.random.default_rng(41)
    imgs = []
    for i in range(18):
        s = ["420", "422", "444"][i % 3]
        imgs.append(synth.random_image(rng, int(rng.integers(100, 900)), int(rng.integers(80, 600)), s, fancy=True))
    planes = [[torch.from_numpy(np.ascontiguousarray(p)).cuda() for p in im.planes] for im in imgs]

    def run(ctx):
        keep = []
        rgbs = [torch.full((im.height, im.width, 3), 0xCD, dtype=torch.uint8, device="cuda") for im in imgs]
        ds = [jdec.make_image(im.width, im.height, (im.h_samp, im.v_samp), planes[i], im.qtabs, rgbs[i],
                              fancy=im.fancy, keep=keep) for i, im in enumerate(imgs)]
        ctx.decode_batch(ds)
        ctx.sync()
        return [r.cpu().numpy() for r in rgbs]

    with jdec.Context(autotune=True, tune_file=str(path)) as ctx:
        got = run(ctx)
        got2 = run(ctx)              # tuned shapes reused
    for i, im in enumerate(imgs):
        want = oracle_rgb(orc, im, 1)
        assert_same(got[i], want, f"autotuned batch image {i}")
        assert np.array_equal(got2[i], want), i
    entries = json.loads(path.read_text())["entries"]
    batch = [e for e in entries if len(e) >= 5 and e[4] == 1]
    # one entry per class present (LLM IDCT with 8-bit or 16-bit tables)
    classes = {3 * v + m for v in (0, 2, 4) for m in (0, 1)}
    assert batch and {e[0] for e in batch} <= classes
    assert all(e[2] in (8, 12, 16, 20, 24, 31, 32) and e[3] in (32, 64, 96) for e in batch)
    before = path.read_text()
    with jdec.Context(tune_file=str(path)) as ctx2:
        got3 = run(ctx2)
    assert path.read_text() == before
    for i in range(len(imgs)):
        assert np.array_equal(got3[i], got[i]), i
