"""Pins for the oracle's colour conversion (Sec. 4.3, Alg. 2) and chroma
upsampling (Sec. 4.2, Alg. 1 and its 4:2:0 reading)."""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def alg2_coefficients():
    """Alg. 2's printed coefficients: ({channel: (cY, cCb, cCr)}, offset)."""
    rows = _rows("alg2_ycbcr_to_rgb.txt")
    offset = float(rows[0][1])
    return {r[0]: tuple(float(v) for v in r[1:4]) for r in rows[1:]}, offset


# ---- Alg. 2 ------------------------------------------------------------------

@pytest.fixture(scope="module")
def cube(orc):
    return orc.ycc_to_rgb_all().astype(np.int64)


def test_cc_matches_floating_point_alg2_exhaustively(cube):
    # All 2^24 (Y, Cb, Cr): the 16-bit fixed-point result is within one unit
    # of Alg. 2 evaluated in double precision and rounded (then saturated).
    coef, offset = alg2_coefficients()
    y = np.arange(256, dtype=np.float64)[:, None, None]
    cb = np.arange(256, dtype=np.float64)[None, :, None] - offset
    cr = np.arange(256, dtype=np.float64)[None, None, :] - offset
    ref = [coef[ch][0] * y + coef[ch][1] * cb + coef[ch][2] * cr for ch in "RGB"]
    exact = 0
    for c in range(3):
        r = np.clip(np.floor(np.broadcast_to(ref[c], (256, 256, 256)) + 0.5), 0, 255)
        d = np.abs(cube[..., c] - r)
        assert d.max() <= 1, c
        exact += int(np.count_nonzero(d == 0))
    assert exact / (3 * 2 ** 24) > 0.99


def test_cc_grey_axis_is_identity(cube):
    y = np.arange(256)
    for c in range(3):
        assert np.array_equal(cube[y, 128, 128, c], y)


def test_cc_monotone_and_saturating(cube):
    # R and B increase with Y at fixed chroma; extremes saturate.
    assert np.all(np.diff(cube[:, :, :, 0], axis=0) >= 0)
    assert np.all(np.diff(cube[:, :, :, 2], axis=0) >= 0)
    assert cube[255, 255, 255, 0] == 255 and cube[0, 0, 0, 2] == 0


# ---- Alg. 1 (h2v1) ------------------------------------------------------------

def alg1_as_printed(In):
    """Alg. 1 of the paper for one 8-sample row, evaluated from its printed
    index table (tests/golden/alg1_h2v1_upsampling.txt)."""
    i = [int(v) for v in In]
    out = [None] * 16
    for o, c, nb, bias in _rows("alg1_h2v1_upsampling.txt"):
        o, c = int(o), int(c)
        out[o] = i[c] if nb == "-" else (3 * i[c] + i[int(nb)] + int(bias)) // 4
    assert None not in out
    return out


def test_h2v1_fancy_equals_alg1_on_one_block_row(orc):
    rng = np.random.default_rng(422)
    rows = rng.integers(0, 256, size=(500, 8)).astype(np.uint8)
    rows[0] = [0, 255, 0, 255, 0, 255, 0, 255]
    rows[1] = 255
    out = orc.upsample(rows, 2, 1, True)
    for r in range(rows.shape[0]):
        assert out[r].tolist() == alg1_as_printed(rows[r])


def test_h2v1_fancy_crosses_block_boundaries(orc):
    # Two adjacent blocks: samples at the seam use the true neighbour, not the
    # block's own edge (only the true image edges replicate).
    row = np.array([[10, 20, 30, 40, 50, 60, 70, 80, 200, 190, 180, 170, 160, 150, 140, 130]], np.uint8)
    out = orc.upsample(row, 2, 1, True)[0].astype(int)
    assert out[15] == (3 * 80 + 200 + 2) // 4
    assert out[16] == (3 * 200 + 80 + 1) // 4
    assert out[0] == 10 and out[31] == 130


# ---- invariants shared by all upsamplers --------------------------------------

@pytest.mark.parametrize("sx,sy", [(2, 1), (2, 2), (1, 1), (1, 2)])
@pytest.mark.parametrize("fancy", [False, True])
def test_constant_in_constant_out(orc, sx, sy, fancy):
    for v in (0, 1, 77, 254, 255):
        p = np.full((5, 7), v, np.uint8)
        assert np.all(orc.upsample(p, sx, sy, fancy) == v)


@pytest.mark.parametrize("sx,sy", [(2, 1), (2, 2), (1, 2)])
def test_replicate_is_nearest_neighbour(orc, sx, sy):
    rng = np.random.default_rng(3)
    p = rng.integers(0, 256, size=(9, 13)).astype(np.uint8)
    want = np.repeat(np.repeat(p, sy, axis=0), sx, axis=1)
    assert np.array_equal(orc.upsample(p, sx, sy, False), want)


def test_fancy_linear_ramps_interpolate_exactly(orc):
    # An output sample of factor-2 upsampling sits 1/4 sample from its nearest
    # source sample; on a ramp of slope 4 the 3:1 filter is exact there.
    x = np.arange(12)
    p = np.tile((20 + 4 * x).astype(np.uint8), (6, 1))
    out = orc.upsample(p, 2, 1, True).astype(int)
    xs = np.arange(2, 22)                                   # interior
    assert np.array_equal(out[0, xs], 20 + 4 * ((xs - 0.5) / 2).astype(float) + 0)
    # vertical ramp through h2v2 (interior rows, slope 8 per chroma row)
    y = np.arange(10)
    pv = np.tile((10 + 8 * y).astype(np.uint8)[:, None], (1, 6))
    outv = orc.upsample(pv, 2, 2, True).astype(int)
    ys = np.arange(2, 18)
    expect = 10 + 8 * (ys - 0.5) / 2
    # 4:2:0 uses one rounding (+8 / +7 over 16): exact within 1/2 unit
    assert np.max(np.abs(outv[ys, 5] - expect)) <= 0.5


@pytest.mark.parametrize("sy", [1, 2])
def test_fancy_output_between_its_sources(orc, sy):
    rng = np.random.default_rng(11 + sy)
    p = rng.integers(0, 256, size=(11, 17)).astype(np.int64)
    out = orc.upsample(p.astype(np.uint8), 2, sy, True).astype(np.int64)
    ch, cw = p.shape
    for oy in range(ch * sy):
        j = oy // sy
        rows = {j}
        if sy == 2:
            rows.add(min(max(j + (1 if oy & 1 else -1), 0), ch - 1))
        for ox in range(cw * 2):
            i = ox // 2
            cols = {i, min(max(i + (1 if ox & 1 else -1), 0), cw - 1)}
            src = [p[r, c] for r in rows for c in cols]
            assert min(src) <= out[oy, ox] <= max(src)


def test_h1v2_is_h2v1_transposed(orc):
    # The vertical-only filter is the horizontal one of Alg. 1 turned by 90
    # degrees: upsampling the transpose must give the transposed output.
    rng = np.random.default_rng(13)
    p = rng.integers(0, 256, size=(9, 14)).astype(np.uint8)
    v = orc.upsample(p, 1, 2, True)
    h = orc.upsample(np.ascontiguousarray(p.T), 2, 1, True)
    assert v.shape == (18, 14)
    assert np.array_equal(v, h.T)


def test_h1v2_vertical_ramp_exact(orc):
    # slope 4 per chroma row: each output row sits 1/4 row from its nearest
    # source row, where the 3:1 filter is exact (interior rows)
    y = np.arange(10)
    p = np.tile((20 + 4 * y).astype(np.uint8)[:, None], (1, 5))
    out = orc.upsample(p, 1, 2, True).astype(float)
    ys = np.arange(2, 18)
    assert np.array_equal(out[ys, 3], 20 + 4 * (ys - 0.5) / 2)


def test_h2v2_edges_replicate_true_edge(orc):
    rng = np.random.default_rng(12)
    p = rng.integers(0, 256, size=(3, 5)).astype(np.int64)
    out = orc.upsample(p.astype(np.uint8), 2, 2, True).astype(np.int64)
    # top-left output: near row 0, far row clamped to 0, left column clamped
    s0 = 4 * p[0, 0]
    assert out[0, 0] == (4 * s0 + 8) >> 4
    # bottom-right output: near row ch-1, far row clamped, right col clamped
    s = 4 * p[2, 4]
    assert out[5, 9] == (4 * s + 7) >> 4
