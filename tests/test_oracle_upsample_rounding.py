"""Pins for the rounding of the oracle's triangular upsampling, from the
sample geometry rather than from the filter formulas.

Alg. 1 (Sec. 4.2) weights a chroma sample 3:1 against its neighbour: that is
linear interpolation at a quarter-sample offset, i.e. chroma samples centred
between the two luma samples they cover.  Here every output sample's position
is worked out in chroma coordinates, ``(ox + 1/2) / s - 1/2``, and its exact
value is the (bi)linear interpolation of the source plane there, with indices
clamped at the true image edges (Fractions, no filter constants).  The oracle's
integer output must then be the exact value rounded to nearest, and an exact
tie must be broken the way the readings state:

* h2v1 and h1v2 (Alg. 1 as printed, +1 / +2 before the divide by 4): even
  outputs round ties down, odd outputs round them up;
* h2v2 (the 4:2:0 reading, +8 / +7 before the divide by 16): even output
  columns round ties up, odd columns round them down.

A mistake in the 4:2:0 branch that the constant, ramp and between-the-sources
pins let through (the biases +8 / +8, the two biases swapped, the far row or
the horizontal neighbour taken on the wrong side) fails here: each is planted
in a copy of the oracle's source, compiled on the CPU, and must be caught.
"""
import ctypes
import os
import re
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ORACLE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")


def _axis_weights(n_src, factor):
    """Per output index along one axis: (i0, i1, w0, w1) with weights in units
    of 1/(2*factor), the linear interpolation at the centred position."""
    rows = []
    for o in range(n_src * factor):
        pos = Fraction(2 * o + 1, 2 * factor) - Fraction(1, 2)
        i0 = pos.numerator // pos.denominator           # floor
        f = pos - i0
        w1 = f * 2 * factor
        assert w1.denominator == 1
        w1 = int(w1)
        cl = lambda v: min(max(v, 0), n_src - 1)
        rows.append((cl(i0), cl(i0 + 1), 2 * factor - w1, w1))
    return rows


def exact_scaled(plane, sx, sy):
    """Exact interpolated value of every output sample, times the common
    denominator (2 sx)(2 sy) (an integer array), and that denominator."""
    p = plane.astype(np.int64)
    ch, cw = p.shape
    wx = _axis_weights(cw, sx) if sx > 1 else [(i, i, 1, 0) for i in range(cw)]
    wy = _axis_weights(ch, sy) if sy > 1 else [(j, j, 1, 0) for j in range(ch)]
    dx = 2 * sx if sx > 1 else 1
    dy = 2 * sy if sy > 1 else 1
    xi0, xi1, xw0, xw1 = (np.array(c) for c in zip(*wx))
    yi0, yi1, yw0, yw1 = (np.array(c) for c in zip(*wy))
    acc = np.zeros((len(wy), len(wx)), np.int64)
    for yi, yw in ((yi0, yw0), (yi1, yw1)):
        for xi, xw in ((xi0, xw0), (xi1, xw1)):
            acc += yw[:, None] * xw[None, :] * p[yi[:, None], xi[None, :]]
    return acc, dx * dy


def rounding_violations(plane, out, sx, sy):
    """Checks `out` (the upsampled plane) against the exact interpolation:
    returns a list of failures (empty when every sample is the exact value
    rounded to nearest with the tie rule of its sampling), and the number of
    ties met in even and odd positions."""
    num, den = exact_scaled(plane, sx, sy)
    got = out.astype(np.int64) * den
    err = got - num
    bad = []
    if np.any(np.abs(err) * 2 > den):
        bad.append(f"{int(np.count_nonzero(np.abs(err) * 2 > den))} outputs farther than 1/2 from the exact value")
    tie = (num % den) * 2 == den
    # position parity that decides the tie: the column for horizontal
    # filters, the row for the vertical-only one
    if sx > 1:
        even = (np.arange(out.shape[1]) % 2 == 0)[None, :].repeat(out.shape[0], 0)
    else:
        even = (np.arange(out.shape[0]) % 2 == 0)[:, None].repeat(out.shape[1], 1)
    up = err * 2 == den
    down = err * 2 == -den
    if sy > 1 and sx > 1:
        want_up, want_down = even, ~even          # +8 even, +7 odd
    else:
        want_up, want_down = ~even, even          # Alg. 1: +1 even, +2 odd
    if np.any(tie & want_up & ~up) or np.any(tie & want_down & ~down):
        bad.append("ties broken against the rule: "
                   f"{int(np.count_nonzero(tie & want_up & ~up))} should round up, "
                   f"{int(np.count_nonzero(tie & want_down & ~down))} should round down")
    return bad, int(np.count_nonzero(tie & even)), int(np.count_nonzero(tie & ~even))


def _planes():
    rng = np.random.default_rng(1311)
    out = [rng.integers(0, 256, size=(23, 37)).astype(np.uint8),
           rng.integers(0, 256, size=(1, 1)).astype(np.uint8),
           rng.integers(0, 256, size=(2, 3)).astype(np.uint8),
           rng.integers(0, 256, size=(9, 1)).astype(np.uint8)]
    # narrow value ranges make ties frequent
    out.append(rng.integers(100, 104, size=(17, 19)).astype(np.uint8))
    out.append((rng.integers(0, 2, size=(13, 29)) * 255).astype(np.uint8))
    return out


@pytest.mark.parametrize("sx,sy", [(2, 2), (2, 1), (1, 2)])
def test_triangular_rounds_exact_interpolation_with_its_tie_rule(orc, sx, sy):
    ties_even = ties_odd = 0
    for p in _planes():
        out = orc.upsample(p, sx, sy, True)
        bad, te, to = rounding_violations(p, out, sx, sy)
        assert not bad, (p.shape, bad)
        ties_even += te
        ties_odd += to
    # the check has power: ties occur in both parities
    assert ties_even > 50 and ties_odd > 50


def test_tie_counts_follow_the_rule(orc):
    # On a plane with many ties the counts of each direction equal the counts
    # of ties in even and odd output columns (4:2:0: up in even, down in odd).
    rng = np.random.default_rng(7)
    p = rng.integers(0, 4, size=(40, 40)).astype(np.uint8) * 4 + 120
    out = orc.upsample(p, 2, 2, True)
    num, den = exact_scaled(p, 2, 2)
    err = out.astype(np.int64) * den - num
    tie = (num % den) * 2 == den
    even = (np.arange(out.shape[1]) % 2 == 0)[None, :]
    assert np.count_nonzero(tie & (err > 0)) == np.count_nonzero(tie & even)
    assert np.count_nonzero(tie & (err < 0)) == np.count_nonzero(tie & ~even)
    assert np.count_nonzero(tie & (err == 0)) == 0


# ---- planted mistakes (in a copy of the oracle, on the CPU) ------------------

PLANTS = {
    "biases +8/+8": [(r"v = \(3 \* s \+ sr \+ 7\) >> 4", "v = (3 * s + sr + 8) >> 4")],
    "biases swapped": [(r"v = \(3 \* s \+ sl \+ 8\) >> 4", "v = (3 * s + sl + 7) >> 4"),
                       (r"v = \(3 \* s \+ sr \+ 7\) >> 4", "v = (3 * s + sr + 8) >> 4")],
    "far row on the wrong side": [(r"\(oy & 1\) \? clampi\(j \+ 1, 0, ch - 1\) : clampi\(j - 1, 0, ch - 1\)",
                                   "(oy & 1) ? clampi(j - 1, 0, ch - 1) : clampi(j + 1, 0, ch - 1)")],
    "left neighbour on the wrong side": [(r"int il = clampi\(i - 1, 0, cw - 1\);",
                                          "int il = clampi(i + 1, 0, cw - 1);")],
}


def _planted_upsampler(tmp_path, name, subs):
    src = open(os.path.join(ORACLE, "orc_upsample.c")).read()
    for pat, rep in subs:
        src, n = re.subn(pat, rep, src)
        assert n == 1, (name, pat)
    c = tmp_path / "orc_upsample_planted.c"
    c.write_text(src)
    so = tmp_path / "liborc_planted.so"
    subprocess.run(["gcc", "-std=c11", "-O1", "-fwrapv", "-fPIC", "-shared", "-I", ORACLE, "-o", str(so), str(c)],
                   check=True)
    lib = ctypes.CDLL(str(so))
    P = ctypes.c_void_p
    lib.orc_upsample.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_int, P, ctypes.c_int64]

    def up(plane, sx, sy):
        plane = np.ascontiguousarray(plane, np.uint8)
        ch, cw = plane.shape
        out = np.zeros((ch * sy, cw * sx), np.uint8)
        lib.orc_upsample(plane.ctypes.data, cw, ch, cw, sx, sy, 1, out.ctypes.data, cw * sx)
        return out
    return up


@pytest.mark.parametrize("name", sorted(PLANTS))
def test_planted_h2v2_mistakes_are_caught(tmp_path, name):
    up = _planted_upsampler(tmp_path, name.replace(" ", "_"), PLANTS[name])
    caught = False
    for p in _planes():
        bad, _, _ = rounding_violations(p, up(p, 2, 2), 2, 2)
        caught |= bool(bad)
    assert caught, name
