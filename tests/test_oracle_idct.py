"""Pins for the oracle's dequantisation + IDCT (Sec. 4.1, Eq. 1-2), for both
factorisations: the default LLM form and the AAN scaled form (Sec. 2).

Every check here compares the oracle with something other than itself:
the transform evaluated in double precision from its defining cosine sums,
the IEEE 1180-1990 accuracy procedure, the closed form of a DC-only block,
forward-DCT round trips, single-coefficient basis functions, linearity, and
(across the two factorisations) agreement with each other.
"""
import functools
import math

import numpy as np
import pytest


def _basis():
    # D[k, n] = C_k / 2 * cos((2n+1) k pi / 16): the JPEG-normalised 1-D basis,
    # so that f = D^T F D is the 2-D inverse of T.81 A.3.3.
    d = np.zeros((8, 8))
    for k in range(8):
        ck = 1 / math.sqrt(2) if k == 0 else 1.0
        for n in range(8):
            d[k, n] = 0.5 * ck * math.cos((2 * n + 1) * k * math.pi / 16)
    return d


D = _basis()


@pytest.fixture(params=[False, True], ids=["llm", "aan"])
def aan(request):
    return request.param


def ref_idct(F):
    """Double-precision Eq. 1 then Eq. 2 with 1/4 C_u C_v normalisation.
    F[..., v, u] (row = vertical frequency) -> f[..., y, x]."""
    F = np.asarray(F, np.float64).reshape(-1, 8, 8)
    return np.einsum("vy,nvu,ux->nyx", D, F, D).reshape(-1, 64)


def ref_fdct(f):
    f = np.asarray(f, np.float64).reshape(-1, 8, 8)
    return np.einsum("vy,nyx,ux->nvu", D, f, D).reshape(-1, 64)


def test_constants_are_rounded_cosine_products(orc):
    k = orc.idct_constants()
    c = [math.cos(i * math.pi / 16) for i in range(8)]
    r2 = math.sqrt(2)
    real = [r2 * c[6], r2 * (c[2] - c[6]), r2 * (c[2] + c[6]), r2 * c[3],
            r2 * (-c[1] + c[3] + c[5] - c[7]), r2 * (c[1] + c[3] - c[5] + c[7]),
            r2 * (c[1] + c[3] + c[5] - c[7]), r2 * (c[1] + c[3] - c[5] - c[7]),
            r2 * (c[3] - c[7]), r2 * (c[1] + c[3]), r2 * (c[3] + c[5]), r2 * (c[3] - c[5])]
    assert np.all(np.abs(k / 8192.0 - np.array(real)) <= 0.5 / 8192 + 1e-12)


def test_zero_in_zero_out(orc, aan):
    z = np.zeros((4, 64), np.int16)
    assert np.all(orc.idct_core_blocks(z, aan=aan) == 0)
    assert np.all(orc.idct_blocks(z, np.full(64, 255, np.uint16), aan=aan) == 128)


def test_dc_only_closed_form_exhaustive(orc, aan):
    # Only F(0,0) != 0: every sample is clamp(128 + floor((F + 4) / 8)).
    F = np.arange(-32768, 32768, dtype=np.int64)
    coef = np.zeros((F.size, 64), np.int16)
    coef[:, 0] = F.astype(np.int16)
    out = orc.idct_blocks(coef, np.ones(64, np.uint16), aan=aan)
    want = np.clip(128 + np.floor_divide(F + 4, 8), 0, 255).astype(np.uint8)
    assert np.array_equal(out, np.repeat(want[:, None], 64, axis=1))


def test_single_coefficient_basis_functions(orc, aan):
    # A lone coefficient a at (v, u) must reproduce a/4 C_u C_v cos cos to
    # within one unit: catches a wrong sign, index or transposition.
    for a in (1000, -731, 64):
        coef = np.zeros((64, 64), np.int16)
        coef[np.arange(64), np.arange(64)] = a
        got = orc.idct_core_blocks(coef, aan=aan)
        ref = ref_idct(coef)
        assert np.max(np.abs(got - ref)) <= 1.0, a


def test_random_blocks_against_double_precision(orc, aan):
    rng = np.random.default_rng(1180)
    # dequantised range of real streams: coefficients in [-1024, 1023], q in 1..255
    coef = rng.integers(-60, 61, size=(20000, 64)).astype(np.int16)
    q = rng.integers(1, 17, size=64).astype(np.uint16)
    got = orc.idct_core_blocks(coef, q, aan=aan)
    ref = ref_idct(coef.astype(np.float64) * q)
    err = got - ref
    assert np.max(np.abs(err)) <= 1.0
    # the clamped, level-shifted samples follow the same bound
    samp = orc.idct_blocks(coef, q, aan=aan).astype(np.float64)
    assert np.max(np.abs(samp - np.clip(ref + 128, 0, 255))) <= 1.0


def test_dequantisation_is_exact_product(orc, aan):
    # F = coef * Q before the transform: scaling Q by 2 equals doubling coef.
    rng = np.random.default_rng(7)
    coef = rng.integers(-500, 501, size=(500, 64)).astype(np.int16)
    q = rng.integers(1, 128, size=64).astype(np.uint16)
    a = orc.idct_core_blocks(coef, q * 2, aan=aan)
    b = orc.idct_core_blocks((coef.astype(np.int32) * 2).astype(np.int16), q, aan=aan)
    assert np.array_equal(a, b)


def _ieee1180_rand(state, L, H):
    # Uniform integer in [-L, H] from the linear congruential generator of the
    # IEEE 1180-1990 procedure (32-bit arithmetic).
    state = (state * 1103515245 + 12345) & 0xFFFFFFFF
    i = state & 0x7FFFFFFE
    x = i / float(0x7FFFFFFF) * (L + H + 1)
    return state, int(x) - L


@functools.lru_cache(maxsize=None)
def _ieee1180_blocks(L, H, n, seed=1):
    s = seed
    out = np.empty((n, 64), np.int64)
    for b in range(n):
        for k in range(64):
            s, out[b, k] = _ieee1180_rand(s, L, H)
    out.setflags(write=False)
    return out


@pytest.mark.parametrize("L,H", [(256, 255), (5, 5), (300, 300)])
@pytest.mark.parametrize("sign", [1, -1])
def test_ieee1180(orc, L, H, sign, aan):
    n = 10000
    f = _ieee1180_blocks(L, H, n) * sign
    # IEEE 1180 rounds half away from zero
    Fr = ref_fdct(f)
    F = np.clip(np.sign(Fr) * np.floor(np.abs(Fr) + 0.5), -2048, 2047)
    ref = np.clip(np.sign(r := ref_idct(F)) * np.floor(np.abs(r) + 0.5), -256, 255)
    got = np.clip(orc.idct_core_blocks(F.astype(np.int16), aan=aan), -256, 255)
    e = (got - ref).reshape(n, 64)
    assert np.max(np.abs(e)) <= 1                              # peak error
    assert np.max(np.mean(e * e, axis=0)) <= 0.06              # per-pixel MSE
    assert np.mean(e * e) <= 0.02                              # overall MSE
    assert np.max(np.abs(np.mean(e, axis=0))) <= 0.015         # per-pixel mean
    assert abs(np.mean(e)) <= 0.0015                           # overall mean


def test_round_trip(orc, aan):
    rng = np.random.default_rng(31)
    smooth = np.clip(128 + 60 * np.sin(np.arange(64).reshape(8, 8) / 5.0)[None]
                     + rng.normal(0, 3, size=(2000, 8, 8)), 0, 255)
    noisy = rng.integers(0, 256, size=(2000, 8, 8)).astype(np.float64)
    for f in (smooth, noisy):
        f = np.rint(f)
        Fr = ref_fdct(f - 128)
        F = np.sign(Fr) * np.floor(np.abs(Fr) + 0.5)
        got = orc.idct_blocks(F.astype(np.int16), np.ones(64, np.uint16), aan=aan).astype(np.int64)
        err = np.abs(got - f.reshape(-1, 64))
        # error = IDCT of the coefficient rounding (<= 0.5 each, orthonormal
        # transform) plus one fixed-point rounding
        assert np.max(err) <= 2
        assert np.mean(err <= 1) > 0.999


def test_linearity_in_the_exact_domain(orc, aan):
    # The row-pass sums are linear in the input; the rounded output of a sum
    # differs from the sum of rounded outputs by at most the rounding slack.
    rng = np.random.default_rng(5)
    a = rng.integers(-200, 201, size=(3000, 64)).astype(np.int16)
    b = rng.integers(-200, 201, size=(3000, 64)).astype(np.int16)
    ab = orc.idct_core_blocks((a.astype(np.int32) + b).astype(np.int16), aan=aan)
    assert np.max(np.abs(ab - orc.idct_core_blocks(a, aan=aan) - orc.idct_core_blocks(b, aan=aan))) <= 2


# ---- the AAN factorisation only ------------------------------------------------

def test_aan_scale_table_and_constants_follow_their_definitions(orc):
    S, (k1, k2, k3, k4) = orc.idct_aan_constants()
    s = np.array([1.0] + [math.sqrt(2) * math.cos(k * math.pi / 16) for k in range(1, 8)])
    exact = 4096.0 * np.outer(s, s)
    assert np.array_equal(S, np.floor(exact + 0.5).astype(np.int32))
    # no entry sits near a rounding boundary, so any evaluation order of the
    # product gives the same table
    assert np.min(np.abs(exact - np.floor(exact) - 0.5)) > 1e-3
    assert S[0, 0] == 4096
    c, sn = math.cos(math.pi / 8), math.sin(math.pi / 8)
    for k, real in ((k1, math.sqrt(2) - 1), (k2, 2 - 2 * c), (k3, 3 - 2 * c - 2 * sn), (k4, 2 * c - 2 * sn - 1)):
        assert abs(k / 2.0 ** 32 - real) <= 0.5 / 2.0 ** 32 + 1e-15


def test_aan_and_llm_agree_on_realistic_blocks(orc):
    # Two independent factorisations of the same transform, both within the
    # IEEE 1180 bounds: on quantised blocks of real-looking content their
    # samples differ by at most one level and rarely at all.
    from paper_1311_5304_gb300 import synth
    img = synth.make_image(512, 512, "444", 75, seed=9, kind="texture", sigma=4.0)
    for c in range(3):
        coef = img.planes[c].reshape(-1, 64)
        a = orc.idct_blocks(coef, img.qtabs[c]).astype(np.int64)
        b = orc.idct_blocks(coef, img.qtabs[c], aan=True).astype(np.int64)
        d = np.abs(a - b)
        assert d.max() <= 1
        assert np.mean(d == 0) > 0.97


@pytest.mark.parametrize("aan", [False, True])
def test_level_shift_inside_the_rounding_constant_is_shift_then_add(orc, aan):
    # The oracle adds the level shift as 128 * 2^18 (AAN: 128 * 2^15) inside
    # the row pass's rounding constant.  floor((P + r + 128 * 2^n) / 2^n) is
    # floor((P + r) / 2^n) + 128 whenever the int32 sum does not wrap, so on
    # every block of real-data range the samples equal the Eq. 2 output
    # (idct_core, no level shift) plus 128, then clamped.  They differ only
    # for adversarial inputs whose sum lies within 2^25 (AAN: 2^22) of the
    # int32 limit, where both sides of the GPU comparison wrap identically.
    rng = np.random.default_rng(1805)
    # dequantised values within the range of 8-bit samples' DCT (|F| < 2^13)
    q = rng.integers(1, 40, size=64).astype(np.uint16)
    coef = np.round(rng.laplace(0, 400, size=(4000, 64)) / q).astype(np.int64)
    coef = np.clip(coef, -(8000 // q.astype(np.int64)), 8000 // q.astype(np.int64)).astype(np.int16)
    core = orc.idct_core_blocks(coef, q, aan=aan).astype(np.int64)
    want = np.clip(core + 128, 0, 255)
    got = orc.idct_blocks(coef, q, aan=aan).astype(np.int64)
    assert np.array_equal(got, want)
    assert np.count_nonzero(want == 0) > 0 and np.count_nonzero(want == 255) > 0
