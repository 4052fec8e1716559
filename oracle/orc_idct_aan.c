/*
 * orc_idct_aan.c -- the Arai-Agui-Nakajima (AAN) scaled 8x8 IDCT of the
 * oracle, the algorithm the decoder of Sec. 2 is based on.
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 *
 * What is computed: the same 2-D transform as orc_idct.c (Eq. 1 column pass,
 * then Eq. 2 row pass, JPEG normalisation: f = 1/8 of the double sum of the
 * 1-D transforms y[n] = X0 + sqrt(2) sum_{k>0} X_k cos((2n+1)k pi/16)), by a
 * different factorisation and fixed point.
 *
 * Scaled inputs.  Writing s_0 = 1, s_k = sqrt(2) cos(k pi/16) (k = 1..7) and
 * w_k = s_k X_k, the 1-D transform needs only five multiplications by
 * constants (derived from the even/odd split, with c = cos(pi/8),
 * s = sin(pi/8)):
 *   even half (e[n] = sum over even k):
 *     P = w2 + w6,  q = sqrt2 (w2 - w6) - P
 *     e0 = w0 + w4 + P,  e3 = w0 + w4 - P,  e1 = w0 - w4 + q,  e2 = w0 - w4 - q
 *   odd half (o[n] = sum over odd k):
 *     a = w5 + w3,  b = w5 - w3,  cc = w1 + w7,  d = w1 - w7
 *     o0 = a + cc
 *     z  = 2c (b + d)
 *     o1 = z - (2c + 2s) b - o0
 *     o2 = sqrt2 (cc - a) - o1
 *     o3 = z - (2c - 2s) d - o2
 *   y[n] = e[n] + o[n],  y[7-n] = e[n] - o[n].
 * In 2-D the column pass takes w(v,u) = s_v s_u F(v,u); its outputs are the
 * column-pass values scaled by s_u, which is exactly the scaled input the row
 * pass needs, so all 64 scale factors fold into the dequantisation table.
 *
 * Fixed point (this implementation's choice; the paper gives none):
 *   prescaled table  QS(v,u) = Q(v,u) * S(v,u),  S(v,u) = round(2^12 s_v s_u)
 *                    (so the working values carry 12 fractional bits)
 *   dequantisation   w = coef * QS                       (int32, wraps)
 *   products         hi(t, K) = floor(t K / 2^32), t and K int32, and
 *     P1(t) = t  + hi(t,  K1)   ~ sqrt2 t,          K1 = round((sqrt2 - 1) 2^32)
 *     P2(t) = 2t + hi(t, -K2)   ~ 2c t,             K2 = round((2 - 2c) 2^32)
 *     P3(t) = 3t - hi(t,  K3)   ~ (2c + 2s) t,      K3 = round((3 - 2c - 2s) 2^32)
 *     P4(t) = t  - hi(t, -K4)   ~ (2c - 2s) t,      K4 = round((2c - 2s - 1) 2^32)
 *   both passes use the flowgraph above with these products and no
 *   intermediate descale; the 2-D value Y is f * 2^15 (12 fractional bits and
 *   the 1/8).  The sample adds the rounding and the level shift in one
 *   constant, as orc_idct.c does: clamp((Y + 2^14 + 128 * 2^15) >> 15, 0, 255)
 *   (the same as ((Y + 2^14) >> 15) + 128 unless the sum wraps).
 * Every intermediate is int32 with two's-complement wrap (-fwrapv); hi() takes
 * the high word of the exact 64-bit product.
 */
#include <math.h>
#include "orc.h"

#define AAN_BITS 12          /* fractional bits of the working values */
#define AAN_SHIFT (AAN_BITS + 3)

static int32_t S[64];        /* round(2^12 s_v s_u), [v*8 + u] */
static int32_t K1, K2, K3, K4;
static int aan_ready = 0;

static int32_t round_i32(double x) { return (int32_t)floor(x + 0.5); }

static void init_aan(void)
{
    if (aan_ready) return;
    const double pi = 3.14159265358979323846;
    double s[8];
    s[0] = 1.0;
    for (int k = 1; k < 8; k++) s[k] = sqrt(2.0) * cos(k * pi / 16.0);
    for (int v = 0; v < 8; v++)
        for (int u = 0; u < 8; u++) S[v * 8 + u] = round_i32(s[v] * s[u] * (double)(1 << AAN_BITS));
    const double c = cos(pi / 8.0), sn = sin(pi / 8.0), two32 = 4294967296.0;
    K1 = round_i32((sqrt(2.0) - 1.0) * two32);
    K2 = round_i32((2.0 - 2.0 * c) * two32);
    K3 = round_i32((3.0 - 2.0 * c - 2.0 * sn) * two32);
    K4 = round_i32((2.0 * c - 2.0 * sn - 1.0) * two32);
    aan_ready = 1;
}

static int32_t hi(int32_t t, int32_t k) { return (int32_t)(((int64_t)t * (int64_t)k) >> 32); }
static int32_t P1(int32_t t) { return t + hi(t, K1); }
static int32_t P2(int32_t t) { return 2 * t + hi(t, -K2); }
static int32_t P3(int32_t t) { return 3 * t - hi(t, K3); }
static int32_t P4(int32_t t) { return t - hi(t, -K4); }

void orc_idct_aan_constants(int32_t scale[64], int32_t k[4])
{
    init_aan();
    for (int i = 0; i < 64; i++) scale[i] = S[i];
    k[0] = K1; k[1] = K2; k[2] = K3; k[3] = K4;
}

/* One 8-point transform of scaled inputs w[0..7] into y[0..7]. */
static void aan8(const int32_t w[8], int32_t y[8])
{
    /* even half */
    const int32_t P = w[2] + w[6];
    const int32_t q = P1(w[2] - w[6]) - P;
    const int32_t e0 = w[0] + w[4] + P, e3 = w[0] + w[4] - P;
    const int32_t e1 = w[0] - w[4] + q, e2 = w[0] - w[4] - q;
    /* odd half */
    const int32_t a = w[5] + w[3], b = w[5] - w[3];
    const int32_t cc = w[1] + w[7], d = w[1] - w[7];
    const int32_t o0 = a + cc;
    const int32_t z = P2(b + d);
    const int32_t o1 = z - P3(b) - o0;
    const int32_t o2 = P1(cc - a) - o1;
    const int32_t o3 = z - P4(d) - o2;
    y[0] = e0 + o0; y[7] = e0 - o0;
    y[1] = e1 + o1; y[6] = e1 - o1;
    y[2] = e2 + o2; y[5] = e2 - o2;
    y[3] = e3 + o3; y[4] = e3 - o3;
}

/* Dequantisation with the prescaled table and both passes: Y = f * 2^15. */
static void aan2d(const int16_t coef[64], const uint16_t q[64], int32_t Y[64])
{
    int32_t w[64], t[64], x[8], y[8];
    init_aan();
    for (int k = 0; k < 64; k++) w[k] = (int32_t)coef[k] * ((int32_t)q[k] * S[k]);
    /* Eq. 1, column pass: for each horizontal frequency u, transform over v */
    for (int u = 0; u < 8; u++) {
        for (int v = 0; v < 8; v++) x[v] = w[v * 8 + u];
        aan8(x, y);
        for (int r = 0; r < 8; r++) t[r * 8 + u] = y[r];
    }
    /* Eq. 2, row pass: for each spatial row, transform over u */
    for (int r = 0; r < 8; r++) {
        aan8(t + 8 * r, y);
        for (int xx = 0; xx < 8; xx++) Y[r * 8 + xx] = y[xx];
    }
}

void orc_idct_aan_block(const int16_t coef[64], const uint16_t q[64], uint8_t out[64])
{
    int32_t Y[64];
    aan2d(coef, q, Y);
    for (int i = 0; i < 64; i++) {
        const int32_t s = (Y[i] + (1 << (AAN_SHIFT - 1)) + (128 << AAN_SHIFT)) >> AAN_SHIFT;
        out[i] = (uint8_t)(s < 0 ? 0 : (s > 255 ? 255 : s));
    }
}

void orc_idct_aan_core(const int16_t coef[64], const uint16_t q[64], int32_t out[64])
{
    int32_t Y[64];
    aan2d(coef, q, Y);
    for (int i = 0; i < 64; i++) out[i] = (Y[i] + (1 << (AAN_SHIFT - 1))) >> AAN_SHIFT;
}

void orc_idct_aan_blocks(const int16_t *coef, const uint16_t q[64], uint8_t *out, int64_t n)
{
    for (int64_t b = 0; b < n; b++) orc_idct_aan_block(coef + 64 * b, q, out + 64 * b);
}

void orc_idct_aan_core_blocks(const int16_t *coef, const uint16_t q[64], int32_t *out, int64_t n)
{
    for (int64_t b = 0; b < n; b++) orc_idct_aan_core(coef + 64 * b, q, out + 64 * b);
}
