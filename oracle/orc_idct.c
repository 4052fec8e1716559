/*
 * orc_idct.c -- dequantisation and the 8x8 fixed-point IDCT of the oracle.
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 *
 * What is computed (Sec. 4.1, Eq. 1 and Eq. 2):
 *   column pass  f(u,y) = sum_v C_v F(u,v) cos((2y+1) v pi / 16)     (Eq. 1)
 *   row pass     f(x,y) = sum_u C_u f(u,y) cos((2x+1) u pi / 16)     (Eq. 2)
 * with the JPEG normalisation that Eq. 1-2 leave out: the 2-D result is
 * 1/4 of the double sum with C_0 = 1/sqrt(2), i.e. 1/8 of the double sum of
 * the 1-D transforms y[n] = X0 + sqrt(2) * sum_{k>0} X_k cos((2n+1)k pi/16).
 *
 * Fixed point: multipliers are round(k * 2^13) (13 fractional bits).  The
 * column pass keeps 2 fractional bits: out = (P + 2^10) >> 11.  The row pass
 * removes them and the 1/8: out = (P + 2^17) >> 18; the level shift +128 is
 * added as 128 * 2^18 inside the same rounding constant, then the sample is
 * saturated to [0, 255] (range-limit clamp).
 *
 * The 1-D transform is evaluated with the Loeffler-Ligtenberg-Moschytz even/odd
 * decomposition: the even half is a 4-point transform of X0, X2, X4, X6 (a
 * butterfly on X0 +- X4 plus one 3-multiply rotation on X2, X6); the odd half
 * computes the four sums o_n = sqrt(2) sum_{k odd} X_k cos((2n+1)k pi/16) with
 * 12 multipliers; outputs are y[n] = e[n] + o[n], y[7-n] = e[n] - o[n].
 * Every quantity is an integer linear form in the inputs, so any exact
 * re-association of the same products gives bit-identical results.
 */
#include <math.h>
#include "orc.h"

#define CONST_BITS 13
#define PASS1_BITS 2

/* Multipliers, indices into K[]: */
enum {
    K_R6 = 0,     /* sqrt2*c6             rotation, both outputs */
    K_R2M6,       /* sqrt2*(c2-c6)        rotation, X2 term      */
    K_R2P6,       /* sqrt2*(c2+c6)        rotation, X6 term      */
    K_S3,         /* sqrt2*c3             shared odd term        */
    K_X7,         /* sqrt2*(-c1+c3+c5-c7)                        */
    K_X5,         /* sqrt2*( c1+c3-c5+c7)                        */
    K_X3,         /* sqrt2*( c1+c3+c5-c7)                        */
    K_X1,         /* sqrt2*( c1+c3-c5-c7)                        */
    K_P71,        /* sqrt2*(c3-c7)        pair X7+X1, negated    */
    K_P53,        /* sqrt2*(c1+c3)        pair X5+X3, negated    */
    K_P73,        /* sqrt2*(c3+c5)        pair X7+X3, negated    */
    K_P51         /* sqrt2*(c3-c5)        pair X5+X1, negated    */
};

static int32_t K[12];
static int k_ready = 0;

static int32_t fix13(double k) { return (int32_t)floor(k * (double)(1 << CONST_BITS) + 0.5); }

static void init_constants(void)
{
    if (k_ready) return;
    const double pi = 3.14159265358979323846;
    double c[8];
    for (int k = 0; k < 8; k++) c[k] = cos(k * pi / 16.0);
    const double r2 = sqrt(2.0);
    K[K_R6]   = fix13(r2 * c[6]);
    K[K_R2M6] = fix13(r2 * (c[2] - c[6]));
    K[K_R2P6] = fix13(r2 * (c[2] + c[6]));
    K[K_S3]   = fix13(r2 * c[3]);
    K[K_X7]   = fix13(r2 * (-c[1] + c[3] + c[5] - c[7]));
    K[K_X5]   = fix13(r2 * ( c[1] + c[3] - c[5] + c[7]));
    K[K_X3]   = fix13(r2 * ( c[1] + c[3] + c[5] - c[7]));
    K[K_X1]   = fix13(r2 * ( c[1] + c[3] - c[5] - c[7]));
    K[K_P71]  = fix13(r2 * (c[3] - c[7]));
    K[K_P53]  = fix13(r2 * (c[1] + c[3]));
    K[K_P73]  = fix13(r2 * (c[3] + c[5]));
    K[K_P51]  = fix13(r2 * (c[3] - c[5]));
    k_ready = 1;
}

void orc_idct_constants(int32_t k[12])
{
    init_constants();
    for (int i = 0; i < 12; i++) k[i] = K[i];
}

/*
 * One 8-point transform.  x[0..7] are the inputs X_0..X_7 (frequency order),
 * p[0..7] receive the undescaled outputs y[0..7] scaled by 2^13 relative to
 * the inputs.  Arithmetic wraps mod 2^32 (-fwrapv).
 */
static void idct8(const int32_t x[8], int32_t p[8])
{
    /* even half: 4-point transform of X0, X2, X4, X6 */
    int32_t a0 = (x[0] + x[4]) * (1 << CONST_BITS);     /* n = 0, 3 */
    int32_t a1 = (x[0] - x[4]) * (1 << CONST_BITS);     /* n = 1, 2 */
    int32_t r  = (x[2] + x[6]) * K[K_R6];
    int32_t b0 = r + x[2] * K[K_R2M6];                  /* sqrt2(c2 X2 + c6 X6) */
    int32_t b1 = r - x[6] * K[K_R2P6];                  /* sqrt2(c6 X2 - c2 X6) */
    int32_t e0 = a0 + b0, e3 = a0 - b0;
    int32_t e1 = a1 + b1, e2 = a1 - b1;

    /* odd half: o_n for n = 0..3 */
    int32_t s71 = x[7] + x[1], s53 = x[5] + x[3];
    int32_t s73 = x[7] + x[3], s51 = x[5] + x[1];
    int32_t sh  = (s73 + s51) * K[K_S3];
    int32_t t7 = x[7] * K[K_X7], t5 = x[5] * K[K_X5];
    int32_t t3 = x[3] * K[K_X3], t1 = x[1] * K[K_X1];
    int32_t m71 = -s71 * K[K_P71], m53 = -s53 * K[K_P53];
    int32_t m73 = -s73 * K[K_P73] + sh, m51 = -s51 * K[K_P51] + sh;
    int32_t o3 = t7 + m71 + m73;       /* sqrt2( c7X1 - c5X3 + c3X5 - c1X7) */
    int32_t o2 = t5 + m53 + m51;       /* sqrt2( c5X1 - c1X3 + c7X5 + c3X7) */
    int32_t o1 = t3 + m53 + m73;       /* sqrt2( c3X1 - c7X3 - c1X5 - c5X7) */
    int32_t o0 = t1 + m71 + m51;       /* sqrt2( c1X1 + c3X3 + c5X5 + c7X7) */

    p[0] = e0 + o0; p[7] = e0 - o0;
    p[1] = e1 + o1; p[6] = e1 - o1;
    p[2] = e2 + o2; p[5] = e2 - o2;
    p[3] = e3 + o3; p[4] = e3 - o3;
}

/* Dequantisation and both passes; ws receives the row-pass sums P. */
static void idct2d_sums(const int16_t coef[64], const uint16_t q[64], int32_t ps[64])
{
    int32_t f[64], ws[64], x[8], p[8];
    init_constants();
    /* dequantisation: F(u,v) = coef * Q, int32 (Sec. 2, Sec. 4.1) */
    for (int k = 0; k < 64; k++) f[k] = (int32_t)coef[k] * (int32_t)q[k];
    /* Eq. 1, column pass: for each horizontal frequency u, transform over v */
    for (int u = 0; u < 8; u++) {
        for (int v = 0; v < 8; v++) x[v] = f[v * 8 + u];
        idct8(x, p);
        for (int y = 0; y < 8; y++)
            ws[y * 8 + u] = (p[y] + (1 << (CONST_BITS - PASS1_BITS - 1))) >> (CONST_BITS - PASS1_BITS);
    }
    /* Eq. 2, row pass: for each spatial row y, transform over u */
    for (int y = 0; y < 8; y++) {
        for (int u = 0; u < 8; u++) x[u] = ws[y * 8 + u];
        idct8(x, p);
        for (int xx = 0; xx < 8; xx++) ps[y * 8 + xx] = p[xx];
    }
}

#define SHIFT2 (CONST_BITS + PASS1_BITS + 3)

void orc_idct_block(const int16_t coef[64], const uint16_t q[64], uint8_t out[64])
{
    int32_t ps[64];
    idct2d_sums(coef, q, ps);
    for (int i = 0; i < 64; i++) {
        /* rounding and level shift in one constant, then range-limit clamp */
        int32_t s = (ps[i] + (1 << (SHIFT2 - 1)) + (128 << SHIFT2)) >> SHIFT2;
        out[i] = (uint8_t)(s < 0 ? 0 : (s > 255 ? 255 : s));
    }
}

void orc_idct_core(const int16_t coef[64], const uint16_t q[64], int32_t out[64])
{
    int32_t ps[64];
    idct2d_sums(coef, q, ps);
    for (int i = 0; i < 64; i++) out[i] = (ps[i] + (1 << (SHIFT2 - 1))) >> SHIFT2;
}

void orc_idct_blocks(const int16_t *coef, const uint16_t q[64], uint8_t *out, int64_t n)
{
    for (int64_t b = 0; b < n; b++) orc_idct_block(coef + 64 * b, q, out + 64 * b);
}

void orc_idct_core_blocks(const int16_t *coef, const uint16_t q[64], int32_t *out, int64_t n)
{
    for (int64_t b = 0; b < n; b++) orc_idct_core(coef + 64 * b, q, out + 64 * b);
}
