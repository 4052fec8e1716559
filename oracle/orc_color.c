/*
 * orc_color.c -- YCbCr -> RGB of the oracle.  TEST INFRASTRUCTURE ONLY.
 *
 * Sec. 4.3, Alg. 2:  R = Y + 1.402 (Cr-128)
 *                    G = Y - 0.34414 (Cb-128) - 0.71414 (Cr-128)
 *                    B = Y + 1.772 (Cb-128)
 * in 16-bit fixed point: each multiplier is round(c * 2^16); each channel's
 * chroma term is rounded once, (sum + 2^15) >> 16, added to Y and saturated
 * to [0, 255].
 */
#include <math.h>
#include "orc.h"

static int cc_ready = 0;
static int32_t M_CR_R, M_CB_G, M_CR_G, M_CB_B;

static int32_t fix16(double c) { return (int32_t)floor(c * 65536.0 + 0.5); }

static void init_cc(void)
{
    if (cc_ready) return;
    M_CR_R = fix16(1.402);
    M_CB_G = fix16(0.34414);
    M_CR_G = fix16(0.71414);
    M_CB_B = fix16(1.772);
    cc_ready = 1;
}

static uint8_t sat8(int32_t v) { return (uint8_t)(v < 0 ? 0 : (v > 255 ? 255 : v)); }

void orc_ycc_to_rgb(int y, int cb, int cr, uint8_t rgb[3])
{
    init_cc();
    int32_t cbs = cb - 128, crs = cr - 128;
    int32_t dr = (M_CR_R * crs + 32768) >> 16;
    int32_t dg = (-M_CB_G * cbs - M_CR_G * crs + 32768) >> 16;
    int32_t db = (M_CB_B * cbs + 32768) >> 16;
    rgb[0] = sat8(y + dr);
    rgb[1] = sat8(y + dg);
    rgb[2] = sat8(y + db);
}

void orc_ycc_to_rgb_all(uint8_t *rgb)
{
    for (int y = 0; y < 256; y++)
        for (int cb = 0; cb < 256; cb++)
            for (int cr = 0; cr < 256; cr++)
                orc_ycc_to_rgb(y, cb, cr, rgb + (((size_t)y * 256 + cb) * 256 + cr) * 3);
}
