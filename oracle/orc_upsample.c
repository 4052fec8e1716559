/*
 * orc_upsample.c -- chroma upsampling of the oracle.  TEST INFRASTRUCTURE ONLY.
 *
 * Sec. 4.2, Alg. 1 (4:2:2, horizontal factor 2, "triangular" weights 3:1):
 *   Out[2i]   = (3 In[i] + In[i-1] + 1) / 4
 *   Out[2i+1] = (3 In[i] + In[i+1] + 2) / 4
 *   Out[0] = In[0], Out[last] = In[last]
 * Alg. 1 prints this for one 8-sample block row; neighbours across block and
 * MCU boundaries are the true neighbouring samples and only the component's
 * true image edges are replicated (reading of Sec. 4.2, where all but the end
 * pixels depend on neighbouring samples).  With the index clamped to
 * [0, cw-1] the edge formulas are the interior formulas: (4a+1)/4 = a and
 * (4a+2)/4 = a for 0 <= a <= 255.
 *
 * Vertical factor 2 (4:2:0) is not printed in the paper ("other subsamplings
 * are handled in a similar manner"); the reading used is the separable 3:1
 * triangular filter with a single rounding:
 *   S[i]      = 3 C[i][near] + C[i][far]      (near = j, far = j-1 for
 *                                              output row 2j, j+1 for 2j+1;
 *                                              far clamped to [0, ch-1])
 *   Out[2i]   = (3 S[i] + S[i-1] + 8) >> 4
 *   Out[2i+1] = (3 S[i] + S[i+1] + 7) >> 4   (S index clamped to [0, cw-1])
 * Vertical factor 2 alone (h1v2, 4:4:0; not in the paper either): Alg. 1
 * turned vertical, the same weights and alternating biases:
 *   Out[x][2j]   = (3 C[x][j] + C[x][j-1] + 1) >> 2
 *   Out[x][2j+1] = (3 C[x][j] + C[x][j+1] + 2) >> 2   (row index clamped to
 *                                                     [0, ch-1])
 * Replication: Out(x, y) = C[x / sx][y / sy].
 */
#include "orc.h"

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Output rows [oy0, oy1) of the upsampled plane. */
void orc_upsample_rows(const uint8_t *in, int cw, int ch, int64_t in_pitch,
                       int sx, int sy, int fancy, uint8_t *out, int64_t out_pitch,
                       int oy0, int oy1)
{
    const int ow = cw * sx;
    for (int oy = oy0; oy < oy1; oy++) {
        for (int ox = 0; ox < ow; ox++) {
            int v;
            if (!fancy || (sx == 1 && sy == 1)) {
                v = in[(int64_t)(oy / sy) * in_pitch + ox / sx];
            } else if (sy == 1) {
                /* h2v1, Alg. 1 */
                const uint8_t *row = in + (int64_t)oy * in_pitch;
                int i = ox >> 1;
                int c = row[i];
                if ((ox & 1) == 0) v = (3 * c + row[clampi(i - 1, 0, cw - 1)] + 1) >> 2;
                else               v = (3 * c + row[clampi(i + 1, 0, cw - 1)] + 2) >> 2;
            } else if (sx == 2) {
                /* h2v2: vertical 3:1 sums, then horizontal 3:1 with one rounding */
                int j = oy >> 1;
                int far = (oy & 1) ? clampi(j + 1, 0, ch - 1) : clampi(j - 1, 0, ch - 1);
                const uint8_t *rn = in + (int64_t)j * in_pitch;
                const uint8_t *rf = in + (int64_t)far * in_pitch;
                int i = ox >> 1;
                int s  = 3 * rn[i] + rf[i];
                if ((ox & 1) == 0) {
                    int il = clampi(i - 1, 0, cw - 1);
                    int sl = 3 * rn[il] + rf[il];
                    v = (3 * s + sl + 8) >> 4;
                } else {
                    int ir = clampi(i + 1, 0, cw - 1);
                    int sr = 3 * rn[ir] + rf[ir];
                    v = (3 * s + sr + 7) >> 4;
                }
            } else {
                /* h1v2: Alg. 1 along columns */
                int j = oy >> 1;
                int c = in[(int64_t)j * in_pitch + ox];
                if ((oy & 1) == 0) v = (3 * c + in[(int64_t)clampi(j - 1, 0, ch - 1) * in_pitch + ox] + 1) >> 2;
                else               v = (3 * c + in[(int64_t)clampi(j + 1, 0, ch - 1) * in_pitch + ox] + 2) >> 2;
            }
            out[(int64_t)oy * out_pitch + ox] = (uint8_t)v;
        }
    }
}

void orc_upsample(const uint8_t *in, int cw, int ch, int64_t in_pitch,
                  int sx, int sy, int fancy, uint8_t *out, int64_t out_pitch)
{
    orc_upsample_rows(in, cw, ch, in_pitch, sx, sy, fancy, out, out_pitch, 0, ch * sy);
}
