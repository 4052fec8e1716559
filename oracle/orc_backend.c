/*
 * orc_backend.c -- the whole data-parallel back-end of the oracle: for each
 * component dequantise + IDCT every block of the padded MCU grid into a sample
 * plane, upsample each chroma plane from its true size, convert every pixel
 * of the W x H image to RGB (Fig. 1 after entropy decoding; Sec. 4).
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 *
 * Geometry (ITU-T T.81 A.1.1; the paper is silent): Hmax, Vmax are the largest
 * sampling factors; the MCU is 8*Hmax x 8*Vmax pixels (Sec. 2: 8x8 for 4:4:4,
 * 16x8 for 4:2:2); component c holds (MCUs_x*h_c) x (MCUs_y*v_c) blocks; its
 * true size is ceil(W*h_c/Hmax) x ceil(H*v_c/Vmax).  Samples of padding blocks
 * are computed but never used past the true edge; only W x H pixels are
 * written (Sec. 4.3: raster output, one image width between vertical
 * neighbours).
 */
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include "orc.h"

void orc_upsample_rows(const uint8_t *in, int cw, int ch, int64_t in_pitch,
                       int sx, int sy, int fancy, uint8_t *out, int64_t out_pitch,
                       int oy0, int oy1);

typedef struct {
    const orc_image *img;
    int hmax, vmax;
    int cw[3], ch[3], sx[3], sy[3];
    uint8_t *plane[3];   int64_t ppitch[3];   /* IDCT output, padded grid */
    uint8_t *up[3];      int64_t upitch[3];   /* upsampled, >= W x H      */
    uint8_t *rgb;        int64_t rgb_pitch;
} job;

static int setup(const orc_image *img, job *J)
{
    memset(J, 0, sizeof(*J));
    J->img = img;
    if (img->width < 1 || img->height < 1) return -1;
    int hmax = 1, vmax = 1;
    for (int c = 0; c < 3; c++) {
        if (img->h_samp[c] < 1 || img->h_samp[c] > 2 || img->v_samp[c] < 1 || img->v_samp[c] > 2) return -1;
        if (img->h_samp[c] > hmax) hmax = img->h_samp[c];
        if (img->v_samp[c] > vmax) vmax = img->v_samp[c];
    }
    J->hmax = hmax; J->vmax = vmax;
    const int mx = (img->width + 8 * hmax - 1) / (8 * hmax);
    const int my = (img->height + 8 * vmax - 1) / (8 * vmax);
    for (int c = 0; c < 3; c++) {
        if (hmax % img->h_samp[c] || vmax % img->v_samp[c]) return -1;
        if (img->blocks_w[c] != mx * img->h_samp[c] || img->blocks_h[c] != my * img->v_samp[c]) return -1;
        J->sx[c] = hmax / img->h_samp[c];
        J->sy[c] = vmax / img->v_samp[c];
        J->cw[c] = (int)(((int64_t)img->width * img->h_samp[c] + hmax - 1) / hmax);
        J->ch[c] = (int)(((int64_t)img->height * img->v_samp[c] + vmax - 1) / vmax);
        J->ppitch[c] = (int64_t)img->blocks_w[c] * 8;
        J->upitch[c] = (int64_t)J->cw[c] * J->sx[c];
    }
    return 0;
}

static int alloc_planes(job *J)
{
    for (int c = 0; c < 3; c++) {
        J->plane[c] = (uint8_t *)malloc((size_t)J->ppitch[c] * J->img->blocks_h[c] * 8);
        J->up[c] = (uint8_t *)malloc((size_t)J->upitch[c] * J->ch[c] * J->sy[c]);
        if (!J->plane[c] || !J->up[c]) return -1;
    }
    return 0;
}

static void free_planes(job *J)
{
    for (int c = 0; c < 3; c++) { free(J->plane[c]); free(J->up[c]); }
}

/* Blocks with linear index in [b0, b1) of component c: IDCT into the plane. */
static void stage_idct(job *J, int c, int64_t b0, int64_t b1)
{
    const orc_image *img = J->img;
    uint8_t blk[64];
    for (int64_t b = b0; b < b1; b++) {
        const int bx = (int)(b % img->blocks_w[c]), by = (int)(b / img->blocks_w[c]);
        if (img->idct)
            orc_idct_aan_block(img->coef[c] + 64 * b, img->qtab[c], blk);
        else
            orc_idct_block(img->coef[c] + 64 * b, img->qtab[c], blk);
        for (int y = 0; y < 8; y++)
            memcpy(J->plane[c] + (int64_t)(by * 8 + y) * J->ppitch[c] + bx * 8, blk + 8 * y, 8);
    }
}

/* Output rows [y0, y1): upsample the three planes for those rows, convert. */
static void stage_rows(job *J, int y0, int y1)
{
    const orc_image *img = J->img;
    for (int c = 0; c < 3; c++)
        orc_upsample_rows(J->plane[c], J->cw[c], J->ch[c], J->ppitch[c], J->sx[c], J->sy[c],
                          img->fancy, J->up[c], J->upitch[c], y0, y1);
    for (int y = y0; y < y1; y++)
        for (int x = 0; x < img->width; x++)
            orc_ycc_to_rgb(J->up[0][(int64_t)y * J->upitch[0] + x],
                           J->up[1][(int64_t)y * J->upitch[1] + x],
                           J->up[2][(int64_t)y * J->upitch[2] + x],
                           J->rgb + (int64_t)y * J->rgb_pitch + 3 * x);
}

int orc_backend_decode(const orc_image *img, uint8_t *rgb, int64_t rgb_pitch)
{
    job J;
    if (setup(img, &J) || rgb_pitch < 3 * (int64_t)img->width) return -1;
    J.rgb = rgb; J.rgb_pitch = rgb_pitch;
    if (alloc_planes(&J)) { free_planes(&J); return -1; }
    for (int c = 0; c < 3; c++)
        stage_idct(&J, c, 0, (int64_t)img->blocks_w[c] * img->blocks_h[c]);
    stage_rows(&J, 0, img->height);
    free_planes(&J);
    return 0;
}

int orc_backend_decode_gray(int32_t width, int32_t height, const int16_t *coef, int32_t blocks_w,
                            int32_t blocks_h, const uint16_t q[64], uint8_t *rgb, int64_t rgb_pitch,
                            int32_t idct)
{
    if (width < 1 || height < 1 || !coef || !q || !rgb || rgb_pitch < 3 * (int64_t)width) return -1;
    if (blocks_w != (width + 7) / 8 || blocks_h != (height + 7) / 8) return -1;
    uint8_t blk[64];
    for (int by = 0; by < blocks_h; by++)
        for (int bx = 0; bx < blocks_w; bx++) {
            if (idct)
                orc_idct_aan_block(coef + 64 * ((int64_t)by * blocks_w + bx), q, blk);
            else
                orc_idct_block(coef + 64 * ((int64_t)by * blocks_w + bx), q, blk);
            for (int y = 0; y < 8; y++) {
                const int py = by * 8 + y;
                if (py >= height) break;
                for (int x = 0; x < 8; x++) {
                    const int px = bx * 8 + x;
                    if (px >= width) break;
                    uint8_t *o = rgb + (int64_t)py * rgb_pitch + 3 * px;
                    o[0] = o[1] = o[2] = blk[8 * y + x];
                }
            }
        }
    return 0;
}

/* ---- threaded driver: same stages, split into contiguous ranges ---------- */
typedef struct { job *J; int t, n, phase; } targ;

static void *worker(void *p)
{
    targ *a = (targ *)p;
    job *J = a->J;
    if (a->phase == 0) {
        for (int c = 0; c < 3; c++) {
            int64_t nb = (int64_t)J->img->blocks_w[c] * J->img->blocks_h[c];
            stage_idct(J, c, nb * a->t / a->n, nb * (a->t + 1) / a->n);
        }
    } else {
        int h = J->img->height;
        stage_rows(J, (int)((int64_t)h * a->t / a->n), (int)((int64_t)h * (a->t + 1) / a->n));
    }
    return NULL;
}

int orc_backend_decode_mt(const orc_image *img, uint8_t *rgb, int64_t rgb_pitch, int nthreads)
{
    job J;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (setup(img, &J) || rgb_pitch < 3 * (int64_t)img->width) return -1;
    J.rgb = rgb; J.rgb_pitch = rgb_pitch;
    if (alloc_planes(&J)) { free_planes(&J); return -1; }
    pthread_t th[256];
    targ args[256];
    for (int phase = 0; phase < 2; phase++) {
        for (int t = 0; t < nthreads; t++) {
            args[t].J = &J; args[t].t = t; args[t].n = nthreads; args[t].phase = phase;
            pthread_create(&th[t], NULL, worker, &args[t]);
        }
        for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    }
    free_planes(&J);
    return nthreads;
}
