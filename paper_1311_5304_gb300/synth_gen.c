/*
 * synth_gen.c -- seeded synthetic images -> quantised DCT coefficient planes
 * (input side of the benchmarks and tests; holds no decode arithmetic).
 *
 * Content of pixel (x, y), every term a pure function of (seed, x, y), so the
 * result does not depend on the number of threads or on banding:
 *   base_c  = smooth per-channel colour field: offset + linear ramps + a
 *             product of sinusoids;
 *   texture = 4 octaves of 2-D gradient noise (cells 24, 10, 4, 2.2 px) plus an
 *             independent 4-octave texture (16, 6, 3, 2.2 px) in the colour
 *             difference direction, scaled by a
 *             patch mask m = clamp(4 (P(x, y) - t), 0, 1) where P is gradient
 *             noise with 192-px cells and t is set from the requested cover;
 *   grain   = i.i.d. Gaussian noise of standard deviation sigma per channel,
 *             from a counter-based generator (SplitMix64 on the pixel index,
 *             Box-Muller).
 * Encoder side (ITU-T T.81): RGB -> YCbCr with the JFIF weights, rounded;
 * box-filter chroma downsampling, rounded; level shift -128; 8x8 forward DCT
 * in double precision (A.3.3); quantisation rounding half away from zero;
 * DC clipped to [-2047, 2047], AC to [-1023, 1023] (baseline-encodable).
 * Padding beyond the image replicates the last row and column.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

static double u01(uint64_t h) { return ((h >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

/* one N(0,1) sample keyed by (seed, stream, index) */
static double gauss(uint64_t seed, uint64_t stream, uint64_t idx)
{
    uint64_t h1 = splitmix64(seed ^ splitmix64(stream * 0x632BE59BD9B4E019ull + idx));
    uint64_t h2 = splitmix64(h1 ^ 0xD1B54A32D192ED03ull);
    double r = sqrt(-2.0 * log(u01(h1)));
    return r * cos(6.283185307179586 * u01(h2));
}

static double grad_noise(uint64_t seed, int oct, double fx, double fy)
{
    double x0 = floor(fx), y0 = floor(fy);
    double tx = fx - x0, ty = fy - y0;
    long ix = (long)x0, iy = (long)y0;
    double v[4];
    for (int c = 0; c < 4; c++) {
        long cx = ix + (c & 1), cy = iy + (c >> 1);
        uint64_t h = splitmix64(seed ^ splitmix64(((uint64_t)(uint32_t)cx << 32 | (uint32_t)cy) + 0x1000003ull * oct));
        double a = 6.283185307179586 * u01(h);
        v[c] = cos(a) * (tx - (c & 1)) + sin(a) * (ty - (c >> 1));
    }
    double u = tx * tx * tx * (tx * (tx * 6 - 15) + 10);
    double w = ty * ty * ty * (ty * (ty * 6 - 15) + 10);
    double a = v[0] + u * (v[1] - v[0]);
    double b = v[2] + u * (v[3] - v[2]);
    return a + w * (b - a);
}

typedef struct {
    int W, H;
    uint64_t seed;
    int kind;          /* 0 gradient, 1 texture */
    double sigma, cover;
    double coef[3][6], base[3], freq[3][2];
    double thresh;
} content_t;

static void content_init(content_t *c, int W, int H, uint64_t seed, int kind, double sigma, double cover)
{
    memset(c, 0, sizeof(*c));
    c->W = W; c->H = H; c->seed = seed; c->kind = kind; c->sigma = sigma; c->cover = cover;
    uint64_t s = splitmix64(seed ^ 0x5EEDull);
    for (int ch = 0; ch < 3; ch++) {
        for (int k = 0; k < 6; k++) { s = splitmix64(s); c->coef[ch][k] = 2.0 * u01(s) - 1.0; }
        s = splitmix64(s); c->base[ch] = 70.0 + 110.0 * u01(s);
        for (int k = 0; k < 2; k++) { s = splitmix64(s); c->freq[ch][k] = 0.5 + 2.5 * u01(s); }
    }
    /* P in [-0.7, 0.7] roughly; threshold so that about `cover` of the area is textured */
    c->thresh = 0.55 - 1.1 * cover;
}

static void content_rgb(const content_t *c, int x, int y, double rgb[3])
{
    const double nx = (double)x / c->W, ny = (double)y / c->H;
    for (int ch = 0; ch < 3; ch++) {
        const double *a = c->coef[ch];
        rgb[ch] = c->base[ch] + 50 * a[0] * nx + 50 * a[1] * ny
                + 25 * a[2] * sin(6.283185307179586 * (c->freq[ch][0] * nx + a[3]))
                  * cos(6.283185307179586 * (c->freq[ch][1] * ny + a[4]))
                + 10 * a[5] * nx * ny;
    }
    if (c->kind == 1) {
        double p = grad_noise(c->seed, 0, x / 192.0, y / 192.0);
        double m = (p - c->thresh) * 4.0;
        m = m < 0 ? 0 : (m > 1 ? 1 : m);
        if (m > 0) {
            double t = grad_noise(c->seed, 1, x / 24.0, y / 24.0) + 0.6 * grad_noise(c->seed, 2, x / 10.0, y / 10.0)
                     + 0.5 * grad_noise(c->seed, 3, x / 4.0, y / 4.0) + 0.45 * grad_noise(c->seed, 8, x / 2.2, y / 2.2);
            /* an independent texture drives the colour difference channels */
            double t2 = grad_noise(c->seed, 5, x / 16.0, y / 16.0) + 0.7 * grad_noise(c->seed, 6, x / 6.0, y / 6.0)
                      + 0.6 * grad_noise(c->seed, 9, x / 3.0, y / 3.0)
                      + 0.9 * grad_noise(c->seed, 10, x / 2.2, y / 2.2);
            double amp = 70.0 * m;
            rgb[0] += amp * (t + 1.0 * t2);
            rgb[1] += amp * (t - 0.5 * t2);
            rgb[2] += amp * (t - 1.2 * t2);
        }
    }
    if (c->sigma > 0) {
        uint64_t idx = ((uint64_t)y * (uint64_t)c->W + (uint64_t)x) * 3;
        for (int ch = 0; ch < 3; ch++) rgb[ch] += c->sigma * gauss(c->seed, 7, idx + ch);
    }
}

/* Rows [y0, y1) of the true image as float RGB (for quality checks). */
int synth_render_rgb(int W, int H, uint64_t seed, int kind, double sigma, double cover, int y0, int y1, float *out)
{
    content_t c;
    content_init(&c, W, H, seed, kind, sigma, cover);
    for (int y = y0; y < y1; y++)
        for (int x = 0; x < W; x++) {
            double v[3];
            content_rgb(&c, x, y, v);
            for (int ch = 0; ch < 3; ch++) out[((size_t)(y - y0) * W + x) * 3 + ch] = (float)v[ch];
        }
    return 0;
}

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }
static double round_half_away(double v) { return v < 0 ? -floor(-v + 0.5) : floor(v + 0.5); }

typedef struct {
    const content_t *c;
    int hs[3], vs[3], hmax, vmax, mx, my;
    const uint16_t *q[3];
    int16_t *planes[3];
    int bw[3];
    int next_row;      /* MCU row counter (shared) */
    pthread_mutex_t mu;
    double D[8][8];
} gen_t;

static void fdct_quant(const gen_t *g, const double in[8][8], const uint16_t *q, int16_t *out)
{
    double t[8][8], F[8][8];
    for (int i = 0; i < 8; i++)
        for (int u = 0; u < 8; u++) {
            double s = 0;
            for (int j = 0; j < 8; j++) s += g->D[u][j] * in[i][j];
            t[i][u] = s;
        }
    for (int v = 0; v < 8; v++)
        for (int u = 0; u < 8; u++) {
            double s = 0;
            for (int i = 0; i < 8; i++) s += g->D[v][i] * t[i][u];
            F[v][u] = s;
        }
    for (int k = 0; k < 64; k++) {
        double z = round_half_away(F[k >> 3][k & 7] / (double)q[k]);
        double lim = k ? 1023.0 : 2047.0;
        out[k] = (int16_t)clampd(z, -lim, lim);
    }
}

static void do_mcu_row(gen_t *g, int r)
{
    const content_t *c = g->c;
    const int mh = 8 * g->vmax, mw = 8 * g->hmax;
    const int pw = g->mx * mw;
    /* full-resolution Y, Cb, Cr of the MCU row (padded width) */
    size_t n = (size_t)mh * pw;
    double *pl = (double *)malloc(3 * n * sizeof(double));
    for (int yy = 0; yy < mh; yy++) {
        int y = r * mh + yy;
        if (y > c->H - 1) y = c->H - 1;
        for (int xx = 0; xx < pw; xx++) {
            int x = xx > c->W - 1 ? c->W - 1 : xx;
            double rgb[3];
            content_rgb(c, x, y, rgb);
            double R = rgb[0], G = rgb[1], B = rgb[2];
            double Y = 0.299 * R + 0.587 * G + 0.114 * B;
            double Cb = -0.168736 * R - 0.331264 * G + 0.5 * B + 128.0;
            double Cr = 0.5 * R - 0.418688 * G - 0.081312 * B + 128.0;
            size_t o = (size_t)yy * pw + xx;
            pl[o] = clampd(floor(Y + 0.5), 0, 255);
            pl[n + o] = clampd(floor(Cb + 0.5), 0, 255);
            pl[2 * n + o] = clampd(floor(Cr + 0.5), 0, 255);
        }
    }
    for (int ch = 0; ch < 3; ch++) {
        const int sx = g->hmax / g->hs[ch], sy = g->vmax / g->vs[ch];
        const double *p = pl + ch * n;
        for (int by = 0; by < g->vs[ch]; by++)
            for (int bx = 0; bx < g->mx * g->hs[ch]; bx++) {
                double blk[8][8];
                for (int i = 0; i < 8; i++)
                    for (int j = 0; j < 8; j++) {
                        double s = 0;
                        int py = (by * 8 + i) * sy, px = (bx * 8 + j) * sx;
                        for (int a = 0; a < sy; a++)
                            for (int b = 0; b < sx; b++) s += p[(size_t)(py + a) * pw + px + b];
                        s /= (double)(sx * sy);
                        if (sx * sy > 1) s = floor(s + 0.5);
                        blk[i][j] = s - 128.0;
                    }
                int64_t brow = (int64_t)r * g->vs[ch] + by;
                fdct_quant(g, blk, g->q[ch], g->planes[ch] + 64 * (brow * g->bw[ch] + bx));
            }
    }
    free(pl);
}

static void *gen_worker(void *arg)
{
    gen_t *g = (gen_t *)arg;
    for (;;) {
        pthread_mutex_lock(&g->mu);
        int r = g->next_row++;
        pthread_mutex_unlock(&g->mu);
        if (r >= g->my) break;
        do_mcu_row(g, r);
    }
    return NULL;
}

/* Quantised coefficient planes of the synthetic image.  planes[c] holds
 * (my*vs[c]) x (mx*hs[c]) blocks of 64 int16 in natural order. */
int synth_make_coefs(int W, int H, const int hs[3], const int vs[3], uint64_t seed, int kind, double sigma,
                     double cover, const uint16_t *q[3], int16_t *planes[3], int nthreads)
{
    content_t c;
    content_init(&c, W, H, seed, kind, sigma, cover);
    gen_t g;
    memset(&g, 0, sizeof g);
    g.c = &c;
    g.hmax = g.vmax = 1;
    for (int ch = 0; ch < 3; ch++) {
        g.hs[ch] = hs[ch]; g.vs[ch] = vs[ch]; g.q[ch] = q[ch]; g.planes[ch] = planes[ch];
        if (hs[ch] > g.hmax) g.hmax = hs[ch];
        if (vs[ch] > g.vmax) g.vmax = vs[ch];
    }
    g.mx = (W + 8 * g.hmax - 1) / (8 * g.hmax);
    g.my = (H + 8 * g.vmax - 1) / (8 * g.vmax);
    for (int ch = 0; ch < 3; ch++) g.bw[ch] = g.mx * hs[ch];
    for (int u = 0; u < 8; u++)
        for (int x = 0; x < 8; x++)
            g.D[u][x] = 0.5 * (u ? 1.0 : sqrt(0.5)) * cos((2 * x + 1) * u * 3.14159265358979323846 / 16.0);
    pthread_mutex_init(&g.mu, NULL);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 128) nthreads = 128;
    pthread_t th[128];
    for (int t = 0; t < nthreads; t++) pthread_create(&th[t], NULL, gen_worker, &g);
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&g.mu);
    return 0;
}
