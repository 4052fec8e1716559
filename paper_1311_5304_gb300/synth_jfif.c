/*
 * synth_jfif.c -- baseline JFIF encoder for the synthetic workloads (input
 * side only: it turns quantised coefficient planes into the byte streams that
 * the host entropy decoder of the serving loop consumes).
 *
 * Follows ITU-T T.81: one interleaved scan of three components (SOF0, 8-bit),
 * DC differences coded by magnitude category, AC coefficients in zig-zag order
 * as run/size symbols with ZRL and EOB, per-image optimal Huffman tables built
 * with the Annex K.2 procedure (a reserved code point keeps the all-ones code
 * unused; lengths limited to 16 bits by moving pairs of symbols up the tree),
 * byte stuffing after 0xFF, optional restart intervals with RSTn markers.
 * Table 0 serves luminance, table 1 both chrominance components.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { uint8_t *buf; int64_t cap, n; uint32_t acc; int nbits; int overflow; } bw_t;

static void put_byte(bw_t *w, int b)
{
    if (w->n < w->cap) w->buf[w->n] = (uint8_t)b; else w->overflow = 1;
    w->n++;
}
static void put_u16(bw_t *w, int v) { put_byte(w, v >> 8); put_byte(w, v & 255); }

static void put_bits(bw_t *w, uint32_t code, int len)
{
    for (int i = len - 1; i >= 0; i--) {
        w->acc = (w->acc << 1) | ((code >> i) & 1);
        if (++w->nbits == 8) {
            put_byte(w, (int)w->acc);
            if (w->acc == 0xFF) put_byte(w, 0);
            w->acc = 0; w->nbits = 0;
        }
    }
}
static void flush_bits(bw_t *w)
{
    while (w->nbits) put_bits(w, 1, 1);   /* pad with 1-bits */
}

static int zz_nat[64];
static void make_zigzag(void)
{
    int k = 0;
    for (int s = 0; s < 15; s++) {
        int lo = s < 8 ? 0 : s - 7, hi = s < 8 ? s : 7;
        if (s & 1) for (int r = lo; r <= hi; r++) zz_nat[k++] = r * 8 + (s - r);
        else       for (int r = hi; r >= lo; r--) zz_nat[k++] = r * 8 + (s - r);
    }
}

static int category(int v) { int a = v < 0 ? -v : v, n = 0; while (a) { n++; a >>= 1; } return n; }

typedef struct { uint8_t bits[17]; uint8_t val[256]; int nval; uint16_t code[256]; uint8_t len[256]; } huff_t;

/* Annex K.2: code sizes from frequencies, then length limiting (K.3). */
static void build_optimal(const int64_t freq_in[256], huff_t *h)
{
    int64_t freq[257];
    int codesize[257], others[257];
    for (int i = 0; i < 256; i++) freq[i] = freq_in[i];
    freq[256] = 1;                                   /* reserved code point */
    for (int i = 0; i < 257; i++) { codesize[i] = 0; others[i] = -1; }
    for (;;) {
        int v1 = -1, v2 = -1;
        for (int i = 0; i < 257; i++)                /* least frequency; ties: larger value */
            if (freq[i] > 0 && (v1 < 0 || freq[i] <= freq[v1])) v1 = i;
        for (int i = 0; i < 257; i++)
            if (freq[i] > 0 && i != v1 && (v2 < 0 || freq[i] <= freq[v2])) v2 = i;
        if (v2 < 0) break;
        freq[v1] += freq[v2]; freq[v2] = 0;
        codesize[v1]++;
        while (others[v1] >= 0) { v1 = others[v1]; codesize[v1]++; }
        others[v1] = v2;
        codesize[v2]++;
        while (others[v2] >= 0) { v2 = others[v2]; codesize[v2]++; }
    }
    int bits[64];
    memset(bits, 0, sizeof bits);
    for (int i = 0; i < 257; i++) if (codesize[i]) bits[codesize[i]]++;
    for (int i = 63; i > 16; i--) {
        while (bits[i] > 0) {
            int j = i - 2;
            while (bits[j] == 0) j--;
            bits[i] -= 2; bits[i - 1] += 1; bits[j + 1] += 2; bits[j] -= 1;
        }
    }
    int i = 16;
    while (bits[i] == 0) i--;
    bits[i]--;                                       /* drop the reserved point */
    memset(h, 0, sizeof(*h));
    for (int l = 1; l <= 16; l++) h->bits[l] = (uint8_t)bits[l];
    /* symbols in order of code size, then value */
    int k = 0;
    for (int l = 1; l <= 32; l++)
        for (int s = 0; s < 256; s++)
            if (codesize[s] == l) h->val[k++] = (uint8_t)s;
    h->nval = k;
    /* canonical codes */
    int code = 0; k = 0;
    for (int l = 1; l <= 16; l++) {
        for (int n = 0; n < h->bits[l]; n++) { h->code[h->val[k]] = (uint16_t)code; h->len[h->val[k]] = (uint8_t)l; code++; k++; }
        code <<= 1;
    }
}

typedef struct {
    int width, height, ncomp, hs[3], vs[3], bw[3], bh[3], mx, my, restart;
    const int16_t *planes[3];
} enc_t;

/* Walks the scan; with count != NULL gathers symbol frequencies, else emits. */
static void scan(const enc_t *e, int64_t dcf[2][256], int64_t acf[2][256],
                 const huff_t dch[2], const huff_t ach[2], bw_t *w)
{
    int pred[3] = {0, 0, 0}, rst = 0;
    int64_t nmcu = (int64_t)e->mx * e->my;
    for (int64_t m = 0; m < nmcu; m++) {
        if (e->restart && m > 0 && m % e->restart == 0) {
            if (w) { flush_bits(w); put_byte(w, 0xFF); put_byte(w, 0xD0 + (rst & 7)); }
            rst++;
            pred[0] = pred[1] = pred[2] = 0;
        }
        int mcx = (int)(m % e->mx), mcy = (int)(m / e->mx);
        for (int c = 0; c < e->ncomp; c++) {
            int t = c ? 1 : 0;
            for (int v = 0; v < e->vs[c]; v++)
                for (int h = 0; h < e->hs[c]; h++) {
                    int64_t bx = (int64_t)mcx * e->hs[c] + h, by = (int64_t)mcy * e->vs[c] + v;
                    const int16_t *b = e->planes[c] + 64 * (by * e->bw[c] + bx);
                    int diff = b[0] - pred[c];
                    pred[c] = b[0];
                    int s = category(diff);
                    if (dcf) dcf[t][s]++;
                    if (w) {
                        put_bits(w, dch[t].code[s], dch[t].len[s]);
                        if (s) put_bits(w, (uint32_t)(diff < 0 ? diff - 1 : diff) & ((1u << s) - 1), s);
                    }
                    int run = 0;
                    for (int k = 1; k < 64; k++) {
                        int a = b[zz_nat[k]];
                        if (a == 0) { run++; continue; }
                        while (run > 15) {
                            if (acf) acf[t][0xF0]++;
                            if (w) put_bits(w, ach[t].code[0xF0], ach[t].len[0xF0]);
                            run -= 16;
                        }
                        int ss = category(a), rs = (run << 4) | ss;
                        if (acf) acf[t][rs]++;
                        if (w) {
                            put_bits(w, ach[t].code[rs], ach[t].len[rs]);
                            put_bits(w, (uint32_t)(a < 0 ? a - 1 : a) & ((1u << ss) - 1), ss);
                        }
                        run = 0;
                    }
                    if (run > 0) {
                        if (acf) acf[t][0x00]++;
                        if (w) put_bits(w, ach[t].code[0], ach[t].len[0]);
                    }
                }
        }
    }
    if (w) flush_bits(w);
}

/* Returns the stream length (may exceed cap: then call again with a larger
 * buffer), or -1 on bad arguments.  Coefficients must lie in [-2047, 2047]
 * (DC differences in [-2047, 2047] as well for 8-bit baseline). */
int64_t synth_jfif_encode_n(int width, int height, int ncomp, const int hs[3], const int vs[3],
                            const int16_t *planes[3], const int bw[3], const int bh[3],
                            const uint16_t *qtabs[3], int restart, uint8_t *out, int64_t cap)
{
    make_zigzag();
    if (ncomp != 1 && ncomp != 3) return -1;
    enc_t e;
    memset(&e, 0, sizeof e);
    e.width = width; e.height = height; e.restart = restart; e.ncomp = ncomp;
    int hmax = 1, vmax = 1;
    for (int c = 0; c < ncomp; c++) {
        e.hs[c] = hs[c]; e.vs[c] = vs[c]; e.bw[c] = bw[c]; e.bh[c] = bh[c]; e.planes[c] = planes[c];
        if (hs[c] > hmax) hmax = hs[c];
        if (vs[c] > vmax) vmax = vs[c];
    }
    e.mx = (width + 8 * hmax - 1) / (8 * hmax);
    e.my = (height + 8 * vmax - 1) / (8 * vmax);
    if (ncomp == 1) {
        /* one component: 8x8 MCUs whatever its sampling factors (T.81 A.2.2) */
        e.hs[0] = e.vs[0] = 1;
        e.mx = (width + 7) / 8;
        e.my = (height + 7) / 8;
    }
    for (int c = 0; c < ncomp; c++)
        if (bw[c] != e.mx * e.hs[c] || bh[c] != e.my * e.vs[c]) return -1;
    const int ntab = ncomp == 1 ? 1 : 2;

    static int64_t dcf[2][256], acf[2][256];
    memset(dcf, 0, sizeof dcf); memset(acf, 0, sizeof acf);
    scan(&e, dcf, acf, NULL, NULL, NULL);
    huff_t dch[2], ach[2];
    for (int t = 0; t < ntab; t++) { build_optimal(dcf[t], &dch[t]); build_optimal(acf[t], &ach[t]); }

    bw_t w = { out, cap, 0, 0, 0, 0 };
    put_u16(&w, 0xFFD8);
    /* APP0 JFIF */
    put_u16(&w, 0xFFE0); put_u16(&w, 16);
    put_byte(&w, 'J'); put_byte(&w, 'F'); put_byte(&w, 'I'); put_byte(&w, 'F'); put_byte(&w, 0);
    put_u16(&w, 0x0101); put_byte(&w, 0); put_u16(&w, 1); put_u16(&w, 1); put_byte(&w, 0); put_byte(&w, 0);
    /* DQT: one table per component (zig-zag order) */
    for (int c = 0; c < ncomp; c++) {
        int big = 0;
        for (int k = 0; k < 64; k++) if (qtabs[c][k] > 255) big = 1;
        put_u16(&w, 0xFFDB); put_u16(&w, 2 + 1 + (big ? 128 : 64));
        put_byte(&w, (big << 4) | c);
        for (int k = 0; k < 64; k++) {
            int q = qtabs[c][zz_nat[k]];
            if (big) put_u16(&w, q); else put_byte(&w, q);
        }
    }
    /* SOF0 */
    put_u16(&w, 0xFFC0); put_u16(&w, 8 + 3 * ncomp); put_byte(&w, 8);
    put_u16(&w, height); put_u16(&w, width); put_byte(&w, ncomp);
    for (int c = 0; c < ncomp; c++) { put_byte(&w, c + 1); put_byte(&w, (e.hs[c] << 4) | e.vs[c]); put_byte(&w, c); }
    /* DHT */
    for (int t = 0; t < ntab; t++)
        for (int cls = 0; cls < 2; cls++) {
            const huff_t *h = cls ? &ach[t] : &dch[t];
            put_u16(&w, 0xFFC4); put_u16(&w, 2 + 1 + 16 + h->nval);
            put_byte(&w, (cls << 4) | t);
            for (int l = 1; l <= 16; l++) put_byte(&w, h->bits[l]);
            for (int k = 0; k < h->nval; k++) put_byte(&w, h->val[k]);
        }
    if (restart) { put_u16(&w, 0xFFDD); put_u16(&w, 4); put_u16(&w, restart); }
    /* SOS */
    put_u16(&w, 0xFFDA); put_u16(&w, 6 + 2 * ncomp); put_byte(&w, ncomp);
    for (int c = 0; c < ncomp; c++) { put_byte(&w, c + 1); put_byte(&w, c ? 0x11 : 0x00); }
    put_byte(&w, 0); put_byte(&w, 63); put_byte(&w, 0);
    scan(&e, NULL, NULL, dch, ach, &w);
    put_u16(&w, 0xFFD9);
    return w.n;
}

int64_t synth_jfif_encode(int width, int height, const int hs[3], const int vs[3],
                          const int16_t *planes[3], const int bw[3], const int bh[3],
                          const uint16_t *qtabs[3], int restart, uint8_t *out, int64_t cap)
{
    return synth_jfif_encode_n(width, height, 3, hs, vs, planes, bw, bh, qtabs, restart, out, cap);
}
