/*
 * orc_huffman.c -- baseline JPEG stream parsing and Huffman (entropy)
 * decoding for the oracle.  TEST INFRASTRUCTURE ONLY (see orc.h).
 *
 * Entropy decoding is the sequential first stage of Fig. 1 (Sec. 2); it stays
 * on the host and outside the data-parallel path.  The decoder follows the
 * procedures of ITU-T T.81 (the paper does not restate them): code tables
 * from BITS/HUFFVAL (Annex C), DECODE with MINCODE/MAXCODE/VALPTR, RECEIVE
 * and EXTEND (F.2.2), DC prediction per component, AC run/size symbols with
 * EOB and ZRL, byte stuffing (0xFF00) and restart markers (F.2.2.5).
 * Coefficients are written in natural order (zig-zag undone).
 */
#include <string.h>
#include "orc.h"

typedef struct {
    int present;
    uint8_t bits[17];        /* bits[l] = number of codes of length l */
    uint8_t val[256];
    int32_t mincode[17], maxcode[18], valptr[17];
} htab;

typedef struct {
    const uint8_t *p, *end;
    uint32_t acc; int nbits;
    int hit_marker;
} bitrd;

/* zig-zag position -> natural index, generated by walking the anti-diagonals
 * of the 8x8 block (T.81 Figure A.6) */
static void make_zigzag(int zz[64])
{
    int k = 0;
    for (int s = 0; s < 15; s++) {
        if (s & 1) {   /* odd diagonal: top-right to bottom-left */
            for (int r = (s < 8 ? 0 : s - 7); r <= (s < 8 ? s : 7); r++) zz[k++] = r * 8 + (s - r);
        } else {       /* even diagonal: bottom-left to top-right */
            for (int r = (s < 8 ? s : 7); r >= (s < 8 ? 0 : s - 7); r--) zz[k++] = r * 8 + (s - r);
        }
    }
}

static int build_htab(htab *t)
{
    /* Annex C: code lengths and codes in canonical order, then F.15 tables */
    int code = 0, k = 0;
    for (int l = 1; l <= 16; l++) {
        t->valptr[l] = k;
        t->mincode[l] = code;
        code += t->bits[l];
        k += t->bits[l];
        t->maxcode[l] = t->bits[l] ? code - 1 : -1;
        if (code > (1 << l)) return -1;
        code <<= 1;
    }
    t->maxcode[17] = 0x7fffffff;
    return k <= 256 ? 0 : -1;
}

static int nextbit(bitrd *b)
{
    if (b->nbits == 0) {
        uint8_t byte = 0;
        if (b->hit_marker || b->p >= b->end) {
            byte = 0;                       /* past the data: zeros */
        } else {
            byte = *b->p;
            if (byte == 0xFF) {
                if (b->p + 1 < b->end && b->p[1] == 0x00) { b->p += 2; }
                else { b->hit_marker = 1; byte = 0; }
            } else {
                b->p++;
            }
        }
        b->acc = byte; b->nbits = 8;
    }
    b->nbits--;
    return (b->acc >> b->nbits) & 1;
}

static int receive(bitrd *b, int s)
{
    int v = 0;
    for (int i = 0; i < s; i++) v = (v << 1) | nextbit(b);
    return v;
}

static int extend(int v, int t)
{
    return (t > 0 && v < (1 << (t - 1))) ? v - (1 << t) + 1 : v;
}

static int decode(bitrd *b, const htab *t)
{
    int l = 1, code = nextbit(b);
    while (l <= 16 && code > t->maxcode[l]) { code = (code << 1) | nextbit(b); l++; }
    if (l > 16) return -1;
    return t->val[t->valptr[l] + code - t->mincode[l]];
}

static int u16be(const uint8_t *p) { return (p[0] << 8) | p[1]; }

int orc_jpeg_decode_coefs(const uint8_t *data, int64_t size, orc_jpeg_info *info,
                          int16_t *planes[3])
{
    int zz[64];
    make_zigzag(zz);
    htab dc[4], ac[4];
    memset(dc, 0, sizeof dc); memset(ac, 0, sizeof ac);
    uint16_t qt[4][64];
    int qt_present[4] = {0, 0, 0, 0};
    int comp_q[3] = {0, 0, 0}, comp_id[3] = {0, 0, 0};
    int restart = 0, have_sof = 0;
    memset(info, 0, sizeof(*info));

    const uint8_t *p = data, *end = data + size;
    if (size < 4 || p[0] != 0xFF || p[1] != 0xD8) return -1;
    p += 2;
    while (p + 4 <= end) {
        if (p[0] != 0xFF) return -2;
        int m = p[1];
        if (m == 0xFF) { p++; continue; }
        if (m == 0xD9) return -3;                  /* EOI before SOS */
        int len = u16be(p + 2);
        const uint8_t *s = p + 4, *se = p + 2 + len;
        if (se > end || len < 2) return -2;
        if (m == 0xDB) {                           /* DQT */
            while (s < se) {
                int pq = s[0] >> 4, tq = s[0] & 15;
                if (tq > 3) return -4;
                s++;
                for (int k = 0; k < 64; k++) {
                    int v = pq ? u16be(s + 2 * k) : s[k];
                    qt[tq][zz[k]] = (uint16_t)v;
                }
                s += pq ? 128 : 64;
                qt_present[tq] = 1;
            }
        } else if (m == 0xC4) {                    /* DHT */
            while (s < se) {
                int tc = s[0] >> 4, th = s[0] & 15;
                if (th > 3 || tc > 1) return -4;
                htab *t = tc ? &ac[th] : &dc[th];
                int total = 0;
                t->bits[0] = 0;
                for (int l = 1; l <= 16; l++) { t->bits[l] = s[l]; total += s[l]; }
                if (total > 256 || s + 17 + total > se) return -4;
                memcpy(t->val, s + 17, (size_t)total);
                if (build_htab(t)) return -4;
                t->present = 1;
                s += 17 + total;
            }
        } else if (m == 0xC0 || m == 0xC1) {       /* SOF0 / SOF1, 8-bit */
            if (s[0] != 8) return -5;
            info->height = u16be(s + 1);
            info->width = u16be(s + 3);
            info->ncomp = s[5];
            if (info->ncomp != 3 || info->width < 1 || info->height < 1) return -5;
            for (int c = 0; c < 3; c++) {
                comp_id[c] = s[6 + 3 * c];
                info->h_samp[c] = s[7 + 3 * c] >> 4;
                info->v_samp[c] = s[7 + 3 * c] & 15;
                comp_q[c] = s[8 + 3 * c] & 3;
                if (info->h_samp[c] < 1 || info->h_samp[c] > 2 || info->v_samp[c] < 1 || info->v_samp[c] > 2)
                    return -5;
            }
            have_sof = 1;
        } else if (m == 0xDD) {                    /* DRI */
            restart = u16be(s);
        } else if (m == 0xDA) {                    /* SOS */
            if (!have_sof) return -6;
            int ns = s[0];
            if (ns != 3) return -6;
            int td[3], ta[3], order[3];
            for (int i = 0; i < 3; i++) {
                int id = s[1 + 2 * i];
                order[i] = -1;
                for (int c = 0; c < 3; c++) if (comp_id[c] == id) order[i] = c;
                if (order[i] < 0) return -6;
                td[i] = s[2 + 2 * i] >> 4; ta[i] = s[2 + 2 * i] & 15;
                if (td[i] > 3 || ta[i] > 3 || !dc[td[i]].present || !ac[ta[i]].present) return -6;
            }
            int hmax = 1, vmax = 1;
            for (int c = 0; c < 3; c++) {
                if (info->h_samp[c] > hmax) hmax = info->h_samp[c];
                if (info->v_samp[c] > vmax) vmax = info->v_samp[c];
            }
            const int mx = (info->width + 8 * hmax - 1) / (8 * hmax);
            const int my = (info->height + 8 * vmax - 1) / (8 * vmax);
            for (int c = 0; c < 3; c++) {
                info->blocks_w[c] = mx * info->h_samp[c];
                info->blocks_h[c] = my * info->v_samp[c];
                if (!qt_present[comp_q[c]]) return -4;
                memcpy(info->qtab[c], qt[comp_q[c]], sizeof(info->qtab[c]));
            }
            if (!planes) return 0;
            bitrd b = { se + 3, end, 0, 0, 0 };
            b.p = se;
            int pred[3] = {0, 0, 0};
            int64_t nmcu = (int64_t)mx * my, todo = restart;
            for (int64_t mcu = 0; mcu < nmcu; mcu++) {
                if (restart && todo == 0) {
                    /* F.2.2.5: byte-align, expect RSTn, reset predictors */
                    b.nbits = 0; b.hit_marker = 0;
                    if (b.p + 1 < b.end && b.p[0] == 0xFF && b.p[1] >= 0xD0 && b.p[1] <= 0xD7) b.p += 2;
                    else return -7;
                    pred[0] = pred[1] = pred[2] = 0;
                    todo = restart;
                }
                const int mcx = (int)(mcu % mx), mcy = (int)(mcu / mx);
                for (int i = 0; i < 3; i++) {
                    const int c = order[i];
                    for (int v = 0; v < info->v_samp[c]; v++)
                        for (int h = 0; h < info->h_samp[c]; h++) {
                            int64_t bx = (int64_t)mcx * info->h_samp[c] + h;
                            int64_t by = (int64_t)mcy * info->v_samp[c] + v;
                            int16_t *blk = planes[c] + 64 * (by * info->blocks_w[c] + bx);
                            memset(blk, 0, 64 * sizeof(int16_t));
                            int t = decode(&b, &dc[td[i]]);
                            if (t < 0 || t > 11) return -8;
                            pred[c] += extend(receive(&b, t), t);
                            blk[0] = (int16_t)pred[c];
                            for (int k = 1; k < 64; k++) {
                                int rs = decode(&b, &ac[ta[i]]);
                                if (rs < 0) return -8;
                                int r = rs >> 4, ss = rs & 15;
                                if (ss == 0) {
                                    if (r == 15) { k += 15; continue; }
                                    break;                        /* EOB */
                                }
                                k += r;
                                if (k > 63 || ss > 10) return -8;
                                blk[zz[k]] = (int16_t)extend(receive(&b, ss), ss);
                            }
                        }
                }
                if (restart) todo--;
            }
            return 0;
        }
        p = se;
    }
    return -9;
}
