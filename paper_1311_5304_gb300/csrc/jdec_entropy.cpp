// jdec_entropy.cpp -- host-side baseline JPEG parsing and entropy (Huffman)
// decoding for the serving path (Sec. 2: the sequential stage that stays on
// the CPU; Sec. 4.5: it overlaps with the data-parallel back-end).
//
// Parsing follows ITU-T T.81 markers (SOI, DQT, SOF0/SOF1, DHT, DRI, SOS).
// Decoding uses a 64-bit bit buffer (byte stuffing 0xFF00 removed, a marker
// ends the data), refilled up to 8 bytes at a time when none of them is 0xFF
// and a byte at a time otherwise.  Per Huffman table, an 11-bit table gives,
// for a code and its magnitude bits that fit in 11 bits together, the
// decoded value, the zero run (AC) and the bits used, so that most
// coefficients take one lookup; other codes go through a 9-bit lookahead
// table of code length and symbol, then the canonical MAXCODE/VALPTR search
// for codes longer than 9 bits (T.81 F.2.2.3).  Coefficients are written in
// natural order into the component planes (zig-zag undone); restart markers
// reset the DC predictors.
#include <cstdint>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <new>
#include <thread>
#include <vector>

#include "jdec_entropy.h"

#include "../../include/jdec.h"

namespace {

constexpr int kLook = 9;
constexpr int kFast = 11;

struct HuffTable {
    bool present = false;
    uint8_t bits[17] = {0};
    uint8_t vals[256] = {0};
    int32_t maxcode[18];     // largest code of each length (-1: none), [17] sentinel
    int32_t valoff[17];      // vals index of the first code of each length minus that code
    uint16_t look[1 << kLook];   // (length << 8) | symbol, length 0 = not in table
    // code + magnitude bits within kFast bits: value << 16 | run << 8 | bits
    // used; end of block: 0x80 << 8 | code length (0: not in table; never
    // holds ZRL or sizes above 11)
    int32_t fast[1 << kFast];
};

inline int extend(int v, int s) { return (s && v < (1 << (s - 1))) ? v - (1 << s) + 1 : v; }

// Fills t.fast: for every kFast-bit prefix whose leading code (length l,
// symbol rs: run rs >> 4, size rs & 15) and its size magnitude bits fit in
// the prefix, the extended value, the run and l + size.  `ac`: AC table
// (end of block flagged, ZRL left to the general path); else DC (run 0, size
// rs).
void build_fast(HuffTable &t, bool ac)
{
    memset(t.fast, 0, sizeof(t.fast));
    int code = 0, k = 0;
    for (int l = 1; l <= kFast; ++l) {
        for (int i = 0; i < t.bits[l]; ++i, ++k, ++code) {
            const int rs = t.vals[k];
            const int run = ac ? rs >> 4 : 0, sz = ac ? rs & 15 : rs;
            if (ac && rs == 0) {
                // end of block: run field 0x80, no value
                const int rest = kFast - l;
                for (int f = 0; f < (1 << rest); ++f) t.fast[(code << rest) | f] = (0x80 << 8) | l;
                continue;
            }
            if ((ac && sz == 0) || sz > (ac ? 10 : 11) || l + sz > kFast) continue;
            const int rest = kFast - l - sz;
            for (int m = 0; m < (1 << sz); ++m) {
                const int v = extend(m, sz);
                const int32_t e = static_cast<int32_t>(static_cast<uint32_t>(v) << 16) | (run << 8) | (l + sz);
                const int base = (((code << sz) | m) << rest);
                for (int f = 0; f < (1 << rest); ++f) t.fast[base | f] = e;
            }
        }
        code <<= 1;
    }
}

bool build_table(HuffTable &t)
{
    int code = 0, k = 0;
    for (int l = 1; l <= 16; ++l) {
        t.valoff[l] = k - code;
        if (t.bits[l]) {
            code += t.bits[l];
            k += t.bits[l];
            t.maxcode[l] = code - 1;
        } else {
            t.maxcode[l] = -1;
        }
        if (code > (1 << l)) return false;
        code <<= 1;
    }
    t.maxcode[17] = 0x7fffffff;
    if (k > 256) return false;
    memset(t.look, 0, sizeof(t.look));
    code = 0;
    k = 0;
    for (int l = 1; l <= kLook; ++l) {
        for (int i = 0; i < t.bits[l]; ++i, ++k, ++code) {
            const int shift = kLook - l;
            for (int f = 0; f < (1 << shift); ++f)
                t.look[(code << shift) | f] = static_cast<uint16_t>((l << 8) | t.vals[k]);
        }
        code <<= 1;
    }
    return true;
}

inline uint64_t load_be64(const uint8_t *p)
{
    uint64_t x;
    memcpy(&x, p, 8);
#if defined(__BYTE_ORDER__) && __BYTE_ORDER__ == __ORDER_LITTLE_ENDIAN__
    x = __builtin_bswap64(x);
#endif
    return x;
}

struct BitReader {
    const uint8_t *p, *end;
    uint64_t acc = 0;   // bits are left-aligned: the next bit is bit 63
    int n = 0;          // valid bits in acc
    bool marker = false;

    void refill()
    {
        // fast path: the next 8 bytes are data bytes with no 0xFF among them
        if (!marker && end - p >= 8) {
            const uint64_t x = load_be64(p);
            const uint64_t y = ~x;   // a 0xFF byte of x is a zero byte of y
            if (((y - 0x0101010101010101ull) & ~y & 0x8080808080808080ull) == 0) {
                const int k = (64 - n) >> 3;   // whole bytes that fit
                if (k > 0) {
                    acc |= (x >> (64 - 8 * k)) << (64 - 8 * k - n);
                    p += k;
                    n += 8 * k;
                }
                return;
            }
        }
        while (n <= 56) {
            uint32_t byte = 0;
            if (!marker && p < end) {
                byte = *p;
                if (byte == 0xFF) {
                    if (p + 1 < end && p[1] == 0x00) {
                        p += 2;
                    } else {
                        marker = true;   // leave p at the marker
                        byte = 0;
                    }
                } else {
                    ++p;
                }
            }
            acc |= static_cast<uint64_t>(byte) << (56 - n);
            n += 8;
        }
    }
    uint32_t peek(int k) { return static_cast<uint32_t>(acc >> (64 - k)); }
    void skip(int k) { acc <<= k; n -= k; }
    int get(int k)
    {
        if (k == 0) return 0;
        if (n < k) refill();
        const int v = static_cast<int>(acc >> (64 - k));
        skip(k);
        return v;
    }
    void reset_at(const uint8_t *q)
    {
        p = q;
        acc = 0;
        n = 0;
        marker = false;
    }
    // Byte position of the next unread whole byte (after discarding the bits
    // left in the buffer): only valid when the buffer holds no more than the
    // current byte's padding.
};

inline int decode_symbol(BitReader &br, const HuffTable &t)
{
    if (br.n < 16) br.refill();
    const uint16_t e = t.look[br.peek(kLook)];
    if (e) {
        br.skip(e >> 8);
        return e & 0xff;
    }
    int l = kLook + 1;
    int code = static_cast<int>(br.peek(l));
    while (l <= 16 && code > t.maxcode[l]) {
        ++l;
        code = static_cast<int>(br.peek(l));
    }
    if (l > 16) return -1;
    br.skip(l);
    return t.vals[t.valoff[l] + code];
}

int u16be(const uint8_t *p) { return (p[0] << 8) | p[1]; }

const int *zigzag()
{
    static int zz[64];
    static bool ready = false;
    if (!ready) {
        int k = 0;
        for (int s = 0; s < 15; ++s) {
            const int lo = s < 8 ? 0 : s - 7, hi = s < 8 ? s : 7;
            if (s & 1)
                for (int r = lo; r <= hi; ++r) zz[k++] = r * 8 + (s - r);
            else
                for (int r = hi; r >= lo; --r) zz[k++] = r * 8 + (s - r);
        }
        ready = true;
    }
    return zz;
}

struct Parsed {
    jdec_jpeg_info info;
    HuffTable dc[4], ac[4];
    int comp_id[3], comp_q[3];
    int scan_order[3], td[3], ta[3];
    const uint8_t *scan = nullptr;
};

jdec_status parse(const uint8_t *data, size_t size, Parsed &P, bool need_tables)
{
    const int *zz = zigzag();
    memset(&P.info, 0, sizeof(P.info));
    uint16_t qt[4][64];
    bool qt_present[4] = {false, false, false, false};
    bool have_sof = false;
    if (!data || size < 4 || data[0] != 0xFF || data[1] != 0xD8) return JDEC_EINVAL;
    const uint8_t *p = data + 2, *end = data + size;
    while (p + 4 <= end) {
        if (p[0] != 0xFF) return JDEC_EINVAL;
        const int m = p[1];
        if (m == 0xFF) {
            ++p;
            continue;
        }
        if (m == 0xD9) return JDEC_EINVAL;
        const int len = u16be(p + 2);
        const uint8_t *s = p + 4, *se = p + 2 + len;
        if (len < 2 || se > end) return JDEC_EINVAL;
        if (m == 0xDB) {
            while (s < se) {
                const int pq = s[0] >> 4, tq = s[0] & 15;
                if (tq > 3 || s + 1 + (pq ? 128 : 64) > se) return JDEC_EINVAL;
                ++s;
                for (int k = 0; k < 64; ++k) qt[tq][zz[k]] = static_cast<uint16_t>(pq ? u16be(s + 2 * k) : s[k]);
                s += pq ? 128 : 64;
                qt_present[tq] = true;
            }
        } else if (m == 0xC4) {
            while (s < se) {
                const int tc = s[0] >> 4, th = s[0] & 15;
                if (tc > 1 || th > 3 || s + 17 > se) return JDEC_EINVAL;
                HuffTable &t = tc ? P.ac[th] : P.dc[th];
                int total = 0;
                for (int l = 1; l <= 16; ++l) {
                    t.bits[l] = s[l];
                    total += s[l];
                }
                if (total > 256 || s + 17 + total > se) return JDEC_EINVAL;
                memcpy(t.vals, s + 17, static_cast<size_t>(total));
                if (need_tables) {
                    if (!build_table(t)) return JDEC_EINVAL;
                    build_fast(t, tc != 0);
                }
                t.present = true;
                s += 17 + total;
            }
        } else if (m == 0xC0 || m == 0xC1) {
            if (len < 8 || s[0] != 8) return JDEC_EUNSUPPORTED;
            P.info.height = u16be(s + 1);
            P.info.width = u16be(s + 3);
            P.info.ncomp = s[5];
            const int nc = P.info.ncomp;
            if (nc != 3 && nc != 1) return JDEC_EUNSUPPORTED;
            if (len < 8 + 3 * nc) return JDEC_EINVAL;
            for (int c = 0; c < nc; ++c) {
                P.comp_id[c] = s[6 + 3 * c];
                P.info.h_samp[c] = static_cast<uint8_t>(s[7 + 3 * c] >> 4);
                P.info.v_samp[c] = static_cast<uint8_t>(s[7 + 3 * c] & 15);
                P.comp_q[c] = s[8 + 3 * c] & 3;
                if (P.info.h_samp[c] < 1 || P.info.h_samp[c] > 4 || P.info.v_samp[c] < 1 || P.info.v_samp[c] > 4)
                    return JDEC_EINVAL;
                if (nc == 3 && (P.info.h_samp[c] > 2 || P.info.v_samp[c] > 2)) return JDEC_EUNSUPPORTED;
            }
            if (nc == 1) {
                // one component: 8x8 MCUs whatever its sampling factors (T.81 A.2.2)
                P.info.h_samp[0] = P.info.v_samp[0] = 1;
                for (int c = 1; c < 3; ++c) P.info.h_samp[c] = P.info.v_samp[c] = 0;
            }
            if (P.info.width < 1 || P.info.height < 1) return JDEC_EINVAL;
            have_sof = true;
        } else if (m >= 0xC2 && m <= 0xCF && m != 0xC4 && m != 0xC8 && m != 0xCC) {
            return JDEC_EUNSUPPORTED;   // progressive, lossless, arithmetic coding
        } else if (m == 0xDD) {
            if (len < 4) return JDEC_EINVAL;
            P.info.restart_interval = u16be(s);
        } else if (m == 0xDA) {
            if (!have_sof) return JDEC_EINVAL;
            const int nc = P.info.ncomp;
            if (s[0] != nc || len < 6 + 2 * nc) return JDEC_EUNSUPPORTED;
            for (int i = 0; i < nc; ++i) {
                const int id = s[1 + 2 * i];
                P.scan_order[i] = -1;
                for (int c = 0; c < nc; ++c)
                    if (P.comp_id[c] == id) P.scan_order[i] = c;
                if (P.scan_order[i] < 0) return JDEC_EINVAL;
                P.td[i] = s[2 + 2 * i] >> 4;
                P.ta[i] = s[2 + 2 * i] & 15;
                if (P.td[i] > 3 || P.ta[i] > 3 || !P.dc[P.td[i]].present || !P.ac[P.ta[i]].present) return JDEC_EINVAL;
            }
            int hmax = 1, vmax = 1;
            for (int c = 0; c < nc; ++c) {
                if (P.info.h_samp[c] > hmax) hmax = P.info.h_samp[c];
                if (P.info.v_samp[c] > vmax) vmax = P.info.v_samp[c];
            }
            const int mx = (P.info.width + 8 * hmax - 1) / (8 * hmax);
            const int my = (P.info.height + 8 * vmax - 1) / (8 * vmax);
            for (int c = 0; c < nc; ++c) {
                P.info.blocks_w[c] = mx * P.info.h_samp[c];
                P.info.blocks_h[c] = my * P.info.v_samp[c];
                if (!qt_present[P.comp_q[c]]) return JDEC_EINVAL;
                memcpy(P.info.qtab[c], qt[P.comp_q[c]], sizeof(P.info.qtab[c]));
            }
            P.scan = se;
            P.info.scan_offset = se - data;
            P.info.scan_bytes = end - se;
            return JDEC_OK;
        }
        p = se;
    }
    return JDEC_EINVAL;
}

// Decoder state that carries from one run of MCUs to the next.
struct ScanState {
    BitReader br;
    int pred[3] = {0, 0, 0};
    long todo = 0;   // MCUs left in the current restart interval
};

int mcus_x(const jdec_jpeg_info &in)
{
    int hmax = 1;
    for (int c = 0; c < 3; ++c)
        if (in.h_samp[c] > hmax) hmax = in.h_samp[c];
    return (in.width + 8 * hmax - 1) / (8 * hmax);
}

int mcus_y(const jdec_jpeg_info &in)
{
    int vmax = 1;
    for (int c = 0; c < 3; ++c)
        if (in.v_samp[c] > vmax) vmax = in.v_samp[c];
    return (in.height + 8 * vmax - 1) / (8 * vmax);
}

// Decodes MCUs [m0, m1) (raster order) into the full-size planes.
jdec_status decode_mcus(const Parsed &P, ScanState &S, int16_t *const planes[3], long m0, long m1)
{
    const int *zz = zigzag();
    const jdec_jpeg_info &in = P.info;
    const int mx = mcus_x(in);
    BitReader &br = S.br;
    for (long mcu = m0; mcu < m1; ++mcu) {
        if (in.restart_interval && S.todo == 0) {
            // expect RSTn at the marker the reader stopped on
            const uint8_t *q = br.p;
            if (!br.marker) {
                // the reader may have buffered padding bits only; skip to the marker
                while (q + 1 < br.end && !(q[0] == 0xFF && q[1] != 0x00)) ++q;
            }
            // fill bytes (0xFF) may precede any marker (T.81 B.1.1.2)
            while (q + 2 < br.end && q[0] == 0xFF && q[1] == 0xFF) ++q;
            if (!(q + 1 < br.end && q[0] == 0xFF && q[1] >= 0xD0 && q[1] <= 0xD7)) return JDEC_EINVAL;
            br.reset_at(q + 2);
            S.pred[0] = S.pred[1] = S.pred[2] = 0;
            S.todo = in.restart_interval;
        }
        const int mcx = static_cast<int>(mcu % mx), mcy = static_cast<int>(mcu / mx);
        for (int i = 0; i < in.ncomp; ++i) {
            const int c = P.scan_order[i];
            const HuffTable &dct = P.dc[P.td[i]], &act = P.ac[P.ta[i]];
            for (int v = 0; v < in.v_samp[c]; ++v)
                for (int h = 0; h < in.h_samp[c]; ++h) {
                    const long bx = static_cast<long>(mcx) * in.h_samp[c] + h;
                    const long by = static_cast<long>(mcy) * in.v_samp[c] + v;
                    int16_t *blk = planes[c] + 64 * (by * in.blocks_w[c] + bx);
                    memset(blk, 0, 64 * sizeof(int16_t));
                    if (br.n < 32) br.refill();
                    const int32_t fd = dct.fast[br.peek(kFast)];
                    if (fd) {
                        br.skip(fd & 0xff);
                        S.pred[c] += fd >> 16;
                    } else {
                        const int t = decode_symbol(br, dct);
                        if (t < 0 || t > 11) return JDEC_EINVAL;
                        S.pred[c] += extend(br.get(t), t);
                    }
                    blk[0] = static_cast<int16_t>(S.pred[c]);
                    for (int k = 1; k < 64; ++k) {
                        if (br.n < 32) br.refill();
                        const int32_t fa = act.fast[br.peek(kFast)];
                        if (fa) {
                            br.skip(fa & 0xff);
                            if (fa & 0x8000) break;   // end of block
                            k += (fa >> 8) & 0xff;
                            if (k > 63) return JDEC_EINVAL;
                            blk[zz[k]] = static_cast<int16_t>(fa >> 16);
                            continue;
                        }
                        const int rs = decode_symbol(br, act);
                        if (rs < 0) return JDEC_EINVAL;
                        const int r = rs >> 4, sz = rs & 15;
                        if (sz == 0) {
                            if (r == 15) {
                                k += 15;
                                continue;
                            }
                            break;
                        }
                        k += r;
                        if (k > 63 || sz > 10) return JDEC_EINVAL;
                        blk[zz[k]] = static_cast<int16_t>(extend(br.get(sz), sz));
                    }
                }
        }
        if (in.restart_interval) --S.todo;
    }
    return JDEC_OK;
}

}  // namespace

// ---- internal interface used by the pipelined decoder (jdec_pipeline.cu) ----
namespace jdec {

struct JpegScan {
    Parsed P;
    const uint8_t *data = nullptr, *end = nullptr;
    ScanState seq;                       // state of the sequential decoder
    std::vector<const uint8_t *> rst;    // start of restart interval i (i >= 1: after RST i-1)
    bool rst_indexed = false;
};

jdec_status scan_open(const uint8_t *data, size_t size, JpegScan **out, jdec_jpeg_info *info)
{
    if (!out) return JDEC_EINVAL;
    JpegScan *J = new (std::nothrow) JpegScan();
    if (!J) return JDEC_ENOMEM;
    const jdec_status st = parse(data, size, J->P, true);
    if (st != JDEC_OK) {
        delete J;
        return st;
    }
    J->data = data;
    J->end = data + size;
    J->seq.br.reset_at(J->P.scan);
    J->seq.br.end = J->end;
    J->seq.todo = J->P.info.restart_interval;
    if (info) *info = J->P.info;
    *out = J;
    return JDEC_OK;
}

void scan_close(JpegScan *J) { delete J; }

// Rows between chunk boundaries that fall on restart-interval starts (chunks
// that begin there decode independently), or 0 when the stream has no
// restart intervals.
int scan_row_step(const JpegScan *J)
{
    const long ri = J->P.info.restart_interval;
    if (ri <= 0) return 0;
    const long mx = mcus_x(J->P.info);
    long step = 1;
    while ((step * mx) % ri != 0) {
        ++step;
        if (step > 65535) return 0;
    }
    return static_cast<int>(step);
}

// Finds every restart marker of the entropy-coded segment (byte-stuffed
// 0xFF00 pairs are data; 0xFFD0..D7 start the next interval).
static void index_restarts(JpegScan *J)
{
    if (J->rst_indexed) return;
    J->rst.clear();
    J->rst.push_back(J->P.scan);
    const uint8_t *q = J->P.scan, *e = J->end;
    while (q + 1 < e) {
        q = static_cast<const uint8_t *>(memchr(q, 0xFF, static_cast<size_t>(e - q - 1)));
        if (!q) break;
        const uint8_t m = q[1];
        if (m >= 0xD0 && m <= 0xD7) {
            J->rst.push_back(q + 2);
            q += 2;
        } else if (m == 0x00 || m == 0xFF) {
            q += (m == 0x00) ? 2 : 1;
        } else {
            break;   // EOI or another marker ends the scan
        }
    }
    J->rst_indexed = true;
}

// Decodes MCU rows [r0, r1) into the full-size planes.  independent = false:
// continue the sequential decoder (rows must follow the previous call's);
// true: start afresh at the restart interval that begins at row r0 (r0 a
// multiple of scan_row_step; safe to run concurrently with other
// independent calls on disjoint rows).
jdec_status scan_decode_rows(JpegScan *J, int16_t *const planes[3], int r0, int r1, bool independent)
{
    const jdec_jpeg_info &in = J->P.info;
    const long mx = mcus_x(in);
    if (r0 < 0 || r1 > mcus_y(in) || r0 > r1) return JDEC_EINVAL;
    for (int c = 0; c < in.ncomp; ++c)
        if (!planes[c]) return JDEC_EINVAL;
    if (!independent) return decode_mcus(J->P, J->seq, planes, r0 * mx, r1 * mx);
    const long ri = in.restart_interval;
    if (ri <= 0 || (r0 * mx) % ri != 0) return JDEC_EINVAL;
    const long interval = r0 * mx / ri;
    if (interval >= static_cast<long>(J->rst.size())) return JDEC_EINVAL;
    ScanState S;
    S.br.reset_at(J->rst[interval]);
    S.br.end = J->end;
    S.todo = ri;
    return decode_mcus(J->P, S, planes, r0 * mx, r1 * mx);
}

// Builds the restart index (call once before concurrent independent calls).
jdec_status scan_prepare_independent(JpegScan *J)
{
    if (J->P.info.restart_interval <= 0) return JDEC_EINVAL;
    index_restarts(J);
    return JDEC_OK;
}

}  // namespace jdec

extern "C" {

JDEC_API jdec_status jdec_jpeg_parse(const uint8_t *data, size_t size, jdec_jpeg_info *info)
{
    if (!info) return JDEC_EINVAL;
    Parsed *P = new (std::nothrow) Parsed();
    if (!P) return JDEC_ENOMEM;
    const jdec_status st = parse(data, size, *P, false);
    if (st == JDEC_OK) *info = P->info;
    delete P;
    return st;
}

JDEC_API jdec_status jdec_entropy_decode(const uint8_t *data, size_t size, int16_t *const planes[3])
{
    if (!planes || !planes[0]) return JDEC_EINVAL;
    jdec::JpegScan *J = nullptr;
    jdec_jpeg_info info;
    jdec_status st = jdec::scan_open(data, size, &J, &info);
    if (st != JDEC_OK) return st;
    st = jdec::scan_decode_rows(J, planes, 0, mcus_y(info), false);
    jdec::scan_close(J);
    return st;
}

JDEC_API jdec_status jdec_entropy_decode_mt(const uint8_t *data, size_t size, int16_t *const planes[3],
                                            int32_t threads)
{
    if (!planes || !planes[0]) return JDEC_EINVAL;
    jdec::JpegScan *J = nullptr;
    jdec_jpeg_info info;
    jdec_status st = jdec::scan_open(data, size, &J, &info);
    if (st != JDEC_OK) return st;
    const int my = mcus_y(info);
    const int step = jdec::scan_row_step(J);
    if (threads <= 1 || step <= 0 || step >= my || jdec::scan_prepare_independent(J) != JDEC_OK) {
        st = jdec::scan_decode_rows(J, planes, 0, my, false);
        jdec::scan_close(J);
        return st;
    }
    // chunks of whole restart-aligned row groups, several per thread
    const int want = std::max(1, my / (4 * threads));
    const int chunk = std::max(step, (want + step - 1) / step * step);
    const int nch = (my + chunk - 1) / chunk;
    std::atomic<int> next{0};
    std::atomic<int> err{0};
    std::vector<std::thread> pool;
    for (int w = 0; w < std::min(threads, nch); ++w)
        pool.emplace_back([&]() {
            for (int k; (k = next.fetch_add(1)) < nch;) {
                const int r0 = k * chunk, r1 = std::min(my, r0 + chunk);
                const jdec_status r = jdec::scan_decode_rows(J, planes, r0, r1, true);
                if (r != JDEC_OK) err.store(static_cast<int>(r));
            }
        });
    for (auto &t : pool) t.join();
    jdec::scan_close(J);
    return static_cast<jdec_status>(err.load());
}

}  // extern "C"
