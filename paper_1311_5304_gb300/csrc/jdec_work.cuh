// jdec_work.cuh -- one work item of the fused back-end: a strip of `wt`
// MCUs walked down a chunk of MCU rows (Sec. 2 MCU tiling; Sec. 4.1-4.3
// stages fused into one pass, Sec. 4.4).
//
// The CTA is split into two warp groups that run as a two-deep pipeline over
// the item's "jobs" (one job per MCU row, plus two chroma-only jobs at the top
// of a 4:2:0 triangular-filtering item):
//   IDCT warps   wait for the job's TMA tile (mbarrier), dequantise + IDCT one
//                block per thread into shared sample planes, refill the TMA
//                stage with the tile two jobs ahead, replicate the true chroma
//                edge into halo columns at image edges, signal FULL[job % 2];
//   colour warps wait FULL[job % 2], upsample chroma and convert 8 pixels of
//                one output row per task to RGB with 8-byte vector stores,
//                signal EMPTY[job % 2].
// The IDCT warps wait EMPTY[job % 2] before overwriting the planes of job-2.
// Luma planes are double-buffered; chroma rows go to a ring of four slots in
// job order, so a 4:2:0 triangular filter finds chroma rows r-1, r, r+1 in
// the three most recent slots and every chroma block is transformed once per
// item (the row above the item is recomputed once).
#pragma once

#include "jdec_device.cuh"

namespace jdec {

enum : int { kBarIdct = 1, kBarFull0 = 2, kBarEmpty0 = 4 };

// The per-image values the work loops use, held in registers for the whole
// item (the batched kernel's descriptors live in global memory).
struct ItemDesc {
    uint8_t *rgb;
    int64_t pitch;
    int W, H, cw, ch, mcus_x, mcus_y, wt, nidct;
    bool aligned8, withhold;
};

__device__ __forceinline__ ItemDesc item_desc(const ImageDesc &d)
{
    ItemDesc t;
    t.rgb = d.rgb;
    t.pitch = d.pitch;
    t.W = d.W; t.H = d.H; t.cw = d.cw; t.ch = d.ch;
    t.mcus_x = d.mcus_x; t.mcus_y = d.mcus_y; t.wt = d.wt; t.nidct = d.nidct;
    t.aligned8 = d.aligned8 != 0;
    t.withhold = d.withhold != 0;
    return t;
}

struct PipeState {
    uint32_t parity;   // bit s = parity of the next completion of stage s
    int job;           // jobs started by this CTA (all items)
    int sync_from;     // first job whose colour warps signal EMPTY (split roles)
};


template <int HM, int VM, bool FANCY>
struct Variant {
    static constexpr bool kHalo = FANCY && HM == 2;            // horizontal neighbours
    static constexpr bool kRing = FANCY && VM == 2;            // vertical neighbours
    static constexpr int kLA = kRing ? 1 : 0;                  // chroma lookahead rows
    static constexpr int kPro = kRing ? 2 : 0;                 // chroma-only jobs per item
    // every warp may transform and then convert each job (triangular 4:2:2
    // and 4:2:0, where colour work is close to IDCT work; faster on full-width
    // strips of large images); else split warp roles
    static constexpr bool kCanUnify = FANCY && HM == 2;
};

// Job k of an item covering MCU rows [r0, r1): its luma row (-1: none) and
// chroma row.
template <int HM, int VM, bool FANCY>
__device__ __forceinline__ void job_rows(int k, int r0, int &yrow, int &crow)
{
    using V = Variant<HM, VM, FANCY>;
    if (k < V::kPro) {
        yrow = -1;
        crow = r0 - 1 + k;
    } else {
        yrow = r0 + k - V::kPro;
        crow = yrow + V::kLA;
    }
}

// Issues the TMA loads of one job into a stage.  Called by one thread.
// `withhold` (testing aid): arm the barrier for the bytes but issue no load,
// so the job's bounded wait runs out.
template <int HM, int VM, bool FANCY>
__device__ __forceinline__ void issue_job(const CUtensorMap *tm, const SmemLayout &L, uint8_t *stage, uint32_t bar,
                                          int mx0, int yrow, int crow, int mcus_y, bool withhold)
{
    using V = Variant<HM, VM, FANCY>;
    const bool do_y = yrow >= 0;
    const bool do_c = crow >= 0 && crow < mcus_y;
    const uint32_t bytes = (do_y ? L.ny * 128 : 0) + (do_c ? 2 * L.nc * 128 : 0);
    mbar_arrive_expect_tx(bar, bytes);
    if (withhold) return;
    if (do_y) tma_load_3d(smem_u32(stage + L.stage_y), &tm[0], bar, 0, mx0 * HM, yrow * VM);
    if (do_c) {
        tma_load_3d(smem_u32(stage + L.stage_c), &tm[1], bar, 0, mx0 - (V::kHalo ? 1 : 0), crow);
        tma_load_3d(smem_u32(stage + L.stage_c + L.cbytes), &tm[2], bar, 0, mx0 - (V::kHalo ? 1 : 0), crow);
    }
}

// Colour conversion of 16 pixels of one row when every pixel has its own
// chroma sample (4:4:4, and 4:4:0 with replication): Cb bytes at cb, Cr bytes
// `cstep` after them, luma at yrow; n1 pixels of the first 8-pixel group and
// n2 (0: none) of the second are written to out.  Samples minus 128 are the
// signed bytes of the words XOR 0x80808080.
__device__ __forceinline__ void row_convert_h1(const uint8_t *cb, int cstep, const uint8_t *yrow, uint8_t *out,
                                               int n1, int n2, bool vec)
{
    uint4 wb = *reinterpret_cast<const uint4 *>(cb);
    uint4 wr = *reinterpret_cast<const uint4 *>(cb + cstep);
    wb.x ^= 0x80808080u; wb.y ^= 0x80808080u; wb.z ^= 0x80808080u; wb.w ^= 0x80808080u;
    wr.x ^= 0x80808080u; wr.y ^= 0x80808080u; wr.z ^= 0x80808080u; wr.w ^= 0x80808080u;
    int Cb[2][8], Cr[2][8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        Cb[0][k] = sbyte_of(wb.x, k); Cb[0][4 + k] = sbyte_of(wb.y, k);
        Cb[1][k] = sbyte_of(wb.z, k); Cb[1][4 + k] = sbyte_of(wb.w, k);
        Cr[0][k] = sbyte_of(wr.x, k); Cr[0][4 + k] = sbyte_of(wr.y, k);
        Cr[1][k] = sbyte_of(wr.z, k); Cr[1][4 + k] = sbyte_of(wr.w, k);
    }
    const uint2 y0 = *reinterpret_cast<const uint2 *>(yrow);
    cc_store8(y0, Cb[0], Cr[0], out, n1, vec);
    if (n2 > 0) {
        const uint2 y1 = *reinterpret_cast<const uint2 *>(yrow + 8);
        cc_store8(y1, Cb[1], Cr[1], out + 24, n2, vec);
    }
}

// ---------------------------------------------------------------------------
// colour warps: one task = 16 pixels (two 8-pixel groups) of one output row
// ---------------------------------------------------------------------------
// CLEAN: the image's rows are 8-byte aligned and its width a multiple of 8,
// so every 8-pixel group inside the image is whole and stored with aligned
// 8-byte stores (no partial or unaligned path in the code).
template <int HM, int VM, bool FANCY, bool CLEAN = false>
__device__ __forceinline__ void cc_task(const ItemDesc &d, const SmemLayout &L, const uint8_t *yplane,
                                        const uint8_t *cslots, int job, int r, int mx0, int wte, int py, int gt)
{
    const int xg = (mx0 * HM + 2 * gt) * 8;
    const int y = r * 8 * VM + py;
    if (xg >= d.W || y >= d.H) return;
    const bool vec = CLEAN || d.aligned8;
    const uint8_t *yrow = yplane + py * L.ypitch + 16 * gt;
    uint8_t *out = d.rgb + static_cast<int64_t>(y) * d.pitch + 3 * xg;
    const uint8_t *slot = cslots + (job & (L.nslot - 1)) * L.slot_bytes;
    int Cb[2][8], Cr[2][8];
    if (HM == 1) {
        // 4:4:4: chroma sample = pixel; 4:4:0 replication: chroma row y/2
        const uint8_t *cb = slot + (VM == 2 ? (py >> 1) : py) * L.lc + 16 * gt;
        const bool two = 2 * gt + 1 < HM * wte && xg + 8 < d.W;
        row_convert_h1(cb, 8 * L.lc, yrow, out, CLEAN ? 8 : min(8, d.W - xg), two ? (CLEAN ? 8 : min(8, d.W - xg - 8)) : 0,
                       vec);
        return;
    } else if (!FANCY) {
        // replication: chroma sample (x/2, y/VM), minus 128 as above
        const uint8_t *cb = slot + (VM == 2 ? (py >> 1) : py) * L.lc + 8 * gt;
        uint2 wb = *reinterpret_cast<const uint2 *>(cb);
        uint2 wr = *reinterpret_cast<const uint2 *>(cb + 8 * L.lc);
        wb.x ^= 0x80808080u; wb.y ^= 0x80808080u;
        wr.x ^= 0x80808080u; wr.y ^= 0x80808080u;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            Cb[0][2 * k] = Cb[0][2 * k + 1] = sbyte_of(wb.x, k);
            Cb[1][2 * k] = Cb[1][2 * k + 1] = sbyte_of(wb.y, k);
            Cr[0][2 * k] = Cr[0][2 * k + 1] = sbyte_of(wr.x, k);
            Cr[1][2 * k] = Cr[1][2 * k + 1] = sbyte_of(wr.y, k);
        }
    } else {
        // h2v1 triangular (Alg. 1); the slot row starts one halo block left
        const uint8_t *cb = slot + py * L.lc + 8 + 8 * gt;
        int c10[10];
        load10(cb, c10);
        tri_h2v1(c10, Cb[0]);
        tri_h2v1(c10 + 4, Cb[1]);
        load10(cb + 8 * L.lc, c10);
        tri_h2v1(c10, Cr[0]);
        tri_h2v1(c10 + 4, Cr[1]);
    }
    const uint2 y0 = *reinterpret_cast<const uint2 *>(yrow);
    cc_store8(y0, Cb[0], Cr[0], out, CLEAN ? 8 : min(8, d.W - xg), vec);
    // the second group may lie past the strip (odd group count) or the image
    if (2 * gt + 1 < HM * wte && xg + 8 < d.W) {
        const uint2 y1 = *reinterpret_cast<const uint2 *>(yrow + 8);
        cc_store8(y1, Cb[1], Cr[1], out + 24, CLEAN ? 8 : min(8, d.W - xg - 8), vec);
    }
}

// 4:2:0 triangular colour conversion of 8 pixels of two output rows: chroma
// near row at pn, far rows at pu (upper output row) and pd (lower), the Cr
// rows `cstep` bytes after the Cb rows; luma at yp and yp + ypitch; RGB to
// out and out + pitch (the second row only when `row2`); n pixels per row.
__device__ __forceinline__ void pair_convert_h2v2(const uint8_t *pn, const uint8_t *pu, const uint8_t *pd, int cstep,
                                                  const uint8_t *yp, int ypitch, uint8_t *out, int64_t pitch, int n,
                                                  bool vec, bool row2)
{
    const uint2 y0 = *reinterpret_cast<const uint2 *>(yp);
    const uint2 y1 = *reinterpret_cast<const uint2 *>(yp + ypitch);
    int Cb0[8], Cr0[8], Cb1[8], Cr1[8];
#pragma unroll
    for (int comp = 0; comp < 2; ++comp) {
        const int o = comp * cstep;
        const uint32_t *wn = reinterpret_cast<const uint32_t *>(pn + o);
        const uint32_t *wu = reinterpret_cast<const uint32_t *>(pu + o);
        const uint32_t *wd = reinterpret_cast<const uint32_t *>(pd + o);
        uint32_t ne, no, nl, nr;
        lanes4(wn[-1], wn[0], wn[1], ne, no, nl, nr);
        tri_h2v2_pairs(ne, no, nl, nr, wu[-1], wu[0], wu[1], comp ? Cr0 : Cb0);
        tri_h2v2_pairs(ne, no, nl, nr, wd[-1], wd[0], wd[1], comp ? Cr1 : Cb1);
    }
    cc_store8(y0, Cb0, Cr0, out, n, vec);
    if (row2) cc_store8(y1, Cb1, Cr1, out + pitch, n, vec);
}

// 4:2:0 triangular filtering: one task = 8 pixels of the two output rows
// 2m and 2m+1 of MCU row r, which share the near chroma row j = 8r + m; the
// far rows are j-1 (row 2m) and j+1 (row 2m+1), clamped to the image.  Chroma
// block row r lives in slot (job - 1) & 3, the rows above and below it in
// (job - 2) & 3 and job & 3.
template <bool CLEAN = false>
__device__ __forceinline__ void cc_task_h2v2_pair(const ItemDesc &d, const SmemLayout &L, const uint8_t *yplane,
                                                  const uint8_t *cslots, int job, int r, int mx0, int m, int g)
{
    const int x0 = (2 * mx0 + g) * 8;
    const int y = 16 * r + 2 * m;
    if (x0 >= d.W || y >= d.H) return;
    const int n = CLEAN ? 8 : min(8, d.W - x0);
    const bool vec = CLEAN || d.aligned8;
    const int j = 8 * r + m;
    const uint8_t *slot = cslots + ((job - 1) & 3) * L.slot_bytes;
    const uint8_t *pn = slot + m * L.lc + 8 + 4 * g;
    const uint8_t *pu = m > 0 ? pn - L.lc
                      : (j > 0 ? cslots + ((job - 2) & 3) * L.slot_bytes + 7 * L.lc + 8 + 4 * g : pn);
    const uint8_t *pd = j + 1 >= d.ch ? pn
                      : (m < 7 ? pn + L.lc : cslots + (job & 3) * L.slot_bytes + 8 + 4 * g);
    uint8_t *out = d.rgb + static_cast<int64_t>(y) * d.pitch + 3 * x0;
    pair_convert_h2v2(pn, pu, pd, 8 * L.lc, yplane + 2 * m * L.ypitch + 8 * g, L.ypitch, out, d.pitch, n, vec,
                      y + 1 < d.H);
}

// 4:4:0 triangular filtering (Alg. 1 along columns): one task = 8 pixels of
// output rows 2m and 2m+1 of MCU row r, near chroma row j = 8r + m, far rows
// j-1 and j+1 clamped to the image; the slots rotate as in the 4:2:0 pair
// task.  No horizontal filter: chroma column = pixel column.
template <bool CLEAN = false>
__device__ __forceinline__ void cc_task_h1v2_pair(const ItemDesc &d, const SmemLayout &L, const uint8_t *yplane,
                                                  const uint8_t *cslots, int job, int r, int mx0, int m, int g)
{
    const int x0 = (mx0 + g) * 8;
    const int y = 16 * r + 2 * m;
    if (x0 >= d.W || y >= d.H) return;
    const int n = CLEAN ? 8 : min(8, d.W - x0);
    const bool vec = CLEAN || d.aligned8;
    const int j = 8 * r + m;
    const uint8_t *slot = cslots + ((job - 1) & 3) * L.slot_bytes;
    const uint8_t *pn = slot + m * L.lc + 8 * g;
    const uint8_t *pu = m > 0 ? pn - L.lc
                      : (j > 0 ? cslots + ((job - 2) & 3) * L.slot_bytes + 7 * L.lc + 8 * g : pn);
    const uint8_t *pd = j + 1 >= d.ch ? pn
                      : (m < 7 ? pn + L.lc : cslots + (job & 3) * L.slot_bytes + 8 * g);
    const uint2 y0 = *reinterpret_cast<const uint2 *>(yplane + 2 * m * L.ypitch + 8 * g);
    const uint2 y1 = *reinterpret_cast<const uint2 *>(yplane + (2 * m + 1) * L.ypitch + 8 * g);
    int Cb0[8], Cr0[8], Cb1[8], Cr1[8];
#pragma unroll
    for (int comp = 0; comp < 2; ++comp) {
        const int off = comp * 8 * L.lc;
        const uint2 wn = *reinterpret_cast<const uint2 *>(pn + off);
        const uint2 wu = *reinterpret_cast<const uint2 *>(pu + off);
        const uint2 wd = *reinterpret_cast<const uint2 *>(pd + off);
        int *c0 = comp ? Cr0 : Cb0, *c1 = comp ? Cr1 : Cb1;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t sel = k < 4 ? 0 : 1;
            const int near = 3 * byte_of(sel ? wn.y : wn.x, k & 3);
            // minus 128: (x - 512) >> 2 = (x >> 2) - 128
            c0[k] = (near + byte_of(sel ? wu.y : wu.x, k & 3) + 1 - 512) >> 2;
            c1[k] = (near + byte_of(sel ? wd.y : wd.x, k & 3) + 2 - 512) >> 2;
        }
    }
    uint8_t *out = d.rgb + static_cast<int64_t>(y) * d.pitch + 3 * x0;
    cc_store8(y0, Cb0, Cr0, out, n, vec);
    if (y + 1 < d.H) cc_store8(y1, Cb1, Cr1, out + d.pitch, n, vec);
}

// Replicates the true chroma edge into halo/padding columns of the 8 rows of
// both components of one chroma slot (strips at the image's left or right
// edge only, triangular filtering only).  Thread `tid` < 16 does one row.
__device__ __forceinline__ void fix_edges(uint8_t *slot, int lc, int mx0, int cw, int used, int tid)
{
    if (tid >= 16) return;
    uint8_t *row = slot + tid * lc;     // rows 0..7: Cb, 8..15: Cr
    if (mx0 == 0) {
        const uint8_t v = row[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) row[k] = v;
    }
    const int lce = cw + 7 - 8 * mx0;   // local column of the last true sample
    if (lce < used - 1) {
        const uint8_t v = row[lce];
        for (int k = lce + 1; k < used; ++k) row[k] = v;
    }
}

// Runs one work item (MCU rows [r0, r1) of one strip) with the whole CTA.
// `smem` is 1024-byte aligned; L is the shared-memory layout.  Returns false
// if a bounded wait gave up (the error word has been set; the CTA must stop).
// `last` = this is the CTA's final item (drain barriers); `reload_q` = load
// this image's dequantisation tables first.
// Writes the dequantisation tables of `d` into shared memory in the layout the
// IDCT expects (packed bytes for dp2a, or transposed int32).
template <int QM>
__device__ __forceinline__ void load_qtables(int *qs, const ImageDesc &d, int tid, int nthreads)
{
    if (QM == kQ8) {
        // word 64*c + 8*pr + v = Q_c(v, 2pr) | Q_c(v, 2pr+1) << 24
        for (int i = tid; i < 96; i += nthreads) {
            const int c = i >> 5, pr = (i >> 3) & 3, v = i & 7;
            qs[64 * c + 8 * pr + v] = d.q[c][8 * v + 2 * pr] | (d.q[c][8 * v + 2 * pr + 1] << 24);
        }
    } else {
        // qs[64*c + 8*u + v] = Q_c(v, u) (prescaled for the AAN transform)
        for (int i = tid; i < 192; i += nthreads) qs[i] = d.q[i >> 6][((i & 7) << 3) | ((i >> 3) & 7)];
    }
}

// One dequantisation + IDCT task (block at shared address blk -> samples at
// dst); EVEN_ALU as for idct8 (the LLM forms).
template <int QM, bool EVEN_ALU = false>
__device__ __forceinline__ void idct_task(uint32_t blk, const int *q, uint8_t *dst, int pitch)
{
    if (QM == kQ8)
        idct_block_q8<EVEN_ALU>(blk, reinterpret_cast<const uint32_t *>(q), dst, pitch);
    else if (QM == kAAN)
        idct_block_aan(blk, q, dst, pitch);
    else
        idct_block<EVEN_ALU>(blk, q, dst, pitch);
}

// The IDCT tasks of one job on threads [0, nthr) (this thread: tid), any
// strip width: luma blocks (nye, rows of HM * wte) when has_y, then chroma
// blocks [lb0, lb0 + nce) of both components when has_c.
template <int HM, int VM, bool FANCY, int QM>
__device__ __forceinline__ void idct_job(uint8_t *stage, uint8_t *yplane, uint8_t *slot, const int *qs,
                                         const SmemLayout &L, bool has_y, bool has_c, int nye, int nce, int lb0,
                                         int wt, int wte, int tid, int nthr)
{
    const int ntask = (has_y ? nye : 0) + (has_c ? 2 * nce : 0);
    for (int t = tid; t < ntask; t += nthr) {
        uint32_t blk;
        const int *q;
        uint8_t *dst;
        int pitch;
        int tc = t;
        if (has_y && t < nye) {
            const int vy = t / (HM * wte), bx = t - vy * (HM * wte);
            blk = smem_u32(stage + L.stage_y + (vy * HM * wt + bx) * 128);
            q = qs;
            dst = yplane + 8 * vy * L.ypitch + 8 * bx;
            pitch = L.ypitch;
        } else {
            if (has_y) tc -= nye;
            const int comp = tc >= nce;
            const int lb = lb0 + (comp ? tc - nce : tc);
            blk = smem_u32(stage + L.stage_c + comp * L.cbytes + lb * 128);
            q = qs + 64 * (1 + comp);
            dst = slot + comp * 8 * L.lc + 8 * lb;
            pitch = L.lc;
        }
        idct_task<QM, HM == 1 && VM == 1>(blk, q, dst, pitch);
    }
}

// The same for strips of exactly FW MCUs (compile-time width) on NT threads:
// every chroma block of the TMA box is transformed, halo blocks included (at
// the image's edges they hold zero-filled blocks, whose samples the edge
// replication then overwrites), so the task list is the same for every job:
// luma tasks 0 .. NY-1, chroma NY .. NY + 2 NC - 1.  Each thread's tasks
// (t = tid + i NT) and their shared-memory offsets are worked out once.
template <int HM, int VM, bool FANCY, int QM, int FW, int NT>
struct FixedIdct {
    static constexpr int kHalo = Variant<HM, VM, FANCY>::kHalo ? 1 : 0;
    static constexpr int NY = HM * VM * FW;
    static constexpr int NC = FW + 2 * kHalo;
    static constexpr int NTASK = NY + 2 * NC;
    static constexpr int NS = (NTASK + NT - 1) / NT;
    uint32_t src[NS];   // offset of the block in a stage
    uint32_t dst[NS];   // offset of the samples in the luma plane (luma) or the chroma slot
    int pitch[NS];
    int qoff[NS];

    __device__ __forceinline__ void init(const SmemLayout &L, int tid)
    {
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            const int t = tid + i * NT;
            if (t < NY) {
                const int vy = t / (HM * FW), bx = t - vy * (HM * FW);
                src[i] = L.stage_y + 128 * t;
                dst[i] = 8 * vy * L.ypitch + 8 * bx;
                pitch[i] = L.ypitch;
                qoff[i] = 0;
            } else {
                const int tc = t - NY;
                const int comp = tc >= NC;
                const int lb = comp ? tc - NC : tc;
                src[i] = L.stage_c + comp * L.cbytes + 128 * lb;
                dst[i] = comp * 8 * L.lc + 8 * lb;
                pitch[i] = L.lc;
                qoff[i] = 64 * (1 + comp);
            }
        }
    }

    __device__ __forceinline__ void run(uint8_t *stage, uint8_t *yplane, uint8_t *slot, const int *qs, bool has_y,
                                        bool has_c, int tid) const
    {
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            const int t = tid + i * NT;
            if (t >= NTASK) break;
            const bool luma = t < NY;
            if (luma ? !has_y : !has_c) continue;
            idct_task<QM, HM == 1 && VM == 1>(smem_u32(stage + src[i]), qs + qoff[i], (luma ? yplane : slot) + dst[i],
                                              pitch[i]);
        }
    }
};

// FW > 0: the strip is decoded as exactly FW MCUs wide (d.wt == FW; a last
// strip that reaches past the image's right edge is padded, see run_share), L
// is the layout for width FW, kFixedIdctThreads threads transform: task lists
// and offsets are compile-time (FixedIdct); the image is CLEAN (see cc_task:
// aligned rows, width a multiple of 8).  FW = 0: any strip, any image.
template <int HM, int VM, bool FANCY, int QM, int FW = 0>
__device__ bool run_work_split(const CUtensorMap *tm, const ItemDesc d, const ImageDesc &qsrc, int strip, int r0,
                               int r1, uint8_t *smem, const SmemLayout &L, PipeState &ps, int *err, bool last,
                               bool reload_q)
{
    using V = Variant<HM, VM, FANCY>;
    const int tid = threadIdx.x;
    const int wt = FW ? FW : d.wt;
    const int mx0 = strip * wt;
    const int wte = FW ? FW : min(wt, d.mcus_x - mx0);
    if (r0 >= r1 || wte <= 0) return true;
    const int njobs = V::kPro + (r1 - r0);
    const int J0 = ps.job;

    uint8_t *stages = smem + L.off_stage;
    uint8_t *yplanes = smem + L.off_y;
    uint8_t *cslots = smem + L.off_c;
    const uint32_t bar0 = smem_u32(smem + L.off_bar);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + L.off_flag);

    const int nidct = FW ? kFixedIdctThreads : d.nidct, ncc = kCtaThreads - nidct;
    if (tid < nidct) {
        // =================== IDCT warps ===================
        int *qs = reinterpret_cast<int *>(smem + L.off_q);
        if (reload_q) {
            // every IDCT thread is past its last use of the previous tables
            load_qtables<QM>(qs, qsrc, tid, nidct);
            named_sync(kBarIdct, nidct);
        }
        const int lb0 = (!FW && V::kHalo && mx0 == 0) ? 1 : 0;
        const int lb1 = FW ? FW + (V::kHalo ? 2 : 0)
                           : min(wte + (V::kHalo ? 2 : 0), d.mcus_x - (mx0 - (V::kHalo ? 1 : 0)));
        const int nce = lb1 - lb0;
        const int nye = VM * HM * wte;
        const int used = 8 * (wte + (V::kHalo ? 2 : 0));
        const bool edge = V::kHalo && (mx0 == 0 || d.cw + 7 - 8 * mx0 < used - 1);
        const uint64_t budget = 2000000000ull;   // 2 s per wait
        FixedIdct<HM, VM, FANCY, QM, FW ? FW : 1, kFixedIdctThreads> fx;
        if (FW) fx.init(L, tid);

        if (tid == 0) {
            fence_proxy_async_smem();
            for (int k = 0; k < 2 && k < njobs; ++k) {
                int yr, cr;
                job_rows<HM, VM, FANCY>(k, r0, yr, cr);
                const int s = (J0 + k) & 1;
                issue_job<HM, VM, FANCY>(tm, L, stages + s * L.stage_bytes, bar0 + 8 * s, mx0, yr, cr, d.mcus_y,
                                          d.withhold);
            }
        }
        for (int k = 0; k < njobs; ++k) {
            const int j = J0 + k, s = j & 1;
            int yrow, crow;
            job_rows<HM, VM, FANCY>(k, r0, yrow, crow);
            const bool do_c = crow >= 0 && crow < d.mcus_y;
            if (j >= ps.sync_from + 2) named_sync(kBarEmpty0 + s, kCtaThreads);
            const bool ok = mbar_wait_bounded(bar0 + 8 * s, (ps.parity >> s) & 1u, budget);
            ps.parity ^= 1u << s;
            if (!ok) *abort_flag = 1;
            uint8_t *stage = stages + s * L.stage_bytes;
            uint8_t *yplane = yplanes + s * L.ybytes;
            uint8_t *slot = cslots + (j & (L.nslot - 1)) * L.slot_bytes;
            if (ok) {
                if (FW)
                    fx.run(stage, yplane, slot, qs, yrow >= 0, do_c, tid);
                else
                    idct_job<HM, VM, FANCY, QM>(stage, yplane, slot, qs, L, yrow >= 0, do_c, nye, nce, lb0, wt, wte,
                                                tid, nidct);
            }
            named_sync(kBarIdct, nidct);
            if (*abort_flag) {
                if (tid == 0) {
                    atomicExch(err, kErrTimeout);
                    // the other stage may still have a copy in flight: wait for it (bounded)
                    if (k + 1 < njobs) mbar_wait_bounded(bar0 + 8 * (s ^ 1), (ps.parity >> (s ^ 1)) & 1u, budget);
                }
                named_arrive(kBarFull0 + s, kCtaThreads);
                return false;
            }
            if (tid == 0 && k + 2 < njobs) {
                int yr, cr;
                job_rows<HM, VM, FANCY>(k + 2, r0, yr, cr);
                fence_proxy_async_smem();
                issue_job<HM, VM, FANCY>(tm, L, stage, bar0 + 8 * s, mx0, yr, cr, d.mcus_y, d.withhold);
            }
            if (edge && do_c) fix_edges(slot, L.lc, mx0, d.cw, used, tid);
            named_arrive(kBarFull0 + s, kCtaThreads);
        }
        ps.job = J0 + njobs;
        if (last) {
            // consume the colour warps' EMPTY signals of the final two jobs, as
            // jobs ps.job and ps.job + 1 would
            for (int jj = ps.job; jj < ps.job + 2; ++jj)
                if (jj >= ps.sync_from + 2) named_sync(kBarEmpty0 + (jj & 1), kCtaThreads);
            ps.sync_from = ps.job;
        }
    } else {
        // =================== colour warps ===================
        const int tc = tid - nidct;
        // tasks: 4:2:0 and 4:4:0 triangular, 8 pixels of a pair of output rows; else
        // 16 pixels of one output row
        const int ngroups = V::kRing ? HM * wte : (HM * wte + 1) >> 1;
        const int rows = V::kRing ? 8 : 8 * VM;
        // this thread's first task (row, group) and the per-step advance
        const int py0 = tc / ngroups, g0 = tc - py0 * ngroups;
        const int dpy = ncc / ngroups, dg = ncc - dpy * ngroups;
        for (int k = 0; k < njobs; ++k) {
            const int j = J0 + k, s = j & 1;
            // keep this thread's copy of the stage parities in step with the
            // IDCT warps' (a unified-role item may follow)
            ps.parity ^= 1u << s;
            named_sync(kBarFull0 + s, kCtaThreads);
            if (*abort_flag) return false;
            if (k >= V::kPro) {
                const int r = r0 + k - V::kPro;
                const uint8_t *yplane = yplanes + s * L.ybytes;
                int py = py0, g = g0;
                while (py < rows) {
                    if (V::kRing && HM == 2)
                        cc_task_h2v2_pair<FW != 0>(d, L, yplane, cslots, j, r, mx0, py, g);
                    else if (V::kRing)
                        cc_task_h1v2_pair<FW != 0>(d, L, yplane, cslots, j, r, mx0, py, g);
                    else
                        cc_task<HM, VM, FANCY, FW != 0>(d, L, yplane, cslots, j, r, mx0, wte, py, g);
                    py += dpy;
                    g += dg;
                    if (g >= ngroups) { g -= ngroups; ++py; }
                }
            }
            named_arrive(kBarEmpty0 + s, kCtaThreads);
        }
        ps.job = J0 + njobs;
        if (last) ps.sync_from = ps.job;
    }
    return true;
}

// Unified roles: every thread takes part in both halves of every job k:
//   wait for job k's TMA tile; IDCT tasks of job k; CTA barrier;
//   (thread 0 refills the consumed stage with job k+2; edge strips replicate
//   the true chroma edge, then a second barrier); colour tasks of job k.
// One barrier per job suffices: a thread that starts the IDCT of job k+1 may
// overlap slower threads' colour tasks of job k because luma planes are
// double-buffered and chroma slots rotate (job k+1 writes neither the plane
// nor the slots that job k reads), and a thread that starts job k+2 has passed
// the barrier of job k+1, which every thread reaches only after finishing the
// colour tasks of job k.  No named barrier is left half-signalled, so an item
// of either kind may follow.
// FW as for run_work_split (all 128 threads transform).
template <int HM, int VM, bool FANCY, int QM, int FW = 0>
__device__ bool run_work_unified(const CUtensorMap *tm, const ItemDesc d, const ImageDesc &qsrc, int strip, int r0,
                                 int r1, uint8_t *smem, const SmemLayout &L, PipeState &ps, int *err, bool reload_q)
{
    using V = Variant<HM, VM, FANCY>;
    const int tid = threadIdx.x;
    const int wt = FW ? FW : d.wt;
    const int mx0 = strip * wt;
    const int wte = FW ? FW : min(wt, d.mcus_x - mx0);
    if (r0 >= r1 || wte <= 0) return true;
    const int njobs = V::kPro + (r1 - r0);
    const int J0 = ps.job;

    uint8_t *stages = smem + L.off_stage;
    uint8_t *yplanes = smem + L.off_y;
    uint8_t *cslots = smem + L.off_c;
    const uint32_t bar0 = smem_u32(smem + L.off_bar);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + L.off_flag);
    int *qs = reinterpret_cast<int *>(smem + L.off_q);
    if (reload_q) {
        // every thread is past the barrier that follows the previous item's
        // last IDCT tasks, so nobody reads the old tables any more
        load_qtables<QM>(qs, qsrc, tid, kCtaThreads);
        __syncthreads();
    }
    const int lb0 = (!FW && V::kHalo && mx0 == 0) ? 1 : 0;
    const int lb1 = FW ? FW + (V::kHalo ? 2 : 0) : min(wte + (V::kHalo ? 2 : 0), d.mcus_x - (mx0 - (V::kHalo ? 1 : 0)));
    const int nce = lb1 - lb0;
    const int nye = VM * HM * wte;
    const int used = 8 * (wte + (V::kHalo ? 2 : 0));
    const bool edge = V::kHalo && (mx0 == 0 || d.cw + 7 - 8 * mx0 < used - 1);
    const uint64_t budget = 2000000000ull;   // 2 s per wait
    FixedIdct<HM, VM, FANCY, QM, FW ? FW : 1, kCtaThreads> fx;
    if (FW) fx.init(L, tid);

    if (tid == 0) {
        // the stages were consumed before the barrier of the previous job
        fence_proxy_async_smem();
        for (int k = 0; k < 2 && k < njobs; ++k) {
            int yr, cr;
            job_rows<HM, VM, FANCY>(k, r0, yr, cr);
            const int s = (J0 + k) & 1;
            issue_job<HM, VM, FANCY>(tm, L, stages + s * L.stage_bytes, bar0 + 8 * s, mx0, yr, cr, d.mcus_y,
                                          d.withhold);
        }
    }
    // colour tasks (see the split version); this thread's first task and the
    // per-step advance
    const int ngroups = V::kRing ? HM * wte : (HM * wte + 1) >> 1;
    const int rows = V::kRing ? 8 : 8 * VM;
    const int py0 = tid / ngroups, g0 = tid - py0 * ngroups;
    const int dpy = kCtaThreads / ngroups, dg = kCtaThreads - dpy * ngroups;

    for (int k = 0; k < njobs; ++k) {
        const int j = J0 + k, s = j & 1;
        int yrow, crow;
        job_rows<HM, VM, FANCY>(k, r0, yrow, crow);
        const bool do_c = crow >= 0 && crow < d.mcus_y;
        const bool ok = mbar_wait_bounded(bar0 + 8 * s, (ps.parity >> s) & 1u, budget);
        ps.parity ^= 1u << s;
        if (!ok) *abort_flag = 1;
        uint8_t *stage = stages + s * L.stage_bytes;
        uint8_t *yplane = yplanes + s * L.ybytes;
        uint8_t *slot = cslots + (j & (L.nslot - 1)) * L.slot_bytes;
        if (ok) {
            if (FW)
                fx.run(stage, yplane, slot, qs, yrow >= 0, do_c, tid);
            else
                idct_job<HM, VM, FANCY, QM>(stage, yplane, slot, qs, L, yrow >= 0, do_c, nye, nce, lb0, wt, wte, tid,
                                            kCtaThreads);
        }
        __syncthreads();
        if (*abort_flag) {
            if (tid == 0) {
                atomicExch(err, kErrTimeout);
                // the other stage may still have a copy in flight: wait for it (bounded)
                if (k + 1 < njobs) mbar_wait_bounded(bar0 + 8 * (s ^ 1), (ps.parity >> (s ^ 1)) & 1u, budget);
            }
            return false;
        }
        if (tid == 0 && k + 2 < njobs) {
            int yr, cr;
            job_rows<HM, VM, FANCY>(k + 2, r0, yr, cr);
            fence_proxy_async_smem();
            issue_job<HM, VM, FANCY>(tm, L, stage, bar0 + 8 * s, mx0, yr, cr, d.mcus_y, d.withhold);
        }
        if (edge && do_c) {
            fix_edges(slot, L.lc, mx0, d.cw, used, tid);
            __syncthreads();
        }
        if (k >= V::kPro) {
            const int r = r0 + k - V::kPro;
            int py = py0, g = g0;
            while (py < rows) {
                if (V::kRing && HM == 2)
                    cc_task_h2v2_pair<FW != 0>(d, L, yplane, cslots, j, r, mx0, py, g);
                else if (V::kRing)
                    cc_task_h1v2_pair<FW != 0>(d, L, yplane, cslots, j, r, mx0, py, g);
                else
                    cc_task<HM, VM, FANCY, FW != 0>(d, L, yplane, cslots, j, r, mx0, wte, py, g);
                py += dpy;
                g += dg;
                if (g >= ngroups) { g -= ngroups; ++py; }
            }
        }
    }
    ps.job = J0 + njobs;
    ps.sync_from = ps.job;
    return true;
}

// One work item with unified roles (UNI, where the variant allows it) or
// split roles (see run_work_split and run_work_unified).  `last` = this is
// the CTA's final item, or the next item may use the other kind of roles:
// the split version then drains its barriers.
template <int HM, int VM, bool FANCY, int QM, bool UNI, int FW = 0>
__device__ __forceinline__ bool run_work(const CUtensorMap *tm, const ItemDesc d, const ImageDesc &qsrc, int strip,
                                         int r0, int r1, uint8_t *smem, const SmemLayout &L, PipeState &ps, int *err,
                                         bool last, bool reload_q)
{
    if (UNI && Variant<HM, VM, FANCY>::kCanUnify)
        return run_work_unified<HM, VM, FANCY, QM, FW>(tm, d, qsrc, strip, r0, r1, smem, L, ps, err, reload_q);
    return run_work_split<HM, VM, FANCY, QM, FW>(tm, d, qsrc, strip, r0, r1, smem, L, ps, err, last, reload_q);
}

}  // namespace jdec

namespace jdec {

// Runs the strip-rows [a, e) of an image (strip-rows concatenated strip after
// strip) as one item per strip.  `last_range`: the CTA decodes nothing after
// them.  FW > 0 (the launch's strip width, d.wt == FW): every strip runs the
// compile-time-width code; a last strip that reaches past the image's right
// edge is decoded as a full one (its blocks beyond the edge are zero-filled by
// TMA, the chroma halo is replaced by the true edge, and no pixel beyond the
// image is written).
template <int HM, int VM, bool FANCY, int QM, bool UNI, int FW>
__device__ __forceinline__ bool run_range(const CUtensorMap *tm, const ItemDesc &id, const ImageDesc &d, long a,
                                          long e, uint8_t *smem, const SmemLayout &L, PipeState &ps, int *err,
                                          bool last_range)
{
    const long nrows = d.row1 - d.row0;
    while (a < e) {
        const int s = static_cast<int>(a / nrows);
        const int rr = static_cast<int>(a - s * nrows);
        const int len = static_cast<int>(min(e - a, nrows - rr));
        a += len;
        const bool last = last_range && a >= e;
        bool ok;
        if (FW) {
            const SmemLayout LF = smem_layout(HM, VM, FANCY, FW ? FW : 1, default_slots(HM, VM, FANCY));
            ok = run_work<HM, VM, FANCY, QM, UNI, FW>(tm, id, d, s, d.row0 + rr, d.row0 + rr + len, smem, LF, ps, err,
                                                      last, false);
        } else {
            ok = run_work<HM, VM, FANCY, QM, UNI>(tm, id, d, s, d.row0 + rr, d.row0 + rr + len, smem, L, ps, err, last,
                                                  false);
        }
        if (!ok) return false;
    }
    return true;
}

// Runs this CTA's share of an image (MCU rows [row0, row1) of every strip):
// CTA b of nctas first takes its even part of the strip-rows before
// d.dyn_start, then claims chunks of d.dyn_chunk strip-rows of the rest from
// the launch's counter (work[0]) until none is left, so that CTAs that
// progress faster take more.  Split roles then consume the colour warps'
// last two EMPTY signals (the drain a final item does).
template <int HM, int VM, bool FANCY, int QM, bool UNI, int FW = 0>
__device__ bool run_share(const CUtensorMap *tm, const ImageDesc &d, int b, uint8_t *smem, const SmemLayout &L,
                          PipeState &ps, int *err, int *work)
{
    const ItemDesc id = item_desc(d);
    const long total = static_cast<long>(d.row1 - d.row0) * d.nstrips;
    const long S = work ? min(static_cast<long>(d.dyn_start), total) : total;
    if (!run_range<HM, VM, FANCY, QM, UNI, FW>(tm, id, d, S * b / d.nctas, S * (b + 1) / d.nctas, smem, L, ps, err,
                                               S >= total))
        return false;
    if (S >= total) return true;
    volatile int *claim = reinterpret_cast<volatile int *>(smem + L.off_flag + 4);
    for (;;) {
        __syncthreads();   // every thread has read the previous claim
        if (threadIdx.x == 0) *claim = atomicAdd(work, 1);
        __syncthreads();
        const long a = S + static_cast<long>(*claim) * d.dyn_chunk;
        if (a >= total) break;
        if (!run_range<HM, VM, FANCY, QM, UNI, FW>(tm, id, d, a, min(a + d.dyn_chunk, total), smem, L, ps, err,
                                                   false))
            return false;
    }
    if (!(UNI && Variant<HM, VM, FANCY>::kCanUnify)) {
        const int nidct = FW ? kFixedIdctThreads : d.nidct;
        if (static_cast<int>(threadIdx.x) < nidct)
            for (int jj = ps.job; jj < ps.job + 2; ++jj)
                if (jj >= ps.sync_from + 2) named_sync(kBarEmpty0 + (jj & 1), kCtaThreads);
        ps.sync_from = ps.job;
    }
    return true;
}

// The end of a single-image launch's CTA: counts it finished; the last one
// resets the launch's counters for the next launch that uses them.
__device__ __forceinline__ void finish_work(int *work)
{
    if (work && threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(work + 1, 1) == static_cast<int>(gridDim.x) - 1) {
            work[0] = 0;
            work[1] = 0;
        }
    }
}

}  // namespace jdec
