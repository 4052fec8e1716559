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
//   colour warps wait FULL[job % 2], upsample chroma and convert 8 pixels (or
//                8 pixels x 2 rows for 4:2:0) per task to RGB with 8-byte
//                vector stores, signal EMPTY[job % 2].
// The IDCT warps wait EMPTY[job % 2] before overwriting the planes of job-2.
// Luma planes are double-buffered; chroma rows go to a ring of four slots in
// job order, so a 4:2:0 triangular filter finds chroma rows r-1, r, r+1 in
// the three most recent slots and every chroma block is transformed once per
// item (the row above the item is recomputed once).
#pragma once

#include "jdec_device.cuh"

namespace jdec {

enum : int { kBarIdct = 1, kBarFull0 = 2, kBarEmpty0 = 4 };

struct PipeState {
    uint32_t parity;   // bit s = parity of the next completion of stage s
    int job;           // jobs started by this CTA (all items)
};

template <int HM, int VM, bool FANCY>
struct Variant {
    static constexpr bool kHalo = FANCY && HM == 2;            // horizontal neighbours
    static constexpr bool kRing = FANCY && HM == 2 && VM == 2; // vertical neighbours
    static constexpr int kLA = kRing ? 1 : 0;                  // chroma lookahead rows
    static constexpr int kPro = kRing ? 2 : 0;                 // chroma-only jobs per item
    static constexpr int kIdctThreads = 32 * (HM == 1 ? 3 : 2);
    static constexpr int kCcThreads = kCtaThreads - kIdctThreads;
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
template <int HM, int VM, bool FANCY>
__device__ __forceinline__ void issue_job(const CUtensorMap *tm, const SmemLayout &L, uint8_t *stage, uint32_t bar,
                                          int mx0, int yrow, int crow, int mcus_y)
{
    using V = Variant<HM, VM, FANCY>;
    const bool do_y = yrow >= 0;
    const bool do_c = crow >= 0 && crow < mcus_y;
    const uint32_t bytes = (do_y ? L.ny * 128 : 0) + (do_c ? 2 * L.nc * 128 : 0);
    mbar_arrive_expect_tx(bar, bytes);
    if (do_y) tma_load_3d(smem_u32(stage + L.stage_y), &tm[0], bar, 0, mx0 * HM, yrow * VM);
    if (do_c) {
        tma_load_3d(smem_u32(stage + L.stage_c), &tm[1], bar, 0, mx0 - (V::kHalo ? 1 : 0), crow);
        tma_load_3d(smem_u32(stage + L.stage_c + L.cbytes), &tm[2], bar, 0, mx0 - (V::kHalo ? 1 : 0), crow);
    }
}

// ---------------------------------------------------------------------------
// colour warps: one task
// ---------------------------------------------------------------------------
template <int HM, int VM, bool FANCY>
__device__ __forceinline__ void cc_task(const ImageDesc &d, const SmemLayout &L, const uint8_t *yplane,
                                        const uint8_t *cslots, int job, int r, int mx0, int t, int ngroups)
{
    const int lc = L.lc;
    const int pr = t / ngroups, g = t - pr * ngroups;
    const int x0 = (mx0 * HM + g) * 8;
    if (x0 >= d.W) return;
    const int n = min(8, d.W - x0);
    const bool vec = d.aligned8 != 0;
    const uint8_t *cb_cur = cslots + (job & (L.nslot - 1)) * L.slot_bytes;
    if (VM == 1) {
        const int y = r * 8 + pr;
        if (y >= d.H) return;
        int Yv[8], Cb[8], Cr[8];
        load8(yplane + pr * L.ypitch + 8 * g, Yv);
        const uint8_t *cb = cb_cur + pr * lc;
        const uint8_t *cr = cb + 8 * lc;
        if (HM == 1) {
            load8(cb + 8 * g, Cb);
            load8(cr + 8 * g, Cr);
        } else if (!FANCY) {
            const uint32_t wb = *reinterpret_cast<const uint32_t *>(cb + 4 * g);
            const uint32_t wr = *reinterpret_cast<const uint32_t *>(cr + 4 * g);
#pragma unroll
            for (int k = 0; k < 8; ++k) { Cb[k] = byte_of(wb, k >> 1); Cr[k] = byte_of(wr, k >> 1); }
        } else {
            int cb6[6], cr6[6];
            load6(cb + 8 + 4 * g, cb6);
            load6(cr + 8 + 4 * g, cr6);
            tri_h2v1(cb6, Cb);
            tri_h2v1(cr6, Cr);
        }
        cc_store8(Yv, Cb, Cr, d.rgb + static_cast<int64_t>(y) * d.pitch + 3 * x0, n, vec);
    } else {
        // output rows 2*pr and 2*pr + 1 of the MCU row share chroma row j
        const int y = r * 16 + 2 * pr;
        if (y >= d.H) return;
        const bool two = y + 1 < d.H;
        int Y0[8], Y1[8], Cb0[8], Cr0[8], Cb1[8], Cr1[8];
        load8(yplane + (2 * pr) * L.ypitch + 8 * g, Y0);
        load8(yplane + (2 * pr + 1) * L.ypitch + 8 * g, Y1);
        if (!FANCY) {
            const uint8_t *cb = cb_cur + pr * lc;
            const uint32_t wb = *reinterpret_cast<const uint32_t *>(cb + 4 * g);
            const uint32_t wr = *reinterpret_cast<const uint32_t *>(cb + 8 * lc + 4 * g);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                Cb0[k] = Cb1[k] = byte_of(wb, k >> 1);
                Cr0[k] = Cr1[k] = byte_of(wr, k >> 1);
            }
        } else {
            // chroma block row b lives in slot (job - 1 + b - r) & 3
            const int j = y >> 1;
            const int ju = max(j - 1, 0), jd = min(j + 1, d.ch - 1);
            auto row_ptr = [&](int jr) {
                return cslots + ((job - 1 + (jr >> 3) - r) & 3) * L.slot_bytes + (jr & 7) * lc + 8 + 4 * g;
            };
            const uint8_t *pn = row_ptr(j), *pu = row_ptr(ju), *pd = row_ptr(jd);
            int n6[6], u6[6], d6[6];
            load6(pn, n6); load6(pu, u6); load6(pd, d6);
            tri_h2v2(n6, u6, Cb0);
            tri_h2v2(n6, d6, Cb1);
            load6(pn + 8 * lc, n6); load6(pu + 8 * lc, u6); load6(pd + 8 * lc, d6);
            tri_h2v2(n6, u6, Cr0);
            tri_h2v2(n6, d6, Cr1);
        }
        uint8_t *out = d.rgb + static_cast<int64_t>(y) * d.pitch + 3 * x0;
        cc_store8(Y0, Cb0, Cr0, out, n, vec);
        if (two) cc_store8(Y1, Cb1, Cr1, out + d.pitch, n, vec);
    }
}

// Replicates the true chroma edge into halo/padding columns of the 8 rows of
// both components of one chroma slot (strips at the image's left or right
// edge only).  `tid` < 16 does one row each.
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

// Runs one work item with the whole CTA.  `smem` is 1024-byte aligned.
// Returns false if a bounded wait gave up (the error word has been set; the
// CTA must stop).  `last` = this is the CTA's final item (drain barriers).
template <int HM, int VM, bool FANCY>
__device__ bool run_work(const CUtensorMap *tm, const ImageDesc &d, int strip, int chunk, uint8_t *smem,
                         PipeState &ps, int *err, bool last)
{
    using V = Variant<HM, VM, FANCY>;
    const SmemLayout L = smem_layout(HM, VM, FANCY, d.wt, d.nslot);
    const int tid = threadIdx.x;
    const int wt = d.wt;
    const int mx0 = strip * wt;
    const int wte = min(wt, d.mcus_x - mx0);
    const int r0 = d.row0 + chunk * d.rows_per_chunk;
    const int r1 = min(r0 + d.rows_per_chunk, d.row1);
    if (r0 >= r1 || wte <= 0) return true;
    const int njobs = V::kPro + (r1 - r0);
    const int J0 = ps.job;

    uint8_t *stages = smem + L.off_stage;
    uint8_t *yplanes = smem + L.off_y;
    uint8_t *cslots = smem + L.off_c;
    const uint32_t bar0 = smem_u32(smem + L.off_bar);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + L.off_flag);

    if (tid < V::kIdctThreads) {
        // =================== IDCT warps ===================
        const int *qs = reinterpret_cast<const int *>(smem + L.off_q);
        const int lb0 = (V::kHalo && mx0 == 0) ? 1 : 0;
        const int lb1 = min(wte + (V::kHalo ? 2 : 0), d.mcus_x - (mx0 - (V::kHalo ? 1 : 0)));
        const int nce = lb1 - lb0;
        const int used = 8 * (wte + (V::kHalo ? 2 : 0));
        const bool edge = V::kHalo && (mx0 == 0 || d.cw + 7 - 8 * mx0 < used - 1);
        const int nye = VM * HM * wte;
        const uint64_t budget = 2000000000ull;   // 2 s per wait

        if (tid == 0) {
            fence_proxy_async_smem();
            for (int k = 0; k < 2 && k < njobs; ++k) {
                int yr, cr;
                job_rows<HM, VM, FANCY>(k, r0, yr, cr);
                const int s = (J0 + k) & 1;
                issue_job<HM, VM, FANCY>(tm, L, stages + s * L.stage_bytes, bar0 + 8 * s, mx0, yr, cr, d.mcus_y);
            }
        }
        for (int k = 0; k < njobs; ++k) {
            const int j = J0 + k, s = j & 1;
            int yrow, crow;
            job_rows<HM, VM, FANCY>(k, r0, yrow, crow);
            const bool do_c = crow >= 0 && crow < d.mcus_y;
            if (j >= 2) named_sync(kBarEmpty0 + s, kCtaThreads);
            const bool ok = mbar_wait_bounded(bar0 + 8 * s, (ps.parity >> s) & 1u, budget);
            ps.parity ^= 1u << s;
            if (!ok) *abort_flag = 1;
            uint8_t *stage = stages + s * L.stage_bytes;
            uint8_t *yplane = yplanes + s * L.ybytes;
            uint8_t *slot = cslots + (j & (L.nslot - 1)) * L.slot_bytes;
            const int ntask = (yrow >= 0 ? nye : 0) + (do_c ? 2 * nce : 0);
            for (int t = tid; ok && t < ntask; t += V::kIdctThreads) {
                uint32_t blk;
                const int *q;
                uint8_t *dst;
                int pitch;
                int tc = t;
                if (yrow >= 0 && t < nye) {
                    const int vy = t / (HM * wte), bx = t - vy * (HM * wte);
                    blk = smem_u32(stage + L.stage_y + (vy * HM * wt + bx) * 128);
                    q = qs;
                    dst = yplane + 8 * vy * L.ypitch + 8 * bx;
                    pitch = L.ypitch;
                } else {
                    if (yrow >= 0) tc -= nye;
                    const int comp = tc >= nce;
                    const int lb = lb0 + (comp ? tc - nce : tc);
                    blk = smem_u32(stage + L.stage_c + comp * L.cbytes + lb * 128);
                    q = qs + 64 * (1 + comp);
                    dst = slot + comp * 8 * L.lc + 8 * lb;
                    pitch = L.lc;
                }
                idct_block(blk, q, dst, pitch);
            }
            named_sync(kBarIdct, V::kIdctThreads);
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
                issue_job<HM, VM, FANCY>(tm, L, stage, bar0 + 8 * s, mx0, yr, cr, d.mcus_y);
            }
            if (edge && do_c) fix_edges(slot, L.lc, mx0, d.cw, used, tid);
            named_arrive(kBarFull0 + s, kCtaThreads);
        }
        ps.job = J0 + njobs;
        if (last) {
            // consume the colour warps' EMPTY signals of the final two jobs, as
            // jobs ps.job and ps.job + 1 would
            for (int jj = ps.job; jj < ps.job + 2; ++jj)
                if (jj >= 2) named_sync(kBarEmpty0 + (jj & 1), kCtaThreads);
        }
    } else {
        // =================== colour warps ===================
        const int tc = tid - V::kIdctThreads;
        const int ngroups = HM * wte;
        const int ntask = 8 * ngroups;   // 8 rows (or row pairs) x 8-pixel groups
        for (int k = 0; k < njobs; ++k) {
            const int j = J0 + k, s = j & 1;
            named_sync(kBarFull0 + s, kCtaThreads);
            if (*abort_flag) return false;
            if (k >= V::kPro) {
                const int r = r0 + k - V::kPro;
                const uint8_t *yplane = yplanes + s * L.ybytes;
                for (int t = tc; t < ntask; t += V::kCcThreads)
                    cc_task<HM, VM, FANCY>(d, L, yplane, cslots, j, r, mx0, t, ngroups);
            }
            named_arrive(kBarEmpty0 + s, kCtaThreads);
        }
        ps.job = J0 + njobs;
    }
    return true;
}

}  // namespace jdec
