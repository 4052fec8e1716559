// jdec_work.cuh -- one work item of the fused back-end: a strip of `wt`
// MCUs walked down a chunk of MCU rows (Sec. 2 MCU tiling; Sec. 4.1-4.3
// stages fused into one pass, Sec. 4.4).
//
// Per MCU row ("step") the CTA
//   1. waits for the TMA copy of the step's coefficient blocks (Y blocks of the
//      row; Cb/Cr blocks of the row plus one halo block left and right when
//      the triangular filter needs neighbours across the strip edge),
//   2. dequantises + IDCTs every block, one thread per block, into shared
//      sample planes (Y plane; Cb/Cr planes kept as a ring of three chroma
//      block rows for 4:2:0 triangular filtering, so each chroma block is
//      transformed once per chunk and the rows above/below come for free),
//   3. refills the TMA stage with the coefficients two steps ahead,
//   4. upsamples chroma and converts to RGB, 8 pixels per thread task,
//      writing the raster output with 8-byte vector stores.
// Chroma rows are processed one step ahead of luma for 4:2:0 triangular
// filtering (the output row pair 2j+1 needs chroma row j+1).
#pragma once

#include "jdec_device.cuh"

namespace jdec {

struct PipeState {
    uint32_t parity;   // bit s = parity of the next completion of stage s
};

template <int HM, int VM, bool FANCY>
struct Variant {
    static constexpr bool kHalo = FANCY && HM == 2;            // horizontal neighbours
    static constexpr bool kRing = FANCY && HM == 2 && VM == 2; // vertical neighbours
    static constexpr int kLA = kRing ? 1 : 0;                  // chroma lookahead rows
};

// Issues the TMA loads of one stage.  y_row < 0: chroma only.  c_row outside
// the grid: chroma skipped.  Called by one thread.
template <int HM, int VM, bool FANCY>
__device__ __forceinline__ void issue_stage(const CUtensorMap *tm, const SmemLayout &L, uint8_t *stage,
                                            uint32_t bar, int mx0, int y_row, int c_row, int mcus_y)
{
    using V = Variant<HM, VM, FANCY>;
    const bool do_y = y_row >= 0;
    const bool do_c = c_row >= 0 && c_row < mcus_y;
    const uint32_t bytes = (do_y ? L.ny * 128 : 0) + (do_c ? 2 * L.nc * 128 : 0);
    mbar_arrive_expect_tx(bar, bytes);
    if (do_y) tma_load_3d(smem_u32(stage + L.stage_y), &tm[0], bar, 0, mx0 * HM, y_row * VM);
    if (do_c) {
        const int cbytes = round_up(L.nc * 128, 1024);
        tma_load_3d(smem_u32(stage + L.stage_c), &tm[1], bar, 0, mx0 - (V::kHalo ? 1 : 0), c_row);
        tma_load_3d(smem_u32(stage + L.stage_c + cbytes), &tm[2], bar, 0, mx0 - (V::kHalo ? 1 : 0), c_row);
    }
}

// Replicates the true chroma edge into halo/padding columns of 8 rows of the
// two chroma planes (only strips at the image's left or right edge).
template <int HM, int VM, bool FANCY>
__device__ __forceinline__ void fix_edges(uint8_t *cb_rows, uint8_t *cr_rows, int lc, int mx0, int cw, int used)
{
    const int tid = threadIdx.x;
    if (tid >= 16) return;
    uint8_t *row = (tid < 8 ? cb_rows : cr_rows) + (tid & 7) * lc;
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

// Runs one work item.  `smem` is 1024-byte aligned.  Returns false if a
// bounded wait gave up (the error word has been set; the CTA must stop).
template <int HM, int VM, bool FANCY>
__device__ bool run_work(const CUtensorMap *tm, const ImageDesc &d, int strip, int chunk,
                         uint8_t *smem, PipeState &ps, int *err)
{
    using V = Variant<HM, VM, FANCY>;
    const SmemLayout L = smem_layout(HM, VM, FANCY, d.wt);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int wt = d.wt;
    const int mx0 = strip * wt;
    const int wte = min(wt, d.mcus_x - mx0);
    const int r0 = d.row0 + chunk * d.rows_per_chunk;
    const int r1 = min(r0 + d.rows_per_chunk, d.row1);
    if (r0 >= r1 || wte <= 0) return true;

    uint8_t *stages = smem + L.off_stage;
    uint8_t *yplane = smem + L.off_y;
    uint8_t *cplane = smem + L.off_c;
    const int *qs = reinterpret_cast<const int *>(smem + L.off_q);
    const uint32_t bar0 = smem_u32(smem + L.off_bar);
    int *flag = reinterpret_cast<int *>(smem + L.off_flag);
    const int ypitch = 8 * HM * wt;
    const int lc = L.lc;
    const int slot_bytes = 8 * lc;
    const int cbytes = round_up(L.nc * 128, 1024);
    const uint64_t budget = 2000000000ull;   // 2 s per wait

    // chroma blocks present in this strip (local indices [lb0, lb1))
    const int lb0 = (V::kHalo && mx0 == 0) ? 1 : 0;
    const int lb1 = min(wte + (V::kHalo ? 2 : 0), d.mcus_x - (mx0 - (V::kHalo ? 1 : 0)));
    const int nce = lb1 - lb0;
    const int used = 8 * (wte + (V::kHalo ? 2 : 0));
    const bool edge = V::kHalo && (mx0 == 0 || d.cw + 7 - 8 * mx0 < used - 1);

    auto cb_slot = [&](int crow) { return cplane + ((V::kRing ? (crow + 3) % 3 : 0)) * slot_bytes; };
    auto cr_slot = [&](int crow) { return cplane + (L.nslot + (V::kRing ? (crow + 3) % 3 : 0)) * slot_bytes; };

    // IDCT of the chroma blocks held by `stage` into the slot of chroma row crow.
    auto chroma_idct = [&](const uint8_t *stage, int crow, int t0) {
        for (int t = t0; t < 2 * nce; t += nt) {
            const int comp = t >= nce;
            const int lb = lb0 + (comp ? t - nce : t);
            const uint32_t blk = smem_u32(stage + L.stage_c + comp * cbytes + lb * 128);
            uint8_t *dst = (comp ? cr_slot(crow) : cb_slot(crow)) + 8 * lb;
            idct_block(blk, qs + 64 * (1 + comp), dst, lc);
        }
    };

    auto wait_stage = [&](int s) -> bool {
        bool ok = mbar_wait_bounded(bar0 + 8 * s, (ps.parity >> s) & 1u, budget);
        ps.parity ^= 1u << s;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicExch(err, kErrTimeout);
            return false;
        }
        return true;
    };

    // ---- prologue: chroma rows r0-1 and r0 for vertical triangular filtering
    if (V::kRing) {
        if (tid == 0) {
            fence_proxy_async_smem();
            issue_stage<HM, VM, FANCY>(tm, L, stages, bar0, mx0, -1, r0 - 1 >= 0 ? r0 - 1 : -1, d.mcus_y);
            issue_stage<HM, VM, FANCY>(tm, L, stages + L.stage_bytes, bar0 + 8, mx0, -1, r0, d.mcus_y);
        }
        if (!wait_stage(0)) return false;
        if (!wait_stage(1)) return false;
        if (r0 > 0) chroma_idct(stages, r0 - 1, tid);
        chroma_idct(stages + L.stage_bytes, r0, tid);
        __syncthreads();
        if (edge) {
            if (r0 > 0) fix_edges<HM, VM, FANCY>(cb_slot(r0 - 1), cr_slot(r0 - 1), lc, mx0, d.cw, used);
            fix_edges<HM, VM, FANCY>(cb_slot(r0), cr_slot(r0), lc, mx0, d.cw, used);
            __syncthreads();
        }
    }

    // ---- main pipeline
    const int nsteps = r1 - r0;
    if (tid == 0) {
        fence_proxy_async_smem();
        issue_stage<HM, VM, FANCY>(tm, L, stages, bar0, mx0, r0, r0 + V::kLA, d.mcus_y);
        if (nsteps > 1)
            issue_stage<HM, VM, FANCY>(tm, L, stages + L.stage_bytes, bar0 + 8, mx0, r0 + 1, r0 + 1 + V::kLA, d.mcus_y);
    }
    const int nye = VM * HM * wte;
    const int rows_out = 8 * VM;
    const int ngroups = HM * wte;
    for (int i = 0; i < nsteps; ++i) {
        const int s = i & 1;
        const int r = r0 + i;
        const int crow = r + V::kLA;
        uint8_t *stage = stages + s * L.stage_bytes;
        if (!wait_stage(s)) return false;

        // phase A: IDCT
        const bool do_c = crow < d.mcus_y;
        const int ntask = nye + (do_c ? 2 * nce : 0);
        for (int t = tid; t < ntask; t += nt) {
            if (t < nye) {
                const int vy = t / (HM * wte), bx = t - vy * (HM * wte);
                const uint32_t blk = smem_u32(stage + L.stage_y + (vy * HM * wt + bx) * 128);
                idct_block(blk, qs, yplane + 8 * vy * ypitch + 8 * bx, ypitch);
            } else {
                const int tc = t - nye;
                const int comp = tc >= nce;
                const int lb = lb0 + (comp ? tc - nce : tc);
                const uint32_t blk = smem_u32(stage + L.stage_c + comp * cbytes + lb * 128);
                uint8_t *dst = (comp ? cr_slot(crow) : cb_slot(crow)) + 8 * lb;
                idct_block(blk, qs + 64 * (1 + comp), dst, lc);
            }
        }
        __syncthreads();
        if (tid == 0 && i + 2 < nsteps) {
            fence_proxy_async_smem();
            issue_stage<HM, VM, FANCY>(tm, L, stage, bar0 + 8 * s, mx0, r + 2, r + 2 + V::kLA, d.mcus_y);
        }
        if (edge && do_c) {
            fix_edges<HM, VM, FANCY>(cb_slot(crow), cr_slot(crow), lc, mx0, d.cw, used);
            __syncthreads();
        }

        // phase B: upsample + colour conversion, 8 pixels per task
        for (int t = tid; t < rows_out * ngroups; t += nt) {
            const int py = t / ngroups, g = t - py * ngroups;
            const int y = r * rows_out + py;
            const int x0 = (mx0 * HM + g) * 8;
            if (y >= d.H || x0 >= d.W) continue;
            int Yv[8], Cb[8], Cr[8];
            load8(yplane + py * ypitch + 8 * g, Yv);
            if (HM == 1) {
                load8(cb_slot(r) + py * lc + 8 * g, Cb);
                load8(cr_slot(r) + py * lc + 8 * g, Cr);
            } else if (!FANCY) {
                const int row = (VM == 2) ? (py >> 1) : py;
                const uint32_t wb = *reinterpret_cast<const uint32_t *>(cb_slot(r) + row * lc + 4 * g);
                const uint32_t wr = *reinterpret_cast<const uint32_t *>(cr_slot(r) + row * lc + 4 * g);
#pragma unroll
                for (int k = 0; k < 8; ++k) { Cb[k] = byte_of(wb, k >> 1); Cr[k] = byte_of(wr, k >> 1); }
            } else if (VM == 1) {
                int cb6[6], cr6[6];
                load6(cb_slot(r) + py * lc + 8 + 4 * g, cb6);
                load6(cr_slot(r) + py * lc + 8 + 4 * g, cr6);
                tri_h2v1(cb6, Cb);
                tri_h2v1(cr6, Cr);
            } else {
                const int j = y >> 1;
                const int jf = min(max(j + ((py & 1) ? 1 : -1), 0), d.ch - 1);
                const int off = 8 + 4 * g;
                int nb[6], fb[6], nr[6], fr[6];
                load6(cb_slot(j >> 3) + (j & 7) * lc + off, nb);
                load6(cb_slot(jf >> 3) + (jf & 7) * lc + off, fb);
                load6(cr_slot(j >> 3) + (j & 7) * lc + off, nr);
                load6(cr_slot(jf >> 3) + (jf & 7) * lc + off, fr);
                tri_h2v2(nb, fb, Cb);
                tri_h2v2(nr, fr, Cr);
            }
            cc_store8(Yv, Cb, Cr, d.rgb + static_cast<int64_t>(y) * d.pitch + 3 * x0, min(8, d.W - x0),
                      d.aligned8 != 0);
        }
        __syncthreads();
    }
    (void)flag;
    return true;
}

}  // namespace jdec
