// jdec_common.h -- definitions shared by the host runtime and the kernels of
// the GB300 back-end (product code; not shared with the CPU oracle).
#pragma once

#include <cstdint>
#include <cuda.h>

namespace jdec {

// Launch shape of the fused kernel: each CTA owns a strip of `wt` MCUs and
// walks down `rows_per_chunk` MCU rows of it.
constexpr int kMaxWT = 32;          // widest strip the shared-memory layout allows
constexpr int kStages = 2;          // coefficient double buffer

// Error codes a kernel writes to the context's device error word.
constexpr int kErrTimeout = 1;      // an mbarrier wait gave up
constexpr int kErrBadWork = 2;      // a work item failed validation on device

// Per-image description as the kernels see it.
struct ImageDesc {
    uint8_t *rgb;           // device
    int64_t pitch;          // bytes per RGB row
    int32_t W, H;
    int32_t mcus_x, mcus_y;
    int32_t cw, ch;         // true chroma size
    int32_t wt;             // MCUs per strip
    int32_t nstrips;
    int32_t rows_per_chunk; // MCU rows per CTA work item
    int32_t nchunks;
    int32_t aligned8;       // rgb and pitch are 8-byte aligned
    int32_t row0, row1;     // MCU rows [row0, row1) covered by the launch
    int32_t pad_;
    int32_t q[3][64];       // dequantisation tables, natural order
};

// Kernel parameters of the single-image launch.
struct DecodeParams {
    CUtensorMap tmap[3];    // coefficient planes, 3-D {64, blocks_w, blocks_h}
    ImageDesc img;
    int *err;               // device error word
};

// Shared-memory carve-up of one CTA; identical on host and device.
struct SmemLayout {
    int ny, nc;             // Y blocks per step, chroma blocks per component per step
    int lc;                 // chroma samples per plane row (with halo blocks)
    int nslot;              // chroma block rows kept (3 for vertical triangular filtering)
    int stage_y, stage_c;   // byte offsets of the chroma regions inside a stage
    int stage_bytes;        // one coefficient stage (1024-aligned regions)
    int off_stage;          // offset of stage 0
    int off_y;              // Y sample plane, (8*VM) x (8*HM*wt)
    int off_c;              // chroma sample planes, 2 x nslot x 8 x lc
    int off_q;              // dequantisation tables, int32 [3][64]
    int off_bar;            // mbarriers, one per stage
    int off_flag;           // CTA-wide flags
    int total;              // bytes, including 1024 of alignment slack
};

__host__ __device__ inline int round_up(int x, int a) { return (x + a - 1) / a * a; }

__host__ __device__ inline SmemLayout smem_layout(int hm, int vm, bool fancy, int wt)
{
    SmemLayout L;
    const int halo = (fancy && hm == 2) ? 1 : 0;
    L.ny = hm * vm * wt;
    L.nc = wt + 2 * halo;
    L.lc = 8 * L.nc;
    L.nslot = (fancy && hm == 2 && vm == 2) ? 3 : 1;
    L.stage_y = 0;
    L.stage_c = round_up(L.ny * 128, 1024);
    L.stage_bytes = L.stage_c + 2 * round_up(L.nc * 128, 1024);
    L.off_stage = 0;
    int off = kStages * L.stage_bytes;
    L.off_y = off;
    off += round_up(8 * vm * 8 * hm * wt, 16);
    L.off_c = off;
    off += round_up(2 * L.nslot * 8 * L.lc, 16);
    L.off_q = off;
    off += 3 * 64 * 4;
    L.off_bar = off;
    off += 8 * kStages;
    L.off_flag = off;
    off += 16;
    L.total = off + 1024;
    return L;
}

}  // namespace jdec
