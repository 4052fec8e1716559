// jdec_common.h -- definitions shared by the host runtime and the kernels of
// the GB300 back-end (product code; not shared with the CPU oracle).
#pragma once

#include <cstdint>
#include <cuda.h>

namespace jdec {

// Launch shape of the fused kernel: the image is cut into strips of `wt` MCUs;
// the strips' MCU rows, concatenated strip after strip, are split into equal
// contiguous ranges, one per CTA (a range may end one strip and start the
// next).
constexpr int kMaxWT = 64;          // widest strip (MCUs) a launch accepts
constexpr int kStages = 2;          // coefficient double buffer

// Kernel variants (sampling x upsampling): 0: 4:4:4, 1/2: 4:2:2, 3/4: 4:2:0,
// 5/6: 4:4:0 (replicate / triangular).
constexpr int kVariants = 7;
// Dequantisation + IDCT modes: the LLM form with 32-bit table entries, the
// LLM form with 8-bit steps (dp2a dequantisation), the AAN scaled form
// (prescaled 32-bit table).
constexpr int kQ16 = 0, kQ8 = 1, kAAN = 2;
constexpr int kQModes = 3;
// A batch launch class is one variant in one mode: class = 3 * variant + mode.
constexpr int kClasses = kQModes * kVariants;

// Error codes a kernel writes to the context's device error word.
constexpr int kErrTimeout = 1;      // an mbarrier wait gave up
constexpr int kErrBadWork = 2;      // reserved: a work item that fails validation on device

// Per-image description as the kernels see it.
struct ImageDesc {
    uint8_t *rgb;           // device
    int64_t pitch;          // bytes per RGB row
    int32_t W, H;
    int32_t mcus_x, mcus_y;
    int32_t cw, ch;         // true chroma size
    int32_t wt;             // MCUs per strip
    int32_t nstrips;
    int32_t nctas;          // CTAs sharing the strip-rows of this image
    int32_t aligned8;       // rgb and pitch are 8-byte aligned
    int32_t qmode;          // kQ16, kQ8 (every step fits in 8 bits) or kAAN
    int32_t row0, row1;     // MCU rows [row0, row1) covered by the launch
    int32_t nslot;          // chroma slots of the shared-memory ring (2 or 4)
    int32_t nidct;          // IDCT threads of the split roles (32, 64 or 96; unified roles: unused)
    int32_t withhold;       // testing aid: arm the load barriers, issue no loads
    int32_t dyn_start;      // single-image launch: strip-rows before this index are split
                            // evenly over the CTAs, the rest claimed in chunks
    int32_t dyn_chunk;      // strip-rows per claimed chunk
    int32_t q[3][64];       // dequantisation tables, natural order (kAAN: prescaled)
};

// Region offsets shared by every variant decoded by one persistent launch:
// each variant keeps its own pitches and stage-internal offsets, but stages,
// planes and slots sit at the same places whatever the variant, so jobs of
// consecutive items of different variants can overlap in the pipeline.
struct UnionLayout {
    int stage_bytes, off_y, ybytes, off_c, slot_bytes, off_q, off_bar, off_flag, total;
    int nslot;   // chroma slots (4 when items of several variants share the layout)
};

// Kernel parameters of the single-image launch.
struct DecodeParams {
    CUtensorMap tmap[3];    // coefficient planes, 3-D {64, blocks_w, blocks_h}
    ImageDesc img;
    int *err;               // device error word
    int *work;              // this launch's two counters: chunks claimed, CTAs finished
                            // (both zero at launch; the last CTA to finish resets them)
};

// Work counters of the single-image launches: a context owns kWorkSlots pairs
// and hands them out in turn, so up to kWorkSlots - 1 of its launches may
// overlap on the GPU.
constexpr int kWorkSlots = 64;

// Threads of a CTA: IDCT warps (producers) + upsample/colour warps (consumers).
constexpr int kWarps = 4;
constexpr int kCtaThreads = 32 * kWarps;
__host__ __device__ inline int default_idct_warps(int hm, int vm) { return (void)hm, (void)vm, 2; }

// Shared-memory carve-up of one CTA; identical on host and device.
//   stages : kStages coefficient tiles written by TMA (1024-aligned regions)
//   y      : 2 luma sample planes (double buffer), (8*VM) x (8*HM*wt) bytes
//   c      : nslot chroma slots (4 for 4:2:0 and 4:4:0 triangular filtering, else 2),
//            each 2 components x 8 rows x lc bytes (halo blocks included)
//   q      : dequantisation tables, 3 components x 64 int32 (transposed) or
//            3 x 32 packed-byte words for the dp2a path
struct SmemLayout {
    int ny, nc;             // Y blocks per step, chroma blocks per component per step
    int lc;                 // bytes per chroma slot row
    int stage_y, stage_c;   // byte offsets of the regions inside a stage
    int cbytes;             // bytes of one chroma component region of a stage
    int stage_bytes;        // one coefficient stage
    int off_stage;          // offset of stage 0
    int ypitch, ybytes;     // luma plane pitch and size
    int off_y;              // luma planes
    int nslot;              // chroma slots
    int slot_bytes;         // one chroma slot (both components)
    int off_c;              // chroma slots
    int off_q;              // dequantisation tables
    int off_bar;            // mbarriers, one per stage
    int off_flag;           // CTA-wide flags
    int total;              // bytes, including 1024 of alignment slack
};

__host__ __device__ inline int round_up(int x, int a) { return (x + a - 1) / a * a; }

// IDCT threads of the split roles in the compile-time-width path (4:4:4,
// 32-MCU strips: 96 blocks per job, one per IDCT thread; the fourth warp
// converts the job's 128 16-pixel tasks, about as much work).
constexpr int kFixedIdctThreads = 96;

// Strip widths with a compile-time-width fast path in the single-image kernel
// (the variants' default widths, 8-bit tables): 4:4:4 32 MCUs, triangular
// 4:2:2 31, triangular 4:2:0 20; 0 = none.
__host__ __device__ inline int fixed_wt(int hm, int vm, bool fancy, int qmode)
{
    if (qmode != kQ8) return 0;
    if (hm == 1 && vm == 1) return 32;
    if (hm == 2 && vm == 1 && fancy) return 31;
    if (hm == 2 && vm == 2 && fancy) return 20;
    return 0;
}

__host__ __device__ inline SmemLayout apply_union(SmemLayout L, const UnionLayout &U)
{
    L.stage_bytes = U.stage_bytes;
    L.off_stage = 0;
    L.off_y = U.off_y;
    L.ybytes = U.ybytes;
    L.nslot = U.nslot;
    L.off_c = U.off_c;
    L.slot_bytes = U.slot_bytes;
    L.off_q = U.off_q;
    L.off_bar = U.off_bar;
    L.off_flag = U.off_flag;
    L.total = U.total;
    return L;
}

// triangular filtering along columns (4:2:0, 4:4:0) keeps a ring of 4 chroma
// block rows: the rows above, at and below the current one, and the one loading
__host__ __device__ inline int default_slots(int hm, int vm, bool fancy) { return (void)hm, (fancy && vm == 2) ? 4 : 2; }

// Chroma blocks loaded on each side of a strip: horizontal triangular
// filtering (4:2:2, 4:2:0) needs one neighbouring block column; the chroma
// TMA box is wt + 2 * chroma_halo blocks wide.
__host__ __device__ inline int chroma_halo(int hm, bool fancy) { return (fancy && hm == 2) ? 1 : 0; }

__host__ __device__ inline SmemLayout smem_layout(int hm, int vm, bool fancy, int wt, int nslot)
{
    SmemLayout L;
    const int halo = chroma_halo(hm, fancy);
    L.ny = hm * vm * wt;
    L.nc = wt + 2 * halo;
    L.lc = round_up(8 * L.nc, 16);
    L.stage_y = 0;
    L.stage_c = round_up(L.ny * 128, 1024);
    L.cbytes = round_up(L.nc * 128, 1024);
    L.stage_bytes = L.stage_c + 2 * L.cbytes;
    L.off_stage = 0;
    int off = kStages * L.stage_bytes;
    L.ypitch = 8 * hm * wt;
    L.ybytes = round_up(8 * vm * L.ypitch, 16);
    L.off_y = off;
    off += 2 * L.ybytes;
    L.nslot = nslot;
    L.slot_bytes = 2 * 8 * L.lc;
    L.off_c = off;
    off += nslot * L.slot_bytes;
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
