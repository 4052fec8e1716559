// jdec_runtime.h -- context state and host-runtime internals of the C ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/jdec.h"
#include "jdec_common.h"

namespace jdec {

struct Geometry {
    int hm, vm;
    bool fancy;
    bool gray;       // one component: decoded as 4:4:4 with all-zero chroma blocks
    bool aan;        // AAN scaled IDCT instead of the LLM form
    int W, H;
    int mcus_x, mcus_y;
    int cw, ch;
    int64_t coef_bytes, rgb_bytes;
};

// Autotuned tile shape.  kind 0: single-image launches, keyed by (variant,
// size class of the image); kind 1: batched launches, keyed by (batch class =
// 3 * variant + dequantisation/IDCT mode, size class of the class's average
// image in the batch).
struct TuneEntry {
    int variant;     // kind 0: 0: 4:4:4, 1/2: 4:2:2, 3/4: 4:2:0, 5/6: 4:4:0 (replicate / triangular); kind 1: class
    int size_class;  // log2 of the MCU count, bucketed
    int wt;
    int nidct;       // IDCT threads of split roles (0: default)
    int kind = 0;
};

struct BatchState;

constexpr int kMaxTune = 128;   // tune-table entries a context holds

}  // namespace jdec

struct jdec_ctx {
    jdec_options opt;
    int device = 0;
    int sms = 0;
    int *d_err = nullptr;         // error word, then kWorkSlots pairs of work counters
    int *d_work = nullptr;
    int work_slot = 0;
    size_t owned_bytes = 0;
    long launches = 0;
    int fail_allocs = 0;   // testing aid: the next n buffer allocations fail (JDEC_TEST_FAIL_ALLOCS)
    // occupancy cache
    int occ_key[32][2];
    int occ_val[32];
    int n_occ = 0;
    // tune table
    jdec::TuneEntry tune[128];
    int n_tune = 0;
    // host-buffer path: device staging
    // device staging of the host-buffer calls: two slots, so that consecutive
    // images of one call overlap their copies
    void *h_coef[2] = {nullptr, nullptr};
    size_t h_coef_cap[2] = {0, 0};
    void *h_rgb[2] = {nullptr, nullptr};
    size_t h_rgb_cap[2] = {0, 0};
    cudaEvent_t band_ev[64];
    int n_band_ev = 0;
    // batched path
    jdec::BatchState *batch = nullptr;
    // pipelined JPEG path: device planes, page-locked staging, streams, events
    void *p_coef = nullptr;
    size_t p_coef_cap = 0;
    void *p_host = nullptr;
    size_t p_host_cap = 0;
    cudaStream_t p_h2d = nullptr, p_comp = nullptr;
    cudaEvent_t p_ev[66];
    int n_p_ev = 0;
    bool p_pending = false;   // p_ev[65] guards the staging buffer until its copies ran
};

namespace jdec {

const char *status_str(jdec_status s);
bool encode_plane_map(CUtensorMap *m, const int16_t *base, int bw, int bh, int box_w, int box_h);
// allow_test: accept the JDEC_TEST_WITHHOLD_LOADS flag (single-image launches only)
jdec_status validate(const jdec_image *img, Geometry *g, bool host_buffers, bool allow_test = false);
void plan_tiles(jdec_ctx *ctx, const Geometry &g, int nrows, int force_wt, int fw, int *wt, int *nctas, int *smem,
                bool *fixed);
void fill_desc(ImageDesc *d, const jdec_image *img, const Geometry &g, int wt, int nctas);
// Dequantisation + IDCT mode of an image: kAAN when asked for, else kQ8 when
// every quantisation step fits in 8 bits, else kQ16.
int qmode_of(const jdec_image *img, const Geometry &g);
bool encode_maps(CUtensorMap maps[3], const jdec_image *img, const Geometry &g, int wt);
// Device address (current device) of a small all-zero coefficient plane that
// stands in for the chroma planes of a grayscale image (null on failure).
const int16_t *zero_plane();
constexpr int kZeroPlaneBlocks = kMaxWT + 2;   // blocks per row of that plane (one row)
jdec_status launch_rows(jdec_ctx *ctx, const jdec_image *img, const Geometry &g, cudaStream_t s, int row0,
                        int row1, int force_wt);
jdec_status launch_image(jdec_ctx *ctx, const jdec_image *img, const Geometry &g, cudaStream_t s, int force_wt);
int occupancy_cached(jdec_ctx *ctx, int hm, int vm, bool fancy, int smem);
jdec_status ensure_buffer(jdec_ctx *ctx, void **buf, size_t *cap, size_t need);

int variant_of(const Geometry &g);
int default_wt(const Geometry &g);
int equal_strips(int mcus_x, int w);   // widest equal strips no wider than w
int size_class_of(const Geometry &g);
int tuned_wt(jdec_ctx *ctx, const Geometry &g);
int tuned_nidct(jdec_ctx *ctx, const Geometry &g);
const TuneEntry *tuned_batch(jdec_ctx *ctx, int cls, int size_class);
int size_class_of_mcus(long mcus);
void load_tune_table(jdec_ctx *ctx);
void save_tune_table(jdec_ctx *ctx);
void autotune_shape(jdec_ctx *ctx, const jdec_image *img, const Geometry &g, cudaStream_t s);

jdec_status decode_host_banded(jdec_ctx *ctx, const jdec_image *img, const Geometry &g, cudaStream_t s);
// n images from host buffers in one call: copies and decodes of consecutive
// images overlap (alternating staging slots); stream-ordered on s as a whole.
jdec_status decode_host_many(jdec_ctx *ctx, const jdec_image *imgs, const Geometry *geo, int n, cudaStream_t s);
jdec_status decode_batch(jdec_ctx *ctx, const jdec_image *imgs, int n, cudaStream_t s);
void release_runtime(jdec_ctx *ctx);
jdec_status decode_jpeg(jdec_ctx *ctx, const uint8_t *data, size_t size, uint8_t *rgb, int64_t pitch, uint32_t flags,
                        int threads, cudaStream_t s);
void release_pipeline(jdec_ctx *ctx);
void release_batch(jdec_ctx *ctx);

}  // namespace jdec
