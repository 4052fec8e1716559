// jdec_api.cu -- host runtime behind the C ABI declared in include/jdec.h:
// validation, tile choice, TMA tensor-map encoding, launches, host-buffer
// staging and the device error word.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "../../include/jdec.h"
#include "jdec_common.h"
#include "jdec_launch.h"
#include "jdec_runtime.h"

using namespace jdec;

namespace jdec {

const char *status_str(jdec_status s)
{
    switch (s) {
    case JDEC_OK: return "ok";
    case JDEC_EINVAL: return "invalid argument";
    case JDEC_ENOMEM: return "out of memory";
    case JDEC_ECUDA: return "CUDA error";
    case JDEC_EUNSUPPORTED: return "unsupported sampling";
    case JDEC_EBUSY: return "exceeds the HBM budget";
    case JDEC_ETIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

// Makes `device` current for the lifetime of the guard, restoring the
// caller's device afterwards.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int device)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != device && cudaSetDevice(device) != cudaSuccess) ok = false;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

static PFN_cuTensorMapEncodeTiled_v12000 get_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 3-D view {64 coefficients, blocks_w, blocks_h} of one plane, box
// {64, box_w, box_h}, 128-byte swizzle (conflict-free thread-per-block reads).
// The element type is declared as uint16: TMA only moves the bytes.
bool encode_plane_map(CUtensorMap *m, const int16_t *base, int bw, int bh, int box_w, int box_h)
{
    auto enc = get_encoder();
    if (!enc) return false;
    cuuint64_t dims[3] = {64, static_cast<cuuint64_t>(bw), static_cast<cuuint64_t>(bh)};
    cuuint64_t strides[2] = {128, static_cast<cuuint64_t>(bw) * 128};
    cuuint32_t box[3] = {64, static_cast<cuuint32_t>(box_w), static_cast<cuuint32_t>(box_h)};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, const_cast<int16_t *>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// A grayscale image is decoded by the 4:4:4 kernel whose chroma tiles come
// from this plane's single row of zero blocks: TMA fills every tile outside it
// with zeros too, an all-zero block transforms to 128, and Alg. 2 maps
// (Y, 128, 128) to (Y, Y, Y), so the output is exactly the grey axis.
static __device__ __align__(256) int16_t g_zero_plane[kZeroPlaneBlocks * 64];

const int16_t *zero_plane()
{
    static const int16_t *addr[64];
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (!addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_zero_plane) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        addr[dev] = static_cast<const int16_t *>(p);
    }
    return addr[dev];
}

jdec_status validate(const jdec_image *img, Geometry *g, bool host_buffers, bool allow_test)
{
    if (!img) return JDEC_EINVAL;
    if (img->width < 1 || img->width > 65535 || img->height < 1 || img->height > 65535) return JDEC_EINVAL;
    if (img->ncomp == 1) {
        // one component: 8x8 MCUs (T.81 A.2.2), output R = G = B = Y
        if (img->h_samp[0] != 1 || img->v_samp[0] != 1) return JDEC_EUNSUPPORTED;
        if (img->flags & ~(JDEC_UPSAMPLE_REPLICATE | JDEC_IDCT_AAN | JDEC_TEST_WITHHOLD_LOADS)) return JDEC_EINVAL;
        if ((img->flags & JDEC_TEST_WITHHOLD_LOADS) && !allow_test) return JDEC_EINVAL;
        g->hm = g->vm = 1;
        g->fancy = false;
        g->gray = true;
        g->aan = (img->flags & JDEC_IDCT_AAN) != 0;
        g->W = img->width; g->H = img->height;
        g->mcus_x = (img->width + 7) / 8;
        g->mcus_y = (img->height + 7) / 8;
        g->cw = img->width;
        g->ch = img->height;
        if (img->blocks_w[0] != g->mcus_x || img->blocks_h[0] != g->mcus_y) return JDEC_EINVAL;
        if (!img->coef[0] || !img->qtab[0]) return JDEC_EINVAL;
        if (!host_buffers && (reinterpret_cast<uintptr_t>(img->coef[0]) & 15)) return JDEC_EINVAL;
        if (!img->rgb || img->rgb_pitch < 3 * static_cast<int64_t>(img->width)) return JDEC_EINVAL;
        g->coef_bytes = static_cast<int64_t>(img->blocks_w[0]) * img->blocks_h[0] * 128;
        g->rgb_bytes = 3 * static_cast<int64_t>(img->width) * img->height;
        return JDEC_OK;
    }
    if (img->ncomp != 3) return JDEC_EINVAL;
    g->gray = false;
    for (int c = 0; c < 3; ++c)
        if (img->h_samp[c] < 1 || img->h_samp[c] > 4 || img->v_samp[c] < 1 || img->v_samp[c] > 4) return JDEC_EINVAL;
    if (img->h_samp[1] != 1 || img->v_samp[1] != 1 || img->h_samp[2] != 1 || img->v_samp[2] != 1)
        return JDEC_EUNSUPPORTED;
    const int hm = img->h_samp[0], vm = img->v_samp[0];
    if (hm > 2 || vm > 2) return JDEC_EUNSUPPORTED;   // 4:4:4, 4:2:2, 4:2:0, 4:4:0
    if (img->flags & ~(JDEC_UPSAMPLE_REPLICATE | JDEC_IDCT_AAN | JDEC_TEST_WITHHOLD_LOADS)) return JDEC_EINVAL;
    if ((img->flags & JDEC_TEST_WITHHOLD_LOADS) && !allow_test) return JDEC_EINVAL;
    g->hm = hm; g->vm = vm;
    g->aan = (img->flags & JDEC_IDCT_AAN) != 0;
    g->fancy = (img->flags & JDEC_UPSAMPLE_REPLICATE) == 0 && (hm == 2 || vm == 2);
    g->W = img->width; g->H = img->height;
    g->mcus_x = (img->width + 8 * hm - 1) / (8 * hm);
    g->mcus_y = (img->height + 8 * vm - 1) / (8 * vm);
    g->cw = (img->width + hm - 1) / hm;
    g->ch = (img->height + vm - 1) / vm;
    for (int c = 0; c < 3; ++c) {
        const int h = c ? 1 : hm, v = c ? 1 : vm;
        if (img->blocks_w[c] != g->mcus_x * h || img->blocks_h[c] != g->mcus_y * v) return JDEC_EINVAL;
        if (!img->coef[c] || !img->qtab[c]) return JDEC_EINVAL;
        if (!host_buffers && (reinterpret_cast<uintptr_t>(img->coef[c]) & 15)) return JDEC_EINVAL;
    }
    if (!img->rgb || img->rgb_pitch < 3 * static_cast<int64_t>(img->width)) return JDEC_EINVAL;
    g->coef_bytes = 0;
    for (int c = 0; c < 3; ++c) g->coef_bytes += static_cast<int64_t>(img->blocks_w[c]) * img->blocks_h[c] * 128;
    g->rgb_bytes = 3 * static_cast<int64_t>(img->width) * img->height;
    return JDEC_OK;
}

// Default strip width (measured on 8192x8192 images with 64 IDCT threads): the
// blocks of one job (MCU row of the strip, halo included) fill whole rounds
// of the IDCT threads, and the colour tasks whole rounds of the colour threads.
int default_wt(const Geometry &g)
{
    if (g.hm == 1 && g.vm == 1) return 32;    // 3 blocks per MCU: 96 blocks
    // 4:4:0, 4 blocks per MCU: 128; triangular at 28 keeps four CTAs per SM
    // with its four chroma slots
    if (g.hm == 1) return g.fancy ? 28 : 32;
    if (g.vm == 1) return g.fancy ? 31 : 32;  // 4 blocks per MCU (+ 4 halo blocks): 128
    return g.fancy ? 20 : 21;                 // 6 blocks per MCU (+ 4 halo blocks): 124 / 126
}

// Strips of (nearly) equal width no wider than `w`: a narrow last strip
// would leave most of its IDCT and colour threads idle.
int equal_strips(int mcus_x, int w)
{
    const int ns = (mcus_x + w - 1) / w;
    return (mcus_x + ns - 1) / ns;
}

// Default strip width of an image whose `nrows` MCU rows are decoded by one
// launch of up to `wave` CTAs: narrower strips while there are too few
// strip-rows to give every CTA a few rows (small images), then equal strips.
static bool enough_rows(const Geometry &g, int nrows, long wave, int w)
{
    const long min_rows = (g.fancy && g.vm == 2) ? 6 : 2;
    return static_cast<long>((g.mcus_x + w - 1) / w) * nrows >= min_rows * wave;
}

static int fit_wt(const Geometry &g, int nrows, long wave)
{
    int w = default_wt(g);
    while (w > 4 && !enough_rows(g, nrows, wave, w)) w = std::max(4, w / 2);
    return equal_strips(g.mcus_x, w);
}

// Strip width (MCUs) and the number of CTAs for `nrows` MCU rows of an image:
// one full wave (occupancy x SMs) or fewer when there are fewer strip-rows.
// fw > 0: the variant's compile-time width; when the image is at least that
// wide, the last strip's padding stays small and there are enough strip-rows
// at that width (and no width is forced or tuned), every strip is fw wide
// (the last one padded) and *fixed is set.
void plan_tiles(jdec_ctx *ctx, const Geometry &g, int nrows, int force_wt, int fw, int *wt, int *nctas, int *smem,
                bool *fixed)
{
    int w = force_wt > 0 ? force_wt : tuned_wt(ctx, g);
    *fixed = false;
    if (w <= 0) {
        const SmemLayout L0 = smem_layout(g.hm, g.vm, g.fancy, default_wt(g), default_slots(g.hm, g.vm, g.fancy));
        const long wave = static_cast<long>(occupancy_cached(ctx, g.hm, g.vm, g.fancy, L0.total)) * ctx->sms;
        // (the padded part of the last strip, decoded but not written, stays
        // within 3 % of the width)
        const long pad = ((g.mcus_x + fw - 1) / fw) * static_cast<long>(fw) - g.mcus_x;
        if (fw > 0 && g.mcus_x >= fw && 100 * pad <= 3L * g.mcus_x && enough_rows(g, nrows, wave, fw)) {
            w = fw;
            *fixed = true;
        } else {
            w = fit_wt(g, nrows, wave);
        }
    }
    w = std::max(1, std::min(w, kMaxWT));
    const SmemLayout L = smem_layout(g.hm, g.vm, g.fancy, w, default_slots(g.hm, g.vm, g.fancy));
    const int occ = occupancy_cached(ctx, g.hm, g.vm, g.fancy, L.total);
    const int nstrips = (g.mcus_x + w - 1) / w;
    const long rows = static_cast<long>(nstrips) * nrows;
    // items shorter than a few rows pay the 4:2:0 chroma prologue too often
    const long min_rows = (g.fancy && g.vm == 2) ? 6 : 1;
    const long cap = std::max(1L, rows / std::min<long>(min_rows, nrows));
    *wt = w;
    *nctas = static_cast<int>(std::min<long>(static_cast<long>(occ) * ctx->sms, cap));
    *smem = L.total;
}

// Even and claimed parts of a launch's strip-rows.  CTAs on one SM progress
// at different rates (the warp schedulers favour some), so an even split of
// the work leaves SMs with fewer and fewer resident CTAs towards the end.
// With unified warp roles the strip-rows are instead cut into chunks of 8
// that the CTAs claim one after another as they finish (measured on 8192^2:
// 4:2:2 -7 %, 4:2:0 -2.5 %; 8 rows beat 2 to 16); launches with fewer chunks
// than CTAs stay even.  Split roles keep the even split: each chunk boundary
// would drain their two-group pipeline (measured slower).
static void plan_dynamic(const Geometry &g, int nrows, bool unified, ImageDesc *d)
{
    (void)g;
    const long total = static_cast<long>(nrows) * d->nstrips;
    const int chunk = 8;
    d->dyn_start = static_cast<int32_t>(total);
    d->dyn_chunk = chunk;
    if (unified && total / chunk >= d->nctas) d->dyn_start = 0;
}

// AAN scale table S(v,u) = round(2^12 s_v s_u), s_0 = 1, s_k = sqrt(2) cos(k pi / 16)
// ([8v + u]); the AAN transform's 2-D input scale folded into dequantisation.
static const int32_t *aan_scale()
{
    static const struct Table {
        int32_t s[64];
        Table()
        {
            const double pi = 3.14159265358979323846;
            double f[8];
            for (int k = 0; k < 8; ++k) f[k] = k ? std::sqrt(2.0) * std::cos(k * pi / 16.0) : 1.0;
            for (int v = 0; v < 8; ++v)
                for (int u = 0; u < 8; ++u) s[8 * v + u] = static_cast<int32_t>(std::floor(4096.0 * f[v] * f[u] + 0.5));
        }
    } table;
    return table.s;
}

int qmode_of(const jdec_image *img, const Geometry &g)
{
    if (g.aan) return kAAN;
    for (int c = 0; c < (g.gray ? 1 : 3); ++c)
        for (int k = 0; k < 64; ++k)
            if (img->qtab[c][k] > 255) return kQ16;
    return kQ8;
}

void fill_desc(ImageDesc *d, const jdec_image *img, const Geometry &g, int wt, int nctas)
{
    memset(d, 0, sizeof(*d));
    d->rgb = img->rgb;
    d->pitch = img->rgb_pitch;
    d->W = g.W; d->H = g.H;
    d->mcus_x = g.mcus_x; d->mcus_y = g.mcus_y;
    d->cw = g.cw; d->ch = g.ch;
    d->wt = wt;
    d->nstrips = (g.mcus_x + wt - 1) / wt;
    d->nctas = nctas;
    d->row0 = 0;
    d->row1 = g.mcus_y;
    d->nslot = default_slots(g.hm, g.vm, g.fancy);
    d->nidct = 32 * default_idct_warps(g.hm, g.vm);
    d->aligned8 = ((reinterpret_cast<uintptr_t>(img->rgb) | static_cast<uintptr_t>(img->rgb_pitch)) & 7) == 0;
    d->withhold = (img->flags & JDEC_TEST_WITHHOLD_LOADS) ? 1 : 0;
    d->qmode = qmode_of(img, g);
    const int32_t *S = aan_scale();
    for (int c = 0; c < 3; ++c) {
        const uint16_t *q = img->qtab[g.gray ? 0 : c];   // grayscale: the chroma blocks are zero
        // AAN: Q * S < 65536 * 2^13 fits int32
        for (int k = 0; k < 64; ++k) d->q[c][k] = g.aan ? static_cast<int32_t>(q[k]) * S[k] : q[k];
    }
}

bool encode_maps(CUtensorMap maps[3], const jdec_image *img, const Geometry &g, int wt)
{
    const int halo = chroma_halo(g.hm, g.fancy);
    if (!encode_plane_map(&maps[0], img->coef[0], img->blocks_w[0], img->blocks_h[0], g.hm * wt, g.vm)) return false;
    if (g.gray) {
        const int16_t *z = zero_plane();
        if (!z) return false;
        return encode_plane_map(&maps[1], z, kZeroPlaneBlocks, 1, wt, 1) &&
               encode_plane_map(&maps[2], z, kZeroPlaneBlocks, 1, wt, 1);
    }
    for (int c = 1; c < 3; ++c)
        if (!encode_plane_map(&maps[c], img->coef[c], img->blocks_w[c], img->blocks_h[c], wt + 2 * halo, 1))
            return false;
    return true;
}

jdec_status launch_rows(jdec_ctx *ctx, const jdec_image *img, const Geometry &g, cudaStream_t s, int row0,
                        int row1, int force_wt)
{
    if (row1 <= row0) return JDEC_OK;
    int wt, nctas, smem;
    bool fixed;
    const int ni = tuned_nidct(ctx, g);
    // the compile-time-width instances run their own split (kFixedIdctThreads
    // IDCT threads) and store whole 8-pixel groups with aligned stores only:
    // 8-byte aligned rows, width a multiple of 8
    const bool clean = ((reinterpret_cast<uintptr_t>(img->rgb) | static_cast<uintptr_t>(img->rgb_pitch)) & 7) == 0 &&
                       g.W % 8 == 0;
    const int fw = ((ni > 0 && ni != kFixedIdctThreads) || !clean) ? 0 : fixed_wt(g.hm, g.vm, g.fancy, qmode_of(img, g));
    plan_tiles(ctx, g, row1 - row0, force_wt, fw, &wt, &nctas, &smem, &fixed);
    DecodeParams p;
    memset(&p, 0, sizeof(p));
    if (!encode_maps(p.tmap, img, g, wt)) return JDEC_ECUDA;
    fill_desc(&p.img, img, g, wt, nctas);
    if (ni > 0) p.img.nidct = ni;
    if (fixed) p.img.nidct = kFixedIdctThreads;
    p.img.row0 = row0;
    p.img.row1 = row1;
    // unified roles pay off on strips of 16 MCUs or more (measured: 4:2:2 on
    // 4000x3000 +10 %, 8192x8192 and 4:2:0 unchanged; narrower strips gain nothing)
    const bool unified = g.fancy && g.hm == 2 && wt >= 16;
    plan_dynamic(g, row1 - row0, unified, &p.img);
    p.err = ctx->d_err;
    p.work = ctx->d_work + 2 * ctx->work_slot;
    ctx->work_slot = (ctx->work_slot + 1) % kWorkSlots;
    const int grid = nctas;
    cudaError_t e = launch_fused(g.hm, g.vm, g.fancy, unified, fixed, p, grid, smem, s);
    if (e != cudaSuccess) return JDEC_ECUDA;
    ctx->launches++;
    return JDEC_OK;
}

jdec_status launch_image(jdec_ctx *ctx, const jdec_image *img, const Geometry &g, cudaStream_t s, int force_wt)
{
    return launch_rows(ctx, img, g, s, 0, g.mcus_y, force_wt);
}

int occupancy_cached(jdec_ctx *ctx, int hm, int vm, bool fancy, int smem)
{
    const int v = (hm == 1) ? (vm == 1 ? 0 : (fancy ? 6 : 5)) : (vm == 1 ? (fancy ? 2 : 1) : (fancy ? 4 : 3));
    for (int i = 0; i < ctx->n_occ; ++i)
        if (ctx->occ_key[i][0] == v && ctx->occ_key[i][1] == smem) return ctx->occ_val[i];
    const int o = fused_occupancy(hm, vm, fancy, smem);
    if (ctx->n_occ < static_cast<int>(sizeof(ctx->occ_val) / sizeof(ctx->occ_val[0]))) {
        ctx->occ_key[ctx->n_occ][0] = v;
        ctx->occ_key[ctx->n_occ][1] = smem;
        ctx->occ_val[ctx->n_occ] = o;
        ctx->n_occ++;
    }
    return o;
}

jdec_status ensure_buffer(jdec_ctx *ctx, void **buf, size_t *cap, size_t need)
{
    if (*cap >= need) return JDEC_OK;
    if (ctx->fail_allocs > 0) {   // injected failure (testing aid); the context stays usable
        --ctx->fail_allocs;
        return JDEC_ENOMEM;
    }
    const size_t others = ctx->owned_bytes - *cap;
    if (ctx->opt.hbm_budget_bytes && others + need > ctx->opt.hbm_budget_bytes) return JDEC_EBUSY;
    if (*buf) cudaFree(*buf);
    ctx->owned_bytes -= *cap;
    *buf = nullptr;
    *cap = 0;
    if (cudaMalloc(buf, need) != cudaSuccess) {
        cudaGetLastError();
        *buf = nullptr;
        return JDEC_ENOMEM;
    }
    *cap = need;
    ctx->owned_bytes += need;
    return JDEC_OK;
}

}  // namespace jdec

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char *jdec_status_str(jdec_status s) { return jdec::status_str(s); }

jdec_status jdec_create(jdec_ctx **out, const jdec_options *opt)
{
    if (!out) return JDEC_EINVAL;
    *out = nullptr;
    jdec_options o;
    memset(&o, 0, sizeof(o));
    if (opt) o = *opt;
    if (o.max_batch <= 0) o.max_batch = 4096;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || o.device < 0 || o.device >= ndev) {
        cudaGetLastError();
        return ndev == 0 ? JDEC_ECUDA : JDEC_EINVAL;
    }
    DeviceGuard dg(o.device);
    if (!dg.ok) return JDEC_ECUDA;
    if (!jdec::get_encoder()) return JDEC_ECUDA;
    jdec_ctx *ctx = new (std::nothrow) jdec_ctx();
    if (!ctx) return JDEC_ENOMEM;
    ctx->opt = o;
    ctx->device = o.device;
    if (cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, o.device) != cudaSuccess) {
        delete ctx;
        return JDEC_ECUDA;
    }
    const size_t words = 32 + 2 * jdec::kWorkSlots;   // error word; counters from a 128-byte boundary
    if (cudaMalloc(&ctx->d_err, words * sizeof(int)) != cudaSuccess ||
        cudaMemset(ctx->d_err, 0, words * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        if (ctx->d_err) cudaFree(ctx->d_err);
        delete ctx;
        return JDEC_ENOMEM;
    }
    ctx->d_work = ctx->d_err + 32;
    jdec::load_tune_table(ctx);
    if (const char *e = getenv("JDEC_TEST_FAIL_ALLOCS")) ctx->fail_allocs = std::max(0, atoi(e));
    *out = ctx;
    return JDEC_OK;
}

jdec_status jdec_decode_coeffs(jdec_ctx *ctx, const jdec_image *img, void *stream)
{
    if (!ctx) return JDEC_EINVAL;
    jdec::Geometry g;
    jdec_status st = jdec::validate(img, &g, false, true);
    if (st != JDEC_OK) return st;
    jdec::DeviceGuard dg(ctx->device);
    if (!dg.ok) return JDEC_ECUDA;
    if (ctx->opt.autotune && !(img->flags & JDEC_TEST_WITHHOLD_LOADS))
        jdec::autotune_shape(ctx, img, g, static_cast<cudaStream_t>(stream));
    return jdec::launch_image(ctx, img, g, static_cast<cudaStream_t>(stream), 0);
}

jdec_status jdec_decode_host(jdec_ctx *ctx, const jdec_image *img, void *stream)
{
    if (!ctx) return JDEC_EINVAL;
    jdec::Geometry g;
    jdec_status st = jdec::validate(img, &g, true);
    if (st != JDEC_OK) return st;
    jdec::DeviceGuard dg(ctx->device);
    if (!dg.ok) return JDEC_ECUDA;
    return jdec::decode_host_banded(ctx, img, g, static_cast<cudaStream_t>(stream));
}

jdec_status jdec_decode_batch(jdec_ctx *ctx, const jdec_image *imgs, int32_t n, void *stream)
{
    if (!ctx || n < 0 || (n > 0 && !imgs) || n > ctx->opt.max_batch) return JDEC_EINVAL;
    if (n == 0) return JDEC_OK;
    jdec::DeviceGuard dg(ctx->device);
    if (!dg.ok) return JDEC_ECUDA;
    return jdec::decode_batch(ctx, imgs, n, static_cast<cudaStream_t>(stream));
}

jdec_status jdec_sync_status(jdec_ctx *ctx, void *stream)
{
    if (!ctx) return JDEC_EINVAL;
    jdec::DeviceGuard dg(ctx->device);
    if (!dg.ok) return JDEC_ECUDA;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return JDEC_ECUDA;
    int h = 0;
    if (cudaMemcpy(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return JDEC_ECUDA;
    if (h != 0) {
        cudaMemset(ctx->d_err, 0, sizeof(int));
        return JDEC_ETIMEOUT;
    }
    return JDEC_OK;
}

jdec_status jdec_destroy(jdec_ctx *ctx)
{
    if (!ctx) return JDEC_EINVAL;
    {
        jdec::DeviceGuard dg(ctx->device);
        jdec::release_runtime(ctx);
        if (ctx->d_err) cudaFree(ctx->d_err);
    }
    delete ctx;
    return JDEC_OK;
}

}  // extern "C"
