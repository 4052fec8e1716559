// jdec_runtime.cu -- host runtime: strip-width autotuner and its table,
// the host-buffer path (row bands whose copies overlap decoding, the
// pipelined execution of Sec. 4.5 with the entropy decoder replaced by the
// host->device copy), and context teardown.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "jdec_launch.h"
#include "jdec_runtime.h"

namespace jdec {

int variant_of(const Geometry &g)
{
    if (g.hm == 1) return g.vm == 1 ? 0 : (g.fancy ? 6 : 5);
    if (g.vm == 1) return g.fancy ? 2 : 1;
    return g.fancy ? 4 : 3;
}

int size_class_of_mcus(long mcus)
{
    int c = 0;
    while ((1L << (c + 1)) <= mcus && c < 40) ++c;
    return c / 2;   // buckets of 4x in MCU count
}

int size_class_of(const Geometry &g) { return size_class_of_mcus(static_cast<long>(g.mcus_x) * g.mcus_y); }

static const TuneEntry *tuned(jdec_ctx *ctx, const Geometry &g)
{
    const int v = variant_of(g), sc = size_class_of(g);
    for (int i = 0; i < ctx->n_tune; ++i)
        if (ctx->tune[i].kind == 0 && ctx->tune[i].variant == v && ctx->tune[i].size_class == sc) return &ctx->tune[i];
    return nullptr;
}

const TuneEntry *tuned_batch(jdec_ctx *ctx, int cls, int size_class)
{
    for (int i = 0; i < ctx->n_tune; ++i)
        if (ctx->tune[i].kind == 1 && ctx->tune[i].variant == cls && ctx->tune[i].size_class == size_class)
            return &ctx->tune[i];
    return nullptr;
}

int tuned_wt(jdec_ctx *ctx, const Geometry &g)
{
    const TuneEntry *t = tuned(ctx, g);
    return t ? t->wt : 0;
}

int tuned_nidct(jdec_ctx *ctx, const Geometry &g)
{
    const TuneEntry *t = tuned(ctx, g);
    return t ? t->nidct : 0;
}

static const char *tune_path(jdec_ctx *ctx)
{
    if (ctx->opt.tune_file && ctx->opt.tune_file[0]) return ctx->opt.tune_file;
    const char *e = getenv("JDEC_TUNE_FILE");
    return (e && e[0]) ? e : nullptr;
}

// Table format: {"gpu": "<name>", "sms": N, "entries": [[variant, size_class, wt, idct_threads, kind], ...]}
// (idct_threads may be omitted or 0: default split; kind may be omitted: 0,
// single-image entry; 1: batch-class entry, whose first field is the class)
void load_tune_table(jdec_ctx *ctx)
{
    const char *path = tune_path(ctx);
    if (!path) return;
    FILE *f = fopen(path, "rb");
    if (!f) return;
    std::vector<char> buf(1 << 16);
    const size_t n = fread(buf.data(), 1, buf.size() - 1, f);
    fclose(f);
    buf[n] = 0;
    const char *p = strstr(buf.data(), "\"sms\"");
    if (!p || !(p = strchr(p, ':'))) return;   // malformed: ignore
    int sms = 0;
    if (sscanf(p + 1, "%d", &sms) != 1 || sms != ctx->sms) return;   // other GPU: ignore
    p = strstr(buf.data(), "\"entries\"");
    if (!p) return;
    p = strchr(p, '[');
    if (!p) return;
    ++p;
    while (ctx->n_tune < kMaxTune) {
        const char *q = strchr(p, '[');
        if (!q) break;
        int v = 0, sc = 0, wt = 0, ni = 0, kind = 0;
        const int got = sscanf(q, "[ %d , %d , %d , %d , %d", &v, &sc, &wt, &ni, &kind);
        if (got < 3) break;
        if (got < 4 || (ni != 32 && ni != 64 && ni != 96)) ni = 0;
        if (got < 5 || (kind != 0 && kind != 1)) kind = 0;
        const bool ok_key = kind == 0 ? (v >= 0 && v < kVariants) : (v >= 0 && v < kClasses);
        if (wt >= 1 && wt <= kMaxWT && ok_key) ctx->tune[ctx->n_tune++] = TuneEntry{v, sc, wt, ni, kind};
        p = strchr(q, ']');
        if (!p) break;
        ++p;
    }
}

void save_tune_table(jdec_ctx *ctx)
{
    const char *path = tune_path(ctx);
    if (!path) return;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, ctx->device) != cudaSuccess) return;
    FILE *f = fopen(path, "wb");
    if (!f) return;
    fprintf(f, "{\"gpu\": \"%s\", \"sms\": %d, \"entries\": [", prop.name, ctx->sms);
    for (int i = 0; i < ctx->n_tune; ++i)
        fprintf(f, "%s[%d, %d, %d, %d, %d]", i ? ", " : "", ctx->tune[i].variant, ctx->tune[i].size_class,
                ctx->tune[i].wt, ctx->tune[i].nidct, ctx->tune[i].kind);
    fprintf(f, "]}\n");
    fclose(f);
}

// Times the candidate strip widths on this image (the output is rewritten
// with identical bytes) and records the fastest for its variant and size
// class.  Runs once per (variant, size class); synchronises the stream.
void autotune_shape(jdec_ctx *ctx, const jdec_image *img, const Geometry &g, cudaStream_t s)
{
    if (tuned_wt(ctx, g) > 0 || ctx->n_tune >= kMaxTune) return;
    // the defaults (20/21, 31/32) fill whole rounds of the IDCT threads
    static const int cand[] = {4, 6, 8, 10, 12, 16, 20, 21, 24, 31, 32, 42};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return; }
    int best = 0;
    float best_ms = 1e30f;
    for (int wt : cand) {
        if (wt > 2 * g.mcus_x && wt != cand[0]) break;
        float tot = 0.f;
        bool ok = true;
        for (int rep = 0; rep < 4 && ok; ++rep) {
            cudaEventRecord(e0, s);
            ok = launch_image(ctx, img, g, s, wt) == JDEC_OK;
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) ok = false;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) tot += ms;   // first launch warms the caches
        }
        if (ok && tot < best_ms) { best_ms = tot; best = wt; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best > 0) {
        ctx->tune[ctx->n_tune++] = TuneEntry{variant_of(g), size_class_of(g), best, 0, 0};
        save_tune_table(ctx);
    }
}

// ---------------------------------------------------------------------------
// Host-buffer path: copy -> decode -> copy back in row bands.
// ---------------------------------------------------------------------------
struct HostStreams {
    cudaStream_t h2d = nullptr, comp = nullptr, d2h = nullptr;
};

static HostStreams &host_streams(jdec_ctx *ctx)
{
    static thread_local HostStreams hs[16];
    HostStreams &h = hs[ctx->device & 15];
    if (!h.h2d) {
        cudaStreamCreateWithFlags(&h.h2d, cudaStreamNonBlocking);
        cudaStreamCreateWithFlags(&h.comp, cudaStreamNonBlocking);
        cudaStreamCreateWithFlags(&h.d2h, cudaStreamNonBlocking);
    }
    return h;
}

static cudaEvent_t band_event(jdec_ctx *ctx, int i)
{
    while (ctx->n_band_ev <= i && ctx->n_band_ev < 64) {
        if (cudaEventCreateWithFlags(&ctx->band_ev[ctx->n_band_ev], cudaEventDisableTiming) != cudaSuccess) return nullptr;
        ctx->n_band_ev++;
    }
    return i < ctx->n_band_ev ? ctx->band_ev[i] : nullptr;
}

// Event indices of the host-buffer calls: per staging slot b, [16b, 16b + nb)
// after the H2D of band k, [16b + 8, 16b + 8 + nb) after its decode; then the
// fork and join of the call and, per slot, "decode done" and "copy-back done".
constexpr int kBands = 8;
constexpr int kEvFork = 32, kEvJoin = 33, kEvCompDone = 34, kEvD2hDone = 36;

// Enqueues one image's banded H2D / decode / D2H on the three host streams,
// staged in slot b.  The slot's previous image (two images earlier in the
// same call, or an earlier call) must have finished decoding before its
// planes are overwritten, and finished copying back before its RGB is.
static jdec_status host_image(jdec_ctx *ctx, const jdec_image *himg, const Geometry &g, int b, HostStreams &hs)
{
    // device staging: the planes (256-byte aligned) + dense RGB
    const int ncomp = g.gray ? 1 : 3;
    size_t off[3] = {0, 0, 0}, tot = 0;
    for (int c = 0; c < ncomp; ++c) {
        off[c] = tot;
        tot += (static_cast<size_t>(himg->blocks_w[c]) * himg->blocks_h[c] * 128 + 255) & ~static_cast<size_t>(255);
    }
    jdec_status st = ensure_buffer(ctx, &ctx->h_coef[b], &ctx->h_coef_cap[b], tot);
    if (st != JDEC_OK) return st;
    const size_t rgb_pitch = 3 * static_cast<size_t>(g.W);
    st = ensure_buffer(ctx, &ctx->h_rgb[b], &ctx->h_rgb_cap[b], rgb_pitch * g.H);
    if (st != JDEC_OK) return st;

    jdec_image dimg = *himg;
    for (int c = 0; c < ncomp; ++c)
        dimg.coef[c] = reinterpret_cast<const int16_t *>(static_cast<uint8_t *>(ctx->h_coef[b]) + off[c]);
    dimg.rgb = static_cast<uint8_t *>(ctx->h_rgb[b]);
    dimg.rgb_pitch = static_cast<int64_t>(rgb_pitch);

    const int nb = std::min(kBands, g.mcus_y);
    const int e0 = 16 * b;
    cudaEvent_t comp_done = band_event(ctx, kEvCompDone + b), d2h_done = band_event(ctx, kEvD2hDone + b);
    for (int i = 0; i < 2 * kBands; ++i)
        if (!band_event(ctx, e0 + i)) return JDEC_ECUDA;
    if (!comp_done || !d2h_done) return JDEC_ECUDA;
    // (waits on an event never recorded return at once)
    if (cudaStreamWaitEvent(hs.h2d, comp_done, 0) != cudaSuccess) return JDEC_ECUDA;
    if (cudaStreamWaitEvent(hs.comp, d2h_done, 0) != cudaSuccess) return JDEC_ECUDA;
    const int lookahead = (g.fancy && g.vm == 2) ? 1 : 0;
    for (int k = 0; k < nb; ++k) {
        const int r0 = static_cast<int>(static_cast<long>(g.mcus_y) * k / nb);
        const int r1 = static_cast<int>(static_cast<long>(g.mcus_y) * (k + 1) / nb);
        for (int c = 0; c < ncomp; ++c) {
            const int v = c ? 1 : g.vm;
            const size_t row_bytes = static_cast<size_t>(himg->blocks_w[c]) * 128;
            const size_t o = static_cast<size_t>(r0) * v * row_bytes;
            const size_t n = static_cast<size_t>(r1 - r0) * v * row_bytes;
            if (cudaMemcpyAsync(static_cast<uint8_t *>(ctx->h_coef[b]) + off[c] + o,
                                reinterpret_cast<const uint8_t *>(himg->coef[c]) + o, n, cudaMemcpyHostToDevice,
                                hs.h2d) != cudaSuccess)
                return JDEC_ECUDA;
        }
        if (cudaEventRecord(band_event(ctx, e0 + k), hs.h2d) != cudaSuccess) return JDEC_ECUDA;
        // decode band k - lookahead once its chroma look-ahead row has arrived
        const int kd = k - lookahead;
        if (kd >= 0) {
            if (cudaStreamWaitEvent(hs.comp, band_event(ctx, e0 + k), 0) != cudaSuccess) return JDEC_ECUDA;
            const int d0 = static_cast<int>(static_cast<long>(g.mcus_y) * kd / nb);
            const int d1 = static_cast<int>(static_cast<long>(g.mcus_y) * (kd + 1) / nb);
            st = launch_rows(ctx, &dimg, g, hs.comp, d0, d1, 0);
            if (st != JDEC_OK) return st;
            if (cudaEventRecord(band_event(ctx, e0 + kBands + kd), hs.comp) != cudaSuccess) return JDEC_ECUDA;
        }
    }
    if (lookahead) {
        const int kd = nb - 1;
        const int d0 = static_cast<int>(static_cast<long>(g.mcus_y) * kd / nb);
        st = launch_rows(ctx, &dimg, g, hs.comp, d0, g.mcus_y, 0);
        if (st != JDEC_OK) return st;
        if (cudaEventRecord(band_event(ctx, e0 + kBands + kd), hs.comp) != cudaSuccess) return JDEC_ECUDA;
    }
    if (cudaEventRecord(comp_done, hs.comp) != cudaSuccess) return JDEC_ECUDA;
    const int mcu_h = 8 * g.vm;
    for (int k = 0; k < nb; ++k) {
        const int r0 = static_cast<int>(static_cast<long>(g.mcus_y) * k / nb);
        const int r1 = static_cast<int>(static_cast<long>(g.mcus_y) * (k + 1) / nb);
        const int y0 = r0 * mcu_h, y1 = std::min(g.H, r1 * mcu_h);
        if (y1 <= y0) continue;
        if (cudaStreamWaitEvent(hs.d2h, band_event(ctx, e0 + kBands + k), 0) != cudaSuccess) return JDEC_ECUDA;
        if (cudaMemcpy2DAsync(himg->rgb + static_cast<int64_t>(y0) * himg->rgb_pitch, himg->rgb_pitch,
                              static_cast<uint8_t *>(ctx->h_rgb[b]) + y0 * rgb_pitch, rgb_pitch, rgb_pitch, y1 - y0,
                              cudaMemcpyDeviceToHost, hs.d2h) != cudaSuccess)
            return JDEC_ECUDA;
    }
    if (cudaEventRecord(d2h_done, hs.d2h) != cudaSuccess) return JDEC_ECUDA;
    return JDEC_OK;
}

jdec_status decode_host_many(jdec_ctx *ctx, const jdec_image *imgs, const Geometry *geo, int n, cudaStream_t s)
{
    HostStreams &hs = host_streams(ctx);
    cudaEvent_t fork = band_event(ctx, kEvFork);
    cudaEvent_t join = band_event(ctx, kEvJoin);
    if (!fork || !join) return JDEC_ECUDA;
    // everything earlier on s happens first ...
    if (cudaEventRecord(fork, s) != cudaSuccess) return JDEC_ECUDA;
    cudaStreamWaitEvent(hs.h2d, fork, 0);
    cudaStreamWaitEvent(hs.comp, fork, 0);
    cudaStreamWaitEvent(hs.d2h, fork, 0);
    jdec_status st = JDEC_OK;
    for (int i = 0; i < n && st == JDEC_OK; ++i) st = host_image(ctx, &imgs[i], geo[i], i & 1, hs);
    // ... and everything later on s waits for the last copy back (also when
    // an image failed to enqueue: what was enqueued still completes first)
    if (cudaEventRecord(join, hs.d2h) != cudaSuccess) return JDEC_ECUDA;
    if (cudaStreamWaitEvent(s, join, 0) != cudaSuccess) return JDEC_ECUDA;
    return st;
}

jdec_status decode_host_banded(jdec_ctx *ctx, const jdec_image *himg, const Geometry &g, cudaStream_t s)
{
    return decode_host_many(ctx, himg, &g, 1, s);
}

void release_runtime(jdec_ctx *ctx)
{
    for (int b = 0; b < 2; ++b) {
        if (ctx->h_coef[b]) cudaFree(ctx->h_coef[b]);
        if (ctx->h_rgb[b]) cudaFree(ctx->h_rgb[b]);
        ctx->h_coef[b] = ctx->h_rgb[b] = nullptr;
        ctx->owned_bytes -= ctx->h_coef_cap[b] + ctx->h_rgb_cap[b];
        ctx->h_coef_cap[b] = ctx->h_rgb_cap[b] = 0;
    }
    for (int i = 0; i < ctx->n_band_ev; ++i) cudaEventDestroy(ctx->band_ev[i]);
    ctx->n_band_ev = 0;
    release_batch(ctx);
    release_pipeline(ctx);
}

}  // namespace jdec

extern "C" JDEC_API jdec_status jdec_decode_host_batch(jdec_ctx *ctx, const jdec_image *imgs, int32_t n, void *stream)
{
    if (!ctx || n < 0 || (n > 0 && !imgs)) return JDEC_EINVAL;
    if (n == 0) return JDEC_OK;
    std::vector<jdec::Geometry> geo(static_cast<size_t>(n));
    for (int i = 0; i < n; ++i) {
        const jdec_status st = jdec::validate(&imgs[i], &geo[i], true);
        if (st != JDEC_OK) return st;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return JDEC_ECUDA;
    if (dev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess) return JDEC_ECUDA;
    const jdec_status st = jdec::decode_host_many(ctx, imgs, geo.data(), n, static_cast<cudaStream_t>(stream));
    if (dev != ctx->device) cudaSetDevice(dev);
    return st;
}
