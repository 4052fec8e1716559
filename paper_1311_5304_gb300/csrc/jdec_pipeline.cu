// jdec_pipeline.cu -- jdec_decode_jpeg: a baseline JPEG stream from host
// memory to device RGB, with host entropy decoding overlapped with the device
// back-end (Sec. 4.5, pipelined execution: the sequential Huffman stage of
// chunk k+1 runs on the CPU while the GPU transforms chunk k).
//
// The MCU rows are cut into chunks.  Each decoded chunk is copied from
// page-locked staging to context-owned device planes on a copy stream and
// handed to the fused kernel for its rows on a compute stream (a 4:2:0
// triangular chunk waits for the next chunk, whose first chroma row its last
// output rows need).  A stream without restart intervals is decoded by the
// calling thread, one chunk after another.  When restart intervals fall on
// chunk boundaries, chunks are decoded independently by `threads` worker
// threads and handed to the GPU in order as they complete.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

#include "jdec_entropy.h"
#include "jdec_launch.h"
#include "jdec_runtime.h"

namespace jdec {

static cudaEvent_t pipe_event(jdec_ctx *ctx, int i)
{
    while (ctx->n_p_ev <= i && ctx->n_p_ev < 66) {
        if (cudaEventCreateWithFlags(&ctx->p_ev[ctx->n_p_ev], cudaEventDisableTiming) != cudaSuccess) return nullptr;
        ctx->n_p_ev++;
    }
    return i < ctx->n_p_ev ? ctx->p_ev[i] : nullptr;
}

static jdec_status ensure_pinned(jdec_ctx *ctx, size_t need)
{
    if (ctx->p_host_cap >= need) return JDEC_OK;
    if (ctx->p_host) cudaFreeHost(ctx->p_host);
    ctx->p_host = nullptr;
    ctx->p_host_cap = 0;
    if (cudaMallocHost(&ctx->p_host, need) != cudaSuccess) {
        cudaGetLastError();
        return JDEC_ENOMEM;
    }
    ctx->p_host_cap = need;
    return JDEC_OK;
}

namespace {

// Completion of the chunks decoded by worker threads.
struct ChunkBoard {
    std::mutex mu;
    std::condition_variable cv;
    std::vector<int> state;   // 0 pending, 1 decoded, < 0 failed (status)
    std::atomic<int> next{0};
    std::atomic<bool> stop{false};
};

}  // namespace

jdec_status decode_jpeg(jdec_ctx *ctx, const uint8_t *data, size_t size, uint8_t *rgb, int64_t pitch, uint32_t flags,
                        int threads, cudaStream_t s)
{
    JpegScan *J = nullptr;
    jdec_jpeg_info in;
    jdec_status st = scan_open(data, size, &J, &in);
    if (st != JDEC_OK) return st;
    struct Closer {
        JpegScan *J;
        ~Closer() { scan_close(J); }
    } closer{J};

    // the image as the back-end sees it (device planes owned by the context)
    const int ncomp = in.ncomp;   // 3, or 1 (grayscale)
    size_t off[3] = {0, 0, 0}, tot = 0;
    for (int c = 0; c < ncomp; ++c) {
        off[c] = tot;
        tot += (static_cast<size_t>(in.blocks_w[c]) * in.blocks_h[c] * 128 + 255) & ~static_cast<size_t>(255);
    }
    st = ensure_buffer(ctx, &ctx->p_coef, &ctx->p_coef_cap, tot);
    if (st != JDEC_OK) return st;
    if (ctx->p_pending) {   // the previous call's copies still read the staging buffer
        cudaEventSynchronize(ctx->p_ev[65]);
        ctx->p_pending = false;
    }
    st = ensure_pinned(ctx, tot);
    if (st != JDEC_OK) return st;
    jdec_image dimg;
    memset(&dimg, 0, sizeof(dimg));
    dimg.width = in.width;
    dimg.height = in.height;
    dimg.ncomp = ncomp;
    for (int c = 0; c < 3; ++c) {
        dimg.h_samp[c] = in.h_samp[c];
        dimg.v_samp[c] = in.v_samp[c];
    }
    for (int c = 0; c < ncomp; ++c) {
        dimg.coef[c] = reinterpret_cast<const int16_t *>(static_cast<uint8_t *>(ctx->p_coef) + off[c]);
        dimg.blocks_w[c] = in.blocks_w[c];
        dimg.blocks_h[c] = in.blocks_h[c];
        dimg.qtab[c] = in.qtab[c];
    }
    dimg.rgb = rgb;
    dimg.rgb_pitch = pitch;
    dimg.flags = flags;
    Geometry g;
    st = validate(&dimg, &g, false);
    if (st != JDEC_OK) return st;
    int16_t *hplanes[3] = {nullptr, nullptr, nullptr};
    for (int c = 0; c < ncomp; ++c)
        hplanes[c] = reinterpret_cast<int16_t *>(static_cast<uint8_t *>(ctx->p_host) + off[c]);

    // chunk boundaries: the context's chunk size, else 8 chunks (about 8
    // per worker when decoding in parallel); parallel chunks are whole
    // restart intervals
    const int my = g.mcus_y;
    const int step = scan_row_step(J);
    const bool parallel = threads > 1 && step > 0 && step < my && scan_prepare_independent(J) == JDEC_OK;
    int chunk = std::max(1, (my + 7) / 8);
    if (ctx->opt.jpeg_chunk_rows > 0) chunk = std::min(ctx->opt.jpeg_chunk_rows, my);
    else if (parallel) chunk = std::max(1, my / (8 * threads));
    if (parallel) chunk = std::max(step, (chunk + step - 1) / step * step);
    std::vector<int> b;
    for (int r = 0; r < my; r += chunk) b.push_back(r);
    while (b.size() > 64) {   // bounded number of events per call
        chunk *= 2;
        b.clear();
        for (int r = 0; r < my; r += chunk) b.push_back(r);
    }
    b.push_back(my);
    const int nch = static_cast<int>(b.size()) - 1;

    if (!ctx->p_h2d) {
        if (cudaStreamCreateWithFlags(&ctx->p_h2d, cudaStreamNonBlocking) != cudaSuccess) return JDEC_ECUDA;
        if (cudaStreamCreateWithFlags(&ctx->p_comp, cudaStreamNonBlocking) != cudaSuccess) return JDEC_ECUDA;
    }
    cudaEvent_t fork = pipe_event(ctx, 64), guard = pipe_event(ctx, 65);
    if (!fork || !guard || !pipe_event(ctx, nch)) return JDEC_ECUDA;
    if (cudaEventRecord(fork, s) != cudaSuccess) return JDEC_ECUDA;
    cudaStreamWaitEvent(ctx->p_h2d, fork, 0);
    cudaStreamWaitEvent(ctx->p_comp, fork, 0);

    // workers (parallel mode)
    ChunkBoard board;
    board.state.assign(nch, 0);
    std::vector<std::thread> pool;
    if (parallel) {
        const int nw = std::min(threads, nch);
        for (int w = 0; w < nw; ++w)
            pool.emplace_back([&]() {
                for (;;) {
                    const int k = board.next.fetch_add(1);
                    if (k >= nch || board.stop.load()) return;
                    const jdec_status r = scan_decode_rows(J, hplanes, b[k], b[k + 1], true);
                    {
                        std::lock_guard<std::mutex> lk(board.mu);
                        board.state[k] = r == JDEC_OK ? 1 : static_cast<int>(r);
                    }
                    board.cv.notify_all();
                }
            });
    }

    const int lookahead = (g.fancy && g.vm == 2) ? 1 : 0;
    for (int k = 0; k < nch && st == JDEC_OK; ++k) {
        if (parallel) {
            std::unique_lock<std::mutex> lk(board.mu);
            board.cv.wait(lk, [&] { return board.state[k] != 0; });
            if (board.state[k] < 0) st = static_cast<jdec_status>(board.state[k]);
        } else {
            st = scan_decode_rows(J, hplanes, b[k], b[k + 1], false);
        }
        if (st != JDEC_OK) break;
        for (int c = 0; c < ncomp; ++c) {
            const int v = c ? 1 : g.vm;
            const size_t row_bytes = static_cast<size_t>(in.blocks_w[c]) * 128;
            const size_t o = static_cast<size_t>(b[k]) * v * row_bytes;
            const size_t n = static_cast<size_t>(b[k + 1] - b[k]) * v * row_bytes;
            if (cudaMemcpyAsync(static_cast<uint8_t *>(ctx->p_coef) + off[c] + o,
                                reinterpret_cast<const uint8_t *>(hplanes[c]) + o, n, cudaMemcpyHostToDevice,
                                ctx->p_h2d) != cudaSuccess) {
                st = JDEC_ECUDA;
                break;
            }
        }
        if (st != JDEC_OK) break;
        cudaEventRecord(ctx->p_ev[k], ctx->p_h2d);
        cudaStreamWaitEvent(ctx->p_comp, ctx->p_ev[k], 0);
        const int kd = k - lookahead;   // chunk whose rows can be transformed now
        if (kd >= 0) st = launch_rows(ctx, &dimg, g, ctx->p_comp, b[kd], b[kd + 1], 0);
    }
    if (st == JDEC_OK && lookahead && nch > 0) st = launch_rows(ctx, &dimg, g, ctx->p_comp, b[nch - 1], b[nch], 0);
    board.stop.store(true);
    for (auto &t : pool) t.join();
    // staging reuse guard and the join back to the caller's stream (also on
    // failure: work already issued must finish before the caller's next use)
    cudaEventRecord(guard, ctx->p_h2d);
    ctx->p_pending = true;
    cudaEventRecord(fork, ctx->p_comp);
    cudaStreamWaitEvent(s, fork, 0);
    cudaStreamWaitEvent(s, guard, 0);
    return st;
}

void release_pipeline(jdec_ctx *ctx)
{
    if (ctx->p_pending && ctx->n_p_ev > 65) cudaEventSynchronize(ctx->p_ev[65]);
    if (ctx->p_coef) cudaFree(ctx->p_coef);
    ctx->owned_bytes -= ctx->p_coef_cap;
    ctx->p_coef = nullptr;
    ctx->p_coef_cap = 0;
    if (ctx->p_host) cudaFreeHost(ctx->p_host);
    ctx->p_host = nullptr;
    ctx->p_host_cap = 0;
    for (int i = 0; i < ctx->n_p_ev; ++i) cudaEventDestroy(ctx->p_ev[i]);
    ctx->n_p_ev = 0;
    if (ctx->p_h2d) cudaStreamDestroy(ctx->p_h2d);
    if (ctx->p_comp) cudaStreamDestroy(ctx->p_comp);
    ctx->p_h2d = ctx->p_comp = nullptr;
}

}  // namespace jdec

extern "C" JDEC_API jdec_status jdec_decode_jpeg(jdec_ctx *ctx, const uint8_t *data, size_t size, uint8_t *rgb,
                                                 int64_t rgb_pitch, uint32_t flags, int32_t threads, void *stream)
{
    if (!ctx || !data || !rgb) return JDEC_EINVAL;
    if (flags & ~(JDEC_UPSAMPLE_REPLICATE | JDEC_IDCT_AAN)) return JDEC_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return JDEC_ECUDA;
    if (dev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess) return JDEC_ECUDA;
    const jdec_status st = jdec::decode_jpeg(ctx, data, size, rgb, rgb_pitch, flags, threads,
                                             static_cast<cudaStream_t>(stream));
    if (dev != ctx->device) cudaSetDevice(dev);
    return st;
}
