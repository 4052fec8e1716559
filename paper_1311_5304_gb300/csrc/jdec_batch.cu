// jdec_batch.cu -- batched decoding of many images with one persistent launch.
//
// Host side of jdec_decode_batch: every image is cut into strips of its
// variant's width; for each variant class (sampling, upsampling, 8-bit or
// 16-bit tables) the strips' MCU rows of its images, concatenated image after
// image, are weighted by their decode cost and split into equal contiguous
// shares, one per resident CTA.  A CTA's work list is its share of every
// class in a fixed class order (a short list of (image, strip, row range)
// items), so all CTAs of an SM run the same variant's code at a time.  The per-image descriptors (TMA tensor
// maps, geometry, quantisation tables) and the item lists are written to
// pinned staging memory and copied to a device buffer that the kernel reads.
// The copy and the launch are recorded once per launch shape as a CUDA graph
// and replayed for later calls of the same shape.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <unordered_map>
#include <vector>

#include "jdec_launch.h"
#include "jdec_runtime.h"

namespace jdec {

namespace {

struct MapKey {
    const void *base;
    int bw, bh, box_w, box_h;
    bool operator==(const MapKey &o) const
    {
        return base == o.base && bw == o.bw && bh == o.bh && box_w == o.box_w && box_h == o.box_h;
    }
};

struct MapKeyHash {
    size_t operator()(const MapKey &k) const
    {
        size_t h = reinterpret_cast<size_t>(k.base);
        h = h * 1000003u ^ static_cast<size_t>(k.bw);
        h = h * 1000003u ^ static_cast<size_t>(k.bh);
        h = h * 1000003u ^ static_cast<size_t>(k.box_w * 1024 + k.box_h);
        return h;
    }
};

struct GraphEntry {
    size_t copy_bytes;
    int nctas, smem;
    size_t off_items, off_first;
    UnionLayout U;
    cudaGraphExec_t exec;
};

}  // namespace

struct BatchState {
    void *d_buf = nullptr;
    size_t d_cap = 0;
    void *h_buf = nullptr;
    size_t h_cap = 0;
    cudaEvent_t copied = nullptr;     // the staging buffer may be rewritten once this fires
    bool copy_pending = false;
    cudaStream_t cap_stream = nullptr;
    std::vector<GraphEntry> graphs;
    std::unordered_map<MapKey, CUtensorMap, MapKeyHash> maps;
    std::vector<BatchItem> items;
    std::vector<int32_t> first;
};

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

static size_t pow2_at_least(size_t x, size_t lo)
{
    size_t p = lo;
    while (p < x) p <<= 1;
    return p;
}

static bool cached_map(BatchState *b, CUtensorMap *out, const int16_t *base, int bw, int bh, int box_w, int box_h)
{
    const MapKey key{base, bw, bh, box_w, box_h};
    auto it = b->maps.find(key);
    if (it != b->maps.end()) {
        *out = it->second;
        return true;
    }
    if (!encode_plane_map(out, base, bw, bh, box_w, box_h)) return false;
    if (b->maps.size() > 65536) b->maps.clear();
    b->maps.emplace(key, *out);
    return true;
}

// Relative decode cost of one padded pixel per variant (measured on
// 8192x8192 images: 4:4:4 is the most expensive per pixel).
static double px_weight(int variant)
{
    static const double w[5] = {1.12, 0.95, 1.05, 0.9, 1.0};
    return w[variant];
}

static jdec_status ensure_host(BatchState *b, size_t need)
{
    if (b->h_cap >= need) return JDEC_OK;
    if (b->h_buf) cudaFreeHost(b->h_buf);
    b->h_buf = nullptr;
    b->h_cap = 0;
    if (cudaMallocHost(&b->h_buf, need) != cudaSuccess) {
        cudaGetLastError();
        return JDEC_ENOMEM;
    }
    b->h_cap = need;
    return JDEC_OK;
}

static void drop_graphs(BatchState *b)
{
    for (auto &g : b->graphs) cudaGraphExecDestroy(g.exec);
    b->graphs.clear();
}

jdec_status decode_batch(jdec_ctx *ctx, const jdec_image *imgs, int n, cudaStream_t s)
{
    std::vector<Geometry> geo(n);
    for (int i = 0; i < n; ++i) {
        jdec_status st = validate(&imgs[i], &geo[i], false);
        if (st != JDEC_OK) return st;
    }
    if (!ctx->batch) {
        ctx->batch = new (std::nothrow) BatchState();
        if (!ctx->batch) return JDEC_ENOMEM;
        if (cudaEventCreateWithFlags(&ctx->batch->copied, cudaEventDisableTiming) != cudaSuccess ||
            cudaStreamCreateWithFlags(&ctx->batch->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
            return JDEC_ECUDA;
    }
    BatchState *b = ctx->batch;

    // ---- per-image strip width and the union of the shared-memory layouts
    std::vector<int> wt(n), var(n), q8(n);
    UnionLayout U;
    memset(&U, 0, sizeof(U));
    for (int i = 0; i < n; ++i) {
        const Geometry &g = geo[i];
        int w = tuned_wt(ctx, g);
        wt[i] = std::max(1, std::min(w > 0 ? w : default_wt(g), kMaxWT));
        var[i] = variant_of(g);
        q8[i] = 1;
        for (int c = 0; c < 3; ++c)
            for (int k = 0; k < 64; ++k)
                if (imgs[i].qtab[c][k] > 255) q8[i] = 0;
        const SmemLayout L = smem_layout(g.hm, g.vm, g.fancy, wt[i], 4);
        U.stage_bytes = std::max(U.stage_bytes, L.stage_bytes);
        U.ybytes = std::max(U.ybytes, L.ybytes);
        U.slot_bytes = std::max(U.slot_bytes, L.slot_bytes);
    }
    U.off_y = kStages * U.stage_bytes;
    U.off_c = U.off_y + 2 * U.ybytes;
    U.off_q = U.off_c + 4 * U.slot_bytes;
    U.off_bar = U.off_q + 3 * 64 * 4;
    U.off_flag = U.off_bar + 8 * kStages;
    U.total = U.off_flag + 16 + 1024;
    const int smem = U.total;
    const int occ = batch_occupancy(smem);

    // ---- cost-balanced split, one variant class at a time: every CTA gets an
    // equal share of each class's strip-rows and runs the classes in the same
    // order, so the CTAs of an SM execute one variant's code at a time.
    struct Seg { int img, strip, rows; double row_cost; };
    std::vector<Seg> segs[10];
    double total[10] = {0.0};
    long total_rows = 0;
    for (int i = 0; i < n; ++i) {
        const Geometry &g = geo[i];
        const int cls = 2 * var[i] + (q8[i] ? 1 : 0);
        const int ns = (g.mcus_x + wt[i] - 1) / wt[i];
        for (int st = 0; st < ns; ++st) {
            const int w = std::min(wt[i], g.mcus_x - st * wt[i]);
            const double rc = 64.0 * g.hm * g.vm * w * px_weight(var[i]);
            segs[cls].push_back(Seg{i, st, g.mcus_y, rc});
            total[cls] += rc * g.mcus_y;
            total_rows += g.mcus_y;
        }
    }
    const int nctas = static_cast<int>(std::max<long>(1, std::min<long>(static_cast<long>(occ) * ctx->sms, total_rows)));
    std::vector<std::vector<BatchItem>> per_cta(nctas);
    for (int cls = 0; cls < 10; ++cls) {
        if (segs[cls].empty()) continue;
        const double share = total[cls] / nctas;
        int cta = 0;
        double acc = 0.0;   // cost of this class assigned to CTAs < cta plus the current CTA's part
        for (const Seg &sg : segs[cls]) {
            int r = 0;
            while (r < sg.rows) {
                const double room = (cta + 1) * share - acc;
                int take = sg.rows - r;
                if (cta < nctas - 1) {
                    const int fit = static_cast<int>(room / sg.row_cost + 0.5);
                    take = std::max(1, std::min(take, fit));
                }
                per_cta[cta].push_back(BatchItem{sg.img, sg.strip, r, r + take});
                r += take;
                acc += take * sg.row_cost;
                if (cta < nctas - 1 && acc >= (cta + 1) * share - 0.5 * sg.row_cost) ++cta;
            }
        }
    }
    b->items.clear();
    b->first.assign(nctas + 1, 0);
    for (int c = 0; c < nctas; ++c) {
        b->first[c] = static_cast<int32_t>(b->items.size());
        b->items.insert(b->items.end(), per_cta[c].begin(), per_cta[c].end());
    }
    b->first[nctas] = static_cast<int32_t>(b->items.size());
    const int nitems = static_cast<int>(b->items.size());

    // ---- staging layout: images | items | cta_first (fixed offsets per bucket)
    const size_t img_bytes = align_up(pow2_at_least(static_cast<size_t>(n), 16) * sizeof(BatchImage), 256);
    const size_t item_bytes = align_up(pow2_at_least(static_cast<size_t>(nitems), 256) * sizeof(BatchItem), 256);
    const size_t first_bytes = align_up(static_cast<size_t>(nctas + 1) * sizeof(int32_t), 256);
    const size_t off_items = img_bytes, off_first = img_bytes + item_bytes;
    const size_t bytes = off_first + first_bytes;

    void *old_dbuf = b->d_buf;
    if (b->d_cap < bytes && b->copy_pending) {
        cudaEventSynchronize(b->copied);   // earlier launches may still read the device buffer
        b->copy_pending = false;
    }
    jdec_status st = ensure_buffer(ctx, &b->d_buf, &b->d_cap, bytes);
    if (b->d_buf != old_dbuf) drop_graphs(b);   // recorded graphs point at the old buffer
    if (st != JDEC_OK) return st;
    if (b->copy_pending) {
        cudaEventSynchronize(b->copied);   // the previous copy still reads the staging buffer
        b->copy_pending = false;
    }
    if (b->h_cap < bytes) {
        drop_graphs(b);
        st = ensure_host(b, bytes);
        if (st != JDEC_OK) return st;
    }
    uint8_t *h = static_cast<uint8_t *>(b->h_buf);
    BatchImage *hi = reinterpret_cast<BatchImage *>(h);
    for (int i = 0; i < n; ++i) {
        const Geometry &g = geo[i];
        BatchImage &bi = hi[i];
        memset(&bi, 0, sizeof(bi));
        const int halo = g.fancy ? 1 : 0;
        if (!cached_map(b, &bi.tmap[0], imgs[i].coef[0], imgs[i].blocks_w[0], imgs[i].blocks_h[0], g.hm * wt[i], g.vm))
            return JDEC_ECUDA;
        for (int c = 1; c < 3; ++c)
            if (!cached_map(b, &bi.tmap[c], imgs[i].coef[c], imgs[i].blocks_w[c], imgs[i].blocks_h[c], wt[i] + 2 * halo, 1))
                return JDEC_ECUDA;
        fill_desc(&bi.desc, &imgs[i], g, wt[i], 1);
        bi.desc.nslot = 4;
        bi.desc.nidct = 64;
        bi.variant = var[i];
    }
    memcpy(h + off_items, b->items.data(), nitems * sizeof(BatchItem));
    memcpy(h + off_first, b->first.data(), (nctas + 1) * sizeof(int32_t));

    // ---- replay (or record) the copy + launch
    GraphEntry *ge = nullptr;
    for (auto &g : b->graphs)
        if (g.copy_bytes == bytes && g.nctas == nctas && g.smem == smem && g.off_items == off_items &&
            g.off_first == off_first && memcmp(&g.U, &U, sizeof(U)) == 0) {
            ge = &g;
            break;
        }
    if (!ge) {
        if (b->graphs.size() >= 64) drop_graphs(b);
        BatchParams p;
        p.imgs = static_cast<const BatchImage *>(b->d_buf);
        p.items = reinterpret_cast<const BatchItem *>(static_cast<uint8_t *>(b->d_buf) + off_items);
        p.cta_first = reinterpret_cast<const int32_t *>(static_cast<uint8_t *>(b->d_buf) + off_first);
        p.U = U;
        p.err = ctx->d_err;
        // make sure the kernel attributes are set outside the capture
        if (batch_occupancy(smem) <= 0) return JDEC_ECUDA;
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return JDEC_ECUDA;
        cudaError_t e1 = cudaMemcpyAsync(b->d_buf, b->h_buf, bytes, cudaMemcpyHostToDevice, b->cap_stream);
        cudaError_t e2 = launch_batch(p, nctas, smem, b->cap_stream);
        cudaError_t e3 = cudaStreamEndCapture(b->cap_stream, &graph);
        if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || !graph) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return JDEC_ECUDA;
        }
        cudaGraphExec_t exec = nullptr;
        cudaError_t e4 = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e4 != cudaSuccess) {
            cudaGetLastError();
            return JDEC_ECUDA;
        }
        b->graphs.push_back(GraphEntry{bytes, nctas, smem, off_items, off_first, U, exec});
        ge = &b->graphs.back();
    }
    if (cudaGraphLaunch(ge->exec, s) != cudaSuccess) return JDEC_ECUDA;
    if (cudaEventRecord(b->copied, s) == cudaSuccess) b->copy_pending = true;
    ctx->launches++;
    return JDEC_OK;
}

void release_batch(jdec_ctx *ctx)
{
    BatchState *b = ctx->batch;
    if (!b) return;
    if (b->copy_pending) cudaEventSynchronize(b->copied);
    drop_graphs(b);
    if (b->d_buf) cudaFree(b->d_buf);
    ctx->owned_bytes -= b->d_cap;
    if (b->h_buf) cudaFreeHost(b->h_buf);
    if (b->copied) cudaEventDestroy(b->copied);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    delete b;
    ctx->batch = nullptr;
}

}  // namespace jdec
