// jdec_batch.cu -- batched decoding of many images in one CUDA graph.
//
// Host side of jdec_decode_batch: every image is cut into strips of its
// variant's width; for each variant class (sampling, upsampling, and the
// dequantisation/IDCT mode: LLM with 8-bit or 16-bit tables, or AAN) the strips' MCU rows of its images, concatenated image after
// image, are weighted by their decode cost and split into equal contiguous
// shares, one per resident CTA of that class's kernel.  Each class runs as one
// persistent launch over its (image, strip, row range) work list, holding
// only that variant's code; the launches follow each other on the stream.
// The per-image descriptors (TMA tensor maps, geometry, quantisation tables)
// and the work lists are written to pinned staging memory and copied to a
// device buffer that the kernels read.  The copy and the launches are
// recorded once per launch shape as a CUDA graph and replayed for later calls
// of the same shape.
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

// One class launch of a batch: grid, shared memory, layout, and where its
// per-CTA item offsets start in the staging buffer.
struct ClassLaunch {
    int cls, nctas, smem;
    size_t first_off;
    UnionLayout U;
    bool operator==(const ClassLaunch &o) const
    {
        return cls == o.cls && nctas == o.nctas && smem == o.smem && first_off == o.first_off &&
               memcmp(&U, &o.U, sizeof(U)) == 0;
    }
};

struct GraphEntry {
    size_t copy_bytes;
    size_t off_items;
    std::vector<ClassLaunch> launches;
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
    if (!base) return false;
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
// 8192x8192 images: 4:4:4 is the most expensive per pixel; 4:4:0 taken as
// 4:2:2, which has as many blocks per pixel).
static double px_weight(int variant)
{
    static const double w[kVariants] = {1.12, 0.95, 1.05, 0.9, 1.0, 0.95, 1.0};
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
            cudaStreamCreateWithFlags(&ctx->batch->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
            release_batch(ctx);   // a later call starts over instead of using half-made state
            return JDEC_ECUDA;
        }
    }
    BatchState *b = ctx->batch;

    // ---- per-image strip width, variant class, and per class the union of
    // its images' shared-memory layouts
    std::vector<int> wt(n), var(n), cls_of(n);
    UnionLayout U[kClasses];
    memset(U, 0, sizeof(U));
    for (int i = 0; i < n; ++i) {
        const Geometry &g = geo[i];
        int w = tuned_wt(ctx, g);
        wt[i] = std::max(1, std::min(w > 0 ? w : equal_strips(g.mcus_x, default_wt(g)), kMaxWT));
        var[i] = variant_of(g);
        cls_of[i] = kQModes * var[i] + qmode_of(&imgs[i], g);
        UnionLayout &u = U[cls_of[i]];
        // one variant per class launch: its own number of chroma slots
        u.nslot = default_slots(g.hm, g.vm, g.fancy);
        const SmemLayout L = smem_layout(g.hm, g.vm, g.fancy, wt[i], u.nslot);
        u.stage_bytes = std::max(u.stage_bytes, L.stage_bytes);
        u.ybytes = std::max(u.ybytes, L.ybytes);
        u.slot_bytes = std::max(u.slot_bytes, L.slot_bytes);
    }
    for (int c = 0; c < kClasses; ++c) {
        UnionLayout &u = U[c];
        u.off_y = kStages * u.stage_bytes;
        u.off_c = u.off_y + 2 * u.ybytes;
        u.off_q = u.off_c + u.nslot * u.slot_bytes;
        u.off_bar = u.off_q + 3 * 64 * 4;
        u.off_flag = u.off_bar + 8 * kStages;
        u.total = u.off_flag + 16 + 1024;
    }

    // ---- per class: cost-balanced split of its strip-rows over one wave of
    // that class's CTAs
    struct Seg { int img, strip, rows; double row_cost; };
    std::vector<Seg> segs[kClasses];
    double total[kClasses] = {0.0};
    long rows_of[kClasses] = {0};
    for (int i = 0; i < n; ++i) {
        const Geometry &g = geo[i];
        const int cls = cls_of[i];
        const int ns = (g.mcus_x + wt[i] - 1) / wt[i];
        for (int st = 0; st < ns; ++st) {
            const int w = std::min(wt[i], g.mcus_x - st * wt[i]);
            const double rc = 64.0 * g.hm * g.vm * w * px_weight(var[i]);
            segs[cls].push_back(Seg{i, st, g.mcus_y, rc});
            total[cls] += rc * g.mcus_y;
            rows_of[cls] += g.mcus_y;
        }
    }
    std::vector<ClassLaunch> launches;
    b->items.clear();
    b->first.clear();
    for (int cls = 0; cls < kClasses; ++cls) {
        if (segs[cls].empty()) continue;
        const int smem = U[cls].total;
        const int occ = batch_class_occupancy(cls, smem);   // also sets the kernel's attributes
        if (occ <= 0) return JDEC_ECUDA;
        const int nctas = static_cast<int>(std::max<long>(1, std::min<long>(static_cast<long>(occ) * ctx->sms,
                                                                            rows_of[cls])));
        std::vector<std::vector<BatchItem>> per_cta(nctas);
        const double share = total[cls] / nctas;
        int cta = 0;
        double acc = 0.0;   // cost assigned to CTAs < cta plus the current CTA's part
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
        launches.push_back(ClassLaunch{cls, nctas, smem, b->first.size(), U[cls]});
        for (int c = 0; c < nctas; ++c) {
            b->first.push_back(static_cast<int32_t>(b->items.size()));
            b->items.insert(b->items.end(), per_cta[c].begin(), per_cta[c].end());
        }
        b->first.push_back(static_cast<int32_t>(b->items.size()));
    }
    const int nitems = static_cast<int>(b->items.size());
    const size_t nfirst = b->first.size();

    // ---- staging layout: images | items | cta_first (fixed offsets per bucket)
    const size_t img_bytes = align_up(pow2_at_least(static_cast<size_t>(n), 16) * sizeof(BatchImage), 256);
    const size_t item_bytes = align_up(pow2_at_least(static_cast<size_t>(nitems), 256) * sizeof(BatchItem), 256);
    const size_t first_bytes = align_up(pow2_at_least(nfirst, 256) * sizeof(int32_t), 256);
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
        const int halo = chroma_halo(g.hm, g.fancy);
        if (!cached_map(b, &bi.tmap[0], imgs[i].coef[0], imgs[i].blocks_w[0], imgs[i].blocks_h[0], g.hm * wt[i], g.vm))
            return JDEC_ECUDA;
        for (int c = 1; c < 3; ++c) {
            // grayscale: zero chroma tiles (see zero_plane)
            const bool ok = g.gray ? cached_map(b, &bi.tmap[c], zero_plane(), kZeroPlaneBlocks, 1, wt[i], 1)
                                   : cached_map(b, &bi.tmap[c], imgs[i].coef[c], imgs[i].blocks_w[c],
                                                imgs[i].blocks_h[c], wt[i] + 2 * halo, 1);
            if (!ok) return JDEC_ECUDA;
        }
        fill_desc(&bi.desc, &imgs[i], g, wt[i], 1);
        bi.desc.nslot = default_slots(g.hm, g.vm, g.fancy);
        bi.desc.nidct = 64;
        bi.variant = var[i];
    }
    memcpy(h + off_items, b->items.data(), nitems * sizeof(BatchItem));
    memcpy(h + off_first, b->first.data(), nfirst * sizeof(int32_t));

    // ---- replay (or record) the copy + the class launches
    GraphEntry *ge = nullptr;
    for (auto &g : b->graphs)
        if (g.copy_bytes == bytes && g.off_items == off_items && g.launches == launches) {
            ge = &g;
            break;
        }
    if (!ge) {
        if (b->graphs.size() >= 64) drop_graphs(b);
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return JDEC_ECUDA;
        cudaError_t e1 = cudaMemcpyAsync(b->d_buf, b->h_buf, bytes, cudaMemcpyHostToDevice, b->cap_stream);
        cudaError_t e2 = cudaSuccess;
        for (const ClassLaunch &cl : launches) {
            BatchParams p;
            p.imgs = static_cast<const BatchImage *>(b->d_buf);
            p.items = reinterpret_cast<const BatchItem *>(static_cast<uint8_t *>(b->d_buf) + off_items);
            p.cta_first = reinterpret_cast<const int32_t *>(static_cast<uint8_t *>(b->d_buf) + off_first) + cl.first_off;
            p.U = cl.U;
            p.err = ctx->d_err;
            if (e2 == cudaSuccess) e2 = launch_batch_class(cl.cls, p, cl.nctas, cl.smem, b->cap_stream);
        }
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
        b->graphs.push_back(GraphEntry{bytes, off_items, launches, exec});
        ge = &b->graphs.back();
    }
    if (cudaGraphLaunch(ge->exec, s) != cudaSuccess) return JDEC_ECUDA;
    if (cudaEventRecord(b->copied, s) == cudaSuccess) b->copy_pending = true;
    ctx->launches += static_cast<long>(launches.size());
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
