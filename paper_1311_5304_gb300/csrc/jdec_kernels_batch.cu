// jdec_kernels_batch.cu -- __global__ entry points of the batched launches.
#include "jdec_batch_types.h"
#include "jdec_kernels.cuh"

namespace jdec {

// One item of a batch with its variant's code and the union layout.
template <int HM, int VM, bool FANCY, int QM>
__device__ __forceinline__ bool batch_item(const BatchParams &p, const BatchImage &bi, const BatchItem &it, uint8_t *smem,
                                           PipeState &ps, bool last, bool reload)
{
    const SmemLayout L = apply_union(smem_layout(HM, VM, FANCY, bi.desc.wt, p.U.nslot), p.U);
    // wt also sizes the layout: read once
    if (reload && threadIdx.x == 0)
        for (int c = 0; c < 3; ++c) {
            tensormap_acquire(&bi.tmap[c]);
            tma_prefetch_map(&bi.tmap[c]);
        }
    // batches hold many small and narrow images: split roles
    return run_work<HM, VM, FANCY, QM, false>(bi.tmap, item_desc(bi.desc), bi.desc, it.strip, it.r0, it.r1, smem, L, ps,
                                              p.err, last, reload);
}

//   jdec_batch_kernel: many images of any variants in one launch (used by the
//     allocation-free entry point, whose static scratch holds one work list);
//     the CTAs claim the (image, strip, row range) items one at a time from
//     the launch's counter, as the class launches below do.
__global__ void __launch_bounds__(kCtaThreads, JDEC_MIN_CTAS) jdec_batch_kernel(const __grid_constant__ BatchParams p)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = align1024(smem_raw);
    if (threadIdx.x == 0) {
        *reinterpret_cast<volatile int *>(smem + p.U.off_flag) = 0;
        for (int s = 0; s < kStages; ++s) mbar_init(smem_u32(smem + p.U.off_bar + 8 * s), 1);
        fence_barrier_init();
    }
    __syncthreads();
    PipeState ps{0u, 0, 0};
    volatile int *claim = reinterpret_cast<volatile int *>(smem + p.U.off_flag + 4);
    int cur = -1;
    for (;;) {
        __syncthreads();   // every thread has read the previous claim
        if (threadIdx.x == 0) *claim = atomicAdd(p.work, 1);
        __syncthreads();
        const int c = *claim;
        if (c >= p.nitems) break;
        const BatchItem it = p.items[p.item0 + c];
        const BatchImage &bi = p.imgs[it.img];
        const bool reload = it.img != cur;
        cur = it.img;
        const bool last = true;   // each item drains the split-role pipeline
        bool ok;
        switch (kQModes * bi.variant + bi.desc.qmode) {
        case 0: ok = batch_item<1, 1, false, kQ16>(p, bi, it, smem, ps, last, reload); break;
        case 1: ok = batch_item<1, 1, false, kQ8>(p, bi, it, smem, ps, last, reload); break;
        case 2: ok = batch_item<1, 1, false, kAAN>(p, bi, it, smem, ps, last, reload); break;
        case 3: ok = batch_item<2, 1, false, kQ16>(p, bi, it, smem, ps, last, reload); break;
        case 4: ok = batch_item<2, 1, false, kQ8>(p, bi, it, smem, ps, last, reload); break;
        case 5: ok = batch_item<2, 1, false, kAAN>(p, bi, it, smem, ps, last, reload); break;
        case 6: ok = batch_item<2, 1, true, kQ16>(p, bi, it, smem, ps, last, reload); break;
        case 7: ok = batch_item<2, 1, true, kQ8>(p, bi, it, smem, ps, last, reload); break;
        case 8: ok = batch_item<2, 1, true, kAAN>(p, bi, it, smem, ps, last, reload); break;
        case 9: ok = batch_item<2, 2, false, kQ16>(p, bi, it, smem, ps, last, reload); break;
        case 10: ok = batch_item<2, 2, false, kQ8>(p, bi, it, smem, ps, last, reload); break;
        case 11: ok = batch_item<2, 2, false, kAAN>(p, bi, it, smem, ps, last, reload); break;
        case 12: ok = batch_item<2, 2, true, kQ16>(p, bi, it, smem, ps, last, reload); break;
        case 13: ok = batch_item<2, 2, true, kQ8>(p, bi, it, smem, ps, last, reload); break;
        case 14: ok = batch_item<2, 2, true, kAAN>(p, bi, it, smem, ps, last, reload); break;
        case 15: ok = batch_item<1, 2, false, kQ16>(p, bi, it, smem, ps, last, reload); break;
        case 16: ok = batch_item<1, 2, false, kQ8>(p, bi, it, smem, ps, last, reload); break;
        case 17: ok = batch_item<1, 2, false, kAAN>(p, bi, it, smem, ps, last, reload); break;
        case 18: ok = batch_item<1, 2, true, kQ16>(p, bi, it, smem, ps, last, reload); break;
        case 19: ok = batch_item<1, 2, true, kQ8>(p, bi, it, smem, ps, last, reload); break;
        case 20: ok = batch_item<1, 2, true, kAAN>(p, bi, it, smem, ps, last, reload); break;
        default: ok = false; break;
        }
        if (!ok) break;
    }
    finish_work(p.work);
}

cudaError_t launch_batch(const BatchParams &p, int grid, int smem, cudaStream_t s)
{
    static ConfigFlags configured;
    cudaError_t e = configure_kernel(jdec_batch_kernel, configured);
    if (e != cudaSuccess) return e;
    jdec_batch_kernel<<<grid, kCtaThreads, smem, s>>>(p);
    return cudaGetLastError();
}

int batch_occupancy(int smem)
{
    static ConfigFlags configured;
    int n = 0;
    if (configure_kernel(jdec_batch_kernel, configured) != cudaSuccess) return 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, jdec_batch_kernel, kCtaThreads, smem) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

//   jdec_batch_class_kernel<HM, VM, FANCY, QM>: the items of one variant
//     class only, so each launch holds one variant's code (no
//     instruction-cache competition between variants, registers allocated
//     for that variant alone).  The CTAs claim the items one at a time from
//     the launch's counter as they finish the previous one: CTAs on one SM
//     progress at different rates, and items of small images cost more per
//     pixel than their share of the pixels says, so a fixed split leaves SMs
//     idle towards the end.  Each item drains the split-role pipeline.
template <int HM, int VM, bool FANCY, int QM>
__global__ void __launch_bounds__(kCtaThreads, JDEC_MIN_CTAS)
    jdec_batch_class_kernel(const __grid_constant__ BatchParams p)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = align1024(smem_raw);
    if (threadIdx.x == 0) {
        *reinterpret_cast<volatile int *>(smem + p.U.off_flag) = 0;
        for (int s = 0; s < kStages; ++s) mbar_init(smem_u32(smem + p.U.off_bar + 8 * s), 1);
        fence_barrier_init();
    }
    __syncthreads();
    PipeState ps{0u, 0, 0};
    volatile int *claim = reinterpret_cast<volatile int *>(smem + p.U.off_flag + 4);
    int cur = -1;
    for (;;) {
        __syncthreads();   // every thread has read the previous claim
        if (threadIdx.x == 0) *claim = atomicAdd(p.work, 1);
        __syncthreads();
        const int c = *claim;
        if (c >= p.nitems) break;
        const BatchItem it = p.items[p.item0 + c];
        const BatchImage &bi = p.imgs[it.img];
        const bool reload = it.img != cur;
        cur = it.img;
        if (!batch_item<HM, VM, FANCY, QM>(p, bi, it, smem, ps, true, reload)) break;
    }
    finish_work(p.work);
}

template <int HM, int VM, bool FANCY, int QM>
static cudaError_t launch_class_t(const BatchParams &p, int grid, int smem, cudaStream_t s)
{
    auto k = jdec_batch_class_kernel<HM, VM, FANCY, QM>;
    static ConfigFlags configured;
    cudaError_t e = configure_kernel(k, configured);
    if (e != cudaSuccess) return e;
    k<<<grid, kCtaThreads, smem, s>>>(p);
    return cudaGetLastError();
}

template <int HM, int VM, bool FANCY, int QM>
static int occupancy_class_t(int smem)
{
    int n = 0;
    auto k = jdec_batch_class_kernel<HM, VM, FANCY, QM>;
    static ConfigFlags configured;
    if (configure_kernel(k, configured) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kCtaThreads, smem) != cudaSuccess) return 0;
    return n;
}

// Class = 3 * variant + mode (variant 0: 4:4:4, 1: 4:2:2 replicate, 2: 4:2:2
// triangular, 3: 4:2:0 replicate, 4: 4:2:0 triangular, 5: 4:4:0 replicate,
// 6: 4:4:0 triangular; mode kQ16, kQ8 or kAAN).
cudaError_t launch_batch_class(int cls, const BatchParams &p, int grid, int smem, cudaStream_t s)
{
    switch (cls) {
    case 0: return launch_class_t<1, 1, false, kQ16>(p, grid, smem, s);
    case 1: return launch_class_t<1, 1, false, kQ8>(p, grid, smem, s);
    case 2: return launch_class_t<1, 1, false, kAAN>(p, grid, smem, s);
    case 3: return launch_class_t<2, 1, false, kQ16>(p, grid, smem, s);
    case 4: return launch_class_t<2, 1, false, kQ8>(p, grid, smem, s);
    case 5: return launch_class_t<2, 1, false, kAAN>(p, grid, smem, s);
    case 6: return launch_class_t<2, 1, true, kQ16>(p, grid, smem, s);
    case 7: return launch_class_t<2, 1, true, kQ8>(p, grid, smem, s);
    case 8: return launch_class_t<2, 1, true, kAAN>(p, grid, smem, s);
    case 9: return launch_class_t<2, 2, false, kQ16>(p, grid, smem, s);
    case 10: return launch_class_t<2, 2, false, kQ8>(p, grid, smem, s);
    case 11: return launch_class_t<2, 2, false, kAAN>(p, grid, smem, s);
    case 12: return launch_class_t<2, 2, true, kQ16>(p, grid, smem, s);
    case 13: return launch_class_t<2, 2, true, kQ8>(p, grid, smem, s);
    case 14: return launch_class_t<2, 2, true, kAAN>(p, grid, smem, s);
    case 15: return launch_class_t<1, 2, false, kQ16>(p, grid, smem, s);
    case 16: return launch_class_t<1, 2, false, kQ8>(p, grid, smem, s);
    case 17: return launch_class_t<1, 2, false, kAAN>(p, grid, smem, s);
    case 18: return launch_class_t<1, 2, true, kQ16>(p, grid, smem, s);
    case 19: return launch_class_t<1, 2, true, kQ8>(p, grid, smem, s);
    case 20: return launch_class_t<1, 2, true, kAAN>(p, grid, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

int batch_class_occupancy(int cls, int smem)
{
    switch (cls) {
    case 0: return occupancy_class_t<1, 1, false, kQ16>(smem);
    case 1: return occupancy_class_t<1, 1, false, kQ8>(smem);
    case 2: return occupancy_class_t<1, 1, false, kAAN>(smem);
    case 3: return occupancy_class_t<2, 1, false, kQ16>(smem);
    case 4: return occupancy_class_t<2, 1, false, kQ8>(smem);
    case 5: return occupancy_class_t<2, 1, false, kAAN>(smem);
    case 6: return occupancy_class_t<2, 1, true, kQ16>(smem);
    case 7: return occupancy_class_t<2, 1, true, kQ8>(smem);
    case 8: return occupancy_class_t<2, 1, true, kAAN>(smem);
    case 9: return occupancy_class_t<2, 2, false, kQ16>(smem);
    case 10: return occupancy_class_t<2, 2, false, kQ8>(smem);
    case 11: return occupancy_class_t<2, 2, false, kAAN>(smem);
    case 12: return occupancy_class_t<2, 2, true, kQ16>(smem);
    case 13: return occupancy_class_t<2, 2, true, kQ8>(smem);
    case 14: return occupancy_class_t<2, 2, true, kAAN>(smem);
    case 15: return occupancy_class_t<1, 2, false, kQ16>(smem);
    case 16: return occupancy_class_t<1, 2, false, kQ8>(smem);
    case 17: return occupancy_class_t<1, 2, false, kAAN>(smem);
    case 18: return occupancy_class_t<1, 2, true, kQ16>(smem);
    case 19: return occupancy_class_t<1, 2, true, kQ8>(smem);
    case 20: return occupancy_class_t<1, 2, true, kAAN>(smem);
    default: return 0;
    }
}

}  // namespace jdec
