// jdec_kernels.cu -- __global__ entry points of the GB300 back-end.
//
//   jdec_fused_kernel<HM, VM, FANCY, Q8, UNI>: one image; CTA b runs share b of the
//     image's strip-rows (see run_share).
//
// Variants: (HM, VM) = (1,1) 4:4:4, (2,1) 4:2:2, (2,2) 4:2:0, (1,2) 4:4:0; FANCY selects
// the triangular filter of Alg. 1 (Sec. 4.2) over replication.
#include <cuda_runtime.h>
#include "jdec_work.cuh"
#include "jdec_launch.h"

// CTAs per SM the register allocation is sized for (128 threads each).
#ifndef JDEC_MIN_CTAS
#define JDEC_MIN_CTAS 4
#endif

namespace jdec {

__device__ __forceinline__ uint8_t *align1024(uint8_t *p)
{
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    return reinterpret_cast<uint8_t *>((a + 1023) & ~static_cast<uintptr_t>(1023));
}

// Raises a kernel's dynamic shared-memory limit to the device's opt-in
// maximum and prefers the largest shared-memory carveout, once per kernel and
// device (`done` has one flag per device ordinal).  Occupancy queries and
// launches of every size then see the same attribute.
struct ConfigFlags {
    bool done[64] = {};
};

template <typename K>
static cudaError_t configure_kernel(K k, ConfigFlags &f)
{
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && f.done[dev]) return cudaSuccess;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess && dev >= 0 && dev < 64) f.done[dev] = true;
    return e;
}

template <int HM, int VM, bool FANCY, bool Q8, bool UNI>
__global__ void __launch_bounds__(kCtaThreads, JDEC_MIN_CTAS) jdec_fused_kernel(const __grid_constant__ DecodeParams p)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = align1024(smem_raw);
    const SmemLayout L = smem_layout(HM, VM, FANCY, p.img.wt, p.img.nslot);
    load_qtables<Q8>(reinterpret_cast<int *>(smem + L.off_q), p.img, threadIdx.x, blockDim.x);
    if (threadIdx.x == 0) {
        *reinterpret_cast<volatile int *>(smem + L.off_flag) = 0;
        for (int s = 0; s < kStages; ++s) mbar_init(smem_u32(smem + L.off_bar + 8 * s), 1);
        fence_barrier_init();
        for (int c = 0; c < 3; ++c) tma_prefetch_map(&p.tmap[c]);
    }
    __syncthreads();
    PipeState ps{0u, 0, 0};
    run_share<HM, VM, FANCY, Q8, UNI>(p.tmap, p.img, blockIdx.x, smem, L, ps, p.err, true);
}

// One item of a batch with its variant's code and the union layout.
template <int HM, int VM, bool FANCY, bool Q8>
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
    return run_work<HM, VM, FANCY, Q8, false>(bi.tmap, item_desc(bi.desc), bi.desc, it.strip, it.r0, it.r1, smem, L, ps,
                                              p.err, last, reload);
}

//   jdec_batch_kernel: many images of any variants in one launch (used by the
//     allocation-free entry point, whose static scratch holds one work list);
//     CTA b runs the items [cta_first[b], cta_first[b+1]) of a flattened
//     (image, strip, row range) work list, pipelined across item boundaries.
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
    const int i0 = p.cta_first[blockIdx.x], i1 = p.cta_first[blockIdx.x + 1];
    int cur = -1;
    for (int i = i0; i < i1; ++i) {
        const BatchItem it = p.items[i];
        const BatchImage &bi = p.imgs[it.img];
        const bool reload = it.img != cur;
        cur = it.img;
        const bool last = i + 1 == i1;
        bool ok;
        const bool q8 = bi.desc.q8 != 0;
        switch (bi.variant) {
        case 0: ok = q8 ? batch_item<1, 1, false, true>(p, bi, it, smem, ps, last, reload)
                        : batch_item<1, 1, false, false>(p, bi, it, smem, ps, last, reload); break;
        case 1: ok = q8 ? batch_item<2, 1, false, true>(p, bi, it, smem, ps, last, reload)
                        : batch_item<2, 1, false, false>(p, bi, it, smem, ps, last, reload); break;
        case 2: ok = q8 ? batch_item<2, 1, true, true>(p, bi, it, smem, ps, last, reload)
                        : batch_item<2, 1, true, false>(p, bi, it, smem, ps, last, reload); break;
        case 3: ok = q8 ? batch_item<2, 2, false, true>(p, bi, it, smem, ps, last, reload)
                        : batch_item<2, 2, false, false>(p, bi, it, smem, ps, last, reload); break;
        case 4: ok = q8 ? batch_item<2, 2, true, true>(p, bi, it, smem, ps, last, reload)
                        : batch_item<2, 2, true, false>(p, bi, it, smem, ps, last, reload); break;
        case 5: ok = q8 ? batch_item<1, 2, false, true>(p, bi, it, smem, ps, last, reload)
                        : batch_item<1, 2, false, false>(p, bi, it, smem, ps, last, reload); break;
        default: ok = q8 ? batch_item<1, 2, true, true>(p, bi, it, smem, ps, last, reload)
                         : batch_item<1, 2, true, false>(p, bi, it, smem, ps, last, reload); break;
        }
        if (!ok) break;
    }
}

//   jdec_batch_class_kernel<HM, VM, FANCY, Q8>: the same work-list walk for
//     the items of one variant class only, so each launch holds one variant's
//     code (no instruction-cache competition between variants, registers
//     allocated for that variant alone).
template <int HM, int VM, bool FANCY, bool Q8>
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
    const int i0 = p.cta_first[blockIdx.x], i1 = p.cta_first[blockIdx.x + 1];
    int cur = -1;
    for (int i = i0; i < i1; ++i) {
        const BatchItem it = p.items[i];
        const BatchImage &bi = p.imgs[it.img];
        const bool reload = it.img != cur;
        cur = it.img;
        if (!batch_item<HM, VM, FANCY, Q8>(p, bi, it, smem, ps, i + 1 == i1, reload)) break;
    }
}

template <int HM, int VM, bool FANCY, bool Q8>
static cudaError_t launch_class_t(const BatchParams &p, int grid, int smem, cudaStream_t s)
{
    auto k = jdec_batch_class_kernel<HM, VM, FANCY, Q8>;
    static ConfigFlags configured;
    cudaError_t e = configure_kernel(k, configured);
    if (e != cudaSuccess) return e;
    k<<<grid, kCtaThreads, smem, s>>>(p);
    return cudaGetLastError();
}

template <int HM, int VM, bool FANCY, bool Q8>
static int occupancy_class_t(int smem)
{
    int n = 0;
    auto k = jdec_batch_class_kernel<HM, VM, FANCY, Q8>;
    static ConfigFlags configured;
    if (configure_kernel(k, configured) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kCtaThreads, smem) != cudaSuccess) return 0;
    return n;
}

// Class = 2 * variant + q8 (variant 0: 4:4:4, 1: 4:2:2 replicate, 2: 4:2:2
// triangular, 3: 4:2:0 replicate, 4: 4:2:0 triangular, 5: 4:4:0 replicate,
// 6: 4:4:0 triangular).
cudaError_t launch_batch_class(int cls, const BatchParams &p, int grid, int smem, cudaStream_t s)
{
    switch (cls) {
    case 0: return launch_class_t<1, 1, false, false>(p, grid, smem, s);
    case 1: return launch_class_t<1, 1, false, true>(p, grid, smem, s);
    case 2: return launch_class_t<2, 1, false, false>(p, grid, smem, s);
    case 3: return launch_class_t<2, 1, false, true>(p, grid, smem, s);
    case 4: return launch_class_t<2, 1, true, false>(p, grid, smem, s);
    case 5: return launch_class_t<2, 1, true, true>(p, grid, smem, s);
    case 6: return launch_class_t<2, 2, false, false>(p, grid, smem, s);
    case 7: return launch_class_t<2, 2, false, true>(p, grid, smem, s);
    case 8: return launch_class_t<2, 2, true, false>(p, grid, smem, s);
    case 9: return launch_class_t<2, 2, true, true>(p, grid, smem, s);
    case 10: return launch_class_t<1, 2, false, false>(p, grid, smem, s);
    case 11: return launch_class_t<1, 2, false, true>(p, grid, smem, s);
    case 12: return launch_class_t<1, 2, true, false>(p, grid, smem, s);
    case 13: return launch_class_t<1, 2, true, true>(p, grid, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

int batch_class_occupancy(int cls, int smem)
{
    switch (cls) {
    case 0: return occupancy_class_t<1, 1, false, false>(smem);
    case 1: return occupancy_class_t<1, 1, false, true>(smem);
    case 2: return occupancy_class_t<2, 1, false, false>(smem);
    case 3: return occupancy_class_t<2, 1, false, true>(smem);
    case 4: return occupancy_class_t<2, 1, true, false>(smem);
    case 5: return occupancy_class_t<2, 1, true, true>(smem);
    case 6: return occupancy_class_t<2, 2, false, false>(smem);
    case 7: return occupancy_class_t<2, 2, false, true>(smem);
    case 8: return occupancy_class_t<2, 2, true, false>(smem);
    case 9: return occupancy_class_t<2, 2, true, true>(smem);
    case 10: return occupancy_class_t<1, 2, false, false>(smem);
    case 11: return occupancy_class_t<1, 2, false, true>(smem);
    case 12: return occupancy_class_t<1, 2, true, false>(smem);
    case 13: return occupancy_class_t<1, 2, true, true>(smem);
    default: return 0;
    }
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

template <int HM, int VM, bool FANCY, bool Q8, bool UNI = false>
static cudaError_t launch_variant(const DecodeParams &p, int grid, int smem, cudaStream_t s)
{
    auto k = jdec_fused_kernel<HM, VM, FANCY, Q8, UNI>;
    static ConfigFlags configured;
    cudaError_t e = configure_kernel(k, configured);
    if (e != cudaSuccess) return e;
    k<<<grid, kCtaThreads, smem, s>>>(p);
    return cudaGetLastError();
}

template <bool Q8>
static cudaError_t launch_q(int hm, int vm, bool fancy, bool uni, const DecodeParams &p, int grid, int smem,
                            cudaStream_t s)
{
    if (hm == 1 && vm == 1) return launch_variant<1, 1, false, Q8>(p, grid, smem, s);
    if (hm == 1) return fancy ? launch_variant<1, 2, true, Q8>(p, grid, smem, s) : launch_variant<1, 2, false, Q8>(p, grid, smem, s);
    if (vm == 1) {
        if (!fancy) return launch_variant<2, 1, false, Q8>(p, grid, smem, s);
        return uni ? launch_variant<2, 1, true, Q8, true>(p, grid, smem, s) : launch_variant<2, 1, true, Q8>(p, grid, smem, s);
    }
    if (!fancy) return launch_variant<2, 2, false, Q8>(p, grid, smem, s);
    return uni ? launch_variant<2, 2, true, Q8, true>(p, grid, smem, s) : launch_variant<2, 2, true, Q8>(p, grid, smem, s);
}

cudaError_t launch_fused(int hm, int vm, bool fancy, bool unified, const DecodeParams &p, int grid, int smem,
                         cudaStream_t s)
{
    return p.img.q8 ? launch_q<true>(hm, vm, fancy, unified, p, grid, smem, s)
                    : launch_q<false>(hm, vm, fancy, unified, p, grid, smem, s);
}

template <int HM, int VM, bool FANCY>
static int occupancy_variant(int smem)
{
    int n = 0;
    auto k = jdec_fused_kernel<HM, VM, FANCY, true, false>;
    static ConfigFlags configured;
    if (configure_kernel(k, configured) != cudaSuccess) return 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kCtaThreads, smem) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

int fused_occupancy(int hm, int vm, bool fancy, int smem)
{
    if (hm == 1 && vm == 1) return occupancy_variant<1, 1, false>(smem);
    if (hm == 1) return fancy ? occupancy_variant<1, 2, true>(smem) : occupancy_variant<1, 2, false>(smem);
    if (vm == 1) return fancy ? occupancy_variant<2, 1, true>(smem) : occupancy_variant<2, 1, false>(smem);
    return fancy ? occupancy_variant<2, 2, true>(smem) : occupancy_variant<2, 2, false>(smem);
}

}  // namespace jdec
