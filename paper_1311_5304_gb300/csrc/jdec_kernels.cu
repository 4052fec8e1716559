// jdec_kernels.cu -- __global__ entry points of the GB300 back-end.
//
//   jdec_fused_kernel<HM, VM, FANCY>: one image; CTA b runs share b of the
//     image's strip-rows (see run_share).
//
// Variants: (HM, VM) = (1,1) 4:4:4, (2,1) 4:2:2, (2,2) 4:2:0; FANCY selects
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

template <int HM, int VM, bool FANCY, bool Q8>
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
    PipeState ps{0u, 0};
    run_share<HM, VM, FANCY, Q8>(p.tmap, p.img, blockIdx.x, smem, L, ps, p.err, true);
}

// One item of a batch with its variant's code and the union layout.
template <int HM, int VM, bool FANCY, bool Q8>
__device__ __forceinline__ bool batch_item(const BatchParams &p, const BatchImage &bi, const BatchItem &it, uint8_t *smem,
                                           PipeState &ps, bool last, bool reload)
{
    const SmemLayout L = apply_union(smem_layout(HM, VM, FANCY, bi.desc.wt, 4), p.U);
    // wt also sizes the layout: read once
    if (reload && threadIdx.x == 0)
        for (int c = 0; c < 3; ++c) {
            tensormap_acquire(&bi.tmap[c]);
            tma_prefetch_map(&bi.tmap[c]);
        }
    return run_work<HM, VM, FANCY, Q8>(bi.tmap, item_desc(bi.desc), bi.desc, it.strip, it.r0, it.r1, smem, L, ps, p.err,
                                       last, reload);
}

//   jdec_batch_kernel: many images of any variants; CTA b runs the items
//     [cta_first[b], cta_first[b+1]) of a flattened (image, strip, row range)
//     work list, pipelined across item boundaries.
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
    PipeState ps{0u, 0};
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
        default: ok = q8 ? batch_item<2, 2, true, true>(p, bi, it, smem, ps, last, reload)
                         : batch_item<2, 2, true, false>(p, bi, it, smem, ps, last, reload); break;
        }
        if (!ok) break;
    }
}

cudaError_t launch_batch(const BatchParams &p, int grid, int smem, cudaStream_t s)
{
    static int configured_smem = 0;
    if (smem > configured_smem) {
        cudaError_t e = cudaFuncSetAttribute(jdec_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        cudaFuncSetAttribute(jdec_batch_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        configured_smem = smem;
    }
    jdec_batch_kernel<<<grid, kCtaThreads, smem, s>>>(p);
    return cudaGetLastError();
}

int batch_occupancy(int smem)
{
    int n = 0;
    cudaFuncSetAttribute(jdec_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(jdec_batch_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, jdec_batch_kernel, kCtaThreads, smem) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

template <int HM, int VM, bool FANCY, bool Q8>
static cudaError_t launch_variant(const DecodeParams &p, int grid, int smem, cudaStream_t s)
{
    auto k = jdec_fused_kernel<HM, VM, FANCY, Q8>;
    static int configured_smem = 0;
    if (smem > configured_smem) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        configured_smem = smem;
    }
    k<<<grid, kCtaThreads, smem, s>>>(p);
    return cudaGetLastError();
}

template <bool Q8>
static cudaError_t launch_q(int hm, int vm, bool fancy, const DecodeParams &p, int grid, int smem, cudaStream_t s)
{
    if (hm == 1) return launch_variant<1, 1, false, Q8>(p, grid, smem, s);
    if (vm == 1)
        return fancy ? launch_variant<2, 1, true, Q8>(p, grid, smem, s) : launch_variant<2, 1, false, Q8>(p, grid, smem, s);
    return fancy ? launch_variant<2, 2, true, Q8>(p, grid, smem, s) : launch_variant<2, 2, false, Q8>(p, grid, smem, s);
}

cudaError_t launch_fused(int hm, int vm, bool fancy, const DecodeParams &p, int grid, int smem, cudaStream_t s)
{
    return p.img.q8 ? launch_q<true>(hm, vm, fancy, p, grid, smem, s) : launch_q<false>(hm, vm, fancy, p, grid, smem, s);
}

template <int HM, int VM, bool FANCY>
static int occupancy_variant(int smem)
{
    int n = 0;
    auto k = jdec_fused_kernel<HM, VM, FANCY, true>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kCtaThreads, smem) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

int fused_occupancy(int hm, int vm, bool fancy, int smem)
{
    if (hm == 1) return occupancy_variant<1, 1, false>(smem);
    if (vm == 1) return fancy ? occupancy_variant<2, 1, true>(smem) : occupancy_variant<2, 1, false>(smem);
    return fancy ? occupancy_variant<2, 2, true>(smem) : occupancy_variant<2, 2, false>(smem);
}

}  // namespace jdec
