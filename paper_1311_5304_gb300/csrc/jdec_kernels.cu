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
    int *qs = reinterpret_cast<int *>(smem + L.off_q);
    if (Q8) {
        // packed per component: word 8*pr + v = Q_c(v, 2pr) | Q_c(v, 2pr+1) << 24
        for (int i = threadIdx.x; i < 96; i += blockDim.x) {
            const int c = i >> 5, pr = (i >> 3) & 3, v = i & 7;
            qs[64 * c + 8 * pr + v] = p.img.q[c][8 * v + 2 * pr] | (p.img.q[c][8 * v + 2 * pr + 1] << 24);
        }
    } else {
        // transposed per component: qs[64*c + 8*u + v] = Q_c(v, u)
        for (int i = threadIdx.x; i < 192; i += blockDim.x)
            qs[i] = p.img.q[i >> 6][((i & 7) << 3) | ((i >> 3) & 7)];
    }
    if (threadIdx.x == 0) {
        *reinterpret_cast<volatile int *>(smem + L.off_flag) = 0;
        for (int s = 0; s < kStages; ++s) mbar_init(smem_u32(smem + L.off_bar + 8 * s), 1);
        fence_barrier_init();
        for (int c = 0; c < 3; ++c) tma_prefetch_map(&p.tmap[c]);
    }
    __syncthreads();
    PipeState ps{0u, 0};
    run_share<HM, VM, FANCY, Q8>(p.tmap, p.img, blockIdx.x, smem, ps, p.err, true);
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
