// jdec_kernels.cu -- __global__ entry point of the single-image launch.
//
//   jdec_fused_kernel<HM, VM, FANCY, QM, UNI>: one image; CTA b runs share b of the
//     image's strip-rows (see run_share).
//
// Variants: (HM, VM) = (1,1) 4:4:4, (2,1) 4:2:2, (2,2) 4:2:0, (1,2) 4:4:0; FANCY selects
// the triangular filter of Alg. 1 (Sec. 4.2) over replication; QM the
// dequantisation + IDCT mode (LLM with 32-bit or 8-bit tables, or AAN).
#include "jdec_kernels.cuh"

namespace jdec {

// FW > 0: the launch's strip width is FW (full strips run compile-time-width
// code, see run_share).
template <int HM, int VM, bool FANCY, int QM, bool UNI, int FW = 0>
__global__ void __launch_bounds__(kCtaThreads, JDEC_MIN_CTAS) jdec_fused_kernel(const __grid_constant__ DecodeParams p)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = align1024(smem_raw);
    const SmemLayout L = smem_layout(HM, VM, FANCY, p.img.wt, p.img.nslot);
    load_qtables<QM>(reinterpret_cast<int *>(smem + L.off_q), p.img, threadIdx.x, blockDim.x);
    if (threadIdx.x == 0) {
        *reinterpret_cast<volatile int *>(smem + L.off_flag) = 0;
        for (int s = 0; s < kStages; ++s) mbar_init(smem_u32(smem + L.off_bar + 8 * s), 1);
        fence_barrier_init();
        for (int c = 0; c < 3; ++c) tma_prefetch_map(&p.tmap[c]);
    }
    __syncthreads();
    PipeState ps{0u, 0, 0};
    run_share<HM, VM, FANCY, QM, UNI, FW>(p.tmap, p.img, blockIdx.x, smem, L, ps, p.err, p.work);
    finish_work(p.work);
}

template <int HM, int VM, bool FANCY, int QM, bool UNI = false, int FW = 0>
static cudaError_t launch_variant(const DecodeParams &p, int grid, int smem, cudaStream_t s)
{
    auto k = jdec_fused_kernel<HM, VM, FANCY, QM, UNI, FW>;
    static ConfigFlags configured;
    cudaError_t e = configure_kernel(k, configured);
    if (e != cudaSuccess) return e;
    k<<<grid, kCtaThreads, smem, s>>>(p);
    return cudaGetLastError();
}

template <int QM>
static cudaError_t launch_q(int hm, int vm, bool fancy, bool uni, const DecodeParams &p, int grid, int smem,
                            cudaStream_t s)
{
    if (hm == 1 && vm == 1) return launch_variant<1, 1, false, QM>(p, grid, smem, s);
    if (hm == 1) return fancy ? launch_variant<1, 2, true, QM>(p, grid, smem, s) : launch_variant<1, 2, false, QM>(p, grid, smem, s);
    if (vm == 1) {
        if (!fancy) return launch_variant<2, 1, false, QM>(p, grid, smem, s);
        return uni ? launch_variant<2, 1, true, QM, true>(p, grid, smem, s) : launch_variant<2, 1, true, QM>(p, grid, smem, s);
    }
    if (!fancy) return launch_variant<2, 2, false, QM>(p, grid, smem, s);
    return uni ? launch_variant<2, 2, true, QM, true>(p, grid, smem, s) : launch_variant<2, 2, true, QM>(p, grid, smem, s);
}

// The compile-time-width instances (see fixed_wt): split roles for 4:4:4,
// unified roles for the triangular 4:2:2 / 4:2:0 strips.
static cudaError_t launch_fixed(int hm, int vm, bool fancy, const DecodeParams &p, int grid, int smem,
                                cudaStream_t s)
{
    if (p.img.qmode != kQ8 || p.img.wt != fixed_wt(hm, vm, fancy, kQ8)) return cudaErrorInvalidValue;
    if (hm == 1 && vm == 1) return launch_variant<1, 1, false, kQ8, false, 32>(p, grid, smem, s);
    if (hm == 2 && vm == 1 && fancy) return launch_variant<2, 1, true, kQ8, true, 31>(p, grid, smem, s);
    if (hm == 2 && vm == 2 && fancy) return launch_variant<2, 2, true, kQ8, true, 20>(p, grid, smem, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_fused(int hm, int vm, bool fancy, bool unified, bool fixed, const DecodeParams &p, int grid,
                         int smem, cudaStream_t s)
{
    if (fixed) return launch_fixed(hm, vm, fancy, p, grid, smem, s);
    switch (p.img.qmode) {
    case kQ16: return launch_q<kQ16>(hm, vm, fancy, unified, p, grid, smem, s);
    case kQ8: return launch_q<kQ8>(hm, vm, fancy, unified, p, grid, smem, s);
    case kAAN: return launch_q<kAAN>(hm, vm, fancy, unified, p, grid, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int HM, int VM, bool FANCY>
static int occupancy_variant(int smem)
{
    int n = 0;
    auto k = jdec_fused_kernel<HM, VM, FANCY, kQ8, false>;
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
