// jdec_kernels.cuh -- shared by the translation units that hold the
// __global__ entry points (jdec_kernels.cu: one image per launch;
// jdec_kernels_batch.cu: the batch kernels).
#pragma once
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
inline cudaError_t configure_kernel(K k, ConfigFlags &f)
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

}  // namespace jdec
