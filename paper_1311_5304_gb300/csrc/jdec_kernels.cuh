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

// The first 1024-byte aligned byte of the dynamic shared-memory window (the
// 128-byte TMA swizzle repeats every 1024 bytes).  The pointer is formed by
// adding an offset to the shared array itself, so every pointer derived from
// it stays a shared-space pointer: shared loads and stores with 32-bit
// addresses instead of generic ones.
__device__ __forceinline__ uint8_t *align1024(uint8_t *p)
{
    return p + ((1024u - (smem_u32(p) & 1023u)) & 1023u);
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
