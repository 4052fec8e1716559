// jdec_launch.h -- host-side launch interface of the kernels TU.
#pragma once

#include <cuda_runtime.h>
#include "jdec_common.h"

namespace jdec {

struct BatchParams;   // jdec_batch_types.h

// unified: every warp transforms and converts (triangular 4:2:2 / 4:2:0 only);
// fixed: the compile-time-width instance for p.img.wt == fixed_wt(...)
// (unified roles for 4:2:2 / 4:2:0, split for 4:4:4 with kFixedIdctThreads IDCT threads)
cudaError_t launch_fused(int hm, int vm, bool fancy, bool unified, bool fixed, const DecodeParams &p, int grid,
                         int smem, cudaStream_t s);
int fused_occupancy(int hm, int vm, bool fancy, int smem);
cudaError_t launch_batch(const BatchParams &p, int grid, int smem, cudaStream_t s);
int batch_occupancy(int smem);
cudaError_t launch_batch_class(int cls, const BatchParams &p, int grid, int smem, cudaStream_t s);
int batch_class_occupancy(int cls, int smem);   // 0 if the class cannot be resident

}  // namespace jdec
