// jdec_batch_types.h -- descriptors and kernel parameters of the batched
// launches (kept apart from jdec_common.h, which the single-image kernel
// shares).
#pragma once

#include "jdec_common.h"

namespace jdec {

// One image of a batched launch (device memory, 128-byte aligned: the tensor
// maps are read from global memory by TMA).
struct alignas(128) BatchImage {
    CUtensorMap tmap[3];
    ImageDesc desc;
    int32_t variant;        // 0: 4:4:4, 1/2: 4:2:2, 3/4: 4:2:0, 5/6: 4:4:0 (replicate / triangular)
};

// A run of MCU rows [r0, r1) of one strip of one image.
struct BatchItem {
    int32_t img, strip, r0, r1;
};

// Kernel parameters of the batched launches: the CTAs claim items item0 ..
// item0 + nitems - 1 one at a time from the counter work[0] (work[1] counts
// finished CTAs; both zero at launch, the last CTA to finish resets them).
struct BatchParams {
    const BatchImage *imgs;
    const BatchItem *items;
    UnionLayout U;
    int *err;
    int *work;
    int32_t item0, nitems;
};

}  // namespace jdec
