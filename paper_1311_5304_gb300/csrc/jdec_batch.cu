// jdec_batch.cu -- batched decoding of many images.
#include <cuda_runtime.h>

#include "jdec_launch.h"
#include "jdec_runtime.h"

namespace jdec {

struct BatchState {
    int unused = 0;
};

jdec_status decode_batch(jdec_ctx *ctx, const jdec_image *imgs, int n, cudaStream_t s)
{
    Geometry g;
    for (int i = 0; i < n; ++i) {
        jdec_status st = validate(&imgs[i], &g, false);
        if (st != JDEC_OK) return st;
    }
    for (int i = 0; i < n; ++i) {
        validate(&imgs[i], &g, false);
        jdec_status st = launch_image(ctx, &imgs[i], g, s, 0);
        if (st != JDEC_OK) return st;
    }
    return JDEC_OK;
}

void release_batch(jdec_ctx *ctx)
{
    delete ctx->batch;
    ctx->batch = nullptr;
}

}  // namespace jdec
