// Batched-sweep TMA step-kernel tiles (float32 storage; see step_tma.cuh).
#include "dmrt.h"
#include "step_tma.cuh"
#include "tma_variants.h"

namespace dmrt {

static const TmaVariant kVariants[] = {
    {DMRT_FP32, DMRT_ROUND_NEAREST, 1, 1, 2, 0, (const void*)step_tma_batch_kernel<1, 1, 2>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 1, 2, 2, 0, (const void*)step_tma_batch_kernel<1, 2, 2>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 1, 4, 2, 0, (const void*)step_tma_batch_kernel<1, 4, 2>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 1, 4, 3, 0, (const void*)step_tma_batch_kernel<1, 4, 3>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 2, 2, 2, 0, (const void*)step_tma_batch_kernel<2, 2, 2>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 2, 4, 2, 0, (const void*)step_tma_batch_kernel<2, 4, 2>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 4, 1, 4, 0, (const void*)step_tma_batch_kernel<4, 1, 4>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 4, 4, 2, 0, (const void*)step_tma_batch_kernel<4, 4, 2>},
};

const TmaVariant* tma_variants_batch(int* n) {
    *n = (int)(sizeof(kVariants) / sizeof(kVariants[0]));
    return kVariants;
}

}  // namespace dmrt
