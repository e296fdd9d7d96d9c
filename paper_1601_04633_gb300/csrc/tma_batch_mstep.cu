// Multi-step batched-sweep kernel tiles (several time steps per launch):
// float32 and mixed storage, both roundings (see step_tma_batch.cuh).
#include "dmrt.h"
#include "step_tma.cuh"
#include "step_tma_batch.cuh"
#include "tma_variants.h"

namespace dmrt {

using Mixed = Split<__half, float>;

static const TmaVariant kVariants[] = {
    {DMRT_FP32, DMRT_ROUND_NEAREST, 1, 2, 2, 0, (const void*)step_tma_batch_mstep_kernel<OneType<float>, 1, 2, 2>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 2, 1, 2, 0, (const void*)step_tma_batch_mstep_kernel<OneType<float>, 2, 1, 2>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 2, 2, 2, 0, (const void*)step_tma_batch_mstep_kernel<OneType<float>, 2, 2, 2>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 2, 2, 3, 0, (const void*)step_tma_batch_mstep_kernel<OneType<float>, 2, 2, 3>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 4, 2, 2, 0, (const void*)step_tma_batch_mstep_kernel<OneType<float>, 4, 2, 2>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 4, 4, 2, 0, (const void*)step_tma_batch_mstep_kernel<OneType<float>, 4, 4, 2>},
    {DMRT_MIXED, DMRT_ROUND_NEAREST, 2, 2, 2, 0, (const void*)step_tma_batch_mstep_kernel<Mixed, 2, 2, 2>},
    {DMRT_MIXED, DMRT_ROUND_NEAREST, 4, 2, 2, 0, (const void*)step_tma_batch_mstep_kernel<Mixed, 4, 2, 2>},
    {DMRT_MIXED, DMRT_ROUND_NEAREST, 4, 4, 2, 0, (const void*)step_tma_batch_mstep_kernel<Mixed, 4, 4, 2>},
    {DMRT_MIXED, DMRT_ROUND_STOCHASTIC, 2, 2, 2, 0, (const void*)step_tma_batch_mstep_kernel<Mixed, 2, 2, 2, true>},
    {DMRT_MIXED, DMRT_ROUND_STOCHASTIC, 4, 2, 2, 0, (const void*)step_tma_batch_mstep_kernel<Mixed, 4, 2, 2, true>},
    {DMRT_MIXED, DMRT_ROUND_STOCHASTIC, 4, 4, 2, 0, (const void*)step_tma_batch_mstep_kernel<Mixed, 4, 4, 2, true>},
};

const TmaVariant* tma_variants_batch_mstep(int* n) {
    *n = (int)(sizeof(kVariants) / sizeof(kVariants[0]));
    return kVariants;
}

}  // namespace dmrt
