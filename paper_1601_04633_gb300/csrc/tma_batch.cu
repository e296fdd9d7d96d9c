// Batched-sweep TMA step-kernel tiles: float32 and mixed storage (see step_tma.cuh).
#include "dmrt.h"
#include "step_tma.cuh"
#include "step_tma_batch.cuh"
#include "tma_variants.h"

namespace dmrt {

static const TmaVariant kVariants[] = {
    {DMRT_FP32, DMRT_ROUND_NEAREST, 1, 1, 2, 0, (const void*)step_tma_batch_kernel<OneType<float>, 1, 1, 2>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 1, 2, 2, 0, (const void*)step_tma_batch_kernel<OneType<float>, 1, 2, 2>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 1, 4, 2, 0, (const void*)step_tma_batch_kernel<OneType<float>, 1, 4, 2>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 1, 4, 3, 0, (const void*)step_tma_batch_kernel<OneType<float>, 1, 4, 3>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 2, 2, 2, 0, (const void*)step_tma_batch_kernel<OneType<float>, 2, 2, 2>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 2, 4, 2, 0, (const void*)step_tma_batch_kernel<OneType<float>, 2, 4, 2>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 4, 1, 4, 0, (const void*)step_tma_batch_kernel<OneType<float>, 4, 1, 4>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 4, 4, 2, 0, (const void*)step_tma_batch_kernel<OneType<float>, 4, 4, 2>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 2, 1, 2, 0, (const void*)step_tma_batch_kernel<OneType<float>, 2, 1, 2>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 2, 1, 3, 0, (const void*)step_tma_batch_kernel<OneType<float>, 2, 1, 3>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 2, 2, 3, 0, (const void*)step_tma_batch_kernel<OneType<float>, 2, 2, 3>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 4, 2, 2, 0, (const void*)step_tma_batch_kernel<OneType<float>, 4, 2, 2>},
    {DMRT_MIXED, DMRT_ROUND_NEAREST, 1, 1, 2, 0, (const void*)step_tma_batch_kernel<Split<__half, float>, 1, 1, 2>},
    {DMRT_MIXED, DMRT_ROUND_NEAREST, 1, 2, 2, 0, (const void*)step_tma_batch_kernel<Split<__half, float>, 1, 2, 2>},
    {DMRT_MIXED, DMRT_ROUND_NEAREST, 1, 4, 2, 0, (const void*)step_tma_batch_kernel<Split<__half, float>, 1, 4, 2>},
    {DMRT_MIXED, DMRT_ROUND_NEAREST, 1, 4, 3, 0, (const void*)step_tma_batch_kernel<Split<__half, float>, 1, 4, 3>},
    {DMRT_MIXED, DMRT_ROUND_NEAREST, 2, 2, 2, 0, (const void*)step_tma_batch_kernel<Split<__half, float>, 2, 2, 2>},
    {DMRT_MIXED, DMRT_ROUND_NEAREST, 2, 4, 2, 0, (const void*)step_tma_batch_kernel<Split<__half, float>, 2, 4, 2>},
    {DMRT_MIXED, DMRT_ROUND_NEAREST, 4, 1, 4, 0, (const void*)step_tma_batch_kernel<Split<__half, float>, 4, 1, 4>},
    {DMRT_MIXED, DMRT_ROUND_NEAREST, 4, 4, 2, 0, (const void*)step_tma_batch_kernel<Split<__half, float>, 4, 4, 2>},
    // (2, 1, 2): registers bounded for 7 blocks per SM (72; shared memory allows 8).
    {DMRT_MIXED, DMRT_ROUND_NEAREST, 2, 1, 2, 0, (const void*)step_tma_batch_kernel<Split<__half, float>, 2, 1, 2, false, false, 7>},
    {DMRT_MIXED, DMRT_ROUND_NEAREST, 2, 1, 3, 0, (const void*)step_tma_batch_kernel<Split<__half, float>, 2, 1, 3>},
    {DMRT_MIXED, DMRT_ROUND_NEAREST, 2, 2, 3, 0, (const void*)step_tma_batch_kernel<Split<__half, float>, 2, 2, 3>},
    {DMRT_MIXED, DMRT_ROUND_NEAREST, 4, 2, 2, 0, (const void*)step_tma_batch_kernel<Split<__half, float>, 4, 2, 2>},
    {DMRT_MIXED, DMRT_ROUND_STOCHASTIC, 1, 1, 2, 0, (const void*)step_tma_batch_kernel<Split<__half, float>, 1, 1, 2, true>},
    {DMRT_MIXED, DMRT_ROUND_STOCHASTIC, 1, 2, 2, 0, (const void*)step_tma_batch_kernel<Split<__half, float>, 1, 2, 2, true>},
    {DMRT_MIXED, DMRT_ROUND_STOCHASTIC, 1, 4, 2, 0, (const void*)step_tma_batch_kernel<Split<__half, float>, 1, 4, 2, true>},
    {DMRT_MIXED, DMRT_ROUND_STOCHASTIC, 1, 4, 3, 0, (const void*)step_tma_batch_kernel<Split<__half, float>, 1, 4, 3, true>},
    {DMRT_MIXED, DMRT_ROUND_STOCHASTIC, 2, 2, 2, 0, (const void*)step_tma_batch_kernel<Split<__half, float>, 2, 2, 2, true>},
    {DMRT_MIXED, DMRT_ROUND_STOCHASTIC, 2, 4, 2, 0, (const void*)step_tma_batch_kernel<Split<__half, float>, 2, 4, 2, true>},
    {DMRT_MIXED, DMRT_ROUND_STOCHASTIC, 4, 1, 4, 0, (const void*)step_tma_batch_kernel<Split<__half, float>, 4, 1, 4, true>},
    {DMRT_MIXED, DMRT_ROUND_STOCHASTIC, 4, 4, 2, 0, (const void*)step_tma_batch_kernel<Split<__half, float>, 4, 4, 2, true>},
    {DMRT_MIXED, DMRT_ROUND_STOCHASTIC, 2, 1, 2, 0, (const void*)step_tma_batch_kernel<Split<__half, float>, 2, 1, 2, true, false, 7>},
    {DMRT_MIXED, DMRT_ROUND_STOCHASTIC, 2, 1, 3, 0, (const void*)step_tma_batch_kernel<Split<__half, float>, 2, 1, 3, true>},
    {DMRT_MIXED, DMRT_ROUND_STOCHASTIC, 2, 2, 3, 0, (const void*)step_tma_batch_kernel<Split<__half, float>, 2, 2, 3, true>},
    {DMRT_MIXED, DMRT_ROUND_STOCHASTIC, 4, 2, 2, 0, (const void*)step_tma_batch_kernel<Split<__half, float>, 4, 2, 2, true>},
    // Tensor-store epilogue.
    {DMRT_FP32, DMRT_ROUND_NEAREST, 2, 2, 2, 1, (const void*)step_tma_batch_kernel<OneType<float>, 2, 2, 2, false, true>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 2, 1, 2, 1, (const void*)step_tma_batch_kernel<OneType<float>, 2, 1, 2, false, true>},
    {DMRT_MIXED, DMRT_ROUND_NEAREST, 2, 2, 2, 1, (const void*)step_tma_batch_kernel<Split<__half, float>, 2, 2, 2, false, true>},
    {DMRT_MIXED, DMRT_ROUND_NEAREST, 4, 2, 2, 1, (const void*)step_tma_batch_kernel<Split<__half, float>, 4, 2, 2, false, true>},
    {DMRT_MIXED, DMRT_ROUND_NEAREST, 4, 4, 2, 1, (const void*)step_tma_batch_kernel<Split<__half, float>, 4, 4, 2, false, true>},
    {DMRT_MIXED, DMRT_ROUND_STOCHASTIC, 2, 2, 2, 1, (const void*)step_tma_batch_kernel<Split<__half, float>, 2, 2, 2, true, true>},
    {DMRT_MIXED, DMRT_ROUND_STOCHASTIC, 4, 2, 2, 1, (const void*)step_tma_batch_kernel<Split<__half, float>, 4, 2, 2, true, true>},
    {DMRT_MIXED, DMRT_ROUND_STOCHASTIC, 4, 4, 2, 1, (const void*)step_tma_batch_kernel<Split<__half, float>, 4, 4, 2, true, true>},
};

const TmaVariant* tma_variants_batch(int* n) {
    *n = (int)(sizeof(kVariants) / sizeof(kVariants[0]));
    return kVariants;
}

}  // namespace dmrt
