// TMA step-kernel tiles: float32 storage, 4 nodes per thread (see step_tma.cuh).
#include "dmrt.h"
#include "step_tma.cuh"
#include "tma_variants.h"

namespace dmrt {

static const TmaVariant kVariants[] = {
    {DMRT_FP32, DMRT_ROUND_NEAREST, 4, 1, 2, 0, (const void*)step_tma_kernel<OneType<float>, 4, 1, 2, false, false>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 4, 1, 3, 0, (const void*)step_tma_kernel<OneType<float>, 4, 1, 3, false, false>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 4, 1, 4, 0, (const void*)step_tma_kernel<OneType<float>, 4, 1, 4, false, false>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 4, 1, 5, 0, (const void*)step_tma_kernel<OneType<float>, 4, 1, 5, false, false>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 4, 1, 6, 0, (const void*)step_tma_kernel<OneType<float>, 4, 1, 6, false, false>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 4, 2, 2, 0, (const void*)step_tma_kernel<OneType<float>, 4, 2, 2, false, false>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 4, 2, 3, 0, (const void*)step_tma_kernel<OneType<float>, 4, 2, 3, false, false>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 4, 2, 4, 0, (const void*)step_tma_kernel<OneType<float>, 4, 2, 4, false, false>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 4, 4, 2, 0, (const void*)step_tma_kernel<OneType<float>, 4, 4, 2, false, false>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 4, 4, 3, 0, (const void*)step_tma_kernel<OneType<float>, 4, 4, 3, false, false>},
};

const TmaVariant* tma_variants_npt4(int* n) {
    *n = (int)(sizeof(kVariants) / sizeof(kVariants[0]));
    return kVariants;
}

}  // namespace dmrt
