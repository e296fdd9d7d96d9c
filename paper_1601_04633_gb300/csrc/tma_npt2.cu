// TMA step-kernel tiles: float32 storage, 2 nodes per thread (see step_tma.cuh).
#include "dmrt.h"
#include "step_tma.cuh"
#include "tma_variants.h"

namespace dmrt {

static const TmaVariant kVariants[] = {
    {DMRT_FP32, DMRT_ROUND_NEAREST, 2, 1, 3, 0, (const void*)step_tma_kernel<OneType<float>, 2, 1, 3, false, false>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 2, 1, 4, 0, (const void*)step_tma_kernel<OneType<float>, 2, 1, 4, false, false>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 2, 1, 5, 0, (const void*)step_tma_kernel<OneType<float>, 2, 1, 5, false, false>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 2, 2, 2, 0, (const void*)step_tma_kernel<OneType<float>, 2, 2, 2, false, false>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 2, 2, 3, 0, (const void*)step_tma_kernel<OneType<float>, 2, 2, 3, false, false>},
    {DMRT_FP32, DMRT_ROUND_NEAREST, 2, 4, 2, 0, (const void*)step_tma_kernel<OneType<float>, 2, 4, 2, false, false>},
};

const TmaVariant* tma_variants_npt2(int* n) {
    *n = (int)(sizeof(kVariants) / sizeof(kVariants[0]));
    return kVariants;
}

}  // namespace dmrt
