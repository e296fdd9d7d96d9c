// TMA step-kernel tiles: float16 storage, nearest and stochastic rounding (see step_tma.cuh).
#include "dmrt.h"
#include "step_tma.cuh"
#include "tma_variants.h"

namespace dmrt {

static const TmaVariant kVariants[] = {
    {DMRT_FP16, DMRT_ROUND_NEAREST, 1, 1, 2, 1, (const void*)step_tma_kernel<OneType<__half>, 1, 1, 2, false, true>},
    {DMRT_FP16, DMRT_ROUND_NEAREST, 1, 2, 2, 1, (const void*)step_tma_kernel<OneType<__half>, 1, 2, 2, false, true>},
    {DMRT_FP16, DMRT_ROUND_NEAREST, 1, 4, 2, 1, (const void*)step_tma_kernel<OneType<__half>, 1, 4, 2, false, true>},
    {DMRT_FP16, DMRT_ROUND_NEAREST, 1, 4, 3, 1, (const void*)step_tma_kernel<OneType<__half>, 1, 4, 3, false, true>},
    {DMRT_FP16, DMRT_ROUND_NEAREST, 1, 4, 4, 1, (const void*)step_tma_kernel<OneType<__half>, 1, 4, 4, false, true>},
    {DMRT_FP16, DMRT_ROUND_NEAREST, 2, 2, 2, 1, (const void*)step_tma_kernel<OneType<__half>, 2, 2, 2, false, true>},
    {DMRT_FP16, DMRT_ROUND_NEAREST, 2, 4, 2, 1, (const void*)step_tma_kernel<OneType<__half>, 2, 4, 2, false, true>},
    {DMRT_FP16, DMRT_ROUND_NEAREST, 2, 4, 3, 1, (const void*)step_tma_kernel<OneType<__half>, 2, 4, 3, false, true>},
    {DMRT_FP16, DMRT_ROUND_NEAREST, 4, 4, 2, 1, (const void*)step_tma_kernel<OneType<__half>, 4, 4, 2, false, true>},
    {DMRT_FP16, DMRT_ROUND_NEAREST, 4, 2, 2, 1, (const void*)step_tma_kernel<OneType<__half>, 4, 2, 2, false, true>},
    {DMRT_FP16, DMRT_ROUND_STOCHASTIC, 1, 1, 2, 1, (const void*)step_tma_kernel<OneType<__half>, 1, 1, 2, true, true>},
    {DMRT_FP16, DMRT_ROUND_STOCHASTIC, 1, 4, 2, 1, (const void*)step_tma_kernel<OneType<__half>, 1, 4, 2, true, true>},
    {DMRT_FP16, DMRT_ROUND_STOCHASTIC, 2, 2, 2, 1, (const void*)step_tma_kernel<OneType<__half>, 2, 2, 2, true, true>},
    {DMRT_FP16, DMRT_ROUND_STOCHASTIC, 4, 4, 2, 1, (const void*)step_tma_kernel<OneType<__half>, 4, 4, 2, true, true>},
    {DMRT_FP16, DMRT_ROUND_STOCHASTIC, 2, 4, 2, 1, (const void*)step_tma_kernel<OneType<__half>, 2, 4, 2, true, true>},
    {DMRT_FP16, DMRT_ROUND_STOCHASTIC, 4, 2, 2, 1, (const void*)step_tma_kernel<OneType<__half>, 4, 2, 2, true, true>},
};

const TmaVariant* tma_variants_fp16(int* n) {
    *n = (int)(sizeof(kVariants) / sizeof(kVariants[0]));
    return kVariants;
}

}  // namespace dmrt
