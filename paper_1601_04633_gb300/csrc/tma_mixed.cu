// TMA step-kernel tiles: mixed storage (flow populations float16, thermal
// populations float32), nearest and stochastic rounding of the flow
// populations (see step_tma.cuh).
#include "dmrt.h"
#include "step_tma.cuh"
#include "tma_variants.h"

namespace dmrt {

using Mixed = Split<__half, float>;

static const TmaVariant kVariants[] = {
    {DMRT_MIXED, DMRT_ROUND_NEAREST, 1, 1, 2, 1, (const void*)step_tma_kernel<Mixed, 1, 1, 2, false, true>},
    {DMRT_MIXED, DMRT_ROUND_NEAREST, 1, 2, 2, 1, (const void*)step_tma_kernel<Mixed, 1, 2, 2, false, true>},
    {DMRT_MIXED, DMRT_ROUND_NEAREST, 1, 4, 2, 1, (const void*)step_tma_kernel<Mixed, 1, 4, 2, false, true>},
    {DMRT_MIXED, DMRT_ROUND_NEAREST, 2, 2, 2, 1, (const void*)step_tma_kernel<Mixed, 2, 2, 2, false, true>},
    {DMRT_MIXED, DMRT_ROUND_NEAREST, 1, 1, 3, 1, (const void*)step_tma_kernel<Mixed, 1, 1, 3, false, true>},
    {DMRT_MIXED, DMRT_ROUND_NEAREST, 1, 1, 4, 1, (const void*)step_tma_kernel<Mixed, 1, 1, 4, false, true>},
    {DMRT_MIXED, DMRT_ROUND_NEAREST, 1, 2, 3, 1, (const void*)step_tma_kernel<Mixed, 1, 2, 3, false, true>},
    {DMRT_MIXED, DMRT_ROUND_NEAREST, 2, 1, 3, 1, (const void*)step_tma_kernel<Mixed, 2, 1, 3, false, true>},
    {DMRT_MIXED, DMRT_ROUND_NEAREST, 2, 1, 2, 1, (const void*)step_tma_kernel<Mixed, 2, 1, 2, false, true>},
    {DMRT_MIXED, DMRT_ROUND_NEAREST, 2, 1, 4, 1, (const void*)step_tma_kernel<Mixed, 2, 1, 4, false, true>},
    {DMRT_MIXED, DMRT_ROUND_NEAREST, 4, 1, 3, 1, (const void*)step_tma_kernel<Mixed, 4, 1, 3, false, true>},
    {DMRT_MIXED, DMRT_ROUND_NEAREST, 4, 1, 4, 1, (const void*)step_tma_kernel<Mixed, 4, 1, 4, false, true>},
    {DMRT_MIXED, DMRT_ROUND_STOCHASTIC, 1, 1, 2, 1, (const void*)step_tma_kernel<Mixed, 1, 1, 2, true, true>},
    {DMRT_MIXED, DMRT_ROUND_STOCHASTIC, 1, 2, 2, 1, (const void*)step_tma_kernel<Mixed, 1, 2, 2, true, true>},
    {DMRT_MIXED, DMRT_ROUND_STOCHASTIC, 1, 4, 2, 1, (const void*)step_tma_kernel<Mixed, 1, 4, 2, true, true>},
    {DMRT_MIXED, DMRT_ROUND_STOCHASTIC, 1, 4, 3, 1, (const void*)step_tma_kernel<Mixed, 1, 4, 3, true, true>},
    {DMRT_MIXED, DMRT_ROUND_STOCHASTIC, 2, 2, 2, 1, (const void*)step_tma_kernel<Mixed, 2, 2, 2, true, true>},
    {DMRT_MIXED, DMRT_ROUND_STOCHASTIC, 2, 4, 2, 1, (const void*)step_tma_kernel<Mixed, 2, 4, 2, true, true>},
    {DMRT_MIXED, DMRT_ROUND_STOCHASTIC, 2, 1, 2, 1, (const void*)step_tma_kernel<Mixed, 2, 1, 2, true, true>},
    {DMRT_MIXED, DMRT_ROUND_STOCHASTIC, 2, 1, 3, 1, (const void*)step_tma_kernel<Mixed, 2, 1, 3, true, true>},
    {DMRT_MIXED, DMRT_ROUND_STOCHASTIC, 4, 1, 3, 1, (const void*)step_tma_kernel<Mixed, 4, 1, 3, true, true>},
};

const TmaVariant* tma_variants_mixed(int* n) {
    *n = (int)(sizeof(kVariants) / sizeof(kVariants[0]));
    return kVariants;
}

}  // namespace dmrt
