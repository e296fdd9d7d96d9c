// TMA step-kernel tiles: THETA32 storage (flow populations float16, theta
// float32, thermal deviations float16), nearest and stochastic rounding of the
// float16 stores (see step_tma.cuh).
#include "dmrt.h"
#include "step_tma.cuh"
#include "tma_variants.h"

namespace dmrt {

static const TmaVariant kVariants[] = {
    {DMRT_THETA32, DMRT_ROUND_NEAREST, 1, 1, 2, 1, (const void*)step_tma_kernel<ThetaSplit, 1, 1, 2, false, true>},
    {DMRT_THETA32, DMRT_ROUND_NEAREST, 2, 1, 2, 1, (const void*)step_tma_kernel<ThetaSplit, 2, 1, 2, false, true>},
    {DMRT_THETA32, DMRT_ROUND_NEAREST, 2, 1, 3, 1, (const void*)step_tma_kernel<ThetaSplit, 2, 1, 3, false, true>},
    {DMRT_THETA32, DMRT_ROUND_NEAREST, 2, 2, 2, 1, (const void*)step_tma_kernel<ThetaSplit, 2, 2, 2, false, true>},
    {DMRT_THETA32, DMRT_ROUND_NEAREST, 4, 1, 3, 1, (const void*)step_tma_kernel<ThetaSplit, 4, 1, 3, false, true>},
    {DMRT_THETA32, DMRT_ROUND_STOCHASTIC, 1, 1, 2, 1, (const void*)step_tma_kernel<ThetaSplit, 1, 1, 2, true, true>},
    {DMRT_THETA32, DMRT_ROUND_STOCHASTIC, 1, 2, 2, 1, (const void*)step_tma_kernel<ThetaSplit, 1, 2, 2, true, true>},
    {DMRT_THETA32, DMRT_ROUND_STOCHASTIC, 2, 1, 2, 1, (const void*)step_tma_kernel<ThetaSplit, 2, 1, 2, true, true>},
    {DMRT_THETA32, DMRT_ROUND_STOCHASTIC, 2, 1, 3, 1, (const void*)step_tma_kernel<ThetaSplit, 2, 1, 3, true, true>},
    {DMRT_THETA32, DMRT_ROUND_STOCHASTIC, 2, 2, 2, 1, (const void*)step_tma_kernel<ThetaSplit, 2, 2, 2, true, true>},
    {DMRT_THETA32, DMRT_ROUND_STOCHASTIC, 2, 4, 2, 1, (const void*)step_tma_kernel<ThetaSplit, 2, 4, 2, true, true>},
    {DMRT_THETA32, DMRT_ROUND_STOCHASTIC, 4, 1, 3, 1, (const void*)step_tma_kernel<ThetaSplit, 4, 1, 3, true, true>},
    {DMRT_THETA32, DMRT_ROUND_STOCHASTIC, 4, 2, 2, 1, (const void*)step_tma_kernel<ThetaSplit, 4, 2, 2, true, true>},
};

const TmaVariant* tma_variants_theta(int* n) {
    *n = (int)(sizeof(kVariants) / sizeof(kVariants[0]));
    return kVariants;
}

}  // namespace dmrt
