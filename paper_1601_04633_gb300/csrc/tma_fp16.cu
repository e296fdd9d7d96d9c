// TMA step-kernel tiles: float16 storage (see step_tma.cuh).
#include "dmrt.h"
#include "step_tma.cuh"
#include "tma_variants.h"

namespace dmrt {

static const TmaVariant kVariants[] = {
    {DMRT_FP16, 1, 1, 2, (const void*)step_tma_kernel<__half, 1, 1, 2>},
    {DMRT_FP16, 1, 2, 2, (const void*)step_tma_kernel<__half, 1, 2, 2>},
    {DMRT_FP16, 1, 4, 2, (const void*)step_tma_kernel<__half, 1, 4, 2>},
    {DMRT_FP16, 1, 4, 3, (const void*)step_tma_kernel<__half, 1, 4, 3>},
    {DMRT_FP16, 1, 4, 4, (const void*)step_tma_kernel<__half, 1, 4, 4>},
    {DMRT_FP16, 2, 2, 2, (const void*)step_tma_kernel<__half, 2, 2, 2>},
    {DMRT_FP16, 2, 4, 2, (const void*)step_tma_kernel<__half, 2, 4, 2>},
    {DMRT_FP16, 2, 4, 3, (const void*)step_tma_kernel<__half, 2, 4, 3>},
    {DMRT_FP16, 4, 4, 2, (const void*)step_tma_kernel<__half, 4, 4, 2>},
};

const TmaVariant* tma_variants_fp16(int* n) {
    *n = (int)(sizeof(kVariants) / sizeof(kVariants[0]));
    return kVariants;
}

}  // namespace dmrt
