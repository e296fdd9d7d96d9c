// TMA step-kernel tiles: bfloat16 storage (see step_tma.cuh).
#include "dmrt.h"
#include "step_tma.cuh"
#include "tma_variants.h"

namespace dmrt {

static const TmaVariant kVariants[] = {
    {DMRT_BF16, 1, 1, 2, (const void*)step_tma_kernel<__nv_bfloat16, 1, 1, 2>},
    {DMRT_BF16, 1, 2, 2, (const void*)step_tma_kernel<__nv_bfloat16, 1, 2, 2>},
    {DMRT_BF16, 1, 4, 2, (const void*)step_tma_kernel<__nv_bfloat16, 1, 4, 2>},
    {DMRT_BF16, 1, 4, 3, (const void*)step_tma_kernel<__nv_bfloat16, 1, 4, 3>},
    {DMRT_BF16, 1, 4, 4, (const void*)step_tma_kernel<__nv_bfloat16, 1, 4, 4>},
    {DMRT_BF16, 2, 2, 2, (const void*)step_tma_kernel<__nv_bfloat16, 2, 2, 2>},
    {DMRT_BF16, 2, 4, 2, (const void*)step_tma_kernel<__nv_bfloat16, 2, 4, 2>},
    {DMRT_BF16, 2, 4, 3, (const void*)step_tma_kernel<__nv_bfloat16, 2, 4, 3>},
    {DMRT_BF16, 4, 4, 2, (const void*)step_tma_kernel<__nv_bfloat16, 4, 4, 2>},
};

const TmaVariant* tma_variants_bf16(int* n) {
    *n = (int)(sizeof(kVariants) / sizeof(kVariants[0]));
    return kVariants;
}

}  // namespace dmrt
