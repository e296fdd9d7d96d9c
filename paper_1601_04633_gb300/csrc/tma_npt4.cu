// TMA step-kernel tiles with 4 node(s) per thread (see step_tma.cuh).
#include "step_tma.cuh"
#include "tma_variants.h"

namespace dmrt {

static const TmaVariant kVariants4[] = {
    {4, 1, 2, (const void*)step_tma_kernel<4, 1, 2>},
    {4, 1, 3, (const void*)step_tma_kernel<4, 1, 3>},
    {4, 1, 4, (const void*)step_tma_kernel<4, 1, 4>},
    {4, 1, 5, (const void*)step_tma_kernel<4, 1, 5>},
    {4, 1, 6, (const void*)step_tma_kernel<4, 1, 6>},
    {4, 2, 2, (const void*)step_tma_kernel<4, 2, 2>},
    {4, 2, 3, (const void*)step_tma_kernel<4, 2, 3>},
    {4, 2, 4, (const void*)step_tma_kernel<4, 2, 4>},
    {4, 4, 2, (const void*)step_tma_kernel<4, 4, 2>},
    {4, 4, 3, (const void*)step_tma_kernel<4, 4, 3>},
};

const TmaVariant* tma_variants_npt4(int* n) {
    *n = (int)(sizeof(kVariants4) / sizeof(kVariants4[0]));
    return kVariants4;
}

}  // namespace dmrt
