// TMA step-kernel tiles with 1 node(s) per thread (see step_tma.cuh).
#include "step_tma.cuh"
#include "tma_variants.h"

namespace dmrt {

static const TmaVariant kVariants1[] = {
    {1, 1, 2, (const void*)step_tma_kernel<1, 1, 2>},
    {1, 1, 3, (const void*)step_tma_kernel<1, 1, 3>},
    {1, 1, 4, (const void*)step_tma_kernel<1, 1, 4>},
    {1, 1, 5, (const void*)step_tma_kernel<1, 1, 5>},
    {1, 2, 2, (const void*)step_tma_kernel<1, 2, 2>},
    {1, 2, 3, (const void*)step_tma_kernel<1, 2, 3>},
    {1, 3, 2, (const void*)step_tma_kernel<1, 3, 2>},
    {1, 4, 2, (const void*)step_tma_kernel<1, 4, 2>},
    {1, 4, 3, (const void*)step_tma_kernel<1, 4, 3>},
};

const TmaVariant* tma_variants_npt1(int* n) {
    *n = (int)(sizeof(kVariants1) / sizeof(kVariants1[0]));
    return kVariants1;
}

}  // namespace dmrt
