// TMA step-kernel tiles with 2 node(s) per thread (see step_tma.cuh).
#include "step_tma.cuh"
#include "tma_variants.h"

namespace dmrt {

static const TmaVariant kVariants2[] = {
    {2, 1, 3, (const void*)step_tma_kernel<2, 1, 3>},
    {2, 1, 4, (const void*)step_tma_kernel<2, 1, 4>},
    {2, 1, 5, (const void*)step_tma_kernel<2, 1, 5>},
    {2, 2, 2, (const void*)step_tma_kernel<2, 2, 2>},
    {2, 2, 3, (const void*)step_tma_kernel<2, 2, 3>},
    {2, 4, 2, (const void*)step_tma_kernel<2, 4, 2>},
};

const TmaVariant* tma_variants_npt2(int* n) {
    *n = (int)(sizeof(kVariants2) / sizeof(kVariants2[0]));
    return kVariants2;
}

}  // namespace dmrt
