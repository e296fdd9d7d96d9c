// Registry of the compiled TMA step-kernel tiles: NPT nodes per thread, R rows
// per work item, S pipeline stages. Each list is defined in its own
// translation unit (tma_npt*.cu) so the instantiations compile in parallel.
#pragma once

namespace dmrt {

struct TmaVariant {
    int npt, R, S;
    const void* func;
};

const TmaVariant* tma_variants_npt4(int* n);
const TmaVariant* tma_variants_npt2(int* n);
const TmaVariant* tma_variants_npt1(int* n);

}  // namespace dmrt
