// Registry of the compiled TMA step-kernel tiles: storage type, NPT nodes per
// thread, R rows per work item, S pipeline stages. Each list is defined in its
// own translation unit (tma_*.cu) so the instantiations compile in parallel.
#pragma once

namespace dmrt {

struct TmaVariant {
    int storage;   // DMRT_FP32, DMRT_FP16, DMRT_BF16, DMRT_MIXED or DMRT_THETA32
    int rounding;  // DMRT_ROUND_NEAREST or DMRT_ROUND_STOCHASTIC
    int npt, R, S;
    int ts;  // 1: tensor-store epilogue through shared-memory output tiles
    const void* func;
};

const TmaVariant* tma_variants_npt4(int* n);
const TmaVariant* tma_variants_npt2(int* n);
const TmaVariant* tma_variants_npt1(int* n);
const TmaVariant* tma_variants_fp16(int* n);
const TmaVariant* tma_variants_bf16(int* n);
const TmaVariant* tma_variants_mixed(int* n);  // float16 flow, float32 thermal
const TmaVariant* tma_variants_theta(int* n);  // float16 flow and deviations, float32 theta
const TmaVariant* tma_variants_batch(int* n);  // batched sweep kernels
const TmaVariant* tma_variants_batch_mstep(int* n);  // batched sweep, several steps per launch

}  // namespace dmrt
