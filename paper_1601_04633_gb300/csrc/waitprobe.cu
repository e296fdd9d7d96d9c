// dmrt_probe_bounded_wait: exercises the failure path of the step kernels'
// bounded device-side waits without faulting or hanging the GPU. One thread
// waits, through the same routine the step kernels use (mbar_wait_bounded), on
// an mbarrier that nothing ever completes; the wait must give up after the
// limit and report it, leaving the context usable.
#include <cuda_runtime.h>

#include "dmrt.h"
#include "step_tma.cuh"

void dmrt_internal_set_error(const char* msg);

namespace {

// [0]: 1 if the wait completed (it must not), 2 if it gave up; [1]: waited ns.
__device__ unsigned long long g_probe[2];

__global__ void wait_probe_kernel(unsigned long long limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    dmrt::mbar_init(&bar, 1);
    dmrt::mbar_fence_init();
    const unsigned long long t0 = dmrt::global_ns();
    const bool done = dmrt::mbar_wait_bounded(&bar, 0u, limit_ns);  // phase 0 never completes
    g_probe[0] = done ? 1ull : 2ull;
    g_probe[1] = dmrt::global_ns() - t0;
}

}  // namespace

extern "C" int dmrt_probe_bounded_wait(int64_t limit_ns, void* stream, int64_t* waited_ns) {
    if (limit_ns < 1000000 || limit_ns > (int64_t)dmrt::kWaitLimitNs) {
        dmrt_internal_set_error("dmrt_probe_bounded_wait: limit must be in [1 ms, 2 s]");
        return DMRT_E_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned long long out[2] = {0, 0};
    wait_probe_kernel<<<1, 32, 0, s>>>((unsigned long long)limit_ns);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyFromSymbolAsync(out, g_probe, sizeof out, 0, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        dmrt_internal_set_error(cudaGetErrorString(e));
        return DMRT_E_CUDA;
    }
    if (waited_ns) *waited_ns = (int64_t)out[1];
    if (out[0] == 2) {
        dmrt_internal_set_error("dmrt_probe_bounded_wait: the wait gave up after its limit, as designed");
        return DMRT_E_TIMEOUT;
    }
    dmrt_internal_set_error("dmrt_probe_bounded_wait: the wait completed although nothing arrived");
    return DMRT_OK;
}
