// dmrt_step_noalloc: one time step that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the point where they step a cavity:
// code that runs while a framework owns all device memory and hands out only
// the input and output buffers, real-time loops where an allocation would
// synchronise the device, or plug-in hosts that forbid allocation inside their
// callbacks. This entry point takes the two population buffers from the
// caller and keeps everything else the step kernel needs (wall temperatures,
// per-row Nusselt values, the step counter and pending flag of the Nusselt
// reduction, the error word) in one file-scope device array of fixed size. Every GPU that
// loads the library holds that array until the process exits.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>

#include "dmrt.h"
#include "step_consts.h"
#include "step_direct.cuh"

// Defined in dmrt.cu: the message dmrt_last_error(NULL) returns.
void dmrt_internal_set_error(const char* msg);

namespace {

// Scratch layout inside the static array (bytes):
//   [0, 8 * MAX)            per-row local Nusselt numbers (double)
//   [8 * MAX, 12 * MAX)     left-wall temperatures (float)
//   [12 * MAX, 16 * MAX)    right-wall temperatures (float)
//   [16 * MAX, + 256)       step counter, latest mean, pending flag, error word
constexpr int kMaxNy = DMRT_NOALLOC_MAX_NY;
constexpr size_t kOffRows = 0;
constexpr size_t kOffHot = 8 * (size_t)kMaxNy;
constexpr size_t kOffCold = 12 * (size_t)kMaxNy;
constexpr size_t kOffMisc = 16 * (size_t)kMaxNy;
constexpr size_t kScratchBytes = kOffMisc + 256;

struct Misc {
    long long step[2];
    double nu_last;
    double nu_sink;  // target of the mean when the caller passes no output
    unsigned pending;
    unsigned err;
};

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

__global__ void noalloc_fill(float* hot, float* cold, const float* hot_src, const float* cold_src,
                             float hot_val, float cold_val, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        hot[i] = hot_src ? hot_src[i] : hot_val;
        cold[i] = cold_src ? cold_src[i] : cold_val;
    }
}

int fail(int code, const char* what, const char* detail) {
    char msg[256];
    std::snprintf(msg, sizeof msg, "dmrt_step_noalloc: %s%s", what, detail ? detail : "");
    dmrt_internal_set_error(msg);
    return code;
}

}  // namespace

extern "C" int dmrt_step_noalloc(const dmrt_params* p, const float* src, float* dst,
                                 const float* theta_hot, const float* theta_cold,
                                 double* nu_mean, void* stream) {
    dmrt_consts k;
    int rc = dmrt_derive(p, &k);
    if (rc) return rc;
    if (p->storage != DMRT_FP32) return fail(DMRT_E_ARG, "float32 storage only", nullptr);
    if (p->ny > kMaxNy) {
        char d[64];
        std::snprintf(d, sizeof d, "%d > %d", p->ny, kMaxNy);
        return fail(DMRT_E_ARG, "ny exceeds DMRT_NOALLOC_MAX_NY: ", d);
    }
    if (!src || !dst || src == dst || (reinterpret_cast<uintptr_t>(src) & 15) ||
        (reinterpret_cast<uintptr_t>(dst) & 15))
        return fail(DMRT_E_ARG, "src and dst must be distinct 16-byte aligned device buffers", nullptr);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(DMRT_E_CUDA, "cudaGetDevice: ", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(DMRT_E_ARG, "device ordinal too large", nullptr);
    void* base = nullptr;
    {
        // First call on a device: look up the device address of the static array
        // (host code only sees a host-side stand-in for the symbol).
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_ptr[dev]) {
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess)
                return fail(DMRT_E_CUDA, "cudaGetSymbolAddress: ", cudaGetErrorString(e));
            g_scratch_ptr[dev] = ptr;
        }
        base = g_scratch_ptr[dev];
    }
    char* b = static_cast<char*>(base);
    Misc* misc = reinterpret_cast<Misc*>(b + kOffMisc);
    float* hot = reinterpret_cast<float*>(b + kOffHot);
    float* cold = reinterpret_cast<float*>(b + kOffCold);
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // The array keeps the previous call's contents: clear the reduction's
    // pending flag, step and error word, and write this call's wall temperatures.
    e = cudaMemsetAsync(misc, 0, sizeof(Misc), s);
    if (e != cudaSuccess) return fail(DMRT_E_CUDA, "cudaMemsetAsync: ", cudaGetErrorString(e));
    noalloc_fill<<<(p->ny + 255) / 256, 256, 0, s>>>(hot, cold, theta_hot, theta_cold,
                                                     (float)p->theta_hot, (float)p->theta_cold, p->ny);

    const dmrt::StepConsts sc = dmrt::make_step_consts(*p, k);

    const int pitch = ((p->nx + 127) / 128) * 128;
    dmrt::StepArgs A;
    A.src = src;
    A.dst = dst;
    A.hot = hot;
    A.cold = cold;
    A.nu_rows = reinterpret_cast<double*>(b + kOffRows);
    A.prev_rows = A.nu_rows;  // summed only by the finalize launch below (nothing is pending before)
    A.nu_ring = nu_mean ? nu_mean : &misc->nu_sink;  // a ring of length 1
    A.nu_last = &misc->nu_last;
    A.pending = &misc->pending;
    A.err = &misc->err;
    A.step_in = &misc->step[0];
    A.step_out = &misc->step[1];
    A.rounding = 0;
    A.cap = 1;
    A.plane = (long long)p->ny * pitch;
    A.nx = p->nx;
    A.ny = p->ny;
    A.pitch = pitch;
    A.row0 = 0;  // a whole cavity: no halo rows, walls on both sides
    A.wall_lo = 1;
    A.wall_hi = 1;
    A.jglob0 = 0;
    A.nu_inv = 1.0 / (double)p->ny;
    const int nxq = (p->nx + 3) / 4;
    int wx = 1;
    while (wx < nxq && wx < 32) wx <<= 1;
    A.wx_log2 = 0;
    while ((1 << A.wx_log2) < wx) ++A.wx_log2;
    const int rows_per_block = (dmrt::kDirectThreads / 32) * (32 / wx);
    const dim3 grid((nxq + wx - 1) / wx, (p->ny + rows_per_block - 1) / rows_per_block, 1);
    dmrt::step_direct_kernel<<<grid, dmrt::kDirectThreads, 0, s>>>(A, sc);
    // The step stores its local Nusselt numbers; one block then sums them into *nu_mean.
    dmrt::StepArgs F = A;
    F.step_in = &misc->step[1];
    dmrt::nu_finalize_kernel<<<1, 256, 0, s>>>(F);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(DMRT_E_CUDA, "step launch: ", cudaGetErrorString(e));
    return DMRT_OK;
}
