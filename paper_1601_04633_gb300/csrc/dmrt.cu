// Host side of libdmrt.so: parameter derivation, workspace layout, the
// init / fields kernels and the C entry points declared in include/dmrt.h.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "dmrt.h"
#include "adjoint.cuh"
#include "step_cluster.cuh"
#include "step_consts.h"
#include "step_direct.cuh"
#include "step_tma.cuh"
#include "step_tma_batch.cuh"
#include "tma_variants.h"

using dmrt::plane_f;
using dmrt::plane_g;
using dmrt::kPlanes;

namespace {

thread_local char g_create_error[256] = "";

struct Layout {
    int pitch;            // elements per row (multiple of 128)
    long long plane;      // elements per plane
    size_t buf_bytes;     // one population buffer (14 planes; mixed storage: 9 float16
                          // flow planes, then 5 float32 thermal planes; THETA32: 9
                          // float16 flow planes, a float32 theta plane, 4 float16
                          // deviation planes)
    size_t off_a, off_b, off_hot, off_cold, off_rows, off_ring, off_misc;
    size_t total;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Bytes per stored flow (f) and thermal (g) population (THETA32: per deviation),
// and of a node's whole thermal block.
int f_bytes(int storage) { return storage == DMRT_FP32 ? 4 : 2; }
int g_bytes(int storage) { return storage == DMRT_FP32 || storage == DMRT_MIXED ? 4 : 2; }
int thermal_bytes(int storage) { return storage == DMRT_THETA32 ? 4 + 4 * 2 : 5 * g_bytes(storage); }

// DMRT_ROUND_AUTO resolved: stochastic rounding for 16-bit and mixed storage,
// nearest (nothing is rounded) for float32.
int resolved_rounding(const dmrt_params& p) {
    if (p.rounding != DMRT_ROUND_AUTO) return p.rounding;
    return p.storage == DMRT_FP32 ? DMRT_ROUND_NEAREST : DMRT_ROUND_STOCHASTIC;
}
dmrt_params resolved(const dmrt_params& p) {
    dmrt_params q = p;
    q.rounding = resolved_rounding(p);
    return q;
}

// halo_rows: extra population rows held by a y-slab (one below, one above its ny rows).
Layout make_layout(const dmrt_params& p, int halo_rows = 0) {
    Layout L;
    L.pitch = ((p.nx + 127) / 128) * 128;
    L.plane = (long long)(p.ny + halo_rows) * L.pitch;
    L.buf_bytes = align256((size_t)L.plane * (9 * f_bytes(p.storage) + thermal_bytes(p.storage)));
    size_t o = 0;
    L.off_a = o; o += L.buf_bytes;
    L.off_b = o; o += L.buf_bytes;
    L.off_hot = o; o += align256((size_t)p.ny * sizeof(float));
    L.off_cold = o; o += align256((size_t)p.ny * sizeof(float));
    L.off_rows = o; o += align256((size_t)2 * p.ny * sizeof(double));  // by source buffer
    L.off_ring = o; o += align256((size_t)p.nu_capacity * sizeof(double));
    L.off_misc = o; o += 256;
    L.total = o;
    return L;
}

// dmrt_step reads the device error word once per this many steps.
constexpr long long kPollSteps = 1LL << 16;

// Scalars kept on the device (one 256-byte block).
struct Misc {
    long long step[2];   // steps recorded in the Nu ring; slot b is current when the
                         // state is in buffer b (a launch reads one slot, writes the other)
    double nu_last;      // mean Nu of the latest step
    unsigned pending;    // the last step's local Nu rows are not yet summed into the ring
    unsigned err;        // error bits
};

}  // namespace

void dmrt_internal_set_error(const char* msg) {
    std::snprintf(g_create_error, sizeof g_create_error, "%s", msg);
}

struct dmrt_ctx {
    dmrt_params p;
    dmrt_consts k;
    Layout L;
    char* ws;
    cudaStream_t stream;
    int cur;             // 0: state in buffer A, 1: in buffer B
    long long t;         // steps enqueued
    dmrt::StepConsts sc;
    int kernel;          // DMRT_KERNEL_DIRECT or DMRT_KERNEL_TMA (resolved)
    // direct kernel
    int wx_log2;
    dim3 grid;
    // TMA kernel
    int npt, R, S, tma_block;
    dmrt::TmaGeo geo;
    int tma_grid;
    size_t tma_smem;
    const void* tma_func;
    dmrt::TmaMaps tmaps[2];  // per source buffer: the step kernel's load and store maps
    // Cluster kernel (runs of steps of a small float32 cavity; single steps and
    // the adjoint use `kernel`): blocks, rows per block, threads, shared memory.
    bool cluster;
    int csize, crows, cthreads;
    size_t csmem;
    // Adjoint: a second stream and events for the overlapped recompute (created at first use).
    cudaStream_t aux;
    cudaEvent_t ev[5];
    cudaGraphExec_t graph[2];
    int graph_len;
    long long nu_floor;  // ring values of steps before this one are unavailable (after a load)
    long long next_poll; // dmrt_step reads the error word once the step count reaches this
    // A y-slab of a larger cavity (rows y0 .. y0 + p.ny - 1 of H rows) holds one
    // halo row on each side (row0 = 1) that its neighbours fill; a whole cavity
    // has row0 = 0, y0 = 0, H = p.ny and both walls.
    bool slab;
    int row0, y0, H, wall_lo, wall_hi;
    char err[256];
};

namespace {

void set_err(dmrt_ctx* c, const char* fmt, ...) {
    char* dst = c ? c->err : g_create_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 256, fmt, ap);
    va_end(ap);
}

int cuda_fail(dmrt_ctx* c, cudaError_t e, const char* what) {
    set_err(c, "%s: %s", what, cudaGetErrorString(e));
    return DMRT_E_CUDA;
}

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

float* buf(dmrt_ctx* c, int which) {
    return reinterpret_cast<float*>(c->ws + (which == 0 ? c->L.off_a : c->L.off_b));
}
Misc* misc(dmrt_ctx* c) { return reinterpret_cast<Misc*>(c->ws + c->L.off_misc); }
// Local Nu rows of the last step taken (it ran from buffer 1 - cur).
double* last_rows(dmrt_ctx* c) {
    return reinterpret_cast<double*>(c->ws + c->L.off_rows) + (size_t)(1 - c->cur) * c->p.ny;
}

dmrt::StepArgs step_args(dmrt_ctx* c, int from) {
    dmrt::StepArgs A;
    A.src = buf(c, from);
    A.dst = buf(c, 1 - from);
    A.hot = reinterpret_cast<const float*>(c->ws + c->L.off_hot);
    A.cold = reinterpret_cast<const float*>(c->ws + c->L.off_cold);
    // Local Nu rows: a step from buffer b writes rows[b] and sums rows[1 - b],
    // those of the step before it.
    double* rows = reinterpret_cast<double*>(c->ws + c->L.off_rows);
    A.nu_rows = rows + (size_t)from * c->p.ny;
    A.prev_rows = rows + (size_t)(1 - from) * c->p.ny;
    A.nu_ring = reinterpret_cast<double*>(c->ws + c->L.off_ring);
    Misc* m = misc(c);
    A.nu_last = &m->nu_last;
    A.pending = &m->pending;
    A.err = &m->err;
    A.step_in = &m->step[from];
    A.step_out = &m->step[1 - from];
    A.rounding = c->p.rounding;
    A.cap = c->p.nu_capacity;
    A.plane = c->L.plane;
    A.nx = c->p.nx;
    A.ny = c->p.ny;
    A.pitch = c->L.pitch;
    A.wx_log2 = c->wx_log2;
    A.row0 = c->row0;
    A.wall_lo = c->wall_lo;
    A.wall_hi = c->wall_hi;
    A.jglob0 = c->y0;
    A.nu_inv = 1.0 / (double)c->H;
    return A;
}

// ---- small kernels ----------------------------------------------------------

__device__ __forceinline__ float elem_to_f(float x) { return x; }
__device__ __forceinline__ float elem_to_f(__half x) { return __half2float(x); }
__device__ __forceinline__ float elem_to_f(__nv_bfloat16 x) { return __bfloat162float(x); }
template <typename E>
__device__ __forceinline__ E elem_from_f(float x);
template <>
__device__ __forceinline__ float elem_from_f<float>(float x) { return x; }
template <>
__device__ __forceinline__ __half elem_from_f<__half>(float x) { return __float2half_rn(x); }
template <>
__device__ __forceinline__ __nv_bfloat16 elem_from_f<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

// Flow and thermal plane bases of a population buffer in layout L.
template <typename L, typename B>
__device__ __forceinline__ auto* f_base(B* S) {
    using Ef = typename L::Ef;
    using T = typename std::conditional<std::is_const<B>::value, const Ef, Ef>::type;
    return reinterpret_cast<T*>(S);
}
template <typename L, typename B>
__device__ __forceinline__ auto* g_base(B* S, long long plane) {
    using Eg = typename L::Eg;
    using T = typename std::conditional<std::is_const<B>::value, const Eg, Eg>::type;
    return reinterpret_cast<T*>(S + (L::kSplit ? (size_t)9 * plane * sizeof(typename L::Ef) : 0));
}
// ThetaSplit: the theta plane and deviation plane k (k = 1..4).
template <typename L, typename B>
__device__ __forceinline__ auto* theta_plane(B* S, long long plane) {
    using T = typename std::conditional<std::is_const<B>::value, const float, float>::type;
    return reinterpret_cast<T*>(S + (size_t)9 * plane * 2);
}
template <typename L, typename B>
__device__ __forceinline__ auto* dev_plane(B* S, long long plane, int k) {
    using Eg = typename L::Eg;
    using T = typename std::conditional<std::is_const<B>::value, const Eg, Eg>::type;
    return reinterpret_cast<T*>(S + (size_t)9 * plane * 2 + (size_t)plane * 4) + (size_t)(k - 1) * plane;
}
// Post-collision thermal population k >= 1 of buffer element s, and theta =
// sum_i g_i, in float64 (stored value + shift; ThetaSplit: w theta + d_k, and
// theta as stored).
template <typename L>
__device__ __forceinline__ double g_moving(const unsigned char* S, long long plane, long long s, int k, double sh1,
                                           double w1) {
    if constexpr (L::kTheta)
        return w1 * (double)theta_plane<L>(S, plane)[s] + (double)elem_to_f(dev_plane<L>(S, plane, k)[s]);
    else
        return (double)elem_to_f(g_base<L>(S, plane)[L::pg(k) * plane + s]) + sh1;
}
template <typename L>
__device__ __forceinline__ double theta_sum(const unsigned char* S, long long plane, long long s, double sh0,
                                            double sh1) {
    if constexpr (L::kTheta) return (double)theta_plane<L>(S, plane)[s];
    const auto* Sg = g_base<L>(S, plane);
    double th = 0.0;
    for (int k = 0; k < 5; ++k) th += (double)elem_to_f(Sg[L::pg(k) * plane + s]) + (k == 0 ? sh0 : sh1);
    return th;
}

// Initial post-collision state: f = 0 (rest, delta-rho = 0) and g at the D2Q5
// equilibrium of theta0 at rest, g_0 = (1 - a) theta / 5, g_1..4 = (4 + a) theta / 20
// (Eq. 42 mapped back through N), stored minus sh0 / sh1 (16-bit thermal storage
// shift; 0 for float32). Also zeroes the padding columns.
template <typename L>
__global__ void init_kernel(unsigned char* __restrict__ S, const double* __restrict__ theta0, double theta_const,
                            double a, double sh0, double sh1, int nx, int ny, int pitch,
                            long long plane, int row0) {
    using Ef = typename L::Ef;
    using Eg = typename L::Eg;
    Ef* Sf = f_base<L>(S);
    Eg* Sg = g_base<L>(S, plane);
    const int rows = (int)(plane / pitch);  // every row held, halo rows (zero) included
    // A block per buffer row (striding over rows), its threads along the row.
    for (int rr = blockIdx.x; rr < rows; rr += gridDim.x) {
        const int j = rr - row0;
        for (int i = threadIdx.x; i < pitch; i += blockDim.x) {
            const long long q = (long long)rr * pitch + i;
            double th = 0.0;
            const bool in = i < nx && j >= 0 && j < ny;
            if (in) th = theta0 ? theta0[(size_t)j * nx + i] : theta_const;
            for (int k = 0; k < 9; ++k) Sf[L::pf(k) * plane + q] = elem_from_f<Ef>(0.f);
            if constexpr (L::kTheta) {
                // At rest g_k = w theta exactly: theta and zero deviations.
                theta_plane<L>(S, plane)[q] = in ? (float)th : 0.f;
                for (int k = 1; k < 5; ++k) dev_plane<L>(S, plane, k)[q] = elem_from_f<Eg>(0.f);
                continue;
            }
            Sg[L::pg(0) * plane + q] = elem_from_f<Eg>(in ? (float)((1.0 - a) * th / 5.0 - sh0) : 0.f);
            const float side = in ? (float)((4.0 + a) * th / 20.0 - sh1) : 0.f;
            for (int k = 1; k < 5; ++k) Sg[L::pg(k) * plane + q] = elem_from_f<Eg>(side);
        }
    }
}

// Macroscopic fields of a post-collision state at the same time level:
// theta = sum g* (the thermal collision keeps theta), u = sum e f*, and
// v = sum e_y f* - G_y(theta) (the force added rho0 G to the momentum).
template <typename L>
__global__ void fields_kernel(const unsigned char* __restrict__ S, float* __restrict__ u,
                              float* __restrict__ v, float* __restrict__ th, int nx, int ny,
                              int pitch, long long plane, float gbeta, float theta_ref,
                              float sh0, float sh1, int row0) {
    const auto* Sf = f_base<L>(S);
    const auto* Sg = g_base<L>(S, plane);
    const long long n = (long long)nx * ny;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(q / nx), i = (int)(q % nx);
        const long long s = (long long)(j + row0) * pitch + i;
        float f[9];
        for (int k = 0; k < 9; ++k) f[k] = elem_to_f(Sf[L::pf(k) * plane + s]);
        float t;
        if constexpr (L::kTheta) {
            t = theta_plane<L>(S, plane)[s];
        } else {
            float g[5];
            for (int k = 0; k < 5; ++k) g[k] = elem_to_f(Sg[L::pg(k) * plane + s]) + (k == 0 ? sh0 : sh1);
            t = g[0] + g[1] + g[2] + g[3] + g[4];
        }
        const float jx = (f[1] - f[3]) + (f[5] - f[6]) - (f[7] - f[8]);
        const float jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
        if (u) u[q] = jx;
        if (v) v[q] = jy - gbeta * (t - theta_ref);
        if (th) th[q] = t;
    }
}

// One plane between the padded device layout and a dense float32 [ny][nx]
// array (16-bit storage: value = stored + shift).
template <typename E>
__global__ void plane_to_f32(const E* __restrict__ P, float* __restrict__ out, int nx, int ny,
                             int pitch, float shift) {
    const long long n = (long long)nx * ny;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(q / nx), i = (int)(q % nx);
        out[q] = elem_to_f(P[(size_t)j * pitch + i]) + shift;
    }
}

template <typename E>
__global__ void plane_from_f32(E* __restrict__ P, const float* __restrict__ in, int nx, int ny,
                               int pitch, float shift) {
    const long long n = (long long)ny * pitch;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(q / pitch), i = (int)(q % pitch);
        P[q] = elem_from_f<E>(i < nx ? in[(size_t)j * nx + i] - shift : 0.f);
    }
}

// THETA32 thermal block <-> dense float32 populations [5][ny][nx] (0-based
// directions 0..4, host planes g_1..g_5): g_k = w theta + d_k (k >= 1) and
// g_0 = w_0 theta - (d_1 + d_3 + d_2 + d_4), formed as the step kernel forms
// them; back: theta = sum_k g_k and d_k = g_k - w theta rounded to the nearest
// float16 (padding columns zero).
__global__ void theta_to_g32(const unsigned char* __restrict__ S, long long plane, int pitch, int nx, int ny,
                             int row0, float w0, float w1, float* __restrict__ out) {
    const long long n = (long long)nx * ny;
    const float* T = reinterpret_cast<const float*>(S + (size_t)9 * plane * 2);
    const __half* D = reinterpret_cast<const __half*>(S + (size_t)9 * plane * 2 + (size_t)plane * 4);
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(q / nx), i = (int)(q % nx);
        const long long s = (long long)(j + row0) * pitch + i;
        const float th = T[s];
        float d[5];
        for (int k = 1; k < 5; ++k) d[k] = __half2float(D[(k - 1) * plane + s]);
        out[q] = fmaf(w0, th, -((d[1] + d[3]) + (d[2] + d[4])));
        for (int k = 1; k < 5; ++k) out[k * n + q] = fmaf(w1, th, d[k]);
    }
}
__global__ void theta_from_g32(unsigned char* __restrict__ S, long long plane, int pitch, int nx, int ny, int row0,
                               float w1, const float* __restrict__ in) {
    const long long n = (long long)nx * ny;
    float* T = reinterpret_cast<float*>(S + (size_t)9 * plane * 2);
    __half* D = reinterpret_cast<__half*>(S + (size_t)9 * plane * 2 + (size_t)plane * 4);
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < (long long)ny * pitch;
         q += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(q / pitch), i = (int)(q % pitch);
        const long long s = (long long)(j + row0) * pitch + i;
        float g[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        if (i < nx)
            for (int k = 0; k < 5; ++k) g[k] = in[k * n + (long long)j * nx + i];
        const float th = g[0] + g[1] + g[2] + g[3] + g[4];
        T[s] = th;
        for (int k = 1; k < 5; ++k) D[(k - 1) * plane + s] = __float2half_rn(fmaf(-w1, th, g[k]));
    }
}

__global__ void fill_kernel(float* p, const double* src, double value, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = (float)(src ? src[i] : value);
}

// Host state arrays are ordered f_1..f_9, g_1..g_5; the device planes are grouped.
int host_plane(int k) { return k < 9 ? plane_f(k) : plane_g(k - 9); }

// Secondary hot-wall Nusselt number per row from the post-collision thermal
// populations of the wall column: the next streaming brings abb theta_w(j) -
// g*_3(0, j) in across the left wall's link (anti-bounce-back, Eq. 45) and takes
// g*_3(0, j) out; Nu_j = H (abb theta_w - 2 g*_3) / (alpha dT). abb = 0 and
// sign = 0 for an adiabatic left wall (no heat crosses it).
template <typename L>
__global__ void nu_flux_kernel(const unsigned char* __restrict__ S, const float* __restrict__ hot,
                               double* __restrict__ out, int ny, int pitch, long long plane, double abb,
                               double g_sign, double sh1, double w1, double scale, int row0) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ny) return;
    const double g3 = g_moving<L>(S, plane, (long long)(j + row0) * pitch, 3, sh1, w1);
    out[j] = scale * (abb * (double)hot[j] - g_sign * 2.0 * g3);
}

// Heat content of each row (sum of theta = sum_i g*_i over the row, Eq. 41) and
// the heat the next streaming brings in across the row's fixed-temperature wall
// links (Eq. 45: anti-bounce-back returns abb theta_w - g* and the wall link
// takes g* out, so the row gains abb theta_w - 2 g*; bounce-back, Eq. 44,
// returns what leaves). One warp per row, float64: lane l adds nodes l, l + 32,
// ... in order, the warp combines the lanes by a butterfly (a fixed order).
template <typename L>
__global__ void energy_rows_kernel(const unsigned char* __restrict__ S, const float* __restrict__ hot,
                                   const float* __restrict__ cold, double* __restrict__ row_theta,
                                   double* __restrict__ row_in, int nx, int ny, int pitch, long long plane,
                                   double abb_l, double sign_l, double abb_r, double sign_r, double sh0,
                                   double sh1, double w1, int row0) {
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= ny) return;  // warp-uniform
    const size_t row = (size_t)(j + row0) * pitch;
    double acc = 0.0;
    for (int i = lane; i < nx; i += 32) acc += theta_sum<L>(S, plane, (long long)(row + i), sh0, sh1);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
        // West-moving g (0-based direction 3) leaves through the left wall,
        // east-moving g (direction 1) through the right wall.
        const double gw = g_moving<L>(S, plane, (long long)row, 3, sh1, w1);
        const double ge = g_moving<L>(S, plane, (long long)(row + nx - 1), 1, sh1, w1);
        row_theta[j] = acc;
        row_in[j] = (abb_l * (double)hot[j] - sign_l * 2.0 * gw) + (abb_r * (double)cold[j] - sign_r * 2.0 * ge);
    }
}

// Sums of n values of x and of y, each in a fixed order (256 partial sums over
// the indices congruent mod 256, added in index order, then combined in a fixed
// tree); one block of 256 threads. out[0] = sum x, out[1] = sum y.
__global__ void sum2_fixed_kernel(const double* __restrict__ x, const double* __restrict__ y, int n,
                                  double* __restrict__ out) {
    __shared__ double px[256], py[256];
    const int t = threadIdx.x;
    double ax = 0.0, ay = 0.0;
    for (int i = t; i < n; i += 256) {
        ax += x[i];
        ay += y[i];
    }
    px[t] = ax;
    py[t] = ay;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (t < w) {
            px[t] += px[t + w];
            py[t] += py[t + w];
        }
        __syncthreads();
    }
    if (t == 0) {
        out[0] = px[0];
        out[1] = py[0];
    }
}

// Call fn with a value of the element type of a one-type storage (float, __half, __nv_bfloat16).
template <typename Fn>
void with_elem(int storage, Fn&& fn) {
    if (storage == DMRT_FP16)
        fn(__half{});
    else if (storage == DMRT_BF16)
        fn(__nv_bfloat16{});
    else
        fn(float{});
}

// Call fn with the population layout of a storage mode.
template <typename Fn>
void with_layout(int storage, Fn&& fn) {
    if (storage == DMRT_FP16)
        fn(dmrt::OneType<__half>{});
    else if (storage == DMRT_BF16)
        fn(dmrt::OneType<__nv_bfloat16>{});
    else if (storage == DMRT_MIXED)
        fn(dmrt::Split<__half, float>{});
    else if (storage == DMRT_THETA32)
        fn(dmrt::ThetaSplit{});
    else
        fn(dmrt::OneType<float>{});
}

// Byte offset of host-order plane k (f_1..f_9, g_1..g_5) in a population
// buffer, and the one-type storage its elements have.
// THETA32: host planes 9..13 (g_1..g_5) are the stored theta (float32) and
// the deviations d_1..d_4 (float16), not populations; dmrt_get_state and
// dmrt_set_state convert them.
size_t plane_offset(const dmrt_params& p, long long plane, int k) {
    if (p.storage == DMRT_MIXED)
        return k < 9 ? (size_t)dmrt::split_f(k) * plane * 2
                     : (size_t)9 * plane * 2 + (size_t)dmrt::split_g(k - 9) * plane * 4;
    if (p.storage == DMRT_THETA32)
        return k < 9 ? (size_t)dmrt::split_f(k) * plane * 2
                     : (size_t)9 * plane * 2 + (k == 9 ? 0 : (size_t)plane * 4 + (size_t)(k - 10) * plane * 2);
    return (size_t)host_plane(k) * plane * f_bytes(p.storage);
}
int plane_storage(const dmrt_params& p, int k) {
    if (p.storage == DMRT_MIXED) return k < 9 ? DMRT_FP16 : DMRT_FP32;
    if (p.storage == DMRT_THETA32) return k == 9 ? DMRT_FP32 : DMRT_FP16;
    return p.storage;
}
size_t plane_elem_bytes(const dmrt_params& p, int k) { return plane_storage(p, k) == DMRT_FP32 ? 4 : 2; }

// Default TMA tile (nodes per thread, rows, stages) per storage mode, the
// fastest measured on the 4096^2 cavity.
void default_tile(int storage, int rounding, int* npt, int* R, int* S) {
    if (storage == DMRT_THETA32 && rounding == DMRT_ROUND_STOCHASTIC) {
        *npt = 4, *R = 2, *S = 2;  // 80.0k against 78.1k MLUPS for (2, 1, 2) on 4096^2
    } else if (storage == DMRT_MIXED || storage == DMRT_THETA32) {
        *npt = 2, *R = 1, *S = 2;
    } else if (storage == DMRT_FP16 || storage == DMRT_BF16) {
        if (rounding == DMRT_ROUND_STOCHASTIC) *npt = 4, *R = 4, *S = 2;
        else *npt = 2, *R = 4, *S = 2;
    } else {
        *npt = 1, *R = 4, *S = 2;
    }
}

const dmrt::TmaVariant* find_tma_variant(int storage, int rounding, int npt, int R, int S) {
    const dmrt::TmaVariant* (*lists[7])(int*) = {dmrt::tma_variants_npt4, dmrt::tma_variants_npt2,
                                                dmrt::tma_variants_npt1, dmrt::tma_variants_fp16,
                                                dmrt::tma_variants_bf16, dmrt::tma_variants_mixed,
                                                dmrt::tma_variants_theta};
    for (auto list : lists) {
        int n = 0;
        const dmrt::TmaVariant* v = list(&n);
        for (int i = 0; i < n; ++i)
            if (v[i].storage == storage && v[i].rounding == rounding && v[i].npt == npt && v[i].R == R &&
                v[i].S == S)
                return &v[i];
    }
    return nullptr;
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    }
    return fn;
}

// 3-D view {xdim, ny, nplanes} (row stride pitch; xdim = pitch when 0) of
// planes of element type `storage` (FP32, FP16 or BF16) starting at base,
// with boxes {width, rows, planes}.
int encode_map(dmrt_ctx* c, CUtensorMap* m, void* base, int storage, int nplanes, int planes, int rows,
               int width = dmrt::kTmaBox, int xdim = 0, int ydim = 0) {
    auto enc = tensor_map_encoder();
    if (!enc) {
        set_err(c, "cuTensorMapEncodeTiled is not available from the driver");
        return DMRT_E_CUDA;
    }
    // Rows: every row the buffers hold (a slab's halo rows included), or ydim.
    const int rows_held = (int)(c->L.plane / c->L.pitch);
    cuuint64_t dims[3] = {(cuuint64_t)(xdim > 0 ? xdim : c->L.pitch), (cuuint64_t)(ydim > 0 ? ydim : rows_held),
                          (cuuint64_t)nplanes};
    const int eb = f_bytes(storage);
    cuuint64_t strides[2] = {(cuuint64_t)c->L.pitch * eb, (cuuint64_t)c->L.plane * eb};
    const CUtensorMapDataType dt = storage == DMRT_FP32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : storage == DMRT_FP16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                          : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    cuuint32_t box[3] = {(cuuint32_t)width, (cuuint32_t)rows, (cuuint32_t)planes};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(m, dt, 3, base, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_err(c, "cuTensorMapEncodeTiled failed (%d)", (int)r);
        return DMRT_E_CUDA;
    }
    return DMRT_OK;
}

// The kernel and tile that parameters p run with on a GPU of `sms` SMs (host
// logic only; AUTO resolves to DIRECT or TMA). Measured choices are noted at
// each rule.
void choose_launch(const dmrt_params& p_in, int sms, int* kernel, int* npt_out, int* R_out, int* S_out) {
    const dmrt_params p = resolved(p_in);
    int want = p.kernel;
    int dn, dr, ds;
    default_tile(p.storage, p.rounding, &dn, &dr, &ds);
    int npt = p.tma_npt > 0 ? p.tma_npt : dn;
    int R = p.tma_rows > 0 ? p.tma_rows : dr;
    int S = p.tma_stages > 0 ? p.tma_stages : ds;
    const bool st16 = p.storage == DMRT_FP16 || p.storage == DMRT_BF16;
    if (p.tma_rows <= 0 && p.ny < R) {
        // Fewer rows than the default tile: one row per item (16-bit storage:
        // one node per thread, the one-row tile compiled for both roundings).
        R = 1;
        if (p.tma_npt <= 0 && st16) npt = 1;
        if (p.tma_stages <= 0) S = npt == 1 ? 2 : 3;
    } else if (p.tma_rows <= 0 && st16 && R == 4) {
        // Small 16-bit grids: one-row items, one node per thread, while they
        // number at most two per SM (64^2: 2.9 against 3.4 us per step with
        // 2-row items); else 2-row items while 4-row items would number fewer
        // than four per SM (512^2: 7.9 against 9.4 us with 4-row items).
        const long long strips = (p.nx + dmrt::tma_strip(2) - 1) / dmrt::tma_strip(2);
        if (p.tma_npt <= 0 && p.tma_stages <= 0 && strips * p.ny <= 2LL * sms) {
            R = 1;
            npt = 1;
            S = 2;
        } else if (strips * ((p.ny + 3) / 4) < 4LL * sms) {
            R = 2;
        }
    }
    if (want == DMRT_KERNEL_AUTO) {
        want = (p.storage != DMRT_FP32 || (p.nx > 2 * dmrt::tma_strip(4) && p.ny >= 4 * R))
                   ? DMRT_KERNEL_TMA
                   : DMRT_KERNEL_DIRECT;
        if (want == DMRT_KERNEL_DIRECT && p.tma_rows <= 0 && p.tma_npt <= 0 && p.tma_stages <= 0) {
            // Small float32 grids: one-row items, one or two nodes per thread,
            // while the one-row items number at most four per SM (one step of a
            // 64^2 cavity 2.7 us against 4.9 us with the direct kernel; 256^2
            // 4.2 against 4.8 us; the direct kernel from about 384^2).
            const long long rows1 = (long long)((p.nx + dmrt::tma_strip(4) - 1) / dmrt::tma_strip(4)) * p.ny;
            if (rows1 <= 4LL * sms) {
                want = DMRT_KERNEL_TMA;
                R = 1;
                if (rows1 <= 2LL * sms) npt = 1, S = 2;
                else npt = 2, S = 3;
            }
        }
    }
    *kernel = want;
    *npt_out = npt;
    *R_out = R;
    *S_out = S;
}

// Resolve the kernel variant and prepare its launch configuration.
// Cluster kernel for runs of steps: float32, a whole cavity, the state of
// both buffers in the shared memory of one cluster of up to 16 blocks.
// The cluster kernel's launch shape for c (blocks, rows per block, threads,
// shared memory); false if the cavity does not fit one cluster on this GPU.
// The cluster kernel compiled for blocks of at most `threads` threads, and its launch.
// The compiled form for a block of `threads` threads whose rows hold
// `nodes` nodes: one node per node thread (blocks up to 640 threads always) or
// a loop over the block's nodes.
const void* cluster_func(int threads, int nodes) {
    if (threads <= 320) return (const void*)dmrt::step_cluster_kernel<320, true>;
    if (threads <= 640) return (const void*)dmrt::step_cluster_kernel<640, true>;
    return nodes <= threads - 64 ? (const void*)dmrt::step_cluster_kernel<1024, true>
                                 : (const void*)dmrt::step_cluster_kernel<1024, false>;
}
cudaError_t launch_cluster_kernel(const cudaLaunchConfig_t& cfg, const dmrt::ClusterArgs& C) {
    const int threads = (int)cfg.blockDim.x, nodes = C.rows_per * C.A[0].nx;
    if (threads <= 320) return cudaLaunchKernelEx(&cfg, dmrt::step_cluster_kernel<320, true>, C);
    if (threads <= 640) return cudaLaunchKernelEx(&cfg, dmrt::step_cluster_kernel<640, true>, C);
    if (nodes <= threads - 64) return cudaLaunchKernelEx(&cfg, dmrt::step_cluster_kernel<1024, true>, C);
    return cudaLaunchKernelEx(&cfg, dmrt::step_cluster_kernel<1024, false>, C);
}

bool cluster_fit(dmrt_ctx* c, int* csize_out, int* crows_out, int* threads_out, size_t* smem_out) {
    const dmrt_params& p = c->p;
    if (p.storage != DMRT_FP32 || c->slab) return false;
    for (int csize : {16, 8}) {
        const int cs = std::min(csize, p.ny);
        const int rows = (p.ny + cs - 1) / cs;
        const int blocks = (p.ny + rows - 1) / rows;
        const size_t smem = dmrt::cluster_smem_bytes(rows, p.nx, p.ny);
        const int threads = dmrt::cluster_threads(rows, p.nx);
        const void* fn = cluster_func(threads, rows * p.nx);
        // At most two nodes per node thread (the kernel takes no more).
        if (smem > (size_t)dmrt::kMaxSmem || rows * p.nx > 2 * (threads - 64)) continue;
        if (blocks > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
            (void)cudaGetLastError();
            continue;
        }
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
            (void)cudaGetLastError();
            continue;
        }
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = blocks;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(blocks);
        cfg.blockDim = dim3(threads);
        cfg.dynamicSmemBytes = smem;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) != cudaSuccess || nclusters < 1) {
            (void)cudaGetLastError();
            continue;
        }
        *csize_out = blocks;
        *crows_out = rows;
        *threads_out = threads;
        *smem_out = smem;
        return true;
    }
    return false;
}

int setup_cluster(dmrt_ctx* c) {
    const dmrt_params& p = c->p;
    c->cluster = false;
    if (p.storage != DMRT_FP32 || c->slab) {
        set_err(c, "the cluster kernel runs float32 storage of a whole cavity only");
        return DMRT_E_ARG;
    }
    if (cluster_fit(c, &c->csize, &c->crows, &c->cthreads, &c->csmem)) {
        c->cluster = true;
        return DMRT_OK;
    }
    set_err(c, "a %d x %d float32 cavity does not fit the shared memory of one thread-block cluster", p.nx, p.ny);
    return DMRT_E_ARG;
}


// AUTO takes the cluster kernel for runs of steps of a small float32 cavity:
// rows split over 16 blocks with at most 1024 nodes per block (e.g. up to
// 128^2), whose state fits the cluster's shared memory, and no tile asked for.
// Measured per step, cluster / one-row TMA items: 16^2 1.23 / 3.11, 32^2 1.23 /
// 2.98, 64^2 1.43 / 2.66, 96^2 1.65 / 2.95, 128^2 2.60 / 2.78 us.
bool auto_cluster(const dmrt_params& p) {
    if (p.kernel != DMRT_KERNEL_AUTO || p.storage != DMRT_FP32) return false;
    if (p.tma_npt > 0 || p.tma_rows > 0 || p.tma_stages > 0) return false;
    const int crows = (p.ny + 15) / 16;
    return (long long)crows * p.nx <= 1024 && dmrt::cluster_smem_bytes(crows, p.nx, p.ny) <= (size_t)dmrt::kMaxSmem;
}

int setup_kernel(dmrt_ctx* c) {
    const dmrt_params& p0 = c->p;
    c->cluster = false;
    if (p0.kernel == DMRT_KERNEL_CLUSTER) {
        int rc = setup_cluster(c);
        if (rc) return rc;
    } else if (auto_cluster(p0) && !c->slab) {
        // Where the cluster does not fit this GPU, AUTO keeps the other kernels.
        c->cluster = cluster_fit(c, &c->csize, &c->crows, &c->cthreads, &c->csmem);
    }
    dmrt_params p = p0;  // single steps and the adjoint: the kernel AUTO picks among the others
    if (p.kernel == DMRT_KERNEL_CLUSTER) p.kernel = DMRT_KERNEL_AUTO;
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev), "cudaGetDevice");
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    int want, npt, R, S;
    choose_launch(p, sms, &want, &npt, &R, &S);
    if (want == DMRT_KERNEL_DIRECT && p.storage != DMRT_FP32) {
        set_err(c, "the direct kernel stores float32 only; 16-bit and mixed storage run the TMA kernel");
        return DMRT_E_ARG;
    }
    c->kernel = want;
    c->npt = npt;
    c->R = R;
    c->S = S;
    c->tma_func = nullptr;
    if (want != DMRT_KERNEL_TMA) {
        // A direct grid of fewer blocks than two per SM gets one more row of
        // blocks, whose first block only sums the previous step's Nusselt rows.
        if ((long long)c->grid.x * c->grid.y < 2LL * sms) c->grid.y += 1;
        return DMRT_OK;
    }
    const dmrt::TmaVariant* v = find_tma_variant(p.storage, p.rounding, npt, R, S);
    if (!v) {
        set_err(c, "no TMA tile with %d nodes/thread, %d rows, %d stages is compiled in for this "
                   "storage and rounding", npt, R, S);
        return DMRT_E_ARG;
    }
    c->tma_func = v->func;
    c->tma_block = R * (256 / npt);
    if (p.ny < R) {
        set_err(c, "TMA kernel needs ny >= %d", R);
        return DMRT_E_ARG;
    }
    const int fb = f_bytes(p.storage), gb = g_bytes(p.storage);
    const int strip = dmrt::tma_strip(std::min(fb, gb));
    c->geo.n_strips = (p.nx + strip - 1) / strip;
    c->geo.n_rowblocks = (p.ny + R - 1) / R;
    const bool split = p.storage == DMRT_MIXED;
    const bool theta = p.storage == DMRT_THETA32;
    c->tma_smem = theta ? dmrt::step_tma_smem_bytes_theta(v->ts != 0, R, S)
                        : dmrt::step_tma_smem_bytes(split, v->ts != 0, R, S, fb, gb);
    if (c->tma_smem > (size_t)dmrt::kMaxSmem) {
        set_err(c, "TMA tile %dx%d needs %zu bytes of shared memory", R, S, c->tma_smem);
        return DMRT_E_ARG;
    }
    CK(cudaFuncSetAttribute(c->tma_func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->tma_smem),
       "set TMA kernel shared memory");
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, c->tma_func, c->tma_block, c->tma_smem),
       "occupancy");
    if (per_sm < 1) {
        set_err(c, "TMA tile %dx%d does not fit on an SM", R, S);
        return DMRT_E_ARG;
    }
    const long long items = (long long)c->geo.n_strips * c->geo.n_rowblocks;
    // A grid smaller than the resident capacity gets one more block, which only
    // sums the previous step's Nusselt rows (off the first item's path).
    c->tma_grid = items < (long long)sms * per_sm ? (int)items + 1 : sms * per_sm;
    for (int b = 0; b < 2; ++b) {
        // Loads from buffer b, stores (nx columns wide) to the other one.
        dmrt::TmaMaps& m = c->tmaps[b];
        std::memset(&m, 0, sizeof m);
        float* dst = buf(c, 1 - b);
        int rc;
        if (theta) {
            // 9 float16 flow planes, the float32 theta plane, 4 float16 deviation
            // planes; theta and the deviations are loaded R + 2 rows high.
            const size_t toff = (size_t)9 * c->L.plane * 2, doff = toff + (size_t)c->L.plane * 4;
            char* src = reinterpret_cast<char*>(buf(c, b));
            char* dd = reinterpret_cast<char*>(dst);
            rc = encode_map(c, &m.ld[0], buf(c, b), DMRT_FP16, 9, 3, R);
            if (!rc) rc = encode_map(c, &m.ld[1], src + toff, DMRT_FP32, 1, 1, R + 2);
            if (!rc) rc = encode_map(c, &m.ld[2], src + doff, DMRT_FP16, 4, 4, R + 2);
            if (!rc) rc = encode_map(c, &m.st[0], dst, DMRT_FP16, 9, 9, R, strip, p.nx, c->row0 + p.ny);
            if (!rc) rc = encode_map(c, &m.st[1], dd + toff, DMRT_FP32, 1, 1, R, strip, p.nx, c->row0 + p.ny);
            if (!rc) rc = encode_map(c, &m.st[2], dd + doff, DMRT_FP16, 4, 4, R, strip, p.nx, c->row0 + p.ny);
        } else if (split) {
            // 9 float16 flow planes, then 5 float32 thermal planes.
            const size_t goff = (size_t)9 * c->L.plane * 2;
            char* g = reinterpret_cast<char*>(buf(c, b)) + goff;
            char* gd = reinterpret_cast<char*>(dst) + goff;
            rc = encode_map(c, &m.ld[0], buf(c, b), DMRT_FP16, 9, 3, R);
            if (!rc) rc = encode_map(c, &m.ld[1], g, DMRT_FP32, 5, 3, R);
            if (!rc) rc = encode_map(c, &m.ld[2], g, DMRT_FP32, 5, 1, R);
            if (!rc) rc = encode_map(c, &m.st[0], dst, DMRT_FP16, 9, 9, R, strip, p.nx, c->row0 + p.ny);
            if (!rc) rc = encode_map(c, &m.st[1], gd, DMRT_FP32, 5, 5, R, strip, p.nx, c->row0 + p.ny);
        } else {
            rc = encode_map(c, &m.ld[0], buf(c, b), p.storage, kPlanes, 6, R);
            if (!rc) rc = encode_map(c, &m.ld[1], buf(c, b), p.storage, kPlanes, 4, R);
            if (!rc) rc = encode_map(c, &m.st[0], dst, p.storage, kPlanes, kPlanes, R, strip, p.nx, c->row0 + p.ny);
        }
        if (rc) return rc;
    }
    return DMRT_OK;
}

int validate(const dmrt_params* p, dmrt_ctx* c) {
    if (!p) {
        set_err(c, "params is NULL");
        return DMRT_E_ARG;
    }
    if (p->nx < 2 || p->ny < 2 || p->nx > 32768 || p->ny > 32768) {
        set_err(c, "grid %d x %d outside [2, 32768]", p->nx, p->ny);
        return DMRT_E_ARG;
    }
    if (!(p->Pr > 0.0) || !(p->Ra >= 0.0) || !std::isfinite(p->Ra) || !std::isfinite(p->Pr)) {
        set_err(c, "need Pr > 0 and finite Ra >= 0 (Pr=%g Ra=%g)", p->Pr, p->Ra);
        return DMRT_E_ARG;
    }
    if (!(p->alpha > 0.0) && !(p->Ma > 0.0 && p->Ra > 0.0)) {
        set_err(c, "give alpha > 0, or Ma > 0 with Ra > 0");
        return DMRT_E_ARG;
    }
    if (p->left_wall < 0 || p->left_wall > 1 || p->right_wall < 0 || p->right_wall > 1) {
        set_err(c, "wall kinds must be DMRT_WALL_FIXED or DMRT_WALL_ADIABATIC");
        return DMRT_E_ARG;
    }
    if (p->storage < DMRT_FP32 || p->storage > DMRT_THETA32) {
        set_err(c, "storage must be DMRT_FP32, DMRT_FP16, DMRT_BF16, DMRT_MIXED or DMRT_THETA32 (got %d)",
                p->storage);
        return DMRT_E_ARG;
    }
    if (p->rounding != DMRT_ROUND_NEAREST && p->rounding != DMRT_ROUND_STOCHASTIC &&
        p->rounding != DMRT_ROUND_AUTO) {
        set_err(c, "rounding must be DMRT_ROUND_NEAREST, DMRT_ROUND_STOCHASTIC or DMRT_ROUND_AUTO");
        return DMRT_E_ARG;
    }
    if (p->rounding == DMRT_ROUND_STOCHASTIC && p->storage == DMRT_FP32) {
        set_err(c, "stochastic rounding applies to 16-bit and mixed storage only");
        return DMRT_E_ARG;
    }
    if (p->kernel < DMRT_KERNEL_AUTO || p->kernel > DMRT_KERNEL_CLUSTER) {
        set_err(c, "kernel must be DMRT_KERNEL_AUTO, _DIRECT, _TMA or _CLUSTER");
        return DMRT_E_ARG;
    }
    if (p->nu_capacity < 1) {
        set_err(c, "nu_capacity must be >= 1");
        return DMRT_E_ARG;
    }
    const double dT = p->theta_hot - p->theta_cold;
    if (!std::isfinite(dT) || (dT == 0.0 && p->Ra > 0.0)) {
        set_err(c, "theta_hot - theta_cold must be finite and nonzero when Ra > 0");
        return DMRT_E_ARG;
    }
    return DMRT_OK;
}

}  // namespace

extern "C" {

void dmrt_default_params(dmrt_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->nx = 64;
    p->ny = 64;
    p->Ra = 1e4;
    p->Pr = 0.01;
    p->alpha = 0.1;
    p->Ma = 0.0;
    p->theta_hot = 0.5;
    p->theta_cold = -0.5;
    p->theta_ref = 0.0;
    p->theta_init = 0.0;
    p->left_wall = DMRT_WALL_FIXED;
    p->right_wall = DMRT_WALL_FIXED;
    p->storage = DMRT_FP32;
    p->kernel = DMRT_KERNEL_AUTO;
    p->nu_capacity = 1 << 20;
    p->tma_rows = 0;
    p->tma_stages = 0;
    p->tma_npt = 0;
    p->rounding = DMRT_ROUND_AUTO;
}

int dmrt_derive(const dmrt_params* p, dmrt_consts* out) {
    int rc = validate(p, nullptr);
    if (rc) return rc;
    const double H = (double)p->ny;
    const double dT = p->theta_hot - p->theta_cold;
    dmrt_consts k;
    // alpha from Ma: Ma = sqrt(3 g beta dT H) and g beta dT = Ra nu alpha / H^3
    // = Ra Pr alpha^2 / H^3 (Eq. 9) give alpha = Ma H / sqrt(3 Ra Pr).
    k.alpha = p->alpha > 0.0 ? p->alpha : p->Ma * H / std::sqrt(3.0 * p->Ra * p->Pr);
    k.nu = p->Pr * k.alpha;
    k.s_nu = 2.0 / (6.0 * k.nu + 1.0);               // Eq. 32
    k.s_e = k.s_eps = k.s_nu;
    k.s_q = 8.0 * (2.0 - k.s_nu) / (8.0 - k.s_nu);    // Eq. 32
    const double inv_k = 0.5 + std::sqrt(3.0) / 6.0;  // 1/sigma_k, Eq. 40
    const double inv_e = 0.5 + std::sqrt(3.0) / 3.0;  // 1/sigma_e = 1/sigma_nu, Eq. 40
    k.sig_k = 1.0 / inv_k;
    k.sig_e = k.sig_nu = 1.0 / inv_e;
    k.a = 10.0 * k.alpha / (inv_k - 0.5) - 4.0;       // Eq. 43
    k.gbeta = dT != 0.0 ? p->Ra * k.nu * k.alpha / (H * H * H) / dT : 0.0;
    k.abb = 2.0 * std::sqrt(3.0) * k.alpha;           // Eq. 45
    k.Ma = std::sqrt(3.0 * k.gbeta * dT * H);
    k.fo_per_step = k.alpha / (H * H);                // Eq. 20
    if (!(k.a > -4.0 && k.a < 1.0)) {
        set_err(nullptr, "a = %g outside (-4, 1): alpha must lie in (0, %.6f)", k.a,
                1.0 / (4.0 * std::sqrt(3.0)));
        return DMRT_E_UNSTABLE;
    }
    if (!(k.s_nu > 0.0 && k.s_nu < 2.0 && k.s_q > 0.0 && k.s_q < 2.0)) {
        set_err(nullptr, "relaxation rate outside (0, 2)");
        return DMRT_E_UNSTABLE;
    }
    if (out) *out = k;
    return DMRT_OK;
}

int dmrt_workspace_size(const dmrt_params* p, size_t* bytes) {
    int rc = validate(p, nullptr);
    if (rc) return rc;
    if (!bytes) return DMRT_E_ARG;
    *bytes = make_layout(*p).total;
    return DMRT_OK;
}

}  // extern "C"

// A context for rows y0 .. y0 + rows - 1 of the cavity pg (the whole cavity:
// y0 = 0, rows = pg->ny, slab = false). The model constants come from the
// whole cavity (H = pg->ny in Eqs. 9 and 18); the context's own parameters are
// those of its rows.
static int create_ctx(const dmrt_params* pg, int y0, int rows, bool slab, const double* theta0, void* workspace,
                      size_t workspace_bytes, void* stream, dmrt_ctx** out) {
    if (!out) {
        set_err(nullptr, "out is NULL");
        return DMRT_E_ARG;
    }
    *out = nullptr;
    dmrt_consts k;
    int rc = dmrt_derive(pg, &k);
    if (rc) return rc;
    if (slab && (y0 < 0 || rows < 1 || y0 + rows > pg->ny)) {
        set_err(nullptr, "slab rows %d .. %d outside the cavity's %d rows", y0, y0 + rows - 1, pg->ny);
        return DMRT_E_ARG;
    }
    if (slab && pg->storage == DMRT_THETA32) {
        // A THETA32 pull reads the source row's theta as well as the crossing
        // populations, which the face messages do not carry.
        set_err(nullptr, "slabs take float32, 16-bit or mixed storage, not THETA32");
        return DMRT_E_ARG;
    }
    dmrt_params pl = resolved(*pg);
    pl.ny = rows;
    const int row0 = slab ? 1 : 0;
    Layout L = make_layout(pl, 2 * row0);
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255)) {
        set_err(nullptr, "workspace must be a 256-byte aligned device pointer");
        return DMRT_E_ARG;
    }
    if (workspace_bytes < L.total) {
        set_err(nullptr, "workspace too small: %zu < %zu bytes", workspace_bytes, L.total);
        return DMRT_E_SPACE;
    }
    dmrt_ctx* c = new (std::nothrow) dmrt_ctx();
    if (!c) {
        set_err(nullptr, "out of host memory");
        return DMRT_E_SPACE;
    }
    const dmrt_params* p = &c->p;
    c->p = pl;
    c->k = k;
    c->L = L;
    c->ws = static_cast<char*>(workspace);
    c->stream = static_cast<cudaStream_t>(stream);
    c->cur = 0;
    c->t = 0;
    c->graph[0] = c->graph[1] = nullptr;
    c->graph_len = 64;
    c->nu_floor = 0;
    c->next_poll = kPollSteps;
    c->err[0] = 0;
    c->slab = slab;
    c->row0 = row0;
    c->y0 = y0;
    c->H = pg->ny;
    c->wall_lo = y0 == 0;
    c->wall_hi = y0 + rows == pg->ny;

    c->sc = dmrt::make_step_consts(*pg, k);  // H of the whole cavity
    const double sh0 = dmrt::thermal_shift0(*pg, k);
    const double sh1 = dmrt::thermal_shift1(*pg, k);

    const int nxq = (p->nx + 3) / 4;
    int wx = 1;
    while (wx < nxq && wx < 32) wx <<= 1;
    c->wx_log2 = 0;
    while ((1 << c->wx_log2) < wx) ++c->wx_log2;
    const int rows_per_block = (dmrt::kDirectThreads / 32) * (32 / wx);
    c->grid = dim3((nxq + wx - 1) / wx, (p->ny + rows_per_block - 1) / rows_per_block, 1);

    auto fail = [&](int code) {
        std::snprintf(g_create_error, sizeof g_create_error, "%s", c->err);
        delete c;
        return code;
    };
    int rc2 = setup_kernel(c);
    if (rc2) return fail(rc2);
    // Zero the scalars and the ring, set the wall profiles, write the initial state.
    if (cudaMemsetAsync(c->ws + L.off_hot, 0, L.total - L.off_hot, c->stream) != cudaSuccess)
        return fail(cuda_fail(c, cudaGetLastError(), "cudaMemsetAsync"));
    fill_kernel<<<(p->ny + 255) / 256, 256, 0, c->stream>>>(
        reinterpret_cast<float*>(c->ws + L.off_hot), nullptr, p->theta_hot, p->ny);
    fill_kernel<<<(p->ny + 255) / 256, 256, 0, c->stream>>>(
        reinterpret_cast<float*>(c->ws + L.off_cold), nullptr, p->theta_cold, p->ny);
    const double* d_theta0 = nullptr;
    if (theta0) {
        // Stage the host field in buffer B (not yet used: it holds 28 to 56 bytes per node).
        double* stage = reinterpret_cast<double*>(c->ws + L.off_b);
        cudaError_t e = cudaMemcpyAsync(stage, theta0, (size_t)p->nx * p->ny * sizeof(double),
                                        cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) return fail(cuda_fail(c, e, "copy theta0"));
        d_theta0 = stage;
    }
    const int init_grid = (int)std::min<long long>(L.plane / L.pitch, 4096);
    with_layout(p->storage, [&](auto tag) {
        using Lt = decltype(tag);
        init_kernel<Lt><<<init_grid, 256, 0, c->stream>>>(reinterpret_cast<unsigned char*>(buf(c, 0)), d_theta0,
                                                          p->theta_init, k.a, sh0, sh1, p->nx, p->ny,
                                                          L.pitch, L.plane, row0);
    });
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(cuda_fail(c, e, "init kernel"));
    // Buffer B: zero (its padding columns must read as zero; the first step
    // writes every node, and a slab's halo rows are filled before they are read).
    e = cudaMemsetAsync(c->ws + L.off_b, 0, L.buf_bytes, c->stream);
    if (e != cudaSuccess) return fail(cuda_fail(c, e, "clear buffer B"));
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(cuda_fail(c, e, "init synchronize"));
    *out = c;
    return DMRT_OK;
}

extern "C" {

int dmrt_create(const dmrt_params* p, const double* theta0, void* workspace,
                size_t workspace_bytes, void* stream, dmrt_ctx** out) {
    if (!p) {
        set_err(nullptr, "params is NULL");
        return DMRT_E_ARG;
    }
    return create_ctx(p, 0, p->ny, false, theta0, workspace, workspace_bytes, stream, out);
}

int dmrt_slab_workspace_size(const dmrt_params* p, int32_t rows, size_t* bytes) {
    int rc = validate(p, nullptr);
    if (rc) return rc;
    if (!bytes || rows < 1 || rows > p->ny) {
        set_err(nullptr, "need 1 <= rows <= ny and a non-NULL bytes");
        return DMRT_E_ARG;
    }
    if (p->storage == DMRT_THETA32) {
        set_err(nullptr, "slabs take float32, 16-bit or mixed storage, not THETA32");
        return DMRT_E_ARG;
    }
    dmrt_params pl = *p;
    pl.ny = rows;
    *bytes = make_layout(pl, 2).total;
    return DMRT_OK;
}

int dmrt_create_slab(const dmrt_params* p, int32_t y0, int32_t rows, const double* theta0, void* workspace,
                     size_t workspace_bytes, void* stream, dmrt_ctx** out) {
    if (!p) {
        set_err(nullptr, "params is NULL");
        return DMRT_E_ARG;
    }
    return create_ctx(p, y0, rows, true, theta0, workspace, workspace_bytes, stream, out);
}

extern "C++" {
// A kernel launch on the stream that may begin while the previous kernel on
// the stream finishes (programmatic stream serialization); the kernel waits
// for that kernel's completion (grid_dep_wait) before touching global memory.
template <typename... KArgs, typename... Args>
static cudaError_t launch_overlapped(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t stream,
                                    Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}
static cudaError_t launch_overlapped(const void* kernel, dim3 grid, dim3 block, size_t smem,
                                     cudaStream_t stream, void** params) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, kernel, params);
}
}  // extern "C++"

// One step from buffer `from` to the other one.
static int launch_step(dmrt_ctx* c, int from) {
    dmrt::StepArgs A = step_args(c, from);
    if (c->kernel == DMRT_KERNEL_TMA) {
        void* params[4] = {&c->tmaps[from], &A, &c->sc, &c->geo};
        cudaError_t e = launch_overlapped(c->tma_func, dim3(c->tma_grid), dim3(c->tma_block), c->tma_smem,
                                          c->stream, params);
        if (e != cudaSuccess) return cuda_fail(c, e, "TMA step launch");
    } else {
        cudaError_t e = launch_overlapped(dmrt::step_direct_kernel, c->grid, dim3(dmrt::kDirectThreads),
                                          c->stream, A, c->sc);
        if (e != cudaSuccess) return cuda_fail(c, e, "step launch");
    }
    return DMRT_OK;
}

static int launch_one(dmrt_ctx* c) {
    int rc = launch_step(c, c->cur);
    if (rc) return rc;
    c->cur ^= 1;
    c->t += 1;
    return DMRT_OK;
}

// Appends kernel node `kp` to graph g after `prev` (none: first node) through a
// programmatic edge: the node's blocks may launch while prev's last blocks run
// and wait in the kernel (grid_dep_wait) for prev to complete. If the edge type
// is refused, an ordinary edge (launch after completion) is used instead.
static cudaError_t add_step_node(cudaGraph_t g, cudaGraphNode_t prev, const cudaKernelNodeParams* kp,
                                 cudaGraphNode_t* node) {
    cudaError_t e = cudaGraphAddKernelNode(node, g, nullptr, 0, kp);
    if (e != cudaSuccess || !prev) return e;
    cudaGraphEdgeData ed;
    std::memset(&ed, 0, sizeof ed);
    ed.from_port = cudaGraphKernelNodePortProgrammatic;
    ed.type = cudaGraphDependencyTypeProgrammatic;
    e = cudaGraphAddDependencies(g, &prev, node, &ed, 1);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        e = cudaGraphAddDependencies(g, &prev, node, nullptr, 1);
    }
    return e;
}

// A graph of graph_len (even) steps starting from buffer `from`, built node by
// node (no stream capture, so it works on any stream, the legacy default included).
static int build_graph(dmrt_ctx* c, int from) {
    cudaGraph_t g;
    CK(cudaGraphCreate(&g, 0), "cudaGraphCreate");
    cudaGraphNode_t prev = nullptr;
    dmrt::StepArgs args[2] = {step_args(c, from), step_args(c, 1 - from)};
    for (int i = 0; i < c->graph_len; ++i) {
        const int src = (i & 1) ? 1 - from : from;
        cudaKernelNodeParams kp = {};
        void* dparams[2] = {&args[i & 1], &c->sc};
        void* tparams[4] = {&c->tmaps[src], &args[i & 1], &c->sc, &c->geo};
        if (c->kernel == DMRT_KERNEL_TMA) {
            kp.func = const_cast<void*>(c->tma_func);
            kp.gridDim = dim3(c->tma_grid);
            kp.blockDim = dim3(c->tma_block);
            kp.sharedMemBytes = (unsigned)c->tma_smem;
            kp.kernelParams = tparams;
        } else {
            kp.func = (void*)dmrt::step_direct_kernel;
            kp.gridDim = c->grid;
            kp.blockDim = dim3(dmrt::kDirectThreads);
            kp.sharedMemBytes = 0;
            kp.kernelParams = dparams;
        }
        cudaGraphNode_t node;
        cudaError_t e = add_step_node(g, prev, &kp, &node);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            return cuda_fail(c, e, "cudaGraphAddKernelNode");
        }
        prev = node;
    }
    cudaError_t e = cudaGraphInstantiate(&c->graph[from], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
    return DMRT_OK;
}

// After a run of steps: sum the last step's local Nusselt numbers into the ring
// (every step sums its predecessor's; the last one has no successor yet).
static int finalize_nu(dmrt_ctx* c) {
    dmrt::nu_finalize_kernel<<<1, 256, 0, c->stream>>>(step_args(c, c->cur));
    CK(cudaGetLastError(), "step launch");
    return DMRT_OK;
}

int dmrt_choose_launch(const dmrt_params* p, int32_t sms, int32_t* kernel, int32_t* npt, int32_t* rows,
                       int32_t* stages) {
    if (!p || sms < 1 || !kernel || !npt || !rows || !stages) {
        set_err(nullptr, "dmrt_choose_launch: NULL argument or sms < 1");
        return DMRT_E_ARG;
    }
    int rc = validate(p, nullptr);
    if (rc) return rc;
    if (auto_cluster(*p)) {
        *kernel = DMRT_KERNEL_CLUSTER;
        *npt = *rows = *stages = 0;
        return DMRT_OK;
    }
    if (p->kernel == DMRT_KERNEL_CLUSTER) {
        // Fits when both buffers' rows fit the shared memory of 16 blocks.
        const int crows = (p->ny + 15) / 16;
        if (p->storage != DMRT_FP32 || dmrt::cluster_smem_bytes(crows, p->nx, p->ny) > (size_t)dmrt::kMaxSmem) {
            set_err(nullptr, "the cluster kernel needs float32 storage and a cavity whose state fits one cluster");
            return DMRT_E_ARG;
        }
        *kernel = DMRT_KERNEL_CLUSTER;
        *npt = *rows = *stages = 0;
        return DMRT_OK;
    }
    int k, n, r, st;
    choose_launch(*p, sms, &k, &n, &r, &st);
    if (k == DMRT_KERNEL_DIRECT && p->storage != DMRT_FP32) {
        set_err(nullptr, "the direct kernel stores float32 only; 16-bit and mixed storage run the TMA kernel");
        return DMRT_E_ARG;
    }
    *kernel = k;
    *npt = k == DMRT_KERNEL_TMA ? n : 0;
    *rows = k == DMRT_KERNEL_TMA ? r : 0;
    *stages = k == DMRT_KERNEL_TMA ? st : 0;
    return DMRT_OK;
}

// Reads the device error word (synchronises the stream): DMRT_E_TIMEOUT or
// DMRT_E_DIVERGED when a bit is set, else DMRT_OK.
static int poll_error(dmrt_ctx* c) {
    unsigned err = 0;
    CK(cudaMemcpyAsync(&err, &misc(c)->err, sizeof err, cudaMemcpyDeviceToHost, c->stream), "read error flag");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    if (err & dmrt::kErrTimeout) {
        set_err(c, "a bounded device-side wait expired after %lld steps", c->t);
        return DMRT_E_TIMEOUT;
    }
    if (err & dmrt::kErrBounds) {
        set_err(c, "an index out of range was seen (bounds-checked build) after %lld steps", c->t);
        return DMRT_E_BOUNDS;
    }
    if (err & dmrt::kErrNonFinite) {
        set_err(c, "non-finite density or temperature after %lld steps", c->t);
        return DMRT_E_DIVERGED;
    }
    return DMRT_OK;
}

// Runs of n >= 2 steps on the cluster kernel: one launch.
// n steps in one cluster launch; with `record`, the state after each step s of
// the launch is also written to record + s * stride.
static int launch_cluster(dmrt_ctx* c, int n, float* record = nullptr, long long stride = 0) {
    dmrt::ClusterArgs C;
    C.A[0] = step_args(c, 0);
    C.A[1] = step_args(c, 1);
    C.K = c->sc;
    C.steps = n;
    C.parity = c->cur;
    C.rows_per = c->crows;
    C.start = nullptr;
    C.record = record;
    C.record_stride = stride;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = c->csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(c->csize);
    cfg.blockDim = dim3(c->cthreads);
    cfg.dynamicSmemBytes = c->csmem;
    cfg.stream = c->stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CK(launch_cluster_kernel(cfg, C), "cluster step launch");
    c->cur ^= n & 1;
    c->t += n;
    return DMRT_OK;
}

// nsteps steps; with `finalize`, the last step's Nusselt rows are summed into
// the ring at the end (without, the next launch sums them). With `record`
// (cluster kernel only), the state after the run's step s is also written to
// record + s * stride.
static int step_run(dmrt_ctx* c, int64_t nsteps, bool finalize, float* record = nullptr, long long stride = 0) {
    if (!c || nsteps < 0) return DMRT_E_ARG;
    if (record && !c->cluster) return DMRT_E_ARG;
    if (c->cluster) {
        while (nsteps > 0) {
            if (c->t >= c->next_poll) {
                c->next_poll = c->t + kPollSteps;
                int rc = poll_error(c);
                if (rc) return rc;
            }
            // Up to the next divergence poll, in one launch.
            const long long n = std::min<long long>(nsteps, std::max<long long>(1, c->next_poll - c->t));
            int rc = n >= 2 ? launch_cluster(c, (int)n, record, stride) : launch_one(c);
            if (rc) return rc;
            if (record && n < 2)
                CK(cudaMemcpyAsync(record, buf(c, c->cur), (size_t)kPlanes * (size_t)c->L.plane * sizeof(float),
                                   cudaMemcpyDeviceToDevice, c->stream),
                   "record");
            if (record) record += n * stride;
            nsteps -= n;
        }
        return finalize ? finalize_nu(c) : DMRT_OK;
    }
    if (c->slab && !(c->wall_lo && c->wall_hi) && nsteps > 1) {
        set_err(c, "a slab with neighbours takes one step at a time (dmrt_slab_step), its halo rows "
                   "exchanged in between");
        return DMRT_E_STATE;
    }
    while (nsteps > 0) {
        if (c->t >= c->next_poll) {
            // Every kPollSteps steps: stop a run that has diverged (the steps
            // enqueued so far complete; the ring holds their Nusselt numbers).
            c->next_poll = c->t + kPollSteps;
            int rc = finalize_nu(c);
            if (!rc) rc = poll_error(c);
            if (rc) return rc;
        }
        if (nsteps >= c->graph_len) {
            if (!c->graph[c->cur]) {
                int rc = build_graph(c, c->cur);
                if (rc) return rc;
            }
            CK(cudaGraphLaunch(c->graph[c->cur], c->stream), "cudaGraphLaunch");
            c->t += c->graph_len;  // even length: the state stays in the same buffer
            nsteps -= c->graph_len;
        } else {
            int rc = launch_one(c);
            if (rc) return rc;
            nsteps -= 1;
        }
    }
    return finalize ? finalize_nu(c) : DMRT_OK;
}

int dmrt_step(dmrt_ctx* c, int64_t nsteps) { return step_run(c, nsteps, true); }

// ---- y-slabs: halo rows --------------------------------------------------------
namespace {

// The plane groups a face message carries: P (the populations moving up,
// e_y = +1: f3 f6 f7 g3) or N (moving down: f5 f8 f9 g5), of one buffer row.
// One-type layout: 4 consecutive planes; split layout: 3 flow planes, then 1
// thermal plane. The message holds each plane's nx values, in plane order.
struct FacePart {
    size_t plane_byte;  // byte offset of the part's first plane in the buffer
    size_t eb;          // bytes per element
    int planes;
};
int face_parts(const dmrt_ctx* c, bool up, FacePart* parts) {
    const long long PL = c->L.plane;
    if (c->p.storage == DMRT_MIXED) {
        parts[0] = {(size_t)(up ? 3 : 6) * PL * 2, 2, 3};
        parts[1] = {(size_t)9 * PL * 2 + (size_t)(up ? 3 : 4) * PL * 4, 4, 1};
        return 2;
    }
    const size_t eb = (size_t)f_bytes(c->p.storage);
    parts[0] = {(size_t)(up ? dmrt::kGroupP : dmrt::kGroupN) * PL * eb, eb, 4};
    return 1;
}
size_t face_bytes(const dmrt_ctx* c) {
    FacePart parts[2];
    const int n = face_parts(c, true, parts);
    size_t b = 0;
    for (int i = 0; i < n; ++i) b += parts[i].eb * parts[i].planes * (size_t)c->p.nx;
    return b;
}
// Copy the face planes of buffer row `brow` of the current state to msg
// (to_msg) or from msg into it; stream-ordered on the context's stream.
int face_copy(dmrt_ctx* c, bool up, int brow, void* msg, bool to_msg) {
    FacePart parts[2];
    const int n = face_parts(c, up, parts);
    char* base = reinterpret_cast<char*>(buf(c, c->cur));
    char* m = static_cast<char*>(msg);
    for (int i = 0; i < n; ++i) {
        const FacePart& f = parts[i];
        char* plane0 = base + f.plane_byte + (size_t)brow * c->L.pitch * f.eb;
        const size_t width = (size_t)c->p.nx * f.eb;
        const size_t spitch = (size_t)c->L.plane * f.eb;
        cudaError_t e = to_msg ? cudaMemcpy2DAsync(m, width, plane0, spitch, width, f.planes,
                                                   cudaMemcpyDeviceToDevice, c->stream)
                               : cudaMemcpy2DAsync(plane0, spitch, m, width, width, f.planes,
                                                   cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "halo row copy");
        m += width * f.planes;
    }
    return DMRT_OK;
}

}  // namespace

int dmrt_slab_halo_bytes(const dmrt_ctx* c, size_t* bytes) {
    if (!c || !bytes) return DMRT_E_ARG;
    *bytes = face_bytes(c);
    return DMRT_OK;
}

int dmrt_slab_pack(dmrt_ctx* c, void* to_below, void* to_above) {
    if (!c) return DMRT_E_ARG;
    if (!c->slab) {
        set_err(c, "not a slab context");
        return DMRT_E_ARG;
    }
    // The neighbour below pulls our first row's downward populations into its
    // top row; the neighbour above pulls our last row's upward populations.
    if (to_below) {
        int rc = face_copy(c, false, c->row0, to_below, true);
        if (rc) return rc;
    }
    if (to_above) {
        int rc = face_copy(c, true, c->row0 + c->p.ny - 1, to_above, true);
        if (rc) return rc;
    }
    return DMRT_OK;
}

int dmrt_slab_unpack(dmrt_ctx* c, const void* from_below, const void* from_above) {
    if (!c) return DMRT_E_ARG;
    if (!c->slab) {
        set_err(c, "not a slab context");
        return DMRT_E_ARG;
    }
    if (from_below) {
        int rc = face_copy(c, true, c->row0 - 1, const_cast<void*>(from_below), false);
        if (rc) return rc;
    }
    if (from_above) {
        int rc = face_copy(c, false, c->row0 + c->p.ny, const_cast<void*>(from_above), false);
        if (rc) return rc;
    }
    return DMRT_OK;
}

int dmrt_slab_step(dmrt_ctx* c, void* to_below, void* to_above) {
    if (!c) return DMRT_E_ARG;
    if (!c->slab) {
        set_err(c, "not a slab context");
        return DMRT_E_ARG;
    }
    int rc = launch_one(c);
    if (rc) return rc;
    return dmrt_slab_pack(c, to_below, to_above);
}

int dmrt_check(dmrt_ctx* c) {
    if (!c) return DMRT_E_ARG;
    return poll_error(c);
}

int64_t dmrt_steps_done(const dmrt_ctx* c) { return c ? c->t : -1; }

int dmrt_nusselt_flux(dmrt_ctx* c, double* nu_mean, double* nu_local) {
    if (!c) return DMRT_E_ARG;
    const dmrt_params& p = c->p;
    const bool fixed = p.left_wall == DMRT_WALL_FIXED;
    const double dT = p.theta_hot - p.theta_cold;
    const double scale = dT != 0.0 ? (double)c->H / (c->k.alpha * dT) : 0.0;
    // Per-row values staged in the idle population buffer (no allocation).
    double* stage = reinterpret_cast<double*>(buf(c, 1 - c->cur));
    with_layout(p.storage, [&](auto tag) {
        using Lt = decltype(tag);
        nu_flux_kernel<Lt><<<(p.ny + 255) / 256, 256, 0, c->stream>>>(
            reinterpret_cast<const unsigned char*>(buf(c, c->cur)), reinterpret_cast<const float*>(c->ws + c->L.off_hot),
            stage, p.ny, c->L.pitch, c->L.plane, fixed ? c->k.abb : 0.0, fixed ? 1.0 : 0.0, (double)c->sc.gsh1,
            (4.0 + c->k.a) / 20.0, scale, c->row0);
    });
    CK(cudaGetLastError(), "flux Nusselt kernel");
    std::vector<double> local((size_t)p.ny);
    CK(cudaMemcpyAsync(local.data(), stage, local.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
       "copy flux Nusselt");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    double sum = 0.0;
    for (double x : local) sum += x;  // rows in order
    if (nu_mean) *nu_mean = sum / (double)c->H;  // a slab: its share of the cavity's mean
    if (nu_local) std::memcpy(nu_local, local.data(), local.size() * sizeof(double));
    return DMRT_OK;
}

int dmrt_energy(dmrt_ctx* c, double* theta_sum, double* wall_in) {
    if (!c) return DMRT_E_ARG;
    const dmrt_params& p = c->p;
    const bool lf = p.left_wall == DMRT_WALL_FIXED, rf = p.right_wall == DMRT_WALL_FIXED;
    // Per-row values and the two sums staged in the idle population buffer (no allocation).
    double* rows = reinterpret_cast<double*>(buf(c, 1 - c->cur));
    double* sums = rows + 2 * (size_t)p.ny;
    const int warps = 8;
    with_layout(p.storage, [&](auto tag) {
        using Lt = decltype(tag);
        energy_rows_kernel<Lt><<<(p.ny + warps - 1) / warps, 32 * warps, 0, c->stream>>>(
            reinterpret_cast<const unsigned char*>(buf(c, c->cur)), reinterpret_cast<const float*>(c->ws + c->L.off_hot),
            reinterpret_cast<const float*>(c->ws + c->L.off_cold), rows, rows + p.ny, p.nx, p.ny, c->L.pitch,
            c->L.plane, lf ? c->k.abb : 0.0, lf ? 1.0 : 0.0, rf ? c->k.abb : 0.0, rf ? 1.0 : 0.0,
            (double)c->sc.gsh0, (double)c->sc.gsh1, (4.0 + c->k.a) / 20.0, c->row0);
    });
    sum2_fixed_kernel<<<1, 256, 0, c->stream>>>(rows, rows + p.ny, p.ny, sums);
    CK(cudaGetLastError(), "energy kernels");
    double h[2];
    CK(cudaMemcpyAsync(h, sums, sizeof h, cudaMemcpyDeviceToHost, c->stream), "copy energy");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    if (theta_sum) *theta_sum = h[0];
    if (wall_in) *wall_in = h[1];
    return DMRT_OK;
}

int dmrt_fields(dmrt_ctx* c, float* u, float* v, float* theta, int on_device) {
    if (!c) return DMRT_E_ARG;
    const dmrt_params& p = c->p;
    const long long n = (long long)p.nx * p.ny;
    float *du = u, *dv = v, *dt = theta;
    if (!on_device) {
        // Host outputs: stage in the idle population buffer (no allocation).
        float* stage = buf(c, 1 - c->cur);
        du = u ? stage : nullptr;
        dv = v ? stage + n : nullptr;
        dt = theta ? stage + 2 * n : nullptr;
    }
    const int blocks = (int)std::min<long long>((n + 255) / 256, 152 * 16);
    with_layout(p.storage, [&](auto tag) {
        using Lt = decltype(tag);
        fields_kernel<Lt><<<blocks, 256, 0, c->stream>>>(reinterpret_cast<const unsigned char*>(buf(c, c->cur)),
                                                         du, dv, dt, p.nx, p.ny, c->L.pitch, c->L.plane,
                                                         c->sc.gbeta, c->sc.theta_ref, c->sc.gsh0, c->sc.gsh1,
                                                         c->row0);
    });
    CK(cudaGetLastError(), "fields kernel");
    if (!on_device) {
        if (u) CK(cudaMemcpyAsync(u, du, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream), "copy u");
        if (v) CK(cudaMemcpyAsync(v, dv, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream), "copy v");
        if (theta) CK(cudaMemcpyAsync(theta, dt, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream), "copy theta");
    }
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    return DMRT_OK;
}

int dmrt_nusselt(dmrt_ctx* c, double* nu_mean, double* nu_local, double* series, int64_t cap,
                 int64_t* count) {
    if (!c || (series && cap < 0)) return DMRT_E_ARG;
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    Misc m;
    CK(cudaMemcpy(&m, misc(c), sizeof m, cudaMemcpyDeviceToHost), "read scalars");
    if (nu_mean) *nu_mean = m.nu_last;
    if (nu_local)
        CK(cudaMemcpy(nu_local, last_rows(c), (size_t)c->p.ny * sizeof(double),
                      cudaMemcpyDeviceToHost), "copy local Nu");
    long long written = 0;
    if (series && cap > 0) {
        const long long R = c->p.nu_capacity;
        const long long recorded = m.step[c->cur];
        long long avail = std::min<long long>(recorded - c->nu_floor, R);
        long long want = std::min<long long>(avail, cap);
        long long first = recorded - want;  // step index of the oldest value returned
        const double* ring = reinterpret_cast<const double*>(c->ws + c->L.off_ring);
        long long done = 0;
        while (done < want) {
            long long slot = (first + done) % R;
            long long run = std::min<long long>(want - done, R - slot);
            CK(cudaMemcpy(series + done, ring + slot, run * sizeof(double), cudaMemcpyDeviceToHost),
               "copy Nu series");
            done += run;
        }
        written = want;
    }
    if (count) *count = written;
    if (m.err & dmrt::kErrTimeout) {
        set_err(c, "a bounded device-side wait expired after %lld steps", c->t);
        return DMRT_E_TIMEOUT;
    }
    if (m.err & dmrt::kErrBounds) {
        set_err(c, "an index out of range was seen (bounds-checked build) after %lld steps", c->t);
        return DMRT_E_BOUNDS;
    }
    if (m.err & dmrt::kErrNonFinite) {
        set_err(c, "non-finite density or temperature after %lld steps", c->t);
        return DMRT_E_DIVERGED;
    }
    return DMRT_OK;
}

int dmrt_set_wall_profiles(dmrt_ctx* c, const double* hot, const double* cold) {
    if (!c) return DMRT_E_ARG;
    const int ny = c->p.ny;
    // Stage through the idle buffer, convert to float on the device.
    double* stage = reinterpret_cast<double*>(buf(c, 1 - c->cur));
    if (hot) {
        CK(cudaMemcpyAsync(stage, hot, ny * sizeof(double), cudaMemcpyHostToDevice, c->stream), "copy hot");
        fill_kernel<<<(ny + 255) / 256, 256, 0, c->stream>>>(
            reinterpret_cast<float*>(c->ws + c->L.off_hot), stage, 0.0, ny);
    }
    if (cold) {
        CK(cudaMemcpyAsync(stage + ny, cold, ny * sizeof(double), cudaMemcpyHostToDevice, c->stream), "copy cold");
        fill_kernel<<<(ny + 255) / 256, 256, 0, c->stream>>>(
            reinterpret_cast<float*>(c->ws + c->L.off_cold), stage + ny, 0.0, ny);
    }
    CK(cudaGetLastError(), "profile kernel");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    return DMRT_OK;
}

// Copy between a dense host array [14][ny][nx] of float32 and the padded
// device planes of the current state. A float32 plane: one 2D copy. A 16-bit
// plane: converted through the idle buffer (which holds at least 28 bytes per
// node; a float32 plane needs 4). THETA32: the thermal block converted to and
// from the five population planes as a whole (20 bytes per node).
static float plane_shift(const dmrt_ctx* c, int host_k) {
    return host_k < 9 ? 0.f : (host_k == 9 ? c->sc.gsh0 : c->sc.gsh1);
}

int dmrt_get_state(dmrt_ctx* c, float* host) {
    if (!c || !host) return DMRT_E_ARG;
    const dmrt_params& p = c->p;
    const size_t n = (size_t)p.nx * p.ny;
    float* stage = buf(c, 1 - c->cur);
    const bool theta = p.storage == DMRT_THETA32;
    for (int k = 0; k < (theta ? 9 : kPlanes); ++k) {
        const char* P = reinterpret_cast<const char*>(buf(c, c->cur)) + plane_offset(p, c->L.plane, k) +
                        (size_t)c->row0 * c->L.pitch * plane_elem_bytes(p, k);
        const int st = plane_storage(p, k);
        if (st == DMRT_FP32) {
            CK(cudaMemcpy2DAsync(host + (size_t)k * n, (size_t)p.nx * sizeof(float), P,
                                 (size_t)c->L.pitch * sizeof(float), (size_t)p.nx * sizeof(float), p.ny,
                                 cudaMemcpyDeviceToHost, c->stream),
               "copy state to host");
            continue;
        }
        with_elem(st, [&](auto tag) {
            using E = decltype(tag);
            plane_to_f32<E><<<1024, 256, 0, c->stream>>>(reinterpret_cast<const E*>(P), stage, p.nx, p.ny,
                                                         c->L.pitch, plane_shift(c, k));
        });
        CK(cudaGetLastError(), "state conversion");
        CK(cudaMemcpyAsync(host + (size_t)k * n, stage, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream),
           "copy state to host");
    }
    if (theta) {
        // The idle buffer holds 30 bytes per node: room for 5 float32 planes.
        theta_to_g32<<<1024, 256, 0, c->stream>>>(reinterpret_cast<const unsigned char*>(buf(c, c->cur)),
                                                  c->L.plane, c->L.pitch, p.nx, p.ny, c->row0, c->sc.w0,
                                                  c->sc.w1, stage);
        CK(cudaGetLastError(), "state conversion");
        CK(cudaMemcpyAsync(host + (size_t)9 * n, stage, 5 * n * sizeof(float), cudaMemcpyDeviceToHost, c->stream),
           "copy state to host");
    }
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    return DMRT_OK;
}

int dmrt_set_state(dmrt_ctx* c, const float* host) {
    if (!c || !host) return DMRT_E_ARG;
    const dmrt_params& p = c->p;
    const size_t n = (size_t)p.nx * p.ny;
    float* stage = buf(c, 1 - c->cur);
    const bool theta = p.storage == DMRT_THETA32;
    for (int k = 0; k < (theta ? 9 : kPlanes); ++k) {
        char* P = reinterpret_cast<char*>(buf(c, c->cur)) + plane_offset(p, c->L.plane, k) +
                  (size_t)c->row0 * c->L.pitch * plane_elem_bytes(p, k);
        const int st = plane_storage(p, k);
        if (st == DMRT_FP32) {
            CK(cudaMemcpy2DAsync(P, (size_t)c->L.pitch * sizeof(float), host + (size_t)k * n,
                                 (size_t)p.nx * sizeof(float), (size_t)p.nx * sizeof(float), p.ny,
                                 cudaMemcpyHostToDevice, c->stream),
               "copy state to device");
            continue;
        }
        CK(cudaMemcpyAsync(stage, host + (size_t)k * n, n * sizeof(float), cudaMemcpyHostToDevice, c->stream),
           "copy state to device");
        with_elem(st, [&](auto tag) {
            using E = decltype(tag);
            plane_from_f32<E><<<1024, 256, 0, c->stream>>>(reinterpret_cast<E*>(P), stage, p.nx, p.ny,
                                                           c->L.pitch, plane_shift(c, k));
        });
        CK(cudaGetLastError(), "state conversion");
    }
    if (theta) {
        CK(cudaMemcpyAsync(stage, host + (size_t)9 * n, 5 * n * sizeof(float), cudaMemcpyHostToDevice, c->stream),
           "copy state to device");
        theta_from_g32<<<1024, 256, 0, c->stream>>>(reinterpret_cast<unsigned char*>(buf(c, c->cur)), c->L.plane,
                                                    c->L.pitch, p.nx, p.ny, c->row0, c->sc.w1, stage);
        CK(cudaGetLastError(), "state conversion");
    }
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    return DMRT_OK;
}

// ---- checkpoint and resume ----------------------------------------------------
namespace {

constexpr char kCkptMagic[8] = {'D', 'M', 'R', 'T', 'C', 'K', 'P', '1'};
constexpr uint32_t kCkptVersion = 1;

struct CkptHeader {
    char magic[8];
    uint32_t version;
    uint32_t header_bytes;
    int32_t nx, ny, storage, rounding;
    int32_t left_wall, right_wall;
    double Ra, Pr, alpha, theta_hot, theta_cold, theta_ref;
    int64_t t;          // steps taken
    int64_t recorded;   // device step counter of the current buffer
    int64_t n_series;   // most recent mean-Nu values saved
    double nu_last;
    uint32_t err;
    uint32_t reserved;
    uint64_t state_bytes;
};

// 64-bit FNV-1a (Fowler, Noll, Vo).
uint64_t fnv1a64(const unsigned char* p, size_t n) {
    uint64_t h = 14695981039346656037ull;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}


size_t ckpt_state_bytes(const dmrt_params& p) {
    size_t s = 0;
    for (int k = 0; k < kPlanes; ++k) s += plane_elem_bytes(p, k) * (size_t)p.nx * p.ny;
    return s;
}

size_t ckpt_bytes(const dmrt_params& p, int64_t n_series) {
    return sizeof(CkptHeader) + 2 * (size_t)p.ny * sizeof(float) + (size_t)p.ny * sizeof(double) +
           (size_t)n_series * sizeof(double) + ckpt_state_bytes(p) + sizeof(uint64_t);
}

}  // namespace

int dmrt_save(dmrt_ctx* c, void* host_buf, size_t cap, size_t* used) {
    if (!c || !used) return DMRT_E_ARG;
    const dmrt_params& p = c->p;
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    Misc m;
    CK(cudaMemcpy(&m, misc(c), sizeof m, cudaMemcpyDeviceToHost), "read scalars");
    const long long recorded = m.step[c->cur];
    const long long n_series = std::min<long long>(recorded - c->nu_floor, p.nu_capacity);
    const size_t need = ckpt_bytes(p, n_series);
    *used = need;
    if (!host_buf) return DMRT_OK;
    if (cap < need) {
        set_err(c, "checkpoint needs %zu bytes, buffer has %zu", need, cap);
        return DMRT_E_SPACE;
    }
    unsigned char* base = static_cast<unsigned char*>(host_buf);
    unsigned char* o = base;
    CkptHeader h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, kCkptMagic, 8);
    h.version = kCkptVersion;
    h.header_bytes = sizeof h;
    h.nx = p.nx;
    h.ny = p.ny;
    h.storage = p.storage;
    h.rounding = p.rounding;
    h.left_wall = p.left_wall;
    h.right_wall = p.right_wall;
    h.Ra = p.Ra;
    h.Pr = p.Pr;
    h.alpha = c->k.alpha;
    h.theta_hot = p.theta_hot;
    h.theta_cold = p.theta_cold;
    h.theta_ref = p.theta_ref;
    h.t = c->t;
    h.recorded = recorded;
    h.n_series = n_series;
    h.nu_last = m.nu_last;
    h.err = m.err;
    h.state_bytes = ckpt_state_bytes(p);
    std::memcpy(o, &h, sizeof h);
    o += sizeof h;
    const size_t ny = (size_t)p.ny, nx = (size_t)p.nx;
    CK(cudaMemcpy(o, c->ws + c->L.off_hot, ny * sizeof(float), cudaMemcpyDeviceToHost), "copy hot wall");
    o += ny * sizeof(float);
    CK(cudaMemcpy(o, c->ws + c->L.off_cold, ny * sizeof(float), cudaMemcpyDeviceToHost), "copy cold wall");
    o += ny * sizeof(float);
    CK(cudaMemcpy(o, last_rows(c), ny * sizeof(double), cudaMemcpyDeviceToHost), "copy local Nu");
    o += ny * sizeof(double);
    // Mean Nu of steps recorded - n_series .. recorded - 1, oldest first (ring slot = step % capacity).
    const double* ring = reinterpret_cast<const double*>(c->ws + c->L.off_ring);
    const long long R = p.nu_capacity;
    for (long long done = 0; done < n_series;) {
        const long long slot = (recorded - n_series + done) % R;
        const long long run = std::min<long long>(n_series - done, R - slot);
        CK(cudaMemcpy(o + done * sizeof(double), ring + slot, run * sizeof(double), cudaMemcpyDeviceToHost),
           "copy Nu series");
        done += run;
    }
    o += n_series * sizeof(double);
    // Population planes in host order (f_1..f_9, g_1..g_5), stored representation, x < nx.
    for (int k = 0; k < kPlanes; ++k) {
        const size_t eb = plane_elem_bytes(p, k);
        const char* P = reinterpret_cast<const char*>(buf(c, c->cur)) + plane_offset(p, c->L.plane, k) +
                        (size_t)c->row0 * c->L.pitch * eb;
        CK(cudaMemcpy2D(o, nx * eb, P, (size_t)c->L.pitch * eb, nx * eb, ny, cudaMemcpyDeviceToHost),
           "copy state plane");
        o += nx * ny * eb;
    }
    const uint64_t sum = fnv1a64(base, (size_t)(o - base));
    std::memcpy(o, &sum, sizeof sum);
    return DMRT_OK;
}

int dmrt_load(dmrt_ctx* c, const void* host_buf, size_t size) {
    if (!c || !host_buf || size < sizeof(CkptHeader) + sizeof(uint64_t)) {
        if (c) set_err(c, "checkpoint buffer missing or shorter than its header");
        return DMRT_E_ARG;
    }
    const dmrt_params& p = c->p;
    const unsigned char* base = static_cast<const unsigned char*>(host_buf);
    CkptHeader h;
    std::memcpy(&h, base, sizeof h);
    if (std::memcmp(h.magic, kCkptMagic, 8) != 0 || h.version != kCkptVersion || h.header_bytes != sizeof h) {
        set_err(c, "not a checkpoint of this format (magic / version)");
        return DMRT_E_STATE;
    }
    if (h.nx != p.nx || h.ny != p.ny || h.storage != p.storage) {
        set_err(c, "checkpoint of a %d x %d grid with storage %d; this context is %d x %d with storage %d", h.nx,
                h.ny, h.storage, p.nx, p.ny, p.storage);
        return DMRT_E_STATE;
    }
    if (h.recorded < 0 || h.n_series < 0 || h.n_series > h.recorded || h.t < 0 ||
        h.state_bytes != ckpt_state_bytes(p)) {
        set_err(c, "inconsistent checkpoint header");
        return DMRT_E_STATE;
    }
    const size_t need = ckpt_bytes(p, h.n_series);
    if (size < need) {
        set_err(c, "checkpoint truncated: %zu bytes of %zu", size, need);
        return DMRT_E_ARG;
    }
    uint64_t sum;
    std::memcpy(&sum, base + need - sizeof sum, sizeof sum);
    if (sum != fnv1a64(base, need - sizeof sum)) {
        set_err(c, "checkpoint checksum mismatch");
        return DMRT_E_STATE;
    }
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    const unsigned char* o = base + sizeof h;
    const size_t ny = (size_t)p.ny, nx = (size_t)p.nx;
    CK(cudaMemcpy(c->ws + c->L.off_hot, o, ny * sizeof(float), cudaMemcpyHostToDevice), "copy hot wall");
    o += ny * sizeof(float);
    CK(cudaMemcpy(c->ws + c->L.off_cold, o, ny * sizeof(float), cudaMemcpyHostToDevice), "copy cold wall");
    o += ny * sizeof(float);
    CK(cudaMemcpy(last_rows(c), o, ny * sizeof(double), cudaMemcpyHostToDevice), "copy local Nu");
    o += ny * sizeof(double);
    // Keep the last min(n_series, capacity) values, each in its step's ring slot.
    double* ring = reinterpret_cast<double*>(c->ws + c->L.off_ring);
    const long long R = p.nu_capacity;
    const long long keep = std::min<long long>(h.n_series, R);
    const unsigned char* series = o + (h.n_series - keep) * sizeof(double);
    for (long long done = 0; done < keep;) {
        const long long slot = (h.recorded - keep + done) % R;
        const long long run = std::min<long long>(keep - done, R - slot);
        CK(cudaMemcpy(ring + slot, series + done * sizeof(double), run * sizeof(double), cudaMemcpyHostToDevice),
           "copy Nu series");
        done += run;
    }
    o += h.n_series * sizeof(double);
    for (int k = 0; k < kPlanes; ++k) {
        const size_t eb = plane_elem_bytes(p, k);
        char* P = reinterpret_cast<char*>(buf(c, c->cur)) + plane_offset(p, c->L.plane, k) +
                  (size_t)c->row0 * c->L.pitch * eb;
        CK(cudaMemcpy2D(P, (size_t)c->L.pitch * eb, o, nx * eb, nx * eb, ny, cudaMemcpyHostToDevice),
           "copy state plane");
        o += nx * ny * eb;
    }
    Misc m;
    std::memset(&m, 0, sizeof m);
    m.step[0] = m.step[1] = h.recorded;
    m.nu_last = h.nu_last;
    m.pending = 0u;
    m.err = h.err;
    CK(cudaMemcpy(misc(c), &m, sizeof m, cudaMemcpyHostToDevice), "write scalars");
    c->t = h.t;
    c->next_poll = h.t + kPollSteps;
    c->nu_floor = h.recorded - keep;
    return DMRT_OK;
}

int dmrt_get_launch(const dmrt_ctx* c, dmrt_launch* out) {
    if (!c || !out) return DMRT_E_ARG;
    if (c->cluster) {
        out->kernel = DMRT_KERNEL_CLUSTER;
        out->tma_npt = out->tma_rows = out->tma_stages = 0;
        out->grid = c->csize;
        out->block = c->cthreads;
        out->smem_bytes = (int64_t)c->csmem;
        out->graph_steps = 0;
        return DMRT_OK;
    }
    out->kernel = c->kernel;
    if (c->kernel == DMRT_KERNEL_TMA) {
        out->tma_npt = c->npt;
        out->tma_rows = c->R;
        out->tma_stages = c->S;
        out->grid = c->tma_grid;
        out->block = c->tma_block;
        out->smem_bytes = (int64_t)c->tma_smem;
    } else {
        out->tma_npt = out->tma_rows = out->tma_stages = 0;
        out->grid = (int32_t)(c->grid.x * c->grid.y);
        out->block = dmrt::kDirectThreads;
        out->smem_bytes = 0;
    }
    out->graph_steps = c->graph_len;
    return DMRT_OK;
}

int dmrt_get_consts(const dmrt_ctx* c, dmrt_consts* out) {
    if (!c || !out) return DMRT_E_ARG;
    *out = c->k;
    return DMRT_OK;
}

const char* dmrt_last_error(const dmrt_ctx* c) { return c ? c->err : g_create_error; }

void dmrt_destroy(dmrt_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    for (int i = 0; i < 2; ++i)
        if (c->graph[i]) cudaGraphExecDestroy(c->graph[i]);
    if (c->aux) {
        cudaStreamSynchronize(c->aux);
        for (cudaEvent_t e : c->ev)
            if (e) cudaEventDestroy(e);
        cudaStreamDestroy(c->aux);
    }
    delete c;
}

}  // extern "C"

// ---- batched sweep ------------------------------------------------------------

// Cavities [first, first + count) of a batch, stepped by launches of their own.
// One group (all cavities) streams the whole batch through HBM on every step;
// smaller groups, each run for all the steps of a call before the next one,
// keep their state resident in L2 between steps.
struct BatchGroup {
    int first, count;
    int total_items;
    int static_per_block;  // items each block takes before drawing from the shared pool
    int grid;
    int* d_ib;             // first item of each of its cavities, then the total (count + 1 entries)
    unsigned* d_ctr;       // its two work-pool counters (by launch parity)
    unsigned* d_sync;      // multi-step launches: two sets of (queue counter, done[], ready[])
    int mgrid;             // blocks of a multi-step launch
    cudaGraphExec_t graph[2];
};

struct dmrt_batch {
    int n;
    std::vector<dmrt_ctx*> sub;
    char* ws;
    cudaStream_t stream;
    dmrt::BatchCavity* d_cav;
    CUtensorMap* d_maps;
    unsigned* d_err;
    std::vector<BatchGroup> groups;
    long long group_bytes;
    int npt, R, S, block;
    size_t smem;
    const void* func;
    int K;                 // steps per launch (1: one launch per step; else the multi-step kernel)
    const void* mfunc;     // the multi-step kernel (K > 1)
    int parity;
    long long t;
    int graph_len;
    char err[256];
};

namespace {

struct BatchLayout {
    std::vector<size_t> off, bytes;
    size_t off_cav, off_maps, off_ib, off_err, off_sync, total;
};

int batch_layout(const dmrt_params* arr, int32_t n, BatchLayout* L) {
    if (!arr || n < 1 || n > 65536) {
        set_err(nullptr, "batch needs 1 <= n <= 65536 cavities");
        return DMRT_E_ARG;
    }
    L->off.resize(n);
    L->bytes.resize(n);
    size_t o = 0;
    for (int i = 0; i < n; ++i) {
        int rc = validate(&arr[i], nullptr);
        if (rc) return rc;
        if (arr[i].storage != DMRT_FP32 && arr[i].storage != DMRT_MIXED) {
            set_err(nullptr, "batched sweep: cavity %d: float32 or mixed storage only", i);
            return DMRT_E_ARG;
        }
        if (arr[i].storage != arr[0].storage) {
            set_err(nullptr, "batched sweep: cavity %d: every cavity needs the same storage", i);
            return DMRT_E_ARG;
        }
        if (resolved_rounding(arr[i]) != resolved_rounding(arr[0])) {
            set_err(nullptr, "batched sweep: cavity %d: every cavity needs the same rounding", i);
            return DMRT_E_ARG;
        }
        L->off[i] = o;
        L->bytes[i] = make_layout(arr[i]).total;
        o += align256(L->bytes[i]);
    }
    L->off_cav = o;
    o += align256((size_t)n * sizeof(dmrt::BatchCavity));
    L->off_maps = o;
    o += align256((size_t)n * 2 * dmrt::kBatchMaps * sizeof(CUtensorMap));
    L->off_ib = o;  // item tables of at most n groups: n + groups entries
    o += align256((size_t)(2 * n) * sizeof(int));
    L->off_err = o;  // the error word, then two pool counters per group
    o += align256(sizeof(unsigned) * (size_t)(1 + 2 * n));
    L->off_sync = o;  // multi-step launches: two synchronisation sets per group (at most n groups)
    o += align256(sizeof(unsigned) * (size_t)(2 * (dmrt::mstep_set_words(0) + 2) * n));
    L->total = o;
    return DMRT_OK;
}

void batch_set_err(dmrt_batch* b, const char* fmt, ...) {
    char* dst = b ? b->err : g_create_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 256, fmt, ap);
    va_end(ap);
}

int batch_cuda_fail(dmrt_batch* b, cudaError_t e, const char* what) {
    batch_set_err(b, "%s: %s", what, cudaGetErrorString(e));
    return DMRT_E_CUDA;
}

#define BCK(call, what)                                              \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return batch_cuda_fail(b, e_, what);  \
    } while (0)

// The kernel arguments of group g's launches (parity points at the launch's parity).
struct GroupArgs {
    const dmrt::BatchCavity* cav;
    const CUtensorMap* maps;
    const int* ib;
    int n_cav, total, per_block;
    unsigned *err, *ctr;
    GroupArgs(const dmrt_batch* b, const BatchGroup& G)
        : cav(b->d_cav + G.first), maps(b->d_maps + (size_t)G.first * 2 * dmrt::kBatchMaps), ib(G.d_ib),
          n_cav(G.count), total(G.total_items), per_block(G.static_per_block), err(b->d_err), ctr(G.d_ctr) {}
    void fill(void** p, int* parity) {
        p[0] = &cav, p[1] = &maps, p[2] = &ib, p[3] = &n_cav, p[4] = &total, p[5] = &per_block;
        p[6] = parity, p[7] = &err, p[8] = &ctr;
    }
};

int batch_launch(dmrt_batch* b, const BatchGroup& G, int parity) {
    GroupArgs a(b, G);
    void* params[9];
    a.fill(params, &parity);
    BCK(cudaLaunchKernel(b->func, dim3(G.grid), dim3(b->block), params, b->smem, b->stream),
        "batch step launch");
    return DMRT_OK;
}

// Arguments of a multi-step launch of group G (K steps from buffer `parity`,
// synchronisation set lp).
struct MstepArgs {
    const dmrt::BatchCavity* cav;
    const CUtensorMap* maps;
    const int* ib;
    int n_cav, per_step, K, parity;
    unsigned *err, *sync;
    int lp;
    MstepArgs(const dmrt_batch* b, const BatchGroup& G, int parity_, int lp_)
        : cav(b->d_cav + G.first), maps(b->d_maps + (size_t)G.first * 2 * dmrt::kBatchMaps), ib(G.d_ib),
          n_cav(G.count), per_step(G.total_items), K(b->K), parity(parity_), err(b->d_err), sync(G.d_sync),
          lp(lp_) {}
    void fill(void** p) {
        p[0] = &cav, p[1] = &maps, p[2] = &ib, p[3] = &n_cav, p[4] = &per_step, p[5] = &K, p[6] = &parity;
        p[7] = &err, p[8] = &sync, p[9] = &lp;
    }
};

// Graph of two multi-step launches (synchronisation sets 0 then 1), 2 K steps
// from buffer `from` (K even: each launch ends in the buffer it started from).
int batch_build_mstep_graph(dmrt_batch* b, BatchGroup& G, int from) {
    cudaGraph_t g;
    BCK(cudaGraphCreate(&g, 0), "cudaGraphCreate");
    cudaGraphNode_t prev = nullptr;
    MstepArgs a[2] = {MstepArgs(b, G, from, 0), MstepArgs(b, G, from, 1)};
    for (int i = 0; i < 2; ++i) {
        cudaKernelNodeParams kp = {};
        void* params[10];
        a[i].fill(params);
        kp.func = const_cast<void*>(b->mfunc);
        kp.gridDim = dim3(G.mgrid);
        kp.blockDim = dim3(b->block);
        kp.sharedMemBytes = (unsigned)b->smem;
        kp.kernelParams = params;
        cudaGraphNode_t node;
        cudaError_t e = add_step_node(g, prev, &kp, &node);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            return batch_cuda_fail(b, e, "cudaGraphAddKernelNode");
        }
        prev = node;
    }
    cudaError_t e = cudaGraphInstantiate(&G.graph[from], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return batch_cuda_fail(b, e, "cudaGraphInstantiate");
    return DMRT_OK;
}

int batch_build_graph(dmrt_batch* b, BatchGroup& G, int from) {
    if (b->K > 1) return batch_build_mstep_graph(b, G, from);
    cudaGraph_t g;
    BCK(cudaGraphCreate(&g, 0), "cudaGraphCreate");
    cudaGraphNode_t prev = nullptr;
    int par[2] = {from, 1 - from};
    GroupArgs a(b, G);
    for (int i = 0; i < b->graph_len; ++i) {
        cudaKernelNodeParams kp = {};
        void* params[9];
        a.fill(params, &par[i & 1]);
        kp.func = const_cast<void*>(b->func);
        kp.gridDim = dim3(G.grid);
        kp.blockDim = dim3(b->block);
        kp.sharedMemBytes = (unsigned)b->smem;
        kp.kernelParams = params;
        cudaGraphNode_t node;
        cudaError_t e = add_step_node(g, prev, &kp, &node);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            return batch_cuda_fail(b, e, "cudaGraphAddKernelNode");
        }
        prev = node;
    }
    cudaError_t e = cudaGraphInstantiate(&G.graph[from], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return batch_cuda_fail(b, e, "cudaGraphInstantiate");
    return DMRT_OK;
}

}  // namespace

extern "C" {

int dmrt_batch_workspace_size(const dmrt_params* arr, int32_t n, size_t* bytes) {
    BatchLayout L;
    int rc = batch_layout(arr, n, &L);
    if (rc) return rc;
    if (!bytes) return DMRT_E_ARG;
    *bytes = L.total;
    return DMRT_OK;
}

int dmrt_batch_create(const dmrt_params* arr, int32_t n, const double* const* theta0,
                      const dmrt_batch_opts* opts, void* workspace, size_t workspace_bytes,
                      void* stream, dmrt_batch** out) {
    if (!out) {
        set_err(nullptr, "out is NULL");
        return DMRT_E_ARG;
    }
    *out = nullptr;
    BatchLayout L;
    int rc = batch_layout(arr, n, &L);
    if (rc) return rc;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255)) {
        set_err(nullptr, "workspace must be a 256-byte aligned device pointer");
        return DMRT_E_ARG;
    }
    if (workspace_bytes < L.total) {
        set_err(nullptr, "workspace too small: %zu < %zu bytes", workspace_bytes, L.total);
        return DMRT_E_SPACE;
    }
    const bool mixed_def = arr[0].storage == DMRT_MIXED;
    const int npt = opts && opts->tma_npt > 0 ? opts->tma_npt : (mixed_def ? 4 : 2);
    const int R = opts && opts->tma_rows > 0 ? opts->tma_rows : 2;
    const int S = opts && opts->tma_stages > 0 ? opts->tma_stages : 2;
    const int K = opts && opts->steps_per_launch > 1 ? opts->steps_per_launch : 1;
    if (K > 1 && K % 2) {
        set_err(nullptr, "steps_per_launch must be even");
        return DMRT_E_ARG;
    }
    const int glen = K > 1 ? 2 * K : (opts && opts->graph_steps > 0 ? opts->graph_steps : 64);
    if (glen % 2) {
        set_err(nullptr, "graph_steps must be even");
        return DMRT_E_ARG;
    }
    int nv = 0;
    const dmrt::TmaVariant* vars = dmrt::tma_variants_batch(&nv);
    const void* func = nullptr;
    const int storage = arr[0].storage;
    // Epilogue: register stores, or tensor stores through shared memory.
    const bool ts = opts && opts->tensor_store > 0;
    for (int i = 0; i < nv; ++i)
        if (vars[i].storage == storage && vars[i].rounding == resolved_rounding(arr[0]) && vars[i].npt == npt &&
            vars[i].R == R && vars[i].S == S && (vars[i].ts != 0) == ts)
            func = vars[i].func;
    if (!func) {
        set_err(nullptr, "no batched tile with %d nodes/thread, %d rows, %d stages%s is compiled in for this storage",
                npt, R, S, ts ? " and tensor stores" : "");
        return DMRT_E_ARG;
    }
    if (ts && K > 1) {
        set_err(nullptr, "the multi-step batched kernel stores from registers (tensor_store must be 0)");
        return DMRT_E_ARG;
    }
    const void* mfunc = nullptr;
    if (K > 1) {
        int nm = 0;
        const dmrt::TmaVariant* mv = dmrt::tma_variants_batch_mstep(&nm);
        for (int i = 0; i < nm; ++i)
            if (mv[i].storage == storage && mv[i].rounding == resolved_rounding(arr[0]) && mv[i].npt == npt &&
                mv[i].R == R && mv[i].S == S)
                mfunc = mv[i].func;
        if (!mfunc) {
            set_err(nullptr, "no multi-step batched tile with %d nodes/thread, %d rows, %d stages is compiled in "
                             "for this storage", npt, R, S);
            return DMRT_E_ARG;
        }
    }
    dmrt_batch* b = new (std::nothrow) dmrt_batch();
    if (!b) {
        set_err(nullptr, "out of host memory");
        return DMRT_E_SPACE;
    }
    b->n = n;
    b->ws = static_cast<char*>(workspace);
    b->stream = static_cast<cudaStream_t>(stream);
    b->npt = npt;
    b->R = R;
    b->S = S;
    b->func = func;
    b->parity = 0;
    b->t = 0;
    b->graph_len = glen;
    b->K = K;
    b->mfunc = mfunc;
    b->err[0] = 0;
    auto fail = [&](int code) {
        std::snprintf(g_create_error, sizeof g_create_error, "%s", b->err[0] ? b->err : g_create_error);
        for (dmrt_ctx* c : b->sub) dmrt_destroy(c);
        delete b;
        return code;
    };
    // Members: ordinary contexts on slices of the workspace.
    for (int i = 0; i < n; ++i) {
        dmrt_ctx* c = nullptr;
        rc = dmrt_create(&arr[i], theta0 ? theta0[i] : nullptr, b->ws + L.off[i], L.bytes[i], stream, &c);
        if (rc) {
            char msg[256];
            std::snprintf(msg, sizeof msg, "cavity %d: %.200s", i, g_create_error);
            std::snprintf(b->err, sizeof b->err, "%s", msg);
            return fail(rc);
        }
        b->sub.push_back(c);
    }
    // Device tables: per-cavity arguments and tensor maps (boxes of R rows).
    std::vector<dmrt::BatchCavity> cav(n);
    std::vector<CUtensorMap> maps((size_t)n * 2 * dmrt::kBatchMaps);
    std::memset(maps.data(), 0, maps.size() * sizeof(maps[0]));
    long long items = 0;
    const bool split = storage == DMRT_MIXED;
    const int fb = split ? 2 : 4, gb = 4;               // bytes per flow / thermal element
    const int halo = dmrt::tma_halo(std::min(fb, gb));  // 16 bytes of the narrowest element
    const int block = R * (256 / npt);
    const int quantum = 32 * npt;                       // strip widths keep warps in one row
    const int w_max = (dmrt::kTmaBox - 2 * halo) / quantum * quantum;
    const int stage_bytes = (int)dmrt::batch_stage_bytes(R, fb, gb);  // the compiled stage
    const bool fill = opts && opts->strip_fill > 0;
    for (int i = 0; i < n; ++i) {
        dmrt_ctx* c = b->sub[i];
        std::memset(&cav[i], 0, sizeof cav[i]);
        cav[i].args[0] = step_args(c, 0);
        cav[i].args[1] = step_args(c, 1);
        cav[i].K = c->sc;
        // Rows per item and stage placement of a strip W nodes wide (the same
        // function the kernel specialises its items on).
        auto geo = [&](int w) { return dmrt::batch_geometry(split, npt, R, w, stage_bytes); };
        // Strip width. Default: the widest strips (fewest halo columns), the
        // cavity's width split evenly. strip_fill: the width, among multiples of
        // the quantum, whose items keep the most of the block's threads busy
        // (rows x threads per row against the block, times the valid share of
        // the strips' nodes); ties go to the wider strip.
        int W;
        if (fill) {
            W = quantum;
            double best = -1.0;
            for (int w = quantum; w <= w_max; w += quantum) {
                const int rc = geo(w).RC;
                const long long ns_w = (c->p.nx + w - 1) / w;
                const double use = (double)rc * (w / npt) / block * c->p.nx / ((double)ns_w * w);
                if (use > best + 1e-12 || (use > best - 1e-12 && w > W)) {
                    best = use;
                    W = w;
                }
            }
        } else {
            const int ns = (c->p.nx + w_max - 1) / w_max;
            W = ((c->p.nx + ns - 1) / ns + quantum - 1) / quantum * quantum;
        }
        const int tpr = W / npt;
        const dmrt::BatchGeo G = geo(W);
        const int RC = G.RC;
        const int WB = W + 2 * halo;
        dmrt::StageOffsets so = G.so;
        dmrt::StageOffsets so_check{};
        if (dmrt::batch_place(split, RC, WB, so_check) > stage_bytes) {
            std::snprintf(b->err, sizeof b->err, "cavity %d: strip of %d nodes does not fit the stage", i, W);
            return fail(DMRT_E_ARG);
        }
        cav[i].so = so;
        cav[i].n_strips = (c->p.nx + W - 1) / W;
        cav[i].n_rowblocks = (c->p.ny + RC - 1) / RC;
        cav[i].item_base = (int)items;
        cav[i].W = W;
        cav[i].WB = WB;
        cav[i].RC = RC;
        cav[i].tpr = tpr;
        cav[i].tpr_magic = (unsigned)((0x100000000ull + (unsigned)tpr - 1) / (unsigned)tpr);
        cav[i].stage_bytes = (unsigned)((size_t)RC * WB * (9 * fb + 5 * gb));
        items += (long long)cav[i].n_strips * cav[i].n_rowblocks;
        for (int bf = 0; bf < 2; ++bf) {
            CUtensorMap* m = &maps[((size_t)i * 2 + bf) * dmrt::kBatchMaps];
            // Loads from buffer bf; the epilogue's stores (W x RC boxes, nx columns) to the other one.
            float* dst = buf(c, 1 - bf);
            const int sm = dmrt::kBatchStoreMap;
            if (split) {  // 9 float16 flow planes, then 5 float32 thermal planes
                char* g = reinterpret_cast<char*>(buf(c, bf)) + (size_t)9 * c->L.plane * 2;
                char* gd = reinterpret_cast<char*>(dst) + (size_t)9 * c->L.plane * 2;
                rc = encode_map(c, &m[0], buf(c, bf), DMRT_FP16, 9, 3, RC, WB);
                if (!rc) rc = encode_map(c, &m[1], g, DMRT_FP32, 5, 3, RC, WB);
                if (!rc) rc = encode_map(c, &m[2], g, DMRT_FP32, 5, 1, RC, WB);
                if (!rc) rc = encode_map(c, &m[sm], dst, DMRT_FP16, 9, 9, RC, W, c->p.nx);
                if (!rc) rc = encode_map(c, &m[sm + 1], gd, DMRT_FP32, 5, 5, RC, W, c->p.nx);
            } else {
                rc = encode_map(c, &m[0], buf(c, bf), DMRT_FP32, kPlanes, 6, RC, WB);
                if (!rc) rc = encode_map(c, &m[1], buf(c, bf), DMRT_FP32, kPlanes, 4, RC, WB);
                if (!rc) rc = encode_map(c, &m[sm], dst, DMRT_FP32, kPlanes, kPlanes, RC, W, c->p.nx);
            }
            if (rc) {
                std::snprintf(b->err, sizeof b->err, "cavity %d: %.200s", i, c->err);
                return fail(rc);
            }
        }
    }
    if (items > 0x7fffffff) {
        batch_set_err(b, "batch has too many work items");
        return fail(DMRT_E_ARG);
    }
    // Groups: consecutive cavities whose two population buffers together take
    // at most group_bytes (a larger cavity forms a group of its own); 0: one
    // group of all cavities. Each group numbers its own items from 0.
    b->group_bytes = opts && opts->group_bytes > 0 ? opts->group_bytes : 0;
    b->d_cav = reinterpret_cast<dmrt::BatchCavity*>(b->ws + L.off_cav);
    b->d_maps = reinterpret_cast<CUtensorMap*>(b->ws + L.off_maps);
    b->d_err = reinterpret_cast<unsigned*>(b->ws + L.off_err);
    int* d_ib_all = reinterpret_cast<int*>(b->ws + L.off_ib);
    unsigned* d_sync_all = reinterpret_cast<unsigned*>(b->ws + L.off_sync);
    size_t sync_words = 0;
    std::vector<int> ib;
    {
        long long acc = 0;
        for (int i = 0; i < n; ++i) {
            const long long bytes = 2LL * (long long)b->sub[i]->L.buf_bytes;
            if (b->groups.empty() || (b->group_bytes > 0 && acc > 0 && acc + bytes > b->group_bytes)) {
                BatchGroup G{};
                G.first = i;
                b->groups.push_back(G);
                acc = 0;
            }
            b->groups.back().count += 1;
            acc += bytes;
        }
        for (size_t g = 0; g < b->groups.size(); ++g) {
            BatchGroup& G = b->groups[g];
            G.d_ib = d_ib_all + ib.size();
            G.d_ctr = b->d_err + 1 + 2 * g;
            G.d_sync = d_sync_all + sync_words;
            sync_words += 2 * (size_t)dmrt::mstep_set_words(G.count);
            int it = 0;
            for (int i = G.first; i < G.first + G.count; ++i) {
                cav[i].item_base = it;
                ib.push_back(it);
                it += cav[i].n_strips * cav[i].n_rowblocks;
            }
            ib.push_back(it);
            G.total_items = it;
        }
    }
    cudaError_t e = cudaMemcpyAsync(b->d_cav, cav.data(), cav.size() * sizeof(cav[0]), cudaMemcpyHostToDevice,
                                    b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_maps, maps.data(), maps.size() * sizeof(maps[0]), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_ib_all, ib.data(), ib.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, sizeof(unsigned) * (1 + 2 * b->groups.size()), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_sync_all, 0, sizeof(unsigned) * sync_words, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return fail(batch_cuda_fail(b, e, "batch tables"));
    // Launch shape: persistent grid of resident blocks.
    b->block = R * (256 / npt);
    b->smem = dmrt::batch_smem_bytes(ts, R, S, split ? 2 : 4, 4);
    int dev = 0, sms = 0, per_sm = 0;
    e = cudaFuncSetAttribute(b->func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, b->func, b->block, b->smem);
    if (e != cudaSuccess) return fail(batch_cuda_fail(b, e, "batch launch shape"));
    if (per_sm < 1) {
        batch_set_err(b, "batched tile does not fit on an SM");
        return fail(DMRT_E_ARG);
    }
    int mper_sm = 0;
    if (K > 1) {
        e = cudaFuncSetAttribute(b->mfunc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&mper_sm, b->mfunc, b->block, b->smem);
        if (e != cudaSuccess) return fail(batch_cuda_fail(b, e, "multi-step launch shape"));
        if (mper_sm < 1) {
            batch_set_err(b, "multi-step batched tile does not fit on an SM");
            return fail(DMRT_E_ARG);
        }
    }
    for (BatchGroup& G : b->groups) {
        // Multi-step launches: every block resident; each takes items from the queue.
        G.mgrid = (int)std::min<long long>((long long)G.total_items * K, (long long)sms * std::max(mper_sm, 1));
        G.grid = (int)std::min<long long>(G.total_items, (long long)sms * per_sm);
        // Three quarters of the items are split statically, the rest are drawn at run time.
        G.static_per_block = (int)((long long)G.total_items * 3 / 4 / G.grid);
    }
    *out = b;
    return DMRT_OK;
}

int dmrt_batch_step(dmrt_batch* b, int64_t nsteps) {
    if (!b || nsteps < 0) return DMRT_E_ARG;
    for (int i = 0; i < b->n; ++i) {
        if (b->sub[i]->cur != b->parity) {
            batch_set_err(b, "cavity %d was stepped on its own by an odd number of steps since the last "
                             "batch step; step it once more first", i);
            return DMRT_E_STATE;
        }
    }
    // Group after group, each for all nsteps steps (independent cavities: the
    // order of the groups does not change any result).
    const int start = b->parity;
    for (BatchGroup& G : b->groups) {
        int parity = start;
        long long done = 0;
        while (done < nsteps) {
            if (nsteps - done >= b->graph_len) {
                if (!G.graph[parity]) {
                    int rc = batch_build_graph(b, G, parity);
                    if (rc) return rc;
                }
                BCK(cudaGraphLaunch(G.graph[parity], b->stream), "cudaGraphLaunch");
                done += b->graph_len;  // even: parity unchanged
            } else {
                int rc = batch_launch(b, G, parity);
                if (rc) return rc;
                parity ^= 1;
                done += 1;
            }
        }
        if (nsteps > 0)  // each cavity's last step: its local Nu rows into its ring
            dmrt::nu_finalize_batch_kernel<<<G.count, 256, 0, b->stream>>>(b->d_cav + G.first, parity);
        BCK(cudaGetLastError(), "batch step launch");
    }
    b->parity = start ^ (int)(nsteps & 1);
    b->t += nsteps;
    for (dmrt_ctx* c : b->sub) {
        c->cur = b->parity;
        c->t += nsteps;
    }
    return DMRT_OK;
}

int dmrt_batch_check(dmrt_batch* b) {
    if (!b) return DMRT_E_ARG;
    BCK(cudaStreamSynchronize(b->stream), "synchronize");
    unsigned err = 0;
    BCK(cudaMemcpy(&err, b->d_err, sizeof err, cudaMemcpyDeviceToHost), "read error flag");
    if (err & dmrt::kErrTimeout) {
        batch_set_err(b, "a bounded device-side wait expired");
        return DMRT_E_TIMEOUT;
    }
    if (err & dmrt::kErrBounds) {
        batch_set_err(b, "an index out of range was seen (bounds-checked build)");
        return DMRT_E_BOUNDS;
    }
    for (int i = 0; i < b->n; ++i) {
        int rc = dmrt_check(b->sub[i]);
        if (rc) {
            batch_set_err(b, "cavity %d: %.200s", i, b->sub[i]->err);
            return rc;
        }
    }
    return DMRT_OK;
}

int32_t dmrt_batch_size(const dmrt_batch* b) { return b ? b->n : 0; }

dmrt_ctx* dmrt_batch_context(dmrt_batch* b, int32_t i) {
    if (!b || i < 0 || i >= b->n) return nullptr;
    return b->sub[i];
}

int dmrt_batch_get_launch(const dmrt_batch* b, dmrt_launch* out) {
    if (!b || !out) return DMRT_E_ARG;
    out->kernel = DMRT_KERNEL_TMA;
    out->tma_npt = b->npt;
    out->tma_rows = b->R;
    out->tma_stages = b->S;
    int grid = 0;
    for (const BatchGroup& G : b->groups) grid = std::max(grid, G.grid);
    out->grid = grid;
    out->block = b->block;
    out->smem_bytes = (int64_t)b->smem;
    out->graph_steps = b->graph_len;
    return DMRT_OK;
}

const char* dmrt_batch_last_error(const dmrt_batch* b) { return b ? b->err : g_create_error; }

void dmrt_batch_destroy(dmrt_batch* b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    for (BatchGroup& G : b->groups)
        for (int i = 0; i < 2; ++i)
            if (G.graph[i]) cudaGraphExecDestroy(G.graph[i]);
    for (dmrt_ctx* c : b->sub) dmrt_destroy(c);
    delete b;
}

int32_t dmrt_batch_group_count(const dmrt_batch* b) { return b ? (int32_t)b->groups.size() : 0; }

}  // extern "C"

// ---- discrete adjoint ------------------------------------------------------------

namespace {

struct AdjLayout {
    long long K, C;  // checkpoint interval and count
    size_t state;    // bytes of one state
    size_t off_ckpt, off_nu0, off_nu1, off_dthw, off_dgb, off_misc, off_rows, off_sdgb, off_sdthw;
    size_t off_seg[2];  // segment slots: one set, or two when the recompute overlaps the reverse sweep
    size_t total_seq;   // bytes with one set of segment slots
    size_t total;       // bytes with two
    size_t total_all;   // bytes with every state stored (from off_ckpt on: C K + 1 states)
    long long n_blocks;  // blocks of the reverse-step grid: one dJ/dgbeta slot each
    bool pairs;          // the sweep's form: pair nodes, or one step per node
};

// The reverse sweep's form: pair nodes (two steps per launch, the first on
// a 3-row window) while their grid takes at most a third of the GPU's
// threads, so that the window's extra rows run on otherwise idle SMs; one
// step per launch above. Tiles of 128 columns; pair tiles of 126 columns with
// one halo column on each side when nx > 128.
bool adj_pairs(const dmrt_ctx* c) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        sms = 152;
    }
    const long long tiles = (long long)((c->p.nx + (c->p.nx <= 128 ? c->p.nx : 126) - 1) /
                                        (c->p.nx <= 128 ? c->p.nx : 126)) * c->p.ny;
    return tiles * dmrt::kPairThreads <= (long long)sms * 2048 / 3;
}
int adj_tile_width(const dmrt_ctx* c, bool pairs) { return pairs && c->p.nx > 128 ? 126 : std::min(c->p.nx, 128); }
int adj_tiles_x(const dmrt_ctx* c, bool pairs) {
    const int tw = adj_tile_width(c, pairs);
    return (c->p.nx + tw - 1) / tw;
}

AdjLayout adjoint_layout(const dmrt_ctx* c, long long N) {
    AdjLayout L;
    L.K = (long long)std::ceil(std::sqrt((double)N));
    if (L.K < 1) L.K = 1;
    // Segments of whole step graphs, so that the forward pass replays graphs only.
    if (L.K > c->graph_len) L.K = (L.K + c->graph_len - 1) / c->graph_len * c->graph_len;
    L.K += L.K & 1;  // even, so that a step's adjoint buffers do not depend on its segment
    L.C = (N + L.K - 1) / L.K;
    L.state = align256((size_t)kPlanes * (size_t)c->L.plane * sizeof(float));
    size_t o = 0;
    L.off_nu0 = o; o += L.state;
    L.off_nu1 = o; o += L.state;
    L.off_dthw = o; o += align256((size_t)c->p.ny * sizeof(double));
    L.pairs = adj_pairs(c);
    L.n_blocks = (long long)adj_tiles_x(c, L.pairs) * c->p.ny;
    L.off_dgb = o; o += align256((size_t)L.n_blocks * sizeof(double));
    L.off_misc = o; o += 256;
    L.off_rows = o; o += align256((size_t)2 * c->p.ny * sizeof(double) + 8);
    L.off_sdgb = o; o += align256((size_t)L.K * L.n_blocks * 4 * sizeof(float2));  // per step and warp
    L.off_sdthw = o; o += align256((size_t)L.K * c->p.ny * sizeof(float));
    L.off_ckpt = o; o += (size_t)L.C * L.state;
    L.off_seg[0] = o; o += (size_t)L.K * L.state;
    L.total_seq = o;
    L.off_seg[1] = o; o += (size_t)L.K * L.state;
    L.total = o;
    L.total_all = L.off_ckpt + (size_t)(L.C * L.K + 1) * L.state;  // s_0 .. s_N, padded to whole segments
    return L;
}

}  // namespace

extern "C" {

int dmrt_adjoint_workspace_size(const dmrt_ctx* c, int64_t nsteps, size_t* bytes) {
    if (!c || !bytes || nsteps < 1) return DMRT_E_ARG;
    *bytes = adjoint_layout(c, nsteps).total;
    return DMRT_OK;
}

int dmrt_adjoint_workspace_min(const dmrt_ctx* c, int64_t nsteps, size_t* bytes) {
    if (!c || !bytes || nsteps < 1) return DMRT_E_ARG;
    *bytes = adjoint_layout(c, nsteps).total_seq;
    return DMRT_OK;
}

int dmrt_adjoint_workspace_all(const dmrt_ctx* c, int64_t nsteps, size_t* bytes) {
    if (!c || !bytes || nsteps < 1) return DMRT_E_ARG;
    *bytes = c->cluster && !c->slab ? adjoint_layout(c, nsteps).total_all : 0;
    return DMRT_OK;
}

int dmrt_adjoint(dmrt_ctx* c, int64_t nsteps, int64_t avg_last, void* workspace, size_t workspace_bytes,
                 double* J, double* dJ_dthetaw, double* dJ_dRa) {
    if (!c) return DMRT_E_ARG;
    if (nsteps < 1 || avg_last < 1 || avg_last > nsteps) {
        set_err(c, "need 1 <= avg_last <= nsteps");
        return DMRT_E_ARG;
    }
    if (c->p.storage != DMRT_FP32) {
        set_err(c, "the adjoint needs float32 storage");
        return DMRT_E_ARG;
    }
    if (c->slab) {
        set_err(c, "the adjoint runs on a whole cavity, not on a slab");
        return DMRT_E_ARG;
    }
    if (avg_last > c->p.nu_capacity) {
        set_err(c, "nu_capacity (%lld) must hold the %lld averaged steps", (long long)c->p.nu_capacity,
                (long long)avg_last);
        return DMRT_E_ARG;
    }
    if ((size_t)kPlanes * (size_t)c->L.plane >= ((size_t)1 << 31)) {
        set_err(c, "the adjoint indexes a state with 32-bit offsets: %lld values per state is too many",
                (long long)kPlanes * (long long)c->L.plane);
        return DMRT_E_ARG;
    }
    const AdjLayout AL = adjoint_layout(c, nsteps);
    // Every forward state stored (no recompute) when the context runs the
    // cluster kernel and the workspace holds them all.
    const bool all = c->cluster && workspace_bytes >= AL.total_all;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) || (workspace_bytes < AL.total_seq && !all)) {
        set_err(c, "adjoint workspace: need %zu bytes (%zu to overlap the recompute with the reverse sweep), "
                   "256-byte aligned", AL.total_seq, AL.total);
        return DMRT_E_SPACE;
    }
    // With room for two sets of segment slots, the recompute of the next segment
    // runs on a second stream while the reverse sweep of the current one runs on
    // the context's stream (the two are latency-bound launches of a few hundred
    // blocks, so they share the GPU); with one set they alternate.
    const bool overlap = !all && workspace_bytes >= AL.total;
    if (overlap && !c->aux) {
        CK(cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking), "adjoint stream");
        for (int i = 0; i < 5; ++i) CK(cudaEventCreateWithFlags(&c->ev[i], cudaEventDisableTiming), "adjoint event");
    }
    cudaStream_t rs = overlap ? c->aux : c->stream;  // the recompute's stream
    char* w = static_cast<char*>(workspace);
    auto ckpt = [&](long long q) { return reinterpret_cast<float*>(w + AL.off_ckpt + (size_t)q * AL.state); };
    auto slot = [&](int set, long long q) {
        return reinterpret_cast<float*>(w + AL.off_seg[set] + (size_t)q * AL.state);
    };
    const size_t copy_bytes = (size_t)kPlanes * (size_t)c->L.plane * sizeof(float);
    const long long N = nsteps, K = AL.K;
    int rc = DMRT_OK;

    // Reverse sweep, segment by segment from the last.
    float* nu_a = reinterpret_cast<float*>(w + AL.off_nu0);
    float* nu_b = reinterpret_cast<float*>(w + AL.off_nu1);
    double* dthw = reinterpret_cast<double*>(w + AL.off_dthw);
    float2* sdgb = reinterpret_cast<float2*>(w + AL.off_sdgb);
    float* sdthw = reinterpret_cast<float*>(w + AL.off_sdthw);
    Misc* scratch = reinterpret_cast<Misc*>(w + AL.off_misc);
    CK(cudaMemsetAsync(nu_a, 0, copy_bytes, c->stream), "zero adjoint");
    CK(cudaMemsetAsync(w + AL.off_dthw, 0, AL.off_rows - AL.off_dthw, c->stream), "zero gradients");
    double* dgb = reinterpret_cast<double*>(w + AL.off_dgb);  // per-block totals, zeroed with the gradients
    dmrt::StepArgs RA = step_args(c, 0);  // recompute: Nusselt output into scratch
    double* ra_rows = reinterpret_cast<double*>(w + AL.off_rows);  // two buffers, alternating by step
    RA.nu_ring = ra_rows + 2 * (size_t)c->p.ny;
    RA.nu_last = RA.nu_ring;
    RA.pending = &scratch->pending;
    RA.err = &scratch->err;
    RA.step_in = &scratch->step[0];
    RA.step_out = &scratch->step[1];
    RA.cap = 1;
    long long* seg_ctr = reinterpret_cast<long long*>(w + AL.off_misc + 128);  // the graphs' segment counters
    dmrt::AdjArgs AA;
    std::memset(&AA, 0, sizeof AA);
    AA.slot[0] = slot(0, 0);
    AA.slot[1] = overlap ? slot(1, 0) : slot(0, 0);
    float* states = reinterpret_cast<float*>(w + AL.off_ckpt);  // with `all`: s_k at states + k * state
    AA.all = all ? states : nullptr;
    AA.nu[0] = nu_a;  // nu_{N+1} = 0
    AA.nu[1] = nu_b;
    AA.hot = reinterpret_cast<const float*>(c->ws + c->L.off_hot);
    AA.cold = reinterpret_cast<const float*>(c->ws + c->L.off_cold);
    AA.dthw = dthw;
    AA.dgbeta = dgb;
    AA.dthw_step = sdthw;
    AA.dgbeta_step = sdgb;
    AA.state = (long long)(AL.state / sizeof(float));
    AA.K = K;
    AA.N = N;
    AA.C = AL.C;
    AA.w_from = N - avg_last;
    AA.n_blocks = AL.n_blocks;
    AA.plane = c->L.plane;
    AA.nsets = overlap ? 2 : 1;
    AA.nx = c->p.nx;
    AA.ny = c->p.ny;
    AA.pitch = c->L.pitch;
    AA.w = (float)(1.0 / (double)avg_last);
    AA.nu_wall = (float)(-9.0 * c->sc.nu_scale / c->p.ny);
    AA.nu_next = (float)(c->sc.nu_scale / c->p.ny);
    AA.tw = adj_tile_width(c, AL.pairs);
    AA.hx = AL.pairs && c->p.nx > 128 ? 1 : 0;
    AA.pairs = AL.pairs ? 1 : 0;
    const dim3 agrid(adj_tiles_x(c, AL.pairs), c->p.ny);
    // The reverse sweep of a segment: one graph of K / 2 pair nodes, or K
    // single-step nodes (programmatic edges), and the fold; graph p reads
    // counter p and leaves the next segment in counter 1 - p, so replays
    // alternate between the two.
    struct Execs {
        cudaGraphExec_t e[2] = {nullptr, nullptr};
        ~Execs() {
            for (cudaGraphExec_t x : e)
                if (x) cudaGraphExecDestroy(x);
        }
    } rg;
    for (int gp = 0; gp < 2; ++gp) {
        dmrt::AdjArgs Ap = AA;
        Ap.seg = seg_ctr + gp;
        Ap.seg_next = seg_ctr + (gp ^ 1);
        cudaGraph_t g;
        CK(cudaGraphCreate(&g, 0), "cudaGraphCreate");
        cudaGraphNode_t prev = nullptr;
        cudaError_t e = cudaSuccess;
        const long long per = AL.pairs ? 2 : 1;  // steps per node
        for (long long i = 0; i < K / per && e == cudaSuccess; ++i) {
            int set = gp, th = (int)(K - 1 - per * i);  // the segment's last step (pair) first
            void* params[4] = {&Ap, &set, &th, &c->sc};
            cudaKernelNodeParams kp = {};
            if (AL.pairs) {
                kp.func = all ? (void*)dmrt::adjoint_pair_kernel<true> : (void*)dmrt::adjoint_pair_kernel<false>;
                kp.blockDim = dim3(dmrt::kPairThreads);
            } else {
                kp.func = all ? (void*)dmrt::adjoint_step_kernel<true> : (void*)dmrt::adjoint_step_kernel<false>;
                kp.blockDim = dim3(128);
            }
            kp.gridDim = agrid;
            kp.kernelParams = params;
            cudaGraphNode_t node;
            e = add_step_node(g, prev, &kp, &node);
            prev = node;
        }
        if (e == cudaSuccess) {
            const long long warps = AL.n_blocks + c->p.ny, per = dmrt::kFoldThreads / 32;
            void* params[2] = {&Ap, &c->sc};
            cudaKernelNodeParams kp = {};
            kp.func = (void*)dmrt::adjoint_fold_kernel;
            kp.gridDim = dim3((unsigned)((warps + per - 1) / per));
            kp.blockDim = dim3(dmrt::kFoldThreads);
            kp.kernelParams = params;
            cudaGraphNode_t node;
            e = cudaGraphAddKernelNode(&node, g, &prev, 1, &kp);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&rg.e[gp], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(c, e, "adjoint graph");
    }
    const long long q_last = AL.C - 1;
    CK(cudaMemcpyAsync(seg_ctr, &q_last, sizeof q_last, cudaMemcpyHostToDevice, c->stream), "segment counter");
    // The segment recompute runs the context's own step kernel. For the TMA
    // kernel every checkpoint and segment slot it reads gets its load maps
    // (float32 storage stores from registers, so no store maps are needed).
    const bool tma_re = !all && c->kernel == DMRT_KERNEL_TMA;
    const int nsets = overlap ? 2 : 1;
    std::vector<dmrt::TmaMaps> ck_maps(tma_re ? (size_t)AL.C : 0), sl_maps(tma_re ? (size_t)(nsets * AL.K) : 0);
    for (size_t q = 0; q < ck_maps.size() + sl_maps.size(); ++q) {
        const bool ck = q < ck_maps.size();
        const size_t qs = q - ck_maps.size();
        dmrt::TmaMaps& m = ck ? ck_maps[q] : sl_maps[qs];
        float* base = ck ? ckpt((long long)q) : slot((int)(qs / AL.K), (long long)(qs % AL.K));
        std::memset(&m, 0, sizeof m);
        rc = encode_map(c, &m.ld[0], base, DMRT_FP32, kPlanes, 6, c->R);
        if (!rc) rc = encode_map(c, &m.ld[1], base, DMRT_FP32, kPlanes, 4, c->R);
        if (rc) return rc;
    }
    // With the recompute on its own stream, a cavity that fits one thread-block
    // cluster recomputes each segment in one cluster launch (on 16 SMs or fewer,
    // so it takes little from the reverse sweep's blocks), writing every state.
    int ccs = 0, ccr = 0, cct = 0;
    size_t ccm = 0;
    const bool cluster_re = overlap && cluster_fit(c, &ccs, &ccr, &cct, &ccm);
    // Recompute of segment q into slot set `set` on stream rs: s_{start + t} into slot t
    // (slot 0: a copy of the checkpoint).
    auto recompute = [&](long long q, int set) -> int {
        const long long start = q * K, len = std::min(start + K, N) - start;
        CK(cudaMemcpyAsync(slot(set, 0), ckpt(q), copy_bytes, cudaMemcpyDeviceToDevice, rs), "segment start");
        if (cluster_re && len > 1) {
            dmrt::ClusterArgs CA;
            CA.A[0] = CA.A[1] = step_args(c, 0);
            CA.K = c->sc;
            CA.steps = (int)(len - 1);
            CA.parity = 0;
            CA.rows_per = ccr;
            CA.start = ckpt(q);
            CA.record = slot(set, 1);
            CA.record_stride = (long long)(AL.state / sizeof(float));
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = ccs;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3(ccs);
            cfg.blockDim = dim3(cct);
            cfg.dynamicSmemBytes = ccm;
            cfg.stream = rs;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            CK(launch_cluster_kernel(cfg, CA), "adjoint recompute launch");
            return DMRT_OK;
        }
        for (long long t = 1; t < len; ++t) {
            RA.src = t == 1 ? ckpt(q) : slot(set, t - 1);
            RA.dst = slot(set, t);
            RA.nu_rows = ra_rows + (size_t)(t & 1) * c->p.ny;
            RA.prev_rows = ra_rows + (size_t)((t + 1) & 1) * c->p.ny;
            if (tma_re) {
                dmrt::TmaMaps& M = t == 1 ? ck_maps[(size_t)q] : sl_maps[(size_t)(set * K + t - 1)];
                void* params[4] = {&M, &RA, &c->sc, &c->geo};
                CK(launch_overlapped(c->tma_func, dim3(c->tma_grid), dim3(c->tma_block), c->tma_smem, rs, params),
                   "adjoint recompute launch");
            } else {
                CK(launch_overlapped(dmrt::step_direct_kernel, c->grid, dim3(dmrt::kDirectThreads), rs, RA, c->sc),
                   "adjoint recompute launch");
            }
        }
        return DMRT_OK;
    };
    // Forward pass with checkpoints every K steps (issued once the sweep's
    // graphs and arguments are ready, so that the GPU does not wait for the
    // host between the passes; J is read from the Nusselt ring at the end).
    // With `all`, every state instead: s_0 copied, s_1 .. s_N written by the
    // cluster kernel as it steps.
    CK(cudaMemcpyAsync(ckpt(0), buf(c, c->cur), copy_bytes, cudaMemcpyDeviceToDevice, c->stream), "checkpoint");
    if (all) {
        const long long sf = (long long)(AL.state / sizeof(float));
        rc = step_run(c, N, true, states + sf, sf);
        if (rc) return rc;
    }
    for (long long q = 0; q < AL.C && !all; ++q) {
        const long long n = std::min(K, N - q * K);
        rc = step_run(c, n, q + 1 == AL.C);  // the last segment sums its last step's rows
        if (rc) return rc;
        if (q + 1 < AL.C)
            CK(cudaMemcpyAsync(ckpt(q + 1), buf(c, c->cur), copy_bytes, cudaMemcpyDeviceToDevice, c->stream),
               "checkpoint");
    }
    // Events (overlap): ev[0] the forward pass done; ev[1 + set] recompute into
    // `set` done; ev[3 + set] reverse sweep from `set` done.
    if (overlap) {
        CK(cudaEventRecord(c->ev[0], c->stream), "event");
        CK(cudaStreamWaitEvent(rs, c->ev[0], 0), "wait");
    }
    if (!all) {
        rc = recompute(AL.C - 1, 0);
        if (rc) return rc;
    }
    if (overlap) CK(cudaEventRecord(c->ev[1], rs), "event");
    for (long long q = AL.C - 1; q >= 0; --q) {
        const int set = (int)((AL.C - 1 - q) & 1) % nsets;
        if (overlap && q >= 1) {
            // Segment q - 1 into the other set, once the sweep that last read it is done.
            if (q + 1 <= AL.C - 1) CK(cudaStreamWaitEvent(rs, c->ev[3 + (set ^ 1)], 0), "wait");
            rc = recompute(q - 1, set ^ 1);
            if (rc) return rc;
            CK(cudaEventRecord(c->ev[1 + (set ^ 1)], rs), "event");
        }
        if (overlap) CK(cudaStreamWaitEvent(c->stream, c->ev[1 + set], 0), "wait");
        CK(cudaGraphLaunch(rg.e[(AL.C - 1 - q) & 1], c->stream), "adjoint sweep launch");
        if (overlap) CK(cudaEventRecord(c->ev[3 + set], c->stream), "event");
        if (!overlap && !all && q >= 1) {
            rc = recompute(q - 1, 0);
            if (rc) return rc;
        }
    }
    dmrt::adjoint_gather_kernel<<<(c->p.ny + 127) / 128, 128, 0, c->stream>>>(AA, c->sc);
    CK(cudaGetLastError(), "adjoint launch");
    std::vector<double> g((size_t)c->p.ny);
    std::vector<double> slots((size_t)AL.n_blocks);
    CK(cudaMemcpyAsync(g.data(), dthw, g.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "read dJ/dtheta_w");
    CK(cudaMemcpyAsync(slots.data(), dgb, slots.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
       "read dJ/dgbeta");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    std::vector<double> series((size_t)avg_last);
    int64_t got = 0;
    rc = dmrt_nusselt(c, nullptr, nullptr, series.data(), avg_last, &got);
    if (rc) return rc;
    double jsum = 0.0;
    for (int64_t q = 0; q < got; ++q) jsum += series[(size_t)q];
    if (J) *J = jsum / (double)avg_last;
    // The Nusselt stencil's own theta_w term, 8 scale / ny per averaged step.
    const double direct = 8.0 * c->sc.nu_scale / (double)c->p.ny;
    if (dJ_dthetaw)
        for (int j = 0; j < c->p.ny; ++j) dJ_dthetaw[j] = g[(size_t)j] + direct;
    double dgbeta = 0.0;
    for (double v : slots) dgbeta += v;  // in block order
    // gbeta = Ra nu alpha / (H^3 dT), so dJ/dRa = dJ/dgbeta * nu alpha / (H^3 dT).
    const double H = (double)c->p.ny, dT = c->p.theta_hot - c->p.theta_cold;
    if (dJ_dRa) *dJ_dRa = dT != 0.0 ? dgbeta * c->k.nu * c->k.alpha / (H * H * H * dT) : 0.0;
    return dmrt_check(c);
}

}  // extern "C"
