// Shared device pieces of the double-MRT step (Li, Yang & Zhang, arXiv 1601.04633,
// Sec. 3): the population layout, per-launch arguments, the per-node collision
// with the buoyancy force, and the fused hot-wall Nusselt reduction.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dmrt {

constexpr int kPlanes = 14;
constexpr unsigned kFull = 0xffffffffu;

// Populations are stored as 14 planes [ny][pitch] (structure of arrays; pitch a
// multiple of 128 elements, padding columns kept at zero). The planes are
// grouped by the y component of their lattice velocity, so that the pull of one
// output row reads three contiguous plane groups from three rows:
//   Z (e_y =  0, source row j):     f1 f2 f4 g1 g2 g4   -> planes 0..5
//   P (e_y = +1, source row j - 1): f3 f6 f7 g3         -> planes 6..9
//   N (e_y = -1, source row j + 1): f5 f8 f9 g5         -> planes 10..13
// (paper numbering, Eqs. 23 and 35). plane_f(k) / plane_g(k) give the plane of
// the 0-based direction k.
__host__ __device__ constexpr int plane_f(int k) {
    return k == 0 ? 0 : k == 1 ? 1 : k == 2 ? 6 : k == 3 ? 2 : k == 4 ? 10 : k == 5 ? 7 : k == 6 ? 8 : k == 7 ? 11 : 12;
}
__host__ __device__ constexpr int plane_g(int k) {
    return k == 0 ? 3 : k == 1 ? 4 : k == 2 ? 9 : k == 3 ? 5 : 13;
}
constexpr int kGroupZ = 0, kGroupP = 6, kGroupN = 10;

// Relaxation constants pre-divided by the squared norms of the rows of the
// transforms (D2Q9: 9,6,6,36,4,4,12,12,36; D2Q5: 5,2,2,20,4), so that
// f* = f - sum_k M[k][i] d_k with d_k = rate_k (m_k - m_k_eq) / norm_k.
// (16-byte aligned, as StepArgs: where a kernel reads them from shared memory,
// neighbouring fields come in 16-byte loads.)
struct alignas(16) StepConsts {
    float se36, snu4, sq12, seps36;  // D2Q9: s_e/36, s_nu/4, s_q/12, s_eps/36
    float sk2, se20, snu4t;          // D2Q5: sigma_k/2, sigma_e/20, sigma_nu/4
    float a;                         // D2Q5 equilibrium parameter (Eq. 43)
    float gbeta, theta_ref;          // G_y = gbeta (theta - theta_ref) (Eq. 27)
    float abb;                       // 2 sqrt(3) alpha (Eq. 45)
    int left_fixed, right_fixed;     // 1 = anti-bounce-back wall, 0 = adiabatic
    float gsh0, gsh1;                // 16-bit storage: g_0, g_1..4 stored minus these
    float w0, w1;                    // D2Q5 rest weights (1 - a)/5 and (4 + a)/20 (Eq. 42)
    double nu_scale;                 // H / (3 (theta_hot - theta_cold))
};

struct alignas(16) StepArgs {
    const float* __restrict__ src;  // post-collision state at time t
    float* __restrict__ dst;        // post-collision state at time t + 1
    const float* __restrict__ hot;  // [ny] left-wall temperature
    const float* __restrict__ cold; // [ny] right-wall temperature
    double* nu_rows;                // [ny] local Nu of this step
    const double* prev_rows;        // [ny] local Nu of the previous step (summed by this step)
    double* nu_ring;                // [cap] mean Nu per step
    double* nu_last;                // mean Nu of the latest summed step
    unsigned* pending;              // 1 while prev_rows holds a step not yet summed into the ring
    unsigned* err;                  // bit 0: non-finite value; bit 1: wait timed out
    const long long* step_in;       // steps taken before this step (read by all)
    long long* step_out;            // written once, = step_in + 1
    int rounding;                   // 16-bit storage: 0 nearest, 1 stochastic
    long long cap;
    long long plane;  // elements per plane = (rows held) * pitch
    int nx, ny, pitch;
    int wx_log2;      // direct kernel: lanes per row segment = 1 << wx_log2
    // A y-slab of a larger cavity holds one halo row below and one above its
    // ny rows: node row j sits in buffer row j + row0 (row0 = 1; 0 for a whole
    // cavity), and only the slab sides that are cavity walls (wall_lo: row 0,
    // wall_hi: row ny - 1) apply the wall rules; across the others the pull
    // reads the halo rows, which the neighbouring slabs fill. jglob0 is the
    // cavity row of node row 0 (it seeds the stochastic rounding, so a slab
    // rounds as the whole cavity would), nu_inv the reciprocal of the row
    // count of the whole cavity (the Nusselt mean of a slab is its share of
    // the cavity's mean; a product, since a float64 division is slow here).
    int row0, wall_lo, wall_hi, jglob0;
    double nu_inv;
};

constexpr unsigned kErrNonFinite = 1u;
constexpr unsigned kErrTimeout = 2u;
constexpr unsigned kErrBounds = 4u;  // an index out of its range (bounds-checked builds)

// Bounds-checked builds (-DDMRT_BOUNDS_CHECK): DMRT_IN(i, lo, hi, err) is true
// when lo <= i < hi, and otherwise records kErrBounds in *err and is false; the
// kernels test it before each global and shared-memory access whose index they
// compute, and skip the access when it is false. Other builds: always true, no
// code.
#ifdef DMRT_BOUNDS_CHECK
__device__ __forceinline__ bool bounds_ok(long long i, long long lo, long long hi, unsigned* err) {
    if (i >= lo && i < hi) return true;
    atomicOr(err, kErrBounds);
    return false;
}
#define DMRT_IN(i, lo, hi, err) ::dmrt::bounds_ok((long long)(i), (long long)(lo), (long long)(hi), (err))
#else
#define DMRT_IN(i, lo, hi, err) true
#endif

// Programmatic dependent launch. In the step graphs each step kernel depends on
// the previous one through a programmatic edge, so its blocks may be launched
// while the previous step's last blocks still run. grid_dep_wait() returns once
// the previous kernel has completed and its memory operations are visible (at
// once for a kernel launched without such an edge); a step kernel calls it
// before its first access to global memory, so nothing it reads or writes
// overlaps the previous step. grid_dep_launch() then allows the next step's
// launch to begin.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ float4 ldg4(const float* p) {
    return __ldg(reinterpret_cast<const float4*>(p));
}

template <int E>
__device__ __forceinline__ float& comp(float4& v) {
    if constexpr (E == 0) return v.x;
    else if constexpr (E == 1) return v.y;
    else if constexpr (E == 2) return v.z;
    else return v.w;
}

__device__ __forceinline__ void set_comp(float4& v, int e, float val) {
    v.x = (e == 0) ? val : v.x;
    v.y = (e == 1) ? val : v.y;
    v.z = (e == 2) ? val : v.z;
    v.w = (e == 3) ? val : v.w;
}

// Collision + force + thermal collision of one node, in place.
// f[0..8]: D2Q9 populations (shifted: they sum to delta-rho, Eq. 33),
// g[0..4]: D2Q5 populations. Directions: f1..f4 = (1,0),(0,1),(-1,0),(0,-1),
// f5..f8 = (1,1),(-1,1),(-1,-1),(1,-1); g1..g4 as f1..f4 (0-based indices).
__device__ __forceinline__ void collide_node(float (&f)[9], float (&g)[5], const StepConsts& K,
                                             float& rho_out, float& theta_out) {
    // Moments m = M f (Eq. 30), with rho0 = 1 so u = jx, v = jy (Eq. 33).
    const float a13 = f[1] - f[3], a24 = f[2] - f[4];
    const float s13 = f[1] + f[3], s24 = f[2] + f[4];
    const float a56 = f[5] - f[6], a78 = f[7] - f[8];
    const float s56 = f[5] + f[6], s78 = f[7] + f[8];
    const float s1234 = s13 + s24, s5678 = s56 + s78;
    const float rho = f[0] + s1234 + s5678;
    const float u = a13 + a56 - a78;
    const float v = a24 + s56 - s78;
    const float e = -4.f * f[0] - s1234 + 2.f * s5678;
    const float pxx = s13 - s24;
    const float pxy = (f[5] + f[7]) - (f[6] + f[8]);
    const float qx = -2.f * a13 + a56 - a78;
    const float qy = -2.f * a24 + s56 - s78;
    const float eps = 4.f * f[0] - 2.f * s1234 + s5678;
    const float uu = u * u + v * v;
    const float theta = g[0] + g[1] + g[2] + g[3] + g[4];  // Eq. 41

    // Buoyancy force (Eqs. 26-27): F_i = 3 (e_i - u).G f_i^eq(rho0 = 1, u) with
    // G = (0, Gy), Gy = gbeta (theta - theta_ref). It is added in moment space:
    // the moments M F of that F are, exactly, (rho, e, eps, jx, qx, jy, qy, pxx,
    // pxy) = (0, 3 Gy v (2 - 3|u|^2), -3 Gy v (2 - 3|u|^2), 0, 6 Gy u v, Gy,
    // Gy (3u^2 - 1), -Gy v (3(u^2 - v^2) + 2), Gy u (1 - 3v^2)), and
    // F = M^-1 (M F), so each term joins its moment's relaxation below
    // (divided by the moment's norm, as M^-1 = M^T diag(1/norm)).
    const float Gy = K.gbeta * (theta - K.theta_ref);
    const float uu_d = u * u - v * v;
    const float g12 = Gy * (1.f / 12.f);
    const float fe = g12 * v * (2.f - 3.f * uu);                // (M F)_e / 36 = -(M F)_eps / 36
    const float fqx = 0.5f * Gy * u * v;                        // (M F)_qx / 12
    const float fqy = g12 * (3.f * u * u - 1.f);                // (M F)_qy / 12
    const float fpxx = -0.25f * Gy * v * (3.f * uu_d + 2.f);    // (M F)_pxx / 4
    const float fpxy = 0.25f * Gy * u * (1.f - 3.f * v * v);    // (M F)_pxy / 4
    const float fjy = Gy * (1.f / 6.f);                         // (M F)_jy / 6

    // Non-equilibrium parts (Eq. 34, m4_eq = -2 drho + 3 |u|^2), scaled, less the force terms.
    const float d3 = K.se36 * (e + 2.f * rho - 3.f * uu) - fe;
    const float d4 = K.snu4 * (pxx - uu_d) - fpxx;
    const float d5 = K.snu4 * (pxy - u * v) - fpxy;
    const float d6 = K.sq12 * (qx + u) - fqx;
    const float d7 = K.sq12 * (qy + v) - fqy;
    const float d8 = K.seps36 * (eps - rho + 3.f * uu) + fe;

    // f* = f - M^-1 (S (m - m_eq) - M F), with M^-1 = M^T diag(1/norm) (Eq. 28).
    f[0] = f[0] + 4.f * d3 - 4.f * d8;
    f[1] = f[1] + d3 - d4 + 2.f * d6 + 2.f * d8;
    f[2] = f[2] + d3 + d4 + 2.f * d7 + 2.f * d8 + fjy;
    f[3] = f[3] + d3 - d4 - 2.f * d6 + 2.f * d8;
    f[4] = f[4] + d3 + d4 - 2.f * d7 + 2.f * d8 - fjy;
    f[5] = f[5] - 2.f * d3 - d5 - d6 - d7 - d8 + fjy;
    f[6] = f[6] - 2.f * d3 + d5 + d6 - d7 - d8 + fjy;
    f[7] = f[7] - 2.f * d3 - d5 + d6 + d7 - d8 - fjy;
    f[8] = f[8] - 2.f * d3 + d5 - d6 + d7 - d8 - fjy;

    // D2Q5: n = N g (Eq. 37, fifth row (0,1,-1,1,-1)), n_eq = (theta, u theta,
    // v theta, a theta, 0) (Eq. 42), g* = g - N^-1 Q (n - n_eq) (Eq. 36).
    const float n1 = g[1] - g[3];
    const float n2 = g[2] - g[4];
    const float n3 = -4.f * g[0] + (g[1] + g[2] + g[3] + g[4]);
    const float n4 = (g[1] + g[3]) - (g[2] + g[4]);
    const float e1 = K.sk2 * (n1 - u * theta);
    const float e2 = K.sk2 * (n2 - v * theta);
    const float e3 = K.se20 * (n3 - K.a * theta);
    const float e4 = K.snu4t * n4;
    g[0] = g[0] + 4.f * e3;
    g[1] = g[1] - e1 - e3 - e4;
    g[2] = g[2] - e2 - e3 + e4;
    g[3] = g[3] + e1 - e3 - e4;
    g[4] = g[4] + e2 - e3 + e4;

    rho_out = rho;
    theta_out = theta;
}

// Collide node E of four (F, Gq hold the pulled populations of 4 nodes) in
// place; invalid nodes (padding) are zeroed so the padding stays zero.
template <int E>
__device__ __forceinline__ void node_update(float4 (&F)[9], float4 (&Gq)[5], const StepConsts& K,
                                            float (&theta4)[4], bool valid, bool& bad) {
    float f[9], g[5];
#pragma unroll
    for (int k = 0; k < 9; ++k) f[k] = comp<E>(F[k]);
#pragma unroll
    for (int k = 0; k < 5; ++k) g[k] = comp<E>(Gq[k]);
    float rho, theta;
    collide_node(f, g, K, rho, theta);
    if (valid) {
        bad |= !(fabsf(rho) < 1e30f) || !(fabsf(theta) < 1e30f);
    } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) f[k] = 0.f;
#pragma unroll
        for (int k = 0; k < 5; ++k) g[k] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) comp<E>(F[k]) = f[k];
#pragma unroll
    for (int k = 0; k < 5; ++k) comp<E>(Gq[k]) = g[k];
    theta4[E] = theta;
}

__device__ __forceinline__ void collide_quad(float4 (&F)[9], float4 (&Gq)[5], const StepConsts& K,
                                             float (&theta4)[4], int nvalid, bool& bad) {
    node_update<0>(F, Gq, K, theta4, nvalid > 0, bad);
    node_update<1>(F, Gq, K, theta4, nvalid > 1, bad);
    node_update<2>(F, Gq, K, theta4, nvalid > 2, bad);
    node_update<3>(F, Gq, K, theta4, nvalid > 3, bad);
}

// Store a collided quad (4 nodes from x0 of row j) to the destination planes.
__device__ __forceinline__ void store_quad(const StepArgs& A, int j, int x0, const float4 (&F)[9],
                                           const float4 (&Gq)[5]) {
    const long long o = (long long)(j + A.row0) * A.pitch + x0;
    if (!DMRT_IN(o, 0, A.plane - 3, A.err)) return;
    float* D = A.dst + o;
#pragma unroll
    for (int k = 0; k < 9; ++k) *reinterpret_cast<float4*>(D + plane_f(k) * A.plane) = F[k];
#pragma unroll
    for (int k = 0; k < 5; ++k) *reinterpret_cast<float4*>(D + plane_g(k) * A.plane) = Gq[k];
}

// Hot-wall Nusselt number (Eqs. 18-19), in two halves so that no step waits
// for its own mean. During a step the thread holding row j's local value
// stores it (nu_report). The mean over the rows is taken by one warp at the
// start of the next step by one block, or by the finalize launch after a run
// of steps (nu_finish_prev), when the rows are complete without any counting.
__device__ __forceinline__ void nu_report(const StepArgs& A, bool has_nu, int j, double nuj) {
    if (has_nu && DMRT_IN(j, 0, A.ny, A.err)) A.nu_rows[j] = nuj;
}

// Called by every thread of a block (it synchronises the block), once per
// step (step = true, at any point of the step's launch) or once after a run of
// steps (step = false). If prev_rows holds a step not yet summed, its ny rows
// are summed in a fixed order and appended to the ring as step step_in - 1: 256
// partial sums, partial p over rows p, p + 256, p + 512, ... in that order,
// kept by lane p % 32 of the warp that takes stream q = p / 32 (warps take
// q = w, w + nwarps, ...), each partial starting from its first row; lane l
// then adds its partials pairwise (nu_combine), and the warp adds the 32 lane
// sums by a butterfly. The order does not depend
// on the block size or on scheduling. A step then advances the step counter
// (step_out = step_in + 1) and marks its own rows as pending; the finalize
// call clears the mark.
// A lane's partial sums of Nusselt rows p[q], q < nq = min(8, ceil(ny / 32))
// (partials q >= nq hold no row), added pairwise: ((p0 + p1) + (p2 + p3)) +
// ((p4 + p5) + (p6 + p7)), a leaf past nq left out (float64 is a slow pipe on
// this GPU, so no zeros are added). Every kernel that sums a step's rows uses
// this order; nq is the same in every lane, so the branches are uniform.
__device__ __forceinline__ int nu_partials(int ny) { return ny >= 256 ? 8 : (ny + 31) / 32; }
__device__ __forceinline__ double nu_combine(const double (&p)[8], int nq) {
    double a = p[0];
    if (nq > 1) a += p[1];
    if (nq > 2) {
        double b = p[2];
        if (nq > 3) b += p[3];
        a += b;
    }
    if (nq > 4) {
        double c = p[4];
        if (nq > 5) c += p[5];
        if (nq > 6) {
            double d = p[6];
            if (nq > 7) d += p[7];
            c += d;
        }
        a += c;
    }
    return a;
}

__device__ __forceinline__ void nu_finish_prev(const StepArgs& A, bool step) {
    __shared__ double part[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const long long t = __ldcg(A.step_in);
    const unsigned pend = __ldcg(A.pending);
    __syncthreads();  // every thread has read the flag before thread 0 rewrites it
    if (pend) {
        for (int q = warp; q < 8; q += nw) {
            double acc = 0.0;
            int r = lane + 32 * q;
            if (r < A.ny) {  // the partial starts from its first row
                acc = __ldcg(A.prev_rows + r);
                r += 256;
            }
            for (; r + 3 * 256 < A.ny; r += 4 * 256) {  // four loads in flight, added in order
                double v[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) v[i] = __ldcg(A.prev_rows + r + 256 * i);
#pragma unroll
                for (int i = 0; i < 4; ++i) acc += v[i];
            }
            for (; r < A.ny; r += 256) acc += __ldcg(A.prev_rows + r);
            part[q][lane] = acc;
        }
        __syncthreads();
        if (warp == 0) {
            double p8[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) p8[q] = part[q][lane];
            double s = nu_combine(p8, nu_partials(A.ny));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
            if (lane == 0) {
                const double mean = s * A.nu_inv;
                if (DMRT_IN((t - 1) % A.cap, 0, A.cap, A.err)) A.nu_ring[(t - 1) % A.cap] = mean;
                *A.nu_last = mean;
            }
        }
        __syncthreads();  // part may be reused by the next call
    }
    if (threadIdx.x == 0) {
        if (step) {
            *A.step_out = t + 1;
            *A.pending = 1u;
        } else {
            *A.pending = 0u;
        }
    }
}

// Sums the last step of a run (one block of 256 threads).
static __global__ void nu_finalize_kernel(StepArgs A) { nu_finish_prev(A, false); }

}  // namespace dmrt
