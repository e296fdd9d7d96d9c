// Fused double-MRT time step for sm_103a (Li, Yang & Zhang, arXiv 1601.04633, Sec. 3).
//
// One launch advances every node of the cavity by one time step:
//   pull-stream the D2Q9 populations f (Eq. 25) and the D2Q5 populations g
//   (Eq. 36) from the previous post-collision buffer, with half-way
//   bounce-back on the no-slip walls, bounce-back on adiabatic walls (Eq. 44)
//   and anti-bounce-back on fixed-temperature walls (Eq. 45);
//   moments (Eqs. 33, 41); D2Q9 MRT relaxation (Eqs. 28-32, 34); buoyancy
//   force (Eqs. 26-27); D2Q5 MRT relaxation (Eqs. 37-43); store to the other
//   buffer; hot-wall Nusselt number from the pre-collision temperature
//   (Eqs. 18-19), reduced in a fixed order so every run gives the same bits.
//
// Layout: structure of arrays, 14 planes (f0..f8, g0..g4), each plane
// [ny][pitch] with pitch a multiple of 128 elements; the padding columns are
// kept at zero. Each thread owns four consecutive nodes of one row and moves
// them with 128-bit loads and stores; the x +- 1 shifts of the pull are done
// with warp shuffles inside a row segment of WX lanes, and only the segment's
// edge lanes read their one halo value from memory (an L1/L2 hit: the
// neighbouring segment reads the same sector).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dmrt {

constexpr int kPlanes = 14;
constexpr int kThreads = 128;  // 4 warps per block
constexpr unsigned kFull = 0xffffffffu;

// Relaxation constants pre-divided by the squared norms of the rows of the
// transforms (D2Q9: 9,6,6,36,4,4,12,12,36; D2Q5: 5,2,2,20,4), so that
// f* = f - sum_k M[k][i] d_k with d_k = rate_k (m_k - m_k_eq) / norm_k.
struct StepConsts {
    float se36, snu4, sq12, seps36;  // D2Q9: s_e/36, s_nu/4, s_q/12, s_eps/36
    float sk2, se20, snu4t;          // D2Q5: sigma_k/2, sigma_e/20, sigma_nu/4
    float a;                         // D2Q5 equilibrium parameter (Eq. 43)
    float gbeta, theta_ref;          // G_y = gbeta (theta - theta_ref) (Eq. 27)
    float abb;                       // 2 sqrt(3) alpha (Eq. 45)
    int left_fixed, right_fixed;     // 1 = anti-bounce-back wall, 0 = adiabatic
    double nu_scale;                 // H / (3 (theta_hot - theta_cold))
};

struct StepArgs {
    const float* __restrict__ src;  // post-collision state at time t
    float* __restrict__ dst;        // post-collision state at time t + 1
    const float* __restrict__ hot;  // [ny] left-wall temperature
    const float* __restrict__ cold; // [ny] right-wall temperature
    double* nu_rows;                // [ny] local Nu of the latest step
    double* nu_ring;                // [cap] mean Nu per step
    double* nu_last;                // mean Nu of the latest step
    unsigned* counter;              // rows reported in the current step
    unsigned* err;                  // bit 0: non-finite density or temperature
    long long* d_step;              // steps recorded so far
    long long cap;
    long long plane;  // elements per plane = ny * pitch
    int nx, ny, pitch;
    int wx_log2;      // lanes per row segment = 1 << wx_log2
};

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

struct Geo {
    int nx, ny, pitch, wx, seg_lane;
};

// Pull one plane for the four nodes (x0..x0+3, j): value at node x is the
// post-collision value of the same plane at x - e (Eq. 25 / Eq. 36). Links
// that leave through the top or bottom wall reflect the node's own opposite
// population (no-slip bounce-back; Eq. 44 for g). Links that leave through
// the left/right walls take  sign * opposite + add  (bounce-back: 1, 0;
// anti-bounce-back, Eq. 45: -1, 2 sqrt(3) alpha theta_w).
template <int EX, int EY>
__device__ __forceinline__ float4 pull(const float* __restrict__ P, const float* __restrict__ Popp,
                                       int j, int x0, const Geo& G, float sign_l, float add_l,
                                       float sign_r, float add_r) {
    const int r = j - EY;
    const bool yin = (r >= 0) && (r < G.ny);
    const int rc = min(max(r, 0), G.ny - 1);
    const float* row = P + (size_t)rc * G.pitch;
    float4 v = ldg4(row + x0);
    float4 out;
    if constexpr (EX == 0) {
        out = v;
    } else if constexpr (EX == 1) {
        float left = __shfl_up_sync(kFull, v.w, 1, G.wx);
        if (G.seg_lane == 0) left = (x0 > 0) ? __ldg(row + x0 - 1) : 0.f;
        out = make_float4(left, v.x, v.y, v.z);
    } else {
        float right = __shfl_down_sync(kFull, v.x, 1, G.wx);
        if (G.seg_lane == G.wx - 1) right = (x0 + 4 < G.pitch) ? __ldg(row + x0 + 4) : 0.f;
        out = make_float4(v.y, v.z, v.w, right);
    }
    const float* orow = Popp + (size_t)j * G.pitch;
    if (!yin) {
        out = ldg4(orow + x0);
    } else {
        if constexpr (EX == 1) {
            if (x0 == 0) out.x = sign_l * __ldg(orow) + add_l;
        }
        if constexpr (EX == -1) {
            const int e = G.nx - 1 - x0;
            if (e >= 0 && e < 4) set_comp(out, e, sign_r * __ldg(orow + G.nx - 1) + add_r);
        }
    }
    return out;
}

// Collision + force + thermal collision of one node, in place.
// f[0..8]: D2Q9 populations (shifted: they sum to delta-rho, Eq. 33),
// g[0..4]: D2Q5 populations. Directions: f1..f4 = (1,0),(0,1),(-1,0),(0,-1),
// f5..f8 = (1,1),(-1,1),(-1,-1),(1,-1); g1..g4 as f1..f4.
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
    // Non-equilibrium parts (Eq. 34, m4_eq = -2 drho + 3 |u|^2), scaled.
    const float d3 = K.se36 * (e + 2.f * rho - 3.f * uu);
    const float d4 = K.snu4 * (pxx - (u * u - v * v));
    const float d5 = K.snu4 * (pxy - u * v);
    const float d6 = K.sq12 * (qx + u);
    const float d7 = K.sq12 * (qy + v);
    const float d8 = K.seps36 * (eps - rho + 3.f * uu);

    float theta = g[0] + g[1] + g[2] + g[3] + g[4];  // Eq. 41

    // Buoyancy force (Eqs. 26-27): F_i = 3 (e_i - u).G f_i_eq(rho0 = 1, u),
    // G = (0, gbeta (theta - theta_ref)).
    const float c3 = 3.f * K.gbeta * (theta - K.theta_ref);
    const float base = 1.f - 1.5f * uu;
    const float cv_m = c3 * (-v), cv_p = c3 * (1.f - v), cv_n = c3 * (-1.f - v);
    const float w1 = 1.f / 9.f, w5 = 1.f / 36.f;
    const float u3 = 3.f * u, v3 = 3.f * v, uu45 = 4.5f * u * u, vv45 = 4.5f * v * v;
    const float upv = u + v, umv = u - v;
    const float qp = base + 4.5f * upv * upv, qm = base + 4.5f * umv * umv;
    const float F0 = cv_m * (4.f / 9.f) * base;
    const float F1 = cv_m * w1 * (base + u3 + uu45);
    const float F2 = cv_p * w1 * (base + v3 + vv45);
    const float F3 = cv_m * w1 * (base - u3 + uu45);
    const float F4 = cv_n * w1 * (base - v3 + vv45);
    const float F5 = cv_p * w5 * (qp + 3.f * upv);
    const float F6 = cv_p * w5 * (qm - 3.f * umv);
    const float F7 = cv_n * w5 * (qp - 3.f * upv);
    const float F8 = cv_n * w5 * (qm + 3.f * umv);

    // f* = f - M^-1 S (m - m_eq) + F, with M^-1 = M^T diag(1/norm) (Eq. 28).
    f[0] = f[0] + 4.f * d3 - 4.f * d8 + F0;
    f[1] = f[1] + d3 - d4 + 2.f * d6 + 2.f * d8 + F1;
    f[2] = f[2] + d3 + d4 + 2.f * d7 + 2.f * d8 + F2;
    f[3] = f[3] + d3 - d4 - 2.f * d6 + 2.f * d8 + F3;
    f[4] = f[4] + d3 + d4 - 2.f * d7 + 2.f * d8 + F4;
    f[5] = f[5] - 2.f * d3 - d5 - d6 - d7 - d8 + F5;
    f[6] = f[6] - 2.f * d3 + d5 + d6 - d7 - d8 + F6;
    f[7] = f[7] - 2.f * d3 - d5 + d6 + d7 - d8 + F7;
    f[8] = f[8] - 2.f * d3 + d5 - d6 + d7 - d8 + F8;

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

__global__ void __launch_bounds__(kThreads) step_kernel(StepArgs A, StepConsts K) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    Geo G;
    G.nx = A.nx;
    G.ny = A.ny;
    G.pitch = A.pitch;
    G.wx = 1 << A.wx_log2;
    G.seg_lane = lane & (G.wx - 1);
    const int rows_per_warp = 32 >> A.wx_log2;
    const int j_raw = (blockIdx.y * (kThreads / 32) + warp) * rows_per_warp + (lane >> A.wx_log2);
    const int x0 = (blockIdx.x * G.wx + G.seg_lane) * 4;
    const bool row_ok = j_raw < A.ny;
    const int j = row_ok ? j_raw : A.ny - 1;
    const bool quad_ok = row_ok && x0 < A.nx;

    const float* S = A.src;
    const long long PL = A.plane;
    // Wall values for the left / right links (only the edge threads use them).
    float add_l_g = 0.f, add_r_g = 0.f;
    if (x0 == 0 && K.left_fixed) add_l_g = K.abb * __ldg(A.hot + j);
    if (x0 <= A.nx - 1 && A.nx - 1 < x0 + 4 && K.right_fixed) add_r_g = K.abb * __ldg(A.cold + j);
    const float sign_l_g = K.left_fixed ? -1.f : 1.f;
    const float sign_r_g = K.right_fixed ? -1.f : 1.f;

    // Pull-stream (opposites: 1<->3, 2<->4, 5<->7, 6<->8).
    float4 F[9], Gq[5];
    F[0] = pull<0, 0>(S + 0 * PL, S + 0 * PL, j, x0, G, 1.f, 0.f, 1.f, 0.f);
    F[1] = pull<1, 0>(S + 1 * PL, S + 3 * PL, j, x0, G, 1.f, 0.f, 1.f, 0.f);
    F[2] = pull<0, 1>(S + 2 * PL, S + 4 * PL, j, x0, G, 1.f, 0.f, 1.f, 0.f);
    F[3] = pull<-1, 0>(S + 3 * PL, S + 1 * PL, j, x0, G, 1.f, 0.f, 1.f, 0.f);
    F[4] = pull<0, -1>(S + 4 * PL, S + 2 * PL, j, x0, G, 1.f, 0.f, 1.f, 0.f);
    F[5] = pull<1, 1>(S + 5 * PL, S + 7 * PL, j, x0, G, 1.f, 0.f, 1.f, 0.f);
    F[6] = pull<-1, 1>(S + 6 * PL, S + 8 * PL, j, x0, G, 1.f, 0.f, 1.f, 0.f);
    F[7] = pull<-1, -1>(S + 7 * PL, S + 5 * PL, j, x0, G, 1.f, 0.f, 1.f, 0.f);
    F[8] = pull<1, -1>(S + 8 * PL, S + 6 * PL, j, x0, G, 1.f, 0.f, 1.f, 0.f);
    Gq[0] = pull<0, 0>(S + 9 * PL, S + 9 * PL, j, x0, G, 1.f, 0.f, 1.f, 0.f);
    Gq[1] = pull<1, 0>(S + 10 * PL, S + 12 * PL, j, x0, G, sign_l_g, add_l_g, 1.f, 0.f);
    Gq[2] = pull<0, 1>(S + 11 * PL, S + 13 * PL, j, x0, G, 1.f, 0.f, 1.f, 0.f);
    Gq[3] = pull<-1, 0>(S + 12 * PL, S + 10 * PL, j, x0, G, 1.f, 0.f, sign_r_g, add_r_g);
    Gq[4] = pull<0, -1>(S + 13 * PL, S + 11 * PL, j, x0, G, 1.f, 0.f, 1.f, 0.f);

    float theta4[4];
    bool bad = false;
    node_update<0>(F, Gq, K, theta4, quad_ok && x0 + 0 < A.nx, bad);
    node_update<1>(F, Gq, K, theta4, quad_ok && x0 + 1 < A.nx, bad);
    node_update<2>(F, Gq, K, theta4, quad_ok && x0 + 2 < A.nx, bad);
    node_update<3>(F, Gq, K, theta4, quad_ok && x0 + 3 < A.nx, bad);

    if (quad_ok) {
        float* D = A.dst + (size_t)j * A.pitch + x0;
#pragma unroll
        for (int k = 0; k < 9; ++k) *reinterpret_cast<float4*>(D + k * PL) = F[k];
#pragma unroll
        for (int k = 0; k < 5; ++k) *reinterpret_cast<float4*>(D + (9 + k) * PL) = Gq[k];
        if (bad) atomicOr(A.err, 1u);
    }

    // Hot-wall Nusselt number (Eqs. 18-19) from the pre-collision theta.
    if (blockIdx.x == 0) {
        const bool has_nu = row_ok && G.seg_lane == 0;
        if (has_nu) {
            const double tw = (double)__ldg(A.hot + j);
            A.nu_rows[j] = K.nu_scale * (8.0 * tw - 9.0 * (double)theta4[0] + (double)theta4[1]);
            __threadfence();
        }
        const unsigned n_here = __popc(__ballot_sync(kFull, has_nu));
        unsigned before = 0;
        if (lane == 0 && n_here) before = atomicAdd(A.counter, n_here);
        before = __shfl_sync(kFull, before, 0);
        if (n_here && before + n_here == (unsigned)A.ny) {
            // Last warp to report: sum the rows in a fixed order (lane-strided,
            // then a butterfly), so the result does not depend on arrival order.
            __threadfence();
            double s = 0.0;
            for (int r = lane; r < A.ny; r += 32) s += __ldcg(A.nu_rows + r);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
            if (lane == 0) {
                const double mean = s / (double)A.ny;
                const long long t = *A.d_step;
                A.nu_ring[t % A.cap] = mean;
                *A.nu_last = mean;
                *A.d_step = t + 1;
                *A.counter = 0u;
            }
        }
    }
}

}  // namespace dmrt
