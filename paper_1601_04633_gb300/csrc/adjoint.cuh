// Discrete adjoint of the double-MRT step (reverse collide-stream), sm_103a.
//
// Forward step k (s = post-collision state, q = pulled state):
//   q_k = P(s_{k-1}; theta_w)   pull with bounce-back / anti-bounce-back (Eqs. 25, 36, 44, 45)
//   s_k = C(q_k; gbeta)          collision + force per node (Eqs. 26-43)
//   Nu(k) from q_k               (Eqs. 18-19)
// Objective J = sum_k w_k Nu(k). Reverse step k (k = N .. 1):
//   lambda_k = P^T-gather of nu_{k+1}       (adjoint of s_k; nu_{N+1} = 0)
//   nu_k     = C'(q_k)^T lambda_k + w_k dNu(k)/dq_k
//   dJ/dgbeta += lambda_k . dC/dgbeta;  dJ/dtheta_w(j) += abb * nu_{k+1}[g east](0, j)
// One thread per node. The transpose of the pull is itself a pull in the
// opposite direction: s_m(x) fed q_m(x + e_m), or, where x + e_m lies outside,
// the wall value of q_opp(m)(x) (sign -1 for anti-bounce-back).
//
// The transposed local Jacobian is written out in closed form. With
// S' = diag(rates / row norms) and A = I - M^T S' M (symmetric),
//   f* = A f + M^T S' m_eq(rho, u) + F(u, theta, gbeta),
//   g* = B g + N^T Q' n_eq(theta, u),   B = I - N^T Q' N (symmetric),
// so, with kappa = S' M lam_f and eta = Q' N lam_g,
//   nu_f = lam_f - M^T kappa + kappa_rho + e_x (kappa_u + F_u + theta eta_1)
//                                        + e_y (kappa_v + F_v + theta eta_2)
//   nu_g = lam_g - N^T eta + (u eta_1 + v eta_2 + a eta_3) + F_theta
// where kappa_rho, kappa_u, kappa_v are kappa contracted with dm_eq/d(rho, u, v)
// (Eq. 34) and F_u, F_v, F_theta the force derivatives contracted with lam_f.
#pragma once
#include "lattice.cuh"

namespace dmrt {

struct AdjArgs {
    const float* __restrict__ s_prev;  // s_{k-1}
    const float* __restrict__ nu_in;   // nu_{k+1}
    float* __restrict__ nu_out;        // nu_k
    const float* __restrict__ hot;
    const float* __restrict__ cold;
    double* dthw;                      // [ny] dJ/dtheta_w, accumulated (the final gather only)
    double* dthw_step;                 // [ny] this step's dJ/dtheta_w terms (written, not accumulated)
    double* dgbeta_step;               // this step's dJ/dgbeta per warp: [gridDim.y][gridDim.x][4]
    long long plane;
    int nx, ny, pitch;
    float w;                           // w_k (0 outside the averaging window)
    float nu_wall, nu_next;            // dNu/dtheta at columns 0 and 1, divided by ny
    int gather_only;                   // only the anti-bounce-back term of nu_in
};

__device__ __forceinline__ void collide_vjp(const float (&f)[9], const float (&g)[5], const float (&lf)[9],
                                            const float (&lg)[5], const StepConsts& K, float (&nf)[9],
                                            float (&ng)[5], float& dgb) {
    // Forward quantities of the pulled state.
    const float u = (f[1] - f[3]) + (f[5] - f[6]) - (f[7] - f[8]);
    const float v = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
    const float th = g[0] + g[1] + g[2] + g[3] + g[4];
    const float uu = u * u + v * v;
    const float base = 1.f - 1.5f * uu;

    // kappa = S' M lam_f (the conserved rows do not contribute).
    const float a13 = lf[1] - lf[3], a24 = lf[2] - lf[4];
    const float s13 = lf[1] + lf[3], s24 = lf[2] + lf[4];
    const float a56 = lf[5] - lf[6], a78 = lf[7] - lf[8];
    const float s56 = lf[5] + lf[6], s78 = lf[7] + lf[8];
    const float s1234 = s13 + s24, s5678 = s56 + s78;
    const float k3 = K.se36 * (-4.f * lf[0] - s1234 + 2.f * s5678);
    const float k4 = K.snu4 * (s13 - s24);
    const float k5 = K.snu4 * ((lf[5] + lf[7]) - (lf[6] + lf[8]));
    const float k6 = K.sq12 * (-2.f * a13 + a56 - a78);
    const float k7 = K.sq12 * (-2.f * a24 + s56 - s78);
    const float k8 = K.seps36 * (4.f * lf[0] - 2.f * s1234 + s5678);
    // kappa contracted with dm_eq/d(rho, u, v), Eq. 34 (rho0 = 1).
    const float kr = -2.f * k3 + k8;
    const float ku = 6.f * u * k3 + 2.f * u * k4 + v * k5 - k6 - 6.f * u * k8;
    const float kv = 6.f * v * k3 - 2.f * v * k4 + u * k5 - k7 - 6.f * v * k8;

    // Force F_i = 3 gbeta (theta - theta_ref)(e_iy - v) w_i P_i,
    // P_i = 1 - 1.5 |u|^2 + 3 e_i.u + 4.5 (e_i.u)^2 (Eqs. 26-27).
    const float c3 = 3.f * K.gbeta * (th - K.theta_ref);
    const int EXs[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const int EYs[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    const float Ws[9] = {4.f / 9.f, 1.f / 9.f, 1.f / 9.f, 1.f / 9.f, 1.f / 9.f,
                         1.f / 36.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f};
    float Fu = 0.f, Fv = 0.f, Fp = 0.f;  // Fp = sum lam_i (e_iy - v) w_i P_i
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const float ex = (float)EXs[i], ey = (float)EYs[i];
        const float eu = ex * u + ey * v;
        const float P = base + 3.f * eu + 4.5f * eu * eu;
        const float lw = lf[i] * Ws[i];
        const float dy = ey - v;
        Fu += lw * dy * (3.f * ex + 9.f * eu * ex - 3.f * u);
        Fv += lw * (dy * (3.f * ey + 9.f * eu * ey - 3.f * v) - P);
        Fp += lw * dy * P;
    }
    Fu *= c3;
    Fv *= c3;
    const float Fth = 3.f * K.gbeta * Fp;
    dgb = 3.f * (th - K.theta_ref) * Fp;

    // eta = Q' N lam_g; N^T eta pattern as in the forward D2Q5 update.
    const float e1 = K.sk2 * (lg[1] - lg[3]);
    const float e2 = K.sk2 * (lg[2] - lg[4]);
    const float e3 = K.se20 * (-4.f * lg[0] + (lg[1] + lg[2] + lg[3] + lg[4]));
    const float e4 = K.snu4t * ((lg[1] + lg[3]) - (lg[2] + lg[4]));

    const float cx = ku + Fu + th * e1;
    const float cy = kv + Fv + th * e2;
    nf[0] = lf[0] + 4.f * k3 - 4.f * k8 + kr;
    nf[1] = lf[1] + k3 - k4 + 2.f * k6 + 2.f * k8 + kr + cx;
    nf[2] = lf[2] + k3 + k4 + 2.f * k7 + 2.f * k8 + kr + cy;
    nf[3] = lf[3] + k3 - k4 - 2.f * k6 + 2.f * k8 + kr - cx;
    nf[4] = lf[4] + k3 + k4 - 2.f * k7 + 2.f * k8 + kr - cy;
    nf[5] = lf[5] - 2.f * k3 - k5 - k6 - k7 - k8 + kr + cx + cy;
    nf[6] = lf[6] - 2.f * k3 + k5 + k6 - k7 - k8 + kr - cx + cy;
    nf[7] = lf[7] - 2.f * k3 - k5 + k6 + k7 - k8 + kr - cx - cy;
    nf[8] = lf[8] - 2.f * k3 + k5 - k6 + k7 - k8 + kr + cx - cy;

    const float cg = u * e1 + v * e2 + K.a * e3 + Fth;
    ng[0] = lg[0] + 4.f * e3 + cg;
    ng[1] = lg[1] - e1 - e3 - e4 + cg;
    ng[2] = lg[2] - e2 - e3 + e4 + cg;
    ng[3] = lg[3] + e1 - e3 - e4 + cg;
    ng[4] = lg[4] + e2 - e3 + e4 + cg;
}

__global__ void __launch_bounds__(128) adjoint_step_kernel(AdjArgs A, StepConsts K) {
    grid_dep_wait();  // launched programmatically after the previous kernel of the sweep
    grid_dep_launch();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    const bool in = i < A.nx;
    const int ic = in ? i : A.nx - 1;
    const long long PL = A.plane;
    const int EX9[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const int EY9[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    const int OP9[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
    const int OP5[5] = {0, 3, 4, 1, 2};
    const float abb = K.abb;

    if (A.gather_only) {
        // Anti-bounce-back on the hot wall: q_east(0, j) = abb theta_w(j) - s_west(0, j).
        if (in && i == 0 && K.left_fixed)
            A.dthw[j] += (double)abb * (double)__ldg(A.nu_in + plane_g(1) * PL + (long long)j * A.pitch);
        return;
    }

    // Offsets within a plane of this node and of its neighbours, and which of
    // the four sides have a neighbour (the walls lie beyond the others).
    const long long c0 = (long long)j * A.pitch + ic;
    const long long P = A.pitch;
    const bool xm = ic > 0, xp = ic + 1 < A.nx, ym = j > 0, yp = j + 1 < A.ny;
    auto inside = [&](int ex, int ey) {
        return (ex > 0 ? xp : ex < 0 ? xm : true) && (ey > 0 ? yp : ey < 0 ? ym : true);
    };
    const float* __restrict__ NI = A.nu_in;
    const float* __restrict__ SP = A.s_prev;

    // lambda_k: transpose of the pull, gathered from nu_{k+1}: the neighbour at
    // x + e_m, or across a wall the node's own opposite (bounce-back; sign -1
    // for anti-bounce-back of g).
    float lf[9], lg[5];
#pragma unroll
    for (int m = 0; m < 9; ++m) {
        const bool ok = inside(EX9[m], EY9[m]);
        lf[m] = __ldg(NI + (ok ? plane_f(m) * PL + c0 + EX9[m] + EY9[m] * P : plane_f(OP9[m]) * PL + c0));
    }
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        const bool ok = inside(EX9[m], EY9[m]);
        const float val = __ldg(NI + (ok ? plane_g(m) * PL + c0 + EX9[m] + EY9[m] * P : plane_g(OP5[m]) * PL + c0));
        const bool fixed = !ok && ((EX9[m] < 0 && K.left_fixed) || (EX9[m] > 0 && K.right_fixed));
        lg[m] = fixed ? -val : val;  // anti-bounce-back (Eq. 45) / bounce-back (Eq. 44)
    }
    // This step's anti-bounce-back term of dJ/dtheta_w(j) (0 for an adiabatic
    // hot wall): written into the step's own row, summed after the segment in
    // step order, so no read-modify-write sits at the end of every step.
    if (in && i == 0)
        A.dthw_step[j] = K.left_fixed ? (double)abb * (double)__ldg(NI + plane_g(1) * PL + (long long)j * A.pitch) : 0.0;

    // q_k at this node: the forward pull of s_{k-1} (the neighbour at x - e_m,
    // or across a wall the wall rule on the node's own opposite).
    float f[9], g[5];
#pragma unroll
    for (int m = 0; m < 9; ++m) {
        const bool ok = inside(-EX9[m], -EY9[m]);
        f[m] = __ldg(SP + (ok ? plane_f(m) * PL + c0 - EX9[m] - EY9[m] * P : plane_f(OP9[m]) * PL + c0));
    }
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        const bool ok = inside(-EX9[m], -EY9[m]);
        const float v = __ldg(SP + (ok ? plane_g(m) * PL + c0 - EX9[m] - EY9[m] * P : plane_g(OP5[m]) * PL + c0));
        if (ok) g[m] = v;
        else if (EX9[m] > 0 && K.left_fixed) g[m] = abb * __ldg(A.hot + j) - v;     // x - e_m < 0
        else if (EX9[m] < 0 && K.right_fixed) g[m] = abb * __ldg(A.cold + j) - v;   // x - e_m >= nx
        else g[m] = v;
    }

    float nf[9], ng[5], dgb;
    collide_vjp(f, g, lf, lg, K, nf, ng, dgb);
    if (A.w != 0.f) {
        // Nu(k) = (1/ny) sum_j scale (8 theta_w - 9 theta(0, j) + theta(1, j)), theta = sum g.
        const float add = i == 0 ? A.w * A.nu_wall : (i == 1 ? A.w * A.nu_next : 0.f);
#pragma unroll
        for (int m = 0; m < 5; ++m) ng[m] += add;
    }
    if (in) {
        float* D = A.nu_out + (long long)j * A.pitch + i;
#pragma unroll
        for (int m = 0; m < 9; ++m) D[plane_f(m) * PL] = nf[m];
#pragma unroll
        for (int m = 0; m < 5; ++m) D[plane_g(m) * PL] = ng[m];
    }
    // dJ/dgbeta: each warp's sum in fp64 by a butterfly, written to the warp's
    // slot of this step; after the segment, each block's four warp sums are
    // added in order and the result to the block's total in step order
    // (adjoint_fold_kernel), so every run gives the same bits.
    // (Each warp writes its own slot; the fold adds a block's four warps in order.)
    double d = in ? (double)dgb : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(kFull, d, o);
    if ((threadIdx.x & 31) == 0)
        A.dgbeta_step[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 4 + (threadIdx.x >> 5)] = d;
}

// After a segment's reverse steps: add each step's per-block dJ/dgbeta and per-row
// dJ/dtheta_w terms to the totals, the segment's last step first (the order in
// which the steps ran), one thread per slot.
__global__ void adjoint_fold_kernel(double* __restrict__ dgbeta, const double* __restrict__ dgbeta_steps,
                                    long long n_blocks, double* __restrict__ dthw,
                                    const double* __restrict__ dthw_steps, int ny, int len) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q < n_blocks) {
        double acc = dgbeta[q];
        for (int t = len - 1; t >= 0; --t) {
            const double* w = dgbeta_steps + ((size_t)t * n_blocks + q) * 4;  // the block's four warps
            acc += ((w[0] + w[1]) + w[2]) + w[3];
        }
        dgbeta[q] = acc;
    }
    if (q < ny) {
        double acc = dthw[q];
        for (int t = len - 1; t >= 0; --t) acc += dthw_steps[(size_t)t * ny + q];
        dthw[q] = acc;
    }
}

}  // namespace dmrt
