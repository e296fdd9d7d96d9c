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
// One thread per node and reverse step. The transpose of the pull is itself a
// pull in the opposite direction: s_m(x) fed q_m(x + e_m), or, where x + e_m
// lies outside, the wall value of q_opp(m)(x) (sign -1 for anti-bounce-back).
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

// The reverse sweep of a segment of K steps (K even) replays one of two
// graphs, each of K / 2 pair nodes (reverse steps k and k - 1 in one launch)
// or K single-step nodes, and a fold node; graph s serves the segments whose
// recomputed states sit in slot set s, so a node's pre-wait addresses depend
// on s and on t, the step within the segment, only (with every state stored,
// on the segment q as well). q comes from a device counter (graph s reads
// counter s; its fold leaves q - 1 in the other); after the wait it selects
// the adjoint buffers and the averaging weight and skips the missing steps of
// a short last segment.
struct AdjArgs {
    const long long* seg;              // the segment q swept by this replay
    long long* seg_next;               // the fold writes q - 1 here (the other graph's counter)
    const float* slot[2];              // set s: s_{qK+t} at slot[s] + t * state (t = 0: the checkpoint's copy)
    const float* all;                  // every state stored (s_k at all + k * state), else null
    float* nu[2];                      // adjoint states: pair P reads nu[P & 1] (single steps: step k reads
                                       // nu[(N - k) & 1]) and writes the other
    const float* __restrict__ hot;
    const float* __restrict__ cold;
    double* dthw;                      // [ny] dJ/dtheta_w totals
    double* dgbeta;                    // [n_blocks] dJ/dgbeta totals, one per tile (block of the step grid)
    float* dthw_step;                  // [K][ny] nu_{k+1}[g east](0, j) by step (0: adiabatic hot wall)
    float2* dgbeta_step;               // [K][n_blocks][4] the segment's dJ/dgbeta by step and warp, as (hi, lo)
    long long state;                   // floats in one state
    long long K, N, C;                 // segment length, steps, segments
    long long w_from;                  // steps k > w_from carry the weight w (the averaging window)
    long long n_blocks;
    long long plane;
    int nsets;                         // slot sets: with 2, segment q uses set (C - 1 - q) & 1
    int nx, ny, pitch;
    int tw, hx;                        // output columns per tile and halo columns on each side
    int pairs;                         // 1: pair nodes (two steps per launch), 0: one step per launch
    float w;                           // w_k inside the averaging window
    float nu_wall, nu_next;            // dNu/dtheta at columns 0 and 1, divided by ny
};

// The half of the local Jacobian that depends on the pulled state only:
// velocity, temperature and, per direction i, the three factors of the force
// derivatives (F_i = 3 gbeta (theta - theta_ref)(e_iy - v) w_i P_i,
// P_i = 1 - 1.5 |u|^2 + 3 e_i.u + 4.5 (e_i.u)^2, Eqs. 26-27):
//   fu_i = (e_iy - v)(3 e_ix + 9 (e_i.u) e_ix - 3 u)       (d/du without w_i)
//   fv_i = (e_iy - v)(3 e_iy + 9 (e_i.u) e_iy - 3 v) - P_i  (d/dv)
//   fp_i = (e_iy - v) P_i                                  (d/dtheta, d/dgbeta)
struct VjpFwd {
    float u, v, th;
    float fu[9], fv[9], fp[9];
};

__device__ __forceinline__ VjpFwd vjp_forward(const float (&f)[9], const float (&g)[5]) {
    VjpFwd F;
    F.u = (f[1] - f[3]) + (f[5] - f[6]) - (f[7] - f[8]);
    F.v = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
    F.th = g[0] + g[1] + g[2] + g[3] + g[4];
    const float u = F.u, v = F.v;
    const float base = 1.f - 1.5f * (u * u + v * v);
    const int EXs[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const int EYs[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const float ex = (float)EXs[i], ey = (float)EYs[i];
        const float eu = ex * u + ey * v;
        const float P = base + 3.f * eu + 4.5f * eu * eu;
        const float dy = ey - v;
        F.fu[i] = dy * (3.f * ex + 9.f * eu * ex - 3.f * u);
        F.fv[i] = dy * (3.f * ey + 9.f * eu * ey - 3.f * v) - P;
        F.fp[i] = dy * P;
    }
    return F;
}

// The other half: nu = C'(q)^T lambda for the pulled state summarised by F.
__device__ __forceinline__ void collide_vjp(const VjpFwd& F, const float (&lf)[9], const float (&lg)[5],
                                            const StepConsts& K, float (&nf)[9], float (&ng)[5], float& dgb) {
    const float u = F.u, v = F.v, th = F.th;

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

    // Force derivatives contracted with lam_f.
    const float c3 = 3.f * K.gbeta * (th - K.theta_ref);
    const float Ws[9] = {4.f / 9.f, 1.f / 9.f, 1.f / 9.f, 1.f / 9.f, 1.f / 9.f,
                         1.f / 36.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f};
    float Fu = 0.f, Fv = 0.f, Fp = 0.f;  // Fp = sum lam_i (e_iy - v) w_i P_i
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const float lw = lf[i] * Ws[i];
        Fu += lw * F.fu[i];
        Fv += lw * F.fv[i];
        Fp += lw * F.fp[i];
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

// A node of the reverse step: its column i, row j, offset within a plane,
// whether it lies inside the cavity, and which of its four sides have a
// neighbour (the walls lie beyond the others).
struct AdjNode {
    int i, j, c0;
    bool in, xm, xp, ym, yp;
    __device__ __forceinline__ bool inside(int ex, int ey) const {
        return (ex > 0 ? xp : ex < 0 ? xm : true) && (ey > 0 ? yp : ey < 0 ? ym : true);
    }
};

// Column i (clamped to the last column when outside), row j (inside).
__device__ __forceinline__ AdjNode adj_node(const AdjArgs& A, int i, int j) {
    AdjNode n;
    n.i = i;
    n.j = j;
    n.in = i < A.nx;
    const int ic = n.in ? i : A.nx - 1;
    n.c0 = j * A.pitch + ic;  // a whole state has fewer than 2^31 values (checked on the host)
    n.xm = ic > 0;
    n.xp = ic + 1 < A.nx;
    n.ym = j > 0;
    n.yp = j + 1 < A.ny;
    return n;
}

// q_k at the node: the forward pull of s_{k-1} (the neighbour at x - e_m, or
// across a wall the wall rule on the node's own opposite).
__device__ __forceinline__ void adj_pull(const float* __restrict__ SP, const AdjNode& n, const AdjArgs& A,
                                         const StepConsts& K, float (&f)[9], float (&g)[5]) {
    const int EX9[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const int EY9[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    const int OP9[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
    const int OP5[5] = {0, 3, 4, 1, 2};
    const int PL = (int)A.plane, P = A.pitch, c0 = n.c0;
#pragma unroll
    for (int m = 0; m < 9; ++m) {
        const bool ok = n.inside(-EX9[m], -EY9[m]);
        f[m] = __ldg(SP + (ok ? plane_f(m) * PL + c0 - EX9[m] - EY9[m] * P : plane_f(OP9[m]) * PL + c0));
    }
    const float hw = __ldg(A.hot + n.j), cw = __ldg(A.cold + n.j);
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        const bool ok = n.inside(-EX9[m], -EY9[m]);
        const float v = __ldg(SP + (ok ? plane_g(m) * PL + c0 - EX9[m] - EY9[m] * P : plane_g(OP5[m]) * PL + c0));
        if (ok) g[m] = v;
        else if (EX9[m] > 0 && K.left_fixed) g[m] = K.abb * hw - v;   // x - e_m < 0
        else if (EX9[m] < 0 && K.right_fixed) g[m] = K.abb * cw - v;  // x - e_m >= nx
        else g[m] = v;
    }
}

// lambda_k: the transpose of the pull, gathered from nu_{k+1} in global
// memory: the neighbour at x + e_m, or across a wall the node's own opposite
// (bounce-back; sign -1 for anti-bounce-back of g).
__device__ __forceinline__ void adj_gather(const float* __restrict__ NI, const AdjNode& n, const AdjArgs& A,
                                           const StepConsts& K, float (&lf)[9], float (&lg)[5]) {
    const int EX9[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const int EY9[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    const int OP9[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
    const int OP5[5] = {0, 3, 4, 1, 2};
    const int PL = (int)A.plane, P = A.pitch, c0 = n.c0;
#pragma unroll
    for (int m = 0; m < 9; ++m) {
        const bool ok = n.inside(EX9[m], EY9[m]);
        lf[m] = __ldg(NI + (ok ? plane_f(m) * PL + c0 + EX9[m] + EY9[m] * P : plane_f(OP9[m]) * PL + c0));
    }
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        const bool ok = n.inside(EX9[m], EY9[m]);
        const float val = __ldg(NI + (ok ? plane_g(m) * PL + c0 + EX9[m] + EY9[m] * P : plane_g(OP5[m]) * PL + c0));
        const bool fixed = !ok && ((EX9[m] < 0 && K.left_fixed) || (EX9[m] > 0 && K.right_fixed));
        lg[m] = fixed ? -val : val;  // anti-bounce-back (Eq. 45) / bounce-back (Eq. 44)
    }
}

// dJ/dgbeta: each warp's sum by a butterfly in float32 pairs (hi, lo) carrying
// the rounding error of every addition (Knuth's two-sum), so the pair holds the
// sum to about float64 accuracy without the float64 pipe, which is slow on this
// GPU; the pair goes to the slot of step t, tile `tile` and the warp's place in
// its 128-lane row, and adjoint_fold_kernel adds the slots in a fixed order, so
// every run gives the same bits. (Lanes combine commutatively, so every lane
// ends with the same pair.)
__device__ __forceinline__ void adj_dgb_store(float dgb, int t, long long tile, const AdjArgs& A) {
    float hi = dgb, lo = 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(kFull, hi, o), l2 = __shfl_xor_sync(kFull, lo, o);
        const float sum = hi + h2, bp = sum - hi;
        const float err = (hi - (sum - bp)) + (h2 - bp);
        hi = sum;
        lo = (lo + l2) + err;
    }
    if ((threadIdx.x & 31) == 0)
        A.dgbeta_step[((size_t)t * A.n_blocks + tile) * 4 + ((threadIdx.x >> 5) & 3)] = make_float2(hi, lo);
}

// ---- two reverse steps per launch ---------------------------------------------
// Pair node: reverse steps k_hi = qK + th + 1 and k_lo = k_hi - 1 (th odd) of a
// tile of tw columns of row j. Step k_hi runs at rows j - 1, j, j + 1 and at
// the tile's columns plus hx halo columns on each side (384 threads: 128
// lanes by 3 rows), with nu_{k_hi + 1} gathered from global memory; its
// output nu_{k_hi} stays in shared memory, where step k_lo (the middle row's
// output lanes) gathers it; only nu_{k_lo} goes to global memory. So the
// launch boundary, and its dependency wait, comes once every two steps, at
// the price of computing step k_hi on the halo as well. Pair P (P-th of the
// sweep, counted from the end) reads nu[P & 1] and writes nu[(P + 1) & 1].
// When the last segment has an odd length its first pair begins with the
// step after the last (k_hi = N + 1): that step is skipped and its output is
// nu_{N+1} = 0.
constexpr int kPairThreads = 384;

__device__ __forceinline__ int pair_smem_index(int row, int plane, int lane) { return (row * kPlanes + plane) * 128 + lane; }

// lambda at the middle-row node (lane l) gathered from nu_{k_hi} in shared memory.
__device__ __forceinline__ void adj_gather_smem(const float* __restrict__ S, int l, const AdjNode& n,
                                                const StepConsts& K, float (&lf)[9], float (&lg)[5]) {
    const int EX9[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const int EY9[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    const int OP9[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
    const int OP5[5] = {0, 3, 4, 1, 2};
#pragma unroll
    for (int m = 0; m < 9; ++m) {
        const bool ok = n.inside(EX9[m], EY9[m]);
        lf[m] = S[ok ? pair_smem_index(1 + EY9[m], plane_f(m), l + EX9[m]) : pair_smem_index(1, plane_f(OP9[m]), l)];
    }
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        const bool ok = n.inside(EX9[m], EY9[m]);
        const float val =
            S[ok ? pair_smem_index(1 + EY9[m], plane_g(m), l + EX9[m]) : pair_smem_index(1, plane_g(OP5[m]), l)];
        const bool fixed = !ok && ((EX9[m] < 0 && K.left_fixed) || (EX9[m] > 0 && K.right_fixed));
        lg[m] = fixed ? -val : val;  // anti-bounce-back (Eq. 45) / bounce-back (Eq. 44)
    }
}

// nu_k at a node from lambda_k and the forward half, with the Nusselt source
// of step k (weight wk) on columns 0 and 1; returns the node's dJ/dgbeta term.
__device__ __forceinline__ float adj_node_step(const VjpFwd& F, const float (&lf)[9], const float (&lg)[5],
                                               const AdjNode& n, float wk, const AdjArgs& A, const StepConsts& K,
                                               float (&nf)[9], float (&ng)[5]) {
    float dgb;
    collide_vjp(F, lf, lg, K, nf, ng, dgb);
    if (wk != 0.f) {
        // Nu(k) = (1/ny) sum_j scale (8 theta_w - 9 theta(0, j) + theta(1, j)), theta = sum g.
        const float add = n.i == 0 ? wk * A.nu_wall : (n.i == 1 ? wk * A.nu_next : 0.f);
#pragma unroll
        for (int m = 0; m < 5; ++m) ng[m] += add;
    }
    return dgb;
}

// ALL: every forward state is stored (s_{qK+t} at all + (qK + t) * state);
// else the segment's states are in slot set `set`.
template <bool ALL>
__global__ void __launch_bounds__(kPairThreads) adjoint_pair_kernel(AdjArgs A, int set, int th, StepConsts K) {
    // Launched programmatically after the previous pair, which writes neither
    // s_{k_hi - 1}, s_{k_lo - 1} (slots th, th - 1 of this graph's set, filled
    // before the replay began, or stored states) nor the segment counter (set
    // by the previous replay's fold): these are read, and the forward halves
    // computed, before waiting for that pair (grid_dep_wait), so their latency
    // overlaps it. nu is read, and anything written, after the wait.
    __shared__ float S[3 * kPlanes * 128];
    grid_dep_launch();
    const int tid = threadIdx.x, l = tid & 127, rr = tid >> 7;  // lane; row j - 1, j, j + 1
    const int j = blockIdx.y, jr = j + rr - 1;
    const int x = blockIdx.x * A.tw - A.hx + l;
    const bool col_ok = x >= 0 && x < A.nx;
    const bool act = col_ok && jr >= 0 && jr < A.ny;                 // step k_hi here
    const bool out = rr == 1 && col_ok && l >= A.hx && l < A.hx + A.tw;  // step k_lo here
    const AdjNode n = adj_node(A, col_ok ? x : A.nx, act ? jr : j);      // (x, jr); clamped when inactive
    const long long q = *A.seg;
    const float* base = ALL ? A.all + q * A.K * A.state : A.slot[set];  // s_{qK}
    VjpFwd F1, F2;
    {
        float f[9], g[5];
        adj_pull(base + th * A.state, n, A, K, f, g);  // s_{k_hi - 1}
        F1 = vjp_forward(f, g);
        if (out) {
            adj_pull(base + (th - 1) * A.state, n, A, K, f, g);  // s_{k_lo - 1}
            F2 = vjp_forward(f, g);
        }
    }
    grid_dep_wait();
    const long long k_hi = q * A.K + th + 1, k_lo = k_hi - 1;
    if (k_lo > A.N) return;  // the last segment may be short
    const long long P = (A.N + 1 - k_hi) / 2;
    const float* __restrict__ NI = A.nu[P & 1];  // nu_{k_hi + 1}
    float* __restrict__ NO = A.nu[(P + 1) & 1];  // nu_{k_lo}
    const int PL = (int)A.plane;
    const long long tile = (long long)blockIdx.y * gridDim.x + blockIdx.x;
    const bool hi_real = k_hi <= A.N;

    // Step k_hi on the 3-row window: nu_{k_hi} into shared memory.
    float dgb1 = 0.f;
    if (act) {
        float nf[9], ng[5];
        if (hi_real) {
            float lf[9], lg[5];
            adj_gather(NI, n, A, K, lf, lg);
            dgb1 = adj_node_step(F1, lf, lg, n, k_hi > A.w_from ? A.w : 0.f, A, K, nf, ng);
            if (out && x == 0)
                A.dthw_step[(size_t)th * A.ny + j] = K.left_fixed ? __ldg(NI + plane_g(1) * PL + j * A.pitch) : 0.f;
        } else {
#pragma unroll
            for (int m = 0; m < 9; ++m) nf[m] = 0.f;  // nu_{N+1} = 0
#pragma unroll
            for (int m = 0; m < 5; ++m) ng[m] = 0.f;
        }
#pragma unroll
        for (int m = 0; m < 9; ++m) S[pair_smem_index(rr, plane_f(m), l)] = nf[m];
#pragma unroll
        for (int m = 0; m < 5; ++m) S[pair_smem_index(rr, plane_g(m), l)] = ng[m];
    }
    __syncthreads();
    if (rr != 1) return;  // the halo rows are done

    // Step k_lo at the middle row's output lanes: nu_{k_lo} to global memory.
    float dgb2 = 0.f;
    if (out) {
        float lf[9], lg[5], nf[9], ng[5];
        adj_gather_smem(S, l, n, K, lf, lg);
        dgb2 = adj_node_step(F2, lf, lg, n, k_lo > A.w_from ? A.w : 0.f, A, K, nf, ng);
        if (x == 0) A.dthw_step[(size_t)(th - 1) * A.ny + j] = K.left_fixed ? S[pair_smem_index(1, plane_g(1), l)] : 0.f;
        float* D = NO + n.c0;
#pragma unroll
        for (int m = 0; m < 9; ++m) D[plane_f(m) * PL] = nf[m];
#pragma unroll
        for (int m = 0; m < 5; ++m) D[plane_g(m) * PL] = ng[m];
    }
    if (hi_real) adj_dgb_store(out ? dgb1 : 0.f, th, tile, A);
    adj_dgb_store(dgb2, th - 1, tile, A);
}

// ---- one reverse step per launch ------------------------------------------------
// For cavities large enough to fill the GPU, where the pair's halo rows would
// be extra work rather than idle SMs put to use: step k = qK + t + 1 at a
// tile of 128 columns of row j, nu_{k+1} from global memory, nu_k to it.
template <bool ALL>
__global__ void __launch_bounds__(128) adjoint_step_kernel(AdjArgs A, int set, int t, StepConsts K) {
    // As in the pair kernel: s_{k-1} and the segment counter before the wait,
    // nu and every write after it.
    grid_dep_launch();
    const long long q = *A.seg;
    const float* base = ALL ? A.all + q * A.K * A.state : A.slot[set];
    const AdjNode n = adj_node(A, blockIdx.x * 128 + threadIdx.x, blockIdx.y);
    VjpFwd F;
    {
        float f[9], g[5];
        adj_pull(base + t * A.state, n, A, K, f, g);
        F = vjp_forward(f, g);
    }
    grid_dep_wait();
    const long long k = q * A.K + t + 1;
    if (k > A.N) return;  // the last segment may be short
    const float* __restrict__ NI = A.nu[(A.N - k) & 1];  // nu_{k+1}
    float* __restrict__ NO = A.nu[(A.N - k + 1) & 1];    // nu_k
    const int PL = (int)A.plane;
    float dgb = 0.f;
    if (n.in) {
        float lf[9], lg[5], nf[9], ng[5];
        adj_gather(NI, n, A, K, lf, lg);
        dgb = adj_node_step(F, lf, lg, n, k > A.w_from ? A.w : 0.f, A, K, nf, ng);
        if (n.i == 0)
            A.dthw_step[(size_t)t * A.ny + n.j] = K.left_fixed ? __ldg(NI + plane_g(1) * PL + n.j * A.pitch) : 0.f;
        float* D = NO + n.c0;
#pragma unroll
        for (int m = 0; m < 9; ++m) D[plane_f(m) * PL] = nf[m];
#pragma unroll
        for (int m = 0; m < 5; ++m) D[plane_g(m) * PL] = ng[m];
    }
    adj_dgb_store(dgb, t, (long long)blockIdx.y * gridDim.x + blockIdx.x, A);
}

// After a segment's reverse steps: add the segment's dJ/dgbeta terms (per block
// of the step grid) and dJ/dtheta_w terms (per row) to the totals, in float64,
// one warp per slot: lane l sums the steps t = l, l + 32, ... in turn, a
// butterfly adds the lanes, and lane 0 adds the result to the total; then the
// next segment goes to the other graph's counter. Fixed order, same bits on
// every run.
constexpr int kFoldThreads = 256;

__global__ void __launch_bounds__(kFoldThreads) adjoint_fold_kernel(AdjArgs A, StepConsts K) {
    const long long q = *A.seg;
    const int len = (int)min(A.K, A.N - q * A.K);
    const long long s = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (s < A.n_blocks + A.ny) {
        double acc = 0.0;
        if (s < A.n_blocks) {
#pragma unroll 4
            for (int t = lane; t < len; t += 32) {
                const float2* w = A.dgbeta_step + ((size_t)t * A.n_blocks + s) * 4;  // the block's four warps
                const float2 w0 = w[0], w1 = w[1], w2 = w[2], w3 = w[3];
                acc += (((double)w0.x + (double)w0.y) + ((double)w1.x + (double)w1.y)) +
                       (((double)w2.x + (double)w2.y) + ((double)w3.x + (double)w3.y));
            }
        } else {
            const long long r = s - A.n_blocks;
#pragma unroll 4
            for (int t = lane; t < len; t += 32) acc += (double)K.abb * (double)A.dthw_step[(size_t)t * A.ny + r];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
        if (lane == 0) {
            if (s < A.n_blocks) A.dgbeta[s] += acc;
            else A.dthw[s - A.n_blocks] += acc;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *A.seg_next = q - 1;
}

// The anti-bounce-back term of step 1 (after the sweep): q_east(0, j) =
// abb theta_w(j) - s_west(0, j) feeds dJ/dtheta_w(j) with abb nu_1[g east](0, j).
// nu_1 is the output of the sweep's last pair, P = (N - 1) / 2, or of step 1.
__global__ void adjoint_gather_kernel(AdjArgs A, StepConsts K) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const float* nu1 = A.pairs ? A.nu[((A.N - 1) / 2 + 1) & 1] : A.nu[A.N & 1];
    if (j < A.ny && K.left_fixed) A.dthw[j] += (double)K.abb * (double)nu1[plane_g(1) * A.plane + (long long)j * A.pitch];
}

}  // namespace dmrt
