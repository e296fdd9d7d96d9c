// Fused double-MRT time step, direct-load variant (sm_103a).
//
// One thread owns four consecutive nodes of one row and moves them with 128-bit
// loads and stores straight from/to global memory; the x +- 1 shifts of the
// pull are warp shuffles inside a row segment of WX lanes, and only the
// segment's edge lanes read one halo value from memory. Used for grids too
// small for the TMA tiles, and kept as a comparison point for the TMA kernel.
//
// Stage order per node (Sec. 3): pull-stream f (Eq. 25) and g (Eq. 36) with the
// walls (bounce-back, Eq. 44; anti-bounce-back, Eq. 45), moments (Eqs. 33, 41),
// D2Q9 MRT + force (Eqs. 26-34), D2Q5 MRT (Eqs. 36-43), store, Nusselt (Eqs. 18-19).
#pragma once
#include "lattice.cuh"

namespace dmrt {

constexpr int kDirectThreads = 128;  // 4 warps per block

struct Geo {
    int nx, ny, pitch, wx, seg_lane;
    int row0, wall_lo, wall_hi;  // see StepArgs
    long long plane;             // elements per plane (bounds-checked builds)
    unsigned* err;
};

// Pull-stream of one plane for the four nodes (x0..x0+3, j): the value at node
// x is the post-collision value of the same plane at x - e. Links that leave
// through the top or bottom wall take the node's own opposite population
// (no-slip bounce-back; Eq. 44 for g). Links that leave through the left/right
// walls take  sign * opposite + add  (bounce-back: 1, 0; anti-bounce-back,
// Eq. 45: -1, 2 sqrt(3) alpha theta_w).
// Two phases, so that all 14 loads are issued before the first is used.
struct PlaneLoad {
    float4 v;
    float edge;
};

template <int EX, int EY>
__device__ __forceinline__ void pull_load(const float* __restrict__ P, const float* __restrict__ Popp,
                                          int j, int x0, int right_e, const Geo& G, PlaneLoad& L) {
    const int r = j - EY;
    const bool yin = (r >= 0 || !G.wall_lo) && (r < G.ny || !G.wall_hi);
    // Source row: row r of plane P, or across a top/bottom wall the node's own
    // row of the opposite plane (bounce-back). Offsets are within one plane.
    const long long oo = (long long)(j + G.row0) * G.pitch;
    const long long ro = yin ? (long long)(r + G.row0) * G.pitch : oo;
    const float* orow = Popp + oo;
    const float* row = (yin ? P : Popp) + ro;
    L.v = DMRT_IN(ro + x0, 0, G.plane - 3, G.err) ? ldg4(row + x0) : make_float4(0.f, 0.f, 0.f, 0.f);
    L.edge = 0.f;
    if constexpr (EX == 1) {
        if (yin && x0 == 0) {
            if (DMRT_IN(oo, 0, G.plane, G.err)) L.edge = __ldg(orow);    // wall partner
        } else if (yin && G.seg_lane == 0) {
            if (DMRT_IN(ro + x0 - 1, 0, G.plane, G.err)) L.edge = __ldg(row + x0 - 1);  // halo
        }
    }
    if constexpr (EX == -1) {
        if (yin && right_e >= 0 && right_e < 4) {
            if (DMRT_IN(oo + G.nx - 1, 0, G.plane, G.err)) L.edge = __ldg(orow + G.nx - 1);
        } else if (yin && G.seg_lane == G.wx - 1 && x0 + 4 < G.pitch) {
            if (DMRT_IN(ro + x0 + 4, 0, G.plane, G.err)) L.edge = __ldg(row + x0 + 4);
        }
    }
}

template <int EX, int EY>
__device__ __forceinline__ float4 pull_finish(const PlaneLoad& L, int j, int x0, int right_e,
                                              const Geo& G, float sign_l, float add_l,
                                              float sign_r, float add_r) {
    const int r = j - EY;
    const bool yin = (r >= 0 || !G.wall_lo) && (r < G.ny || !G.wall_hi);
    const float4 v = L.v;
    float4 out;
    if constexpr (EX == 0) {
        out = v;
    } else if constexpr (EX == 1) {
        float left = __shfl_up_sync(kFull, v.w, 1, G.wx);
        if (G.seg_lane == 0) left = L.edge;
        out = make_float4(left, v.x, v.y, v.z);
        if (yin && x0 == 0) out.x = sign_l * L.edge + add_l;
    } else {
        float right = __shfl_down_sync(kFull, v.x, 1, G.wx);
        if (G.seg_lane == G.wx - 1) right = L.edge;
        out = make_float4(v.y, v.z, v.w, right);
        if (yin && right_e >= 0 && right_e < 4) set_comp(out, right_e, sign_r * L.edge + add_r);
    }
    return yin ? out : v;
}

// The nodes of tile (bx, by) of the direct grid: 128 threads (4 warps), each
// with four consecutive nodes of one row; rows of WX lanes per warp segment.
__device__ __forceinline__ void direct_tile(const StepArgs& A, const StepConsts& K, int bx, int by) {
    const int lane = threadIdx.x & 31;
    const int warp = (threadIdx.x & (kDirectThreads - 1)) >> 5;
    Geo G;
    G.nx = A.nx;
    G.ny = A.ny;
    G.pitch = A.pitch;
    G.row0 = A.row0;
    G.wall_lo = A.wall_lo;
    G.wall_hi = A.wall_hi;
    G.plane = A.plane;
    G.err = A.err;
    G.wx = 1 << A.wx_log2;
    G.seg_lane = lane & (G.wx - 1);
    const int rows_per_warp = 32 >> A.wx_log2;
    const int j_raw = (by * (kDirectThreads / 32) + warp) * rows_per_warp + (lane >> A.wx_log2);
    const int x0 = (bx * G.wx + G.seg_lane) * 4;
    const bool row_ok = j_raw < A.ny;
    const int j = row_ok ? j_raw : A.ny - 1;
    const bool quad_ok = row_ok && x0 < A.nx;

    const float* S = A.src;
    const long long PL = A.plane;
    float add_l_g = 0.f, add_r_g = 0.f;
    const bool j_in = DMRT_IN(j, 0, A.ny, A.err);
    if (x0 == 0 && K.left_fixed && j_in) add_l_g = K.abb * __ldg(A.hot + j);
    if (x0 <= A.nx - 1 && A.nx - 1 < x0 + 4 && K.right_fixed && j_in) add_r_g = K.abb * __ldg(A.cold + j);
    const float sign_l_g = K.left_fixed ? -1.f : 1.f;
    const float sign_r_g = K.right_fixed ? -1.f : 1.f;

    // Opposites: 1<->3, 2<->4, 5<->7, 6<->8 (0-based directions).
    const int right_e = A.nx - 1 - x0;
    PlaneLoad L[kPlanes];
#define DMRT_PF(k) (S + plane_f(k) * PL)
#define DMRT_PG(k) (S + plane_g(k) * PL)
    pull_load<0, 0>(DMRT_PF(0), DMRT_PF(0), j, x0, right_e, G, L[0]);
    pull_load<1, 0>(DMRT_PF(1), DMRT_PF(3), j, x0, right_e, G, L[1]);
    pull_load<0, 1>(DMRT_PF(2), DMRT_PF(4), j, x0, right_e, G, L[2]);
    pull_load<-1, 0>(DMRT_PF(3), DMRT_PF(1), j, x0, right_e, G, L[3]);
    pull_load<0, -1>(DMRT_PF(4), DMRT_PF(2), j, x0, right_e, G, L[4]);
    pull_load<1, 1>(DMRT_PF(5), DMRT_PF(7), j, x0, right_e, G, L[5]);
    pull_load<-1, 1>(DMRT_PF(6), DMRT_PF(8), j, x0, right_e, G, L[6]);
    pull_load<-1, -1>(DMRT_PF(7), DMRT_PF(5), j, x0, right_e, G, L[7]);
    pull_load<1, -1>(DMRT_PF(8), DMRT_PF(6), j, x0, right_e, G, L[8]);
    pull_load<0, 0>(DMRT_PG(0), DMRT_PG(0), j, x0, right_e, G, L[9]);
    pull_load<1, 0>(DMRT_PG(1), DMRT_PG(3), j, x0, right_e, G, L[10]);
    pull_load<0, 1>(DMRT_PG(2), DMRT_PG(4), j, x0, right_e, G, L[11]);
    pull_load<-1, 0>(DMRT_PG(3), DMRT_PG(1), j, x0, right_e, G, L[12]);
    pull_load<0, -1>(DMRT_PG(4), DMRT_PG(2), j, x0, right_e, G, L[13]);
#undef DMRT_PF
#undef DMRT_PG

    float4 F[9], Gq[5];
    F[0] = pull_finish<0, 0>(L[0], j, x0, right_e, G, 1.f, 0.f, 1.f, 0.f);
    F[1] = pull_finish<1, 0>(L[1], j, x0, right_e, G, 1.f, 0.f, 1.f, 0.f);
    F[2] = pull_finish<0, 1>(L[2], j, x0, right_e, G, 1.f, 0.f, 1.f, 0.f);
    F[3] = pull_finish<-1, 0>(L[3], j, x0, right_e, G, 1.f, 0.f, 1.f, 0.f);
    F[4] = pull_finish<0, -1>(L[4], j, x0, right_e, G, 1.f, 0.f, 1.f, 0.f);
    F[5] = pull_finish<1, 1>(L[5], j, x0, right_e, G, 1.f, 0.f, 1.f, 0.f);
    F[6] = pull_finish<-1, 1>(L[6], j, x0, right_e, G, 1.f, 0.f, 1.f, 0.f);
    F[7] = pull_finish<-1, -1>(L[7], j, x0, right_e, G, 1.f, 0.f, 1.f, 0.f);
    F[8] = pull_finish<1, -1>(L[8], j, x0, right_e, G, 1.f, 0.f, 1.f, 0.f);
    Gq[0] = pull_finish<0, 0>(L[9], j, x0, right_e, G, 1.f, 0.f, 1.f, 0.f);
    Gq[1] = pull_finish<1, 0>(L[10], j, x0, right_e, G, sign_l_g, add_l_g, 1.f, 0.f);
    Gq[2] = pull_finish<0, 1>(L[11], j, x0, right_e, G, 1.f, 0.f, 1.f, 0.f);
    Gq[3] = pull_finish<-1, 0>(L[12], j, x0, right_e, G, 1.f, 0.f, sign_r_g, add_r_g);
    Gq[4] = pull_finish<0, -1>(L[13], j, x0, right_e, G, 1.f, 0.f, 1.f, 0.f);

    float theta4[4];
    bool bad = false;
    collide_quad(F, Gq, K, theta4, quad_ok ? min(4, A.nx - x0) : 0, bad);
    if (quad_ok) {
        store_quad(A, j, x0, F, Gq);
        if (bad) atomicOr(A.err, kErrNonFinite);
    }

    if (bx == 0) {
        const bool has_nu = row_ok && G.seg_lane == 0;
        double nuj = 0.0;
        if (has_nu && j_in) {
            const double tw = (double)__ldg(A.hot + j);
            nuj = K.nu_scale * (8.0 * tw - 9.0 * (double)theta4[0] + (double)theta4[1]);
        }
        nu_report(A, has_nu, j, nuj);
    }
}

// Internal linkage: every translation unit that launches it compiles its own copy.
static __global__ void __launch_bounds__(kDirectThreads, 4) step_direct_kernel(StepArgs A, StepConsts K) {
    grid_dep_wait();
    grid_dep_launch();
    // The previous step's mean Nusselt number: the first block, or, when the
    // grid has one row of blocks more than the cavity needs (small grids, where
    // it would delay the first block's nodes), the first block of that row,
    // which does nothing else.
    const int work_y = (A.ny + (kDirectThreads >> A.wx_log2) - 1) / (kDirectThreads >> A.wx_log2);
    if (blockIdx.y >= work_y) {
        if (blockIdx.x == 0) nu_finish_prev(A, true);
        return;
    }
    if (blockIdx.x == 0 && blockIdx.y == 0 && gridDim.y == work_y) nu_finish_prev(A, true);
    direct_tile(A, K, blockIdx.x, blockIdx.y);
}

}  // namespace dmrt
