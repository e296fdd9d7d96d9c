// Fused double-MRT time step, TMA-pipelined persistent variant (sm_103a).
//
// Work items are (strip, row block): a strip is 248 nodes of a row, a row block
// R consecutive rows. For one item the pull-stream needs, per plane group
// (see lattice.cuh), R rows of 256 floats starting 4 nodes left of the strip
// (one halo column each side, rounded out to 16-byte alignment):
//   group Z (6 planes) from rows j0 .. j0+R-1,
//   group P (4 planes) from rows j0-1 .. j0+R-2,
//   group N (4 planes) from rows j0+1 .. j0+R.
// Each is one 3-D tensor copy (cp.async.bulk.tensor, box 256 x R x planes) into
// a shared-memory stage; S stages form a ring guarded by mbarriers, so while
// the block computes one item the copies of the next S-1 items are in flight.
// Out-of-range boxes (the left of the first strip, the rows above and below
// the cavity) are zero-filled by the copy engine and replaced by the wall
// rules. Each thread owns NPT (4, 2 or 1) consecutive nodes of a row, reads
// them from shared memory (vector reads; a shifted plane takes two aligned
// reads), collides in registers and stores with NPT-wide vector stores; a row
// of a strip is 256 / NPT threads. One elected thread issues the copies.
//
// Every wait is bounded (%globaltimer): on expiry the block records
// kErrTimeout, waits (bounded) for the copies it issued and returns.
#pragma once
#include <cuda.h>

#include "lattice.cuh"

namespace dmrt {

constexpr int kTmaStrip = 248;      // nodes per strip
constexpr int kTmaBox = 256;        // floats per box row (strip + halos, aligned)
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s

struct TmaGeo {
    int n_strips;
    int n_rowblocks;
};

__host__ __device__ constexpr int tma_stage_floats(int R) { return kPlanes * R * kTmaBox; }
__host__ __device__ constexpr size_t tma_smem_bytes(int R, int S) {
    return (size_t)S * tma_stage_floats(R) * sizeof(float) + (size_t)S * 8;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait until the barrier's phase with the given parity completed, at most
// kWaitLimitNs; returns false on expiry.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > kWaitLimitNs) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

template <int NPT>
struct VecOf;
template <>
struct VecOf<4> {
    using T = float4;
};
template <>
struct VecOf<2> {
    using T = float2;
};
template <>
struct VecOf<1> {
    using T = float;
};

template <int NPT>
__device__ __forceinline__ void vec_get(const float* p, float (&o)[NPT]) {
    if constexpr (NPT == 4) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        o[0] = v.x, o[1] = v.y, o[2] = v.z, o[3] = v.w;
    } else if constexpr (NPT == 2) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        o[0] = v.x, o[1] = v.y;
    } else {
        o[0] = *p;
    }
}

template <int NPT>
__device__ __forceinline__ void vec_ldg(const float* p, float (&o)[NPT]) {
    if constexpr (NPT == 4) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(p));
        o[0] = v.x, o[1] = v.y, o[2] = v.z, o[3] = v.w;
    } else if constexpr (NPT == 2) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(p));
        o[0] = v.x, o[1] = v.y;
    } else {
        o[0] = __ldg(p);
    }
}

template <int NPT>
__device__ __forceinline__ void vec_put(float* p, const float (&o)[NPT]) {
    if constexpr (NPT == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
    } else if constexpr (NPT == 2) {
        *reinterpret_cast<float2*>(p) = make_float2(o[0], o[1]);
    } else {
        *p = o[0];
    }
}

// NPT consecutive values of a shared-memory plane row for nodes n0..n0+NPT-1,
// shifted for a pull with lattice x-velocity EX: node n takes the value at
// n - EX. The row starts 4 nodes left of the strip, so node n sits at n + 4.
template <int EX, int NPT>
__device__ __forceinline__ void lds_pull(const float* rowp, int n0, float (&o)[NPT]) {
    const float* p = rowp + 4 + n0;
    if constexpr (EX == 0 || NPT == 1) {
        vec_get<NPT>(p - EX, o);
    } else if constexpr (EX == 1) {
        float a[NPT], b[NPT];
        vec_get<NPT>(p - NPT, a);
        vec_get<NPT>(p, b);
        o[0] = a[NPT - 1];
#pragma unroll
        for (int e = 1; e < NPT; ++e) o[e] = b[e - 1];
    } else {
        float b[NPT], c[NPT];
        vec_get<NPT>(p, b);
        vec_get<NPT>(p + NPT, c);
#pragma unroll
        for (int e = 0; e < NPT - 1; ++e) o[e] = b[e + 1];
        o[NPT - 1] = c[0];
    }
}

// Collide NPT nodes in place; nodes at or beyond nvalid (padding) are zeroed.
template <int NPT>
__device__ __forceinline__ void collide_nodes(float (&F)[9][NPT], float (&Gq)[5][NPT],
                                              const StepConsts& K, float (&theta)[NPT], int nvalid,
                                              bool& bad) {
#pragma unroll
    for (int e = 0; e < NPT; ++e) {
        float f[9], g[5];
#pragma unroll
        for (int k = 0; k < 9; ++k) f[k] = F[k][e];
#pragma unroll
        for (int k = 0; k < 5; ++k) g[k] = Gq[k][e];
        float rho, th;
        collide_node(f, g, K, rho, th);
        const bool valid = e < nvalid;
        if (valid) bad |= !(fabsf(rho) < 1e30f) || !(fabsf(th) < 1e30f);
#pragma unroll
        for (int k = 0; k < 9; ++k) F[k][e] = valid ? f[k] : 0.f;
#pragma unroll
        for (int k = 0; k < 5; ++k) Gq[k][e] = valid ? g[k] : 0.f;
        theta[e] = th;
    }
}

// Position in the block's sequence of work items blockIdx.x, blockIdx.x + G,
// blockIdx.x + 2G, ... with item = rowblock * n_strips + strip, advanced
// without divisions (they would cost as much as a node's arithmetic).
struct ItemCursor {
    int strip, rb, dstrip, drb;
    __device__ __forceinline__ void init(int first, int G, int n_strips) {
        strip = first % n_strips;
        rb = first / n_strips;
        dstrip = G % n_strips;
        drb = G / n_strips;
    }
    __device__ __forceinline__ void advance(int n_strips) {
        strip += dstrip;
        rb += drb;
        if (strip >= n_strips) {
            strip -= n_strips;
            ++rb;
        }
    }
};

template <int NPT, int R, int S>
__global__ void __launch_bounds__(R * (256 / NPT)) step_tma_kernel(const __grid_constant__ CUtensorMap map6,
                                                          const __grid_constant__ CUtensorMap map4,
                                                          StepArgs A, StepConsts K, TmaGeo T) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    float* stages = reinterpret_cast<float*>(smem_raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + (size_t)S * tma_stage_floats(R) * sizeof(float));
    constexpr int TPR = 256 / NPT;  // threads per row of a strip
    const int tid = threadIdx.x;
    const int rg = tid / TPR;  // row of the block this thread works on
    const int t = tid % TPR;   // node group within the strip
    const int G = gridDim.x;
    constexpr uint32_t kStageBytes = (uint32_t)(kPlanes * R * kTmaBox * sizeof(float));

    // After an expired wait in an earlier launch the state is already invalid:
    // return at once instead of waiting again.
    if (*reinterpret_cast<volatile unsigned*>(A.err) & kErrTimeout) return;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
        mbar_fence_init();
    }
    __syncthreads();

    auto issue = [&](const ItemCursor& c, int s) {
        const int x = c.strip * kTmaStrip - 4;
        const int j0 = c.rb * R;
        float* st = stages + (size_t)s * tma_stage_floats(R);
        mbar_expect_tx(&bars[s], kStageBytes);
        tma_load_3d(st, &map6, x, j0, kGroupZ, &bars[s]);
        tma_load_3d(st + kGroupP * R * kTmaBox, &map4, x, j0 - 1, kGroupP, &bars[s]);
        tma_load_3d(st + kGroupN * R * kTmaBox, &map4, x, j0 + 1, kGroupN, &bars[s]);
    };

    // Producer (thread 0): issues items ahead of the consumers, S - 1 in flight.
    ItemCursor pc;
    pc.init(blockIdx.x, G, T.n_strips);
    int issued = 0;  // items issued by this block (thread 0's count)
    if (tid == 0) {
        for (int q = 0; q < S - 1 && pc.rb < T.n_rowblocks; ++q) {
            issue(pc, q);
            pc.advance(T.n_strips);
            issued = q + 1;
        }
    }

    const float* Sg = A.src;
    const long long PL = A.plane;
    const float sign_l_g = K.left_fixed ? -1.f : 1.f;
    const float sign_r_g = K.right_fixed ? -1.f : 1.f;
    bool timed_out = false;
    ItemCursor cc;  // consumer: the item being computed
    cc.init(blockIdx.x, G, T.n_strips);
    int k = 0, s = 0;
    uint32_t phase = 0;
    for (; cc.rb < T.n_rowblocks; ++k) {
        if (tid == 0 && pc.rb < T.n_rowblocks) {
            // Item k + S - 1 goes to the stage of item k - 1, released by the
            // barrier that ended it.
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(pc, s == 0 ? S - 1 : s - 1);
            pc.advance(T.n_strips);
            issued = k + S;
        }
        const bool ok = mbar_wait_bounded(&bars[s], phase);

        const int strip = cc.strip;
        const int j = cc.rb * R + rg;
        const int n0 = NPT * t;
        const int x0 = strip * kTmaStrip + n0;
        const bool row_ok = j < A.ny;
        const bool mine = ok && row_ok && n0 < kTmaStrip && x0 < A.nx;
        float theta[NPT];
#pragma unroll
        for (int e = 0; e < NPT; ++e) theta[e] = 0.f;
        if (mine) {
            const float* st = stages + (size_t)s * tma_stage_floats(R);
            auto rowp = [&](int plane) { return st + (plane * R + rg) * kTmaBox; };
            float F[9][NPT], Gq[5][NPT];
            lds_pull<0>(rowp(plane_f(0)), n0, F[0]);
            lds_pull<1>(rowp(plane_f(1)), n0, F[1]);
            lds_pull<0>(rowp(plane_f(2)), n0, F[2]);
            lds_pull<-1>(rowp(plane_f(3)), n0, F[3]);
            lds_pull<0>(rowp(plane_f(4)), n0, F[4]);
            lds_pull<1>(rowp(plane_f(5)), n0, F[5]);
            lds_pull<-1>(rowp(plane_f(6)), n0, F[6]);
            lds_pull<-1>(rowp(plane_f(7)), n0, F[7]);
            lds_pull<1>(rowp(plane_f(8)), n0, F[8]);
            lds_pull<0>(rowp(plane_g(0)), n0, Gq[0]);
            lds_pull<1>(rowp(plane_g(1)), n0, Gq[1]);
            lds_pull<0>(rowp(plane_g(2)), n0, Gq[2]);
            lds_pull<-1>(rowp(plane_g(3)), n0, Gq[3]);
            lds_pull<0>(rowp(plane_g(4)), n0, Gq[4]);

            // Walls. Bottom row: links from below (f2, f5, f6, g2) bounce back from
            // the node's own opposites (f4, f7, f8, g4); top row the reverse.
            const float* rowj = Sg + (size_t)j * A.pitch;
            if (j == 0) {
                vec_ldg<NPT>(rowj + plane_f(4) * PL + x0, F[2]);
                vec_ldg<NPT>(rowj + plane_f(7) * PL + x0, F[5]);
                vec_ldg<NPT>(rowj + plane_f(8) * PL + x0, F[6]);
                vec_ldg<NPT>(rowj + plane_g(4) * PL + x0, Gq[2]);
            }
            if (j == A.ny - 1) {
                vec_ldg<NPT>(rowj + plane_f(2) * PL + x0, F[4]);
                vec_ldg<NPT>(rowj + plane_f(5) * PL + x0, F[7]);
                vec_ldg<NPT>(rowj + plane_f(6) * PL + x0, F[8]);
                vec_ldg<NPT>(rowj + plane_g(2) * PL + x0, Gq[4]);
            }
            // Left wall (node x = 0): links with e_x = +1 (f1, f5, f8, g1).
            if (x0 == 0) {
                F[1][0] = __ldg(rowj + plane_f(3) * PL);
                F[5][0] = __ldg(rowj + plane_f(7) * PL);
                F[8][0] = __ldg(rowj + plane_f(6) * PL);
                const float add = K.left_fixed ? K.abb * __ldg(A.hot + j) : 0.f;
                Gq[1][0] = sign_l_g * __ldg(rowj + plane_g(3) * PL) + add;
            }
            // Right wall (node x = nx - 1): links with e_x = -1 (f3, f6, f7, g3).
            const int re = A.nx - 1 - x0;
            if (re < NPT) {
                const int xr = A.nx - 1;
                const float v3 = __ldg(rowj + plane_f(1) * PL + xr);
                const float v6 = __ldg(rowj + plane_f(8) * PL + xr);
                const float v7 = __ldg(rowj + plane_f(5) * PL + xr);
                const float add = K.right_fixed ? K.abb * __ldg(A.cold + j) : 0.f;
                const float vg = sign_r_g * __ldg(rowj + plane_g(1) * PL + xr) + add;
#pragma unroll
                for (int e = 0; e < NPT; ++e) {
                    if (e == re) {
                        F[3][e] = v3;
                        F[6][e] = v6;
                        F[7][e] = v7;
                        Gq[3][e] = vg;
                    }
                }
            }

            bool bad = false;
            collide_nodes<NPT>(F, Gq, K, theta, min(NPT, A.nx - x0), bad);
            float* D = A.dst + (size_t)j * A.pitch + x0;
#pragma unroll
            for (int k = 0; k < 9; ++k) vec_put<NPT>(D + plane_f(k) * PL, F[k]);
#pragma unroll
            for (int k = 0; k < 5; ++k) vec_put<NPT>(D + plane_g(k) * PL, Gq[k]);
            if (bad) atomicOr(A.err, kErrNonFinite);
        }
        // Nusselt number of row j from the first warp of the row's thread group
        // in the first strip; nodes 0 and 1 sit in lane 0 (or lanes 0 and 1).
        if (strip == 0 && t < 32) {
            float th1 = NPT > 1 ? theta[NPT > 1 ? 1 : 0] : 0.f;
            if constexpr (NPT == 1) th1 = __shfl_down_sync(kFull, theta[0], 1);
            const bool has_nu = mine && t == 0;
            double nuj = 0.0;
            if (has_nu) {
                const double tw = (double)__ldg(A.hot + j);
                nuj = K.nu_scale * (8.0 * tw - 9.0 * (double)theta[0] + (double)th1);
            }
            nu_report(A, has_nu, j, nuj);
        }
        // All threads are done with stage s; a timeout anywhere ends the block.
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        cc.advance(T.n_strips);
        if (++s == S) {
            s = 0;
            phase ^= 1u;
        }
    }
    if (timed_out && tid == 0) {
        atomicOr(A.err, kErrTimeout);
        // Let the copies this block issued land before its shared memory is released.
        for (int q = k; q < issued; ++q) mbar_wait_bounded(&bars[q % S], (uint32_t)((q / S) & 1));
    }
}

}  // namespace dmrt
