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
// rules. Threads read their 4 nodes per row from shared memory (two aligned
// 128-bit reads for a shifted plane), collide in registers and store with
// 128-bit stores. One elected thread issues the copies.
//
// Every wait is bounded (%globaltimer): on expiry the block records
// kErrTimeout, waits (bounded) for the copies it issued and returns.
#pragma once
#include <cuda.h>

#include "lattice.cuh"

namespace dmrt {

constexpr int kTmaStrip = 248;      // nodes per strip
constexpr int kTmaBox = 256;        // floats per box row (strip + halos, aligned)
constexpr int kTmaQuads = kTmaStrip / 4;  // active threads per row (62 of 64)
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

// Four consecutive values of a shared-memory plane row for nodes 4t..4t+3,
// shifted for a pull with lattice x-velocity EX (the row starts 4 nodes left
// of the strip, so node n sits at index n + 4).
template <int EX>
__device__ __forceinline__ float4 lds_pull(const float* rowp, int t) {
    const float* p = rowp + 4 + 4 * t;
    const float4 b = *reinterpret_cast<const float4*>(p);
    if constexpr (EX == 0) {
        return b;
    } else if constexpr (EX == 1) {
        const float4 a = *reinterpret_cast<const float4*>(p - 4);
        return make_float4(a.w, b.x, b.y, b.z);
    } else {
        const float4 c = *reinterpret_cast<const float4*>(p + 4);
        return make_float4(b.y, b.z, b.w, c.x);
    }
}

template <int R, int S>
__global__ void __launch_bounds__(64 * R) step_tma_kernel(const __grid_constant__ CUtensorMap map6,
                                                          const __grid_constant__ CUtensorMap map4,
                                                          StepArgs A, StepConsts K, TmaGeo T) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    float* stages = reinterpret_cast<float*>(smem_raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + (size_t)S * tma_stage_floats(R) * sizeof(float));
    const int tid = threadIdx.x;
    const int rg = tid >> 6;  // row of the block this thread works on
    const int t = tid & 63;   // quad within the strip
    const long long items = (long long)T.n_strips * T.n_rowblocks;
    const long long G = gridDim.x;
    constexpr uint32_t kStageBytes = (uint32_t)(kPlanes * R * kTmaBox * sizeof(float));

    // After an expired wait in an earlier launch the state is already invalid:
    // return at once instead of waiting again.
    if (*reinterpret_cast<volatile unsigned*>(A.err) & kErrTimeout) return;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
        mbar_fence_init();
    }
    __syncthreads();

    auto issue = [&](long long it, int s) {
        const int strip = (int)(it % T.n_strips);
        const int j0 = (int)(it / T.n_strips) * R;
        const int x = strip * kTmaStrip - 4;
        float* st = stages + (size_t)s * tma_stage_floats(R);
        mbar_expect_tx(&bars[s], kStageBytes);
        tma_load_3d(st, &map6, x, j0, kGroupZ, &bars[s]);
        tma_load_3d(st + kGroupP * R * kTmaBox, &map4, x, j0 - 1, kGroupP, &bars[s]);
        tma_load_3d(st + kGroupN * R * kTmaBox, &map4, x, j0 + 1, kGroupN, &bars[s]);
    };

    long long issued = 0;  // items issued by this block (thread 0's count)
    if (tid == 0) {
        for (int k = 0; k < S - 1; ++k) {
            const long long it = blockIdx.x + (long long)k * G;
            if (it < items) {
                issue(it, k);
                issued = k + 1;
            }
        }
    }

    const float* Sg = A.src;
    const long long PL = A.plane;
    const float sign_l_g = K.left_fixed ? -1.f : 1.f;
    const float sign_r_g = K.right_fixed ? -1.f : 1.f;
    bool timed_out = false;
    long long k = 0;
    for (;; ++k) {
        const long long it = blockIdx.x + k * G;
        if (it >= items) break;
        if (tid == 0) {
            const long long nxt = blockIdx.x + (k + S - 1) * G;
            if (nxt < items) {
                // The stage of item k-1, released by the barrier that ended it.
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(nxt, (int)((k + S - 1) % S));
                issued = k + S;
            }
        }
        const int s = (int)(k % S);
        const bool ok = mbar_wait_bounded(&bars[s], (uint32_t)((k / S) & 1));

        const int strip = (int)(it % T.n_strips);
        const int j = (int)(it / T.n_strips) * R + rg;
        const int x0 = strip * kTmaStrip + 4 * t;
        const bool row_ok = j < A.ny;
        const bool quad_ok = ok && row_ok && t < kTmaQuads && x0 < A.nx;
        float theta4[4] = {0.f, 0.f, 0.f, 0.f};
        if (quad_ok) {
            const float* st = stages + (size_t)s * tma_stage_floats(R);
            auto rowp = [&](int plane) { return st + (plane * R + rg) * kTmaBox; };
            float4 F[9], Gq[5];
            F[0] = lds_pull<0>(rowp(plane_f(0)), t);
            F[1] = lds_pull<1>(rowp(plane_f(1)), t);
            F[2] = lds_pull<0>(rowp(plane_f(2)), t);
            F[3] = lds_pull<-1>(rowp(plane_f(3)), t);
            F[4] = lds_pull<0>(rowp(plane_f(4)), t);
            F[5] = lds_pull<1>(rowp(plane_f(5)), t);
            F[6] = lds_pull<-1>(rowp(plane_f(6)), t);
            F[7] = lds_pull<-1>(rowp(plane_f(7)), t);
            F[8] = lds_pull<1>(rowp(plane_f(8)), t);
            Gq[0] = lds_pull<0>(rowp(plane_g(0)), t);
            Gq[1] = lds_pull<1>(rowp(plane_g(1)), t);
            Gq[2] = lds_pull<0>(rowp(plane_g(2)), t);
            Gq[3] = lds_pull<-1>(rowp(plane_g(3)), t);
            Gq[4] = lds_pull<0>(rowp(plane_g(4)), t);

            // Walls. Bottom row: links from below (f2, f5, f6, g2) bounce back from
            // the node's own opposites (f4, f7, f8, g4); top row the reverse.
            const float* rowj = Sg + (size_t)j * A.pitch;
            if (j == 0) {
                F[2] = ldg4(rowj + plane_f(4) * PL + x0);
                F[5] = ldg4(rowj + plane_f(7) * PL + x0);
                F[6] = ldg4(rowj + plane_f(8) * PL + x0);
                Gq[2] = ldg4(rowj + plane_g(4) * PL + x0);
            }
            if (j == A.ny - 1) {
                F[4] = ldg4(rowj + plane_f(2) * PL + x0);
                F[7] = ldg4(rowj + plane_f(5) * PL + x0);
                F[8] = ldg4(rowj + plane_f(6) * PL + x0);
                Gq[4] = ldg4(rowj + plane_g(2) * PL + x0);
            }
            // Left wall (node x = 0): links with e_x = +1 (f1, f5, f8, g1).
            if (x0 == 0) {
                F[1].x = __ldg(rowj + plane_f(3) * PL);
                F[5].x = __ldg(rowj + plane_f(7) * PL);
                F[8].x = __ldg(rowj + plane_f(6) * PL);
                const float add = K.left_fixed ? K.abb * __ldg(A.hot + j) : 0.f;
                Gq[1].x = sign_l_g * __ldg(rowj + plane_g(3) * PL) + add;
            }
            // Right wall (node x = nx - 1): links with e_x = -1 (f3, f6, f7, g3).
            const int re = A.nx - 1 - x0;
            if (re < 4) {
                const int xr = A.nx - 1;
                set_comp(F[3], re, __ldg(rowj + plane_f(1) * PL + xr));
                set_comp(F[6], re, __ldg(rowj + plane_f(8) * PL + xr));
                set_comp(F[7], re, __ldg(rowj + plane_f(5) * PL + xr));
                const float add = K.right_fixed ? K.abb * __ldg(A.cold + j) : 0.f;
                set_comp(Gq[3], re, sign_r_g * __ldg(rowj + plane_g(1) * PL + xr) + add);
            }

            bool bad = false;
            collide_quad(F, Gq, K, theta4, min(4, A.nx - x0), bad);
            store_quad(A, j, x0, F, Gq);
            if (bad) atomicOr(A.err, kErrNonFinite);
        }
        // Nusselt number of row j from the first warp of the row's thread group
        // in the first strip (lane 0 holds nodes 0 and 1).
        if (strip == 0 && t < 32) {
            const bool has_nu = quad_ok && t == 0;
            double nuj = 0.0;
            if (has_nu) {
                const double tw = (double)__ldg(A.hot + j);
                nuj = K.nu_scale * (8.0 * tw - 9.0 * (double)theta4[0] + (double)theta4[1]);
            }
            nu_report(A, has_nu, j, nuj);
        }
        // All threads are done with stage s; a timeout anywhere ends the block.
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
    }
    if (timed_out && tid == 0) {
        atomicOr(A.err, kErrTimeout);
        // Let the copies this block issued land before its shared memory is released.
        for (long long q = k; q < issued; ++q) mbar_wait_bounded(&bars[q % S], (uint32_t)((q / S) & 1));
    }
}

}  // namespace dmrt
