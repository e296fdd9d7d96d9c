// Fused double-MRT time step, TMA-pipelined persistent variant (sm_103a).
//
// Work items are (strip, row block): a strip is 256 - 2 HALO nodes of a row
// (248 for float32 storage, 240 for 16-bit and mixed storage), a row block R
// consecutive rows. For one item the pull-stream needs, per plane group (see
// lattice.cuh), R rows of 256 elements starting HALO nodes left of the strip
// (one halo column each side, rounded out so the copy starts on a 16-byte
// boundary; HALO = 16 bytes / size of the narrowest stored element):
//   group Z (e_y = 0) from rows j0 .. j0+R-1,
//   group P (e_y = +1) from rows j0-1 .. j0+R-2,
//   group N (e_y = -1) from rows j0+1 .. j0+R.
// One-type storage (all planes float32, float16 or bfloat16) takes one 3-D
// tensor copy per group (cp.async.bulk.tensor, box 256 x R x planes: 6, 4, 4).
// Mixed storage (flow planes float16, thermal planes float32, in two blocks)
// takes six: three for the flow groups (3 planes each) and three for the
// thermal groups (3, 1, 1 planes). The copies land in a shared-memory stage;
// S stages form a ring guarded by mbarriers, so while
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
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "lattice.cuh"

namespace dmrt {

constexpr int kTmaBox = 256;  // elements per box row (strip + halos, aligned)
constexpr int kMaxSmem = 232448;  // dynamic shared memory a block may opt in to (227 KB)
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s

__host__ __device__ constexpr int tma_halo(int elem_bytes) { return 16 / elem_bytes; }
__host__ __device__ constexpr int tma_strip(int elem_bytes) { return kTmaBox - 2 * tma_halo(elem_bytes); }

struct TmaGeo {
    int n_strips;
    int n_rowblocks;
};

// Stage of R rows with the 9 flow planes in f_bytes and the 5 thermal planes in
// g_bytes per element, plus one mbarrier per stage.
__host__ __device__ constexpr size_t tma_stage_bytes_fg(int R, int f_bytes, int g_bytes) {
    return (size_t)R * kTmaBox * (9 * f_bytes + 5 * g_bytes);
}
__host__ __device__ constexpr size_t tma_smem_bytes_fg(int R, int S, int f_bytes, int g_bytes) {
    return (size_t)S * tma_stage_bytes_fg(R, f_bytes, g_bytes) + (size_t)S * 8;
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

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
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
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  unsigned long long limit_ns = kWaitLimitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > limit_ns) return false;
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

// Tensor store of a shared-memory box (bulk-group completion), and the bulk-group
// bookkeeping: commit, wait until the committed stores have read their shared
// memory (.read) or have completed.
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, const void* src, int x, int y, int z) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(smem_u32(src)), "r"(x), "r"(y), "r"(z)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// Make this thread's shared-memory writes visible to the copy engine.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---- typed storage -----------------------------------------------------------
// Populations are stored as float32, or rounded (to nearest, or stochastically)
// to float16 / bfloat16 (the collision always runs in float32). 16-bit storage keeps the thermal
// populations shifted by their rest weight times theta_ref: a stored g_i is
// g_i - w_i theta_ref (w_0 = (1-a)/5, w_1..4 = (4+a)/20); the flow populations
// are already shifted by w_i rho0 (Eq. 33).
__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(__half x) { return __half2float(x); }
__device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }

// Only 16-bit storage is shifted; float32 values are stored as they are.
template <typename E>
constexpr bool kShifted = !std::is_same<E, float>::value;

template <typename E, int N>
struct alignas(sizeof(E) * N) Pack {
    E v[N];
};

// N consecutive stored values (aligned to N elements) as floats.
template <typename E, int N>
__device__ __forceinline__ void vec_get(const E* p, float (&o)[N]) {
    const Pack<E, N> q = *reinterpret_cast<const Pack<E, N>*>(p);
#pragma unroll
    for (int e = 0; e < N; ++e) o[e] = to_f(q.v[e]);
}

// Global loads through L2 (ld.global.cg), not the non-coherent cache: the
// multi-step batched kernel reads state written earlier in the same launch.
template <typename E, int N>
__device__ __forceinline__ void vec_ldg(const E* p, float (&o)[N], float shift) {
    Pack<E, N> q;
    if constexpr (sizeof(Pack<E, N>) == 16) {
        const uint4 r = __ldcg(reinterpret_cast<const uint4*>(p));
        q = *reinterpret_cast<const Pack<E, N>*>(&r);
    } else if constexpr (sizeof(Pack<E, N>) == 8) {
        const uint2 r = __ldcg(reinterpret_cast<const uint2*>(p));
        q = *reinterpret_cast<const Pack<E, N>*>(&r);
    } else if constexpr (sizeof(Pack<E, N>) == 4) {
        const unsigned r = __ldcg(reinterpret_cast<const unsigned*>(p));
        q = *reinterpret_cast<const Pack<E, N>*>(&r);
    } else {
        const unsigned short r = __ldcg(reinterpret_cast<const unsigned short*>(p));
        q = *reinterpret_cast<const Pack<E, N>*>(&r);
    }
#pragma unroll
    for (int e = 0; e < N; ++e) o[e] = kShifted<E> ? to_f(q.v[e]) + shift : to_f(q.v[e]);
}

template <typename E>
__device__ __forceinline__ float ldg_one(const E* p, float shift) {
    float o[1];
    vec_ldg<E, 1>(p, o, shift);
    return o[0];
}

// Two float32 values converted to a packed pair of E, the first in the low half
// (the lower address). Rounding to nearest even: one paired conversion.
template <typename E>
__device__ __forceinline__ unsigned pack2_rn(float lo, float hi);
template <>
__device__ __forceinline__ unsigned pack2_rn<__half>(float lo, float hi) {
    unsigned d;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}
template <>
__device__ __forceinline__ unsigned pack2_rn<__nv_bfloat16>(float lo, float hi) {
    unsigned d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

// Stochastic rounding (used for 16-bit stores when requested) by the
// conversion instruction of this GPU family: for each value a uniform random
// integer is added below the bits that are kept and the result is truncated
// toward zero, so x is rounded up in magnitude with probability equal to its
// distance from the lower neighbour in units of the spacing (Croci et al.,
// "Stochastic rounding: implementation, error analysis and applications",
// R. Soc. Open Sci. 2022). The random word holds one 16-bit field per value
// (high value: bits 16-31, low value: bits 0-15); bfloat16 uses all 16 bits of
// a field, float16 its low 13 (the bits a normal float16 discards). Each field
// is filled from bits 16-31 of that value's own draw, so a value's rounding
// depends on its own draw only, whatever it is paired with.
template <typename E>
__device__ __forceinline__ unsigned pack2_rs(float lo, float hi, unsigned rlo, unsigned rhi);
template <>
__device__ __forceinline__ unsigned pack2_rs<__half>(float lo, float hi, unsigned rlo, unsigned rhi) {
    unsigned d;
    asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(__byte_perm(rlo, rhi, 0x7632)));
    return d;
}
template <>
__device__ __forceinline__ unsigned pack2_rs<__nv_bfloat16>(float lo, float hi, unsigned rlo, unsigned rhi) {
    unsigned d;
    asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(__byte_perm(rlo, rhi, 0x7632)));
    return d;
}

// Integer hash "lowbias32" (C. Wellons, "Prospecting for hash functions", 2018).
__device__ __forceinline__ unsigned hash32(unsigned x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// Linear congruential step (Numerical Recipes constants); the high bits are used.
__device__ __forceinline__ unsigned lcg(unsigned& r) {
    r = r * 1664525u + 1013904223u;
    return r;
}

// Store of N nodes' values (shifted for 16-bit storage), rounded to nearest
// or, with SR, stochastically; r[e] is node e's random state, so a node draws
// the same bits whatever the number of nodes per thread.
template <typename E, int N, bool SR>
__device__ __forceinline__ void vec_put(E* p, const float (&o)[N], float shift, unsigned (&r)[N]) {
    if constexpr (!kShifted<E>) {
        Pack<E, N> q;
#pragma unroll
        for (int e = 0; e < N; ++e) q.v[e] = o[e];
        *reinterpret_cast<Pack<E, N>*>(p) = q;
    } else if constexpr (N == 1) {
        const unsigned d = SR ? pack2_rs<E>(o[0] - shift, 0.f, lcg(r[0]), 0u) : pack2_rn<E>(o[0] - shift, 0.f);
        *reinterpret_cast<unsigned short*>(p) = (unsigned short)d;
    } else {
        static_assert(N == 2 || N == 4 || N == 8, "16-bit stores take pairs of nodes");
        unsigned w[N / 2];
#pragma unroll
        for (int e = 0; e < N; e += 2) {
            if constexpr (SR) {
                const unsigned r0 = lcg(r[e]);
                const unsigned r1 = lcg(r[e + 1]);
                w[e / 2] = pack2_rs<E>(o[e] - shift, o[e + 1] - shift, r0, r1);
            } else {
                w[e / 2] = pack2_rn<E>(o[e] - shift, o[e + 1] - shift);
            }
        }
        if constexpr (N == 2) *reinterpret_cast<unsigned*>(p) = w[0];
        else if constexpr (N == 4) *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
        else *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// NPT consecutive values of a shared-memory plane row for nodes n0..n0+NPT-1,
// shifted for a pull with lattice x-velocity EX: node n takes the value at
// n - EX. The row starts HALO nodes left of the strip, so node n sits at n + HALO.
// (HALO is the layout's: 16 bytes of its narrowest stored type.)
template <int EX, int NPT, int HALO, typename E>
__device__ __forceinline__ void lds_pull(const E* rowp, int n0, float (&o)[NPT], float shift) {
    const E* p = rowp + HALO + n0;
    if constexpr (EX == 0 || NPT == 1) {
        vec_get<E, NPT>(p - EX, o);
    } else if constexpr (EX == 1) {
        float a[NPT], b[NPT];
        vec_get<E, NPT>(p - NPT, a);
        vec_get<E, NPT>(p, b);
        o[0] = a[NPT - 1];
#pragma unroll
        for (int e = 1; e < NPT; ++e) o[e] = b[e - 1];
    } else {
        float b[NPT], c[NPT];
        vec_get<E, NPT>(p, b);
        vec_get<E, NPT>(p + NPT, c);
#pragma unroll
        for (int e = 0; e < NPT - 1; ++e) o[e] = b[e + 1];
        o[NPT - 1] = c[0];
    }
    if constexpr (kShifted<E>) {
#pragma unroll
        for (int e = 0; e < NPT; ++e) o[e] += shift;
    }
}

// NPT consecutive nodes n0.. of a shared-memory row together with their left
// neighbours (l[e] = node n0 + e - 1) and, for lds_three, right neighbours
// (r[e] = node n0 + e + 1): the unshifted vector and one shifted read per side.
template <int NPT, int HALO, typename E>
__device__ __forceinline__ void lds_left_own(const E* rowp, int n0, float (&l)[NPT], float (&c)[NPT]) {
    const E* p = rowp + HALO + n0;
    float a[NPT];
    vec_get<E, NPT>(p - NPT, a);
    vec_get<E, NPT>(p, c);
    l[0] = a[NPT - 1];
#pragma unroll
    for (int e = 1; e < NPT; ++e) l[e] = c[e - 1];
}
template <int NPT, int HALO, typename E>
__device__ __forceinline__ void lds_right_own(const E* rowp, int n0, float (&r)[NPT], float (&c)[NPT]) {
    const E* p = rowp + HALO + n0;
    float b[NPT];
    vec_get<E, NPT>(p, c);
    vec_get<E, NPT>(p + NPT, b);
#pragma unroll
    for (int e = 0; e < NPT - 1; ++e) r[e] = c[e + 1];
    r[NPT - 1] = b[0];
}
template <int NPT, int HALO, typename E>
__device__ __forceinline__ void lds_three(const E* rowp, int n0, float (&l)[NPT], float (&c)[NPT],
                                          float (&r)[NPT]) {
    const E* p = rowp + HALO + n0;
    float a[NPT], b[NPT];
    vec_get<E, NPT>(p - NPT, a);
    vec_get<E, NPT>(p, c);
    vec_get<E, NPT>(p + NPT, b);
    l[0] = a[NPT - 1];
#pragma unroll
    for (int e = 1; e < NPT; ++e) l[e] = c[e - 1];
#pragma unroll
    for (int e = 0; e < NPT - 1; ++e) r[e] = c[e + 1];
    r[NPT - 1] = b[0];
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
        const bool valid = NPT == 1 || e < nvalid;  // one node per thread: only valid nodes get here
        if (valid) bad |= !(fabsf(rho) < 1e30f) || !(fabsf(th) < 1e30f);
#pragma unroll
        for (int k = 0; k < 9; ++k) F[k][e] = valid ? f[k] : 0.f;
#pragma unroll
        for (int k = 0; k < 5; ++k) Gq[k][e] = valid ? g[k] : (k == 0 ? K.gsh0 : K.gsh1);
        theta[e] = valid ? th : 0.f;
    }
}

// Population layouts. OneType<E>: 14 planes of E, grouped Z/P/N (lattice.cuh).
// Split<EF, EG>: the 9 flow planes of EF (Z f1 f2 f4, P f3 f6 f7, N f5 f8 f9)
// followed by the 5 thermal planes of EG (Z g1 g2 g4, P g3, N g5), paper numbering.
__host__ __device__ constexpr int split_f(int k) {
    return k == 0 ? 0 : k == 1 ? 1 : k == 3 ? 2 : k == 2 ? 3 : k == 5 ? 4 : k == 6 ? 5 : k == 4 ? 6 : k == 7 ? 7 : 8;
}
__host__ __device__ constexpr int split_g(int k) { return k == 0 ? 0 : k == 1 ? 1 : k == 3 ? 2 : k == 2 ? 3 : 4; }

template <typename E>
struct OneType {
    using Ef = E;
    using Eg = E;
    static constexpr bool kSplit = false;
    static constexpr bool kTheta = false;
    static constexpr int kHalo = tma_halo(sizeof(E));
    __host__ __device__ static constexpr int pf(int k) { return plane_f(k); }
    __host__ __device__ static constexpr int pg(int k) { return plane_g(k); }
};

template <typename EF, typename EG>
struct Split {
    using Ef = EF;
    using Eg = EG;
    static constexpr bool kSplit = true;
    static constexpr bool kTheta = false;
    static constexpr int kHalo = tma_halo(sizeof(EF) < sizeof(EG) ? sizeof(EF) : sizeof(EG));
    __host__ __device__ static constexpr int pf(int k) { return split_f(k); }
    __host__ __device__ static constexpr int pg(int k) { return split_g(k); }
};

// ThetaSplit: the 9 flow planes in float16 as in Split, then the thermal
// block: one float32 plane holding theta = sum_i g_i (Eq. 41), then four
// float16 planes holding d_k = g_k - w theta for the moving directions k = 1..4
// (0-based: +x, +y, -x, -y; w = (4 + a)/20, the D2Q5 rest weight of Eq. 42),
// deviation plane k - 1. The rest population is g_0 = w_0 theta - (d_1 + d_2 +
// d_3 + d_4) (w_0 = (1 - a)/5), so a node's stored populations sum to its
// theta whatever the rounding of the deviations. Pulling g_k into a node needs
// the source node's theta and d_k, and g_0 the node's own four deviations: the
// thermal block is staged with one halo row on each side (R + 2 rows) instead
// of by plane group. Eg is the deviations' type; pg is not used.
struct ThetaSplit {
    using Ef = __half;
    using Eg = __half;
    static constexpr bool kSplit = true;
    static constexpr bool kTheta = true;
    static constexpr int kHalo = tma_halo(2);
    __host__ __device__ static constexpr int pf(int k) { return split_f(k); }
    __host__ __device__ static constexpr int pg(int k) { return k; }
};

// ThetaSplit stage of R rows: the flow groups (9 planes x R rows of float16),
// then theta (R + 2 rows of float32), then the deviations (4 planes x (R + 2)
// rows of float16); every part starts 128-byte aligned.
__host__ __device__ constexpr size_t theta_stage_th(int R) { return (size_t)9 * R * kTmaBox * 2; }
__host__ __device__ constexpr size_t theta_stage_d(int R) { return theta_stage_th(R) + (size_t)(R + 2) * kTmaBox * 4; }
__host__ __device__ constexpr size_t theta_stage_bytes(int R) { return theta_stage_d(R) + (size_t)4 * (R + 2) * kTmaBox * 2; }
// Shared-memory output tile of one item for the tensor-store epilogue: the
// item's R rows x W nodes (W = strip width) of every plane, [plane][row][node];
// split layouts put the thermal planes at a 128-byte aligned offset (a tensor
// copy's shared-memory address must be 128-byte aligned).
__host__ __device__ constexpr size_t round128(size_t x) { return (x + 127) & ~size_t(127); }
__host__ __device__ constexpr size_t out_g_offset(bool split, int R, int W, int f_bytes) {
    return split ? round128((size_t)9 * R * W * f_bytes) : 0;
}
__host__ __device__ constexpr size_t out_tile_bytes(bool split, int R, int W, int f_bytes, int g_bytes) {
    return split ? round128(out_g_offset(true, R, W, f_bytes) + (size_t)5 * R * W * g_bytes)
                 : round128((size_t)kPlanes * R * W * f_bytes);
}
// ThetaSplit output tile of R rows x W nodes: flow [9][R][W] float16, theta
// [R][W] float32, deviations [4][R][W] float16, each part 128-byte aligned.
__host__ __device__ constexpr size_t theta_out_th(int R, int W) { return round128((size_t)9 * R * W * 2); }
__host__ __device__ constexpr size_t theta_out_d(int R, int W) {
    return theta_out_th(R, W) + round128((size_t)R * W * 4);
}
__host__ __device__ constexpr size_t theta_out_bytes(int R, int W) {
    return theta_out_d(R, W) + round128((size_t)4 * R * W * 2);
}

// Tensor maps of the single-cavity TMA kernel for one source buffer: loads
// from the source (one-type layout: 6-plane and 4-plane boxes; split layout:
// 3-plane flow, 3-plane and 1-plane thermal boxes; ThetaSplit: 3-plane flow
// boxes, a theta box and a 4-plane deviation box of R + 2 rows) and the
// epilogue's stores to the destination (one-type: one 14-plane box; split: a
// 9-plane flow and a 5-plane thermal box; ThetaSplit: flow, theta and
// deviation boxes). The store maps span nx columns, so the padding columns
// of the last strip are never written.
struct TmaMaps {
    CUtensorMap ld[3];
    CUtensorMap st[3];
};

template <typename E, int NPT, bool SR>
__device__ __forceinline__ void put_vals(E* p, const float (&o)[NPT], float shift, unsigned (&r)[NPT]) {
    vec_put<E, NPT, SR>(p, o, shift, r);
}

// Where each plane group starts in a shared-memory stage, every start 128-byte
// aligned (a tensor copy's destination must be). One-type layout: groups Z, P,
// N of the 14 planes at elements 0, zP, zN. Split layout: the flow groups Z, P,
// N at flow elements 0, zP, zN; the thermal block at byte g_bytes, its groups
// Z, P, N at thermal elements 0, gP, gN. Each group is [plane][row][WB].
struct StageOffsets {
    int zP, zN;
    int g_bytes;
    int gP, gN;
    int d_bytes;  // ThetaSplit: theta at byte g_bytes, the deviation planes at byte d_bytes
};

// Pull, collide and store one work item (strip, row block) from its shared-
// memory stage, and report the Nusselt number of the rows it owns in the
// first strip. Called by every thread of the block (the Nusselt report is a
// warp collective); `ok` is false when the stage's wait expired.
// Geometry: strips of W nodes, shared-memory rows of WB elements (kHalo left
// of the strip), RC rows per item, plane groups placed as `so` says.
// TS: store the results into the shared-memory output tile `out` (see
// out_tile_bytes) for the block's tensor store, instead of to global memory.
template <typename L, int NPT, bool SR, bool TS = false>
__device__ __forceinline__ void process_item(const unsigned char* stage, const StepArgs& A, const StepConsts& K,
                                             int strip, int rb, int rg, int t, bool ok,
                                             unsigned salt, int W, int WB, int RC, const StageOffsets& so,
                                             unsigned char* out = nullptr, unsigned stage_cap = 0,
                                             unsigned out_cap = 0) {
    using Ef = typename L::Ef;
    using Eg = typename L::Eg;
    constexpr int HALO = L::kHalo;
    const long long PL = A.plane;
    const Ef* Sf = reinterpret_cast<const Ef*>(A.src);
    const Eg* Sgg = L::kSplit ? reinterpret_cast<const Eg*>(reinterpret_cast<const unsigned char*>(A.src) +
                                                            (size_t)9 * PL * sizeof(Ef))
                              : reinterpret_cast<const Eg*>(A.src);
    const Ef* stf = reinterpret_cast<const Ef*>(stage);
    const Eg* stg = L::kSplit ? reinterpret_cast<const Eg*>(stage + so.g_bytes) : reinterpret_cast<const Eg*>(stage);
    const float sh0 = K.gsh0, sh1 = K.gsh1;  // thermal storage shifts (0 unless g is 16-bit)
    const float sign_l_g = K.left_fixed ? -1.f : 1.f;
    const float sign_r_g = K.right_fixed ? -1.f : 1.f;
    const int j = rb * RC + rg;
    const int n0 = NPT * t;
    const int x0 = strip * W + n0;
    const bool row_ok = j < A.ny;
    const bool mine = ok && row_ok && rg < RC && n0 < W && x0 < A.nx;
    float theta[NPT];
#pragma unroll
    for (int e = 0; e < NPT; ++e) theta[e] = 0.f;
    // Plane p of a layout whose groups start at planes 0, p_P, p_N and at
    // elements 0, oP, oN of the stage.
    auto grouped = [&](int plane, int p_P, int p_N, int oP, int oN) {
        const int g0 = plane >= p_N ? p_N : plane >= p_P ? p_P : 0;
        const int off = plane >= p_N ? oN : plane >= p_P ? oP : 0;
        return off + ((plane - g0) * RC + rg) * WB;
    };
    auto rowf = [&](int plane) {
        return stf + (L::kSplit ? grouped(plane, 3, 6, so.zP, so.zN)
                                : grouped(plane, kGroupP, kGroupN, so.zP, so.zN));
    };
    auto rowg = [&](int plane) {
        return stg + (L::kSplit ? grouped(plane, 3, 4, so.gP, so.gN)
                                : grouped(plane, kGroupP, kGroupN, so.zP, so.zN));
    };
    bool bc = true;  // every index of this item in range (checked in bounds-checked builds)
#ifdef DMRT_BOUNDS_CHECK
    if (mine) {
        // The stage rows read (one shifted vector each way), the wall columns
        // and destination rows of every plane, the output tile, and the rows of
        // the wall-temperature and Nusselt arrays.
        bc = DMRT_IN(j, 0, A.ny, A.err) && DMRT_IN(HALO + n0 - NPT, 0, WB, A.err) &&
             DMRT_IN(HALO + n0 + 2 * NPT - 1, 0, WB, A.err);
        for (int k = 0; k < 9 && bc; ++k) {
            const long long b = (long long)(rowf(L::pf(k)) - stf) * (long long)sizeof(Ef);
            bc = DMRT_IN(b, 0, stage_cap, A.err) && DMRT_IN(b + (long long)WB * sizeof(Ef) - 1, 0, stage_cap, A.err);
        }
        if constexpr (L::kTheta) {
            // Theta rows rg .. rg + 2 and the same rows of the 4 deviation planes.
            const long long bt = so.g_bytes + (long long)(rg + 2) * WB * 4;
            const long long bd = so.d_bytes + ((long long)3 * (RC + 2) + rg + 2) * WB * 2;
            bc = bc && DMRT_IN(bt + (long long)WB * 4 - 1, 0, stage_cap, A.err) &&
                 DMRT_IN(bd + (long long)WB * 2 - 1, 0, stage_cap, A.err);
        } else {
            for (int k = 0; k < 5 && bc; ++k) {
                const long long b =
                    (long long)(rowg(L::pg(k)) - stg) * (long long)sizeof(Eg) + (L::kSplit ? so.g_bytes : 0);
                bc = DMRT_IN(b, 0, stage_cap, A.err) && DMRT_IN(b + (long long)WB * sizeof(Eg) - 1, 0, stage_cap, A.err);
            }
        }
        // Destination offsets within the flow and thermal blocks (ThetaSplit: a
        // thermal block of 6 float16-sized planes, theta taking two).
        const long long nfp = L::kSplit ? 9 : kPlanes, ngp = L::kTheta ? 6 : L::kSplit ? 5 : kPlanes;
        const long long ro = (long long)(j + A.row0) * A.pitch;
        bc = bc && DMRT_IN(ro + x0 + NPT - 1, 0, PL, A.err) && DMRT_IN(ro + A.nx - 1, 0, PL, A.err) &&
             DMRT_IN((nfp - 1) * PL + ro + x0, 0, nfp * PL, A.err) &&
             DMRT_IN((ngp - 1) * PL + ro + x0, 0, ngp * PL, A.err);
        if (TS)
            bc = bc && DMRT_IN(rg, 0, RC, A.err) && DMRT_IN(n0 + NPT - 1, 0, W, A.err) &&
                 DMRT_IN((long long)(L::kTheta ? theta_out_bytes(RC, W)
                                               : out_tile_bytes(L::kSplit, RC, W, sizeof(Ef), sizeof(Eg))) - 1,
                         0, out_cap, A.err);
    }
#endif
    if (mine && bc) {
        float F[9][NPT], Gq[5][NPT];
        lds_pull<0, NPT, HALO>(rowf(L::pf(0)), n0, F[0], 0.f);
        lds_pull<1, NPT, HALO>(rowf(L::pf(1)), n0, F[1], 0.f);
        lds_pull<0, NPT, HALO>(rowf(L::pf(2)), n0, F[2], 0.f);
        lds_pull<-1, NPT, HALO>(rowf(L::pf(3)), n0, F[3], 0.f);
        lds_pull<0, NPT, HALO>(rowf(L::pf(4)), n0, F[4], 0.f);
        lds_pull<1, NPT, HALO>(rowf(L::pf(5)), n0, F[5], 0.f);
        lds_pull<-1, NPT, HALO>(rowf(L::pf(6)), n0, F[6], 0.f);
        lds_pull<-1, NPT, HALO>(rowf(L::pf(7)), n0, F[7], 0.f);
        lds_pull<1, NPT, HALO>(rowf(L::pf(8)), n0, F[8], 0.f);
        // ThetaSplit: the node's own theta and deviations (g*_k = w theta + d_k of
        // the previous step's collision at this node, for g_0 and the walls).
        float thc[NPT], d1o[NPT], d2o[NPT], d3o[NPT], d4o[NPT];
        if constexpr (L::kTheta) {
            const float* sth = reinterpret_cast<const float*>(stage + so.g_bytes) + rg * WB;  // row j - 1
            const Eg* sd = reinterpret_cast<const Eg*>(stage + so.d_bytes) + rg * WB;
            const int DPB = (RC + 2) * WB;  // elements of one deviation plane in the stage
            float thl[NPT], thr[NPT], thd[NPT], thu[NPT], dv[NPT];
            lds_three<NPT, HALO>(sth + WB, n0, thl, thc, thr);
            lds_pull<0, NPT, HALO>(sth, n0, thd, 0.f);
            lds_pull<0, NPT, HALO>(sth + 2 * WB, n0, thu, 0.f);
            // g_k pulled from the source node x - e_k: w theta(source) + d_k(source).
            lds_left_own<NPT, HALO>(sd + WB, n0, dv, d1o);  // k = 1 (+x) from x - 1
#pragma unroll
            for (int e = 0; e < NPT; ++e) Gq[1][e] = fmaf(K.w1, thl[e], dv[e]);
            lds_right_own<NPT, HALO>(sd + 2 * DPB + WB, n0, dv, d3o);  // k = 3 (-x) from x + 1
#pragma unroll
            for (int e = 0; e < NPT; ++e) Gq[3][e] = fmaf(K.w1, thr[e], dv[e]);
            lds_pull<0, NPT, HALO>(sd + DPB, n0, dv, 0.f);  // k = 2 (+y) from row j - 1
            lds_pull<0, NPT, HALO>(sd + DPB + WB, n0, d2o, 0.f);
#pragma unroll
            for (int e = 0; e < NPT; ++e) Gq[2][e] = fmaf(K.w1, thd[e], dv[e]);
            lds_pull<0, NPT, HALO>(sd + 3 * DPB + 2 * WB, n0, dv, 0.f);  // k = 4 (-y) from row j + 1
            lds_pull<0, NPT, HALO>(sd + 3 * DPB + WB, n0, d4o, 0.f);
#pragma unroll
            for (int e = 0; e < NPT; ++e) {
                Gq[4][e] = fmaf(K.w1, thu[e], dv[e]);
                Gq[0][e] = fmaf(K.w0, thc[e], -((d1o[e] + d3o[e]) + (d2o[e] + d4o[e])));
            }
        } else {
            lds_pull<0, NPT, HALO>(rowg(L::pg(0)), n0, Gq[0], sh0);
            lds_pull<1, NPT, HALO>(rowg(L::pg(1)), n0, Gq[1], sh1);
            lds_pull<0, NPT, HALO>(rowg(L::pg(2)), n0, Gq[2], sh1);
            lds_pull<-1, NPT, HALO>(rowg(L::pg(3)), n0, Gq[3], sh1);
            lds_pull<0, NPT, HALO>(rowg(L::pg(4)), n0, Gq[4], sh1);
        }

        // Walls. Bottom row: links from below (f2, f5, f6, g2) bounce back from
        // the node's own opposites (f4, f7, f8, g4); top row the reverse.
        const Ef* rowjf = Sf + (size_t)(j + A.row0) * A.pitch;
        const Eg* rowjg = Sgg + (size_t)(j + A.row0) * A.pitch;
        if (j == 0 && A.wall_lo) {
            vec_ldg<Ef, NPT>(rowjf + L::pf(4) * PL + x0, F[2], 0.f);
            vec_ldg<Ef, NPT>(rowjf + L::pf(7) * PL + x0, F[5], 0.f);
            vec_ldg<Ef, NPT>(rowjf + L::pf(8) * PL + x0, F[6], 0.f);
            if constexpr (L::kTheta) {
#pragma unroll
                for (int e = 0; e < NPT; ++e) Gq[2][e] = fmaf(K.w1, thc[e], d4o[e]);
            } else {
                vec_ldg<Eg, NPT>(rowjg + L::pg(4) * PL + x0, Gq[2], sh1);
            }
        }
        if (j == A.ny - 1 && A.wall_hi) {
            vec_ldg<Ef, NPT>(rowjf + L::pf(2) * PL + x0, F[4], 0.f);
            vec_ldg<Ef, NPT>(rowjf + L::pf(5) * PL + x0, F[7], 0.f);
            vec_ldg<Ef, NPT>(rowjf + L::pf(6) * PL + x0, F[8], 0.f);
            if constexpr (L::kTheta) {
#pragma unroll
                for (int e = 0; e < NPT; ++e) Gq[4][e] = fmaf(K.w1, thc[e], d2o[e]);
            } else {
                vec_ldg<Eg, NPT>(rowjg + L::pg(2) * PL + x0, Gq[4], sh1);
            }
        }
        // Left wall (node x = 0): links with e_x = +1 (f1, f5, f8, g1).
        if (x0 == 0) {
            F[1][0] = ldg_one(rowjf + L::pf(3) * PL, 0.f);
            F[5][0] = ldg_one(rowjf + L::pf(7) * PL, 0.f);
            F[8][0] = ldg_one(rowjf + L::pf(6) * PL, 0.f);
            const float add = K.left_fixed ? K.abb * __ldg(A.hot + j) : 0.f;
            float g3;
            if constexpr (L::kTheta) g3 = fmaf(K.w1, thc[0], d3o[0]);
            else g3 = ldg_one(rowjg + L::pg(3) * PL, sh1);
            Gq[1][0] = sign_l_g * g3 + add;
        }
        // Right wall (node x = nx - 1): links with e_x = -1 (f3, f6, f7, g3).
        const int re = A.nx - 1 - x0;
        if (re < NPT) {
            const int xr = A.nx - 1;
            const float v3 = ldg_one(rowjf + L::pf(1) * PL + xr, 0.f);
            const float v6 = ldg_one(rowjf + L::pf(8) * PL + xr, 0.f);
            const float v7 = ldg_one(rowjf + L::pf(5) * PL + xr, 0.f);
            const float add = K.right_fixed ? K.abb * __ldg(A.cold + j) : 0.f;
            float vg = 0.f;
            if constexpr (!L::kTheta) vg = sign_r_g * ldg_one(rowjg + L::pg(1) * PL + xr, sh1) + add;
#pragma unroll
            for (int e = 0; e < NPT; ++e) {
                if (e == re) {
                    F[3][e] = v3;
                    F[6][e] = v6;
                    F[7][e] = v7;
                    if constexpr (L::kTheta) Gq[3][e] = sign_r_g * fmaf(K.w1, thc[e], d1o[e]) + add;
                    else Gq[3][e] = vg;
                }
            }
        }

        bool bad = false;
        collide_nodes<NPT>(F, Gq, K, theta, min(NPT, A.nx - x0), bad);
        Ef* Df;
        Eg* Dg;
        long long DP;  // plane stride of the destination, elements
        if constexpr (TS) {
            DP = (long long)RC * W;
            Df = reinterpret_cast<Ef*>(out) + rg * W + n0;
            Dg = reinterpret_cast<Eg*>(out + out_g_offset(L::kSplit, RC, W, sizeof(Ef))) + rg * W + n0;
        } else {
            DP = PL;
            Df = reinterpret_cast<Ef*>(A.dst) + (size_t)(j + A.row0) * A.pitch + x0;
            Dg = (L::kSplit ? reinterpret_cast<Eg*>(reinterpret_cast<unsigned char*>(A.dst) +
                                                    (size_t)9 * PL * sizeof(Ef))
                            : reinterpret_cast<Eg*>(A.dst)) +
                 (size_t)(j + A.row0) * A.pitch + x0;
        }
        // Stochastic rounding: each node's bits come from a hash of its index and the step.
        unsigned r[NPT];
#pragma unroll
        for (int e = 0; e < NPT; ++e)
            r[e] = SR ? hash32(((unsigned)(j + A.jglob0) * (unsigned)A.pitch + (unsigned)(x0 + e)) ^ salt) : 0u;
#pragma unroll
        for (int k = 0; k < 9; ++k) put_vals<Ef, NPT, SR>(Df + L::pf(k) * DP, F[k], 0.f, r);
        if constexpr (L::kTheta) {
            // theta (the collision keeps it) and d_k = g*_k - w theta, k = 1..4.
            float* Dth;
            Eg* Dd;
            if constexpr (TS) {
                Dth = reinterpret_cast<float*>(out + theta_out_th(RC, W)) + rg * W + n0;
                Dd = reinterpret_cast<Eg*>(out + theta_out_d(RC, W)) + rg * W + n0;
            } else {
                unsigned char* tb = reinterpret_cast<unsigned char*>(A.dst) + (size_t)9 * PL * sizeof(Ef);
                const size_t o = (size_t)(j + A.row0) * A.pitch + x0;
                Dth = reinterpret_cast<float*>(tb) + o;
                Dd = reinterpret_cast<Eg*>(tb + (size_t)PL * 4) + o;
            }
            Pack<float, NPT> tq;
#pragma unroll
            for (int e = 0; e < NPT; ++e) tq.v[e] = theta[e];
            *reinterpret_cast<Pack<float, NPT>*>(Dth) = tq;
#pragma unroll
            for (int k = 1; k < 5; ++k) {
                float dv[NPT];
#pragma unroll
                for (int e = 0; e < NPT; ++e) dv[e] = fmaf(-K.w1, theta[e], Gq[k][e]);
                put_vals<Eg, NPT, SR>(Dd + (k - 1) * DP, dv, 0.f, r);
            }
        } else {
#pragma unroll
            for (int k = 0; k < 5; ++k) put_vals<Eg, NPT, SR>(Dg + L::pg(k) * DP, Gq[k], k == 0 ? sh0 : sh1, r);
        }
        if (bad) atomicOr(A.err, kErrNonFinite);
    }
    // Nusselt number of row j from the first warp of the row's thread group
    // in the first strip; nodes 0 and 1 sit in lane 0 (or lanes 0 and 1).
    if (strip == 0 && t < 32) {
        float th1 = NPT > 1 ? theta[NPT > 1 ? 1 : 0] : 0.f;
        if constexpr (NPT == 1) th1 = __shfl_down_sync(kFull, theta[0], 1);
        const bool has_nu = mine && bc && t == 0;
        double nuj = 0.0;
        if (has_nu) {
            const double tw = (double)__ldg(A.hot + j);
            nuj = K.nu_scale * (8.0 * tw - 9.0 * (double)theta[0] + (double)th1);
        }
        nu_report(A, has_nu, j, nuj);
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

// Shared memory of the single-cavity kernel: S input stages, with TS two
// output tiles, and S mbarriers.
__host__ __device__ constexpr size_t step_tma_smem_bytes_theta(bool ts, int R, int S) {
    return (size_t)S * theta_stage_bytes(R) + (ts ? 2 * theta_out_bytes(R, kTmaBox - 2 * tma_halo(2)) : 0) +
           (size_t)S * 8;
}
__host__ __device__ constexpr size_t step_tma_smem_bytes(bool split, bool ts, int R, int S, int f_bytes,
                                                         int g_bytes) {
    return (size_t)S * tma_stage_bytes_fg(R, f_bytes, g_bytes) +
           (ts ? 2 * out_tile_bytes(split, R, kTmaBox - 2 * tma_halo(f_bytes < g_bytes ? f_bytes : g_bytes),
                                    f_bytes, g_bytes)
               : 0) +
           (size_t)S * 8;
}

// Epilogue. TS false: every thread stores its nodes to global memory. TS true:
// results go through a shared-memory output tile (two, alternating) and leave
// by tensor store: one elected thread stores item k after the barrier that
// ends it; before that barrier it waits until the store of item k - 1 has read
// its tile, which item k + 1 then overwrites.
template <typename L, int NPT, int R, int S, bool SR, bool TS>
__global__ void __launch_bounds__(R * (256 / NPT)) step_tma_kernel(const __grid_constant__ TmaMaps M,
                                                          StepArgs A, StepConsts K, TmaGeo T) {
    using Ef = typename L::Ef;
    using Eg = typename L::Eg;
    constexpr uint32_t kStageBytes =
        (uint32_t)(L::kTheta ? theta_stage_bytes(R) : tma_stage_bytes_fg(R, sizeof(Ef), sizeof(Eg)));
    constexpr int HALO = L::kHalo;
    constexpr int STRIP = kTmaBox - 2 * HALO;
    constexpr size_t kOutBytes =
        L::kTheta ? theta_out_bytes(R, STRIP) : out_tile_bytes(L::kSplit, R, STRIP, sizeof(Ef), sizeof(Eg));
    constexpr size_t kOutG = L::kTheta ? theta_out_th(R, STRIP) : out_g_offset(L::kSplit, R, STRIP, sizeof(Ef));
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* stages = smem_raw;
    unsigned char* outs = smem_raw + (size_t)S * kStageBytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(outs + (TS ? 2 * kOutBytes : 0));
    constexpr int TPR = 256 / NPT;   // threads per row of a strip
    constexpr int PB = R * kTmaBox;  // elements of one plane in a stage
    constexpr StageOffsets kSO =
        L::kTheta   ? StageOffsets{3 * PB, 6 * PB, (int)theta_stage_th(R), 0, 0, (int)theta_stage_d(R)}
        : L::kSplit ? StageOffsets{3 * PB, 6 * PB, (int)(9 * PB * sizeof(Ef)), 3 * PB, 4 * PB, 0}
                    : StageOffsets{kGroupP * PB, kGroupN * PB, 0, 0, 0, 0};
    const int tid = threadIdx.x;
    const int rg = tid / TPR;  // row of the block this thread works on
    const int t = tid % TPR;   // node group within the strip
    // Blocks beyond the item count (small grids: one) only sum the previous
    // step's Nusselt rows, which otherwise delay block 0's first item.
    const int n_items = T.n_strips * T.n_rowblocks;
    const bool nu_extra = (int)gridDim.x > n_items;
    const int G = nu_extra ? n_items : (int)gridDim.x;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
        mbar_fence_init();
    }
    grid_dep_wait();
    grid_dep_launch();
    // After an expired wait in an earlier launch the state is already invalid:
    // return at once instead of waiting again. One thread reads the word and
    // the barrier hands its answer to the whole block, so either every thread
    // of the block returns here or none does (the barrier also publishes the
    // mbarrier initialisation).
    if (__syncthreads_or(tid == 0 && (*reinterpret_cast<volatile unsigned*>(A.err) & kErrTimeout))) return;
    // The previous step's mean Nusselt number: block 0 before its first item, or
    // the extra block.
    if (nu_extra ? (int)blockIdx.x == n_items : blockIdx.x == 0) nu_finish_prev(A, true);
    if ((int)blockIdx.x >= G) return;

    // One item: every plane's R rows of row block rb, groups P and N taken one
    // row below / above (their e_y). One-type layout: ld[0] has 6-plane boxes
    // (group Z), ld[1] 4-plane boxes (P, N). Split layout: ld[0] has 3-plane
    // flow boxes, ld[1] 3-plane thermal boxes, ld[2] 1-plane thermal boxes.
    // ThetaSplit: ld[0] as Split, ld[1] theta boxes and ld[2] 4-plane
    // deviation boxes of R + 2 rows from the row below the item's first.
    auto issue = [&](const ItemCursor& c, int s) {
        const int x = c.strip * STRIP - HALO;
        const int j0 = c.rb * R + A.row0;  // buffer row of the item's first row
        unsigned char* st = stages + (size_t)s * kStageBytes;
        mbar_expect_tx(&bars[s], kStageBytes);
        if constexpr (!L::kSplit) {
            Ef* e = reinterpret_cast<Ef*>(st);
            tma_load_3d(e, &M.ld[0], x, j0, kGroupZ, &bars[s]);
            tma_load_3d(e + kGroupP * PB, &M.ld[1], x, j0 - 1, kGroupP, &bars[s]);
            tma_load_3d(e + kGroupN * PB, &M.ld[1], x, j0 + 1, kGroupN, &bars[s]);
        } else {
            Ef* f = reinterpret_cast<Ef*>(st);
            tma_load_3d(f, &M.ld[0], x, j0, 0, &bars[s]);
            tma_load_3d(f + 3 * PB, &M.ld[0], x, j0 - 1, 3, &bars[s]);
            tma_load_3d(f + 6 * PB, &M.ld[0], x, j0 + 1, 6, &bars[s]);
            if constexpr (L::kTheta) {
                tma_load_3d(st + kSO.g_bytes, &M.ld[1], x, j0 - 1, 0, &bars[s]);
                tma_load_3d(st + kSO.d_bytes, &M.ld[2], x, j0 - 1, 0, &bars[s]);
            } else {
                Eg* g = reinterpret_cast<Eg*>(st + (size_t)9 * PB * sizeof(Ef));
                tma_load_3d(g, &M.ld[1], x, j0, 0, &bars[s]);
                tma_load_3d(g + 3 * PB, &M.ld[2], x, j0 - 1, 3, &bars[s]);
                tma_load_3d(g + 4 * PB, &M.ld[2], x, j0 + 1, 4, &bars[s]);
            }
        }
    };
    // Item (strip, rb) from output tile o: a box of STRIP x R x planes at the
    // strip's first node (a multiple of 16 bytes).
    auto store = [&](int strip, int rb, const unsigned char* o) {
        const int x = strip * STRIP;
        const int j0 = rb * R + A.row0;
        tma_store_3d(&M.st[0], o, x, j0, 0);
        if constexpr (L::kSplit) tma_store_3d(&M.st[1], o + kOutG, x, j0, 0);
        if constexpr (L::kTheta) tma_store_3d(&M.st[2], o + theta_out_d(R, STRIP), x, j0, 0);
        bulk_commit();
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

    // Stochastic rounding: per-step salt (the step count is only written by the
    // previous launch, so every block reads the same value).
    unsigned salt = 0;
    if constexpr (SR) salt = hash32((unsigned)*A.step_in * 0x9e3779b9u + 0x632be5abu);
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

        unsigned char* out = outs + (size_t)(k & 1) * kOutBytes;
        process_item<L, NPT, SR, TS>(stages + (size_t)s * kStageBytes, A, K, cc.strip, cc.rb, rg, t, ok, salt,
                                     STRIP, kTmaBox, R, kSO, out, kStageBytes, (unsigned)kOutBytes);
        if constexpr (TS) {
            fence_async_smem();
            if (tid == 0) bulk_wait_read_all();  // item k - 1's store has read the other tile
        }
        // All threads are done with stage s and have filled tile k & 1; a
        // timeout anywhere ends the block.
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        if (TS && tid == 0) store(cc.strip, cc.rb, out);
        cc.advance(T.n_strips);
        if (++s == S) {
            s = 0;
            phase ^= 1u;
        }
    }
    if (TS && tid == 0) bulk_wait_all();  // the stores have read their tiles and written global memory
    if (timed_out && tid == 0) {
        atomicOr(A.err, kErrTimeout);
        // Let the copies this block issued land before its shared memory is released.
        for (int q = k; q < issued; ++q) mbar_wait_bounded(&bars[q % S], (uint32_t)((q / S) & 1));
    }
}

}  // namespace dmrt
