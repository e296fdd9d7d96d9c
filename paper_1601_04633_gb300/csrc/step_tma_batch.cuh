// Batched step: one launch advances every cavity of a sweep (float32 or mixed
// storage), built on the single-cavity item routine of step_tma.cuh.
#pragma once

#include "step_tma.cuh"

namespace dmrt {

// ---- batched sweep ------------------------------------------------------------
// One launch steps every cavity of a batch. The work items of all cavities
// form one list, cavity after cavity (strip fastest, then row block), which
// the blocks of the persistent grid share out as described at the kernel.
// Each cavity has its own strip geometry: strips of W nodes (a multiple of
// 32 NPT, so that every warp stays within one row), boxes WB = W + 2 HALO
// elements wide and RC rows tall (as many rows as the block's threads and the
// stage's shared memory allow), so narrow cavities keep the block's lanes busy.
// Float32 storage (one-type layout, two tensor maps per buffer: 6-plane and
// 4-plane boxes) or mixed storage (split layout, three: 3-plane flow boxes,
// 3-plane and 1-plane thermal boxes); then the epilogue's store maps into the
// other buffer (one-type: one 14-plane box W x RC; split: a 9-plane flow and a
// 5-plane thermal box), spanning nx columns; maps[(c * 2 + buffer) * 5 + k].
constexpr int kBatchMaps = 5;
constexpr int kBatchStoreMap = 3;

// Shared memory of a batched block: S stages, with TS two output tiles, and S
// mbarriers. A stage holds 5/4 of R rows of 256 elements per plane, so that
// strips whose threads per row divide the block keep every thread busy: a
// block of R 256 / NPT threads computes R 256 / W rows of a W-node strip, and
// those rows with their halo columns (W + 2 HALO elements each) take
// R 256 (1 + 2 HALO / W) elements, at most 5/4 of R 256 for W >= 8 HALO. An
// output tile holds an item's results without halos (at most R 256 nodes of
// every plane, the split layout's thermal block 128-byte aligned).
__host__ __device__ constexpr size_t batch_stage_bytes(int R, int f_bytes, int g_bytes) {
    return round128(tma_stage_bytes_fg(R, f_bytes, g_bytes) * 5 / 4);
}
__host__ __device__ constexpr size_t batch_out_bytes(int R, int f_bytes, int g_bytes) {
    return round128(tma_stage_bytes_fg(R, f_bytes, g_bytes) + 128);
}
__host__ __device__ constexpr size_t batch_smem_bytes(bool ts, int R, int S, int f_bytes, int g_bytes) {
    return (size_t)S * batch_stage_bytes(R, f_bytes, g_bytes) + (ts ? 2 * batch_out_bytes(R, f_bytes, g_bytes) : 0) +
           (size_t)S * 8;
}
// Geometry of a W-node strip in a batched tile (NPT nodes per thread, R rows,
// float32 one-type or mixed split layout, stage of stage_bytes): rows per item
// RC, as many as the block's threads and the stage allow, and the places of the
// plane groups in the stage, each 128-byte aligned (a tensor copy's
// destination must be). A pure function of the tile and W: the host builds
// the cavity records with it, and the kernel specialises its items on it.
struct BatchGeo {
    int RC;
    StageOffsets so;
};
__host__ __device__ constexpr long long batch_r128(long long bytes) { return (bytes + 127) / 128 * 128; }
__host__ __device__ constexpr long long batch_place(bool split, int rc, int WB, StageOffsets& so) {
    const long long row = (long long)rc * WB;
    if (!split) {
        const long long zP = batch_r128(6 * row * 4), zN = batch_r128(zP + 4 * row * 4);
        so = StageOffsets{(int)(zP / 4), (int)(zN / 4), 0, 0, 0, 0};
        return zN + 4 * row * 4;
    }
    const long long zP = batch_r128(3 * row * 2), zN = batch_r128(zP + 3 * row * 2), g0 = batch_r128(zN + 3 * row * 2);
    const long long gP = batch_r128(3 * row * 4), gN = batch_r128(gP + row * 4);
    so = StageOffsets{(int)(zP / 2), (int)(zN / 2), (int)g0, (int)(gP / 4), (int)(gN / 4), 0};
    return g0 + gN + row * 4;
}
__host__ __device__ constexpr BatchGeo batch_geometry(bool split, int npt, int R, int W, long long stage_bytes) {
    const int halo = tma_halo(split ? 2 : 4);
    const int WB = W + 2 * halo;
    const int block = R * (256 / npt);
    int rc = block / (W / npt);
    if (rc < 1) rc = 1;
    StageOffsets so{};
    while (rc > 1 && batch_place(split, rc, WB, so) > stage_bytes) --rc;
    batch_place(split, rc, WB, so);
    return BatchGeo{rc, so};
}

// A cavity's record, 16-byte aligned and sized so that the single-step kernel
// copies it into shared memory with the item's stage (one bulk copy), and the
// consumers read its arguments and constants there.
struct alignas(16) BatchCavity {
    StepArgs args[2];  // by source buffer: args[b] reads buffer b, writes 1 - b
    StepConsts K;
    int n_strips, n_rowblocks;
    int item_base;     // index of the cavity's first item in the batch list
    int W, WB, RC;     // strip width, box width, rows per item
    int tpr;           // threads per row = W / NPT
    unsigned tpr_magic;  // ceil(2^32 / tpr): tid / tpr = umulhi(tid, tpr_magic), exact for tid < 2^32 / tpr
    StageOffsets so;   // plane groups in the stage
    unsigned stage_bytes;  // bytes the item's tensor copies bring
};
static_assert(sizeof(BatchCavity) % 16 == 0, "bulk copies move multiples of 16 bytes");

// Bulk copy (not tensor-shaped) of `bytes` (a multiple of 16, both addresses
// 16-byte aligned) from global to shared memory, completing on an mbarrier.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Work distribution: block b first takes the static items [b Q, (b + 1) Q)
// (contiguous, so mostly one cavity), then draws single items from the
// dynamic pool [G Q, total) through a per-launch counter. Items of narrow
// cavities cost more per node (every item carries side walls and the Nusselt
// rows), so a static split by item count leaves a long tail; the pool evens it
// out. Which block computes an item does not change its result. The producer
// (thread 0) picks the items and passes each one's (cavity, strip, row block)
// to the consumers through shared memory with the stage; an item of -1 ends
// the block. Counters: ctr[parity] serves this launch; this launch zeroes
// ctr[1 - parity] for the next one. The producer's own latency is on the
// block's critical path (it computes its share of each item after issuing the
// next copies), so it reserves its next pool item one item ahead (the atomic
// completes while the item is computed) and finds an item's cavity in the
// compact item_base array (first item of each cavity; n_cav + 1 entries,
// cached in L1) rather than in the cavity records.
// TS: results go through a shared-memory output tile (two, alternating) and
// leave by tensor stores issued by one thread after the item's barrier, as in
// the single-cavity kernel, with the cavity's own store maps.
// MINB: blocks per SM that the registers must leave room for (1: no bound
// beyond the block size).
template <typename L, int NPT, int R, int S, bool SR = false, bool TS = false, int MINB = 1>
__global__ void __launch_bounds__(R * (256 / NPT), MINB)
    step_tma_batch_kernel(const BatchCavity* __restrict__ cav, const CUtensorMap* __restrict__ maps,
                          const int* __restrict__ item_base, int n_cav, int total_items, int static_per_block,
                          int parity, unsigned* batch_err, unsigned* ctr) {
    using Ef = typename L::Ef;
    using Eg = typename L::Eg;
    constexpr size_t kStageBytes = batch_stage_bytes(R, sizeof(Ef), sizeof(Eg));  // a multiple of 128
    constexpr size_t kOutBytes = batch_out_bytes(R, sizeof(Ef), sizeof(Eg));
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* stages = smem_raw;
    unsigned char* outs = smem_raw + (size_t)S * kStageBytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(outs + (TS ? 2 * kOutBytes : 0));
    __shared__ int4 stage_item[S];  // (cavity, strip, row block, item) of each stage; cavity -1: no more items
    __shared__ BatchCavity stage_cav[S];  // the record of each stage's cavity (copied with the stage)
    constexpr int HALO = L::kHalo;
    const int tid = threadIdx.x;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
        mbar_fence_init();
    }
    grid_dep_wait();
    grid_dep_launch();
    // A block-uniform decision (one reader, handed out by the barrier, which
    // also publishes the mbarrier initialisation): every thread returns or none.
    if (__syncthreads_or(tid == 0 && (*reinterpret_cast<volatile unsigned*>(batch_err) & kErrTimeout))) return;
    if (blockIdx.x == 0 && tid == 0) ctr[1 - parity] = 0u;
    // The previous step's mean Nusselt number of each cavity: blocks 0, 1, ...
    // before their first item.
    for (int cc = blockIdx.x; cc < n_cav; cc += gridDim.x) nu_finish_prev(cav[cc].args[parity], true);

    // Producer state (thread 0 only).
    int next_static = blockIdx.x * static_per_block;
    const int static_end = next_static + static_per_block;
    const int pool_base = gridDim.x * static_per_block;
    bool drained = false;
    int reserved = -1;  // pool item reserved ahead (-1: none)
    int pc = 0;  // cavity of the last item issued (items issued by a block increase)
    auto next_item = [&]() -> int {
        int it;
        if (next_static < static_end) {
            it = next_static++;
            if (next_static < static_end) return it;
        } else {
            if (drained) return -1;
            it = reserved >= 0 ? reserved : pool_base + (int)atomicAdd(&ctr[parity], 1u);
            if (it >= total_items) {
                drained = true;
                return -1;
            }
        }
        // The block's next item comes from the pool: reserve it now.
        reserved = pool_base + (int)atomicAdd(&ctr[parity], 1u);
        return it;
    };
    auto issue = [&](int it, int s) {
        if (it < 0) {
            stage_item[s] = make_int4(-1, 0, 0, -1);
            mbar_arrive(&bars[s]);  // completes the phase with nothing to load
            return;
        }
        while (pc + 1 < n_cav && __ldg(item_base + pc + 1) <= it) ++pc;
        const BatchCavity& bc = cav[pc];
        const int local = it - bc.item_base;
        const int rb = local / bc.n_strips;
        const int strip = local - rb * bc.n_strips;
        stage_item[s] = make_int4(pc, strip, rb, it);
        const int x = strip * bc.W - HALO;
        const int j0 = rb * bc.RC;
        const CUtensorMap* m = maps + ((size_t)pc * 2 + parity) * kBatchMaps;
        unsigned char* st = stages + (size_t)s * kStageBytes;
        mbar_expect_tx(&bars[s], bc.stage_bytes + (uint32_t)sizeof(BatchCavity));
        bulk_load(&stage_cav[s], &bc, (uint32_t)sizeof(BatchCavity), &bars[s]);
        if constexpr (!L::kSplit) {
            Ef* e = reinterpret_cast<Ef*>(st);
            tma_load_3d(e, m, x, j0, kGroupZ, &bars[s]);
            tma_load_3d(e + bc.so.zP, m + 1, x, j0 - 1, kGroupP, &bars[s]);
            tma_load_3d(e + bc.so.zN, m + 1, x, j0 + 1, kGroupN, &bars[s]);
        } else {
            Ef* f = reinterpret_cast<Ef*>(st);
            Eg* g = reinterpret_cast<Eg*>(st + bc.so.g_bytes);
            tma_load_3d(f, m, x, j0, 0, &bars[s]);
            tma_load_3d(f + bc.so.zP, m, x, j0 - 1, 3, &bars[s]);
            tma_load_3d(f + bc.so.zN, m, x, j0 + 1, 6, &bars[s]);
            tma_load_3d(g, m + 1, x, j0, 0, &bars[s]);
            tma_load_3d(g + bc.so.gP, m + 2, x, j0 - 1, 3, &bars[s]);
            tma_load_3d(g + bc.so.gN, m + 2, x, j0 + 1, 4, &bars[s]);
        }
    };

    int issued = 0;
    if (tid == 0) {
        for (int q = 0; q < S - 1; ++q) {
            issue(next_item(), q);
            issued = q + 1;
        }
    }
    bool timed_out = false;
    int k = 0, s = 0;
    uint32_t phase = 0;
    for (;; ++k) {
        if (tid == 0) {
            // Item k + S - 1 goes to the stage of item k - 1, released by the
            // barrier that ended it.
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(next_item(), s == 0 ? S - 1 : s - 1);
            issued = k + S;
        }
        const bool ok = mbar_wait_bounded(&bars[s], phase);
        // Every thread reads the same entry; a thread whose wait expired may
        // read a stale one, and the barrier below then ends the block anyway.
        const int4 w = stage_item[s];
        const bool work = ok && w.x >= 0 && DMRT_IN(w.x, 0, n_cav, batch_err);
        // The cavity's record, copied into shared memory with the stage (a stage
        // without an item holds a stale record: only its geometry is read, and
        // the item routine then touches no memory).
        const BatchCavity& bc = stage_cav[s];
        // Stochastic rounding: the cavity's per-step salt, as its own context would
        // use (its step count was written by the previous launch: read-only here).
        unsigned salt = 0;
        if constexpr (SR)
            if (work) salt = hash32((unsigned)__ldg(bc.args[parity].step_in) * 0x9e3779b9u + 0x632be5abu);
        unsigned char* out = outs + (size_t)(k & 1) * kOutBytes;
        unsigned char* st = stages + (size_t)s * kStageBytes;
        // The item with the strip geometry known at compile time: strip widths are
        // multiples of 32 NPT that fit a box, so 64, 128 or 192 with 2 nodes per
        // thread and 128 with 4 (one-node tiles take the geometry at run time).
        auto item_w = [&](auto wc) {
            constexpr int W = decltype(wc)::value;
            constexpr BatchGeo G = batch_geometry(L::kSplit, NPT, R, W, (long long)kStageBytes);
            constexpr int TPR = W / NPT;
            if (work && !DMRT_IN(bc.RC, G.RC, G.RC + 1, batch_err)) return;  // the record's RC is G.RC
            const int rg = work ? tid / TPR : 0;
            const int t = work ? tid - rg * TPR : tid;
            process_item<L, NPT, SR, TS>(st, bc.args[parity], bc.K, work ? w.y : 1, w.z, rg, t, work, salt, W, W + 2 * HALO,
                                         G.RC, G.so, out, (unsigned)kStageBytes, (unsigned)kOutBytes);
        };
        auto item_any = [&]() {
            const int rg = work ? (int)__umulhi((unsigned)tid, bc.tpr_magic) : 0;
            const int t = work ? tid - rg * bc.tpr : tid;
            process_item<L, NPT, SR, TS>(st, bc.args[parity], bc.K, work ? w.y : 1, w.z, rg, t, work, salt, bc.W, bc.WB,
                                         bc.RC, bc.so, out, (unsigned)kStageBytes, (unsigned)kOutBytes);
        };
        const int Wrec = work ? bc.W : 0;
        if constexpr (NPT == 2) {
            if (Wrec == 128) item_w(std::integral_constant<int, 128>{});
            else if (Wrec == 192) item_w(std::integral_constant<int, 192>{});
            else if (Wrec == 64) item_w(std::integral_constant<int, 64>{});
            else item_any();
        } else if constexpr (NPT == 4) {
            if (Wrec == 128) item_w(std::integral_constant<int, 128>{});
            else item_any();
        } else {
            item_any();
        }
        if constexpr (TS) {
            fence_async_smem();
            if (tid == 0) bulk_wait_read_all();  // item k - 1's store has read the other tile
        }
        // One barrier per item: it releases the stage and tells every thread
        // whether any wait expired; with none expired, w is the same valid
        // entry in every thread, so the end test is block-uniform.
        if (__syncthreads_count(!ok)) {
            timed_out = true;
            break;
        }
        if (w.x < 0) break;
        if (TS && tid == 0 && work) {
            // The item's tile (W x RC nodes of every plane) to the other buffer.
            const CUtensorMap* m = maps + ((size_t)w.x * 2 + parity) * kBatchMaps + kBatchStoreMap;
            const int x = w.y * bc.W, j0 = w.z * bc.RC;
            tma_store_3d(m, out, x, j0, 0);
            if constexpr (L::kSplit) tma_store_3d(m + 1, out + out_g_offset(true, bc.RC, bc.W, sizeof(Ef)), x, j0, 0);
            bulk_commit();
        }
        if (++s == S) {
            s = 0;
            phase ^= 1u;
        }
    }
    if (TS && tid == 0) bulk_wait_all();  // the stores have read their tiles and written global memory
    if (timed_out && tid == 0) {
        atomicOr(batch_err, kErrTimeout);
        for (int q = k; q < issued; ++q) mbar_wait_bounded(&bars[q % S], (uint32_t)((q / S) & 1));
    }
}

// Sums each cavity's last step of a run (one block of 256 threads per cavity).
static __global__ void nu_finalize_batch_kernel(const BatchCavity* __restrict__ cav, int parity) {
    nu_finish_prev(cav[blockIdx.x].args[parity], false);
}

}  // namespace dmrt

namespace dmrt {

// ---- batched sweep, several time steps per launch ------------------------------
// The cavities of a batch are independent: step s + 1 of cavity c needs only
// cavity c's step s to be complete (its pull reads neighbouring rows of that
// state, and it overwrites the buffer step s read). So one launch can advance
// every cavity by K steps without a grid-wide barrier between them: the work
// list is every (step, cavity, item) in step-major order, handed out one item
// at a time from a queue counter, and an item of step s + 1 of cavity c is
// loaded only once cavity c's step s is complete. Blocks keep their copy
// pipeline full across step boundaries, and no launch boundary (ramp, tail,
// launch gap) sits between steps.
//
// Progress: a block waits for a dependency only when it has computed every
// item it has loaded (the producer first tries without waiting; if the next
// item's cavity is not ready it lets the block compute the current item and
// waits after that). A waited-for step is always earlier than the step of the
// waiting block's earliest held item, and every item of an earlier step was
// taken from the queue by a running block, so no wait can be circular. Every
// wait is bounded (%globaltimer); on expiry the launch records kErrTimeout.
//
// Completion of a cavity's step: every thread fences its stores, the block
// barrier follows, thread 0 counts the item (done[c]); the block completing
// the cavity's step sums the step's per-row Nusselt numbers in warp 0 (the
// same fixed order as nu_finish_prev: partial p over rows p, p + 256, ...;
// lane l adds its partials pairwise, then a butterfly), appends the mean to
// the cavity's ring, and publishes ready[c] = s + 1 (a fence, then the store).
// The consumer of ready[c] acquires it and orders the following tensor copies
// after it with a proxy fence. Loads of the wall columns (ld.global.cg in
// process_item) bypass the non-coherent cache, since the state they read was
// written by this launch.
//
// Synchronisation words: two sets of (queue counter, done[n], ready[n]), by
// launch parity lp; a launch zeroes the other set for the next one.
__host__ __device__ constexpr int mstep_set_words(int n_cav) { return 32 + 2 * n_cav; }

__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Waits (bounded) until *p >= want; acquire: later reads see what the publisher wrote before.
__device__ __forceinline__ bool wait_at_least(const unsigned* p, unsigned want,
                                              unsigned long long limit_ns = kWaitLimitNs) {
    if (*reinterpret_cast<const volatile unsigned*>(p) >= want) {
        __threadfence();
        return true;
    }
    const unsigned long long t0 = global_ns();
    while (*reinterpret_cast<const volatile unsigned*>(p) < want) {
        if (global_ns() - t0 > limit_ns) return false;
        __nanosleep(64);
    }
    __threadfence();
    return true;
}

template <typename L, int NPT, int R, int S, bool SR = false>
__global__ void __launch_bounds__(R * (256 / NPT))
    step_tma_batch_mstep_kernel(const BatchCavity* __restrict__ cav, const CUtensorMap* __restrict__ maps,
                                const int* __restrict__ item_base, int n_cav, int items_per_step, int K,
                                int parity, unsigned* batch_err, unsigned* sync, int lp) {
    using Ef = typename L::Ef;
    using Eg = typename L::Eg;
    constexpr size_t kStageBytes = batch_stage_bytes(R, sizeof(Ef), sizeof(Eg));
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* stages = smem_raw;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + (size_t)S * kStageBytes);
    // (cavity, strip, row block, step) of each stage; cavity -1: no more items, -2: abort.
    __shared__ int4 stage_item[S];
    constexpr int HALO = L::kHalo;
    const int tid = threadIdx.x;
    const int words = mstep_set_words(n_cav);
    unsigned* set = sync + (size_t)lp * words;
    unsigned* ctr = set;
    unsigned* done = set + 32;
    unsigned* ready = set + 32 + n_cav;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
        mbar_fence_init();
    }
    grid_dep_wait();
    grid_dep_launch();
    if (__syncthreads_or(tid == 0 && (*reinterpret_cast<volatile unsigned*>(batch_err) & kErrTimeout))) return;
    {
        // The previous launch used the other set and has completed: zero it for the next one.
        unsigned* other = sync + (size_t)(1 - lp) * words;
        for (int i = blockIdx.x * blockDim.x + tid; i < words; i += gridDim.x * blockDim.x) other[i] = 0u;
    }
    const int total = K * items_per_step;

    // Producer state (thread 0): the next item to issue (a queue index, or
    // >= total for the end), one reserved after it, and the count issued.
    int next_g = 0, resv_g = 0, issued = 0;
    if (tid == 0) {
        next_g = (int)atomicAdd(ctr, 1u);
        resv_g = next_g < total ? (int)atomicAdd(ctr, 1u) : total;
    }
    auto decode = [&](int g, int& c, int& st, int& local) {
        st = g / items_per_step;
        const int r = g - st * items_per_step;
        int lo = 0, hi = n_cav - 1;  // last cavity whose first item <= r
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(item_base + mid) <= r) lo = mid;
            else hi = mid - 1;
        }
        c = lo;
        local = r - __ldg(item_base + c);
    };
    // Issue the next item into stage `s` if its cavity's previous step is
    // complete (wait: spin up to the limit; else one look). Returns false if
    // not issued (not ready, or the wait expired: *expired then true).
    auto try_issue = [&](int s, bool wait, bool* expired) -> bool {
        if (next_g >= total) {
            stage_item[s] = make_int4(-1, 0, 0, 0);
            mbar_arrive(&bars[s]);  // completes the phase with nothing to load
            return true;
        }
        int c, st, local;
        decode(next_g, c, st, local);
        if (st > 0) {
            const unsigned* rp = ready + c;
            if (wait) {
                if (!wait_at_least(rp, (unsigned)st)) {
                    *expired = true;
                    stage_item[s] = make_int4(-2, 0, 0, 0);
                    mbar_arrive(&bars[s]);
                    return false;
                }
            } else {
                if (*reinterpret_cast<const volatile unsigned*>(rp) < (unsigned)st) return false;
                __threadfence();
            }
            fence_proxy_async_global();  // the tensor copies below read what the publisher's blocks wrote
        }
        const BatchCavity& bc = cav[c];
        const int rb = local / bc.n_strips;
        const int strip = local - rb * bc.n_strips;
        stage_item[s] = make_int4(c, strip, rb, st);
        const int src = parity ^ (st & 1);
        const int x = strip * bc.W - HALO;
        const int j0 = rb * bc.RC;
        const CUtensorMap* m = maps + ((size_t)c * 2 + src) * kBatchMaps;
        unsigned char* sp = stages + (size_t)s * kStageBytes;
        mbar_expect_tx(&bars[s], bc.stage_bytes);
        if constexpr (!L::kSplit) {
            Ef* e = reinterpret_cast<Ef*>(sp);
            tma_load_3d(e, m, x, j0, kGroupZ, &bars[s]);
            tma_load_3d(e + bc.so.zP, m + 1, x, j0 - 1, kGroupP, &bars[s]);
            tma_load_3d(e + bc.so.zN, m + 1, x, j0 + 1, kGroupN, &bars[s]);
        } else {
            Ef* f = reinterpret_cast<Ef*>(sp);
            Eg* g = reinterpret_cast<Eg*>(sp + bc.so.g_bytes);
            tma_load_3d(f, m, x, j0, 0, &bars[s]);
            tma_load_3d(f + bc.so.zP, m, x, j0 - 1, 3, &bars[s]);
            tma_load_3d(f + bc.so.zN, m, x, j0 + 1, 6, &bars[s]);
            tma_load_3d(g, m + 1, x, j0, 0, &bars[s]);
            tma_load_3d(g + bc.so.gP, m + 2, x, j0 - 1, 3, &bars[s]);
            tma_load_3d(g + bc.so.gN, m + 2, x, j0 + 1, 4, &bars[s]);
        }
        next_g = resv_g;
        resv_g = next_g < total ? (int)atomicAdd(ctr, 1u) : total;
        return true;
    };

    bool timed_out = false;
    uint32_t phase = 0;
    int k = 0;
    for (int s = 0;; ++k) {
        bool expired = false;
        if (tid == 0) {
            // Items k .. k + S - 1 may be in flight; their stages were released
            // by the barriers that ended items k - S .. k - 1. Item k itself is
            // waited for only when it is not loaded yet: then every item this
            // block took is computed, and it holds nothing another block needs.
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            while (issued < k + S) {
                if (!try_issue(issued % S, issued == k, &expired)) break;
                ++issued;
            }
        }
        const bool ok = mbar_wait_bounded(&bars[s], phase);
        const int4 w = stage_item[s];
        const bool work = ok && w.x >= 0 && DMRT_IN(w.x, 0, n_cav, batch_err);
        const BatchCavity& bc = cav[work ? w.x : 0];
        const int tpr = bc.tpr;
        const int rg = tid / tpr;
        const int t = tid - rg * tpr;
        const int src = parity ^ (w.w & 1);
        unsigned salt = 0;
        if constexpr (SR)
            if (work)
                salt = hash32((unsigned)(__ldcg(bc.args[parity].step_in) + w.w) * 0x9e3779b9u + 0x632be5abu);
        process_item<L, NPT, SR>(stages + (size_t)s * kStageBytes, bc.args[src], bc.K, work ? w.y : 1, w.z, rg, t,
                                 work, salt, bc.W, bc.WB, bc.RC, bc.so, nullptr, (unsigned)kStageBytes);
        __threadfence();  // this thread's stores (state, Nusselt rows) before the item is counted
        if (__syncthreads_count(!ok || w.x == -2)) {
            timed_out = true;
            break;
        }
        if (w.x < 0) break;
        // Count the item; the block completing the cavity's step sums its Nusselt rows.
        if (tid < 32) {
            unsigned last = 0;
            if (tid == 0) {
                const unsigned want = (unsigned)((w.w + 1) * (bc.n_strips * bc.n_rowblocks));
                last = atomicAdd(done + w.x, 1u) + 1u == want;
            }
            last = __shfl_sync(kFull, last, 0);
            if (last) {
                __threadfence();
                const StepArgs& A = bc.args[src];
                double acc8[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    double acc = 0.0;
                    int r = tid + 32 * q;
                    if (r < A.ny) {  // the partial starts from its first row
                        acc = __ldcg(A.nu_rows + r);
                        r += 256;
                    }
                    for (; r + 3 * 256 < A.ny; r += 4 * 256) {
                        double v[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) v[i] = __ldcg(A.nu_rows + r + 256 * i);
#pragma unroll
                        for (int i = 0; i < 4; ++i) acc += v[i];
                    }
                    for (; r < A.ny; r += 256) acc += __ldcg(A.nu_rows + r);
                    acc8[q] = acc;
                }
                double sum = nu_combine(acc8, nu_partials(A.ny));
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(kFull, sum, o);
                if (tid == 0) {
                    const long long t0 = __ldcg(bc.args[parity].step_in);
                    const double mean = sum * A.nu_inv;
                    A.nu_ring[(t0 + w.w) % A.cap] = mean;
                    *A.nu_last = mean;
                    if (w.w == K - 1) {
                        // After the launch's K steps (K even) the state is back in
                        // buffer `parity`, whose step counter slot now holds t0 + K;
                        // every step's rows are summed, so nothing is pending.
                        *const_cast<long long*>(bc.args[parity].step_in) = t0 + K;
                        *A.pending = 0u;
                    }
                    __threadfence();
                    *reinterpret_cast<volatile unsigned*>(ready + w.x) = (unsigned)(w.w + 1);
                }
            }
        }
        if (++s == S) {
            s = 0;
            phase ^= 1u;
        }
    }
    if (timed_out && tid == 0) {
        atomicOr(batch_err, kErrTimeout);
        // Wait (bounded) for the copies this block issued before releasing its shared memory.
        for (int q = k; q < issued; ++q) mbar_wait_bounded(&bars[q % S], (uint32_t)((q / S) & 1));
    }
}

}  // namespace dmrt
