// Fused double-MRT steps for small float32 cavities, the whole state held on
// chip: one thread-block cluster (up to 16 blocks on 16 SMs) keeps both
// population buffers of the cavity in its blocks' shared memory and runs many
// time steps per launch.
//
// Block r of the cluster owns rows [r rows_per, (r + 1) rows_per) of the
// cavity; its shared memory holds those rows of both buffers plus one halo row
// below and one above, 14 planes [row][x] each, in the device plane order of
// lattice.cuh. One thread per node (looping when a block has more nodes than
// threads). Every pull reads this block's shared memory: when a thread stores
// its node of the block's first row it also stores the downward-moving
// populations (e_y = -1) into the halo row above of the previous block's
// destination buffer, and for the last row the upward-moving ones (e_y = +1)
// into the halo row below of the next block's (distributed shared memory
// stores, which do not wait for a reply). Between steps one cluster barrier
// (release / acquire at cluster scope) publishes the new buffers, halo rows
// included. The walls are the same rules, in the same arithmetic, as the other
// step kernels, and the collision is the same routine, so every step gives
// the other kernels' bits. No step touches global memory except the wall
// temperatures, the Nusselt ring and the error word.
//
// Nusselt number (Eqs. 18-19): the pre-collision temperatures at x = 0 and 1 of
// each row are staged in shared memory (double-buffered by step parity). After
// the step's cluster barrier, an extra warp of each block (it owns no nodes)
// computes its rows' values and writes them into block 0's shared row array
// (distributed shared memory, by step parity), and a second extra warp of
// block 0 sums the previous step's rows in the fixed order of nu_finish_prev
// (partial p over rows p, p + 256, ...; lane l adds its partials pairwise;
// butterfly over the lanes) and appends the mean to the ring, while the other
// warps compute the next step; one more barrier after the last step lets it
// sum that step too.
//
// The launch starts from the state in global buffer `parity` (copied in), and
// ends by copying the final state to global buffer parity ^ (K & 1), the last
// step's per-row Nusselt values to its rows array, the step counter slot and
// a cleared pending flag: afterwards the context is exactly as after K steps
// of the other kernels. The cluster barrier is the hardware's (every block
// executes the same K iterations, so every block arrives); there is no
// spin-wait in this kernel.
#pragma once
#include <cooperative_groups.h>

#include "lattice.cuh"

namespace dmrt {

struct ClusterArgs {
    StepArgs A[2];   // global buffers and Nusselt arrays, by source buffer
    StepConsts K;
    int steps;       // time steps of the launch
    int parity;      // global buffer holding the state at launch
    int rows_per;    // rows per block
    // Recompute mode (start != nullptr; the adjoint's segment recompute):
    // start from the state at `start` (same layout as a population buffer) and
    // touch nothing but the record (no Nusselt numbers, no context buffers or
    // counters). In either mode, with record != nullptr, the state after step
    // s is also written to record + s * record_stride.
    const float* start;
    float* record;
    long long record_stride;  // floats between recorded states
};

// Means kept in block 0's shared memory between their flushes to the ring.
constexpr int kClusterNuChunk = 1024;

// Threads of a cluster block: one per node of its rows (at most 960), rounded up
// to whole warps, and two Nusselt warps (rows; block 0: the sums).
__host__ __device__ constexpr int cluster_threads(int rows_per, int nx) {
    return ((rows_per * nx + 31) / 32 * 32 < 960 ? (rows_per * nx + 31) / 32 * 32 : 960) + 64;
}

__host__ __device__ constexpr size_t cluster_smem_bytes(int rows_per, int nx, int ny) {
    return (size_t)2 * kPlanes * (rows_per + 2) * nx * sizeof(float)  // both buffers, with halo rows
           + (((size_t)6 * rows_per * sizeof(float) + 15) & ~size_t(15))  // theta at x = 0, 1 (by step parity); walls
           + (size_t)kClusterNuChunk * sizeof(double)                  // means not yet in the ring (block 0)
           + (size_t)2 * ny * sizeof(double);                         // Nusselt rows (block 0), by step parity
}

// Sum of rows[0..ny) by warp 0 in the fixed order of nu_finish_prev (the result in every lane).
__device__ __forceinline__ double warp_fixed_sum(const double* rows, int ny, int lane) {
    double p8[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int r0q = lane + 32 * q;
        double acc = r0q < ny ? rows[r0q] : 0.0;
        for (int r = r0q + 256; r < ny; r += 256) acc += rows[r];
        p8[q] = acc;
    }
    double s = nu_combine(p8, nu_partials(ny));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    return s;
}

// Bulk copy (asynchronous proxy) of `bytes` bytes, a multiple of 16, from this
// block's shared memory to global memory; both addresses 16-byte aligned.
__device__ __forceinline__ void cluster_bulk_s2g(float* g, const float* s, unsigned bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(g),
                 "r"((unsigned)__cvta_generic_to_shared(s)), "r"(bytes)
                 : "memory");
}

// MAXT: the largest block it is launched with (the compiler may give a block of
// at most 320 or 640 threads more registers per thread, hence more
// independent instructions in flight along a node's chain). ONE: every block
// has at most one node per node thread (rows_per * nx <= blockDim.x - 64);
// otherwise a thread has a second node, nwork further on (the host keeps
// blocks within two nodes per node thread). A thread's nodes, and with them
// every shared-memory offset, are fixed across steps.
template <int MAXT, bool ONE>
__global__ void __launch_bounds__(MAXT) step_cluster_kernel(const __grid_constant__ ClusterArgs C) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int csize = (int)cl.num_blocks();
    const StepArgs& A0 = C.A[C.parity];
    const StepConsts& K = C.K;
    const int nx = A0.nx, ny = A0.ny, pitch = A0.pitch;
    const long long PL = A0.plane;
    const int RP = C.rows_per;
    const int r0 = rank * RP;
    const int nr = max(0, min(RP, ny - r0));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int plane_sm = (RP + 2) * nx;  // floats per plane in shared memory: rows -1 .. RP
    const int nwork = (int)blockDim.x - 64;  // node threads; then the two Nusselt warps
    const bool nu_warp = (int)threadIdx.x >= nwork;
    const bool sum_warp = (int)threadIdx.x >= nwork + 32;

    extern __shared__ __align__(16) unsigned char smem_c[];
    float* sb[2] = {reinterpret_cast<float*>(smem_c), reinterpret_cast<float*>(smem_c) + kPlanes * plane_sm};
    float* th01 = reinterpret_cast<float*>(smem_c) + 2 * kPlanes * plane_sm;  // [step parity][row][x = 0, 1]
    float* walls = th01 + 4 * RP;  // hot and cold wall temperatures of this block's rows
    double* nur = reinterpret_cast<double*>(smem_c + cluster_smem_bytes(RP, nx, ny) - (size_t)2 * ny * sizeof(double));
    double* means = nur - kClusterNuChunk;

    grid_dep_wait();
    grid_dep_launch();
    const bool rec = C.start != nullptr;
    // Recorded states: in the form for the largest blocks, when the rows fill
    // the pitch (a block's rows are then one contiguous run per plane, 16-byte
    // aligned in shared memory and in global memory), one lane of the
    // Nusselt-rows warp copies them out in bulk after each step's barrier, off
    // the node warps' path; else every node thread stores its node. (The forms
    // for smaller blocks keep the stores: the copy code there cost their
    // unrecorded steps 6-10 % through register allocation.)
    const bool bulk_rec = MAXT == 1024 && C.record != nullptr && pitch == nx && (nx & 3) == 0;
    // The state of this block's rows and of the rows next to them, from global
    // buffer `parity` (recompute mode: from `start`); halo rows beyond the
    // cavity's walls read as zero in both buffers (the wall rules replace
    // what a pull would take from them).
    for (int i = threadIdx.x; i < (nr + 2) * nx; i += blockDim.x) {
        const int rr = i / nx - 1, x = i - (rr + 1) * nx;
        const int j = r0 + rr;
        if (!DMRT_IN(i, 0, plane_sm, A0.err)) continue;
        if (j < 0 || j >= ny) {
#pragma unroll
            for (int p = 0; p < kPlanes; ++p) sb[0][p * plane_sm + i] = sb[1][p * plane_sm + i] = 0.f;
            continue;
        }
        if (!DMRT_IN((long long)j * pitch + x, 0, PL, A0.err)) continue;
        const float* src = (rec ? C.start : A0.src) + (size_t)j * pitch + x;
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) sb[0][p * plane_sm + i] = src[p * PL];
    }
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
        walls[r] = __ldg(A0.hot + r0 + r);
        walls[RP + r] = __ldg(A0.cold + r0 + r);
    }
    const long long t0 = *A0.step_in;
    if (!rec && rank == 0 && warp == 0 && *A0.pending) {
        // Rows of an earlier step not yet summed (a single step launched before).
        const double sum = warp_fixed_sum(A0.prev_rows, ny, lane);
        if (lane == 0) {
            A0.nu_ring[(t0 - 1) % A0.cap] = sum * A0.nu_inv;
            *A0.nu_last = sum * A0.nu_inv;
        }
    }
    cl.sync();

    const float sign_l_g = K.left_fixed ? -1.f : 1.f;
    const float sign_r_g = K.right_fixed ? -1.f : 1.f;
    bool bad = false;
    // The halo rows this block fills in its neighbours' buffers: the row above
    // the previous block's RP rows, the row below the next block's rows.
    float* const below0 = rank > 0 ? cl.map_shared_rank(sb[0], rank - 1) + (size_t)(RP + 1) * nx : nullptr;
    float* const below1 = rank > 0 ? cl.map_shared_rank(sb[1], rank - 1) + (size_t)(RP + 1) * nx : nullptr;
    float* const above0 = rank + 1 < csize ? cl.map_shared_rank(sb[0], rank + 1) : nullptr;
    float* const above1 = rank + 1 < csize ? cl.map_shared_rank(sb[1], rank + 1) : nullptr;
    double* nu_rows0 = cl.map_shared_rank(nur, 0);
    // The spare warps' Nusselt work (Eqs. 18-19). Rows of step q: from the
    // temperatures at x = 0 and 1 into block 0's row array (by step parity).
    auto nu_rows_of = [&](int q) {
        const float* th = th01 + (q & 1) * 2 * RP;
        double* dst = nu_rows0 + (size_t)(q & 1) * ny;
        for (int r = lane; r < nr; r += 32) {
            const int j = r0 + r;
            if (!DMRT_IN(j, 0, ny, A0.err)) continue;
            dst[j] = K.nu_scale * (8.0 * (double)walls[r] - 9.0 * (double)th[2 * r] + (double)th[2 * r + 1]);
        }
    };
    // Block 0: the mean of step q's rows, kept in shared memory; a full chunk
    // goes to the ring (global stores only once per kClusterNuChunk steps), and
    // only the chunk's last `cap` means, so that no two lanes write one slot (a
    // smaller ring wraps within a chunk).
    auto nu_mean_of = [&](int q) {
        const double sum = warp_fixed_sum(nur + (size_t)(q & 1) * ny, ny, lane);
        if (lane == 0) means[q % kClusterNuChunk] = sum * A0.nu_inv;
        __syncwarp();
        if (q % kClusterNuChunk == kClusterNuChunk - 1 || q == C.steps - 1) {
            const int first = q - q % kClusterNuChunk;
            const long long n = q - first + 1;
            const int q0 = (int)(n > A0.cap ? n - A0.cap : 0);
            for (int k = q0 + lane; k <= q - first; k += 32) A0.nu_ring[(t0 + first + k) % A0.cap] = means[k];
            if (lane == 0) *A0.nu_last = means[q - first];
        }
    };
    // One node's step s: node i of the block (row r, column x, cavity row j)
    // from buffer S into Dst, the halo rows into the neighbours' Dbelow/Dabove.
    auto node_step = [&](int s, int i, int r, int x, int j, const float* S, float* Dst, float* Dbelow,
                         float* Dabove) {
        if (!DMRT_IN(i + nx, 0, plane_sm, A0.err) || !DMRT_IN(j, 0, ny, A0.err) || !DMRT_IN(r, 0, RP, A0.err))
            return;
        // Post-collision value of plane p at (x, local row rr = -1 .. nr) of
        // this step's state. (Across the cavity's bottom and top walls the
        // halo rows hold zeros, replaced by the wall rules below.)
        auto at = [&](int p, int rr, int xx) -> float { return S[p * plane_sm + (rr + 1) * nx + xx]; };
        auto own = [&](int p) { return S[p * plane_sm + (r + 1) * nx + x]; };
        // Pull (Eqs. 25, 36): value of direction k at x comes from x - e_k, where
        // that node exists; links across a wall are replaced below.
        float f[9], g[5];
        const int xl = x > 0 ? x - 1 : x, xr = x + 1 < nx ? x + 1 : x;
        f[0] = own(plane_f(0));
        f[1] = at(plane_f(1), r, xl);
        f[2] = at(plane_f(2), r - 1, x);
        f[3] = at(plane_f(3), r, xr);
        f[4] = at(plane_f(4), r + 1, x);
        f[5] = at(plane_f(5), r - 1, xl);
        f[6] = at(plane_f(6), r - 1, xr);
        f[7] = at(plane_f(7), r + 1, xr);
        f[8] = at(plane_f(8), r + 1, xl);
        g[0] = own(plane_g(0));
        g[1] = at(plane_g(1), r, xl);
        g[2] = at(plane_g(2), r - 1, x);
        g[3] = at(plane_g(3), r, xr);
        g[4] = at(plane_g(4), r + 1, x);
        // Bottom wall (j = 0): f2, f5, f6, g2 from the node's own opposites; top the reverse.
        if (j == 0) {
            f[2] = own(plane_f(4));
            f[5] = own(plane_f(7));
            f[6] = own(plane_f(8));
            g[2] = own(plane_g(4));
        }
        if (j == ny - 1) {
            f[4] = own(plane_f(2));
            f[7] = own(plane_f(5));
            f[8] = own(plane_f(6));
            g[4] = own(plane_g(2));
        }
        // Left wall (x = 0): links with e_x = +1.
        if (x == 0) {
            f[1] = own(plane_f(3));
            f[5] = own(plane_f(7));
            f[8] = own(plane_f(6));
            const float add = K.left_fixed ? K.abb * walls[r] : 0.f;
            g[1] = sign_l_g * own(plane_g(3)) + add;
        }
        // Right wall (x = nx - 1): links with e_x = -1.
        if (x == nx - 1) {
            f[3] = own(plane_f(1));
            f[6] = own(plane_f(8));
            f[7] = own(plane_f(5));
            const float add = K.right_fixed ? K.abb * walls[RP + r] : 0.f;
            g[3] = sign_r_g * own(plane_g(1)) + add;
        }
        float rho, theta;
        collide_node(f, g, K, rho, theta);
        bad |= !(fabsf(rho) < 1e30f) || !(fabsf(theta) < 1e30f);
#pragma unroll
        for (int k = 0; k < 9; ++k) Dst[plane_f(k) * plane_sm + nx + i] = f[k];
#pragma unroll
        for (int k = 0; k < 5; ++k) Dst[plane_g(k) * plane_sm + nx + i] = g[k];
        // The neighbours' halo rows: downward-moving populations (0-based
        // directions f 4, 7, 8 and g 4) of the first row to the previous
        // block, upward-moving ones (f 2, 5, 6 and g 2) of the last row to
        // the next block.
        if (r == 0 && Dbelow) {
            Dbelow[plane_f(4) * plane_sm + x] = f[4];
            Dbelow[plane_f(7) * plane_sm + x] = f[7];
            Dbelow[plane_f(8) * plane_sm + x] = f[8];
            Dbelow[plane_g(4) * plane_sm + x] = g[4];
        }
        if (r == nr - 1 && Dabove) {
            Dabove[plane_f(2) * plane_sm + x] = f[2];
            Dabove[plane_f(5) * plane_sm + x] = f[5];
            Dabove[plane_f(6) * plane_sm + x] = f[6];
            Dabove[plane_g(2) * plane_sm + x] = g[2];
        }
        if (C.record && !bulk_rec) {
            float* d = C.record + (size_t)s * C.record_stride + (size_t)j * pitch + x;
#pragma unroll
            for (int k = 0; k < 9; ++k) d[plane_f(k) * PL] = f[k];
#pragma unroll
            for (int k = 0; k < 5; ++k) d[plane_g(k) * PL] = g[k];
        }
        if (x == 0) th01[(s & 1) * 2 * RP + 2 * r] = theta;
        if (x == 1) th01[(s & 1) * 2 * RP + 2 * r + 1] = theta;
    };
    const int r1 = (int)threadIdx.x / nx, x1 = (int)threadIdx.x - r1 * nx;  // ONE: this thread's node
    const bool has1 = !nu_warp && (int)threadIdx.x < nr * nx;
    const int i2 = (int)threadIdx.x + nwork, r2 = i2 / nx, x2 = i2 - r2 * nx;  // !ONE: the second node
    const bool has2 = !nu_warp && i2 < nr * nx;
    for (int s = 0; s < C.steps; ++s) {
        const bool odd = (s & 1) != 0;
        const float* S = odd ? sb[1] : sb[0];
        float* Dst = odd ? sb[0] : sb[1];
        float* Dbelow = odd ? below0 : below1;
        float* Dabove = odd ? above0 : above1;
        if (has1) node_step(s, (int)threadIdx.x, r1, x1, r0 + r1, S, Dst, Dbelow, Dabove);
        if constexpr (!ONE) {
            // A block holds at most two nodes per node thread (checked on the host).
            if (has2) node_step(s, i2, r2, x2, r0 + r2, S, Dst, Dbelow, Dabove);
        }
        cl.sync();  // step s's state, halo rows and wall-side temperatures are visible
        const bool copier = bulk_rec && nu_warp && !sum_warp && lane == 0 && nr > 0;
        if (copier) {
            // The state after step s (this block's rows of Dst) to its record;
            // the copies have read Dst before this thread reaches the next
            // barrier, after which step s + 2 overwrites it.
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            float* g = C.record + (size_t)s * C.record_stride + (size_t)r0 * pitch;
            const float* src = Dst + nx;  // local row 0
#pragma unroll 1
            for (int p = 0; p < kPlanes; ++p)
                cluster_bulk_s2g(g + p * PL, src + p * plane_sm, (unsigned)(nr * nx * 4));
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
        if (!rec && nu_warp) {
            // Off the node warps' path, on two warps: this block's rows of step s
            // into block 0's row array; in block 0, the sum of step s - 1, whose
            // rows every block wrote before this barrier.
            if (!sum_warp) nu_rows_of(s);
            else if (rank == 0 && s > 0) nu_mean_of(s - 1);
        }
        if (copier) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    }
    if (bulk_rec && nu_warp && !sum_warp && lane == 0 && nr > 0)
        asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");  // the records written
    if (!rec && C.steps > 0) {
        cl.sync();  // the last step's rows
        if (rank == 0 && sum_warp) nu_mean_of(C.steps - 1);
    }
    // The final state to global buffer parity ^ (K & 1); the last step's rows to
    // the rows array of its source buffer; the step counter slot of the final
    // buffer; nothing pending.
    const int pend = C.parity ^ (C.steps & 1);
    const float* fin = sb[C.steps & 1];
    float* dstg = const_cast<float*>(C.A[pend].src);
    for (int i = threadIdx.x; i < (rec ? 0 : nr * nx); i += blockDim.x) {
        const int r = i / nx, x = i - r * nx;
        if (!DMRT_IN(i + nx, 0, plane_sm, A0.err) || !DMRT_IN((long long)(r0 + r) * pitch + x, 0, PL, A0.err))
            continue;
        float* d = dstg + (size_t)(r0 + r) * pitch + x;
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) d[p * PL] = fin[p * plane_sm + nx + i];
    }
    if (!rec && rank == 0 && C.steps > 0) {
        const double* last = nur + (size_t)((C.steps - 1) & 1) * ny;
        double* rows = C.A[C.parity ^ ((C.steps - 1) & 1)].nu_rows;
        for (int r = threadIdx.x; r < ny; r += blockDim.x) rows[r] = last[r];
        if (threadIdx.x == 0) {
            *const_cast<long long*>(C.A[pend].step_in) = t0 + C.steps;
            *A0.pending = 0u;
        }
    }
    if (bad) atomicOr(A0.err, kErrNonFinite);
}

}  // namespace dmrt
