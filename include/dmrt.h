/*
 * dmrt — double-MRT thermal lattice Boltzmann time step on one GB300 (sm_103a).
 *
 * C ABI of libdmrt.so. The method is the one of Li, Yang & Zhang, "Double MRT
 * thermal lattice Boltzmann method for simulating natural convection of low
 * Prandtl number fluids" (arXiv 1601.04633):
 *   - Sec. 2 (Eqs. 1-17): side-heated square cavity, left wall theta_hot,
 *     right wall theta_cold, adiabatic top and bottom, no-slip everywhere;
 *   - Sec. 3.1 (Eqs. 22-34): D2Q9 MRT flow lattice with the Boussinesq force
 *     (Eqs. 26-27) and bounce-back no-slip walls;
 *   - Sec. 3.2 (Eqs. 35-45): D2Q5 MRT temperature lattice, bounce-back on
 *     adiabatic walls (Eq. 44), anti-bounce-back on fixed-temperature walls (Eq. 45);
 *   - Eqs. 18-19: hot-wall Nusselt number, recorded every time step.
 *
 * Conventions (every entry point):
 *   - Return 0 on success or a negative DMRT_E_* code; nothing throws.
 *     dmrt_last_error() gives a message for the most recent failure of a context.
 *   - Device memory is never allocated by the library. The caller provides one
 *     device workspace of dmrt_workspace_size() bytes (256-byte aligned) at
 *     creation and keeps it alive until dmrt_destroy(). Host memory for the
 *     context itself is malloc'd by dmrt_create and freed by dmrt_destroy.
 *   - All device work is enqueued on the CUDA stream given at creation
 *     (a cudaStream_t passed as void*; NULL = the legacy default stream).
 *     dmrt_step only enqueues; calls that return data to the host synchronise
 *     that stream.
 *   - A context is not thread-safe; distinct contexts are independent.
 *   - Grid: nodes (i, j), 0 <= i < nx, 0 <= j < ny, cell-centred at x = i + 1/2,
 *     y = j + 1/2 (lattice units, dx = dt = c = 1). Walls lie at x = 0, nx and
 *     y = 0, ny (half-way bounce-back). H = ny. Host field arrays are row-major
 *     [ny][nx] (index j * nx + i).
 */
#ifndef DMRT_H
#define DMRT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define DMRT_OK 0
#define DMRT_E_ARG (-1)      /* invalid argument or size */
#define DMRT_E_UNSTABLE (-2) /* parameters outside the model's valid range */
#define DMRT_E_CUDA (-3)     /* a CUDA runtime call failed */
#define DMRT_E_DIVERGED (-4) /* a non-finite density or temperature was seen */
#define DMRT_E_TIMEOUT (-5)  /* a bounded device-side wait ran out (2 s per wait) */
#define DMRT_E_SPACE (-6)    /* workspace or host buffer too small */
#define DMRT_E_STATE (-7)    /* checkpoint does not match this context */
#define DMRT_E_BOUNDS (-8)   /* bounds-checked build (libdmrt_bc.so, compiled with
                                DMRT_BOUNDS_CHECK): a kernel computed an index outside
                                its array and skipped that access */

/* Population storage precision. MIXED: the flow populations f in float16 and
 * the thermal populations g in float32 (38 bytes per node and buffer instead of
 * 56); the rounding mode applies to the float16 flow stores. THETA32: the flow
 * populations in float16, the temperature theta = sum_i g_i (Eq. 41) in
 * float32 and the four moving thermal populations as float16 deviations
 * d_i = g_i - w theta (i = 1..4 in 0-based directions; w = (4 + a)/20, the
 * weight of a moving direction in the D2Q5 equilibrium at rest, Eq. 42), the
 * rest population being g_0 = w_0 theta - (d_1 + d_2 + d_3 + d_4) with
 * w_0 = (1 - a)/5 (30 bytes per node and buffer); the rounding mode applies to
 * every float16 store. A node's stored thermal populations sum to its theta
 * (up to float32 arithmetic) whatever the deviations' rounding, so the
 * rounding moves heat between neighbours but creates none. dmrt_get_state
 * returns the populations these values stand for; dmrt_set_state stores theta
 * = sum_i g_i and each deviation rounded to nearest. THETA32 runs the
 * single-cavity TMA kernel only (no batch, slab, cluster, direct kernel or
 * adjoint). 16-bit, mixed and THETA32 storage have no counterpart in the paper
 * (which stores double). */
#define DMRT_FP32 0
#define DMRT_FP16 1
#define DMRT_BF16 2
#define DMRT_MIXED 3
#define DMRT_THETA32 4

/* Rounding of 16-bit population stores. NEAREST: round to nearest even.
 * STOCHASTIC: round up with probability equal to the distance to the lower
 * neighbour in units of the spacing, so that the expected stored value equals
 * the float32 value and increments smaller than half a unit in the last place
 * are kept on average; the random bits come from a per-node, per-step hash
 * (deterministic: a run repeats bit for bit), 13 per value for float16 and 16
 * for bfloat16, consumed by the GPU's stochastically rounding conversion
 * instruction. Float32 storage rounds nothing. AUTO (the default of
 * dmrt_default_params): STOCHASTIC for FP16, BF16 and MIXED storage, nothing
 * for FP32. Rounding to nearest loses the increments below half a unit in the
 * last place on every step; over long runs that biases the hot-wall Nusselt
 * number by more than 1e-3 (mixed storage: -3.1e-3 over 1e6 steps of the
 * 256^2, Ra 1e5 cavity), which stochastic rounding avoids. */
#define DMRT_ROUND_NEAREST 0
#define DMRT_ROUND_STOCHASTIC 1
#define DMRT_ROUND_AUTO 2

/* Step kernel variants. All compute the same step; they differ only in how
 * the populations reach the registers. DIRECT: 128-bit loads straight from
 * global memory, x-shifts by warp shuffles. TMA: a persistent kernel that
 * stages (strip x row-block) tiles in shared memory with 3-D tensor copies
 * through a multi-stage mbarrier pipeline. AUTO picks TMA for grids wider
 * than 496 nodes and for float32 grids whose one-row items (248-node strips x
 * rows) number at most 4 per SM, with tile (1, 1, 2) up to 2 per SM and (2, 1,
 * 3) beyond (e.g. 112^2 to 256^2), DIRECT otherwise (e.g. 384^2); for runs of
 * steps of a float32 cavity whose rows split over 16 blocks give at most 1024
 * nodes per block (e.g. up to 128^2), and no tile asked for, the CLUSTER kernel
 * below where the GPU fits it (64^2: 1.43 against 2.66 us per step). TMA tiles
 * compiled in, as (nodes per
 * thread, rows R, stages S): NPT 4 with (R,S) in (1,2) (1,3) (1,4) (1,5) (1,6)
 * (2,2) (2,3) (2,4) (4,2) (4,3); NPT 2 with (1,3) (1,4) (1,5) (2,2) (2,3)
 * (4,2); NPT 1 with (1,2) (1,3) (1,4) (1,5) (2,2) (2,3) (3,2) (4,2) (4,3).
 * Default (1, 4, 2). FP16 / BF16 storage, rounding to nearest (default (2, 4, 2)):
 * (1,1,2) (1,2,2) (1,4,2) (1,4,3) (1,4,4) (2,2,2) (2,4,2) (2,4,3) (4,2,2) (4,4,2);
 * stochastic (default (4, 4, 2)): (1,1,2) (1,4,2) (2,2,2) (2,4,2) (4,2,2) (4,4,2);
 * with fewer rows than the default tile, or one-row items at most 2 per SM,
 * (1, 1, 2); 4-row items fewer than 4 per SM, 2-row items. MIXED storage (default (2, 1, 2)), nearest:
 * (1,1,2) (1,1,3) (1,1,4) (1,2,2) (1,2,3) (1,4,2) (2,1,2) (2,1,3) (2,1,4)
 * (2,2,2) (4,1,3) (4,1,4); stochastic: (1,1,2) (1,2,2) (1,4,2) (1,4,3) (2,1,2)
 * (2,1,3) (2,2,2) (2,4,2) (4,1,3). THETA32 storage, nearest (default
 * (2, 1, 2)): (1,1,2) (2,1,2) (2,1,3) (2,2,2) (4,1,3); stochastic (default
 * (4, 2, 2)): (1,1,2) (1,2,2) (2,1,2) (2,1,3) (2,2,2) (2,4,2) (4,1,3) (4,2,2). */
#define DMRT_KERNEL_AUTO 0
#define DMRT_KERNEL_DIRECT 1
#define DMRT_KERNEL_TMA 2
/* CLUSTER: for small float32 cavities (both buffers, with one halo row per
 * block, in the shared memory of one thread-block cluster of up to 16 blocks,
 * e.g. up to 160^2): each dmrt_step call runs as one launch that keeps the
 * state on chip between steps (one cluster barrier per step); single steps and
 * the adjoint use the kernel AUTO picks among the others. The same bits as the
 * other kernels. DMRT_E_ARG at creation if the cavity does not fit. */
#define DMRT_KERNEL_CLUSTER 3

/* Wall kinds for the left and right (vertical) walls. Top and bottom are
 * always adiabatic (Eqs. 7-8, 44). */
#define DMRT_WALL_FIXED 0     /* fixed temperature, anti-bounce-back (Eq. 45) */
#define DMRT_WALL_ADIABATIC 1 /* zero heat flux, bounce-back (Eq. 44) */

typedef struct {
    int32_t nx, ny;     /* nodes; H = ny. 2 <= nx, ny <= 32768 */
    double Ra;          /* Rayleigh number g beta dT H^3 / (nu alpha) (Eq. 9), >= 0 */
    double Pr;          /* Prandtl number nu / alpha (Eq. 9), > 0 */
    double alpha;       /* lattice thermal diffusivity; if <= 0 it is derived from Ma */
    double Ma;          /* Mach number u_c / c_s (Eq. 9), used only when alpha <= 0:
                           alpha = Ma H / sqrt(3 Ra Pr) */
    double theta_hot;   /* left wall temperature (Eq. 14) */
    double theta_cold;  /* right wall temperature (Eq. 15) */
    double theta_ref;   /* buoyancy reference temperature theta_l (Eq. 27) */
    double theta_init;  /* uniform initial temperature when no field is given */
    int32_t left_wall;  /* DMRT_WALL_FIXED or DMRT_WALL_ADIABATIC */
    int32_t right_wall; /* DMRT_WALL_FIXED or DMRT_WALL_ADIABATIC */
    int32_t storage;    /* DMRT_FP32, DMRT_FP16, DMRT_BF16, DMRT_MIXED or DMRT_THETA32 (16-bit,
                           mixed and THETA32 storage run the TMA kernel; arithmetic is
                           float32 in every case) */
    int32_t kernel;     /* DMRT_KERNEL_AUTO, _DIRECT, _TMA or _CLUSTER */
    int64_t nu_capacity; /* length of the device ring of mean-Nu values, >= 1 */
    int32_t tma_rows;   /* TMA kernel: rows per work item (0 = the storage's default tile) */
    int32_t tma_stages; /* TMA kernel: pipeline stages (0 = default) */
    int32_t tma_npt;    /* TMA kernel: nodes per thread, 4, 2 or 1 (0 = default) */
    int32_t rounding;   /* 16-bit stores (all populations for FP16 / BF16, the flow
                           populations for MIXED): DMRT_ROUND_NEAREST, DMRT_ROUND_STOCHASTIC
                           or DMRT_ROUND_AUTO (stochastic unless the storage is FP32) */
} dmrt_params;

/* Constants derived from dmrt_params (Eqs. 9, 31-32, 38-40, 43, 45). */
typedef struct {
    double nu;        /* kinematic viscosity Pr * alpha */
    double alpha;     /* thermal diffusivity */
    double s_e, s_nu, s_q, s_eps;  /* D2Q9 rates (Eq. 32) */
    double sig_k, sig_e, sig_nu;   /* D2Q5 rates (Eq. 40) */
    double a;         /* D2Q5 equilibrium parameter (Eq. 43) */
    double gbeta;     /* buoyancy per unit theta: G_y = gbeta (theta - theta_ref) */
    double abb;       /* 2 sqrt(3) alpha (Eq. 45) */
    double Ma;        /* Mach number sqrt(3 gbeta dT H) */
    double fo_per_step; /* Fourier number per step alpha / H^2 (Eq. 20) */
} dmrt_consts;

typedef struct dmrt_ctx dmrt_ctx;

/* Fill *p with defaults: 64x64, Ra 1e4, Pr 0.01, alpha 0.1, walls +-0.5,
 * theta_ref 0, theta_init 0, fixed-temperature side walls, FP32, ring 2^20,
 * rounding DMRT_ROUND_AUTO. */
void dmrt_default_params(dmrt_params* p);

/* Validate *p and derive the model constants (host only, no GPU needed).
 * Errors: DMRT_E_ARG (sizes, Pr <= 0, Ra < 0, no alpha and no Ma, walls equal
 * with Ra > 0), DMRT_E_UNSTABLE (a outside (-4, 1), a rate outside (0, 2)). */
int dmrt_derive(const dmrt_params* p, dmrt_consts* out);

/* Device workspace bytes a context with these parameters needs. */
int dmrt_workspace_size(const dmrt_params* p, size_t* bytes);

/* Create a context. theta0: optional host array [ny][nx] of initial
 * temperatures (NULL = theta_init everywhere). The initial state is the
 * equilibrium at rest: f_i = 0 (delta-rho = 0, u = 0; the flow populations are
 * stored shifted by w_i rho0, Eq. 33) and g_i = g_i_eq(theta0, u = 0) (Eq. 42);
 * it counts as a post-collision state, so the first step starts with streaming.
 * workspace: device pointer, 256-byte aligned, of at least
 * dmrt_workspace_size() bytes; the context uses it until dmrt_destroy.
 * stream: cudaStream_t as void*. Synchronises the stream before returning. */
int dmrt_create(const dmrt_params* p, const double* theta0, void* workspace,
                size_t workspace_bytes, void* stream, dmrt_ctx** out);

/* Enqueue nsteps time steps (nsteps >= 0). One step is one fused kernel:
 * pull-stream f and g with the walls, moments, D2Q9 MRT collision (Eq. 28),
 * buoyancy force (Eq. 26), D2Q5 MRT collision (Eq. 36), store, and the
 * hot-wall Nusselt number of the pre-collision temperature (Eqs. 18-19)
 * appended to the ring. Does not synchronise, except to poll for divergence:
 * each time the context's step count passes a multiple of 65536, it waits for
 * the steps enqueued so far and reads the device error word; if a step saw a
 * non-finite value it returns DMRT_E_DIVERGED (DMRT_E_TIMEOUT for an expired
 * wait) without enqueueing the remaining steps (dmrt_steps_done tells how
 * many were taken). */
int dmrt_step(dmrt_ctx* c, int64_t nsteps);

/* Synchronise the stream and report DMRT_E_DIVERGED if any step so far saw a
 * non-finite density or temperature. */
int dmrt_check(dmrt_ctx* c);

/* Time steps taken so far. */
int64_t dmrt_steps_done(const dmrt_ctx* c);

/* Macroscopic fields at the current time level (pre-collision u, v, theta of
 * the last step; Eqs. 33, 41), float32 arrays [ny][nx] owned by the caller.
 * on_device != 0: u, v, theta are device pointers; else host pointers.
 * Any of u, v, theta may be NULL. Synchronises. */
int dmrt_fields(dmrt_ctx* c, float* u, float* v, float* theta, int on_device);

/* Hot-wall Nusselt numbers (Eqs. 18-19), host outputs, all nullable:
 *   nu_mean:  mean Nu of the last step;
 *   nu_local: [ny] local Nu of the last step;
 *   series:   up to cap most recent per-step mean values, oldest first;
 *   count:    number of values written to series.
 * Nu_j = H (8 theta_w(j) - 9 theta(0,j) + theta(1,j)) / (3 (theta_hot - theta_cold)).
 * Synchronises; returns DMRT_E_DIVERGED if a non-finite value was seen. */
int dmrt_nusselt(dmrt_ctx* c, double* nu_mean, double* nu_local, double* series,
                 int64_t cap, int64_t* count);

/* Replace the left (hot) and right (cold) wall temperatures by per-row
 * profiles theta_w(j) (host arrays [ny], nullable = keep). Used by Eq. 45 and
 * by the Nusselt number. */
int dmrt_set_wall_profiles(dmrt_ctx* c, const double* hot, const double* cold);

/* Secondary hot-wall Nusselt number of the current state, from the heat the
 * next streaming carries across the hot wall's links (Eq. 45 with Fourier's
 * law behind Eqs. 18-19): Nu_j = H (2 sqrt(3) alpha theta_w(j) - 2 g*_3(0, j)) /
 * (alpha (theta_hot - theta_cold)), g* the post-collision thermal populations
 * of the wall column; 0 for an adiabatic left wall. Exactly 1 in the
 * conduction limit, like the wall-gradient estimator of dmrt_nusselt, which it
 * matches to the discretisation level otherwise. Host outputs, both nullable:
 * nu_mean (mean over rows), nu_local [ny]. Synchronises. */
int dmrt_nusselt_flux(dmrt_ctx* c, double* nu_mean, double* nu_local);

/* Heat content and wall heat input of the current state, summed in float64 on
 * the GPU in a fixed order (the same bits for the same state), host outputs,
 * both nullable:
 *   theta_sum: sum over all nodes of theta = sum_i g*_i (Eq. 41; the thermal
 *              collision conserves theta, so this is the heat content of the
 *              current time level);
 *   wall_in:   the heat the next streaming brings in across the side walls:
 *              sum over rows of (2 sqrt(3) alpha theta_w(j) - 2 g*_4(0, j)) for a
 *              fixed-temperature left wall (anti-bounce-back, Eq. 45, returns
 *              2 sqrt(3) alpha theta_w - g*_4 and the wall link removes g*_4) plus
 *              the same with theta_c(j) and g*_2(nx-1, j) for a fixed right wall
 *              (paper numbering: g_2 moves in +x, g_4 in -x); bounce-back walls
 *              (Eq. 44, the top and bottom ones always) carry no heat.
 * Hence the next step's theta_sum equals theta_sum + wall_in up to float32
 * rounding. Synchronises. */
int dmrt_energy(dmrt_ctx* c, double* theta_sum, double* wall_in);

/* Post-collision population state at the current time level as a dense host
 * float32 array [14][ny][nx]: planes f_1..f_9 (Eq. 23 order; f stored shifted
 * so that sum f_i = delta-rho, Eq. 33) then g_1..g_5 (Eq. 35 order).
 * get: device -> host; set: host -> device (replaces the state; the step
 * count and the Nusselt ring are unchanged). Both synchronise. */
int dmrt_get_state(dmrt_ctx* c, float* host);
int dmrt_set_state(dmrt_ctx* c, const float* host);

/* ---- Checkpoint and resume (the paper has no counterpart) ----
 *
 * dmrt_save writes a self-describing checkpoint of everything a later step
 * reads into a caller-owned host buffer: the population state of the current
 * time level in its stored representation (bit for bit, also for 16-bit and
 * mixed storage), the step count and the device step counter (which seeds the
 * stochastic rounding), the wall profiles, the local and latest mean Nusselt
 * numbers, the recorded part of the Nusselt ring (at most nu_capacity values)
 * and the error word, followed by a 64-bit FNV-1a checksum. Layout:
 * little-endian header (magic "DMRTCKP1", version, grid, storage, the
 * physical parameters it was taken with), then the sections in that order.
 * With host_buf == NULL only *used is set to the size needed. Errors:
 * DMRT_E_ARG (c or used NULL), DMRT_E_SPACE (cap < needed; *used is set).
 * Synchronises the context's stream.
 *
 * dmrt_load restores such a checkpoint into a context created with the same
 * nx, ny and storage (its own Ra, Pr, walls and rounding govern the steps
 * after it). Stepping after a load continues bit for bit as the saved context
 * would have. The Nusselt ring keeps the last min(saved, nu_capacity) values.
 * Errors: DMRT_E_ARG (NULL or too short), DMRT_E_STATE (wrong magic, version,
 * grid or storage, or a checksum mismatch; the context is unchanged).
 * Synchronises. */
int dmrt_save(dmrt_ctx* c, void* host_buf, size_t cap, size_t* used);
int dmrt_load(dmrt_ctx* c, const void* host_buf, size_t size);

/* ---- Failure-path check of the bounded waits (the paper has no counterpart) ----
 *
 * The TMA step kernels wait on mbarriers for their tensor copies; every such
 * wait gives up after 2 s, records the failure (dmrt_check then returns
 * DMRT_E_TIMEOUT) and lets the kernel end, so a copy that never completes
 * cannot hang the GPU. dmrt_probe_bounded_wait runs that wait routine on an
 * mbarrier that nothing ever completes, with limit_ns in [1 ms, 2 s], on the
 * given stream (cudaStream_t as void*), and returns DMRT_E_TIMEOUT when the
 * wait gave up as designed (*waited_ns, nullable: the time it waited),
 * DMRT_OK if it completed (a defect), DMRT_E_ARG or DMRT_E_CUDA otherwise.
 * Uses a file-scope device word; allocates nothing. Synchronises the stream. */
int dmrt_probe_bounded_wait(int64_t limit_ns, void* stream, int64_t* waited_ns);

/* ---- One step without any device allocation (the paper has no counterpart) ----
 *
 * For callers that cannot allocate device memory where they step a cavity: code
 * running while a framework owns all device memory and hands out only input and
 * output buffers, real-time loops in which a cudaMalloc would synchronise the
 * device, or plug-in hosts that forbid allocation inside their callbacks.
 * dmrt_step_noalloc advances one time step (the same fused step as dmrt_step,
 * run by the direct-load kernel) from src to dst and allocates nothing: the
 * scratch the step needs (per-row Nusselt values, the step counter and pending
 * flag of the Nusselt reduction, the wall temperatures, the error word) lives in one
 * file-scope device array of 16 * DMRT_NOALLOC_MAX_NY + 256 bytes (about 128 KB)
 * that every GPU which loads the library holds until the process exits.
 *
 *   p:          problem parameters, as for dmrt_create (kernel and tma_* ignored);
 *               ny must not exceed DMRT_NOALLOC_MAX_NY (else DMRT_E_ARG, with the
 *               reason in dmrt_last_error(NULL)).
 *   src, dst:   distinct 16-byte aligned device buffers, each 14 * ny * pitch
 *               floats, pitch = nx rounded up to a multiple of 128: the
 *               post-collision populations at time t (read) and t + 1 (written),
 *               14 planes [ny][pitch]. The planes are those of dmrt_set_state
 *               (host order f_1..f_9, g_1..g_5, numbered 1..14), arranged on the
 *               device as host planes 1 2 4 10 11 13 3 6 7 12 5 8 9 14. Padding
 *               columns are ignored on input.
 *   theta_hot, theta_cold: device float arrays [ny] of wall temperatures, or NULL
 *               for the constant theta_hot / theta_cold of p.
 *   nu_mean:    device pointer to one double that receives the step's mean
 *               hot-wall Nusselt number (the value dmrt_nusselt reports as
 *               nu_mean after the same step), or NULL.
 *   stream:     cudaStream_t as void*; the call only enqueues work on it.
 *
 * The first call on a device looks up the array's device address (host code
 * only sees a host-side stand-in for it), so make that first call before any
 * stream capture. Every call shares the array and clears what must start at
 * zero; calls that overlap on the GPU (other streams, other threads) race on it,
 * so order them. Non-finite values are not reported by this call. */
#define DMRT_NOALLOC_MAX_NY 8192
int dmrt_step_noalloc(const dmrt_params* p, const float* src, float* dst,
                      const float* theta_hot, const float* theta_cold, double* nu_mean,
                      void* stream);

/* ---- One cavity split into y-slabs (for several GPUs) ------------------------
 *
 * A cavity can be cut into slabs of whole rows, one context per slab (one per
 * GPU, or several on one GPU), that step together. The streaming of Eqs. 25
 * and 36 moves populations by at most one row, so a slab's step needs only its
 * own rows plus one row on each side: from the row below, the populations that
 * move up (e_y = +1: f_3, f_6, f_7 of Eq. 23 and g_3 of Eq. 35); from the row
 * above, those that move down (f_5, f_8, f_9, g_5). A slab context holds these
 * two halo rows next to its own and fills them from its neighbours' messages
 * between steps; the walls of Eqs. 14-17 and 44-45 apply only at the slab sides
 * that are cavity walls. The constants (Ra, gbeta, the Nusselt scale) are those
 * of the whole cavity (H = p->ny), and every slab's state is bit for bit the
 * state of the same rows of the whole cavity stepped as one context, for every
 * storage mode (stochastic rounding draws on the cavity row index).
 *
 * dmrt_slab_workspace_size / dmrt_create_slab: as dmrt_workspace_size /
 *   dmrt_create, for rows y0 .. y0 + rows - 1 of the cavity p (1 <= rows,
 *   y0 + rows <= p->ny); theta0 is NULL or the slab's own [rows][nx] initial
 *   temperatures. All other entry points work on a slab as on a cavity of
 *   `rows` rows (fields, state, checkpoints, wall profiles: the slab's rows),
 *   except that: the Nusselt means (dmrt_nusselt, its ring, dmrt_nusselt_flux)
 *   are the slab's share of the cavity's mean (its rows' sum divided by the
 *   cavity's p->ny), so the cavity's mean is the sum over slabs; dmrt_energy
 *   sums the slab's rows; dmrt_step takes at most one step on a slab that has
 *   a neighbour (DMRT_E_STATE otherwise); dmrt_adjoint refuses a slab.
 *
 * Messages: dmrt_slab_halo_bytes() bytes each, device memory owned by the
 *   caller (the library allocates nothing), the face planes of one row in the
 *   slab's storage type.
 * dmrt_slab_pack(c, to_below, to_above): enqueue copies of the current state's
 *   first row's downward populations into to_below and of its last row's
 *   upward populations into to_above (either NULL to skip).
 * dmrt_slab_unpack(c, from_below, from_above): enqueue copies of the messages
 *   of the neighbour below (its to_above) and above (its to_below) into the
 *   current state's halo rows (either NULL to skip; a side that is a cavity
 *   wall needs none).
 * dmrt_slab_step(c, to_below, to_above): one time step (the fused step kernel,
 *   reading the halo rows), then dmrt_slab_pack of the new state.
 * A run: create the slabs; pack and unpack once (the halo rows of the initial
 *   state); then per time step: dmrt_slab_step on every slab, deliver each
 *   message to its neighbour (a copy on one GPU, a send/receive between GPUs),
 *   dmrt_slab_unpack on every slab. dmrt_slab_step leaves the step's Nusselt
 *   rows to be summed by the next step; dmrt_step(c, 0) sums the last one. All
 *   copies are enqueued on the slab's stream; ordering them against the
 *   transfer between slabs is the caller's. */
int dmrt_slab_workspace_size(const dmrt_params* p, int32_t rows, size_t* bytes);
int dmrt_create_slab(const dmrt_params* p, int32_t y0, int32_t rows, const double* theta0, void* workspace,
                     size_t workspace_bytes, void* stream, dmrt_ctx** out);
int dmrt_slab_halo_bytes(const dmrt_ctx* c, size_t* bytes);
int dmrt_slab_pack(dmrt_ctx* c, void* to_below, void* to_above);
int dmrt_slab_unpack(dmrt_ctx* c, const void* from_below, const void* from_above);
int dmrt_slab_step(dmrt_ctx* c, void* to_below, void* to_above);

/* Launch configuration a context resolved to (for reports and tuning). */
typedef struct {
    int32_t kernel;       /* DMRT_KERNEL_DIRECT or DMRT_KERNEL_TMA */
    int32_t tma_npt, tma_rows, tma_stages;
    int32_t grid, block;  /* blocks per step launch, threads per block */
    int64_t smem_bytes;   /* dynamic shared memory per block */
    int32_t graph_steps;  /* steps per captured CUDA graph */
} dmrt_launch;
int dmrt_get_launch(const dmrt_ctx* c, dmrt_launch* out);

/* The kernel and tile (nodes per thread, rows, stages) that dmrt_create would
 * choose for parameters p on a GPU with sms streaming multiprocessors: host
 * logic only, no device call (the rules are listed at DMRT_KERNEL_AUTO and the
 * storage modes' tile lists). The tile is 0, 0, 0 for the direct kernel. Errors
 * as dmrt_derive; DMRT_E_ARG for a NULL pointer, sms < 1, or the direct kernel
 * asked for with 16-bit or mixed storage. */
int dmrt_choose_launch(const dmrt_params* p, int32_t sms, int32_t* kernel, int32_t* npt, int32_t* rows,
                       int32_t* stages);

/* Derived constants of a context. */
int dmrt_get_consts(const dmrt_ctx* c, dmrt_consts* out);

/* Message for the last failure on c (or of the last failed dmrt_create when c
 * is NULL). Never NULL. */
const char* dmrt_last_error(const dmrt_ctx* c);

/* Release the context (not the caller's workspace). Synchronises. NULL is a no-op. */
void dmrt_destroy(dmrt_ctx* c);

/* ---- Discrete adjoint ---------------------------------------------------------
 *
 * Gradient of J = mean hot-wall Nusselt number (Eqs. 18-19) over the last
 * avg_last of nsteps steps, with respect to the hot-wall temperature profile
 * theta_w(j) (which enters Eq. 45 and the Nusselt stencil) and to Ra (which
 * enters through the buoyancy scale of Eq. 27), by a hand-written reverse
 * (transposed collide-stream) kernel: the exact adjoint of the discrete
 * float32 step, with the gradients accumulated in float64 in a fixed order
 * (the results repeat bit for bit). Memory: sqrt(N) checkpoints of the state
 * plus a sqrt(N)-step segment that is recomputed from its checkpoint, by the
 * context's own step kernel, before being swept backwards. The sweep of a
 * segment is one CUDA-graph replay: nodes chained by programmatic edges, each
 * two reverse steps (small cavities: the first step on a 3-row window, its
 * result kept in shared memory for the second) or one (cavities that fill the
 * GPU), and a fold of the segment's gradient terms; the graphs are built on
 * each call and released before it returns.
 *
 * dmrt_adjoint starts from the context's current state and wall profiles,
 * advances the context by nsteps (its state, step count and Nusselt ring are
 * those of a dmrt_step(c, nsteps) call), and returns J, dJ/dtheta_w (host
 * array [ny]) and dJ/dRa (each output nullable). Float32 storage only;
 * nu_capacity >= avg_last. workspace: device memory of
 * dmrt_adjoint_workspace_size() bytes, 256-byte aligned, used only during the
 * call: then each segment's recompute runs on a second stream (created on the
 * first such call, released by dmrt_destroy) while the reverse sweep of the
 * segment after it runs on the context's stream. A workspace of at least
 * dmrt_adjoint_workspace_min() bytes (one set of segment states fewer) also
 * works: recompute and sweep then alternate on the context's stream. When the
 * context steps with the cluster kernel (DMRT_KERNEL_CLUSTER, or AUTO on a
 * small float32 cavity), a workspace of dmrt_adjoint_workspace_all() bytes
 * (nonzero only then: about N + 1 states) stores every state of the forward
 * pass as the kernel steps, and no segment is recomputed. All three give the
 * same bits. Synchronises; DMRT_E_DIVERGED if the forward run diverged. */
int dmrt_adjoint_workspace_size(const dmrt_ctx* c, int64_t nsteps, size_t* bytes);
int dmrt_adjoint_workspace_min(const dmrt_ctx* c, int64_t nsteps, size_t* bytes);
int dmrt_adjoint_workspace_all(const dmrt_ctx* c, int64_t nsteps, size_t* bytes);
int dmrt_adjoint(dmrt_ctx* c, int64_t nsteps, int64_t avg_last, void* workspace, size_t workspace_bytes,
                 double* J, double* dJ_dthetaw, double* dJ_dRa);

/* ---- Batched sweep: many independent cavities per launch ----------------------
 *
 * Steps n independent side-heated cavities (any sizes and parameters; all
 * float32, or all mixed storage with one rounding mode) with one launch per time
 * step of a persistent TMA kernel over the
 * concatenated work items of all cavities, replayed from CUDA graphs. Each
 * member is also an ordinary context (dmrt_batch_context), so dmrt_fields,
 * dmrt_nusselt, dmrt_get_state, ... work on it, and stepping the members one
 * by one with dmrt_step is the sequential alternative. The paper's four cases
 * (Table 1) are such a sweep over (Ra, Pr). */
typedef struct dmrt_batch dmrt_batch;

/* Tile of the batched kernel: nodes per thread, rows per item, pipeline stages
 * (0 = default: 2, 2, 2 for FLOAT32, 4, 2, 2 for MIXED storage), and steps
 * per CUDA graph (0 = 64; must be even). Compiled tiles (npt, R, S), for both
 * storages and roundings: (1,1,2) (1,2,2) (1,4,2) (1,4,3) (2,1,2) (2,1,3)
 * (2,2,2) (2,2,3) (2,4,2) (4,1,4) (4,2,2) (4,4,2).
 * group_bytes: 0 = one launch per time step steps every cavity (the state
 * streams through HBM on every step). > 0 = the cavities are split, in index
 * order, into groups whose two population buffers take at most group_bytes
 * together (a larger cavity is a group of its own), and dmrt_batch_step runs
 * the groups one after another, each for all of the call's steps with
 * launches over its own cavities: a group small enough for the L2 cache
 * (e.g. 32 to 96 MB of the GB300's 126 MB) is read from and written to L2
 * between its steps. Every cavity's results are the same bits either way.
 * steps_per_launch: 0 or 1 = one launch per time step (graphs of graph_steps
 * launches). K > 1 (even) = a persistent kernel advances every cavity of a
 * group by K steps in one launch, with no grid-wide barrier between the steps:
 * a cavity's next step starts as soon as that cavity's previous step is
 * complete (a per-cavity counter, acquired before the tensor copies of the
 * next step; bounded waits, DMRT_E_TIMEOUT on expiry); graphs hold two such
 * launches. Compiled multi-step tiles: FP32 (1,2,2) (2,1,2) (2,2,2) (2,2,3)
 * (4,2,2) (4,4,2); MIXED, both roundings, (2,2,2) (4,2,2) (4,4,2). The same
 * bits as one launch per step. */
typedef struct {
    int32_t tma_npt, tma_rows, tma_stages, graph_steps;
    int64_t group_bytes;
    int32_t steps_per_launch;
    int32_t tensor_store;  /* 0: stores from registers; 1: the results of an item go
                              through a shared-memory tile and leave by tensor stores
                              (per-cavity store maps; one launch per step only).
                              Compiled: FP32 (2,1,2) (2,2,2); MIXED, both roundings,
                              (2,2,2) (4,2,2) (4,4,2). The same bits either way. */
    int32_t strip_fill;    /* 0: each cavity in the widest strips the stage allows
                              (fewest halo columns); 1: in the strip width that keeps
                              the most of the block's threads busy (an item's rows
                              times threads per row against the block, times the
                              valid share of the strips' nodes). The same bits
                              either way. */
} dmrt_batch_opts;

/* Device workspace for a batch of n cavities (the members' workspaces plus the
 * kernel's tables). Errors as dmrt_derive for any member; DMRT_E_ARG for n < 1,
 * FP16 / BF16 storage, or members stored or rounded differently. */
int dmrt_batch_workspace_size(const dmrt_params* arr, int32_t n, size_t* bytes);

/* Create a batch. arr: n parameter sets; theta0: NULL, or n host pointers (each
 * NULL or an [ny][nx] initial temperature field); opts: NULL for defaults;
 * workspace: 256-byte aligned device memory of dmrt_batch_workspace_size()
 * bytes, kept alive by the caller until dmrt_batch_destroy. Synchronises. */
int dmrt_batch_create(const dmrt_params* arr, int32_t n, const double* const* theta0,
                      const dmrt_batch_opts* opts, void* workspace, size_t workspace_bytes,
                      void* stream, dmrt_batch** out);

/* Enqueue nsteps time steps of every member. DMRT_E_STATE if a member was
 * stepped on its own by an odd number of steps since the last batch step. */
int dmrt_batch_step(dmrt_batch* b, int64_t nsteps);

/* Synchronise; DMRT_E_TIMEOUT or DMRT_E_DIVERGED (first member concerned). */
int dmrt_batch_check(dmrt_batch* b);

int32_t dmrt_batch_size(const dmrt_batch* b);

/* Number of cavity groups (1 unless dmrt_batch_opts.group_bytes > 0). */
int32_t dmrt_batch_group_count(const dmrt_batch* b);

/* Member i as a context (borrowed: do not destroy it), or NULL. */
dmrt_ctx* dmrt_batch_context(dmrt_batch* b, int32_t i);

int dmrt_batch_get_launch(const dmrt_batch* b, dmrt_launch* out);
const char* dmrt_batch_last_error(const dmrt_batch* b);

/* Release the batch and its member contexts (not the workspace). */
void dmrt_batch_destroy(dmrt_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* DMRT_H */
