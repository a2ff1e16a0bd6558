/*
 * lbm.h -- C ABI of the GB300 thermal lattice Boltzmann library.
 *
 * The library advances the double-distribution thermal lattice Boltzmann
 * scheme of Hu, Zhang & Geng (arXiv 1608.06345) on one GPU: per time step,
 * every cell pulls its 2Q populations g_i (mass/momentum, Eq. (13a)) and h_i
 * (internal energy, Eq. (13b)) from its upwind neighbours, takes the moments
 * of Eq. (14)/(15), evaluates the fourth-order Hermite equilibrium of Eq. (18)
 * and relaxes both populations with the explicit BGK step of Eq. (16)/(17).
 * Velocity sets: D2Q37 (Table I) and D3Q107 (Table II).
 *
 * Conventions shared by every entry point:
 *  - Every call returns an lbm_status; on failure lbm_last_error() gives a
 *    thread-local, human-readable message.  No call aborts the process.
 *  - Cell index of (x, y, z) is x + nx*(y + ny*z).  Scalar fields hold N =
 *    nx*ny*nz doubles; velocity fields are component-major, D*N doubles
 *    (u_x of every cell, then u_y, then u_z).
 *  - Host pointers are caller-owned and only read/written during the call.
 *    Device pointers are caller-owned and must stay valid until the stream
 *    work that uses them has completed.
 *  - All GPU work of an instance is issued on the stream given at creation
 *    (NULL = the legacy default stream).  Calls that return host results
 *    synchronise that stream.
 *  - Units are the non-dimensional units of the paper's Sec. II: p = rho T,
 *    velocities in units of sqrt(R T0); lattice spacing 1, time step 1, so
 *    that xi_i = r c_i with the integer c_i of Tables I/II (Sec. V maps step
 *    n to t = n / (X r)).  tau_f, tau_g are relaxation times in time steps.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_instance* lbm_handle;

enum lbm_status {
  LBM_OK = 0,
  LBM_EINVAL = 1,     /* invalid argument (message says which) */
  LBM_ENOMEM = 2,     /* device or host allocation failed, or caller buffer too small */
  LBM_ECUDA = 3,      /* a CUDA runtime call failed */
  LBM_ENONFINITE = 4, /* a step produced a non-finite density or temperature */
  LBM_ETIMEOUT = 5,   /* reserved for a bounded device-side wait that gives up; no
                         kernel of this library waits on the device, so no call
                         returns it */
  LBM_EBUSY = 6       /* a pool's memory budget is full */
};

enum lbm_lattice { LBM_D2Q37 = 0, LBM_D3Q107 = 1 };

/* Boundary kind per axis (both ends of an axis share it).
 * LBM_ZERO_GRADIENT is the "open" boundary of Sec. V: a pull from outside
 * [0, n-1] reads the edge cell's stored populations. */
enum lbm_bc { LBM_PERIODIC = 0, LBM_ZERO_GRADIENT = 1 };

/* Compute / storage precision of the populations.
 *  LBM_F64      FP64 arithmetic, FP64 storage.
 *  LBM_F32      FP32 arithmetic, FP32 storage.
 *  LBM_F32_S16F / LBM_F32_S16BF: FP32 arithmetic; populations stored in
 *               FP16 / BF16 as relative deviations from the instance's
 *               reference equilibrium (rho0, u = 0, T0). */
enum lbm_prec { LBM_F64 = 0, LBM_F32 = 1, LBM_F32_S16F = 2, LBM_F32_S16BF = 3 };

typedef struct {
  int nx, ny, nz;       /* cells per axis; nz = 1 for D2Q37 */
  int bc[3];            /* lbm_bc per axis x, y, z */
  int prec;             /* lbm_prec */
  void* stream;         /* cudaStream_t for all work of the instance; NULL = default stream */
  void* device_mem;     /* optional caller-owned device buffer of >= lbm_state_bytes()
                           bytes, 256-byte aligned; NULL = the library allocates */
  size_t device_bytes;  /* size of device_mem */
  double rho0, T0;      /* reference state (rho0, u = 0, T0) whose equilibrium the
                           stored populations are deviations from (see below) */
} lbm_grid;

/* The reference state.  The populations are stored as deviations
 * g_i - gref_i, h_i - href_i from the equilibrium gref_i = F_i(rho0, 0, T0),
 * href_i = (delta/2) T0 gref_i: an exact change of variables that changes
 * only the rounding.  Where the flow is near the reference the deviations
 * are small and keep more bits than the populations (FP32 resolves the
 * momentum of a flow near rest about 50 times better); where it is far from
 * it (|g - gref| > |g|, e.g. a density below half of rho0) they keep fewer,
 * about log2(|g - gref| / |g|) bits fewer.
 *   rho0 > 0      that reference;
 *   rho0 < 0      no reference, populations stored whole (gref = 0): FP64
 *                 and FP32 storage only;
 *   rho0 = 0, NaN the precision's default: whole storage for LBM_F64,
 *                 rho0 = 1 for LBM_F32 and 16-bit storage.
 * T0 that is not positive (NaN included) means 1.0.  16-bit storage needs a
 * reference near the flow's state (the codec stores (g - gref)/gref); a
 * negative rho0 there fails with LBM_EINVAL. */

/* Device bytes an instance needs: two copies of the 2Q population planes
 * (double buffer) plus a small tail (error word, reduction partials).
 * Returns 0 for invalid arguments. */
size_t lbm_state_bytes(int lattice, const lbm_grid* grid);

/* Create an instance.  gamma sets delta = 2/(gamma-1) - D (Eq. (3)); it must
 * give delta >= 0, i.e. 1 < gamma <= (D+2)/D.  tau_f relaxes g, tau_g relaxes
 * h (Eq. (16)/(17); the paper uses one tau); both must exceed 0.5.
 * Errors: LBM_EINVAL (bad lattice, gamma, tau, dims, bc, prec, nz != 1 in 2D,
 * more than 2^31-1 cells), LBM_ENOMEM (allocation or device_mem too small),
 * LBM_ECUDA.  On success *out owns the instance until lbm_destroy. */
int lbm_create(lbm_handle* out, int lattice, double gamma, double tau_f, double tau_g,
               const lbm_grid* grid);

/* Release an instance and any memory the library allocated for it.  NULL-safe. */
int lbm_destroy(lbm_handle h);

/* Set the state to the equilibrium of the given fields (host arrays):
 * g_i = F_i(rho, u, T) of Eq. (18), h_i = (delta/2) T F_i.  Copies the
 * fields to the device through the instance's idle buffer and synchronises. */
int lbm_init(lbm_handle h, const double* rho, const double* u, const double* T);

/* As lbm_init with device arrays; asynchronous on the instance's stream. */
int lbm_init_device(lbm_handle h, const double* rho, const double* u, const double* T);

/* Advance n >= 0 time steps (pull-stream + BGK collide of g and h per step:
 * Eq. (16)/(17) with the convection done by exact streaming, xi_i dt = c_i dx,
 * which the time mapping of Sec. V implies).  Asynchronous on the instance's
 * stream.  Runs of at least twice the graph
 * length (lbm_set_graph_steps, default 64) replay a captured CUDA graph of
 * that many steps instead of launching each step; the arithmetic is the same. */
int lbm_step(lbm_handle h, long n);

/* Steps per CUDA graph replay of lbm_step (even, 0..4096); 0 launches every
 * step separately (the plain one-launch-per-step path).  Execution control
 * with no counterpart in the paper. */
int lbm_set_graph_steps(lbm_handle h, int steps);

/* Advance n >= 0 time steps of the finite-difference variant of Sec. III:
 * forward Euler in time, the convection xi_i . grad q_i discretised along
 * each axis by the third-order upwind difference (the paper's printed g_j is
 * read as g_i), and the BGK relaxation of Eq. (16)/(17) from the cell's own
 * moments; lambda = dt/dx (> 0), tau_f and tau_g in units of dt.  Boundaries
 * as for lbm_step.  Forward Euler with this stencil is stable only for small
 * lambda (about 0.07 at tau = 0.8 on rough fields; the largest velocity
 * 3 r moves 3 r lambda cells per step).  Asynchronous; plain launches. */
int lbm_step_fd(lbm_handle h, long n, double lambda);

/* Kernel of lbm_step_fd (execution control; both compute Eq. (16)/(17) with
 * the same per-value arithmetic and agree to rounding):
 *  - LBM_FD_AUTO (default): LBM_FD_CELL;
 *  - LBM_FD_CELL: one thread per cell, every stencil value read from global
 *    memory;
 *  - LBM_FD_MARCH: blocks of 32 columns march along y; the lattice's (c, -c)
 *    pairs are split over the block's warps, each streaming its planes' rows
 *    through its own shared-memory ring (D2Q37 only; LBM_EINVAL otherwise). */
enum lbm_fd_kernel { LBM_FD_AUTO = 0, LBM_FD_CELL = 1, LBM_FD_MARCH = 2 };
int lbm_set_fd_kernel(lbm_handle h, int kernel);

/* rho, u, T of the stored (post-collision) state, Eq. (14)/(15), into host
 * arrays of N, D*N, N doubles.  Synchronises; returns LBM_ENONFINITE if any
 * step since creation met a non-finite density or temperature. */
int lbm_moments(lbm_handle h, double* rho, double* u, double* T);

/* As lbm_moments into device arrays; asynchronous, no status check. */
int lbm_moments_device(lbm_handle h, double* rho, double* u, double* T);

/* Grid totals of the stored state in FP64: out[0] = mass = sum g,
 * out[1..D] = momentum = sum xi g, out[D+1] = total energy
 * = sum (xi^2/2 g + h) (Eq. (14)).  Deterministic (fixed reduction order).
 * Synchronises; LBM_ENONFINITE as for lbm_moments. */
int lbm_conserved(lbm_handle h, double* out);

/* Synchronise the instance's stream and report LBM_ENONFINITE / LBM_ECUDA. */
int lbm_sync(lbm_handle h);

/* Time steps taken since the last init. */
long lbm_steps_done(lbm_handle h);

/* Copy the raw population planes of the current state to or from host
 * memory of lbm_raw_state_bytes() bytes, for checkpoint/restore.
 * Synchronous.  Velocity order of lbm_lattice_table.  Layout:
 *  - FP64/FP32 storage: 2Q planes of N values (g for velocities 0..Q-1,
 *    then h), the values g_i - gref_i and h_i - href_i;
 *  - 16-bit storage: Q planes of N 4-byte pairs (g_i in the low 16 bits, h_i
 *    in the high 16 bits), the values (g_i - gref_i)/gref_i and
 *    (h_i - href_i)/hscale_i.
 * gref_i = F_i(rho0, u = 0, T0) is the instance's reference equilibrium
 * (zero for whole storage), href_i = (delta/2) T0 gref_i, hscale_i = href_i
 * (gref_i when delta = 0). */
size_t lbm_raw_state_bytes(lbm_handle h);
int lbm_get_state(lbm_handle h, void* host, size_t bytes);
int lbm_set_state(lbm_handle h, const void* host, size_t bytes);

/* The library's own refined velocity set (Tables I/II, weights refined in
 * FP64 so that the isotropy conditions of degree <= 8 hold to round-off):
 * *q = Q; c[Q*D] integer velocities (row-major), w[Q] weights, *r the
 * scaling factor (xi_i = r c_i).  Any output pointer may be NULL. */
int lbm_lattice_table(int lattice, int* q, int* c, double* w, double* r);

/* Grid totals (as lbm_conserved: out[0] mass, out[1..D] momentum, out[D+1]
 * energy) of a raw state held in device memory, computed without allocating
 * anything.  The paper has no counterpart: this serves callers that cannot
 * call cudaMalloc when they need the totals -- e.g. a serving pool that has
 * reserved the whole device budget, or code holding populations in its own
 * arena without a library instance.
 *  state         device pointer to the planes in the layout of lbm_get_state
 *                (deviations from the reference equilibrium of rho0, T0);
 *                plane p starts plane_stride elements (pairs, for 16-bit
 *                storage) after plane p - 1.  It must be memory of the
 *                current device (or managed memory) and aligned to the
 *                storage word (8 bytes for FP64, 4 bytes otherwise); host
 *                pointers, other devices' memory and misaligned pointers
 *                fail with LBM_EINVAL before anything is launched.  The
 *                caller guarantees that the planes' extent, (2Q-1)
 *                plane_stride + ncells elements (Q-1 and pairs for 16-bit
 *                storage), lies inside the allocation
 *  ncells        cells per plane, 0 <= ncells <= 16777216 (4096^2 or 256^3);
 *                larger sizes fail with LBM_EINVAL
 *  lattice, prec, gamma, rho0, T0: as given to lbm_create (the same
 *                defaults: see the reference state above)
 *  stream        cudaStream_t to run on (NULL = default stream); the call
 *                synchronises it before returning
 *  out           host array of D + 2 doubles
 * The block partials live in one static device array of about 160 KB that
 * every GPU loading the library keeps until exit.  The first call on a
 * device looks up that array's device address (make it before any stream
 * capture).  That address is kept per device index for the life of the
 * process; after a cudaDeviceReset the array is mapped anew, so a process
 * that resets a device must not call this entry point again.  All calls
 * share the array: calls that overlap on the GPU race and give wrong
 * totals.  No cudaMalloc, cudaFree or allocating library routine is called. */
int lbm_conserved_noalloc(int lattice, int prec, double gamma, double rho0, double T0, const void* state,
                          long long ncells, long long plane_stride, void* stream, double* out);

/* Launch shapes of the step kernel (execution control with no counterpart in
 * the paper; every shape computes the same step, the stage-4, 7 and 8
 * shapes up to the summation order of the moments).  Each (lattice, precision) has a small
 * table of compiled candidates (how the pulled values are staged --
 * registers, shared memory by cp.async, g in registers and h in shared
 * memory (stages 0-3), the velocities of each cell split over 4 warps
 * (stage 4; stage 7 with the per-cell equilibrium coefficients formed once
 * and shared), for 16-bit storage the (g, h) pairs held packed in registers
 * (stage 6) or half of them so and half in shared memory (stage 9), or two
 * lanes per cell, one for c and one for -c of every
 * (c, -c) pair, whose moment sums meet by warp shuffles (stage 8) -- and
 * the cells per thread block); index 0 is the default.
 * lbm_shape_info describes candidate `index` (LBM_EINVAL past the end). */
int lbm_shape_info(int lattice, int prec, int index, int* stage, int* block);

/* Select a candidate shape for this instance's steps. */
int lbm_set_shape(lbm_handle h, int index);

/* Current shape index of the instance (-1 for NULL). */
int lbm_get_shape(lbm_handle h);

/* Time every candidate shape on this instance's own buffers (reps launches
 * each, CUDA events on its stream; the trials write only the idle buffer,
 * so the state does not change), select the fastest and return its index
 * and mean time per step in microseconds.  Synchronises. */
int lbm_autotune(lbm_handle h, int reps, int* best_index, double* best_us);

/* ------------------------------------------------------------------------
 * Continuous-batching pool: many independent instances of one lattice and
 * precision (shock tubes and periodic boxes of different sizes, gamma, tau,
 * step counts) resident in one device arena and advanced together by one
 * batched launch per time step.  Instances are admitted against the memory
 * budget as they arrive and retired when their results are read; each
 * instance computes exactly what it would alone (bitwise).  Serving machinery
 * with no counterpart in the paper; the step itself is lbm_step's.
 * Typical loop: lbm_pool_run(1) -> submit arrivals while the bundle runs
 * (LBM_EBUSY = wait for results) -> lbm_pool_sync -> lbm_pool_poll each
 * ticket -> lbm_pool_result for finished ones.
 * ------------------------------------------------------------------------ */
typedef struct lbm_pool* lbm_pool_handle;

typedef struct {
  int lattice;          /* lbm_lattice of every instance */
  int prec;             /* lbm_prec of every instance */
  size_t budget_bytes;  /* device bytes for instance states (the admission budget) */
  int max_instances;    /* resident instances at most */
  int max_tiles;        /* work-list entries at most (0 = sized from the budget) */
  int bundle_steps;     /* time steps per lbm_pool_run bundle (one CUDA graph) */
  void* stream;         /* cudaStream_t; NULL = the pool creates its own stream */
  void* device_mem;     /* optional caller-owned device buffer of >= lbm_pool_bytes(),
                           256-byte aligned; NULL = the library allocates */
  size_t device_bytes;
} lbm_pool_config;

/* Device bytes a pool needs (arena + slot table + work list); 0 if invalid. */
size_t lbm_pool_bytes(const lbm_pool_config* cfg);

/* Create a pool.  Errors: LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA. */
int lbm_pool_create(lbm_pool_handle* out, const lbm_pool_config* cfg);

/* Destroy a pool (synchronises; NULL-safe). */
int lbm_pool_destroy(lbm_pool_handle p);

/* Arena bytes an instance of this grid takes (two population buffers). */
size_t lbm_pool_instance_bytes(lbm_pool_handle p, const lbm_grid* grid);

/* Admit an instance: validate as lbm_create (grid->prec must equal the
 * pool's; grid->stream and grid->device_mem are ignored), set it to the
 * equilibrium of the host fields rho, u, T (as lbm_init) and give it `steps`
 * time steps to take from the next lbm_pool_run on.  May be called while a
 * bundle runs: the copies and the initialisation use the pool's own
 * admission stream, which it synchronises (the host arrays are copied when
 * it returns), not the pool stream.  LBM_EBUSY if no slot, budget or
 * work-list room is free now (nothing changes; retry after results are
 * read). */
int lbm_pool_submit(lbm_pool_handle p, double gamma, double tau_f, double tau_g, const lbm_grid* grid,
                    const double* rho, const double* u, const double* T, long steps, long long* ticket);

/* Enqueue `bundles` step bundles: each advances every resident instance
 * that has steps left by up to bundle_steps steps.  Asynchronous. */
int lbm_pool_run(lbm_pool_handle p, int bundles);

/* Synchronise the pool's stream and read the instances' error words: an
 * instance that met a non-finite state stops stepping on the device and is
 * reported finished (its lbm_pool_result returns LBM_ENONFINITE). */
int lbm_pool_sync(lbm_pool_handle p);

/* *done = 1 once all the instance's steps are enqueued (its result can be
 * read), else 0; *steps_done gets the steps enqueued so far.  Either pointer
 * may be NULL.  LBM_EINVAL for an unknown ticket. */
int lbm_pool_poll(lbm_pool_handle p, long long ticket, int* done, long* steps_done);

/* rho, u, T of a finished instance into host arrays (as lbm_moments), then
 * retire it and free its memory.  Synchronises.  LBM_EBUSY if it still has
 * steps left; LBM_ENONFINITE if it met a non-finite state (the arrays are
 * filled with NaN and the instance is retired all the same). */
int lbm_pool_result(lbm_pool_handle p, long long ticket, double* rho, double* u, double* T);

/* out[6]: resident instances, finished-but-unread instances, arena bytes in
 * use, arena bytes, work-list entries, persistent grid blocks. */
int lbm_pool_stats(lbm_pool_handle p, long long* out);

/* ------------------------------------------------------------------------
 * Slab decomposition of one grid along its slowest axis (y for D2Q37, z for
 * D3Q107) over nranks ranks: host-side plan, pack and unpack.  The paper
 * has no parallel design; this is the halo exchange a multi-GPU run of the
 * step would use.  A step pulls from at most 3 cells away per axis
 * (|c_a| <= 3 in Tables I/II), so a slab with 3 ghost layers on each side,
 * refreshed before every step, steps its owned cells exactly as the whole
 * grid would: ghost layer begin - k (k = 1..3) is read only by the
 * velocities with c_axis >= k, ghost layer end + k - 1 only by those with
 * c_axis <= -k, and only those populations travel.  At a zero-gradient end
 * the ghost layers repeat the edge layer (the clamped pull).
 * These calls work on host arrays in the raw FP64 layout of lbm_get_state
 * (2Q planes of plane_stride values: g for velocities 0..Q-1 in the order of
 * lbm_lattice_table, then h; cell x + nx (y + ny z) of the rank's local
 * grid local_n, its owned layers plus 3 ghost layers per side).  Every box
 * of this build has one GPU, so no device transport is provided; a rank
 * steps its local grid with the split axis' boundary set to zero-gradient.
 * ------------------------------------------------------------------------ */
typedef struct {
  int lattice, axis;      /* lattice; split axis (1 = y for D2Q37, 2 = z for D3Q107) */
  int n[3];               /* global grid */
  int periodic;           /* 1: periodic split axis, 0: zero-gradient ends */
  int nranks, rank;
  int begin, end;         /* owned global layers [begin, end) along the axis */
  int lo, hi;             /* neighbour ranks below / above; -1 at a zero-gradient end */
  int layer_cells;        /* cells per layer (nx in 2D, nx ny in 3D) */
  int local_n[3];         /* local grid: n with end - begin + 6 layers along the axis;
                             local layer k is global layer begin - 3 + k */
  long long msg_values;   /* doubles in each message (either direction) */
} lbm_slab;

/* Plan of rank `rank`: layers split as evenly as possible (rank r owns
 * [L r / nranks, L (r+1) / nranks)).  LBM_EINVAL for a bad lattice, grid or
 * rank, or a slab thinner than 3 layers. */
int lbm_slab_plan(int lattice, const int n[3], int periodic, int nranks, int rank, lbm_slab* out);

/* Pack the two messages of msg_values doubles: to_hi (for the rank above)
 * holds, for k = 1..3, owned layer end - k of every population with
 * c_axis >= k (g planes, then h); to_lo (for the rank below) owned layer
 * begin + k - 1 of those with c_axis <= -k.  Either output may be NULL. */
int lbm_slab_pack(const lbm_slab* s, const double* state, long long plane_stride, double* to_lo, double* to_hi);

/* Unpack the neighbours' messages into the ghost layers: from_lo (the rank
 * below's to_hi) and from_hi (the rank above's to_lo); at a zero-gradient
 * end the ghost layers get copies of the edge layer (every plane) and the
 * message pointer of that side may be NULL. */
int lbm_slab_unpack(const lbm_slab* s, double* state, long long plane_stride, const double* from_lo,
                    const double* from_hi);

/* General Hermite quadrature (the construction of Sec. IV, for any/* General Hermite quadrature (the construction of Sec. IV, for any
 * symmetric integer velocity set): the velocities are all sign flips and
 * axis permutations of the ngroups representatives reps[ngroups*D]
 * (D = 1..3); find one weight per group w_group[ngroups] and the scale r
 * (xi = r c) such that sum_i w_i (r c_i)^alpha equals the moment E[x^alpha]
 * of the unit Gaussian for each of the nconds even monomial classes
 * exps[nconds*D] (odd moments vanish by symmetry).  nconds == ngroups keeps
 * r = r_in; nconds == ngroups + 1 solves r starting from r_in.  *q gets the
 * number of velocities, *max_residual the largest relative condition error.
 * E.g. D2Q9: reps {0,0, 1,0, 1,1}, exps {0,0, 2,0, 4,0, 2,2} -> r = sqrt 3,
 * w = 4/9, 1/9, 1/36.  LBM_EINVAL with a message if there is no solution. */
int lbm_quadrature(int D, int ngroups, const int* reps, int nconds, const int* exps, double r_in, int* q,
                   double* w_group, double* r, double* max_residual);

/* Thread-local message of the last failed call on this thread ("" if none). */
const char* lbm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
