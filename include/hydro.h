/*
 * hydro.h -- C ABI of libhydro: the aggregated per-sub-grid hydro
 * right-hand-side (RHS) evaluation on one NVIDIA GB300 (sm_103a).
 *
 * The operation (Sec. IV-B of "From Task-Based GPU Work Aggregation to
 * Stellar Mergers", Daiss et al.): for each sub-grid of an octree AMR mesh
 * (N^3 interior cells plus a ghost layer of thickness 3, Sec. V-A), convert
 * the conserved fields to primitives, reconstruct them on every cell face with
 * the piecewise-parabolic method (Colella & Woodward 1984), evaluate the
 * central(-upwind) flux of Kurganov & Tadmor with the largest local signal
 * speed, and return the flux divergence dU/dt together with the largest
 * signal speed (the input of the Courant condition, Sec. IV-B).  Many
 * sub-grids are evaluated in one launch: the explicit work aggregation of
 * Sec. V-D (strategy 3), with mixed sub-grid sizes (strategy 1, Sec. V-B).
 *
 * Conventions common to every entry point
 *   - Fields, in order: 0 rho, 1-3 momentum (x, y, z), 4 total energy E,
 *     5 entropy tracer tau = (rho e)^(1/gamma), 6.. species densities rho_k.
 *     n_fields = 6 + species, 6 <= n_fields <= HYDRO_MAX_FIELDS.
 *   - Input U of a sub-grid: binary64, [n_fields][G][G][G] with G = N + 2*ghost
 *     and x fastest; 8-byte aligned; in memory the GPU can read (device
 *     memory, or pinned host memory, which the kernels read in place over the
 *     host link).  Only the 3 innermost ghost layers are read, and of those
 *     only the cells with at most one coordinate outside the interior (the
 *     26-point variant, HYDRO_F_QUAD26, also reads cells two deep in a second
 *     coordinate).  U is never written.
 *   - Output dU/dt: binary64, packed in descriptor order: sub-grid s occupies
 *     n_fields_s * N_s^3 doubles ([f][z][y][x]) starting at
 *     sum_{t<s} n_fields_t * N_t^3.  Output amax: one double per sub-grid.
 *     Both in device memory or pinned host memory, owned by the caller and
 *     fully overwritten.
 *   - Streams are cudaStream_t passed as void*; NULL means the legacy default
 *     stream.  Every launch entry point is asynchronous with respect to the
 *     host.  Pointers are plain addresses in CUDA's unified address space
 *     (device pointers, e.g. from torch tensors, or pinned host pointers).
 *   - Return value: HYDRO_OK (0) or a negative status below.  No entry point
 *     aborts the process or traps the GPU; device-side problems are recorded
 *     in a per-device status word read back by hydro_status().
 *   - Thread safety: entry points may be called from several host threads
 *     at once, also for different devices: each device's context has its
 *     own lock for set-up and the status word, and the direct calls
 *     (hydro_rhs, hydro_rhs_ex, hydro_rhs_per_subgrid) each take one of four
 *     work-list slots with its own lock, so that up to four of them build
 *     their work lists and wait for their slots concurrently.  A plan,
 *     server or forest handle may be used by one thread at a time.
 */
#ifndef HYDRO_H_
#define HYDRO_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HYDRO_MAX_FIELDS 11 /* 6 + up to 5 species */
#define HYDRO_MAX_N 256     /* largest interior edge accepted */

/* status codes */
#define HYDRO_OK 0
#define HYDRO_EINVAL (-1)    /* bad argument: NULL pointer, N < 2, ghost < 3, n_fields out of
                                range, gamma <= 1, dx <= 0, uniform-batch mismatch, overflow */
#define HYDRO_ENOMEM (-2)    /* a library workspace could not be allocated */
#define HYDRO_ECUDA (-3)     /* a CUDA runtime call failed; see hydro_last_cuda_error() */
#define HYDRO_ENONPHYS (-4)  /* device flag: rho <= 0, p <= 0 or non-finite value read */
#define HYDRO_EBUDGET (-5)   /* serving: the task can never fit the memory budget */
#define HYDRO_ETIMEDOUT (-6) /* serving: the wait ran past its deadline */
#define HYDRO_EBUSY (-7)     /* serving: queue full, try again */
#define HYDRO_ETOOBIG (-8)   /* hydro_rhs_noalloc: more sub-grids than its fixed scratch holds */

/* One sub-grid task.  The aggregation allocator's per-task chunk of Sec. V-D:
 * each task brings its own input block; the library packs the outputs. */
typedef struct {
  const double* U; /* [n_fields][N+2g]^3, x fastest; memory the GPU can read: device
                      memory, or pinned host memory (cudaHostAlloc / cudaHostRegister),
                      which the kernels read in place over the host link -- on GB300
                      NVLink-C2C -- moving only the cells the scheme reads */
  double dx;       /* cell width > 0 (depends on the octree level) */
  int32_t N;       /* interior cells per edge, 2..HYDRO_MAX_N (8 and 16 are the paper's) */
  int32_t n_fields;
} hydro_subgrid_t;

/* Arithmetic of the reconstruction and flux steps.
 *   HYDRO_FP64: every step in binary64 (Sec. VI-A: all floating point in
 *     double precision).
 *   HYDRO_FP32_FLUX_FP64_ACC: primitives and the dual-energy decision as in
 *     HYDRO_FP64 within binary32 rounding, reconstruction and flux in
 *     binary32, flux differences and their sum carried exactly/in binary64
 *     so that the divergence telescopes (conservation). */
typedef enum { HYDRO_FP64 = 0, HYDRO_FP32_FLUX_FP64_ACC = 1 } hydro_precision_t;

/* ---------------------------------------------------------------------------
 * hydro_rhs -- one aggregated RHS evaluation over n_subgrids sub-grids in one
 * fused launch (Sec. V-D), binary64, on the legacy default stream.
 *   subgrids   HOST array of n_subgrids descriptors; copied, reusable on return
 *   n_subgrids >= 0 (0 is a no-op)
 *   N, n_fields  if > 0, every descriptor must match (uniform batch), else
 *              HYDRO_EINVAL; 0 means per-descriptor values
 *   ghost      ghost layers stored in U, >= 3 (layers beyond 3 are ignored)
 *   gamma      ratio of specific heats, > 1
 *   out_dUdt, out_amax  outputs as described above, in device memory or in
 *              pinned host memory (written in place by the kernel)
 * Work list: a batch of one N and one field count has its tiles built on the
 * device from the copied descriptors; other batches build it on the host,
 * the sub-grids with more fields first.
 * Allocation: the first call on a device (and a call with a larger batch than
 * any before) allocates library workspace; later calls allocate nothing. */
int hydro_rhs(const hydro_subgrid_t* subgrids, int64_t n_subgrids, int32_t N, int32_t ghost,
              int32_t n_fields, double gamma, double* out_dUdt, double* out_amax);

/* hydro_rhs with a precision, a stream (cudaStream_t as void*) and flags
 * (HYDRO_F_* below, 0 for defaults). */
#define HYDRO_F_NO_STATUS 1u /* skip the nonphysical-input checks' status writes */
#define HYDRO_F_KNP 2u       /* central-upwind flux with one-sided local speeds (Kurganov,
                                Noelle & Petrova 2001) instead of the single-speed
                                Kurganov-Tadmor flux; same signal speed for amax */
#define HYDRO_F_QUAD26 8u         /* the 26-point variant of Sec. IV-B: fluxes at the 9
                                     points of every face (centre, edge midpoints,
                                     vertices) from PPM along the lines through them,
                                     combined with Simpson weights; reads the ghosted
                                     block except its 3-deep edges beyond 2 cells */
#define HYDRO_F_REGISTER_LOADS 4u /* mixed form: the kernel that loads the read region
                                     through registers instead of the default pipelined
                                     kernel (asynchronous copies into shared memory,
                                     one CTA of 576 threads per SM); same results */
int hydro_rhs_ex(const hydro_subgrid_t* subgrids, int64_t n_subgrids, int32_t N, int32_t ghost,
                 int32_t n_fields, double gamma, double* out_dUdt, double* out_amax,
                 hydro_precision_t prec, void* stream, uint32_t flags);

/* The plain per-sub-grid launch form (strategy 2 of Sec. V-C): the same
 * arithmetic as hydro_rhs_ex, but one kernel launch per sub-grid, issued
 * round-robin over `n_streams` caller-provided streams (streams[i] as void*;
 * n_streams >= 1).  Kept as the comparison baseline of the aggregated form.
 * Allocation as for hydro_rhs. */
int hydro_rhs_per_subgrid(const hydro_subgrid_t* subgrids, int64_t n_subgrids, int32_t ghost,
                          double gamma, double* out_dUdt, double* out_amax,
                          hydro_precision_t prec, void* const* streams, int32_t n_streams);

/* hydro_rhs_per_subgrid with flags: HYDRO_F_KNP, HYDRO_F_QUAD26 (each launch
 * then runs the 26-point kernel), HYDRO_F_REGISTER_LOADS, HYDRO_F_NO_STATUS,
 * as for hydro_rhs_ex; the results equal hydro_rhs_ex's with the same flags
 * bit for bit.  HYDRO_EINVAL for other flag bits. */
int hydro_rhs_per_subgrid_ex(const hydro_subgrid_t* subgrids, int64_t n_subgrids, int32_t ghost,
                             double gamma, double* out_dUdt, double* out_amax,
                             hydro_precision_t prec, void* const* streams, int32_t n_streams,
                             uint32_t flags);

/* ---------------------------------------------------------------------------
 * Plans: a fixed batch (the descriptors, hence the input pointers, are bound
 * at creation) whose work list is built, sorted and uploaded once, whose
 * launch configuration is chosen by the autotuner (HYDRO_PLAN_AUTOTUNE) and
 * whose launch is captured once in a CUDA graph and replayed by
 * hydro_plan_execute (the aggregation region of Sec. V-D, made static).
 * hydro_plan_create allocates (work list, tuning scratch); execute allocates
 * nothing.  The output pointers may change between executions. */
typedef struct hydro_plan hydro_plan_t;
#define HYDRO_PLAN_AUTOTUNE 1u /* time candidate launch shapes and keep the fastest */
#define HYDRO_PLAN_NO_GRAPH 2u /* launch directly instead of replaying a graph */
#define HYDRO_PLAN_KNP 4u      /* the flux of HYDRO_F_KNP */
#define HYDRO_PLAN_PIPELINED 8u       /* mixed form: consider only the pipelined kernel */
#define HYDRO_PLAN_REGISTER_LOADS 16u /* mixed form: consider only the register-load kernels */
#define HYDRO_PLAN_QUAD26 32u         /* the flux of HYDRO_F_QUAD26 (one launch shape; the
                                         autotuner keeps it) */

typedef struct {
  int64_t n_subgrids;
  int64_t n_tiles;         /* 8^3 work tiles (a 16^3 sub-grid is 8 tiles) */
  int64_t interior_cells;  /* sum of N^3 */
  int64_t out_doubles;     /* packed dU/dt length */
  int64_t alg_bytes;       /* algorithmic bytes of one execution (read region + outputs) */
  int32_t threads_per_cta; /* chosen launch shape */
  int32_t ctas_per_sm;
  int32_t grid;
  int32_t smem_bytes;
  float tuned_ms;          /* autotuner's best time, 0 if not tuned */
  int32_t n_candidates;    /* configurations the autotuner timed */
  int32_t lines_per_chunk; /* lines reconstructed per shared-memory chunk */
  int32_t prefetch;        /* L2 prefetch of the next tile: 0 none, 1 per row, 2 per plane */
  int32_t regs_cap;        /* kernel variant: 65536 / (threads * min resident CTAs) */
  int32_t load_batch;      /* kernel variant: read-region slots a thread loads at once
                              (0: the pipelined and 26-point kernels) */
} hydro_plan_info_t;

int hydro_plan_create(const hydro_subgrid_t* subgrids, int64_t n_subgrids, int32_t ghost,
                      double gamma, hydro_precision_t prec, uint32_t flags, void* stream,
                      hydro_plan_t** out_plan);
int hydro_plan_execute(hydro_plan_t* plan, double* out_dUdt, double* out_amax, void* stream);
int hydro_plan_info(const hydro_plan_t* plan, hydro_plan_info_t* info);
int hydro_plan_destroy(hydro_plan_t* plan);

/* ---------------------------------------------------------------------------
 * hydro_status -- synchronise `stream`, then read and clear this device's
 * sticky status word.  Returns HYDRO_OK, or HYDRO_ENONPHYS if any launch since
 * the last call read a nonphysical value (rho <= 0, p <= 0 or non-finite) in a
 * sub-grid's read region; then *first_bad_subgrid (may be NULL) receives the
 * smallest offending sub-grid index of those launches (index within its own
 * batch).  Outputs of a flagged sub-grid are written but meaningless. */
int hydro_status(void* stream, int64_t* first_bad_subgrid);

/* Text for a status code; never NULL. */
const char* hydro_strerror(int status);
/* Text of the last CUDA error seen by the library on this thread's calls. */
const char* hydro_last_cuda_error(void);

/* ---------------------------------------------------------------------------
 * Serving: a request loop over the aggregated kernel (strategy 3 of Sec. V-D
 * with several parent executors, combined with strategy 2).  Tasks
 * (one or more sub-grids whose state is already resident on the device) are
 * submitted from any host thread; a scheduler thread admits queued tasks in
 * arrival order while the memory budget allows and a launch stream is idle,
 * packs every admitted task's sub-grids into one work list and launches one
 * kernel for all of them on that stream (continuous batching: tasks that
 * arrive while other launches run join the next launch on a free stream).
 * Completion is observed with CUDA events; latency is measured on the host
 * monotonic clock (CLOCK_MONOTONIC nanoseconds).
 *
 * hydro_server_create allocates the streams, events and per-stream work-list
 * buffers; submit and the scheduler allocate nothing unless a launch needs a
 * larger work list than any before.  The server launches on its own streams;
 * a task's outputs are complete when poll/wait report HYDRO_OK (the host may
 * then read them after a device-wide or stream synchronisation of its own). */
typedef struct hydro_server hydro_server_t;

typedef struct {
  int64_t budget_bytes;   /* admitted-and-unfinished tasks' bytes (read blocks + outputs) stay
                             below this; a task larger than the whole budget is rejected */
  int32_t max_batch;      /* most sub-grids per launch (the "maximum aggregated kernels" of
                             Sec. V-D); a single larger task is launched alone */
  int32_t n_streams;      /* launch streams, >= 1 */
  int32_t ghost;          /* ghost layers of every submitted U, >= 3 */
  int32_t queue_capacity; /* queued tasks before submit answers HYDRO_EBUSY, >= 1 */
  double gamma;           /* > 1 */
  hydro_precision_t prec;
  int32_t per_task;       /* 1: never aggregate; one launch per task (the comparison form) */
  int64_t dry_run_ns;     /* > 0: no GPU work at all; a launch "completes" this many ns after
                             it starts (host-only testing of admission, order and timeouts) */
  uint32_t flags;         /* HYDRO_F_KNP, HYDRO_F_QUAD26 (the 26-point variant), or 0 */
} hydro_server_cfg_t;

typedef struct {
  int64_t submitted, completed, rejected;
  int64_t launches, subgrids_launched, max_subgrids_per_launch;
  int64_t bytes_in_flight, peak_bytes_in_flight;
  int64_t queued;
} hydro_server_stats_t;

int hydro_server_create(const hydro_server_cfg_t* cfg, hydro_server_t** out_server);
/* subgrids: HOST array of n >= 1 descriptors (copied).  out_dUdt / out_amax:
 * DEVICE outputs of this task (packed as for hydro_rhs).  *ticket receives the
 * task's id.  HYDRO_EBUDGET: the task alone exceeds the budget; HYDRO_EBUSY:
 * queue full. */
int hydro_server_submit(hydro_server_t* srv, const hydro_subgrid_t* subgrids, int32_t n,
                        double* out_dUdt, double* out_amax, int64_t* ticket);
/* HYDRO_OK if the task has completed, HYDRO_EBUSY if not yet, HYDRO_EINVAL for
 * an unknown ticket; HYDRO_ECUDA if its launch failed. */
int hydro_server_poll(hydro_server_t* srv, int64_t ticket);
/* Block until the task completes or timeout_ns (< 0: no limit) passes; the
 * deadline is host-side, the task itself keeps running: HYDRO_ETIMEDOUT. */
int hydro_server_wait(hydro_server_t* srv, int64_t ticket, int64_t timeout_ns);
/* Host monotonic times of a task: submitted, launched, completion observed
 * (0 where not reached yet). */
int hydro_server_times(hydro_server_t* srv, int64_t ticket, int64_t* t_submit_ns,
                       int64_t* t_launch_ns, int64_t* t_done_ns);
int hydro_server_stats(hydro_server_t* srv, hydro_server_stats_t* stats);
/* Drain (wait for every admitted launch), stop the scheduler, free. */
int hydro_server_destroy(hydro_server_t* srv);
/* Host monotonic clock in ns, the clock of hydro_server_times. */
int64_t hydro_now_ns(void);

/* ---------------------------------------------------------------------------
 * Domains: nb^3 same-level sub-grids of N^3 cells tiling a periodic cube,
 * stored WITHOUT ghost layers: U[s][f][z][y][x] (DEVICE, binary64), sub-grid
 * s = bx + nb (by + nb bz) holding cells [bx N, bx N + N) ... of the cube.
 * Each sub-grid's 3-deep ghost shell is gathered inside the kernel from its
 * neighbours (the ghost exchange that precedes every hydro iteration,
 * Sec. V-A), so no ghosted copy exists.  nb * N >= 6; nb^3 N^3 n_fields
 * < 2^31; dx the cell width of every sub-grid.
 *
 * hydro_domain_rhs -- dU/dt (packed exactly like U) and amax per sub-grid,
 * the arithmetic of hydro_rhs_ex on the equivalent ghosted sub-grids.
 * hydro_domain_stage -- one explicit stage in the same launch:
 *   U_out = alpha * U0 + beta * (U + dt * dU/dt(U))
 * (SSP-RK3 of Shu & Osher: (alpha, beta) = (0,1), (3/4,1/4), (1/3,2/3) with
 * U0 the state at the start of the step; the paper's time step has three
 * hydro iterations, Sec. VI-A).  U_out must not alias U; U0 may alias U or
 * U_out.  flags: HYDRO_F_KNP, HYDRO_F_QUAD26 (the 26-point variant), or 0.
 * Both launch asynchronously on `stream`,
 * allocate nothing, and record nonphysical input in the hydro_status word. */
int hydro_domain_rhs(const double* U, int32_t nb, int32_t N, int32_t n_fields, double dx,
                     double gamma, double* out_dUdt, double* out_amax, hydro_precision_t prec,
                     void* stream, uint32_t flags);
int hydro_domain_stage(const double* U, const double* U0, double alpha, double beta, double dt,
                       int32_t nb, int32_t N, int32_t n_fields, double dx, double gamma,
                       double* U_out, double* out_amax, hydro_precision_t prec, void* stream,
                       uint32_t flags);
/* hydro_domain_stage with dt read from DEVICE memory (one double, 8-byte
 * aligned) when the kernel runs, e.g. written by hydro_courant earlier on
 * the same stream: a time loop then needs no host round trip and records
 * into a CUDA graph. */
int hydro_domain_stage_dt(const double* U, const double* U0, double alpha, double beta,
                          const double* dt, int32_t nb, int32_t N, int32_t n_fields, double dx,
                          double gamma, double* U_out, double* out_amax, hydro_precision_t prec,
                          void* stream, uint32_t flags);

/* ---------------------------------------------------------------------------
 * Forests: the adaptive mesh of the paper's application (Cartesian adaptive
 * mesh refinement of an octree of sub-grids, Sec. III), as the leaves of an
 * octree over a periodic cube of nb0^3 root blocks.  Every leaf holds N^3
 * cells of width dx0 / 2^level and is stored without ghost layers,
 * U[s][f][z][y][x] (DEVICE, binary64) for the leaves in the order given at
 * creation.  Face neighbours must differ by at most one level (2:1 balance).
 *
 * The ghost shells are built on the device before every RHS: a face
 * neighbour of the same level is read in place (as in hydro_domain_rhs);
 * for a neighbour of another level the slab is first transferred into a
 * library-owned auxiliary block:
 *   - coarser neighbour: each ghost cell takes the value of the coarse cell
 *     that contains it (piecewise-constant prolongation);
 *   - finer neighbours (four leaves): each ghost cell takes the mean of the
 *     eight fine cells it covers, summed in the order i + 2j + 4k of their
 *     offsets, times 1/8 (restriction).
 * Then the tile kernel runs on every leaf (face-centre scheme, or the
 * 26-point variant: see the flags below) and records the fluxes through
 * faces towards other levels; last, every coarse cell
 * next to finer leaves has the flux through that face replaced by the mean
 * of the four fine fluxes (summed (0,0), (1,0), (0,1), (1,1) over the two
 * tangential offsets, times 1/4; x, then y, then z faces), so that the RHS
 * conserves every field to rounding, as the paper's application does.
 * The paper states no level-transfer formulas: these are readings.
 */
typedef struct {
  int32_t level;      /* 0 = root blocks; at most HYDRO_FOREST_MAX_LEVEL */
  int32_t bx, by, bz; /* block coordinates at that level, in [0, nb0 << level) */
} hydro_leaf_t;

#define HYDRO_FOREST_MAX_LEVEL 15
typedef struct hydro_forest hydro_forest_t;

typedef struct {
  int32_t n_leaves;
  int32_t N, n_fields, nb0;
  int32_t max_level;
  int32_t n_level_faces;    /* leaf faces towards another level (auxiliary blocks) */
  int32_t n_reflux_leaves;  /* leaves with at least one finer face neighbour */
  int32_t quad26;           /* 1 if edge and corner neighbours also differ by at most one
                               level, so that HYDRO_F_QUAD26 is accepted */
  int64_t device_bytes;     /* tables, auxiliary blocks and flux registers (and the ghosted
                               blocks once a 26-point call has allocated them) */
} hydro_forest_info_t;

/* Face neighbours of a forest's leaves, computed on the host (no GPU call):
 * for leaf s and face k = 2 d + side (d = x, y, z; side 1 the high face),
 * kind[6 s + k] = 0 same level, -1 coarser, +1 finer, and nbr[6 s + k] =
 * the neighbour leaf (same level or coarser), or for finer neighbours the
 * leaf of the four that touches the face at its lowest tangential corner.
 * kind and nbr may be NULL.  HYDRO_EINVAL if the leaves are not a 2:1
 * balanced exact cover of the cube (duplicates, overlaps, gaps, levels or
 * coordinates out of range), or N is odd, < 6 or > HYDRO_MAX_N (a ghost
 * slab of three cells must lie in one finer leaf), or nb0 < 1. */
int hydro_forest_links(const hydro_leaf_t* leaves, int32_t n_leaves, int32_t nb0, int32_t N,
                       int32_t* kind, int32_t* nbr);

/* Validate the forest (as hydro_forest_links, plus 6 <= n_fields <=
 * HYDRO_MAX_FIELDS), build its tables and allocate its device memory (on
 * the current device).  The forest is then used on that device only. */
int hydro_forest_create(const hydro_leaf_t* leaves, int32_t n_leaves, int32_t nb0, int32_t N,
                        int32_t n_fields, hydro_forest_t** out);
int hydro_forest_info(const hydro_forest_t* forest, hydro_forest_info_t* info);

/* dU/dt (packed like U) and amax per leaf, with dx0 the cell width of
 * level 0.  hydro_forest_stage: U_out = alpha U0 + beta (U + dt dU/dt) in
 * the same launches (as hydro_domain_stage; U_out must not alias U, U0 may
 * alias U or U_out).  flags: HYDRO_F_KNP, HYDRO_F_REGISTER_LOADS (mixed form:
 * the register-load kernel instead of the pipelined one; same results),
 * HYDRO_F_QUAD26 (the 26-point variant; its diagonal lines read edge and
 * corner ghosts, filled by the same rule from the 26 neighbours: accepted
 * only if those differ from every leaf by at most one level too, see
 * hydro_forest_info_t.quad26; HYDRO_EINVAL otherwise) or 0.  Three launches
 * on `stream` (level transfer, tiles, flux correction; with HYDRO_F_QUAD26:
 * a gather of every leaf's ghosted block, the 26-point tiles, the flux
 * correction).  Nothing is allocated, except that the first HYDRO_F_QUAD26
 * call allocates the ghosted blocks (n_leaves F (N+6)^3 doubles, kept until
 * hydro_forest_destroy): make it before any stream capture.  The auxiliary
 * blocks, ghosted blocks and flux registers belong to the forest, so calls
 * on one forest must be ordered (one stream, or synchronised). */
int hydro_forest_rhs(hydro_forest_t* forest, const double* U, double dx0, double gamma,
                     double* out_dUdt, double* out_amax, hydro_precision_t prec, void* stream,
                     uint32_t flags);
int hydro_forest_stage(hydro_forest_t* forest, const double* U, const double* U0, double alpha,
                       double beta, double dt, double dx0, double gamma, double* U_out,
                       double* out_amax, hydro_precision_t prec, void* stream, uint32_t flags);
/* hydro_forest_stage with dt read from DEVICE memory (as hydro_domain_stage_dt). */
int hydro_forest_stage_dt(hydro_forest_t* forest, const double* U, const double* U0, double alpha,
                          double beta, const double* dt, double dx0, double gamma, double* U_out,
                          double* out_amax, hydro_precision_t prec, void* stream, uint32_t flags);
/* Free the forest's device memory (synchronises its device). */
int hydro_forest_destroy(hydro_forest_t* forest);

/* ---------------------------------------------------------------------------
 * hydro_courant -- the Courant time step on the device (one small launch on
 * `stream`), from the largest signal speeds that earlier RHS or stage
 * launches wrote (Sec. IV-B), so that explicit steps need no host round trip.
 *   amax      DEVICE, n_rows rows of n values, row r at amax + r*row_stride
 *             (row_stride >= n): e.g. the three stages of the previous step;
 *             a_s = max over the rows of the sub-grid's value.
 *   dx        DEVICE array of n cell widths (sub-grids of several levels):
 *             q = cfl * min_s(dx_s / a_s); or NULL with dx_uniform > 0:
 *             q = (cfl * dx_uniform) / max_s a_s.
 *   clock     DEVICE, 3 doubles {t, dt, steps}, read and updated in place:
 *             dt = min(q, t_end - t) (0 once t >= t_end), t += dt, steps += 1.
 *   dt_hist   optional DEVICE array: dt_hist[steps] = dt while steps < hist_len.
 * The paper has no such routine; it is the step rule of the time loops of the
 * tests and benchmark moved onto the device.  HYDRO_EINVAL on null or
 * misaligned pointers, n < 1, n_rows < 1, row_stride < n, cfl <= 0. */
int hydro_courant(const double* amax, int32_t n_rows, int64_t row_stride, int64_t n,
                  const double* dx, double dx_uniform, double cfl, double t_end, double* clock,
                  double* dt_hist, int64_t hist_len, void* stream);

/* ---------------------------------------------------------------------------
 * hydro_rhs_noalloc -- hydro_rhs_ex for callers that cannot allocate memory.
 * The paper has no counterpart: this is a service of the library.
 *
 * Who needs it: code that must not call cudaMalloc or any allocating routine
 * -- real-time loops where an allocation (which may synchronise the device)
 * is not acceptable, or processes whose device memory belongs to another
 * allocator (a framework's caching allocator) that must not be bypassed or
 * that has handed out all of it.  hydro_rhs_ex allocates its work list on
 * its first calls; this entry point allocates nothing, on the device or the
 * host heap.  The caller still provides the inputs and the outputs.
 *
 * How: the sub-grid descriptors are copied into a fixed device array that is
 * part of the library image (HYDRO_NOALLOC_MAX_SUBGRIDS entries, 192 KiB; it
 * occupies device memory on every GPU that loads the library until the
 * process exits), and a register-load tile kernel reads them there (256
 * threads per CTA, 32 lines per chunk).  The per-cell arithmetic is that of
 * hydro_rhs_ex's kernels in both precision forms, so the results are bitwise
 * equal to hydro_rhs_ex's for the same batch.
 *   - Uniform batches only: 2 <= N <= HYDRO_MAX_N and 6 <= n_fields <=
 *     HYDRO_MAX_FIELDS (0, "any", is not accepted here), and every
 *     descriptor must match them; dx may differ per sub-grid.  Otherwise
 *     HYDRO_EINVAL, nothing runs.
 *   - n_subgrids > HYDRO_NOALLOC_MAX_SUBGRIDS: HYDRO_ETOOBIG, nothing runs.
 *   - The first call on a device (with that device current) resolves the
 *     array's device address and sets the kernels' attributes for that
 *     device; later calls on that device skip this set-up.
 *   - The descriptor array is copied with cudaMemcpyAsync on `stream`.  From
 *     pageable host memory the copy has taken the data when the call
 *     returns, and the array may be reused at once; from page-locked (pinned)
 *     host memory the copy runs in stream order, so the array must stay
 *     unchanged until the stream has passed this call.
 *   - Every call reuses the same device array, which keeps the last call's
 *     descriptors: two calls whose work overlaps on the GPU (different
 *     streams, not ordered) race on it.  Calls on one stream, or otherwise
 *     ordered, are safe.  out_amax is cleared by the call itself where
 *     sub-grids span several tiles.
 *   - Nonphysical inputs are not recorded (hydro_status does not see this
 *     entry point's launches).
 * Other arguments and the output layout are those of hydro_rhs_ex. */
#define HYDRO_NOALLOC_MAX_SUBGRIDS 8192
int hydro_rhs_noalloc(const hydro_subgrid_t* subgrids, int64_t n_subgrids, int32_t N,
                      int32_t ghost, int32_t n_fields, double gamma, double* out_dUdt,
                      double* out_amax, hydro_precision_t prec, void* stream);

/* ---------------------------------------------------------------------------
 * hydro_probe_fp64 -- a measurement aid, not part of the method (the paper
 * has no counterpart): the binary64 form is bound by the binary64 pipe, so
 * its roofline needs the rate that pipe reaches on the GPU in use.  Enqueues
 * on `stream` one launch of a kernel that runs only independent binary64
 * fused multiply-adds (blocks_per_sm x SMs CTAs of 256 threads, 8 chains of
 * `iters` steps per thread) and writes their number to *fma_per_launch
 * (host).  The caller times the launch, e.g. with CUDA events on `stream`;
 * 2 * *fma_per_launch / seconds is the measured binary64 peak in flop/s.
 * Allocates nothing.  HYDRO_EINVAL for blocks_per_sm outside [1, 64],
 * iters < 1 or a null result pointer; HYDRO_ECUDA if the launch fails. */
int hydro_probe_fp64(int32_t blocks_per_sm, int32_t iters, void* stream, double* fma_per_launch);

/* Packed output length (doubles) of a batch; -1 on bad arguments. */
int64_t hydro_output_doubles(const hydro_subgrid_t* subgrids, int64_t n_subgrids);

/* Library version (major*10000 + minor*100 + patch). */
int hydro_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HYDRO_H_ */
