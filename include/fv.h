/*
 * fv.h -- C ABI of the GB300 temporally adaptive finite-volume hot path.
 *
 * The library advances the inviscid compressible Euler equations (the
 * integral balance law of Eq. 1 with no source term) on an unstructured
 * tetrahedral mesh with the temporally adaptive explicit scheme of
 * Algorithm 2 (Sec. 2.2): every cell gets a local explicit time step, cells
 * are binned into levels k = 0..L-1 with dt_k = 2^k dt_min (neighbours at
 * most one level apart), and one cycle ("iteration" in the paper) runs
 * 2^(L-1) subiterations in which level k starts a step every 2^k
 * subiterations.  Each level step is a predictor/corrector (Heun) step in
 * flux form; states of neighbours on other levels are interpolated linearly
 * in time; a coarse cell takes the time integral of the fine-side fluxes on a
 * level interface, so the method conserves mass, momentum and energy.
 * Fluxes: least-squares gradients, MUSCL reconstruction with the minmod
 * limiter, exact Godunov Riemann solver (Newton on the star pressure).
 *
 * Conventions (all entry points):
 *  - Every call returns FV_OK (0) or a negative FV_ERR_* code and never
 *    aborts; fv_last_error() returns a message for the calling thread's last
 *    failure.
 *  - Device work is enqueued on `stream` (a cudaStream_t, NULL = legacy
 *    default stream) and is asynchronous unless stated otherwise.
 *  - Host arrays passed in are read during the call only (copied).
 *    Device pointers passed in are borrowed, never freed, and must stay
 *    valid until the work enqueued on `stream` has finished.
 *  - Cell data exchanged with the caller are in the caller's tet order,
 *    structure of arrays: component c of cell i at [c * n_tets + i].
 *  - A mesh handle is not thread-safe; distinct handles are independent.
 *  - The library owns the device memory it allocates for a mesh (freed by
 *    fv_mesh_free) and calls cudaSetDevice(cfg.device) inside every call.
 */
#ifndef FV_H
#define FV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FV_OK 0
#define FV_ERR_INVALID_ARG (-1) /* bad argument or call out of order */
#define FV_ERR_BAD_MESH (-2)    /* inverted/degenerate tet, non-manifold or untagged face */
#define FV_ERR_CUDA (-3)        /* a CUDA runtime call failed */
#define FV_ERR_NONPHYSICAL (-4) /* density or pressure not positive/finite */
#define FV_ERR_RIEMANN (-5)     /* vacuum generation or Newton non-convergence */
#define FV_ERR_TIMEOUT (-6)     /* a bounded device wait gave up */
#define FV_ERR_NOMEM (-7)       /* device allocation failed */

/* face boundary tags (face_bc) */
#define FV_BC_INTERIOR 0
#define FV_BC_WALL 1         /* slip wall: ghost mirrors the normal velocity */
#define FV_BC_TRANSMISSIVE 2 /* ghost copies the interior state */

/* precision modes */
#define FV_FP64 0      /* everything in FP64 */
#define FV_FP32_FLUX 1 /* reconstruction and Riemann flux in FP32; state,
                          residual sums and flux time integrals in FP64 */

/* initial guess of the Newton iteration on the star pressure */
#define FV_GUESS_TWO_RAREFACTION 0
#define FV_GUESS_MLP 1

typedef struct fv_config {
  double gamma;        /* ratio of specific heats (1.4) */
  double cfl;          /* CFL number of the local time step (0.5) */
  double newton_tol;   /* relative change that stops Newton (1e-10) */
  int max_levels;      /* L: number of temporal levels, 1..8 */
  int newton_max_iter; /* Newton iterations before FV_ERR_RIEMANN (50) */
  int precision;       /* FV_FP64 or FV_FP32_FLUX */
  int guess;           /* FV_GUESS_TWO_RAREFACTION at load; fv_mlp_load selects FV_GUESS_MLP */
  int device;          /* CUDA device ordinal */
} fv_config;

typedef struct fv_mesh fv_mesh;

/* Fills *cfg with the defaults shown above (device 0). */
void fv_config_default(fv_config *cfg);

/*
 * Builds a mesh from host arrays (copied): node coordinates xyz[3*n_nodes]
 * (x,y,z per node), tets[4*n_tets] node indices (positively oriented:
 * det[x1-x0, x2-x0, x3-x0] > 0), face_bc[4*n_tets] where entry 4*t+j tags the
 * face of tet t opposite its local node j (FV_BC_*; interior faces 0).
 * Extracts faces, computes FP64 geometry (Sec. 2.1: the solver works on cells
 * and faces), renumbers cells along a Morton curve and uploads everything to
 * the device.  Synchronous.  Errors: FV_ERR_INVALID_ARG (NULL argument,
 * invalid configuration, or an empty mesh: n_tets or n_nodes <= 0, refused
 * before any device call), FV_ERR_BAD_MESH, FV_ERR_NOMEM, FV_ERR_CUDA.
 * *out is NULL on failure.
 */
int fv_mesh_load(const double *xyz, int64_t n_nodes, const int64_t *tets, int64_t n_tets,
                 const int8_t *face_bc, const fv_config *cfg, fv_mesh **out);

/* Releases every device and host resource of the mesh (NULL is a no-op).
 * Synchronises the device first. */
void fv_mesh_free(fv_mesh *m);

/* Number of cells / faces of the mesh. */
int64_t fv_mesh_cells(const fv_mesh *m);
int64_t fv_mesh_faces(const fv_mesh *m);

/*
 * Sets the state from primitives prim_soa[5*n_tets] = (rho, u, v, w, p),
 * caller's cell order; host memory (on_device = 0) or device memory
 * (on_device = 1).  Resets the cycle (levels must be reassigned), the
 * interface accumulators and the boundary flux ledger; keeps the time.
 * Errors: FV_ERR_INVALID_ARG, FV_ERR_CUDA.
 */
int fv_set_state(fv_mesh *m, const double *prim_soa, int on_device, void *stream);

/*
 * Writes the conserved state U^n = (rho, rho u, rho v, rho w, E) to
 * cons_soa[5*n_tets] in the caller's cell order, host (on_device = 0,
 * synchronous) or device (on_device = 1, asynchronous) memory.
 */
int fv_get_state(fv_mesh *m, double *cons_soa, int on_device, void *stream);

/*
 * Alg. 2 (time steps, then levels): computes every cell's local explicit time step
 * dt_i = 2 CFL V_i / sum_f A_f (|u_i . n_f| + c_i), dt_min = min_i dt_i, the
 * level k_i = max{k <= L-1 : 2^k dt_min <= dt_i}, then lowers levels until
 * neighbours differ by at most one (Sec. 2.2), and builds the level-sorted
 * cell and face lists.  Starts a cycle.  dt_min_out (may be NULL) receives
 * dt_min and level_counts_out[L] (may be NULL) the cells per level; either
 * non-NULL makes the call synchronous.  Errors: FV_ERR_INVALID_ARG (a cycle
 * is in progress), FV_ERR_CUDA.
 */
int fv_assign_levels(fv_mesh *m, double *dt_min_out, int32_t *level_counts_out, void *stream);

/* Local explicit time step dt_i of every cell (caller's order) computed by
 * the last level assignment (the time-step computation of Alg. 2): host dt_out[n_tets].  The
 * assignment evaluates dt_i in FP32 with a certified relative bound (at
 * most 2^-12, typically ~3e-6) and in FP64 wherever the minimum or a level
 * decision needs the exact value: those entries, dt_min and every level are
 * bit for bit the all-FP64 evaluation; the other entries are the FP32
 * estimates.  Synchronous.
 * Errors: FV_ERR_INVALID_ARG before any level assignment. */
int fv_get_local_dt(fv_mesh *m, double *dt_out);

/* The evolving level distribution (the paper follows it in Sec. 5: the
 * share of cells and of the cost C(tau) per level, iteration by iteration):
 * for the last n = min(cycles run since the state was set, 4096,
 * max_cycles) cycles, oldest first, counts_out[q*8 + k] = cells of level k
 * in cycle q (k < 8; 0 above the mesh's levels) and dtmin_out[q] = its
 * dt_min; *n_out = n.  Host arrays; synchronous. */
int fv_level_history(fv_mesh *m, int max_cycles, int32_t *counts_out, double *dtmin_out, int *n_out);

/* Level of every cell (caller's order) of the current cycle: host int8
 * array levels_out[n_tets].  Synchronous. */
int fv_get_levels(fv_mesh *m, int8_t *levels_out);

/*
 * The level-compacted lists of the current cycle (host, synchronous, any
 * pointer may be NULL): cells_out[n_tets] caller's cell indices sorted by
 * (level, no finer neighbour) with cell_off_out[2L+1] bucket offsets, and
 * face_level_out[n_faces] / face_off_out[L+1] the face level of every face
 * in library face order and the offsets of the face list sorted by level.
 * A phase of level tau touches a prefix or a contiguous segment of them.
 */
int fv_get_level_lists(fv_mesh *m, int64_t *cells_out, int32_t *cell_off_out,
                       int8_t *face_level_out, int32_t *face_off_out);

/*
 * The residual R_i = -(1/V_i) sum_f sigma_f F_f A_f (Eq. 1, S = 0) of every
 * cell of level `level`, with every cell's state taken at the start
 * (stage 1) or the end (stage 2) of that level's current step: U^n at the
 * step start, the predicted U* at its end, and linear interpolation in time
 * for neighbours on other levels.  Writes R_soa_dev[5*n_tets] (device
 * memory, caller's order); entries of other cells are 0.  Changes no state.
 * Errors: FV_ERR_INVALID_ARG when no cycle is active, when stage 2 is asked
 * before the level's predictor ran, or when some level's state is not
 * defined at that time (a finer level that has not reached it).
 */
int fv_residual_level(fv_mesh *m, int level, int stage, double *R_soa_dev, void *stream);

/*
 * Runs the next n_phases phases of the current cycle.  The phases of one
 * cycle in FV_ORDER_FINEST_FIRST, for s = 1..2^(L-1): B(s) starts levels
 * 0..tau(s) (the subiteration loop of Alg. 2: predictor fluxes on faces of
 * level <= tau, U* of those cells), then E(s,k) for k = 0,1,.. while
 * s mod 2^k == 0 (corrector fluxes on faces of level k, flux time integrals,
 * U^{n+1} of level-k cells): 3 * 2^(L-1) - 1 phases.  In FV_ORDER_PAPER
 * (fv_set_order): for s > 1 the commit of levels 0..tau(s), B(s), then the
 * correctors of tau' = tau(s) down to 0, and a final commit of every level:
 * 4 * 2^(L-1) - 1 phases.  Completing the last phase ends the cycle (time
 * advances by 2^(L-1) dt_min).  A pause/resume hook for phase-by-phase
 * checks.  Errors: FV_ERR_INVALID_ARG (no active cycle, or past its end).
 */
int fv_advance_phases(fv_mesh *m, int n_phases, void *stream);

/*
 * The order of the level steps inside a cycle (Alg. 2, Sec. 2.2).
 * FV_ORDER_FINEST_FIRST (the default): a level's corrector runs when its
 * step's end time is reached, finest level first, and a coarse cell takes
 * the finer side's accumulated integral on each face to a finer neighbour
 * at once.  FV_ORDER_PAPER: the order of Alg. 2's loops -- every level that
 * begins a step at subiteration s is predicted, then corrected coarsest
 * first at the end time of its step, before the finer levels advance: finer
 * neighbours enter its gradients extrapolated linearly in time, each face
 * to a finer neighbour enters with the provisional integral dt_k F1 A, and
 * when the level's next step begins (Alg. 2's "intensive correction"; Alg.
 * 3's extra subiteration for the last one) the provisional integrals are
 * replaced by the finer side's.  Both conserve mass, momentum and energy
 * exactly and coincide with one level.  FV_ORDER_PAPER needs 5 doubles per
 * cell more in the FP32-flux mode; batches, the persistent cycle and
 * fv_residual_level take FV_ORDER_FINEST_FIRST only (the persistent cycle
 * falls back to the graph path).  Between cycles only; drops a captured
 * graph.  Errors: FV_ERR_INVALID_ARG (bad order, inside a cycle or a batch),
 * FV_ERR_NOMEM.
 */
#define FV_ORDER_FINEST_FIRST 0
#define FV_ORDER_PAPER 1
int fv_set_order(fv_mesh *m, int order);
int fv_get_order(fv_mesh *m, int *order_out);

/*
 * Advances n_cycles complete cycles (Alg. 2), each starting with level
 * assignment; a cycle already in progress is completed first and counts as
 * one.  *t_out (may be NULL) receives the time reached; the call then
 * synchronises the stream.  Device-side errors (non-physical state, Riemann
 * failure) are sticky and reported by fv_status.
 */
int fv_advance(fv_mesh *m, int n_cycles, double *t_out, void *stream);

/* Physical time of the mesh (synchronous). */
int fv_get_time(fv_mesh *m, double *t_out);

/* Sets the physical time (only between cycles). */
int fv_set_time(fv_mesh *m, double t);

/*
 * Sum over boundary faces of the time-integrated flux that left the domain
 * since the last fv_set_state, out5[5] (host, synchronous).  With
 * sum_i V_i U_i this gives the conservation ledger.
 */
int fv_boundary_ledger(fv_mesh *m, double *out5);

/* Cell volumes in the caller's order, host vol_out[n_tets] (synchronous). */
int fv_cell_volumes(fv_mesh *m, double *vol_out);

/*
 * Sticky device status of the mesh (synchronous): FV_OK, or the first of
 * FV_ERR_NONPHYSICAL / FV_ERR_RIEMANN raised by a kernel since the last
 * fv_set_state.
 */
int fv_status(fv_mesh *m);

/*
 * Sets the conserved state U = (rho, rho u, rho v, rho w, E) from
 * cons_soa[5*n_tets] (caller's order), host (on_device = 0, synchronous) or
 * device (on_device = 1) memory.  Same resets as fv_set_state.
 */
int fv_set_conserved(fv_mesh *m, const double *cons_soa, int on_device, void *stream);

/*
 * Work counters since the last fv_set_state/fv_set_conserved (synchronous):
 * completed cycles, cell updates weighted as in the cost model of Sec. 2.2
 * (sum over cycles of sum_k 2^(L-1-k) |Omega_k|) and face flux evaluations
 * (predictor + corrector: sum over cycles of sum_k 2 * 2^(L-1-k) |faces of
 * level k|).  Any pointer may be NULL.
 */
int fv_work_counters(fv_mesh *m, int64_t *cycles, int64_t *cell_updates, int64_t *face_evals);

/*
 * Whether fv_advance replays a captured CUDA graph of one whole cycle
 * (default 1).  The graph is captured on the first fv_advance that starts a
 * cycle on a non-legacy stream and replayed afterwards; the legacy default
 * stream always runs the kernels one by one.
 */
int fv_use_graph(fv_mesh *m, int enable);

/*
 * Grid sizes of the four phase kernels (primitives, gradients, fluxes,
 * updates) in blocks per SM (1..64; defaults 8, 8, 16, 8).  Results do not
 * depend on them; the autotuner in paper_1704_01144_gb300/autotune.py picks
 * them by timing and caches its choice.  Setting them drops a captured graph.
 */
int fv_set_launch(fv_mesh *m, const int32_t per_sm[4]);
int fv_get_launch(fv_mesh *m, int32_t per_sm[4]);

/*
 * Gradient-flux fusion for latency-bound phases (FP32-flux mode with the
 * two-rarefaction guess; other modes ignore it): a phase whose face list
 * has at most max_faces faces computes both cells' least-squares gradients
 * inside its flux kernel (a cell's gradient once per face of the cell)
 * rather than in a gradient kernel of its own -- one dependent launch and
 * one chain of gathers less, for more arithmetic per face.  The choice is
 * taken on the device for every phase from the face count of the current
 * level assignment, so a captured cycle follows the level distribution.
 * Both ways compute the same operations on the same values.  0 turns the
 * fusion off and is the default (FV_FUSE_FACES_DEFAULT): on a GB300 a
 * dependent launch in a CUDA graph costs about 2 us while the recomputed
 * gradients cost more, so fusion has measured slower for every threshold.
 * A nonzero threshold adds one launch per phase.  Setting it drops a
 * captured graph.  Errors: FV_ERR_INVALID_ARG (NULL argument, negative
 * count, inside a cycle or a batch).
 */
#define FV_FUSE_FACES_DEFAULT 0
int fv_set_fusion(fv_mesh *m, int64_t max_faces);
int fv_get_fusion(fv_mesh *m, int64_t *max_faces_out);

/*
 * FP32-flux mode: the arithmetic of the predictor's residual sum
 * (Alg. 2, "Extensive prediction": U* = U^n - (dt_k/V) sum sigma F1 A).
 * FV_SUM_FP64 widens each FP32 flux and forms the sum and U* in FP64 from the
 * FP64 U^n; FV_SUM_FP32 forms both in FP32 from the FP32 shadow of U^n.
 * Either way U* is then rounded to its FP32 record, which only ever feeds the
 * FP32 reconstruction of later fluxes; the corrector's sums, U^n and the flux
 * time integrals are FP64 in both.  The FP64 mode ignores the setting.
 * The default is FV_SUM_FP32: on a GB300 the FP64 sum costs 11 % of the
 * cycle on the 1M-tet blast and on the 80M-tet ground blast, and moves the
 * error against the FP64 reference by less than its own spread (9.1e-7
 * against 9.3e-7 after 3 cycles of the 1M-tet blast).
 * Setting it drops a captured graph.  Errors: FV_ERR_INVALID_ARG (NULL mesh,
 * unknown value, inside a cycle or a batch).
 */
#define FV_SUM_FP32 0
#define FV_SUM_FP64 1
#define FV_PREDICTOR_SUM_DEFAULT FV_SUM_FP32
int fv_set_predictor_sum(fv_mesh *m, int sum);
int fv_get_predictor_sum(fv_mesh *m, int *sum_out);

/*
 * FP32-flux mode with the two-rarefaction guess and no fusion: whether the
 * flux kernel stages the records it gathers (face geometry, both cells'
 * primitives and gradients) through shared memory with asynchronous copies,
 * those of the next face in flight while the current face's Riemann problem
 * is solved (1), or loads them into registers when it reaches each face
 * (0).  Both compute the same operations on the same values (bitwise equal
 * results).  Other modes ignore the setting.  Setting it drops a captured
 * graph.  Errors: FV_ERR_INVALID_ARG (NULL argument, inside a cycle or a
 * batch).
 */
#define FV_FLUX_STAGING_DEFAULT 0
int fv_set_flux_staging(fv_mesh *m, int enable);
int fv_get_flux_staging(fv_mesh *m, int *enabled_out);

/*
 * The per-cell gather of the update kernels (Alg. 2, "Flow sum on cells"):
 * FV_GATHER_THREAD, one thread per cell reads its four faces' values and
 * adds them in face order; FV_GATHER_QUAD, four lanes per cell each read one
 * face's value and the first lane adds them in the same order (a warp-level
 * gather; bitwise the same results).  Both are deterministic and use no
 * atomics.  The paper's order, the FP64 predictor sum, batches and the
 * persistent cycle use the per-thread gather.  Setting it drops a captured
 * graph.  Errors: FV_ERR_INVALID_ARG
 * (NULL argument, unknown value, inside a cycle or a batch).
 */
#define FV_GATHER_THREAD 0
#define FV_GATHER_QUAD 1
#define FV_GATHER_DEFAULT FV_GATHER_THREAD
int fv_set_gather(fv_mesh *m, int gather);
int fv_get_gather(fv_mesh *m, int *gather_out);

/* kernel classes of the profiler */
#define FV_PROF_LEVELS 0 /* level assignment: dt, levels, sorts */
#define FV_PROF_PRIM 1   /* primitives at the phase time */
#define FV_PROF_GRAD 2   /* least-squares gradients */
#define FV_PROF_FLUX 3   /* reconstruction + Riemann flux */
#define FV_PROF_UPDATE 4 /* per-cell gather and update */
#define FV_PROF_N 5

/*
 * Per-kernel-class timing with CUDA events recorded on the launching stream
 * around every launch (graphs are bypassed while enabled).  Enabling clears
 * the totals.  fv_profile_read synchronises and returns, per class, the
 * summed kernel time in ms and the number of launches.
 */
int fv_profile_enable(fv_mesh *m, int enable);
int fv_profile_read(fv_mesh *m, double ms_out[FV_PROF_N], int64_t launches_out[FV_PROF_N]);

/*
 * Batches: many meshes of uneven sizes and level counts advanced together.
 * Each mesh keeps its own schedule (Alg. 2 with its own L, dt_min and
 * levels); a batch cycle lasts 2^(Lmax-1) batch subiterations, during which a
 * mesh with L levels completes 2^(Lmax-L) of its own cycles.  Every kernel
 * launch covers all meshes (one per kernel kind and phase; level assignment
 * batched over the meshes starting a cycle), and on a non-legacy stream the
 * whole batch cycle is captured once and replayed as one CUDA graph.
 * Results are bitwise those of each mesh advanced on its own.
 *
 * fv_batch_create: 1..64 distinct meshes sharing device, precision, gamma
 * and Newton settings; the batch references (does not own) them and their
 * states must be set.  fv_batch_advance: n_cycles batch cycles, asynchronous
 * on `stream`; a mesh inside a cycle of its own is FV_ERR_INVALID_ARG.
 * fv_batch_info: subiterations per batch cycle and kernels per batch cycle.
 */
typedef struct fv_batch fv_batch;
int fv_batch_create(fv_mesh *const *meshes, int n, fv_batch **out);
int fv_batch_advance(fv_batch *b, int n_cycles, void *stream);
int fv_batch_info(fv_batch *b, int *subiterations, int *kernel_launches);
int fv_batch_use_graph(fv_batch *b, int enable);
/* grid sizes of a batch's phase kernels, as fv_set_launch */
int fv_batch_set_launch(fv_batch *b, const int32_t per_sm[4]);
int fv_batch_get_launch(fv_batch *b, int32_t per_sm[4]);
void fv_batch_free(fv_batch *b);

/*
 * The device Godunov flux (Sec. 2.1) on a batch of face states, for tests
 * and data harvesting: for i < count, with primitives WL_dev/WR_dev
 * [5*count] = (rho, u, v, w, p) and unit normals n_dev[3*count]
 * (structure of arrays), writes the flux per unit area F_dev[5*count] and
 * the Newton iterations iters_dev[count] (-1 where the solver failed; 0
 * where no Riemann problem is solved: a transmissive boundary).
 * bc = FV_BC_INTERIOR: exact Riemann problem between WL and WR;
 * FV_BC_WALL / FV_BC_TRANSMISSIVE: boundary flux of WL (WR unused).
 * Arithmetic follows cfg->precision; gamma, newton_tol and newton_max_iter
 * come from cfg.  Device pointers; asynchronous on `stream`.  count = 0 is a
 * no-op (FV_OK; no pointer is read).  Errors: FV_ERR_INVALID_ARG (NULL
 * pointer, count < 0 or > 2^31 - 1, unknown bc or precision, bad gas or
 * Newton settings), FV_ERR_CUDA.
 */
int fv_godunov_flux_batch(const double *WL_dev, const double *WR_dev, const double *n_dev,
                          int64_t count, const fv_config *cfg, int bc, double *F_dev,
                          int32_t *iters_dev, void *stream);

/*
 * Measured fused-multiply-add ceiling of the device in TFLOP/s (2 flops per
 * FMA): precision FV_FP64 or FV_FP32_FLUX (FP32).  Runs a timed probe
 * kernel (well under a second); synchronous.  The denominator of the
 * roofline of ALU-bound kernels.
 */
int fv_probe_fma_peak(int device, int precision, double *tflops_out);

/* ---------------------------------------------------------------------
 * Sharded runs (Sec. 3.3 and Sec. 4.3: a spatial domain decomposition in
 * which every cell belongs to one subdomain, ghost cells copy the
 * neighbouring subdomains' border cells, border faces are computed on both
 * sides, and cells are weighted by their temporal level for the
 * partition).  A subdomain is an fv_mesh of its own cells plus ghost layers;
 * the caller drives its cycles phase by phase and moves the packed ghost
 * records between subdomains (a device copy, NCCL or host staging).  The
 * partition, the ghost layers and the driver are in the Python package
 * (shard.py).
 *
 * The level assignment of Alg. 2 in three calls, so that a sharded run can
 * take the minimum local step over all subdomains and give its ghost cells
 * their owners' levels before the lists are sorted:
 *  fv_levels_local_dt: the local steps and this mesh's minimum (synchronous,
 *    written to *dt_min_out);
 *  fv_levels_classify: the levels from dt_min (the global minimum): the
 *    classification and the L-1 smoothing sweeps;
 *  fv_levels_sort: the level-sorted lists; starts a cycle, as
 *    fv_assign_levels does (fv_advance_phases runs its phases).
 * fv_levels_local_dt, fv_levels_classify(its result), fv_levels_sort is
 * fv_assign_levels.  Errors: FV_ERR_INVALID_ARG (NULL argument, out of
 * order, dt_min not positive and finite, inside a cycle), FV_ERR_CUDA.
 * ------------------------------------------------------------------- */
int fv_levels_local_dt(fv_mesh *m, double *dt_min_out, void *stream);
int fv_levels_classify(fv_mesh *m, double dt_min, void *stream);
int fv_levels_sort(fv_mesh *m, void *stream);

/*
 * A halo plan: n cells of mesh m, given in the caller's order of its tets
 * (the order fv_set_state uses), whose records fv_halo_pack writes into a
 * device buffer and fv_halo_unpack reads back from one, record k for
 * cells[k].  what = FV_HALO_LEVELS: one int8 level per cell (n bytes);
 * FV_HALO_STATE: FV_HALO_STATE_DOUBLES doubles per cell (U^n and the
 * predicted state of the mode, bit copies).  Buffers are device memory
 * owned by the caller; asynchronous on `stream`.  The plan copies `cells`
 * (host memory) and keeps a device copy; fv_halo_free releases it (before
 * its mesh).  Errors: FV_ERR_INVALID_ARG (NULL argument, a cell outside the
 * mesh, unknown `what`, unpacking into a mesh inside a batch), FV_ERR_NOMEM,
 * FV_ERR_CUDA.
 */
typedef struct fv_halo fv_halo;
#define FV_HALO_LEVELS 1
#define FV_HALO_STATE 2
#define FV_HALO_STATE_DOUBLES 20
int fv_halo_create(fv_mesh *m, const int64_t *cells, int64_t n, fv_halo **out);
int fv_halo_pack(fv_halo *h, int what, void *buf_dev, void *stream);
int fv_halo_unpack(fv_halo *h, int what, const void *buf_dev, void *stream);
int64_t fv_halo_size(fv_halo *h); /* n, or -1 for a NULL plan */
void fv_halo_free(fv_halo *h);

/* Largest n_cells fv_assign_levels_noalloc accepts (its static scratch). */
#define FV_NOALLOC_MAX_CELLS (1 << 22)

/*
 * Level assignment that allocates nothing, for callers that cannot call
 * cudaMalloc when they need it: a host application that gives the library
 * only memory from its own fixed-budget pool and accounts for every byte of
 * it, or one running under an allocator that must see every device
 * allocation.  The paper has no counterpart of this entry point.
 *
 * Same result as the level part of fv_assign_levels, on caller-owned device
 * arrays: dt_min = min_i dt_dev[i]; k_i = max{k <= max_levels-1 :
 * 2^k dt_min <= dt_i}; then max_levels-1 sweeps of
 * k_i <- min(k_i, 1 + min_j k_nbr(i,j)).  Inputs: dt_dev[n_cells] positive
 * finite local time steps (nothing checks this on the device: a zero,
 * negative, infinite or NaN entry gives undefined levels and dt_min);
 * nbr_dev[4*n_cells] with nbr_dev[j*n_cells + i]
 * the neighbour of cell i across its face j (any negative value: boundary).
 * Outputs: levels_dev[n_cells] and *dt_min_dev.  All four pointers are
 * device memory owned by the caller.  Asynchronous on `stream`.
 *
 * Scratch: one static device array of 256 + FV_NOALLOC_MAX_CELLS bytes that
 * every GPU which loads this library holds until the process exits.  The
 * first call on a device looks up that array's device address (with the
 * device current) and caches it for the life of the process, so make that
 * first call before any stream capture, and do not call it after a
 * cudaDeviceReset.  All calls share the array and each re-initialises what
 * it uses; calls that overlap on the GPU (other streams or threads on the
 * same device) race on it.
 * Errors: FV_ERR_INVALID_ARG for a NULL pointer, n_cells outside
 * [1, FV_NOALLOC_MAX_CELLS], max_levels outside [1, 8] or a current device
 * numbered 64 or above; FV_ERR_CUDA.
 */
int fv_assign_levels_noalloc(const double *dt_dev, const int32_t *nbr_dev, int64_t n_cells,
                             int max_levels, int8_t *levels_dev, double *dt_min_dev,
                             void *stream);

/* ---------------------------------------------------------------------
 * Learned starting guess of the exact Riemann solver's Newton iteration.
 * Sec. 2.1 computes face fluxes from the exact Riemann problem; the paper
 * has no learned component, so the network and its inputs are readings:
 * a 6 -> 64 -> 64 -> 1 perceptron with tanh-form GELU activations whose
 * inputs are the face-frame primitives normalised by the pair's mean state,
 * x = ((rL-rb)/rb, (uL-ub)/ab, (pL-pb)/pb, (rR-rb)/rb, (uR-ub)/ab, (pR-pb)/pb)
 * (u: normal velocities; rb, ub, pb: means; ab = sqrt(gamma pb / rb)), and
 * whose output is y = log(p* / pb) (FV_MLP_TARGET_PBAR) or
 * y = log(p* / p_TR) / s(q) (FV_MLP_TARGET_TR), with p_TR the two-rarefaction
 * guess, q = p_TR / min(pL, pR) - 1 and s(q) = (q / (1 + q))^3 for q > 0
 * (0 otherwise: the two-rarefaction guess is then exact).
 * Newton keeps its stopping rule (newton_tol), so the converged flux does
 * not depend on the guess beyond that tolerance; a non-finite or
 * non-positive guess falls back to the two-rarefaction guess.
 * Parameters (FP32, FV_MLP_PARAMS values, rows = output units):
 * W1[64][6], b1[64], W2[64][64], b2[64], w3[64], b3.
 * ------------------------------------------------------------------- */
#define FV_MLP_PARAMS 4673
#define FV_MLP_PACKED_BYTES 10240 /* bfloat16 weight fragments + FP32 biases */
#define FV_MLP_TARGET_PBAR 0
#define FV_MLP_TARGET_TR 1

typedef struct fv_train_config {
  int epochs;     /* passes over the selected samples */
  int batch;      /* samples per Adam step (1 .. 2^20) */
  double lr0;     /* learning rate of the first step ... */
  double lr1;     /* ... decayed along a half cosine to this one */
  double beta1;   /* Adam moment decay rates and epsilon (0.9, 0.999, 1e-8) */
  double beta2;
  double eps;
  uint64_t seed;  /* shuffle seed (splitmix64 stream) */
} fv_train_config;

/* Glorot-uniform weights, zero biases, from a splitmix64 stream seeded by
 * `seed`, into host memory params[FV_MLP_PARAMS]. */
int fv_mlp_init(float *params, int n_params, uint64_t seed);

/* Packs device FP32 parameters into the fused kernels' layout (bfloat16
 * B-fragments of W1 and W2, FP32 biases and output weights, the target
 * mode, the gate) in packed_dev (FV_MLP_PACKED_BYTES, 16-byte aligned,
 * caller-owned).  gate: a face takes the learned guess only where the
 * two-rarefaction estimate shows a shock, q = p_TR / min(pL, pR) - 1 > gate
 * (that estimate is exact for two rarefactions and third-order accurate for
 * weak shocks); a negative gate consults the network on every face.  A warp
 * evaluates the network when any of its faces passes the gate.
 * Asynchronous on `stream`. */
int fv_mlp_pack(const float *params_dev, int n_params, int target, double gate, void *packed_dev,
                void *stream);

/* The bfloat16 tensor-core inference the flux kernel fuses, on its own:
 * y_dev[i] = network(x_dev[6*i .. 6*i+5]) for i < count.  Device pointers;
 * asynchronous. */
int fv_mlp_infer(const void *packed_dev, const float *x_dev, int64_t count, float *y_dev, void *stream);

/* The same inference with CUDA's tanhf in the activations instead of the
 * hardware tanh approximation the flux kernel uses: a check that separates
 * the approximation's error from the bfloat16 quantisation (the flux kernels
 * never call it).  Arguments and errors as fv_mlp_infer. */
int fv_mlp_infer_exact_tanh(const void *packed_dev, const float *x_dev, int64_t count, float *y_dev,
                            void *stream);

/* Training data from harvested pairs pairs_dev[6*count] = (rL, uL, pL, rR,
 * uR, pR) in the face frame: the exact star pressure pstar_dev[count] (FP64
 * Newton to a relative change of 1e-14), the features x_dev[6*count], the
 * targets y_dev[count] (FP32) and, if q_dev is not NULL, the shock strength
 * of the two-rarefaction estimate q_dev[count] (see fv_mlp_pack's gate).
 * Synchronous.  FV_ERR_RIEMANN if a pair has no star state (its entries are
 * NaN). */
int fv_mlp_label(const double *pairs_dev, int64_t count, double gamma, int target, float *x_dev,
                 float *y_dev, double *pstar_dev, float *q_dev, void *stream);

/* Mean squared loss over samples sel_dev[0..count-1] (NULL: 0..count-1) and
 * its gradient grad_dev[FV_MLP_PARAMS] (NULL: loss only), by the FP32
 * training kernels; sums in a fixed order.  Synchronous. */
int fv_mlp_loss_grad(const float *params_dev, const float *x_dev, const float *y_dev,
                     const int32_t *sel_dev, int64_t count, float *grad_dev, double *loss_out,
                     void *stream);

/* One Adam step (step = 1, 2, ...) on device arrays params, m, v (FP32,
 * FV_MLP_PARAMS each) from grad_dev.  Asynchronous. */
int fv_mlp_adam(float *params_dev, float *m_dev, float *v_dev, const float *grad_dev, int step,
                double lr, double beta1, double beta2, double eps, void *stream);

/* Trains params_dev in place: tc->epochs passes over the samples listed in
 * sel_host[n_sel] (host; NULL: 0..n_sel-1), each pass in a fresh
 * Fisher-Yates order, one Adam step per minibatch of tc->batch samples.
 * loss_hist_dev (NULL or fv_mlp_train_steps() floats) receives each step's
 * minibatch loss.  Deterministic for a given seed.  Synchronous. */
int fv_mlp_train(float *params_dev, const float *x_dev, const float *y_dev, const int32_t *sel_host,
                 int64_t n_sel, const fv_train_config *tc, float *loss_hist_dev, void *stream);
int fv_mlp_train_steps(const fv_train_config *tc, int64_t n_sel);

/* Installs the network in the mesh (packed into mesh-owned device memory,
 * with target and gate as in fv_mlp_pack) and selects FV_GUESS_MLP: the
 * flux kernel then evaluates it on the tensor cores for the faces the gate
 * passes and starts Newton from its guess there.  Synchronous.  Not
 * inside a cycle; batches (fv_batch_create) take only meshes with the
 * two-rarefaction guess and get their network from fv_batch_mlp_load. */
int fv_mlp_load(fv_mesh *m, const float *params_dev, int n_params, int target, double gate);

/* FV_GUESS_TWO_RAREFACTION, or FV_GUESS_MLP after fv_mlp_load. */
int fv_set_guess(fv_mesh *m, int guess);

/* The same for a batch: one network (packed into batch-owned memory) for
 * every instance, evaluated in the batched flux kernel; results equal each
 * mesh advanced alone with the same network.  Synchronous. */
int fv_batch_mlp_load(fv_batch *b, const float *params_dev, int n_params, int target, double gate);
int fv_batch_set_guess(fv_batch *b, int guess);

/* Riemann pairs of the mesh's current state U^n (the reconstructed face
 * states the flux kernel sees, in its precision): pair j of face
 * (a j + b) mod F, with a coprime to F and a, b drawn from `seed`, so a call
 * repeats no face; written as pairs_dev[6*j ..] = (rL, uL, pL, rR, uR, pR)
 * in the face frame (a wall face: its mirrored problem).  count <= faces.
 * Asynchronous on `stream`; not inside a cycle. */
int fv_harvest_pairs(fv_mesh *m, double *pairs_dev, int64_t count, uint64_t seed, void *stream);

/* fv_godunov_flux_batch for interior faces with the learned guess of the
 * packed network (fv_mlp_pack); iters_dev shows what the guess saves. */
int fv_godunov_flux_batch_mlp(const double *WL_dev, const double *WR_dev, const double *n_dev,
                              int64_t count, const fv_config *cfg, const void *packed_dev,
                              double *F_dev, int32_t *iters_dev, void *stream);

/*
 * Runs each whole cycle of fv_advance as one cooperative (persistent)
 * launch: after the level assignment, every phase of Alg. 2's cycle runs in
 * a single kernel whose blocks stay resident and separate the kernel kinds
 * of each phase (primitives, gradients, fluxes, updates) by a grid barrier,
 * instead of four launches per phase.  Results are bitwise those of the
 * per-kernel path.  The barrier waits a bounded time; if it gives up, the
 * cycle stops and fv_status reports FV_ERR_TIMEOUT.  Applies to the
 * two-rarefaction guess and unprofiled runs (others use the per-kernel
 * path).  Not inside a cycle.
 */
int fv_use_persistent(fv_mesh *m, int enable);

/* Failure detection of the persistent cycle's grid barrier: `rounds`
 * barriers over one block per SM; with `unreachable` nonzero each barrier
 * waits for one block more than exists, so every wait runs out (about a
 * second at most) and the kernel returns.  *status_out gets the device
 * status bits (4 = a barrier timed out).  Returns FV_OK, FV_ERR_TIMEOUT or
 * FV_ERR_CUDA.  Synchronous. */
int fv_barrier_selftest(int device, int rounds, int unreachable, int *status_out);

/* Message of the calling thread's last failed call ("" if none). */
const char *fv_last_error(void);

/* Library version string. */
const char *fv_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FV_H */
