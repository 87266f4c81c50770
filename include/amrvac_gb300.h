/*
 * amrvac_gb300 -- C ABI of the GB300 (sm_103a) implementation of the
 * MPI-AMRVAC hot path (Keppens, Teunissen, Xia, Porth, arXiv:2004.03275):
 * the conservative finite-volume Euler update on a block quadtree/octree and
 * the geometric-multigrid implicit diffusion step of the reaction-diffusion
 * module.
 *
 * Conventions for every call:
 *  - returns an int status: AMR_OK (0) or a negative amr_status; no exception
 *    or abort crosses the boundary; amr_last_error / mg_last_error give text.
 *  - handles own all device memory they allocate; the caller owns host
 *    buffers, device buffers it passes in, and the CUDA stream.
 *  - state arrays that cross the boundary are float64, layout
 *    [leaf][variable][cell] with leaves in Morton order and cells ordered
 *    i fastest, then j, then k (i + nx*(j + nx*k)).
 *  - `on_device` = 1 means the pointer is device memory readable/writable by
 *    the handle's stream; 0 means host memory (pageable or pinned).
 *  - calls on one handle are not thread safe; different handles are independent.
 */
#ifndef AMRVAC_GB300_H
#define AMRVAC_GB300_H
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  AMR_OK = 0,
  AMR_ERR_INVALID_ARG = -1,   /* bad config or argument; nothing was changed */
  AMR_ERR_OOM = -2,           /* device or host allocation failed */
  AMR_ERR_CUDA = -3,          /* a CUDA runtime call failed (text in last_error) */
  AMR_ERR_NONPHYSICAL = -4,   /* rho <= 0 or p <= 0 (or NaN) met on the device */
  AMR_ERR_TIMEOUT = -5,       /* a bounded device wait gave up */
  MG_ERR_NOT_CONVERGED = -6,  /* multigrid hit max_cycles before rtol */
  AMR_ERR_CAPACITY = -7,      /* the tree would exceed max_blocks */
  AMR_ERR_UNBALANCED = -8     /* a given leaf set is not a 2:1 balanced cover */
} amr_status;

enum { AMR_FLUX_TVDLF = 0, AMR_FLUX_HLL = 1, AMR_FLUX_HLLC = 2 };
enum { AMR_LIM_MINMOD = 0, AMR_LIM_VANLEER = 1, AMR_LIM_KOREN = 2, AMR_LIM_NONE = 3, AMR_LIM_MC = 4,
       AMR_LIM_CADA = 5 };
enum { AMR_SSPRK2 = 2, AMR_SSPRK3 = 3 };
enum { AMR_BC_PERIODIC = 0, AMR_BC_OUTFLOW = 1 };
enum { AMR_FP64 = 0, AMR_FP32 = 1 };
enum { AMR_NB_BOUNDARY = -1 };
enum { MG_BC_PERIODIC = 0, MG_BC_NEUMANN = 1 };
enum { RD_GRAY_SCOTT = 0, RD_SCHNAKENBERG = 1 };
enum { RD_IMEX = 0, RD_SPLIT = 1, RD_EXPLICIT = 2 };

/* ------------------------------------------------------------------------
 * Block-tree finite-volume Euler solver.
 *
 * Problem (Sec. 1.1, Eq. (eq) with S = 0): dU/dt + div F(U) = 0 for the HD
 * variables U = (rho, rho v, E), E = rho v^2/2 + p/(gamma-1), primitive
 * V = (rho, v, p).  Fluxes: TVDLF (local Lax-Friedrichs) and HLL from the
 * signal-speed bounds (Sec. 1.2, phys_get_cmax / phys_get_cbounds), HLLC
 * (Sec. 2.4); limited MUSCL reconstruction of V with minmod / van Leer / Koren
 * (Koren: Sec. 2.3.1); SSP Runge-Kutta in two or three stages (Sec. 2.3.2,
 * 2.4); CFL time step dt = cfl / max_cells sum_d (|v_d| + c)/dx_d (Sec. 1.2).
 * Grid (Sec. 1.3): blocks of block_nx^ndim cells, base_nblocks blocks per
 * dimension on level 1, refinement ratio 2 up to max_level, Lohner-type
 * estimator of weighted second derivatives; refine if one cell exceeds
 * refine_tol, coarsen if all cells of all siblings are below
 * coarsen_frac*refine_tol; 2:1 balance across faces, edges and corners.
 * ------------------------------------------------------------------------ */
typedef struct amr_handle amr_handle;

typedef struct {
  int ndim;             /* 1, 2 or 3 */
  int block_nx;         /* cells per block side: 8 or 16 (block_nx1.. of Sec. 1.3) */
  int base_nblocks[3];  /* blocks per dimension on level 1 (domain_nx / block_nx) */
  int max_level;        /* refine_max_level; 1 = uniform block grid */
  double xmin[3], xmax[3];  /* xprobmin / xprobmax */
  double gamma;
  int flux;             /* AMR_FLUX_* */
  int limiter;          /* AMR_LIM_* */
  int rk;               /* AMR_SSPRK2 or AMR_SSPRK3 */
  double cfl;
  int bc[3][2];         /* [dim][low, high]: AMR_BC_PERIODIC (both sides) or AMR_BC_OUTFLOW */
  int precision;        /* AMR_FP64 (plain) or AMR_FP32 (state, reconstruction, fluxes in float;
                           conserved totals in float64) */
  double refine_tol;    /* estimator threshold for refinement */
  double coarsen_frac;  /* coarsen below coarsen_frac * refine_tol */
  double wavefilter;    /* estimator filter epsilon (0.01 typical) */
  unsigned refine_var_mask; /* primitive variables used by the estimator: bit 0 rho,
                               bits 1..ndim velocity, bit ndim+1 p */
  long long max_blocks; /* leaf capacity; a regrid that would exceed it fails with
                           AMR_ERR_CAPACITY and leaves the tree unchanged */
  void* stream;         /* cudaStream_t owned by the caller; NULL = legacy default stream */
} amr_config;

/* Creates the level-1 block grid (base_nblocks), state zero, t = 0.
 * Errors: AMR_ERR_INVALID_ARG (unsupported ndim/block_nx/limits), AMR_ERR_OOM, AMR_ERR_CUDA. */
int amr_create(const amr_config* cfg, amr_handle** out);
int amr_destroy(amr_handle* h);
const char* amr_last_error(const amr_handle* h);

/* Number of leaves and their level / block coordinates (Morton order).
 * coords has 3 ints per leaf; unused dimensions are 0.  cap = leaves the
 * arrays can hold; AMR_ERR_INVALID_ARG if cap < number of leaves. */
int amr_num_leaves(const amr_handle* h, long long* n);
int amr_leaf_info(const amr_handle* h, int* level, int* coords, long long cap);

/* Replaces the tree by the given leaves (any order; stored in Morton order).
 * The leaves must cover the domain and be 2:1 balanced, else
 * AMR_ERR_UNBALANCED and nothing changes.  State becomes zero. */
int amr_set_leaves(amr_handle* h, long long n, const int* level, const int* coords);

/* Sets the state of every leaf from a float64 array [leaf][var][cell]
 * (n_values = leaves * (ndim+2) * block_nx^ndim).  primitive = 1: the values
 * are (rho, v_1..v_ndim, p) and are converted on the device (Sec. 1.1,
 * phys_to_conserved); 0: conserved (rho, m_1..m_ndim, E).  Recomputes the
 * CFL step.  Synchronous.  A host array in page-locked (pinned) memory is read
 * in place by the conversion kernel (zero copy); pageable host memory is staged
 * through a device buffer. */
int amr_set_state(amr_handle* h, const double* W, long long n_values, int on_device, int primitive);

/* Initial condition from a host callback: prim_at(x, V, user) writes the primitive state
 * V = (rho, v_1..v_ndim, p) at the cell centre x[3] (unused dimensions 0).  The current tree
 * is sampled, then regridded (amr_regrid, the handle's estimator and thresholds) and resampled
 * max_level - 1 times, so that the initial tree resolves the callback's features (Sec. 1.3);
 * the state is the last sampling.  Synchronous; errors of amr_regrid / amr_set_state. */
typedef void (*amr_prim_fn)(const double x[3], double* V, void* user);
int amr_set_state_fn(amr_handle* h, amr_prim_fn prim_at, void* user);

/* Copies the conserved state to a float64 array [leaf][var][cell] (converted
 * on the device for the FP32 path).  cap_values = capacity in doubles.
 * Synchronous.  A pinned host array is written in place by the conversion
 * kernel; pageable host memory is staged through a device buffer. */
int amr_read_state(amr_handle* h, double* U, long long cap_values, int on_device);

/* Sets the simulation time t (a one-thread control kernel on the handle's stream,
 * which also refreshes the float copy of the next step's dt).  Synchronous. */
int amr_set_time(amr_handle* h, double t);

/* One SSPRK step with dt = min(cfl-step, t_end - t).  Synchronous; returns the
 * dt taken (0 if t >= t_end) and the new time.  AMR_ERR_NONPHYSICAL if a
 * non-positive density or pressure was met. */
int amr_step(amr_handle* h, double t_end, double* dt_taken, double* t_now);

/* nsteps SSPRK steps queued on the handle's stream as CUDA-graph launches
 * (steps after t_end are no-ops on the device).  Asynchronous: call amr_sync
 * to wait and to collect the status. */
int amr_run(amr_handle* h, int nsteps, double t_end);
int amr_sync(amr_handle* h, double* t_now, double* dt_last);

/* Refinement estimator (max over each leaf's cells), computed on the device,
 * copied to err[leaf]; cap = capacity.  Synchronous. */
int amr_estimate(amr_handle* h, double* err, long long cap);

/* Estimator -> flags -> refine / coarsen with 2:1 balance -> new leaves filled
 * by limited prolongation (new children) or restriction (new parents).
 * Synchronous.  Errors: AMR_ERR_CAPACITY (tree unchanged). */
int amr_regrid(amr_handle* h);

/* FP64 sum over leaves and cells of U dV, per conserved variable, as of the
 * last step (or set_state / regrid).  totals has ndim+2 entries. */
int amr_conserved_totals(amr_handle* h, double* totals);

/* Face-neighbour table, for checks: for leaf i and face f = 2*d + side,
 * kind[i*2*ndim + f] = 0 same level, 1 coarser, 2 finer, -1 domain boundary
 * (outflow); nbr[...] = leaf index of the same-level or coarser neighbour, or
 * of the first finer neighbour (tangential offset 0), -1 at a boundary.
 * cap = entries the arrays can hold (leaves * 2 * ndim). */
int amr_face_neighbors(const amr_handle* h, int* kind, int* nbr, long long cap);

/* Face ghost values of one leaf after the device ghost fill, float64
 * [var][face][layer 0..1][tangential cell]; for checks.  Synchronous. */
int amr_face_ghosts(amr_handle* h, long long leaf, double* out, long long cap);

/* One step like amr_step, launched kernel by kernel (no graph) with a CUDA
 * event recorded on the handle's stream after every kernel: ms[i] = duration
 * of kernel i, kind[i] = 0 stage update, 1 ghost fill, 2 reflux, 3 reduction.
 * cap = capacity of ms / kind; *nkernels = kernels of the step.  Synchronous.
 * For measurement only (the events add a little launch overhead). */
int amr_profile_step(amr_handle* h, double t_end, float* ms, int* kind, int cap, int* nkernels);

/* Launch shapes of the float32 2D stage kernel for 16^2 leaves (the project's stage-kernel
 * tuner; the paper has no counterpart).  Per stage kind k (0 first, 1 middle, 2 last with the
 * CFL and totals reductions): choice[2k] = warps (= leaves) per CTA (2, 4 or 8; 4 for the
 * last stage), choice[2k+1] = 1 for a grid of resident CTAs looping over the leaf groups,
 * 0 for one CTA per group.  Before the first captured step of a float32 2D 16^2 handle on a
 * uniform grid with SSPRK3, a tuner times every candidate on the handle's state (5 launches
 * after a warm-up, CUDA events; neither the state nor the time advances) and keeps the
 * fastest per kind; every candidate computes the same state bit for bit.
 * amr_march_tuning: the current choice (host int[6]) and, when tuned, the chosen launch's
 * time per kind in microseconds (host float[3] or NULL; 0 where not measured).
 * amr_set_march_tuning: use `choice` (host int[6]) and skip the tuner; invalid values give
 * AMR_ERR_INVALID_ARG and leave the choice unchanged. */
int amr_march_tuning(amr_handle* h, int* choice, float* us);
int amr_set_march_tuning(amr_handle* h, const int* choice);

/* Device launch counters: kernels launched by this handle since creation. */
int amr_kernel_launches(const amr_handle* h, long long* n);

/* ------------------------------------------------------------------------
 * CFL step and conserved totals without any device allocation.
 *
 * The paper has no counterpart: this is a service for callers that cannot
 * allocate device memory themselves -- code that runs under a fixed memory
 * budget owned by a pool allocator of an enclosing framework (which hands out
 * its buffers and forbids cudaMalloc beside it), or latency-critical loops
 * that cannot afford cudaMalloc's implicit device synchronisation.
 *
 * Computes, for a uniform block grid (every leaf on level 1, leaves in Morton
 * order as amr_leaf_info reports them for a fresh handle), the same two
 * results that amr_set_state leaves behind: dt_cfl = cfl / max over cells of
 * sum_d (|v_d| + c)/dx_d and totals[v] = sum of U dV (float64).
 *  - cfg: geometry and gamma/cfl as for amr_create (precision, flux, limiter,
 *    rk, refinement fields and max_blocks are ignored); cfg->stream is used.
 *  - U: device pointer, float64 conserved state [leaf][var][cell],
 *    nleaves = product of cfg->base_nblocks.  Not modified.
 *  - dt_cfl (host, 1 double), totals (host, ndim+2 doubles): outputs.
 * Errors: AMR_ERR_INVALID_ARG (bad config or nleaves not matching the grid),
 * AMR_ERR_CAPACITY if nleaves > AMR_NOALLOC_MAX_LEAVES, AMR_ERR_NONPHYSICAL
 * (outputs still written), AMR_ERR_CUDA.
 * Memory: the scratch is one fixed array of about 0.7 MB in the library's
 * device image, present on every GPU that loads the library until exit; no
 * call allocates.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress); make that first call before any stream
 * capture.  Every call on a device shares the array and keeps the previous
 * call's contents (the call resets what must start at zero): calls that
 * overlap on the GPU (different streams or threads) race.  The looked-up
 * address is kept for the life of the process, so the call must not be used
 * across a device reset (cudaDeviceReset) of that device.
 * Synchronous: the call waits for cfg->stream and reads its results back
 * into the host outputs before it returns.
 * ------------------------------------------------------------------------ */
#define AMR_NOALLOC_MAX_LEAVES 16384
int amr_reduce_noalloc(const amr_config* cfg, const double* U, long long nleaves, double* dt_cfl, double* totals);

/* ------------------------------------------------------------------------
 * Batched Helmholtz multigrid (Sec. 2.5.1, Eq. (diff-helmholtz); Sec. 1.4).
 * Solves (lambda_i - lap_h) x = b for n_inst independent square (cube) grids
 * of side n_cells[i] on [0, L]^ndim, cell-centred 5/7-point Laplacian, with
 * periodic or zero-flux (Neumann, Sec. 2.5.2) boundaries: a Neumann boundary
 * cell sums only its in-domain neighbours, (sum - count x) / h^2.  Red-black Gauss-Seidel smoothing (nu1 pre, nu2 post),
 * restriction = mean of 2^ndim children, cell-centred (bi/tri)linear
 * prolongation, coarsening while the side is even and > coarse_max, exact
 * solve on the coarsest grid.  Iterates until max|b - A x| <= rtol * max|b|
 * per instance (the paper's max-residual rule, Sec. 2.5.2), or max_cycles.
 * precision AMR_FP32: V-cycles in float on the correction, iterate, residual
 * and norms in float64 (defect correction); AMR_FP64: everything float64.
 * ------------------------------------------------------------------------ */
typedef struct mg_handle mg_handle;

typedef struct {
  int ndim;             /* 2 or 3 */
  int n_inst;           /* number of independent grids */
  const int* n_cells;   /* [n_inst] cells per side, n_cells[i]^ndim < 2^31 (host pointer, copied);
                           a larger instance fails with AMR_ERR_INVALID_ARG */
  const double* lambda; /* [n_inst] Helmholtz constants > 0 (host pointer, copied) */
  double L;             /* domain side */
  int nu1, nu2, max_cycles;
  double rtol;
  int coarse_max;       /* 8 */
  int precision;        /* AMR_FP32 or AMR_FP64 */
  void* stream;
  int bc;               /* MG_BC_PERIODIC or MG_BC_NEUMANN */
} mg_config;

int mg_create(const mg_config* cfg, mg_handle** out);
int mg_destroy(mg_handle* h);
const char* mg_last_error(const mg_handle* h);
/* Total unknowns = sum_i n_cells[i]^ndim; b and x are packed instance after
 * instance, each x-fastest.  x holds the initial guess on entry and the
 * solution on return.  cycles[n_inst] (host, may be NULL) gets the V-cycles
 * per instance, relres[n_inst] (host, may be NULL) the final max-norm
 * relative residuals.  Synchronous.  MG_ERR_NOT_CONVERGED if an instance
 * did not reach rtol (x then holds the last iterate). */
int mg_solve(mg_handle* h, const double* b, double* x, int on_device, int* cycles, double* relres);
int mg_num_unknowns(const mg_handle* h, long long* n);
/* kernels this handle has launched so far (graph nodes included) */
int mg_kernel_launches(const mg_handle* h, long long* n);
/* One more V-cycle (Sec. 1.4; the correction of the current defect, as one loop iteration
 * of mg_solve, which must have run before) over every instance, converged or not, its
 * kernels launched one by one with a CUDA event
 * after each: kind[i] and us[i] = microseconds between consecutive events for kernel i, for
 * up to cap kernels; *nkernels = kernels of the cycle.  Kinds: 0 2D red-black sweep, 1 copy,
 * 2 3D half sweep, 3 residual + restriction, 4 coarsest solve, 5 prolongation, 6 float32
 * update (X += e, R -= A e), 7 zero correction, 8 float64 correction, 9 float64 defect,
 * 10 the coarse depths of 2D instances in shared memory (one CTA per instance).
 * The iterate advances by that cycle.  Synchronous; for measurement only.
 * AMR_ERR_INVALID_ARG before the first mg_solve. */
int mg_profile_vcycle(mg_handle* h, int* kind, float* us, int cap, int* nkernels);
/* 2D: the strip height of the red-black sweep used for levels of side `side`, chosen by
 * the autotuner at mg_create: per depth of the batch, the sweep of all instances' levels
 * of that depth is timed with each candidate height (4..64, or the side-based default
 * clamp(side/32, 8, 64)) and the fastest kept; cached per (sides, precision, boundary
 * kind) for the process.  Every height gives the same iterate bit for bit.
 * AMR_ERR_INVALID_ARG for a side that is not swept. */
int mg_strip_height(const mg_handle* h, int side, int* height);

/* ------------------------------------------------------------------------
 * Reaction-diffusion steps (Sec. 2.5): w = (u, v), dw/dt = F0(w) + F1(w), with
 * F0 the reaction terms of Eq. (gray-scott) (model RD_GRAY_SCOTT: F, k) or
 * Eq. (schnakenberg) (RD_SCHNAKENBERG: kappa, a, b) and F1 = D lap_h w.
 * Schemes:
 *  RD_IMEX, Eq. (imex): reaction explicit, diffusion implicit through the
 *    batched multigrid above with lambda = 2/(dt D) per species; guess w_n.
 *  RD_SPLIT, Eqs. (splitting), (diff-helmholtz): w* = w_n + dt F0(w_n), then
 *    (lambda - lap_h) w_{n+1} = lambda w* with lambda = 1/(dt D); guess w*.
 *  RD_EXPLICIT: three-stage SSP Runge-Kutta on F0 + F1 (no multigrid); stable
 *    for dt below about h^2 / (2 ndim max(Du, Dv)) (Sec. 2.5.1).
 * Both species of all instances form one multigrid batch.  Boundaries: bc
 * (MG_BC_PERIODIC or MG_BC_NEUMANN, zero flux).
 * ------------------------------------------------------------------------ */
typedef struct rd_handle rd_handle;

typedef struct {
  int ndim, n_inst;
  const int* n_cells;   /* [n_inst] (host, copied) */
  double L, Du, Dv, F, k, dt;
  int nu1, nu2, max_cycles;
  double rtol;
  int coarse_max;
  int precision;        /* AMR_FP32 (float smoothing) or AMR_FP64 */
  void* stream;
  int model;            /* RD_GRAY_SCOTT or RD_SCHNAKENBERG */
  double kappa, a, b;   /* Schnakenberg constants */
  int scheme;           /* RD_IMEX, RD_SPLIT or RD_EXPLICIT */
  int bc;               /* MG_BC_PERIODIC or MG_BC_NEUMANN */
} rd_config;

int rd_create(const rd_config* cfg, rd_handle** out);
int rd_destroy(rd_handle* h);
const char* rd_last_error(const rd_handle* h);
/* u, v packed instance after instance (as mg_solve). Synchronous. */
int rd_set_state(rd_handle* h, const double* u, const double* v, int on_device);
int rd_read_state(rd_handle* h, double* u, double* v, int on_device);
/* nsteps steps of the configured scheme; cycles (host, may be NULL) receives
 * [step][2*n_inst] V-cycles (species-major: u of every instance, then v; 0 for
 * RD_EXPLICIT).  Synchronous.  Without a learned guess each implicit step is one
 * graph launch whose multigrid convergence loop runs on the device (a graph
 * conditional node), and the host waits once per 256 steps; MG_ERR_NOT_CONVERGED
 * is then reported after those steps (the state has advanced through them). */
int rd_step(rd_handle* h, int nsteps, int* cycles);
int rd_kernel_launches(const rd_handle* h, long long* n);

/* ------------------------------------------------------------------------
 * Multigrid on a 2D block quadtree (Sec. 1.4: AMR-compatible multigrid; Sec.
 * 2.5.2 runs it on a three-level mesh), float64: solves (lambda - lap_h) x = b
 * on the leaf cells of a periodic, 2:1-balanced (faces and corners) quadtree
 * over a square base of nbx x nby (nbx == nby) blocks of B^2 cells (B = 8 or
 * 16), level-1 cell size L / (nbx B), level-l cell size halved per level.
 * Composite operator: the 5-point stencil of each leaf cell's level; a coarser
 * neighbour contributes (2/3) C^ + (1/3) f0 (C^: the coarse value moved along
 * the face by a linear slope), a refined neighbour (4/3) m - (1/3) f0 (m: mean of
 * the two finer cells on the face; flux matching, conservative).  Full
 * approximation scheme over the tree levels with red-black Gauss-Seidel (nu1,
 * nu2), the base level solved in correction form (A e = b - A x from e = 0) by the
 * uniform multigrid above until its residual is below base_rtol of max|b - A x|.
 * Leaves: level[k] >= 1 and block coordinates (coords[2k], coords[2k+1]) at
 * that level, any order; leaf data [leaf][B*B] in that order, x fastest.
 * ------------------------------------------------------------------------ */
typedef struct mgt_handle mgt_handle;

typedef struct {
  int nbx, nby, B;
  double L, lambda;     /* lambda >= 0 */
  int nu1, nu2, max_cycles;
  double rtol;          /* stop when max|b - A x| over leaf cells <= rtol max|b| */
  double base_rtol;     /* base-level solves: residual reduction factor (1e-3) */
  int coarse_max;       /* the base multigrid's coarsest side */
  void* stream;         /* NULL: the handle creates its own */
} mgt_config;

/* Copies the tree; AMR_ERR_INVALID_ARG if the leaves leave a gap, overlap, or break
 * the 2:1 balance. */
int mgt_create(const mgt_config* cfg, int nleaves, const int* level, const int* coords, mgt_handle** out);
int mgt_destroy(mgt_handle* h);
const char* mgt_last_error(const mgt_handle* h);
int mgt_num_leaves(const mgt_handle* h, long long* n);
/* x: guess in, solution out (host or device, as b).  fixed_cycles > 0 runs exactly
 * that many V-cycles; 0 iterates to rtol (MG_ERR_NOT_CONVERGED after max_cycles).
 * cycles, relres (host, may be NULL): V-cycles run, final relative residual.
 * Synchronous. */
int mgt_solve(mgt_handle* h, const double* b, double* x, int on_device, int fixed_cycles, int* cycles,
              double* relres);
/* the composite operator: Ax = (lambda - lap_h) x on the leaf cells.  Synchronous. */
int mgt_apply(mgt_handle* h, const double* x, double* Ax, int on_device);
int mgt_kernel_launches(const mgt_handle* h, long long* n);

/* Gray-Scott IMEX steps (Eq. (imex), Eq. (gray-scott)) on the leaves of the same kind
 * of quadtree: the composite Laplacian above for the explicit parts, the tree multigrid
 * (lambda = 2/(dt D) per species, guess w_n) for the implicit stage.  The tree is fixed
 * (no regrid).  mg.lambda is ignored; state [leaf][B*B] per species, float64. */
typedef struct rdt_handle rdt_handle;

typedef struct {
  mgt_config mg;
  double Du, Dv, F, k, dt;
} rdt_config;

int rdt_create(const rdt_config* cfg, int nleaves, const int* level, const int* coords, rdt_handle** out);
int rdt_destroy(rdt_handle* h);
const char* rdt_last_error(const rdt_handle* h);
int rdt_set_state(rdt_handle* h, const double* u, const double* v, int on_device);
int rdt_read_state(rdt_handle* h, double* u, double* v, int on_device);
/* cycles (host, may be NULL): [step][2] V-cycles (u, v).  Synchronous. */
int rdt_step(rdt_handle* h, int nsteps, int* cycles);
int rdt_kernel_launches(const rdt_handle* h, long long* n);
int rdt_num_leaves(const rdt_handle* h, long long* n);
/* the current leaves: level[n], coords[2n] (host, capacity cap leaves) */
int rdt_leaves(const rdt_handle* h, int* level, int* coords, long long cap);
/* Regrid (the paper adapts the Gray-Scott mesh; the criterion is a reading): Lohner
 * estimator of u (per direction, filter eps, neighbours by the level values), refine
 * leaves above refine_tol up to max_level, coarsen groups of four sibling leaves below
 * coarsen_frac * refine_tol, 2:1 balance over faces and corners; fields copied, prolonged
 * with minmod slopes, or restricted (means).  New leaves in Morton order of their lower
 * corner at max_level; err_out (host, may be NULL) gets the old leaves' estimator and
 * nleaves_out the new count.  The state keeps its float64 layout [leaf][B*B]. */
int rdt_regrid(rdt_handle* h, double refine_tol, double coarsen_frac, double eps, int max_level, double* err_out,
               long long* nleaves_out);

/* ------------------------------------------------------------------------
 * Learned multigrid initial guess (no counterpart in the paper; the project's
 * addition to the implicit diffusion stage of Eq. (imex)).
 *
 * Network: 4 periodic convolutions with 3^ndim taps and bias, channels
 * 5 -> 16 -> 16 -> 16 -> 2, GELU (erf form) after layers 1..3; bf16 weights and
 * activations, fp32 accumulation on the tensor cores.  Parameters are float32,
 * flat, per layer W[cout][cin][tap] (tap x fastest over offsets -1, 0, 1 per
 * dimension) followed by b[cout]; training keeps float32 master weights (Adam,
 * beta 0.9/0.999, eps 1e-8).  Images are device float32 [N][C][D][H][W]
 * (D = 1 in 2D); H and W multiples of 16 (2D) or D of 4 and H, W of 8 (3D).
 * Loss (cnn_set_loss): mean over both output channels and over pixels at least
 * `margin` cells from every image edge of (out - target)^2 (CNN_LOSS_MSE, the
 * default), or of q^2 (CNN_LOSS_OPERATOR) with
 *   q = (1 + kappa_c) e - (1/(2 ndim)) * sum of e over the 2 ndim face neighbours,
 *   e = out - target.
 * With target = (w* - w_n)/scale, q is the residual lambda g - A X of the guess
 * X = w_n + scale * out under the Helmholtz operator A = lambda - lap_h of
 * Eq. (diff-helmholtz), divided by scale * 2 ndim / h^2; kappa_c = lambda_c h^2 /
 * (2 ndim) per species.  The operator loss needs margin >= 1.
 * ------------------------------------------------------------------------ */
#define CNN_LOSS_MSE 0
#define CNN_LOSS_OPERATOR 1
typedef struct cnn_handle cnn_handle;

/* He-normal initial weights from `seed`, zero biases; stream NULL = own stream. */
int cnn_create(int ndim, unsigned long long seed, void* stream, cnn_handle** out);
int cnn_destroy(cnn_handle* h);
const char* cnn_last_error(const cnn_handle* h);
int cnn_num_params(const cnn_handle* h, long long* n);
/* host float32 arrays of exactly cnn_num_params values; set also resets Adam */
int cnn_set_params(cnn_handle* h, const float* params, long long n);
int cnn_get_params(cnn_handle* h, float* params, long long n);
/* in: device [N][5][...]; out: device [N][2][...].  Synchronous. */
int cnn_forward(cnn_handle* h, const float* in, int N, int D, int H, int W, float* out);
/* loss (host, may be NULL) and its gradient (host float32 [n params], may be NULL) */
int cnn_gradient(cnn_handle* h, const float* in, const float* target, int N, int D, int H, int W, int margin,
                 float* grad, float* loss);
/* one Adam step on the batch; loss (host) if not NULL */
int cnn_train_step(cnn_handle* h, const float* in, const float* target, int N, int D, int H, int W, int margin,
                   float lr, float* loss);
/* Loss of the following cnn_gradient / cnn_train_step calls: kind CNN_LOSS_MSE or
 * CNN_LOSS_OPERATOR; kappa (host, 2 values, finite, >= 0) is read for the operator
 * loss only and may be NULL for MSE.  AMR_ERR_INVALID_ARG otherwise; a later
 * gradient call with margin < 1 under the operator loss is AMR_ERR_INVALID_ARG. */
int cnn_set_loss(cnn_handle* h, int kind, const double* kappa);
/* Inference.  2D images whose sides are multiples of 32 (W) and 16 (H) run one fused
 * kernel for all four layers (activations stay in shared memory; nothing is allocated),
 * with GELU in its tanh form (Hendrycks and Gimpel, 2016; within 4.7e-4 of the erf form,
 * plus the hardware tanh's error of order 2^-11 times |z|/2): outputs agree with
 * cnn_forward to the bf16 tolerance of the network.  Other shapes: cnn_forward.
 * Arguments and layouts as cnn_forward.  Synchronous. */
int cnn_infer(cnn_handle* h, const float* in, int N, int D, int H, int W, float* out);
/* Parameters to / from a file: 8-byte magic "AMRVCNN1", int32 ndim, int32 0, int64 count,
 * count float32 values (host byte order).  cnn_load checks the magic, ndim and count
 * (AMR_ERR_INVALID_ARG otherwise, handle unchanged) and resets Adam like cnn_set_params.
 * File errors: AMR_ERR_INVALID_ARG with the path in cnn_last_error. */
int cnn_save(cnn_handle* h, const char* path);
int cnn_load(cnn_handle* h, const char* path);
int cnn_kernel_launches(const cnn_handle* h, long long* n);

/* Multigrid initial guess of rd_step: net = NULL restores the previous-step
 * guess w_n; otherwise X = w_n + scale * net(u_n, v_n, c2, c3, dt) per species
 * (c2, c3 as set by rd_set_guess_inputs) (the network predicts the increment over the previous-step
 * guess).  The multigrid still iterates to rtol.  The handle keeps a pointer to
 * net (not owned).  Sides must be multiples of 16 (2D) or 8 (3D). */
int rd_set_guess(rd_handle* h, cnn_handle* net, double scale);
/* Input channels 2 and 3 of the network, for rd_set_guess and rd_extract_crops:
 * RD_GUESS_IN_PREV (default) = (u*_prev, v*_prev), the previous step's solution;
 * RD_GUESS_IN_RESIDUAL = the residual of the previous-step guess, per species
 * (lambda g - A w_n) * h^2 / (2 ndim) / scale, A = lambda - lap_h of
 * Eq. (diff-helmholtz) with the handle's boundaries.  With target (w* - w_n)/scale
 * the network's ideal map is then the local inverse of the normalised operator. */
#define RD_GUESS_IN_PREV 0
#define RD_GUESS_IN_RESIDUAL 1
int rd_set_guess_inputs(rd_handle* h, int kind);
/* Max-norm relative residuals max|b - A x| / max|b| of the initial guess and of
 * the final iterate of the last multigrid solve, per (species, instance):
 * initial[2*n_inst], final[2*n_inst] (host, either may be NULL). */
int rd_last_residuals(rd_handle* h, double* initial, double* final_);
/* Training pairs from the last rd_step: for crop k of side `crop` with lowest
 * corner corner[3k..3k+2] (periodic) in instance inst[k]: in[k] (device float
 * [5][crop^ndim]) = (u_n, v_n, c2, c3, dt), channels 2 and 3 as set by
 * rd_set_guess_inputs, and target[k] (device float [2][crop^ndim]) =
 * (w* - w_n) / scale for u and v. */
int rd_extract_crops(rd_handle* h, int ncrops, const int* inst, const int* corner, int crop, double scale, float* in,
                     float* target);

#ifdef __cplusplus
}
#endif
#endif
