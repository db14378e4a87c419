/*
 * dpsim: GPU (GB300, sm_103a) Newton-step solver for two-phase oil-water flow
 * in a naturally fractured reservoir, dual-porosity model.
 *
 * Method: Shen, Cui, Liu, Zhu, Zhong, Chen et al., "Numerical Simulation of
 * Two-phase Flow in Natural Fractured Reservoirs Using Dual Porosity Method
 * on Parallel Computers".
 *   - model: Section 2 (Darcy law Eq. 1-2, mass conservation, constraints,
 *     dual-porosity system Eq. "prob", transfer term q_mf, perforation rate,
 *     well index and Peaceman radius);
 *   - discretisation: Section 3 (FIM, unknowns p, s_w per cell and p_b per
 *     well, backward Euler, cell-centred finite differences, F(x) = 0 of
 *     size N = 2n + tau, Eq. "nonlinear");
 *   - nonlinear solver: Algorithm 1 (inexact Newton) with the forcing terms
 *     of Section 3.1;
 *   - linear solver: Section 3.2 (block Jacobian, decoupling
 *     D^-1 A x = D^-1 b of Eq. "decoupled-eq" by a Gauss-Jordan step, GMRES
 *     preconditioned by CPR-FPF).
 *
 * Conventions shared by every entry point:
 *   - SI units throughout (m, m^2, Pa, Pa s, kg/m^3, m^3/s, s).
 *   - A "location" is a grid block (i, j, k), loc = i + nx (j + ny k).  Each
 *     location has a fracture cell c = 2 loc and a matrix cell c = 2 loc + 1.
 *     n_cells = 2 nx ny nz.  Well w owns block row n_cells + w.
 *   - Every block row has two unknowns: (p, s_w) for a cell, (p_b, dummy)
 *     for a well; every residual row pair is (oil, water) for a cell and
 *     (well equation, dummy) for a well.
 *   - Host pointers are read during the call only (the library copies what
 *     it keeps).  Device memory is owned by the dp_sim and obtained through
 *     the dp_allocator given at creation (cudaMallocAsync when NULL).
 *   - All work is ordered on the CUDA stream given at creation.  Calls that
 *     return host results synchronise that stream before returning.
 *   - Return value: DP_OK (0) or a negative DP_E* code; sim_last_error()
 *     gives a message.  A failed call leaves the dp_sim usable unless it
 *     returned DP_ECUDA or DP_ENOMEM.
 */
#ifndef DPSIM_H
#define DPSIM_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DP_OK 0
#define DP_EINVAL (-1)   /* bad argument or size */
#define DP_ENOMEM (-2)   /* the allocator returned NULL; the dp_sim must be destroyed
                            (sim_destroy then returns every block it holds) */
#define DP_ECUDA (-3)    /* a CUDA call failed; the dp_sim must be destroyed */
#define DP_ELINEAR (-4)  /* FGMRES did not reach its tolerance */
#define DP_ENEWTON (-5)  /* Newton did not converge; the old state is restored */
#define DP_ETIMEOUT (-6) /* a bounded device-side wait gave up */

/* Structured grid (Section 4, Example 1 layout): nx x ny x nz blocks of
 * size dx x dy x dz; top_depth is the depth of the top face (gravity). */
typedef struct { int32_t nx, ny, nz; double dx, dy, dz, top_depth; } dp_grid;

/* Rock (Section 2): isotropic fracture and matrix permeabilities (m^2) and
 * reference porosities per location ([nx ny nz] each, host pointers), the
 * shape factor sigma (m^-2) of the transfer term, rock compressibility
 * (1/Pa) and its reference pressure (Pa). */
typedef struct {
  const double *kf, *km, *phi_f, *phi_m;
  double sigma, c_rock, p_ref;
} dp_rock;

/* Fluids (Section 2): viscosities (Pa s), compressibilities (1/Pa) of the
 * linear densities rho = rho_ref (1 + c (p - p_ref)), Corey end points
 * s_wc, s_or (krw = S^2, kro = (1-S)^2 of the normalised saturation), and
 * the gravitational acceleration g (m/s^2).
 * Capillary pressure (Section 2 constraints, p_w = p_o - p_cow(s_w)):
 * pc_n[k] points (0..256) of the table of continuum k (0 fracture, 1 matrix),
 * pc_table[k] -> pc_n[k] pairs (s_w, p_cow in Pa) with s_w strictly
 * ascending, read once by sim_create (host memory).  p_cow is linear
 * between points and constant outside; with no table it is zero.  It enters
 * the water potential of the fluxes and of the fracture-matrix transfer;
 * densities and perforation rates use the oil pressure p. */
typedef struct {
  double mu_o, mu_w, c_o, c_w, rho_o_ref, rho_w_ref, p_ref, swc, sor, g;
  int32_t pc_n[2];
  const double *pc_table[2];
} dp_fluid;

/* Vertical well perforating the fracture cells of column (i, j), layers
 * k_top..k_bot (Section 2, perforation rate and well index).  kind
 * DP_WELL_RATE_INJ: water injector at a reservoir-volume rate target (m^3/s);
 * DP_WELL_BHP: well at a bottom-hole pressure target (Pa);
 * DP_WELL_OIL_RATE: producer at an oil mass-rate target (kg/s, the oil
 * leaving through its perforations; the producers of Section 4's examples).  rw: wellbore
 * radius (m); skin: skin factor.  limit (Pa, 0: none; kinds 0 and 2): a
 * maximum BHP for an injector, a minimum BHP for an oil-rate producer; after
 * each Newton update of sim_advance a well past its limit switches to BHP
 * control at the limit for the rest of that timestep (each timestep starts on
 * the well's own control).  wi (m^3): > 0 gives every perforation this well
 * index, 0 takes Peaceman's from kf, dx, dy, dz, rw and skin. */
typedef enum { DP_WELL_RATE_INJ = 0, DP_WELL_BHP = 1, DP_WELL_OIL_RATE = 2 } dp_well_kind;
typedef struct {
  int32_t kind, i, j, k_top, k_bot;
  double target, rw, skin;
  double limit, wi;
} dp_well;

/* Device memory provider.  alloc returns device memory usable on `stream`
 * (or NULL); free releases it.  ctx is passed back unchanged. */
typedef struct {
  void *(*alloc)(size_t bytes, void *stream, void *ctx);
  void (*free)(void *ptr, size_t bytes, void *stream, void *ctx);
  void *ctx;
} dp_allocator;

/* Solver options.  eta_mode 0: fixed forcing term eta_fixed; 1-3: the three
 * forcing terms of Section 3.1, clipped to [eta_min, eta_max] (eta_max on a
 * timestep's first Newton iteration).  With b = -R and the previous solve's
 * linear residual r = b - J y (J as assembled), every norm taken in the
 * scaled norm of Algorithm 1's ||b|| (sim_get_norms out[0]): 1 is
 * ||b(x^l) - r^{l-1}|| / ||b(x^{l-1})||, 2 is (||b(x^l)|| - ||r^{l-1}||) /
 * ||b(x^{l-1})||, 3 is eta_gamma (||b(x^l)|| / ||b(x^{l-1})||)^eta_beta.  precond:
 * 0 none, 1 block ILU(0) only, 2 CPR-FPF.  precision: 0 FP64 everywhere;
 * 1 the preconditioner in FP32 inside FP64 FGMRES: ILU(0) factors, AMG
 * levels and the CPR stage residuals (from an FP32 copy of the decoupled
 * operator); the Arnoldi products, restart residuals and orthogonalisation
 * stay FP64; 2 as 1, with the operator, prolongation and restriction values
 * of the AMG levels >= 1 (not the coarsest, solved by its FP64 inverse)
 * stored in BF16 and widened to FP32 as they are read (levels run inside the
 * cluster kernel keep FP32 values).  amg_gs_levels: AMG levels 0..amg_gs_levels-1 are smoothed by
 * multicolour Gauss-Seidel (forward colour order before the coarse
 * correction, reverse after), the coarser ones by one l1-Jacobi sweep
 * before and after, x += (b - A x) / sum_j |a_ij| (Baker, Falgout, Kolev and
 * Yang 2011): one parallel phase per sweep instead of one per colour. */
typedef struct {
  double newton_tol, newton_atol; int32_t newton_max;
  int32_t eta_mode;
  double eta_fixed, eta_gamma, eta_beta, eta_min, eta_max;
  int32_t gmres_restart, gmres_maxit;
  double amg_theta; int32_t amg_coarse_max, amg_max_levels;
  int32_t precond;
  double ds_max;
  int32_t precision;
  int32_t use_graphs;   /* capture the FGMRES iteration in a CUDA graph */
  int32_t amg_gs_levels;
  int32_t cluster_rows;  /* AMG levels of at most this many rows run inside one
                            thread-block-cluster launch per V-cycle (with
                            use_graphs); < 0: never; 0: the library default,
                            20000 rows when one of those levels uses
                            Gauss-Seidel, else never */
  int32_t amg_refresh;   /* 0: the prolongators and coarse operators are recomputed
                            every Newton iteration; 1: only at the first Newton
                            iteration of a timestep (level 0, the pressure block,
                            always takes the current values) */
  int32_t decouple;      /* D of Eq. "decoupled-eq", per cell block row (well rows
                            unchanged): 0 the modified Gauss-Jordan step, read as
                            the elimination of the pressure row's saturation
                            coefficient by the water row of the diagonal block,
                            D_i^-1 = [[1, -a01/a11], [0, 1]] (the per-cell
                            Quasi-IMPES form); 1 ABF, D_i = the diagonal block;
                            2 True-IMPES, D_i^-1 = [[1, -c01/c11], [0, 1]] with c
                            the sums of block column i over all rows (Section 3.2
                            names Quasi-IMPES and ABF beside its own choice) */
  int32_t schur;         /* 1: eliminate every matrix cell exactly before the solve (a
                            matrix cell couples only to its own fracture cell, Section
                            2), y_m = A_mm^-1 (-R_m - A_mf y_f); the decoupling, ILU(0),
                            AMG and FGMRES work on the fracture-and-well system with
                            S_ff = A_ff - A_fm A_mm^-1 A_mf (half the unknowns); 0: the
                            full system */
  double reorth;         /* classical Gram-Schmidt of FGMRES's Arnoldi step: a second
                            pass when ||w - V h||^2 < reorth ||w||^2 after the first
                            (the test of Daniel, Gragg, Kaufman and Stewart; 0.5 its
                            usual constant, >= 1: always two passes, 0: one pass);
                            finite, >= 0 */
} dp_options;

typedef struct {
  int32_t newton_iters, linear_iters, converged, amg_levels;
  double res0, res, lin_relres, eta;
  double ms_setup, ms_solve;   /* device time of the last solve_step parts */
} dp_stats;

typedef struct dp_sim dp_sim;

/* Launch scheduling (no counterpart in the paper): the short, latency-bound
 * kernels of a solve (the well rows of level 0's Gauss-Seidel and of the
 * ILU(0) forward sweep, level 0's pipelined colour kernels, the V-cycle below
 * level 0 and its transfers) are launched as programmatic dependents of the
 * kernel before them on the stream, so that their launch and the loads that
 * do not depend on that kernel overlap its end.  The environment variable
 * DPSIM_PDL, read once per process, is a bit mask of the classes to launch
 * that way (1 level-0 well rows, 2 the V-cycle below level 0, 4 the latter
 * letting their own dependents in early, 8 level 0's colour kernels, 16 the
 * ILU(0) forward well rows; default 31, all); results do not depend on it. */

/* Create a realisation: copies grid, rock, fluid and wells, computes the
 * well indices (Peaceman's radius for a vertical well, Section 2), builds
 * the block pattern (fracture 7-point stencil, fracture-matrix pairs, well
 * rows and columns) and the transmissibilities on the device.  `stream` is
 * a cudaStream_t (NULL: the default stream).  `alloc` may be NULL.  The
 * state is set to zero; call sim_set_state before assembling. */
int sim_create(const dp_grid *grid, const dp_rock *rock, const dp_fluid *fluid,
               const dp_well *wells, int32_t nwells, const dp_options *opts,
               const dp_allocator *alloc, void *stream, dp_sim **out);

void sim_destroy(dp_sim *sim);

/* Sizes: block rows n_cells + nwells, nonzero 2x2 blocks, cells, wells. */
int sim_sizes(const dp_sim *sim, int32_t *nb, int32_t *nnzb, int32_t *ncells,
              int32_t *nwells);

/* Set the state (host pointers: p[n_cells] Pa, sw[n_cells], bhp[nwells] Pa)
 * as both the current Newton iterate and the old time level x^n. */
int sim_set_state(dp_sim *sim, const double *p, const double *sw, const double *bhp);

/* Set only the current Newton iterate (host pointers); x^n is kept. */
int sim_set_iterate(dp_sim *sim, const double *p, const double *sw, const double *bhp);

/* Same as sim_set_state with DEVICE pointers (stream-ordered copy). */
int sim_set_state_device(dp_sim *sim, const double *p, const double *sw, const double *bhp);

/* Copy the current iterate to host arrays (synchronises). */
int sim_get_state(dp_sim *sim, double *p, double *sw, double *bhp);

/* Residual R and Jacobian J of F(x) = 0 at the current iterate for a step
 * of length dt (s) from x^n (Section 3, Eq. "nonlinear"), and the scaled
 * residual norms of Algorithm 1.  Stream-ordered; does not synchronise. */
int sim_assemble(dp_sim *sim, double dt);

/* Copy the last assembled Jacobian (BSR: rowptr[nb+1], col[nnzb],
 * val[4 nnzb] row-major 2x2 blocks) and residual res[2 nb] to host arrays;
 * any pointer may be NULL.  Valid between sim_assemble and sim_solve_step. */
int sim_get_jacobian(dp_sim *sim, int32_t *rowptr, int32_t *col, double *val, double *res);

/* Scaled residual norms and balances of the last assembly (synchronises):
 * out[0] ||R~||_2, out[1] ||R~||_inf, out[2..3] sum of oil / water cell
 * residuals, out[4..5] oil / water mass change since x^n, out[6..7] oil /
 * water mass rate injected by the wells. */
int sim_get_norms(dp_sim *sim, double *out8);

/* One linear solve of Algorithm 1 at the assembled iterate: decoupling
 * (Eq. "decoupled-eq"), pressure extraction, block ILU(0), AMG setup (first
 * call) or value refresh, CPR-FPF preconditioned FGMRES to the forcing term
 * eta, and the update x += y (saturation change limited to +-ds_max, s_w
 * kept in [0, 1]).  Synchronises; fills *stats when not NULL.  DP_ELINEAR:
 * FGMRES did not reach eta within gmres_maxit iterations; no update is made
 * (the state is unchanged; call sim_assemble before solving again). */
int sim_solve_step(dp_sim *sim, dp_stats *stats);

/* One backward-Euler timestep of length dt by Algorithm 1.  On failure the
 * old state is restored and DP_ENEWTON (Newton did not converge within
 * newton_max iterations) or DP_ELINEAR (a linear solve failed) returned. */
int sim_advance(dp_sim *sim, double dt, dp_stats *stats);

/* A simulation period [0, t_end] (seconds) by sim_advance timesteps, as the
 * paper's examples run theirs (800 and 1600 days): dt0 first; after a
 * converged step the next is min(2 h, dt_max) (h the step just taken); a step
 * whose Newton iteration or linear solve fails is retried at h / 2 (a cut);
 * the last step ends at t_end.  Returns DP_OK at t_end; DP_ENEWTON when a retry would fall
 * below dt_min or after max_steps accepted steps (the state is that of the
 * last accepted step, stats->t its time); other codes as sim_advance.
 * DP_EINVAL: sim NULL, t_end, dt0 or dt_min not > 0, dt_max < dt0, or
 * max_steps < 1.  stats (may be NULL): accepted steps, cuts, Newton and
 * FGMRES iterations summed over the accepted steps, the time reached. */
typedef struct {
  int32_t steps, cuts, newton_iters, linear_iters;
  double t;
} dp_run_stats;
int sim_run(dp_sim *sim, double t_end, double dt0, double dt_max, double dt_min,
            int32_t max_steps, dp_run_stats *stats);

/* Batched timesteps of many realisations (no counterpart in the paper,
 * which advances one grid on many processors; here many independent grids
 * share one GPU).  Advances sims[k] by dt[k] for k < n, like sim_advance,
 * with up to `threads` host threads (0: one per realisation, at most 16)
 * taking realisations from a common queue in order, so that realisations of
 * uneven size keep the GPU busy; each realisation runs on the stream given
 * at its creation, and the kernels of realisations on different streams
 * overlap on the device (realisations that share a stream are serialised by
 * it).  A sim may appear once per call.  Results are those of sim_advance on
 * each realisation alone, bit for bit.  stats[k] and status[k] (may be NULL)
 * receive each realisation's statistics and return code.  Returns DP_OK when
 * every realisation returned DP_OK, else the first failing code. */
int sim_advance_many(dp_sim *const *sims, int32_t n, const double *dt, int32_t threads,
                     dp_stats *stats, int32_t *status);

/* Batched timesteps in lockstep (no counterpart in the paper; the batched
 * engine of many uneven-size realisations on one GPU).  A batch groups n
 * realisations created with the FP32 preconditioner (precision 1 or 2),
 * CPR-FPF (precond 2), l1-Jacobi below AMG level 0 (amg_gs_levels <= 1), the
 * V-cycle outside the cluster kernel (cluster_rows < 0) and equal
 * gmres_restart and gmres_maxit; the realisations must not be used by other
 * calls while batch_advance runs, nor destroyed before it returns.
 * batch_advance does one timestep of each realisation k by dt[k] (Algorithm
 * 1, as sim_advance): every Newton iteration assembles and sets up each
 * realisation still iterating (up to 16 host threads, each realisation on
 * the stream it was created with, so these must differ to overlap), then
 * runs their FGMRES iterations together on `stream`:
 * every phase of the Arnoldi step (the ILU(0) sweeps of each colour, the
 * CPR stage residuals, each level of the V-cycle, the operator product, the
 * Gram-Schmidt passes, the Givens rotations) is one launch over a work list
 * of (realisation, block) tiles, in which each realisation runs the blocks
 * of its own launch; each launch's list holds only the realisations still
 * iterating.  At most 256 realisations a batch.  Each realisation's result is that of sim_advance on it
 * alone, bit for bit, whatever the other members of the batch.  `stream`:
 * a cudaStream_t (NULL: the default stream); batch_advance returns after
 * every stream involved has synchronised.  stats[k], status[k] (may
 * be NULL) as sim_advance's; returns DP_OK when all succeeded, else the
 * first failing code.  batch_create returns DP_EINVAL for an unsupported or
 * repeated realisation.  The batch's own device memory (work lists and
 * argument records, a few bytes per tile) comes from cudaMalloc;
 * batch_destroy touches neither the realisations nor the stream. */
typedef struct dp_batch dp_batch;
int batch_create(dp_sim *const *sims, int32_t n, void *stream, dp_batch **out);
int batch_advance(dp_batch *batch, const double *dt, dp_stats *stats, int32_t *status);
void batch_destroy(dp_batch *batch);
const char *batch_last_error(const dp_batch *batch);
/* kernel launches of the batch and its realisations since their creation */
int64_t batch_launch_count(const dp_batch *batch);
/* Where a batch's time goes, since its creation (host wall clock, ms):
 * ms3[0] the per-realisation assembly, convergence tests and set-up, ms3[1]
 * the batched FGMRES, ms3[2] the per-realisation updates; counts3: lockstep
 * Newton rounds, FGMRES cycles, batched Arnoldi steps.  Either may be NULL. */
int batch_profile(const dp_batch *batch, double *ms3, int64_t *counts3);

/* A non-blocking CUDA stream owned by the caller until dp_stream_destroy:
 * for callers whose framework hands out pooled streams (many realisations
 * need as many distinct streams to overlap).  No counterpart in the paper. */
int dp_stream_create(void **stream);
int dp_stream_destroy(void *stream);

/* Block rows and blocks of the system the linear solver works on: the full
 * one, or the fracture-and-well one with the Schur option (the sizes of
 * sim_get_decoupled's arrays and sim_get_colours' array). */
int sim_solver_sizes(dp_sim *sim, int32_t *nb, int32_t *nnzb);

/* Autotuning of launch shapes (no counterpart in the paper): for every AMG
 * level, times each lanes-per-row variant (1..32) of the kernel of its
 * smoother's level operator, of the prolongation and of the restriction;
 * for level 0 in colour order, the kernel of its Gauss-Seidel colours and
 * residual (see sim_set_l0_kernel); and the V-cycle schedule below the
 * cluster level (one cluster launch or a launch per phase).  Each candidate
 * runs `reps` times, timed with CUDA events on the simulation stream on the
 * level's own work vectors, and the fastest is kept; the Arnoldi steps'
 * CUDA graphs are captured again on the next solve.  Colourings, aggregates
 * and operators do not change, but the summation order of some of those
 * kernels does, so results differ from the untuned schedule at rounding
 * level (and a schedule picked by timing can differ between runs).  Needs
 * the AMG hierarchy: call after one sim_solve_step or sim_advance with
 * precond 2.  `report` (may be NULL) receives one text line per decision.
 * Returns DP_ETIMEOUT (and the realisation must be destroyed) when a timed
 * kernel's bounded device wait gave up. */
int sim_autotune(dp_sim *sim, int32_t reps, char *report, int32_t report_len);

/* Sets the kernel of level 0's Gauss-Seidel colours and residual when level
 * 0 runs in the ILU(0) colour order (what sim_autotune chooses; the default
 * is 1):
 *    1  a thread per row;
 *    0  a CTA's rows and their entries staged in shared memory first;
 *   -1, -2, -3  a persistent kernel whose producer warp brings tiles of
 *       256 rows into shared memory with bulk asynchronous copies while the
 *       other warps compute the previous tile: two stages of up to 8
 *       entries a row on average (-1), three of 6 (-2), two of 4 (-3); a
 *       tile with more entries brings its row pointers only.  They need the
 *       level's arrays at 16-byte boundaries (else they run as 1); their
 *       waits are bounded, and one that gives up makes the next
 *       sim_solve_step return DP_ETIMEOUT;
 *    2, 4, 8  lanes per row (a row's entries split between the lanes).
 * 1, 0, -1, -2 and -3 sum a row's products in the same order and give the
 * same results bit for bit; 2, 4 and 8 differ from them at rounding level.
 * Returns DP_EINVAL for another value.  Takes effect from the next solve. */
int sim_set_l0_kernel(dp_sim *sim, int32_t variant);

/* Device bytes the realisation holds through its allocator now, and the
 * most it has held at once (both may be NULL).  Host only, no CUDA call. */
int sim_footprint(dp_sim *s, uint64_t *current, uint64_t *peak);

/* ------------------------------------------------------------- serving
 * A request server for timestep solves of many realisations on one GPU
 * (no counterpart in the paper, whose field runs advance one model on a CPU
 * cluster).  Realisations are registered once (host copies of their inputs
 * and state are kept); a request asks for one sim_advance of one
 * realisation by dt.  `workers` host threads serve the queue concurrently
 * (continuous batching: a request that arrives while others run starts as
 * soon as a worker and device memory are free, and its kernels overlap
 * theirs on the device).  A realisation that has been served stays
 * resident (state, operator, ILU(0) factors, AMG hierarchy) on its own
 * stream.  Admission is by device footprint: a request whose realisation is
 * not resident is admitted when its estimated footprint (the largest bytes
 * per block row measured so far, times its block rows; a guess of 4096 B per
 * row before any measurement, under which an over-budget realisation waits
 * until nothing else runs and is then served alone) fits in hbm_budget after evicting idle resident
 * realisations, least recently used first; an evicted realisation's state
 * goes back to its host copy, and the realisation is rebuilt (operator
 * pattern and AMG set-up) when next served.  Requests are taken in arrival
 * order, skipping those whose realisation is busy or does not fit yet.
 * Results are those of sim_advance on the realisation alone: bit for bit
 * while it stays resident; within the Newton tolerance after an eviction
 * (the AMG aggregates are then rebuilt from the current iterate). */
typedef struct dp_server dp_server;

typedef struct dp_srv_result {
  int32_t status;       /* sim_advance's return code; DP_ENOMEM if the realisation
                           cannot fit in the budget by the measured estimate */
  int32_t realisation;  /* id from srv_add */
  int32_t loaded;       /* 1 if the realisation was (re)built for this request */
  int32_t evicted;      /* realisations evicted to admit it */
  double t_submit_ms;   /* server clock (ms since srv_create): request arrival */
  double t_start_ms;    /* a worker took it */
  double t_done_ms;     /* its result was ready */
  dp_stats stats;
} dp_srv_result;

typedef struct dp_srv_info {
  int32_t registered, resident, queued, running;
  int64_t served, loads, evictions;
  int64_t launches;      /* library kernel launches made for served requests */
  uint64_t resident_bytes, peak_resident_bytes, budget_bytes;
  double bytes_per_row;  /* current admission estimate */
} dp_srv_info;

/* workers >= 1 concurrent requests; hbm_budget > 0 bytes; opts as for
 * sim_create (copied).  Device: the calling thread's current device; the
 * default stream-ordered allocator is used. */
int srv_create(int32_t workers, uint64_t hbm_budget, const dp_options *opts, dp_server **out);
/* Copies the inputs (as for sim_create) and the initial state (p, sw: n_cells
 * each; bhp: nwells).  Returns the realisation id in *id. */
int srv_add(dp_server *srv, const dp_grid *grid, const dp_rock *rock, const dp_fluid *fluid,
            const dp_well *wells, int32_t nwells, const double *p, const double *sw,
            const double *bhp, int32_t *id);
/* Queues one timestep of realisation id by dt (> 0); returns at once with a
 * ticket.  Requests of one realisation run in the order submitted. */
int srv_submit(dp_server *srv, int32_t id, double dt, int64_t *ticket);
/* Blocks until the request is served, then fills *out (once per ticket). */
int srv_wait(dp_server *srv, int64_t ticket, dp_srv_result *out);
/* Waits until realisation id has no queued or running request and copies
 * its state to host arrays (n_cells, n_cells, nwells doubles). */
int srv_get_state(dp_server *srv, int32_t id, double *p, double *sw, double *bhp);
int srv_info(dp_server *srv, dp_srv_info *out);
/* Serves what is queued, stops the workers and frees every realisation. */
int srv_destroy(dp_server *srv);

/* Test access to intermediate results (host arrays, synchronise):
 * the last Newton update y[2 nb]; the decoupled matrix values and
 * right-hand side; the greedy colouring of the block rows (returns the
 * number of colours); the well indices per perforation (returns the count). */
int sim_get_update(dp_sim *sim, double *y);
int sim_get_decoupled(dp_sim *sim, double *val, double *rhs);
int sim_get_colours(dp_sim *sim, int32_t *colour);
int sim_well_index(dp_sim *sim, double *wi);
/* The wells' current controls: kind[nwells] and target[nwells] (host
 * arrays; synchronises).  After sim_advance they show the controls the
 * timestep ended on (a switched well: DP_WELL_BHP at its limit).
 * DP_EINVAL: sim NULL, or kind/target NULL with nwells > 0. */
int sim_well_controls(dp_sim *sim, int32_t *kind, double *target);
/* Per well, the oil and water mass rates (kg/s, positive into the
 * reservoir: an injector's water rate is > 0, a producer's rates are <= 0)
 * summed over its perforations at the current state with the controls in
 * force (Section 2, perforation rate).  q_oil[nwells], q_water[nwells]: host
 * or device arrays; synchronises.  DP_EINVAL: sim NULL, or an array NULL
 * with nwells > 0. */
int sim_well_rates(dp_sim *sim, double *q_oil, double *q_water);

/* AMG hierarchy of the pressure stage after the first sim_solve_step:
 * level sizes (returns the number of levels) and level arrays (CSR of the
 * level operator, aggregate of each row or -1, greedy colour of each row:
 * -1 on a level smoothed by l1-Jacobi, which uses no colouring and gets
 * none); any pointer may be NULL. */
int sim_amg_level_info(dp_sim *sim, int32_t level, int32_t *n, int32_t *nnz, int32_t *nagg);
int sim_amg_level_arrays(dp_sim *sim, int32_t level, int32_t *rowptr, int32_t *col,
                         double *val, int32_t *agg, int32_t *colour);
/* Entries of level `level`'s prolongation P (n x nagg; R = P^T has as
 * many; 0 on the coarsest level) and how the V-cycle treats the level:
 * 0 Gauss-Seidel, 1 l1-Jacobi, 2 a direct solve (the coarsest level's dense
 * inverse or LU); returns the number of levels.  For the algorithmic bytes
 * of a V-cycle.  Either pointer may be NULL; DP_EINVAL as
 * sim_amg_level_info. */
int sim_amg_transfer_info(dp_sim *sim, int32_t level, int32_t *p_nnz, int32_t *smoother);

/* Time every launch of one kernel (by name, e.g. "bsr_spmv") with CUDA
 * events on the simulation stream; NULL stops.  A name with a dot names a
 * region instead, timed from before its first launch to after its last:
 * "sweep.gs", each level-0 Gauss-Seidel sweep in the ILU(0) colour order;
 * "sweep.ilu_fwd" and "sweep.ilu_bwd", each forward and backward sweep of
 * an ILU(0) application;
 * "cycle.coarse", the part of each V-cycle below level 0 (its levels 1 and
 * below, between level 0's restriction and prolongation) when level 0 runs
 * in that order.
 * sim_kernel_timing returns the accumulated milliseconds and the count of
 * launches (regions) since the last reset. */
int sim_time_kernel(dp_sim *sim, const char *name);
int sim_kernel_timing(dp_sim *sim, double *ms, int64_t *launches, int32_t reset);

/* Number of kernel launches made by this dp_sim since creation. */
int64_t sim_launch_count(const dp_sim *sim);

/* Message of the last error on this dp_sim ("" when none). */
const char *sim_last_error(const dp_sim *sim);

/* Scaled residual norms computed without allocating any device memory.
 *
 * The paper has no counterpart of this call; it is a service for callers
 * that must not allocate.  Examples: a serving loop that admits work by its
 * device-memory footprint and keeps that budget exact, and that cannot
 * afford the device-wide synchronisation cudaMalloc/cudaFree imply while
 * other realisations are in flight; or a host program whose device memory
 * is owned by another framework's pool.  It returns the same two numbers as
 * out[0] and out[1] of sim_get_norms (the scaled residual's 2-norm and
 * max-norm, cell rows scaled by dt / (rho_ref phi_ref V), well rows by their
 * target), from a residual the caller already holds on the device.
 *
 * Arguments: grid and fluid are host pointers (only nx, ny, nz, dx, dy, dz
 * and rho_o_ref, rho_w_ref are read); phi_f[nx ny nz], phi_m[nx ny nz],
 * well_kind[nwells], well_target[nwells], res[2 (2 nx ny nz + nwells)] (the
 * layout of sim_get_jacobian's res) and out2[2] are DEVICE pointers; dt is
 * the step length (s); stream is a cudaStream_t (NULL: default stream).
 * The result is written to out2 in stream order; the call does not
 * synchronise.  err (may be NULL) receives a message of at most err_len
 * bytes on failure.
 *
 * Limits and sharing: the block partial sums live in one static device
 * array of 64 KiB (4096 blocks x 2 doubles) that every GPU loading the
 * library keeps until the process exits; problems with more than 8,388,608
 * block rows are rejected with DP_EINVAL and a message.  Every call
 * overwrites the whole part of the array it reads, so nothing needs
 * clearing between calls, but calls that overlap on the GPU (on different
 * streams, or from different threads) share that array and race: order
 * them on one stream.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current and keeps
 * it for the life of the process; make that first call before any stream
 * capture.  A program that resets the device (cudaDeviceReset) invalidates
 * the kept address and must not call this entry point after the reset.  No cudaMalloc, cudaFree or
 * allocating library routine is called.  Returns DP_OK, DP_EINVAL or
 * DP_ECUDA. */
int dp_residual_norms_noalloc(const dp_grid *grid, const dp_fluid *fluid, const double *phi_f,
                              const double *phi_m, int32_t nwells, const int32_t *well_kind,
                              const double *well_target, const double *res, double dt,
                              double *out2, void *stream, char *err, size_t err_len);

#ifdef __cplusplus
}
#endif
#endif
