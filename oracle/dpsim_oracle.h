/*
 * CPU FP64 oracle for the dual-porosity oil-water Newton-step solve.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, sequential restatement of
 * the method of "Numerical Simulation of Two-phase Flow in Natural Fractured
 * Reservoirs Using Dual Porosity Method on Parallel Computers" (Shen et al.):
 * the dual-porosity model (Section 2, Eq. "prob"), the fully implicit
 * cell-centred discretisation (Section 3), the inexact Newton method
 * (Algorithm 1), decoupling (Eq. "decoupled-eq") and GMRES with the CPR-FPF
 * preconditioner (Section 3.2).  Only tests, the smoke check and the timed
 * CPU baseline of the benchmark may load it.  It shares no code, header or
 * constant table with the CUDA library.
 *
 * Every exported function returns 0 on success, a negative code on failure.
 */
#ifndef DPSIM_ORACLE_H
#define DPSIM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { int32_t nx, ny, nz; double dx, dy, dz, top_depth; } og_grid;
typedef struct {
  const double *kf, *km, *phi_f, *phi_m; /* [nL] each, SI */
  double sigma, c_rock, p_ref;
} og_rock;
typedef struct {
  double mu_o, mu_w, c_o, c_w, rho_o_ref, rho_w_ref, p_ref, swc, sor, g;
  int32_t pc_n[2];            /* points of the p_cow(s_w) tables: [0] fracture, [1] matrix;
                                 0: p_cow = 0 in that continuum */
  const double *pc_table[2];  /* pc_n[k] pairs (s_w, p_cow in Pa), s_w strictly ascending;
                                 linear between points, constant outside (copied) */
} og_fluid;
typedef struct {
  int32_t kind, i, j, k_top, k_bot;  /* kind 0: water rate injector, 1: BHP, 2: oil-rate
                                        producer */
  double target, rw, skin;   /* target: m^3/s (kind 0), Pa (kind 1), oil kg/s (kind 2) */
  double limit;              /* kinds 0 and 2: BHP limit (Pa; 0 none): an injector above
                                it, or a producer below it, switches to BHP control */
  double wi;                 /* > 0: well index of every perforation (m^3), else Peaceman */
} og_well;
typedef struct {
  double newton_tol, newton_atol; int32_t newton_max;
  int32_t eta_mode;       /* 0 fixed, 1..3 the three forcing-term choices */
  double eta_fixed, eta_gamma, eta_beta, eta_min, eta_max;
  int32_t gmres_restart, gmres_maxit;
  double amg_theta; int32_t amg_coarse_max, amg_max_levels;
  int32_t precond;        /* 0 none, 1 block ILU(0) only, 2 CPR-FPF */
  double ds_max;
  int32_t amg_gs_levels;  /* levels 0..amg_gs_levels-1 smoothed by multicolour
                             Gauss-Seidel, coarser levels by l1-Jacobi */
  int32_t amg_refresh;    /* 0: P, R and the coarse operators recomputed every
                             Newton iteration; 1: only at the first Newton
                             iteration of a timestep (level 0 always current) */
  int32_t decouple;       /* 0: the paper's modified Gauss-Jordan step (per cell,
                             eliminate the pressure row's saturation coefficient
                             with the diagonal block; the Quasi-IMPES form);
                             1: ABF, the inverse of the diagonal block; 2: True-
                             IMPES, weights from the block-column sums */
  int32_t schur;          /* 1: eliminate every matrix cell exactly (its 2x2 block
                             couples only to its own fracture cell) and solve the
                             fracture-and-well system; 0: the full system */
  double reorth;          /* Gram-Schmidt in FGMRES: a second classical pass when
                             ||w - V h||^2 < reorth ||w||^2 after the first (0.5:
                             the DGKS test; 0: one pass; 1: always two) */
} og_options;
typedef struct {
  int32_t newton_iters, linear_iters, converged, amg_levels;
  double res0, res, lin_relres, eta;
} og_stats;

int  oracle_create(const og_grid *g, const og_rock *r, const og_fluid *f,
                   const og_well *w, int32_t nwells, const og_options *o,
                   void **out);
void oracle_destroy(void *h);
int  oracle_sizes(void *h, int32_t *nb, int32_t *nnzb);
/* block rows and blocks of the system the linear solver sees (the full one,
 * or the fracture-and-well one with schur = 1) */
int  oracle_solver_sizes(void *h, int32_t *nb, int32_t *nnzb);
/* the wells' current controls (kind, target) after the last timestep */
int  oracle_well_controls(void *h, int32_t *kind, double *target);
/* per well, the oil and water mass rates (kg/s, positive into the reservoir)
 * summed over its perforations at the current state and controls */
int  oracle_well_rates(void *h, double *q_oil, double *q_water);
/* p_cow(s_w) and its slope from a table of n (s_w, p_cow) pairs */
void oracle_cap_pressure(int32_t n, const double *table, double sw, double *pc, double *dpc);
int  oracle_set_state(void *h, const double *p, const double *sw, const double *bhp);
int  oracle_set_iterate(void *h, const double *p, const double *sw, const double *bhp);
int  oracle_get_state(void *h, double *p, double *sw, double *bhp);
int  oracle_assemble(void *h, double dt);
int  oracle_get_jacobian(void *h, int32_t *rowptr, int32_t *col, double *val, double *res);
int  oracle_get_norms(void *h, double *out8);
/* one linear solve and update; -4 (no update made) when FGMRES does not
 * reach the forcing term */
int  oracle_solve_step(void *h, og_stats *st);
/* one timestep; -5 (Newton) or -4 (a linear solve) with the old state back */
int  oracle_advance(void *h, double dt, og_stats *st);
/* A simulation period [0, t_end] by timesteps of oracle_advance: dt0 first;
 * after a converged step the next is min(2 h, dt_max) (h the step taken);
 * a step whose Newton iteration or linear solve fails is retried at h / 2 (a
 * cut), and the run stops with OG_ENEWTON once that would fall below dt_min
 * or after max_steps accepted steps; the last step ends at t_end. */
typedef struct {
  int32_t steps, cuts, newton_iters, linear_iters;
  double t;                 /* time reached (s) */
} og_run_stats;
int  oracle_run(void *h, double t_end, double dt0, double dt_max, double dt_min,
                int32_t max_steps, og_run_stats *st);
int  oracle_get_update(void *h, double *y);
int  oracle_get_decoupled(void *h, double *val, double *rhs);
int  oracle_get_colours(void *h, int32_t *colour);
int  oracle_amg_level_info(void *h, int32_t level, int32_t *n, int32_t *nnz, int32_t *nagg);
int  oracle_amg_level_arrays(void *h, int32_t level, int32_t *rowptr, int32_t *col,
                             double *val, int32_t *agg, int32_t *colour);
int  oracle_well_index(void *h, double *wi);

/* Component entry points used by the pinning tests. */
int  oracle_greedy_colour(int32_t n, const int32_t *rowptr, const int32_t *col,
                          int32_t *colour);
int  oracle_ilu0_solve(int32_t n, const int32_t *rowptr, const int32_t *col,
                       const double *val, const int32_t *colour,
                       const double *b, double *x);
/* strength graph (max(|a_ij|, |a_ji|) >= theta sqrt(|a_ii a_jj|)) of a CSR
 * matrix with sorted rows and its MIS(2): state[i] = 2 for a root, 0
 * otherwise; returns the number of roots */
int  oracle_mis2(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val,
                 double theta, int32_t *state);
int  oracle_amg_create(int32_t n, const int32_t *rowptr, const int32_t *col,
                       const double *val, double theta, int32_t coarse_max,
                       int32_t max_levels, void **out);
/* levels 0..gs_levels-1 smoothed by multicolour Gauss-Seidel, the coarser
 * ones by l1-Jacobi (default: Gauss-Seidel on every level) */
int  oracle_amg_set_smoother(void *amg, int32_t gs_levels);
int  oracle_amg_vcycle(void *amg, const double *b, double *x);
int  oracle_amg_info(void *amg, int32_t level, int32_t *n, int32_t *nnz, int32_t *nagg);
int  oracle_amg_arrays(void *amg, int32_t level, int32_t *rowptr, int32_t *col,
                       double *val, int32_t *agg, int32_t *colour);
void oracle_amg_destroy(void *amg);
int  oracle_fgmres_bsr(int32_t n, const int32_t *rowptr, const int32_t *col,
                       const double *val, const double *b, double *x,
                       int32_t precond, int32_t restart, int32_t maxit, double tol,
                       int32_t *iters, double *relres);
int  oracle_fgmres_amg(int32_t n, const int32_t *rowptr, const int32_t *col,
                       const double *val, const double *b, double *x,
                       double theta, int32_t coarse_max, int32_t restart,
                       int32_t maxit, double tol, int32_t *iters, double *relres);
uint32_t oracle_hash32(uint32_t i);

#ifdef __cplusplus
}
#endif
#endif
