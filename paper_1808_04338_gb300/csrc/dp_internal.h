// Internal declarations of the dpsim CUDA library (not part of the C ABI).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "dpsim.h"

namespace dp {

constexpr int kBlock = 256;
// the last-CTA tickets of the long-row tails: a root count and
// kTicketGroups group counts, each on its own 128-byte line
constexpr int kTicketGroups = 128, kTicketStride = 32;
constexpr int kTicketWords = (kTicketGroups + 1) * kTicketStride;

// Error propagation inside the library: every CUDA call is checked, the
// first failure is recorded on the Sim and the entry point returns DP_ECUDA.
struct Err {
  int code = DP_OK;
  std::string msg;
};

#define DP_CUDA(sim, call)                                                     \
  do {                                                                         \
    cudaError_t e__ = (call);                                                  \
    if (e__ != cudaSuccess) {                                                  \
      (sim)->fail(DP_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e__)); \
      return DP_ECUDA;                                                         \
    }                                                                          \
  } while (0)

#define DP_TRY(expr)                 \
  do {                               \
    int rc__ = (expr);               \
    if (rc__ != DP_OK) return rc__;  \
  } while (0)

// Physical constants passed to the physics kernels by value.
struct Phys {
  int nx, ny, nz, nL, nc, nw, nb;
  double dx, dy, dz, top_depth, V;
  double mu_o, mu_w, c_o, c_w, rho_o_ref, rho_w_ref, p_ref, swc, sor, g;
  double inv_span, inv_mu_o, inv_mu_w;
  double sigma, c_rock, p_ref_rock;
  double drho_o, drho_w;          // rho_ref c per phase (the density slopes)
  int pc_n[2];                    // capillary tables: points per continuum
  const double *pc_tab[2];        //   device (s_w, p_cow) pairs, or null
};

// 2x2-block sparse row matrix (device pointers), natural row order.
struct Bsr {
  int n = 0, nnz = 0;
  int *rowptr = nullptr, *col = nullptr, *diag = nullptr;
  double *val = nullptr;
};

// One AMG level: scalar CSR operator plus the transfer operators to the next.
struct Level {
  int n = 0, nnz = 0, nagg = 0;
  int *rowptr = nullptr, *col = nullptr, *dpos = nullptr;
  double *val = nullptr;
  float *valf = nullptr;                 // FP32 copy (precision mode 1)
  int *tpos = nullptr;                   // position of the transposed entry
  uint8_t *strong = nullptr;
  int *agg = nullptr;
  int *colour = nullptr, ncolour = 0;
  int *clist = nullptr;                  // rows sorted by (colour, index)
  std::vector<int> cstart;               // host: colour c rows clist[cstart[c]..cstart[c+1])
  int *cstart_dev = nullptr;             // the same on the device
  int *ell_col = nullptr, *ell_src = nullptr, *ell_off = nullptr, *ell_K = nullptr;
  double *ell_val = nullptr;             // padded per-colour copy (cluster cycle)
  float *ell_valf = nullptr;
  long long ell_total = 0;
  double *fdiag = nullptr, *ratio = nullptr;
  // prolongator P (n x nagg), restriction R = P^T (nagg x n), AP = A P
  int p_nnz = 0, r_nnz = 0, ap_nnz = 0;
  int *p_rowptr = nullptr, *p_col = nullptr;
  double *p_val = nullptr;
  float *p_valf = nullptr;
  int *r_rowptr = nullptr, *r_col = nullptr, *r_src = nullptr;
  double *r_val = nullptr;
  float *r_valf = nullptr;
  // precision 2, levels >= 1: BF16 copies of the operator, P and R values
  // (stored in BF16, computed in FP32)
  __nv_bfloat16 *valh = nullptr, *p_valh = nullptr, *r_valh = nullptr;
  int *ap_rowptr = nullptr, *ap_col = nullptr;
  double *ap_val = nullptr;
  bool l1 = false;                        // l1-Jacobi smoothing (dinv = 1 / sum_j |a_ij|)
  double *dinv = nullptr;                 // 1 / a_ii
  float *dinvf = nullptr;
  int *ap_off = nullptr, *ap_pos = nullptr, *rap_off = nullptr, *rap_pos = nullptr;
  // lanes per row of the level kernels (operator, P, R) and of the products
  int G = 1, p_G = 1, r_G = 1, ap_G = 1, rap_G = 1;
  // V-cycle work vectors
  double *x = nullptr, *b = nullptr, *r = nullptr;
  float *xf = nullptr, *bf = nullptr, *rf = nullptr;
};

struct Sim;

// ---------------------------------------------------------------- memory
void *dalloc(Sim *s, size_t bytes);
void dfree(Sim *s, void *p);

// ---------------------------------------------------------------- launches
// Bookkeeping around every kernel launch: launch count, optional CUDA-event
// timing of one named kernel.
struct LaunchScope {
  Sim *s;
  bool timed;
  LaunchScope(Sim *s, const char *name);
  ~LaunchScope();
};
// CUDA-event timing of a region of launches (one whole colour sweep, say),
// when the name being timed is the region's name exactly: one event before
// its first launch and one after its last, none between them (an event
// between two launches would end a programmatic dependence).  Region names
// hold a dot, which no kernel name does.
struct RegionScope {
  Sim *s;
  bool timed;
  RegionScope(Sim *s, const char *name);
  ~RegionScope();
};
// After an allocation has failed nothing more is launched for the
// realisation (its calls return DP_ENOMEM until it is destroyed), so no
// kernel can be handed a buffer that was never obtained.
#define DP_LAUNCH(sim, name, grid, block, smem, ...)                    \
  do {                                                                  \
    if ((sim)->alloc_failed) break;                                     \
    ::dp::LaunchScope ls__((sim), #name);                               \
    name<<<(grid), (block), (smem), (sim)->stream>>>(__VA_ARGS__);      \
  } while (0)

// A launch as a programmatic dependent of the kernel before it on the
// stream: its CTAs may be scheduled once every CTA of that kernel has
// triggered (griddepcontrol.launch_dependents) or exited, before that
// kernel's completion.  The kernel must execute griddep_wait() before it
// touches anything the kernel before it writes, and write nothing before
// it (launch_pdl, after Sim).  cls: kPdlWells, the level-0 well rows;
// kPdlCoarse, the kernels of the V-cycle's transfers and coarse levels;
// kPdlL0, level 0's pipelined colour kernels (Gauss-Seidel and residual);
// kPdlIluW, the ILU(0) forward sweep's long rows (the wells).
#define DP_LAUNCH_PDL(sim, cls, name, grid, block, smem, ...)                         \
  do {                                                                               \
    if ((sim)->alloc_failed) break;                                                  \
    ::dp::LaunchScope ls__((sim), #name);                                            \
    ::dp::launch_pdl((sim), (cls), name, dim3(grid), dim3(block), (smem), __VA_ARGS__); \
  } while (0)
constexpr int kPdlWells = 1, kPdlCoarse = 2, kPdlL0 = 8, kPdlIluW = 16;
// Waits until the grids this one depends on have completed and their
// writes are visible (a no-op in a kernel launched without the attribute).
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Lets the programmatic dependents of this grid be scheduled once every CTA
// has executed it (or exited); it orders nothing: they still wait in
// griddep_wait for this grid's completion.
__device__ __forceinline__ void griddep_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
// Which launches are programmatic dependents, a bit mask (the environment's
// DPSIM_PDL, by default all): the classes above, and 4, the dependents'
// own dependents let in as soon as they have passed their wait
// (pdl_trigger)
int pdl_mode();
inline bool pdl_trigger() { return (pdl_mode() & 4) != 0; }

// Storage order of the Krylov operator's copy: locations in chunks of
// kChunk; storage rows 2 kChunk c .. of chunk c hold its fracture rows (cells
// 2 loc), then its matrix rows (2 loc + 1); the well rows follow.  A warp
// streams rows of one kind and length from contiguous memory, and the
// storage rows of a chunk are, as a set, the natural rows 2 kChunk c .. of
// the same chunk, so a CTA of one chunk writes its outputs contiguously.
// nL = 0 (no matrix rows in the operator) gives the identity.
constexpr int kChunk = 64;
__host__ __device__ __forceinline__ int row_of_pair(int q, int nL, int nc) {
  if (q >= nc) return q;
  int c = q / (2 * kChunk), w = q - 2 * kChunk * c;
  int k = nL - kChunk * c < kChunk ? nL - kChunk * c : kChunk;   // locations of chunk c
  return w < k ? 2 * (kChunk * c + w) : 2 * (kChunk * c + w - k) + 1;
}
__host__ __device__ __forceinline__ int storage_row(int i, int nL, int nc) {
  if (i >= nc) return i;
  int loc = i >> 1, c = loc / kChunk, w = loc - kChunk * c;
  int k = nL - kChunk * c < kChunk ? nL - kChunk * c : kChunk;
  return 2 * kChunk * c + ((i & 1) ? k + w : w);
}

inline int nblk(long long n, int b = kBlock) {
  long long g = (n + b - 1) / b;
  return (int)(g > 0 ? g : 1);
}

// ---------------------------------------------------------------- kernels
// dp_phys.cu (compiled without FMA contraction: results must equal the
// oracle's bit for bit)
int phys_build_pattern(Sim *s);
int phys_save_old(Sim *s);
int phys_well_controls(Sim *s, bool restore);
int phys_well_rates(Sim *s, double *q);   // device q[2 nw]: oil rates, then water rates
int phys_assemble(Sim *s);
int phys_norms(Sim *s);
int phys_norm_weights(Sim *s);    // s->norm_w, once the porosities are on the device
int phys_decouple_extract(Sim *s);
int phys_decoupled_natural(Sim *s, double *out);
int phys_solver_view(Sim *s);     // K and the solver view, after phys_build_pattern
int phys_schur_reduce(Sim *s);    // K's values and residual from A and R (Schur option)
int phys_schur_back(Sim *s);      // the full update y from K's update
int phys_update(Sim *s);

// dp_sim.cu: the parts of a Newton step that the batched driver shares with
// sim_solve_step and sim_advance
int solve_prepare(Sim *s, double *eta, bool norms_current = false);
int solve_update(Sim *s, int rc);
int solve_finish(Sim *s, int rc, int it, double rr, double eta, float ms_setup, float ms_solve,
                 dp_stats *st);
void new_timestep(Sim *s);
int device_waits(Sim *s);   // DP_ETIMEOUT when a kernel's bounded wait gave up
int timestep_begin(Sim *s);
int timestep_restore(Sim *s);

// dp_amg.cu (integer setup and bit-exact smoothed-aggregation numerics)
int scan_i32(Sim *s, const int *in, int *out, int n, int *total);  // out[n] = total
int greedy_colour(Sim *s, int n, const int *rowptr, const int *col, int *colour,
                  int *ncolour);
int colour_lists(Sim *s, int n, const int *colour, int ncolour, int *clist,
                 std::vector<int> &cstart, int *iperm_or_null);
int amg_setup(Sim *s);
int amg_refresh(Sim *s);
int level_dinv(Sim *s, Level &L);
void amg_free(Sim *s);

// dp_la.cu (linear algebra of the Krylov loop and the preconditioner)
int ilu_setup(Sim *s);
int ilu_factor(Sim *s);
int ilu_apply(Sim *s, const double *r, double *z);
int bsr_spmv(Sim *s, const double *x, double *y);                 // y = A x
int bsr_residual(Sim *s, const double *b, const double *x, double *r);  // r = b - A x
int lin_residual(Sim *s);          // s->lq = R + A y, A the assembled Jacobian
// tpos[e] = position of entry (j, i) for every entry (i, j) of a structurally
// symmetric block pattern with sorted rows
int block_tpos(Sim *s, int n, const int *rowptr, const int *col, int *tpos);
int vcycle(Sim *s, int level, const double *b, double *x);
int coarse_factor(Sim *s);
int cpr_apply(Sim *s, const double *r, double *z);
int fgmres(Sim *s, double tol, int *iters, double *relres);
int la_alloc(Sim *s);
int mixed_refresh(Sim *s, bool coarse);
int l0_refresh(Sim *s, bool coarse);
int lanes_for(double mean_len);
void graphs_free(Sim *s);
int autotune(Sim *s, int reps, std::string &report);

// dp_cycle.cu (the coarse levels of the V-cycle in one cluster launch)
constexpr int kClusterMaxRows = 20000;   // default of dp_options.cluster_rows
int cluster_setup(Sim *s);
int cluster_refresh(Sim *s);
template <typename T> int coarse_cycle(Sim *s, int l0, const T *b, T *x);

struct Timing {
  int kernel_id = -1;            // hashed name being timed, -1 none
  std::string name;
  std::vector<cudaEvent_t> ev;   // pairs
  size_t used = 0;
  double ms = 0.0;
  int64_t launches = 0;
};

struct Sim {
  // problem
  Phys ph{};
  dp_options opt{};
  std::vector<dp_well> wells;
  int nperf = 0;
  cudaStream_t stream = nullptr;
  dp_allocator alloc{};
  bool own_alloc = true;
  std::vector<std::pair<void *, size_t>> blocks;
  size_t cur_bytes = 0, peak_bytes = 0;   // device bytes held through the allocator
  bool alloc_failed = false;              // the allocator returned NULL once (sticky)
  Err err;
  Timing timing;
  int64_t launches = 0;
  std::string last_error;

  // device: static data
  double *kf = nullptr, *km = nullptr, *phi_f = nullptr, *phi_m = nullptr;
  int *perf_cell = nullptr, *perf_well = nullptr;   // sorted by (cell, well)
  double *perf_wi = nullptr;
  int *well_kind = nullptr;                          // current controls (switched by
  double *well_target = nullptr;                     //   sim_advance)
  int *well_ctl_kind = nullptr;                      // the wells' own controls
  double *well_ctl_target = nullptr, *well_limit = nullptr;
  bool well_limits = false;                          // some well has a BHP limit
  std::vector<double> wi_host;                       // per perforation, well order
  Bsr A;                                             // Jacobian, decoupled in place
  double *trans = nullptr;                           // per entry: T or WI
  // device: state and residual
  double *p = nullptr, *sw = nullptr, *bhp = nullptr;
  double *pn = nullptr, *swn = nullptr, *bhpn = nullptr, *Mn = nullptr;
  double *R = nullptr, *bh = nullptr, *y = nullptr;
  double *pr = nullptr;                              // cell properties, 8 x nc (SoA)
  double *fconn = nullptr;   // per connection (3 faces a location, then its f-m link): F
  int *atpos = nullptr;      // position of the transposed block of each Jacobian entry
  double *Macc = nullptr;                            // phase masses at the iterate, 2 x nc
  double dt = 1.0, inv_dt = 1.0;
  double *norm_part = nullptr;                       // reduction partials
  double *norm_w = nullptr;                          // 1/(rho_ref phi_ref V), 2 x nc
  double *norm_out = nullptr;                        // 10 doubles (phys_norms)
  double *h_norms = nullptr;                         // pinned host copy
  int norm_blocks = 0;
  bool assembled = false, decoupled = false;
  // colouring of the block rows
  int *colour = nullptr;
  int ncolour = 0;
  // ILU(0) factor in (colour, index) row order
  int *perm = nullptr, *iperm = nullptr;
  int *lu_rowptr = nullptr, *lu_col = nullptr, *lu_src = nullptr, *lu_dpos = nullptr;
  double *lu_val = nullptr;
  float *lu_valf = nullptr;
  int *upd_ptr = nullptr, *upd_e2 = nullptr, *upd_q = nullptr;   // IKJ update lists
  // split layout of the factor: L blocks, inverted pivots, U blocks
  int lu_nL = 0;
  int *lu_Lptr = nullptr, *lu_Uptr = nullptr, *lu_dst = nullptr, *lu_colp = nullptr;
  double *ilu_zp = nullptr;       // colour-order work vector (2 nb values of the sweep type)
  double *ilu_zp2 = nullptr;      // the FP32 second application's result (2 nb floats)
  // maps of the decoupling's entry-parallel writes: natural row of each
  // entry, its block in the factor's split layout, its factor-order position
  int *erow = nullptr, *ilupos = nullptr, *l0pos = nullptr;
  // The system the linear solver sees: K is the assembled Jacobian A (full
  // system), or with the Schur option the fracture-and-well system whose
  // rows are the fracture cells (row loc) and the wells (row nL + w).  Its
  // storage-order copy maps storage row q to row row_of_pair(q, sv_sL,
  // sv_sc); rows below sv_cells are cell rows (decoupled), rows from
  // sv_long0 on are the long well rows.
  Bsr K;
  int sv_sL = 0, sv_sc = 0, sv_cells = 0, sv_long0 = 0;
  double *Rk = nullptr;           // residual of K's rows (R itself for the full system)
  double *yk = nullptr;           // update of K's rows (y itself for the full system)
  int *kmap = nullptr, *pos_fm = nullptr, *pos_mf = nullptr;   // Schur: entry maps
  double *Minv = nullptr;         // Schur: inverted matrix-cell block of each location
  double *fct = nullptr;          // per cell row: the weight w_i, or D_i^-1 (4 values, ABF)
  int *btpos = nullptr;           // transpose position of each block entry (True-IMPES)
  std::vector<int> lu_cstart;
  std::vector<int> lu_cmaxlen;   // longest row (blocks) of each colour
  // AMG hierarchy (level 0 shares the block pattern)
  std::vector<Level> lev;
  bool amg_ready = false;
  double *ap = nullptr;                              // pressure values (nnzb)
  // the decoupled matrix again in storage order (row_of_pair), with its
  // pressure rows (entries (0,0) and (0,1) of every block) as separate arrays
  int *srowptr = nullptr, *scol = nullptr;
  double *sval = nullptr, *sa00 = nullptr, *sa01 = nullptr;
  float *svalf = nullptr;   // precision 1: FP32 copy of sval (CPR stage residuals)
  float *spf = nullptr;     //   and the (a00, a01) pair of every block, FP32
  float *z1f = nullptr, *r1f = nullptr;   // FP32 stage vectors of the CPR preconditioner
  double *coarse_lu = nullptr;
  double *coarse_inv = nullptr;
  // level-0 pressure values in the colour order of the ILU(0) pattern (the
  // same greedy colouring), for contiguous Gauss-Seidel colour sweeps
  // Level 0 in colour order: when its Gauss-Seidel runs on the ILU(0)
  // colouring (l0_lu), the level's vectors are kept in that colour order, so
  // that the sweeps, the residual and the transfers stream them contiguously
  // (natural order would read each at stride 2: one location's fracture and
  // matrix rows fall in different colours).
  bool l0c = false;
  int *l0_colp = nullptr;                                 // colour position of each column
  // the colour positions of the stage operator copy's columns (scol), so
  // that the FP32 stage residuals gather z1 and z2 in the ILU(0) colour
  // order (precision >= 1, level 0 in colour order); z2c: z2 in that order
  int *scolc = nullptr;
  float *z2c = nullptr;
  int *r0_colp = nullptr;                                 // R0's columns, colour positions
  int *p0c_rowptr = nullptr, *p0c_col = nullptr, *p0c_src = nullptr;  // P0, rows in colour order
  double *p0c_val = nullptr, *dinv_c = nullptr;
  float *p0c_valf = nullptr, *dinv_cf = nullptr;
  bool l0_lu = false;
  int l0_G = 1;       // lanes per row of the level-0 colour-order sweeps (autotuned; 1: a thread)
  int shapes = 0;     // bumped whenever launch shapes change (autotune, AMG set-up)
  double *l0_pv = nullptr;
  float *l0_pvf = nullptr;   // inverse from the LU factors (n <= kInverseMax), row-major
  int *coarse_piv = nullptr;
  int coarse_n = 0;
  int cl_level = -1, cl_size = 0;                    // first level of the cluster cycle
  void *cl_lev64 = nullptr, *cl_lev32 = nullptr;     // device level descriptors
  double *omega = nullptr;                           // device scalars
  unsigned long long *rho_bits = nullptr;
  int *counter = nullptr, *h_counter = nullptr;      // device / pinned host
  // Krylov workspace
  int m = 30;
  double *V = nullptr, *Z = nullptr, *w = nullptr;
  double *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *hy = nullptr;
  double *dots_part = nullptr, *dots = nullptr, *scal = nullptr;
  double *h_res = nullptr;                           // pinned host scalars
  int dot_blocks = 0;
  double *z1 = nullptr, *r1 = nullptr, *rp = nullptr, *xp = nullptr;
  // CUDA graphs of the FGMRES iterations j = 0..m-1 (captured on first use)
  std::vector<cudaGraphExec_t> graph;
  std::vector<long long> graph_launches;
  cudaStream_t cap_stream = nullptr;
  // Newton bookkeeping
  double prev_res = 0.0;
  int newton_iter = 0;
  double last_norms[10] = {0};
  // forcing terms 1-2 (Section 3.1): the linear residual lq = R + A y of the
  // last solve (A as assembled), valid from the second Newton iteration on
  double *lq = nullptr;
  bool have_lq = false;
  dp_stats last{};

  // device flag of the bounded waits (set by a kernel whose wait gave up)
  int *dev_err = nullptr;
  unsigned *tickets = nullptr;   // the last-CTA tickets of the long-row tails (zeroed)
  bool waits_used = false;   // a kernel with bounded waits ran since the flag was read

  // Records a failure's message; a CUDA failure or a device wait that gave
  // up also marks the realisation unusable (every later call returns that
  // code), other codes do not.
  void fail(int code, const std::string &m) {
    if ((code == DP_ECUDA || code == DP_ETIMEOUT) && err.code == 0) { err.code = code; err.msg = m; }
    last_error = m;
  }
};

template <typename... P, typename... A>
inline void launch_pdl(Sim *s, int cls, void (*k)(P...), dim3 grid, dim3 block, size_t smem,
                       A &&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = (pdl_mode() & cls) ? 1 : 0;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
  if (e != cudaSuccess) s->fail(DP_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
}

}  // namespace dp

// The opaque handle of the C ABI is the library's realisation.
struct dp_sim : dp::Sim {};
