// Batched Newton steps of many realisations (batch_create / batch_advance,
// include/dpsim.h).  The realisations advance in lockstep: each Newton
// iteration assembles and sets up every realisation still iterating (a pool
// of host threads, each realisation on its own stream), then runs their
// FGMRES iterations together on the batch's stream, one launch per phase of
// the Arnoldi step over a work list of (realisation, block) tiles.  A tile runs the
// kernel body of dp_kernels.cuh with the block index and grid size of the
// realisation's own launch, so every realisation computes exactly what it
// computes alone (sim_advance), whatever else is in the batch.  Each
// launch's work list (a segment table passed by value) holds only the
// realisations still iterating, so a launch costs the work left, not the
// batch's size.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "dp_internal.h"
#include "dp_kernels.cuh"

namespace dp {

struct Tile {
  int m, bx;   // realisation, block of its own launch
};

// The realisations of one batched launch, passed by value: the active ones
// (those a launch covers), and the first block of each in the launch; a
// block finds its realisation by bisection.  At most kMaxBatch realisations.
constexpr int kMaxBatch = 256;
struct Seg {
  int n;
  int start[kMaxBatch + 1];
  short id[kMaxBatch];
};

// ---------------------------------------------------------------- argument records
// One record per realisation for each phase; gx is the grid of the
// realisation's own launch, `js` strides add j (the Arnoldi column) times
// the stride to a base pointer.
struct ALuF {   // ILU(0) forward sweep of one colour
  int var;      // 0 copy (first colour), 1 two lanes per row, 2 warp per row, 3 warp + pivots
  int gx, r0, r1, nL;
  const int *perm, *Lptr, *colp;
  const float *lu;
  const void *rhs;
  long long rjs;
  float *zp;
};
struct ALuB {   // ILU(0) backward sweep of one colour
  int var;      // 0 thread per row, 1 warp per row
  int gx, r0, r1, nL, n;
  const int *Uptr, *colp;
  const float *lu;
  float *zp;
};
struct ARes {   // result gather of the ILU(0) work vector
  int gx, n;
  const int *iperm;
  const float *zp;
  const double *base;
  double *out;
  long long ojs;
  float *outT;
  const float *inj;
  int inj_perm;
};
struct APres {  // pressure rows of b - A x, FP32 pairs
  int gx, n, nL, nc, nlong;
  const int *rowptr, *col;
  const float2 *pf;
  const float *x;
  const double *b;
  long long bjs;
  float *rp;
  const int *omap;
};
struct AResid {  // b - A x, FP32 copy of the operator
  int gx, n, nL, nc, nlong;
  const int *rowptr, *col;
  const float *valf;
  const float *x;
  const double *b;
  long long bjs;
  float *y;
};
struct AFillF { int gx; long long n; float *x; };
struct ACopyF { int gx; long long n; const float *src; float *dst; };
struct AGsC {   // level-0 Gauss-Seidel colour in colour order
  int var;      // 0 first colour from zero, 1 G lanes per row, 2 warp per row
  int G, gx, r0, r1;
  const int *rowptr, *colp;
  const float *pv, *dinv, *b;
  float *x;
};
struct AResC {  // level-0 residual rows in colour order
  int var;      // 0 G lanes per row, 1 warp per row
  int G, gx, r0, r1;
  const int *rowptr, *colp;
  const float *pv, *b;
  float *x, *r;
};
struct ACsr {   // y (+)= A x, G lanes per row, values FP32 or BF16
  int G, gx, n;
  const int *rowptr, *col;
  const float *val;
  const __nv_bfloat16 *valh;
  const float *x;
  float *y;
  int add;
};
struct AJac {   // l1-Jacobi: pre-smoothing (x, r out) or a sweep (r out)
  int G, gx, n;
  const int *rowptr, *col;
  const float *val;
  const __nv_bfloat16 *valh;
  const float *d, *b;
  float *x, *r;
};
struct ADense { int gx, n; const double *inv; const float *b; float *x; };
struct AInj { int gx, n; const float *xp; float *zf; const int *imap; };
struct ASpmv {  // FP64 operator product (MODE 0) or residual (MODE 1)
  int gx, n, nL, nc, nlong;
  const int *rowptr, *col;
  const double *val;
  const double *x;
  long long xjs;
  const double *b;
  double *y;
};
struct ADot {   // partial dot products of V_0.. against w
  int gx;
  long long N;
  const double *V;
  long long ldv;
  const double *w;
  double *part;
  const double *gate;
};
struct ADotF {  // their fixed-order sum
  int nblocks;
  const double *part;
  double *dots, *H;
  int m;
  double *scal;
  double reorth;
  double *dst;   // mode 0 (a norm's square): its slot
};
struct AProj { int gx; long long N; const double *V; long long ldv; const double *c; double *w; const double *scal; };
struct AGiv { double *H, *cs, *sn, *g; int m; double *scal; };
struct ABack { const double *H, *g; int m; double *y; const int *jend; };
struct AAxpy { int gx; long long N; const double *Z; long long ldv; const double *c; double *x; const int *jend; };
struct AScale { int gx; long long N; const double *src; const double *alpha; double *y; };
struct AFillD { int gx; long long n; double *x; };
struct AInitG { double *g; int m; const double *beta; };
struct ASqrt { double *v; };
struct AGather { const double *scal; double *out; };

#define TILE(A)                                                   \
  int lo_ = 0, hi_ = seg.n;                                       \
  while (hi_ - lo_ > 1) {                                         \
    int mid_ = (lo_ + hi_) >> 1;                                  \
    if (seg.start[mid_] <= (int)blockIdx.x) lo_ = mid_;           \
    else hi_ = mid_;                                              \
  }                                                               \
  Tile t{seg.id[lo_], (int)blockIdx.x - seg.start[lo_]};          \
  const A &a = args[t.m];

// ---------------------------------------------------------------- batched kernels
#define KB_SWITCH_G(G, CALL)                          \
  switch (G) {                                        \
    case 1: { constexpr int GG = 1; CALL; } break;    \
    case 2: { constexpr int GG = 2; CALL; } break;    \
    case 4: { constexpr int GG = 4; CALL; } break;    \
    case 8: { constexpr int GG = 8; CALL; } break;    \
    case 16: { constexpr int GG = 16; CALL; } break;  \
    default: { constexpr int GG = 32; CALL; } break;  \
  }

template <typename TR>
__global__ void __launch_bounds__(kBlock) kb_ilu_fwd(const ALuF *args, const Seg seg, int j) {
  TILE(ALuF)
  const TR *rhs = reinterpret_cast<const TR *>(a.rhs) + (long long)j * a.rjs;
  switch (a.var) {
    case 0: k_ilu_fwd_copy_b<float, TR>(t.bx, a.gx, a.r0, a.r1, a.perm, rhs, a.zp); break;
    case 1: k_ilu_fwd_b<float, TR>(t.bx, a.gx, a.r0, a.r1, a.perm, a.Lptr, a.colp, a.lu, rhs, a.zp); break;
    case 2:
      k_ilu_fwd_w_b<float, TR, false>(t.bx, a.gx, a.r0, a.r1, a.nL, a.perm, a.Lptr, a.colp, a.lu,
                                      rhs, a.zp);
      break;
    default:
      k_ilu_fwd_w_b<float, TR, true>(t.bx, a.gx, a.r0, a.r1, a.nL, a.perm, a.Lptr, a.colp, a.lu,
                                     rhs, a.zp);
  }
}

__global__ void __launch_bounds__(kBlock) kb_ilu_bwd(const ALuB *args, const Seg seg, int) {
  TILE(ALuB)
  if (a.var == 0) k_ilu_bwd_r_b<float>(t.bx, a.gx, a.r0, a.r1, a.nL, a.n, a.Uptr, a.colp, a.lu, a.zp);
  else k_ilu_bwd_w_b<float>(t.bx, a.gx, a.r0, a.r1, a.nL, a.n, a.Uptr, a.colp, a.lu, a.zp);
}

__global__ void __launch_bounds__(kBlock) kb_ilu_result(const ARes *args, const Seg seg, int j) {
  TILE(ARes)
  k_ilu_result_b<float>(t.bx, a.gx, a.n, a.iperm, a.zp, a.base, a.out + (long long)j * a.ojs,
                        a.outT, a.inj, a.inj_perm);
}

__global__ void __launch_bounds__(kBlock) kb_presid(const APres *args, const Seg seg, int j) {
  TILE(APres)
  k_bsr_presid_f32_b(t.bx, a.gx, a.n, a.nL, a.nc, a.nlong, a.rowptr, a.col, a.pf, a.x,
                     a.b + (long long)j * a.bjs, a.rp, a.omap, X0Init{});
}

__global__ void __launch_bounds__(kBlock) kb_resid(const AResid *args, const Seg seg, int j) {
  TILE(AResid)
  k_bsr_resid_f32_b(t.bx, a.gx, a.n, a.nL, a.nc, a.nlong, a.rowptr, a.col, a.valf, a.x,
                    a.b + (long long)j * a.bjs, a.y);
}

__global__ void __launch_bounds__(kBlock) kb_fill_f(const AFillF *args, const Seg seg, int) {
  TILE(AFillF)
  long long i = (long long)t.bx * blockDim.x + threadIdx.x;
  if (i < a.n) a.x[i] = 0.f;
}

__global__ void __launch_bounds__(kBlock) kb_copy_f(const ACopyF *args, const Seg seg, int) {
  TILE(ACopyF)
  long long i = (long long)t.bx * blockDim.x + threadIdx.x;
  if (i < a.n) a.dst[i] = a.src[i];
}

__global__ void __launch_bounds__(kBlock) kb_gs_c(const AGsC *args, const Seg seg, int) {
  TILE(AGsC)
  if (a.var == 0) {
    k_gs_c_first_b<float>(t.bx, a.gx, a.r0, a.r1, a.dinv, a.b, a.x);
  } else if (a.var == 1) {
    if (a.G == 1) k_gs_c_b<float>(t.bx, a.gx, a.r0, a.r1, a.rowptr, a.colp, a.pv, a.dinv, a.b, a.x);
    else if (a.G == 0)
      k_sweep_cs_b<float, false>(t.bx, a.gx, a.r0, a.r1, a.rowptr, a.colp, a.pv, a.dinv, a.b, a.x,
                                 nullptr);
    else
      KB_SWITCH_G(a.G, (k_gs_cg_b<GG, float>(t.bx, a.gx, a.r0, a.r1, a.rowptr, a.colp, a.pv,
                                              a.dinv, a.b, a.x)))
  } else {
    k_gs_c_w_b<float>(t.bx, a.gx, a.r0, a.r1, a.rowptr, a.colp, a.pv, a.dinv, a.b, a.x);
  }
}

__global__ void __launch_bounds__(kBlock) kb_resid_c(const AResC *args, const Seg seg, int) {
  TILE(AResC)
  if (a.var == 0) {
    if (a.G == 1) k_resid_c_b<float>(t.bx, a.gx, a.r0, a.r1, a.rowptr, a.colp, a.pv, a.b, a.x, a.r);
    else if (a.G == 0)
      k_sweep_cs_b<float, true>(t.bx, a.gx, a.r0, a.r1, a.rowptr, a.colp, a.pv, nullptr, a.b, a.x,
                                a.r);
    else
      KB_SWITCH_G(a.G, (k_resid_cg_b<GG, float>(t.bx, a.gx, a.r0, a.r1, a.rowptr, a.colp, a.pv,
                                                 a.b, a.x, a.r)))
  } else {
    k_resid_c_w_b<float>(t.bx, a.gx, a.r0, a.r1, a.rowptr, a.colp, a.pv, a.b, a.x, a.r);
  }
}


__global__ void __launch_bounds__(kBlock) kb_csr_mv(const ACsr *args, const Seg seg, int) {
  TILE(ACsr)
  if (a.valh)
    KB_SWITCH_G(a.G, (k_csr_mv_b<GG, float, __nv_bfloat16>(t.bx, a.gx, a.n, a.rowptr, a.col,
                                                             a.valh, a.x, a.y, a.add)))
  else
    KB_SWITCH_G(a.G, (k_csr_mv_b<GG, float>(t.bx, a.gx, a.n, a.rowptr, a.col, a.val, a.x, a.y,
                                             a.add)))
}

__global__ void __launch_bounds__(kBlock) kb_jacobi_pre(const AJac *args, const Seg seg, int) {
  TILE(AJac)
  if (a.valh)
    KB_SWITCH_G(a.G, (k_jacobi_pre_b<GG, float, __nv_bfloat16>(t.bx, a.gx, a.n, a.rowptr, a.col,
                                                                 a.valh, a.d, a.b, a.x, a.r)))
  else
    KB_SWITCH_G(a.G, (k_jacobi_pre_b<GG, float>(t.bx, a.gx, a.n, a.rowptr, a.col, a.val, a.d, a.b,
                                                 a.x, a.r)))
}

__global__ void __launch_bounds__(kBlock) kb_jacobi_sweep(const AJac *args, const Seg seg, int) {
  TILE(AJac)
  if (a.valh)
    KB_SWITCH_G(a.G, (k_jacobi_sweep_b<GG, float, __nv_bfloat16>(t.bx, a.gx, a.n, a.rowptr, a.col,
                                                                   a.valh, a.d, a.b, a.x, a.r)))
  else
    KB_SWITCH_G(a.G, (k_jacobi_sweep_b<GG, float>(t.bx, a.gx, a.n, a.rowptr, a.col, a.val, a.d,
                                                   a.b, a.x, a.r)))
}

__global__ void __launch_bounds__(kBlock) kb_dense_mv(const ADense *args, const Seg seg, int) {
  TILE(ADense)
  k_dense_mv_b<float>(t.bx, a.gx, a.n, a.inv, a.b, a.x);
}

__global__ void __launch_bounds__(kBlock) kb_inject(const AInj *args, const Seg seg, int) {
  TILE(AInj)
  k_inject_f32_b(t.bx, a.gx, a.n, a.xp, a.zf, a.imap);
}

template <int MODE>
__global__ void __launch_bounds__(kBlock) kb_spmv(const ASpmv *args, const Seg seg, int j) {
  TILE(ASpmv)
  k_bsr_spmv_b<MODE>(t.bx, a.gx, a.n, a.nL, a.nc, a.nlong, a.rowptr, a.col, a.val,
                     a.x + (long long)j * a.xjs, a.b, a.y);
}

// v0: the first vector of this chunk of V
template <int NV, bool SELF>
__global__ void __launch_bounds__(kBlock, kDotBlocks / 152) kb_multidot(const ADot *args,
                                                                        const Seg seg,
                                                                        int v0) {
  TILE(ADot)
  k_multidot_b<NV, SELF>(t.bx, a.gx, a.N, a.V + (long long)v0 * a.ldv, a.ldv, a.w, a.part, v0,
                         a.gate);
}

__global__ void __launch_bounds__(kBlock) kb_dot_final(const ADotF *args, const Seg seg, int nv, int j,
                                                       int mode) {
  TILE(ADotF)
  double *dots = mode == 0 ? a.dst : a.dots;
  k_dot_final_b(t.bx, 1, a.part, a.nblocks, nv, dots, a.H, a.m, j, mode, a.scal, a.reorth);
}

__global__ void __launch_bounds__(kBlock) kb_project(const AProj *args, const Seg seg, int j, int pass) {
  TILE(AProj)
  k_project_b(t.bx, a.gx, a.N, a.V, a.ldv, j + 1, a.c, a.w, const_cast<double *>(a.V) + (long long)(j + 1) * a.ldv,
              a.scal, pass);
}

__global__ void __launch_bounds__(kBlock) kb_givens(const AGiv *args, const Seg seg, int j) {
  TILE(AGiv)
  k_givens_b(t.bx, 1, a.H, a.cs, a.sn, a.g, a.m, j, a.scal + 3);
}

__global__ void __launch_bounds__(kBlock) kb_backsub(const ABack *args, const Seg seg, int) {
  TILE(ABack)
  k_backsub_b(t.bx, 1, a.H, a.g, a.m, a.jend[t.m], a.y);
}

__global__ void __launch_bounds__(kBlock) kb_multi_axpy(const AAxpy *args, const Seg seg, int) {
  TILE(AAxpy)
  k_multi_axpy_b(t.bx, a.gx, a.N, a.Z, a.ldv, a.jend[t.m], a.c, 1.0, a.x);
}

__global__ void __launch_bounds__(kBlock) kb_scale(const AScale *args, const Seg seg, int) {
  TILE(AScale)
  k_scale_b(t.bx, a.gx, a.N, a.src, a.alpha, 1, a.y);
}

__global__ void __launch_bounds__(kBlock) kb_fill_d(const AFillD *args, const Seg seg, int) {
  TILE(AFillD)
  long long i = (long long)t.bx * blockDim.x + threadIdx.x;
  if (i < a.n) a.x[i] = 0.0;
}

__global__ void __launch_bounds__(kBlock) kb_init_g(const AInitG *args, const Seg seg, int) {
  TILE(AInitG)
  k_init_g_b(t.bx, 1, a.g, a.m, a.beta);
}

__global__ void __launch_bounds__(kBlock) kb_sqrt(const ASqrt *args, const Seg seg, int) {
  TILE(ASqrt)
  if (threadIdx.x == 0) k_sqrt_inplace_b(t.bx, 1, a.v);
}

// scal[0..3] of every realisation into one array for a single copy to the host
__global__ void __launch_bounds__(kBlock) kb_gather(const AGather *args, const Seg seg, int) {
  TILE(AGather)
  if (threadIdx.x < 4) a.out[4 * t.m + threadIdx.x] = a.scal[threadIdx.x];
}

// ---------------------------------------------------------------- phases
// A phase: one batched launch; its argument records (one per realisation)
// live in device memory from the batch's set-up, its work list is made at
// each launch from the realisations active then.
struct Phase {
  int kind = 0;
  void *args = nullptr;
  std::vector<int> grid;    // blocks of each realisation's own launch (0: not in it)
  int p0 = 0, p1 = 0;       // kind-specific uniform parameters (a template choice)
};

enum Kind {
  K_ILU_FWD_D, K_ILU_FWD_F, K_ILU_BWD, K_ILU_RES, K_PRES, K_RESID, K_FILL_F, K_COPY_F, K_GS_C,
  K_RES_C, K_CSR, K_JAC_PRE, K_JAC_SWEEP, K_DENSE, K_INJ, K_SPMV0, K_SPMV1, K_DOT, K_DOT_FINAL,
  K_PROJECT, K_GIVENS, K_BACKSUB, K_AXPY, K_SCALE, K_FILL_D, K_INIT_G, K_SQRT, K_GATHER
};

}  // namespace dp

struct dp_batch {
  std::vector<dp::Sim *> m;
  cudaStream_t stream = nullptr;
  int nm = 0, mres = 30, maxit = 300;
  bool built = false;
  std::vector<int> shapes;   // each member's Sim::shapes when the plan was built
  // the batch's own device memory (cudaMalloc: it never touches a member's
  // allocator, so that it can be released after its members)
  std::vector<void *> blocks;
  // activity masks: the Arnoldi step's, and two for the restart prologue
  // the active realisations of the Arnoldi step (s), of the first cycle's
  // start (a) and of a restart (b); host arrays from which each launch's
  // work list is made
  std::vector<unsigned char> h_act;
  // jend per realisation for the cycle's end (host copy pageable, so that
  // an upload is staged before cudaMemcpyAsync returns)
  std::vector<int> h_jend;
  int *jend = nullptr;
  double *gath = nullptr, *h_gath = nullptr;   // scal[0..3] of every member
  double *h_norms = nullptr;                   // 10 norms of every member
  // phases
  std::vector<dp::Phase> step;         // one Arnoldi step (column j)
  dp::Phase norm_b[3];                  // ||b||: multidot, final (into scal[0]), sqrt
  dp::Phase rst[4];                     // restart residual, multidot, final (scal[1]), sqrt
  dp::Phase scale_b, scale_r, fill_x, fill_h, init_g0, init_g1;
  dp::Phase backsub, axpy, gather;
  std::string err;
  int64_t launches = 0;
  // captured Arnoldi steps: key (column j, activity mask) -> the executable
  // graph and the launches it holds; the same Newton rounds recur with the
  // same masks in every timestep, so the cache is replayed from the second on
  std::map<std::string, std::pair<cudaGraphExec_t, int64_t>> graphs;
  // the per-realisation parts (assembly, set-up, update) run on the
  // realisations' own streams from a pool of host threads
  std::vector<cudaEvent_t> ev;   // per realisation: its set-up is queued
  cudaEvent_t solved = nullptr;  // the batched FGMRES is queued
  int device = 0;
  std::vector<std::thread> workers;
  std::mutex mu;
  std::condition_variable cv, done_cv;
  std::function<void(int)> task;
  int ntask = 0, generation = 0, busy = 0;
  std::atomic<int> next{0};
  bool quit = false;
  // host wall time (ms) since creation: the per-realisation parts (assembly
  // and set-up; update), the batched FGMRES; lockstep counts
  double ms_setup = 0.0, ms_fgmres = 0.0, ms_update = 0.0;
  int64_t newton_rounds = 0, arnoldi_steps = 0, cycles = 0;
};

namespace dp {

static void graphs_clear(dp_batch *b) {
  for (auto &g : b->graphs) cudaGraphExecDestroy(g.second.first);
  b->graphs.clear();
}

static void *balloc(dp_batch *b, size_t bytes) {
  void *p = nullptr;
  if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) return nullptr;
  b->blocks.push_back(p);
  return p;
}

template <typename A>
static int add_phase(dp_batch *b, Phase &ph, int kind, const std::vector<A> &args,
                     const std::vector<int> &grid, int p0 = 0, int p1 = 0) {
  ph.kind = kind;
  ph.p0 = p0;
  ph.p1 = p1;
  ph.grid = grid;
  ph.args = balloc(b, sizeof(A) * std::max(b->nm, 1));
  if (!ph.args) return DP_ENOMEM;
  if (cudaMemcpyAsync(ph.args, args.data(), sizeof(A) * b->nm, cudaMemcpyHostToDevice,
                      b->stream) != cudaSuccess)
    return DP_ECUDA;
  return DP_OK;
}

// The work list of a launch: the realisations flagged in `act` (host) that
// take part in the phase, with their first blocks.  Returns the blocks.
static int make_seg(dp_batch *b, const Phase &ph, const unsigned char *act, Seg &sg) {
  sg.n = 0;
  int total = 0;
  for (int k = 0; k < b->nm; ++k) {
    if (!act[k] || ph.grid[k] <= 0) continue;
    sg.id[sg.n] = (short)k;
    sg.start[sg.n] = total;
    total += ph.grid[k];
    ++sg.n;
  }
  sg.start[sg.n] = total;
  return total;
}

static int launch(dp_batch *b, const Phase &ph, const unsigned char *act, int j) {
  Seg sg;
  int nbl = make_seg(b, ph, act, sg);
  if (nbl == 0) return DP_OK;
  dim3 g(nbl), t(kBlock);
  cudaStream_t st = b->stream;
#define KB(name, A, ...) name<<<g, t, 0, st>>>(reinterpret_cast<const A *>(ph.args), sg, __VA_ARGS__)
  switch (ph.kind) {
    case K_ILU_FWD_D: KB(kb_ilu_fwd<double>, ALuF, j); break;
    case K_ILU_FWD_F: KB(kb_ilu_fwd<float>, ALuF, j); break;
    case K_ILU_BWD: KB(kb_ilu_bwd, ALuB, j); break;
    case K_ILU_RES: KB(kb_ilu_result, ARes, j); break;
    case K_PRES: KB(kb_presid, APres, j); break;
    case K_RESID: KB(kb_resid, AResid, j); break;
    case K_FILL_F: KB(kb_fill_f, AFillF, j); break;
    case K_COPY_F: KB(kb_copy_f, ACopyF, j); break;
    case K_GS_C: KB(kb_gs_c, AGsC, j); break;
    case K_RES_C: KB(kb_resid_c, AResC, j); break;
    case K_CSR: KB(kb_csr_mv, ACsr, j); break;
    case K_JAC_PRE: KB(kb_jacobi_pre, AJac, j); break;
    case K_JAC_SWEEP: KB(kb_jacobi_sweep, AJac, j); break;
    case K_DENSE: KB(kb_dense_mv, ADense, j); break;
    case K_INJ: KB(kb_inject, AInj, j); break;
    case K_SPMV0: KB(kb_spmv<0>, ASpmv, j); break;
    case K_SPMV1: KB(kb_spmv<1>, ASpmv, j); break;
    case K_DOT: {
      // p0: vectors in this chunk (1..8), p1: SELF; the chunk's first vector is passed as j
      int v0 = j;
#define KB_DOT(NVC)                                                                   \
  case NVC:                                                                           \
    if (ph.p1) KB((kb_multidot<NVC, true>), ADot, v0); else KB((kb_multidot<NVC, false>), ADot, v0); \
    break;
      switch (ph.p0) { KB_DOT(1) KB_DOT(2) KB_DOT(3) KB_DOT(4) KB_DOT(5) KB_DOT(6) KB_DOT(7) KB_DOT(8) }
#undef KB_DOT
      break;
    }
    case K_PROJECT: KB(kb_project, AProj, j, ph.p0); break;
    case K_GIVENS: KB(kb_givens, AGiv, j); break;
    case K_BACKSUB: KB(kb_backsub, ABack, j); break;
    case K_AXPY: KB(kb_multi_axpy, AAxpy, j); break;
    case K_SCALE: KB(kb_scale, AScale, j); break;
    case K_FILL_D: KB(kb_fill_d, AFillD, j); break;
    case K_INIT_G: KB(kb_init_g, AInitG, j); break;
    case K_SQRT: KB(kb_sqrt, ASqrt, j); break;
    case K_GATHER: KB(kb_gather, AGather, j); break;
    default: break;
  }
#undef KB
  b->launches += 1;
  return cudaGetLastError() == cudaSuccess ? DP_OK : DP_ECUDA;
}

// the dot-product final sum for nv vectors of column j in `mode` (a launch
// parameter, not a record field)
static int launch_final(dp_batch *b, const Phase &ph, const unsigned char *act, int nv, int j,
                        int mode) {
  Seg sg;
  int nbl = make_seg(b, ph, act, sg);
  if (nbl == 0) return DP_OK;
  kb_dot_final<<<nbl, kBlock, 0, b->stream>>>(reinterpret_cast<const ADotF *>(ph.args), sg, nv, j,
                                              mode);
  b->launches += 1;
  return cudaGetLastError() == cudaSuccess ? DP_OK : DP_ECUDA;
}

// ---------------------------------------------------------------- the plan
// Which realisations the batch takes: the FP32 preconditioner (precision 1
// or 2) with CPR-FPF, the level-0 Gauss-Seidel in the ILU(0) colour order,
// l1-Jacobi below level 0, the coarsest level by its explicit inverse, the
// coarse levels not in the cluster kernel, equal FGMRES restart and limit.
static const char *unsupported(const Sim *s, const Sim *s0) {
  const dp_options &o = s->opt;
  if (o.precond != 2) return "the batch needs the CPR-FPF preconditioner (precond 2)";
  if (o.precision < 1) return "the batch needs the FP32 preconditioner (precision 1 or 2)";
  if (o.amg_gs_levels > 1) return "the batch needs l1-Jacobi below AMG level 0 (amg_gs_levels <= 1)";
  if (o.cluster_rows >= 0 && o.use_graphs)
    return "the batch needs the V-cycle outside the cluster kernel (cluster_rows < 0)";
  if (o.gmres_restart != s0->opt.gmres_restart || o.gmres_maxit != s0->opt.gmres_maxit)
    return "the realisations of a batch need equal gmres_restart and gmres_maxit";
  if (s->amg_ready) {
    if (s->lev.size() < 2) return "a realisation with one AMG level";
    if (!s->l0c || s->cl_level >= 0) return "a realisation whose level 0 is not in colour order";
    const Level &Lc = s->lev.back();
    if (!s->coarse_inv || s->coarse_n != Lc.n) return "a realisation without the coarsest inverse";
    for (size_t l = 1; l + 1 < s->lev.size(); ++l)
      if (!s->lev[l].l1) return "a realisation with Gauss-Seidel below level 0";
  }
  return nullptr;
}

// per realisation, the ILU(0) sweeps as (variant, r0, r1, grid) in order
struct Sweep { int var, r0, r1, grid; };
static void ilu_sweeps(const Sim *s, std::vector<Sweep> &fwd, std::vector<Sweep> &bwd) {
  int nc = s->ncolour;
  int last = nc - 1;
  while (last >= 0 && s->lu_cstart[last + 1] <= s->lu_cstart[last]) --last;
  int first = 0;
  while (first < nc && s->lu_cstart[first + 1] <= s->lu_cstart[first]) ++first;
  for (int c = 0; c < nc; ++c) {
    int r0 = s->lu_cstart[c], r1 = s->lu_cstart[c + 1];
    if (r1 <= r0) continue;
    bool lng = s->lu_cmaxlen[c] > kLongRow;
    if (c == last && lng) fwd.push_back({3, r0, r1, nblk(32LL * (r1 - r0))});
    else if (lng) fwd.push_back({2, r0, r1, nblk(32LL * (r1 - r0))});
    else if (c == first) fwd.push_back({0, r0, r1, nblk((r1 - r0 + kRes - 1) / kRes)});
    else fwd.push_back({1, r0, r1, nblk(2LL * (r1 - r0))});
  }
  for (int c = nc - 1; c >= 0; --c) {
    int r0 = s->lu_cstart[c], r1 = s->lu_cstart[c + 1];
    if (r1 <= r0) continue;
    bool lng = s->lu_cmaxlen[c] > kLongRow;
    if (c == last && lng) continue;
    if (lng) bwd.push_back({1, r0, r1, nblk(32LL * (r1 - r0))});
    else bwd.push_back({0, r0, r1, nblk((r1 - r0 + kRes - 1) / kRes)});
  }
}

// level-0 Gauss-Seidel colours (forward, from zero when pre-smoothing) and
// the residual's runs, as in gs_sweep_c and resid_c
// Lanes per row of a member's level-0 colour kernels inside the batch: the
// member's own choice, except that the pipelined persistent kernel (-1; a
// launch walks one member's tiles) runs as the thread-per-row kernel, whose
// results are the same bit for bit.
static int batch_lanes(int l0_G) { return l0_G < 0 ? 1 : l0_G; }

static void gs_colours(const Sim *s, bool forward, bool from_zero, std::vector<Sweep> &out) {
  int nc = s->ncolour;
  bool first = from_zero;
  for (int t = 0; t < nc; ++t) {
    int c = forward ? t : nc - 1 - t;
    int r0 = s->lu_cstart[c], r1 = s->lu_cstart[c + 1];
    if (r1 <= r0) continue;
    if (first) { first = false; out.push_back({0, r0, r1, nblk(r1 - r0)}); continue; }
    if (s->lu_cmaxlen[c] > kLongRow) out.push_back({2, r0, r1, nblk(32LL * (r1 - r0))});
    else out.push_back({1, r0, r1, nblk((long long)(r1 - r0) * std::max(s->l0_G, 1))});
  }
}
static void resid_runs(const Sim *s, std::vector<Sweep> &out) {
  int nc = s->ncolour, c = 0;
  while (c < nc) {
    int r0 = s->lu_cstart[c];
    bool lng = s->lu_cmaxlen[c] > kLongRow;
    int c1 = c + 1;
    while (c1 < nc && (s->lu_cmaxlen[c1] > kLongRow) == lng) ++c1;
    int r1 = s->lu_cstart[c1];
    if (r1 > r0)
      out.push_back({lng ? 1 : 0, r0, r1,
                     lng ? nblk(32LL * (r1 - r0)) : nblk((long long)(r1 - r0) * std::max(s->l0_G, 1))});
    c = c1;
  }
}

template <typename A>
static int phase_from(dp_batch *b, int kind, const std::vector<std::vector<std::pair<A, int>>> &per,
                      size_t t, int p0 = 0, int p1 = 0) {
  std::vector<A> args(b->nm);
  std::vector<int> grid(b->nm, 0);
  for (int k = 0; k < b->nm; ++k)
    if (t < per[k].size()) { args[k] = per[k][t].first; grid[k] = per[k][t].second; }
  Phase ph;
  DP_TRY(add_phase(b, ph, kind, args, grid, p0, p1));
  b->step.push_back(ph);
  return DP_OK;
}

// The ILU(0) application (LU)^-1 rhs into each realisation's work vector:
// rhs_js = 2 nb for the Arnoldi column v_j, else 0; TR the rhs type.
static int plan_ilu(dp_batch *b, bool rhs_double, std::vector<const void *> rhs,
                    std::vector<long long> rjs) {
  size_t nf = 0, nbw = 0;
  std::vector<std::vector<std::pair<ALuF, int>>> F(b->nm);
  std::vector<std::vector<std::pair<ALuB, int>>> B(b->nm);
  for (int k = 0; k < b->nm; ++k) {
    Sim *s = b->m[k];
    std::vector<Sweep> fw, bw;
    ilu_sweeps(s, fw, bw);
    for (auto &w : fw) {
      ALuF a{};
      a.var = w.var; a.gx = w.grid; a.r0 = w.r0; a.r1 = w.r1; a.nL = s->lu_nL;
      a.perm = s->perm; a.Lptr = s->lu_Lptr; a.colp = s->lu_colp; a.lu = s->lu_valf;
      a.rhs = rhs[k]; a.rjs = rjs[k]; a.zp = reinterpret_cast<float *>(s->ilu_zp);
      F[k].push_back({a, w.grid});
    }
    for (auto &w : bw) {
      ALuB a{};
      a.var = w.var; a.gx = w.grid; a.r0 = w.r0; a.r1 = w.r1; a.nL = s->lu_nL; a.n = s->K.n;
      a.Uptr = s->lu_Uptr; a.colp = s->lu_colp; a.lu = s->lu_valf;
      a.zp = reinterpret_cast<float *>(s->ilu_zp);
      B[k].push_back({a, w.grid});
    }
    nf = std::max(nf, F[k].size());
    nbw = std::max(nbw, B[k].size());
  }
  for (size_t t = 0; t < nf; ++t) DP_TRY(phase_from(b, rhs_double ? K_ILU_FWD_D : K_ILU_FWD_F, F, t));
  for (size_t t = 0; t < nbw; ++t) DP_TRY(phase_from(b, K_ILU_BWD, B, t));
  return DP_OK;
}

template <typename A>
static int one_phase(dp_batch *b, std::vector<Phase> *into, Phase *ph, int kind,
                     const std::vector<A> &args, const std::vector<int> &grid, int p0 = 0,
                     int p1 = 0) {
  Phase q;
  DP_TRY(add_phase(b, q, kind, args, grid, p0, p1));
  if (into) into->push_back(q);
  if (ph) *ph = q;
  return DP_OK;
}

// the whole plan: the Arnoldi step (as cpr_apply and arnoldi_step run it for
// the FP32 preconditioner) and the pieces of the restart cycle
static int build_plan(dp_batch *b) {
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return DP_ECUDA;
  graphs_clear(b);   // they hold the old records' addresses
  for (void *p : b->blocks) cudaFree(p);
  b->blocks.clear();
  b->step.clear();
  int nm = b->nm;
  std::vector<int> one(nm, 1), gridN(nm), gridNb(nm), dotg(nm);
  std::vector<long long> Ns(nm);
  for (int k = 0; k < nm; ++k) {
    Sim *s = b->m[k];
    long long N = 2LL * s->K.n;
    Ns[k] = N;
    gridN[k] = (int)std::min<long long>(nblk(N), kDotBlocks * 4);
    gridNb[k] = nblk(N);
    dotg[k] = dot_blocks(N);
  }
  // ---- z_j = M v_j: ILU(0) of v_j
  {
    std::vector<const void *> rhs(nm);
    std::vector<long long> rjs(nm);
    for (int k = 0; k < nm; ++k) { rhs[k] = b->m[k]->V; rjs[k] = Ns[k]; }
    DP_TRY(plan_ilu(b, true, rhs, rjs));
  }
  {  // z1 (FP64 and FP32) from the work vector
    std::vector<ARes> a(nm);
    std::vector<int> g(nm);
    for (int k = 0; k < nm; ++k) {
      Sim *s = b->m[k];
      int n = s->K.n;
      a[k] = ARes{nblk((n + kRes - 1) / kRes), n, s->iperm, reinterpret_cast<const float *>(s->ilu_zp),
                  nullptr, s->z1, 0, s->z1f, nullptr, 0};
      g[k] = a[k].gx;
    }
    DP_TRY(one_phase(b, &b->step, nullptr, K_ILU_RES, a, g));
  }
  {  // pressure rows of v_j - A z1 into level 0's right-hand side (colour order)
    std::vector<APres> a(nm);
    std::vector<int> g(nm);
    for (int k = 0; k < nm; ++k) {
      Sim *s = b->m[k];
      a[k] = APres{1 + nblk(s->sv_long0), s->K.n, s->sv_sL, s->sv_sc, s->sv_long0, s->srowptr,
                   s->scol, reinterpret_cast<const float2 *>(s->spf), s->z1f, s->V, Ns[k],
                   s->lev[0].bf, s->iperm};
      g[k] = a[k].gx;
    }
    DP_TRY(one_phase(b, &b->step, nullptr, K_PRES, a, g));
  }
  // ---- the V-cycle from level 0 (colour order)
  {
    std::vector<AFillF> a(nm);
    std::vector<int> g(nm);
    for (int k = 0; k < nm; ++k) {
      Level &L = b->m[k]->lev[0];
      a[k] = AFillF{nblk(L.n), L.n, L.xf};
      g[k] = a[k].gx;
    }
    DP_TRY(one_phase(b, &b->step, nullptr, K_FILL_F, a, g));
  }
  auto gs_phases = [&](bool forward, bool from_zero) -> int {
    std::vector<std::vector<std::pair<AGsC, int>>> P(nm);
    size_t np = 0;
    for (int k = 0; k < nm; ++k) {
      Sim *s = b->m[k];
      std::vector<Sweep> cs;
      gs_colours(s, forward, from_zero, cs);
      for (auto &w : cs) {
        AGsC a{w.var, batch_lanes(s->l0_G), w.grid, w.r0, w.r1, s->lu_rowptr, s->l0_colp, s->l0_pvf,
               s->dinv_cf, s->lev[0].bf, s->lev[0].xf};
        P[k].push_back({a, w.grid});
      }
      np = std::max(np, P[k].size());
    }
    for (size_t t = 0; t < np; ++t) DP_TRY(phase_from(b, K_GS_C, P, t));
    return DP_OK;
  };
  DP_TRY(gs_phases(true, true));
  {
    std::vector<std::vector<std::pair<AResC, int>>> P(nm);
    size_t np = 0;
    for (int k = 0; k < nm; ++k) {
      Sim *s = b->m[k];
      std::vector<Sweep> rs;
      resid_runs(s, rs);
      for (auto &w : rs) {
        AResC a{w.var, batch_lanes(s->l0_G), w.grid, w.r0, w.r1, s->lu_rowptr, s->l0_colp, s->l0_pvf,
                s->lev[0].bf, s->lev[0].xf, s->lev[0].rf};
        P[k].push_back({a, w.grid});
      }
      np = std::max(np, P[k].size());
    }
    for (size_t t = 0; t < np; ++t) DP_TRY(phase_from(b, K_RES_C, P, t));
  }
  {  // restriction from level 0: R0 with its columns in colour order
    std::vector<ACsr> a(nm);
    std::vector<int> g(nm);
    for (int k = 0; k < nm; ++k) {
      Sim *s = b->m[k];
      Level &L = s->lev[0], &N = s->lev[1];
      a[k] = ACsr{L.r_G, nblk((long long)N.n * L.r_G), N.n, L.r_rowptr, s->r0_colp, L.r_valf,
                  nullptr, L.rf, N.bf, 0};
      g[k] = a[k].gx;
    }
    DP_TRY(one_phase(b, &b->step, nullptr, K_CSR, a, g));
  }
  int maxlev = 0;
  for (int k = 0; k < nm; ++k) maxlev = std::max(maxlev, (int)b->m[k]->lev.size());
  // down: levels 1.. (pre-smoothing and restriction; the coarsest by its inverse)
  for (int l = 1; l < maxlev; ++l) {
    std::vector<AJac> pre(nm);
    std::vector<ACsr> rr(nm);
    std::vector<ADense> dn(nm);
    std::vector<int> gp(nm, 0), gr(nm, 0), gd(nm, 0);
    for (int k = 0; k < nm; ++k) {
      Sim *s = b->m[k];
      int last = (int)s->lev.size() - 1;
      if (l > last) continue;
      Level &L = s->lev[l];
      if (l == last) {
        dn[k] = ADense{nblk(32LL * L.n), L.n, s->coarse_inv, L.bf, L.xf};
        gd[k] = dn[k].gx;
        continue;
      }
      Level &N = s->lev[l + 1];
      pre[k] = AJac{L.G, nblk((long long)L.n * L.G), L.n, L.rowptr, L.col, L.valf, L.valh,
                    L.dinvf, L.bf, L.xf, L.rf};
      gp[k] = pre[k].gx;
      rr[k] = ACsr{L.r_G, nblk((long long)N.n * L.r_G), N.n, L.r_rowptr, L.r_col, L.r_valf,
                   L.r_valh, L.rf, N.bf, 0};
      gr[k] = rr[k].gx;
    }
    DP_TRY(one_phase(b, &b->step, nullptr, K_JAC_PRE, pre, gp));
    DP_TRY(one_phase(b, &b->step, nullptr, K_CSR, rr, gr));
    DP_TRY(one_phase(b, &b->step, nullptr, K_DENSE, dn, gd));
  }
  // up: prolongation and post-smoothing, coarse to fine
  for (int l = maxlev - 2; l >= 1; --l) {
    std::vector<ACsr> pp(nm);
    std::vector<AJac> post(nm);
    std::vector<ACopyF> cp(nm);
    std::vector<int> gpp(nm, 0), gpo(nm, 0), gc(nm, 0);
    for (int k = 0; k < nm; ++k) {
      Sim *s = b->m[k];
      int last = (int)s->lev.size() - 1;
      if (l >= last) continue;
      Level &L = s->lev[l], &N = s->lev[l + 1];
      pp[k] = ACsr{L.p_G, nblk((long long)L.n * L.p_G), L.n, L.p_rowptr, L.p_col, L.p_valf,
                   L.p_valh, N.xf, L.xf, 1};
      gpp[k] = pp[k].gx;
      post[k] = AJac{L.G, nblk((long long)L.n * L.G), L.n, L.rowptr, L.col, L.valf, L.valh,
                     L.dinvf, L.bf, L.xf, L.rf};
      gpo[k] = post[k].gx;
      cp[k] = ACopyF{nblk(L.n), L.n, L.rf, L.xf};
      gc[k] = cp[k].gx;
    }
    DP_TRY(one_phase(b, &b->step, nullptr, K_CSR, pp, gpp));
    DP_TRY(one_phase(b, &b->step, nullptr, K_JAC_SWEEP, post, gpo));
    DP_TRY(one_phase(b, &b->step, nullptr, K_COPY_F, cp, gc));
  }
  {  // prolongation to level 0 (rows in colour order), post-smoothing backward
    std::vector<ACsr> a(nm);
    std::vector<int> g(nm);
    for (int k = 0; k < nm; ++k) {
      Sim *s = b->m[k];
      Level &L = s->lev[0], &N = s->lev[1];
      a[k] = ACsr{L.p_G, nblk((long long)L.n * L.p_G), L.n, s->p0c_rowptr, s->p0c_col,
                  s->p0c_valf, nullptr, N.xf, L.xf, 1};
      g[k] = a[k].gx;
    }
    DP_TRY(one_phase(b, &b->step, nullptr, K_CSR, a, g));
  }
  DP_TRY(gs_phases(false, false));
  {  // the coarse correction into the FP32 z1
    std::vector<AInj> a(nm);
    std::vector<int> g(nm);
    for (int k = 0; k < nm; ++k) {
      Sim *s = b->m[k];
      a[k] = AInj{nblk(s->K.n), s->K.n, s->lev[0].xf, s->z1f, s->iperm};
      g[k] = a[k].gx;
    }
    DP_TRY(one_phase(b, &b->step, nullptr, K_INJ, a, g));
  }
  {  // v_j - A z2 in FP32
    std::vector<AResid> a(nm);
    std::vector<int> g(nm);
    for (int k = 0; k < nm; ++k) {
      Sim *s = b->m[k];
      a[k] = AResid{1 + nblk(2LL * s->sv_long0), s->K.n, s->sv_sL, s->sv_sc, s->sv_long0,
                    s->srowptr, s->scol, s->svalf, s->z1f, s->V, Ns[k], s->r1f};
      g[k] = a[k].gx;
    }
    DP_TRY(one_phase(b, &b->step, nullptr, K_RESID, a, g));
  }
  {
    std::vector<const void *> rhs(nm);
    std::vector<long long> rjs(nm, 0);
    for (int k = 0; k < nm; ++k) rhs[k] = b->m[k]->r1f;
    DP_TRY(plan_ilu(b, false, rhs, rjs));
  }
  {  // z_j = z2 + F (v_j - A z2), z2 = z1 + P e
    std::vector<ARes> a(nm);
    std::vector<int> g(nm);
    for (int k = 0; k < nm; ++k) {
      Sim *s = b->m[k];
      int n = s->K.n;
      a[k] = ARes{nblk((n + kRes - 1) / kRes), n, s->iperm, reinterpret_cast<const float *>(s->ilu_zp),
                  s->z1, s->Z, Ns[k], nullptr, s->lev[0].xf, 1};
      g[k] = a[k].gx;
    }
    DP_TRY(one_phase(b, &b->step, nullptr, K_ILU_RES, a, g));
  }
  // ---- w = A z_j, Gram-Schmidt, Givens
  {
    std::vector<ASpmv> a(nm);
    std::vector<int> g(nm);
    for (int k = 0; k < nm; ++k) {
      Sim *s = b->m[k];
      a[k] = ASpmv{1 + nblk(2LL * s->sv_long0), s->K.n, s->sv_sL, s->sv_sc, s->sv_long0, s->srowptr,
                   s->scol, s->sval, s->Z, Ns[k], nullptr, s->w};
      g[k] = a[k].gx;
    }
    DP_TRY(one_phase(b, &b->step, nullptr, K_SPMV0, a, g));
  }
  // the dot phases of the step are launched by run_step with the chunking of
  // column j; their records are these (V, w, partials, with and without gate)
  std::vector<ADot> d0(nm), d1(nm), dn(nm), dr(nm);
  std::vector<ADotF> f(nm), fn(nm), fr(nm);
  std::vector<AProj> pj(nm);
  std::vector<AGiv> gv(nm);
  std::vector<ABack> bs(nm);
  std::vector<AAxpy> ax(nm);
  std::vector<AScale> scb(nm), scr(nm);
  std::vector<AFillD> fx(nm), fh(nm);
  std::vector<AInitG> ig0(nm), ig1(nm);
  std::vector<ASqrt> sq0(nm), sq1(nm);
  std::vector<AGather> ga(nm);
  std::vector<ASpmv> rs(nm);
  std::vector<int> gsp(nm), gfh(nm), gfx(nm);
  for (int k = 0; k < nm; ++k) {
    Sim *s = b->m[k];
    long long N = Ns[k];
    d0[k] = ADot{dotg[k], N, s->V, N, s->w, s->dots_part, nullptr};
    d1[k] = ADot{dotg[k], N, s->V, N, s->w, s->dots_part, s->scal + 4};
    dn[k] = ADot{dotg[k], N, s->bh, 0, s->bh, s->dots_part, nullptr};
    dr[k] = ADot{dotg[k], N, s->V, 0, s->V, s->dots_part, nullptr};
    f[k] = ADotF{dotg[k], s->dots_part, s->dots, s->H, s->m, s->scal, s->opt.reorth, nullptr};
    fn[k] = ADotF{dotg[k], s->dots_part, s->dots, s->H, s->m, s->scal, 0.0, s->scal + 0};
    fr[k] = ADotF{dotg[k], s->dots_part, s->dots, s->H, s->m, s->scal, 0.0, s->scal + 1};
    pj[k] = AProj{gridN[k], N, s->V, N, s->dots, s->w, s->scal};
    gv[k] = AGiv{s->H, s->cs, s->sn, s->g, s->m, s->scal};
    bs[k] = ABack{s->H, s->g, s->m, s->hy, b->jend};
    ax[k] = AAxpy{gridN[k], N, s->Z, N, s->hy, s->yk, b->jend};
    scb[k] = AScale{gridNb[k], N, s->bh, s->scal + 0, s->V};
    scr[k] = AScale{gridNb[k], N, s->V, s->scal + 1, s->V};
    fx[k] = AFillD{gridNb[k], N, s->yk};
    long long nh = (long long)(s->m + 1) * s->m;
    fh[k] = AFillD{nblk(nh), nh, s->H};
    gfh[k] = fh[k].gx;
    gfx[k] = gridNb[k];
    ig0[k] = AInitG{s->g, s->m, s->scal + 0};
    ig1[k] = AInitG{s->g, s->m, s->scal + 1};
    sq0[k] = ASqrt{s->scal + 0};
    sq1[k] = ASqrt{s->scal + 1};
    ga[k] = AGather{s->scal, b->gath};
    rs[k] = ASpmv{1 + nblk(2LL * s->sv_long0), s->K.n, s->sv_sL, s->sv_sc, s->sv_long0, s->srowptr,
                  s->scol, s->sval, s->yk, 0, s->bh, s->V};
    gsp[k] = rs[k].gx;
  }
  Phase pd0, pd1, pf, pp, pg;
  DP_TRY(one_phase(b, nullptr, &pd0, K_DOT, d0, dotg));
  DP_TRY(one_phase(b, nullptr, &pd1, K_DOT, d1, dotg));
  DP_TRY(one_phase(b, nullptr, &pf, K_DOT_FINAL, f, one));
  DP_TRY(one_phase(b, nullptr, &pp, K_PROJECT, pj, gridN));
  DP_TRY(one_phase(b, nullptr, &pg, K_GIVENS, gv, one));
  // the step's tail is kept as five phases at the end of `step`: dots without
  // gate, dots with gate, final, project, Givens (run_step launches them)
  b->step.push_back(pd0);
  b->step.push_back(pd1);
  b->step.push_back(pf);
  b->step.push_back(pp);
  b->step.push_back(pg);
  DP_TRY(one_phase(b, nullptr, &b->norm_b[0], K_DOT, dn, dotg, 1, 0));
  DP_TRY(one_phase(b, nullptr, &b->norm_b[1], K_DOT_FINAL, fn, one));
  DP_TRY(one_phase(b, nullptr, &b->norm_b[2], K_SQRT, sq0, one));
  DP_TRY(one_phase(b, nullptr, &b->rst[0], K_SPMV1, rs, gsp));
  DP_TRY(one_phase(b, nullptr, &b->rst[1], K_DOT, dr, dotg, 1, 0));
  DP_TRY(one_phase(b, nullptr, &b->rst[2], K_DOT_FINAL, fr, one));
  DP_TRY(one_phase(b, nullptr, &b->rst[3], K_SQRT, sq1, one));
  DP_TRY(one_phase(b, nullptr, &b->scale_b, K_SCALE, scb, gridNb));
  DP_TRY(one_phase(b, nullptr, &b->scale_r, K_SCALE, scr, gridNb));
  DP_TRY(one_phase(b, nullptr, &b->fill_x, K_FILL_D, fx, gfx));
  DP_TRY(one_phase(b, nullptr, &b->fill_h, K_FILL_D, fh, gfh));
  DP_TRY(one_phase(b, nullptr, &b->init_g0, K_INIT_G, ig0, one));
  DP_TRY(one_phase(b, nullptr, &b->init_g1, K_INIT_G, ig1, one));
  DP_TRY(one_phase(b, nullptr, &b->backsub, K_BACKSUB, bs, one));
  DP_TRY(one_phase(b, nullptr, &b->axpy, K_AXPY, ax, gridN));
  DP_TRY(one_phase(b, nullptr, &b->gather, K_GATHER, ga, one));
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return DP_ECUDA;
  b->shapes.assign(nm, 0);
  for (int k = 0; k < nm; ++k) b->shapes[k] = b->m[k]->shapes;
  b->built = true;
  return DP_OK;
}

// One Arnoldi step for column j over the realisations flagged in act:
// every phase of cpr_apply and arnoldi_step, then the scalars gathered.
static int run_step(dp_batch *b, int j, const unsigned char *act) {
  size_t ntail = 5;
  size_t nbody = b->step.size() - ntail;
  for (size_t p = 0; p < nbody; ++p) DP_TRY(launch(b, b->step[p], act, j));
  const Phase &pd0 = b->step[nbody], &pd1 = b->step[nbody + 1], &pf = b->step[nbody + 2],
              &pp = b->step[nbody + 3], &pg = b->step[nbody + 4];
  int nv = j + 1;
  // first Gram-Schmidt pass (with w.w), its final sum in mode 3, projection
  for (int pass = 0; pass < 2; ++pass) {
    const Phase &pd = pass == 0 ? pd0 : pd1;
    for (int v0 = 0; v0 < nv; v0 += kDotVec) {
      Phase q = pd;
      q.p0 = std::min(kDotVec, nv - v0);
      q.p1 = v0 == 0 ? 1 : 0;
      DP_TRY(launch(b, q, act, v0));
    }
    DP_TRY(launch_final(b, pf, act, nv, j, pass == 0 ? 3 : 4));
    Phase q = pp;
    q.p0 = pass;
    DP_TRY(launch(b, q, act, j));
  }
  DP_TRY(launch(b, pg, act, j));
  DP_TRY(launch(b, b->gather, act, 0));
  return DP_OK;
}

// run_step through the graph cache: captured the first time a (j, mask)
// comes (thread-local capture: the member streams' host threads keep
// working meanwhile), replayed after; on the legacy default stream (which
// cannot be captured) the launches are made directly
constexpr size_t kMaxGraphs = 4096;
static int run_step_graph(dp_batch *b, int j, const unsigned char *act) {
  // the legacy default stream cannot be captured: launch directly there
  if (b->stream == nullptr || b->stream == cudaStreamLegacy) return run_step(b, j, act);
  std::string key(reinterpret_cast<const char *>(&j), sizeof j);
  key.append(reinterpret_cast<const char *>(act), (size_t)b->nm);
  auto it = b->graphs.find(key);
  if (it == b->graphs.end()) {
    if (b->graphs.size() >= kMaxGraphs) graphs_clear(b);
    int64_t l0 = b->launches;
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return DP_ECUDA;
    int rc = run_step(b, j, act);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (rc != DP_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return rc != DP_OK ? rc : DP_ECUDA;
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return DP_ECUDA;
    it = b->graphs.emplace(key, std::make_pair(ex, b->launches - l0)).first;
    b->launches = l0;
  }
  if (cudaGraphLaunch(it->second.first, b->stream) != cudaSuccess) return DP_ECUDA;
  b->launches += it->second.second;
  return DP_OK;
}

static int fetch_gather(dp_batch *b) {
  if (cudaMemcpyAsync(b->h_gath, b->gath, 32 * (size_t)b->nm, cudaMemcpyDeviceToHost, b->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return DP_ECUDA;
  return DP_OK;
}

// FGMRES of fgmres() for the realisations `in` (with their tolerances), in
// lockstep: the same restart cycles, Arnoldi steps and stopping tests per
// realisation.  rc/it/rr receive each one's outcome.
static int batch_fgmres(dp_batch *b, const std::vector<int> &in, const std::vector<double> &tol,
                        std::vector<int> &rc, std::vector<int> &it, std::vector<double> &rr) {
  int nm = b->nm;
  unsigned char *hs = b->h_act.data(), *ha = hs + nm, *hb = hs + 2 * nm;
  const unsigned char *act = hs, *act_a = ha, *act_b = hb;
  std::vector<int> total(nm, 0), jend(nm, 0);
  std::vector<char> conv(nm, 0), live(nm, 0), stop(nm, 0);
  std::vector<double> bnorm(nm, 0.0), res(nm, 0.0);
  for (int k : in) live[k] = 1;
  // x = 0, ||b|| into scal[0]
  for (int k = 0; k < nm; ++k) hs[k] = live[k], ha[k] = 0, hb[k] = 0;
  DP_TRY(launch(b, b->fill_x, act, 0));
  DP_TRY(launch(b, b->norm_b[0], act, 0));
  DP_TRY(launch_final(b, b->norm_b[1], act, 1, 0, 0));
  DP_TRY(launch(b, b->norm_b[2], act, 0));
  DP_TRY(launch(b, b->gather, act, 0));
  DP_TRY(fetch_gather(b));
  for (int k : in) {
    bnorm[k] = b->h_gath[4 * k + 0];
    res[k] = bnorm[k];
    if (bnorm[k] == 0.0) { conv[k] = 1; res[k] = 0.0; }
  }
  auto running = [&](int k) { return live[k] && !conv[k] && !stop[k] && total[k] < b->maxit; };
  for (;;) {
    // the members that start (or restart) a cycle
    std::vector<int> cyc;
    for (int k = 0; k < nm; ++k) if (running(k)) cyc.push_back(k);
    if (cyc.empty()) break;
    // restart residual of those with total > 0: r = b - A x, ||r|| into scal[1]
    bool any_r = false;
    for (int k = 0; k < nm; ++k) {
      hs[k] = 0;
      ha[k] = 0;
      hb[k] = 0;
    }
    for (int k : cyc) { if (total[k] > 0) { hb[k] = 1; any_r = true; } }
    if (any_r) {
      for (int p = 0; p < 2; ++p) DP_TRY(launch(b, b->rst[p], act_b, 0));
      DP_TRY(launch_final(b, b->rst[2], act_b, 1, 0, 0));
      DP_TRY(launch(b, b->rst[3], act_b, 0));
      DP_TRY(launch(b, b->gather, act_b, 0));
      DP_TRY(fetch_gather(b));
    }
    std::vector<int> go;
    for (int k : cyc) {
      double beta = total[k] > 0 ? b->h_gath[4 * k + 1] : bnorm[k];
      res[k] = beta;
      if (beta <= tol[k] * bnorm[k]) { conv[k] = 1; continue; }
      go.push_back(k);
    }
    if (go.empty()) continue;
    for (int k = 0; k < nm; ++k) { hs[k] = 0; ha[k] = 0; hb[k] = 0; }
    for (int k : go) { if (total[k] > 0) hb[k] = 1; else ha[k] = 1; hs[k] = 1; }
    DP_TRY(launch(b, b->scale_b, act_a, 0));
    DP_TRY(launch(b, b->scale_r, act_b, 0));
    DP_TRY(launch(b, b->fill_h, act, 0));
    DP_TRY(launch(b, b->init_g0, act_a, 0));
    DP_TRY(launch(b, b->init_g1, act_b, 0));
    for (int k : go) jend[k] = 0;
    ++b->cycles;
    std::vector<char> in_cycle(nm, 0);
    for (int k : go) in_cycle[k] = 1;
    for (int j = 0; j < b->mres; ++j) {
      bool any = false;
      for (int k = 0; k < nm; ++k) {
        hs[k] = in_cycle[k] && total[k] < b->maxit;
        any = any || hs[k];
      }
      if (!any) break;
      DP_TRY(run_step_graph(b, j, act));
      ++b->arnoldi_steps;
      DP_TRY(fetch_gather(b));
      for (int k = 0; k < nm; ++k) {
        if (!hs[k]) continue;
        ++total[k];
        jend[k] = j + 1;
        double hn = b->h_gath[4 * k + 2];
        res[k] = b->h_gath[4 * k + 3];
        if (res[k] <= tol[k] * bnorm[k]) { conv[k] = 1; in_cycle[k] = 0; }
        else if (hn == 0.0) in_cycle[k] = 0;
      }
    }
    // x += Z y for the members of the cycle
    for (int k = 0; k < nm; ++k) { hs[k] = 0; b->h_jend[k] = jend[k]; }
    for (int k : go) hs[k] = 1;
    if (cudaMemcpyAsync(b->jend, b->h_jend.data(), 4 * (size_t)nm, cudaMemcpyHostToDevice, b->stream) !=
        cudaSuccess)
      return DP_ECUDA;
    DP_TRY(launch(b, b->backsub, act, 0));
    DP_TRY(launch(b, b->axpy, act, 0));
    for (int k : go) if (jend[k] == 0) stop[k] = 1;
  }
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return DP_ECUDA;
  for (int k : in) {
    rc[k] = conv[k] ? DP_OK : DP_ELINEAR;
    it[k] = total[k];
    rr[k] = bnorm[k] > 0.0 ? res[k] / bnorm[k] : 0.0;
  }
  return DP_OK;
}

}  // namespace dp

using namespace dp;

static int bfail(dp_batch *b, int rc, const std::string &msg) {
  if (b) b->err = msg;
  return rc;
}

// The worker pool: run(fn, n) calls fn(0..n-1) on the workers (each index
// once) and returns when all are done.
static void worker_main(dp_batch *b) {
  cudaSetDevice(b->device);
  int seen = 0;
  for (;;) {
    std::function<void(int)> fn;
    int n = 0;
    {
      std::unique_lock<std::mutex> lk(b->mu);
      b->cv.wait(lk, [&] { return b->quit || b->generation != seen; });
      if (b->quit) return;
      seen = b->generation;
      fn = b->task;
      n = b->ntask;
    }
    for (;;) {
      int k = b->next.fetch_add(1);
      if (k >= n) break;
      fn(k);
    }
    std::lock_guard<std::mutex> lk(b->mu);
    if (--b->busy == 0) b->done_cv.notify_all();
  }
}

static void pool_run(dp_batch *b, int n, const std::function<void(int)> &fn) {
  if (n <= 0) return;
  if (b->workers.empty()) {
    for (int k = 0; k < n; ++k) fn(k);
    return;
  }
  std::unique_lock<std::mutex> lk(b->mu);
  b->task = fn;
  b->ntask = n;
  b->next.store(0);
  b->busy = (int)b->workers.size();
  ++b->generation;
  b->cv.notify_all();
  b->done_cv.wait(lk, [&] { return b->busy == 0; });
}

extern "C" int batch_create(dp_sim *const *sims, int32_t n, void *stream, dp_batch **out) {
  if (!out) return DP_EINVAL;
  *out = nullptr;
  if (n < 1 || !sims) return DP_EINVAL;
  for (int k = 0; k < n; ++k) {
    if (!sims[k]) return DP_EINVAL;
    for (int q = 0; q < k; ++q)
      if (sims[q] == sims[k]) return DP_EINVAL;
    if (unsupported(sims[k], sims[0])) return DP_EINVAL;
  }
  dp_batch *b = new (std::nothrow) dp_batch();
  if (!b) return DP_ENOMEM;
  b->nm = n;
  b->stream = (cudaStream_t)stream;
  for (int k = 0; k < n; ++k) b->m.push_back(static_cast<Sim *>(sims[k]));
  b->mres = b->m[0]->m;
  b->maxit = b->m[0]->opt.gmres_maxit;
  if (n > kMaxBatch) {
    delete b;
    return DP_EINVAL;
  }
  if (cudaMalloc(&b->jend, 4 * (size_t)n) != cudaSuccess ||
      cudaMalloc(&b->gath, 32 * (size_t)n) != cudaSuccess) {
    batch_destroy(b);
    return DP_ENOMEM;
  }
  b->h_act.assign(3 * (size_t)n, 0);
  b->h_jend.assign(n, 0);
  cudaGetDevice(&b->device);
  b->ev.assign(n, nullptr);
  for (int k = 0; k < n; ++k)
    if (cudaEventCreateWithFlags(&b->ev[k], cudaEventDisableTiming) != cudaSuccess) {
      batch_destroy(b);
      return DP_ECUDA;
    }
  if (cudaEventCreateWithFlags(&b->solved, cudaEventDisableTiming) != cudaSuccess) {
    batch_destroy(b);
    return DP_ECUDA;
  }
  int nw = std::min(n, 16);
  for (int k = 0; k < nw && n > 1; ++k) b->workers.emplace_back(worker_main, b);
  if (cudaMallocHost(&b->h_gath, 32 * (size_t)n) != cudaSuccess ||
      cudaMallocHost(&b->h_norms, 80 * (size_t)n) != cudaSuccess) {
    batch_destroy(b);
    return DP_ECUDA;
  }
  *out = b;
  return DP_OK;
}

// Touches neither the members nor the batch's stream (either may be gone
// already); cudaFree waits for the device.
extern "C" void batch_destroy(dp_batch *b) {
  if (!b) return;
  {
    std::lock_guard<std::mutex> lk(b->mu);
    b->quit = true;
  }
  b->cv.notify_all();
  for (std::thread &t : b->workers) t.join();
  for (cudaEvent_t e : b->ev)
    if (e) cudaEventDestroy(e);
  if (b->solved) cudaEventDestroy(b->solved);
  for (void *p : b->blocks) cudaFree(p);
  if (b->jend) cudaFree(b->jend);
  if (b->gath) cudaFree(b->gath);
  if (b->h_gath) cudaFreeHost(b->h_gath);
  if (b->h_norms) cudaFreeHost(b->h_norms);
  dp::graphs_clear(b);
  delete b;
}

extern "C" const char *batch_last_error(const dp_batch *b) { return b ? b->err.c_str() : ""; }

extern "C" int batch_profile(const dp_batch *b, double *ms3, int64_t *counts3) {
  if (!b) return DP_EINVAL;
  if (ms3) { ms3[0] = b->ms_setup; ms3[1] = b->ms_fgmres; ms3[2] = b->ms_update; }
  if (counts3) { counts3[0] = b->newton_rounds; counts3[1] = b->cycles; counts3[2] = b->arnoldi_steps; }
  return DP_OK;
}

extern "C" int64_t batch_launch_count(const dp_batch *b) {
  if (!b) return 0;
  int64_t n = b->launches;
  for (Sim *s : b->m) n += s->launches;
  return n;
}

extern "C" int batch_advance(dp_batch *b, const double *dt, dp_stats *stats, int32_t *status) {
  if (!b || !dt) return DP_EINVAL;
  int nm = b->nm;
  for (int k = 0; k < nm; ++k)
    if (!(dt[k] > 0.0)) return DP_EINVAL;
  for (Sim *s : b->m) {
    if (s->err.code == DP_ECUDA) return bfail(b, DP_ECUDA, "a realisation is unusable");
    if (s->alloc_failed) return bfail(b, DP_ENOMEM, "a realisation's allocator failed");
  }
  std::vector<int> rc(nm, DP_OK), lin(nm, 0), perr(nm, DP_OK);
  std::vector<char> newton(nm, 1), conv(nm, 0), linfail(nm, 0), solving(nm, 0), rebuilt(nm, 0);
  std::vector<double> res0(nm, 0.0), res(nm, 0.0), eta(nm, 0.0);
  std::vector<std::string> why(nm);
  std::vector<int> all(nm);
  for (int k = 0; k < nm; ++k) all[k] = k;
  pool_run(b, nm, [&](int k) { perr[k] = timestep_begin(b->m[k]); });
  for (int k = 0; k < nm; ++k)
    if (perr[k] != DP_OK) return bfail(b, perr[k], "timestep set-up");
  int newton_max = b->m[0]->opt.newton_max;
  for (int l = 0; l <= newton_max; ++l) {
    std::vector<int> iter;
    for (int k = 0; k < nm; ++k) if (newton[k]) iter.push_back(k);
    if (iter.empty()) break;
    // assembly, convergence test and set-up of each realisation, on its own
    // stream; the batch's stream then waits for every set-up
    using clk = std::chrono::steady_clock;
    auto ms_since = [](clk::time_point t0) {
      return std::chrono::duration<double, std::milli>(clk::now() - t0).count();
    };
    auto t0 = clk::now();
    ++b->newton_rounds;
    pool_run(b, (int)iter.size(), [&](int q) {
      int k = iter[q];
      Sim *s = b->m[k];
      solving[k] = 0;
      int r = sim_assemble(static_cast<dp_sim *>(s), dt[k]);
      if (r == DP_OK &&
          (cudaMemcpyAsync(b->h_norms + 10 * k, s->norm_out, 80, cudaMemcpyDeviceToHost,
                           s->stream) != cudaSuccess ||
           cudaStreamSynchronize(s->stream) != cudaSuccess))
        r = DP_ECUDA;
      if (r != DP_OK) { perr[k] = r; return; }
      std::memcpy(s->last_norms, b->h_norms + 10 * k, 80);
      res[k] = s->last_norms[0];
      if (l == 0) res0[k] = res[k];
      const dp_options &o = s->opt;
      if (res[k] <= o.newton_tol * res0[k] || s->last_norms[1] <= o.newton_atol) {
        conv[k] = 1;
        newton[k] = 0;
        return;
      }
      if (l == o.newton_max) { newton[k] = 0; return; }
      bool had = s->amg_ready;
      r = solve_prepare(s, &eta[k], true);
      if (r == DP_OK && cudaEventRecord(b->ev[k], s->stream) != cudaSuccess) r = DP_ECUDA;
      if (r != DP_OK) { perr[k] = r; return; }
      rebuilt[k] = !had;
      const char *w = unsupported(s, b->m[0]);
      if (w) { why[k] = w; perr[k] = DP_EINVAL; return; }
      solving[k] = 1;
    });
    b->ms_setup += ms_since(t0);
    t0 = clk::now();
    std::vector<int> solve;
    bool rebuild = !b->built;
    for (int k = 0; k < nm && !rebuild; ++k) rebuild = b->shapes[k] != b->m[k]->shapes;
    for (int k : iter) {
      if (perr[k] != DP_OK) return bfail(b, perr[k], why[k].empty() ? "assembly or set-up" : why[k]);
      if (solving[k]) {
        solve.push_back(k);
        if (rebuilt[k]) rebuild = true;
        if (cudaStreamWaitEvent(b->stream, b->ev[k], 0) != cudaSuccess)
          return bfail(b, DP_ECUDA, "event");
      }
    }
    if (solve.empty()) continue;
    if (rebuild) {
      int r = build_plan(b);
      if (r != DP_OK) return bfail(b, r, "batch plan");
    }
    std::vector<int> frc(nm, DP_OK), fit(nm, 0);
    std::vector<double> frr(nm, 0.0);
    int r = batch_fgmres(b, solve, eta, frc, fit, frr);
    if (r != DP_OK) return bfail(b, r, "batched FGMRES");
    if (cudaEventRecord(b->solved, b->stream) != cudaSuccess) return bfail(b, DP_ECUDA, "event");
    b->ms_fgmres += ms_since(t0);
    t0 = clk::now();
    // the updates, each on its own stream after the batched FGMRES
    pool_run(b, (int)solve.size(), [&](int q) {
      int k = solve[q];
      Sim *s = b->m[k];
      int ru = cudaStreamWaitEvent(s->stream, b->solved, 0) == cudaSuccess ? DP_OK : DP_ECUDA;
      if (ru == DP_OK) ru = solve_update(s, frc[k]);
      if (ru == DP_OK && cudaStreamSynchronize(s->stream) != cudaSuccess) ru = DP_ECUDA;
      if (ru != DP_OK) { perr[k] = ru; return; }
      dp_stats ls{};
      int rf = solve_finish(s, frc[k], fit[k], frr[k], eta[k], 0.f, 0.f, &ls);
      if (rf != DP_OK && rf != DP_ELINEAR) { perr[k] = rf; return; }
      lin[k] += ls.linear_iters;
      if (rf == DP_ELINEAR) { linfail[k] = 1; newton[k] = 0; return; }
      if (s->well_limits) perr[k] = phys_well_controls(s, false);
    });
    for (int k : solve)
      if (perr[k] != DP_OK) return bfail(b, perr[k], "update");
    b->ms_update += ms_since(t0);
  }
  int first = DP_OK;
  for (int k = 0; k < nm; ++k) {
    Sim *s = b->m[k];
    dp_stats &L = s->last;
    L.newton_iters = s->newton_iter; L.linear_iters = lin[k]; L.converged = conv[k];
    L.res0 = res0[k]; L.res = res[k]; L.amg_levels = (int)s->lev.size();
    L.ms_setup = 0.0; L.ms_solve = 0.0;
    if (stats) stats[k] = L;
    rc[k] = DP_OK;
    if (!conv[k]) {
      int r = timestep_restore(s);
      if (r != DP_OK) return bfail(b, r, "restore");
      rc[k] = linfail[k] ? DP_ELINEAR : DP_ENEWTON;
      s->fail(rc[k], linfail[k] ? "a linear solve did not reach its forcing term; the old state is restored"
                                : "Newton did not converge");
    }
    if (status) status[k] = rc[k];
    if (rc[k] != DP_OK && first == DP_OK) first = rc[k];
  }
  for (Sim *s : b->m)
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return bfail(b, DP_ECUDA, "sync");
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bfail(b, DP_ECUDA, "sync");
  return first;
}
