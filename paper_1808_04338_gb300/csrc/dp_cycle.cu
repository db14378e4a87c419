// The coarse part of the AMG V-cycle in one launch of one thread-block
// cluster.
//
// Below a size threshold every level of the hierarchy is small, but its
// multicolour Gauss-Seidel still needs one ordered phase per colour (17-46
// colours per level on the 8M-unknown problem), and even l1-Jacobi needs a
// few phases per level.  Launching a kernel per phase costs more than the
// phase's work.  Here one cluster of CTAs (up to
// 16 CTAs of 512 threads, one per SM of a GPC) runs all phases of levels l0..L-1: the colour
// sweeps, residuals, restrictions, the dense coarsest solve and the
// prolongations, separated by hardware cluster barriers (barrier.cluster
// with release/acquire semantics).  Vectors that other CTAs write are read
// through L2 (ld.global.cg) so that no stale L1 line is used after a
// barrier; the operators, which do not change during the launch, are read
// through the read-only path.  The arithmetic is that of the per-launch
// cycle (the same colour order, the same row formulas).
#include <cooperative_groups.h>

#include <algorithm>

#include "dp_internal.h"

namespace cg = cooperative_groups;

namespace dp {

template <typename T>
struct LevelDev {
  int n, ncolour, lanes;
  int l1;                         // l1-Jacobi smoothing; dinv = 1 / sum_j |a_ij|
  const int *rowptr, *col, *clist, *cstart;
  const T *val, *dinv;
  const int *r_rowptr, *r_col;   // restriction to the next level
  const T *r_val;
  int nn;                         // rows of the next level
  int r_lanes, p_lanes;
  const int *p_rowptr, *p_col;   // prolongation from the next level
  const T *p_val;
  T *x, *b, *r;
  // padded column-major copy of the rows of each colour: entry k of the
  // t-th row of colour c at ell_off[c] + k * (rows of c) + t
  const int *ell_col, *ell_off, *ell_K;
  const T *ell_val;
};

// sum over a row's entries owned by one lane of a group of G lanes, with the
// vector read through L2
template <typename T>
__device__ __forceinline__ T row_dot_l2(int e0, int e1, int lane, int G, const int *__restrict__ col,
                                        const T *__restrict__ val, const T *x) {
  T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
  int e = e0 + lane;
  for (; e + 3 * G < e1; e += 4 * G) {
    int c0 = __ldg(col + e), c1 = __ldg(col + e + G), c2 = __ldg(col + e + 2 * G),
        c3 = __ldg(col + e + 3 * G);
    T v0 = __ldg(val + e), v1 = __ldg(val + e + G), v2 = __ldg(val + e + 2 * G),
      v3 = __ldg(val + e + 3 * G);
    T x0 = __ldcg(x + c0), x1 = __ldcg(x + c1), x2 = __ldcg(x + c2), x3 = __ldcg(x + c3);
    s0 = fma(v0, x0, s0);
    s1 = fma(v1, x1, s1);
    s2 = fma(v2, x2, s2);
    s3 = fma(v3, x3, s3);
  }
  for (; e < e1; e += G) s0 = fma(__ldg(val + e), __ldcg(x + __ldg(col + e)), s0);
  return (s0 + s1) + (s2 + s3);
}

// sum_j a_ij b_j d_j over the lane's entries: the residual of the l1-Jacobi
// pre-smoothing from zero without storing x first (b through L2, d constant)
template <typename T>
__device__ __forceinline__ T row_dot_bd(int e0, int e1, int lane, int G, const int *__restrict__ col,
                                        const T *__restrict__ val, const T *b,
                                        const T *__restrict__ d) {
  T s0 = T(0), s1 = T(0);
  int e = e0 + lane;
  for (; e + G < e1; e += 2 * G) {
    int c0 = __ldg(col + e), c1 = __ldg(col + e + G);
    T v0 = __ldg(val + e), v1 = __ldg(val + e + G);
    T b0 = __ldcg(b + c0), b1 = __ldcg(b + c1);
    s0 = fma(v0, b0 * __ldg(d + c0), s0);
    s1 = fma(v1, b1 * __ldg(d + c1), s1);
  }
  if (e < e1) {
    int c0 = __ldg(col + e);
    s0 = fma(__ldg(val + e), __ldcg(b + c0) * __ldg(d + c0), s0);
  }
  return s0 + s1;
}

template <typename T>
__device__ __forceinline__ T group_reduce(T v, int G) {
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, G);
  return v;
}

// Rows [0, count) of a phase spread over the cluster's threads in groups of
// G lanes; the trip count is uniform across a warp so that the shuffles see
// every lane.  f(q, lane, valid) returns the lane's partial sum of row slot q;
// done(q, sum) runs on lane 0 of the group.
template <typename T, typename F, typename D>
__device__ __forceinline__ void for_rows(int count, int G, int gt, int nt, F f, D done) {
  int groups = nt / G, gid = gt / G, lane = gt % G;
  for (int base = 0; base < count; base += groups) {
    int q = base + gid;
    bool valid = q < count;
    T s = f(q, lane, valid);
    s = group_reduce<T>(s, G);
    if (valid && lane == 0) done(q, s);
  }
}

// One Gauss-Seidel sweep over the colours of a level from its ELL copy.  A
// lane loads the column indices and values of up to eight of its row's
// entries at once (no row-pointer indirection), then the eight x values:
// two dependent round trips per colour phase.  The fields are copied into
// registers first: the L2 loads and stores are opaque to the compiler, which
// would otherwise reload the descriptor after each of them.
template <typename T>
__device__ void gs_sweep_cl(const LevelDev<T> &Ld, const T *b, T *x, bool forward, int gt, int nt,
                            cg::cluster_group &cl) {
  const int ncolour = Ld.ncolour;
  const int *__restrict__ clist = Ld.clist;
  const int *__restrict__ cstart = Ld.cstart;
  const int *__restrict__ ecol = Ld.ell_col;
  const int *__restrict__ eoff = Ld.ell_off;
  const int *__restrict__ eK = Ld.ell_K;
  const T *__restrict__ eval = Ld.ell_val;
  const T *__restrict__ dinv = Ld.dinv;
  for (int t = 0; t < ncolour; ++t) {
    int c = forward ? t : ncolour - 1 - t;
    int r0 = __ldg(cstart + c), ncr = __ldg(cstart + c + 1) - r0;
    int off = __ldg(eoff + c), K = __ldg(eK + c);
    int G = 1;
    while (G < 32 && 8 * G < K) G <<= 1;
    int groups = nt / G, gid = gt / G, lane = gt % G;
    for (int base = 0; base < ncr; base += groups) {
      int q = base + gid;
      bool valid = q < ncr;
      int i = 0;
      T di = T(0);
      if (valid && lane == 0) { i = __ldg(clist + r0 + q); di = __ldg(dinv + i); }
      T s = T(0);
      if (valid) {
        for (int kb = 0; kb < K; kb += 8 * G) {
          int ci[8];
          T v[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            int k = kb + lane + G * u;
            ci[u] = k < K ? __ldg(ecol + off + (size_t)k * ncr + q) : -1;
            v[u] = k < K ? __ldg(eval + off + (size_t)k * ncr + q) : T(0);
          }
          T xv[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) xv[u] = ci[u] >= 0 ? __ldcg(x + ci[u]) : T(0);
#pragma unroll
          for (int u = 0; u < 8; ++u) s = fma(v[u], xv[u], s);
        }
      }
      T bi = T(0), xi = T(0);
      if (valid && lane == 0) { bi = __ldcg(b + i); xi = __ldcg(x + i); }
      s = group_reduce<T>(s, G);
      if (valid && lane == 0 && di != T(0)) __stcg(x + i, fma(bi - s, di, xi));
    }
    cl.sync();
  }
}

// Dense solve with the FP64 LU factors and row pivots of the coarsest level,
// by the first CTA of the cluster only.
template <typename T>
__device__ void dense_solve_cta(int n, const double *a, const int *piv, const T *b, T *x) {
  __shared__ double xs[4096];
  int t = threadIdx.x, nt = blockDim.x;
  for (int i = t; i < n; i += nt) xs[i] = double(__ldcg(b + i));
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (t == 0) {
      int p = piv[k];
      if (p != k && p >= 0 && p < n) { double tmp = xs[k]; xs[k] = xs[p]; xs[p] = tmp; }
    }
    __syncthreads();
    double xk = xs[k];
    for (int i = k + 1 + t; i < n; i += nt) xs[i] -= a[(size_t)i * n + k] * xk;
    __syncthreads();
  }
  for (int i = n - 1; i >= 0; --i) {
    if (t == 0) { double d = a[(size_t)i * n + i]; xs[i] = d != 0.0 ? xs[i] / d : 0.0; }
    __syncthreads();
    double xi = xs[i];
    for (int r = t; r < i; r += nt) xs[r] -= a[(size_t)r * n + i] * xi;
    __syncthreads();
  }
  for (int i = t; i < n; i += nt) __stcg(x + i, T(xs[i]));
}

// l1-Jacobi pre-smoothing from zero and the residual in one phase:
// x_i = b_i d_i, r_i = b_i - sum_j a_ij b_j d_j.
template <typename T>
__device__ void jacobi_pre_cl(const LevelDev<T> &L, const T *b, T *x, T *r, int gt, int nt) {
  const int G = L.lanes;
  const int *__restrict__ rowptr = L.rowptr;
  const int *__restrict__ col = L.col;
  const T *__restrict__ val = L.val;
  const T *__restrict__ d = L.dinv;
  for_rows<T>(
      L.n, G, gt, nt,
      [&](int i, int lane, bool valid) -> T {
        return valid ? row_dot_bd<T>(__ldg(rowptr + i), __ldg(rowptr + i + 1), lane, G, col, val, b,
                                     d)
                     : T(0);
      },
      [&](int i, T s) {
        T bi = __ldcg(b + i);
        __stcg(x + i, bi * __ldg(d + i));
        __stcg(r + i, bi - s);
      });
}

// One l1-Jacobi sweep through t (t_i = x_i + (b_i - (A x)_i) d_i), then
// t copied back into x: two phases.
template <typename T>
__device__ void jacobi_post_cl(const LevelDev<T> &L, const T *b, T *x, T *t, int gt, int nt,
                               cg::cluster_group &cl) {
  const int G = L.lanes;
  const int *__restrict__ rowptr = L.rowptr;
  const int *__restrict__ col = L.col;
  const T *__restrict__ val = L.val;
  const T *__restrict__ d = L.dinv;
  for_rows<T>(
      L.n, G, gt, nt,
      [&](int i, int lane, bool valid) -> T {
        return valid ? row_dot_l2<T>(__ldg(rowptr + i), __ldg(rowptr + i + 1), lane, G, col, val, x)
                     : T(0);
      },
      [&](int i, T s) { __stcg(t + i, fma(__ldcg(b + i) - s, __ldg(d + i), __ldcg(x + i))); });
  cl.sync();
  for (int i = gt; i < L.n; i += nt) __stcg(x + i, __ldcg(t + i));
  cl.sync();
}

constexpr int kClusterThreads = 512;

// x = inv b for the coarsest level from its explicit FP64 inverse: one phase
template <typename T>
__device__ void dense_mv_cl(int n, const double *__restrict__ inv, const T *b, T *x, int gt,
                            int nt) {
  int G = 1;
  while (G < 32 && 4 * G < n) G <<= 1;
  for_rows<double>(
      n, G, gt, nt,
      [&](int i, int lane, bool valid) -> double {
        double s0 = 0.0, s1 = 0.0;
        if (valid) {
          const double *row = inv + (size_t)i * n;
          int j = lane;
          for (; j + G < n; j += 2 * G) {
            s0 = fma(__ldg(row + j), double(__ldcg(b + j)), s0);
            s1 = fma(__ldg(row + j + G), double(__ldcg(b + j + G)), s1);
          }
          if (j < n) s0 = fma(__ldg(row + j), double(__ldcg(b + j)), s0);
        }
        return s0 + s1;
      },
      [&](int i, double s) { __stcg(x + i, T(s)); });
}

template <typename T>
__global__ void __launch_bounds__(kClusterThreads, 1)
    k_coarse_cycle(const LevelDev<T> *__restrict__ lv, int l0, int nl, const T *b0, T *x0,
                   const double *lu, const int *piv, const double *inv, int dense_n) {
  cg::cluster_group cl = cg::this_cluster();
  int gt = (int)cl.block_rank() * blockDim.x + threadIdx.x;
  int nt = (int)cl.num_blocks() * blockDim.x;
  // descending half: pre-smoothing, residual, restriction
  for (int l = l0; l < nl - 1; ++l) {
    const LevelDev<T> &L = lv[l];
    const T *b = l == l0 ? b0 : L.b;
    T *x = l == l0 ? x0 : L.x;
    const int n = L.n, G = L.lanes, nn = L.nn, rG = L.r_lanes;
    const int *__restrict__ rowptr = L.rowptr;
    const int *__restrict__ col = L.col;
    const T *__restrict__ val = L.val;
    const int *__restrict__ rrp = L.r_rowptr;
    const int *__restrict__ rcol = L.r_col;
    const T *__restrict__ rval = L.r_val;
    T *r = L.r, *nb = lv[l + 1].b;
    if (L.l1) {
      jacobi_pre_cl<T>(L, b, x, r, gt, nt);
    } else {
      for (int i = gt; i < n; i += nt) __stcg(x + i, T(0));
      cl.sync();
      gs_sweep_cl<T>(L, b, x, true, gt, nt, cl);
      for_rows<T>(
          n, G, gt, nt,
          [&](int i, int lane, bool valid) -> T {
            return valid ? row_dot_l2<T>(__ldg(rowptr + i), __ldg(rowptr + i + 1), lane, G, col,
                                         val, x)
                         : T(0);
          },
          [&](int i, T s) { __stcg(r + i, __ldcg(b + i) - s); });
    }
    cl.sync();
    for_rows<T>(
        nn, rG, gt, nt,
        [&](int I, int lane, bool valid) -> T {
          return valid ? row_dot_l2<T>(__ldg(rrp + I), __ldg(rrp + I + 1), lane, rG, rcol, rval, r)
                       : T(0);
        },
        [&](int I, T s) { __stcg(nb + I, s); });
    cl.sync();
  }
  // coarsest level
  {
    const LevelDev<T> &L = lv[nl - 1];
    const T *b = nl - 1 == l0 ? b0 : L.b;
    T *x = nl - 1 == l0 ? x0 : L.x;
    if (dense_n == L.n && L.n > 0 && inv) {
      dense_mv_cl<T>(L.n, inv, b, x, gt, nt);
      cl.sync();
    } else if (dense_n == L.n && L.n > 0) {
      if (cl.block_rank() == 0) dense_solve_cta<T>(L.n, lu, piv, b, x);
      cl.sync();
    } else if (L.l1) {
      jacobi_pre_cl<T>(L, b, x, L.r, gt, nt);
      cl.sync();
      jacobi_post_cl<T>(L, b, x, L.r, gt, nt, cl);
    } else {
      for (int i = gt; i < L.n; i += nt) __stcg(x + i, T(0));
      cl.sync();
      gs_sweep_cl<T>(L, b, x, true, gt, nt, cl);
      gs_sweep_cl<T>(L, b, x, false, gt, nt, cl);
    }
  }
  // ascending half: prolongation, post-smoothing
  for (int l = nl - 2; l >= l0; --l) {
    const LevelDev<T> &L = lv[l];
    const LevelDev<T> &N = lv[l + 1];
    const T *b = l == l0 ? b0 : L.b;
    T *x = l == l0 ? x0 : L.x;
    const int n = L.n, pG = L.p_lanes;
    const int *__restrict__ prp = L.p_rowptr;
    const int *__restrict__ pcol = L.p_col;
    const T *__restrict__ pval = L.p_val;
    const T *nx = N.x;
    for_rows<T>(
        n, pG, gt, nt,
        [&](int i, int lane, bool valid) -> T {
          return valid ? row_dot_l2<T>(__ldg(prp + i), __ldg(prp + i + 1), lane, pG, pcol, pval, nx)
                       : T(0);
        },
        [&](int i, T s) { __stcg(x + i, __ldcg(x + i) + s); });
    cl.sync();
    if (L.l1) jacobi_post_cl<T>(L, b, x, L.r, gt, nt, cl);
    else gs_sweep_cl<T>(L, b, x, false, gt, nt, cl);
  }
}

// lanes per row inside the cluster: rows are few, so shorten the chains
static int cluster_lanes(double mean_len) {
  int g = 1;
  while (g < 32 && 4.0 * g < mean_len) g *= 2;
  return g;
}

template <typename T>
static const T *pick(const double *d, const float *f) {
  if constexpr (sizeof(T) == 8) return (const T *)d; else return (const T *)f;
}
template <typename T>
static T *pickw(double *d, float *f) {
  if constexpr (sizeof(T) == 8) return (T *)d; else return (T *)f;
}

template <typename T>
static int upload_levels(Sim *s, void **dst) {
  int nl = (int)s->lev.size();
  std::vector<LevelDev<T>> h(nl);
  for (int l = 0; l < nl; ++l) {
    Level &L = s->lev[l];
    LevelDev<T> &d = h[l];
    d.n = L.n;
    d.l1 = L.l1 ? 1 : 0;
    d.ncolour = L.ncolour;
    d.lanes = cluster_lanes(L.n ? (double)L.nnz / L.n : 0.0);
    d.rowptr = L.rowptr; d.col = L.col; d.clist = L.clist; d.cstart = L.cstart_dev;
    d.val = pick<T>(L.val, L.valf);
    d.dinv = pick<T>(L.dinv, L.dinvf);
    d.x = pickw<T>(L.x, L.xf); d.b = pickw<T>(L.b, L.bf); d.r = pickw<T>(L.r, L.rf);
    d.ell_col = L.ell_col; d.ell_off = L.ell_off; d.ell_K = L.ell_K;
    d.ell_val = pick<T>(L.ell_val, L.ell_valf);
    if (l + 1 < nl) {
      d.nn = s->lev[l + 1].n;
      d.r_rowptr = L.r_rowptr; d.r_col = L.r_col; d.r_val = pick<T>(L.r_val, L.r_valf);
      d.p_rowptr = L.p_rowptr; d.p_col = L.p_col; d.p_val = pick<T>(L.p_val, L.p_valf);
      d.r_lanes = cluster_lanes(d.nn ? (double)L.r_nnz / d.nn : 0.0);
      d.p_lanes = cluster_lanes(L.n ? (double)L.p_nnz / L.n : 0.0);
    } else {
      d.nn = 0; d.r_rowptr = d.r_col = d.p_rowptr = d.p_col = nullptr;
      d.r_val = d.p_val = nullptr; d.r_lanes = d.p_lanes = 1;
    }
  }
  if (!*dst) {
    *dst = dalloc(s, sizeof(LevelDev<T>) * std::max(nl, 1));
    if (!*dst) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
  }
  DP_CUDA(s, cudaMemcpyAsync(*dst, h.data(), sizeof(LevelDev<T>) * nl, cudaMemcpyHostToDevice,
                             s->stream));
  DP_CUDA(s, cudaStreamSynchronize(s->stream));
  return DP_OK;
}

__global__ void k_ell_maxlen(int n, const int *rowptr, const int *colour, int *K) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicMax(&K[colour[i]], rowptr[i + 1] - rowptr[i]);
}

// Fill the padded copy: padding entries point at the row itself with source
// -1 (value 0).
__global__ void k_ell_fill(int n, const int *clist, const int *colour, const int *cstart,
                           const int *eoff, const int *eK, const int *rowptr, const int *col,
                           int *ecol, int *esrc) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  int i = clist[q], c = colour[i];
  int r0 = cstart[c], ncr = cstart[c + 1] - r0, t = q - r0, K = eK[c], off = eoff[c];
  int e0 = rowptr[i], len = rowptr[i + 1] - e0;
  for (int k = 0; k < K; ++k) {
    size_t p = (size_t)off + (size_t)k * ncr + t;
    ecol[p] = k < len ? col[e0 + k] : i;
    esrc[p] = k < len ? e0 + k : -1;
  }
}

template <typename T>
__global__ void k_ell_values(long long total, const int *esrc, const T *val, T *eval) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < total) { int q = esrc[p]; eval[p] = q >= 0 ? val[q] : T(0); }
}

static int ell_build(Sim *s, Level &L) {
  int nc = L.ncolour;
  L.ell_off = (int *)dalloc(s, (size_t)(nc + 1) * 4);
  L.ell_K = (int *)dalloc(s, (size_t)std::max(nc, 1) * 4);
  if (!L.ell_off || !L.ell_K) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
  DP_CUDA(s, cudaMemsetAsync(L.ell_K, 0, (size_t)std::max(nc, 1) * 4, s->stream));
  DP_LAUNCH(s, k_ell_maxlen, nblk(L.n), kBlock, 0, L.n, L.rowptr, L.colour, L.ell_K);
  std::vector<int> K(std::max(nc, 1)), off(nc + 1, 0);
  DP_CUDA(s, cudaMemcpyAsync(K.data(), L.ell_K, (size_t)std::max(nc, 1) * 4, cudaMemcpyDeviceToHost,
                             s->stream));
  DP_CUDA(s, cudaStreamSynchronize(s->stream));
  long long total = 0;
  for (int c = 0; c < nc; ++c) {
    off[c] = (int)total;
    total += (long long)K[c] * (L.cstart[c + 1] - L.cstart[c]);
  }
  off[nc] = (int)total;
  if (total >= (1LL << 31)) { s->fail(DP_EINVAL, "coarse level too large for its padded copy"); return DP_EINVAL; }
  L.ell_total = total;
  DP_CUDA(s, cudaMemcpyAsync(L.ell_off, off.data(), (size_t)(nc + 1) * 4, cudaMemcpyHostToDevice,
                             s->stream));
  size_t m = (size_t)std::max(total, 1LL);
  L.ell_col = (int *)dalloc(s, m * 4);
  L.ell_src = (int *)dalloc(s, m * 4);
  L.ell_val = (double *)dalloc(s, m * 8);
  L.ell_valf = (float *)dalloc(s, m * 4);
  if (!L.ell_col || !L.ell_src || !L.ell_val || !L.ell_valf) {
    s->fail(DP_ENOMEM, "allocation failed");
    return DP_ENOMEM;
  }
  DP_LAUNCH(s, k_ell_fill, nblk(L.n), kBlock, 0, L.n, L.clist, L.colour, L.cstart_dev, L.ell_off,
            L.ell_K, L.rowptr, L.col, L.ell_col, L.ell_src);
  DP_CUDA(s, cudaGetLastError());
  return DP_OK;
}

// Copy the current level values into the padded copies (every Newton step,
// after the hierarchy's values and their FP32 copies are refreshed).
int cluster_refresh(Sim *s) {
  if (s->cl_level < 0) return DP_OK;
  bool f32 = s->opt.precision >= 1;
  for (int l = s->cl_level; l < (int)s->lev.size(); ++l) {
    Level &L = s->lev[l];
    if (!L.ell_src) continue;
    if (f32)
      DP_LAUNCH(s, k_ell_values<float>, nblk(L.ell_total), kBlock, 0, L.ell_total, L.ell_src,
                L.valf, L.ell_valf);
    else
      DP_LAUNCH(s, k_ell_values<double>, nblk(L.ell_total), kBlock, 0, L.ell_total, L.ell_src,
                L.val, L.ell_val);
  }
  DP_CUDA(s, cudaGetLastError());
  return DP_OK;
}

// Decide the first level run by the cluster kernel and the cluster size; copy
// the level descriptors and colour starts to the device.  Called after the
// hierarchy is built.
int cluster_setup(Sim *s) {
  s->cl_level = -1;
  if (s->lev.empty()) return DP_OK;
  for (Level &L : s->lev) {
    if (!L.cstart_dev) {
      L.cstart_dev = (int *)dalloc(s, (L.cstart.size() + 1) * 4);
      if (!L.cstart_dev) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
    }
    DP_CUDA(s, cudaMemcpyAsync(L.cstart_dev, L.cstart.data(), L.cstart.size() * 4,
                               cudaMemcpyHostToDevice, s->stream));
  }
  // cluster size: 16 CTAs if the GPU can place them, else 8
  int csize = 0;
  for (int c : {16, 8}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c);
    cfg.blockDim = dim3(kClusterThreads);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = c; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (c > 8) {
      cudaFuncSetAttribute(k_coarse_cycle<float>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      cudaFuncSetAttribute(k_coarse_cycle<double>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    }
    int nc1 = 0, nc2 = 0;
    if (cudaOccupancyMaxActiveClusters(&nc1, k_coarse_cycle<float>, &cfg) == cudaSuccess &&
        cudaOccupancyMaxActiveClusters(&nc2, k_coarse_cycle<double>, &cfg) == cudaSuccess &&
        nc1 > 0 && nc2 > 0) {
      csize = c;
      break;
    }
    cudaGetLastError();
  }
  s->cl_size = csize;
  if (csize == 0 || !s->opt.use_graphs) return DP_OK;  // the per-launch cycle stays in use
  int rows = s->opt.cluster_rows == 0 ? kClusterMaxRows : s->opt.cluster_rows;
  int first = -1;
  for (int l = 0; l < (int)s->lev.size() && rows > 0; ++l)
    if (s->lev[l].n <= rows) { first = l; break; }
  if (first < 0) return DP_OK;
  // By default the cluster runs only where it saves launches: a level with
  // multicolour Gauss-Seidel has one phase per colour, an l1-Jacobi level
  // five, and on GB300 five full-GPU launches of a small level (graph
  // launched) cost less than the same phases on the cluster's 16 SMs.
  bool gs = false;
  for (int l = first; l < (int)s->lev.size(); ++l) gs |= !s->lev[l].l1;
  if (s->opt.cluster_rows == 0 && !gs) return DP_OK;
  for (int l = first; l < (int)s->lev.size(); ++l)
    if (!s->lev[l].l1) DP_TRY(ell_build(s, s->lev[l]));   // Gauss-Seidel levels only
  DP_TRY(upload_levels<double>(s, &s->cl_lev64));
  DP_TRY(upload_levels<float>(s, &s->cl_lev32));
  s->cl_level = first;
  return DP_OK;
}

template <typename T>
int coarse_cycle(Sim *s, int l0, const T *b, T *x) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(s->cl_size);
  cfg.blockDim = dim3(kClusterThreads);
  cfg.stream = s->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = s->cl_size; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const LevelDev<T> *lv = (const LevelDev<T> *)(sizeof(T) == 8 ? s->cl_lev64 : s->cl_lev32);
  int nl = (int)s->lev.size();
  {
    LaunchScope ls(s, "k_coarse_cycle");
    DP_CUDA(s, cudaLaunchKernelEx(&cfg, k_coarse_cycle<T>, lv, l0, nl, b, x,
                                  (const double *)s->coarse_lu, (const int *)s->coarse_piv,
                                  (const double *)s->coarse_inv, s->coarse_n));
  }
  return DP_OK;
}

template int coarse_cycle<double>(Sim *, int, const double *, double *);
template int coarse_cycle<float>(Sim *, int, const float *, float *);

}  // namespace dp
