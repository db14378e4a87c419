// Linear algebra of the Newton-step solve (Section 3.2): block SpMV, block
// ILU(0) in colour order, the AMG V-cycle with multicolour Gauss-Seidel, the
// dense coarsest solve, the CPR-FPF preconditioner and flexible GMRES.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "dp_internal.h"

namespace dp {

// ---------------------------------------------------------------- BSR SpMV
// Two lanes per block row, one per output component: lane c of row i reads
// row c of every 2x2 block (one 16-byte load; the two lanes of a row read
// the two halves of the same 32-byte block), x_j (16 bytes, shared by the
// pair) and accumulates its own output with FMAs, so no FP64 reduction
// across lanes is needed.  A warp covers 16 block rows.
template <int MODE>  // MODE 0: y = A x; 1: y = b - A x
__global__ void __launch_bounds__(kBlock) k_bsr_spmv(int n, const int *__restrict__ rowptr,
                                                     const int *__restrict__ col,
                                                     const double *__restrict__ val,
                                                     const double *__restrict__ x,
                                                     const double *__restrict__ b,
                                                     double *__restrict__ y) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int row = t >> 1, comp = t & 1;
  if (row >= n) return;
  int e0 = __ldg(rowptr + row), e1 = __ldg(rowptr + row + 1);
  const double2 *v2 = reinterpret_cast<const double2 *>(val) + comp;
  const double2 *x2 = reinterpret_cast<const double2 *>(x);
  double s = 0.0;
#pragma unroll 4
  for (int e = e0; e < e1; ++e) {
    double2 a = __ldg(v2 + 2 * (size_t)e);
    double2 xj = __ldg(x2 + __ldg(col + e));
    s = fma(a.x, xj.x, s);
    s = fma(a.y, xj.y, s);
  }
  y[2 * (size_t)row + comp] = MODE == 0 ? s : b[2 * (size_t)row + comp] - s;
}

// Pressure component of b - A x: rp_i = b_{i,0} - sum_j (a00 x_j0 + a01 x_j1)
// (reads the first half of every block only).
__global__ void __launch_bounds__(kBlock) k_bsr_presid(int n, const int *__restrict__ rowptr,
                                                       const int *__restrict__ col,
                                                       const double *__restrict__ val,
                                                       const double *__restrict__ x,
                                                       const double *__restrict__ b,
                                                       double *__restrict__ rp) {
  int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  int e0 = __ldg(rowptr + row), e1 = __ldg(rowptr + row + 1);
  const double2 *v2 = reinterpret_cast<const double2 *>(val);
  const double2 *x2 = reinterpret_cast<const double2 *>(x);
  double s = 0.0;
#pragma unroll 4
  for (int e = e0; e < e1; ++e) {
    double2 a = __ldg(v2 + 2 * (size_t)e);
    double2 xj = __ldg(x2 + __ldg(col + e));
    s = fma(a.x, xj.x, s);
    s = fma(a.y, xj.y, s);
  }
  rp[row] = b[2 * (size_t)row] - s;
}

int bsr_spmv(Sim *s, const double *x, double *y) {
  DP_LAUNCH(s, k_bsr_spmv<0>, nblk(2LL * s->A.n), kBlock, 0, s->A.n, s->A.rowptr, s->A.col,
            s->A.val, x, nullptr, y);
  return DP_OK;
}

int bsr_residual(Sim *s, const double *b, const double *x, double *r) {
  DP_LAUNCH(s, k_bsr_spmv<1>, nblk(2LL * s->A.n), kBlock, 0, s->A.n, s->A.rowptr, s->A.col,
            s->A.val, x, b, r);
  return DP_OK;
}

// ---------------------------------------------------------------- ILU(0)
// Rows are ordered by (colour, index); the factor is stored row by row in
// that order with each row's blocks sorted by the permuted position of
// their column: L blocks, the inverted pivot block, U blocks.

__global__ void k_perm_len(int n, const int *perm, const int *rowptr, int *len) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) { int i = perm[r]; len[r] = rowptr[i + 1] - rowptr[i]; }
}

__global__ void k_lu_pattern(int n, const int *perm, const int *iperm, const int *rowptr,
                             const int *col, const int *lu_rowptr, int *lu_col, int *lu_src,
                             int *lu_dpos) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  int i = perm[r], s0 = rowptr[i], m = rowptr[i + 1] - s0, d0 = lu_rowptr[r];
  for (int t = 0; t < m; ++t) { lu_col[d0 + t] = col[s0 + t]; lu_src[d0 + t] = s0 + t; }
  for (int a = 1; a < m; ++a) {           // insertion sort by permuted position
    int c = lu_col[d0 + a], sidx = lu_src[d0 + a], key = iperm[c], b = a - 1;
    while (b >= 0 && iperm[lu_col[d0 + b]] > key) {
      lu_col[d0 + b + 1] = lu_col[d0 + b];
      lu_src[d0 + b + 1] = lu_src[d0 + b];
      --b;
    }
    lu_col[d0 + b + 1] = c;
    lu_src[d0 + b + 1] = sidx;
  }
  for (int t = 0; t < m; ++t) if (lu_col[d0 + t] == i) lu_dpos[r] = d0 + t;
}

__device__ __forceinline__ void mul2(const double *a, const double *b, double *o) {
  double t0 = a[0] * b[0] + a[1] * b[2];
  double t1 = a[0] * b[1] + a[1] * b[3];
  double t2 = a[2] * b[0] + a[3] * b[2];
  double t3 = a[2] * b[1] + a[3] * b[3];
  o[0] = t0; o[1] = t1; o[2] = t2; o[3] = t3;
}

__device__ __forceinline__ void inv2(double *a) {
  double det = a[0] * a[3] - a[1] * a[2];
  double id = 1.0 / det;
  double o0 = a[3] * id, o1 = -a[1] * id, o2 = -a[2] * id, o3 = a[0] * id;
  a[0] = o0; a[1] = o1; a[2] = o2; a[3] = o3;
}

// IKJ block ILU(0) of the rows [r0, r1) of one colour: all their L blocks
// refer to rows of earlier colours, which are final.
__global__ void k_ilu_factor(int r0, int r1, const int *perm, const int *iperm,
                             const int *lu_rowptr, const int *lu_col, const int *lu_src,
                             const int *lu_dpos, const double *aval, double *lu) {
  int r = r0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= r1) return;
  int s0 = lu_rowptr[r], s1 = lu_rowptr[r + 1], dp = lu_dpos[r];
  for (int e = s0; e < s1; ++e) {
    const double *src = aval + 4 * (size_t)lu_src[e];
    double *dst = lu + 4 * (size_t)e;
    dst[0] = src[0]; dst[1] = src[1]; dst[2] = src[2]; dst[3] = src[3];
  }
  for (int e = s0; e < dp; ++e) {
    int k = lu_col[e], rk = iperm[k];
    double lik[4];
    mul2(lu + 4 * (size_t)e, lu + 4 * (size_t)lu_dpos[rk], lik);   // A_ik U_kk^-1
    double *le = lu + 4 * (size_t)e;
    le[0] = lik[0]; le[1] = lik[1]; le[2] = lik[2]; le[3] = lik[3];
    int ku0 = lu_dpos[rk] + 1, ku1 = lu_rowptr[rk + 1];
    for (int e2 = e + 1; e2 < s1; ++e2) {
      int j = lu_col[e2];
      int q = -1;
      for (int t = ku0; t < ku1; ++t) if (lu_col[t] == j) { q = t; break; }
      if (q < 0) continue;
      double u[4];
      mul2(lik, lu + 4 * (size_t)q, u);
      double *aij = lu + 4 * (size_t)e2;
      aij[0] -= u[0]; aij[1] -= u[1]; aij[2] -= u[2]; aij[3] -= u[3];
    }
  }
  inv2(lu + 4 * (size_t)dp);
}

// Forward sweep of one colour, two lanes per row (one per component):
// z_i = r_i - sum_{L} L_ik z_k (unit lower triangle).
__global__ void __launch_bounds__(kBlock) k_ilu_fwd(int r0, int r1, const int *__restrict__ perm,
                                                    const int *__restrict__ lu_rowptr,
                                                    const int *__restrict__ lu_col,
                                                    const int *__restrict__ lu_dpos,
                                                    const double *__restrict__ lu,
                                                    const double *__restrict__ rhs, double *z) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int r = r0 + (t >> 1), comp = t & 1;
  if (r >= r1) return;
  int i = __ldg(perm + r);
  const double2 *v2 = reinterpret_cast<const double2 *>(lu) + comp;
  const double2 *z2 = reinterpret_cast<const double2 *>(z);
  double s = 0.0;
  int ea = __ldg(lu_rowptr + r), eb = __ldg(lu_dpos + r);
#pragma unroll 4
  for (int e = ea; e < eb; ++e) {
    double2 a = __ldg(v2 + 2 * (size_t)e);
    double2 xk = z2[__ldg(lu_col + e)];
    s = fma(a.x, xk.x, s);
    s = fma(a.y, xk.y, s);
  }
  z[2 * (size_t)i + comp] = rhs[2 * (size_t)i + comp] - s;
}

// Backward sweep of one colour: z_i = U_ii^-1 (z_i - sum_{U} U_ij z_j).  The
// two lanes of a row exchange their partial results for the 2x2 product.
__global__ void __launch_bounds__(kBlock) k_ilu_bwd(int r0, int r1, const int *__restrict__ perm,
                                                    const int *__restrict__ lu_rowptr,
                                                    const int *__restrict__ lu_col,
                                                    const int *__restrict__ lu_dpos,
                                                    const double *__restrict__ lu, double *z) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int r = r0 + (t >> 1), comp = t & 1;
  bool valid = r < r1;                  // no early exit: the pair shuffles
  int i = valid ? __ldg(perm + r) : 0;
  const double2 *v2 = reinterpret_cast<const double2 *>(lu);
  const double2 *z2 = reinterpret_cast<const double2 *>(z);
  int dp = valid ? __ldg(lu_dpos + r) : 0, eb = valid ? __ldg(lu_rowptr + r + 1) : 0;
  double s = 0.0;
#pragma unroll 4
  for (int e = dp + 1; e < eb; ++e) {
    double2 a = __ldg(v2 + 2 * (size_t)e + comp);
    double2 xj = z2[__ldg(lu_col + e)];
    s = fma(a.x, xj.x, s);
    s = fma(a.y, xj.y, s);
  }
  double yi = valid ? z[2 * (size_t)i + comp] - s : 0.0;
  double yo = __shfl_xor_sync(0xffffffffu, yi, 1);
  if (valid) {
    double y0 = comp == 0 ? yi : yo, y1 = comp == 0 ? yo : yi;
    double2 d = __ldg(v2 + 2 * (size_t)dp + comp);
    z[2 * (size_t)i + comp] = fma(d.x, y0, d.y * y1);
  }
}

int ilu_setup(Sim *s) {
  int n = s->A.n;
  s->colour = (int *)dalloc(s, (size_t)n * 4);
  s->perm = (int *)dalloc(s, (size_t)n * 4);
  s->iperm = (int *)dalloc(s, (size_t)n * 4);
  s->lu_rowptr = (int *)dalloc(s, ((size_t)n + 1) * 4);
  s->lu_dpos = (int *)dalloc(s, (size_t)n * 4);
  s->lu_col = (int *)dalloc(s, (size_t)s->A.nnz * 4);
  s->lu_src = (int *)dalloc(s, (size_t)s->A.nnz * 4);
  s->lu_val = (double *)dalloc(s, (size_t)s->A.nnz * 32);
  s->lu_valf = (float *)dalloc(s, (size_t)s->A.nnz * 16);
  int *len = (int *)dalloc(s, (size_t)n * 4);
  if (!s->colour || !s->perm || !s->iperm || !s->lu_rowptr || !s->lu_dpos || !s->lu_col ||
      !s->lu_src || !s->lu_val || !s->lu_valf || !len) {
    s->fail(DP_ENOMEM, "allocation failed");
    return DP_ENOMEM;
  }
  DP_TRY(greedy_colour(s, n, s->A.rowptr, s->A.col, s->colour, &s->ncolour));
  DP_TRY(colour_lists(s, n, s->colour, s->ncolour, s->perm, s->lu_cstart, s->iperm));
  DP_LAUNCH(s, k_perm_len, nblk(n), kBlock, 0, n, s->perm, s->A.rowptr, len);
  int nnz = 0;
  DP_TRY(scan_i32(s, len, s->lu_rowptr, n, &nnz));
  DP_LAUNCH(s, k_lu_pattern, nblk(n), kBlock, 0, n, s->perm, s->iperm, s->A.rowptr, s->A.col,
            s->lu_rowptr, s->lu_col, s->lu_src, s->lu_dpos);
  DP_CUDA(s, cudaGetLastError());
  dfree(s, len);
  return DP_OK;
}

int ilu_factor(Sim *s) {
  for (int c = 0; c < s->ncolour; ++c) {
    int r0 = s->lu_cstart[c], r1 = s->lu_cstart[c + 1];
    if (r1 > r0)
      DP_LAUNCH(s, k_ilu_factor, nblk(r1 - r0, 128), 128, 0, r0, r1, s->perm, s->iperm,
                s->lu_rowptr, s->lu_col, s->lu_src, s->lu_dpos, s->A.val, s->lu_val);
  }
  DP_CUDA(s, cudaGetLastError());
  return DP_OK;
}

int ilu_apply(Sim *s, const double *r, double *z) {
  for (int c = 0; c < s->ncolour; ++c) {
    int r0 = s->lu_cstart[c], r1 = s->lu_cstart[c + 1];
    if (r1 > r0)
      DP_LAUNCH(s, k_ilu_fwd, nblk(2LL * (r1 - r0)), kBlock, 0, r0, r1, s->perm, s->lu_rowptr,
                s->lu_col, s->lu_dpos, s->lu_val, r, z);
  }
  for (int c = s->ncolour - 1; c >= 0; --c) {
    int r0 = s->lu_cstart[c], r1 = s->lu_cstart[c + 1];
    if (r1 > r0)
      DP_LAUNCH(s, k_ilu_bwd, nblk(2LL * (r1 - r0)), kBlock, 0, r0, r1, s->perm, s->lu_rowptr,
                s->lu_col, s->lu_dpos, s->lu_val, z);
  }
  return DP_OK;
}

// ---------------------------------------------------------------- AMG cycle

// Scalar CSR kernels of the AMG levels: G lanes per row (G chosen per level
// from its mean row length), partial sums combined with shuffles inside the
// group; every lane reaches the shuffles (no early exit).
template <int G>
__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, G);
  return v;
}

// One colour of Gauss-Seidel: x_i = (b_i - sum_{j != i} a_ij x_j) / a_ii.
template <int G>
__global__ void __launch_bounds__(kBlock) k_gs_colour(int r0, int r1, const int *__restrict__ clist,
                                                      const int *__restrict__ rowptr,
                                                      const int *__restrict__ col,
                                                      const double *__restrict__ val,
                                                      const int *__restrict__ dpos,
                                                      const double *__restrict__ b, double *x) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int q = r0 + t / G, lane = t % G;
  bool valid = q < r1;
  int i = valid ? clist[q] : 0;
  int e0 = valid ? rowptr[i] : 0, e1 = valid ? rowptr[i + 1] : 0, dp = valid ? dpos[i] : -1;
  double s = 0.0, d = 0.0;
  for (int e = e0 + lane; e < e1; e += G) {
    double a = val[e];
    if (e == dp) d = a;
    else s = fma(a, x[col[e]], s);
  }
  if (G > 1) { s = group_sum<G>(s); d = group_sum<G>(d); }
  if (valid && lane == 0 && d != 0.0) x[i] = (b[i] - s) / d;
}

// r = b - A x
template <int G>
__global__ void __launch_bounds__(kBlock) k_csr_resid(int n, const int *__restrict__ rowptr,
                                                      const int *__restrict__ col,
                                                      const double *__restrict__ val,
                                                      const double *__restrict__ b,
                                                      const double *__restrict__ x,
                                                      double *__restrict__ r) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int i = t / G, lane = t % G;
  bool valid = i < n;
  int e0 = valid ? rowptr[i] : 0, e1 = valid ? rowptr[i + 1] : 0;
  double s = 0.0;
  for (int e = e0 + lane; e < e1; e += G) s = fma(val[e], x[col[e]], s);
  if (G > 1) s = group_sum<G>(s);
  if (valid && lane == 0) r[i] = b[i] - s;
}

// y = A x (add = 0) or y += A x (add = 1)
template <int G>
__global__ void __launch_bounds__(kBlock) k_csr_mv(int n, const int *__restrict__ rowptr,
                                                   const int *__restrict__ col,
                                                   const double *__restrict__ val,
                                                   const double *__restrict__ x,
                                                   double *__restrict__ y, int add) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int i = t / G, lane = t % G;
  bool valid = i < n;
  int e0 = valid ? rowptr[i] : 0, e1 = valid ? rowptr[i + 1] : 0;
  double s = 0.0;
  for (int e = e0 + lane; e < e1; e += G) s = fma(val[e], x[col[e]], s);
  if (G > 1) s = group_sum<G>(s);
  if (valid && lane == 0) y[i] = add ? y[i] + s : s;
}

// lanes per row for a mean row length
int lanes_for(double mean_len) {
  int g = 1;
  while (g < 32 && 2.0 * g < mean_len) g *= 2;
  return g;
}

#define DP_SWITCH_G(G, LAUNCH)                       \
  switch (G) {                                      \
    case 1: { constexpr int GG = 1; LAUNCH; } break;  \
    case 2: { constexpr int GG = 2; LAUNCH; } break;  \
    case 4: { constexpr int GG = 4; LAUNCH; } break;  \
    case 8: { constexpr int GG = 8; LAUNCH; } break;  \
    case 16: { constexpr int GG = 16; LAUNCH; } break; \
    default: { constexpr int GG = 32; LAUNCH; } break; \
  }

static int csr_resid(Sim *s, const Level &L, const double *b, const double *x, double *r) {
  long long thr = (long long)L.n * L.G;
  DP_SWITCH_G(L.G, DP_LAUNCH(s, k_csr_resid<GG>, nblk(thr), kBlock, 0, L.n, L.rowptr, L.col,
                             L.val, b, x, r));
  return DP_OK;
}

static int csr_mv(Sim *s, int n, int G, const int *rowptr, const int *col, const double *val,
                  const double *x, double *y, int add) {
  long long thr = (long long)n * G;
  DP_SWITCH_G(G, DP_LAUNCH(s, k_csr_mv<GG>, nblk(thr), kBlock, 0, n, rowptr, col, val, x, y, add));
  return DP_OK;
}

// coarsest level: dense copy, LU with partial pivoting, solve (one block)
__global__ void k_csr_to_dense(int n, const int *rowptr, const int *col, const double *val,
                               double *a) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int j = 0; j < n; ++j) a[(size_t)i * n + j] = 0.0;
  for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) a[(size_t)i * n + col[e]] = val[e];
}

__global__ void __launch_bounds__(1024) k_dense_lu(int n, double *a, int *piv) {
  __shared__ double sv[1024];
  __shared__ int si[1024];
  int t = threadIdx.x, nt = blockDim.x;
  for (int k = 0; k < n; ++k) {
    double best = -1.0;
    int bi = n;
    for (int i = k + t; i < n; i += nt) {
      double v = fabs(a[(size_t)i * n + k]);
      if (v > best || (v == best && i < bi)) { best = v; bi = i; }
    }
    sv[t] = best; si[t] = bi;
    __syncthreads();
    for (int o = nt / 2; o > 0; o >>= 1) {
      if (t < o) {
        double v = sv[t + o];
        int i = si[t + o];
        if (v > sv[t] || (v == sv[t] && i < si[t])) { sv[t] = v; si[t] = i; }
      }
      __syncthreads();
    }
    int p = si[0];
    if (p < k || p >= n) p = k;           // no finite candidate (NaN column)
    __syncthreads();
    if (t == 0) piv[k] = p;
    if (p != k)
      for (int j = t; j < n; j += nt) {
        double tmp = a[(size_t)k * n + j];
        a[(size_t)k * n + j] = a[(size_t)p * n + j];
        a[(size_t)p * n + j] = tmp;
      }
    __syncthreads();
    double d = a[(size_t)k * n + k];
    if (d != 0.0) {
      for (int i = k + 1 + t; i < n; i += nt) a[(size_t)i * n + k] /= d;
      __syncthreads();
      int m = n - k - 1;
      for (int q = t; q < m * m; q += nt) {
        int i = k + 1 + q / m, j = k + 1 + q % m;
        a[(size_t)i * n + j] -= a[(size_t)i * n + k] * a[(size_t)k * n + j];
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(1024) k_dense_solve(int n, const double *a, const int *piv,
                                                      const double *b, double *x) {
  int t = threadIdx.x, nt = blockDim.x;
  for (int i = t; i < n; i += nt) x[i] = b[i];
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (t == 0) {
      int p = piv[k];
      if (p != k && p >= 0 && p < n) { double tmp = x[k]; x[k] = x[p]; x[p] = tmp; }
    }
    __syncthreads();
    double xk = x[k];
    for (int i = k + 1 + t; i < n; i += nt) x[i] -= a[(size_t)i * n + k] * xk;
    __syncthreads();
  }
  for (int i = n - 1; i >= 0; --i) {
    if (t == 0) { double d = a[(size_t)i * n + i]; x[i] = d != 0.0 ? x[i] / d : 0.0; }
    __syncthreads();
    double xi = x[i];
    for (int r = t; r < i; r += nt) x[r] -= a[(size_t)r * n + i] * xi;
    __syncthreads();
  }
}

constexpr int kDenseMax = 4096;

int coarse_factor(Sim *s) {
  Level &L = s->lev.back();
  int n = L.n;
  if (n > kDenseMax || n == 0) { s->coarse_n = 0; return DP_OK; }
  if (!s->coarse_lu || s->coarse_n != n) {
    if (s->coarse_lu) dfree(s, s->coarse_lu);
    if (s->coarse_piv) dfree(s, s->coarse_piv);
    s->coarse_lu = (double *)dalloc(s, (size_t)n * n * 8);
    s->coarse_piv = (int *)dalloc(s, (size_t)n * 4);
    if (!s->coarse_lu || !s->coarse_piv) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
  }
  s->coarse_n = n;
  DP_LAUNCH(s, k_csr_to_dense, nblk(n), kBlock, 0, n, L.rowptr, L.col, L.val, s->coarse_lu);
  DP_LAUNCH(s, k_dense_lu, 1, 1024, 0, n, s->coarse_lu, s->coarse_piv);
  DP_CUDA(s, cudaGetLastError());
  return DP_OK;
}

static int gs_sweep(Sim *s, Level &L, const double *b, double *x, bool forward) {
  for (int t = 0; t < L.ncolour; ++t) {
    int c = forward ? t : L.ncolour - 1 - t;
    int r0 = L.cstart[c], r1 = L.cstart[c + 1];
    if (r1 > r0) {
      long long thr = (long long)(r1 - r0) * L.G;
      DP_SWITCH_G(L.G, DP_LAUNCH(s, k_gs_colour<GG>, nblk(thr), kBlock, 0, r0, r1, L.clist,
                                 L.rowptr, L.col, L.val, L.dpos, b, x));
    }
  }
  return DP_OK;
}

int vcycle(Sim *s, int l, const double *b, double *x) {
  Level &L = s->lev[l];
  int n = L.n;
  if (l == (int)s->lev.size() - 1) {
    if (s->coarse_n == n && n > 0) {
      DP_LAUNCH(s, k_dense_solve, 1, 1024, 0, n, s->coarse_lu, s->coarse_piv, b, x);
      return DP_OK;
    }
    DP_CUDA(s, cudaMemsetAsync(x, 0, (size_t)n * 8, s->stream));
    DP_TRY(gs_sweep(s, L, b, x, true));
    DP_TRY(gs_sweep(s, L, b, x, false));
    return DP_OK;
  }
  Level &N = s->lev[l + 1];
  DP_CUDA(s, cudaMemsetAsync(x, 0, (size_t)n * 8, s->stream));
  DP_TRY(gs_sweep(s, L, b, x, true));
  DP_TRY(csr_resid(s, L, b, x, L.r));
  DP_TRY(csr_mv(s, N.n, L.r_G, L.r_rowptr, L.r_col, L.r_val, L.r, N.b, 0));
  DP_TRY(vcycle(s, l + 1, N.b, N.x));
  DP_TRY(csr_mv(s, n, L.p_G, L.p_rowptr, L.p_col, L.p_val, N.x, x, 1));
  DP_TRY(gs_sweep(s, L, b, x, false));
  return DP_OK;
}

// ---------------------------------------------------------------- CPR-FPF
// z1 = F r;  z2 = z1 + P V(R (r - A z1));  z = z2 + F (r - A z2)

__global__ void k_inject_add(int n, const double *xp, double *z) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[2 * i] += xp[i];
}

__global__ void k_axpy1(long long n, const double *x, double *y) {  // y += x
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += x[i];
}

int cpr_apply(Sim *s, const double *r, double *z) {
  int nb = s->A.n;
  long long N = 2LL * nb;
  if (s->opt.precond == 0) {
    DP_CUDA(s, cudaMemcpyAsync(z, r, N * 8, cudaMemcpyDeviceToDevice, s->stream));
    return DP_OK;
  }
  if (s->opt.precond == 1) return ilu_apply(s, r, z);
  DP_TRY(ilu_apply(s, r, s->z1));
  DP_LAUNCH(s, k_bsr_presid, nblk(nb), kBlock, 0, nb, s->A.rowptr, s->A.col, s->A.val, s->z1, r,
            s->rp);
  DP_TRY(vcycle(s, 0, s->rp, s->xp));
  DP_LAUNCH(s, k_inject_add, nblk(nb), kBlock, 0, nb, s->xp, s->z1);
  DP_TRY(bsr_residual(s, r, s->z1, s->r1));
  DP_TRY(ilu_apply(s, s->r1, z));
  DP_LAUNCH(s, k_axpy1, nblk(N), kBlock, 0, N, s->z1, z);
  return DP_OK;
}

// ---------------------------------------------------------------- FGMRES
// Deterministic reductions: a fixed grid of kDotBlocks blocks writes one
// partial per vector, a single warp sums the partials in block order.
constexpr int kDotBlocks = 608;   // 4 x 152 SMs
constexpr int kDotVec = 8;        // vectors per pass

__global__ void __launch_bounds__(kBlock) k_multidot(long long N, const double *__restrict__ V,
                                                     long long ldv, int nv,
                                                     const double *__restrict__ w,
                                                     double *__restrict__ part, int part_off) {
  double acc[kDotVec];
#pragma unroll
  for (int k = 0; k < kDotVec; ++k) acc[k] = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    double wi = w[i];
#pragma unroll
    for (int k = 0; k < kDotVec; ++k)
      if (k < nv) acc[k] += V[k * ldv + i] * wi;
  }
  __shared__ double sh[kBlock / 32][kDotVec];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kDotVec; ++k) {
    double v = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[wid][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double v = 0.0;
    for (int q = 0; q < kBlock / 32; ++q) v += sh[q][threadIdx.x];
    part[(size_t)blockIdx.x * 32 + part_off + threadIdx.x] = v;
  }
}

// dots[k] = sum_b part[b][k] (fixed order); mode 1: also add into H[:, j];
// mode 2: dots[0] = sqrt(sum), H[j+1][j] = it.
__global__ void k_dot_final(const double *part, int nblocks, int nv, double *dots, double *H,
                            int m, int j, int mode) {
  int k = threadIdx.x;
  if (k >= nv) return;
  double v = 0.0;
  for (int b = 0; b < nblocks; ++b) v += part[(size_t)b * 32 + k];
  if (mode == 2) { v = sqrt(v); dots[0] = v; H[(size_t)(j + 1) * m + j] = v; return; }
  dots[k] = v;
  if (mode == 1) H[(size_t)k * m + j] += v;
}

// w -= sum_k c_k V_k (sign -1) or w += sum_k c_k V_k (sign +1)
__global__ void __launch_bounds__(kBlock) k_multi_axpy(long long N, const double *__restrict__ V,
                                                       long long ldv, int nv,
                                                       const double *__restrict__ c, double sign,
                                                       double *__restrict__ w) {
  __shared__ double cs[32];
  if (threadIdx.x < nv) cs[threadIdx.x] = sign * c[threadIdx.x];
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    double acc = w[i];
    for (int k = 0; k < nv; ++k) acc += cs[k] * V[k * ldv + i];
    w[i] = acc;
  }
}

__global__ void k_scale(long long N, const double *x, const double *alpha, int invert, double *y) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double a = *alpha;
  if (invert) a = a != 0.0 ? 1.0 / a : 0.0;
  if (i < N) y[i] = x[i] * a;
}

// Givens rotations on column j of the Hessenberg matrix and the rotated
// right-hand side g; res_out = |g_{j+1}|.
__global__ void k_givens(double *H, double *cs, double *sn, double *g, int m, int j,
                         double *res_out) {
  if (threadIdx.x != 0) return;
  for (int i = 0; i < j; ++i) {
    double a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
    H[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
    H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
  }
  double a = H[(size_t)j * m + j], c = H[(size_t)(j + 1) * m + j];
  double r = sqrt(a * a + c * c);
  if (r == 0.0) { cs[j] = 1.0; sn[j] = 0.0; }
  else { cs[j] = a / r; sn[j] = c / r; }
  H[(size_t)j * m + j] = r;
  H[(size_t)(j + 1) * m + j] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  *res_out = fabs(g[j + 1]);
}

__global__ void k_backsub(const double *H, const double *g, int m, int jend, double *y) {
  if (threadIdx.x != 0) return;
  for (int i = jend - 1; i >= 0; --i) {
    double s = g[i];
    for (int k = i + 1; k < jend; ++k) s -= H[(size_t)i * m + k] * y[k];
    double d = H[(size_t)i * m + i];
    y[i] = d != 0.0 ? s / d : 0.0;
  }
}

__global__ void k_init_g(double *g, int m, const double *beta) {
  int i = threadIdx.x;
  if (i <= m) g[i] = i == 0 ? *beta : 0.0;
}

static int dots(Sim *s, const double *V, long long ldv, int nv, const double *w, int mode, int j) {
  long long N = 2LL * s->A.n;
  for (int v0 = 0; v0 < nv; v0 += kDotVec) {
    int cnt = std::min(kDotVec, nv - v0);
    DP_LAUNCH(s, k_multidot, kDotBlocks, kBlock, 0, N, V + (long long)v0 * ldv, ldv, cnt, w,
              s->dots_part, v0);
  }
  DP_LAUNCH(s, k_dot_final, 1, 32, 0, s->dots_part, kDotBlocks, nv, s->dots, s->H, s->m, j, mode);
  return DP_OK;
}

// ||x|| into s->scal[slot] (device) via the dot machinery
static int norm_into(Sim *s, const double *x, double *dst) {
  long long N = 2LL * s->A.n;
  DP_LAUNCH(s, k_multidot, kDotBlocks, kBlock, 0, N, x, 0LL, 1, x, s->dots_part, 0);
  DP_LAUNCH(s, k_dot_final, 1, 32, 0, s->dots_part, kDotBlocks, 1, dst, s->H, s->m, 0, 0);
  return DP_OK;
}

__global__ void k_sqrt_inplace(double *v) { v[0] = sqrt(v[0]); }

// One Arnoldi step of FGMRES for column j: z_j = M v_j, w = A z_j, two
// passes of classical Gram-Schmidt, h_{j+1,j} = ||w||, v_{j+1} = w / h, the
// Givens rotations, and |g_{j+1}| into scal[3].
static int arnoldi_step(Sim *s, int j) {
  int m = s->m;
  long long N = 2LL * s->A.n;
  int gridN = (int)std::min<long long>(nblk(N), kDotBlocks * 4);
  double *vj = s->V + (long long)j * N, *zj = s->Z + (long long)j * N;
  DP_TRY(cpr_apply(s, vj, zj));
  DP_TRY(bsr_spmv(s, zj, s->w));
  for (int pass = 0; pass < 2; ++pass) {
    DP_TRY(dots(s, s->V, N, j + 1, s->w, 1, j));
    DP_LAUNCH(s, k_multi_axpy, gridN, kBlock, 0, N, s->V, N, j + 1, s->dots, -1.0, s->w);
  }
  DP_LAUNCH(s, k_multidot, kDotBlocks, kBlock, 0, N, s->w, 0LL, 1, s->w, s->dots_part, 0);
  DP_LAUNCH(s, k_dot_final, 1, 32, 0, s->dots_part, kDotBlocks, 1, s->scal + 2, s->H, m, j, 2);
  DP_LAUNCH(s, k_scale, nblk(N), kBlock, 0, N, s->w, s->scal + 2, 1, s->V + (long long)(j + 1) * N);
  DP_LAUNCH(s, k_givens, 1, 32, 0, s->H, s->cs, s->sn, s->g, m, j, s->scal + 3);
  return DP_OK;
}

void graphs_free(Sim *s) {
  for (cudaGraphExec_t &g : s->graph)
    if (g) { cudaGraphExecDestroy(g); g = nullptr; }
  s->graph.clear();
  s->graph_launches.clear();
}

// Run Arnoldi step j, from a CUDA graph captured on its first use (the
// capture goes through a private stream; the graph is launched on the
// simulation stream).
static int arnoldi_step_graph(Sim *s, int j) {
  if ((int)s->graph.size() < s->m) {
    s->graph.assign(s->m, nullptr);
    s->graph_launches.assign(s->m, 0);
  }
  if (!s->graph[j]) {
    if (!s->cap_stream) DP_CUDA(s, cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking));
    cudaStream_t user = s->stream;
    // the captured work must follow what is already queued on the user stream
    DP_CUDA(s, cudaStreamSynchronize(user));
    s->stream = s->cap_stream;
    DP_CUDA(s, cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
    int64_t l0 = s->launches;
    int rc = arnoldi_step(s, j);
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(s->cap_stream, &g);
    s->stream = user;
    int64_t kernels = s->launches - l0;   // kernels recorded, not yet run
    s->launches = l0;
    if (rc != DP_OK) { if (g) cudaGraphDestroy(g); return rc; }
    if (ce != cudaSuccess) { s->fail(DP_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ce)); return DP_ECUDA; }
    cudaGraphExec_t ex = nullptr;
    ce = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) { s->fail(DP_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce)); return DP_ECUDA; }
    s->graph[j] = ex;
    s->graph_launches[j] = kernels;
  }
  DP_CUDA(s, cudaGraphLaunch(s->graph[j], s->stream));
  s->launches += s->graph_launches[j];
  return DP_OK;
}

int fgmres(Sim *s, double tol, int *iters, double *relres) {
  int m = s->m, maxit = s->opt.gmres_maxit;
  long long N = 2LL * s->A.n;
  bool use_graph = s->opt.use_graphs && s->timing.kernel_id < 0;
  double *x = s->y;
  DP_CUDA(s, cudaMemsetAsync(x, 0, N * 8, s->stream));
  DP_TRY(norm_into(s, s->bh, s->scal + 0));
  DP_LAUNCH(s, k_sqrt_inplace, 1, 1, 0, s->scal + 0);
  DP_CUDA(s, cudaMemcpyAsync(s->h_res, s->scal, 8, cudaMemcpyDeviceToHost, s->stream));
  DP_CUDA(s, cudaStreamSynchronize(s->stream));
  double bnorm = s->h_res[0];
  int total = 0;
  bool conv = false;
  double res = bnorm;
  if (bnorm == 0.0) { conv = true; res = 0.0; }
  int gridN = (int)std::min<long long>(nblk(N), kDotBlocks * 4);
  while (!conv && total < maxit) {
    DP_TRY(bsr_residual(s, s->bh, x, s->V));
    DP_TRY(norm_into(s, s->V, s->scal + 1));
    DP_LAUNCH(s, k_sqrt_inplace, 1, 1, 0, s->scal + 1);
    DP_CUDA(s, cudaMemcpyAsync(s->h_res + 1, s->scal + 1, 8, cudaMemcpyDeviceToHost, s->stream));
    DP_CUDA(s, cudaStreamSynchronize(s->stream));
    double beta = s->h_res[1];
    res = beta;
    if (beta <= tol * bnorm) { conv = true; break; }
    DP_LAUNCH(s, k_scale, nblk(N), kBlock, 0, N, s->V, s->scal + 1, 1, s->V);
    DP_CUDA(s, cudaMemsetAsync(s->H, 0, (size_t)(m + 1) * m * 8, s->stream));
    DP_LAUNCH(s, k_init_g, 1, 64, 0, s->g, m, s->scal + 1);
    int jend = 0;
    for (int j = 0; j < m && total < maxit; ++j) {
      if (use_graph) DP_TRY(arnoldi_step_graph(s, j));
      else DP_TRY(arnoldi_step(s, j));
      DP_CUDA(s, cudaMemcpyAsync(s->h_res + 2, s->scal + 2, 16, cudaMemcpyDeviceToHost, s->stream));
      DP_CUDA(s, cudaStreamSynchronize(s->stream));
      DP_CUDA(s, cudaGetLastError());
      ++total;
      jend = j + 1;
      double hn = s->h_res[2];
      res = s->h_res[3];
      if (res <= tol * bnorm) { conv = true; break; }
      if (hn == 0.0) break;
    }
    DP_LAUNCH(s, k_backsub, 1, 32, 0, s->H, s->g, m, jend, s->hy);
    DP_LAUNCH(s, k_multi_axpy, gridN, kBlock, 0, N, s->Z, N, jend, s->hy, 1.0, x);
    if (jend == 0) break;
  }
  DP_CUDA(s, cudaGetLastError());
  *iters = total;
  *relres = bnorm > 0.0 ? res / bnorm : 0.0;
  return conv ? DP_OK : DP_ELINEAR;
}

int la_alloc(Sim *s) {
  int m = std::max(1, std::min(s->opt.gmres_restart, 30));
  s->m = m;
  long long N = 2LL * s->A.n;
  s->V = (double *)dalloc(s, (size_t)(m + 1) * N * 8);
  s->Z = (double *)dalloc(s, (size_t)m * N * 8);
  s->w = (double *)dalloc(s, (size_t)N * 8);
  s->H = (double *)dalloc(s, (size_t)(m + 1) * m * 8);
  s->cs = (double *)dalloc(s, (size_t)m * 8);
  s->sn = (double *)dalloc(s, (size_t)m * 8);
  s->g = (double *)dalloc(s, (size_t)(m + 1) * 8);
  s->hy = (double *)dalloc(s, (size_t)m * 8);
  s->dots_part = (double *)dalloc(s, (size_t)kDotBlocks * 32 * 8);
  s->dots = (double *)dalloc(s, 32 * 8);
  s->scal = (double *)dalloc(s, 8 * 8);
  s->z1 = (double *)dalloc(s, (size_t)N * 8);
  s->r1 = (double *)dalloc(s, (size_t)N * 8);
  s->rp = (double *)dalloc(s, (size_t)s->A.n * 8);
  s->xp = (double *)dalloc(s, (size_t)s->A.n * 8);
  if (!s->V || !s->Z || !s->w || !s->H || !s->cs || !s->sn || !s->g || !s->hy || !s->dots_part ||
      !s->dots || !s->scal || !s->z1 || !s->r1 || !s->rp || !s->xp) {
    s->fail(DP_ENOMEM, "allocation failed");
    return DP_ENOMEM;
  }
  return DP_OK;
}

int mixed_refresh(Sim *) { return DP_OK; }

}  // namespace dp
