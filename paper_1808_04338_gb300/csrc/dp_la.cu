// Linear algebra of the Newton-step solve (Section 3.2): block SpMV, block
// ILU(0) in colour order, the AMG V-cycle with multicolour Gauss-Seidel, the
// dense coarsest solve, the CPR-FPF preconditioner and flexible GMRES.
#include <algorithm>
#include <cstdio>
#include <string>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "dp_internal.h"
#include "dp_kernels.cuh"
#include "dp_tma.cuh"

namespace dp {

// ---------------------------------------------------------------- BSR SpMV
// Two lanes per block row, one per output component: lane c of row i reads
// row c of every 2x2 block (one 16-byte load; the two lanes of a row read
// the two halves of the same 32-byte block), x_j (16 bytes, shared by the
// pair) and accumulates its own output with FMAs, so no FP64 reduction
// across lanes is needed.  A warp covers 16 block rows.
//
// The operator is read from its storage-order copy (chunks of fracture rows
// then matrix rows, then wells): pair q processes storage row q, whose
// blocks are contiguous with those of pair q+1.  A CTA takes 128 storage
// rows, which are, as a set, the natural rows q0..q0+127, and each lane
// stores its result at natural row row_of_pair(q): the fracture and matrix
// rows of a location are 16 bytes apart, so a 32-byte sector of y is
// written in halves by two warps of the same CTA, which meet in L2 (DRAM
// sees whole sectors).  Staging the results in shared memory for one
// coalesced store instead made the short matrix-row warps wait at the CTA
// barrier for the fracture rows (0.170 against 0.151 ms a product at 8M
// unknowns).


template <int MODE>  // MODE 0: y = A x; 1: y = b - A x
__global__ void __launch_bounds__(kBlock) k_bsr_spmv(int n, int nL, int nc, int nlong,
                                                     const int *__restrict__ rowptr,
                                                     const int *__restrict__ col,
                                                     const double *__restrict__ val,
                                                     const double *__restrict__ x,
                                                     const double *__restrict__ b,
                                                     double *__restrict__ y) {
  k_bsr_spmv_b<MODE>(blockIdx.x, gridDim.x, n, nL, nc, nlong, rowptr, col, val, x, b, y);
}

// lq = R + A y over every block row of the Jacobian as assembled (natural
// order): the linear residual of the Newton equation A y = -R, whose scaled
// norms the forcing terms 1 and 2 of Section 3.1 take.  Two lanes per cell
// block row, one per component, the rows taken in the storage order of the
// Krylov operator's copy (as in k_bsr_spmv) so that a warp's rows have one
// length; the well rows a warp each in block 0.  Natural order throughout.
__global__ void __launch_bounds__(kBlock) k_lin_residual(int n, int nL, int nc,
                                                         const int *__restrict__ rowptr,
                                                         const int *__restrict__ col,
                                                         const double *__restrict__ val,
                                                         const double *__restrict__ R,
                                                         const double *__restrict__ y,
                                                         double *__restrict__ lq) {
  const double2 *y2 = reinterpret_cast<const double2 *>(y);
  if (blockIdx.x == 0) {   // the well rows (long): a warp per row, lanes over its blocks
    int lane = threadIdx.x & 31;
    for (int i = nc + (threadIdx.x >> 5); i < n; i += blockDim.x >> 5) {
      double a0 = 0.0, a1 = 0.0;
      for (int e = __ldg(rowptr + i) + lane, e1 = __ldg(rowptr + i + 1); e < e1; e += 32) {
        const double *b = val + 4 * (size_t)e;
        double2 x = __ldg(y2 + __ldg(col + e));
        a0 = fma(__ldg(b), x.x, fma(__ldg(b + 1), x.y, a0));
        a1 = fma(__ldg(b + 2), x.x, fma(__ldg(b + 3), x.y, a1));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
      }
      if (lane == 0) {
        lq[2 * (size_t)i] = R[2 * (size_t)i] + a0;
        lq[2 * (size_t)i + 1] = R[2 * (size_t)i + 1] + a1;
      }
    }
    return;
  }
  // cell rows in the storage order (row_of_pair): a warp holds rows of one
  // kind (fracture rows of up to 8 blocks, or matrix rows of 2), two lanes a row
  long long t = (long long)(blockIdx.x - 1) * blockDim.x + threadIdx.x;
  int q = (int)(t >> 1), comp = (int)(t & 1);
  if (q >= nc) return;
  int i = row_of_pair(q, nL, nc);
  const double2 *v2 = reinterpret_cast<const double2 *>(val) + comp;
  double a = R[2 * (size_t)i + comp];
#pragma unroll 4
  for (int e = __ldg(rowptr + i), e1 = __ldg(rowptr + i + 1); e < e1; ++e) {
    double2 b = __ldg(v2 + 2 * (size_t)e);
    double2 x = __ldg(y2 + __ldg(col + e));
    a = fma(b.x, x.x, fma(b.y, x.y, a));
  }
  lq[2 * (size_t)i + comp] = a;
}

int lin_residual(Sim *s) {
  const Bsr &A = s->A;
  // the assembled Jacobian of the full system (also with the Schur option)
  DP_LAUNCH(s, k_lin_residual, 1 + nblk(2LL * s->ph.nc), kBlock, 0, A.n, s->ph.nL, s->ph.nc,
            A.rowptr, A.col, A.val, s->R, s->y, s->lq);
  DP_CUDA(s, cudaGetLastError());
  return DP_OK;
}

// Pressure component of b - A x: rp_i = b_{i,0} - sum_j (a00 x_j0 + a01 x_j1),
// from the contiguous copies of the (0,0) and (0,1) entries that the
// decoupling writes (the 2x2 blocks would be read half-used).
__global__ void __launch_bounds__(kBlock) k_bsr_presid(int n, int nL, int nc, int nlong,
                                                       const int *__restrict__ rowptr,
                                                       const int *__restrict__ col,
                                                       const double *__restrict__ a00,
                                                       const double *__restrict__ a01,
                                                       const double *__restrict__ x,
                                                       const double *__restrict__ b,
                                                       double *__restrict__ rp,
                                                       const int *__restrict__ omap) {
  if (blockIdx.x == 0) {   // the well rows, a warp per row (as in k_bsr_spmv)
    int lane = threadIdx.x & 31;
    const double2 *x2 = reinterpret_cast<const double2 *>(x);
    for (int row = nlong + (threadIdx.x >> 5); row < n; row += blockDim.x >> 5) {
      double s = 0.0;
      for (int e = __ldg(rowptr + row) + lane, e1 = __ldg(rowptr + row + 1); e < e1; e += 32) {
        double2 xj = __ldg(x2 + __ldg(col + e));
        s = fma(__ldg(a00 + e), xj.x, fma(__ldg(a01 + e), xj.y, s));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) rp[omap ? omap[row] : row] = b[2 * (size_t)row] - s;
    }
    return;
  }
  // a CTA takes storage rows q0..q0+255 (two chunks: the natural rows
  // q0..q0+255 as a set); each thread stores its own row's result (the
  // fracture and matrix halves of a sector meet in L2, as in k_bsr_spmv)
  int t = (blockIdx.x - 1) * kBlock + threadIdx.x;
  if (t < nlong) {
    int row = row_of_pair(t, nL, nc);
    int e0 = __ldg(rowptr + t), e1 = __ldg(rowptr + t + 1);
    const double2 *x2 = reinterpret_cast<const double2 *>(x);
    double s = 0.0;
#pragma unroll 4
    for (int e = e0; e < e1; ++e) {
      double2 xj = __ldg(x2 + __ldg(col + e));
      s = fma(__ldg(a00 + e), xj.x, s);
      s = fma(__ldg(a01 + e), xj.y, s);
    }
    rp[omap ? __ldg(omap + row) : row] = b[2 * (size_t)row] - s;
  }
}

// Residuals inside the CPR preconditioner with the FP32 preconditioner
// (precision 1), from an FP32 copy of the decoupled operator: the stage
// residuals feed the FP32 ILU(0) and the FP32 V-cycle only, so products in
// FP32 (the vectors read in FP64 and rounded) change nothing that the
// preconditioner's own rounding does not already, and take the stage
// residuals off GB300's FP64 pipe.  FGMRES itself (its Arnoldi products,
// restart residuals and orthogonalisation) stays in FP64; a flexible method
// takes any preconditioner.
//
// r = b - A x: the layout and work split of k_bsr_spmv (a CTA of 128
// storage rows writing its natural rows through shared memory), FP32 values
// (16-byte blocks: the lane of component c reads that row as a float2).
__global__ void __launch_bounds__(kBlock) k_bsr_resid_f32(int n, int nL, int nc, int nlong,
                                                         const int *__restrict__ rowptr,
                                                         const int *__restrict__ col,
                                                         const float *__restrict__ valf,
                                                         const float *__restrict__ x,
                                                         const double *__restrict__ b,
                                                         float *__restrict__ y) {
  k_bsr_resid_f32_b(blockIdx.x, gridDim.x, n, nL, nc, nlong, rowptr, col, valf, x, b, y);
}

// The pressure rows of b - A x from the FP32 (a00, a01) pairs, written in
// FP32 straight into the V-cycle's level-0 right-hand side (natural order).
__global__ void __launch_bounds__(kBlock) k_bsr_presid_f32(int n, int nL, int nc, int nlong,
                                                          const int *__restrict__ rowptr,
                                                          const int *__restrict__ col,
                                                          const float2 *__restrict__ pf,
                                                          const float *__restrict__ x,
                                                          const double *__restrict__ b,
                                                          float *__restrict__ rp,
                                                          const int *__restrict__ omap,
                                                          X0Init xi) {
  k_bsr_presid_f32_b(blockIdx.x, gridDim.x, n, nL, nc, nlong, rowptr, col, pf, x, b, rp, omap, xi);
}

int bsr_spmv(Sim *s, const double *x, double *y) {
  DP_LAUNCH(s, k_bsr_spmv<0>, 1 + nblk(2LL * s->sv_long0), kBlock, 0, s->K.n, s->sv_sL, s->sv_sc,
            s->sv_long0,
            s->srowptr, s->scol, s->sval, x, nullptr, y);
  return DP_OK;
}

int bsr_residual(Sim *s, const double *b, const double *x, double *r) {
  DP_LAUNCH(s, k_bsr_spmv<1>, 1 + nblk(2LL * s->sv_long0), kBlock, 0, s->K.n, s->sv_sL, s->sv_sc,
            s->sv_long0,
            s->srowptr, s->scol, s->sval, x, b, r);
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


template <typename T>
__device__ __forceinline__ void mul2(const T *a, const T *b, T *o) {
  T t0 = a[0] * b[0] + a[1] * b[2];
  T t1 = a[0] * b[1] + a[1] * b[3];
  T t2 = a[2] * b[0] + a[3] * b[2];
  T t3 = a[2] * b[1] + a[3] * b[3];
  o[0] = t0; o[1] = t1; o[2] = t2; o[3] = t3;
}

template <typename T>
__device__ __forceinline__ void inv2(T *a) {
  T det = a[0] * a[3] - a[1] * a[2];
  T id = T(1) / det;
  T o0 = a[3] * id, o1 = -a[1] * id, o2 = -a[2] * id, o3 = a[0] * id;
  a[0] = o0; a[1] = o1; a[2] = o2; a[3] = o3;
}

// Update lists of the IKJ factorisation, built once from the pattern: for
// every L block e = (i, k) of a row, the pairs (e2, q) such that block e2 =
// (i, j) of the same row, j after k in the ordering, receives
// A_ij -= L_ik U_kj with q the position of U_kj in row k.
__device__ __forceinline__ int find_in(const int *col, int lo, int hi, int c) {
  for (int t = lo; t < hi; ++t) if (col[t] == c) return t;
  return -1;
}

__global__ void k_ilu_upd(int n, int fill, const int *iperm, const int *lu_rowptr,
                          const int *lu_col, const int *lu_dpos, const int *upd_ptr, int *cnt,
                          int *upd_e2, int *upd_q) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  int s1 = lu_rowptr[r + 1], dp = lu_dpos[r];
  for (int e = lu_rowptr[r]; e < dp; ++e) {
    int rk = iperm[lu_col[e]];
    int ku0 = lu_dpos[rk] + 1, ku1 = lu_rowptr[rk + 1];
    int c = 0, base = fill ? upd_ptr[e] : 0;
    for (int e2 = e + 1; e2 < s1; ++e2) {
      int q = find_in(lu_col, ku0, ku1, lu_col[e2]);
      if (q < 0) continue;
      if (fill) { upd_e2[base + c] = e2; upd_q[base + c] = q; }
      ++c;
    }
    if (!fill) cnt[e] = c;
  }
}

// Storage of the factor ("split layout"): the L blocks of all rows first
// (row r's at Lptr[r]..Lptr[r+1]), then the inverted pivot block of every
// row (at nL + r), then the U blocks (at nL + n + Uptr[r]..); every block's
// column as its permuted position (colp), so that the sweeps work on a
// vector kept in colour order: a colour's rows, their pivots and their
// results are contiguous, and with the greedy colouring of this pattern each
// location has one row per colour, so the neighbours a row gathers sit
// compactly in the earlier colours' segments.

// IKJ block ILU(0) of the rows [r0, r1) of one colour, in precision T: all
// their L blocks refer to rows of earlier colours, which are final.  The
// decoupling has already written the rows' values into the split layout.
// The loops run over the row's entries e in factor order (lu_rowptr, lu_dpos);
// dst[e] is the entry's block in the split layout and the update lists hold
// split-layout positions.
template <typename T>
__global__ void k_ilu_factor(int r0, int r1, int nL, const int *lu_rowptr, const int *lu_dpos,
                             const int *dst, const int *colp, const int *upd_ptr,
                             const int *__restrict__ upd_e2, const int *__restrict__ upd_q,
                             T *lu) {
  int r = r0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= r1) return;
  // every block moves as one 16-byte (FP32) or two 16-byte (FP64) accesses;
  // the index arrays are read-only
  int s0 = __ldg(lu_rowptr + r), dp = __ldg(lu_dpos + r);
  for (int e = s0; e < dp; ++e) {
    int k = __ldg(dst + e);
    int rk = __ldg(colp + k);
    T a[4], piv[4], lik[4];
    Blk<T>::load(lu + 4 * (size_t)k, a);
    Blk<T>::load(lu + 4 * ((size_t)nL + rk), piv);
    mul2<T>(a, piv, lik);                                            // A_ik U_kk^-1
    Blk<T>::store(lu + 4 * (size_t)k, lik);
    for (int p = __ldg(upd_ptr + e), p1 = __ldg(upd_ptr + e + 1); p < p1; ++p) {
      T ukj[4], u[4], c[4];
      Blk<T>::load(lu + 4 * (size_t)__ldg(upd_q + p), ukj);
      mul2<T>(lik, ukj, u);
      T *aij = lu + 4 * (size_t)__ldg(upd_e2 + p);
      Blk<T>::load(aij, c);
      c[0] -= u[0]; c[1] -= u[1]; c[2] -= u[2]; c[3] -= u[3];
      Blk<T>::store(aij, c);
    }
  }
  T d[4];
  Blk<T>::load(lu + 4 * ((size_t)nL + r), d);
  inv2<T>(d);
  Blk<T>::store(lu + 4 * ((size_t)nL + r), d);
}

// Forward sweep of one colour, two lanes per row (one per component):
// zp_r = r_{perm[r]} - sum_{L} L_rk zp_k (unit lower triangle), zp in colour
// order; the right-hand side (natural order) in TR.
template <typename T, typename TR>
__global__ void __launch_bounds__(kBlock) k_ilu_fwd(int r0, int r1, const int *__restrict__ perm,
                                                    const int *__restrict__ Lptr,
                                                    const int *__restrict__ colp,
                                                    const T *__restrict__ lu,
                                                    const TR *__restrict__ rhs, T *zp) {
  griddep_launch_dependents();   // the long rows after this colour (k_ilu_fwd_wp)
  k_ilu_fwd_b<T, TR>(blockIdx.x, gridDim.x, r0, r1, perm, Lptr, colp, lu, rhs, zp);
}

// the same, followed in its last CTA by the next colour's long rows (the
// wells; PIVOT: they are the last colour, their pivots applied as well)
template <typename T, typename TR, bool PIVOT>
__global__ void __launch_bounds__(kBlock, kTailMinBlocks) k_ilu_fwd_t(int r0, int r1, const int *__restrict__ perm,
                                                      const int *__restrict__ Lptr,
                                                      const int *__restrict__ colp,
                                                      const T *__restrict__ lu,
                                                      const TR *__restrict__ rhs, T *zp, int nL,
                                                      Tail tl) {
  for (int bx = blockIdx.x; bx < tl.nb; bx += gridDim.x)
    k_ilu_fwd_b<T, TR>(bx, tl.nb, r0, r1, perm, Lptr, colp, lu, rhs, zp);
  __shared__ int last;
  __syncthreads();
  if (threadIdx.x == 0) last = tail_ticket(tl.ticket);
  __syncthreads();
  if (last)
    ilu_fwd_tail<T, TR, PIVOT>(tl, threadIdx.x >> 5, blockDim.x >> 5, threadIdx.x & 31, nL, perm,
                               Lptr, colp, lu, rhs, zp);
}


// Forward sweep of the first colour, whose rows have no L blocks: zp_r =
// r_{perm[r]}, a copy.  A thread takes kRes rows (r, r + S, ...) with their
// permutation loads, then their right-hand-side loads, issued together.
template <typename T, typename TR>
__global__ void __launch_bounds__(kBlock) k_ilu_fwd_copy(int r0, int r1, const int *__restrict__ perm,
                                                     const TR *__restrict__ rhs, T *zp) {
  k_ilu_fwd_copy_b<T, TR>(blockIdx.x, gridDim.x, r0, r1, perm, rhs, zp);
}

// Backward sweep of one colour (short rows): zp_r = D_r (zp_r - sum_{U}
// U_rj zp_j) with D_r the inverted pivot; a thread per row, kRes rows per
// thread, each row's pivot block and y loaded with its U pointers before the
// U gathers (a two-lanes-per-row version, one output component a lane, was
// 2% slower on the cell colours and 2.3 times slower on the colour before
// the wells, whose rows have at most one U block).
template <typename T>
__global__ void __launch_bounds__(kBlock) k_ilu_bwd_r(int r0, int r1, int nL, int n,
                                                      const int *__restrict__ Uptr,
                                                      const int *__restrict__ colp,
                                                      const T *__restrict__ lu, T *zp) {
  k_ilu_bwd_r_b<T>(blockIdx.x, gridDim.x, r0, r1, nL, n, Uptr, colp, lu, zp);
}


// PIVOT: the colour is the last one (no U blocks), so the backward sweep's
// first step for it, z_r = D_r (y_r - 0), follows at once in the same launch.
template <typename T, typename TR, bool PIVOT>
__global__ void __launch_bounds__(kBlock) k_ilu_fwd_w(int r0, int r1, int nL,
                                                      const int *__restrict__ perm,
                                                      const int *__restrict__ Lptr,
                                                      const int *__restrict__ colp,
                                                      const T *__restrict__ lu,
                                                      const TR *__restrict__ rhs, T *zp) {
  k_ilu_fwd_w_b<T, TR, PIVOT>(blockIdx.x, gridDim.x, r0, r1, nL, perm, Lptr, colp, lu, rhs, zp);
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_ilu_bwd_w(int r0, int r1, int nL, int n,
                                                      const int *__restrict__ Uptr,
                                                      const int *__restrict__ colp,
                                                      const T *__restrict__ lu, T *zp) {
  k_ilu_bwd_w_b<T>(blockIdx.x, gridDim.x, r0, r1, nL, n, Uptr, colp, lu, zp);
}

// Split-layout position of each factor entry, and the permuted column of
// each split-layout block.
__global__ void k_ilu_split(int n, int nL, const int *iperm, const int *lu_rowptr,
                            const int *lu_col, const int *lu_dpos, const int *Lptr,
                            const int *Uptr, int *dst, int *colp) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  int s0 = lu_rowptr[r], dp = lu_dpos[r], s1 = lu_rowptr[r + 1];
  for (int e = s0; e < s1; ++e) {
    int d = e < dp ? Lptr[r] + (e - s0) : (e == dp ? nL + r : nL + n + Uptr[r] + (e - dp - 1));
    dst[e] = d;
    colp[d] = iperm[lu_col[e]];
  }
}

// For natural entry e: its row, its block in the split layout and its
// factor-order position (inverse of lu_src).
__global__ void k_entry_maps(int n, const int *rowptr, const int *lu_rowptr, const int *lu_src,
                             const int *dst, int *erow, int *ilupos, int *l0pos) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  for (int e = rowptr[r]; e < rowptr[r + 1]; ++e) erow[e] = r;
  for (int f = lu_rowptr[r]; f < lu_rowptr[r + 1]; ++f) {
    ilupos[lu_src[f]] = dst[f];
    l0pos[lu_src[f]] = f;
  }
}

// Position of entry (j, i) for every entry (i, j) of the structurally
// symmetric block pattern (columns sorted within rows).
__global__ void k_block_tpos(int n, const int *rowptr, const int *col, int *tpos) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
    int j = col[e], lo = rowptr[j], hi = rowptr[j + 1], t = -1;
    while (lo < hi) {
      int m = (lo + hi) >> 1, c = col[m];
      if (c == i) { t = m; break; }
      if (c < i) lo = m + 1; else hi = m;
    }
    tpos[e] = t;
  }
}

__global__ void k_remap(long long n, const int *map, int *v) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = map[v[i]];
}

__global__ void k_lu_lens(int n, const int *lu_rowptr, const int *lu_dpos, int *nl, int *nu) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  nl[r] = lu_dpos[r] - lu_rowptr[r];
  nu[r] = lu_rowptr[r + 1] - lu_dpos[r] - 1;
}

// longest row of each colour (blocks), for choosing the sweep variant
__global__ void k_colour_maxlen(int n, const int *cstart_dev, int ncolour, const int *rowptr,
                                int *out) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  int c = -1, len = 0;
  if (r < n) {
    c = 0;
    while (c + 1 < ncolour && r >= cstart_dev[c + 1]) ++c;
    len = rowptr[r + 1] - rowptr[r];
  }
  // one atomic per colour present in the warp (rows of a colour are
  // contiguous, so a warp spans one or two colours)
  unsigned same = __match_any_sync(0xffffffffu, c);
  int m = __reduce_max_sync(same, len);
  if (c >= 0 && (threadIdx.x & 31) == __ffs(same) - 1) atomicMax(out + c, m);
}


int block_tpos(Sim *s, int n, const int *rowptr, const int *col, int *tpos) {
  DP_LAUNCH(s, k_block_tpos, nblk(n), kBlock, 0, n, rowptr, col, tpos);
  DP_CUDA(s, cudaGetLastError());
  return DP_OK;
}

int ilu_setup(Sim *s) {
  int n = s->K.n;
  s->colour = (int *)dalloc(s, (size_t)n * 4);
  s->perm = (int *)dalloc(s, (size_t)n * 4);
  s->iperm = (int *)dalloc(s, (size_t)n * 4);
  s->lu_rowptr = (int *)dalloc(s, ((size_t)n + 1) * 4 + 16);   // + the bulk copies' overrun
  s->lu_dpos = (int *)dalloc(s, (size_t)n * 4);
  s->lu_col = (int *)dalloc(s, (size_t)s->K.nnz * 4);
  s->lu_src = (int *)dalloc(s, (size_t)s->K.nnz * 4);
  s->lu_val = (double *)dalloc(s, (size_t)s->K.nnz * 32);
  s->lu_valf = (float *)dalloc(s, (size_t)s->K.nnz * 16);
  int *len = (int *)dalloc(s, (size_t)n * 4);
  if (!s->colour || !s->perm || !s->iperm || !s->lu_rowptr || !s->lu_dpos || !s->lu_col ||
      !s->lu_src || !s->lu_val || !s->lu_valf || !len) {
    s->fail(DP_ENOMEM, "allocation failed");
    return DP_ENOMEM;
  }
  DP_TRY(greedy_colour(s, n, s->K.rowptr, s->K.col, s->colour, &s->ncolour));
  DP_TRY(colour_lists(s, n, s->colour, s->ncolour, s->perm, s->lu_cstart, s->iperm));
  DP_LAUNCH(s, k_perm_len, nblk(n), kBlock, 0, n, s->perm, s->K.rowptr, len);
  int nnz = 0;
  DP_TRY(scan_i32(s, len, s->lu_rowptr, n, &nnz));
  DP_LAUNCH(s, k_lu_pattern, nblk(n), kBlock, 0, n, s->perm, s->iperm, s->K.rowptr, s->K.col,
            s->lu_rowptr, s->lu_col, s->lu_src, s->lu_dpos);
  {
    int nc = s->ncolour;
    int *dev = (int *)dalloc(s, (size_t)(2 * nc + 2) * 4);
    if (!dev) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
    DP_CUDA(s, cudaMemcpyAsync(dev, s->lu_cstart.data(), (size_t)(nc + 1) * 4,
                               cudaMemcpyHostToDevice, s->stream));
    DP_CUDA(s, cudaMemsetAsync(dev + nc + 1, 0, (size_t)nc * 4, s->stream));
    DP_LAUNCH(s, k_colour_maxlen, nblk(n), kBlock, 0, n, dev, nc, s->lu_rowptr, dev + nc + 1);
    s->lu_cmaxlen.assign(nc, 0);
    DP_CUDA(s, cudaMemcpyAsync(s->lu_cmaxlen.data(), dev + nc + 1, (size_t)nc * 4,
                               cudaMemcpyDeviceToHost, s->stream));
    DP_CUDA(s, cudaStreamSynchronize(s->stream));
    dfree(s, dev);
  }
  // update lists of the factorisation
  int *cnt = (int *)dalloc(s, (size_t)nnz * 4);
  s->upd_ptr = (int *)dalloc(s, ((size_t)nnz + 1) * 4);
  if (!cnt || !s->upd_ptr) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
  DP_CUDA(s, cudaMemsetAsync(cnt, 0, (size_t)nnz * 4, s->stream));
  DP_LAUNCH(s, k_ilu_upd, nblk(n), kBlock, 0, n, 0, s->iperm, s->lu_rowptr, s->lu_col, s->lu_dpos,
            s->upd_ptr, cnt, nullptr, nullptr);
  int npairs = 0;
  DP_TRY(scan_i32(s, cnt, s->upd_ptr, nnz, &npairs));
  s->upd_e2 = (int *)dalloc(s, (size_t)std::max(npairs, 1) * 4);
  s->upd_q = (int *)dalloc(s, (size_t)std::max(npairs, 1) * 4);
  if (!s->upd_e2 || !s->upd_q) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
  DP_LAUNCH(s, k_ilu_upd, nblk(n), kBlock, 0, n, 1, s->iperm, s->lu_rowptr, s->lu_col, s->lu_dpos,
            s->upd_ptr, cnt, s->upd_e2, s->upd_q);
  // split layout: L and U row pointers, each entry's block, permuted columns
  int *nu = cnt;   // reused: n <= nnz
  s->lu_Lptr = (int *)dalloc(s, ((size_t)n + 1) * 4);
  s->lu_Uptr = (int *)dalloc(s, ((size_t)n + 1) * 4);
  s->lu_dst = (int *)dalloc(s, (size_t)nnz * 4);
  s->lu_colp = (int *)dalloc(s, (size_t)nnz * 4);
  s->ilu_zp = (double *)dalloc(s, (size_t)2 * n * 8);
  s->ilu_zp2 = (double *)dalloc(s, (size_t)2 * n * 4);   // the FP32 second result
  if (!s->lu_Lptr || !s->lu_Uptr || !s->lu_dst || !s->lu_colp || !s->ilu_zp || !s->ilu_zp2) {
    s->fail(DP_ENOMEM, "allocation failed");
    return DP_ENOMEM;
  }
  DP_LAUNCH(s, k_lu_lens, nblk(n), kBlock, 0, n, s->lu_rowptr, s->lu_dpos, len, nu);
  int nL = 0, nU = 0;
  DP_TRY(scan_i32(s, len, s->lu_Lptr, n, &nL));
  DP_TRY(scan_i32(s, nu, s->lu_Uptr, n, &nU));
  if (nL + nU + n != nnz) { s->fail(DP_EINVAL, "ILU(0) pattern without a pivot per row"); return DP_EINVAL; }
  s->lu_nL = nL;
  DP_LAUNCH(s, k_ilu_split, nblk(n), kBlock, 0, n, nL, s->iperm, s->lu_rowptr, s->lu_col,
            s->lu_dpos, s->lu_Lptr, s->lu_Uptr, s->lu_dst, s->lu_colp);
  if (npairs > 0) {
    DP_LAUNCH(s, k_remap, nblk(npairs), kBlock, 0, (long long)npairs, s->lu_dst, s->upd_e2);
    DP_LAUNCH(s, k_remap, nblk(npairs), kBlock, 0, (long long)npairs, s->lu_dst, s->upd_q);
  }
  // maps for the decoupling's writes
  s->erow = (int *)dalloc(s, (size_t)nnz * 4);
  s->ilupos = (int *)dalloc(s, (size_t)nnz * 4);
  s->l0pos = (int *)dalloc(s, (size_t)nnz * 4);
  s->fct = (double *)dalloc(s, (size_t)n * 32);
  s->btpos = (int *)dalloc(s, (size_t)nnz * 4);
  if (!s->erow || !s->ilupos || !s->l0pos || !s->fct || !s->btpos) {
    s->fail(DP_ENOMEM, "allocation failed");
    return DP_ENOMEM;
  }
  DP_LAUNCH(s, k_entry_maps, nblk(n), kBlock, 0, n, s->K.rowptr, s->lu_rowptr, s->lu_src,
            s->lu_dst, s->erow, s->ilupos, s->l0pos);
  DP_LAUNCH(s, k_block_tpos, nblk(n), kBlock, 0, n, s->K.rowptr, s->K.col, s->btpos);
  DP_CUDA(s, cudaGetLastError());
  dfree(s, cnt);
  dfree(s, len);
  return DP_OK;
}

int ilu_factor(Sim *s) {
  bool f32 = s->opt.precision >= 1;
  for (int c = 0; c < s->ncolour; ++c) {
    int r0 = s->lu_cstart[c], r1 = s->lu_cstart[c + 1];
    if (r1 <= r0) continue;
    if (f32)
      DP_LAUNCH(s, k_ilu_factor<float>, nblk(r1 - r0, 128), 128, 0, r0, r1, s->lu_nL,
                s->lu_rowptr, s->lu_dpos, s->lu_dst, s->lu_colp, s->upd_ptr, s->upd_e2, s->upd_q,
                s->lu_valf);
    else
      DP_LAUNCH(s, k_ilu_factor<double>, nblk(r1 - r0, 128), 128, 0, r0, r1, s->lu_nL,
                s->lu_rowptr, s->lu_dpos, s->lu_dst, s->lu_colp, s->upd_ptr, s->upd_e2, s->upd_q,
                s->lu_val);
  }
  DP_CUDA(s, cudaGetLastError());
  return DP_OK;
}

// CTAs of a launch with a long-row tail: one wave (kTailMinBlocks an SM) at
// most, walking the launch's nb blocks of rows
static int tail_grid(int nb) {
  static const int slots = []() {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return std::max(nsm, 1) * kTailMinBlocks;
  }();
  return std::max(1, std::min(nb, slots));
}

// The same long rows as a programmatic dependent of the colour launch before
// them (class kPdlIluW), a one-warp CTA per row: the row's pointers, its
// first 64 L blocks and their columns, its permutation and (PIVOT) its
// inverted pivot, which no kernel of the solve writes, are loaded before
// griddep_wait; zp and the right-hand side after it.  The products and
// their order are k_ilu_fwd_w_b's, so the results are the same bit for bit.
template <typename T, typename TR, bool PIVOT>
__global__ void __launch_bounds__(32) k_ilu_fwd_wp(int r0, int nL, const int *__restrict__ perm,
                                                   const int *__restrict__ Lptr,
                                                   const int *__restrict__ colp,
                                                   const T *__restrict__ lu, const TR *rhs,
                                                   T *zp) {
  using T2 = typename V2<T>::t;
  const T2 *z2 = reinterpret_cast<const T2 *>(zp);
  int r = r0 + (int)blockIdx.x, lane = threadIdx.x;
  int e = __ldg(Lptr + r) + lane, eb = __ldg(Lptr + r + 1);
  bool h0 = e < eb, h1 = e + 32 < eb;
  T a0[4] = {T(0), T(0), T(0), T(0)}, a1[4] = {T(0), T(0), T(0), T(0)}, d[4];
  int c0 = 0, c1 = 0;
  if (h0) {
    V4<T>::load(lu + 4 * (size_t)e, a0);
    c0 = __ldg(colp + e);
  }
  if (h1) {
    V4<T>::load(lu + 4 * (size_t)(e + 32), a1);
    c1 = __ldg(colp + e + 32);
  }
  int i = lane == 0 ? __ldg(perm + r) : 0;
  if (PIVOT && lane == 0) V4<T>::load(lu + 4 * ((size_t)nL + r), d);
  griddep_wait();
  T s0 = T(0), s1 = T(0);
  if (h0) {
    T2 xk = z2[c0];
    s0 = fma(a0[0], xk.x, fma(a0[1], xk.y, s0));
    s1 = fma(a0[2], xk.x, fma(a0[3], xk.y, s1));
  }
  if (h1) {
    T2 xk = z2[c1];
    s0 = fma(a1[0], xk.x, fma(a1[1], xk.y, s0));
    s1 = fma(a1[2], xk.x, fma(a1[3], xk.y, s1));
  }
  for (e += 64; e < eb; e += 32) {
    T a[4];
    V4<T>::load(lu + 4 * (size_t)e, a);
    T2 xk = z2[__ldg(colp + e)];
    s0 = fma(a[0], xk.x, fma(a[1], xk.y, s0));
    s1 = fma(a[2], xk.x, fma(a[3], xk.y, s1));
  }
  s0 = warp_sum(s0);
  s1 = warp_sum(s1);
  if (lane == 0) {
    T y0 = T(rhs[2 * (size_t)i]) - s0, y1 = T(rhs[2 * (size_t)i + 1]) - s1;
    if (PIVOT) {
      y0 = y0 - T(0);   // the backward sweep's y - (sum over no U blocks)
      y1 = y1 - T(0);
      zp[2 * (size_t)r] = fma(d[0], y0, d[1] * y1);
      zp[2 * (size_t)r + 1] = fma(d[2], y0, d[3] * y1);
    } else {
      zp[2 * (size_t)r] = y0;
      zp[2 * (size_t)r + 1] = y1;
    }
  }
}

// (LU)^-1 r with the factor in T and r (natural order) in TR; the result
// is left in the colour-order work vector s->ilu_zp, from which the caller
// gathers it (ilu_result) while converting or accumulating.
template <typename T, typename TR>
static int ilu_apply_t(Sim *s, const T *lu, const TR *r, T *zpo = nullptr) {
  int n = s->K.n, nL = s->lu_nL, nc = s->ncolour;
  T *zp = zpo ? zpo : reinterpret_cast<T *>(s->ilu_zp);
  // with kPdlIluW the long rows are a launch of their own, a programmatic
  // dependent of the colour before them; otherwise that colour's last CTA
  // takes them (a tail)
  bool wp = (pdl_mode() & kPdlIluW) != 0;
  // the last colour is solved forward and its pivots applied in one launch:
  // its rows have no U blocks, so that is also the backward sweep's first step
  int last = nc - 1;
  while (last >= 0 && s->lu_cstart[last + 1] <= s->lu_cstart[last]) --last;
  int first = 0;
  while (first < nc && s->lu_cstart[first + 1] <= s->lu_cstart[first]) ++first;
  {
  RegionScope region(s, "sweep.ilu_fwd");   // the forward sweep's launches, timed as one
  for (int c = 0; c < nc; ++c) {
    int r0 = s->lu_cstart[c], r1 = s->lu_cstart[c + 1];
    if (r1 <= r0) continue;
    int nx = c + 1;   // the next non-empty colour
    while (nx < nc && s->lu_cstart[nx + 1] <= s->lu_cstart[nx]) ++nx;
    if (!wp && c != first && s->lu_cmaxlen[c] <= kLongRow && nx < nc &&
        s->lu_cmaxlen[nx] > kLongRow) {
      // a short colour followed by a long one: its last CTA takes the long rows
      Tail tl;
      tl.w0 = s->lu_cstart[nx];
      tl.w1 = s->lu_cstart[nx + 1];
      tl.ticket = s->tickets;
      tl.nb = nblk(2LL * (r1 - r0));
      if (nx == last)
        DP_LAUNCH(s, (k_ilu_fwd_t<T, TR, true>), tail_grid(tl.nb), kBlock, 0, r0, r1, s->perm,
                  s->lu_Lptr, s->lu_colp, lu, r, zp, nL, tl);
      else
        DP_LAUNCH(s, (k_ilu_fwd_t<T, TR, false>), tail_grid(tl.nb), kBlock, 0, r0, r1, s->perm,
                  s->lu_Lptr, s->lu_colp, lu, r, zp, nL, tl);
      c = nx;
      continue;
    }
    if (wp && c != first && s->lu_cmaxlen[c] > kLongRow) {
      if (c == last)
        DP_LAUNCH_PDL(s, kPdlIluW, (k_ilu_fwd_wp<T, TR, true>), r1 - r0, 32, 0, r0, nL, s->perm,
                      s->lu_Lptr, s->lu_colp, lu, r, zp);
      else
        DP_LAUNCH_PDL(s, kPdlIluW, (k_ilu_fwd_wp<T, TR, false>), r1 - r0, 32, 0, r0, nL, s->perm,
                      s->lu_Lptr, s->lu_colp, lu, r, zp);
    } else if (c == last && s->lu_cmaxlen[c] > kLongRow)
      DP_LAUNCH(s, (k_ilu_fwd_w<T, TR, true>), nblk(32LL * (r1 - r0)), kBlock, 0, r0, r1, nL,
                s->perm, s->lu_Lptr, s->lu_colp, lu, r, zp);
    else if (s->lu_cmaxlen[c] > kLongRow)
      DP_LAUNCH(s, (k_ilu_fwd_w<T, TR, false>), nblk(32LL * (r1 - r0)), kBlock, 0, r0, r1, nL,
                s->perm, s->lu_Lptr, s->lu_colp, lu, r, zp);
    else if (c == first)   // no L blocks
      DP_LAUNCH(s, (k_ilu_fwd_copy<T, TR>), nblk((r1 - r0 + kRes - 1) / kRes), kBlock, 0, r0, r1,
                s->perm, r, zp);
    else
      DP_LAUNCH(s, (k_ilu_fwd<T, TR>), nblk(2LL * (r1 - r0)), kBlock, 0, r0, r1, s->perm,
                s->lu_Lptr, s->lu_colp, lu, r, zp);
  }
  }
  RegionScope region(s, "sweep.ilu_bwd");   // the backward sweep's launches, timed as one
  for (int c = nc - 1; c >= 0; --c) {
    int r0 = s->lu_cstart[c], r1 = s->lu_cstart[c + 1];
    if (r1 <= r0) continue;
    if (c == last && s->lu_cmaxlen[c] > kLongRow) continue;   // done with the forward launch
    if (s->lu_cmaxlen[c] > kLongRow)
      DP_LAUNCH(s, k_ilu_bwd_w<T>, nblk(32LL * (r1 - r0)), kBlock, 0, r0, r1, nL, n,
                s->lu_Uptr, s->lu_colp, lu, zp);
    else
      DP_LAUNCH(s, k_ilu_bwd_r<T>, nblk((r1 - r0 + kRes - 1) / kRes), kBlock, 0, r0, r1, nL, n,
                s->lu_Uptr, s->lu_colp, lu, zp);
  }
  return DP_OK;
}

// out_i = base_i + zp_{iperm[i]} (base may be NULL: out_i = zp_{iperm[i]}),
// natural order, FP64; two lanes per block row.
// out_i = base_i + zp_{iperm[i]} (base may be NULL), natural order, FP64,
// and optionally the result in T.  A thread takes kRes rows (i, i + S, ...,
// S the thread count), all their index loads first, then all their gathers:
// with one row per thread the launch is a chain of dependent loads per
// thread and stays far below the bandwidth.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_ilu_result(int n, const int *__restrict__ iperm,
                                                       const T *__restrict__ zp,
                                                       const double *__restrict__ base,
                                                       double *__restrict__ out,
                                                       T *__restrict__ outT,
                                                       const float *__restrict__ inj,
                                                       int inj_perm, const T *__restrict__ zb) {
  k_ilu_result_b<T>(blockIdx.x, gridDim.x, n, iperm, zp, base, out, outT, inj, inj_perm, zb);
}

// out = base + result; with inj, out = (base + inj injected) + result, inj
// (a level-0 vector, natural or, with inj_perm, colour order) added to the
// base's pressure component first.  out may be NULL (only outT written);
// zb, a colour-order vector in T, may stand for the base (widened exactly);
// zp: the colour-order result (s->ilu_zp by default).
template <typename T>
static int ilu_result(Sim *s, const double *base, double *out, T *outT = nullptr,
                      const float *inj = nullptr, int inj_perm = 0, const T *zb = nullptr,
                      const T *zp = nullptr) {
  int n = s->K.n;
  DP_LAUNCH(s, k_ilu_result<T>, nblk((n + kRes - 1) / kRes), kBlock, 0, n, s->iperm,
            zp ? zp : reinterpret_cast<const T *>(s->ilu_zp), base, out, outT, inj, inj_perm, zb);
  return DP_OK;
}

int ilu_apply(Sim *s, const double *r, double *z) {
  DP_TRY((ilu_apply_t<double, double>(s, s->lu_val, r)));
  return ilu_result<double>(s, nullptr, z);
}

// ---------------------------------------------------------------- AMG cycle


// One colour of Gauss-Seidel: x_i = (b_i - sum_{j != i} a_ij x_j) / a_ii,
// evaluated as x_i + (b_i - (A x)_i) / a_ii with 1/a_ii precomputed per level
// (0 where a_ii = 0: the row is left as is).
template <int G, typename T, typename TV = T>
__global__ void __launch_bounds__(kBlock) k_gs_colour(int r0, int r1, const int *__restrict__ clist,
                                                      const int *__restrict__ rowptr,
                                                      const int *__restrict__ col,
                                                      const TV *__restrict__ val,
                                                      const T *__restrict__ dinv,
                                                      const T *__restrict__ b, T *x) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int q = r0 + t / G, lane = t % G;
  bool valid = q < r1;
  int i = valid ? clist[q] : 0;
  int e0 = valid ? rowptr[i] : 0, e1 = valid ? rowptr[i + 1] : 0;
  T s = row_dot<G, T, TV>(e0, e1, lane, col, val, x);
  if (G > 1) s = group_sum<G, T>(s);
  if (valid && lane == 0) {
    T di = dinv[i];
    if (di != T(0)) x[i] = fma(b[i] - s, di, x[i]);
  }
}

// ---- the V-cycle's transfer and coarse-level kernels as programmatic
// dependents (launched by DP_LAUNCH_PDL): each loads what no kernel of a
// V-cycle writes (row pointers, the first round of a row's columns and
// values, 1/a_ii) before griddep_wait, and the vectors after it; with trig
// set it then lets its own dependents launch.  Their arithmetic is that of
// the batch's k_jacobi_pre_b, k_jacobi_sweep_b, k_csr_mv_b and k_dense_mv_b,
// term for term.

// the first round of a row's entries for G lanes: entries e0+lane+kG,
// k = 0..3, those below e1
template <int G, typename T, typename TV>
struct RowHead {
  int e, e1;
  int c[4];
  T v[4];
  __device__ __forceinline__ void load(int e0, int e1_, int lane, const int *__restrict__ col,
                                       const TV *__restrict__ val) {
    e = e0 + lane;
    e1 = e1_;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      bool h = e + k * G < e1;
      c[k] = h ? __ldg(col + e + k * G) : 0;
      v[k] = h ? ldv<T>(val + e + k * G) : T(0);
    }
  }
};

// row_dot's sum (four accumulators, the remainder into the first) with
// the head's entries taken from registers; X(c) is the vector entry.
template <int G, typename T, typename TV, typename F>
__device__ __forceinline__ T row_dot_head(const RowHead<G, T, TV> &h, const int *__restrict__ col,
                                          const TV *__restrict__ val, F X) {
  T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
  int e = h.e, e1 = h.e1;
  if (e + 3 * G < e1) {
    s0 = fma(h.v[0], X(h.c[0]), s0);
    s1 = fma(h.v[1], X(h.c[1]), s1);
    s2 = fma(h.v[2], X(h.c[2]), s2);
    s3 = fma(h.v[3], X(h.c[3]), s3);
    for (e += 4 * G; e + 3 * G < e1; e += 4 * G) {
      int c0 = __ldg(col + e), c1 = __ldg(col + e + G), c2 = __ldg(col + e + 2 * G),
          c3 = __ldg(col + e + 3 * G);
      T v0 = ldv<T>(val + e), v1 = ldv<T>(val + e + G), v2 = ldv<T>(val + e + 2 * G),
        v3 = ldv<T>(val + e + 3 * G);
      s0 = fma(v0, X(c0), s0);
      s1 = fma(v1, X(c1), s1);
      s2 = fma(v2, X(c2), s2);
      s3 = fma(v3, X(c3), s3);
    }
    for (; e < e1; e += G) s0 = fma(ldv<T>(val + e), X(__ldg(col + e)), s0);
  } else {   // at most three entries, all in the head
    if (e < e1) s0 = fma(h.v[0], X(h.c[0]), s0);
    if (e + G < e1) s0 = fma(h.v[1], X(h.c[1]), s0);
    if (e + 2 * G < e1) s0 = fma(h.v[2], X(h.c[2]), s0);
  }
  return (s0 + s1) + (s2 + s3);
}

// l1-Jacobi pre-smoothing from x = 0 fused with the residual: x_i = b_i d_i
// and r_i = b_i - sum_j a_ij b_j d_j (d = 1 / sum_j |a_ij|, 0 for an empty row).
template <int G, typename T, typename TV = T>
__global__ void __launch_bounds__(kBlock) k_jacobi_pre_p(int n, const int *__restrict__ rowptr,
                                                         const int *__restrict__ col,
                                                         const TV *__restrict__ val,
                                                         const T *__restrict__ d, const T *b,
                                                         T *x, T *r, int trig) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int i = t / G, lane = t % G;
  bool valid = i < n;
  int e0 = valid ? rowptr[i] : 0, e1 = valid ? rowptr[i + 1] : 0;
  RowHead<G, T, TV> h;
  h.load(e0, e1, lane, col, val);
  T di = valid && lane == 0 ? d[i] : T(0);
  griddep_wait();
  if (trig) griddep_launch_dependents();
  T s = row_dot_head<G>(h, col, val, [&](int c) { return __ldg(b + c) * __ldg(d + c); });
  if (G > 1) s = group_sum<G, T>(s);
  if (valid && lane == 0) {
    T bi = b[i];
    x[i] = bi * di;
    r[i] = bi - s;
  }
}

// One l1-Jacobi sweep: t_i = x_i + (b_i - (A x)_i) d_i for every row from
// the old x (t must not alias x).
template <int G, typename T, typename TV = T>
__global__ void __launch_bounds__(kBlock) k_jacobi_sweep_p(int n, const int *__restrict__ rowptr,
                                                           const int *__restrict__ col,
                                                           const TV *__restrict__ val,
                                                           const T *__restrict__ d, const T *b,
                                                           const T *x, T *tout, int trig) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int i = t / G, lane = t % G;
  bool valid = i < n;
  int e0 = valid ? rowptr[i] : 0, e1 = valid ? rowptr[i + 1] : 0;
  RowHead<G, T, TV> h;
  h.load(e0, e1, lane, col, val);
  T di = valid && lane == 0 ? d[i] : T(0);
  griddep_wait();
  if (trig) griddep_launch_dependents();
  T s = row_dot_head<G>(h, col, val, [&](int c) { return x[c]; });
  if (G > 1) s = group_sum<G, T>(s);
  if (valid && lane == 0) tout[i] = fma(b[i] - s, di, x[i]);
}

// y = A x (add = 0) or y += A x (add = 1)
template <int G, typename T, typename TV = T>
__global__ void __launch_bounds__(kBlock) k_csr_mv_p(int n, const int *__restrict__ rowptr,
                                                     const int *__restrict__ col,
                                                     const TV *__restrict__ val, const T *x, T *y,
                                                     int add, int trig) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int i = t / G, lane = t % G;
  bool valid = i < n;
  int e0 = valid ? rowptr[i] : 0, e1 = valid ? rowptr[i + 1] : 0;
  RowHead<G, T, TV> h;
  h.load(e0, e1, lane, col, val);
  griddep_wait();
  if (trig) griddep_launch_dependents();
  T s = row_dot_head<G>(h, col, val, [&](int c) { return x[c]; });
  if (G > 1) s = group_sum<G, T>(s);
  if (valid && lane == 0) y[i] = add ? y[i] + s : s;
}

// x = inv b on the coarsest level, a warp per row, FP64 accumulation: the
// row's first 64 entries of the inverse are loaded before the wait
template <typename T>
__global__ void k_dense_mv_p(int n, const double *__restrict__ inv, const T *b, T *x, int trig) {
  int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  bool valid = w < n;
  const double *row = inv + (size_t)(valid ? w : 0) * n;
  double a0 = valid && lane < n ? row[lane] : 0.0, a1 = valid && lane + 32 < n ? row[lane + 32] : 0.0;
  griddep_wait();
  if (trig) griddep_launch_dependents();
  if (!valid) return;   // whole warps leave together
  double s = 0.0;
  if (lane < n) s = fma(a0, double(b[lane]), s);
  if (lane + 32 < n) s = fma(a1, double(b[lane + 32]), s);
  for (int j = lane + 64; j < n; j += 32) s = fma(row[j], double(b[j]), s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) x[w] = T(s);
}

// r = b - A x
template <int G, typename T, typename TV = T>
__global__ void __launch_bounds__(kBlock) k_csr_resid(int n, const int *__restrict__ rowptr,
                                                      const int *__restrict__ col,
                                                      const TV *__restrict__ val,
                                                      const T *__restrict__ b,
                                                      const T *__restrict__ x, T *__restrict__ r) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int i = t / G, lane = t % G;
  bool valid = i < n;
  int e0 = valid ? rowptr[i] : 0, e1 = valid ? rowptr[i + 1] : 0;
  T s = row_dot<G, T, TV>(e0, e1, lane, col, val, x);
  if (G > 1) s = group_sum<G, T>(s);
  if (valid && lane == 0) r[i] = b[i] - s;
}


// Lanes per row for a mean row length: enough lanes that each walks about
// eight entries (two rounds of four loads in flight), no more, because on
// GB300 FP64 issue is scarce (1.2 TFLOP/s for the whole GPU) and every lane
// of a group takes part in the log2(G) shuffle additions.
int lanes_for(double mean_len) {
  int g = 1;
  while (g < 32 && 8.0 * g < mean_len) g *= 2;
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

// The arrays of a level in precision T.
template <typename T> struct LV;
template <> struct LV<double> {
  static const double *val(const Level &L) { return L.val; }
  static const double *dinv(const Level &L) { return L.dinv; }
  static const double *pval(const Level &L) { return L.p_val; }
  static const double *rval(const Level &L) { return L.r_val; }
  static double *x(const Level &L) { return L.x; }
  static double *b(const Level &L) { return L.b; }
  static double *r(const Level &L) { return L.r; }
};
template <> struct LV<float> {
  static const float *val(const Level &L) { return L.valf; }
  static const float *dinv(const Level &L) { return L.dinvf; }
  static const float *pval(const Level &L) { return L.p_valf; }
  static const float *rval(const Level &L) { return L.r_valf; }
  static float *x(const Level &L) { return L.xf; }
  static float *b(const Level &L) { return L.bf; }
  static float *r(const Level &L) { return L.rf; }
};

// In the FP32 cycle a level whose values also have a BF16 copy (precision 2,
// levels >= 1) is read from that copy.
template <typename T>
static bool use_bf16(const __nv_bfloat16 *h) {
  return std::is_same<T, float>::value && h != nullptr;
}

template <typename T>
static int csr_resid(Sim *s, const Level &L, const T *b, const T *x, T *r) {
  long long thr = (long long)L.n * L.G;
  if constexpr (std::is_same<T, float>::value) {
    if (use_bf16<T>(L.valh)) {
      DP_SWITCH_G(L.G, DP_LAUNCH(s, (k_csr_resid<GG, float, __nv_bfloat16>), nblk(thr), kBlock, 0,
                                 L.n, L.rowptr, L.col, L.valh, b, x, r));
      return DP_OK;
    }
  }
  DP_SWITCH_G(L.G, DP_LAUNCH(s, (k_csr_resid<GG, T>), nblk(thr), kBlock, 0, L.n, L.rowptr, L.col,
                             LV<T>::val(L), b, x, r));
  return DP_OK;
}

// y = A x or y += A x for the V-cycle's transfers, as a programmatic
// dependent; trig: let the next launch start once past the wait (always
// for level 0's prolongation, whose next launch is the wells' rows)
template <typename T>
static int csr_mv(Sim *s, int n, int G, const int *rowptr, const int *col, const T *val,
                  const T *x, T *y, int add, bool trig = pdl_trigger()) {
  long long thr = (long long)n * G;
  DP_SWITCH_G(G, DP_LAUNCH_PDL(s, kPdlCoarse, (k_csr_mv_p<GG, T>), nblk(thr), kBlock, 0, n, rowptr,
                               col, val, x, y, add, (int)trig));
  return DP_OK;
}

// A transfer operator (P or R) of a level, from its BF16 copy when it has one.
template <typename T>
static int transfer_mv(Sim *s, int n, int G, const int *rowptr, const int *col, const T *val,
                       const __nv_bfloat16 *valh, const T *x, T *y, int add) {
  if constexpr (std::is_same<T, float>::value) {
    if (use_bf16<T>(valh)) {
      long long thr = (long long)n * G;
      DP_SWITCH_G(G, DP_LAUNCH_PDL(s, kPdlCoarse, (k_csr_mv_p<GG, float, __nv_bfloat16>),
                                   nblk(thr), kBlock, 0, n, rowptr, col, valh, x, y, add,
                                   (int)pdl_trigger()));
      return DP_OK;
    }
  }
  return csr_mv<T>(s, n, G, rowptr, col, val, x, y, add);
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

constexpr int kDenseMax = 4096;
constexpr int kInverseMax = 1024;   // coarsest levels up to this size keep an explicit inverse

// Solve with the FP64 LU factors; b and x in T, the solve itself in FP64 in
// shared memory.
template <typename T>
__global__ void __launch_bounds__(1024) k_dense_solve(int n, const double *a, const int *piv,
                                                      const T *b, T *x) {
  __shared__ double xs[kDenseMax];
  int t = threadIdx.x, nt = blockDim.x;
  for (int i = t; i < n; i += nt) xs[i] = double(b[i]);
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
  for (int i = t; i < n; i += nt) x[i] = T(xs[i]);
}

// Inverse of the coarsest operator from its LU factors and row pivots, one
// column per thread: the solve of k_dense_solve applied to the unit vector
// e_c (the same steps in the same order), kept in column c of `inv`.
__global__ void k_dense_inverse(int n, const double *a, const int *piv, double *inv) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + c] = i == c ? 1.0 : 0.0;
  for (int k = 0; k < n; ++k) {
    int p = piv[k];
    if (p != k && p >= 0 && p < n) {
      double tmp = inv[(size_t)k * n + c];
      inv[(size_t)k * n + c] = inv[(size_t)p * n + c];
      inv[(size_t)p * n + c] = tmp;
    }
    double xk = inv[(size_t)k * n + c];
    for (int i = k + 1; i < n; ++i) inv[(size_t)i * n + c] -= a[(size_t)i * n + k] * xk;
  }
  for (int i = n - 1; i >= 0; --i) {
    double d = a[(size_t)i * n + i];
    double xi = d != 0.0 ? inv[(size_t)i * n + c] / d : 0.0;
    inv[(size_t)i * n + c] = xi;
    for (int r = 0; r < i; ++r) inv[(size_t)r * n + c] -= a[(size_t)r * n + i] * xi;
  }
}


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
    if (s->coarse_inv) dfree(s, s->coarse_inv);
    s->coarse_inv = nullptr;
    if (n <= kInverseMax) {
      s->coarse_inv = (double *)dalloc(s, (size_t)n * n * 8);
      if (!s->coarse_inv) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
    }
  }
  s->coarse_n = n;
  DP_LAUNCH(s, k_csr_to_dense, nblk(n), kBlock, 0, n, L.rowptr, L.col, L.val, s->coarse_lu);
  DP_LAUNCH(s, k_dense_lu, 1, 1024, 0, n, s->coarse_lu, s->coarse_piv);
  if (s->coarse_inv)
    DP_LAUNCH(s, k_dense_inverse, nblk(n, 128), 128, 0, n, s->coarse_lu, s->coarse_piv,
              s->coarse_inv);
  DP_CUDA(s, cudaGetLastError());
  return DP_OK;
}

// l1-Jacobi: pre-smoothing from zero fused with the residual into r, and a
// sweep after the coarse correction into r (free by then), where the
// prolongation of the level above reads the result.
template <typename T>
static int jacobi_pre(Sim *s, Level &L, const T *b, T *x, T *r) {
  long long thr = (long long)L.n * L.G;
  if constexpr (std::is_same<T, float>::value) {
    if (use_bf16<T>(L.valh)) {
      DP_SWITCH_G(L.G, DP_LAUNCH_PDL(s, kPdlCoarse, (k_jacobi_pre_p<GG, float, __nv_bfloat16>),
                                     nblk(thr), kBlock, 0, L.n, L.rowptr, L.col, L.valh, L.dinvf,
                                     b, x, r, (int)pdl_trigger()));
      return DP_OK;
    }
  }
  DP_SWITCH_G(L.G, DP_LAUNCH_PDL(s, kPdlCoarse, (k_jacobi_pre_p<GG, T>), nblk(thr), kBlock, 0,
                                 L.n, L.rowptr, L.col, LV<T>::val(L), LV<T>::dinv(L), b, x, r,
                                 (int)pdl_trigger()));
  return DP_OK;
}

template <typename T>
static int jacobi_post(Sim *s, Level &L, const T *b, T *x, T *r) {
  long long thr = (long long)L.n * L.G;
  bool done = false;
  if constexpr (std::is_same<T, float>::value) {
    if (use_bf16<T>(L.valh)) {
      DP_SWITCH_G(L.G, DP_LAUNCH_PDL(s, kPdlCoarse, (k_jacobi_sweep_p<GG, float, __nv_bfloat16>),
                                     nblk(thr), kBlock, 0, L.n, L.rowptr, L.col, L.valh, L.dinvf,
                                     b, x, r, (int)pdl_trigger()));
      done = true;
    }
  }
  if (!done)
    DP_SWITCH_G(L.G, DP_LAUNCH_PDL(s, kPdlCoarse, (k_jacobi_sweep_p<GG, T>), nblk(thr), kBlock,
                                   0, L.n, L.rowptr, L.col, LV<T>::val(L), LV<T>::dinv(L), b, x,
                                   r, (int)pdl_trigger()));
  return DP_OK;
}

// One colour of Gauss-Seidel on level 0 from its colour-ordered copy: the
// rows q of a colour are contiguous in the ILU(0) pattern (row q is natural
// row perm[q], entries lu_col[e] with values pv[e]), so a sweep streams the
// operator once instead of touching every row's sectors for every colour.
// Operator data read once per sweep is loaded evict-first (ld.global.cs) so
// that the vectors stay in L2 between colours.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_gs_lu(int r0, int r1, const int *__restrict__ perm,
                                                  const int *__restrict__ lu_rowptr,
                                                  const int *__restrict__ lu_col,
                                                  const T *__restrict__ pv,
                                                  const T *__restrict__ dinv,
                                                  const T *__restrict__ b, T *x) {
  int q = r0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= r1) return;
  int i = __ldcs(perm + q);
  int e = __ldcs(lu_rowptr + q), e1 = __ldcs(lu_rowptr + q + 1);
  // the row's first eight entries (a cell row's whole stencil) in one batch
  // of predicated loads, then their eight gathers of x, so that a thread waits
  // for two memory round trips instead of one pair per two entries
  constexpr int kB = 8;
  int c[kB];
  T v[kB];
#pragma unroll
  for (int k = 0; k < kB; ++k) {
    bool in = e + k < e1;
    c[k] = in ? __ldcs(lu_col + e + k) : 0;
    v[k] = in ? __ldcs(pv + e + k) : T(0);
  }
  T s0 = T(0), s1 = T(0);
#pragma unroll
  for (int k = 0; k < kB; k += 2) {
    if (e + k < e1) s0 = fma(v[k], x[c[k]], s0);
    if (e + k + 1 < e1) s1 = fma(v[k + 1], x[c[k + 1]], s1);
  }
  for (e += kB; e < e1; ++e) s0 = fma(__ldcs(pv + e), x[__ldcs(lu_col + e)], s0);
  T s = s0 + s1;
  T di = dinv[i];
  if (di != T(0)) x[i] = fma(b[i] - s, di, x[i]);
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_gs_lu_w(int r0, int r1, const int *__restrict__ perm,
                                                    const int *__restrict__ lu_rowptr,
                                                    const int *__restrict__ lu_col,
                                                    const T *__restrict__ pv,
                                                    const T *__restrict__ dinv,
                                                    const T *__restrict__ b, T *x) {
  int q = r0 + (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  int lane = threadIdx.x & 31;
  if (q >= r1) return;   // whole warps
  T s = T(0);
  for (int e = __ldg(lu_rowptr + q) + lane, e1 = __ldg(lu_rowptr + q + 1); e < e1; e += 32)
    s = fma(__ldg(pv + e), x[__ldg(lu_col + e)], s);
  s = warp_sum(s);
  if (lane == 0) {
    int i = __ldg(perm + q);
    T di = dinv[i];
    if (di != T(0)) x[i] = fma(b[i] - s, di, x[i]);
  }
}

template <typename T>
__global__ void k_gather_vals(long long n, const int *__restrict__ src, const double *__restrict__ v,
                              T *__restrict__ out) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) out[e] = T(v[__ldg(src + e)]);
}

// The colour-ordered level-0 values (used when level 0 is smoothed by
// Gauss-Seidel: its colouring is the ILU(0) colouring, same pattern and same
// algorithm): gathered here when first needed, then written by the
// decoupling every Newton step.  With them, level 0 runs in colour order
// (Sim::l0c): the colour positions of the copy's columns and of R0's columns
// and P0 with its rows in colour order are built once; 1/a_ii in colour order
// every Newton step, P0's values whenever the coarse values are refreshed.
__global__ void k_perm_rows(int n, const int *perm, const int *rowptr, const int *col,
                            const int *prow, int *pcol, int *psrc) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  int i = perm[q], e0 = rowptr[i], m = rowptr[i + 1] - e0, d0 = prow[q];
  for (int k = 0; k < m; ++k) { pcol[d0 + k] = col[e0 + k]; psrc[d0 + k] = e0 + k; }
}

__global__ void k_map_copy(long long n, const int *map, const int *in, int *out) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) out[e] = map[in[e]];
}

static int l0c_setup(Sim *s) {
  Level &L = s->lev[0];
  int n = L.n;
  s->l0_colp = (int *)dalloc(s, (size_t)std::max(L.nnz, 1) * 4 + 16);
  s->r0_colp = (int *)dalloc(s, (size_t)std::max(L.r_nnz, 1) * 4);
  s->p0c_rowptr = (int *)dalloc(s, ((size_t)n + 1) * 4);
  s->p0c_col = (int *)dalloc(s, (size_t)std::max(L.p_nnz, 1) * 4);
  s->p0c_src = (int *)dalloc(s, (size_t)std::max(L.p_nnz, 1) * 4);
  int *len = (int *)dalloc(s, (size_t)n * 4);
  bool f32 = s->opt.precision >= 1;
  if (f32) {
    s->p0c_valf = (float *)dalloc(s, (size_t)std::max(L.p_nnz, 1) * 4);
    s->dinv_cf = (float *)dalloc(s, (size_t)n * 4);
    s->scolc = (int *)dalloc(s, (size_t)std::max(s->K.nnz, 1) * 4);
    s->z2c = (float *)dalloc(s, (size_t)s->K.n * 8);
    if (!s->scolc || !s->z2c) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
  } else {
    s->p0c_val = (double *)dalloc(s, (size_t)std::max(L.p_nnz, 1) * 8);
    s->dinv_c = (double *)dalloc(s, (size_t)n * 8);
  }
  if (!s->l0_colp || !s->r0_colp || !s->p0c_rowptr || !s->p0c_col || !s->p0c_src || !len ||
      (f32 ? (!s->p0c_valf || !s->dinv_cf) : (!s->p0c_val || !s->dinv_c))) {
    s->fail(DP_ENOMEM, "allocation failed");
    return DP_ENOMEM;
  }
  DP_LAUNCH(s, k_map_copy, nblk(L.nnz), kBlock, 0, (long long)L.nnz, s->iperm, s->lu_col,
            s->l0_colp);
  DP_LAUNCH(s, k_map_copy, nblk(L.r_nnz), kBlock, 0, (long long)L.r_nnz, s->iperm, L.r_col,
            s->r0_colp);
  if (s->scolc)
    DP_LAUNCH(s, k_map_copy, nblk(s->K.nnz), kBlock, 0, (long long)s->K.nnz, s->iperm, s->scol,
              s->scolc);
  DP_LAUNCH(s, k_perm_len, nblk(n), kBlock, 0, n, s->perm, L.p_rowptr, len);
  int pn = 0;
  DP_TRY(scan_i32(s, len, s->p0c_rowptr, n, &pn));
  DP_LAUNCH(s, k_perm_rows, nblk(n), kBlock, 0, n, s->perm, L.p_rowptr, L.p_col, s->p0c_rowptr,
            s->p0c_col, s->p0c_src);
  DP_CUDA(s, cudaGetLastError());
  dfree(s, len);
  s->l0c = true;
  return DP_OK;
}

int l0_refresh(Sim *s, bool coarse) {
  if (s->lev.empty() || s->opt.precond != 2) return DP_OK;
  Level &L = s->lev[0];
  bool first = false;
  if (!s->l0_lu) {
    if (L.l1 || L.ncolour != s->ncolour || L.rowptr != s->K.rowptr) return DP_OK;
    for (int c = 0; c <= L.ncolour; ++c)
      if (L.cstart[c] != s->lu_cstart[c]) return DP_OK;
    size_t nnz = (size_t)std::max(L.nnz, 1);
    if (s->opt.precision >= 1) s->l0_pvf = (float *)dalloc(s, nnz * 4 + 16);
    else s->l0_pv = (double *)dalloc(s, nnz * 8 + 32);
    if (!s->l0_pvf && !s->l0_pv) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
    s->l0_lu = true;
    first = true;
    // later Newton steps: the decoupling writes the copy
    if (s->l0_pvf)
      DP_LAUNCH(s, k_gather_vals<float>, nblk(L.nnz), kBlock, 0, (long long)L.nnz, s->lu_src,
                L.val, s->l0_pvf);
    else
      DP_LAUNCH(s, k_gather_vals<double>, nblk(L.nnz), kBlock, 0, (long long)L.nnz, s->lu_src,
                L.val, s->l0_pv);
    if (s->lev.size() > 1) DP_TRY(l0c_setup(s));
  }
  if (s->l0c) {
    if (s->dinv_cf)
      DP_LAUNCH(s, k_gather_vals<float>, nblk(L.n), kBlock, 0, (long long)L.n, s->perm, L.dinv,
                s->dinv_cf);
    else
      DP_LAUNCH(s, k_gather_vals<double>, nblk(L.n), kBlock, 0, (long long)L.n, s->perm, L.dinv,
                s->dinv_c);
    if (coarse || first) {
      if (s->p0c_valf)
        DP_LAUNCH(s, k_gather_vals<float>, nblk(L.p_nnz), kBlock, 0, (long long)L.p_nnz,
                  s->p0c_src, L.p_val, s->p0c_valf);
      else
        DP_LAUNCH(s, k_gather_vals<double>, nblk(L.p_nnz), kBlock, 0, (long long)L.p_nnz,
                  s->p0c_src, L.p_val, s->p0c_val);
    }
  }
  DP_CUDA(s, cudaGetLastError());
  return DP_OK;
}

// Level 0 in colour order (Sim::l0c): row q of the colour copy is the q-th
// row of the ILU(0) ordering, its columns are colour positions (colp), and
// b, x, 1/a_ii and the residual are colour-ordered vectors, so every access
// but the column gathers is contiguous.  The same row formulas as k_gs_lu.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_gs_c(int r0, int r1, const int *__restrict__ rowptr,
                                                 const int *__restrict__ colp,
                                                 const T *__restrict__ pv,
                                                 const T *__restrict__ dinv,
                                                 const T *__restrict__ b, T *x) {
  k_gs_c_b<T>(blockIdx.x, gridDim.x, r0, r1, rowptr, colp, pv, dinv, b, x);
}

// The first colour of a Gauss-Seidel sweep that starts from x = 0: every
// x_j a row reads is still zero, so the row formula reduces to
// x_i = fma(b_i, 1/a_ii, 0) (the same value bit for bit: the sum is +0).
template <typename T>
__global__ void k_gs_c_first(int r0, int r1, const T *__restrict__ dinv, const T *__restrict__ b,
                             T *__restrict__ x) {
  k_gs_c_first_b<T>(blockIdx.x, gridDim.x, r0, r1, dinv, b, x);
}


// Level-0 long rows (the wells) launched as programmatic dependents of the
// launch before them, a CTA of one warp per row: what no kernel of the
// V-cycle writes (the row's pointers, columns and values, 1/a_ii) is loaded
// before griddep_wait, so the rows' launch and these loads overlap the end
// of the kernel before; b and x are read after it.  The first 64 entries of
// a row stay in registers, longer rows read the rest after the wait.  The
// products and their order are warp_row_c's, so the results equal
// the batch's well rows (k_gs_c_w_b, k_resid_c_w_b) bit for bit.
template <typename T, bool RESID>
__device__ __forceinline__ void row_c_wp(int q, const int *__restrict__ rowptr,
                                         const int *__restrict__ colp, const T *__restrict__ pv,
                                         const T *__restrict__ dinv, const T *b, T *x, T *r) {
  int lane = threadIdx.x;
  int e = __ldg(rowptr + q) + lane, e1 = __ldg(rowptr + q + 1);
  bool h0 = e < e1, h1 = e + 32 < e1;
  T v0 = h0 ? __ldg(pv + e) : T(0), v1 = h1 ? __ldg(pv + e + 32) : T(0);
  int c0 = h0 ? __ldg(colp + e) : 0, c1 = h1 ? __ldg(colp + e + 32) : 0;
  T di = (!RESID && lane == 0) ? dinv[q] : T(0);
  griddep_wait();
  griddep_launch_dependents();   // the colour launch after the wells (backward sweep)
  T bq = lane == 0 ? b[q] : T(0);
  T s = T(0);
  if (h1) {
    s = fma(v0, x[c0], s);
    s = fma(v1, x[c1], s);
    for (e += 64; e + 32 < e1; e += 64) {
      T w0 = __ldg(pv + e), w1 = __ldg(pv + e + 32);
      int d0 = __ldg(colp + e), d1 = __ldg(colp + e + 32);
      s = fma(w0, x[d0], s);
      s = fma(w1, x[d1], s);
    }
    if (e < e1) s = fma(__ldg(pv + e), x[__ldg(colp + e)], s);
  } else if (h0) {
    s = fma(v0, x[c0], s);
  }
  s = warp_sum(s);
  if (lane == 0) {
    if (RESID) r[q] = bq - s;
    else if (di != T(0)) x[q] = fma(bq - s, di, x[q]);
  }
}

template <typename T>
__global__ void __launch_bounds__(32) k_gs_c_wp(int r0, const int *__restrict__ rowptr,
                                                const int *__restrict__ colp,
                                                const T *__restrict__ pv,
                                                const T *__restrict__ dinv, const T *b, T *x) {
  row_c_wp<T, false>(r0 + (int)blockIdx.x, rowptr, colp, pv, dinv, b, x, nullptr);
}

template <typename T>
__global__ void __launch_bounds__(32) k_resid_c_wp(int r0, const int *__restrict__ rowptr,
                                                   const int *__restrict__ colp,
                                                   const T *__restrict__ pv, const T *b, T *x,
                                                   T *r) {
  row_c_wp<T, true>(r0 + (int)blockIdx.x, rowptr, colp, pv, nullptr, b, x, r);
}

// r = b - A x over the rows [r0, r1) of the colour copy, a thread per row.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_resid_c(int r0, int r1, const int *__restrict__ rowptr,
                                                    const int *__restrict__ colp,
                                                    const T *__restrict__ pv,
                                                    const T *__restrict__ b,
                                                    const T *__restrict__ x, T *__restrict__ r) {
  k_resid_c_b<T>(blockIdx.x, gridDim.x, r0, r1, rowptr, colp, pv, b, x, r);
}

template <int G, typename T>
__global__ void __launch_bounds__(kBlock) k_gs_cg(int r0, int r1, const int *__restrict__ rowptr,
                                                  const int *__restrict__ colp,
                                                  const T *__restrict__ pv,
                                                  const T *__restrict__ dinv,
                                                  const T *__restrict__ b, T *x) {
  k_gs_cg_b<G, T>(blockIdx.x, gridDim.x, r0, r1, rowptr, colp, pv, dinv, b, x);
}

template <int G, typename T>
__global__ void __launch_bounds__(kBlock) k_resid_cg(int r0, int r1, const int *__restrict__ rowptr,
                                                     const int *__restrict__ colp,
                                                     const T *__restrict__ pv,
                                                     const T *__restrict__ b, const T *x,
                                                     T *__restrict__ r) {
  k_resid_cg_b<G, T>(blockIdx.x, gridDim.x, r0, r1, rowptr, colp, pv, b, x, r);
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_gs_cs(int r0, int r1, const int *__restrict__ rowptr,
                                                  const int *__restrict__ colp,
                                                  const T *__restrict__ pv,
                                                  const T *__restrict__ dinv,
                                                  const T *__restrict__ b, T *x) {
  k_sweep_cs_b<T, false>(blockIdx.x, gridDim.x, r0, r1, rowptr, colp, pv, dinv, b, x, nullptr);
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_resid_cs(int r0, int r1, const int *__restrict__ rowptr,
                                                     const int *__restrict__ colp,
                                                     const T *__restrict__ pv,
                                                     const T *__restrict__ b, T *x,
                                                     T *__restrict__ r) {
  k_sweep_cs_b<T, true>(blockIdx.x, gridDim.x, r0, r1, rowptr, colp, pv, nullptr, b, x, r);
}

// Level-0 Gauss-Seidel colour (RESID false) or residual rows (RESID true)
// as a pipelined persistent kernel: each CTA walks tiles of kTT consecutive
// rows of [r0, r1) (tile blockIdx.x, + gridDim.x, ...).  A producer warp
// brings a tile's row pointers, columns and values into shared memory with
// bulk asynchronous copies (S stages, full/empty mbarriers), so the matrix
// stream of the next tiles is in flight while the kTT consumer threads (a
// thread per row) gather x for the current one (stage_row_sum); 1/a_ii
// and b are read per thread before the wait.  A stage holds CAPR entries a
// row on average;
// a tile with more entries brings only its row pointers and its threads
// read their entries from global memory.  The row's products are summed as
// in k_gs_c (entries 1, 3, 5, 7 into one accumulator, the others into the
// second), so every row's result is that kernel's bit for bit.  The copies
// start at 16-byte boundaries below the tile's first row pointer and entry
// and read up to three elements past the last one: the row pointer, column
// and value arrays are allocated with 16 (32 for FP64 values) spare bytes.
// A bounded wait that gives up sets *err and ends the thread (the producer
// first lets its copies in flight land, again with a bound).
constexpr int kTT = 256;
template <typename T, int CAPR> struct TStage {
  int rp[kTT + 8];
  int col[CAPR * kTT];
  T val[CAPR * kTT];
};

// a barrier of the kTT consumer threads only (named barrier 1; the
// producer warp is not waited for)
__device__ __forceinline__ void consumers_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kTT) : "memory");
}

// The producer warp of the pipelined kernels: the CTA's tiles are tiles
// B, B + G, ... of each of the nph row ranges [pr0[p], pr1[p]) in turn
// (the consumers take them in the same order).  The warp's 32 lanes read
// the row-pointer bounds of 32 coming tiles at once, then lane 0 issues
// their copies one by one as stages come free (the bounds shuffled from
// the lane that read them): the row pointers always, the columns and
// values when they fit the stage.  A stage's full barrier expects exactly
// the bytes copied into it.  When a wait gives up the warp sets *err, lets
// the copies in flight land (bounded) and ends.
template <typename T, int S, int CAPR>
__device__ __forceinline__ void tile_producer(int nph, const int *pr0, const int *pr1, int B, int G,
                                              const int *__restrict__ rowptr,
                                              const int *__restrict__ colp,
                                              const T *__restrict__ pv, TStage<T, CAPR> *st,
                                              uint64_t *full, uint64_t *empty, int *err) {
  constexpr int kCap = CAPR * kTT;
  const int lane = threadIdx.x & 31;
  auto mine = [&](int p) {
    int ntile = (pr1[p] - pr0[p] + kTT - 1) / kTT;
    return ntile > B ? (ntile - 1 - B) / G + 1 : 0;
  };
  int total = 0;
  for (int p = 0; p < nph; ++p) total += mine(p);
  int i = 0;
  bool ok = true;
  for (int base = 0; base < total && ok; base += 32) {
    int q0 = 0, nrow = 0, e0 = 0, e1 = 0;
    if (base + lane < total) {
      int p = 0, rem = base + lane;
      while (rem >= mine(p)) rem -= mine(p++);
      q0 = pr0[p] + (B + rem * G) * kTT;
      nrow = min(kTT, pr1[p] - q0);
      e0 = __ldg(rowptr + q0);
      e1 = __ldg(rowptr + q0 + nrow);
    }
    int cnt = min(32, total - base);
    for (int j = 0; j < cnt; ++j, ++i) {
      int tq0 = __shfl_sync(0xffffffffu, q0, j), tn = __shfl_sync(0xffffffffu, nrow, j);
      int te0 = __shfl_sync(0xffffffffu, e0, j), te1 = __shfl_sync(0xffffffffu, e1, j);
      int k = i % S;
      int w = 1;
      if (lane == 0 && i >= S) w = mbar_wait(&empty[k], (i / S - 1) & 1);
      if (!__shfl_sync(0xffffffffu, w, 0)) {
        ok = false;
        break;
      }
      if (lane == 0) {
        int aq = tq0 & ~3, nrp = (tq0 + tn + 1 - aq + 3) & ~3;
        int ae = te0 & ~3, ne = (te1 - ae + 3) & ~3;
        bool fits = ne <= kCap;
        mbar_arrive_tx(&full[k], (uint32_t)(4 * nrp + (fits ? ne * (4 + (int)sizeof(T)) : 0)));
        bulk_load(st[k].rp, rowptr + aq, 4u * nrp, &full[k]);
        if (fits && ne > 0) {
          bulk_load(st[k].col, colp + ae, 4u * ne, &full[k]);
          bulk_load(st[k].val, pv + ae, (uint32_t)sizeof(T) * ne, &full[k]);
        }
      }
    }
  }
  if (!ok && lane == 0) {   // the copies in flight land before the warp ends
    atomicExch(err, 1);
    for (int j = max(0, i - S); j < i; ++j) mbar_wait(&full[j % S], (j / S) & 1);
  }
}

template <typename T, bool RESID, int S, int CAPR>
__device__ __forceinline__ void sweep_tma_body(int r0, int r1, const int *__restrict__ rowptr,
                                               const int *__restrict__ colp,
                                               const T *__restrict__ pv,
                                               const T *__restrict__ dinv,
                                               const T *__restrict__ b, T *x,
                                               T *__restrict__ r, int *err) {
  constexpr int kCap = CAPR * kTT;
  extern __shared__ __align__(128) unsigned char tma_smem[];
  TStage<T, CAPR> *st = reinterpret_cast<TStage<T, CAPR> *>(tma_smem);
  __shared__ __align__(8) uint64_t full[S], empty[S];
  griddep_launch_dependents();   // the wells' rows after this colour (k_gs_c_wp, k_resid_c_wp)
  int ntile = (r1 - r0 + kTT - 1) / kTT;
  int mine = (int)blockIdx.x < ntile ? (ntile - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  if (threadIdx.x == 0) {
    for (int k = 0; k < S; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], kTT);
    }
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x >= kTT) {   // the producer warp
    tile_producer<T, S, CAPR>(1, &r0, &r1, (int)blockIdx.x, (int)gridDim.x, rowptr, colp, pv, st,
                              full, empty, err);
    return;
  }
  int t = threadIdx.x;
  __shared__ int abort_flag;
  volatile int *abort_v = &abort_flag;
  if (t == 0) abort_flag = 0;
  consumers_sync();
  // launched as a programmatic dependent (kPdlL0), the producer has been
  // bringing in the operator's tiles, which no kernel of the cycle writes,
  // while the kernel before finished; b and x are read after this
  griddep_wait();
  for (int i = 0; i < mine; ++i) {
    int k = i % S;
    int q0 = r0 + ((int)blockIdx.x + i * (int)gridDim.x) * kTT, nrow = min(kTT, r1 - q0);
    int q = q0 + t;
    bool in = t < nrow;
    T bq = T(0), dq = T(0);
    if (in) {
      bq = b[q];
      if (!RESID) dq = dinv[q];
    }
    // a consumer that gives up marks the CTA, which skips the rest
    bool ok = !*abort_v && mbar_wait(&full[k], (i / S) & 1);
    if (!ok) *abort_v = 1;
    if (ok && in) {
      const int *rp = st[k].rp + (q0 & 3);
      int ae = rp[0] & ~3;
      bool fits = ((rp[nrow] - ae + 3) & ~3) <= kCap;
      int e = rp[t], e1 = rp[t + 1];
      T sum = fits ? stage_row_sum<T>(e1 - e, st[k].col + (e - ae), st[k].val + (e - ae), x)
                   : stage_row_sum<T>(e1 - e, colp + e, pv + e, x);
      if (RESID) r[q] = bq - sum;
      else if (dq != T(0)) x[q] = fma(bq - sum, dq, x[q]);
    }
    mbar_arrive(&empty[k]);
  }
  if (*abort_v) atomicExch(err, 1);
}

template <typename T, int S, int CAPR>
__global__ void __launch_bounds__(kTT + 32) k_gs_c_tma(int r0, int r1, const int *__restrict__ rowptr,
                                                       const int *__restrict__ colp,
                                                       const T *__restrict__ pv,
                                                       const T *__restrict__ dinv,
                                                       const T *__restrict__ b, T *x, int *err) {
  sweep_tma_body<T, false, S, CAPR>(r0, r1, rowptr, colp, pv, dinv, b, x, nullptr, err);
}

template <typename T, int S, int CAPR>
__global__ void __launch_bounds__(kTT + 32) k_resid_c_tma(int r0, int r1,
                                                          const int *__restrict__ rowptr,
                                                          const int *__restrict__ colp,
                                                          const T *__restrict__ pv,
                                                          const T *__restrict__ b, T *x,
                                                          T *__restrict__ r, int *err) {
  sweep_tma_body<T, true, S, CAPR>(r0, r1, rowptr, colp, pv, nullptr, b, x, r, err);
}

// grid of a pipelined kernel: its tiles, at most the CTAs that fit on the
// GPU at once (queried once per kernel, thread-safe; ID tells the kernels
// of one signature apart)
template <int ID, typename K>
static int tma_grid(K kern, int smem, int rows) {
  static const int slots = [&]() {
    int dev = 0, nsm = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kTT + 32, smem);
    return std::max(n, 1) * std::max(nsm, 1);
  }();
  return std::max(1, std::min((rows + kTT - 1) / kTT, slots));
}

// the pipelined variants: -1 two stages of up to 8 entries a row, -2 three
// stages of 6, -3 two stages of 4 (level 0's mixed fracture/matrix tiles
// average about 5, so those bring their row pointers only)
template <typename T, int S, int CAPR>
static void gs_tma(Sim *s, int r0, int r1, const T *pv, const T *dinv, const T *b, T *x) {
  constexpr int smem = S * (int)sizeof(TStage<T, CAPR>);
  DP_LAUNCH_PDL(s, kPdlL0, (k_gs_c_tma<T, S, CAPR>),
                (tma_grid<16 * S + CAPR>(k_gs_c_tma<T, S, CAPR>, smem, r1 - r0)), kTT + 32, smem, r0,
                r1, s->lu_rowptr, s->l0_colp, pv, dinv, b, x, s->dev_err);
}
template <typename T, int S, int CAPR>
static void resid_tma(Sim *s, int r0, int r1, const T *pv, const T *b, T *x, T *r) {
  constexpr int smem = S * (int)sizeof(TStage<T, CAPR>);
  DP_LAUNCH_PDL(s, kPdlL0, (k_resid_c_tma<T, S, CAPR>),
                (tma_grid<16 * S + CAPR>(k_resid_c_tma<T, S, CAPR>, smem, r1 - r0)), kTT + 32, smem,
                r0, r1, s->lu_rowptr, s->l0_colp, pv, b, x, r, s->dev_err);
}
template <typename T>
static void sweep_tma(Sim *s, int G, int r0, int r1, const T *pv, const T *dinv, const T *b, T *x,
                      T *r) {
  s->waits_used = true;
  if (r) {
    if (G == -1) resid_tma<T, 2, 8>(s, r0, r1, pv, b, x, r);
    else if (G == -2) resid_tma<T, 3, 6>(s, r0, r1, pv, b, x, r);
    else resid_tma<T, 2, 4>(s, r0, r1, pv, b, x, r);
  } else {
    if (G == -1) gs_tma<T, 2, 8>(s, r0, r1, pv, dinv, b, x);
    else if (G == -2) gs_tma<T, 3, 6>(s, r0, r1, pv, dinv, b, x);
    else gs_tma<T, 2, 4>(s, r0, r1, pv, dinv, b, x);
  }
}


// One whole Gauss-Seidel sweep of level 0 in colour order as a single
// cooperative persistent launch (the CTAs are resident together): the
// sweep's phases (the colours in sweep order, and for the pre-smoothing
// first the initialisation x = b/a_ii on colour 0's rows, x = 0 on the
// others) are separated by grid barriers.  Short-row colours go tile by tile
// through the producer/consumer pipeline of sweep_tma_body; the producer
// warp walks all of the sweep's tiles without waiting at the barriers (the
// matrix does not change), so the next colour's tiles are already in
// shared memory when its phase starts.  Long-row colours (the wells) take a
// consumer warp per row.  Every row's arithmetic is that of k_gs_c_first,
// k_gs_c and k_gs_c_wp, so the sweep's result is theirs bit for bit.  The
// barrier counts arrivals on bar[0] (the k-th barrier is passed at (k+1)
// gridDim.x arrivals) and the last CTA to finish resets it (with bar[1],
// the exit count) for the next launch; its waits, like the pipeline's,
// give up after kWaitNs, set *err and end the CTA, and a CTA that finds
// *err set does no more.
constexpr int kSweepPhases = 8;
struct SweepPlan {
  int n;                      // rows of level 0
  int nphase;
  int kind[kSweepPhases];     // 0: initialisation, 1: short rows (tiles), 2: long rows
  int r0[kSweepPhases], r1[kSweepPhases];
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// grid barrier of the consumer threads (every one of them reaches it: none
// leaves the kernel before); false, for all of the CTA's consumers, when
// the CTA has given up (abort_flag) or the wait gave up or *err is set
__device__ __forceinline__ bool grid_barrier(unsigned *cnt, unsigned target, int *err,
                                             volatile int *abort_flag) {
  consumers_sync();
  if (threadIdx.x == 0) {
    if (*abort_flag || *(volatile int *)err) {
      *abort_flag = 1;
    } else {
      __threadfence();
      atomicAdd(cnt, 1u);
      uint64_t t0 = global_ns();
      while (ld_acquire(cnt) < target) {
        if (*(volatile int *)err || global_ns() - t0 > kWaitNs) {
          *abort_flag = 1;
          break;
        }
        __nanosleep(64);
      }
      __threadfence();
    }
    if (*abort_flag) atomicExch(err, 1);
  }
  consumers_sync();
  return !*abort_flag;
}

template <typename T, int S, int CAPR>
__global__ void __launch_bounds__(kTT + 32) k_gs_c_sweep(SweepPlan plan,
                                                         const int *__restrict__ rowptr,
                                                         const int *__restrict__ colp,
                                                         const T *__restrict__ pv,
                                                         const T *__restrict__ dinv,
                                                         const T *__restrict__ b, T *x,
                                                         unsigned *bar, int *err) {
  constexpr int kCap = CAPR * kTT;
  extern __shared__ __align__(128) unsigned char tma_smem[];
  TStage<T, CAPR> *st = reinterpret_cast<TStage<T, CAPR> *>(tma_smem);
  __shared__ __align__(8) uint64_t full[S], empty[S];
  __shared__ int abort_flag;
  const int G = (int)gridDim.x, B = (int)blockIdx.x;
  if (threadIdx.x == 0) {
    for (int k = 0; k < S; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], kTT);
    }
    mbar_init_fence();
    abort_flag = 0;
  }
  __syncthreads();
  if (threadIdx.x >= kTT) {   // the producer warp, over the sweep's short-row phases
    int pr0[kSweepPhases], pr1[kSweepPhases], nph = 0;
    for (int p = 0; p < plan.nphase; ++p)
      if (plan.kind[p] == 1) {
        pr0[nph] = plan.r0[p];
        pr1[nph++] = plan.r1[p];
      }
    tile_producer<T, S, CAPR>(nph, pr0, pr1, B, G, rowptr, colp, pv, st, full, empty, err);
    return;
  }
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  volatile int *abort_v = &abort_flag;
  int i = 0, nbar = 0;
  for (int p = 0; p < plan.nphase; ++p) {
    if (p > 0 && !grid_barrier(bar, (unsigned)(++nbar) * (unsigned)G, err, abort_v)) return;
    int r0 = plan.r0[p], r1 = plan.r1[p];
    if (plan.kind[p] == 0) {   // x = b/a_ii on [r0, r1), 0 elsewhere
      for (int q = B * kTT + t; q < plan.n; q += G * kTT) {
        T v = T(0);
        if (q >= r0 && q < r1) {
          T di = dinv[q];
          v = di != T(0) ? fma(b[q] - T(0), di, T(0)) : T(0);
        }
        x[q] = v;
      }
    } else if (plan.kind[p] == 2) {   // a warp per row
      for (int q = r0 + B * (kTT / 32) + warp; q < r1; q += G * (kTT / 32))
        warp_row_c<T, false>(q, lane, rowptr, colp, pv, dinv, b, x, nullptr);
    } else {
      int ntile = (r1 - r0 + kTT - 1) / kTT;
      for (int tile = B; tile < ntile; tile += G, ++i) {
        int k = i % S;
        int q0 = r0 + tile * kTT, nrow = min(kTT, r1 - q0);
        int q = q0 + t;
        bool in = t < nrow;
        T bq = T(0), dq = T(0);
        if (in) {
          bq = b[q];
          dq = dinv[q];
        }
        // a consumer that gives up does not leave: it marks the CTA, which
        // then skips its work up to the next barrier and ends there
        bool ok = !*abort_v && mbar_wait(&full[k], (i / S) & 1);
        if (!ok) *abort_v = 1;
        if (ok && in) {
          const int *rp = st[k].rp + (q0 & 3);
          int ae = rp[0] & ~3;
          bool fits = ((rp[nrow] - ae + 3) & ~3) <= kCap;
          int e = rp[t], e1 = rp[t + 1];
          T sum = fits ? stage_row_sum<T>(e1 - e, st[k].col + (e - ae), st[k].val + (e - ae), x)
                       : stage_row_sum<T>(e1 - e, colp + e, pv + e, x);
          if (dq != T(0)) x[q] = fma(bq - sum, dq, x[q]);
        }
        mbar_arrive(&empty[k]);
      }
    }
  }
  consumers_sync();
  if (t == 0) {
    if (*abort_v) {
      atomicExch(err, 1);
    } else if (atomicAdd(bar + 1, 1u) == (unsigned)G - 1) {   // the last CTA out
      bar[0] = 0;
      bar[1] = 0;
      __threadfence();
    }
  }
}

// the persistent sweep: grid = the CTAs resident at once (capped by the
// largest phase's tiles), launched cooperatively
template <typename T, int S, int CAPR>
static int gs_sweep_persistent(Sim *s, const SweepPlan &plan, const T *pv, const T *dinv,
                               const T *b, T *x) {
  constexpr int smem = S * (int)sizeof(TStage<T, CAPR>);
  auto kern = k_gs_c_sweep<T, S, CAPR>;
  static const int slots = [&]() {
    int dev = 0, nsm = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kTT + 32, smem);
    return std::max(n, 1) * std::max(nsm, 1);
  }();
  int tiles = 1;
  for (int p = 0; p < plan.nphase; ++p)
    tiles = std::max(tiles, (plan.r1[p] - plan.r0[p] + kTT - 1) / kTT);
  int grid = std::min(slots, tiles);
  if (s->alloc_failed) return DP_ENOMEM;
  s->waits_used = true;
  LaunchScope ls(s, "k_gs_c_sweep");
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kTT + 32);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  DP_CUDA(s, cudaLaunchKernelEx(&cfg, kern, plan, (const int *)s->lu_rowptr,
                                (const int *)s->l0_colp, pv, dinv, b, x,
                                (unsigned *)(s->dev_err + 4), s->dev_err));
  return DP_OK;
}

template <typename T> struct L0C;
template <> struct L0C<double> {
  static const double *pv(const Sim *s) { return s->l0_pv; }
  static const double *dinv(const Sim *s) { return s->dinv_c; }
  static const double *pval(const Sim *s) { return s->p0c_val; }
};
template <> struct L0C<float> {
  static const float *pv(const Sim *s) { return s->l0_pvf; }
  static const float *dinv(const Sim *s) { return s->dinv_cf; }
  static const float *pval(const Sim *s) { return s->p0c_valf; }
};

// level 0 runs in colour order (see Sim::l0c): not when the hierarchy has one
// level or the cluster cycle takes level 0 itself
static bool l0c_on(const Sim *s) { return s->l0c && s->lev.size() > 1 && s->cl_level != 0; }

// The level-0 colour kernel to launch: the autotuned one, except that the
// bulk-copy kernel (-1) needs its arrays at 16-byte boundaries (an
// allocator passed by the caller may give less) and otherwise runs as the
// thread-per-row kernel, which has the same results.
template <typename T>
static int l0_lanes(const Sim *s) {
  if (s->l0_G >= 0) return s->l0_G;
  auto a16 = [](const void *p) { return ((uintptr_t)p & 15) == 0; };
  return a16(s->lu_rowptr) && a16(s->l0_colp) && a16(L0C<T>::pv(s)) ? s->l0_G : 1;
}

// from_zero: x = 0 on entry (the pre-smoothing), so the first colour is the
// reduced formula of k_gs_c_first; preset: the kernel that wrote b has also
// written that x (X0Init), so the sweep starts with the second colour
template <typename T>
static int gs_sweep_c(Sim *s, const T *b, T *x, bool forward, bool from_zero = false,
                      bool preset = false) {
  RegionScope region(s, "sweep.gs");   // the sweep's launches, timed as one
  int nc = s->ncolour, G = l0_lanes<T>(s);
  if (G <= -4 && nc + 1 <= kSweepPhases) {   // the whole sweep in one launch
    SweepPlan plan{};
    plan.n = s->lu_cstart[nc];
    bool first = from_zero;
    for (int t = 0; t < nc; ++t) {
      int c = forward ? t : nc - 1 - t;
      int r0 = s->lu_cstart[c], r1 = s->lu_cstart[c + 1];
      if (r1 <= r0) continue;
      int kind = s->lu_cmaxlen[c] > kLongRow ? 2 : 1;
      if (first) {
        first = false;
        if (preset) continue;
        kind = 0;
      }
      plan.kind[plan.nphase] = kind;
      plan.r0[plan.nphase] = r0;
      plan.r1[plan.nphase] = r1;
      ++plan.nphase;
    }
    if (plan.nphase == 0) {   // nothing left to do (or no rows: x = 0)
      if (from_zero && !preset)
        DP_CUDA(s, cudaMemsetAsync(x, 0, (size_t)plan.n * sizeof(T), s->stream));
      return DP_OK;
    }
    return gs_sweep_persistent<T, 3, 6>(s, plan, L0C<T>::pv(s), L0C<T>::dinv(s), b, x);
  }
  if (G <= -4) G = 1;
  if (from_zero && !preset)
    DP_CUDA(s, cudaMemsetAsync(x, 0, (size_t)s->lu_cstart[nc] * sizeof(T), s->stream));
  std::vector<int> order;   // the non-empty colours in sweep order
  for (int t = 0; t < nc; ++t) {
    int c = forward ? t : nc - 1 - t;
    if (s->lu_cstart[c + 1] > s->lu_cstart[c]) order.push_back(c);
  }
  auto lng = [&](int c) { return s->lu_cmaxlen[c] > kLongRow; };
  bool first = from_zero;
  for (size_t t = 0; t < order.size(); ++t) {
    int c = order[t];
    int r0 = s->lu_cstart[c], r1 = s->lu_cstart[c + 1];
    if (first) {
      first = false;
      if (!preset)
        DP_LAUNCH(s, k_gs_c_first<T>, nblk(r1 - r0), kBlock, 0, r0, r1, L0C<T>::dinv(s), b, x);
      continue;
    }
    if (lng(c))
      DP_LAUNCH_PDL(s, kPdlWells, k_gs_c_wp<T>, r1 - r0, 32, 0, r0, s->lu_rowptr, s->l0_colp,
                    L0C<T>::pv(s), L0C<T>::dinv(s), b, x);
    else if (G > 1) {
      DP_SWITCH_G(G, DP_LAUNCH(s, (k_gs_cg<GG, T>), nblk((long long)(r1 - r0) * GG), kBlock,
                                     0, r0, r1, s->lu_rowptr, s->l0_colp, L0C<T>::pv(s),
                                     L0C<T>::dinv(s), b, x));
    } else if (G == 0)
      DP_LAUNCH(s, k_gs_cs<T>, nblk(r1 - r0), kBlock, 0, r0, r1, s->lu_rowptr, s->l0_colp,
                L0C<T>::pv(s), L0C<T>::dinv(s), b, x);
    else if (G < 0)
      sweep_tma<T>(s, G, r0, r1, L0C<T>::pv(s), L0C<T>::dinv(s), b, x, nullptr);
    else
      DP_LAUNCH(s, k_gs_c<T>, nblk(r1 - r0), kBlock, 0, r0, r1, s->lu_rowptr, s->l0_colp,
                L0C<T>::pv(s), L0C<T>::dinv(s), b, x);
  }
  return DP_OK;
}

template <typename T>
static int resid_c(Sim *s, const T *b, const T *x, T *r) {
  int nc = s->ncolour, c = 0, G = l0_lanes<T>(s);
  if (G <= -4) G = 1;   // the persistent sweep's residual: a thread per row
  while (c < nc) {   // runs of short-row colours in one launch, long-row colours a warp per row
    int r0 = s->lu_cstart[c];
    bool lng = s->lu_cmaxlen[c] > kLongRow;
    int c1 = c + 1;
    while (c1 < nc && (s->lu_cmaxlen[c1] > kLongRow) == lng) ++c1;
    int r1 = s->lu_cstart[c1];
    if (r1 > r0) {
      if (lng)
        DP_LAUNCH_PDL(s, kPdlWells, k_resid_c_wp<T>, r1 - r0, 32, 0, r0, s->lu_rowptr, s->l0_colp,
                      L0C<T>::pv(s), b, (T *)x, r);
      else if (G > 1) {
        DP_SWITCH_G(G, DP_LAUNCH(s, (k_resid_cg<GG, T>), nblk((long long)(r1 - r0) * GG),
                                       kBlock, 0, r0, r1, s->lu_rowptr, s->l0_colp,
                                       L0C<T>::pv(s), b, x, r));
      } else if (G == 0)
        DP_LAUNCH(s, k_resid_cs<T>, nblk(r1 - r0), kBlock, 0, r0, r1, s->lu_rowptr, s->l0_colp,
                  L0C<T>::pv(s), b, (T *)x, r);
      else if (G < 0)
        sweep_tma<T>(s, G, r0, r1, L0C<T>::pv(s), nullptr, b, (T *)x, r);
      else
        DP_LAUNCH(s, k_resid_c<T>, nblk(r1 - r0), kBlock, 0, r0, r1, s->lu_rowptr, s->l0_colp,
                  L0C<T>::pv(s), b, x, r);
    }
    c = c1;
  }
  return DP_OK;
}

template <typename T>
static int gs_sweep(Sim *s, Level &L, const T *b, T *x, bool forward) {
  const T *pv = nullptr;
  if (&L == &s->lev[0] && s->l0_lu) {
    if constexpr (sizeof(T) == 8) pv = (const T *)s->l0_pv; else pv = (const T *)s->l0_pvf;
  }
  if (pv) {
    for (int t = 0; t < L.ncolour; ++t) {
      int c = forward ? t : L.ncolour - 1 - t;
      int r0 = s->lu_cstart[c], r1 = s->lu_cstart[c + 1];
      if (r1 <= r0) continue;
      if (s->lu_cmaxlen[c] > kLongRow)
        DP_LAUNCH(s, k_gs_lu_w<T>, nblk(32LL * (r1 - r0)), kBlock, 0, r0, r1, s->perm,
                  s->lu_rowptr, s->lu_col, pv, LV<T>::dinv(L), b, x);
      else
        DP_LAUNCH(s, k_gs_lu<T>, nblk(r1 - r0), kBlock, 0, r0, r1, s->perm, s->lu_rowptr,
                  s->lu_col, pv, LV<T>::dinv(L), b, x);
    }
    return DP_OK;
  }
  for (int t = 0; t < L.ncolour; ++t) {
    int c = forward ? t : L.ncolour - 1 - t;
    int r0 = L.cstart[c], r1 = L.cstart[c + 1];
    if (r1 > r0) {
      long long thr = (long long)(r1 - r0) * L.G;
      bool done = false;
      if constexpr (std::is_same<T, float>::value) {
        if (use_bf16<T>(L.valh)) {
          DP_SWITCH_G(L.G, DP_LAUNCH(s, (k_gs_colour<GG, float, __nv_bfloat16>), nblk(thr), kBlock,
                                     0, r0, r1, L.clist, L.rowptr, L.col, L.valh, L.dinvf, b, x));
          done = true;
        }
      }
      if (!done)
        DP_SWITCH_G(L.G, DP_LAUNCH(s, (k_gs_colour<GG, T>), nblk(thr), kBlock, 0, r0, r1, L.clist,
                                   L.rowptr, L.col, LV<T>::val(L), LV<T>::dinv(L), b, x));
    }
  }
  return DP_OK;
}

// V(1,1) cycle from level l in precision T: pre-smoothing (colours forward,
// or one l1-Jacobi sweep), residual, restriction, coarse correction,
// prolongation, post-smoothing (colours reversed, or one l1-Jacobi sweep);
// dense LU on the coarsest level.  *res: where the result is, x or, after an
// l1-Jacobi post-smoothing (which cannot run in place), the level's r; the
// prolongation above reads it there.
// x_preset: level 0 in colour order and the pre-smoothing's first colour
// (and x = 0 on the other rows) already written with b (X0Init)
template <typename T>
static int vcycle_r(Sim *s, int l, const T *b, T *x, const T **res, bool x_preset = false) {
  *res = x;
  if (l == s->cl_level) return coarse_cycle<T>(s, l, b, x);
  const T *nres = nullptr;
  if (l == 0 && l0c_on(s)) {   // b and x in colour order
    Level &L = s->lev[0], &N = s->lev[1];
    T *r = LV<T>::r(L), *nb = LV<T>::b(N), *nx = LV<T>::x(N);
    DP_TRY(gs_sweep_c<T>(s, b, x, true, true, x_preset));   // from x = 0
    DP_TRY(resid_c<T>(s, b, x, r));
    DP_TRY(csr_mv<T>(s, N.n, L.r_G, L.r_rowptr, s->r0_colp, LV<T>::rval(L), r, nb, 0));
    {
      RegionScope region(s, "cycle.coarse");   // levels 1 and below, timed as one
      DP_TRY(vcycle_r<T>(s, 1, nb, nx, &nres));
    }
    DP_TRY(csr_mv<T>(s, L.n, L.p_G, s->p0c_rowptr, s->p0c_col, L0C<T>::pval(s), nres, x, 1,
                     true));
    return gs_sweep_c<T>(s, b, x, false);
  }
  Level &L = s->lev[l];
  int n = L.n;
  if (l == (int)s->lev.size() - 1) {
    if (s->coarse_n == n && n > 0) {
      if (s->coarse_inv)
        DP_LAUNCH_PDL(s, kPdlCoarse, k_dense_mv_p<T>, nblk(32LL * n), kBlock, 0, n,
                      s->coarse_inv, b, x, (int)pdl_trigger());
      else
        DP_LAUNCH(s, k_dense_solve<T>, 1, 1024, 0, n, s->coarse_lu, s->coarse_piv, b, x);
      return DP_OK;
    }
    if (L.l1) {
      DP_TRY(jacobi_pre<T>(s, L, b, x, LV<T>::r(L)));
      DP_TRY(jacobi_post<T>(s, L, b, x, LV<T>::r(L)));
      *res = LV<T>::r(L);
      return DP_OK;
    }
    DP_CUDA(s, cudaMemsetAsync(x, 0, (size_t)n * sizeof(T), s->stream));
    DP_TRY(gs_sweep<T>(s, L, b, x, true));
    DP_TRY(gs_sweep<T>(s, L, b, x, false));
    return DP_OK;
  }
  Level &N = s->lev[l + 1];
  T *r = LV<T>::r(L), *nb = LV<T>::b(N), *nx = LV<T>::x(N);
  if (L.l1) {
    DP_TRY(jacobi_pre<T>(s, L, b, x, r));
  } else {
    DP_CUDA(s, cudaMemsetAsync(x, 0, (size_t)n * sizeof(T), s->stream));
    DP_TRY(gs_sweep<T>(s, L, b, x, true));
    DP_TRY(csr_resid<T>(s, L, b, x, r));
  }
  DP_TRY(transfer_mv<T>(s, N.n, L.r_G, L.r_rowptr, L.r_col, LV<T>::rval(L), L.r_valh, r, nb, 0));
  DP_TRY(vcycle_r<T>(s, l + 1, nb, nx, &nres));
  DP_TRY(transfer_mv<T>(s, n, L.p_G, L.p_rowptr, L.p_col, LV<T>::pval(L), L.p_valh, nres, x, 1));
  if (L.l1) {
    DP_TRY(jacobi_post<T>(s, L, b, x, r));
    *res = r;
  } else {
    DP_TRY(gs_sweep<T>(s, L, b, x, false));
  }
  return DP_OK;
}

// the V-cycle with its result in x
template <typename T>
static int vcycle_t(Sim *s, int l, const T *b, T *x, bool x_preset = false) {
  const T *res = x;
  DP_TRY(vcycle_r<T>(s, l, b, x, &res, x_preset));
  if (res != x)
    DP_CUDA(s, cudaMemcpyAsync(x, res, (size_t)s->lev[l].n * sizeof(T), cudaMemcpyDeviceToDevice,
                               s->stream));
  return DP_OK;
}

int vcycle(Sim *s, int l, const double *b, double *x) { return vcycle_t<double>(s, l, b, x); }

// ---------------------------------------------------------------- autotuning
// Lanes per row of the AMG level kernels, chosen by timing: for every level,
// the level-operator kernel of its smoother (l1-Jacobi sweep, else the
// residual, which shares the Gauss-Seidel colour kernels' lane count), the
// prolongation and the restriction, each launched `reps` times per candidate
// with CUDA events on the simulation stream on the level's own work vectors.
// Colourings, aggregates and operators are not touched.
template <typename F>
static int time_launches(Sim *s, int reps, F launch, float *ms) {
  cudaEvent_t a = nullptr, b = nullptr;
  DP_CUDA(s, cudaEventCreate(&a));
  DP_CUDA(s, cudaEventCreate(&b));
  int rc = launch();   // warm-up
  if (rc == DP_OK) {
    cudaEventRecord(a, s->stream);
    for (int k = 0; k < reps && rc == DP_OK; ++k) rc = launch();
    cudaEventRecord(b, s->stream);
    if (cudaEventSynchronize(b) != cudaSuccess) rc = DP_ECUDA;
    else cudaEventElapsedTime(ms, a, b);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc == DP_ECUDA) s->fail(DP_ECUDA, "autotune timing");
  return rc;
}

template <typename T>
static int tune_level(Sim *s, int l, int reps, std::string &rep) {
  static const int cand[] = {1, 2, 4, 8, 16, 32};
  Level &L = s->lev[l];
  bool last = l + 1 == (int)s->lev.size();
  if (L.n == 0) return DP_OK;
  T *x = LV<T>::x(L), *b = LV<T>::b(L), *r = LV<T>::r(L);
  auto pick = [&](const char *what, int &field, auto launch_g) -> int {
    int old = field, best = old;
    float best_ms = 1e30f;
    char buf[160];
    std::string line;
    for (int g : cand) {
      float ms = 0.f;
      auto one = [&]() { return launch_g(g); };
      DP_TRY(time_launches(s, reps, one, &ms));
      std::snprintf(buf, sizeof buf, " %d:%.1f", g, 1000.f * ms / reps);
      line += buf;
      if (ms < best_ms) { best_ms = ms; best = g; }
    }
    field = best;
    std::snprintf(buf, sizeof buf, "level %d %s lanes %d -> %d (us per launch:%s)\n", l, what, old,
                  best, line.c_str());
    rep += buf;
    return DP_OK;
  };
  // level operator
  auto op = [&](int g) -> int {
    long long thr = (long long)L.n * g;
    if (L.l1) {
      DP_SWITCH_G(g, DP_LAUNCH_PDL(s, kPdlCoarse, (k_jacobi_sweep_p<GG, T>), nblk(thr), kBlock,
                                   0, L.n, L.rowptr, L.col, LV<T>::val(L), LV<T>::dinv(L), b, x,
                                   r, (int)pdl_trigger()));
    } else {
      DP_SWITCH_G(g, DP_LAUNCH(s, (k_csr_resid<GG, T>), nblk(thr), kBlock, 0, L.n, L.rowptr,
                               L.col, LV<T>::val(L), b, x, r));
    }
    return DP_OK;
  };
  DP_TRY(pick(L.l1 ? "l1-Jacobi sweep" : "residual", L.G, op));
  if (last) return DP_OK;
  Level &N = s->lev[l + 1];
  T *nx = LV<T>::x(N), *nb = LV<T>::b(N);
  auto prol = [&](int g) -> int {
    return csr_mv<T>(s, L.n, g, L.p_rowptr, L.p_col, LV<T>::pval(L), nx, r, 0);
  };
  auto restr = [&](int g) -> int {
    return csr_mv<T>(s, N.n, g, L.r_rowptr, L.r_col, LV<T>::rval(L), r, nb, 0);
  };
  DP_TRY(pick("prolongation", L.p_G, prol));
  DP_TRY(pick("restriction", L.r_G, restr));
  return DP_OK;
}

// Level 0 in colour order: the kernel of its short-row Gauss-Seidel colours
// and residual, timed as a V-cycle uses them (a forward sweep, the
// residual, a backward sweep) on the level's own vectors: a thread per row (1), a CTA's rows staged in shared memory
// (0), the tiles brought in by a producer warp's bulk copies (-1, -2, -3),
// or 2, 4, 8 lanes per row.
template <typename T>
static int tune_l0(Sim *s, int reps, std::string &rep) {
  if (!l0c_on(s)) return DP_OK;
  Level &L = s->lev[0];
  T *x = LV<T>::x(L), *b = LV<T>::b(L), *r = LV<T>::r(L);
  // 0: the CTA's rows staged in shared memory; -1, -2, -3: the pipelined bulk-copy kernels
  static const int cand[] = {1, 0, -1, -2, -3, -4, 2, 4, 8};
  int old = s->l0_G, best = old;
  float best_ms = 1e30f;
  std::string line;
  char buf[160];
  for (int g : cand) {
    s->l0_G = g;
    float ms = 0.f;
    auto one = [&]() -> int {
      DP_TRY(gs_sweep_c<T>(s, b, x, true));
      DP_TRY(resid_c<T>(s, b, x, r));
      return gs_sweep_c<T>(s, b, x, false);
    };
    int rc = time_launches(s, reps, one, &ms);
    if (rc != DP_OK) { s->l0_G = old; return rc; }
    std::snprintf(buf, sizeof buf, " %d:%.1f", g, 1000.f * ms / reps);
    line += buf;
    if (ms < best_ms) { best_ms = ms; best = g; }
  }
  s->l0_G = best;
  std::snprintf(buf, sizeof buf, "level 0 colour sweeps and residual lanes %d -> %d (us per two sweeps+residual:%s)\n",
                old, best, line.c_str());
  rep += buf;
  return DP_OK;
}

// The schedule of the coarse V-cycle: the levels from cl_level on in one
// thread-block-cluster launch (a persistent launch with cluster barriers
// between the colour phases) or one launch per phase; timed as whole
// V-cycles from level 0 on the level's own vectors.
template <typename T>
static int tune_cycle(Sim *s, int reps, std::string &rep) {
  if (s->cl_level < 0) return DP_OK;
  Level &L = s->lev[0];
  T *x = LV<T>::x(L), *b = LV<T>::b(L);
  int keep = s->cl_level;
  float ms[2] = {0.f, 0.f};
  for (int k = 0; k < 2; ++k) {
    s->cl_level = k == 0 ? keep : -1;
    auto one = [&]() -> int { return vcycle_t<T>(s, 0, b, x); };
    int rc = time_launches(s, reps, one, &ms[k]);
    if (rc != DP_OK) { s->cl_level = keep; return rc; }
  }
  s->cl_level = ms[1] < ms[0] ? -1 : keep;
  char buf[200];
  std::snprintf(buf, sizeof buf,
                "V-cycle schedule: cluster launch from level %d %.1f us, per-phase launches %.1f us -> %s\n",
                keep, 1000.f * ms[0] / reps, 1000.f * ms[1] / reps,
                s->cl_level < 0 ? "per-phase launches" : "cluster launch");
  rep += buf;
  return DP_OK;
}

int autotune(Sim *s, int reps, std::string &rep) {
  if (!s->amg_ready || s->opt.precond != 2) {
    s->fail(DP_EINVAL, "autotune needs the AMG hierarchy (one CPR-FPF solve first)");
    return DP_EINVAL;
  }
  reps = std::max(1, std::min(reps, 1000));
  for (int l = 0; l < (int)s->lev.size(); ++l) {
    if (s->opt.precision >= 1) DP_TRY(tune_level<float>(s, l, reps, rep));
    else DP_TRY(tune_level<double>(s, l, reps, rep));
  }
  if (s->opt.precision >= 1) {
    DP_TRY(tune_l0<float>(s, reps, rep));
    DP_TRY(tune_cycle<float>(s, reps, rep));
  } else {
    DP_TRY(tune_l0<double>(s, reps, rep));
    DP_TRY(tune_cycle<double>(s, reps, rep));
  }
  DP_CUDA(s, cudaStreamSynchronize(s->stream));
  graphs_free(s);   // the Arnoldi steps are captured again with the new launch shapes
  ++s->shapes;      // and a batch holding this realisation rebuilds its plan
  return DP_OK;
}

// ---------------------------------------------------------------- CPR-FPF
// z1 = F r;  z2 = z1 + P V(R (r - A z1));  z = z2 + F (r - A z2)

template <typename T>
__global__ void k_inject_add(int n, const T *xp, double *z, const int *imap) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[2 * i] += double(xp[imap ? __ldg(imap + i) : i]);
}

// The injection into the FP32 copy of z1 only (updated in FP32: no
// conversions on the FP64 pipe); the FP64 z1 takes the same correction in
// the final result gather (ilu_result's inj).
__global__ void k_inject_f32(int n, const float *xp, float *zf, const int *imap) {
  k_inject_f32_b(blockIdx.x, gridDim.x, n, xp, zf, imap);
}

// z2 = z1 + P e in the ILU(0) colour order, FP32: the pressure component
// of row q gets the level-0 correction of the same position (level 0 runs
// in that order), the other is z1's; the same sum as k_inject_f32's.
__global__ void __launch_bounds__(kBlock) k_inject_colour_f32(int n, const float2 *__restrict__ z1,
                                                              const float *__restrict__ xp,
                                                              float2 *__restrict__ z2) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  float2 v = z1[q];
  v.x += xp[q];
  z2[q] = v;
}


__global__ void k_to_f32(long long n, const double *x, float *y) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = float(x[i]);
}


int cpr_apply(Sim *s, const double *r, double *z) {
  int nb = s->K.n;
  long long N = 2LL * nb;
  bool f32 = s->opt.precision >= 1;
  if (s->opt.precond == 0) {
    DP_CUDA(s, cudaMemcpyAsync(z, r, N * 8, cudaMemcpyDeviceToDevice, s->stream));
    return DP_OK;
  }
  if (!f32) {
    if (s->opt.precond == 1) return ilu_apply(s, r, z);
    DP_TRY(ilu_apply(s, r, s->z1));
    const int *m = l0c_on(s) ? s->iperm : nullptr;   // level-0 vectors in colour order
    DP_LAUNCH(s, k_bsr_presid, 1 + nblk(s->sv_long0), kBlock, 0, nb, s->sv_sL, s->sv_sc,
              s->sv_long0, s->srowptr, s->scol, s->sa00, s->sa01, s->z1, r, s->rp, m);
    DP_TRY(vcycle(s, 0, s->rp, s->xp));
    DP_LAUNCH(s, k_inject_add<double>, nblk(nb), kBlock, 0, nb, s->xp, s->z1, m);
    DP_TRY(bsr_residual(s, r, s->z1, s->r1));
    DP_TRY((ilu_apply_t<double, double>(s, s->lu_val, s->r1)));
    return ilu_result<double>(s, s->z1, z);           // z = z2 + F (r - A z2)
  }
  // FP32 factor, FP32 V-cycle, FP32 stage residuals
  if (s->opt.precond == 1) {
    DP_TRY((ilu_apply_t<float, double>(s, s->lu_valf, r)));
    return ilu_result<float>(s, nullptr, z);
  }
  // the stage residuals from the FP32 copy of the operator
  // (z1 and z2 also kept in FP32 for the residuals' gathers; r - A z2 in FP32)
  // z1 in FP32 only: the colour-order result itself (s->ilu_zp, kept for
  // the final sum; the second application writes s->ilu_zp2), or, when level
  // 0 is not in colour order, gathered into natural order (z1f)
  Level &L0 = s->lev[0];
  DP_TRY((ilu_apply_t<float, double>(s, s->lu_valf, r)));
  const int *m = l0c_on(s) ? s->iperm : nullptr;     // level-0 vectors in colour order
  // with level 0 in colour order, z1 stays in the ILU(0) colour order: the
  // stage residuals gather it, and z2, there through the colour positions
  // of the operator's columns (scolc), so z1 is not gathered into natural
  // order at all; the products see the same values as from natural order
  bool cz = m && s->scolc && s->z2c;
  const float *z1s = cz ? reinterpret_cast<const float *>(s->ilu_zp) : s->z1f;
  const int *scs = cz ? s->scolc : s->scol;
  if (!cz) DP_TRY(ilu_result<float>(s, nullptr, nullptr, s->z1f));
  X0Init xi;   // in colour order, the pre-smoothing's start written with b
  if (m) {
    int f = 0;
    while (f < s->ncolour && s->lu_cstart[f + 1] <= s->lu_cstart[f]) ++f;
    if (f < s->ncolour) {
      xi.x = L0.xf;
      xi.dinv = s->dinv_cf;
      xi.f0 = s->lu_cstart[f];
      xi.f1 = s->lu_cstart[f + 1];
    }
  }
  DP_LAUNCH(s, k_bsr_presid_f32, 1 + nblk(s->sv_long0), kBlock, 0, nb, s->sv_sL, s->sv_sc,
            s->sv_long0, s->srowptr, scs, reinterpret_cast<const float2 *>(s->spf), z1s, r, L0.bf,
            m, xi);
  DP_TRY(vcycle_t<float>(s, 0, L0.bf, L0.xf, xi.x != nullptr));
  const float *z2s = s->z1f;
  if (cz) {
    DP_LAUNCH(s, k_inject_colour_f32, nblk(nb), kBlock, 0, nb,
              reinterpret_cast<const float2 *>(s->ilu_zp), L0.xf, reinterpret_cast<float2 *>(s->z2c));
    z2s = s->z2c;
  } else {
    DP_LAUNCH(s, k_inject_f32, nblk(nb), kBlock, 0, nb, L0.xf, s->z1f, m);
  }
  DP_LAUNCH(s, k_bsr_resid_f32, 1 + nblk(2LL * s->sv_long0), kBlock, 0, nb, s->sv_sL, s->sv_sc,
            s->sv_long0, s->srowptr, scs, s->svalf, z2s, r, s->r1f);
  float *zp2 = reinterpret_cast<float *>(s->ilu_zp2);
  DP_TRY((ilu_apply_t<float, float>(s, s->lu_valf, s->r1f, zp2)));
  // z = z2 + F (r - A z2), z2 = z1 + P e formed here (z1 from the first result)
  return ilu_result<float>(s, nullptr, z, nullptr, L0.xf, m ? 1 : 0,
                           reinterpret_cast<const float *>(s->ilu_zp), zp2);
}

// ---------------------------------------------------------------- FGMRES

// part[b][part_off + k] = block b's share of V_k . w for k < NV; with SELF
// also w . w into slot 31.  A gate that points at 0.0 makes the launch a
// no-op (the reorthogonalisation pass of an Arnoldi step that needs none).
// Each thread takes two double2 of w and of every V_k per trip (4 elements)
// and issues all of those loads before the FMAs, so that enough bytes are in
// flight to cover HBM latency; N is even and the vectors 16-byte aligned.
template <int NV, bool SELF>
__global__ void __launch_bounds__(kBlock, kDotBlocks / 152) k_multidot(long long N, const double *__restrict__ V,
                                                     long long ldv,
                                                     const double *__restrict__ w,
                                                     double *__restrict__ part, int part_off,
                                                     const double *__restrict__ gate) {
  k_multidot_b<NV, SELF>(blockIdx.x, gridDim.x, N, V, ldv, w, part, part_off, gate);
}

// dots[k] = sum_b part[b][k] (fixed order); mode 1: also add into H[:, j];
// mode 2: dots[0] = sqrt(sum), H[j+1][j] = it.
// Modes 3 and 4 are the two passes of classical Gram-Schmidt with the DGKS
// test (Daniel, Gragg, Kaufman and Stewart 1976): both add the projections
// into H[:, j] and take ||w - V h||^2 = w.w - h.h (slot 31 holds w.w).
// Mode 3 sets scal[4] = 1 when that is below reorth * w.w (cancellation: a
// second pass is needed; reorth >= 1: always), else stores beta = h_{j+1,j}
// in H and scal[2].
// Mode 4 runs only when scal[4] = 1 and stores beta.
// 256 threads: lane k of group g sums the partials of blocks g, g+8, ...;
// the eight group sums are then added in group order.
__global__ void __launch_bounds__(256) k_dot_final(const double *part, int nblocks, int nv,
                                                   double *dots, double *H, int m, int j,
                                                   int mode, double *scal, double reorth) {
  k_dot_final_b(blockIdx.x, gridDim.x, part, nblocks, nv, dots, H, m, j, mode, scal, reorth);
}

// One projection of the Arnoldi step: w - V c.  Pass 0 writes it back into
// w when scal[4] = 1 (a second pass follows), else writes the normalised
// vector (w - V c) / scal[2] into out; pass 1 runs only when scal[4] = 1 and
// writes the normalised vector.
__global__ void __launch_bounds__(kBlock) k_project(long long N, const double *__restrict__ V,
                                                    long long ldv, int nv,
                                                    const double *__restrict__ c,
                                                    double *__restrict__ w,
                                                    double *__restrict__ out,
                                                    const double *__restrict__ scal, int pass) {
  k_project_b(blockIdx.x, gridDim.x, N, V, ldv, nv, c, w, out, scal, pass);
}

// w -= sum_k c_k V_k (sign -1) or w += sum_k c_k V_k (sign +1)
__global__ void __launch_bounds__(kBlock) k_multi_axpy(long long N, const double *__restrict__ V,
                                                       long long ldv, int nv,
                                                       const double *__restrict__ c, double sign,
                                                       double *__restrict__ w) {
  k_multi_axpy_b(blockIdx.x, gridDim.x, N, V, ldv, nv, c, sign, w);
}

// y = x * alpha, or x / alpha (the reciprocal taken once per block: an FP64
// division is a long instruction sequence on GB300)
__global__ void k_scale(long long N, const double *x, const double *alpha, int invert, double *y) {
  k_scale_b(blockIdx.x, gridDim.x, N, x, alpha, invert, y);
}

// Givens rotations on column j of the Hessenberg matrix and the rotated
// right-hand side g; res_out = |g_{j+1}|.
__global__ void k_givens(double *H, double *cs, double *sn, double *g, int m, int j,
                         double *res_out) {
  k_givens_b(blockIdx.x, gridDim.x, H, cs, sn, g, m, j, res_out);
}

__global__ void k_backsub(const double *H, const double *g, int m, int jend, double *y) {
  k_backsub_b(blockIdx.x, gridDim.x, H, g, m, jend, y);
}

__global__ void k_init_g(double *g, int m, const double *beta) {
  k_init_g_b(blockIdx.x, gridDim.x, g, m, beta);
}

// V^T w (and, for modes 3 and 4, w.w) reduced by k_dot_final in `mode`;
// `gate` as for k_multidot.
static int dots(Sim *s, const double *V, long long ldv, int nv, const double *w, int mode, int j,
                const double *gate = nullptr) {
  long long N = 2LL * s->K.n;
  int nblocks = dot_blocks(N);
  for (int v0 = 0; v0 < nv; v0 += kDotVec) {
    int cnt = std::min(kDotVec, nv - v0);
    const double *Vb = V + (long long)v0 * ldv;
#define DP_MD(NVC)                                                                             \
  case NVC:                                                                                    \
    if (mode >= 3 && v0 == 0)                                                                  \
      DP_LAUNCH(s, (k_multidot<NVC, true>), nblocks, kBlock, 0, N, Vb, ldv, w, s->dots_part,   \
                v0, gate);                                                                     \
    else                                                                                       \
      DP_LAUNCH(s, (k_multidot<NVC, false>), nblocks, kBlock, 0, N, Vb, ldv, w,                \
                s->dots_part, v0, gate);                                                       \
    break;
    switch (cnt) {
      DP_MD(1) DP_MD(2) DP_MD(3) DP_MD(4) DP_MD(5) DP_MD(6) DP_MD(7) DP_MD(8)
    }
#undef DP_MD
  }
  DP_LAUNCH(s, k_dot_final, 1, 256, 0, s->dots_part, nblocks, nv, s->dots, s->H, s->m, j, mode,
            s->scal, s->opt.reorth);
  return DP_OK;
}

// ||x|| into s->scal[slot] (device) via the dot machinery
static int norm_into(Sim *s, const double *x, double *dst) {
  long long N = 2LL * s->K.n;
  int nblocks = dot_blocks(N);
  DP_LAUNCH(s, (k_multidot<1, false>), nblocks, kBlock, 0, N, x, 0LL, x, s->dots_part, 0,
            (const double *)nullptr);
  DP_LAUNCH(s, k_dot_final, 1, 256, 0, s->dots_part, nblocks, 1, dst, s->H, s->m, 0, 0, s->scal,
            0.0);
  return DP_OK;
}

__global__ void k_sqrt_inplace(double *v) {
  k_sqrt_inplace_b(blockIdx.x, gridDim.x, v);
}

// One Arnoldi step of FGMRES for column j: z_j = M v_j, w = A z_j, then
// classical Gram-Schmidt against v_0..v_j with the DGKS test: the second
// pass runs only when the first left less than reorth ||w||^2, and
// h_{j+1,j} = ||w - V h|| comes from w.w - h.h, so each pass reads the basis
// twice (dots, projection) and the projection writes v_{j+1} normalised.
// Then the Givens rotations, and |g_{j+1}| into scal[3].
static int arnoldi_step(Sim *s, int j) {
  int m = s->m;
  long long N = 2LL * s->K.n;
  int gridN = (int)std::min<long long>(nblk(N), kDotBlocks * 4);
  double *vj = s->V + (long long)j * N, *zj = s->Z + (long long)j * N;
  double *vnext = s->V + (long long)(j + 1) * N;
  DP_TRY(cpr_apply(s, vj, zj));
  DP_TRY(bsr_spmv(s, zj, s->w));
  DP_TRY(dots(s, s->V, N, j + 1, s->w, 3, j));
  DP_LAUNCH(s, k_project, gridN, kBlock, 0, N, s->V, N, j + 1, s->dots, s->w, vnext, s->scal, 0);
  DP_TRY(dots(s, s->V, N, j + 1, s->w, 4, j, s->scal + 4));
  DP_LAUNCH(s, k_project, gridN, kBlock, 0, N, s->V, N, j + 1, s->dots, s->w, vnext, s->scal, 1);
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
  long long N = 2LL * s->K.n;
  bool use_graph = s->opt.use_graphs && s->timing.kernel_id < 0;
  double *x = s->yk;
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
    // v_0 = r / ||r||.  The first cycle starts from x = 0, where r = b - A 0
    // = b exactly and ||r|| = ||b|| is already in scal[0]: no product.
    const double *beta_dev = s->scal + 0;
    double beta = bnorm;
    if (total > 0) {
      DP_TRY(bsr_residual(s, s->bh, x, s->V));
      DP_TRY(norm_into(s, s->V, s->scal + 1));
      DP_LAUNCH(s, k_sqrt_inplace, 1, 1, 0, s->scal + 1);
      DP_CUDA(s, cudaMemcpyAsync(s->h_res + 1, s->scal + 1, 8, cudaMemcpyDeviceToHost, s->stream));
      DP_CUDA(s, cudaStreamSynchronize(s->stream));
      beta = s->h_res[1];
      beta_dev = s->scal + 1;
    }
    res = beta;
    if (beta <= tol * bnorm) { conv = true; break; }
    DP_LAUNCH(s, k_scale, nblk(N), kBlock, 0, N, total > 0 ? s->V : s->bh, beta_dev, 1, s->V);
    DP_CUDA(s, cudaMemsetAsync(s->H, 0, (size_t)(m + 1) * m * 8, s->stream));
    DP_LAUNCH(s, k_init_g, 1, 64, 0, s->g, m, beta_dev);
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
  long long N = 2LL * s->K.n;
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
  if (s->opt.precision >= 1) {
    s->z1f = (float *)dalloc(s, (size_t)N * 4);
    s->r1f = (float *)dalloc(s, (size_t)N * 4);
    if (!s->z1f || !s->r1f) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
  }
  s->rp = (double *)dalloc(s, (size_t)s->K.n * 8);
  s->xp = (double *)dalloc(s, (size_t)s->K.n * 8);
  if (!s->V || !s->Z || !s->w || !s->H || !s->cs || !s->sn || !s->g || !s->hy || !s->dots_part ||
      !s->dots || !s->scal || !s->z1 || !s->r1 || !s->rp || !s->xp) {
    s->fail(DP_ENOMEM, "allocation failed");
    return DP_ENOMEM;
  }
  return DP_OK;
}

__global__ void k_to_f32_i(long long n, const double *x, float *y) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = float(x[i]);
}

__global__ void k_to_bf16(long long n, const double *x, __nv_bfloat16 *y) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = __double2bfloat16(x[i]);
}

// BF16 copy of n FP64 values into *dst (allocated on first use).
static int to_bf16(Sim *s, long long n, const double *src, __nv_bfloat16 **dst) {
  if (n <= 0) return DP_OK;
  if (!*dst) {
    *dst = (__nv_bfloat16 *)dalloc(s, (size_t)n * 2);
    if (!*dst) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
  }
  DP_LAUNCH(s, k_to_bf16, nblk(n), kBlock, 0, n, src, *dst);
  return DP_OK;
}

// FP32 copies of the AMG operators, transfer operators and inverse
// diagonals (precisions 1 and 2), refreshed with the FP64 values: every
// level, or (coarse = false) the level-0 operator and scaling only.  With
// precision 2 the operators of levels >= 1 below the coarsest, and their
// prolongation and restriction, also get BF16 copies, which the FP32 cycle
// reads instead (values rounded to 8 significant bits; the scalings 1/a_ii
// and every vector stay FP32, the arithmetic FP32).
int mixed_refresh(Sim *s, bool coarse) {
  for (size_t l = 0; l < s->lev.size(); ++l) {
    if (!coarse) {
      // level 0 only; in colour order its FP32 values and 1/a_ii come from the
      // decoupling and from l0_refresh instead
      Level &L = s->lev[0];
      if (!s->l0c) {
        DP_LAUNCH(s, k_to_f32_i, nblk(L.nnz), kBlock, 0, (long long)L.nnz, L.val, L.valf);
        DP_LAUNCH(s, k_to_f32_i, nblk(L.n), kBlock, 0, (long long)L.n, L.dinv, L.dinvf);
      }
      break;
    }
    Level &L = s->lev[l];
    DP_LAUNCH(s, k_to_f32_i, nblk(L.nnz), kBlock, 0, (long long)L.nnz, L.val, L.valf);
    DP_LAUNCH(s, k_to_f32_i, nblk(L.n), kBlock, 0, (long long)L.n, L.dinv, L.dinvf);
    bool last = l + 1 == s->lev.size();
    if (!last) {
      DP_LAUNCH(s, k_to_f32_i, nblk(L.p_nnz), kBlock, 0, (long long)L.p_nnz, L.p_val, L.p_valf);
      DP_LAUNCH(s, k_to_f32_i, nblk(L.r_nnz), kBlock, 0, (long long)L.r_nnz, L.r_val, L.r_valf);
    }
    if (s->opt.precision == 2 && l >= 1 && !last) {
      DP_TRY(to_bf16(s, L.nnz, L.val, &L.valh));
      DP_TRY(to_bf16(s, L.p_nnz, L.p_val, &L.p_valh));
      DP_TRY(to_bf16(s, L.r_nnz, L.r_val, &L.r_valh));
    }
  }
  DP_CUDA(s, cudaGetLastError());
  return DP_OK;
}

}  // namespace dp
