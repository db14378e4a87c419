/*
 * CPU FP64 oracle: dual-porosity two-phase (oil-water) fully implicit
 * Newton step with CPR-FPF preconditioned flexible GMRES.
 *
 * TEST INFRASTRUCTURE ONLY: tests, the smoke check and the CPU baseline of
 * the benchmark load it; the CUDA library never does.  Plain sequential C,
 * FP64 throughout, compiled with -ffp-contract=off so that every expression
 * is evaluated exactly as written.  Where the paper is silent, the reading
 * taken is stated at the function that implements it.
 *
 * Paper sections followed (Shen, Cui, Liu, Zhu, Zhong, Chen et al.):
 *   Section 2      Darcy law (Eq. 1-2), two-phase mass conservation, the
 *                  constraints (Phi = p - rho g z, so + sw = 1, p_cow = 0),
 *                  the dual-porosity system Eq. "prob", the transfer term
 *                  q_mf with upstream weighting, the perforation rate, the
 *                  well index and Peaceman's effective radius.
 *   Section 3      FIM with unknowns (p, sw) per cell and p_b per well,
 *                  backward Euler, cell-centred finite differences,
 *                  F(x) = 0 with N = 2n + tau (Eq. "nonlinear").
 *   Section 3.1    Algorithm 1 (inexact Newton) and the forcing terms.
 *   Section 3.2    block Jacobian, decoupling D^-1 A x = D^-1 b
 *                  (Eq. "decoupled-eq") by a modified Gauss-Jordan step,
 *                  CPR-FPF preconditioner, GMRES (Section 4, Example 3).
 */
#include "dpsim_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define OG_OK 0
#define OG_EINVAL (-1)
#define OG_ENOMEM (-2)
#define OG_ELINEAR (-4)
#define OG_ENEWTON (-5)

/* ------------------------------------------------------------------ */
/* small containers                                                    */
/* ------------------------------------------------------------------ */

typedef struct {            /* scalar CSR, rows sorted by column */
  int n, ncol, nnz;
  int *rowptr, *col;
  double *val;
} og_csr;

typedef struct {            /* 2x2-block BSR, blocks row-major [a00 a01 a10 a11] */
  int n, nnz;
  int *rowptr, *col, *diag;
  double *val;
} og_bsr;

static void *zalloc(size_t n, size_t s) {
  if (n == 0) n = 1;
  return calloc(n, s);
}

static void csr_free(og_csr *a) {
  free(a->rowptr); free(a->col); free(a->val);
  memset(a, 0, sizeof(*a));
}

static void sort_int(int *a, int n) {          /* insertion sort, short rows */
  for (int i = 1; i < n; ++i) {
    int v = a[i], j = i - 1;
    while (j >= 0 && a[j] > v) { a[j + 1] = a[j]; --j; }
    a[j + 1] = v;
  }
}

static int find_col(const int *col, int lo, int hi, int c) {
  for (int e = lo; e < hi; ++e) if (col[e] == c) return e;
  return -1;
}

static double dot(const double *a, const double *b, int n) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

static double nrm2(const double *a, int n) { return sqrt(dot(a, a, n)); }

/* ------------------------------------------------------------------ */
/* 2x2 block helpers                                                   */
/* ------------------------------------------------------------------ */

/* inverse of [[a b][c d]] = (1/(ad - bc)) [[d -b][-c a]] */
static void inv2(const double *a, double *o) {
  double det = a[0] * a[3] - a[1] * a[2];
  double id = 1.0 / det;
  o[0] = a[3] * id; o[1] = -a[1] * id; o[2] = -a[2] * id; o[3] = a[0] * id;
}

static void mul2(const double *a, const double *b, double *o) {  /* o = a b */
  double t0 = a[0] * b[0] + a[1] * b[2];
  double t1 = a[0] * b[1] + a[1] * b[3];
  double t2 = a[2] * b[0] + a[3] * b[2];
  double t3 = a[2] * b[1] + a[3] * b[3];
  o[0] = t0; o[1] = t1; o[2] = t2; o[3] = t3;
}

static void mv2(const double *a, const double *x, double *y) {  /* y = a x */
  double y0 = a[0] * x[0] + a[1] * x[1];
  double y1 = a[2] * x[0] + a[3] * x[1];
  y[0] = y0; y[1] = y1;
}

/* y = A x for a block matrix, x and y of length 2n */
static void bsr_mv(const og_bsr *A, const double *x, double *y) {
  for (int i = 0; i < A->n; ++i) {
    double s0 = 0.0, s1 = 0.0;
    for (int e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e) {
      const double *a = A->val + 4 * (size_t)e;
      const double *xj = x + 2 * (size_t)A->col[e];
      s0 += a[0] * xj[0] + a[1] * xj[1];
      s1 += a[2] * xj[0] + a[3] * xj[1];
    }
    y[2 * i] = s0; y[2 * i + 1] = s1;
  }
}

static void csr_mv(const og_csr *A, const double *x, double *y) {
  for (int i = 0; i < A->n; ++i) {
    double s = 0.0;
    for (int e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e) s += A->val[e] * x[A->col[e]];
    y[i] = s;
  }
}

/* ------------------------------------------------------------------ */
/* Greedy first-fit colouring in natural row order.                    */
/* The paper does not say how its ILU orders unknowns; the reading     */
/* taken is the textbook greedy colouring: row i gets the smallest     */
/* colour not used by an adjacent row of smaller index.                */
/* ------------------------------------------------------------------ */

static int greedy_colour(int n, const int *rowptr, const int *col, int *colour) {
  int ncol = 0;
  int cap = 64;
  int *used = (int *)zalloc((size_t)cap, sizeof(int));
  for (int i = 0; i < n; ++i) {
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      int j = col[e];
      if (j < i) {
        int c = colour[j];
        if (c >= cap) {
          int nc = 2 * c + 2;
          used = (int *)realloc(used, (size_t)nc * sizeof(int));
          for (int t = cap; t < nc; ++t) used[t] = -1;
          cap = nc;
        }
        used[c] = i + 1;       /* mark colour c as used by row i */
      }
    }
    int c = 0;
    while (c < cap && used[c] == i + 1) ++c;
    colour[i] = c;
    if (c + 1 > ncol) ncol = c + 1;
  }
  free(used);
  return ncol;
}

int oracle_greedy_colour(int32_t n, const int32_t *rowptr, const int32_t *col,
                         int32_t *colour) {
  return greedy_colour(n, rowptr, col, colour);
}

/* ------------------------------------------------------------------ */
/* Block ILU(0) (Section 3.2: the full-system stage of CPR-FPF).       */
/* Rows are ordered by (colour, index); the factorisation is the       */
/* textbook IKJ incomplete LU restricted to the matrix pattern, done   */
/* on the permuted matrix:                                             */
/*   for i: for k < i in row i: L_ik = A_ik U_kk^-1;                    */
/*          for j > k in row i and in row k: A_ij -= L_ik A_kj.         */
/* ------------------------------------------------------------------ */

typedef struct {
  og_bsr M;          /* permuted factor: L (unit, strictly lower), U, pattern of A */
  double *dinv;      /* [4n] inverse of U_ii */
  int *perm;         /* perm[new] = old */
  int *iperm;        /* iperm[old] = new */
  double *t1, *t2;   /* work vectors, 2n */
} og_ilu;

static void ilu_free(og_ilu *f) {
  free(f->M.rowptr); free(f->M.col); free(f->M.diag); free(f->M.val);
  free(f->dinv); free(f->perm); free(f->iperm); free(f->t1); free(f->t2);
  memset(f, 0, sizeof(*f));
}

/* Build the permuted pattern once (integer setup). */
static int ilu_setup(og_ilu *f, const og_bsr *A, const int *colour) {
  int n = A->n;
  f->perm = (int *)zalloc((size_t)n, sizeof(int));
  f->iperm = (int *)zalloc((size_t)n, sizeof(int));
  int maxc = 0;
  for (int i = 0; i < n; ++i) if (colour[i] > maxc) maxc = colour[i];
  int pos = 0;
  for (int c = 0; c <= maxc; ++c)
    for (int i = 0; i < n; ++i)
      if (colour[i] == c) { f->perm[pos] = i; f->iperm[i] = pos; ++pos; }
  f->M.n = n; f->M.nnz = A->nnz;
  f->M.rowptr = (int *)zalloc((size_t)n + 1, sizeof(int));
  f->M.col = (int *)zalloc((size_t)A->nnz, sizeof(int));
  f->M.diag = (int *)zalloc((size_t)n, sizeof(int));
  f->M.val = (double *)zalloc(4 * (size_t)A->nnz, sizeof(double));
  f->dinv = (double *)zalloc(4 * (size_t)n, sizeof(double));
  f->t1 = (double *)zalloc(2 * (size_t)n, sizeof(double));
  f->t2 = (double *)zalloc(2 * (size_t)n, sizeof(double));
  int e = 0;
  for (int i = 0; i < n; ++i) {
    int old = f->perm[i];
    f->M.rowptr[i] = e;
    for (int q = A->rowptr[old]; q < A->rowptr[old + 1]; ++q) f->M.col[e++] = f->iperm[A->col[q]];
    sort_int(f->M.col + f->M.rowptr[i], e - f->M.rowptr[i]);
  }
  f->M.rowptr[n] = e;
  for (int i = 0; i < n; ++i) f->M.diag[i] = find_col(f->M.col, f->M.rowptr[i], f->M.rowptr[i + 1], i);
  return 0;
}

static void ilu_factor(og_ilu *f, const og_bsr *A) {
  int n = A->n;
  og_bsr *M = &f->M;
  /* copy A into the permuted pattern */
  for (int i = 0; i < n; ++i) {
    int old = f->perm[i];
    for (int e = M->rowptr[i]; e < M->rowptr[i + 1]; ++e) {
      int qo = find_col(A->col, A->rowptr[old], A->rowptr[old + 1], f->perm[M->col[e]]);
      memcpy(M->val + 4 * (size_t)e, A->val + 4 * (size_t)qo, 4 * sizeof(double));
    }
  }
  for (int i = 0; i < n; ++i) {
    for (int e = M->rowptr[i]; e < M->rowptr[i + 1]; ++e) {
      int k = M->col[e];
      if (k >= i) break;
      double *lik = M->val + 4 * (size_t)e;
      double t[4];
      mul2(lik, f->dinv + 4 * (size_t)k, t);          /* L_ik = A_ik U_kk^-1 */
      memcpy(lik, t, sizeof(t));
      for (int e2 = e + 1; e2 < M->rowptr[i + 1]; ++e2) {   /* j > k in row i */
        int j = M->col[e2];
        int qk = find_col(M->col, M->diag[k] + 1, M->rowptr[k + 1], j);
        if (qk < 0) continue;
        double u[4];
        mul2(lik, M->val + 4 * (size_t)qk, u);
        double *aij = M->val + 4 * (size_t)e2;
        aij[0] -= u[0]; aij[1] -= u[1]; aij[2] -= u[2]; aij[3] -= u[3];
      }
    }
    inv2(M->val + 4 * (size_t)M->diag[i], f->dinv + 4 * (size_t)i);
  }
}

/* z = (LU)^-1 r, vectors in natural order */
static void ilu_apply(const og_ilu *f, const double *r, double *z) {
  const og_bsr *M = &f->M;
  int n = M->n;
  double *y = f->t1;
  for (int i = 0; i < n; ++i) {                      /* forward, unit L */
    int old = f->perm[i];
    double s0 = r[2 * old], s1 = r[2 * old + 1];
    for (int e = M->rowptr[i]; e < M->diag[i]; ++e) {
      const double *l = M->val + 4 * (size_t)e;
      const double *yk = y + 2 * (size_t)M->col[e];
      s0 -= l[0] * yk[0] + l[1] * yk[1];
      s1 -= l[2] * yk[0] + l[3] * yk[1];
    }
    y[2 * i] = s0; y[2 * i + 1] = s1;
  }
  double *x = f->t2;
  for (int i = n - 1; i >= 0; --i) {                 /* backward */
    double s[2] = {y[2 * i], y[2 * i + 1]};
    for (int e = M->diag[i] + 1; e < M->rowptr[i + 1]; ++e) {
      const double *u = M->val + 4 * (size_t)e;
      const double *xj = x + 2 * (size_t)M->col[e];
      s[0] -= u[0] * xj[0] + u[1] * xj[1];
      s[1] -= u[2] * xj[0] + u[3] * xj[1];
    }
    mv2(f->dinv + 4 * (size_t)i, s, x + 2 * (size_t)i);
  }
  for (int i = 0; i < n; ++i) {
    int old = f->perm[i];
    z[2 * old] = x[2 * i]; z[2 * old + 1] = x[2 * i + 1];
  }
}

int oracle_ilu0_solve(int32_t n, const int32_t *rowptr, const int32_t *col,
                      const double *val, const int32_t *colour,
                      const double *b, double *x) {
  og_bsr A = {n, rowptr[n], (int *)rowptr, (int *)col, NULL, (double *)val};
  og_ilu f; memset(&f, 0, sizeof(f));
  ilu_setup(&f, &A, colour);
  ilu_factor(&f, &A);
  ilu_apply(&f, b, x);
  ilu_free(&f);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Smoothed-aggregation AMG for the pressure stage of CPR-FPF.         */
/* The paper names CPR-FPF only (Section 3.2); the pressure solver     */
/* taken here is one V(1,1) cycle of smoothed aggregation:             */
/*   strength  S_ij: max(|a_ij|,|a_ji|) >= theta sqrt(|a_ii a_jj|)     */
/*   MIS(2) on S by synchronous rounds of (state, hash, index) maxima  */
/*   aggregates grown from the MIS(2) roots (distance 1, then 2)       */
/*   P = (I - omega D^-1 A) T, omega = (4/3) / max_i sum_j|a_ij|/|a_ii| */
/*   A_c = P^T A P, coarsest level by dense LU with partial pivoting   */
/*   smoother: multicolour Gauss-Seidel (forward before, reverse after) */
/* ------------------------------------------------------------------ */

uint32_t oracle_hash32(uint32_t i) {
  uint32_t h = i * 0x9E3779B1u;
  h ^= h >> 16; h *= 0x85EBCA6Bu;
  h ^= h >> 13; h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

typedef struct {
  og_csr A;          /* level operator */
  unsigned char *strong;  /* strength flag per entry of A (setup) */
  int *agg;          /* aggregate of each row, -1 when not aggregated */
  int nagg;
  int *colour; int ncolour;
  og_csr P, R;       /* prolongator n x nagg and its transpose */
  double *x, *b, *r; /* work */
} og_level;

typedef struct {
  int nlev;
  og_level lev[32];
  int smoother;      /* levels from this one on use l1-Jacobi, the finer ones multicolour GS */
  double theta;
  int coarse_max, max_levels;
  int dense_n;       /* coarsest dense LU size (0: coarsest uses GS) */
  double *lu; int *piv;
} og_amg;

/* strength flags per entry, symmetric by construction */
static unsigned char *strength(const og_csr *A, double theta) {
  unsigned char *s = (unsigned char *)zalloc((size_t)A->nnz, 1);
  double *diag = (double *)zalloc((size_t)A->n, sizeof(double));
  for (int i = 0; i < A->n; ++i)
    for (int e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e)
      if (A->col[e] == i) diag[i] = A->val[e];
  for (int i = 0; i < A->n; ++i) {
    for (int e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e) {
      int j = A->col[e];
      if (j == i) continue;
      int et = find_col(A->col, A->rowptr[j], A->rowptr[j + 1], i);
      double aji = et >= 0 ? A->val[et] : 0.0;
      double lhs = fmax(fabs(A->val[e]), fabs(aji));
      double rhs = theta * sqrt(fabs(diag[i] * diag[j]));
      s[e] = (lhs >= rhs) ? 1 : 0;
    }
  }
  free(diag);
  return s;
}

typedef struct { int state; uint32_t h; int idx; } tup;   /* state 0 out, 1 undecided, 2 in */

static int tup_gt(tup a, tup b) {
  if (a.state != b.state) return a.state > b.state;
  if (a.h != b.h) return a.h > b.h;
  return a.idx > b.idx;
}

/* MIS(2) by synchronous rounds (Bell, Dalton, Olson 2012): each round every
 * node takes the maximum tuple over its distance-2 strong neighbourhood; an
 * undecided node that is its own maximum joins the set, an undecided node
 * whose maximum is in the set leaves it.  Nodes without strong neighbours
 * start outside (they are not aggregated). */
static void mis2(const og_csr *A, const unsigned char *s, int *state) {
  int n = A->n;
  tup *t0 = (tup *)zalloc((size_t)n, sizeof(tup));
  tup *t1 = (tup *)zalloc((size_t)n, sizeof(tup));
  for (int i = 0; i < n; ++i) {
    int deg = 0;
    for (int e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e) deg += s[e];
    state[i] = deg > 0 ? 1 : 0;
  }
  for (;;) {
    int und = 0;
    for (int i = 0; i < n; ++i) und += (state[i] == 1);
    if (!und) break;
    for (int i = 0; i < n; ++i) { t0[i].state = state[i]; t0[i].h = oracle_hash32((uint32_t)i); t0[i].idx = i; }
    for (int pass = 0; pass < 2; ++pass) {
      for (int i = 0; i < n; ++i) {
        tup m = t0[i];
        for (int e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e)
          if (s[e] && tup_gt(t0[A->col[e]], m)) m = t0[A->col[e]];
        t1[i] = m;
      }
      tup *tt = t0; t0 = t1; t1 = tt;
    }
    for (int i = 0; i < n; ++i) {
      if (state[i] != 1) continue;
      if (t0[i].idx == i) state[i] = 2;
      else if (t0[i].state == 2) state[i] = 0;
    }
  }
  free(t0); free(t1);
}

int oracle_mis2(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val,
                double theta, int32_t *state) {
  if (n < 1 || !rowptr || !col || !val || !state) return OG_EINVAL;
  og_csr A = {n, n, rowptr[n], (int *)rowptr, (int *)col, (double *)val};
  unsigned char *s = strength(&A, theta);
  mis2(&A, s, state);
  free(s);
  int roots = 0;
  for (int i = 0; i < n; ++i) roots += state[i] == 2;
  return roots;
}

/* Aggregates: roots numbered in index order; a distance-1 node joins the
 * strongly connected root with the largest (hash, index); a distance-2 node
 * joins the aggregate of its strongly connected, already assigned neighbour
 * with the largest (hash, index), using the assignment after the first pass. */
static int aggregate(const og_csr *A, const unsigned char *s, const int *state, int *agg) {
  int n = A->n, nagg = 0;
  for (int i = 0; i < n; ++i) agg[i] = (state[i] == 2) ? nagg++ : -1;
  int *a1 = (int *)zalloc((size_t)n, sizeof(int));
  memcpy(a1, agg, (size_t)n * sizeof(int));
  for (int i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    int best = -1; uint32_t bh = 0;
    for (int e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e) {
      int j = A->col[e];
      if (!s[e] || state[j] != 2) continue;
      uint32_t h = oracle_hash32((uint32_t)j);
      if (best < 0 || h > bh || (h == bh && j > best)) { best = j; bh = h; }
    }
    if (best >= 0) a1[i] = agg[best];
  }
  int *a2 = (int *)zalloc((size_t)n, sizeof(int));
  memcpy(a2, a1, (size_t)n * sizeof(int));
  for (int i = 0; i < n; ++i) {
    if (a1[i] >= 0) continue;
    int best = -1; uint32_t bh = 0;
    for (int e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e) {
      int j = A->col[e];
      if (!s[e] || a1[j] < 0) continue;
      uint32_t h = oracle_hash32((uint32_t)j);
      if (best < 0 || h > bh || (h == bh && j > best)) { best = j; bh = h; }
    }
    if (best >= 0) a2[i] = a1[best];
  }
  memcpy(agg, a2, (size_t)n * sizeof(int));
  free(a1); free(a2);
  return nagg;
}

/* Sparse product C = L R (Gustavson): for each row r of L, for each entry
 * (r,k) in column order, for each entry (k,c) of R in column order,
 * C_rc += L_rk R_kc.  Every C_rc is a sum taken in increasing k. */
static void spgemm(const og_csr *L, const og_csr *R, og_csr *C) {
  int n = L->n, nc = R->ncol;
  int *mark = (int *)zalloc((size_t)nc, sizeof(int));
  double *acc = (double *)zalloc((size_t)nc, sizeof(double));
  int *list = (int *)zalloc((size_t)nc, sizeof(int));
  for (int c = 0; c < nc; ++c) mark[c] = -1;
  int cap = L->nnz + 16, nnz = 0;
  int *col = (int *)zalloc((size_t)cap, sizeof(int));
  double *val = (double *)zalloc((size_t)cap, sizeof(double));
  int *rowptr = (int *)zalloc((size_t)n + 1, sizeof(int));
  for (int r = 0; r < n; ++r) {
    int len = 0;
    for (int e = L->rowptr[r]; e < L->rowptr[r + 1]; ++e) {
      int k = L->col[e];
      double lv = L->val[e];
      for (int q = R->rowptr[k]; q < R->rowptr[k + 1]; ++q) {
        int c = R->col[q];
        if (mark[c] != r) { mark[c] = r; acc[c] = 0.0; list[len++] = c; }
        acc[c] = acc[c] + lv * R->val[q];
      }
    }
    sort_int(list, len);
    if (nnz + len > cap) {
      while (nnz + len > cap) cap *= 2;
      col = (int *)realloc(col, (size_t)cap * sizeof(int));
      val = (double *)realloc(val, (size_t)cap * sizeof(double));
    }
    rowptr[r] = nnz;
    for (int t = 0; t < len; ++t) { col[nnz] = list[t]; val[nnz] = acc[list[t]]; ++nnz; }
  }
  rowptr[n] = nnz;
  free(mark); free(acc); free(list);
  C->n = n; C->ncol = nc; C->nnz = nnz; C->rowptr = rowptr; C->col = col; C->val = val;
}

static void transpose(const og_csr *A, og_csr *T) {
  int n = A->n, m = A->ncol;
  T->n = m; T->ncol = n; T->nnz = A->nnz;
  T->rowptr = (int *)zalloc((size_t)m + 1, sizeof(int));
  T->col = (int *)zalloc((size_t)A->nnz, sizeof(int));
  T->val = (double *)zalloc((size_t)A->nnz, sizeof(double));
  for (int e = 0; e < A->nnz; ++e) T->rowptr[A->col[e] + 1]++;
  for (int c = 0; c < m; ++c) T->rowptr[c + 1] += T->rowptr[c];
  int *fill = (int *)zalloc((size_t)m, sizeof(int));
  for (int i = 0; i < n; ++i)                 /* rows in increasing i: sorted */
    for (int e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e) {
      int c = A->col[e];
      int p = T->rowptr[c] + fill[c]++;
      T->col[p] = i; T->val[p] = A->val[e];
    }
  free(fill);
}

/* P = (I - omega D_F^-1 A_F) T with T the 0/1 aggregate injection and A_F
 * the filtered operator of smoothed aggregation: the strong off-diagonal
 * entries of A, with every weak off-diagonal entry of a row added to its
 * diagonal, d_i = a_ii + sum_{j weak} a_ij (increasing j).  Entry (i, J) of
 * P is [agg(i) == J] - (omega / d_i) * sum_{k in F(i), agg(k) = J} aF_ik, the
 * sum taken in increasing k; omega = (4/3) / max_i sum_{j in F(i)} |aF_ij| / |d_i|.
 * A row whose filtered diagonal is zero keeps its row of T. */
static void smoothed_prolongator(const og_csr *A, const unsigned char *strong,
                                 const int *agg, int nagg, og_csr *P) {
  int n = A->n;
  og_csr F = {n, A->ncol, A->nnz, NULL, NULL, NULL};
  F.rowptr = (int *)zalloc((size_t)n + 1, sizeof(int));
  F.col = (int *)zalloc((size_t)A->nnz, sizeof(int));
  F.val = (double *)zalloc((size_t)A->nnz, sizeof(double));
  double *diag = (double *)zalloc((size_t)n, sizeof(double));
  int nnz = 0;
  for (int i = 0; i < n; ++i) {
    double d = 0.0;
    for (int e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e) if (A->col[e] == i) d = A->val[e];
    for (int e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e)
      if (A->col[e] != i && !strong[e]) d = d + A->val[e];
    diag[i] = d;
    F.rowptr[i] = nnz;
    for (int e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e) {
      int j = A->col[e];
      if (j == i) { F.col[nnz] = j; F.val[nnz] = d; ++nnz; }
      else if (strong[e]) { F.col[nnz] = j; F.val[nnz] = A->val[e]; ++nnz; }
    }
  }
  F.rowptr[n] = nnz; F.nnz = nnz;
  double rho = 0.0;
  for (int i = 0; i < n; ++i) {
    if (diag[i] == 0.0) continue;
    double s = 0.0;
    for (int e = F.rowptr[i]; e < F.rowptr[i + 1]; ++e) s = s + fabs(F.val[e]);
    double ratio = s / fabs(diag[i]);
    if (ratio > rho) rho = ratio;
  }
  double omega = rho > 0.0 ? (4.0 / 3.0) / rho : 0.0;
  og_csr T = {n, nagg, 0, NULL, NULL, NULL};
  T.rowptr = (int *)zalloc((size_t)n + 1, sizeof(int));
  for (int i = 0; i < n; ++i) T.rowptr[i + 1] = T.rowptr[i] + (agg[i] >= 0);
  T.nnz = T.rowptr[n];
  T.col = (int *)zalloc((size_t)T.nnz, sizeof(int));
  T.val = (double *)zalloc((size_t)T.nnz, sizeof(double));
  for (int i = 0; i < n; ++i) if (agg[i] >= 0) { T.col[T.rowptr[i]] = agg[i]; T.val[T.rowptr[i]] = 1.0; }
  og_csr FT;
  spgemm(&F, &T, &FT);                         /* A_F T, sums in increasing k */
  P->n = n; P->ncol = nagg; P->nnz = FT.nnz;
  P->rowptr = FT.rowptr; P->col = FT.col; P->val = FT.val;
  for (int i = 0; i < n; ++i) {
    double w = diag[i] != 0.0 ? omega / diag[i] : 0.0;
    for (int e = P->rowptr[i]; e < P->rowptr[i + 1]; ++e) {
      double t = (agg[i] == P->col[e]) ? 1.0 : 0.0;
      P->val[e] = t - w * P->val[e];
    }
  }
  csr_free(&T);
  csr_free(&F);
  free(diag);
}

static void dense_lu(double *a, int *piv, int n) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    double m = fabs(a[(size_t)k * n + k]);
    for (int i = k + 1; i < n; ++i) {
      double v = fabs(a[(size_t)i * n + k]);
      if (v > m) { m = v; p = i; }
    }
    piv[k] = p;
    if (p != k)
      for (int j = 0; j < n; ++j) {
        double t = a[(size_t)k * n + j]; a[(size_t)k * n + j] = a[(size_t)p * n + j]; a[(size_t)p * n + j] = t;
      }
    double d = a[(size_t)k * n + k];
    if (d == 0.0) continue;
    for (int i = k + 1; i < n; ++i) {
      double l = a[(size_t)i * n + k] / d;
      a[(size_t)i * n + k] = l;
      for (int j = k + 1; j < n; ++j) a[(size_t)i * n + j] -= l * a[(size_t)k * n + j];
    }
  }
}

static void dense_lu_solve(const double *a, const int *piv, int n, const double *b, double *x) {
  for (int i = 0; i < n; ++i) x[i] = b[i];
  for (int k = 0; k < n; ++k) {
    int p = piv[k];
    if (p != k) { double t = x[k]; x[k] = x[p]; x[p] = t; }
    for (int i = k + 1; i < n; ++i) x[i] -= a[(size_t)i * n + k] * x[k];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int j = i + 1; j < n; ++j) s -= a[(size_t)i * n + j] * x[j];
    double d = a[(size_t)i * n + i];
    x[i] = d != 0.0 ? s / d : 0.0;
  }
}

static void amg_free(og_amg *m) {
  for (int l = 0; l < m->nlev; ++l) {
    og_level *L = &m->lev[l];
    csr_free(&L->A); csr_free(&L->P); csr_free(&L->R);
    free(L->agg); free(L->colour); free(L->x); free(L->b); free(L->r); free(L->strong);
  }
  free(m->lu); free(m->piv);
  double theta = m->theta;
  int cmax = m->coarse_max, mlev = m->max_levels, sm = m->smoother;
  memset(m, 0, sizeof(*m));
  m->theta = theta; m->coarse_max = cmax; m->max_levels = mlev; m->smoother = sm;
}

static void csr_copy(const og_csr *a, og_csr *b) {
  b->n = a->n; b->ncol = a->ncol; b->nnz = a->nnz;
  b->rowptr = (int *)zalloc((size_t)a->n + 1, sizeof(int));
  b->col = (int *)zalloc((size_t)a->nnz, sizeof(int));
  b->val = (double *)zalloc((size_t)a->nnz, sizeof(double));
  memcpy(b->rowptr, a->rowptr, ((size_t)a->n + 1) * sizeof(int));
  memcpy(b->col, a->col, (size_t)a->nnz * sizeof(int));
  memcpy(b->val, a->val, (size_t)a->nnz * sizeof(double));
}

#define OG_DENSE_MAX 4096

/* Coarsest level: dense LU when small enough, else Gauss-Seidel sweeps. */
static void amg_coarsest_factor(og_amg *m) {
  og_level *L = &m->lev[m->nlev - 1];
  int n = L->A.n;
  free(m->lu); free(m->piv); m->lu = NULL; m->piv = NULL; m->dense_n = 0;
  if (n > OG_DENSE_MAX || n == 0) return;
  m->dense_n = n;
  m->lu = (double *)zalloc((size_t)n * n, sizeof(double));
  m->piv = (int *)zalloc((size_t)n, sizeof(int));
  for (int i = 0; i < n; ++i)
    for (int e = L->A.rowptr[i]; e < L->A.rowptr[i + 1]; ++e)
      m->lu[(size_t)i * n + L->A.col[e]] = L->A.val[e];
  dense_lu(m->lu, m->piv, n);
}

/* Full setup on first use: integer structure (strength, MIS(2), aggregates,
 * colourings) and values. */
static int amg_setup(og_amg *m, const og_csr *A0) {
  amg_free(m);
  m->nlev = 1;
  csr_copy(A0, &m->lev[0].A);
  for (int l = 0;; ++l) {
    og_level *L = &m->lev[l];
    int n = L->A.n;
    L->colour = (int *)zalloc((size_t)n, sizeof(int));
    L->ncolour = greedy_colour(n, L->A.rowptr, L->A.col, L->colour);
    L->x = (double *)zalloc((size_t)n, sizeof(double));
    L->b = (double *)zalloc((size_t)n, sizeof(double));
    L->r = (double *)zalloc((size_t)n, sizeof(double));
    L->agg = (int *)zalloc((size_t)n, sizeof(int));
    for (int i = 0; i < n; ++i) L->agg[i] = -1;
    if (n <= m->coarse_max || l + 1 >= m->max_levels) break;
    unsigned char *s = strength(&L->A, m->theta);
    int *state = (int *)zalloc((size_t)n, sizeof(int));
    mis2(&L->A, s, state);
    int nagg = aggregate(&L->A, s, state, L->agg);
    free(state);
    L->strong = s;
    if (nagg == 0 || nagg >= n) { for (int i = 0; i < n; ++i) L->agg[i] = -1; break; }
    L->nagg = nagg;
    smoothed_prolongator(&L->A, L->strong, L->agg, nagg, &L->P);
    transpose(&L->P, &L->R);
    og_csr AP;
    spgemm(&L->A, &L->P, &AP);
    og_level *N = &m->lev[l + 1];
    spgemm(&L->R, &AP, &N->A);
    csr_free(&AP);
    m->nlev++;
  }
  amg_coarsest_factor(m);
  return 0;
}

/* Numeric refresh with the integer structure kept (values of level 0 new);
 * with coarse = 0 only level 0 takes the new values and the transfer and
 * coarse operators of the last refresh stay. */
static void amg_refresh(og_amg *m, const double *val0, int coarse) {
  memcpy(m->lev[0].A.val, val0, (size_t)m->lev[0].A.nnz * sizeof(double));
  if (!coarse) return;
  for (int l = 0; l + 1 < m->nlev; ++l) {
    og_level *L = &m->lev[l];
    csr_free(&L->P); csr_free(&L->R);
    smoothed_prolongator(&L->A, L->strong, L->agg, L->nagg, &L->P);
    transpose(&L->P, &L->R);
    og_csr AP, C;
    spgemm(&L->A, &L->P, &AP);
    spgemm(&L->R, &AP, &C);
    memcpy(m->lev[l + 1].A.val, C.val, (size_t)C.nnz * sizeof(double));
    csr_free(&AP); csr_free(&C);
  }
  amg_coarsest_factor(m);
}

/* One Gauss-Seidel sweep over the colours in the given direction:
 * x_i = (b_i - sum_{j != i} a_ij x_j) / a_ii for every row of a colour. */
static void gs_sweep(const og_level *L, const double *b, double *x, int forward) {
  for (int t = 0; t < L->ncolour; ++t) {
    int c = forward ? t : L->ncolour - 1 - t;
    for (int i = 0; i < L->A.n; ++i) {
      if (L->colour[i] != c) continue;
      double s = b[i], d = 0.0;
      for (int e = L->A.rowptr[i]; e < L->A.rowptr[i + 1]; ++e) {
        int j = L->A.col[e];
        if (j == i) d = L->A.val[e];
        else s -= L->A.val[e] * x[j];
      }
      if (d != 0.0) x[i] = s / d;
    }
  }
}

/* One l1-Jacobi sweep (Baker, Falgout, Kolev, Yang 2011):
 * x_i <- x_i + (b_i - (A x)_i) / sum_j |a_ij|, all rows from the old x. */
static void l1_jacobi(const og_level *L, const double *b, double *x, double *t) {
  for (int i = 0; i < L->A.n; ++i) {
    double s = 0.0, l1 = 0.0;
    for (int e = L->A.rowptr[i]; e < L->A.rowptr[i + 1]; ++e) {
      s += L->A.val[e] * x[L->A.col[e]];
      l1 += fabs(L->A.val[e]);
    }
    t[i] = l1 != 0.0 ? x[i] + (b[i] - s) / l1 : x[i];
  }
  memcpy(x, t, sizeof(double) * (size_t)L->A.n);
}

static void smooth(const og_amg *m, int l, const double *b, double *x, int forward) {
  const og_level *L = &m->lev[l];
  if (l >= m->smoother) l1_jacobi(L, b, x, L->r);   /* r is free while smoothing */
  else gs_sweep(L, b, x, forward);
}

static void vcycle(og_amg *m, int l, const double *b, double *x) {
  og_level *L = &m->lev[l];
  int n = L->A.n;
  if (l == m->nlev - 1) {
    if (m->dense_n == n && n > 0) { dense_lu_solve(m->lu, m->piv, n, b, x); return; }
    for (int i = 0; i < n; ++i) x[i] = 0.0;
    smooth(m, l, b, x, 1); smooth(m, l, b, x, 0);
    return;
  }
  for (int i = 0; i < n; ++i) x[i] = 0.0;
  smooth(m, l, b, x, 1);                              /* pre-smoothing */
  csr_mv(&L->A, x, L->r);
  for (int i = 0; i < n; ++i) L->r[i] = b[i] - L->r[i];
  og_level *N = &m->lev[l + 1];
  csr_mv(&L->R, L->r, N->b);                          /* restrict */
  vcycle(m, l + 1, N->b, N->x);
  double *px = L->r;
  csr_mv(&L->P, N->x, px);                            /* prolong */
  for (int i = 0; i < n; ++i) x[i] += px[i];
  smooth(m, l, b, x, 0);                              /* post-smoothing */
}

int oracle_amg_create(int32_t n, const int32_t *rowptr, const int32_t *col,
                      const double *val, double theta, int32_t coarse_max,
                      int32_t max_levels, void **out) {
  og_amg *m = (og_amg *)zalloc(1, sizeof(og_amg));
  m->theta = theta; m->coarse_max = coarse_max; m->max_levels = max_levels > 30 ? 30 : max_levels;
  m->smoother = 30;
  og_csr A = {n, n, rowptr[n], (int *)rowptr, (int *)col, (double *)val};
  amg_setup(m, &A);
  *out = m;
  return 0;
}

int oracle_amg_set_smoother(void *amg, int32_t gs_levels) {
  if (!amg || gs_levels < 0) return OG_EINVAL;
  ((og_amg *)amg)->smoother = gs_levels;
  return 0;
}

int oracle_amg_vcycle(void *amg, const double *b, double *x) {
  vcycle((og_amg *)amg, 0, b, x);
  return 0;
}

int oracle_amg_info(void *amg, int32_t level, int32_t *n, int32_t *nnz, int32_t *nagg) {
  og_amg *m = (og_amg *)amg;
  if (level < 0 || level >= m->nlev) return OG_EINVAL;
  *n = m->lev[level].A.n; *nnz = m->lev[level].A.nnz; *nagg = m->lev[level].nagg;
  return m->nlev;
}

int oracle_amg_arrays(void *amg, int32_t level, int32_t *rowptr, int32_t *col,
                      double *val, int32_t *agg, int32_t *colour) {
  og_amg *m = (og_amg *)amg;
  if (level < 0 || level >= m->nlev) return OG_EINVAL;
  og_level *L = &m->lev[level];
  if (rowptr) memcpy(rowptr, L->A.rowptr, ((size_t)L->A.n + 1) * sizeof(int));
  if (col) memcpy(col, L->A.col, (size_t)L->A.nnz * sizeof(int));
  if (val) memcpy(val, L->A.val, (size_t)L->A.nnz * sizeof(double));
  if (agg) memcpy(agg, L->agg, (size_t)L->A.n * sizeof(int));
  if (colour) memcpy(colour, L->colour, (size_t)L->A.n * sizeof(int));
  return 0;
}

void oracle_amg_destroy(void *amg) {
  if (!amg) return;
  amg_free((og_amg *)amg);
  free(amg);
}

/* ------------------------------------------------------------------ */
/* Flexible GMRES(m), right preconditioned (Section 3.2 / Example 3:    */
/* GMRES with the CPR preconditioner).  Classical Gram-Schmidt applied  */
/* twice, Givens rotations, zero initial guess, stop when the rotated   */
/* residual |g_{j+1}| <= tol * ||b|| or after maxit iterations.         */
/* ------------------------------------------------------------------ */

typedef void (*op_fn)(void *ctx, const double *x, double *y);

static int fgmres(int n, op_fn A, void *actx, op_fn M, void *mctx,
                  const double *b, double *x, int m, int maxit, double tol, double reorth,
                  int *iters, double *relres) {
  double *V = (double *)zalloc((size_t)(m + 1) * n, sizeof(double));
  double *Z = (double *)zalloc((size_t)m * n, sizeof(double));
  double *H = (double *)zalloc((size_t)(m + 1) * m, sizeof(double));
  double *cs = (double *)zalloc((size_t)m, sizeof(double));
  double *sn = (double *)zalloc((size_t)m, sizeof(double));
  double *g = (double *)zalloc((size_t)m + 1, sizeof(double));
  double *y = (double *)zalloc((size_t)m, sizeof(double));
  double *w = (double *)zalloc((size_t)n, sizeof(double));
  double *h = (double *)zalloc((size_t)m + 1, sizeof(double));
  for (int i = 0; i < n; ++i) x[i] = 0.0;
  double bnorm = nrm2(b, n);
  int total = 0, conv = 0;
  double res = bnorm;
  if (bnorm == 0.0) { conv = 1; res = 0.0; }
  while (!conv && total < maxit) {
    A(actx, x, w);
    for (int i = 0; i < n; ++i) V[i] = b[i] - w[i];
    double beta = nrm2(V, n);
    res = beta;
    if (beta <= tol * bnorm) { conv = 1; break; }
    for (int i = 0; i < n; ++i) V[i] /= beta;
    memset(H, 0, sizeof(double) * (size_t)(m + 1) * m);
    memset(g, 0, sizeof(double) * ((size_t)m + 1));
    g[0] = beta;
    int j, jend = 0;
    for (j = 0; j < m && total < maxit; ++j) {
      double *vj = V + (size_t)j * n, *zj = Z + (size_t)j * n;
      if (M) M(mctx, vj, zj); else memcpy(zj, vj, sizeof(double) * (size_t)n);
      A(actx, zj, w);
      double wn = nrm2(w, n), hn = 0.0;
      for (int pass = 0; pass < 2; ++pass) {            /* classical Gram-Schmidt */
        for (int i = 0; i <= j; ++i) h[i] = dot(V + (size_t)i * n, w, n);
        for (int i = 0; i <= j; ++i) {
          const double *vi = V + (size_t)i * n;
          for (int q = 0; q < n; ++q) w[q] -= h[i] * vi[q];
          H[(size_t)i * m + j] += h[i];
        }
        hn = nrm2(w, n);
        /* a second pass only after cancellation (Daniel, Gragg, Kaufman and
         * Stewart's test): ||w - V h||^2 < reorth ||w||^2; reorth >= 1: always */
        if (!(reorth >= 1.0 || hn * hn < reorth * (wn * wn))) break;
      }
      H[(size_t)(j + 1) * m + j] = hn;
      if (hn != 0.0) {
        double *v1 = V + (size_t)(j + 1) * n;
        for (int q = 0; q < n; ++q) v1[q] = w[q] / hn;
      }
      for (int i = 0; i < j; ++i) {                      /* old rotations */
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
      ++total;
      jend = j + 1;
      res = fabs(g[j + 1]);
      if (res <= tol * bnorm) { conv = 1; break; }
      if (hn == 0.0) break;
    }
    for (int i = jend - 1; i >= 0; --i) {                /* back substitution */
      double s = g[i];
      for (int k = i + 1; k < jend; ++k) s -= H[(size_t)i * m + k] * y[k];
      double d = H[(size_t)i * m + i];
      y[i] = d != 0.0 ? s / d : 0.0;
    }
    for (int i = 0; i < jend; ++i) {
      const double *zi = Z + (size_t)i * n;
      for (int q = 0; q < n; ++q) x[q] += y[i] * zi[q];
    }
    if (jend == 0) break;
  }
  *iters = total;
  *relres = bnorm > 0.0 ? res / bnorm : 0.0;
  free(V); free(Z); free(H); free(cs); free(sn); free(g); free(y); free(w); free(h);
  return conv ? 0 : OG_ELINEAR;
}

/* ------------------------------------------------------------------ */
/* CPR-FPF (Section 3.2): a full-system stage F (block ILU(0) of the    */
/* decoupled matrix), a pressure stage (AMG V-cycle on the pressure     */
/* block), and the full-system stage again, composed multiplicatively:  */
/*   z1 = F r;  z2 = z1 + P V(R (r - A z1));  z = z2 + F (r - A z2)     */
/* R takes the pressure component of each block row, P injects it.     */
/* ------------------------------------------------------------------ */

typedef struct {
  const og_bsr *A;
  og_ilu *ilu;
  og_amg *amg;
  int mode;          /* 1 ILU only, 2 CPR-FPF */
  double *r1, *z1, *rp, *xp;
} og_cpr;

static void op_bsr(void *ctx, const double *x, double *y) { bsr_mv((const og_bsr *)ctx, x, y); }

static void op_cpr(void *ctx, const double *r, double *z) {
  og_cpr *c = (og_cpr *)ctx;
  int n = c->A->n;
  if (c->mode == 1) { ilu_apply(c->ilu, r, z); return; }
  ilu_apply(c->ilu, r, c->z1);                        /* z1 = F r */
  bsr_mv(c->A, c->z1, c->r1);
  for (int i = 0; i < 2 * n; ++i) c->r1[i] = r[i] - c->r1[i];
  for (int i = 0; i < n; ++i) c->rp[i] = c->r1[2 * i];  /* restrict to pressure */
  vcycle(c->amg, 0, c->rp, c->xp);
  for (int i = 0; i < n; ++i) c->z1[2 * i] += c->xp[i];  /* z2 */
  bsr_mv(c->A, c->z1, c->r1);
  for (int i = 0; i < 2 * n; ++i) c->r1[i] = r[i] - c->r1[i];
  ilu_apply(c->ilu, c->r1, z);
  for (int i = 0; i < 2 * n; ++i) z[i] += c->z1[i];
}

int oracle_fgmres_bsr(int32_t n, const int32_t *rowptr, const int32_t *col,
                      const double *val, const double *b, double *x,
                      int32_t precond, int32_t restart, int32_t maxit, double tol,
                      int32_t *iters, double *relres) {
  og_bsr A = {n, rowptr[n], (int *)rowptr, (int *)col, NULL, (double *)val};
  og_ilu f; memset(&f, 0, sizeof(f));
  og_cpr c; memset(&c, 0, sizeof(c));
  int it = 0; double rr = 0.0;
  int rc;
  if (precond == 1) {
    int *colour = (int *)zalloc((size_t)n, sizeof(int));
    greedy_colour(n, rowptr, col, colour);
    ilu_setup(&f, &A, colour);
    ilu_factor(&f, &A);
    free(colour);
    c.A = &A; c.ilu = &f; c.mode = 1;
    rc = fgmres(2 * n, op_bsr, &A, op_cpr, &c, b, x, restart, maxit, tol, 1.0, &it, &rr);
    ilu_free(&f);
  } else {
    rc = fgmres(2 * n, op_bsr, &A, NULL, NULL, b, x, restart, maxit, tol, 1.0, &it, &rr);
  }
  *iters = it; *relres = rr;
  return rc;
}

static void op_csr(void *ctx, const double *x, double *y) { csr_mv((const og_csr *)ctx, x, y); }
static void op_amg(void *ctx, const double *r, double *z) { vcycle((og_amg *)ctx, 0, r, z); }

int oracle_fgmres_amg(int32_t n, const int32_t *rowptr, const int32_t *col,
                      const double *val, const double *b, double *x,
                      double theta, int32_t coarse_max, int32_t restart,
                      int32_t maxit, double tol, int32_t *iters, double *relres) {
  og_csr A = {n, n, rowptr[n], (int *)rowptr, (int *)col, (double *)val};
  og_amg *m = NULL;
  oracle_amg_create(n, rowptr, col, val, theta, coarse_max, 20, (void **)&m);
  int it = 0; double rr = 0.0;
  int rc = fgmres(n, op_csr, &A, op_amg, m, b, x, restart, maxit, tol, 1.0, &it, &rr);
  oracle_amg_destroy(m);
  *iters = it; *relres = rr;
  return rc;
}

/* ------------------------------------------------------------------ */
/* The simulator: grid, properties, assembly, Newton.                  */
/* ------------------------------------------------------------------ */

typedef struct {
  int cell;          /* fracture cell perforated */
  int well;
  double wi;
} og_perf;

typedef struct {
  og_grid g; og_fluid f; og_options o;
  double sigma, c_rock, p_ref_rock;
  double *kf, *km, *phi_f, *phi_m;
  int nwells; og_well *wells;
  int *ctl_kind; double *ctl_target;   /* the wells' own controls (restored each timestep) */
  int cap; double *pc_own[2];          /* some p_cow table given; the tables (copies) */
  int nL, nc, nb;
  og_bsr J;          /* Jacobian, natural order; decoupled in place by solve (full system) */
  og_bsr K;          /* with schur: the fracture-and-well system, decoupled in place */
  double *RK;        /* with schur: its residual [2 (nL + nwells)] */
  double *yk;        /* with schur: its update */
  int *kmap;         /* with schur: entry of J each entry of K copies (-1: S_ff) */
  int *pos_fm, *pos_mf; /* with schur: blocks (f, m) and (m, f) of each location */
  double *Minv;      /* with schur: inverted (m, m) block of each location */
  double *R;         /* residual [2 nb] */
  double *p, *sw, *bhp, *pn, *swn, *bhpn;
  double *Mn;        /* accumulation at the old time level [2 nc] */
  double dt, inv_dt;
  int nperf; og_perf *perf;
  int *colour; int ncolour;
  og_ilu ilu;
  og_amg amg; int amg_ready;
  og_csr Ap;
  double *y, *bh;    /* Newton update and decoupled right-hand side */
  double norms[8];
  double prev_res;
  int newton_iter;
  /* forcing terms 1-2 of Section 3.1 need the linear residual of the last
   * solve: lq = R + J y with J as assembled (Ja keeps J's assembled values
   * when the full system is decoupled in place), and its scaled norms at the
   * next assembly: lin_norms[0] = ||R~(lq)||_2, lin_norms[1] = ||R~(R - lq)||_2 */
  double *Ja, *lq;
  int have_lq;
  double lin_norms[2];
} og_sim;

/* Peaceman's effective radius for a vertical well (Section 2, the first
 * line of the Peaceman system, with D_x, D_y, k_x, k_y of the block) and the
 * well index W = 2 pi k h w_frac / (ln(r_e/r_w) + s) with k h = sqrt(kx ky) dz
 * and w_frac = 1. */
static double well_index(double kx, double ky, double dx, double dy, double dz,
                         double rw, double skin) {
  double ryx = ky / kx, rxy = kx / ky;
  double re = 0.28 * sqrt(sqrt(ryx) * dx * dx + sqrt(rxy) * dy * dy)
              / (pow(ryx, 0.25) + pow(rxy, 0.25));
  double wfrac = 1.0;
  return (((2.0 * M_PI) * sqrt(kx * ky)) * dz) * wfrac / (log(re / rw) + skin);
}

static void cell_ijk(const og_sim *s, int loc, int *i, int *j, int *k) {
  *i = loc % s->g.nx;
  *j = (loc / s->g.nx) % s->g.ny;
  *k = loc / (s->g.nx * s->g.ny);
}

/* Two-point transmissibility of a connection between cells a < b.
 * Fracture-fracture: harmonic mean, 2 A ka kb / (D (ka + kb)).
 * Fracture-matrix of one location: shape-factor transfer sigma km V
 * (Warren-Root / Gilman-Kazemi, the reading of omega in q_mf).
 * Also returns z_a - z_b (cell-centre depth difference). */
static double conn_trans(const og_sim *s, int a, int b, double *dzab) {
  int la = a / 2, lb = b / 2;
  double V = (s->g.dx * s->g.dy) * s->g.dz;
  if (la == lb) { *dzab = 0.0; return (s->sigma * s->km[la]) * V; }
  int ia, ja, ka, ib, jb, kb;
  cell_ijk(s, la, &ia, &ja, &ka);
  cell_ijk(s, lb, &ib, &jb, &kb);
  double A, D;
  if (ka != kb) { A = s->g.dx * s->g.dy; D = s->g.dz; }
  else if (ja != jb) { A = s->g.dx * s->g.dz; D = s->g.dy; }
  else { A = s->g.dy * s->g.dz; D = s->g.dx; }
  double za = s->g.top_depth + ((double)ka + 0.5) * s->g.dz;
  double zb = s->g.top_depth + ((double)kb + 0.5) * s->g.dz;
  *dzab = za - zb;
  double k1 = s->kf[la], k2 = s->kf[lb];
  return ((2.0 * A) * (k1 * k2)) / (D * (k1 + k2));
}

/* Cell properties (Section 2): linear densities rho = rho_ref (1 + c (p -
 * p_ref)), porosity phi = phi_ref (1 + c_r (p - p_ref)), Corey relative
 * permeabilities krw = S^2, kro = (1 - S)^2 of the normalised saturation
 * S = clamp((sw - swc)/(1 - swc - sor), 0, 1), mobilities kr / mu, and their
 * derivatives. */
typedef struct {
  double rho[2], drho[2], phi, dphi, lam[2], dlam[2];
  double pc, dpc;              /* p_cow(s_w) of the cell's continuum and d/ds_w */
} og_props;

/* Capillary pressure p_cow(s_w) (Section 2: p_w = p_o - p_cow(s_w)) from a
 * table of (s_w, p_cow) pairs: linear between neighbouring points, constant
 * (zero slope) below the first and above the last; no table: zero. */
static void cap_pressure(int n, const double *t, double sw, double *pc, double *dpc) {
  if (n == 0) { *pc = 0.0; *dpc = 0.0; return; }
  if (sw <= t[0]) { *pc = t[1]; *dpc = 0.0; return; }
  if (sw >= t[2 * (n - 1)]) { *pc = t[2 * n - 1]; *dpc = 0.0; return; }
  int k = 0;
  while (sw >= t[2 * (k + 1)]) ++k;      /* t[2k] <= sw < t[2k + 2] */
  double ds = t[2 * k + 2] - t[2 * k];
  double dp = t[2 * k + 3] - t[2 * k + 1];
  *dpc = dp / ds;
  *pc = t[2 * k + 1] + dp * ((sw - t[2 * k]) / ds);
}

static void props(const og_sim *s, int c, double p, double sw, og_props *q) {
  int loc = c / 2;
  double phi_ref = (c % 2 == 0) ? s->phi_f[loc] : s->phi_m[loc];
  double dp = p - s->f.p_ref;
  q->rho[0] = s->f.rho_o_ref * (1.0 + s->f.c_o * dp);
  q->rho[1] = s->f.rho_w_ref * (1.0 + s->f.c_w * dp);
  q->drho[0] = s->f.rho_o_ref * s->f.c_o;
  q->drho[1] = s->f.rho_w_ref * s->f.c_w;
  q->phi = phi_ref * (1.0 + s->c_rock * (p - s->p_ref_rock));
  q->dphi = phi_ref * s->c_rock;
  double inv_span = 1.0 / ((1.0 - s->f.swc) - s->f.sor);
  double S = (sw - s->f.swc) * inv_span, dS;
  if (S <= 0.0) { S = 0.0; dS = 0.0; }
  else if (S >= 1.0) { S = 1.0; dS = 0.0; }
  else dS = inv_span;
  double inv_mu_o = 1.0 / s->f.mu_o, inv_mu_w = 1.0 / s->f.mu_w;
  double so = 1.0 - S;
  q->lam[1] = (S * S) * inv_mu_w;
  q->dlam[1] = ((2.0 * S) * dS) * inv_mu_w;
  q->lam[0] = (so * so) * inv_mu_o;
  q->dlam[0] = (-((2.0 * so) * dS)) * inv_mu_o;
  int k = c % 2;
  cap_pressure(s->f.pc_n[k], s->f.pc_table[k], sw, &q->pc, &q->dpc);
}

/* Mass of each phase in a cell, V phi rho s, and its derivatives. */
static void accumulation(const og_sim *s, int c, double sw, const og_props *q,
                         double M[2], double dM[4]) {
  double V = (s->g.dx * s->g.dy) * s->g.dz;
  double Vphi = V * q->phi;
  double so = 1.0 - sw;
  M[0] = (Vphi * q->rho[0]) * so;
  M[1] = (Vphi * q->rho[1]) * sw;
  dM[0] = (V * ((q->dphi * q->rho[0]) + (q->phi * q->drho[0]))) * so;
  dM[1] = -(Vphi * q->rho[0]);
  dM[2] = (V * ((q->dphi * q->rho[1]) + (q->phi * q->drho[1]))) * sw;
  dM[3] = Vphi * q->rho[1];
  (void)c;
}

/* Mass flux from a to b (a < b) of each phase, F = T (rho lambda)_up dPhi
 * with dPhi = p_alpha,a - p_alpha,b - rho_avg g (z_a - z_b), the phase
 * pressures p_o = p and p_w = p - p_cow(s_w); upstream a when dPhi >= 0.
 * dFa, dFb: derivatives with respect to (p, sw) of a and of b, laid out as
 * [phase][variable]. */
static void flux(double T, double gdz, double pa, double pb,
                 const og_props *qa, const og_props *qb, int cap,
                 double F[2], double dFa[4], double dFb[4]) {
  for (int al = 0; al < 2; ++al) {
    int capw = cap && al == 1;                  /* water with a p_cow table */
    double ppa = capw ? pa - qa->pc : pa;       /* phase pressures */
    double ppb = capw ? pb - qb->pc : pb;
    double dpot = (ppa - ppb) - ((0.5 * (qa->rho[al] + qb->rho[al])) * gdz);
    double ddpa = 1.0 - ((0.5 * qa->drho[al]) * gdz);
    double ddpb = -1.0 - ((0.5 * qb->drho[al]) * gdz);
    double mob, mpa, msa, mpb, msb;
    if (dpot >= 0.0) {
      mob = qa->rho[al] * qa->lam[al];
      mpa = qa->drho[al] * qa->lam[al]; msa = qa->rho[al] * qa->dlam[al];
      mpb = 0.0; msb = 0.0;
    } else {
      mob = qb->rho[al] * qb->lam[al];
      mpb = qb->drho[al] * qb->lam[al]; msb = qb->rho[al] * qb->dlam[al];
      mpa = 0.0; msa = 0.0;
    }
    F[al] = (T * mob) * dpot;
    dFa[2 * al + 0] = T * ((mpa * dpot) + (mob * ddpa));
    dFb[2 * al + 0] = T * ((mpb * dpot) + (mob * ddpb));
    if (capw) {   /* dPhi_w/ds_w,a = -p_cow'(s_w,a), dPhi_w/ds_w,b = +p_cow'(s_w,b) */
      dFa[2 * al + 1] = T * ((msa * dpot) - (mob * qa->dpc));
      dFb[2 * al + 1] = T * ((msb * dpot) + (mob * qb->dpc));
    } else {
      dFa[2 * al + 1] = T * (msa * dpot);
      dFb[2 * al + 1] = T * (msb * dpot);
    }
  }
}

/* Perforation mass rate into the cell (Section 2, q_{alpha,i}):
 * producer q = WI rho lambda (p_b - p); water injector q_w = WI rho_w
 * lambda_t (p_b - p), q_o = 0.  dq: [phase][d/dp, d/dsw], dqb: d/dp_b. */
static void perf_rate(int kind, double wi, double pc, double pb, const og_props *q,
                      double Q[2], double dq[4], double dqb[2]) {
  double dpw = pb - pc;
  if (kind == 0) {
    double lt = q->lam[0] + q->lam[1], dlt = q->dlam[0] + q->dlam[1];
    Q[0] = 0.0; dq[0] = 0.0; dq[1] = 0.0; dqb[0] = 0.0;
    Q[1] = ((wi * q->rho[1]) * lt) * dpw;
    dq[2] = (((wi * q->drho[1]) * lt) * dpw) - ((wi * q->rho[1]) * lt);
    dq[3] = ((wi * q->rho[1]) * dlt) * dpw;
    dqb[1] = (wi * q->rho[1]) * lt;
  } else {
    for (int al = 0; al < 2; ++al) {
      Q[al] = ((wi * q->rho[al]) * q->lam[al]) * dpw;
      dq[2 * al + 0] = (((wi * q->drho[al]) * q->lam[al]) * dpw) - ((wi * q->rho[al]) * q->lam[al]);
      dq[2 * al + 1] = ((wi * q->rho[al]) * q->dlam[al]) * dpw;
      dqb[al] = (wi * q->rho[al]) * q->lam[al];
    }
  }
}

static int perf_of(const og_sim *s, int cell, int well) {
  for (int t = 0; t < s->nperf; ++t)
    if (s->perf[t].cell == cell && s->perf[t].well == well) return t;
  return -1;
}

/* Residual R and Jacobian J at the current iterate (Eq. "prob" discretised
 * by backward Euler and two-point fluxes; Eq. "nonlinear").  Cell rows:
 *   R_c = (M_c - M_c^n)/dt + sum over neighbours d of F(c -> d) - q_c,
 * the sum taken in increasing d (well columns last); well rows: the rate
 * constraint sum WI lambda_t (p_b - p) - Q = 0 of a water injector or
 * p_b - p_target = 0 of a BHP well, padded with a dummy unknown. */
static void assemble(og_sim *s) {
  og_bsr *J = &s->J;
  memset(J->val, 0, sizeof(double) * 4 * (size_t)J->nnz);
  for (int c = 0; c < s->nc; ++c) {
    og_props qc;
    props(s, c, s->p[c], s->sw[c], &qc);
    double M[2], dM[4];
    accumulation(s, c, s->sw[c], &qc, M, dM);
    double r0 = (M[0] - s->Mn[2 * c]) * s->inv_dt;
    double r1 = (M[1] - s->Mn[2 * c + 1]) * s->inv_dt;
    double *dg = J->val + 4 * (size_t)J->diag[c];
    double d0 = dM[0] * s->inv_dt, d1 = dM[1] * s->inv_dt;
    double d2 = dM[2] * s->inv_dt, d3 = dM[3] * s->inv_dt;
    for (int e = J->rowptr[c]; e < J->rowptr[c + 1]; ++e) {
      int d = J->col[e];
      if (d == c) continue;
      double *off = J->val + 4 * (size_t)e;
      if (d < s->nc) {
        og_props qd;
        props(s, d, s->p[d], s->sw[d], &qd);
        double dzab, F[2], dFa[4], dFb[4];
        int a = c < d ? c : d, b = c < d ? d : c;
        double T = conn_trans(s, a, b, &dzab);
        double gdz = s->f.g * dzab;
        if (c < d) {
          flux(T, gdz, s->p[c], s->p[d], &qc, &qd, s->cap, F, dFa, dFb);
          r0 = r0 + F[0]; r1 = r1 + F[1];
          d0 = d0 + dFa[0]; d1 = d1 + dFa[1]; d2 = d2 + dFa[2]; d3 = d3 + dFa[3];
          off[0] = dFb[0]; off[1] = dFb[1]; off[2] = dFb[2]; off[3] = dFb[3];
        } else {
          flux(T, gdz, s->p[d], s->p[c], &qd, &qc, s->cap, F, dFa, dFb);
          r0 = r0 + (-F[0]); r1 = r1 + (-F[1]);
          d0 = d0 + (-dFb[0]); d1 = d1 + (-dFb[1]); d2 = d2 + (-dFb[2]); d3 = d3 + (-dFb[3]);
          off[0] = -dFa[0]; off[1] = -dFa[1]; off[2] = -dFa[2]; off[3] = -dFa[3];
        }
      } else {
        int w = d - s->nc;
        int t = perf_of(s, c, w);
        double Q[2], dq[4], dqb[2];
        perf_rate(s->wells[w].kind, s->perf[t].wi, s->p[c], s->bhp[w], &qc, Q, dq, dqb);
        r0 = r0 - Q[0]; r1 = r1 - Q[1];
        d0 = d0 - dq[0]; d1 = d1 - dq[1]; d2 = d2 - dq[2]; d3 = d3 - dq[3];
        off[0] = -dqb[0]; off[1] = 0.0; off[2] = -dqb[1]; off[3] = 0.0;
      }
    }
    dg[0] = d0; dg[1] = d1; dg[2] = d2; dg[3] = d3;
    s->R[2 * c] = r0; s->R[2 * c + 1] = r1;
  }
  for (int w = 0; w < s->nwells; ++w) {
    int row = s->nc + w;
    double pb = s->bhp[w];
    double *dg = J->val + 4 * (size_t)J->diag[row];
    if (s->wells[w].kind == 0) {
      double acc = 0.0, accd = 0.0;
      for (int e = J->rowptr[row]; e < J->rowptr[row + 1]; ++e) {
        int c = J->col[e];
        if (c == row) continue;
        int t = perf_of(s, c, w);
        og_props q;
        props(s, c, s->p[c], s->sw[c], &q);
        double lt = q.lam[0] + q.lam[1], dlt = q.dlam[0] + q.dlam[1];
        double wl = s->perf[t].wi * lt;
        acc = acc + (wl * (pb - s->p[c]));
        accd = accd + wl;
        double *off = J->val + 4 * (size_t)e;
        off[0] = -wl; off[1] = (s->perf[t].wi * dlt) * (pb - s->p[c]); off[2] = 0.0; off[3] = 0.0;
      }
      s->R[2 * row] = acc - s->wells[w].target;
      dg[0] = accd;
    } else if (s->wells[w].kind == 2) {
      /* oil-rate producer: the oil mass leaving through the perforations
       * (-sum of the perforation rates into the cells) equals the target */
      double acc = 0.0, accd = 0.0;
      for (int e = J->rowptr[row]; e < J->rowptr[row + 1]; ++e) {
        int c = J->col[e];
        if (c == row) continue;
        int t = perf_of(s, c, w);
        og_props q;
        props(s, c, s->p[c], s->sw[c], &q);
        double Q[2], dq[4], dqb[2];
        perf_rate(2, s->perf[t].wi, s->p[c], pb, &q, Q, dq, dqb);
        acc = acc + Q[0];
        accd = accd + dqb[0];
        double *off = J->val + 4 * (size_t)e;
        off[0] = dq[0]; off[1] = dq[1]; off[2] = 0.0; off[3] = 0.0;
      }
      s->R[2 * row] = acc + s->wells[w].target;
      dg[0] = accd;
    } else {
      s->R[2 * row] = pb - s->wells[w].target;
      dg[0] = 1.0;
    }
    dg[1] = 0.0; dg[2] = 0.0; dg[3] = 1.0;
    s->R[2 * row + 1] = 0.0;
  }
}

/* Scaled residual norms (Algorithm 1's ||b||) and mass-balance sums.
 * Cell rows scaled by dt / (rho_ref phi_ref V), well rows by the target.
 * With a linear residual lq of the last solve (forcing terms 1-2), its
 * scaled 2-norm and that of R - lq, in the same scaling. */
static void norms(og_sim *s) {
  double V = (s->g.dx * s->g.dy) * s->g.dz;
  double s2 = 0.0, sinf = 0.0, sro = 0.0, srw = 0.0, dmo = 0.0, dmw = 0.0, wo = 0.0, ww = 0.0;
  double lq2 = 0.0, ld2 = 0.0;
  int lin = s->have_lq && (s->o.eta_mode == 1 || s->o.eta_mode == 2);
  for (int c = 0; c < s->nc; ++c) {
    int loc = c / 2;
    double phi_ref = (c % 2 == 0) ? s->phi_f[loc] : s->phi_m[loc];
    for (int al = 0; al < 2; ++al) {
      double rref = al == 0 ? s->f.rho_o_ref : s->f.rho_w_ref;
      double v = (s->R[2 * c + al] * s->dt) / ((rref * phi_ref) * V);
      s2 += v * v;
      if (fabs(v) > sinf) sinf = fabs(v);
      if (lin) {
        double a = (s->lq[2 * c + al] * s->dt) / ((rref * phi_ref) * V);
        double d = ((s->R[2 * c + al] - s->lq[2 * c + al]) * s->dt) / ((rref * phi_ref) * V);
        lq2 += a * a;
        ld2 += d * d;
      }
    }
    sro += s->R[2 * c]; srw += s->R[2 * c + 1];
    og_props q;
    props(s, c, s->p[c], s->sw[c], &q);
    double M[2], dM[4];
    accumulation(s, c, s->sw[c], &q, M, dM);
    dmo += M[0] - s->Mn[2 * c]; dmw += M[1] - s->Mn[2 * c + 1];
  }
  for (int t = 0; t < s->nperf; ++t) {
    int c = s->perf[t].cell, w = s->perf[t].well;
    og_props q;
    props(s, c, s->p[c], s->sw[c], &q);
    double Q[2], dq[4], dqb[2];
    perf_rate(s->wells[w].kind, s->perf[t].wi, s->p[c], s->bhp[w], &q, Q, dq, dqb);
    wo += Q[0]; ww += Q[1];
  }
  for (int w = 0; w < s->nwells; ++w) {
    double sc = s->wells[w].kind == 0 ? fmax(s->wells[w].target, 1e-12) : s->wells[w].target;
    int row = 2 * (s->nc + w);
    double v = s->R[row] / sc;
    s2 += v * v;
    if (fabs(v) > sinf) sinf = fabs(v);
    if (lin) {
      double a = s->lq[row] / sc, d = (s->R[row] - s->lq[row]) / sc;
      lq2 += a * a;
      ld2 += d * d;
    }
  }
  s->lin_norms[0] = sqrt(lq2); s->lin_norms[1] = sqrt(ld2);
  s->norms[0] = sqrt(s2); s->norms[1] = sinf;
  s->norms[2] = sro; s->norms[3] = srw;
  s->norms[4] = dmo; s->norms[5] = dmw; s->norms[6] = wo; s->norms[7] = ww;
}

static void save_old(og_sim *s) {
  memcpy(s->pn, s->p, sizeof(double) * (size_t)s->nc);
  memcpy(s->swn, s->sw, sizeof(double) * (size_t)s->nc);
  memcpy(s->bhpn, s->bhp, sizeof(double) * (size_t)s->nwells);
  for (int c = 0; c < s->nc; ++c) {
    og_props q;
    props(s, c, s->p[c], s->sw[c], &q);
    double M[2], dM[4];
    accumulation(s, c, s->sw[c], &q, M, dM);
    s->Mn[2 * c] = M[0]; s->Mn[2 * c + 1] = M[1];
  }
}

/* ------------------------------------------------------------------ */
/* Exact elimination of the matrix continuum (schur = 1).  A matrix cell m
 * of location loc couples only to itself and its fracture cell f (Section 2:
 * the matrix exchanges fluid with its own fracture only), so from
 *   A_mm y_m + A_mf y_f = -R_m
 * y_m = A_mm^-1 (-R_m - A_mf y_f), and the fracture row becomes
 *   (A_ff - A_fm A_mm^-1 A_mf) y_f + sum_j A_fj y_j = -(R_f - A_fm A_mm^-1 R_m).
 * The fracture-and-well system K keeps the fracture rows (row loc) and the
 * well rows (row nL + w); its blocks are those of J except the fracture
 * diagonal blocks, which take S_ff. */

static const og_bsr *solver_op(const og_sim *s) { return s->o.schur ? &s->K : &s->J; }

static int kcol(const og_sim *s, int c) {        /* column of J -> column of K, -1: dropped */
  if (c >= s->nc) return s->nL + (c - s->nc);
  return (c & 1) ? -1 : c >> 1;
}

static void schur_pattern(og_sim *s) {
  og_bsr *J = &s->J, *K = &s->K;
  int nk = s->nL + s->nwells;
  K->n = nk;
  K->rowptr = (int *)zalloc((size_t)nk + 1, sizeof(int));
  int cnt = 0;
  for (int r = 0; r < nk; ++r) {
    int jr = r < s->nL ? 2 * r : s->nc + (r - s->nL);
    K->rowptr[r] = cnt;
    for (int e = J->rowptr[jr]; e < J->rowptr[jr + 1]; ++e) if (kcol(s, J->col[e]) >= 0) ++cnt;
  }
  K->rowptr[nk] = cnt;
  K->nnz = cnt;
  K->col = (int *)zalloc((size_t)cnt, sizeof(int));
  K->diag = (int *)zalloc((size_t)nk, sizeof(int));
  K->val = (double *)zalloc(4 * (size_t)cnt, sizeof(double));
  s->kmap = (int *)zalloc((size_t)cnt, sizeof(int));
  for (int r = 0; r < nk; ++r) {
    int jr = r < s->nL ? 2 * r : s->nc + (r - s->nL), k = K->rowptr[r];
    for (int e = J->rowptr[jr]; e < J->rowptr[jr + 1]; ++e) {
      int c = kcol(s, J->col[e]);
      if (c < 0) continue;
      K->col[k] = c;
      s->kmap[k] = (r < s->nL && c == r) ? -1 : e;
      if (c == r) K->diag[r] = k;
      ++k;
    }
  }
  s->pos_fm = (int *)zalloc((size_t)s->nL, sizeof(int));
  s->pos_mf = (int *)zalloc((size_t)s->nL, sizeof(int));
  for (int loc = 0; loc < s->nL; ++loc) {
    int f = 2 * loc, m = f + 1;
    s->pos_fm[loc] = find_col(J->col, J->rowptr[f], J->rowptr[f + 1], m);
    s->pos_mf[loc] = find_col(J->col, J->rowptr[m], J->rowptr[m + 1], f);
  }
  s->Minv = (double *)zalloc(4 * (size_t)s->nL, sizeof(double));
  s->RK = (double *)zalloc(2 * (size_t)nk, sizeof(double));
  s->yk = (double *)zalloc(2 * (size_t)nk, sizeof(double));
}

static void schur_reduce(og_sim *s) {
  og_bsr *J = &s->J, *K = &s->K;
  for (int k = 0; k < K->nnz; ++k)
    if (s->kmap[k] >= 0) memcpy(K->val + 4 * (size_t)k, J->val + 4 * (size_t)s->kmap[k], 32);
  for (int w = 0; w < s->nwells; ++w) {
    s->RK[2 * (s->nL + w)] = s->R[2 * (s->nc + w)];
    s->RK[2 * (s->nL + w) + 1] = s->R[2 * (s->nc + w) + 1];
  }
  for (int loc = 0; loc < s->nL; ++loc) {
    int f = 2 * loc, m = f + 1;
    const double *amm = J->val + 4 * (size_t)J->diag[m];
    const double *amf = J->val + 4 * (size_t)s->pos_mf[loc];
    const double *afm = J->val + 4 * (size_t)s->pos_fm[loc];
    const double *aff = J->val + 4 * (size_t)J->diag[f];
    double det = (amm[0] * amm[3]) - (amm[1] * amm[2]);
    double *mi = s->Minv + 4 * (size_t)loc;
    if (fabs(det) < 1e-300) { mi[0] = 0.0; mi[1] = 0.0; mi[2] = 0.0; mi[3] = 0.0; }
    else {
      mi[0] = amm[3] / det; mi[1] = (-amm[1]) / det;
      mi[2] = (-amm[2]) / det; mi[3] = amm[0] / det;
    }
    double x00 = (afm[0] * mi[0]) + (afm[1] * mi[2]);
    double x01 = (afm[0] * mi[1]) + (afm[1] * mi[3]);
    double x10 = (afm[2] * mi[0]) + (afm[3] * mi[2]);
    double x11 = (afm[2] * mi[1]) + (afm[3] * mi[3]);
    double *sk = K->val + 4 * (size_t)K->diag[loc];
    sk[0] = aff[0] - ((x00 * amf[0]) + (x01 * amf[2]));
    sk[1] = aff[1] - ((x00 * amf[1]) + (x01 * amf[3]));
    sk[2] = aff[2] - ((x10 * amf[0]) + (x11 * amf[2]));
    sk[3] = aff[3] - ((x10 * amf[1]) + (x11 * amf[3]));
    double rm0 = s->R[2 * m], rm1 = s->R[2 * m + 1];
    s->RK[2 * loc] = s->R[2 * f] - ((x00 * rm0) + (x01 * rm1));
    s->RK[2 * loc + 1] = s->R[2 * f + 1] - ((x10 * rm0) + (x11 * rm1));
  }
}

/* y of the full system from the fracture-and-well update yk. */
static void schur_back(og_sim *s) {
  const og_bsr *J = &s->J;
  for (int w = 0; w < s->nwells; ++w) {
    s->y[2 * (s->nc + w)] = s->yk[2 * (s->nL + w)];
    s->y[2 * (s->nc + w) + 1] = s->yk[2 * (s->nL + w) + 1];
  }
  for (int loc = 0; loc < s->nL; ++loc) {
    int f = 2 * loc, m = f + 1;
    double yf0 = s->yk[2 * loc], yf1 = s->yk[2 * loc + 1];
    const double *amf = J->val + 4 * (size_t)s->pos_mf[loc];
    const double *mi = s->Minv + 4 * (size_t)loc;
    double t0 = (-s->R[2 * m]) - ((amf[0] * yf0) + (amf[1] * yf1));
    double t1 = (-s->R[2 * m + 1]) - ((amf[2] * yf0) + (amf[3] * yf1));
    s->y[2 * f] = yf0;
    s->y[2 * f + 1] = yf1;
    s->y[2 * m] = (mi[0] * t0) + (mi[1] * t1);
    s->y[2 * m + 1] = (mi[2] * t0) + (mi[3] * t1);
  }
}

int oracle_create(const og_grid *g, const og_rock *r, const og_fluid *f,
                  const og_well *w, int32_t nwells, const og_options *o, void **out) {
  if (!g || !r || !f || !o || !out || g->nx < 1 || g->ny < 1 || g->nz < 1 || nwells < 0)
    return OG_EINVAL;
  for (int k = 0; k < 2; ++k) {
    if (f->pc_n[k] < 0 || f->pc_n[k] > 256 || (f->pc_n[k] > 0 && !f->pc_table[k])) return OG_EINVAL;
    for (int i = 0; i < f->pc_n[k]; ++i) {
      if (!isfinite(f->pc_table[k][2 * i]) || !isfinite(f->pc_table[k][2 * i + 1])) return OG_EINVAL;
      if (i > 0 && !(f->pc_table[k][2 * i] > f->pc_table[k][2 * i - 2])) return OG_EINVAL;
    }
  }
  og_sim *s = (og_sim *)zalloc(1, sizeof(og_sim));
  s->g = *g; s->f = *f; s->o = *o;
  for (int k = 0; k < 2; ++k) {
    s->pc_own[k] = (double *)zalloc((size_t)(2 * f->pc_n[k] + 1), sizeof(double));
    if (f->pc_n[k]) memcpy(s->pc_own[k], f->pc_table[k], sizeof(double) * 2 * (size_t)f->pc_n[k]);
    s->f.pc_table[k] = s->pc_own[k];
    if (f->pc_n[k]) s->cap = 1;
  }
  s->sigma = r->sigma; s->c_rock = r->c_rock; s->p_ref_rock = r->p_ref;
  s->nL = g->nx * g->ny * g->nz;
  s->nc = 2 * s->nL;
  s->nwells = nwells;
  s->nb = s->nc + nwells;
  s->kf = (double *)zalloc((size_t)s->nL, sizeof(double));
  s->km = (double *)zalloc((size_t)s->nL, sizeof(double));
  s->phi_f = (double *)zalloc((size_t)s->nL, sizeof(double));
  s->phi_m = (double *)zalloc((size_t)s->nL, sizeof(double));
  memcpy(s->kf, r->kf, sizeof(double) * (size_t)s->nL);
  memcpy(s->km, r->km, sizeof(double) * (size_t)s->nL);
  memcpy(s->phi_f, r->phi_f, sizeof(double) * (size_t)s->nL);
  memcpy(s->phi_m, r->phi_m, sizeof(double) * (size_t)s->nL);
  s->wells = (og_well *)zalloc((size_t)nwells, sizeof(og_well));
  if (nwells) memcpy(s->wells, w, sizeof(og_well) * (size_t)nwells);
  s->ctl_kind = (int *)zalloc((size_t)nwells, sizeof(int));
  s->ctl_target = (double *)zalloc((size_t)nwells, sizeof(double));
  for (int q = 0; q < nwells; ++q) { s->ctl_kind[q] = w[q].kind; s->ctl_target[q] = w[q].target; }
  /* perforations: fracture cells of every layer k_top..k_bot */
  s->nperf = 0;
  for (int q = 0; q < nwells; ++q) {
    const og_well *W = &w[q];
    if (W->i < 0 || W->i >= g->nx || W->j < 0 || W->j >= g->ny || W->k_top < 0 ||
        W->k_bot >= g->nz || W->k_top > W->k_bot || W->rw <= 0.0 || W->kind < 0 || W->kind > 2 ||
        W->limit < 0.0 || W->wi < 0.0) { oracle_destroy(s); return OG_EINVAL; }
    s->nperf += W->k_bot - W->k_top + 1;
  }
  s->perf = (og_perf *)zalloc((size_t)s->nperf, sizeof(og_perf));
  int t = 0;
  for (int q = 0; q < nwells; ++q) {
    const og_well *W = &w[q];
    for (int k = W->k_top; k <= W->k_bot; ++k) {
      int loc = W->i + g->nx * (W->j + g->ny * k);
      s->perf[t].cell = 2 * loc;
      s->perf[t].well = q;
      s->perf[t].wi = W->wi > 0.0 ? W->wi
                                  : well_index(s->kf[loc], s->kf[loc], g->dx, g->dy, g->dz, W->rw, W->skin);
      ++t;
    }
  }
  /* block pattern: per row the connected cells and wells, sorted */
  og_bsr *J = &s->J;
  J->n = s->nb;
  J->rowptr = (int *)zalloc((size_t)s->nb + 1, sizeof(int));
  int cap = 9 * s->nc + 2 * s->nperf + s->nb + 16;
  J->col = (int *)zalloc((size_t)cap, sizeof(int));
  int e = 0, nxy = g->nx * g->ny;
  for (int c = 0; c < s->nc; ++c) {
    int loc = c / 2, i, j, k;
    cell_ijk(s, loc, &i, &j, &k);
    J->rowptr[c] = e;
    int start = e;
    J->col[e++] = c;
    if (c % 2 == 0) {
      J->col[e++] = c + 1;
      if (k > 0) J->col[e++] = 2 * (loc - nxy);
      if (j > 0) J->col[e++] = 2 * (loc - g->nx);
      if (i > 0) J->col[e++] = 2 * (loc - 1);
      if (i < g->nx - 1) J->col[e++] = 2 * (loc + 1);
      if (j < g->ny - 1) J->col[e++] = 2 * (loc + g->nx);
      if (k < g->nz - 1) J->col[e++] = 2 * (loc + nxy);
      for (int q = 0; q < s->nperf; ++q)
        if (s->perf[q].cell == c) J->col[e++] = s->nc + s->perf[q].well;
    } else {
      J->col[e++] = c - 1;
    }
    sort_int(J->col + start, e - start);
  }
  for (int q = 0; q < nwells; ++q) {
    int row = s->nc + q;
    J->rowptr[row] = e;
    int start = e;
    J->col[e++] = row;
    for (int p = 0; p < s->nperf; ++p) if (s->perf[p].well == q) J->col[e++] = s->perf[p].cell;
    sort_int(J->col + start, e - start);
  }
  J->rowptr[s->nb] = e;
  J->nnz = e;
  J->diag = (int *)zalloc((size_t)s->nb, sizeof(int));
  for (int row = 0; row < s->nb; ++row) J->diag[row] = find_col(J->col, J->rowptr[row], J->rowptr[row + 1], row);
  J->val = (double *)zalloc(4 * (size_t)e, sizeof(double));
  s->R = (double *)zalloc(2 * (size_t)s->nb, sizeof(double));
  s->p = (double *)zalloc((size_t)s->nc, sizeof(double));
  s->sw = (double *)zalloc((size_t)s->nc, sizeof(double));
  s->bhp = (double *)zalloc((size_t)nwells, sizeof(double));
  s->pn = (double *)zalloc((size_t)s->nc, sizeof(double));
  s->swn = (double *)zalloc((size_t)s->nc, sizeof(double));
  s->bhpn = (double *)zalloc((size_t)nwells, sizeof(double));
  s->Mn = (double *)zalloc(2 * (size_t)s->nc, sizeof(double));
  s->y = (double *)zalloc(2 * (size_t)s->nb, sizeof(double));
  s->bh = (double *)zalloc(2 * (size_t)s->nb, sizeof(double));
  if (o->schur) schur_pattern(s);
  const og_bsr *A = solver_op(s);
  s->colour = (int *)zalloc((size_t)A->n, sizeof(int));
  s->ncolour = greedy_colour(A->n, A->rowptr, A->col, s->colour);
  ilu_setup(&s->ilu, A, s->colour);
  s->Ap.n = A->n; s->Ap.ncol = A->n; s->Ap.nnz = A->nnz;
  s->Ap.rowptr = A->rowptr; s->Ap.col = A->col;
  s->Ap.val = (double *)zalloc((size_t)A->nnz, sizeof(double));
  s->amg.theta = o->amg_theta; s->amg.coarse_max = o->amg_coarse_max;
  s->amg.smoother = o->amg_gs_levels;
  s->amg.max_levels = o->amg_max_levels > 30 ? 30 : o->amg_max_levels;
  s->dt = 1.0; s->inv_dt = 1.0;
  *out = s;
  return OG_OK;
}

void oracle_destroy(void *h) {
  og_sim *s = (og_sim *)h;
  if (!s) return;
  free(s->kf); free(s->km); free(s->phi_f); free(s->phi_m); free(s->wells); free(s->perf);
  free(s->ctl_kind); free(s->ctl_target); free(s->pc_own[0]); free(s->pc_own[1]);
  free(s->J.rowptr); free(s->J.col); free(s->J.diag); free(s->J.val);
  free(s->Ja); free(s->lq);
  free(s->R); free(s->p); free(s->sw); free(s->bhp); free(s->pn); free(s->swn); free(s->bhpn);
  free(s->Mn); free(s->y); free(s->bh); free(s->colour); free(s->Ap.val);
  if (s->o.schur) {
    free(s->K.rowptr); free(s->K.col); free(s->K.diag); free(s->K.val);
    free(s->RK); free(s->yk); free(s->kmap); free(s->pos_fm); free(s->pos_mf); free(s->Minv);
  }
  ilu_free(&s->ilu);
  amg_free(&s->amg);
  free(s);
}

int oracle_sizes(void *h, int32_t *nb, int32_t *nnzb) {
  og_sim *s = (og_sim *)h;
  *nb = s->nb; *nnzb = s->J.nnz;
  return 0;
}

int oracle_well_controls(void *h, int32_t *kind, double *target) {
  og_sim *s = (og_sim *)h;
  for (int w = 0; w < s->nwells; ++w) { kind[w] = s->wells[w].kind; target[w] = s->wells[w].target; }
  return s->nwells;
}

/* The perforation rates of Section 2 (WI rho_alpha lambda_alpha (p_b - p)
 * for a producer, WI rho_w lambda_t (p_b - p) for a water injector), summed
 * per well over its perforations from the top layer down. */
int oracle_well_rates(void *h, double *q_oil, double *q_water) {
  og_sim *s = (og_sim *)h;
  for (int w = 0; w < s->nwells; ++w) {
    double qo = 0.0, qw = 0.0;
    for (int t = 0; t < s->nperf; ++t) {
      if (s->perf[t].well != w) continue;
      int c = s->perf[t].cell;
      og_props q;
      props(s, c, s->p[c], s->sw[c], &q);
      double Q[2], dq[4], dqb[2];
      perf_rate(s->wells[w].kind, s->perf[t].wi, s->p[c], s->bhp[w], &q, Q, dq, dqb);
      qo = qo + Q[0];
      qw = qw + Q[1];
    }
    q_oil[w] = qo;
    q_water[w] = qw;
  }
  return s->nwells;
}

void oracle_cap_pressure(int32_t n, const double *table, double sw, double *pc, double *dpc) {
  cap_pressure(n, table, sw, pc, dpc);
}

int oracle_solver_sizes(void *h, int32_t *nb, int32_t *nnzb) {
  og_sim *s = (og_sim *)h;
  const og_bsr *A = solver_op(s);
  *nb = A->n; *nnzb = A->nnz;
  return 0;
}

int oracle_set_iterate(void *h, const double *p, const double *sw, const double *bhp) {
  og_sim *s = (og_sim *)h;
  memcpy(s->p, p, sizeof(double) * (size_t)s->nc);
  memcpy(s->sw, sw, sizeof(double) * (size_t)s->nc);
  if (s->nwells) memcpy(s->bhp, bhp, sizeof(double) * (size_t)s->nwells);
  return 0;
}

int oracle_set_state(void *h, const double *p, const double *sw, const double *bhp) {
  og_sim *s = (og_sim *)h;
  oracle_set_iterate(h, p, sw, bhp);
  save_old(s);
  s->newton_iter = 0;            /* a new old time level starts a new timestep */
  s->prev_res = 0.0; s->have_lq = 0;
  return 0;
}

int oracle_get_state(void *h, double *p, double *sw, double *bhp) {
  og_sim *s = (og_sim *)h;
  memcpy(p, s->p, sizeof(double) * (size_t)s->nc);
  memcpy(sw, s->sw, sizeof(double) * (size_t)s->nc);
  if (s->nwells) memcpy(bhp, s->bhp, sizeof(double) * (size_t)s->nwells);
  return 0;
}

int oracle_assemble(void *h, double dt) {
  og_sim *s = (og_sim *)h;
  if (!(dt > 0.0)) return OG_EINVAL;
  s->dt = dt;
  s->inv_dt = 1.0 / dt;
  assemble(s);
  norms(s);
  return 0;
}

int oracle_get_jacobian(void *h, int32_t *rowptr, int32_t *col, double *val, double *res) {
  og_sim *s = (og_sim *)h;
  if (rowptr) memcpy(rowptr, s->J.rowptr, sizeof(int) * ((size_t)s->nb + 1));
  if (col) memcpy(col, s->J.col, sizeof(int) * (size_t)s->J.nnz);
  if (val) memcpy(val, s->J.val, sizeof(double) * 4 * (size_t)s->J.nnz);
  if (res) memcpy(res, s->R, sizeof(double) * 2 * (size_t)s->nb);
  return 0;
}

int oracle_get_norms(void *h, double *out8) {
  memcpy(out8, ((og_sim *)h)->norms, 8 * sizeof(double));
  return 0;
}

int oracle_well_index(void *h, double *wi) {
  og_sim *s = (og_sim *)h;
  for (int t = 0; t < s->nperf; ++t) wi[t] = s->perf[t].wi;
  return s->nperf;
}

/* Decoupling by one Gauss-Jordan step per block row (the paper's "modified
 * Gauss-Jordan elimination", Eq. "decoupled-eq"): the water row of the
 * diagonal block is the pivot that removes the saturation coefficient from
 * the oil row, D_i^-1 = [[1, -a01/a11], [0, 1]], applied to the whole block
 * row and to the right-hand side b = -R.  Well rows are left as they are. */
/* Decoupling D^-1 A x = D^-1 b (Section 3.2, Eq. "decoupled-eq") per cell
 * block row; well rows unchanged.  decouple 0: the modified Gauss-Jordan step
 * of the paper read as the elimination of the pressure row's saturation
 * coefficient by the water row of the diagonal block, D_i^-1 = [[1, -w_i],
 * [0, 1]] with w_i = a01/a11 (the per-cell Quasi-IMPES form); 1: ABF
 * (alternate block factorisation), D_i = the diagonal block; 2: True-IMPES,
 * w_i = c01/c11 from the sums of block column i over all rows (taken before
 * any row changes, rows in increasing order). */
static void decouple(og_sim *s) {
  og_bsr *J = s->o.schur ? &s->K : &s->J;              /* the system the solver sees */
  const double *R = s->o.schur ? s->RK : s->R;
  int nb = J->n, ncell = s->o.schur ? s->nL : s->nc;    /* rows below ncell are cell rows */
  int mode = s->o.decouple;
  double *w = NULL;
  if (mode == 2) {
    double *c01 = (double *)zalloc((size_t)ncell, sizeof(double));
    double *c11 = (double *)zalloc((size_t)ncell, sizeof(double));
    for (int k = 0; k < nb; ++k)
      for (int e = J->rowptr[k]; e < J->rowptr[k + 1]; ++e) {
        int j = J->col[e];
        if (j >= ncell) continue;
        const double *a = J->val + 4 * (size_t)e;
        c01[j] = c01[j] + a[1];
        c11[j] = c11[j] + a[3];
      }
    w = (double *)zalloc((size_t)ncell, sizeof(double));
    for (int j = 0; j < ncell; ++j) w[j] = fabs(c11[j]) < 1e-300 ? 0.0 : c01[j] / c11[j];
    free(c01);
    free(c11);
  }
  for (int i = 0; i < nb; ++i) {
    double b0 = -R[2 * i], b1 = -R[2 * i + 1];
    if (i >= ncell) { s->bh[2 * i] = b0; s->bh[2 * i + 1] = b1; continue; }
    const double *dg = J->val + 4 * (size_t)J->diag[i];
    if (mode == 1) {
      double d00 = dg[0], d01 = dg[1], d10 = dg[2], d11 = dg[3];
      double det = (d00 * d11) - (d01 * d10);
      if (fabs(det) < 1e-300) { s->bh[2 * i] = b0; s->bh[2 * i + 1] = b1; continue; }
      double i00 = d11 / det, i01 = (-d01) / det, i10 = (-d10) / det, i11 = d00 / det;
      for (int e = J->rowptr[i]; e < J->rowptr[i + 1]; ++e) {
        double *a = J->val + 4 * (size_t)e;
        double v0 = a[0], v1 = a[1], v2 = a[2], v3 = a[3];
        a[0] = (i00 * v0) + (i01 * v2);
        a[1] = (i00 * v1) + (i01 * v3);
        a[2] = (i10 * v0) + (i11 * v2);
        a[3] = (i10 * v1) + (i11 * v3);
      }
      s->bh[2 * i] = (i00 * b0) + (i01 * b1);
      s->bh[2 * i + 1] = (i10 * b0) + (i11 * b1);
      continue;
    }
    double fct;
    if (mode == 2) fct = w[i];
    else {
      double a01 = dg[1], a11 = dg[3];
      fct = fabs(a11) < 1e-300 ? 0.0 : a01 / a11;
    }
    for (int e = J->rowptr[i]; e < J->rowptr[i + 1]; ++e) {
      double *a = J->val + 4 * (size_t)e;
      a[0] = a[0] - (fct * a[2]);
      a[1] = a[1] - (fct * a[3]);
    }
    s->bh[2 * i] = b0 - (fct * b1);
    s->bh[2 * i + 1] = b1;
  }
  free(w);
}

int oracle_get_decoupled(void *h, double *val, double *rhs) {
  og_sim *s = (og_sim *)h;
  const og_bsr *A = solver_op(s);
  if (val) memcpy(val, A->val, sizeof(double) * 4 * (size_t)A->nnz);
  if (rhs) memcpy(rhs, s->bh, sizeof(double) * 2 * (size_t)A->n);
  return 0;
}

int oracle_get_colours(void *h, int32_t *colour) {
  og_sim *s = (og_sim *)h;
  memcpy(colour, s->colour, sizeof(int) * (size_t)solver_op(s)->n);
  return s->ncolour;
}

int oracle_amg_level_info(void *h, int32_t level, int32_t *n, int32_t *nnz, int32_t *nagg) {
  og_sim *s = (og_sim *)h;
  if (!s->amg_ready) return OG_EINVAL;
  return oracle_amg_info(&s->amg, level, n, nnz, nagg);
}

int oracle_amg_level_arrays(void *h, int32_t level, int32_t *rowptr, int32_t *col,
                            double *val, int32_t *agg, int32_t *colour) {
  og_sim *s = (og_sim *)h;
  if (!s->amg_ready) return OG_EINVAL;
  return oracle_amg_arrays(&s->amg, level, rowptr, col, val, agg, colour);
}

/* Forcing term eta_l of Algorithm 1 (Section 3.1).  Choice 0 is a fixed
 * eta; choices 1-3 are the three formulas given, clipped to
 * [eta_min, eta_max]; the first Newton iteration uses eta_max.  With the
 * right-hand side b = -R and the linear residual r^{l-1} = b(x^{l-1}) -
 * A y^{l-1} = -lq of the previous solve, in the scaled norm of ||b||:
 *   1: ||b(x^l) - r^{l-1}|| / ||b(x^{l-1})|| = ||R~(R - lq)|| / prev_res,
 *   2: (||b(x^l)|| - ||r^{l-1}||) / ||b(x^{l-1})|| = (res - ||R~(lq)||) / prev_res,
 *   3: gamma (||b(x^l)|| / ||b(x^{l-1})||)^beta. */
static double forcing(og_sim *s, double res) {
  const og_options *o = &s->o;
  if (o->eta_mode == 0) return o->eta_fixed;
  if (s->newton_iter == 0 || s->prev_res <= 0.0) return o->eta_max;
  double eta;
  if (o->eta_mode == 1) eta = s->lin_norms[1] / s->prev_res;
  else if (o->eta_mode == 2) eta = (res - s->lin_norms[0]) / s->prev_res;
  else eta = o->eta_gamma * pow(res / s->prev_res, o->eta_beta);
  if (eta < o->eta_min) eta = o->eta_min;
  if (eta > o->eta_max) eta = o->eta_max;
  return eta;
}

/* lq = R + J y over the full system, J as assembled (the linear residual of
 * the Newton equation J y = -R, up to its sign). */
static void linear_residual(og_sim *s) {
  const double *jv = s->o.schur ? s->J.val : s->Ja;
  for (int i = 0; i < s->nb; ++i) {
    double a0 = s->R[2 * i], a1 = s->R[2 * i + 1];
    for (int e = s->J.rowptr[i]; e < s->J.rowptr[i + 1]; ++e) {
      const double *b = jv + 4 * (size_t)e;
      int j = s->J.col[e];
      a0 += b[0] * s->y[2 * j] + b[1] * s->y[2 * j + 1];
      a1 += b[2] * s->y[2 * j] + b[3] * s->y[2 * j + 1];
    }
    s->lq[2 * i] = a0; s->lq[2 * i + 1] = a1;
  }
}

/* One linear solve of Algorithm 1 at the assembled iterate, and the update
 * x <- x + y with the saturation change limited to +-ds_max and sw kept in
 * [0, 1].  When FGMRES does not reach its tolerance no update is made (the
 * state and the Newton counters stay as they were) and OG_ELINEAR is
 * returned. */
int oracle_solve_step(void *h, og_stats *st) {
  og_sim *s = (og_sim *)h;
  double eta = forcing(s, s->norms[0]);
  int lin = s->o.eta_mode == 1 || s->o.eta_mode == 2;
  if (lin && !s->o.schur) {
    if (!s->Ja) s->Ja = (double *)zalloc(4 * (size_t)s->J.nnz, sizeof(double));
    memcpy(s->Ja, s->J.val, sizeof(double) * 4 * (size_t)s->J.nnz);
  }
  if (s->o.schur) schur_reduce(s);
  og_bsr *A = s->o.schur ? &s->K : &s->J;
  decouple(s);
  for (int e = 0; e < A->nnz; ++e) s->Ap.val[e] = A->val[4 * (size_t)e];
  if (s->o.precond >= 1) ilu_factor(&s->ilu, A);
  if (s->o.precond == 2) {
    if (!s->amg_ready) { amg_setup(&s->amg, &s->Ap); s->amg_ready = 1; }
    else amg_refresh(&s->amg, s->Ap.val, s->o.amg_refresh == 0 || s->newton_iter == 0);
  }
  og_cpr c; memset(&c, 0, sizeof(c));
  c.A = A; c.ilu = &s->ilu; c.amg = &s->amg; c.mode = s->o.precond;
  int n2 = 2 * A->n;
  c.r1 = (double *)zalloc((size_t)n2, sizeof(double));
  c.z1 = (double *)zalloc((size_t)n2, sizeof(double));
  c.rp = (double *)zalloc((size_t)A->n, sizeof(double));
  c.xp = (double *)zalloc((size_t)A->n, sizeof(double));
  int it = 0; double rr = 0.0;
  double *ys = s->o.schur ? s->yk : s->y;
  int rc = fgmres(n2, op_bsr, A, s->o.precond ? op_cpr : NULL, &c, s->bh, ys,
                  s->o.gmres_restart, s->o.gmres_maxit, eta, s->o.reorth, &it, &rr);
  free(c.r1); free(c.z1); free(c.rp); free(c.xp);
  if (st) {
    st->linear_iters = it; st->lin_relres = rr; st->eta = eta;
    st->amg_levels = s->amg.nlev; st->converged = rc == 0;
  }
  if (rc != 0) return OG_ELINEAR;
  if (s->o.schur) schur_back(s);
  if (lin) {
    if (!s->lq) s->lq = (double *)zalloc(2 * (size_t)s->nb, sizeof(double));
    linear_residual(s);
    s->have_lq = 1;
  }
  for (int cc = 0; cc < s->nc; ++cc) {
    s->p[cc] += s->y[2 * cc];
    double ds = s->y[2 * cc + 1];
    if (ds > s->o.ds_max) ds = s->o.ds_max;
    if (ds < -s->o.ds_max) ds = -s->o.ds_max;
    double v = s->sw[cc] + ds;
    if (v < 0.0) v = 0.0;
    if (v > 1.0) v = 1.0;
    s->sw[cc] = v;
  }
  for (int w = 0; w < s->nwells; ++w) s->bhp[w] += s->y[2 * (s->nc + w)];
  s->prev_res = s->norms[0];
  s->newton_iter++;
  return OG_OK;
}

int oracle_get_update(void *h, double *y) {
  og_sim *s = (og_sim *)h;
  memcpy(y, s->y, sizeof(double) * 2 * (size_t)s->nb);
  return 0;
}

/* Well controls (the examples' wells have rate targets and BHP limits): a
 * timestep starts with every well on its own control; after a Newton update
 * an injector whose BHP exceeds its limit, or an oil-rate producer whose BHP
 * falls below its limit, switches to BHP control at the limit for the rest
 * of the timestep.  Returns the number of wells switched. */
static int switch_controls(og_sim *s) {
  int n = 0;
  for (int w = 0; w < s->nwells; ++w) {
    og_well *W = &s->wells[w];
    if (W->limit <= 0.0) continue;
    if ((W->kind == 0 && s->bhp[w] > W->limit) || (W->kind == 2 && s->bhp[w] < W->limit)) {
      W->kind = 1;
      W->target = W->limit;
      ++n;
    }
  }
  return n;
}

/* One backward-Euler timestep by Algorithm 1: assemble; stop when
 * ||R~|| <= tol ||R~_0|| or ||R~||_inf <= atol; otherwise solve and update.
 * On failure the state of the old time level is restored: OG_ENEWTON when
 * Newton did not converge, OG_ELINEAR when a linear solve did not reach its
 * forcing term. */
int oracle_advance(void *h, double dt, og_stats *st) {
  og_sim *s = (og_sim *)h;
  for (int w = 0; w < s->nwells; ++w) {
    s->wells[w].kind = s->ctl_kind[w];
    s->wells[w].target = s->ctl_target[w];
  }
  save_old(s);
  s->newton_iter = 0;
  s->prev_res = 0.0; s->have_lq = 0;
  int lin = 0, conv = 0, lin_fail = 0;
  double res0 = 0.0, res = 0.0;
  for (int l = 0; l <= s->o.newton_max; ++l) {
    oracle_assemble(h, dt);
    res = s->norms[0];
    if (l == 0) res0 = res;
    if (res <= s->o.newton_tol * res0 || s->norms[1] <= s->o.newton_atol) { conv = 1; break; }
    if (l == s->o.newton_max) break;
    og_stats ls; memset(&ls, 0, sizeof(ls));
    if (oracle_solve_step(h, &ls) != OG_OK) { lin += ls.linear_iters; lin_fail = 1; break; }
    lin += ls.linear_iters;
    switch_controls(s);
  }
  if (st) {
    st->newton_iters = s->newton_iter; st->linear_iters = lin; st->converged = conv;
    st->res0 = res0; st->res = res; st->amg_levels = s->amg.nlev;
  }
  if (!conv) {
    memcpy(s->p, s->pn, sizeof(double) * (size_t)s->nc);
    memcpy(s->sw, s->swn, sizeof(double) * (size_t)s->nc);
    memcpy(s->bhp, s->bhpn, sizeof(double) * (size_t)s->nwells);
    return lin_fail ? OG_ELINEAR : OG_ENEWTON;
  }
  return OG_OK;
}

/* The time loop of a whole simulation period (the paper's examples run 800
 * and 1600 days): halve a step whose Newton iteration fails, double after a
 * converged one up to dt_max, end exactly at t_end. */
int oracle_run(void *h, double t_end, double dt0, double dt_max, double dt_min,
               int32_t max_steps, og_run_stats *st) {
  og_run_stats r;
  memset(&r, 0, sizeof(r));
  if (!h || !(t_end > 0.0) || !(dt0 > 0.0) || !(dt_max >= dt0) || !(dt_min > 0.0) ||
      max_steps < 1)
    return OG_EINVAL;
  double t = 0.0, dt = dt0;
  int rc = OG_OK;
  while (t_end - t > 1e-9 * t_end) {
    if (r.steps >= max_steps) { rc = OG_ENEWTON; break; }
    double hstep = dt < t_end - t ? dt : t_end - t;
    og_stats a;
    memset(&a, 0, sizeof(a));
    int rc1 = oracle_advance(h, hstep, &a);
    if (rc1 == OG_ENEWTON || rc1 == OG_ELINEAR) {
      r.cuts += 1;
      dt = 0.5 * hstep;
      if (dt < dt_min) { rc = OG_ENEWTON; break; }
      continue;
    }
    if (rc1 != OG_OK) { rc = rc1; break; }
    t = t + hstep;
    r.steps += 1;
    r.newton_iters += a.newton_iters;
    r.linear_iters += a.linear_iters;
    dt = 2.0 * hstep < dt_max ? 2.0 * hstep : dt_max;
  }
  r.t = t;
  if (st) *st = r;
  return rc;
}
