// Physics kernels: block pattern, transmissibilities, residual and Jacobian
// assembly, norms, decoupling, pressure extraction and the Newton update.
//
// Compiled with -fmad=false: every floating-point expression is evaluated
// as written (no fused multiply-add), so that the assembled Jacobian, the
// decoupled matrix and the pressure block are bit-identical to a plain
// sequential CPU evaluation of the same formulas.  The AMG strength graph
// and aggregates are computed from those values and must not depend on the
// processor that evaluated them.
#include <algorithm>
#include <cmath>

#include "dp_internal.h"

namespace dp {

// ---------------------------------------------------------------- physics

// Cell properties (Section 2): linear densities, porosity, Corey relative
// permeabilities of the normalised saturation, mobilities and derivatives.
struct Props {
  double rho[2], drho[2], phi, dphi, lam[2], dlam[2];
  double pc, dpc;   // capillary pressure and slope (set only where a table is given)
};

// Capillary pressure p_cow(s_w) (Section 2: p_w = p_o - p_cow(s_w)) from a
// table of n (s_w, p_cow) pairs: the line through the two points around s_w,
// constant with zero slope at and beyond the end points; zero with no table.
__device__ __forceinline__ void cap_pressure(int n, const double *t, double sw, double &pc,
                                             double &dpc) {
  if (n == 0) { pc = 0.0; dpc = 0.0; return; }
  if (sw <= t[0]) { pc = t[1]; dpc = 0.0; return; }
  if (sw >= t[2 * (n - 1)]) { pc = t[2 * n - 1]; dpc = 0.0; return; }
  int k = 0;
  while (sw >= t[2 * (k + 1)]) ++k;      // t[2k] <= sw < t[2k + 2]
  double ds = t[2 * k + 2] - t[2 * k];
  double dp = t[2 * k + 3] - t[2 * k + 1];
  dpc = dp / ds;
  pc = t[2 * k + 1] + dp * ((sw - t[2 * k]) / ds);
}

__device__ __forceinline__ void props(const Phys &P, const double *phi_f, const double *phi_m,
                                      int c, double p, double sw, Props &q) {
  int loc = c >> 1;
  double phi_ref = (c & 1) == 0 ? phi_f[loc] : phi_m[loc];
  double dp = p - P.p_ref;
  q.rho[0] = P.rho_o_ref * (1.0 + P.c_o * dp);
  q.rho[1] = P.rho_w_ref * (1.0 + P.c_w * dp);
  q.drho[0] = P.rho_o_ref * P.c_o;
  q.drho[1] = P.rho_w_ref * P.c_w;
  q.phi = phi_ref * (1.0 + P.c_rock * (p - P.p_ref_rock));
  q.dphi = phi_ref * P.c_rock;
  double S = (sw - P.swc) * P.inv_span, dS;
  if (S <= 0.0) { S = 0.0; dS = 0.0; }
  else if (S >= 1.0) { S = 1.0; dS = 0.0; }
  else dS = P.inv_span;
  double so = 1.0 - S;
  q.lam[1] = (S * S) * P.inv_mu_w;
  q.dlam[1] = ((2.0 * S) * dS) * P.inv_mu_w;
  q.lam[0] = (so * so) * P.inv_mu_o;
  q.dlam[0] = (-((2.0 * so) * dS)) * P.inv_mu_o;
}

// Phase masses V phi rho s of a cell and their derivatives [phase][p, sw].
__device__ __forceinline__ void accumulation(const Phys &P, double sw, const Props &q,
                                             double M[2], double dM[4]) {
  double Vphi = P.V * q.phi;
  double so = 1.0 - sw;
  M[0] = (Vphi * q.rho[0]) * so;
  M[1] = (Vphi * q.rho[1]) * sw;
  dM[0] = (P.V * ((q.dphi * q.rho[0]) + (q.phi * q.drho[0]))) * so;
  dM[1] = -(Vphi * q.rho[0]);
  dM[2] = (P.V * ((q.dphi * q.rho[1]) + (q.phi * q.drho[1]))) * sw;
  dM[3] = Vphi * q.rho[1];
}

// Mass flux a -> b (a < b) per phase with upstream mobility (Section 2:
// Darcy flux with potential Phi = p - rho g z, upstream weighting).  GRAV =
// false is the same evaluation for gdz = 0: the gravity terms are then exact
// zeros (x - (y * 0) == x for the finite values here, and p_a - p_b is never
// -0), so the result is identical bit for bit.
// CAP: the water potential carries -p_cow(s_w) of each side (phase pressure
// p_w = p - p_cow), which adds -/+ p_cow' to the saturation derivatives.
template <bool GRAV, bool CAP>
__device__ __forceinline__ void flux(double T, double gdz, double pa, double pb, const Props &qa,
                                     const Props &qb, double F[2], double dFa[4], double dFb[4]) {
#pragma unroll
  for (int al = 0; al < 2; ++al) {
    const bool capw = CAP && al == 1;
    double ppa = capw ? pa - qa.pc : pa;
    double ppb = capw ? pb - qb.pc : pb;
    double dpot, ddpa, ddpb;
    if (GRAV) {
      dpot = (ppa - ppb) - ((0.5 * (qa.rho[al] + qb.rho[al])) * gdz);
      ddpa = 1.0 - ((0.5 * qa.drho[al]) * gdz);
      ddpb = -1.0 - ((0.5 * qb.drho[al]) * gdz);
    } else {
      dpot = ppa - ppb;
      ddpa = 1.0;
      ddpb = -1.0;
    }
    double mob, mpa, msa, mpb, msb;
    if (dpot >= 0.0) {
      mob = qa.rho[al] * qa.lam[al];
      mpa = qa.drho[al] * qa.lam[al];
      msa = qa.rho[al] * qa.dlam[al];
      mpb = 0.0; msb = 0.0;
    } else {
      mob = qb.rho[al] * qb.lam[al];
      mpb = qb.drho[al] * qb.lam[al];
      msb = qb.rho[al] * qb.dlam[al];
      mpa = 0.0; msa = 0.0;
    }
    F[al] = (T * mob) * dpot;
    dFa[2 * al + 0] = T * ((mpa * dpot) + (mob * ddpa));
    dFb[2 * al + 0] = T * ((mpb * dpot) + (mob * ddpb));
    if (capw) {
      dFa[2 * al + 1] = T * ((msa * dpot) - (mob * qa.dpc));
      dFb[2 * al + 1] = T * ((msb * dpot) + (mob * qb.dpc));
    } else {
      dFa[2 * al + 1] = T * (msa * dpot);
      dFb[2 * al + 1] = T * (msb * dpot);
    }
  }
}

// Perforation mass rate into a fracture cell (Section 2, q_{alpha,i}):
// producer WI rho lambda (p_b - p); water injector WI rho_w lambda_t (p_b - p).
__device__ __forceinline__ void perf_rate(int kind, double wi, double pc, double pb, const Props &q,
                                          double Q[2], double dq[4], double dqb[2]) {
  double dpw = pb - pc;
  if (kind == 0) {
    double lt = q.lam[0] + q.lam[1], dlt = q.dlam[0] + q.dlam[1];
    Q[0] = 0.0; dq[0] = 0.0; dq[1] = 0.0; dqb[0] = 0.0;
    Q[1] = ((wi * q.rho[1]) * lt) * dpw;
    dq[2] = (((wi * q.drho[1]) * lt) * dpw) - ((wi * q.rho[1]) * lt);
    dq[3] = ((wi * q.rho[1]) * dlt) * dpw;
    dqb[1] = (wi * q.rho[1]) * lt;
  } else {
#pragma unroll
    for (int al = 0; al < 2; ++al) {
      Q[al] = ((wi * q.rho[al]) * q.lam[al]) * dpw;
      dq[2 * al + 0] = (((wi * q.drho[al]) * q.lam[al]) * dpw) - ((wi * q.rho[al]) * q.lam[al]);
      dq[2 * al + 1] = ((wi * q.rho[al]) * q.dlam[al]) * dpw;
      dqb[al] = (wi * q.rho[al]) * q.lam[al];
    }
  }
}

__device__ __forceinline__ void loc_ijk(const Phys &P, int loc, int &i, int &j, int &k) {
  i = loc % P.nx;
  j = (loc / P.nx) % P.ny;
  k = loc / (P.nx * P.ny);
}

__device__ __forceinline__ double depth(const Phys &P, int k) {
  return P.top_depth + ((double)k + 0.5) * P.dz;
}

// ---------------------------------------------------------------- pattern

// Perforations of a cell: [lo, hi) in the (cell, well)-sorted list.
__device__ __forceinline__ void perf_range(const int *pc_cell, int np, int c, int &lo, int &hi) {
  int a = 0, b = np;
  while (a < b) { int m = (a + b) >> 1; if (pc_cell[m] < c) a = m + 1; else b = m; }
  lo = a;
  b = np;
  while (a < b) { int m = (a + b) >> 1; if (pc_cell[m] <= c) a = m + 1; else b = m; }
  hi = a;
}

__global__ void k_pattern_count(Phys P, const int *pc_cell, int np, const int *pw_start,
                                int *len) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= P.nb) return;
  if (r >= P.nc) { int w = r - P.nc; len[r] = 1 + pw_start[w + 1] - pw_start[w]; return; }
  if (r & 1) { len[r] = 2; return; }
  int i, j, k;
  loc_ijk(P, r >> 1, i, j, k);
  int lo, hi;
  perf_range(pc_cell, np, r, lo, hi);
  len[r] = 2 + (i > 0) + (i < P.nx - 1) + (j > 0) + (j < P.ny - 1) + (k > 0) + (k < P.nz - 1) +
           (hi - lo);
}

// Two-point transmissibility between cells a < b (fracture-fracture
// harmonic mean, or the shape-factor transfer sigma km V of one location).
__device__ __forceinline__ double conn_trans(const Phys &P, const double *kf, const double *km,
                                             int a, int b) {
  int la = a >> 1, lb = b >> 1;
  if (la == lb) return (P.sigma * km[la]) * P.V;
  int ia, ja, ka, ib, jb, kb;
  loc_ijk(P, la, ia, ja, ka);
  loc_ijk(P, lb, ib, jb, kb);
  double A, D;
  if (ka != kb) { A = P.dx * P.dy; D = P.dz; }
  else if (ja != jb) { A = P.dx * P.dz; D = P.dy; }
  else { A = P.dy * P.dz; D = P.dx; }
  double k1 = kf[la], k2 = kf[lb];
  return ((2.0 * A) * (k1 * k2)) / (D * (k1 + k2));
}

__global__ void k_pattern_fill(Phys P, const double *kf, const double *km, const int *pc_cell,
                               const int *pc_well, const double *pc_wi, int np,
                               const int *pw_start, const int *pw_cell, const double *pw_wi,
                               const int *rowptr, int *col, int *diag, double *trans) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= P.nb) return;
  int e0 = rowptr[r];
  if (r >= P.nc) {                       // well row: perforated cells, then itself
    int w = r - P.nc, s = pw_start[w], t = pw_start[w + 1];
    for (int q = s; q < t; ++q) { col[e0 + q - s] = pw_cell[q]; trans[e0 + q - s] = pw_wi[q]; }
    col[e0 + t - s] = r;
    trans[e0 + t - s] = 0.0;
    diag[r] = e0 + t - s;
    return;
  }
  int c[16];
  int n = 0;
  int loc = r >> 1;
  if (r & 1) { c[n++] = r - 1; c[n++] = r; }
  else {
    int i, j, k, nxy = P.nx * P.ny;
    loc_ijk(P, loc, i, j, k);
    if (k > 0) c[n++] = 2 * (loc - nxy);
    if (j > 0) c[n++] = 2 * (loc - P.nx);
    if (i > 0) c[n++] = 2 * (loc - 1);
    c[n++] = r;
    c[n++] = r + 1;
    if (i < P.nx - 1) c[n++] = 2 * (loc + 1);
    if (j < P.ny - 1) c[n++] = 2 * (loc + P.nx);
    if (k < P.nz - 1) c[n++] = 2 * (loc + nxy);
  }
  for (int a = 1; a < n; ++a) {          // sorted ascending
    int v = c[a], b = a - 1;
    while (b >= 0 && c[b] > v) { c[b + 1] = c[b]; --b; }
    c[b + 1] = v;
  }
  for (int a = 0; a < n; ++a) {
    int d = c[a];
    col[e0 + a] = d;
    if (d == r) { diag[r] = e0 + a; trans[e0 + a] = 0.0; }
    else trans[e0 + a] = conn_trans(P, kf, km, min(r, d), max(r, d));
  }
  if (!(r & 1)) {
    int lo, hi;
    perf_range(pc_cell, np, r, lo, hi);
    for (int q = lo; q < hi; ++q) {      // wells after all cells, by well index
      col[e0 + n] = P.nc + pc_well[q];
      trans[e0 + n] = pc_wi[q];
      ++n;
    }
  }
}

__global__ void k_storage_len(int nb, int nL, int nc, const int *rowptr, int *len) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nb) return;
  int i = row_of_pair(q, nL, nc);
  len[q] = rowptr[i + 1] - rowptr[i];
}

__global__ void k_storage_cols(int nb, int nL, int nc, const int *rowptr, const int *col,
                               const int *srowptr, int *scol) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nb) return;
  int i = row_of_pair(q, nL, nc);
  int e0 = rowptr[i], m = rowptr[i + 1] - e0, d0 = srowptr[q];
  for (int k = 0; k < m; ++k) scol[d0 + k] = col[e0 + k];
}

// Peaceman's radius for a vertical well and the well index
// W = 2 pi k h w_frac / (ln(r_e / r_w) + s), k h = sqrt(kx ky) dz, w_frac = 1.
static double well_index_host(double kx, double ky, double dx, double dy, double dz, double rw,
                              double skin) {
  double ryx = ky / kx, rxy = kx / ky;
  double re = 0.28 * std::sqrt(std::sqrt(ryx) * dx * dx + std::sqrt(rxy) * dy * dy) /
              (std::pow(ryx, 0.25) + std::pow(rxy, 0.25));
  double wfrac = 1.0;
  return (((2.0 * M_PI) * std::sqrt(kx * ky)) * dz) * wfrac / (std::log(re / rw) + skin);
}

int phys_build_pattern(Sim *s) {
  Phys &P = s->ph;
  // perforations, well by well (cells ascending), with their well indices
  std::vector<double> kf_host;  // only the perforated locations are needed
  int np = 0;
  for (auto &w : s->wells) np += w.k_bot - w.k_top + 1;
  s->nperf = np;
  std::vector<int> locs;
  for (auto &w : s->wells)
    for (int k = w.k_top; k <= w.k_bot; ++k) locs.push_back(w.i + P.nx * (w.j + P.ny * k));
  std::vector<double> kfp(np);
  for (int q = 0; q < np; ++q)
    DP_CUDA(s, cudaMemcpyAsync(&kfp[q], s->kf + locs[q], sizeof(double), cudaMemcpyDeviceToHost,
                               s->stream));
  DP_CUDA(s, cudaStreamSynchronize(s->stream));
  std::vector<int> pw_start(P.nw + 1, 0), pw_cell(np);
  std::vector<double> pw_wi(np);
  s->wi_host.resize(np);
  int q = 0;
  for (int w = 0; w < P.nw; ++w) {
    const dp_well &W = s->wells[w];
    pw_start[w] = q;
    for (int k = W.k_top; k <= W.k_bot; ++k, ++q) {
      pw_cell[q] = 2 * locs[q];
      pw_wi[q] = W.wi > 0.0 ? W.wi : well_index_host(kfp[q], kfp[q], P.dx, P.dy, P.dz, W.rw, W.skin);
      s->wi_host[q] = pw_wi[q];
    }
  }
  pw_start[P.nw] = np;
  std::vector<int> order(np);
  for (int t = 0; t < np; ++t) order[t] = t;
  std::vector<int> pw_well(np);
  for (int w = 0; w < P.nw; ++w)
    for (int t = pw_start[w]; t < pw_start[w + 1]; ++t) pw_well[t] = w;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return pw_cell[a] != pw_cell[b] ? pw_cell[a] < pw_cell[b] : pw_well[a] < pw_well[b];
  });
  std::vector<int> pc_cell(np), pc_well(np);
  std::vector<double> pc_wi(np);
  for (int t = 0; t < np; ++t) {
    pc_cell[t] = pw_cell[order[t]];
    pc_well[t] = pw_well[order[t]];
    pc_wi[t] = pw_wi[order[t]];
  }
  for (int t = 1; t < np; ++t)
    if (pc_cell[t] == pc_cell[t - 1] && pc_well[t] == pc_well[t - 1]) {
      s->fail(DP_EINVAL, "a well perforates the same cell twice");
      return DP_EINVAL;
    }
  size_t npb = (size_t)std::max(np, 1);
  int *d_pc_cell = (int *)dalloc(s, npb * 4), *d_pc_well = (int *)dalloc(s, npb * 4);
  double *d_pc_wi = (double *)dalloc(s, npb * 8);
  int *d_pw_start = (int *)dalloc(s, (P.nw + 1) * 4), *d_pw_cell = (int *)dalloc(s, npb * 4);
  double *d_pw_wi = (double *)dalloc(s, npb * 8);
  if (!d_pc_cell || !d_pc_well || !d_pc_wi || !d_pw_start || !d_pw_cell || !d_pw_wi) {
    s->fail(DP_ENOMEM, "allocation failed");
    return DP_ENOMEM;
  }
  if (np) {
    DP_CUDA(s, cudaMemcpyAsync(d_pc_cell, pc_cell.data(), np * 4, cudaMemcpyHostToDevice, s->stream));
    DP_CUDA(s, cudaMemcpyAsync(d_pc_well, pc_well.data(), np * 4, cudaMemcpyHostToDevice, s->stream));
    DP_CUDA(s, cudaMemcpyAsync(d_pc_wi, pc_wi.data(), np * 8, cudaMemcpyHostToDevice, s->stream));
    DP_CUDA(s, cudaMemcpyAsync(d_pw_cell, pw_cell.data(), np * 4, cudaMemcpyHostToDevice, s->stream));
    DP_CUDA(s, cudaMemcpyAsync(d_pw_wi, pw_wi.data(), np * 8, cudaMemcpyHostToDevice, s->stream));
  }
  DP_CUDA(s, cudaMemcpyAsync(d_pw_start, pw_start.data(), (P.nw + 1) * 4, cudaMemcpyHostToDevice,
                             s->stream));
  s->perf_cell = d_pc_cell;
  s->perf_well = d_pc_well;
  s->perf_wi = d_pc_wi;
  // row lengths, row pointers, columns and per-entry transmissibilities
  int *len = (int *)dalloc(s, (size_t)P.nb * 4);
  s->A.n = P.nb;
  s->A.rowptr = (int *)dalloc(s, (size_t)(P.nb + 1) * 4);
  s->A.diag = (int *)dalloc(s, (size_t)P.nb * 4);
  if (!len || !s->A.rowptr || !s->A.diag) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
  DP_LAUNCH(s, k_pattern_count, nblk(P.nb), kBlock, 0, P, d_pc_cell, np, d_pw_start, len);
  int nnz = 0;
  DP_TRY(scan_i32(s, len, s->A.rowptr, P.nb, &nnz));
  s->A.nnz = nnz;
  s->A.col = (int *)dalloc(s, (size_t)nnz * 4);
  s->A.val = (double *)dalloc(s, (size_t)nnz * 32);
  s->trans = (double *)dalloc(s, (size_t)nnz * 8);
  s->ap = (double *)dalloc(s, (size_t)nnz * 8);
  s->sval = (double *)dalloc(s, (size_t)nnz * 32);
  if (s->opt.precision >= 1) {   // the preconditioner's residuals in FP32
    s->svalf = (float *)dalloc(s, (size_t)nnz * 16);
    s->spf = (float *)dalloc(s, (size_t)nnz * 8);
    if (!s->svalf || !s->spf) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
  } else {
    s->sa00 = (double *)dalloc(s, (size_t)nnz * 8);
    s->sa01 = (double *)dalloc(s, (size_t)nnz * 8);
    if (!s->sa00 || !s->sa01) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
  }
  s->scol = (int *)dalloc(s, (size_t)nnz * 4);
  s->srowptr = (int *)dalloc(s, ((size_t)P.nb + 1) * 4);
  s->atpos = (int *)dalloc(s, (size_t)nnz * 4);
  s->fconn = (double *)dalloc(s, (size_t)P.nL * 64);
  if (!s->A.col || !s->A.val || !s->trans || !s->ap || !s->sval || !s->scol || !s->srowptr ||
      !s->atpos || !s->fconn) {
    s->fail(DP_ENOMEM, "allocation failed");
    return DP_ENOMEM;
  }
  DP_LAUNCH(s, k_pattern_fill, nblk(P.nb), kBlock, 0, P, s->kf, s->km, d_pc_cell, d_pc_well,
            d_pc_wi, np, d_pw_start, d_pw_cell, d_pw_wi, s->A.rowptr, s->A.col, s->A.diag,
            s->trans);
  DP_CUDA(s, cudaGetLastError());
  DP_TRY(block_tpos(s, P.nb, s->A.rowptr, s->A.col, s->atpos));
  // the storage-order pattern of the Krylov operator's copy
  DP_LAUNCH(s, k_storage_len, nblk(P.nb), kBlock, 0, P.nb, P.nL, P.nc, s->A.rowptr, len);
  int snnz = 0;
  DP_TRY(scan_i32(s, len, s->srowptr, P.nb, &snnz));
  DP_LAUNCH(s, k_storage_cols, nblk(P.nb), kBlock, 0, P.nb, P.nL, P.nc, s->A.rowptr, s->A.col,
            s->srowptr, s->scol);
  DP_CUDA(s, cudaGetLastError());
  dfree(s, len);
  dfree(s, d_pw_start);
  dfree(s, d_pw_cell);
  dfree(s, d_pw_wi);
  return DP_OK;
}

// ---------------------------------------------------------------- assembly

// Cell properties stored structure-of-arrays, [k * nc + c]: rho_o, rho_w,
// lam_o, lam_w, dlam_o, dlam_w, phi, dphi.  Evaluated once per cell so that
// the connections that use a cell read them instead of re-evaluating.

__global__ void __launch_bounds__(kBlock) k_props(Phys P, const double *phi_f, const double *phi_m,
                                                  const double *p, const double *sw, double *pr) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= P.nc) return;
  Props q;
  props(P, phi_f, phi_m, c, p[c], sw[c], q);
  size_t n = (size_t)P.nc;
  pr[c] = q.rho[0];
  pr[n + c] = q.rho[1];
  pr[2 * n + c] = q.lam[0];
  pr[3 * n + c] = q.lam[1];
  pr[4 * n + c] = q.dlam[0];
  pr[5 * n + c] = q.dlam[1];
  pr[6 * n + c] = q.phi;
  pr[7 * n + c] = q.dphi;
}

// The same values as props(): the stored fields, and the density slopes
// rho_ref c formed once on the host (the same products props() forms).
__device__ __forceinline__ void load_props(const Phys &P, const double *phi_f, const double *phi_m,
                                           const double *__restrict__ pr, int c, Props &q) {
  size_t n = (size_t)P.nc;
  q.rho[0] = pr[c];
  q.rho[1] = pr[n + c];
  q.lam[0] = pr[2 * n + c];
  q.lam[1] = pr[3 * n + c];
  q.dlam[0] = pr[4 * n + c];
  q.dlam[1] = pr[5 * n + c];
  q.phi = pr[6 * n + c];
  q.dphi = pr[7 * n + c];
  q.drho[0] = P.drho_o;
  q.drho[1] = P.drho_w;
}

struct AsmArgs {
  Phys P;
  const int *rowptr, *col, *diag, *tpos;
  const double *trans, *phi_f, *phi_m, *pr;
  const double *p, *sw, *bhp, *Mn;
  const int *well_kind;
  const double *well_target;
  double *val, *R, *Macc;
  double2 *fconn;
  double inv_dt;
};

// Connection c of the cell graph: c = 3 loc + axis for the face between
// location loc and its neighbour along x, y or z (when there is one), c =
// 3 nL + loc for the fracture-matrix link of loc.  The two cells a < b.
__device__ __forceinline__ int conn_of(const Phys &P, int r, int d) {
  int la = min(r, d) >> 1, lb = max(r, d) >> 1;
  if (la == lb) return 3 * P.nL + la;
  int diff = lb - la;
  int axis = (diff == 1 && P.nx > 1) ? 0 : ((diff == P.nx && P.ny > 1) ? 1 : 2);
  return 3 * la + axis;
}

__device__ __forceinline__ int find_entry(const int *__restrict__ rowptr,
                                          const int *__restrict__ col, int r, int d) {
  for (int e = rowptr[r], e1 = rowptr[r + 1]; e < e1; ++e)
    if (col[e] == d) return e;
  return -1;
}

// Each connection's flux once (face-based): one thread per connection a < b
// evaluates the flux a -> b with the expressions and operand order of the
// row-wise evaluation, writes the two off-diagonal blocks, dF/dx_b into row
// a and -dF/dx_a into row b, and keeps F for the two rows' sums.  (The row
// of b used to evaluate the same flux again from its side; the values are
// the same, bit for bit: the same call with the same arguments.)
template <bool GRAV, bool CAP>
__global__ void __launch_bounds__(kBlock) k_conn_flux(AsmArgs a) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  const Phys &P = a.P;
  if (c >= 4 * P.nL) return;
  int la, lb;
  if (c < 3 * P.nL) {
    la = c / 3;
    int axis = c - 3 * la, i, j, k;
    loc_ijk(P, la, i, j, k);
    if (axis == 0) { if (i + 1 >= P.nx) return; lb = la + 1; }
    else if (axis == 1) { if (j + 1 >= P.ny) return; lb = la + P.nx; }
    else { if (k + 1 >= P.nz) return; lb = la + P.nx * P.ny; }
  } else {
    la = lb = c - 3 * P.nL;
  }
  int ca = 2 * la, cb = la == lb ? ca + 1 : 2 * lb;
  int eab = find_entry(a.rowptr, a.col, ca, cb), eba = find_entry(a.rowptr, a.col, cb, ca);
  if (eab < 0 || eba < 0) return;
  Props qa, qb;
  load_props(P, a.phi_f, a.phi_m, a.pr, ca, qa);
  load_props(P, a.phi_f, a.phi_m, a.pr, cb, qb);
  if (CAP) {
    cap_pressure(P.pc_n[ca & 1], P.pc_tab[ca & 1], a.sw[ca], qa.pc, qa.dpc);
    cap_pressure(P.pc_n[cb & 1], P.pc_tab[cb & 1], a.sw[cb], qb.pc, qb.dpc);
  }
  double gdz = 0.0;
  if (GRAV) {
    double dzab = 0.0;
    if (la != lb) {
      int ia, ja, ka, ib, jb, kb;
      loc_ijk(P, la, ia, ja, ka);
      loc_ijk(P, lb, ib, jb, kb);
      dzab = depth(P, ka) - depth(P, kb);
    }
    gdz = P.g * dzab;
  }
  double F[2], dFa[4], dFb[4];
  flux<GRAV, CAP>(a.trans[eab], gdz, a.p[ca], a.p[cb], qa, qb, F, dFa, dFb);
  double *oab = a.val + 4 * (size_t)eab, *oba = a.val + 4 * (size_t)eba;
  oab[0] = dFb[0]; oab[1] = dFb[1]; oab[2] = dFb[2]; oab[3] = dFb[3];
  oba[0] = -dFa[0]; oba[1] = -dFa[1]; oba[2] = -dFa[2]; oba[3] = -dFa[3];
  a.fconn[c] = make_double2(F[0], F[1]);
}

// One thread per block row, after k_conn_flux.  Threads [0, nL) take the
// fracture rows, [nL, nc) the matrix rows and [nc, nb) the well rows, so
// that a warp holds rows of one kind and equal length.  Cell rows:
// accumulation, then the connections in increasing column order: a cell
// neighbour d adds +F (d > r) or -F (d < r) of their connection to the
// residual and minus the transposed block (d, r) to the diagonal block
// (that block is -dF/dx_r written by k_conn_flux, so this adds exactly the
// dF/dx_r the row-wise evaluation added); then the perforations.  Well
// rows: the rate or pressure constraint.
template <bool GRAV, bool CAP>
__global__ void __launch_bounds__(kBlock) k_assemble(AsmArgs a) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  const Phys &P = a.P;
  int r;
  if (t < P.nL) r = 2 * t;
  else if (t < P.nc) r = 2 * (t - P.nL) + 1;
  else if (t < P.nb) r = t;
  else return;
  int e0 = a.rowptr[r], e1 = a.rowptr[r + 1];
  if (r < P.nc) {
    double pc = a.p[r], swc = a.sw[r];
    Props qc;
    load_props(P, a.phi_f, a.phi_m, a.pr, r, qc);
    if (CAP) cap_pressure(P.pc_n[r & 1], P.pc_tab[r & 1], swc, qc.pc, qc.dpc);
    double M[2], dM[4];
    accumulation(P, swc, qc, M, dM);
    a.Macc[2 * r] = M[0];
    a.Macc[2 * r + 1] = M[1];
    double r0 = (M[0] - a.Mn[2 * r]) * a.inv_dt;
    double r1 = (M[1] - a.Mn[2 * r + 1]) * a.inv_dt;
    double d0 = dM[0] * a.inv_dt, d1 = dM[1] * a.inv_dt;
    double d2 = dM[2] * a.inv_dt, d3 = dM[3] * a.inv_dt;
    for (int e = e0; e < e1; ++e) {
      int d = a.col[e];
      if (d == r) continue;
      double *off = a.val + 4 * (size_t)e;
      double T = a.trans[e];
      if (d < P.nc) {
        double2 F = a.fconn[conn_of(P, r, d)];
        int te = a.tpos[e];
        if (te < 0) continue;
        double2 t01 = *reinterpret_cast<const double2 *>(a.val + 4 * (size_t)te);
        double2 t23 = *reinterpret_cast<const double2 *>(a.val + 4 * (size_t)te + 2);
        if (r < d) { r0 = r0 + F.x; r1 = r1 + F.y; }
        else { r0 = r0 + (-F.x); r1 = r1 + (-F.y); }
        d0 = d0 + (-t01.x); d1 = d1 + (-t01.y); d2 = d2 + (-t23.x); d3 = d3 + (-t23.y);
      } else {
        int w = d - P.nc;
        double Q[2], dq[4], dqb[2];
        perf_rate(a.well_kind[w], T, pc, a.bhp[w], qc, Q, dq, dqb);
        r0 = r0 - Q[0]; r1 = r1 - Q[1];
        d0 = d0 - dq[0]; d1 = d1 - dq[1]; d2 = d2 - dq[2]; d3 = d3 - dq[3];
        off[0] = -dqb[0]; off[1] = 0.0; off[2] = -dqb[1]; off[3] = 0.0;
      }
    }
    double *dg = a.val + 4 * (size_t)a.diag[r];
    dg[0] = d0; dg[1] = d1; dg[2] = d2; dg[3] = d3;
    a.R[2 * r] = r0;
    a.R[2 * r + 1] = r1;
    return;
  }
  int w = r - P.nc;
  double pb = a.bhp[w];
  double *dg = a.val + 4 * (size_t)a.diag[r];
  if (a.well_kind[w] == 0) {
    double acc = 0.0, accd = 0.0;
    for (int e = e0; e < e1; ++e) {
      int c = a.col[e];
      if (c == r) continue;
      Props q;
      load_props(P, a.phi_f, a.phi_m, a.pr, c, q);
      double lt = q.lam[0] + q.lam[1], dlt = q.dlam[0] + q.dlam[1];
      double wi = a.trans[e];
      double wl = wi * lt;
      acc = acc + (wl * (pb - a.p[c]));
      accd = accd + wl;
      double *off = a.val + 4 * (size_t)e;
      off[0] = -wl; off[1] = (wi * dlt) * (pb - a.p[c]); off[2] = 0.0; off[3] = 0.0;
    }
    a.R[2 * r] = acc - a.well_target[w];
    dg[0] = accd;
  } else if (a.well_kind[w] == 2) {
    // oil-rate producer: the perforation oil rates into the cells sum to
    // minus the target (the oil leaving the reservoir equals the target)
    double acc = 0.0, accd = 0.0;
    for (int e = e0; e < e1; ++e) {
      int c = a.col[e];
      if (c == r) continue;
      Props q;
      load_props(P, a.phi_f, a.phi_m, a.pr, c, q);
      double Q[2], dq[4], dqb[2];
      perf_rate(2, a.trans[e], a.p[c], pb, q, Q, dq, dqb);
      acc = acc + Q[0];
      accd = accd + dqb[0];
      double *off = a.val + 4 * (size_t)e;
      off[0] = dq[0]; off[1] = dq[1]; off[2] = 0.0; off[3] = 0.0;
    }
    a.R[2 * r] = acc + a.well_target[w];
    dg[0] = accd;
  } else {
    for (int e = e0; e < e1; ++e) {
      if (a.col[e] == r) continue;
      double *off = a.val + 4 * (size_t)e;
      off[0] = 0.0; off[1] = 0.0; off[2] = 0.0; off[3] = 0.0;
    }
    a.R[2 * r] = pb - a.well_target[w];
    dg[0] = 1.0;
  }
  dg[1] = 0.0; dg[2] = 0.0; dg[3] = 1.0;
  a.R[2 * r + 1] = 0.0;
}

__global__ void k_save_old(Phys P, const double *phi_f, const double *phi_m, const double *p,
                           const double *sw, const double *bhp, double *pn, double *swn,
                           double *bhpn, double *Mn) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < P.nw) bhpn[c] = bhp[c];
  if (c >= P.nc) return;
  Props q;
  props(P, phi_f, phi_m, c, p[c], sw[c], q);
  double M[2], dM[4];
  accumulation(P, sw[c], q, M, dM);
  pn[c] = p[c];
  swn[c] = sw[c];
  Mn[2 * c] = M[0];
  Mn[2 * c + 1] = M[1];
}

int phys_save_old(Sim *s) {
  Phys &P = s->ph;
  int n = std::max(P.nc, P.nw);
  DP_LAUNCH(s, k_save_old, nblk(n), kBlock, 0, P, s->phi_f, s->phi_m, s->p, s->sw, s->bhp, s->pn,
            s->swn, s->bhpn, s->Mn);
  DP_CUDA(s, cudaGetLastError());
  return DP_OK;
}

// Per well, the oil and water mass rates into the reservoir summed over its
// perforations (Section 2's perforation rates).  One thread per well; the
// perforations are sorted by (cell, well), so a well's own perforations come
// in increasing cell order, from the top layer down.
__global__ void k_well_rates(Phys P, const double *phi_f, const double *phi_m, const double *p,
                             const double *sw, const double *bhp, const int *perf_cell,
                             const int *perf_well, const double *perf_wi, int np,
                             const int *well_kind, double *q_oil, double *q_water) {
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= P.nw) return;
  double qo = 0.0, qw = 0.0;
  for (int t = 0; t < np; ++t) {
    if (perf_well[t] != w) continue;
    int c = perf_cell[t];
    Props q;
    props(P, phi_f, phi_m, c, p[c], sw[c], q);
    double Q[2], dq[4], dqb[2];
    perf_rate(well_kind[w], perf_wi[t], p[c], bhp[w], q, Q, dq, dqb);
    qo = qo + Q[0];
    qw = qw + Q[1];
  }
  q_oil[w] = qo;
  q_water[w] = qw;
}

int phys_well_rates(Sim *s, double *q) {
  if (s->ph.nw == 0) return DP_OK;
  DP_LAUNCH(s, k_well_rates, nblk(s->ph.nw), kBlock, 0, s->ph, s->phi_f, s->phi_m, s->p, s->sw,
            s->bhp, s->perf_cell, s->perf_well, s->perf_wi, s->nperf, s->well_kind, q,
            q + s->ph.nw);
  DP_CUDA(s, cudaGetLastError());
  return DP_OK;
}

// Well controls.  restore: every well back on its own control (start of a
// timestep).  Otherwise, after a Newton update: an injector above its BHP
// limit, or an oil-rate producer below it, goes on BHP control at the limit.
__global__ void k_well_controls(int nw, int restore, const int *ctl_kind, const double *ctl_target,
                                const double *limit, const double *bhp, int *kind, double *target) {
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nw) return;
  if (restore) {
    kind[w] = ctl_kind[w];
    target[w] = ctl_target[w];
    return;
  }
  double lim = limit[w];
  if (lim <= 0.0) return;
  int k = kind[w];
  if ((k == 0 && bhp[w] > lim) || (k == 2 && bhp[w] < lim)) {
    kind[w] = 1;
    target[w] = lim;
  }
}

int phys_well_controls(Sim *s, bool restore) {
  if (s->ph.nw == 0) return DP_OK;
  DP_LAUNCH(s, k_well_controls, nblk(s->ph.nw), kBlock, 0, s->ph.nw, restore ? 1 : 0,
            s->well_ctl_kind, s->well_ctl_target, s->well_limit, s->bhp, s->well_kind,
            s->well_target);
  DP_CUDA(s, cudaGetLastError());
  return DP_OK;
}

int phys_assemble(Sim *s) {
  DP_LAUNCH(s, k_props, nblk(s->ph.nc), kBlock, 0, s->ph, s->phi_f, s->phi_m, s->p, s->sw, s->pr);
  AsmArgs a;
  a.P = s->ph;
  a.rowptr = s->A.rowptr; a.col = s->A.col; a.diag = s->A.diag; a.tpos = s->atpos;
  a.trans = s->trans; a.phi_f = s->phi_f; a.phi_m = s->phi_m; a.pr = s->pr; a.Macc = s->Macc;
  a.p = s->p; a.sw = s->sw; a.bhp = s->bhp; a.Mn = s->Mn;
  a.well_kind = s->well_kind; a.well_target = s->well_target;
  a.val = s->A.val; a.R = s->R;
  a.fconn = reinterpret_cast<double2 *>(s->fconn);
  a.inv_dt = s->inv_dt;
  bool grav = s->ph.g != 0.0, cap = s->ph.pc_n[0] > 0 || s->ph.pc_n[1] > 0;
  void (*k_conn_flux_sel)(AsmArgs) =
      cap ? (grav ? k_conn_flux<true, true> : k_conn_flux<false, true>)
          : (grav ? k_conn_flux<true, false> : k_conn_flux<false, false>);
  void (*k_assemble_sel)(AsmArgs) =
      cap ? (grav ? k_assemble<true, true> : k_assemble<false, true>)
          : (grav ? k_assemble<true, false> : k_assemble<false, false>);
  DP_LAUNCH(s, k_conn_flux_sel, nblk(4LL * s->ph.nL), kBlock, 0, a);
  DP_LAUNCH(s, k_assemble_sel, nblk(s->ph.nb), kBlock, 0, a);
  DP_CUDA(s, cudaGetLastError());
  return DP_OK;
}

// ---------------------------------------------------------------- norms
// Scaled residual (cell rows by dt / (rho_ref phi_ref V), well rows by
// their target), phase residual sums, mass change and well inflow.  Two
// passes with a fixed reduction order (deterministic for a given size).

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// The cell rows' weights of the scaled residual, 1 / (rho_ref phi_ref V) per
// cell and phase, formed once (an FP64 division per entry is a long
// instruction sequence on this GPU; the norms then multiply).
__global__ void k_norm_weights(Phys P, const double *phi_f, const double *phi_m, double *w) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= P.nc) return;
  int loc = c >> 1;
  double phi_ref = (c & 1) == 0 ? phi_f[loc] : phi_m[loc];
  w[2 * c] = 1.0 / ((P.rho_o_ref * phi_ref) * P.V);
  w[2 * c + 1] = 1.0 / ((P.rho_w_ref * phi_ref) * P.V);
}

int phys_norm_weights(Sim *s) {
  DP_LAUNCH(s, k_norm_weights, nblk(s->ph.nc), kBlock, 0, s->ph, s->phi_f, s->phi_m, s->norm_w);
  DP_CUDA(s, cudaGetLastError());
  return DP_OK;
}

// With lq (the linear residual of the last solve; null when the forcing term
// does not use it) also the squared scaled norms of lq and of R - lq, in the
// scaling of the residual norm.
__global__ void __launch_bounds__(kBlock) k_norms_part(Phys P, const double *__restrict__ w,
                                                       const double *R,
                                                       const double *Macc, const double *Mn,
                                                       const int *well_kind,
                                                       const double *well_target, double dt,
                                                       const double *__restrict__ lq,
                                                       double *part) {
  double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // s2, max, sro, srw, dmo, dmw, |lq|^2, |R-lq|^2
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < P.nb; r += gridDim.x * blockDim.x) {
    if (r < P.nc) {
#pragma unroll
      for (int al = 0; al < 2; ++al) {   // explicit FMAs: this kernel is FP64-bound
        double x = (R[2 * r + al] * dt) * w[2 * r + al];
        v[0] = fma(x, x, v[0]);
        v[1] = fmax(v[1], fabs(x));
        if (lq) {
          double a = (lq[2 * r + al] * dt) * w[2 * r + al];
          double d = x - a;   // R~(R - lq), scaled as R and lq are
          v[6] = fma(a, a, v[6]);
          v[7] = fma(d, d, v[7]);
        }
      }
      v[2] += R[2 * r];
      v[3] += R[2 * r + 1];
      v[4] += Macc[2 * r] - Mn[2 * r];
      v[5] += Macc[2 * r + 1] - Mn[2 * r + 1];
    } else {
      int w = r - P.nc;
      double sc = well_kind[w] == 0 ? fmax(well_target[w], 1e-12) : well_target[w];
      double x = R[2 * r] / sc;
      v[0] = fma(x, x, v[0]);
      v[1] = fmax(v[1], fabs(x));
      if (lq) {
        double a = lq[2 * r] / sc, d = (R[2 * r] - lq[2 * r]) / sc;
        v[6] = fma(a, a, v[6]);
        v[7] = fma(d, d, v[7]);
      }
    }
  }
  __shared__ double sh[kBlock / 32][8];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    double t = k == 1 ? warp_max(v[k]) : warp_sum(v[k]);
    if (lane == 0) sh[wid][k] = t;
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    int k = threadIdx.x;
    double t = 0.0;
    for (int q = 0; q < kBlock / 32; ++q) t = k == 1 ? fmax(t, sh[q][k]) : t + sh[q][k];
    part[blockIdx.x * 8 + k] = t;
  }
}

// One block: partials and perforation rates summed in a fixed order.
__global__ void __launch_bounds__(kBlock) k_norms_final(Phys P, const double *phi_f,
                                                        const double *phi_m, const double *p,
                                                        const double *sw, const double *bhp,
                                                        const int *perf_cell, const int *perf_well,
                                                        const double *perf_wi, int np,
                                                        const int *well_kind, const double *part,
                                                        int nparts, double *out) {
  double v[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) {
    for (int k = 0; k < 6; ++k) v[k] = k == 1 ? fmax(v[k], part[b * 8 + k]) : v[k] + part[b * 8 + k];
    v[8] += part[b * 8 + 6];
    v[9] += part[b * 8 + 7];
  }
  for (int t = threadIdx.x; t < np; t += blockDim.x) {
    int c = perf_cell[t], w = perf_well[t];
    Props q;
    props(P, phi_f, phi_m, c, p[c], sw[c], q);
    double Q[2], dq[4], dqb[2];
    perf_rate(well_kind[w], perf_wi[t], p[c], bhp[w], q, Q, dq, dqb);
    v[6] += Q[0];
    v[7] += Q[1];
  }
  __shared__ double sh[kBlock / 32][10];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 10; ++k) {
    double t = k == 1 ? warp_max(v[k]) : warp_sum(v[k]);
    if (lane == 0) sh[wid][k] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double o[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int q = 0; q < kBlock / 32; ++q)
      for (int k = 0; k < 10; ++k) o[k] = k == 1 ? fmax(o[k], sh[q][k]) : o[k] + sh[q][k];
    out[0] = sqrt(o[0]);
    for (int k = 1; k < 8; ++k) out[k] = o[k];
    out[8] = sqrt(o[8]);   // ||R~(lq)||_2
    out[9] = sqrt(o[9]);   // ||R~(R - lq)||_2
  }
}

int phys_norms(Sim *s) {
  Phys &P = s->ph;
  bool lin = s->have_lq && (s->opt.eta_mode == 1 || s->opt.eta_mode == 2);
  DP_LAUNCH(s, k_norms_part, s->norm_blocks, kBlock, 0, P, s->norm_w, s->R, s->Macc,
            s->Mn, s->well_kind, s->well_target, s->dt, lin ? s->lq : nullptr, s->norm_part);
  DP_LAUNCH(s, k_norms_final, 1, kBlock, 0, P, s->phi_f, s->phi_m, s->p, s->sw, s->bhp, s->perf_cell,
            s->perf_well, s->perf_wi, s->nperf, s->well_kind, s->norm_part, s->norm_blocks,
            s->norm_out);
  DP_CUDA(s, cudaGetLastError());
  return DP_OK;
}

// ---------------------------------------------------------------- decoupling
// Per cell block row (Eq. "decoupled-eq"), well rows unchanged; the pressure
// block takes entry (0,0) of every decoupled block.  Mode 0: the paper's
// modified Gauss-Jordan step, read as the elimination of the pressure row's
// saturation coefficient by the water row of the diagonal block, D_i^-1 =
// [[1, -a01/a11], [0, 1]] (the per-cell Quasi-IMPES form); mode 1: ABF,
// D_i^-1 = the inverse of the diagonal block; mode 2: True-IMPES, the weight
// c01/c11 from the sums of block column i over all rows, in increasing row
// order (read through the transpose positions of row i's entries).
//
// Two passes: one thread per row takes the row's weight or inverse (the
// divisions once per row) and the right-hand side; then one thread per
// entry, in natural order (coalesced reads of the Jacobian), writes the
// decoupled block wherever it is consumed: the pressure block ap (natural
// order), the storage-order copy of the Krylov operator (sval, and
// sa00/sa01 for the pressure residual), the ILU(0) factor's starting values
// in its split layout and precision, and the colour-ordered level-0 copy of
// the Gauss-Seidel sweeps.  The Jacobian itself is left as assembled.
__global__ void __launch_bounds__(kBlock) k_decouple_rows(int nb, int nc, int mode,
                                                          const int *rowptr, const int *diag,
                                                          const int *tpos, const double *val,
                                                          const double *R, double *fct,
                                                          double *bh) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  double b0 = -R[2 * i], b1 = -R[2 * i + 1];
  if (i >= nc) {
    bh[2 * i] = b0;
    bh[2 * i + 1] = b1;
    return;
  }
  const double *dg = val + 4 * (size_t)diag[i];
  if (mode == 1) {
    double d00 = dg[0], d01 = dg[1], d10 = dg[2], d11 = dg[3];
    double det = (d00 * d11) - (d01 * d10);
    double *f = fct + 4 * (size_t)i;
    if (fabs(det) < 1e-300) {
      f[0] = 1.0; f[1] = 0.0; f[2] = 0.0; f[3] = 1.0;   // row left as it is
      bh[2 * i] = b0;
      bh[2 * i + 1] = b1;
      return;
    }
    double i00 = d11 / det, i01 = (-d01) / det, i10 = (-d10) / det, i11 = d00 / det;
    f[0] = i00; f[1] = i01; f[2] = i10; f[3] = i11;
    bh[2 * i] = (i00 * b0) + (i01 * b1);
    bh[2 * i + 1] = (i10 * b0) + (i11 * b1);
    return;
  }
  double w;
  if (mode == 2) {
    double c01 = 0.0, c11 = 0.0;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      const double *a = val + 4 * (size_t)tpos[e];
      c01 = c01 + a[1];
      c11 = c11 + a[3];
    }
    w = fabs(c11) < 1e-300 ? 0.0 : c01 / c11;
  } else {
    double a01 = dg[1], a11 = dg[3];
    w = fabs(a11) < 1e-300 ? 0.0 : a01 / a11;
  }
  fct[i] = w;
  bh[2 * i] = b0 - (w * b1);
  bh[2 * i + 1] = b1;
}

struct DecArgs {
  long long nnz;
  int nc, sL, sc, mode;   // rows below nc are cell rows; storage mapping (sL, sc)
  const int *erow, *rowptr, *srowptr, *ilupos, *l0pos;
  const double *val, *fct;
  double *ap, *sval, *sa00, *sa01;
  float *svalf, *spf;   // FP32 copies for the preconditioner's residuals, or null
  void *lu;         // split-layout factor values (float or double), or null
  void *l0;         // colour-ordered level-0 pressure values, or null
};

template <typename T>
__global__ void __launch_bounds__(kBlock) k_decouple(DecArgs a) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.nnz) return;
  int i = __ldg(a.erow + e);
  const double2 *v2 = reinterpret_cast<const double2 *>(a.val) + 2 * e;
  double2 u = v2[0], w = v2[1];
  double n0 = u.x, n1 = u.y, n2 = w.x, n3 = w.y;
  if (i < a.nc) {
    if (a.mode == 1) {
      const double *f = a.fct + 4 * (size_t)i;
      double i00 = f[0], i01 = f[1], i10 = f[2], i11 = f[3];
      bool keep = i00 == 1.0 && i01 == 0.0 && i10 == 0.0 && i11 == 1.0;   // singular pivot
      double v0 = n0, v1 = n1, v2 = n2, v3 = n3;
      if (!keep) {
        n0 = (i00 * v0) + (i01 * v2);
        n1 = (i00 * v1) + (i01 * v3);
        n2 = (i10 * v0) + (i11 * v2);
        n3 = (i10 * v1) + (i11 * v3);
      }
    } else {
      double f = a.fct[i];
      n0 = n0 - (f * n2);
      n1 = n1 - (f * n3);
    }
  }
  a.ap[e] = n0;
  int si = storage_row(i, a.sL, a.sc);
  size_t q = (size_t)(__ldg(a.srowptr + si) + (int)(e - __ldg(a.rowptr + i)));
  double2 *sv = reinterpret_cast<double2 *>(a.sval) + 2 * q;
  sv[0] = make_double2(n0, n1);
  sv[1] = make_double2(n2, n3);
  if (a.sa00) {
    a.sa00[q] = n0;
    a.sa01[q] = n1;
  }
  if (a.svalf) {
    reinterpret_cast<float4 *>(a.svalf)[q] = make_float4(float(n0), float(n1), float(n2), float(n3));
    reinterpret_cast<float2 *>(a.spf)[q] = make_float2(float(n0), float(n1));
  }
  if (a.lu) {
    T *d = reinterpret_cast<T *>(a.lu) + 4 * (size_t)__ldg(a.ilupos + e);
    d[0] = T(n0); d[1] = T(n1); d[2] = T(n2); d[3] = T(n3);
  }
  if (a.l0) reinterpret_cast<T *>(a.l0)[__ldg(a.l0pos + e)] = T(n0);
}

int phys_decouple_extract(Sim *s) {
  int mode = s->opt.decouple;
  const Bsr &K = s->K;
  DP_LAUNCH(s, k_decouple_rows, nblk(K.n), kBlock, 0, K.n, s->sv_cells, mode, K.rowptr, K.diag,
            s->btpos, K.val, s->Rk, s->fct, s->bh);
  DecArgs a;
  a.nnz = K.nnz; a.nc = s->sv_cells; a.sL = s->sv_sL; a.sc = s->sv_sc; a.mode = mode;
  a.erow = s->erow; a.rowptr = K.rowptr; a.srowptr = s->srowptr;
  a.ilupos = s->ilupos; a.l0pos = s->l0pos;
  a.val = K.val; a.fct = s->fct;
  a.ap = s->ap; a.sval = s->sval; a.sa00 = s->sa00; a.sa01 = s->sa01;
  a.svalf = s->svalf; a.spf = s->spf;
  bool f32 = s->opt.precision >= 1;
  a.lu = s->opt.precond >= 1 ? (f32 ? (void *)s->lu_valf : (void *)s->lu_val) : nullptr;
  a.l0 = s->l0_lu ? (f32 ? (void *)s->l0_pvf : (void *)s->l0_pv) : nullptr;
  if (f32) DP_LAUNCH(s, k_decouple<float>, nblk(K.nnz), kBlock, 0, a);
  else DP_LAUNCH(s, k_decouple<double>, nblk(K.nnz), kBlock, 0, a);
  DP_CUDA(s, cudaGetLastError());
  return DP_OK;
}

// The decoupled matrix in natural order, from its storage-order copy (test
// access: the Jacobian itself stays as assembled).
__global__ void k_natural_from_storage(long long nnz, int nc, int nL, const int *erow,
                                       const int *rowptr, const int *srowptr, const double *sval,
                                       double *out) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnz) return;
  int i = erow[e];
  size_t q = (size_t)(srowptr[storage_row(i, nL, nc)] + (int)(e - rowptr[i]));
  for (int k = 0; k < 4; ++k) out[4 * e + k] = sval[4 * q + k];
}

int phys_decoupled_natural(Sim *s, double *out) {
  DP_LAUNCH(s, k_natural_from_storage, nblk(s->K.nnz), kBlock, 0, (long long)s->K.nnz, s->sv_sc,
            s->sv_sL, s->erow, s->K.rowptr, s->srowptr, s->sval, out);
  DP_CUDA(s, cudaGetLastError());
  return DP_OK;
}

// ---------------------------------------------------------------- Schur option
// Exact elimination of the matrix continuum: a matrix cell m of location loc
// couples only to itself and to its fracture cell f, so y_m = A_mm^-1 (-R_m
// - A_mf y_f), and the fracture row takes S_ff = A_ff - A_fm A_mm^-1 A_mf and
// the residual R_f - A_fm A_mm^-1 R_m.  K keeps the fracture rows (row loc)
// and the well rows (row nL + w); its other blocks are copies of A's.  The
// formulas are evaluated as written, in the order the oracle uses.

__device__ __forceinline__ int kcol(int c, int nL, int nc) {   // -1: a matrix column, dropped
  return c >= nc ? nL + (c - nc) : ((c & 1) ? -1 : c >> 1);
}

__global__ void k_schur_len(int nk, int nL, int nc, const int *rowptr, const int *col, int *len) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nk) return;
  int jr = r < nL ? 2 * r : nc + (r - nL), c = 0;
  for (int e = rowptr[jr]; e < rowptr[jr + 1]; ++e) c += kcol(col[e], nL, nc) >= 0;
  len[r] = c;
}

__global__ void k_schur_fill(int nk, int nL, int nc, const int *rowptr, const int *col,
                             const int *krowptr, int *kcolv, int *kdiag, int *kmap) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nk) return;
  int jr = r < nL ? 2 * r : nc + (r - nL), k = krowptr[r];
  for (int e = rowptr[jr]; e < rowptr[jr + 1]; ++e) {
    int c = kcol(col[e], nL, nc);
    if (c < 0) continue;
    kcolv[k] = c;
    kmap[k] = (r < nL && c == r) ? -1 : e;
    if (c == r) kdiag[r] = k;
    ++k;
  }
}

__device__ __forceinline__ int find_col_in(const int *col, int lo, int hi, int c) {
  while (lo < hi) {
    int m = (lo + hi) >> 1;
    if (col[m] == c) return m;
    if (col[m] < c) lo = m + 1; else hi = m;
  }
  return -1;
}

__global__ void k_schur_pos(int nL, const int *rowptr, const int *col, int *pos_fm, int *pos_mf) {
  int loc = blockIdx.x * blockDim.x + threadIdx.x;
  if (loc >= nL) return;
  int f = 2 * loc, m = f + 1;
  pos_fm[loc] = find_col_in(col, rowptr[f], rowptr[f + 1], m);
  pos_mf[loc] = find_col_in(col, rowptr[m], rowptr[m + 1], f);
}

__global__ void k_schur_copy(long long nnzk, const int *kmap, const double *val, double *kval) {
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nnzk) return;
  int e = kmap[k];
  if (e < 0) return;
  const double2 *src = reinterpret_cast<const double2 *>(val) + 2 * (size_t)e;
  double2 *dst = reinterpret_cast<double2 *>(kval) + 2 * k;
  dst[0] = src[0];
  dst[1] = src[1];
}

__global__ void k_schur_loc(int nL, int nc, int nw, const int *diag, const int *pos_fm,
                            const int *pos_mf, const int *kdiag, const double *val,
                            const double *R, double *kval, double *RK, double *Minv) {
  int loc = blockIdx.x * blockDim.x + threadIdx.x;
  if (loc < nw) {
    RK[2 * (nL + loc)] = R[2 * (nc + loc)];
    RK[2 * (nL + loc) + 1] = R[2 * (nc + loc) + 1];
  }
  if (loc >= nL) return;
  int f = 2 * loc, m = f + 1;
  const double *amm = val + 4 * (size_t)diag[m];
  const double *amf = val + 4 * (size_t)pos_mf[loc];
  const double *afm = val + 4 * (size_t)pos_fm[loc];
  const double *aff = val + 4 * (size_t)diag[f];
  double det = (amm[0] * amm[3]) - (amm[1] * amm[2]);
  double m0, m1, m2, m3;
  if (fabs(det) < 1e-300) { m0 = 0.0; m1 = 0.0; m2 = 0.0; m3 = 0.0; }
  else { m0 = amm[3] / det; m1 = (-amm[1]) / det; m2 = (-amm[2]) / det; m3 = amm[0] / det; }
  double *mi = Minv + 4 * (size_t)loc;
  mi[0] = m0; mi[1] = m1; mi[2] = m2; mi[3] = m3;
  double x00 = (afm[0] * m0) + (afm[1] * m2);
  double x01 = (afm[0] * m1) + (afm[1] * m3);
  double x10 = (afm[2] * m0) + (afm[3] * m2);
  double x11 = (afm[2] * m1) + (afm[3] * m3);
  double *sk = kval + 4 * (size_t)kdiag[loc];
  sk[0] = aff[0] - ((x00 * amf[0]) + (x01 * amf[2]));
  sk[1] = aff[1] - ((x00 * amf[1]) + (x01 * amf[3]));
  sk[2] = aff[2] - ((x10 * amf[0]) + (x11 * amf[2]));
  sk[3] = aff[3] - ((x10 * amf[1]) + (x11 * amf[3]));
  double rm0 = R[2 * m], rm1 = R[2 * m + 1];
  RK[2 * loc] = R[2 * f] - ((x00 * rm0) + (x01 * rm1));
  RK[2 * loc + 1] = R[2 * f + 1] - ((x10 * rm0) + (x11 * rm1));
}

__global__ void k_schur_back(int nL, int nc, int nw, const int *pos_mf, const double *val,
                             const double *Minv, const double *R, const double *yk, double *y) {
  int loc = blockIdx.x * blockDim.x + threadIdx.x;
  if (loc < nw) {
    y[2 * (nc + loc)] = yk[2 * (nL + loc)];
    y[2 * (nc + loc) + 1] = yk[2 * (nL + loc) + 1];
  }
  if (loc >= nL) return;
  int f = 2 * loc, m = f + 1;
  double yf0 = yk[2 * loc], yf1 = yk[2 * loc + 1];
  const double *amf = val + 4 * (size_t)pos_mf[loc];
  const double *mi = Minv + 4 * (size_t)loc;
  double t0 = (-R[2 * m]) - ((amf[0] * yf0) + (amf[1] * yf1));
  double t1 = (-R[2 * m + 1]) - ((amf[2] * yf0) + (amf[3] * yf1));
  y[2 * f] = yf0;
  y[2 * f + 1] = yf1;
  y[2 * m] = (mi[0] * t0) + (mi[1] * t1);
  y[2 * m + 1] = (mi[2] * t0) + (mi[3] * t1);
}

int phys_solver_view(Sim *s) {
  Phys &P = s->ph;
  if (!s->opt.schur) {
    s->K = s->A;
    s->sv_sL = P.nL; s->sv_sc = P.nc; s->sv_cells = P.nc; s->sv_long0 = P.nc;
    s->Rk = s->R;
    s->yk = s->y;
    return DP_OK;
  }
  Bsr &K = s->K;
  int nk = P.nL + P.nw;
  K.n = nk;
  K.rowptr = (int *)dalloc(s, ((size_t)nk + 1) * 4);
  K.diag = (int *)dalloc(s, (size_t)nk * 4);
  int *len = (int *)dalloc(s, (size_t)nk * 4);
  if (!K.rowptr || !K.diag || !len) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
  DP_LAUNCH(s, k_schur_len, nblk(nk), kBlock, 0, nk, P.nL, P.nc, s->A.rowptr, s->A.col, len);
  int nnz = 0;
  DP_TRY(scan_i32(s, len, K.rowptr, nk, &nnz));
  K.nnz = nnz;
  K.col = (int *)dalloc(s, (size_t)nnz * 4);
  K.val = (double *)dalloc(s, (size_t)nnz * 32);
  s->kmap = (int *)dalloc(s, (size_t)nnz * 4);
  s->pos_fm = (int *)dalloc(s, (size_t)P.nL * 4);
  s->pos_mf = (int *)dalloc(s, (size_t)P.nL * 4);
  s->Minv = (double *)dalloc(s, (size_t)P.nL * 32);
  s->Rk = (double *)dalloc(s, (size_t)nk * 16);
  s->yk = (double *)dalloc(s, (size_t)nk * 16);
  if (!K.col || !K.val || !s->kmap || !s->pos_fm || !s->pos_mf || !s->Minv || !s->Rk || !s->yk) {
    s->fail(DP_ENOMEM, "allocation failed");
    return DP_ENOMEM;
  }
  DP_LAUNCH(s, k_schur_fill, nblk(nk), kBlock, 0, nk, P.nL, P.nc, s->A.rowptr, s->A.col, K.rowptr,
            K.col, K.diag, s->kmap);
  DP_LAUNCH(s, k_schur_pos, nblk(P.nL), kBlock, 0, P.nL, s->A.rowptr, s->A.col, s->pos_fm,
            s->pos_mf);
  dfree(s, len);
  // K's rows are already grouped (fracture rows, then wells): its storage
  // order is its natural order
  dfree(s, s->srowptr);
  dfree(s, s->scol);
  s->srowptr = K.rowptr;
  s->scol = K.col;
  s->sv_sL = 0; s->sv_sc = 0; s->sv_cells = P.nL; s->sv_long0 = P.nL;
  DP_CUDA(s, cudaGetLastError());
  return DP_OK;
}

int phys_schur_reduce(Sim *s) {
  Phys &P = s->ph;
  DP_LAUNCH(s, k_schur_copy, nblk(s->K.nnz), kBlock, 0, (long long)s->K.nnz, s->kmap, s->A.val,
            s->K.val);
  DP_LAUNCH(s, k_schur_loc, nblk(std::max(P.nL, P.nw)), kBlock, 0, P.nL, P.nc, P.nw, s->A.diag,
            s->pos_fm, s->pos_mf, s->K.diag, s->A.val, s->R, s->K.val, s->Rk, s->Minv);
  DP_CUDA(s, cudaGetLastError());
  return DP_OK;
}

int phys_schur_back(Sim *s) {
  Phys &P = s->ph;
  DP_LAUNCH(s, k_schur_back, nblk(std::max(P.nL, P.nw)), kBlock, 0, P.nL, P.nc, P.nw, s->pos_mf,
            s->A.val, s->Minv, s->R, s->yk, s->y);
  DP_CUDA(s, cudaGetLastError());
  return DP_OK;
}

// ---------------------------------------------------------------- update
__global__ void k_update(int nc, int nw, double ds_max, const double *y, double *p, double *sw,
                         double *bhp) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < nw) bhp[c] += y[2 * (nc + c)];
  if (c >= nc) return;
  p[c] += y[2 * c];
  double ds = y[2 * c + 1];
  if (ds > ds_max) ds = ds_max;
  if (ds < -ds_max) ds = -ds_max;
  double v = sw[c] + ds;
  if (v < 0.0) v = 0.0;
  if (v > 1.0) v = 1.0;
  sw[c] = v;
}

int phys_update(Sim *s) {
  int n = std::max(s->ph.nc, s->ph.nw);
  DP_LAUNCH(s, k_update, nblk(n), kBlock, 0, s->ph.nc, s->ph.nw, s->opt.ds_max, s->y, s->p, s->sw,
            s->bhp);
  DP_CUDA(s, cudaGetLastError());
  return DP_OK;
}

}  // namespace dp
