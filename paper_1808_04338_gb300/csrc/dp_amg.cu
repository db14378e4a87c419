// Integer setup (scans, greedy colouring, strength, MIS(2), aggregation,
// sparse products) and the numeric smoothed-aggregation hierarchy of the
// pressure stage of CPR-FPF (Section 3.2).
//
// Compiled with -fmad=false.  The aggregates of level l+1 are computed from
// the values of the Galerkin product of level l, so every product and sum
// of the setup is evaluated in a fixed order without contraction: each
// sparse product entry C_rc = sum_k L_rk R_kc is accumulated in increasing
// k, exactly like a sequential row-by-row (Gustavson) product.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>

#include "dp_internal.h"
#include "dp_tma.cuh"

namespace dp {

// ---------------------------------------------------------------- scan
// Exclusive prefix sum of int32 with the total stored in out[n].
constexpr int kScanBlock = 1024;

__global__ void k_scan_block(const int *in, int *out, int n, long long *bsum) {
  __shared__ long long ws[32];
  int i = blockIdx.x * kScanBlock + threadIdx.x;
  long long v = i < n ? in[i] : 0;
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long t = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += t;
  }
  if (lane == 31) ws[wid] = x;
  __syncthreads();
  if (wid == 0) {
    long long y = ws[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long t = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) y += t;
    }
    ws[lane] = y;
  }
  __syncthreads();
  long long excl = x - v + (wid > 0 ? ws[wid - 1] : 0);
  if (i < n) out[i] = (int)excl;
  if (threadIdx.x == kScanBlock - 1) bsum[blockIdx.x] = ws[31];
}

__global__ void k_scan_top(long long *bsum, int nb, int *out, int n, int *overflow) {
  if (threadIdx.x != 0) return;
  long long run = 0;
  for (int b = 0; b < nb; ++b) { long long t = bsum[b]; bsum[b] = run; run += t; }
  out[n] = (int)run;
  *overflow = run > 2147483647LL;
}

__global__ void k_scan_add(int *out, int n, const long long *bsum) {
  int i = blockIdx.x * kScanBlock + threadIdx.x;
  if (i < n) out[i] = (int)(out[i] + bsum[blockIdx.x]);
}

int scan_i32(Sim *s, const int *in, int *out, int n, int *total) {
  int nb = nblk(n, kScanBlock);
  long long *bsum = (long long *)dalloc(s, (size_t)nb * 8);
  if (!bsum) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
  if (n > 0) DP_LAUNCH(s, k_scan_block, nb, kScanBlock, 0, in, out, n, bsum);
  else DP_CUDA(s, cudaMemsetAsync(bsum, 0, 8, s->stream));
  DP_LAUNCH(s, k_scan_top, 1, 32, 0, bsum, n > 0 ? nb : 0, out, n, s->counter + 2);
  if (n > 0) DP_LAUNCH(s, k_scan_add, nb, kScanBlock, 0, out, n, bsum);
  DP_CUDA(s, cudaGetLastError());
  if (total) {
    int h[2];
    DP_CUDA(s, cudaMemcpyAsync(&h[0], out + n, 4, cudaMemcpyDeviceToHost, s->stream));
    DP_CUDA(s, cudaMemcpyAsync(&h[1], s->counter + 2, 4, cudaMemcpyDeviceToHost, s->stream));
    DP_CUDA(s, cudaStreamSynchronize(s->stream));
    if (h[1]) { s->fail(DP_EINVAL, "prefix sum exceeds int32"); dfree(s, bsum); return DP_EINVAL; }
    *total = h[0];
  }
  dfree(s, bsum);
  return DP_OK;
}

// ---------------------------------------------------------------- colouring
// Greedy first-fit colouring in natural row order: row i takes the smallest
// colour unused by its neighbours of smaller index.  Evaluated in rounds: a
// row is coloured once all its lower-index neighbours are (colours written
// earlier in the same round count), so the result is the same function of
// the pattern whatever the timing.  All rounds run in one cooperative
// launch, separated by grid barriers (bounded waits; a failure sets
// err[0]): each round every thread tries the uncoloured rows of its
// grid-stride set and counts those still waiting in pend[round % 3]; after
// the barrier every thread reads that count, and the launch ends when it
// is 0.  Three rotating counts: the one reset during round r was last read
// after barrier r - 2.
constexpr int kMaxColours = 256;

__global__ void __launch_bounds__(kBlock) k_colour_rounds(int n, const int *__restrict__ rowptr,
                                                         const int *__restrict__ col,
                                                         int *colour, int *pend, int *overflow,
                                                         unsigned *bar, int *err) {
  volatile int *vc = colour;
  const int G = (int)gridDim.x;
  for (int round = 0; round < (1 << 20); ++round) {
    if (blockIdx.x == 0 && threadIdx.x == 0) pend[(round + 1) % 3] = 0;
    int waiting = 0;
    for (int i = (int)blockIdx.x * kBlock + threadIdx.x; i < n; i += G * kBlock) {
      if (vc[i] >= 0) continue;
      unsigned long long used[kMaxColours / 64] = {0, 0, 0, 0};
      bool ready = true;
      for (int e = __ldg(rowptr + i), e1 = __ldg(rowptr + i + 1); e < e1; ++e) {
        int j = __ldg(col + e);
        if (j >= i) continue;
        int c = vc[j];
        if (c < 0) { ready = false; break; }
        if (c < kMaxColours) used[c >> 6] |= 1ull << (c & 63);
      }
      if (!ready) { ++waiting; continue; }
      int c = 0;
      while (c < kMaxColours && (used[c >> 6] >> (c & 63)) & 1ull) ++c;
      if (c >= kMaxColours) { *overflow = 1; c = kMaxColours - 1; }
      vc[i] = c;
    }
    if (waiting) atomicAdd(pend + round % 3, waiting);
    if (!grid_sync_all(bar, (unsigned)(round + 1) * (unsigned)G, err)) return;
    if (*(volatile int *)(pend + round % 3) == 0) break;
  }
  grid_exit(bar);
}

__global__ void k_fill_i32(int *a, int n, int v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

// the largest colour (out[0]) and whether a row was left uncoloured (out[1])
__global__ void k_colour_check(const int *a, int n, int *out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  atomicMax(out, a[i]);
  if (a[i] < 0) out[1] = 1;
}

// the cooperative launch of k_colour_rounds: its CTAs resident together
static int colour_rounds(Sim *s, int n, const int *rowptr, const int *col, int *colour) {
  static const int slots = []() {
    int dev = 0, nsm = 0, k = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, k_colour_rounds, kBlock, 0);
    return std::max(k, 1) * std::max(nsm, 1);
  }();
  int grid = std::max(1, std::min(slots, nblk(n)));
  if (s->alloc_failed) return DP_ENOMEM;
  LaunchScope ls(s, "k_colour_rounds");
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kBlock);
  cfg.stream = s->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  // counter: [1] overflow, [3] err, [4..6] the rotating counts; dev_err + 4: the barrier's
  DP_CUDA(s, cudaLaunchKernelEx(&cfg, k_colour_rounds, n, rowptr, col, colour, s->counter + 4,
                                s->counter + 1, (unsigned *)(s->dev_err + 4), s->counter + 3));
  return DP_OK;
}

int greedy_colour(Sim *s, int n, const int *rowptr, const int *col, int *colour, int *ncolour) {
  DP_LAUNCH(s, k_fill_i32, nblk(n), kBlock, 0, colour, n, -1);
  if (n > 0) {
    DP_CUDA(s, cudaMemsetAsync(s->counter, 0, 32, s->stream));   // overflow, err, counts
    DP_TRY(colour_rounds(s, n, rowptr, col, colour));
    DP_CUDA(s, cudaMemcpyAsync(s->h_counter, s->counter, 16, cudaMemcpyDeviceToHost, s->stream));
    DP_CUDA(s, cudaStreamSynchronize(s->stream));
    if (s->h_counter[3]) {
      s->fail(DP_ETIMEOUT, "greedy colouring: a bounded device-side wait gave up");
      return DP_ETIMEOUT;
    }
    if (s->h_counter[1]) { s->fail(DP_EINVAL, "greedy colouring needs more than 256 colours"); return DP_EINVAL; }
  }
  DP_CUDA(s, cudaMemsetAsync(s->counter, 0, 8, s->stream));
  DP_LAUNCH(s, k_colour_check, nblk(n), kBlock, 0, colour, n, s->counter);
  DP_CUDA(s, cudaMemcpyAsync(s->h_counter, s->counter, 8, cudaMemcpyDeviceToHost, s->stream));
  DP_CUDA(s, cudaStreamSynchronize(s->stream));
  if (n > 0 && s->h_counter[1]) {
    s->fail(DP_EINVAL, "greedy colouring left a row uncoloured");
    return DP_EINVAL;
  }
  *ncolour = n > 0 ? s->h_counter[0] + 1 : 0;
  return DP_OK;
}

// Rows sorted by (colour, index), a stable counting sort over the colours:
// per block of kBlock rows the count of each colour (colour-major array
// cnt[c * nb + block]); one exclusive scan of those counts gives every
// (colour, block) its first position; within a block a row's place among
// its colour's rows of smaller index comes from the warps' match masks and
// the earlier warps' counts.
__global__ void __launch_bounds__(kBlock) k_colour_count(const int *__restrict__ colour, int n,
                                                        int ncolour, int nb, int *__restrict__ cnt) {
  __shared__ int hist[kMaxColours];
  for (int c = threadIdx.x; c < ncolour; c += blockDim.x) hist[c] = 0;
  __syncthreads();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(&hist[colour[i]], 1);
  __syncthreads();
  for (int c = threadIdx.x; c < ncolour; c += blockDim.x)
    cnt[(size_t)c * nb + blockIdx.x] = hist[c];
}

__global__ void __launch_bounds__(kBlock) k_colour_place(const int *__restrict__ colour, int n,
                                                        int ncolour, int nb,
                                                        const int *__restrict__ off,
                                                        int *__restrict__ clist,
                                                        int *__restrict__ iperm) {
  constexpr int kW = kBlock / 32;
  __shared__ int wcnt[kW][kMaxColours];
  for (int k = threadIdx.x; k < kW * kMaxColours; k += blockDim.x) (&wcnt[0][0])[k] = 0;
  __syncthreads();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  bool in = i < n;
  int c = in ? colour[i] : -1;
  unsigned same = __match_any_sync(0xffffffffu, c);
  int rank = __popc(same & ((1u << lane) - 1u));
  if (in && rank == 0) wcnt[w][c] = __popc(same);
  __syncthreads();
  if (!in) return;
  int p = off[(size_t)c * nb + blockIdx.x] + rank;
  for (int v = 0; v < w; ++v) p += wcnt[v][c];
  clist[p] = i;
  if (iperm) iperm[i] = p;
}

__global__ void k_colour_starts(const int *__restrict__ off, int nb, int ncolour, int n,
                                int *__restrict__ out) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < ncolour) out[c] = off[(size_t)c * nb];
  if (c == ncolour) out[c] = n;
}

// Rows sorted by (colour, index): clist, the colour starts, and optionally
// the inverse map (row -> position).
int colour_lists(Sim *s, int n, const int *colour, int ncolour, int *clist,
                 std::vector<int> &cstart, int *iperm) {
  cstart.assign(ncolour + 1, 0);
  if (n == 0 || ncolour == 0) return DP_OK;
  int nb = nblk(n);
  long long m = (long long)ncolour * nb;
  int *cnt = (int *)dalloc(s, (size_t)m * 4), *off = (int *)dalloc(s, ((size_t)m + 1) * 4);
  int *st = (int *)dalloc(s, ((size_t)ncolour + 1) * 4);
  if (!cnt || !off || !st) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
  DP_LAUNCH(s, k_colour_count, nb, kBlock, 0, colour, n, ncolour, nb, cnt);
  int total = 0;
  DP_TRY(scan_i32(s, cnt, off, (int)m, &total));
  DP_LAUNCH(s, k_colour_place, nb, kBlock, 0, colour, n, ncolour, nb, off, clist, iperm);
  DP_LAUNCH(s, k_colour_starts, nblk(ncolour + 1), kBlock, 0, off, nb, ncolour, n, st);
  DP_CUDA(s, cudaMemcpyAsync(cstart.data(), st, ((size_t)ncolour + 1) * 4, cudaMemcpyDeviceToHost,
                             s->stream));
  DP_CUDA(s, cudaStreamSynchronize(s->stream));
  dfree(s, st);
  dfree(s, off);
  dfree(s, cnt);
  return DP_OK;
}

// ---------------------------------------------------------------- helpers

__device__ __forceinline__ int find_sorted(const int *col, int lo, int hi, int c) {
  while (lo < hi) {
    int m = (lo + hi) >> 1;
    int v = col[m];
    if (v == c) return m;
    if (v < c) lo = m + 1; else hi = m;
  }
  return -1;
}

// heap sort of keys with a payload, in place (deterministic)
__device__ void heap_sort2(int *key, int *pay, int n) {
  auto sift = [&](int root, int end) {
    while (2 * root + 1 < end) {
      int child = 2 * root + 1;
      if (child + 1 < end && key[child] < key[child + 1]) ++child;
      if (key[root] < key[child]) {
        int t = key[root]; key[root] = key[child]; key[child] = t;
        if (pay) { t = pay[root]; pay[root] = pay[child]; pay[child] = t; }
        root = child;
      } else return;
    }
  };
  for (int st = n / 2 - 1; st >= 0; --st) sift(st, n);
  for (int end = n - 1; end > 0; --end) {
    int t = key[0]; key[0] = key[end]; key[end] = t;
    if (pay) { t = pay[0]; pay[0] = pay[end]; pay[end] = t; }
    sift(0, end);
  }
}

__global__ void k_diag_pos(int n, const int *rowptr, const int *col, int *dpos) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dpos[i] = find_sorted(col, rowptr[i], rowptr[i + 1], i);
}

__global__ void k_tpos(int n, const int *rowptr, const int *col, int *tpos) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
    int j = col[e];
    tpos[e] = find_sorted(col, rowptr[j], rowptr[j + 1], i);
  }
}

// ---------------------------------------------------------------- strength
// S_ij (i != j): max(|a_ij|, |a_ji|) >= theta sqrt(|a_ii a_jj|), symmetric.
__global__ void k_strength(int n, const int *rowptr, const int *col, const int *dpos,
                           const int *tpos, const double *val, double theta, uint8_t *strong,
                           int *state) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double aii = dpos[i] >= 0 ? val[dpos[i]] : 0.0;
  int deg = 0;
  for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
    int j = col[e];
    uint8_t sflag = 0;
    if (j != i) {
      double ajj = dpos[j] >= 0 ? val[dpos[j]] : 0.0;
      double aji = tpos[e] >= 0 ? val[tpos[e]] : 0.0;
      double lhs = fmax(fabs(val[e]), fabs(aji));
      double rhs = theta * sqrt(fabs(aii * ajj));
      sflag = lhs >= rhs ? 1 : 0;
    }
    strong[e] = sflag;
    deg += sflag;
  }
  state[i] = deg > 0 ? 1 : 0;
}

// ---------------------------------------------------------------- MIS(2)
// Synchronous rounds (Bell, Dalton, Olson 2012) on (state, hash, index)
// tuples packed into 64 bits: state in bits 62-63, hash 30-61, index 0-29.
__device__ __forceinline__ uint32_t hash32(uint32_t i) {
  uint32_t h = i * 0x9E3779B1u;
  h ^= h >> 16; h *= 0x85EBCA6Bu;
  h ^= h >> 13; h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

__global__ void k_tuple_init(int n, const int *state, unsigned long long *t) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n)
    t[i] = ((unsigned long long)state[i] << 62) | ((unsigned long long)hash32((uint32_t)i) << 30) |
           (unsigned long long)i;
}

__global__ void k_tuple_max(int n, const int *rowptr, const int *col, const uint8_t *strong,
                            const unsigned long long *tin, unsigned long long *tout) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned long long m = tin[i];
  for (int e = rowptr[i]; e < rowptr[i + 1]; ++e)
    if (strong[e]) { unsigned long long t = tin[col[e]]; if (t > m) m = t; }
  tout[i] = m;
}

__global__ void k_mis_update(int n, const unsigned long long *t, int *state, int *undecided) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || state[i] != 1) return;
  unsigned long long m = t[i];
  if ((int)(m & 0x3FFFFFFFull) == i) state[i] = 2;
  else if ((m >> 62) == 2ull) state[i] = 0;
  else atomicAdd(undecided, 1);
}

__global__ void k_root_flag(int n, const int *state, int *flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = state[i] == 2;
}

__global__ void k_agg_roots(int n, const int *state, const int *pos, int *agg) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) agg[i] = state[i] == 2 ? pos[i] : -1;
}

// pass 1: a node next to roots joins the root with the largest (hash, index)
__global__ void k_agg_pass1(int n, const int *rowptr, const int *col, const uint8_t *strong,
                            const int *state, const int *agg, int *a1) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int v = agg[i];
  if (v < 0) {
    int best = -1;
    uint32_t bh = 0;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      int j = col[e];
      if (!strong[e] || state[j] != 2) continue;
      uint32_t h = hash32((uint32_t)j);
      if (best < 0 || h > bh || (h == bh && j > best)) { best = j; bh = h; }
    }
    if (best >= 0) v = agg[best];
  }
  a1[i] = v;
}

// pass 2: a remaining node joins the aggregate of its assigned neighbour
// with the largest (hash, index), as assigned after pass 1
__global__ void k_agg_pass2(int n, const int *rowptr, const int *col, const uint8_t *strong,
                            const int *a1, int *a2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int v = a1[i];
  if (v < 0) {
    int best = -1;
    uint32_t bh = 0;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      int j = col[e];
      if (!strong[e] || a1[j] < 0) continue;
      uint32_t h = hash32((uint32_t)j);
      if (best < 0 || h > bh || (h == bh && j > best)) { best = j; bh = h; }
    }
    if (best >= 0) v = a1[best];
  }
  a2[i] = v;
}

// ---------------------------------------------------------------- prolongator
// Pattern of P: the aggregates of the filtered row F(i) = {i} u {strong j}.
__global__ void k_p_collect(int n, const int *rowptr, const int *col, const uint8_t *strong,
                            const int *agg, int *scratch, int *cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int base = rowptr[i], m = 0;
  for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
    int k = col[e];
    if ((k == i || strong[e]) && agg[k] >= 0) scratch[base + m++] = agg[k];
  }
  heap_sort2(scratch + base, nullptr, m);
  int u = 0;
  for (int t = 0; t < m; ++t)
    if (u == 0 || scratch[base + t] != scratch[base + u - 1]) scratch[base + u++] = scratch[base + t];
  cnt[i] = u;
}

__global__ void k_copy_rows(int n, const int *src_rowptr, const int *scratch, const int *dst_rowptr,
                            int *dst_col) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int s0 = src_rowptr[i], d0 = dst_rowptr[i], m = dst_rowptr[i + 1] - d0;
  for (int t = 0; t < m; ++t) dst_col[d0 + t] = scratch[s0 + t];
}

// Filtered diagonal d_i = a_ii + sum_{j weak} a_ij (increasing j) and the
// Gershgorin ratio sum_{F(i)} |aF_ij| / |d_i| whose maximum sets omega.
__global__ void k_filtered_diag(int n, const int *rowptr, const int *col, const uint8_t *strong,
                                const double *val, double *fdiag, unsigned long long *rho_bits) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  bool valid = i < n;                   // every lane reaches the shuffles
  double d = 0.0;
  int e0 = valid ? rowptr[i] : 0, e1 = valid ? rowptr[i + 1] : 0;
  for (int e = e0; e < e1; ++e) if (col[e] == i) d = val[e];
  for (int e = e0; e < e1; ++e) if (col[e] != i && !strong[e]) d = d + val[e];
  if (valid) fdiag[i] = d;
  double ratio = 0.0;
  if (d != 0.0) {
    double s = 0.0;
    for (int e = e0; e < e1; ++e) {
      if (col[e] == i) s = s + fabs(d);
      else if (strong[e]) s = s + fabs(val[e]);
    }
    ratio = s / fabs(d);
  }
  // maximum over the block first (exact), then one atomic per warp
  for (int o = 16; o > 0; o >>= 1) ratio = fmax(ratio, __shfl_xor_sync(0xffffffffu, ratio, o));
  if ((threadIdx.x & 31) == 0 && ratio > 0.0)
    atomicMax(rho_bits, (unsigned long long)__double_as_longlong(ratio));  // ratio >= 0
}

__global__ void k_omega(const unsigned long long *rho_bits, double *omega) {
  double rho = __longlong_as_double((long long)*rho_bits);
  *omega = rho > 0.0 ? (4.0 / 3.0) / rho : 0.0;
}

// P_iJ = [agg(i) == J] - (omega / d_i) * sum_{k in F(i), agg(k) = J} aF_ik
__global__ void k_p_values(int n, const int *rowptr, const int *col, const uint8_t *strong,
                           const double *val, const double *fdiag, const int *agg,
                           const double *omega, const int *p_rowptr, const int *p_col,
                           double *p_val) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int q0 = p_rowptr[i], q1 = p_rowptr[i + 1];
  for (int q = q0; q < q1; ++q) p_val[q] = 0.0;
  double d = fdiag[i];
  for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
    int k = col[e];
    double af;
    if (k == i) af = d;
    else if (strong[e]) af = val[e];
    else continue;
    int J = agg[k];
    if (J < 0) continue;
    int q = find_sorted(p_col, q0, q1, J);
    if (q >= 0) p_val[q] = p_val[q] + af * 1.0;
  }
  double w = d != 0.0 ? *omega / d : 0.0;
  int ai = agg[i];
  for (int q = q0; q < q1; ++q) {
    double t = (ai == p_col[q]) ? 1.0 : 0.0;
    p_val[q] = t - w * p_val[q];
  }
}

// ---------------------------------------------------------------- transpose
__global__ void k_col_count(int nnz, const int *col, int *cnt) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < nnz) atomicAdd(&cnt[col[e]], 1);
}

__global__ void k_transpose_fill(int n, const int *rowptr, const int *col, const int *t_rowptr,
                                 int *fill, int *t_col, int *t_src) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
    int c = col[e];
    int p = t_rowptr[c] + atomicAdd(&fill[c], 1);
    t_col[p] = i;
    t_src[p] = e;
  }
}

__global__ void k_sort_rows(int n, const int *rowptr, int *key, int *pay) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  heap_sort2(key + rowptr[i], pay + rowptr[i], rowptr[i + 1] - rowptr[i]);
}

__global__ void k_gather(int nnz, const int *src, const double *in, double *out) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < nnz) out[e] = in[src[e]];
}

// ---------------------------------------------------------------- SpGEMM
// C = L R.  Symbolic: per row, the sorted union of the columns of the rows
// of R named by the row of L.  Numeric: per row of C, for each entry (r, k)
// of L in increasing k and each (k, c) of R, C_rc += L_rk R_kc.
__global__ void k_spgemm_ub(int n, const int *lrp, const int *lcol, const int *rrp, int *ub) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  int s = 0;
  for (int e = lrp[r]; e < lrp[r + 1]; ++e) { int k = lcol[e]; s += rrp[k + 1] - rrp[k]; }
  ub[r] = s;
}

// Symbolic product, a warp per output row: the row's products (at most
// kExpCap) are gathered into shared memory in the order of the entries of L
// and R, sorted there (bitonic) and deduplicated with ballots; a longer row
// is expanded, heap-sorted and deduplicated in its own scratch by the
// warp's first lane.  Either way the row's scratch starts with its sorted
// distinct columns, and cnt[r] is their count.
constexpr int kExpWarps = 4, kExpCap = 1024;
__global__ void __launch_bounds__(32 * kExpWarps) k_spgemm_expand_w(int n, const int *lrp,
                                                                    const int *lcol,
                                                                    const int *rrp,
                                                                    const int *rcol,
                                                                    const int *off, int *scratch,
                                                                    int *cnt) {
  __shared__ int buf[kExpWarps][kExpCap];
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int r = blockIdx.x * kExpWarps + w;
  if (r >= n) return;   // whole warps
  int base = off[r], m = off[r + 1] - base;
  if (m > kExpCap) {
    if (lane == 0) {
      int t = 0;
      for (int e = lrp[r]; e < lrp[r + 1]; ++e) {
        int k = lcol[e];
        for (int q = rrp[k]; q < rrp[k + 1]; ++q) scratch[base + t++] = rcol[q];
      }
      heap_sort2(scratch + base, nullptr, m);
      int u = 0;
      for (int i = 0; i < m; ++i)
        if (u == 0 || scratch[base + i] != scratch[base + u - 1]) scratch[base + u++] = scratch[base + i];
      cnt[r] = u;
    }
    return;
  }
  int *b = buf[w];
  int t = 0;
  for (int e = __ldg(lrp + r), e1 = __ldg(lrp + r + 1); e < e1; ++e) {
    int k = __ldg(lcol + e), q0 = __ldg(rrp + k), q1 = __ldg(rrp + k + 1);
    for (int q = q0 + lane; q < q1; q += 32) b[t + q - q0] = __ldg(rcol + q);
    t += q1 - q0;
  }
  int p2 = 1;
  while (p2 < m) p2 <<= 1;
  for (int i = m + lane; i < p2; i += 32) b[i] = 0x7fffffff;
  __syncwarp();
  for (int size = 2; size <= p2; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = lane; i < (p2 >> 1); i += 32) {
        int lo = 2 * i - (i & (stride - 1)), hi = lo + stride;
        bool asc = (lo & size) == 0;
        int a = b[lo], c = b[hi];
        if ((a > c) == asc) { b[lo] = c; b[hi] = a; }
      }
      __syncwarp();
    }
  int u = 0;
  for (int i0 = 0; i0 < m; i0 += 32) {
    int i = i0 + lane;
    bool keep = i < m && (i == 0 || b[i] != b[i - 1]);
    unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (keep) scratch[base + u + __popc(bal & ((1u << lane) - 1u))] = b[i];
    u += __popc(bal);
  }
  if (lane == 0) cnt[r] = u;
}

// Positions of every product in the output: for row r, the products are
// enumerated (entry (r, k) of L in increasing k, entry (k, c) of R in
// increasing c) and pos[off[r] + t] is the index of C_rc for product t.  A
// warp per row: the lanes take the products of each entry (r, k) together.
__global__ void __launch_bounds__(kBlock) k_spgemm_positions_w(int n, const int *lrp,
                                                              const int *lcol, const int *rrp,
                                                              const int *rcol, const int *off,
                                                              const int *crp, const int *ccol,
                                                              int *pos) {
  int r = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (r >= n) return;   // whole warps
  int c0 = crp[r], c1 = crp[r + 1], t = off[r];
  for (int e = __ldg(lrp + r), e1 = __ldg(lrp + r + 1); e < e1; ++e) {
    int k = __ldg(lcol + e), q0 = __ldg(rrp + k), q1 = __ldg(rrp + k + 1);
    for (int q = q0 + lane; q < q1; q += 32) pos[t + q - q0] = find_sorted(ccol, c0, c1, __ldg(rcol + q));
    t += q1 - q0;
  }
}

// Numeric product with G lanes per output row: the entries (r, k) of L are
// taken one after the other in increasing k; the lanes share the entries of
// row k of R (distinct columns, so distinct outputs) and synchronise before
// the next k.  Every output is therefore a sum in increasing k.
template <int G>
__global__ void k_spgemm_numeric(int n, const int *lrp, const int *lcol, const double *lval,
                                 const int *rrp, const double *rval, const int *off,
                                 const int *pos, const int *crp, double *cval) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int r = t / G, lane = t % G;
  if (r >= n) return;                   // groups of G lanes leave together
  unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
  int c0 = crp[r], c1 = crp[r + 1];
  for (int q = c0 + lane; q < c1; q += G) cval[q] = 0.0;
  if (G > 1) __syncwarp(gmask);
  int base = off[r];
  for (int e = lrp[r]; e < lrp[r + 1]; ++e) {
    int k = lcol[e];
    double lv = lval[e];
    int q0 = rrp[k], q1 = rrp[k + 1];
    for (int q = q0 + lane; q < q1; q += G) {
      int p = pos[base + q - q0];
      if (p >= 0) cval[p] = cval[p] + lv * rval[q];
    }
    base += q1 - q0;
    if (G > 1) __syncwarp(gmask);
  }
}

#define DP_SWITCH_G2(G, LAUNCH)                      \
  switch (G) {                                      \
    case 1: { constexpr int GG = 1; LAUNCH; } break;  \
    case 2: { constexpr int GG = 2; LAUNCH; } break;  \
    case 4: { constexpr int GG = 4; LAUNCH; } break;  \
    case 8: { constexpr int GG = 8; LAUNCH; } break;  \
    case 16: { constexpr int GG = 16; LAUNCH; } break; \
    default: { constexpr int GG = 32; LAUNCH; } break; \
  }

struct Product {                          // C = L R, pattern and product positions
  int G = 1;
  int *off = nullptr, *pos = nullptr;
};

static int spgemm_numeric(Sim *s, const Product &pr, int n, const int *lrp, const int *lcol,
                          const double *lval, const int *rrp, const double *rval, const int *crp,
                          double *cval) {
  long long thr = (long long)n * pr.G;
  DP_SWITCH_G2(pr.G, DP_LAUNCH(s, k_spgemm_numeric<GG>, nblk(thr), kBlock, 0, n, lrp, lcol, lval,
                               rrp, rval, pr.off, pr.pos, crp, cval));
  return DP_OK;
}

static int spgemm_symbolic(Sim *s, int n, const int *lrp, const int *lcol, const int *rrp,
                           const int *rcol, int **crp_out, int **ccol_out, int *nnz_out,
                           Product *prod) {
  int *ub = (int *)dalloc(s, (size_t)(n + 1) * 4), *off = (int *)dalloc(s, (size_t)(n + 1) * 4);
  int *crp = (int *)dalloc(s, (size_t)(n + 1) * 4);
  if (!ub || !off || !crp) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
  DP_LAUNCH(s, k_spgemm_ub, nblk(n), kBlock, 0, n, lrp, lcol, rrp, ub);
  int tot = 0;
  DP_TRY(scan_i32(s, ub, off, n, &tot));
  prod->G = lanes_for(n > 0 ? (double)tot / n : 0.0);
  int *scratch = (int *)dalloc(s, (size_t)std::max(tot, 1) * 4);
  if (!scratch) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
  DP_LAUNCH(s, k_spgemm_expand_w, nblk(n, kExpWarps), 32 * kExpWarps, 0, n, lrp, lcol, rrp, rcol,
            off, scratch, ub);
  int nnz = 0;
  DP_TRY(scan_i32(s, ub, crp, n, &nnz));
  int *ccol = (int *)dalloc(s, (size_t)std::max(nnz, 1) * 4);
  if (!ccol) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
  DP_LAUNCH(s, k_copy_rows, nblk(n), kBlock, 0, n, off, scratch, crp, ccol);
  DP_CUDA(s, cudaGetLastError());
  dfree(s, scratch);
  dfree(s, ub);
  prod->off = off;
  prod->pos = (int *)dalloc(s, (size_t)std::max(tot, 1) * 4);
  if (!prod->pos) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
  DP_LAUNCH(s, k_spgemm_positions_w, nblk(32LL * n), kBlock, 0, n, lrp, lcol, rrp, rcol, off, crp,
            ccol, prod->pos);
  *crp_out = crp;
  *ccol_out = ccol;
  *nnz_out = nnz;
  return DP_OK;
}

// ---------------------------------------------------------------- hierarchy

// Smoother scaling of a level operator: 1 / a_ii for Gauss-Seidel, or
// 1 / sum_j |a_ij| for l1-Jacobi (0 where that is zero: the row is left as is)
__global__ void k_level_dinv(int n, const int *dpos, const int *rowptr, const double *val, int l1,
                             double *dinv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double d = 0.0;
  if (l1) {
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) d += fabs(val[e]);
  } else {
    d = dpos[i] >= 0 ? val[dpos[i]] : 0.0;
  }
  dinv[i] = d != 0.0 ? 1.0 / d : 0.0;
}

int level_dinv(Sim *s, Level &L) {
  if (L.dpos)
    DP_LAUNCH(s, k_level_dinv, nblk(L.n), kBlock, 0, L.n, L.dpos, L.rowptr, L.val, L.l1 ? 1 : 0,
              L.dinv);
  return DP_OK;
}

static int level_prepare(Sim *s, Level &L) {
  int n = L.n;
  L.G = lanes_for(n > 0 ? (double)L.nnz / n : 0.0);
  L.dpos = (int *)dalloc(s, (size_t)n * 4);
  L.tpos = (int *)dalloc(s, (size_t)std::max(L.nnz, 1) * 4);
  L.colour = (int *)dalloc(s, (size_t)n * 4);
  L.clist = (int *)dalloc(s, (size_t)n * 4);
  L.x = (double *)dalloc(s, (size_t)n * 8);
  L.b = (double *)dalloc(s, (size_t)n * 8);
  L.r = (double *)dalloc(s, (size_t)n * 8);
  L.xf = (float *)dalloc(s, (size_t)n * 4);
  L.bf = (float *)dalloc(s, (size_t)n * 4);
  L.rf = (float *)dalloc(s, (size_t)n * 4);
  if (!L.dpos || !L.tpos || !L.colour || !L.clist || !L.x || !L.b || !L.r || !L.xf || !L.bf || !L.rf) {
    s->fail(DP_ENOMEM, "allocation failed");
    return DP_ENOMEM;
  }
  DP_LAUNCH(s, k_diag_pos, nblk(n), kBlock, 0, n, L.rowptr, L.col, L.dpos);
  DP_LAUNCH(s, k_tpos, nblk(n), kBlock, 0, n, L.rowptr, L.col, L.tpos);
  if (L.rowptr == s->K.rowptr && L.col == s->K.col && s->colour && s->perm && s->ncolour > 0) {
    // level 0 is the pattern the ILU(0) coloured: its colouring and lists are those
    DP_CUDA(s, cudaMemcpyAsync(L.colour, s->colour, (size_t)n * 4, cudaMemcpyDeviceToDevice,
                               s->stream));
    DP_CUDA(s, cudaMemcpyAsync(L.clist, s->perm, (size_t)n * 4, cudaMemcpyDeviceToDevice,
                               s->stream));
    L.ncolour = s->ncolour;
    L.cstart = s->lu_cstart;
  } else if (L.l1) {
    // an l1-Jacobi level uses no colouring: none is made (colours -1)
    DP_LAUNCH(s, k_fill_i32, nblk(n), kBlock, 0, L.colour, n, -1);
    L.ncolour = 0;
    L.cstart.assign(1, 0);
  } else {
    DP_TRY(greedy_colour(s, n, L.rowptr, L.col, L.colour, &L.ncolour));
    DP_TRY(colour_lists(s, n, L.colour, L.ncolour, L.clist, L.cstart, nullptr));
  }
  return DP_OK;
}

// numeric part of one level -> values of the next level's operator
static int level_numeric(Sim *s, Level &L, Level &N) {
  int n = L.n;
  DP_CUDA(s, cudaMemsetAsync(s->rho_bits, 0, 8, s->stream));
  DP_LAUNCH(s, k_filtered_diag, nblk(n), kBlock, 0, n, L.rowptr, L.col, L.strong, L.val, L.fdiag,
            s->rho_bits);
  DP_LAUNCH(s, k_omega, 1, 1, 0, s->rho_bits, s->omega);
  DP_LAUNCH(s, k_p_values, nblk(n), kBlock, 0, n, L.rowptr, L.col, L.strong, L.val, L.fdiag,
            L.agg, s->omega, L.p_rowptr, L.p_col, L.p_val);
  DP_LAUNCH(s, k_gather, nblk(L.r_nnz), kBlock, 0, L.r_nnz, L.r_src, L.p_val, L.r_val);
  Product ap{L.ap_G, L.ap_off, L.ap_pos}, rap{L.rap_G, L.rap_off, L.rap_pos};
  DP_TRY(spgemm_numeric(s, ap, n, L.rowptr, L.col, L.val, L.p_rowptr, L.p_val, L.ap_rowptr,
                        L.ap_val));
  DP_TRY(spgemm_numeric(s, rap, L.nagg, L.r_rowptr, L.r_col, L.r_val, L.ap_rowptr, L.ap_val,
                        N.rowptr, N.val));
  DP_TRY(level_dinv(s, N));
  DP_CUDA(s, cudaGetLastError());
  return DP_OK;
}

static bool verbose() {
  static int v = -1;
  if (v < 0) { const char *e = std::getenv("DPSIM_VERBOSE"); v = e && *e && *e != '0'; }
  return v == 1;
}

static double now_ms() {
  return std::chrono::duration<double, std::milli>(
             std::chrono::steady_clock::now().time_since_epoch()).count();
}

// wall-clock phase log of the set-up (DPSIM_VERBOSE=1), after a sync
static void phase(Sim *s, const char *what, int level, double &t) {
  if (!verbose()) return;
  cudaStreamSynchronize(s->stream);
  double t1 = now_ms();
  std::fprintf(stderr, "[dpsim] amg level %d %-12s %9.2f ms\n", level, what, t1 - t);
  t = t1;
}

int amg_setup(Sim *s) {
  double tp = now_ms();
  graphs_free(s);
  amg_free(s);
  const dp_options &o = s->opt;
  s->lev.clear();
  s->lev.reserve(32);
  Level L0;
  L0.n = s->K.n;
  L0.nnz = s->K.nnz;
  L0.rowptr = s->K.rowptr;
  L0.col = s->K.col;
  L0.val = s->ap;
  L0.l1 = o.amg_gs_levels <= 0;
  L0.dinv = (double *)dalloc(s, (size_t)L0.n * 8);
  L0.dinvf = (float *)dalloc(s, (size_t)L0.n * 4);
  if (!L0.dinv || !L0.dinvf) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
  s->lev.push_back(L0);
  int maxlev = std::min(std::max(o.amg_max_levels, 1), 30);
  for (int l = 0;; ++l) {
    Level &L = s->lev[l];
    DP_TRY(level_prepare(s, L));
    DP_TRY(level_dinv(s, L));
    phase(s, "prepare", l, tp);
    L.agg = (int *)dalloc(s, (size_t)L.n * 4);
    if (!L.agg) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
    DP_LAUNCH(s, k_fill_i32, nblk(L.n), kBlock, 0, L.agg, L.n, -1);
    if (L.n <= o.amg_coarse_max || l + 1 >= maxlev) break;
    int n = L.n;
    // strength and MIS(2)
    L.strong = (uint8_t *)dalloc(s, (size_t)std::max(L.nnz, 1));
    int *state = (int *)dalloc(s, (size_t)n * 4);
    unsigned long long *t0 = (unsigned long long *)dalloc(s, (size_t)n * 8);
    unsigned long long *t1 = (unsigned long long *)dalloc(s, (size_t)n * 8);
    if (!L.strong || !state || !t0 || !t1) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
    DP_LAUNCH(s, k_strength, nblk(n), kBlock, 0, n, L.rowptr, L.col, L.dpos, L.tpos, L.val,
              o.amg_theta, L.strong, state);
    for (int round = 0; round < 100000; ++round) {
      DP_LAUNCH(s, k_tuple_init, nblk(n), kBlock, 0, n, state, t0);
      DP_LAUNCH(s, k_tuple_max, nblk(n), kBlock, 0, n, L.rowptr, L.col, L.strong, t0, t1);
      DP_LAUNCH(s, k_tuple_max, nblk(n), kBlock, 0, n, L.rowptr, L.col, L.strong, t1, t0);
      DP_CUDA(s, cudaMemsetAsync(s->counter, 0, 4, s->stream));
      DP_LAUNCH(s, k_mis_update, nblk(n), kBlock, 0, n, t0, state, s->counter);
      DP_CUDA(s, cudaMemcpyAsync(s->h_counter, s->counter, 4, cudaMemcpyDeviceToHost, s->stream));
      DP_CUDA(s, cudaStreamSynchronize(s->stream));
      if (s->h_counter[0] == 0) break;
    }
    // aggregates
    phase(s, "mis2", l, tp);
    int *flag = (int *)t1, *pos = (int *)dalloc(s, ((size_t)n + 1) * 4);
    int *a1 = (int *)t0;
    if (!pos) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
    DP_LAUNCH(s, k_root_flag, nblk(n), kBlock, 0, n, state, flag);
    int nagg = 0;
    DP_TRY(scan_i32(s, flag, pos, n, &nagg));
    DP_LAUNCH(s, k_agg_roots, nblk(n), kBlock, 0, n, state, pos, L.agg);
    DP_LAUNCH(s, k_agg_pass1, nblk(n), kBlock, 0, n, L.rowptr, L.col, L.strong, state, L.agg, a1);
    DP_LAUNCH(s, k_agg_pass2, nblk(n), kBlock, 0, n, L.rowptr, L.col, L.strong, a1, L.agg);
    DP_CUDA(s, cudaGetLastError());
    dfree(s, state); dfree(s, t0); dfree(s, t1); dfree(s, pos);
    if (nagg == 0 || nagg >= n) {
      DP_LAUNCH(s, k_fill_i32, nblk(L.n), kBlock, 0, L.agg, L.n, -1);
      break;
    }
    L.nagg = nagg;
    phase(s, "aggregate", l, tp);
    // prolongator pattern
    int *scratch = (int *)dalloc(s, (size_t)std::max(L.nnz, 1) * 4);
    int *cnt = (int *)dalloc(s, ((size_t)n + 1) * 4);
    L.p_rowptr = (int *)dalloc(s, ((size_t)n + 1) * 4);
    L.fdiag = (double *)dalloc(s, (size_t)n * 8);
    if (!scratch || !cnt || !L.p_rowptr || !L.fdiag) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
    DP_LAUNCH(s, k_p_collect, nblk(n), kBlock, 0, n, L.rowptr, L.col, L.strong, L.agg, scratch, cnt);
    DP_TRY(scan_i32(s, cnt, L.p_rowptr, n, &L.p_nnz));
    L.p_col = (int *)dalloc(s, (size_t)std::max(L.p_nnz, 1) * 4);
    L.p_val = (double *)dalloc(s, (size_t)std::max(L.p_nnz, 1) * 8);
    L.p_valf = (float *)dalloc(s, (size_t)std::max(L.p_nnz, 1) * 4);
    if (!L.p_col || !L.p_val || !L.p_valf) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
    DP_LAUNCH(s, k_copy_rows, nblk(n), kBlock, 0, n, L.rowptr, scratch, L.p_rowptr, L.p_col);
    dfree(s, scratch);
    dfree(s, cnt);
    // R = P^T pattern and value map
    int na = nagg;
    int *ccount = (int *)dalloc(s, ((size_t)na + 1) * 4), *fill = (int *)dalloc(s, (size_t)na * 4);
    L.r_rowptr = (int *)dalloc(s, ((size_t)na + 1) * 4);
    L.r_col = (int *)dalloc(s, (size_t)std::max(L.p_nnz, 1) * 4);
    L.r_src = (int *)dalloc(s, (size_t)std::max(L.p_nnz, 1) * 4);
    L.r_val = (double *)dalloc(s, (size_t)std::max(L.p_nnz, 1) * 8);
    L.r_valf = (float *)dalloc(s, (size_t)std::max(L.p_nnz, 1) * 4);
    if (!ccount || !fill || !L.r_rowptr || !L.r_col || !L.r_src || !L.r_val || !L.r_valf) {
      s->fail(DP_ENOMEM, "allocation failed");
      return DP_ENOMEM;
    }
    DP_CUDA(s, cudaMemsetAsync(ccount, 0, (size_t)na * 4, s->stream));
    DP_CUDA(s, cudaMemsetAsync(fill, 0, (size_t)na * 4, s->stream));
    DP_LAUNCH(s, k_col_count, nblk(L.p_nnz), kBlock, 0, L.p_nnz, L.p_col, ccount);
    DP_TRY(scan_i32(s, ccount, L.r_rowptr, na, &L.r_nnz));
    DP_LAUNCH(s, k_transpose_fill, nblk(n), kBlock, 0, n, L.p_rowptr, L.p_col, L.r_rowptr, fill,
              L.r_col, L.r_src);
    DP_LAUNCH(s, k_sort_rows, nblk(na, 64), 64, 0, na, L.r_rowptr, L.r_col, L.r_src);
    dfree(s, ccount);
    dfree(s, fill);
    phase(s, "P, R", l, tp);
    // AP = A P and A_c = R (A P) patterns
    Product pap, prap;
    DP_TRY(spgemm_symbolic(s, n, L.rowptr, L.col, L.p_rowptr, L.p_col, &L.ap_rowptr, &L.ap_col,
                           &L.ap_nnz, &pap));
    L.ap_G = pap.G; L.ap_off = pap.off; L.ap_pos = pap.pos;
    L.ap_val = (double *)dalloc(s, (size_t)std::max(L.ap_nnz, 1) * 8);
    Level N;
    N.n = na;
    N.l1 = l + 1 >= o.amg_gs_levels;
    DP_TRY(spgemm_symbolic(s, na, L.r_rowptr, L.r_col, L.ap_rowptr, L.ap_col, &N.rowptr, &N.col,
                           &N.nnz, &prap));
    L.rap_G = prap.G; L.rap_off = prap.off; L.rap_pos = prap.pos;
    N.dinv = (double *)dalloc(s, (size_t)std::max(na, 1) * 8);
    N.dinvf = (float *)dalloc(s, (size_t)std::max(na, 1) * 4);
    if (!N.dinv || !N.dinvf) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
    L.p_G = lanes_for((double)L.p_nnz / n);
    L.r_G = lanes_for((double)L.p_nnz / na);
    N.val = (double *)dalloc(s, (size_t)std::max(N.nnz, 1) * 8);
    N.valf = (float *)dalloc(s, (size_t)std::max(N.nnz, 1) * 4);
    if (!L.ap_val || !N.val || !N.valf) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
    phase(s, "RAP symbolic", l, tp);
    DP_TRY(level_numeric(s, L, N));
    phase(s, "numeric", l, tp);
    s->lev.push_back(N);
  }
  // level 0 FP32 operator copy
  s->lev[0].valf = (float *)dalloc(s, (size_t)s->lev[0].nnz * 4);
  if (!s->lev[0].valf) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
  DP_TRY(coarse_factor(s));
  DP_TRY(cluster_setup(s));
  s->amg_ready = true;
  return DP_OK;
}

int amg_refresh(Sim *s) {
  DP_TRY(level_dinv(s, s->lev[0]));
  for (size_t l = 0; l + 1 < s->lev.size(); ++l) DP_TRY(level_numeric(s, s->lev[l], s->lev[l + 1]));
  DP_TRY(coarse_factor(s));
  return DP_OK;
}

void amg_free(Sim *s) {
  for (size_t l = 0; l < s->lev.size(); ++l) {
    Level &L = s->lev[l];
    void *ptrs[] = {L.dpos, L.tpos, L.strong, L.agg, L.colour, L.clist, L.fdiag, L.ratio,
                    L.p_rowptr, L.p_col, L.p_val, L.p_valf, L.r_rowptr, L.r_col, L.r_src,
                    L.r_val, L.r_valf, L.ap_rowptr, L.ap_col, L.ap_val, L.x, L.b, L.r,
                    L.xf, L.bf, L.rf, L.valf, L.dinv, L.dinvf, L.ap_off, L.ap_pos, L.rap_off,
                    L.cstart_dev, L.ell_col, L.ell_src, L.ell_off, L.ell_K, L.ell_val,
                    L.ell_valf, L.valh, L.p_valh, L.r_valh,
                    L.rap_pos};
    for (void *p : ptrs) if (p) dfree(s, p);
    if (l > 0) { dfree(s, L.rowptr); dfree(s, L.col); dfree(s, L.val); }
  }
  s->lev.clear();
  s->cl_level = -1;
  if (s->coarse_lu) dfree(s, s->coarse_lu);
  if (s->coarse_piv) dfree(s, s->coarse_piv);
  if (s->coarse_inv) dfree(s, s->coarse_inv);
  s->coarse_inv = nullptr;
  if (s->l0_pv) dfree(s, s->l0_pv);
  if (s->l0_pvf) dfree(s, s->l0_pvf);
  s->l0_pv = nullptr;
  s->l0_pvf = nullptr;
  s->l0_lu = false;
  for (void *p : {(void *)s->l0_colp, (void *)s->r0_colp, (void *)s->p0c_rowptr,
                  (void *)s->p0c_col, (void *)s->p0c_src, (void *)s->p0c_val,
                  (void *)s->p0c_valf, (void *)s->dinv_c, (void *)s->dinv_cf,
                  (void *)s->scolc, (void *)s->z2c})
    if (p) dfree(s, p);
  s->l0_colp = s->r0_colp = s->p0c_rowptr = s->p0c_col = s->p0c_src = s->scolc = nullptr;
  s->z2c = nullptr;
  s->p0c_val = s->dinv_c = nullptr;
  s->p0c_valf = s->dinv_cf = nullptr;
  s->l0c = false;
  s->coarse_lu = nullptr;
  s->coarse_piv = nullptr;
  s->coarse_n = 0;
  s->amg_ready = false;
}

}  // namespace dp
