// Scaled residual norms with no device allocation.
//
// The reduction keeps its per-block partial sums in a file-scope device
// array instead of memory obtained from an allocator.  Every GPU that loads
// the library holds this array (64 KiB) until the process exits.  In host
// code the array's name is only a host-side stand-in for the device object,
// so the device address is looked up once per device with
// cudaGetSymbolAddress and that address is passed to the kernels.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "dpsim.h"

namespace {

constexpr int kThreads = 256;
constexpr int kRowsPerThread = 8;
constexpr int kRowsPerBlock = kThreads * kRowsPerThread;     // 2048 block rows
constexpr int kMaxBlocks = 4096;
constexpr long long kMaxRows = (long long)kMaxBlocks * kRowsPerBlock;  // 8,388,608
constexpr int kMaxDevices = 64;

// Partial sums of the blocks: [block][0] sum of squares, [block][1] maximum.
static __device__ __align__(256) double g_partials[kMaxBlocks * 2];

// Device address of g_partials per device, looked up on the first call with
// that device current and kept until the process exits (a device reset
// invalidates it; the header tells callers not to call after one).
std::mutex g_lock;
double *g_addr[kMaxDevices] = {nullptr};

struct Scale {
  long long nc, nb;
  double V, dt, rho_o_ref, rho_w_ref;
};

// One partial per block of 2048 block rows: cell rows are scaled by
// dt / (rho_ref phi_ref V), well rows by their target (rate wells by at
// least 1e-12); the block's sum of squares and maximum go to its slot.
__global__ void __launch_bounds__(kThreads) k_norms_part_static(
    Scale sc, const double *res, const double *phi_f, const double *phi_m,
    const int32_t *well_kind, const double *well_target, double *partials) {
  double s2 = 0.0, mx = 0.0;
  long long base = (long long)blockIdx.x * kRowsPerBlock;
  for (int t = 0; t < kRowsPerThread; ++t) {
    long long r = base + (long long)t * kThreads + threadIdx.x;
    if (r >= sc.nb) break;
    if (r < sc.nc) {
      long long loc = r >> 1;
      double phi_ref = (r & 1) == 0 ? phi_f[loc] : phi_m[loc];
      for (int al = 0; al < 2; ++al) {
        double rref = al == 0 ? sc.rho_o_ref : sc.rho_w_ref;
        double x = (res[2 * r + al] * sc.dt) / ((rref * phi_ref) * sc.V);
        s2 += x * x;
        mx = fmax(mx, fabs(x));
      }
    } else {
      long long w = r - sc.nc;
      double d = well_kind[w] == 0 ? fmax(well_target[w], 1e-12) : well_target[w];
      double x = res[2 * r] / d;
      s2 += x * x;
      mx = fmax(mx, fabs(x));
    }
  }
  __shared__ double sh[kThreads / 32][2];
  for (int o = 16; o > 0; o >>= 1) {
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sh[wid][0] = s2; sh[wid][1] = mx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) { a += sh[q][0]; b = fmax(b, sh[q][1]); }
    partials[2 * blockIdx.x] = a;
    partials[2 * blockIdx.x + 1] = b;
  }
}

// Sum the partials in block order (deterministic) and write ||.||_2, ||.||_inf.
__global__ void k_norms_final_static(const double *partials, int nblocks, double *out2) {
  __shared__ double sa[32], sb[32];
  int lane = threadIdx.x;
  double a = 0.0, b = 0.0;
  for (int q = lane; q < nblocks; q += 32) { a += partials[2 * q]; b = fmax(b, partials[2 * q + 1]); }
  sa[lane] = a;
  sb[lane] = b;
  __syncwarp();
  if (lane == 0) {
    double s = 0.0, m = 0.0;
    for (int q = 0; q < 32; ++q) { s += sa[q]; m = fmax(m, sb[q]); }
    out2[0] = sqrt(s);
    out2[1] = m;
  }
}

void set_error(char *err, size_t err_len, const char *msg) {
  if (err && err_len) {
    std::strncpy(err, msg, err_len - 1);
    err[err_len - 1] = '\0';
  }
}

}  // namespace

extern "C" int dp_residual_norms_noalloc(const dp_grid *grid, const dp_fluid *fluid,
                                         const double *phi_f, const double *phi_m,
                                         int32_t nwells, const int32_t *well_kind,
                                         const double *well_target, const double *res, double dt,
                                         double *out2, void *stream, char *err, size_t err_len) {
  set_error(err, err_len, "");
  if (!grid || !fluid || !phi_f || !phi_m || !res || !out2 || nwells < 0 ||
      (nwells > 0 && (!well_kind || !well_target)) || !(dt > 0.0) || grid->nx < 1 ||
      grid->ny < 1 || grid->nz < 1) {
    set_error(err, err_len, "dp_residual_norms_noalloc: invalid argument");
    return DP_EINVAL;
  }
  long long nc = 2LL * grid->nx * grid->ny * grid->nz;
  long long nb = nc + nwells;
  if (nb > kMaxRows) {
    char msg[160];
    std::snprintf(msg, sizeof msg,
                  "dp_residual_norms_noalloc: %lld block rows exceed the static scratch limit of "
                  "%lld block rows",
                  nb, kMaxRows);
    set_error(err, err_len, msg);
    return DP_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_error(err, err_len, "dp_residual_norms_noalloc: no usable current device");
    return DP_ECUDA;
  }
  double *partials = nullptr;
  {
    std::lock_guard<std::mutex> g(g_lock);
    if (!g_addr[dev]) {
      void *p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_partials);
      if (e != cudaSuccess) {
        set_error(err, err_len, cudaGetErrorString(e));
        return DP_ECUDA;
      }
      g_addr[dev] = static_cast<double *>(p);
    }
    partials = g_addr[dev];
  }
  Scale sc;
  sc.nc = nc;
  sc.nb = nb;
  sc.V = (grid->dx * grid->dy) * grid->dz;
  sc.dt = dt;
  sc.rho_o_ref = fluid->rho_o_ref;
  sc.rho_w_ref = fluid->rho_w_ref;
  int nblocks = (int)((nb + kRowsPerBlock - 1) / kRowsPerBlock);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_norms_part_static<<<nblocks, kThreads, 0, st>>>(sc, res, phi_f, phi_m, well_kind, well_target,
                                                     partials);
  k_norms_final_static<<<1, 32, 0, st>>>(partials, nblocks, out2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(err, err_len, cudaGetErrorString(e));
    return DP_ECUDA;
  }
  return DP_OK;
}
