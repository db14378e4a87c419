// C ABI of the dpsim library (include/dpsim.h): realisation set-up, state
// transfer, assembly, the Newton-step solve and the timestep driver of
// Algorithm 1.  Host code only orchestrates; every numerical step runs in
// the library's kernels on the caller's stream.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "dp_internal.h"


namespace dp {

// NVTX range around a stage of the solve (visible in Nsight timelines; a
// no-op unless a tool is attached).
struct Range {
  explicit Range(const char *name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

// ---------------------------------------------------------------- memory
static void *default_alloc(size_t bytes, void *stream, void *) {
  void *p = nullptr;
  if (cudaMallocAsync(&p, bytes, (cudaStream_t)stream) != cudaSuccess) return nullptr;
  return p;
}
static void default_free(void *p, size_t, void *stream, void *) {
  cudaFreeAsync(p, (cudaStream_t)stream);
}

void *dalloc(Sim *s, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~(size_t)255;
  void *p = s->alloc.alloc(bytes, (void *)s->stream, s->alloc.ctx);
  if (p) {
    s->blocks.push_back({p, bytes});
    s->cur_bytes += bytes;
    s->peak_bytes = std::max(s->peak_bytes, s->cur_bytes);
  } else {
    s->alloc_failed = true;
    s->last_error = "the device allocator returned NULL";
  }
  return p;
}

void dfree(Sim *s, void *p) {
  if (!p) return;
  for (size_t i = 0; i < s->blocks.size(); ++i)
    if (s->blocks[i].first == p) {
      s->alloc.free(p, s->blocks[i].second, (void *)s->stream, s->alloc.ctx);
      s->cur_bytes -= s->blocks[i].second;
      s->blocks[i] = s->blocks.back();
      s->blocks.pop_back();
      return;
    }
}

// ---------------------------------------------------------------- launches
LaunchScope::LaunchScope(Sim *sim, const char *name) : s(sim), timed(false) {
  ++s->launches;
  Timing &t = s->timing;
  if (t.kernel_id >= 0 && std::strstr(name, t.name.c_str())) {
    if (t.used + 2 > t.ev.size()) {
      for (int k = 0; k < 64; ++k) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        t.ev.push_back(e);
      }
    }
    cudaEventRecord(t.ev[t.used], s->stream);
    timed = true;
  }
}

LaunchScope::~LaunchScope() {
  if (!timed) return;
  Timing &t = s->timing;
  cudaEventRecord(t.ev[t.used + 1], s->stream);
  t.used += 2;
  t.launches += 1;
}

// Event pairs are taken the same way for a region; its count is the number
// of regions timed.
RegionScope::RegionScope(Sim *sim, const char *name) : s(sim), timed(false) {
  Timing &t = s->timing;
  if (t.kernel_id < 0 || t.name != name) return;
  if (t.used + 2 > t.ev.size()) {
    for (int k = 0; k < 64; ++k) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      t.ev.push_back(e);
    }
  }
  cudaEventRecord(t.ev[t.used], s->stream);
  timed = true;
}

RegionScope::~RegionScope() {
  if (!timed) return;
  Timing &t = s->timing;
  cudaEventRecord(t.ev[t.used + 1], s->stream);
  t.used += 2;
  t.launches += 1;
}

int pdl_mode() {
  static const int mode = [] {
    const char *v = std::getenv("DPSIM_PDL");
    char *end = nullptr;
    long m = v ? std::strtol(v, &end, 10) : -1;
    return v && *v && end && !*end && m >= 0 && m <= 31 ? (int)m : 31;
  }();
  return mode;
}

// A realisation whose allocator failed, or that met a CUDA failure, does no
// further work.
static int unusable(Sim *s) {
  if (s->err.code) return s->err.code;
  return s->alloc_failed ? DP_ENOMEM : DP_OK;
}

static int check(Sim *s) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { s->fail(DP_ECUDA, cudaGetErrorString(e)); return DP_ECUDA; }
  if (s->err.code) return s->err.code;
  return s->alloc_failed ? DP_ENOMEM : DP_OK;
}

// Reads and clears the flag of the kernels with bounded device waits (after
// they ran): DP_ETIMEOUT when one of their waits gave up.
int device_waits(Sim *s) {
  if (!s->waits_used || !s->dev_err) return DP_OK;
  s->waits_used = false;
  int h = 0;
  DP_CUDA(s, cudaMemcpyAsync(&h, s->dev_err, 4, cudaMemcpyDeviceToHost, s->stream));
  DP_CUDA(s, cudaStreamSynchronize(s->stream));
  if (h) {
    s->fail(DP_ETIMEOUT, "a bounded device-side wait gave up (a bulk copy did not land)");
    return DP_ETIMEOUT;
  }
  return DP_OK;
}

// Forcing term of Algorithm 1 (Section 3.1): fixed, or one of the three
// formulas clipped to [eta_min, eta_max]; eta_max on the first iteration.
// With b = -R and the previous solve's linear residual r^{l-1} = -lq
// (lq = R + A y), in the scaled norm of ||b||: 1 takes ||b(x^l) - r^{l-1}||
// = ||R~(R - lq)|| (last_norms[9]), 2 takes ||r^{l-1}|| = ||R~(lq)||
// (last_norms[8]), 3 the ratio of residual norms alone.
static double forcing(Sim *s, double res) {
  const dp_options &o = s->opt;
  if (o.eta_mode == 0) return o.eta_fixed;
  if (s->newton_iter == 0 || s->prev_res <= 0.0) return o.eta_max;
  double eta;
  if (o.eta_mode == 1) eta = s->last_norms[9] / s->prev_res;
  else if (o.eta_mode == 2) eta = (res - s->last_norms[8]) / s->prev_res;
  else eta = o.eta_gamma * std::pow(res / s->prev_res, o.eta_beta);
  return std::min(std::max(eta, o.eta_min), o.eta_max);
}

static int read_norms(Sim *s) {
  DP_CUDA(s, cudaMemcpyAsync(s->h_norms, s->norm_out, 80, cudaMemcpyDeviceToHost, s->stream));
  DP_CUDA(s, cudaStreamSynchronize(s->stream));
  std::memcpy(s->last_norms, s->h_norms, 80);
  return DP_OK;
}

}  // namespace dp

using namespace dp;

static bool bad_opts(const dp_options *o) {
  return !o || o->gmres_restart < 1 || o->gmres_maxit < 1 || o->newton_max < 0 ||
         o->amg_coarse_max < 1 || o->amg_max_levels < 1 || o->precond < 0 || o->precond > 2 ||
         o->precision < 0 || o->precision > 2 || !(o->ds_max > 0.0) || o->amg_gs_levels < 0 ||
         o->amg_refresh < 0 || o->amg_refresh > 1 || o->decouple < 0 || o->decouple > 2 ||
         o->schur < 0 || o->schur > 1 || !(o->reorth >= 0.0) || !std::isfinite(o->reorth);
}

extern "C" int sim_create(const dp_grid *grid, const dp_rock *rock, const dp_fluid *fluid,
                          const dp_well *wells, int32_t nwells, const dp_options *opts,
                          const dp_allocator *alloc, void *stream, dp_sim **out) {
  if (!out) return DP_EINVAL;
  *out = nullptr;
  if (!grid || !rock || !fluid || nwells < 0 || (nwells > 0 && !wells) || bad_opts(opts))
    return DP_EINVAL;
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || !(grid->dx > 0) || !(grid->dy > 0) ||
      !(grid->dz > 0))
    return DP_EINVAL;
  long long nL = (long long)grid->nx * grid->ny * grid->nz;
  if (2 * nL + nwells >= (1LL << 29)) return DP_EINVAL;   // 30-bit row indices in MIS(2)
  if (!rock->kf || !rock->km || !rock->phi_f || !rock->phi_m) return DP_EINVAL;
  for (int w = 0; w < nwells; ++w) {
    const dp_well &W = wells[w];
    if (W.kind < 0 || W.kind > 2 || W.i < 0 || W.i >= grid->nx || W.j < 0 || W.j >= grid->ny ||
        W.k_top < 0 || W.k_bot >= grid->nz || W.k_top > W.k_bot || !(W.rw > 0.0) ||
        !(W.limit >= 0.0) || !(W.wi >= 0.0) || !std::isfinite(W.limit) || !std::isfinite(W.wi))
      return DP_EINVAL;
  }
  for (int k = 0; k < 2; ++k) {
    int n = fluid->pc_n[k];
    if (n < 0 || n > 256 || (n > 0 && !fluid->pc_table[k])) return DP_EINVAL;
    for (int i = 0; i < n; ++i) {
      const double *t = fluid->pc_table[k];
      if (!std::isfinite(t[2 * i]) || !std::isfinite(t[2 * i + 1])) return DP_EINVAL;
      if (i > 0 && !(t[2 * i] > t[2 * i - 2])) return DP_EINVAL;
    }
  }
  dp_sim *s = new (std::nothrow) dp_sim();
  if (!s) return DP_ENOMEM;
  s->opt = *opts;
  s->stream = (cudaStream_t)stream;
  if (alloc && alloc->alloc && alloc->free) { s->alloc = *alloc; s->own_alloc = false; }
  else { s->alloc.alloc = default_alloc; s->alloc.free = default_free; s->alloc.ctx = nullptr; }
  s->wells.assign(wells, wells + nwells);
  Phys &P = s->ph;
  P.nx = grid->nx; P.ny = grid->ny; P.nz = grid->nz;
  P.nL = (int)nL; P.nc = 2 * P.nL; P.nw = nwells; P.nb = P.nc + nwells;
  P.dx = grid->dx; P.dy = grid->dy; P.dz = grid->dz; P.top_depth = grid->top_depth;
  P.V = (grid->dx * grid->dy) * grid->dz;
  P.mu_o = fluid->mu_o; P.mu_w = fluid->mu_w; P.c_o = fluid->c_o; P.c_w = fluid->c_w;
  P.rho_o_ref = fluid->rho_o_ref; P.rho_w_ref = fluid->rho_w_ref; P.p_ref = fluid->p_ref;
  P.swc = fluid->swc; P.sor = fluid->sor; P.g = fluid->g;
  P.inv_span = 1.0 / ((1.0 - fluid->swc) - fluid->sor);
  P.inv_mu_o = 1.0 / fluid->mu_o;
  P.inv_mu_w = 1.0 / fluid->mu_w;
  P.sigma = rock->sigma; P.c_rock = rock->c_rock; P.p_ref_rock = rock->p_ref;
  P.drho_o = fluid->rho_o_ref * fluid->c_o;   // the products props() forms, once
  P.drho_w = fluid->rho_w_ref * fluid->c_w;
  auto fail = [&](int rc) { sim_destroy(s); return rc; };
  for (int k = 0; k < 2; ++k) {
    P.pc_n[k] = fluid->pc_n[k];
    P.pc_tab[k] = nullptr;
    if (P.pc_n[k] == 0) continue;
    size_t bytes = (size_t)P.pc_n[k] * 16;
    double *t = (double *)dalloc(s, bytes);
    if (!t) return fail(DP_ENOMEM);
    if (cudaMemcpyAsync(t, fluid->pc_table[k], bytes, cudaMemcpyHostToDevice, s->stream) !=
        cudaSuccess)
      return fail(DP_ECUDA);
    P.pc_tab[k] = t;
  }
  size_t nl8 = (size_t)P.nL * 8;
  s->kf = (double *)dalloc(s, nl8);
  s->km = (double *)dalloc(s, nl8);
  s->phi_f = (double *)dalloc(s, nl8);
  s->phi_m = (double *)dalloc(s, nl8);
  s->well_kind = (int *)dalloc(s, (size_t)std::max(nwells, 1) * 4);
  s->well_target = (double *)dalloc(s, (size_t)std::max(nwells, 1) * 8);
  s->well_ctl_kind = (int *)dalloc(s, (size_t)std::max(nwells, 1) * 4);
  s->well_ctl_target = (double *)dalloc(s, (size_t)std::max(nwells, 1) * 8);
  s->well_limit = (double *)dalloc(s, (size_t)std::max(nwells, 1) * 8);
  s->counter = (int *)dalloc(s, 64);
  s->omega = (double *)dalloc(s, 8);
  s->rho_bits = (unsigned long long *)dalloc(s, 8);
  if (!s->kf || !s->km || !s->phi_f || !s->phi_m || !s->well_kind || !s->well_target ||
      !s->well_ctl_kind || !s->well_ctl_target || !s->well_limit ||
      !s->counter || !s->omega || !s->rho_bits)
    return fail(DP_ENOMEM);
  if (cudaMallocHost(&s->h_counter, 64) != cudaSuccess ||
      cudaMallocHost(&s->h_res, 64) != cudaSuccess || cudaMallocHost(&s->h_norms, 128) != cudaSuccess)
    return fail(DP_ECUDA);
  cudaStream_t st = s->stream;
  if (cudaMemcpyAsync(s->kf, rock->kf, nl8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(s->km, rock->km, nl8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(s->phi_f, rock->phi_f, nl8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(s->phi_m, rock->phi_m, nl8, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return fail(DP_ECUDA);
  std::vector<int> kinds(std::max(nwells, 1), 0);
  std::vector<double> targets(std::max(nwells, 1), 0.0), limits(std::max(nwells, 1), 0.0);
  for (int w = 0; w < nwells; ++w) {
    kinds[w] = wells[w].kind; targets[w] = wells[w].target;
    limits[w] = wells[w].kind == DP_WELL_BHP ? 0.0 : wells[w].limit;
    if (limits[w] > 0.0) s->well_limits = true;
  }
  if (cudaMemcpyAsync(s->well_kind, kinds.data(), kinds.size() * 4, cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(s->well_target, targets.data(), targets.size() * 8, cudaMemcpyHostToDevice,
                      st) != cudaSuccess ||
      cudaMemcpyAsync(s->well_ctl_kind, kinds.data(), kinds.size() * 4, cudaMemcpyHostToDevice,
                      st) != cudaSuccess ||
      cudaMemcpyAsync(s->well_ctl_target, targets.data(), targets.size() * 8,
                      cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(s->well_limit, limits.data(), limits.size() * 8, cudaMemcpyHostToDevice,
                      st) != cudaSuccess ||
      cudaMemsetAsync(s->counter, 0, 64, st) != cudaSuccess)
    return fail(DP_ECUDA);
  int rc = phys_build_pattern(s);
  if (rc) return fail(rc);
  size_t nc8 = (size_t)P.nc * 8, nw8 = (size_t)std::max(nwells, 1) * 8, nb16 = (size_t)P.nb * 16;
  s->p = (double *)dalloc(s, nc8); s->sw = (double *)dalloc(s, nc8);
  s->bhp = (double *)dalloc(s, nw8);
  s->pn = (double *)dalloc(s, nc8); s->swn = (double *)dalloc(s, nc8);
  s->bhpn = (double *)dalloc(s, nw8);
  s->Mn = (double *)dalloc(s, 2 * nc8);
  s->R = (double *)dalloc(s, nb16); s->bh = (double *)dalloc(s, nb16);
  s->y = (double *)dalloc(s, nb16);
  s->pr = (double *)dalloc(s, 8 * nc8);
  s->Macc = (double *)dalloc(s, 2 * nc8);
  s->norm_blocks = std::min(nblk(P.nb), 1024);
  s->norm_part = (double *)dalloc(s, (size_t)s->norm_blocks * 64);
  s->norm_out = (double *)dalloc(s, 80);
  s->dev_err = (int *)dalloc(s, 64);   // [0] the wait flag, [4..5] the grid barrier's counts
  s->tickets = (unsigned *)dalloc(s, (size_t)kTicketWords * 4);
  s->norm_w = (double *)dalloc(s, 2 * nc8);
  if (!s->p || !s->sw || !s->bhp || !s->pn || !s->swn || !s->bhpn || !s->Mn || !s->R || !s->bh ||
      !s->y || !s->norm_part || !s->norm_out || !s->norm_w || !s->pr || !s->Macc || !s->dev_err ||
      !s->tickets)
    return fail(DP_ENOMEM);
  if ((rc = phys_norm_weights(s))) return fail(rc);
  cudaMemsetAsync(s->p, 0, nc8, st); cudaMemsetAsync(s->sw, 0, nc8, st);
  cudaMemsetAsync(s->bhp, 0, nw8, st); cudaMemsetAsync(s->Mn, 0, 2 * nc8, st);
  cudaMemsetAsync(s->y, 0, nb16, st); cudaMemsetAsync(s->dev_err, 0, 64, st);
  cudaMemsetAsync(s->tickets, 0, (size_t)kTicketWords * 4, st);
  if ((rc = phys_solver_view(s))) return fail(rc);
  if ((rc = ilu_setup(s))) return fail(rc);
  if ((rc = la_alloc(s))) return fail(rc);
  if (cudaStreamSynchronize(st) != cudaSuccess) return fail(DP_ECUDA);
  if ((rc = check(s))) return fail(rc);
  *out = s;
  return DP_OK;
}

extern "C" void sim_destroy(dp_sim *s) {
  if (!s) return;
  cudaStreamSynchronize(s->stream);
  graphs_free(s);
  if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
  amg_free(s);
  while (!s->blocks.empty()) dfree(s, s->blocks.back().first);
  for (cudaEvent_t e : s->timing.ev) cudaEventDestroy(e);
  if (s->h_counter) cudaFreeHost(s->h_counter);
  if (s->h_res) cudaFreeHost(s->h_res);
  if (s->h_norms) cudaFreeHost(s->h_norms);
  cudaStreamSynchronize(s->stream);
  delete s;
}

extern "C" int sim_sizes(const dp_sim *s, int32_t *nb, int32_t *nnzb, int32_t *ncells,
                         int32_t *nwells) {
  if (!s) return DP_EINVAL;
  if (nb) *nb = s->ph.nb;
  if (nnzb) *nnzb = s->A.nnz;
  if (ncells) *ncells = s->ph.nc;
  if (nwells) *nwells = s->ph.nw;
  return DP_OK;
}

static int copy_state(dp_sim *s, const double *p, const double *sw, const double *bhp,
                      cudaMemcpyKind kind) {
  if (!s || !p || !sw || (s->ph.nw > 0 && !bhp)) return DP_EINVAL;
  DP_CUDA(s, cudaMemcpyAsync(s->p, p, (size_t)s->ph.nc * 8, kind, s->stream));
  DP_CUDA(s, cudaMemcpyAsync(s->sw, sw, (size_t)s->ph.nc * 8, kind, s->stream));
  if (s->ph.nw) DP_CUDA(s, cudaMemcpyAsync(s->bhp, bhp, (size_t)s->ph.nw * 8, kind, s->stream));
  s->assembled = s->decoupled = false;
  return DP_OK;
}

namespace dp {

// A new old time level starts a new timestep of Algorithm 1: the Newton
// counters that the forcing terms use start again.
void new_timestep(Sim *s) {
  s->newton_iter = 0;
  s->prev_res = 0.0;
  s->have_lq = false;
}

// The start of a timestep: the wells back on their own controls, x^n saved,
// the Newton counters reset.
int timestep_begin(Sim *s) {
  if (s->well_limits) DP_TRY(phys_well_controls(s, true));
  DP_TRY(phys_save_old(s));
  new_timestep(s);
  return DP_OK;
}

// The old time level copied back into the iterate (a failed timestep).
int timestep_restore(Sim *s) {
  size_t nc8 = (size_t)s->ph.nc * 8;
  DP_CUDA(s, cudaMemcpyAsync(s->p, s->pn, nc8, cudaMemcpyDeviceToDevice, s->stream));
  DP_CUDA(s, cudaMemcpyAsync(s->sw, s->swn, nc8, cudaMemcpyDeviceToDevice, s->stream));
  if (s->ph.nw)
    DP_CUDA(s, cudaMemcpyAsync(s->bhp, s->bhpn, (size_t)s->ph.nw * 8, cudaMemcpyDeviceToDevice,
                               s->stream));
  return DP_OK;
}

}  // namespace dp

extern "C" int sim_set_state(dp_sim *s, const double *p, const double *sw, const double *bhp) {
  DP_TRY(copy_state(s, p, sw, bhp, cudaMemcpyDefault));
  DP_TRY(phys_save_old(s));
  new_timestep(s);
  return check(s);
}

extern "C" int sim_set_state_device(dp_sim *s, const double *p, const double *sw,
                                    const double *bhp) {
  DP_TRY(copy_state(s, p, sw, bhp, cudaMemcpyDeviceToDevice));
  DP_TRY(phys_save_old(s));
  new_timestep(s);
  return check(s);
}

extern "C" int sim_set_iterate(dp_sim *s, const double *p, const double *sw, const double *bhp) {
  DP_TRY(copy_state(s, p, sw, bhp, cudaMemcpyDefault));
  return check(s);
}

extern "C" int sim_get_state(dp_sim *s, double *p, double *sw, double *bhp) {
  if (!s || !p || !sw || (s->ph.nw > 0 && !bhp)) return DP_EINVAL;
  DP_CUDA(s, cudaMemcpyAsync(p, s->p, (size_t)s->ph.nc * 8, cudaMemcpyDefault, s->stream));
  DP_CUDA(s, cudaMemcpyAsync(sw, s->sw, (size_t)s->ph.nc * 8, cudaMemcpyDefault, s->stream));
  if (s->ph.nw)
    DP_CUDA(s, cudaMemcpyAsync(bhp, s->bhp, (size_t)s->ph.nw * 8, cudaMemcpyDefault, s->stream));
  DP_CUDA(s, cudaStreamSynchronize(s->stream));
  return check(s);
}

extern "C" int sim_assemble(dp_sim *s, double dt) {
  Range range("assemble");
  if (!s || !(dt > 0.0)) return DP_EINVAL;
  DP_TRY(unusable(s));
  s->dt = dt;
  s->inv_dt = 1.0 / dt;
  DP_TRY(phys_assemble(s));
  DP_TRY(phys_norms(s));
  s->assembled = true;
  s->decoupled = false;
  return check(s);
}

extern "C" int sim_get_jacobian(dp_sim *s, int32_t *rowptr, int32_t *col, double *val,
                                double *res) {
  if (!s) return DP_EINVAL;
  if (rowptr)
    DP_CUDA(s, cudaMemcpyAsync(rowptr, s->A.rowptr, ((size_t)s->A.n + 1) * 4, cudaMemcpyDefault,
                               s->stream));
  if (col)
    DP_CUDA(s, cudaMemcpyAsync(col, s->A.col, (size_t)s->A.nnz * 4, cudaMemcpyDefault, s->stream));
  if (val)
    DP_CUDA(s, cudaMemcpyAsync(val, s->A.val, (size_t)s->A.nnz * 32, cudaMemcpyDefault, s->stream));
  if (res)
    DP_CUDA(s, cudaMemcpyAsync(res, s->R, (size_t)s->A.n * 16, cudaMemcpyDefault, s->stream));
  DP_CUDA(s, cudaStreamSynchronize(s->stream));
  return check(s);
}

extern "C" int sim_get_norms(dp_sim *s, double *out8) {
  if (!s || !out8) return DP_EINVAL;
  DP_TRY(read_norms(s));
  std::memcpy(out8, s->last_norms, 64);
  return DP_OK;
}

namespace dp {

// The first part of a linear solve of Algorithm 1 at the assembled iterate:
// the forcing term, the decoupling (with the Schur option, the reduction
// first), the ILU(0) factorisation and the AMG set-up or value refresh.
int solve_prepare(Sim *s, double *eta, bool norms_current) {
  if (!norms_current) DP_TRY(read_norms(s));
  *eta = forcing(s, s->last_norms[0]);
  {
    Range range("decouple");
    if (s->opt.schur) DP_TRY(phys_schur_reduce(s));
    DP_TRY(phys_decouple_extract(s));
  }
  s->decoupled = true;
  if (s->opt.precond >= 1) {
    Range range("ilu_factor");
    DP_TRY(ilu_factor(s));
  }
  if (s->opt.precond == 2) {
    Range range("amg");
    bool coarse = !s->amg_ready || s->opt.amg_refresh == 0 || s->newton_iter == 0;
    if (!s->amg_ready) DP_TRY(amg_setup(s));
    else if (coarse) DP_TRY(amg_refresh(s));
    else DP_TRY(level_dinv(s, s->lev[0]));   // level 0 only: its values are s->ap
    if (s->opt.precision >= 1) DP_TRY(mixed_refresh(s, coarse));
    DP_TRY(l0_refresh(s, coarse));
    if (coarse) DP_TRY(cluster_refresh(s));
  }
  return DP_OK;
}

// After FGMRES returned rc (DP_OK or DP_ELINEAR) with `it` iterations and
// relative residual rr: the update (none after DP_ELINEAR), the linear
// residual of the forcing terms 1-2, stream-ordered.
int solve_update(Sim *s, int rc) {
  if (rc != DP_OK) return DP_OK;
  if (s->opt.schur) DP_TRY(phys_schur_back(s));
  if (s->opt.eta_mode == 1 || s->opt.eta_mode == 2) {
    if (!s->lq) s->lq = (double *)dalloc(s, (size_t)s->ph.nb * 16);
    if (!s->lq) { s->fail(DP_ENOMEM, "allocation of the linear residual failed"); return DP_ENOMEM; }
    DP_TRY(lin_residual(s));
  }
  return phys_update(s);
}

// The bookkeeping of a finished solve (after the stream has synchronised):
// statistics, and on success the Newton counters of the forcing terms.
int solve_finish(Sim *s, int rc, int it, double rr, double eta, float ms_setup, float ms_solve,
                 dp_stats *st) {
  s->assembled = false;
  dp_stats &L = s->last;
  L.linear_iters = it; L.lin_relres = rr; L.eta = eta;
  L.amg_levels = (int)s->lev.size(); L.converged = rc == DP_OK;
  L.ms_setup = ms_setup; L.ms_solve = ms_solve;
  if (st) *st = L;
  DP_TRY(device_waits(s));
  if (rc == DP_ELINEAR) {
    s->fail(DP_ELINEAR, "FGMRES did not reach the forcing term; no update was made");
    DP_TRY(check(s));
    return DP_ELINEAR;
  }
  s->prev_res = s->last_norms[0];
  s->have_lq = s->opt.eta_mode == 1 || s->opt.eta_mode == 2;
  s->newton_iter++;
  DP_TRY(check(s));
  return DP_OK;
}

}  // namespace dp

extern "C" int sim_solve_step(dp_sim *s, dp_stats *st) {
  if (!s) return DP_EINVAL;
  DP_TRY(unusable(s));
  if (!s->assembled) { s->fail(DP_EINVAL, "sim_solve_step before sim_assemble"); return DP_EINVAL; }
  cudaEvent_t e0, e1, e2;
  cudaEventCreate(&e0); cudaEventCreate(&e1); cudaEventCreate(&e2);
  cudaEventRecord(e0, s->stream);
  double eta = 0.0;
  int rc = solve_prepare(s, &eta);
  cudaEventRecord(e1, s->stream);
  int it = 0;
  double rr = 0.0;
  if (rc == DP_OK) {
    Range range("fgmres");
    rc = fgmres(s, eta, &it, &rr);
  }
  if (rc == DP_OK || rc == DP_ELINEAR) {
    int ru = solve_update(s, rc);
    if (ru != DP_OK) rc = ru;
  }
  cudaEventRecord(e2, s->stream);
  cudaError_t se = cudaStreamSynchronize(s->stream);
  float ms1 = 0.f, ms2 = 0.f;
  cudaEventElapsedTime(&ms1, e0, e1);
  cudaEventElapsedTime(&ms2, e1, e2);
  cudaEventDestroy(e0); cudaEventDestroy(e1); cudaEventDestroy(e2);
  DP_CUDA(s, se);
  if (rc != DP_OK && rc != DP_ELINEAR) return rc;
  return solve_finish(s, rc, it, rr, eta, ms1, ms2, st);
}

extern "C" int sim_advance(dp_sim *s, double dt, dp_stats *st) {
  if (!s || !(dt > 0.0)) return DP_EINVAL;
  DP_TRY(unusable(s));
  Range range("timestep");
  DP_TRY(timestep_begin(s));
  int lin = 0;
  bool conv = false, lin_fail = false;
  double res0 = 0.0, res = 0.0, ms_setup = 0.0, ms_solve = 0.0;
  for (int l = 0; l <= s->opt.newton_max; ++l) {
    DP_TRY(sim_assemble(s, dt));
    DP_TRY(read_norms(s));
    res = s->last_norms[0];
    if (l == 0) res0 = res;
    if (res <= s->opt.newton_tol * res0 || s->last_norms[1] <= s->opt.newton_atol) { conv = true; break; }
    if (l == s->opt.newton_max) break;
    dp_stats ls{};
    int rc = sim_solve_step(s, &ls);
    if (rc != DP_OK && rc != DP_ELINEAR) return rc;
    lin += ls.linear_iters;
    ms_setup += ls.ms_setup;
    ms_solve += ls.ms_solve;
    if (rc == DP_ELINEAR) { lin_fail = true; break; }
    if (s->well_limits) DP_TRY(phys_well_controls(s, false));
  }
  dp_stats &L = s->last;
  L.newton_iters = s->newton_iter; L.linear_iters = lin; L.converged = conv;
  L.res0 = res0; L.res = res; L.amg_levels = (int)s->lev.size();
  L.ms_setup = ms_setup; L.ms_solve = ms_solve;
  if (st) *st = L;
  if (!conv) {
    DP_TRY(timestep_restore(s));
    DP_CUDA(s, cudaStreamSynchronize(s->stream));
    if (lin_fail) {
      s->fail(DP_ELINEAR, "a linear solve did not reach its forcing term; the old state is restored");
      return DP_ELINEAR;
    }
    s->fail(DP_ENEWTON, "Newton did not converge");
    return DP_ENEWTON;
  }
  return check(s);
}

extern "C" int sim_run(dp_sim *s, double t_end, double dt0, double dt_max, double dt_min,
                       int32_t max_steps, dp_run_stats *st) {
  dp_run_stats r{};
  if (!s || !(t_end > 0.0) || !(dt0 > 0.0) || !(dt_max >= dt0) || !(dt_min > 0.0) ||
      max_steps < 1)
    return DP_EINVAL;
  double t = 0.0, dt = dt0;
  int rc = DP_OK;
  while (t_end - t > 1e-9 * t_end) {
    if (r.steps >= max_steps) { rc = DP_ENEWTON; break; }
    double h = dt < t_end - t ? dt : t_end - t;
    dp_stats a{};
    int rc1 = sim_advance(s, h, &a);
    if (rc1 == DP_ENEWTON || rc1 == DP_ELINEAR) {   // rolled back: retry at half the step
      r.cuts += 1;
      dt = 0.5 * h;
      if (dt < dt_min) { rc = DP_ENEWTON; break; }
      continue;
    }
    if (rc1 != DP_OK) { rc = rc1; break; }
    t = t + h;
    r.steps += 1;
    r.newton_iters += a.newton_iters;
    r.linear_iters += a.linear_iters;
    dt = 2.0 * h < dt_max ? 2.0 * h : dt_max;
  }
  r.t = t;
  if (st) *st = r;
  if (rc == DP_ENEWTON) s->fail(DP_ENEWTON, "sim_run: timestep below dt_min or step limit");
  return rc;
}

extern "C" int dp_stream_create(void **stream) {
  if (!stream) return DP_EINVAL;
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    *stream = nullptr;
    return DP_ECUDA;
  }
  *stream = (void *)st;
  return DP_OK;
}

extern "C" int dp_stream_destroy(void *stream) {
  if (!stream) return DP_EINVAL;
  return cudaStreamDestroy((cudaStream_t)stream) == cudaSuccess ? DP_OK : DP_ECUDA;
}

extern "C" int sim_solver_sizes(dp_sim *s, int32_t *nb, int32_t *nnzb) {
  if (!s) return DP_EINVAL;
  if (nb) *nb = s->K.n;
  if (nnzb) *nnzb = s->K.nnz;
  return DP_OK;
}

extern "C" int sim_set_l0_kernel(dp_sim *s, int32_t variant) {
  if (!s || variant < -4 || variant > 8 || (variant > 2 && variant != 4 && variant != 8))
    return DP_EINVAL;
  DP_TRY(unusable(s));
  if (s->l0_G != variant) {
    s->l0_G = variant;
    graphs_free(s);   // the Arnoldi steps are captured again
    ++s->shapes;      // and a batch holding this realisation rebuilds its plan
  }
  return DP_OK;
}

extern "C" int sim_autotune(dp_sim *s, int32_t reps, char *report, int32_t report_len) {
  if (!s || reps < 1 || (report && report_len < 1)) return DP_EINVAL;
  DP_TRY(unusable(s));
  std::string rep;
  DP_TRY(autotune(s, reps, rep));
  DP_TRY(device_waits(s));
  if (report) {
    size_t n = std::min(rep.size(), (size_t)report_len - 1);
    std::memcpy(report, rep.data(), n);
    report[n] = 0;
  }
  return DP_OK;
}

extern "C" int sim_footprint(dp_sim *s, uint64_t *current, uint64_t *peak) {
  if (!s) return DP_EINVAL;
  if (current) *current = s->cur_bytes;
  if (peak) *peak = s->peak_bytes;
  return DP_OK;
}

extern "C" int sim_advance_many(dp_sim *const *sims, int32_t n, const double *dt, int32_t threads,
                                dp_stats *stats, int32_t *status) {
  if (n < 0 || (n > 0 && (!sims || !dt))) return DP_EINVAL;
  for (int k = 0; k < n; ++k) {
    if (!sims[k] || !(dt[k] > 0.0)) return DP_EINVAL;
    for (int q = 0; q < k; ++q)
      if (sims[q] == sims[k]) return DP_EINVAL;
  }
  int nt = threads > 0 ? threads : std::min<int>(n, 16);
  nt = std::max(1, std::min(nt, n));
  std::vector<int> rc(n, DP_OK);
  std::atomic<int> next{0};
  auto worker = [&]() {
    for (;;) {
      int k = next.fetch_add(1);
      if (k >= n) return;
      dp_stats st{};
      rc[k] = sim_advance(sims[k], dt[k], &st);
      if (stats) stats[k] = st;
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
  worker();
  for (auto &th : pool) th.join();
  int first = DP_OK;
  for (int k = 0; k < n; ++k) {
    if (status) status[k] = rc[k];
    if (first == DP_OK && rc[k] != DP_OK) first = rc[k];
  }
  return first;
}

extern "C" int sim_get_update(dp_sim *s, double *y) {
  if (!s || !y) return DP_EINVAL;
  DP_CUDA(s, cudaMemcpyAsync(y, s->y, (size_t)s->A.n * 16, cudaMemcpyDefault, s->stream));
  DP_CUDA(s, cudaStreamSynchronize(s->stream));
  return check(s);
}

extern "C" int sim_get_decoupled(dp_sim *s, double *val, double *rhs) {
  if (!s) return DP_EINVAL;
  if (!s->decoupled) { s->fail(DP_EINVAL, "no decoupled system yet"); return DP_EINVAL; }
  if (val) {
    double *tmp = (double *)dalloc(s, (size_t)s->K.nnz * 32);
    if (!tmp) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
    int rc = phys_decoupled_natural(s, tmp);
    if (rc == DP_OK &&
        cudaMemcpyAsync(val, tmp, (size_t)s->K.nnz * 32, cudaMemcpyDefault, s->stream) != cudaSuccess)
      rc = DP_ECUDA;
    cudaStreamSynchronize(s->stream);
    dfree(s, tmp);
    if (rc != DP_OK) { s->fail(rc, "sim_get_decoupled"); return rc; }
  }
  if (rhs) DP_CUDA(s, cudaMemcpyAsync(rhs, s->bh, (size_t)s->K.n * 16, cudaMemcpyDefault, s->stream));
  DP_CUDA(s, cudaStreamSynchronize(s->stream));
  return check(s);
}

extern "C" int sim_well_controls(dp_sim *s, int32_t *kind, double *target) {
  if (!s || (s->ph.nw > 0 && (!kind || !target))) return DP_EINVAL;
  if (s->ph.nw == 0) return DP_OK;
  DP_CUDA(s, cudaMemcpyAsync(kind, s->well_kind, (size_t)s->ph.nw * 4, cudaMemcpyDefault, s->stream));
  DP_CUDA(s, cudaMemcpyAsync(target, s->well_target, (size_t)s->ph.nw * 8, cudaMemcpyDefault,
                             s->stream));
  DP_CUDA(s, cudaStreamSynchronize(s->stream));
  return check(s);
}

extern "C" int sim_well_rates(dp_sim *s, double *q_oil, double *q_water) {
  if (!s || (s->ph.nw > 0 && (!q_oil || !q_water))) return DP_EINVAL;
  if (s->ph.nw == 0) return DP_OK;
  size_t nw8 = (size_t)s->ph.nw * 8;
  double *q = (double *)dalloc(s, 2 * nw8);
  if (!q) { s->fail(DP_ENOMEM, "allocation failed"); return DP_ENOMEM; }
  int rc = phys_well_rates(s, q);
  if (rc == DP_OK &&
      (cudaMemcpyAsync(q_oil, q, nw8, cudaMemcpyDefault, s->stream) != cudaSuccess ||
       cudaMemcpyAsync(q_water, q + s->ph.nw, nw8, cudaMemcpyDefault, s->stream) != cudaSuccess))
    rc = DP_ECUDA;
  cudaStreamSynchronize(s->stream);
  dfree(s, q);
  if (rc != DP_OK) { s->fail(rc, "sim_well_rates"); return rc; }
  return check(s);
}

extern "C" int sim_get_colours(dp_sim *s, int32_t *colour) {
  if (!s || !colour) return DP_EINVAL;
  DP_CUDA(s, cudaMemcpyAsync(colour, s->colour, (size_t)s->K.n * 4, cudaMemcpyDefault, s->stream));
  DP_CUDA(s, cudaStreamSynchronize(s->stream));
  DP_TRY(check(s));
  return s->ncolour;
}

extern "C" int sim_well_index(dp_sim *s, double *wi) {
  if (!s || !wi) return DP_EINVAL;
  std::copy(s->wi_host.begin(), s->wi_host.end(), wi);
  return (int)s->wi_host.size();
}

extern "C" int sim_amg_level_info(dp_sim *s, int32_t level, int32_t *n, int32_t *nnz,
                                  int32_t *nagg) {
  if (!s || !s->amg_ready || level < 0 || level >= (int)s->lev.size()) return DP_EINVAL;
  const Level &L = s->lev[level];
  if (n) *n = L.n;
  if (nnz) *nnz = L.nnz;
  if (nagg) *nagg = L.nagg;
  return (int)s->lev.size();
}

extern "C" int sim_amg_transfer_info(dp_sim *s, int32_t level, int32_t *p_nnz,
                                     int32_t *smoother) {
  if (!s || !s->amg_ready || level < 0 || level >= (int)s->lev.size()) return DP_EINVAL;
  const Level &L = s->lev[level];
  bool last = level + 1 == (int)s->lev.size();
  if (p_nnz) *p_nnz = last ? 0 : L.p_nnz;
  if (smoother) *smoother = last && s->coarse_n == L.n && L.n > 0 ? 2 : L.l1 ? 1 : 0;
  return (int)s->lev.size();
}

extern "C" int sim_amg_level_arrays(dp_sim *s, int32_t level, int32_t *rowptr, int32_t *col,
                                    double *val, int32_t *agg, int32_t *colour) {
  if (!s || !s->amg_ready || level < 0 || level >= (int)s->lev.size()) return DP_EINVAL;
  const Level &L = s->lev[level];
  cudaStream_t st = s->stream;
  if (rowptr) DP_CUDA(s, cudaMemcpyAsync(rowptr, L.rowptr, ((size_t)L.n + 1) * 4, cudaMemcpyDefault, st));
  if (col) DP_CUDA(s, cudaMemcpyAsync(col, L.col, (size_t)L.nnz * 4, cudaMemcpyDefault, st));
  if (val) DP_CUDA(s, cudaMemcpyAsync(val, L.val, (size_t)L.nnz * 8, cudaMemcpyDefault, st));
  if (agg) DP_CUDA(s, cudaMemcpyAsync(agg, L.agg, (size_t)L.n * 4, cudaMemcpyDefault, st));
  if (colour) DP_CUDA(s, cudaMemcpyAsync(colour, L.colour, (size_t)L.n * 4, cudaMemcpyDefault, st));
  DP_CUDA(s, cudaStreamSynchronize(st));
  return check(s);
}

extern "C" int sim_time_kernel(dp_sim *s, const char *name) {
  if (!s) return DP_EINVAL;
  Timing &t = s->timing;
  if (!name || !*name) { t.kernel_id = -1; t.name.clear(); return DP_OK; }
  t.kernel_id = 1;
  t.name = name;
  t.used = 0;
  t.ms = 0.0;
  t.launches = 0;
  return DP_OK;
}

extern "C" int sim_kernel_timing(dp_sim *s, double *ms, int64_t *launches, int32_t reset) {
  if (!s) return DP_EINVAL;
  Timing &t = s->timing;
  DP_CUDA(s, cudaStreamSynchronize(s->stream));
  for (size_t k = 0; k + 1 < t.used; k += 2) {
    float e = 0.f;
    cudaEventElapsedTime(&e, t.ev[k], t.ev[k + 1]);
    t.ms += e;
  }
  t.used = 0;
  if (ms) *ms = t.ms;
  if (launches) *launches = t.launches;
  if (reset) { t.ms = 0.0; t.launches = 0; }
  return check(s);
}

extern "C" int64_t sim_launch_count(const dp_sim *s) { return s ? s->launches : 0; }

extern "C" const char *sim_last_error(const dp_sim *s) {
  return s ? s->last_error.c_str() : "null dp_sim";
}
