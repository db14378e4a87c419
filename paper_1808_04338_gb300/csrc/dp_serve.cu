// Request server for timestep solves of many realisations on one GPU
// (include/dpsim.h, "serving").  Host code only: worker threads take
// requests from one queue, keep the realisations they have served resident
// on the device (each on its own stream), and admit a realisation that is
// not resident by its device footprint, evicting idle ones least recently
// used first.  Every numerical step is the library's sim_advance.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/dpsim.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Realisation {
  dp_grid grid{};
  dp_rock rock{};
  dp_fluid fluid{};
  std::vector<dp_well> wells;
  std::vector<double> kf, km, phi_f, phi_m;
  std::vector<double> p, sw, bhp;   // host state: the initial one, or saved at eviction
  long long rows = 0;               // block rows: cells + wells
  dp_sim *sim = nullptr;
  cudaStream_t stream = nullptr;
  uint64_t bytes = 0;               // accounted device bytes while resident (or reserved)
  bool busy = false;                // a worker is serving, loading or evicting it
  int pending = 0;                  // queued requests
  uint64_t last_use = 0;
};

struct Request {
  int64_t ticket;
  int32_t id;
  double dt;
  double t_submit;
};

}  // namespace

struct dp_server {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::vector<Realisation *> real;
  std::deque<Request> queue;
  std::unordered_map<int64_t, dp_srv_result> done;
  std::vector<std::thread> workers;
  bool stop = false;
  dp_options opts{};
  int device = 0;
  uint64_t budget = 0, resident_bytes = 0, peak_resident = 0;
  double bytes_per_row = 0.0;       // largest measured peak bytes per block row
  int64_t next_ticket = 0, served = 0, loads = 0, evictions = 0, launches = 0;
  int running = 0;
  uint64_t use_clock = 0;
  Clock::time_point t0 = Clock::now();

  double now_ms() const {
    return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
  }
  uint64_t estimate(const Realisation &r) const {
    double per_row = bytes_per_row > 0.0 ? 1.05 * bytes_per_row : 4096.0;
    return (uint64_t)(per_row * (double)r.rows) + (1u << 20);
  }
  void worker();
  // Under the lock: can request q start now?  On success fills `victims`
  // (idle resident realisations to evict, least recently used first).
  bool admissible(const Request &q, std::vector<int> &victims, bool &never);
};

bool dp_server::admissible(const Request &q, std::vector<int> &victims, bool &never) {
  victims.clear();
  never = false;
  Realisation &r = *real[q.id];
  if (r.busy) return false;
  if (r.sim) return true;
  uint64_t need = estimate(r);
  if (need > budget) {
    // refused only on a measured estimate; before any measurement the guess
    // may be pessimistic, so the request waits until nothing else holds
    // device memory and then runs alone (and its footprint is measured)
    if (bytes_per_row > 0.0) { never = true; return true; }
    if (running > 0) return false;
    need = budget;
  }
  uint64_t have = resident_bytes;
  if (have + need <= budget) return true;
  std::vector<int> idle;
  for (int k = 0; k < (int)real.size(); ++k)
    if (k != q.id && real[k]->sim && !real[k]->busy) idle.push_back(k);
  std::sort(idle.begin(), idle.end(),
            [&](int a, int b) { return real[a]->last_use < real[b]->last_use; });
  for (int k : idle) {
    victims.push_back(k);
    have -= real[k]->bytes;
    if (have + need <= budget) return true;
  }
  victims.clear();
  return false;
}

void dp_server::worker() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    // the first queued request that can start now
    std::vector<int> victims;
    bool never = false;
    auto it = queue.begin();
    for (; it != queue.end(); ++it)
      if (admissible(*it, victims, never)) break;
    if (it == queue.end()) {
      if (stop && queue.empty()) return;
      cv_work.wait(lk);
      continue;
    }
    Request q = *it;
    queue.erase(it);
    Realisation &r = *real[q.id];
    --r.pending;
    dp_srv_result res{};
    res.realisation = q.id;
    res.t_submit_ms = q.t_submit;
    res.t_start_ms = now_ms();
    if (never) {
      res.status = DP_ENOMEM;
      res.t_done_ms = res.t_start_ms;
      done[q.ticket] = res;
      cv_done.notify_all();
      cv_work.notify_all();
      continue;
    }
    r.busy = true;
    ++running;
    bool load = r.sim == nullptr;
    uint64_t reserved = 0;
    for (int k : victims) {
      real[k]->busy = true;
      resident_bytes -= real[k]->bytes;
      ++evictions;
    }
    if (load) {
      reserved = estimate(r);
      r.bytes = reserved;
      resident_bytes += reserved;
      ++loads;
    }
    peak_resident = std::max(peak_resident, resident_bytes);
    lk.unlock();

    int rc = DP_OK;
    for (int k : victims) {   // state back to the host copy, then free it all
      Realisation &v = *real[k];
      int e = sim_get_state(v.sim, v.p.data(), v.sw.data(), v.bhp.data());
      sim_destroy(v.sim);
      cudaStreamSynchronize(v.stream);
      cudaStreamDestroy(v.stream);
      v.sim = nullptr;
      v.stream = nullptr;
      if (e != DP_OK) rc = e;
    }
    if (rc == DP_OK && load) {
      if (cudaStreamCreateWithFlags(&r.stream, cudaStreamNonBlocking) != cudaSuccess) {
        r.stream = nullptr;
        rc = DP_ECUDA;
      } else {
        r.rock.kf = r.kf.data(); r.rock.km = r.km.data();
        r.rock.phi_f = r.phi_f.data(); r.rock.phi_m = r.phi_m.data();
        rc = sim_create(&r.grid, &r.rock, &r.fluid, r.wells.data(), (int32_t)r.wells.size(),
                        &opts, nullptr, (void *)r.stream, &r.sim);
        if (rc == DP_OK) rc = sim_set_state(r.sim, r.p.data(), r.sw.data(), r.bhp.data());
      }
    }
    int64_t l0 = (r.sim && !load) ? sim_launch_count(r.sim) : 0;
    if (rc == DP_OK) rc = sim_advance(r.sim, q.dt, &res.stats);
    int64_t nl = r.sim ? sim_launch_count(r.sim) - l0 : 0;
    uint64_t peak = 0;
    if (r.sim) sim_footprint(r.sim, nullptr, &peak);
    bool drop = rc != DP_OK && rc != DP_ENEWTON && rc != DP_ELINEAR && r.sim;
    if (drop) {   // a failed CUDA call: the realisation is rebuilt when next served
      sim_destroy(r.sim);
      r.sim = nullptr;
    }
    if (!r.sim && r.stream) {
      cudaStreamSynchronize(r.stream);
      cudaStreamDestroy(r.stream);
      r.stream = nullptr;
    }

    lk.lock();
    for (int k : victims) {
      real[k]->busy = false;
      real[k]->bytes = 0;
    }
    resident_bytes -= r.bytes;
    r.bytes = r.sim ? std::max<uint64_t>(peak, 1) : 0;
    resident_bytes += r.bytes;
    peak_resident = std::max(peak_resident, resident_bytes);
    if (r.sim && r.rows > 0)
      bytes_per_row = std::max(bytes_per_row, (double)peak / (double)r.rows);
    r.busy = false;
    r.last_use = ++use_clock;
    launches += nl;
    --running;
    ++served;
    res.status = rc;
    res.loaded = load ? 1 : 0;
    res.evicted = (int32_t)victims.size();
    res.t_done_ms = now_ms();
    done[q.ticket] = res;
    cv_done.notify_all();
    cv_work.notify_all();
  }
}

extern "C" int srv_create(int32_t workers, uint64_t hbm_budget, const dp_options *opts,
                          dp_server **out) {
  if (!out) return DP_EINVAL;
  *out = nullptr;
  if (workers < 1 || workers > 256 || hbm_budget == 0 || !opts) return DP_EINVAL;
  dp_server *s = new (std::nothrow) dp_server();
  if (!s) return DP_ENOMEM;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return DP_ECUDA;
  }
  s->opts = *opts;
  s->budget = hbm_budget;
  try {
    for (int w = 0; w < workers; ++w) s->workers.emplace_back([s] { s->worker(); });
  } catch (...) {
    {
      std::lock_guard<std::mutex> g(s->mu);
      s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->workers) t.join();
    delete s;
    return DP_ENOMEM;
  }
  *out = s;
  return DP_OK;
}

extern "C" int srv_add(dp_server *srv, const dp_grid *grid, const dp_rock *rock,
                       const dp_fluid *fluid, const dp_well *wells, int32_t nwells,
                       const double *p, const double *sw, const double *bhp, int32_t *id) {
  if (!srv || !grid || !rock || !fluid || !id || nwells < 0 || (nwells > 0 && (!wells || !bhp)) ||
      !p || !sw)
    return DP_EINVAL;
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return DP_EINVAL;
  if (!rock->kf || !rock->km || !rock->phi_f || !rock->phi_m) return DP_EINVAL;
  Realisation *r = new (std::nothrow) Realisation();
  if (!r) return DP_ENOMEM;
  size_t nL = (size_t)grid->nx * grid->ny * grid->nz;
  try {
    r->grid = *grid;
    r->rock = *rock;
    r->fluid = *fluid;
    r->wells.assign(wells, wells + nwells);
    r->kf.assign(rock->kf, rock->kf + nL);
    r->km.assign(rock->km, rock->km + nL);
    r->phi_f.assign(rock->phi_f, rock->phi_f + nL);
    r->phi_m.assign(rock->phi_m, rock->phi_m + nL);
    r->p.assign(p, p + 2 * nL);
    r->sw.assign(sw, sw + 2 * nL);
    r->bhp.assign(std::max(nwells, 1), 0.0);
    if (nwells > 0) std::copy(bhp, bhp + nwells, r->bhp.begin());
  } catch (...) {
    delete r;
    return DP_ENOMEM;
  }
  r->rows = (long long)(2 * nL) + nwells;
  std::lock_guard<std::mutex> g(srv->mu);
  *id = (int32_t)srv->real.size();
  srv->real.push_back(r);
  return DP_OK;
}

extern "C" int srv_submit(dp_server *srv, int32_t id, double dt, int64_t *ticket) {
  if (!srv || !ticket || !(dt > 0.0)) return DP_EINVAL;
  {
    std::lock_guard<std::mutex> g(srv->mu);
    if (id < 0 || id >= (int32_t)srv->real.size() || srv->stop) return DP_EINVAL;
    *ticket = srv->next_ticket++;
    srv->queue.push_back({*ticket, id, dt, srv->now_ms()});
    ++srv->real[id]->pending;
  }
  srv->cv_work.notify_one();
  return DP_OK;
}

extern "C" int srv_wait(dp_server *srv, int64_t ticket, dp_srv_result *out) {
  if (!srv || !out) return DP_EINVAL;
  std::unique_lock<std::mutex> lk(srv->mu);
  if (ticket < 0 || ticket >= srv->next_ticket) return DP_EINVAL;
  for (;;) {
    auto it = srv->done.find(ticket);
    if (it != srv->done.end()) {
      *out = it->second;
      srv->done.erase(it);
      return DP_OK;
    }
    bool queued = false;
    for (const Request &q : srv->queue) queued |= q.ticket == ticket;
    if (!queued && srv->running == 0) return DP_EINVAL;   // already collected
    srv->cv_done.wait(lk);
  }
}

extern "C" int srv_get_state(dp_server *srv, int32_t id, double *p, double *sw, double *bhp) {
  if (!srv || !p || !sw) return DP_EINVAL;
  std::unique_lock<std::mutex> lk(srv->mu);
  if (id < 0 || id >= (int32_t)srv->real.size()) return DP_EINVAL;
  Realisation &r = *srv->real[id];
  if (!r.wells.empty() && !bhp) return DP_EINVAL;
  srv->cv_done.wait(lk, [&] { return !r.busy && r.pending == 0; });
  if (r.sim) {
    r.busy = true;   // keep workers away while the copy runs
    lk.unlock();
    std::vector<double> b(std::max<size_t>(r.wells.size(), 1));
    int rc = sim_get_state(r.sim, p, sw, b.data());
    if (bhp) std::copy(b.begin(), b.begin() + r.wells.size(), bhp);
    lk.lock();
    r.busy = false;
    srv->cv_work.notify_all();
    return rc;
  }
  std::copy(r.p.begin(), r.p.end(), p);
  std::copy(r.sw.begin(), r.sw.end(), sw);
  if (bhp) std::copy(r.bhp.begin(), r.bhp.begin() + r.wells.size(), bhp);
  return DP_OK;
}

extern "C" int srv_info(dp_server *srv, dp_srv_info *out) {
  if (!srv || !out) return DP_EINVAL;
  std::lock_guard<std::mutex> g(srv->mu);
  dp_srv_info i{};
  i.registered = (int32_t)srv->real.size();
  for (auto *r : srv->real) i.resident += r->sim ? 1 : 0;
  i.queued = (int32_t)srv->queue.size();
  i.running = srv->running;
  i.served = srv->served;
  i.loads = srv->loads;
  i.evictions = srv->evictions;
  i.launches = srv->launches;
  i.resident_bytes = srv->resident_bytes;
  i.peak_resident_bytes = srv->peak_resident;
  i.budget_bytes = srv->budget;
  i.bytes_per_row = srv->bytes_per_row;
  *out = i;
  return DP_OK;
}

extern "C" int srv_destroy(dp_server *srv) {
  if (!srv) return DP_EINVAL;
  {
    std::lock_guard<std::mutex> g(srv->mu);
    srv->stop = true;
  }
  srv->cv_work.notify_all();
  for (auto &t : srv->workers) t.join();
  for (auto *r : srv->real) {
    if (r->sim) sim_destroy(r->sim);
    if (r->stream) {
      cudaStreamSynchronize(r->stream);
      cudaStreamDestroy(r->stream);
    }
    delete r;
  }
  delete srv;
  return DP_OK;
}
