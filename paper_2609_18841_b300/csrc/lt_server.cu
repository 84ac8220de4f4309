// Continuous-batching request server over lindtebd contexts.
//
// A request is one ensemble (an lt_config: method, chain, rates, trajectories)
// run for n_steps time steps.  Each admitted request owns a context and its
// stream, so the steps of all active requests are queued side by side and the
// GPU interleaves their kernels; the ensemble stays resident on the device from
// admission to retirement.  Every tick admits queued requests in arrival order
// while their device footprint fits the budget (and the active count is below
// its cap), queues one time step for every active request, and retires those
// whose last step has completed (ensemble density measured, context freed).
// Requests never share a context, so each result is bit-identical to running
// the request alone.  The paper has no serving layer; this is the runtime
// around its trajectory and QSD integrators.
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "lt_internal.cuh"

namespace {

struct Request {
  int64_t id = 0;
  lt_config cfg{};
  std::vector<double> gl, gg, gd;
  std::vector<uint8_t> occ;
  int32_t n_steps = 0, done = 0;
  lt_ctx ctx = nullptr;
  cudaEvent_t last = nullptr;  // recorded after the newest queued step
  uint64_t bytes = 0;
  double t_submit = 0, t_start = 0, t_done = 0;
  std::vector<double> mean, sem;
  lt_status status = LT_OK;
  uint64_t updates = 0;  // two-site updates the request executed (its context's counter)
  std::string error;  // the context's last error when the request failed
  int state = 0;      // 0 queued, 1 active, 2 finished (status tells success)
};

}  // namespace

struct lt_server_s {
  uint64_t budget = 0, used = 0;
  int max_active = 0, num_sms = 0;
  std::deque<int64_t> queue;
  std::vector<int64_t> active;
  std::map<int64_t, Request> reqs;
  int64_t next_id = 1;
  int32_t finished = 0;
  std::chrono::steady_clock::time_point t0;
  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

// Device bytes lt_create allocates for cfg, with the occupancy-dependent grids
// of the bond and environment scratch bounded above (2 and 8 CTAs per SM).
uint64_t context_bytes(const lt_config* cfg, int num_sms) {
  const uint64_t L = cfg->L, chi = cfg->chi_max, nt = cfg->n_traj, nb = L - 1;
  const uint64_t celt = cfg->precision == LT_MIXED ? 8 : 16;
  const uint64_t d = cfg->method == LT_MPDO || cfg->method == LT_PURIFIED ? 4 : 2;
  const uint64_t slot = d * chi * chi;
  uint64_t b = nt * L * slot * celt;                       // site tensors
  b += nt * nb * chi * 8 + nt * nb * 4 + nt * nb * 8;      // Lambda, dims, truncation
  b += nt * 4 * 5 + 2 * 4;                                 // flags, channels, lists, counts
  b += nt * L * 8 + nt * 8 + nt * 3 * L * 8 + 3 * L * 8;   // density, log weights, rates, rates table
  b += 4 + 64 * 4 + LT_NCOUNTERS * 8 + 8 * nb * d * d * d * d * 16;  // error word, histogram, counters, gates
  b += (2 * L * L + 2 * L) * 8;                            // reduction buffer
  const uint64_t need = bond_smem_bytes((int)chi, celt, (int)d);
  if (need > 200 * 1024) {
    b += 2ull * num_sms * need;                              // bond scratch when not in shared memory
    if (celt == 8) b += (uint64_t)num_sms / 2 * LT_CL_STATE * 4;  // cluster Jacobi state
  }
  uint64_t env_grid = nt < 8ull * num_sms ? nt : 8ull * num_sms;
  const uint64_t cap = (uint64_t)env_grid_cap((int)L, (int)chi, celt, num_sms);
  if (env_grid > cap) env_grid = cap;
  b += env_grid * (cfg->method == LT_MPDO       ? (uint64_t)mpdo_scratch_bytes((int)L, (int)chi)
                   : cfg->method == LT_PURIFIED ? (uint64_t)purified_scratch_bytes((int)L, (int)chi)
                                                : env_scratch_elems((int)L, (int)chi) * celt);
  return b;
}

void retire(lt_server_s* s, Request& r, lt_status st) {
  if (r.last) cudaEventDestroy(r.last);
  r.last = nullptr;
  if (r.ctx) {
    if (st != LT_OK) {
      const char* e = lt_last_error(r.ctx);
      r.error = e ? e : "";
    } else {
      uint64_t cnt[LT_NCOUNTERS] = {0};
      if (lt_get_counters(r.ctx, cnt, 0) == LT_OK) r.updates = cnt[0];
    }
    s->used -= r.bytes;
    lt_destroy(r.ctx);
    r.ctx = nullptr;
  }
  r.status = st;
  r.state = 2;
  r.t_done = s->now();
  s->finished++;
}

}  // namespace

extern "C" {

lt_status lt_context_bytes(const lt_config* cfg, int32_t num_sms, uint64_t* out) {
  if (!cfg || !out || num_sms < 1 || cfg->L < 2 || cfg->chi_max < 1 || cfg->chi_max > LT_MAX_CHI ||
      cfg->n_traj < 1)
    return LT_ERR_ARG;
  *out = context_bytes(cfg, num_sms);
  return LT_OK;
}

lt_status lt_admit_plan(uint64_t budget, uint64_t used, int32_t max_active, int32_t n_active,
                        const uint64_t* queued_bytes, int32_t n_queued, int32_t* n_admit) {
  if (!n_admit || n_queued < 0 || (n_queued > 0 && !queued_bytes) || max_active < 1 || n_active < 0)
    return LT_ERR_ARG;
  int32_t k = 0;
  while (k < n_queued && n_active + k < max_active && used + queued_bytes[k] <= budget) {
    used += queued_bytes[k];
    ++k;
  }
  *n_admit = k;
  return LT_OK;
}

lt_status lt_server_create(uint64_t hbm_budget_bytes, int32_t max_active, lt_server* out) {
  if (!out) return LT_ERR_ARG;
  *out = nullptr;
  if (hbm_budget_bytes == 0 || max_active < 1) return LT_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return LT_ERR_CUDA;
  lt_server_s* s = new (std::nothrow) lt_server_s();
  if (!s) return LT_ERR_OOM;
  s->budget = hbm_budget_bytes;
  s->max_active = max_active;
  s->num_sms = sms;
  s->t0 = std::chrono::steady_clock::now();
  *out = s;
  return LT_OK;
}

lt_status lt_server_destroy(lt_server s) {
  if (!s) return LT_ERR_ARG;
  for (auto& kv : s->reqs) {
    Request& r = kv.second;
    if (r.last) cudaEventDestroy(r.last);
    if (r.ctx) lt_destroy(r.ctx);
  }
  delete s;
  return LT_OK;
}

lt_status lt_server_submit(lt_server s, const lt_config* cfg, int32_t n_steps, int64_t* out_id) {
  if (!s || !cfg || !out_id || n_steps < 1 || cfg->L < 2 || cfg->L > 1024 || cfg->n_traj < 1 ||
      cfg->chi_max < 1 || cfg->chi_max > LT_MAX_CHI)
    return LT_ERR_ARG;
  const int64_t id = s->next_id++;
  Request& r = s->reqs[id];
  r.id = id;
  r.cfg = *cfg;
  const int L = cfg->L;
  // the request outlives the caller's arrays: keep copies
  auto copy = [L](const double* p, std::vector<double>& v) {
    v.assign(L, 0.0);
    if (p) std::memcpy(v.data(), p, sizeof(double) * L);
  };
  copy(cfg->gamma_loss, r.gl);
  copy(cfg->gamma_gain, r.gg);
  copy(cfg->gamma_deph, r.gd);
  r.cfg.gamma_loss = r.gl.data();
  r.cfg.gamma_gain = r.gg.data();
  r.cfg.gamma_deph = r.gd.data();
  if (cfg->product_occ) {
    r.occ.assign(cfg->product_occ, cfg->product_occ + L);
    r.cfg.product_occ = r.occ.data();
  }
  r.n_steps = n_steps;
  r.bytes = context_bytes(&r.cfg, s->num_sms);
  r.t_submit = s->now();
  s->queue.push_back(id);
  *out_id = id;
  return LT_OK;
}

lt_status lt_server_tick(lt_server s, int32_t* n_queued, int32_t* n_active, int32_t* n_finished) {
  if (!s) return LT_ERR_ARG;
  // 1. admission in arrival order (head of line waits for room)
  while (!s->queue.empty()) {
    Request& r = s->reqs[s->queue.front()];
    if (r.bytes > s->budget) {  // can never fit
      s->queue.pop_front();
      retire(s, r, LT_ERR_OOM);
      continue;
    }
    uint64_t bytes = r.bytes;
    int32_t k = 0;
    lt_admit_plan(s->budget, s->used, s->max_active, (int32_t)s->active.size(), &bytes, 1, &k);
    if (k == 0) break;
    s->queue.pop_front();
    lt_ctx ctx = nullptr;
    lt_status st = lt_create(&r.cfg, nullptr, &ctx);
    if (st == LT_ERR_OOM && !s->active.empty()) {  // the estimate was short: wait for room
      s->queue.push_front(r.id);
      break;
    }
    if (st != LT_OK) {
      retire(s, r, st);
      continue;
    }
    if (cudaEventCreateWithFlags(&r.last, cudaEventDisableTiming) != cudaSuccess) {
      lt_destroy(ctx);
      retire(s, r, LT_ERR_CUDA);
      continue;
    }
    r.ctx = ctx;
    r.bytes = ctx->dev_bytes;
    s->used += r.bytes;
    r.t_start = s->now();
    r.state = 1;
    s->active.push_back(r.id);
  }
  // 2. one time step for every active request (at most two in flight each)
  for (int64_t id : s->active) {
    Request& r = s->reqs[id];
    if (r.done >= r.n_steps) continue;
    if (r.done > 0) cudaEventSynchronize(r.last);
    lt_status st = lt_step(r.ctx, 1);
    if (st != LT_OK) {
      r.status = st;
      r.done = r.n_steps;
      continue;
    }
    cudaEventRecord(r.last, lt_stream(r.ctx) ? (cudaStream_t)lt_stream(r.ctx) : nullptr);
    r.done++;
  }
  // 3. retirement of requests whose last step has completed
  std::vector<int64_t> still;
  for (int64_t id : s->active) {
    Request& r = s->reqs[id];
    bool pending = r.done < r.n_steps;
    if (!pending && r.status == LT_OK && cudaEventQuery(r.last) == cudaErrorNotReady) {
      cudaGetLastError();  // "not ready" is a state, not an error for later launches to report
      pending = true;
    }
    if (pending) {
      still.push_back(id);
      continue;
    }
    lt_status st = r.status;
    if (st == LT_OK) {
      r.mean.assign(r.cfg.L, 0.0);
      r.sem.assign(r.cfg.L, 0.0);
      st = lt_measure_density(r.ctx, r.mean.data(), r.sem.data(), nullptr);
    }
    retire(s, r, st);
  }
  s->active.swap(still);
  if (n_queued) *n_queued = (int32_t)s->queue.size();
  if (n_active) *n_active = (int32_t)s->active.size();
  if (n_finished) *n_finished = s->finished;
  return LT_OK;
}

lt_status lt_server_result(lt_server s, int64_t id, double* mean, double* sem, double* times) {
  if (!s) return LT_ERR_ARG;
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return LT_ERR_ARG;
  const Request& r = it->second;
  if (r.state != 2) return LT_ERR_STATE;
  if (times) {
    times[0] = r.t_submit;
    times[1] = r.t_start;
    times[2] = r.t_done;
  }
  if (r.status != LT_OK) return r.status;
  if (mean) std::memcpy(mean, r.mean.data(), sizeof(double) * r.cfg.L);
  if (sem) std::memcpy(sem, r.sem.data(), sizeof(double) * r.cfg.L);
  return LT_OK;
}

lt_status lt_server_updates(lt_server s, int64_t id, uint64_t* updates) {
  if (!s || !updates) return LT_ERR_ARG;
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return LT_ERR_ARG;
  const Request& r = it->second;
  *updates = r.updates;
  if (r.state == 1 && r.ctx) {  // active: the context's counter so far (synchronises its stream)
    uint64_t cnt[LT_NCOUNTERS] = {0};
    if (lt_get_counters(r.ctx, cnt, 0) == LT_OK) *updates = cnt[0];
  }
  return LT_OK;
}

const char* lt_server_error(lt_server s, int64_t id) {
  if (!s) return "";
  auto it = s->reqs.find(id);
  return it == s->reqs.end() ? "" : it->second.error.c_str();
}

lt_status lt_server_usage(lt_server s, uint64_t* used_bytes, uint64_t* budget_bytes) {
  if (!s) return LT_ERR_ARG;
  if (used_bytes) *used_bytes = s->used;
  if (budget_bytes) *budget_bytes = s->budget;
  return LT_OK;
}

}  // extern "C"
