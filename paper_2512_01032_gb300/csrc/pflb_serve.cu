// pflb_serve.cu -- request server with continuous batching over the lattice
// and batch C API (host code only).
//
// Each tick: set each resident request's ramp force for its own step count
// and launch steps_per_tick steps for all of them (one persistent batch
// kernel per step, or one fused launch per request); while the GPU runs,
// admit queued requests in arrival order while the budget holds; then
// synchronise once, read each stepped request's diagnostics of the last
// step and retire the finished ones.  The batch is rebuilt only when the
// resident set changes.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <deque>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "../../include/pflb.h"
#include "pflb_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

double seconds(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double>(b - a).count();
}

pflb_status sfail(pflb_status s, const std::string &m) {
  pflb::set_last_error(m.c_str());
  return s;
}

struct Request {
  int64_t ticket = 0;
  int nx = 0, ny = 0, nz = 0;
  std::vector<uint8_t> solid;
  std::vector<double> normal, theta;
  pflb_params params{};
  pflb_solve_spec spec{};
  size_t bytes = 0;
  pflb_lattice *L = nullptr;
  pflb_solve_result res{};
  Clock::time_point t_submit, t_admit;
  std::vector<double> phi;

  pflb_geometry geometry() const {
    pflb_geometry g{};
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.solid = solid.empty() ? nullptr : solid.data();
    g.wall_normal = normal.empty() ? nullptr : normal.data();
    g.theta_deg = theta.empty() ? nullptr : theta.data();
    return g;
  }
  double beta_at(int64_t step) const {
    const double b = spec.beta0 + spec.dbeta * (double)(step / spec.ramp_every);
    return std::min(b, spec.beta_max);
  }
};

}  // namespace

struct pflb_server {
  pflb_server_config cfg{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool poisoned = false;
  int64_t next_ticket = 1;
  std::map<int64_t, std::unique_ptr<Request>> reqs;
  std::deque<Request *> queue;
  std::vector<Request *> active;
  pflb_batch *batch = nullptr;
  bool batch_dirty = true;
  size_t bytes_in_use = 0, peak_bytes = 0;
  int64_t cells_in_use = 0;
  std::vector<double> latencies;
  bool any_submit = false;
  Clock::time_point t_first, t_last_done;
  double cell_updates = 0;
  int64_t ticks = 0, completed = 0, failed = 0, rejected = 0;
  double admit_s = 0, wait_s = 0, retire_s = 0;
};

static pflb_status server_poison(pflb_server *s, const std::string &m) {
  s->poisoned = true;
  return sfail(PFLB_ERR_STATE, m);
}

extern "C" pflb_status pflb_server_create(const pflb_server_config *cfg, void *cuda_stream,
                                          pflb_server **out) {
  if (!out || !cfg) return sfail(PFLB_ERR_ARG, "null config or output");
  *out = nullptr;
  if (cfg->steps_per_tick < 1) return sfail(PFLB_ERR_ARG, "steps_per_tick must be >= 1");
  if (cfg->storage < PFLB_STORAGE_FP64 || cfg->storage > PFLB_STORAGE_BF16)
    return sfail(PFLB_ERR_ARG, "unknown storage");
  if (cfg->max_active < 0 || cfg->max_active_cells < 0 || cfg->hbm_budget_bytes == 0)
    return sfail(PFLB_ERR_ARG, "need a positive budget and max_active >= 0");
  pflb_server *s = new (std::nothrow) pflb_server();
  if (!s) return sfail(PFLB_ERR_OOM, "host allocation failed");
  s->cfg = *cfg;
  if (cuda_stream) {
    s->stream = (cudaStream_t)cuda_stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete s;
      return sfail(PFLB_ERR_CUDA, std::string("stream: ") + cudaGetErrorString(e));
    }
    s->own_stream = true;
  }
  *out = s;
  return PFLB_OK;
}

extern "C" pflb_status pflb_server_submit(pflb_server *s, const pflb_geometry *geom,
                                          const pflb_params *params,
                                          const pflb_solve_spec *spec, int64_t *ticket) {
  if (!s || !geom || !params || !spec || !ticket) return sfail(PFLB_ERR_ARG, "null argument");
  if (s->poisoned) return sfail(PFLB_ERR_STATE, "server poisoned by an earlier error");
  const int tick = s->cfg.steps_per_tick;
  if (spec->ramp_every < 1 || spec->ramp_every % tick || spec->max_steps < tick ||
      spec->max_steps % tick)
    return sfail(PFLB_ERR_ARG, "ramp_every and max_steps must be positive multiples of "
                               "steps_per_tick");
  if (!(spec->length > 0) || !std::isfinite(spec->p_ref))
    return sfail(PFLB_ERR_ARG, "need length > 0 and a finite p_ref");
  if (spec->drive != 0 && spec->drive != 1) return sfail(PFLB_ERR_ARG, "drive must be 0 or 1");
  if (spec->drive == 1 && geom->nx < 3) return sfail(PFLB_ERR_ARG, "pressure drive needs nx >= 3");
  if (params->storage != s->cfg.storage)
    return sfail(PFLB_ERR_ARG, "request storage differs from the server's");
  if (geom->nx < 1 || geom->ny < 1 || geom->nz < 1) return sfail(PFLB_ERR_ARG, "bad dimensions");
  const int64_t bytes = pflb_estimate_bytes(geom, params->storage);
  if (bytes <= 0) return sfail(PFLB_ERR_ARG, "geometry rejected by the footprint estimate");
  auto r = std::make_unique<Request>();
  r->ticket = s->next_ticket++;
  r->nx = geom->nx;
  r->ny = geom->ny;
  r->nz = geom->nz;
  const size_t N = (size_t)geom->nx * geom->ny * geom->nz;
  if (geom->solid) r->solid.assign(geom->solid, geom->solid + N);
  if (geom->wall_normal) r->normal.assign(geom->wall_normal, geom->wall_normal + 3 * N);
  if (geom->theta_deg) r->theta.assign(geom->theta_deg, geom->theta_deg + N);
  r->params = *params;
  r->spec = *spec;
  r->bytes = (size_t)bytes;
  r->t_submit = Clock::now();
  if (!s->any_submit) {
    s->any_submit = true;
    s->t_first = r->t_submit;
  }
  if (r->bytes > s->cfg.hbm_budget_bytes) {
    r->res.state = PFLB_REQ_REJECTED;
    s->rejected++;
  } else {
    r->res.state = PFLB_REQ_QUEUED;
    s->queue.push_back(r.get());
  }
  *ticket = r->ticket;
  s->reqs[r->ticket] = std::move(r);
  return PFLB_OK;
}

static void retire(pflb_server *s, Request *r, int state) {
  const auto now = Clock::now();
  r->res.state = state;
  r->res.latency_s = seconds(r->t_submit, now);
  if (state == PFLB_REQ_DONE) {
    s->latencies.push_back(r->res.latency_s);
    s->completed++;
  } else {
    s->failed++;
  }
  s->t_last_done = now;
  pflb_destroy(r->L);
  r->L = nullptr;
  s->bytes_in_use -= r->bytes;
  s->cells_in_use -= (int64_t)r->nx * r->ny * r->nz;
  // the geometry copies are no longer needed
  std::vector<uint8_t>().swap(r->solid);
  std::vector<double>().swap(r->normal);
  std::vector<double>().swap(r->theta);
}

// Pressure drive: P = beta p_ref at the inlet plane, 0 at the outlet plane,
// each change reached linearly over `ramp` steps (from rest at admission):
// a sudden inlet jump sends a pressure wave through the light phase.
static pflb_status set_drive_boundaries(Request *r, int64_t step, int64_t ramp) {
  pflb_xbc in{}, out{};
  in.type = out.type = PFLB_XBC_PRESSURE;
  in.P = r->beta_at(step) * r->spec.p_ref;
  out.P = 0.0;
  in.ramp_steps = out.ramp_steps = ramp;
  return pflb_set_x_boundaries(r->L, &in, &out);
}

static pflb_status admit(pflb_server *s) {
  while (!s->queue.empty()) {
    Request *r = s->queue.front();
    if (s->cfg.max_active > 0 && (int)s->active.size() >= s->cfg.max_active) break;
    if (s->bytes_in_use + r->bytes > s->cfg.hbm_budget_bytes) break;
    const int64_t cells = (int64_t)r->nx * r->ny * r->nz;
    if (s->cfg.max_active_cells > 0 && !s->active.empty() &&
        s->cells_in_use + cells > s->cfg.max_active_cells)
      break;
    s->queue.pop_front();
    const pflb_geometry g = r->geometry();
    pflb_status st = pflb_create(&g, &r->params, s->stream, &r->L);
    if (st == PFLB_OK)
      st = pflb_init_tanh(r->L, r->spec.init_shape, r->spec.center, r->spec.R, r->spec.normal,
                          0.0);
    if (st == PFLB_OK) st = pflb_set_region(r->L, r->spec.region);
    if (st == PFLB_OK && r->spec.drive == 1)
      st = set_drive_boundaries(r, 0, s->cfg.steps_per_tick);
    if (st != PFLB_OK) {
      // the request cannot run (e.g. its parameters are invalid): fail it,
      // keep serving the others
      if (r->L) pflb_destroy(r->L);
      r->L = nullptr;
      r->res.state = PFLB_REQ_FAILED;
      r->res.latency_s = seconds(r->t_submit, Clock::now());
      s->failed++;
      continue;
    }
    r->t_admit = Clock::now();
    r->res.queue_s = seconds(r->t_submit, r->t_admit);
    r->res.state = PFLB_REQ_RUNNING;
    s->bytes_in_use += r->bytes;
    s->cells_in_use += cells;
    s->peak_bytes = std::max(s->peak_bytes, s->bytes_in_use);
    s->active.push_back(r);
    s->batch_dirty = true;
  }
  return PFLB_OK;
}

extern "C" pflb_status pflb_server_tick(pflb_server *s, int *n_active) {
  if (!s) return sfail(PFLB_ERR_ARG, "null server");
  if (s->poisoned) return sfail(PFLB_ERR_STATE, "server poisoned by an earlier error");
  const int n = s->cfg.steps_per_tick;
  // 1. launch this tick's steps for the resident requests (asynchronous)
  std::vector<Request *> stepped = s->active;
  if (!stepped.empty()) {
    for (Request *r : stepped) {
      if (r->spec.drive == 1) {
        if (set_drive_boundaries(r, r->res.steps, s->cfg.steps_per_tick) != PFLB_OK)
          return server_poison(s, std::string("boundaries: ") + pflb_last_error());
        continue;
      }
      const double F = r->beta_at(r->res.steps) * r->spec.p_ref / r->spec.length;
      const double f[3] = {F * r->spec.dir[0], F * r->spec.dir[1], F * r->spec.dir[2]};
      if (pflb_set_force(r->L, f) != PFLB_OK) return server_poison(s, "set_force failed");
    }
    if (s->cfg.batched) {
      if (s->batch_dirty) {
        pflb_batch_destroy(s->batch);
        s->batch = nullptr;
        std::vector<pflb_lattice *> ls;
        for (Request *r : stepped) ls.push_back(r->L);
        if (pflb_batch_create(ls.data(), (int)ls.size(), s->stream, &s->batch) != PFLB_OK)
          return server_poison(s, std::string("batch: ") + pflb_last_error());
        s->batch_dirty = false;
      }
      if (pflb_batch_step(s->batch, n, 1) != PFLB_OK)
        return server_poison(s, std::string("batch step: ") + pflb_last_error());
    } else {
      for (Request *r : stepped)
        if (pflb_step_ex(r->L, n, 1) != PFLB_OK)
          return server_poison(s, std::string("step: ") + pflb_last_error());
    }
  }
  // 2. admission while the GPU runs; new requests start at the next tick
  const auto t0 = Clock::now();
  admit(s);
  const auto t1 = Clock::now();
  // 3. wait, then check and retire the requests that were stepped
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return server_poison(s, std::string("sync: ") + cudaGetErrorString(e));
  const auto t2 = Clock::now();
  s->admit_s += seconds(t0, t1);
  s->wait_s += seconds(t1, t2);
  std::vector<Request *> keep;
  bool changed = false;
  for (Request *r : stepped) {
    pflb_diag_t d{};
    const pflb_status st = pflb_last_diag(r->L, &d);
    r->res.steps += n;
    s->cell_updates += (double)r->nx * r->ny * r->nz * n;
    r->res.beta = r->beta_at(r->res.steps - 1);
    r->res.region_mass = d.region_mass;
    r->res.mass = d.mass;
    r->res.u_max = d.u_max;
    if (st == PFLB_ERR_NAN || d.nonfinite > 0) {
      retire(s, r, PFLB_REQ_FAILED);
      changed = true;
    } else if (st != PFLB_OK) {
      return server_poison(s, std::string("diag: ") + pflb_last_error());
    } else if (d.region_mass > r->spec.threshold || r->res.steps >= r->spec.max_steps) {
      r->res.broke_through = d.region_mass > r->spec.threshold;
      if (r->spec.keep_phi) {
        r->phi.resize((size_t)r->nx * r->ny * r->nz);
        if (pflb_read(r->L, PFLB_FIELD_PHI, r->phi.data()) != PFLB_OK)
          return server_poison(s, std::string("read: ") + pflb_last_error());
      }
      retire(s, r, PFLB_REQ_DONE);
      changed = true;
    } else {
      keep.push_back(r);
    }
  }
  // requests admitted in this tick follow the ones still running
  for (size_t k = stepped.size(); k < s->active.size(); ++k) keep.push_back(s->active[k]);
  if (changed) s->batch_dirty = true;
  s->active.swap(keep);
  if (!stepped.empty()) s->ticks++;
  s->retire_s += seconds(t2, Clock::now());
  if (n_active) *n_active = (int)s->active.size();
  return PFLB_OK;
}

extern "C" pflb_status pflb_server_poll(pflb_server *s, int64_t ticket, pflb_solve_result *out) {
  if (!s || !out) return sfail(PFLB_ERR_ARG, "null argument");
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return sfail(PFLB_ERR_ARG, "unknown ticket");
  *out = it->second->res;
  return PFLB_OK;
}

extern "C" pflb_status pflb_server_fetch_phi(pflb_server *s, int64_t ticket, double *out,
                                             int64_t n) {
  if (!s || !out) return sfail(PFLB_ERR_ARG, "null argument");
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return sfail(PFLB_ERR_ARG, "unknown ticket");
  const Request *r = it->second.get();
  if (r->res.state != PFLB_REQ_DONE || r->phi.empty())
    return sfail(PFLB_ERR_STATE, "request not finished or submitted without keep_phi");
  if (n < (int64_t)r->phi.size()) return sfail(PFLB_ERR_ARG, "output too small");
  std::copy(r->phi.begin(), r->phi.end(), out);
  return PFLB_OK;
}

extern "C" pflb_status pflb_server_stats_get(pflb_server *s, pflb_server_stats *out) {
  if (!s || !out) return sfail(PFLB_ERR_ARG, "null argument");
  pflb_server_stats st{};
  st.submitted = (int64_t)s->reqs.size();
  st.completed = s->completed;
  st.failed = s->failed;
  st.rejected = s->rejected;
  st.active = (int64_t)s->active.size();
  st.queued = (int64_t)s->queue.size();
  std::vector<double> l = s->latencies;
  std::sort(l.begin(), l.end());
  auto pct = [&](double q) {  // nearest rank
    if (l.empty()) return 0.0;
    size_t k = (size_t)std::ceil(q * (double)l.size());
    return l[std::min(l.size(), std::max<size_t>(k, 1)) - 1];
  };
  st.p50_s = pct(0.50);
  st.p99_s = pct(0.99);
  st.max_s = l.empty() ? 0.0 : l.back();
  double sum = 0;
  for (double v : l) sum += v;
  st.mean_s = l.empty() ? 0.0 : sum / (double)l.size();
  st.makespan_s = (s->any_submit && s->completed) ? seconds(s->t_first, s->t_last_done) : 0.0;
  st.solves_per_s = st.makespan_s > 0 ? (double)s->completed / st.makespan_s : 0.0;
  st.cell_updates = s->cell_updates;
  st.bytes_in_use = s->bytes_in_use;
  st.peak_bytes = s->peak_bytes;
  st.ticks = s->ticks;
  st.admit_s = s->admit_s;
  st.wait_s = s->wait_s;
  st.retire_s = s->retire_s;
  *out = st;
  return PFLB_OK;
}

extern "C" void pflb_server_destroy(pflb_server *s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  pflb_batch_destroy(s->batch);
  for (Request *r : s->active) pflb_destroy(r->L);
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  delete s;
}
