// server.cu -- the request server (cl_server_*, include/cl.h): complex-
// Langevin trajectories of different extents and couplings admitted as they
// arrive, resident in HBM with their Philox step counters, advanced
// concurrently (continuous batching: every resident chain has its own stream
// and a few chunks of steps queued on it, and a chain that finishes frees its
// slot for the next request at once).  Host-side scheduling only; every step
// runs through the same launch sequence as cl_step / cl_cool.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <thread>
#include <vector>

#include "../../include/cl.h"
#include "launch.h"
#include "runtime.h"

using namespace clgc;
using namespace clrt;

namespace {

const int INFLIGHT = 2;  // chunks queued per chain ahead of the host

struct Chain {
  cl_lattice* lat = nullptr;
  cudaStream_t st = nullptr;
  int L[4] = {0, 0, 0, 0};
  int prec = 0;
  size_t bytes = 0;
  // the request it is serving
  bool busy = false;
  cl_request req;
  double t_submit = 0, t_admit = 0;
  int enq_steps = 0;
  cudaEvent_t ev[INFLIGHT] = {nullptr, nullptr};
  int ev_head = 0, ev_count = 0;
  cudaEvent_t final_ev = nullptr;
  bool final_enqueued = false;
  ObsOut* h_obs = nullptr;     // pinned
  CoolState* h_cs = nullptr;   // pinned
  CoolState* h_ccs = nullptr;  // pinned [INFLIGHT]: cooling state after each queued chunk
  int chunk_n[INFLIGHT] = {0, 0};
  bool runaway = false;        // a chunk ended above the runaway bound: no further chunks
};

struct Pending {
  cl_request req;
  double t_submit;
};

void destroy_chain(Chain* c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  if (c->lat) cl_free(c->lat);
  for (cudaEvent_t e : c->ev)
    if (e) cudaEventDestroy(e);
  if (c->final_ev) cudaEventDestroy(c->final_ev);
  if (c->h_obs) cudaFreeHost(c->h_obs);
  if (c->h_cs) cudaFreeHost(c->h_cs);
  if (c->h_ccs) cudaFreeHost(c->h_ccs);
  if (c->st) cudaStreamDestroy(c->st);
  delete c;
}

cl_params params_of(const cl_request& r, cl_precision prec) {
  cl_params p;
  std::memset(&p, 0, sizeof(p));
  for (int mu = 0; mu < 4; ++mu) p.L[mu] = r.L[mu];
  p.beta = r.beta;
  p.theta_re = r.theta_re;
  p.theta_im = r.theta_im;
  p.prec = prec;
  p.seed = r.seed;
  p.start = r.start;
  p.gauge_sigma = r.gauge_sigma;
  return p;
}

}  // namespace

struct cl_server {
  cl_server_config cfg;
  std::chrono::steady_clock::time_point t0;
  std::deque<Pending> queue;
  std::vector<Chain*> active;
  std::vector<Chain*> pool;  // idle chains kept for reuse by same-shape requests
  std::deque<cl_result> done;
  size_t bytes = 0;  // device bytes of active + pooled chains
  cl_server_stats stats;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

cl_status check_request(const cl_server* s, const cl_request* r) {
  if (!r) return fail(CL_ERR_INVALID, "NULL request");
  for (int mu = 0; mu < 4; ++mu)
    if (r->L[mu] < 1) return fail(CL_ERR_INVALID, "lattice extent < 1");
  if (r->n_steps < 0 || !(r->eps >= 0.0)) return fail(CL_ERR_INVALID, "bad n_steps or eps");
  if (r->start != CL_START_COLD && r->start != CL_START_HOT) return fail(CL_ERR_INVALID, "bad start");
  cl_params p = params_of(*r, s->cfg.prec);
  size_t b = 0;
  cl_status st = cl_lattice_bytes(&p, &b);
  if (st != CL_OK) return st;
  if ((double)b > s->cfg.hbm_budget_bytes)
    return fail(CL_ERR_INVALID, "request larger than the whole memory budget");
  return CL_OK;
}

// Enqueue up to `n` steps of chain c on its stream.
cl_status enqueue_steps(cl_server* s, Chain* c, int n) {
  cl_cool_params cp = s->cfg.cool;
  cp.eps = c->req.eps;
  if (s->cfg.use_graphs) return cl_replay(c->lat, n);
  for (int i = 0; i < n; ++i) {
    cl_status st = enqueue_step(c->lat, c->req.eps, s->cfg.cool_enabled ? &cp : nullptr);
    if (st != CL_OK) return st;
  }
  return CL_OK;
}

// Keep INFLIGHT chunks queued; after the last step, the observables and the
// cooling report are copied to pinned host memory behind final_ev.
bool watch_runaway(const cl_server* s) { return s->cfg.cool_enabled && s->cfg.runaway_un > 0.0; }

cl_status feed(cl_server* s, Chain* c) {
  while (!c->final_enqueued && c->ev_count < INFLIGHT) {
    const int k = c->runaway ? 0 : std::min(s->cfg.chunk_steps, c->req.n_steps - c->enq_steps);
    if (k > 0) {
      cl_status st = enqueue_steps(s, c, k);
      if (st != CL_OK) return st;
      c->enq_steps += k;
      const int slot = (c->ev_head + c->ev_count) % INFLIGHT;
      // the cooling state after the chunk: the host checks it for a runaway
      if (watch_runaway(s))
        CK(cudaMemcpyAsync(&c->h_ccs[slot], c->lat->cs, sizeof(CoolState), cudaMemcpyDeviceToHost, c->st));
      c->chunk_n[slot] = k;
      CK(cudaEventRecord(c->ev[slot], c->st));
      c->ev_count++;
    }
    if (c->enq_steps == c->req.n_steps || c->runaway) {
      cl_status st = do_obs(c->lat, c->lat->obs, nullptr);
      if (st != CL_OK) return st;
      CK(cudaMemcpyAsync(c->h_obs, c->lat->obs, sizeof(ObsOut), cudaMemcpyDeviceToHost, c->st));
      CK(cudaMemcpyAsync(c->h_cs, c->lat->cs, sizeof(CoolState), cudaMemcpyDeviceToHost, c->st));
      CK(cudaEventRecord(c->final_ev, c->st));
      c->final_enqueued = true;
    }
  }
  return CL_OK;
}

cl_status new_chain(cl_server* s, const cl_params& p, Chain** out) {
  *out = nullptr;
  Chain* c = new Chain();
  for (int mu = 0; mu < 4; ++mu) c->L[mu] = p.L[mu];
  c->prec = (int)p.prec;
  cl_status st = cl_lattice_bytes(&p, &c->bytes);
  cudaError_t e = cudaSuccess;
  if (st == CL_OK) e = cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking);
  for (int i = 0; i < INFLIGHT && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&c->ev[i], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->final_ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_obs, sizeof(ObsOut));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_cs, sizeof(CoolState));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_ccs, INFLIGHT * sizeof(CoolState));
  if (st == CL_OK && e != cudaSuccess) st = fail(CL_ERR_CUDA, std::string("server chain: ") + cudaGetErrorString(e));
  if (st == CL_OK) st = cl_init_lattice(&p, (void*)c->st, &c->lat);
  if (st == CL_OK && s->cfg.blocks_from_autotune) {
    cl_cool_params cp = s->cfg.cool;
    cp.eps = 0.005;
    st = cl_autotune(c->lat, cp.eps, &cp, 2, 1, nullptr, nullptr);
  }
  if (st != CL_OK) {
    destroy_chain(c);
    return st;
  }
  *out = c;
  return CL_OK;
}

// Admit the head of the queue while a slot and the memory budget allow it
// (first come, first served: a request that does not fit blocks those behind).
cl_status admit(cl_server* s) {
  while (!s->queue.empty() && (int)s->active.size() < s->cfg.max_slots) {
    const Pending& pd = s->queue.front();
    const int prec = (int)s->cfg.prec;
    cl_params p = params_of(pd.req, s->cfg.prec);
    Chain* c = nullptr;
    for (size_t i = 0; i < s->pool.size(); ++i) {
      Chain* q = s->pool[i];
      if (q->prec == prec && q->L[0] == p.L[0] && q->L[1] == p.L[1] && q->L[2] == p.L[2] && q->L[3] == p.L[3]) {
        c = q;
        s->pool.erase(s->pool.begin() + i);
        break;
      }
    }
    if (c) {
      cl_status st = cl_reset_lattice(c->lat, &p);
      if (st != CL_OK) {
        s->bytes -= c->bytes;
        destroy_chain(c);
        return st;
      }
    } else {
      size_t need = 0;
      cl_status st = cl_lattice_bytes(&p, &need);
      if (st != CL_OK) return st;
      // make room by dropping idle chains, least recently used first
      while ((double)(s->bytes + need) > s->cfg.hbm_budget_bytes && !s->pool.empty()) {
        Chain* q = s->pool.front();
        s->pool.erase(s->pool.begin());
        s->bytes -= q->bytes;
        destroy_chain(q);
      }
      if ((double)(s->bytes + need) > s->cfg.hbm_budget_bytes) break;  // wait for memory
      st = new_chain(s, p, &c);
      if (st != CL_OK) return st;
      s->bytes += c->bytes;
    }
    c->busy = true;
    c->req = pd.req;
    c->t_submit = pd.t_submit;
    c->t_admit = s->now();
    c->enq_steps = 0;
    c->ev_head = c->ev_count = 0;
    c->final_enqueued = false;
    c->runaway = false;
    s->queue.pop_front();
    {
      cl_status st = cl_set_adaptive_step(c->lat, s->cfg.k_ref);
      if (st != CL_OK) return st;
    }
    if (s->cfg.use_graphs) {
      cl_cool_params cp = s->cfg.cool;
      cp.eps = c->req.eps;
      cl_status st = cl_capture_step(c->lat, c->req.eps, s->cfg.cool_enabled ? &cp : nullptr);
      if (st != CL_OK) return st;
    }
    s->active.push_back(c);
    s->stats.admitted++;
    if ((int)s->active.size() > s->stats.peak_active) s->stats.peak_active = (int)s->active.size();
    if (s->bytes > s->stats.peak_bytes) s->stats.peak_bytes = s->bytes;
    cl_status st = feed(s, c);
    if (st != CL_OK) return st;
  }
  return CL_OK;
}

// Retire finished chunks and chains; returns the number of state changes.
cl_status collect(cl_server* s, int* changes) {
  for (size_t i = 0; i < s->active.size();) {
    Chain* c = s->active[i];
    while (c->ev_count > 0) {
      cudaError_t e = cudaEventQuery(c->ev[c->ev_head]);
      if (e == cudaErrorNotReady) break;
      CK(e);
      if (watch_runaway(s) && !c->runaway) {
        const CoolState& cs = c->h_ccs[c->ev_head];
        if (cs.nonfinite || !(cs.un_after <= s->cfg.runaway_un)) {
          c->runaway = true;
          s->stats.runaways++;
        }
      }
      c->ev_head = (c->ev_head + 1) % INFLIGHT;
      c->ev_count--;
      (*changes)++;
    }
    bool finished = false;
    if (c->final_enqueued) {
      cudaError_t e = cudaEventQuery(c->final_ev);
      if (e != cudaErrorNotReady) {
        CK(e);
        finished = true;
      }
    }
    if (!finished) {
      cl_status st = feed(s, c);
      if (st != CL_OK) return st;
      ++i;
      continue;
    }
    cl_result r;
    std::memset(&r, 0, sizeof(r));
    r.tag = c->req.tag;
    r.n_steps = c->enq_steps;
    to_cl_obs(*c->h_obs, &r.obs);
    to_report(*c->h_cs, &r.last_cool);
    r.status = c->runaway ? CL_ERR_RUNAWAY
               : (c->h_obs->nonfinite != 0.0 || c->h_cs->nonfinite ? CL_ERR_NONFINITE : CL_OK);
    r.t_submit = c->t_submit;
    r.t_admit = c->t_admit;
    r.t_done = s->now();
    s->done.push_back(r);
    s->stats.completed++;
    c->busy = false;
    s->active.erase(s->active.begin() + i);
    s->pool.push_back(c);
    (*changes)++;
  }
  return CL_OK;
}

}  // namespace

extern "C" {

cl_status cl_server_create(const cl_server_config* cfg, cl_server** out) {
  if (!cfg || !out) return fail(CL_ERR_INVALID, "NULL argument");
  *out = nullptr;
  if (cfg->max_slots < 1 || cfg->chunk_steps < 1 || !(cfg->hbm_budget_bytes > 0.0))
    return fail(CL_ERR_INVALID, "bad server configuration");
  if (cfg->prec != CL_FP64 && cfg->prec != CL_FP32_STORAGE && cfg->prec != CL_DF64)
    return fail(CL_ERR_INVALID, "bad precision");
  if (!(cfg->k_ref >= 0.0)) return fail(CL_ERR_INVALID, "k_ref must be >= 0");
  if (!(cfg->runaway_un >= 0.0)) return fail(CL_ERR_INVALID, "runaway_un must be >= 0");
  if (cfg->cool_enabled) {
    cl_status st = check_cool(&cfg->cool);
    if (st != CL_OK) return st;
  }
  cl_server* s = new cl_server();
  s->cfg = *cfg;
  s->t0 = std::chrono::steady_clock::now();
  std::memset(&s->stats, 0, sizeof(s->stats));
  *out = s;
  return CL_OK;
}

double cl_server_clock(const cl_server* s) { return s ? s->now() : 0.0; }

cl_status cl_server_submit(cl_server* s, const cl_request* req, double t_submit) {
  if (!s) return fail(CL_ERR_INVALID, "NULL server");
  cl_status st = check_request(s, req);
  if (st != CL_OK) return st;
  s->queue.push_back(Pending{*req, t_submit >= 0.0 ? t_submit : s->now()});
  s->stats.submitted++;
  return CL_OK;
}

cl_status cl_server_poll(cl_server* s, cl_result* out, int max_out, int* n_out) {
  if (!s || (max_out > 0 && !out)) return fail(CL_ERR_INVALID, "bad arguments");
  int changes = 0;
  cl_status st = collect(s, &changes);
  if (st == CL_OK) st = admit(s);
  int n = 0;
  while (n < max_out && !s->done.empty()) {
    out[n++] = s->done.front();
    s->done.pop_front();
  }
  if (n_out) *n_out = n;
  return st;
}

cl_status cl_server_stats_get(const cl_server* s, cl_server_stats* out) {
  if (!s || !out) return fail(CL_ERR_INVALID, "NULL argument");
  *out = s->stats;
  out->active = (int)s->active.size();
  out->queued = (int)s->queue.size();
  out->pooled = (int)s->pool.size();
  out->bytes_in_use = s->bytes;
  return CL_OK;
}

cl_status cl_server_run_trace(cl_server* s, int n, const cl_request* reqs, const double* arrival_s,
                              cl_result* results) {
  if (!s || n < 0 || (n > 0 && (!reqs || !arrival_s || !results))) return fail(CL_ERR_INVALID, "bad arguments");
  for (int i = 0; i < n; ++i) {
    cl_status st = check_request(s, &reqs[i]);
    if (st != CL_OK) return st;
    if (i > 0 && arrival_s[i] < arrival_s[i - 1]) return fail(CL_ERR_INVALID, "arrivals must be sorted");
  }
  const double base = s->now();
  int next = 0, got = 0;
  std::vector<cl_result> buf(64);
  while (got < n) {
    const double t = s->now() - base;
    while (next < n && arrival_s[next] <= t) {
      // latency is measured from the scheduled arrival, so host lag counts
      s->queue.push_back(Pending{reqs[next], base + arrival_s[next]});
      s->stats.submitted++;
      ++next;
    }
    int k = 0;
    cl_status st = cl_server_poll(s, buf.data(), (int)buf.size(), &k);
    if (st != CL_OK) return st;
    for (int j = 0; j < k; ++j) results[got++] = buf[j];
    if (k == 0) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  return CL_OK;
}

void cl_server_free(cl_server* s) {
  if (!s) return;
  for (Chain* c : s->active) destroy_chain(c);
  for (Chain* c : s->pool) destroy_chain(c);
  delete s;
}

}  // extern "C"
