// capi.cu -- the C-ABI runtime of libcl.so (include/cl.h): lattice state in
// HBM, the CL step / cooling / observables orchestration and host <-> device
// link exchange.  All arithmetic runs in the kernels (kernels.cu,
// k_update_*.cu); this file only allocates, sequences launches and copies.
#include <climits>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include <algorithm>
#include <chrono>
#include <thread>
#include <array>
#include <mutex>
#include <map>

#include <nvtx3/nvToolsExt.h>

#include "../../include/cl.h"
#include "launch.h"
#include "runtime.h"

using namespace clgc;
using namespace clrt;

namespace {
thread_local std::string g_err;
}  // namespace

namespace clrt {

const double KAPPA_Q = -1.0 / (256.0 * 9.86960440108935861883);  // q_L = kappa [Tr F F ...]

cl_status fail(cl_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

}  // namespace clrt

namespace clgc {
// Error text for entry points defined in other translation units.
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace clgc


namespace clrt {

// Internal precision codes equal cl_precision: 0 FP64, 1 FP32 storage, 2 DF64.
size_t real_size(const cl_lattice* l) { return l->prec == 1 ? 4 : 8; }
size_t align256(size_t n) { return (n + 255) / 256 * 256; }

cudaEvent_t take_event(cl_lattice* l) {
  if (!l->ev_pool->empty()) {
    cudaEvent_t e = l->ev_pool->back();
    l->ev_pool->pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Launch through f(); with timing on, bracket it by two events on the
// lattice's stream and remember them under `phase`.
const char* const PHASE_NAMES[CL_NPHASE] = {"clover", "update", "cool_grad", "cool_rule", "cool_omega",
                                            "cool_apply", "obs", "force", "cool_grad_omega"};

// NVTX range around the enqueue of one phase (a profiler shows the phases by
// name; without one attached the calls cost a few nanoseconds).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

template <typename Fn>
cudaError_t timed(cl_lattice* l, int phase, Fn f, int kernels = 1) {
  l->launches += kernels;
  NvtxRange r(PHASE_NAMES[phase]);
  if (!l->timing) return f();
  cudaEvent_t a = take_event(l), b = take_event(l);
  if (!a || !b) return cudaErrorMemoryAllocation;
  cudaEventRecord(a, l->st);
  cudaError_t e = f();
  cudaEventRecord(b, l->st);
  l->ev_pending->push_back({phase, {a, b}});
  return e;
}

cudaError_t resolve_timing(cl_lattice* l) {
  if (l->ev_pending->empty()) return cudaSuccess;
  cudaError_t e = cudaStreamSynchronize(l->st);
  if (e != cudaSuccess) return e;
  for (auto& p : *l->ev_pending) {
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, p.second.first, p.second.second);
    if (e != cudaSuccess) return e;
    l->phase_ms[p.first] += ms;
    l->phase_n[p.first] += 1;
    l->ev_pool->push_back(p.second.first);
    l->ev_pool->push_back(p.second.second);
  }
  l->ev_pending->clear();
  return cudaSuccess;
}

cl_status ensure_stage(cl_lattice* l) {
  if (l->stage) return CL_OK;
  CK(cudaMalloc(&l->stage, sizeof(double) * 18 * 4 * (size_t)l->g.V));
  return CL_OK;
}

bool theta_nonzero(const cl_lattice* l) { return l->p.theta_re != 0.0 || l->p.theta_im != 0.0; }

// The link-inverse pass: FP64 and DF64 only (the FP32-storage kernels form
// each inverse from its link where they use it).
bool needs_inverse_pass(const cl_lattice* l) { return l->prec != 1; }

// Link inverses, plaquettes and D = P - P^{-1}, then (theta != 0) the clover
// field scaled by (sre + i sim), then the per-plaquette drift contributions.
cudaError_t do_force(cl_lattice* l, bool th, double sre, double sim) {
  cudaError_t e = cudaSuccess;
  if (needs_inverse_pass(l))
    e = timed(l, CL_PHASE_CLOVER, [&] { return launch_link_inverse(l->prec, l->g, l->U, l->Ui, l->st); });
  if (e == cudaSuccess)
    e = timed(l, CL_PHASE_CLOVER, [&] { return launch_plaq(l->prec, l->g, l->U, l->Ui, l->Pq, l->Dq, l->st); });
  if (e == cudaSuccess && th)
    e = timed(l, CL_PHASE_CLOVER, [&] {
      return launch_clover_rot(l->prec, l->g, l->U, l->Ui, l->Dq, l->F, sre, sim, l->st);
    });
  if (e == cudaSuccess)
    e = timed(l, CL_PHASE_FORCE, [&] {
      return launch_plaq_force(l->prec, th, l->g, l->U, l->Ui, l->Pq, l->Dq, l->F, l->Gq, l->C, l->p.beta,
                               l->st);
    }, (th && l->prec != 1) ? 2 : 1);  // FP64 and DF64 split the theta force in two kernels
  return e;
}

cl_status do_steps(cl_lattice* l, double eps, int n) {
  const bool th = theta_nonzero(l);
  // F^ = -i theta kappa F: -i (a + ib) kappa = kappa b - i kappa a
  const double sre = KAPPA_Q * l->p.theta_im, sim = -KAPPA_Q * l->p.theta_re;
  for (int i = 0; i < n; ++i) {
    CK(do_force(l, th, sre, sim));
    const bool adaptive = l->k_ref > 0.0;
    if (adaptive) {
      // drift into the plaquette buffer (dead once the force has run) with
      // max |K|, then the step size on the device, then the update from the
      // stored drift
      CK(timed(l, CL_PHASE_UPDATE, [&] {
        return launch_update_gather(l->prec, 2, l->g, l->U, l->C, l->Pq, eps, l->p.seed, l->sd, false, l->st);
      }));
      CK(timed(l, CL_PHASE_UPDATE, [&] { return launch_step_eps(l->sd, eps, l->k_ref, l->st); }));
      CK(timed(l, CL_PHASE_UPDATE, [&] {
        return launch_update_gather(l->prec, 3, l->g, l->U, l->Pq, l->Un, eps, l->p.seed, l->sd, true, l->st);
      }));
    } else {
      CK(timed(l, CL_PHASE_UPDATE, [&] {
        return launch_update_gather(l->prec, 0, l->g, l->U, l->C, l->Un, eps, l->p.seed, l->sd, false, l->st);
      }));
    }
    // one-thread bookkeeping kernel: counted as a launch, not timed (so the update
    // phase's per-launch time stays that of the update kernel)
    CK(launch_step_bump(l->sd, eps, adaptive, l->st));
    l->launches++;
    std::swap(l->U, l->Un);
    l->step++;
  }
  return CL_OK;
}

CoolArgs cool_args(const cl_cool_params* cp) {
  CoolArgs a;
  a.eps = cp->eps;
  a.alpha = cp->alpha;
  a.tol_rel = cp->tol_rel;
  a.d_floor = cp->d_floor;
  a.d_guard = cp->d_guard;
  a.mode = (int)cp->mode;
  a.n_min = cp->n_min;
  a.n_max = cp->n_max;
  a.forced_sweeps = cp->forced_sweeps;
  return a;
}

cl_status check_cool(const cl_cool_params* cp) {
  if (!cp) return fail(CL_ERR_INVALID, "NULL cooling parameters");
  if ((int)cp->mode < 0 || (int)cp->mode > 3) return fail(CL_ERR_INVALID, "bad cooling mode");
  if (cp->forced_sweeps < 0 && (cp->n_max < 0 || cp->n_min < 0 || cp->n_min > cp->n_max))
    return fail(CL_ERR_INVALID, "bad sweep bounds");
  if (!(cp->eps >= 0.0) || !(cp->alpha >= 0.0)) return fail(CL_ERR_INVALID, "bad eps/alpha");
  return CL_OK;
}

// Enqueue the whole cooling loop; the device rule decides how many sweeps
// actually run (later launches return at once once it says done).
//
// D_0 and D_1 (FP64, FP32 storage) run single-pass sweeps: their strength
// needs only the unitarity norm, so after the first sweep each apply also
// sums the norm of the links it writes (one record per tile), the rule
// decides the next sweep from those records, and one kernel forms the
// gradient and Omega together (f stays in registers): rule, gradient +
// Omega, apply per sweep instead of gradient, rule, Omega, apply.  D_2 needs
// sum |f_ax| before Omega, so it keeps the four-kernel sweep, as does the
// DF64 form.
cl_status do_cool(cl_lattice* l, const cl_cool_params* cp) {
  CoolArgs a = cool_args(cp);
  const int n_iter = cp->forced_sweeps >= 0 ? cp->forced_sweeps : cp->n_max;
  const bool single_pass = (cp->mode == CL_D0 || cp->mode == CL_D1) && l->prec != 2;
  if (single_pass) {
    // sweep 0: the rule's first inputs from a plain gradient pass
    CK(timed(l, CL_PHASE_COOL_GRAD, [&] {
      return launch_cool_grad(l->prec, l->g, l->U, l->f, l->partials, nullptr, l->st);
    }));
    CK(timed(l, CL_PHASE_COOL_RULE, [&] { return launch_cool_adapt(l->g, l->partials, a, l->cs, 1, l->st); }));
    if (n_iter == 0) return CL_OK;
    CK(timed(l, CL_PHASE_COOL_OMEGA, [&] {
      return launch_cool_omega(l->prec, l->g, l->f, l->Om, l->Omi, cp->eps, l->cs, l->st);
    }));
    CK(timed(l, CL_PHASE_COOL_APPLY, [&] {
      return launch_cool_apply_tiles(l->prec, l->g, l->U, l->Om, l->Omi, l->crec, l->cs, l->st);
    }));
    for (int k = 1; k <= n_iter; ++k) {
      CK(timed(l, CL_PHASE_COOL_RULE, [&] { return launch_cool_adapt_tiles(l->g, l->crec, a, l->cs, l->st); }));
      if (k == n_iter) break;
      CK(timed(l, CL_PHASE_COOL_GRAD_OMEGA, [&] {
        return launch_cool_grad_omega(l->prec, l->g, l->U, l->Om, l->Omi, cp->eps, l->cs, l->st);
      }));
      CK(timed(l, CL_PHASE_COOL_APPLY, [&] {
        return launch_cool_apply_tiles(l->prec, l->g, l->U, l->Om, l->Omi, l->crec, l->cs, l->st);
      }));
    }
    return CL_OK;
  }
  for (int k = 0; k <= n_iter; ++k) {
    // the first gradient of a call always runs: the done flag still holds
    // the previous call's decision until the rule resets it (first = 1)
    CK(timed(l, CL_PHASE_COOL_GRAD, [&] {
      return launch_cool_grad(l->prec, l->g, l->U, l->f, l->partials, k == 0 ? nullptr : l->cs, l->st);
    }));
    CK(timed(l, CL_PHASE_COOL_RULE, [&] { return launch_cool_adapt(l->g, l->partials, a, l->cs, k == 0, l->st); }));
    if (k == n_iter) break;
    CK(timed(l, CL_PHASE_COOL_OMEGA, [&] {
      return launch_cool_omega(l->prec, l->g, l->f, l->Om, l->Omi, cp->eps, l->cs, l->st);
    }));
    CK(timed(l, CL_PHASE_COOL_APPLY, [&] { return launch_cool_apply(l->prec, l->g, l->U, l->Om, l->Omi, l->cs, l->st); }));
  }
  return CL_OK;
}

cl_status do_obs(cl_lattice* l, ObsOut* dst, double* q_site) {
  if (needs_inverse_pass(l))
    CK(timed(l, CL_PHASE_OBS, [&] { return launch_link_inverse(l->prec, l->g, l->U, l->Ui, l->st); }));
  CK(timed(l, CL_PHASE_OBS, [&] { return launch_plaq(l->prec, l->g, l->U, l->Ui, l->Pq, l->Dq, l->st); }));
  CK(timed(l, CL_PHASE_OBS, [&] { return launch_clover_rot(l->prec, l->g, l->U, l->Ui, l->Dq, l->F, 1.0, 0.0, l->st); }));
  CK(timed(l, CL_PHASE_OBS, [&] { return launch_obs(l->prec, l->g, l->U, l->F, 1, l->partials, q_site, l->st); }));
  CK(timed(l, CL_PHASE_OBS, [&] {
    return launch_obs_final(l->g, l->partials, l->p.beta, l->p.theta_re, l->p.theta_im, dst, l->st);
  }));
  return CL_OK;
}

void to_cl_obs(const ObsOut& o, cl_obs* out) {
  out->plaq_re = o.plaq_re;
  out->plaq_im = o.plaq_im;
  out->un = o.un;
  out->q_re = o.q_re;
  out->q_im = o.q_im;
  out->sw_re = o.sw_re;
  out->sw_im = o.sw_im;
  out->s_re = o.s_re;
  out->s_im = o.s_im;
  out->max_det_dev = o.max_det_dev;
}

void to_report(const CoolState& c, cl_cool_report* r) {
  r->sweeps = c.sweeps;
  r->alpha_ad_last = c.alpha_ad_last;
  r->un_before = c.un_before;
  r->un_after = c.un_after;
}

}  // namespace clrt

namespace clrt {

// Device bytes of one lattice (the buffers cl_init_lattice allocates).
size_t lattice_bytes(int V, int prec) {
  const size_t Vs = (size_t)V, esz = prec == 1 ? 8 : 16, real = prec == 1 ? 4 : 8;
  (void)real;  // the cooling fields and the parked force partials live inside C (see cl_init_lattice)
  const size_t inverses = prec == 1 ? 0 : 4;  // the FP32-storage form keeps no inverse field
  return esz * 9 * Vs * (4 + 4 + inverses + 6 + 6 + 24 + 6) + sizeof(double) * NQ_OBS * (size_t)reduce_blocks(V) +
         sizeof(CoolState) + sizeof(ObsOut) + sizeof(uint32_t);
}

// Start field, step counter and cooling state from l->p (cold or Haar start,
// then the optional random SL(3,C) gauge transformation).
cudaError_t init_state(cl_lattice* l) {
  const cl_params* params = &l->p;
  l->step = 0;
  cudaError_t e = cudaMemsetAsync(l->cs, 0, sizeof(CoolState), l->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(l->sd, 0, sizeof(StepDev), l->st);
  if (e == cudaSuccess)
    e = params->start == CL_START_HOT ? launch_hot(l->prec, l->g, l->U, params->seed, l->st)
                                      : launch_cold(l->prec, l->g, l->U, l->st);
  l->launches++;
  if (e == cudaSuccess && params->gauge_sigma > 0.0) {
    e = launch_gauge_omega(l->prec, l->g, l->Om, l->Omi, params->seed, params->gauge_sigma, l->st);
    if (e == cudaSuccess) e = launch_cool_apply(l->prec, l->g, l->U, l->Om, l->Omi, nullptr, l->st);
    l->launches += 2;
  }
  return e;
}

}  // namespace clrt

extern "C" {

cl_status cl_init_lattice(const cl_params* params, void* cuda_stream, cl_lattice** out) {
  if (!params || !out) return fail(CL_ERR_INVALID, "NULL argument");
  *out = nullptr;
  long long V = 1;
  for (int mu = 0; mu < 4; ++mu) {
    if (params->L[mu] < 1) return fail(CL_ERR_INVALID, "lattice extent < 1");
    V *= params->L[mu];
    if (V * 6 * 9 > INT_MAX) return fail(CL_ERR_INVALID, "lattice too large");
  }
  if (params->prec != CL_FP64 && params->prec != CL_FP32_STORAGE && params->prec != CL_DF64)
    return fail(CL_ERR_INVALID, "bad precision");
  if (params->start != CL_START_COLD && params->start != CL_START_HOT)
    return fail(CL_ERR_INVALID, "bad start");
  cl_lattice* l = new cl_lattice();
  std::memset(l, 0, sizeof(*l));
  l->p = *params;
  for (int mu = 0; mu < 4; ++mu) l->g.L[mu] = params->L[mu];
  l->g.V = (int)V;
  l->prec = (int)params->prec;
  l->esz = l->prec == 1 ? 8 : 16;
  l->st = (cudaStream_t)cuda_stream;
  l->ev_pool = new std::vector<cudaEvent_t>();
  l->ev_pending = new std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>>();
  cl_status s = CL_OK;
  auto alloc = [&](void** p, size_t bytes) {
    if (s != CL_OK) return;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess)
      s = fail(e == cudaErrorMemoryAllocation ? CL_ERR_OOM : CL_ERR_CUDA,
               std::string("cudaMalloc: ") + cudaGetErrorString(e));
  };
  const size_t Vs = (size_t)V;
  alloc(&l->U, l->esz * 4 * 9 * Vs);
  alloc(&l->Un, l->esz * 4 * 9 * Vs);
  if (needs_inverse_pass(l)) alloc(&l->Ui, l->esz * 4 * 9 * Vs);  // FP32 storage forms inverses in place
  alloc(&l->Pq, l->esz * 6 * 9 * Vs);
  alloc(&l->Dq, l->esz * 6 * 9 * Vs);
  alloc(&l->C, l->esz * 24 * 9 * Vs);

  alloc(&l->F, l->esz * 6 * 9 * Vs);

  alloc((void**)&l->partials, sizeof(double) * NQ_OBS * (size_t)reduce_blocks(l->g.V));
  alloc((void**)&l->cs, sizeof(CoolState));
  alloc((void**)&l->obs, sizeof(ObsOut));
  alloc((void**)&l->sd, sizeof(StepDev));
  if (s != CL_OK) {
    cl_free(l);
    return s;
  }
  // Buffers that live inside C, whose 24 planes of drift contributions are
  // dead outside the CL step's force -> update window:
  //  * Gq, the split force's parked partial sums: plane p at C plane 4p + 1
  //    (Gq points at plane 1; the force kernels index it GQ_PLANE * p), the
  //    slot that stage b writes only after reading the partial back;
  //  * the cooling fields f (8 FP64 per site, [a][V]) and the packed
  //    Hermitian Omega, Omega^{-1} (9 reals per site each), then, on a
  //    256-byte boundary, the single-pass apply's tile records (16 bytes per
  //    tile, at most V / 128 + L3 tiles); used only by the cooling sweeps and
  //    the start's gauge transformation, never while C holds drift
  //    contributions.  They need at most 64 + 144 + 17 bytes per site plus
  //    256, and C has 24 * 9 * 8 bytes per site or more.
  {
    char* c = (char*)l->C;
    l->Gq = c + l->esz * 9 * Vs;
    l->f = c;
    l->Om = c + sizeof(double) * 8 * Vs;
    l->Omi = c + sizeof(double) * 8 * Vs + real_size(l) * 9 * Vs;
    l->crec = (double*)(c + align256(sizeof(double) * 8 * Vs + 2 * real_size(l) * 9 * Vs));
  }
  cudaError_t e = l->prec == 2 ? prepare_df64_kernels() : cudaSuccess;
  if (e == cudaSuccess) e = init_state(l);
  if (e != cudaSuccess) {
    cl_free(l);
    return fail(CL_ERR_CUDA, std::string("init: ") + cudaGetErrorString(e));
  }
  *out = l;
  return CL_OK;
}

cl_status cl_reset_lattice(cl_lattice* l, const cl_params* params) {
  if (!l || !params) return fail(CL_ERR_INVALID, "NULL argument");
  for (int mu = 0; mu < 4; ++mu)
    if (params->L[mu] != l->p.L[mu]) return fail(CL_ERR_INVALID, "reset needs the same extents");
  if (params->prec != l->p.prec) return fail(CL_ERR_INVALID, "reset needs the same precision");
  if (params->start != CL_START_COLD && params->start != CL_START_HOT)
    return fail(CL_ERR_INVALID, "bad start");
  CK(cudaStreamSynchronize(l->st));
  CK(resolve_timing(l));
  for (int v = 0; v < 2; ++v)
    if (l->gexec[v]) {
      cudaGraphExecDestroy(l->gexec[v]);
      l->gexec[v] = nullptr;
    }
  l->p = *params;
  CK(init_state(l));
  return CL_OK;
}

cl_status cl_lattice_bytes(const cl_params* params, size_t* bytes) {
  if (!params || !bytes) return fail(CL_ERR_INVALID, "NULL argument");
  long long V = 1;
  for (int mu = 0; mu < 4; ++mu) {
    if (params->L[mu] < 1) return fail(CL_ERR_INVALID, "lattice extent < 1");
    V *= params->L[mu];
    if (V * 6 * 9 > INT_MAX) return fail(CL_ERR_INVALID, "lattice too large");
  }
  if (params->prec != CL_FP64 && params->prec != CL_FP32_STORAGE && params->prec != CL_DF64)
    return fail(CL_ERR_INVALID, "bad precision");
  *bytes = lattice_bytes((int)V, (int)params->prec);
  return CL_OK;
}

cl_status cl_step(cl_lattice* l, double eps, int n_steps) {
  if (!l) return fail(CL_ERR_INVALID, "NULL lattice");
  if (!(eps >= 0.0) || n_steps < 0) return fail(CL_ERR_INVALID, "bad eps or n_steps");
  return do_steps(l, eps, n_steps);
}

cl_status cl_cool(cl_lattice* l, const cl_cool_params* cp, cl_cool_report* report) {
  if (!l) return fail(CL_ERR_INVALID, "NULL lattice");
  cl_status s = check_cool(cp);
  if (s != CL_OK) return s;
  s = do_cool(l, cp);
  if (s != CL_OK || !report) return s;
  CoolState c;
  CK(cudaMemcpyAsync(&c, l->cs, sizeof(c), cudaMemcpyDeviceToHost, l->st));
  CK(cudaStreamSynchronize(l->st));
  to_report(c, report);
  if (c.nonfinite) return fail(CL_ERR_NONFINITE, "non-finite links during cooling");
  return CL_OK;
}

cl_status cl_cool_last_report(cl_lattice* l, cl_cool_report* report) {
  if (!l || !report) return fail(CL_ERR_INVALID, "NULL argument");
  CoolState c;
  CK(cudaMemcpyAsync(&c, l->cs, sizeof(c), cudaMemcpyDeviceToHost, l->st));
  CK(cudaStreamSynchronize(l->st));
  to_report(c, report);
  if (c.nonfinite) return fail(CL_ERR_NONFINITE, "non-finite links during cooling");
  return CL_OK;
}

cl_status cl_observables(cl_lattice* l, cl_obs* out) {
  if (!l || !out) return fail(CL_ERR_INVALID, "NULL argument");
  cl_status s = do_obs(l, l->obs, nullptr);
  if (s != CL_OK) return s;
  ObsOut o;
  CK(cudaMemcpyAsync(&o, l->obs, sizeof(o), cudaMemcpyDeviceToHost, l->st));
  CK(cudaStreamSynchronize(l->st));
  to_cl_obs(o, out);
  if (o.nonfinite != 0.0) return fail(CL_ERR_NONFINITE, "non-finite links");
  return CL_OK;
}

cl_status cl_trajectory(cl_lattice* l, double eps, int n_steps, const cl_cool_params* cp,
                        int obs_every, cl_obs* obs_out, cl_cool_report* rep_out,
                        double runaway_un) {
  if (!l) return fail(CL_ERR_INVALID, "NULL lattice");
  if (!(eps >= 0.0) || n_steps < 0) return fail(CL_ERR_INVALID, "bad eps or n_steps");
  if (cp) {
    cl_status s = check_cool(cp);
    if (s != CL_OK) return s;
  }
  const int nrec = obs_every > 0 ? n_steps / obs_every : 0;
  ObsOut* dobs = nullptr;
  CoolState* dcs = nullptr;
  if (nrec > 0) {
    CK(cudaMalloc(&dobs, sizeof(ObsOut) * nrec));
    cudaError_t e = cudaMalloc(&dcs, sizeof(CoolState) * nrec);
    if (e != cudaSuccess) {
      cudaFree(dobs);
      return fail(CL_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
  }
  cl_status s = CL_OK;
  int rec = 0;
  for (int i = 0; i < n_steps && s == CL_OK; ++i) {
    s = do_steps(l, eps, 1);
    if (s == CL_OK && cp) s = do_cool(l, cp);
    if (s == CL_OK && nrec > 0 && (i + 1) % obs_every == 0) {
      s = do_obs(l, dobs + rec, nullptr);
      if (s == CL_OK && cp) {
        cudaError_t e = cudaMemcpyAsync(dcs + rec, l->cs, sizeof(CoolState), cudaMemcpyDeviceToDevice, l->st);
        if (e != cudaSuccess) s = fail(CL_ERR_CUDA, cudaGetErrorString(e));
      }
      ++rec;
    }
  }
  if (s == CL_OK && nrec > 0) {
    std::vector<ObsOut> ho(nrec);
    std::vector<CoolState> hc(nrec);
    cudaError_t e = cudaMemcpyAsync(ho.data(), dobs, sizeof(ObsOut) * nrec, cudaMemcpyDeviceToHost, l->st);
    if (e == cudaSuccess && cp)
      e = cudaMemcpyAsync(hc.data(), dcs, sizeof(CoolState) * nrec, cudaMemcpyDeviceToHost, l->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(l->st);
    if (e != cudaSuccess) {
      s = fail(CL_ERR_CUDA, cudaGetErrorString(e));
    } else {
      for (int k = 0; k < nrec; ++k) {
        if (obs_out) to_cl_obs(ho[k], obs_out + k);
        if (rep_out) {
          if (cp) to_report(hc[k], rep_out + k);
          else std::memset(rep_out + k, 0, sizeof(cl_cool_report));
        }
        if (ho[k].nonfinite != 0.0 && s == CL_OK) s = fail(CL_ERR_NONFINITE, "non-finite links");
        if (runaway_un > 0.0 && ho[k].un > runaway_un && s == CL_OK)
          s = fail(CL_ERR_RUNAWAY, "unitarity norm above the runaway bound");
      }
    }
  }
  if (dobs) cudaFree(dobs);
  if (dcs) cudaFree(dcs);
  return s;
}

cl_status cl_get_links_device(cl_lattice* l, double* dev_aos) {
  if (!l || !dev_aos) return fail(CL_ERR_INVALID, "NULL argument");
  CK(launch_soa_to_aos(l->prec, l->g, l->U, dev_aos, 4, l->st));
  l->launches++;
  return CL_OK;
}

cl_status cl_set_links_device(cl_lattice* l, const double* dev_aos) {
  if (!l || !dev_aos) return fail(CL_ERR_INVALID, "NULL argument");
  CK(launch_aos_to_soa(l->prec, l->g, dev_aos, l->U, 4, l->st));
  l->launches++;
  return CL_OK;
}

// The device's view of page-locked host memory (cudaHostAlloc, a registered
// range, a framework's pinned tensor), else NULL (pageable memory).  The
// layout kernels then read or write the host array directly over the
// host link, one pass instead of a copy through the staging buffer plus a
// pass over it.
static void* device_view(const void* host) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
    cudaGetLastError();  // not a pointer CUDA knows: clear the error, take the copy path
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

cl_status cl_get_links(cl_lattice* l, double* host_aos) {
  if (!l || !host_aos) return fail(CL_ERR_INVALID, "NULL argument");
  if (double* dv = (double*)device_view(host_aos)) {
    cl_status s = cl_get_links_device(l, dv);
    if (s != CL_OK) return s;
    CK(cudaStreamSynchronize(l->st));
    return CL_OK;
  }
  cl_status s = ensure_stage(l);
  if (s != CL_OK) return s;
  s = cl_get_links_device(l, l->stage);
  if (s != CL_OK) return s;
  CK(cudaMemcpyAsync(host_aos, l->stage, sizeof(double) * 18 * 4 * (size_t)l->g.V,
                     cudaMemcpyDeviceToHost, l->st));
  CK(cudaStreamSynchronize(l->st));
  return CL_OK;
}

cl_status cl_set_links(cl_lattice* l, const double* host_aos) {
  if (!l || !host_aos) return fail(CL_ERR_INVALID, "NULL argument");
  if (const double* dv = (const double*)device_view(host_aos)) {
    cl_status s = cl_set_links_device(l, dv);
    if (s != CL_OK) return s;
    // the host buffer may be reused on return: wait for the pass that reads it
    CK(cudaStreamSynchronize(l->st));
    return CL_OK;
  }
  cl_status s = ensure_stage(l);
  if (s != CL_OK) return s;
  CK(cudaMemcpyAsync(l->stage, host_aos, sizeof(double) * 18 * 4 * (size_t)l->g.V,
                     cudaMemcpyHostToDevice, l->st));
  s = cl_set_links_device(l, l->stage);
  if (s != CL_OK) return s;
  // the host buffer may be reused on return: wait for the copy only
  CK(cudaStreamSynchronize(l->st));
  return CL_OK;
}

cl_status cl_get_step(const cl_lattice* l, uint64_t* step) {
  if (!l || !step) return fail(CL_ERR_INVALID, "NULL argument");
  *step = l->step;
  return CL_OK;
}

cl_status cl_set_step(cl_lattice* l, uint64_t step) {
  if (!l) return fail(CL_ERR_INVALID, "NULL lattice");
  if (step > 0xffffffffull) return fail(CL_ERR_INVALID, "step beyond the 32-bit Philox counter word");
  l->step = step;
  static thread_local uint32_t v;
  v = (uint32_t)step;
  static_assert(offsetof(StepDev, step) == 0, "the step word leads StepDev");
  CK(cudaMemcpyAsync(reinterpret_cast<uint32_t*>(l->sd), &v, sizeof(uint32_t), cudaMemcpyHostToDevice, l->st));
  CK(cudaStreamSynchronize(l->st));
  return CL_OK;
}

cl_status cl_set_adaptive_step(cl_lattice* l, double k_ref) {
  if (!l) return fail(CL_ERR_INVALID, "NULL lattice");
  if (!(k_ref >= 0.0)) return fail(CL_ERR_INVALID, "k_ref must be >= 0");
  l->k_ref = k_ref;
  return CL_OK;
}

cl_status cl_get_langevin_time(cl_lattice* l, double* t, double* eps_last, double* kmax_last) {
  if (!l) return fail(CL_ERR_INVALID, "NULL lattice");
  StepDev h;
  CK(cudaMemcpyAsync(&h, l->sd, sizeof(StepDev), cudaMemcpyDeviceToHost, l->st));
  CK(cudaStreamSynchronize(l->st));
  if (t) *t = h.t;
  if (eps_last) *eps_last = h.eps_n;
  if (kmax_last) *kmax_last = h.kmax;
  return CL_OK;
}

cl_status cl_drift(cl_lattice* l, double* host_aos) {
  if (!l || !host_aos) return fail(CL_ERR_INVALID, "NULL argument");
  cl_status s = ensure_stage(l);
  if (s != CL_OK) return s;
  const bool th = theta_nonzero(l);
  CK(do_force(l, th, KAPPA_Q * l->p.theta_im, -KAPPA_Q * l->p.theta_re));
  CK(launch_update_gather(l->prec, 1, l->g, l->U, l->C, l->Un, 0.0, l->p.seed, l->sd, false, l->st));
  CK(launch_soa_to_aos(l->prec, l->g, l->Un, l->stage, 4, l->st));
  l->launches += 2;
  CK(cudaMemcpyAsync(host_aos, l->stage, sizeof(double) * 18 * 4 * (size_t)l->g.V,
                     cudaMemcpyDeviceToHost, l->st));
  CK(cudaStreamSynchronize(l->st));
  return CL_OK;
}

cl_status cl_cool_gradient(cl_lattice* l, double* host_f) {
  if (!l || !host_f) return fail(CL_ERR_INVALID, "NULL argument");
  CK(launch_cool_grad(l->prec, l->g, l->U, l->f, l->partials, nullptr, l->st));
  l->launches++;
  const size_t n = 8 * (size_t)l->g.V;
  CK(cudaMemcpyAsync(host_f, l->f, sizeof(double) * n, cudaMemcpyDeviceToHost, l->st));
  CK(cudaStreamSynchronize(l->st));
  if (l->prec == 2) {  // DF64 keeps f as (hi, lo) float pairs: widen in place
    for (size_t i = 0; i < n; ++i) {
      float hl[2];
      std::memcpy(hl, host_f + i, sizeof(hl));
      host_f[i] = (double)hl[0] + (double)hl[1];
    }
  }
  return CL_OK;
}

cl_status cl_noise_sample(cl_precision prec, uint64_t seed, uint32_t step, int mu, int site0, int nsites,
                          double* host_out) {
  if (!host_out) return fail(CL_ERR_INVALID, "NULL argument");
  if (prec != CL_FP64 && prec != CL_FP32_STORAGE && prec != CL_DF64) return fail(CL_ERR_INVALID, "bad precision");
  if (nsites < 0 || site0 < 0 || mu < 0 || mu > 3 || (long long)site0 + nsites > INT_MAX)
    return fail(CL_ERR_INVALID, "bad site range or direction");
  if (nsites == 0) return CL_OK;
  double* d = nullptr;
  const size_t bytes = sizeof(double) * 8 * (size_t)nsites;
  cudaError_t e = cudaMalloc(&d, bytes);
  if (e != cudaSuccess)
    return fail(e == cudaErrorMemoryAllocation ? CL_ERR_OOM : CL_ERR_CUDA, cudaGetErrorString(e));
  e = launch_noise_sample((int)prec, site0, nsites, seed, step, mu, d, 0);
  if (e == cudaSuccess) e = cudaMemcpy(host_out, d, bytes, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return fail(CL_ERR_CUDA, cudaGetErrorString(e));
  return CL_OK;
}

cl_status cl_selftest_convert(uint64_t seed, int64_t n, int64_t* bad_f2d, int64_t* bad_d2f) {
  if (!bad_f2d || !bad_d2f || n < 0) return fail(CL_ERR_INVALID, "NULL argument or n < 0");
  unsigned long long* d = nullptr;
  cudaError_t e = cudaMalloc(&d, 2 * sizeof(unsigned long long));
  if (e != cudaSuccess)
    return fail(e == cudaErrorMemoryAllocation ? CL_ERR_OOM : CL_ERR_CUDA, cudaGetErrorString(e));
  unsigned long long h[2] = {0, 0};
  e = cudaMemset(d, 0, sizeof(h));
  if (e == cudaSuccess) e = launch_selftest_convert(seed, (long long)n, d, 0);
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return fail(CL_ERR_CUDA, cudaGetErrorString(e));
  *bad_f2d = (int64_t)h[0];
  *bad_d2f = (int64_t)h[1];
  return CL_OK;
}

cl_status cl_selftest_box_muller(uint64_t seed, int64_t n, int64_t* ulp_ln, int64_t* ulp_sincos) {
  if (!ulp_ln || !ulp_sincos || n < 0) return fail(CL_ERR_INVALID, "NULL argument or n < 0");
  unsigned long long* d = nullptr;
  cudaError_t e = cudaMalloc(&d, 2 * sizeof(unsigned long long));
  if (e != cudaSuccess)
    return fail(e == cudaErrorMemoryAllocation ? CL_ERR_OOM : CL_ERR_CUDA, cudaGetErrorString(e));
  unsigned long long h[2] = {0, 0};
  e = cudaMemset(d, 0, sizeof(h));
  if (e == cudaSuccess) e = launch_selftest_box_muller(seed, (long long)n, d, 0);
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return fail(CL_ERR_CUDA, cudaGetErrorString(e));
  *ulp_ln = (int64_t)h[0];
  *ulp_sincos = (int64_t)h[1];
  return CL_OK;
}

cl_status cl_qdensity(cl_lattice* l, double* host_q) {
  if (!l || !host_q) return fail(CL_ERR_INVALID, "NULL argument");
  if (!l->qsite) CK(cudaMalloc(&l->qsite, sizeof(double) * 2 * (size_t)l->g.V));
  cl_status s = do_obs(l, l->obs, l->qsite);
  if (s != CL_OK) return s;
  CK(cudaMemcpyAsync(host_q, l->qsite, sizeof(double) * 2 * (size_t)l->g.V,
                     cudaMemcpyDeviceToHost, l->st));
  CK(cudaStreamSynchronize(l->st));
  return CL_OK;
}

cl_status cl_launch_count(const cl_lattice* l, int64_t* count) {
  if (!l || !count) return fail(CL_ERR_INVALID, "NULL argument");
  *count = l->launches;
  return CL_OK;
}

// ------------------------------------------------------------- graphs
}  // extern "C"

namespace clrt {

// Enqueue one step of the hot path (CL step, then cooling when cp != NULL).
cl_status enqueue_step(cl_lattice* l, double eps, const cl_cool_params* cp) {
  cl_status s = do_steps(l, eps, 1);
  if (s == CL_OK && cp) s = do_cool(l, cp);
  return s;
}

cl_status check_step_args(const cl_lattice* l, double eps, const cl_cool_params* cp) {
  if (!l) return fail(CL_ERR_INVALID, "NULL lattice");
  if (!l->st) return fail(CL_ERR_INVALID, "graphs need a non-default stream (cl_init_lattice)");
  if (!(eps >= 0.0)) return fail(CL_ERR_INVALID, "bad eps");
  return cp ? check_cool(cp) : CL_OK;
}

}  // namespace clrt

extern "C" {

cl_status cl_capture_step(cl_lattice* l, double eps, const cl_cool_params* cp) {
  cl_status s = check_step_args(l, eps, cp);
  if (s != CL_OK) return s;
  for (int v = 0; v < 2; ++v)
    if (l->gexec[v]) {
      cudaGraphExecDestroy(l->gexec[v]);
      l->gexec[v] = nullptr;
    }
  const int timing = l->timing;
  void* const U0 = l->U;
  void* const Un0 = l->Un;
  l->timing = 0;
  // two variants: the update writes the other link buffer, so replays alternate
  for (int v = 0; v < 2 && s == CL_OK; ++v) {
    l->gU[v] = l->U;
    const uint64_t step0 = l->step;
    const int64_t n0 = l->launches;
    cudaError_t e = cudaStreamBeginCapture(l->st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      s = fail(CL_ERR_CUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
      break;
    }
    s = enqueue_step(l, eps, cp);
    l->glaunches = l->launches - n0;
    cudaGraph_t gr = nullptr;
    e = cudaStreamEndCapture(l->st, &gr);
    l->step = step0;
    l->launches = n0;
    if (s == CL_OK && e != cudaSuccess) s = fail(CL_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
    if (s == CL_OK) {
      e = cudaGraphInstantiate(&l->gexec[v], gr, 0);
      if (e != cudaSuccess) s = fail(CL_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    if (gr) cudaGraphDestroy(gr);
  }
  l->timing = timing;
  // each variant swapped the buffers once: after two they are back in place
  l->U = U0;
  l->Un = Un0;
  if (s != CL_OK)
    for (int v = 0; v < 2; ++v)
      if (l->gexec[v]) {
        cudaGraphExecDestroy(l->gexec[v]);
        l->gexec[v] = nullptr;
      }
  return s;
}

cl_status cl_replay(cl_lattice* l, int n_steps) {
  if (!l || n_steps < 0) return fail(CL_ERR_INVALID, "bad arguments");
  if (!l->gexec[0]) return fail(CL_ERR_INVALID, "no captured step (cl_capture_step)");
  for (int i = 0; i < n_steps; ++i) {
    const int v = (l->U == l->gU[0]) ? 0 : 1;
    CK(cudaGraphLaunch(l->gexec[v], l->st));
    l->launches += l->glaunches;
    std::swap(l->U, l->Un);
    l->step++;
  }
  return CL_OK;
}

struct cl_batch {
  std::vector<cl_lattice*> lats;
  std::vector<double> eps;
  std::vector<cl_cool_params> cps;
  int with_cooling;
  cudaStream_t origin;
  cudaEvent_t fork, done;
  std::vector<cudaEvent_t> joins, ready;
  cudaGraphExec_t exec[2];
  std::vector<void*> startU[2];  // per lattice, the link buffer each variant starts from
  // fused mode: one launch per kernel family over the blocks of every chain
  int fused;
  void* dmem;                    // descriptors of both variants, work lists, chain lists (one allocation)
};

namespace {

void drop_graphs(cl_batch* b) {
  for (int v = 0; v < 2; ++v)
    if (b->exec[v]) {
      cudaGraphExecDestroy(b->exec[v]);
      b->exec[v] = nullptr;
    }
  if (b->dmem) {
    cudaFree(b->dmem);
    b->dmem = nullptr;
  }
  for (cudaEvent_t e : b->joins)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : b->ready)
    if (e) cudaEventDestroy(e);
  b->joins.clear();
  b->ready.clear();
}

cl_status check_batch_member(const cl_batch* b, const cl_lattice* l, double eps, const cl_cool_params* cp) {
  cl_status s = check_step_args(l, eps, cp);
  if (s != CL_OK) return s;
  for (const cl_lattice* m : b->lats)
    if (m == l || m->st == l->st)
      return fail(CL_ERR_INVALID, "batch lattices need distinct lattices on distinct streams");
  return CL_OK;
}

// ---- fused mode
// Host plan of a fused step: the work lists of every kernel family and the
// chain lists of the per-chain kernels, offsets into one device allocation.
struct FusedPlan {
  std::vector<WorkItem> items;
  std::vector<int> ints;
  struct List {
    size_t off;
    int n;
  };
  List fam[ENS_NFAM + 3];  // + the gradient of the first sweep (all chains), the first Omega (all), spare
  List all_chains, adaptive_chains, adaptive_flags, sp_chains, four_chains;
  int n_iter;
  bool any_adaptive;
};
enum { ENS_FIRST_GRAD = ENS_NFAM, ENS_FIRST_OMEGA = ENS_NFAM + 1 };

bool single_pass_chain(const cl_lattice* l, const cl_cool_params& cp) {
  return (cp.mode == CL_D0 || cp.mode == CL_D1) && l->prec != 2;
}

FusedPlan plan_fused(const cl_batch* b) {
  FusedPlan P;
  const int n = (int)b->lats.size();
  auto add = [&](int fam, auto pred, auto blocks) {
    P.fam[fam].off = P.items.size();
    for (int i = 0; i < n; ++i)
      if (pred(i)) {
        const int nb = blocks(b->lats[i]->g.V);
        for (int vb = 0; vb < nb; ++vb) P.items.push_back(WorkItem{i, vb});
      }
    P.fam[fam].n = (int)(P.items.size() - P.fam[fam].off);
  };
  auto th = [&](int i) { return theta_nonzero(b->lats[i]); };
  auto ad = [&](int i) { return b->lats[i]->k_ref > 0.0; };
  auto sp = [&](int i) { return b->with_cooling && single_pass_chain(b->lats[i], b->cps[i]); };
  auto cool = [&](int i) { return b->with_cooling != 0; };
  auto four = [&](int i) { return b->with_cooling && !single_pass_chain(b->lats[i], b->cps[i]); };
  auto all = [&](int) { return true; };
  auto tiles = [](int V) { return (V + ENS_BLOCK - 1) / ENS_BLOCK; };
  auto x4 = [&](int V) { return 4 * tiles(V); };
  auto x6 = [&](int V) { return 6 * tiles(V); };
  auto red = [](int V) { return reduce_blocks(V); };
  add(ENS_INVERSE, [&](int i) { return needs_inverse_pass(b->lats[i]); }, x4);
  add(ENS_PLAQ, all, x6);
  add(ENS_CLOVER, th, x6);
  add(ENS_FORCE_WILSON, [&](int i) { return !th(i); }, x6);
  add(ENS_FORCE_THETA, th, x6);
  add(ENS_UPDATE, [&](int i) { return !ad(i); }, x4);
  add(ENS_DRIFTMAX, ad, x4);
  add(ENS_UPDATE_X, ad, x4);
  add(ENS_FIRST_GRAD, cool, red);
  add(ENS_FIRST_OMEGA, cool, tiles);
  add(ENS_COOL_GRAD, four, red);
  add(ENS_COOL_OMEGA, four, tiles);
  add(ENS_COOL_APPLY, four, x4);
  add(ENS_COOL_GRAD_OMEGA, sp, red);
  P.fam[ENS_COOL_APPLY_UN].off = P.items.size();
  for (int i = 0; i < n; ++i)
    if (sp(i)) {
      const int nt = cool_tiles(b->lats[i]->g);
      for (int t = 0; t < nt; ++t) P.items.push_back(WorkItem{i, t});
    }
  P.fam[ENS_COOL_APPLY_UN].n = (int)(P.items.size() - P.fam[ENS_COOL_APPLY_UN].off);
  P.all_chains.off = P.ints.size();
  for (int i = 0; i < n; ++i) P.ints.push_back(i);
  P.all_chains.n = n;
  P.adaptive_chains.off = P.ints.size();
  for (int i = 0; i < n; ++i)
    if (ad(i)) P.ints.push_back(i);
  P.adaptive_chains.n = (int)(P.ints.size() - P.adaptive_chains.off);
  P.adaptive_flags.off = P.ints.size();
  for (int i = 0; i < n; ++i) P.ints.push_back(ad(i) ? 1 : 0);
  P.adaptive_flags.n = n;
  P.sp_chains.off = P.ints.size();
  for (int i = 0; i < n; ++i)
    if (sp(i)) P.ints.push_back(i);
  P.sp_chains.n = (int)(P.ints.size() - P.sp_chains.off);
  P.four_chains.off = P.ints.size();
  for (int i = 0; i < n; ++i)
    if (four(i)) P.ints.push_back(i);
  P.four_chains.n = (int)(P.ints.size() - P.four_chains.off);
  P.any_adaptive = P.adaptive_chains.n > 0;
  P.n_iter = 0;
  if (b->with_cooling)
    for (const cl_cool_params& cp : b->cps) P.n_iter = std::max(P.n_iter, cp.forced_sweeps >= 0 ? cp.forced_sweeps : cp.n_max);
  return P;
}

ChainDesc describe(const cl_lattice* l, double eps, const cl_cool_params& cp, bool swapped) {
  ChainDesc c;
  std::memset(&c, 0, sizeof(c));
  int st = 1;
  for (int mu = 0; mu < 4; ++mu) {
    c.L[mu] = l->g.L[mu];
    c.stride[mu] = st;
    st *= l->g.L[mu];
  }
  c.V = l->g.V;
  c.U = swapped ? l->Un : l->U;
  c.Un = swapped ? l->U : l->Un;
  c.Ui = l->Ui;
  c.Pq = l->Pq;
  c.Dq = l->Dq;
  c.F = l->F;
  c.C = l->C;
  c.Gq = l->Gq;
  c.f = l->f;
  c.Om = l->Om;
  c.Omi = l->Omi;
  c.partials = l->partials;
  c.arec = l->crec;
  c.cs = l->cs;
  c.sd = l->sd;
  c.beta = l->p.beta;
  c.sre = KAPPA_Q * l->p.theta_im;  // F^ = -i theta kappa F, as in do_steps
  c.sim = -KAPPA_Q * l->p.theta_re;
  c.eps = eps;
  c.sqrt_eps = sqrt(eps);
  c.k_ref = l->k_ref;
  c.seed = l->p.seed;
  c.ca = cool_args(&cp);
  return c;
}

// One fused step of every chain, enqueued on st from descriptor table cd.
// Each chain runs exactly the kernels and the order of its own step: the CL
// step (force by theta, update by step-size mode), then its cooling sweeps,
// single-pass for D_0 / D_1 and four kernels otherwise, up to the largest
// sweep count of the batch (a chain's own rule marks it done at its count;
// later launches skip its blocks).  Returns the number of launches.
cl_status enqueue_fused_step(const cl_batch* b, const FusedPlan& P, const ChainDesc* cd, const WorkItem* w,
                             const int* ints, cudaStream_t st, int64_t* launches) {
  const int prec = b->lats[0]->prec;
  int64_t nl = 0;
  auto fam = [&](int f, int list, int arg) -> cudaError_t {
    if (P.fam[list].n == 0) return cudaSuccess;
    nl += (f == ENS_FORCE_THETA && prec == 0) ? 2 : 1;
    return launch_ens(prec, f, cd, w + P.fam[list].off, P.fam[list].n, arg, st);
  };
  CK(fam(ENS_INVERSE, ENS_INVERSE, 0));
  CK(fam(ENS_PLAQ, ENS_PLAQ, 0));
  CK(fam(ENS_CLOVER, ENS_CLOVER, 0));
  CK(fam(ENS_FORCE_WILSON, ENS_FORCE_WILSON, 0));
  CK(fam(ENS_FORCE_THETA, ENS_FORCE_THETA, 0));
  if (P.any_adaptive) {
    CK(fam(ENS_DRIFTMAX, ENS_DRIFTMAX, 0));
    CK(launch_ens_step_eps(cd, ints + P.adaptive_chains.off, P.adaptive_chains.n, st));
    ++nl;
    CK(fam(ENS_UPDATE_X, ENS_UPDATE_X, 0));
  }
  CK(fam(ENS_UPDATE, ENS_UPDATE, 0));
  CK(launch_ens_step_bump(cd, ints + P.all_chains.off, ints + P.adaptive_flags.off, P.all_chains.n, st));
  ++nl;
  if (b->with_cooling) {
    const int* all = ints + P.all_chains.off;
    const int n = P.all_chains.n;
    CK(fam(ENS_COOL_GRAD, ENS_FIRST_GRAD, 1));
    CK(launch_ens_cool_adapt(cd, all, n, 1, st));
    ++nl;
    if (P.n_iter > 0) {
      CK(fam(ENS_COOL_OMEGA, ENS_FIRST_OMEGA, 0));
      CK(fam(ENS_COOL_APPLY, ENS_COOL_APPLY, 0));
      CK(fam(ENS_COOL_APPLY_UN, ENS_COOL_APPLY_UN, 0));
    }
    for (int k = 1; k <= P.n_iter; ++k) {
      CK(fam(ENS_COOL_GRAD, ENS_COOL_GRAD, 0));
      // the rule: four-kernel chains from the gradient's records, single-pass
      // chains from their apply's tile records
      if (P.four_chains.n) {
        CK(launch_ens_cool_adapt(cd, ints + P.four_chains.off, P.four_chains.n, 0, st));
        ++nl;
      }
      if (P.sp_chains.n) {
        CK(launch_ens_cool_adapt_tiles(cd, ints + P.sp_chains.off, P.sp_chains.n, st));
        ++nl;
      }
      if (k == P.n_iter) break;
      CK(fam(ENS_COOL_OMEGA, ENS_COOL_OMEGA, 0));
      CK(fam(ENS_COOL_GRAD_OMEGA, ENS_COOL_GRAD_OMEGA, 0));
      CK(fam(ENS_COOL_APPLY, ENS_COOL_APPLY, 0));
      CK(fam(ENS_COOL_APPLY_UN, ENS_COOL_APPLY_UN, 0));
    }
  }
  *launches = nl;
  return CL_OK;
}

// Fused launches need members of one precision, FP64 or FP32 storage.
bool fusable(const cl_batch* b) {
  for (const cl_lattice* l : b->lats)
    if (l->prec == 2 || l->prec != b->lats[0]->prec) return false;
  return true;
}

// Fused capture: the plan and both descriptor variants go to the device in
// one allocation; each variant's step is captured from the origin stream.
cl_status capture_batch_fused(cl_batch* b) {
  const int n = (int)b->lats.size();
  if (!fusable(b)) return fail(CL_ERR_INVALID, "fused batches need FP64 or FP32-storage members of one precision");
  for (int i = 0; i < n; ++i) CK(cudaStreamSynchronize(b->lats[i]->st));
  FusedPlan P = plan_fused(b);
  std::vector<ChainDesc> cd(2 * (size_t)n);
  for (int v = 0; v < 2; ++v)
    for (int i = 0; i < n; ++i) cd[(size_t)v * n + i] = describe(b->lats[i], b->eps[i], b->cps[i], v == 1);
  const size_t cd_bytes = sizeof(ChainDesc) * cd.size(), w_bytes = sizeof(WorkItem) * P.items.size(),
               i_bytes = sizeof(int) * P.ints.size();
  const size_t w_off = (cd_bytes + 255) / 256 * 256, i_off = w_off + (w_bytes + 255) / 256 * 256;
  CK(cudaMalloc(&b->dmem, i_off + i_bytes + 16));
  char* base = (char*)b->dmem;
  CK(cudaMemcpy(base, cd.data(), cd_bytes, cudaMemcpyHostToDevice));
  if (w_bytes) CK(cudaMemcpy(base + w_off, P.items.data(), w_bytes, cudaMemcpyHostToDevice));
  if (i_bytes) CK(cudaMemcpy(base + i_off, P.ints.data(), i_bytes, cudaMemcpyHostToDevice));
  const WorkItem* w = (const WorkItem*)(base + w_off);
  const int* ints = (const int*)(base + i_off);
  cl_status s = CL_OK;
  int64_t nl = 0;
  for (int v = 0; v < 2 && s == CL_OK; ++v) {
    b->startU[v].assign(n, nullptr);
    for (int i = 0; i < n; ++i) b->startU[v][i] = v == 0 ? b->lats[i]->U : b->lats[i]->Un;
    cudaError_t e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return fail(CL_ERR_CUDA, std::string("fused capture: ") + cudaGetErrorString(e));
    s = enqueue_fused_step(b, P, (const ChainDesc*)base + (size_t)v * n, w, ints, b->origin, &nl);
    cudaGraph_t gr = nullptr;
    e = cudaStreamEndCapture(b->origin, &gr);
    if (s == CL_OK && e != cudaSuccess) s = fail(CL_ERR_CUDA, std::string("fused capture: ") + cudaGetErrorString(e));
    if (s == CL_OK) {
      e = cudaGraphInstantiate(&b->exec[v], gr, 0);
      if (e != cudaSuccess) s = fail(CL_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    if (gr) cudaGraphDestroy(gr);
  }
  // launches are shared by all chains: counted once, on the first member
  for (int i = 0; i < n; ++i) b->lats[i]->glaunches = i == 0 ? nl : 0;
  if (s != CL_OK) drop_graphs(b);
  return s;
}

// (Re)capture the batch graph: one step of every member, forked from the
// origin stream to each member's stream and joined back; two variants (the
// members' link buffers before and after one swap).
cl_status capture_batch(cl_batch* b) {
  drop_graphs(b);
  if (b->fused && !b->lats.empty()) {
    b->joins.assign(b->lats.size(), nullptr);
    b->ready.assign(b->lats.size(), nullptr);
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i < b->lats.size() && e == cudaSuccess; ++i)
      e = cudaEventCreateWithFlags(&b->ready[i], cudaEventDisableTiming);
    if (e != cudaSuccess) return fail(CL_ERR_CUDA, std::string("batch setup: ") + cudaGetErrorString(e));
    return capture_batch_fused(b);
  }
  const int n = (int)b->lats.size();
  if (n == 0) return CL_OK;
  cudaError_t e = cudaSuccess;
  b->joins.assign(n, nullptr);
  b->ready.assign(n, nullptr);
  for (int i = 0; i < n && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&b->joins[i], cudaEventDisableTiming);
  for (int i = 0; i < n && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&b->ready[i], cudaEventDisableTiming);
  // the members' pending work must finish before the capture
  for (int i = 0; i < n && e == cudaSuccess; ++i) e = cudaStreamSynchronize(b->lats[i]->st);
  if (e != cudaSuccess) return fail(CL_ERR_CUDA, std::string("batch setup: ") + cudaGetErrorString(e));
  std::vector<void*> U0(n), Un0(n);
  std::vector<int> timing(n);
  for (int i = 0; i < n; ++i) {
    U0[i] = b->lats[i]->U;
    Un0[i] = b->lats[i]->Un;
    timing[i] = b->lats[i]->timing;
    b->lats[i]->timing = 0;
  }
  cl_status s = CL_OK;
  for (int v = 0; v < 2 && s == CL_OK; ++v) {
    std::vector<uint64_t> step0(n);
    std::vector<int64_t> n0(n);
    b->startU[v].assign(n, nullptr);
    e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaEventRecord(b->fork, b->origin);
    for (int i = 0; i < n; ++i) {
      step0[i] = b->lats[i]->step;
      n0[i] = b->lats[i]->launches;
    }
    for (int i = 0; i < n && e == cudaSuccess && s == CL_OK; ++i) {
      cl_lattice* l = b->lats[i];
      b->startU[v][i] = l->U;
      e = cudaStreamWaitEvent(l->st, b->fork, 0);
      if (e == cudaSuccess) s = enqueue_step(l, b->eps[i], b->with_cooling ? &b->cps[i] : nullptr);
      l->glaunches = l->launches - n0[i];
      if (e == cudaSuccess && s == CL_OK) e = cudaEventRecord(b->joins[i], l->st);
      if (e == cudaSuccess && s == CL_OK) e = cudaStreamWaitEvent(b->origin, b->joins[i], 0);
    }
    cudaGraph_t gr = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->origin, &gr);
    for (int i = 0; i < n; ++i) {
      b->lats[i]->step = step0[i];
      b->lats[i]->launches = n0[i];
    }
    if (s == CL_OK && (e != cudaSuccess || e2 != cudaSuccess))
      s = fail(CL_ERR_CUDA, std::string("batch capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    if (s == CL_OK) {
      e = cudaGraphInstantiate(&b->exec[v], gr, 0);
      if (e != cudaSuccess) s = fail(CL_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    if (gr) cudaGraphDestroy(gr);
  }
  // each variant swapped the buffers once: after two they are back in place
  for (int i = 0; i < n; ++i) {
    b->lats[i]->timing = timing[i];
    b->lats[i]->U = U0[i];
    b->lats[i]->Un = Un0[i];
  }
  if (s != CL_OK) drop_graphs(b);
  return s;
}

}  // namespace

void cl_batch_free(cl_batch* b) {
  if (!b) return;
  if (b->origin) cudaStreamSynchronize(b->origin);
  drop_graphs(b);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->done) cudaEventDestroy(b->done);
  if (b->origin) cudaStreamDestroy(b->origin);
  delete b;
}

cl_status cl_batch_create(int n, cl_lattice* const* lats, const double* eps,
                          const cl_cool_params* cps, int with_cooling, cl_batch** out) {
  if (!out || n < 1 || !lats || !eps || (with_cooling && !cps)) return fail(CL_ERR_INVALID, "bad batch arguments");
  *out = nullptr;
  cl_batch* b = new cl_batch();
  b->with_cooling = with_cooling ? 1 : 0;
  b->origin = nullptr;
  b->fork = nullptr;
  b->done = nullptr;
  b->exec[0] = b->exec[1] = nullptr;
  b->fused = 0;
  b->dmem = nullptr;
  for (int i = 0; i < n; ++i) {
    cl_status s = check_batch_member(b, lats[i], eps[i], with_cooling ? &cps[i] : nullptr);
    if (s != CL_OK) {
      delete b;
      return s;
    }
    b->lats.push_back(lats[i]);
    b->eps.push_back(eps[i]);
    cl_cool_params cp;
    std::memset(&cp, 0, sizeof(cp));
    if (with_cooling) cp = cps[i];
    b->cps.push_back(cp);
  }
  // fused launches by default where they apply (measured faster than the
  // per-chain graph on the 64-chain ensemble; see cl_batch_set_fused)
  b->fused = fusable(b) ? 1 : 0;
  cudaError_t e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
  cl_status s = e == cudaSuccess ? capture_batch(b)
                                 : fail(CL_ERR_CUDA, std::string("batch setup: ") + cudaGetErrorString(e));
  if (s != CL_OK) {
    cl_batch_free(b);
    return s;
  }
  *out = b;
  return CL_OK;
}

cl_status cl_batch_add(cl_batch* b, cl_lattice* lat, double eps, const cl_cool_params* cp) {
  if (!b) return fail(CL_ERR_INVALID, "NULL batch");
  if (b->with_cooling && !cp) return fail(CL_ERR_INVALID, "this batch cools: cp is needed");
  cl_status s = check_batch_member(b, lat, eps, b->with_cooling ? cp : nullptr);
  if (s != CL_OK) return s;
  CK(cudaStreamSynchronize(b->origin));
  b->lats.push_back(lat);
  b->eps.push_back(eps);
  cl_cool_params c;
  std::memset(&c, 0, sizeof(c));
  if (b->with_cooling) c = *cp;
  b->cps.push_back(c);
  const int fused0 = b->fused;
  if (b->fused && !fusable(b)) b->fused = 0;  // a member of another precision: per-chain graphs
  s = capture_batch(b);
  if (s != CL_OK) {
    b->lats.pop_back();
    b->eps.pop_back();
    b->cps.pop_back();
    b->fused = fused0;
    cl_status s2 = capture_batch(b);
    (void)s2;
  }
  return s;
}

cl_status cl_batch_remove(cl_batch* b, cl_lattice* lat) {
  if (!b || !lat) return fail(CL_ERR_INVALID, "NULL argument");
  size_t i = 0;
  while (i < b->lats.size() && b->lats[i] != lat) ++i;
  if (i == b->lats.size()) return fail(CL_ERR_INVALID, "lattice is not in the batch");
  CK(cudaStreamSynchronize(b->origin));
  b->lats.erase(b->lats.begin() + i);
  b->eps.erase(b->eps.begin() + i);
  b->cps.erase(b->cps.begin() + i);
  return capture_batch(b);
}

cl_status cl_batch_set_fused(cl_batch* b, int fused) {
  if (!b) return fail(CL_ERR_INVALID, "NULL batch");
  CK(cudaStreamSynchronize(b->origin));
  const int old = b->fused;
  b->fused = fused ? 1 : 0;
  cl_status s = capture_batch(b);
  if (s != CL_OK) {
    b->fused = old;
    cl_status s2 = capture_batch(b);
    (void)s2;
  }
  return s;
}

cl_status cl_batch_get_fused(const cl_batch* b, int* fused) {
  if (!b || !fused) return fail(CL_ERR_INVALID, "NULL argument");
  *fused = b->fused;
  return CL_OK;
}

cl_status cl_batch_size(const cl_batch* b, int* n) {
  if (!b || !n) return fail(CL_ERR_INVALID, "NULL argument");
  *n = (int)b->lats.size();
  return CL_OK;
}

cl_status cl_batch_run(cl_batch* b, int n_steps) {
  if (!b || n_steps < 0) return fail(CL_ERR_INVALID, "bad arguments");
  const int n = (int)b->lats.size();
  if (n_steps == 0 || n == 0) return CL_OK;
  // order against work already queued on the lattices' own streams
  for (int i = 0; i < n; ++i) {
    CK(cudaEventRecord(b->ready[i], b->lats[i]->st));
    CK(cudaStreamWaitEvent(b->origin, b->ready[i], 0));
  }
  for (int k = 0; k < n_steps; ++k) {
    int v = -1;
    for (int w = 0; w < 2 && v < 0; ++w) {
      bool ok = true;
      for (int i = 0; i < n && ok; ++i) ok = b->lats[i]->U == b->startU[w][i];
      if (ok) v = w;
    }
    if (v < 0) return fail(CL_ERR_INVALID, "a batch lattice was stepped outside the batch");
    CK(cudaGraphLaunch(b->exec[v], b->origin));
    for (cl_lattice* l : b->lats) {
      std::swap(l->U, l->Un);
      l->step++;
      l->launches += l->glaunches;
    }
  }
  // later calls on a lattice's own stream see the batch's result
  CK(cudaEventRecord(b->done, b->origin));
  for (cl_lattice* l : b->lats) CK(cudaStreamWaitEvent(l->st, b->done, 0));
  return CL_OK;
}

cl_status cl_batch_synchronize(cl_batch* b) {
  if (!b) return fail(CL_ERR_INVALID, "NULL batch");
  CK(cudaStreamSynchronize(b->origin));
  return CL_OK;
}

// ------------------------------------------------------------- autotuner
namespace {

const int TUNE_CANDIDATES[] = {32, 64, 128, 256};
const int N_TUNE_CANDIDATES = 4;
// the timing phase that holds each tunable family's kernels
const int TUNE_PHASE[NTUNE] = {CL_PHASE_CLOVER, CL_PHASE_FORCE, CL_PHASE_UPDATE, CL_PHASE_COOL_OMEGA,
                               CL_PHASE_COOL_APPLY};

struct TuneKey {
  int device, prec, theta, L[4];
  bool operator<(const TuneKey& o) const {
    return std::memcmp(this, &o, sizeof(TuneKey)) < 0;
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::array<int, NTUNE>>* g_tune_cache = nullptr;

TuneKey tune_key(const cl_lattice* l) {
  TuneKey k;
  std::memset(&k, 0, sizeof(k));
  cudaGetDevice(&k.device);
  k.prec = l->prec;
  k.theta = theta_nonzero(l) ? 1 : 0;
  for (int mu = 0; mu < 4; ++mu) k.L[mu] = l->g.L[mu];
  return k;
}

bool valid_block(int b) { return b == 0 || (b >= 32 && b <= TUNE_MAX_BLOCK && b % 32 == 0); }

}  // namespace

cl_status cl_set_blocks(cl_lattice* l, const int* blocks) {
  if (!l || !blocks) return fail(CL_ERR_INVALID, "NULL argument");
  for (int f = 0; f < NTUNE; ++f)
    if (!valid_block(blocks[f])) return fail(CL_ERR_INVALID, "block size must be 0 or a multiple of 32 in [32, 256]");
  for (int f = 0; f < NTUNE; ++f) l->g.blk[f] = blocks[f];
  return CL_OK;
}

cl_status cl_get_blocks(cl_lattice* l, int* blocks) {
  if (!l || !blocks) return fail(CL_ERR_INVALID, "NULL argument");
  for (int f = 0; f < NTUNE; ++f) blocks[f] = block_of(l->g, f);
  return CL_OK;
}

cl_status cl_autotune(cl_lattice* l, double eps, const cl_cool_params* cp, int reps, int use_cache,
                      int* blocks_out, double* ms_out) {
  if (!l || !cp || reps < 1) return fail(CL_ERR_INVALID, "bad arguments");
  if (!(eps >= 0.0)) return fail(CL_ERR_INVALID, "bad eps");
  cl_status s = check_cool(cp);
  if (s != CL_OK) return s;
  const TuneKey key = tune_key(l);
  if (use_cache && !ms_out) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (g_tune_cache) {
      auto it = g_tune_cache->find(key);
      if (it != g_tune_cache->end()) {
        for (int f = 0; f < NTUNE; ++f) l->g.blk[f] = it->second[f];
        if (blocks_out) cl_get_blocks(l, blocks_out);
        return CL_OK;
      }
    }
  }
  CK(resolve_timing(l));
  CK(cudaStreamSynchronize(l->st));
  // snapshot everything a trial step changes; the trials run on the lattice's
  // own buffers and the snapshot is put back afterwards
  const size_t link_bytes = l->esz * 4 * 9 * (size_t)l->g.V;
  void* saved = nullptr;
  CK(cudaMalloc(&saved, link_bytes));
  CoolState cs0;
  StepDev sd0;
  cudaError_t e = cudaMemcpyAsync(saved, l->U, link_bytes, cudaMemcpyDeviceToDevice, l->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&cs0, l->cs, sizeof(cs0), cudaMemcpyDeviceToHost, l->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&sd0, l->sd, sizeof(StepDev), cudaMemcpyDeviceToHost, l->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(l->st);
  if (e != cudaSuccess) {
    cudaFree(saved);
    return fail(CL_ERR_CUDA, std::string("autotune snapshot: ") + cudaGetErrorString(e));
  }
  const uint64_t step0 = l->step;
  const int64_t launches0 = l->launches;
  const int timing0 = l->timing;
  double ms0[CL_NPHASE];
  int64_t n0[CL_NPHASE];
  std::memcpy(ms0, l->phase_ms, sizeof(ms0));
  std::memcpy(n0, l->phase_n, sizeof(n0));
  int blk0[NTUNE];
  std::memcpy(blk0, l->g.blk, sizeof(blk0));
  cl_cool_params tcp = *cp;
  tcp.forced_sweeps = 2;  // the Omega and apply kernels must run in every trial
  double table[N_TUNE_CANDIDATES][NTUNE];
  for (int c = 0; c < N_TUNE_CANDIDATES && s == CL_OK; ++c) {
    for (int f = 0; f < NTUNE; ++f) l->g.blk[f] = TUNE_CANDIDATES[c];
    e = cudaMemcpyAsync(l->U, saved, link_bytes, cudaMemcpyDeviceToDevice, l->st);
    if (e != cudaSuccess) {
      s = fail(CL_ERR_CUDA, cudaGetErrorString(e));
      break;
    }
    l->timing = 0;
    s = enqueue_step(l, eps, &tcp);  // warm-up
    if (s != CL_OK) break;
    l->timing = 1;
    for (int i = 0; i < CL_NPHASE; ++i) {
      l->phase_ms[i] = 0.0;
      l->phase_n[i] = 0;
    }
    for (int r = 0; r < reps && s == CL_OK; ++r) s = enqueue_step(l, eps, &tcp);
    if (s != CL_OK) break;
    e = resolve_timing(l);
    if (e != cudaSuccess) {
      s = fail(CL_ERR_CUDA, cudaGetErrorString(e));
      break;
    }
    for (int f = 0; f < NTUNE; ++f) table[c][f] = l->phase_ms[TUNE_PHASE[f]] / reps;
  }
  l->timing = 0;
  resolve_timing(l);
  // restore the lattice
  e = cudaMemcpyAsync(l->U, saved, link_bytes, cudaMemcpyDeviceToDevice, l->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(l->cs, &cs0, sizeof(cs0), cudaMemcpyHostToDevice, l->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(l->sd, &sd0, sizeof(StepDev), cudaMemcpyHostToDevice, l->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(l->st);
  cudaFree(saved);
  l->step = step0;
  l->launches = launches0;
  l->timing = timing0;
  std::memcpy(l->phase_ms, ms0, sizeof(ms0));
  std::memcpy(l->phase_n, n0, sizeof(n0));
  if (s == CL_OK && e != cudaSuccess) s = fail(CL_ERR_CUDA, std::string("autotune restore: ") + cudaGetErrorString(e));
  if (s != CL_OK) {
    std::memcpy(l->g.blk, blk0, sizeof(blk0));
    return s;
  }
  std::array<int, NTUNE> best;
  for (int f = 0; f < NTUNE; ++f) {
    int bc = 0;
    for (int c = 1; c < N_TUNE_CANDIDATES; ++c)
      if (table[c][f] < table[bc][f]) bc = c;
    best[f] = TUNE_CANDIDATES[bc];
    l->g.blk[f] = best[f];
  }
  if (ms_out)
    for (int c = 0; c < N_TUNE_CANDIDATES; ++c)
      for (int f = 0; f < NTUNE; ++f) ms_out[c * NTUNE + f] = table[c][f];
  if (blocks_out) cl_get_blocks(l, blocks_out);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (!g_tune_cache) g_tune_cache = new std::map<TuneKey, std::array<int, NTUNE>>();
    (*g_tune_cache)[key] = best;
  }
  return CL_OK;
}

// ------------------------------------------------------------- checkpoints
namespace {

const uint32_t CKPT_MAGIC = 0x4b434c43u;  // "CLCK"
const uint32_t CKPT_VERSION = 2;

struct CkptHeader {
  uint32_t magic, version;
  int32_t L[4];
  int32_t prec;
  int32_t blk[NTUNE];
  uint64_t step;
  double k_ref;
  cl_params params;
  StepDev sd;
  CoolState cs;
  uint64_t link_bytes;  // the link field in its device storage (SoA), copied verbatim
};

size_t link_field_bytes(const cl_lattice* l) { return l->esz * 36 * (size_t)l->g.V; }
size_t ckpt_bytes(const cl_lattice* l) { return sizeof(CkptHeader) + link_field_bytes(l); }

}  // namespace

cl_status cl_state_size(const cl_lattice* l, size_t* bytes) {
  if (!l || !bytes) return fail(CL_ERR_INVALID, "NULL argument");
  *bytes = ckpt_bytes(l);
  return CL_OK;
}

cl_status cl_save_state(cl_lattice* l, void* host, size_t bytes) {
  if (!l || !host) return fail(CL_ERR_INVALID, "NULL argument");
  if (bytes < ckpt_bytes(l)) return fail(CL_ERR_INVALID, "buffer smaller than cl_state_size");
  CkptHeader h;
  std::memset(&h, 0, sizeof(h));
  h.magic = CKPT_MAGIC;
  h.version = CKPT_VERSION;
  for (int mu = 0; mu < 4; ++mu) h.L[mu] = l->g.L[mu];
  h.prec = l->prec;
  for (int f = 0; f < NTUNE; ++f) h.blk[f] = l->g.blk[f];
  h.step = l->step;
  h.k_ref = l->k_ref;
  h.params = l->p;
  h.link_bytes = link_field_bytes(l);
  CK(cudaMemcpyAsync(&h.sd, l->sd, sizeof(StepDev), cudaMemcpyDeviceToHost, l->st));
  CK(cudaMemcpyAsync(&h.cs, l->cs, sizeof(CoolState), cudaMemcpyDeviceToHost, l->st));
  CK(cudaMemcpyAsync((char*)host + sizeof(CkptHeader), l->U, h.link_bytes, cudaMemcpyDeviceToHost, l->st));
  CK(cudaStreamSynchronize(l->st));
  std::memcpy(host, &h, sizeof(h));
  return CL_OK;
}

cl_status cl_load_state(cl_lattice* l, const void* host, size_t bytes) {
  if (!l || !host) return fail(CL_ERR_INVALID, "NULL argument");
  if (bytes < sizeof(CkptHeader)) return fail(CL_ERR_INVALID, "buffer too small for a checkpoint");
  CkptHeader h;
  std::memcpy(&h, host, sizeof(h));
  if (h.magic != CKPT_MAGIC || h.version != CKPT_VERSION) return fail(CL_ERR_INVALID, "not a checkpoint");
  for (int mu = 0; mu < 4; ++mu)
    if (h.L[mu] != l->g.L[mu]) return fail(CL_ERR_INVALID, "checkpoint of other extents");
  if (h.prec != l->prec) return fail(CL_ERR_INVALID, "checkpoint of the other precision");
  if (h.link_bytes != link_field_bytes(l) || bytes < ckpt_bytes(l))
    return fail(CL_ERR_INVALID, "truncated checkpoint");
  CK(cudaStreamSynchronize(l->st));
  for (int v = 0; v < 2; ++v)
    if (l->gexec[v]) {  // the captured steps carry the old parameters
      cudaGraphExecDestroy(l->gexec[v]);
      l->gexec[v] = nullptr;
    }
  l->p = h.params;
  l->k_ref = h.k_ref;
  for (int f = 0; f < NTUNE; ++f) l->g.blk[f] = h.blk[f];
  l->step = h.step;
  CK(cudaMemcpyAsync(l->U, (const char*)host + sizeof(CkptHeader), h.link_bytes, cudaMemcpyHostToDevice,
                     l->st));
  CK(cudaMemcpyAsync(l->sd, &h.sd, sizeof(StepDev), cudaMemcpyHostToDevice, l->st));
  CK(cudaMemcpyAsync(l->cs, &h.cs, sizeof(CoolState), cudaMemcpyHostToDevice, l->st));
  CK(cudaStreamSynchronize(l->st));
  return CL_OK;
}

cl_status cl_stream_create(void** out) {
  if (!out) return fail(CL_ERR_INVALID, "NULL argument");
  *out = nullptr;
  cudaStream_t st = nullptr;
  CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  *out = (void*)st;
  return CL_OK;
}

cl_status cl_stream_destroy(void* stream) {
  if (!stream) return fail(CL_ERR_INVALID, "NULL stream");
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  CK(cudaStreamDestroy((cudaStream_t)stream));
  return CL_OK;
}

cl_status cl_set_timing(cl_lattice* l, int on) {
  if (!l) return fail(CL_ERR_INVALID, "NULL lattice");
  CK(resolve_timing(l));
  for (int i = 0; i < CL_NPHASE; ++i) {
    l->phase_ms[i] = 0.0;
    l->phase_n[i] = 0;
  }
  l->timing = on ? 1 : 0;
  return CL_OK;
}

cl_status cl_get_timing(cl_lattice* l, double* ms, int64_t* launches) {
  if (!l) return fail(CL_ERR_INVALID, "NULL lattice");
  CK(resolve_timing(l));
  for (int i = 0; i < CL_NPHASE; ++i) {
    if (ms) ms[i] = l->phase_ms[i];
    if (launches) launches[i] = l->phase_n[i];
  }
  return CL_OK;
}

cl_status cl_synchronize(cl_lattice* l) {
  if (!l) return fail(CL_ERR_INVALID, "NULL lattice");
  CK(cudaStreamSynchronize(l->st));
  return CL_OK;
}

namespace {
// Poll a stream until its work is done or timeout_s seconds have passed.
cl_status bounded_wait(cudaStream_t st, double timeout_s) {
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaStreamQuery(st);
    if (e == cudaSuccess) return CL_OK;
    if (e != cudaErrorNotReady) return fail(CL_ERR_CUDA, std::string("cudaStreamQuery: ") + cudaGetErrorString(e));
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (el >= timeout_s) return fail(CL_ERR_TIMEOUT, "work still running after the time limit");
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}
}  // namespace

cl_status cl_wait(cl_lattice* l, double timeout_s) {
  if (!l || !(timeout_s >= 0.0)) return fail(CL_ERR_INVALID, "NULL lattice or bad time limit");
  return bounded_wait(l->st, timeout_s);
}

cl_status cl_batch_wait(cl_batch* b, double timeout_s) {
  if (!b || !(timeout_s >= 0.0)) return fail(CL_ERR_INVALID, "NULL batch or bad time limit");
  return bounded_wait(b->origin, timeout_s);
}

void cl_free(cl_lattice* l) {
  if (!l) return;
  void* bufs[] = {l->U, l->Un, l->Ui, l->Pq, l->Dq, l->C, l->F, l->partials, l->cs, l->obs,
                  l->stage, l->qsite, l->sd};
  for (int v = 0; v < 2; ++v)
    if (l->gexec[v]) cudaGraphExecDestroy(l->gexec[v]);
  if (l->st) cudaStreamSynchronize(l->st);
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (l->ev_pending) {
    for (auto& p : *l->ev_pending) {
      cudaEventDestroy(p.second.first);
      cudaEventDestroy(p.second.second);
    }
    delete l->ev_pending;
  }
  if (l->ev_pool) {
    for (cudaEvent_t e : *l->ev_pool) cudaEventDestroy(e);
    delete l->ev_pool;
  }
  delete l;
}

const char* cl_status_str(cl_status s) {
  switch (s) {
    case CL_OK: return "ok";
    case CL_ERR_INVALID: return "invalid argument";
    case CL_ERR_OOM: return "out of device memory";
    case CL_ERR_CUDA: return "CUDA error";
    case CL_ERR_NONFINITE: return "non-finite links";
    case CL_ERR_RUNAWAY: return "runaway (unitarity norm above bound)";
    case CL_ERR_TIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

const char* cl_last_error(void) { return g_err.c_str(); }

int cl_version(void) { return 1; }

}  // extern "C"
