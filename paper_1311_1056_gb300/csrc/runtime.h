// runtime.h -- internal state of a lattice and the launch sequencing shared
// by the C-ABI entry points (capi.cu) and the request server (server.cu).
// Not part of the public interface (include/cl.h).
#pragma once
#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "../../include/cl.h"
#include "launch.h"

struct cl_lattice {
  cl_params p;
  clgc::GeoH g;
  int prec;
  size_t esz;  // bytes of one complex element (16 or 8)
  cudaStream_t st;
  void* U;     // links, SoA [4][9][V]
  void* Un;    // second link buffer (CL update target)
  void* Ui;    // link inverses [4][9][V]
  void* Pq;    // plaquettes [6][9][V]
  void* Dq;    // P - P^{-1} [6][9][V]
  void* C;     // per-plaquette drift contributions [24][9][V]
  void* Gq;    // partial sums of transported dual fields: plane p at C plane 4p + 1 (inside C)
  void* F;     // clover field, SoA [6][9][V]
  void* f;     // cooling gradient [8][V] (FP64 in both forms; inside C)
  void* Om;    // packed Hermitian Omega [9][V] (inside C)
  void* Omi;   // and its inverse (inside C)
  double* crec;  // single-pass apply's tile records, 2 doubles per tile (inside C)
  double* partials;
  clgc::CoolState* cs;
  clgc::ObsOut* obs;
  double* stage;  // AoS double staging, V*4*18 (allocated on first use)
  double* qsite;  // per-site q_L (on first use)
  uint64_t step;        // host mirror of sd->step
  clgc::StepDev* sd;    // device step state: Philox step word, adaptive eps, Langevin time
  double k_ref;         // > 0: adaptive step size eps_n = eps min(1, k_ref / K_max)
  int64_t launches;
  // step graphs (cl_capture_step): variant v starts from the link buffer in gU[v]
  cudaGraphExec_t gexec[2];
  void* gU[2];
  int64_t glaunches;  // kernels in one captured step
  // optional per-phase CUDA-event timing (cl_set_timing)
  int timing;
  std::vector<cudaEvent_t>* ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>>* ev_pending;
  double phase_ms[CL_NPHASE];
  int64_t phase_n[CL_NPHASE];
};

namespace clrt {

// Records msg as the calling thread's last error (cl_last_error) and returns s.
cl_status fail(cl_status s, const std::string& msg);

#define CK(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return ::clrt::fail(e_ == cudaErrorMemoryAllocation ? CL_ERR_OOM : CL_ERR_CUDA, \
                          std::string(#call) + ": " + cudaGetErrorString(e_));     \
  } while (0)

cl_status check_cool(const cl_cool_params* cp);
size_t lattice_bytes(int V, int prec);
cudaError_t init_state(cl_lattice* l);
// Enqueue n CL steps / one cooling call / the observables into dst (device).
cl_status do_steps(cl_lattice* l, double eps, int n);
cl_status do_cool(cl_lattice* l, const cl_cool_params* cp);
cl_status do_obs(cl_lattice* l, clgc::ObsOut* dst, double* q_site);
// One step of the hot path: CL step, then cooling when cp != NULL.
cl_status enqueue_step(cl_lattice* l, double eps, const cl_cool_params* cp);
void to_cl_obs(const clgc::ObsOut& o, cl_obs* out);
void to_report(const clgc::CoolState& c, cl_cool_report* r);

}  // namespace clrt
