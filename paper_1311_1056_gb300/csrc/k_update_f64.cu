// k_update_f64.cu -- the CL-step kernels (k_update.cuh) for double links.
#include "ensemble.cuh"
#include "k_update.cuh"
#include "launch.h"

namespace clgc {

namespace {
typedef vec2_of<double>::type V2;
// 1-D grid, plane (or direction) fastest: the blocks resident at one time
// cover every plane of a range of sites, so shared neighbours stay in cache.
inline dim3 grid(int V, int planes, int bs) { return dim3((unsigned)(((V + bs - 1) / bs) * planes)); }
}  // namespace

cudaError_t launch_link_inverse_f64(const GeoH& h, const void* U, void* Ui, cudaStream_t st) {
  Geo g = make_geo(h.L, h.V);
  k_link_inverse<double><<<grid(g.V, 4, block_of(h, TUNE_CLOVER)), block_of(h, TUNE_CLOVER), 0, st>>>(g, (const V2*)U, (V2*)Ui);
  return cudaGetLastError();
}

cudaError_t launch_plaq_f64(const GeoH& h, const void* U, const void* Ui, void* Pq, void* Dq,
                           cudaStream_t st) {
  Geo g = make_geo(h.L, h.V);
  k_plaq<double><<<grid(g.V, 6, block_of(h, TUNE_CLOVER)), block_of(h, TUNE_CLOVER), 0, st>>>(g, (const V2*)U, (const V2*)Ui, (V2*)Pq, (V2*)Dq);
  return cudaGetLastError();
}

cudaError_t launch_clover_rot_f64(const GeoH& h, const void* U, const void* Ui, const void* Dq,
                                 void* F, double sre, double sim, cudaStream_t st) {
  Geo g = make_geo(h.L, h.V);
  k_clover_rot<double><<<grid(g.V, 6, block_of(h, TUNE_CLOVER)), block_of(h, TUNE_CLOVER), 0, st>>>(g, (const V2*)U, (const V2*)Ui, (const V2*)Dq,
                                                  (V2*)F, sre, sim);
  return cudaGetLastError();
}

cudaError_t launch_plaq_force_f64(bool theta, const GeoH& h, const void* U, const void* Ui,
                                 const void* Pq, const void* Dq, const void* F, void* Gq, void* C,
                                 double beta, cudaStream_t st) {
  Geo g = make_geo(h.L, h.V);
  const double b6 = (double)(beta / 6.0);
  if (!theta) {
    k_plaq_force_wilson<double><<<grid(g.V, 6, block_of(h, TUNE_FORCE)), block_of(h, TUNE_FORCE), 0, st>>>(g, (const V2*)U, (const V2*)Ui, (const V2*)Dq,
                                                         (V2*)C, b6);
    return cudaGetLastError();
  }
  k_plaq_force_a<double><<<grid(g.V, 6, block_of(h, TUNE_FORCE)), block_of(h, TUNE_FORCE), 0, st>>>(g, (const V2*)U, (const V2*)Ui, (const V2*)Dq,
                                                  (const V2*)F, (V2*)Gq, (V2*)C, b6);
  k_plaq_force_b<double><<<grid(g.V, 6, block_of(h, TUNE_FORCE)), block_of(h, TUNE_FORCE), 0, st>>>(g, (const V2*)U, (const V2*)Ui, (const V2*)Pq,
                                                  (const V2*)Dq, (const V2*)F, (const V2*)Gq, (V2*)C, b6);
  return cudaGetLastError();
}

cudaError_t launch_update_gather_f64(int mode, const GeoH& h, const void* U, const void* C, void* out,
                                    double eps, uint64_t seed, StepDev* sd, bool adaptive, cudaStream_t st) {
  Geo g = make_geo(h.L, h.V);
  UpdArgs a;
  a.beta = 0.0;
  a.eps = eps;
  a.sqrt_eps = sqrt(eps);
  a.seed = seed;
  a.sd = sd;
  a.adaptive = adaptive ? 1 : 0;
  const int bs = block_of(h, TUNE_UPDATE);
  const dim3 gr = grid(g.V, 4, bs);
  const V2* u = (const V2*)U;
  const V2* c = (const V2*)C;
  V2* o = (V2*)out;
  switch (mode) {
    case MODE_DRIFT: k_update_gather<double, MODE_DRIFT><<<gr, bs, 0, st>>>(g, u, c, o, a); break;
    case MODE_DRIFTMAX: k_update_gather<double, MODE_DRIFTMAX><<<gr, bs, 0, st>>>(g, u, c, o, a); break;
    case MODE_UPDATE_X: k_update_gather<double, MODE_UPDATE_X><<<gr, bs, 0, st>>>(g, u, c, o, a); break;
    default: k_update_gather<double, MODE_UPDATE><<<gr, bs, 0, st>>>(g, u, c, o, a); break;
  }
  return cudaGetLastError();
}

}  // namespace clgc

// ------------------------------------------------ precision dispatch
namespace clgc {
cudaError_t launch_link_inverse_f32(const GeoH&, const void*, void*, cudaStream_t);
cudaError_t launch_plaq_f32(const GeoH&, const void*, const void*, void*, void*, cudaStream_t);
cudaError_t launch_clover_rot_f32(const GeoH&, const void*, const void*, const void*, void*, double,
                                  double, cudaStream_t);
cudaError_t launch_plaq_force_f32(bool, const GeoH&, const void*, const void*, const void*,
                                  const void*, const void*, void*, void*, double, cudaStream_t);
cudaError_t launch_update_gather_f32(int, const GeoH&, const void*, const void*, void*, double,
                                     uint64_t, StepDev*, bool, cudaStream_t);
cudaError_t launch_link_inverse_df64(const GeoH&, const void*, void*, cudaStream_t);
cudaError_t launch_plaq_df64(const GeoH&, const void*, const void*, void*, void*, cudaStream_t);
cudaError_t launch_clover_rot_df64(const GeoH&, const void*, const void*, const void*, void*, double,
                                  double, cudaStream_t);
cudaError_t launch_plaq_force_df64(bool, const GeoH&, const void*, const void*, const void*,
                                  const void*, const void*, void*, void*, double, cudaStream_t);
cudaError_t launch_update_gather_df64(int, const GeoH&, const void*, const void*, void*, double,
                                     uint64_t, StepDev*, bool, cudaStream_t);

cudaError_t launch_link_inverse(int prec, const GeoH& h, const void* U, void* Ui, cudaStream_t st) {
  if (prec == 0) return launch_link_inverse_f64(h, U, Ui, st);
  if (prec == 1) return launch_link_inverse_f32(h, U, Ui, st);
  return launch_link_inverse_df64(h, U, Ui, st);
}
cudaError_t launch_plaq(int prec, const GeoH& h, const void* U, const void* Ui, void* Pq, void* Dq,
                        cudaStream_t st) {
  if (prec == 0) return launch_plaq_f64(h, U, Ui, Pq, Dq, st);
  if (prec == 1) return launch_plaq_f32(h, U, Ui, Pq, Dq, st);
  return launch_plaq_df64(h, U, Ui, Pq, Dq, st);
}
cudaError_t launch_clover_rot(int prec, const GeoH& h, const void* U, const void* Ui, const void* Dq,
                              void* F, double sre, double sim, cudaStream_t st) {
  if (prec == 0) return launch_clover_rot_f64(h, U, Ui, Dq, F, sre, sim, st);
  if (prec == 1) return launch_clover_rot_f32(h, U, Ui, Dq, F, sre, sim, st);
  return launch_clover_rot_df64(h, U, Ui, Dq, F, sre, sim, st);
}
cudaError_t launch_plaq_force(int prec, bool theta, const GeoH& h, const void* U, const void* Ui,
                              const void* Pq, const void* Dq, const void* F, void* Gq, void* C,
                              double beta, cudaStream_t st) {
  if (prec == 0) return launch_plaq_force_f64(theta, h, U, Ui, Pq, Dq, F, Gq, C, beta, st);
  if (prec == 1) return launch_plaq_force_f32(theta, h, U, Ui, Pq, Dq, F, Gq, C, beta, st);
  return launch_plaq_force_df64(theta, h, U, Ui, Pq, Dq, F, Gq, C, beta, st);
}
cudaError_t launch_update_gather(int prec, int mode, const GeoH& h, const void* U, const void* C,
                                 void* out, double eps, uint64_t seed, StepDev* sd, bool adaptive,
                                 cudaStream_t st) {
  if (prec == 0) return launch_update_gather_f64(mode, h, U, C, out, eps, seed, sd, adaptive, st);
  if (prec == 1) return launch_update_gather_f32(mode, h, U, C, out, eps, seed, sd, adaptive, st);
  return launch_update_gather_df64(mode, h, U, C, out, eps, seed, sd, adaptive, st);
}
}  // namespace clgc

namespace clgc {
// After an update: step += 1 and t += the step size taken (one thread).
__device__ __forceinline__ void step_bump(StepDev* sd, double eps, int adaptive) {
  sd->step += 1u;
  sd->t += adaptive ? sd->eps_n : eps;
}
__global__ void k_step_bump(StepDev* sd, double eps, int adaptive) { step_bump(sd, eps, adaptive); }

// Adaptive step size from the drift pass's max |K|^2: eps_n = eps min(1, k_ref / K_max);
// clears the running max for the next step.
__device__ __forceinline__ void step_eps(StepDev* sd, double eps, double k_ref) {
  const double kmax = sqrt(__longlong_as_double((long long)sd->kmax2_bits));
  const double e = kmax > k_ref ? eps * (k_ref / kmax) : eps;
  sd->eps_n = e;
  sd->sqrt_eps_n = sqrt(e);
  sd->kmax = kmax;
  sd->kmax2_bits = 0ull;
}
__global__ void k_step_eps(StepDev* sd, double eps, double k_ref) { step_eps(sd, eps, k_ref); }

// The same for the chains of a fused batch, one thread per listed chain.
__global__ void k_ens_step_eps(const ChainDesc* __restrict__ cd, const int* __restrict__ chains, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const ChainDesc& c = cd[chains[i]];
  step_eps(c.sd, c.eps, c.k_ref);
}
__global__ void k_ens_step_bump(const ChainDesc* __restrict__ cd, const int* __restrict__ chains,
                                const int* __restrict__ adaptive, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const ChainDesc& c = cd[chains[i]];
  step_bump(c.sd, c.eps, adaptive[i]);
}

cudaError_t launch_ens_step_eps(const ChainDesc* cd, const int* chains, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_ens_step_eps<<<(n + 127) / 128, 128, 0, st>>>(cd, chains, n);
  return cudaGetLastError();
}
cudaError_t launch_ens_step_bump(const ChainDesc* cd, const int* chains, const int* adaptive, int n,
                                 cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_ens_step_bump<<<(n + 127) / 128, 128, 0, st>>>(cd, chains, adaptive, n);
  return cudaGetLastError();
}

cudaError_t launch_step_bump(StepDev* sd, double eps, bool adaptive, cudaStream_t st) {
  k_step_bump<<<1, 1, 0, st>>>(sd, eps, adaptive ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_step_eps(StepDev* sd, double eps, double k_ref, cudaStream_t st) {
  k_step_eps<<<1, 1, 0, st>>>(sd, eps, k_ref);
  return cudaGetLastError();
}
cudaError_t launch_ens_step_f64(int fam, const ChainDesc* cd, const WorkItem* w, int nw, cudaStream_t st) {
  return launch_ens_step_family<double>(fam, cd, w, nw, st);
}

}  // namespace clgc
