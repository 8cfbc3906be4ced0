// k_update_f32.cu -- the CL-step kernels (k_update.cuh) for float links.
#include "ensemble.cuh"
#include "k_update.cuh"
#include "launch.h"

namespace clgc {

namespace {
typedef vec2_of<float>::type V2;
// 1-D grid, plane (or direction) fastest: the blocks resident at one time
// cover every plane of a range of sites, so shared neighbours stay in cache.
inline dim3 grid(int V, int planes, int bs) { return dim3((unsigned)(((V + bs - 1) / bs) * planes)); }
}  // namespace

cudaError_t launch_link_inverse_f32(const GeoH& h, const void* U, void* Ui, cudaStream_t st) {
  Geo g = make_geo(h.L, h.V);
  k_link_inverse<float><<<grid(g.V, 4, block_of(h, TUNE_CLOVER)), block_of(h, TUNE_CLOVER), 0, st>>>(g, (const V2*)U, (V2*)Ui);
  return cudaGetLastError();
}

cudaError_t launch_plaq_f32(const GeoH& h, const void* U, const void* Ui, void* Pq, void* Dq,
                           cudaStream_t st) {
  Geo g = make_geo(h.L, h.V);
  k_plaq<float><<<grid(g.V, 6, block_of(h, TUNE_CLOVER)), block_of(h, TUNE_CLOVER), 0, st>>>(g, (const V2*)U, (const V2*)Ui, (V2*)Pq, (V2*)Dq);
  return cudaGetLastError();
}

cudaError_t launch_clover_rot_f32(const GeoH& h, const void* U, const void* Ui, const void* Dq,
                                 void* F, double sre, double sim, cudaStream_t st) {
  Geo g = make_geo(h.L, h.V);
  k_clover_rot<float><<<grid(g.V, 6, block_of(h, TUNE_CLOVER)), block_of(h, TUNE_CLOVER), 0, st>>>(g, (const V2*)U, (const V2*)Ui, (const V2*)Dq,
                                                  (V2*)F, sre, sim);
  return cudaGetLastError();
}

cudaError_t launch_plaq_force_f32(bool theta, const GeoH& h, const void* U, const void* Ui,
                                 const void* Pq, const void* Dq, const void* F, void* Gq, void* C,
                                 double beta, cudaStream_t st) {
  Geo g = make_geo(h.L, h.V);
  const float b6 = (float)(beta / 6.0);
  if (!theta) {
    k_plaq_force_wilson<float><<<grid(g.V, 6, block_of(h, TUNE_FORCE)), block_of(h, TUNE_FORCE), 0, st>>>(g, (const V2*)U, (const V2*)Ui, (const V2*)Dq,
                                                         (V2*)C, b6);
    return cudaGetLastError();
  }
  k_plaq_force_ab<float><<<grid(g.V, 6, block_of(h, TUNE_FORCE)), block_of(h, TUNE_FORCE), 0, st>>>(g, (const V2*)U, (const V2*)Ui, (const V2*)Pq,
                                                      (const V2*)Dq, (const V2*)F, (V2*)C, b6);
  return cudaGetLastError();
}

cudaError_t launch_update_gather_f32(int mode, const GeoH& h, const void* U, const void* C, void* out,
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
    case MODE_DRIFT: k_update_gather<float, MODE_DRIFT><<<gr, bs, 0, st>>>(g, u, c, o, a); break;
    case MODE_DRIFTMAX: k_update_gather<float, MODE_DRIFTMAX><<<gr, bs, 0, st>>>(g, u, c, o, a); break;
    case MODE_UPDATE_X: k_update_gather<float, MODE_UPDATE_X><<<gr, bs, 0, st>>>(g, u, c, o, a); break;
    default: k_update_gather<float, MODE_UPDATE><<<gr, bs, 0, st>>>(g, u, c, o, a); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_ens_step_f32(int fam, const ChainDesc* cd, const WorkItem* w, int nw, cudaStream_t st) {
  return launch_ens_step_family<float>(fam, cd, w, nw, st);
}

}  // namespace clgc
