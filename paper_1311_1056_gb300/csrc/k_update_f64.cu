// k_update_f64.cu -- the CL-step kernels (k_update.cuh) for double links.
#include "k_update.cuh"
#include "launch.h"

namespace clgc {

namespace {
typedef vec2_of<double>::type V2;
// 1-D grid, plane (or direction) fastest: the blocks resident at one time
// cover every plane of a range of sites, so shared neighbours stay in cache.
inline dim3 grid(int V, int planes) { return dim3((unsigned)(((V + 127) / 128) * planes)); }
}  // namespace

cudaError_t launch_link_inverse_f64(const GeoH& h, const void* U, void* Ui, cudaStream_t st) {
  Geo g = make_geo(h.L, h.V);
  k_link_inverse<double><<<grid(g.V, 4), 128, 0, st>>>(g, (const V2*)U, (V2*)Ui);
  return cudaGetLastError();
}

cudaError_t launch_plaq_f64(const GeoH& h, const void* U, const void* Ui, void* Pq, void* Dq,
                           cudaStream_t st) {
  Geo g = make_geo(h.L, h.V);
  k_plaq<double><<<grid(g.V, 6), 128, 0, st>>>(g, (const V2*)U, (const V2*)Ui, (V2*)Pq, (V2*)Dq);
  return cudaGetLastError();
}

cudaError_t launch_clover_rot_f64(const GeoH& h, const void* U, const void* Ui, const void* Dq,
                                 void* F, double sre, double sim, cudaStream_t st) {
  Geo g = make_geo(h.L, h.V);
  k_clover_rot<double><<<grid(g.V, 6), 128, 0, st>>>(g, (const V2*)U, (const V2*)Ui, (const V2*)Dq,
                                                  (V2*)F, sre, sim);
  return cudaGetLastError();
}

cudaError_t launch_plaq_force_f64(bool theta, const GeoH& h, const void* U, const void* Ui,
                                 const void* Pq, const void* Dq, const void* F, void* Gq, void* C,
                                 double beta, cudaStream_t st) {
  Geo g = make_geo(h.L, h.V);
  const double b6 = (double)(beta / 6.0);
  if (!theta) {
    k_plaq_force_wilson<double><<<grid(g.V, 6), 128, 0, st>>>(g, (const V2*)U, (const V2*)Ui, (const V2*)Dq,
                                                         (V2*)C, b6);
    return cudaGetLastError();
  }
  k_plaq_force_a<double><<<grid(g.V, 6), 128, 0, st>>>(g, (const V2*)U, (const V2*)Ui, (const V2*)Dq,
                                                  (const V2*)F, (V2*)Gq, (V2*)C, b6);
  k_plaq_force_b<double><<<grid(g.V, 6), 128, 0, st>>>(g, (const V2*)U, (const V2*)Ui, (const V2*)Pq,
                                                  (const V2*)Dq, (const V2*)F, (const V2*)Gq, (V2*)C, b6);
  return cudaGetLastError();
}

cudaError_t launch_update_gather_f64(int mode, const GeoH& h, const void* U, const void* C, void* out,
                                    double eps, uint64_t seed, const uint32_t* step, cudaStream_t st) {
  Geo g = make_geo(h.L, h.V);
  UpdArgs a;
  a.beta = 0.0;
  a.eps = eps;
  a.sqrt_eps = sqrt(eps);
  a.seed = seed;
  a.step = step;
  if (mode == MODE_DRIFT)
    k_update_gather<double, MODE_DRIFT><<<grid(g.V, 4), 128, 0, st>>>(g, (const V2*)U, (const V2*)C, (V2*)out, a);
  else
    k_update_gather<double, MODE_UPDATE><<<grid(g.V, 4), 128, 0, st>>>(g, (const V2*)U, (const V2*)C, (V2*)out, a);
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
                                     uint64_t, const uint32_t*, cudaStream_t);

cudaError_t launch_link_inverse(int prec, const GeoH& h, const void* U, void* Ui, cudaStream_t st) {
  return prec == 0 ? launch_link_inverse_f64(h, U, Ui, st) : launch_link_inverse_f32(h, U, Ui, st);
}
cudaError_t launch_plaq(int prec, const GeoH& h, const void* U, const void* Ui, void* Pq, void* Dq,
                        cudaStream_t st) {
  return prec == 0 ? launch_plaq_f64(h, U, Ui, Pq, Dq, st) : launch_plaq_f32(h, U, Ui, Pq, Dq, st);
}
cudaError_t launch_clover_rot(int prec, const GeoH& h, const void* U, const void* Ui, const void* Dq,
                              void* F, double sre, double sim, cudaStream_t st) {
  return prec == 0 ? launch_clover_rot_f64(h, U, Ui, Dq, F, sre, sim, st)
                   : launch_clover_rot_f32(h, U, Ui, Dq, F, sre, sim, st);
}
cudaError_t launch_plaq_force(int prec, bool theta, const GeoH& h, const void* U, const void* Ui,
                              const void* Pq, const void* Dq, const void* F, void* Gq, void* C,
                              double beta, cudaStream_t st) {
  return prec == 0 ? launch_plaq_force_f64(theta, h, U, Ui, Pq, Dq, F, Gq, C, beta, st)
                   : launch_plaq_force_f32(theta, h, U, Ui, Pq, Dq, F, Gq, C, beta, st);
}
cudaError_t launch_update_gather(int prec, int mode, const GeoH& h, const void* U, const void* C,
                                 void* out, double eps, uint64_t seed, const uint32_t* step, cudaStream_t st) {
  return prec == 0 ? launch_update_gather_f64(mode, h, U, C, out, eps, seed, step, st)
                   : launch_update_gather_f32(mode, h, U, C, out, eps, seed, step, st);
}
}  // namespace clgc

namespace clgc {
// Advances the device step counter after an update (one thread).
__global__ void k_step_bump(uint32_t* step) { *step += 1u; }

cudaError_t launch_step_bump(uint32_t* step, cudaStream_t st) {
  k_step_bump<<<1, 1, 0, st>>>(step);
  return cudaGetLastError();
}
}  // namespace clgc
