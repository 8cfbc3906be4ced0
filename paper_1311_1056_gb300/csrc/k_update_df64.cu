// k_update_df64.cu -- the CL-step kernels (k_update.cuh) for double-float
// links (df64.cuh): the link algebra, the noise, the exponential and the
// re-projection in double-float on the FP32 pipe, the matrices of the
// out-of-line products in a shared-memory workspace (Work, su3.cuh).
#include "k_update.cuh"
#include "launch.h"

namespace clgc {

namespace {
typedef vec2_of<df64>::type V2;
// host split of a double into the hi + lo floats of a df64
inline df64 df_host(double d) {
  const float h = (float)d;
  return df64(h, (float)(d - (double)h));
}
// 1-D grid, plane (or direction) fastest: the blocks resident at one time
// cover every plane of a range of sites, so shared neighbours stay in cache.
inline dim3 grid(int V, int planes, int bs) { return dim3((unsigned)(((V + bs - 1) / bs) * planes)); }
// dynamic shared memory of a kernel with nslot workspace matrices per thread
inline size_t ws_bytes(int nslot, int bs) { return (size_t)nslot * sizeof(mat<df64>) * (size_t)bs; }
const int NSLOT_PLAQ = 5, NSLOT_CLOVER = 4, NSLOT_WILSON = 4, NSLOT_FORCE = 5, NSLOT_UPDATE = 3;

template <typename K>
cudaError_t allow_ws(K kernel, int nslot) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)ws_bytes(nslot, TUNE_MAX_BLOCK));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  return e;
}
}  // namespace

cudaError_t prepare_df64_kernels() {
  cudaError_t e = allow_ws(k_plaq<df64>, NSLOT_PLAQ);
  if (e == cudaSuccess) e = allow_ws(k_clover_rot<df64>, NSLOT_CLOVER);
  if (e == cudaSuccess) e = allow_ws(k_plaq_force_wilson<df64>, NSLOT_WILSON);
  if (e == cudaSuccess) e = allow_ws(k_plaq_force_a<df64>, NSLOT_FORCE);
  if (e == cudaSuccess) e = allow_ws(k_plaq_force_b<df64>, NSLOT_FORCE);
  if (e == cudaSuccess) e = allow_ws(k_update_gather<df64, MODE_UPDATE>, NSLOT_UPDATE);
  if (e == cudaSuccess) e = allow_ws(k_update_gather<df64, MODE_DRIFT>, NSLOT_UPDATE);
  if (e == cudaSuccess) e = allow_ws(k_update_gather<df64, MODE_DRIFTMAX>, NSLOT_UPDATE);
  if (e == cudaSuccess) e = allow_ws(k_update_gather<df64, MODE_UPDATE_X>, NSLOT_UPDATE);
  return e;
}

cudaError_t launch_link_inverse_df64(const GeoH& h, const void* U, void* Ui, cudaStream_t st) {
  Geo g = make_geo(h.L, h.V);
  k_link_inverse<df64><<<grid(g.V, 4, block_of(h, TUNE_CLOVER)), block_of(h, TUNE_CLOVER), 0, st>>>(g, (const V2*)U, (V2*)Ui);
  return cudaGetLastError();
}

cudaError_t launch_plaq_df64(const GeoH& h, const void* U, const void* Ui, void* Pq, void* Dq,
                           cudaStream_t st) {
  Geo g = make_geo(h.L, h.V);
  const int bs = block_of(h, TUNE_CLOVER);
  k_plaq<df64><<<grid(g.V, 6, bs), bs, ws_bytes(NSLOT_PLAQ, bs), st>>>(g, (const V2*)U, (const V2*)Ui, (V2*)Pq, (V2*)Dq);
  return cudaGetLastError();
}

cudaError_t launch_clover_rot_df64(const GeoH& h, const void* U, const void* Ui, const void* Dq,
                                 void* F, double sre, double sim, cudaStream_t st) {
  Geo g = make_geo(h.L, h.V);
  const int bs = block_of(h, TUNE_CLOVER);
  k_clover_rot<df64><<<grid(g.V, 6, bs), bs, ws_bytes(NSLOT_CLOVER, bs), st>>>(g, (const V2*)U, (const V2*)Ui, (const V2*)Dq,
                                                  (V2*)F, sre, sim);
  return cudaGetLastError();
}

cudaError_t launch_plaq_force_df64(bool theta, const GeoH& h, const void* U, const void* Ui,
                                 const void* Pq, const void* Dq, const void* F, void* Gq, void* C,
                                 double beta, cudaStream_t st) {
  Geo g = make_geo(h.L, h.V);
  const df64 b6 = df_host(beta / 6.0);
  const int bs = block_of(h, TUNE_FORCE);
  if (!theta) {
    k_plaq_force_wilson<df64><<<grid(g.V, 6, bs), bs, ws_bytes(NSLOT_WILSON, bs), st>>>(g, (const V2*)U, (const V2*)Ui, (const V2*)Dq,
                                                         (V2*)C, b6);
    return cudaGetLastError();
  }
  k_plaq_force_a<df64><<<grid(g.V, 6, bs), bs, ws_bytes(NSLOT_FORCE, bs), st>>>(g, (const V2*)U, (const V2*)Ui, (const V2*)Dq,
                                                  (const V2*)F, (V2*)Gq, (V2*)C, b6);
  k_plaq_force_b<df64><<<grid(g.V, 6, bs), bs, ws_bytes(NSLOT_FORCE, bs), st>>>(g, (const V2*)U, (const V2*)Ui, (const V2*)Pq,
                                                  (const V2*)Dq, (const V2*)F, (const V2*)Gq, (V2*)C, b6);
  return cudaGetLastError();
}

cudaError_t launch_update_gather_df64(int mode, const GeoH& h, const void* U, const void* C, void* out,
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
  const size_t sm = ws_bytes(NSLOT_UPDATE, bs);
  const V2* u = (const V2*)U;
  const V2* c = (const V2*)C;
  V2* o = (V2*)out;
  switch (mode) {
    case MODE_DRIFT: k_update_gather<df64, MODE_DRIFT><<<gr, bs, sm, st>>>(g, u, c, o, a); break;
    case MODE_DRIFTMAX: k_update_gather<df64, MODE_DRIFTMAX><<<gr, bs, sm, st>>>(g, u, c, o, a); break;
    case MODE_UPDATE_X: k_update_gather<df64, MODE_UPDATE_X><<<gr, bs, sm, st>>>(g, u, c, o, a); break;
    default: k_update_gather<df64, MODE_UPDATE><<<gr, bs, sm, st>>>(g, u, c, o, a); break;
  }
  return cudaGetLastError();
}

}  // namespace clgc

