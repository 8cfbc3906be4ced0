// k_update_f32.cu -- instantiation of the CL update kernel for float links.
#include "k_update.cuh"
#include "launch.h"

namespace clgc {

cudaError_t launch_cl_update_f32(bool theta, int mode, const GeoH& h, const void* U, const void* F,
                                void* out, double beta, double eps, uint64_t seed, uint32_t step,
                                cudaStream_t st) {
  typedef vec2_of<float>::type V2;
  Geo g = make_geo(h.L, h.V);
  UpdArgs a;
  a.beta = beta;
  a.eps = eps;
  a.sqrt_eps = sqrt(eps);
  a.seed = seed;
  a.step = step;
  dim3 grid((unsigned)((g.V + 127) / 128), 4);
  const V2* u = (const V2*)U;
  const V2* f = (const V2*)F;
  V2* o = (V2*)out;
  if (theta) {
    if (mode == MODE_DRIFT) k_cl_update<float, true, MODE_DRIFT><<<grid, 128, 0, st>>>(g, u, f, o, a);
    else k_cl_update<float, true, MODE_UPDATE><<<grid, 128, 0, st>>>(g, u, f, o, a);
  } else {
    if (mode == MODE_DRIFT) k_cl_update<float, false, MODE_DRIFT><<<grid, 128, 0, st>>>(g, u, f, o, a);
    else k_cl_update<float, false, MODE_UPDATE><<<grid, 128, 0, st>>>(g, u, f, o, a);
  }
  return cudaGetLastError();
}

}  // namespace clgc
