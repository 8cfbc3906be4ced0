// ensemble.cuh -- fused-batch wrappers of the CL-step kernels (k_update.cuh):
// one launch runs the blocks of every chain of a batch.  Block i of a launch
// reads its work item (chain, block index the chain's own launch would have
// used) and the chain's descriptor, then runs the same kernel body with that
// chain's geometry, buffers and parameters, so each chain's arithmetic is
// exactly that of its own launches.  Included by k_update_f64.cu and
// k_update_f32.cu, which instantiate it for their link type.
#pragma once
#include "k_update.cuh"
#include "launch.h"

namespace clgc {

__device__ __forceinline__ Geo geo_of(const ChainDesc& c) {
  Geo g;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    g.L[mu] = c.L[mu];
    g.stride[mu] = c.stride[mu];
  }
  g.V = c.V;
  return g;
}

template <typename T>
__global__ void __launch_bounds__(TUNE_MAX_BLOCK) k_ens_inverse(const ChainDesc* __restrict__ cd,
                                                                const WorkItem* __restrict__ w) {
  typedef typename vec2_of<T>::type V2;
  const WorkItem it = w[blockIdx.x];
  const ChainDesc& c = cd[it.chain];
  k_link_inverse_body<T>(geo_of(c), (const V2*)c.U, (V2*)c.Ui, it.vb);
}

template <typename T>
__global__ void __launch_bounds__(TUNE_MAX_BLOCK) k_ens_plaq(const ChainDesc* __restrict__ cd,
                                                             const WorkItem* __restrict__ w) {
  typedef typename vec2_of<T>::type V2;
  const WorkItem it = w[blockIdx.x];
  const ChainDesc& c = cd[it.chain];
  k_plaq_body<T>(geo_of(c), (const V2*)c.U, (const V2*)c.Ui, (V2*)c.Pq, (V2*)c.Dq, it.vb);
}

template <typename T>
__global__ void __launch_bounds__(TUNE_MAX_BLOCK) k_ens_clover(const ChainDesc* __restrict__ cd,
                                                               const WorkItem* __restrict__ w) {
  typedef typename vec2_of<T>::type V2;
  const WorkItem it = w[blockIdx.x];
  const ChainDesc& c = cd[it.chain];
  k_clover_rot_body<T>(geo_of(c), (const V2*)c.U, (const V2*)c.Ui, (const V2*)c.Dq, (V2*)c.F, c.sre, c.sim, it.vb);
}

template <typename T>
__global__ void __launch_bounds__(TUNE_MAX_BLOCK) k_ens_force_wilson(const ChainDesc* __restrict__ cd,
                                                                     const WorkItem* __restrict__ w) {
  typedef typename vec2_of<T>::type V2;
  const WorkItem it = w[blockIdx.x];
  const ChainDesc& c = cd[it.chain];
  k_plaq_force_wilson_body<T>(geo_of(c), (const V2*)c.U, (const V2*)c.Ui, (const V2*)c.Dq, (V2*)c.C,
                              (T)(c.beta / 6.0), it.vb);
}

template <typename T>
__global__ void __launch_bounds__(TUNE_MAX_BLOCK) k_ens_force_a(const ChainDesc* __restrict__ cd,
                                                                const WorkItem* __restrict__ w) {
  typedef typename vec2_of<T>::type V2;
  const WorkItem it = w[blockIdx.x];
  const ChainDesc& c = cd[it.chain];
  k_plaq_force_a_body<T>(geo_of(c), (const V2*)c.U, (const V2*)c.Ui, (const V2*)c.Dq, (const V2*)c.F, (V2*)c.Gq,
                         (V2*)c.C, (T)(c.beta / 6.0), it.vb);
}

template <typename T>
__global__ void __launch_bounds__(TUNE_MAX_BLOCK) k_ens_force_b(const ChainDesc* __restrict__ cd,
                                                                const WorkItem* __restrict__ w) {
  typedef typename vec2_of<T>::type V2;
  const WorkItem it = w[blockIdx.x];
  const ChainDesc& c = cd[it.chain];
  k_plaq_force_b_body<T>(geo_of(c), (const V2*)c.U, (const V2*)c.Ui, (const V2*)c.Pq, (const V2*)c.Dq,
                         (const V2*)c.F, (const V2*)c.Gq, (V2*)c.C, (T)(c.beta / 6.0), it.vb);
}

template <typename T>
__global__ void __maxnreg__(FORCE_AB_MAXNREG) k_ens_force_ab(const ChainDesc* __restrict__ cd,
                                                                 const WorkItem* __restrict__ w) {
  typedef typename vec2_of<T>::type V2;
  const WorkItem it = w[blockIdx.x];
  const ChainDesc& c = cd[it.chain];
  k_plaq_force_ab_body<T>(geo_of(c), (const V2*)c.U, (const V2*)c.Ui, (const V2*)c.Pq, (const V2*)c.Dq,
                          (const V2*)c.F, (V2*)c.C, (T)(c.beta / 6.0), it.vb);
}

// The update modes as the runtime runs them: MODE_UPDATE reads C and writes
// Un at the fixed step size; MODE_DRIFTMAX writes the drift into Pq (dead
// after the force); MODE_UPDATE_X reads it back and writes Un at the device
// step size.
template <typename T, int MODE>
__global__ void __launch_bounds__(TUNE_MAX_BLOCK) k_ens_update(const ChainDesc* __restrict__ cd,
                                                               const WorkItem* __restrict__ w) {
  typedef typename vec2_of<T>::type V2;
  const WorkItem it = w[blockIdx.x];
  const ChainDesc& c = cd[it.chain];
  UpdArgs a;
  a.beta = 0.0;
  a.eps = c.eps;
  a.sqrt_eps = c.sqrt_eps;
  a.seed = c.seed;
  a.sd = c.sd;
  a.adaptive = MODE == MODE_UPDATE_X ? 1 : 0;
  const V2* in = (const V2*)(MODE == MODE_UPDATE_X ? c.Pq : c.C);
  V2* out = (V2*)(MODE == MODE_DRIFTMAX ? c.Pq : c.Un);
  k_update_gather_body<T, MODE>(geo_of(c), (const V2*)c.U, in, out, a, it.vb);
}

// Launch family fam of the CL step for link type T (FP64 runs the theta
// force as its two kernels).
template <typename T>
cudaError_t launch_ens_step_family(int fam, const ChainDesc* cd, const WorkItem* w, int nw, cudaStream_t st) {
  if (nw <= 0) return cudaSuccess;
  const unsigned n = (unsigned)nw;
  switch (fam) {
    case ENS_INVERSE: k_ens_inverse<T><<<n, ENS_BLOCK, 0, st>>>(cd, w); break;
    case ENS_PLAQ: k_ens_plaq<T><<<n, ENS_BLOCK, 0, st>>>(cd, w); break;
    case ENS_CLOVER: k_ens_clover<T><<<n, ENS_BLOCK, 0, st>>>(cd, w); break;
    case ENS_FORCE_WILSON: k_ens_force_wilson<T><<<n, ENS_BLOCK, 0, st>>>(cd, w); break;
    case ENS_FORCE_THETA:
      if constexpr (sizeof(T) == 8) {  // FP64: the split form (only it is instantiated)
        k_ens_force_a<T><<<n, ENS_BLOCK, 0, st>>>(cd, w);
        k_ens_force_b<T><<<n, ENS_BLOCK, 0, st>>>(cd, w);
      } else {
        k_ens_force_ab<T><<<n, ENS_BLOCK, 0, st>>>(cd, w);
      }
      break;
    case ENS_UPDATE: k_ens_update<T, MODE_UPDATE><<<n, ENS_BLOCK, 0, st>>>(cd, w); break;
    case ENS_DRIFTMAX: k_ens_update<T, MODE_DRIFTMAX><<<n, ENS_BLOCK, 0, st>>>(cd, w); break;
    case ENS_UPDATE_X: k_ens_update<T, MODE_UPDATE_X><<<n, ENS_BLOCK, 0, st>>>(cd, w); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace clgc
