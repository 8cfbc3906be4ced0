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
const int NSLOT_PLAQ = 3, NSLOT_CLOVER = 3, NSLOT_WILSON = 4, NSLOT_FORCE = 4, NSLOT_UPDATE = 3;
const int DF_FORCE_BLOCK = 128;  // the DF64 force kernels' largest block (their launch bound)

// Plaquettes of the DF64 form in three workspace slots (four blocks of 128
// per SM): P = ((U_mu(x) U_nu(x+mu)) U_mu(x+nu)^{-1}) U_nu(x)^{-1}, the same
// three products as k_plaq associated to the left.
__global__ void __launch_bounds__(TUNE_MAX_BLOCK) k_plaq_df(Geo g, const float4* __restrict__ U,
                                                       const float4* __restrict__ Ui, float4* __restrict__ Pq,
                                                       float4* __restrict__ Dq) {
  const int p = blockIdx.x % 6, mu = plane_mu(p), nu = plane_nu(p);
  const int s = (blockIdx.x / 6) * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int x[4];
  site_coords(g, s, x);
  Work<df64, 3> ws(0);
  mat<df64>&a = ws[0], &b = ws[1], &c = ws[2];
  load(a, U, mu, s, g.V);
  load(b, U, nu, hop(g, s, x, mu, 1), g.V);
  mul(c, a, b);  // U_mu(x) U_nu(x+mu)
  load(a, Ui, mu, hop(g, s, x, nu, 1), g.V);
  mul(b, c, a);
  load(a, Ui, nu, s, g.V);
  mul(c, b, a);  // P
  store(Pq, p, s, g.V, c);
  adj(b, c);
#pragma unroll
  for (int k = 0; k < 9; ++k) c.e[k] = csub(c.e[k], b.e[k]);
  store(Dq, p, s, g.V, c);
}

// The clover field of the DF64 form (k_clover_rot's leaves) in three
// workspace slots: the carried leaves are formed with in-place left
// products, w <- w d, so no product needs a slot of its own.
__global__ void __launch_bounds__(TUNE_MAX_BLOCK) k_clover_rot_df(Geo g, const float4* __restrict__ U,
                                                             const float4* __restrict__ Ui,
                                                             const float4* __restrict__ Dq, float4* __restrict__ F,
                                                             df64 sre, df64 sim) {
  const int p = blockIdx.x % 6, mu = plane_mu(p), nu = plane_nu(p);
  const int s = (blockIdx.x / 6) * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int x[4];
  site_coords(g, s, x);
  const int xmm = hop(g, s, x, mu, -1), xmn = hop(g, s, x, nu, -1);
  const int xmm_mn = hop2(g, s, x, mu, -1, nu, -1);
  Work<df64, 3> ws(0);
  mat<df64>&acc = ws[0], &w = ws[1], &d = ws[2];
  load(acc, Dq, p, s, g.V);
  // L2 = U_mu(x-mu)^{-1} D(x-mu) U_mu(x-mu)
  load(w, Ui, mu, xmm, g.V);
  load(d, Dq, p, xmm, g.V);
  mul_left_inplace_df(w, d);
  load(d, U, mu, xmm, g.V);
  mul_acc<+1>(acc, w, d);
  // L3 + L4 = U_nu(x-nu)^{-1} [D(x-nu) + U_mu(x-mu-nu)^{-1} D(x-mu-nu) U_mu(x-mu-nu)] U_nu(x-nu)
  load(w, Ui, mu, xmm_mn, g.V);
  load(d, Dq, p, xmm_mn, g.V);
  mul_left_inplace_df(w, d);
  load(d, U, mu, xmm_mn, g.V);
  mul_left_inplace_df(w, d);
  load(d, Dq, p, xmn, g.V);
#pragma unroll
  for (int k = 0; k < 9; ++k) d.e[k] = cadd(d.e[k], w.e[k]);
  load(w, Ui, nu, xmn, g.V);
  mul_left_inplace_df(w, d);
  load(d, U, nu, xmn, g.V);
  mul_acc<+1>(acc, w, d);
  const cx<df64> sc = {sre, sim};
#pragma unroll
  for (int k = 0; k < 9; ++k) acc.e[k] = cmul(acc.e[k], sc);
  store(F, p, s, g.V, acc);
}

// The theta force of the DF64 form: the stages of k_update.cuh rescheduled so
// that four workspace slots suffice (Gh and three more; the FP64 stages hold
// five matrices at their peak), which lets three blocks of 128 threads share
// an SM instead of two.  The matrices given up early are re-read from memory
// (D from Dq, the slot-0 partial from C), and (ab) G2 (ab)^{-1} is formed as
// ((ab) G2 b^{-1}) a^{-1}, the same four products.
__device__ __forceinline__ void force_stage_a_df(mat<df64>& Gh, const Geo& g, int s, const int x[4], int p,
                                                 const float4* __restrict__ U, const float4* __restrict__ Ui,
                                                 const float4* __restrict__ Dq, const float4* __restrict__ F,
                                                 float4* C, df64 beta6) {
  const int mu = plane_mu(p), nu = plane_nu(p), pc = 5 - p;
  const unsigned long long m = (p == 1 || p == 4) ? 0x8000000000000000ull : 0ull;
  const int c1 = hop(g, s, x, mu, 1);
  Work<df64, 3> ws(1);  // slot 0 holds Gh
  mat<df64>&D = ws[0], &t = ws[1], &q = ws[2];
  // corner c0: slot 0 partial = [D, G0] - (beta/6) D, formed in t
  load(D, Dq, p, s, g.V);
  load_signed(Gh, F, pc, s, g.V, m);
  scaled(t, -beta6, D);
  commutator_acc(t, D, Gh);
  store(C, 4 * p + 0, s, g.V, t);
  // corner c1: G1^ = a G1 a^{-1}; slot 2 partial = slot 0 partial + [D, G1^]
  load_signed(t, F, pc, c1, g.V, m);
  load(q, U, mu, s, g.V);
  mul(D, q, t);  // a G1
  load(q, Ui, mu, s, g.V);
  mul(t, D, q);  // G1^
#pragma unroll
  for (int k = 0; k < 9; ++k) Gh.e[k] = cadd(Gh.e[k], t.e[k]);
  load(D, Dq, p, s, g.V);
  load_rw(q, C, 4 * p + 0, s, g.V);
  commutator_acc(q, D, t);
  store(C, 4 * p + 2, s, g.V, q);
  // corner c2: G2^ = ((ab) G2 b^{-1}) a^{-1}
  load(q, U, mu, s, g.V);
  load(t, U, nu, c1, g.V);
  mul(D, q, t);  // ab
  load_signed(q, F, pc, hop(g, c1, x, nu, 1), g.V, m);
  mul(t, D, q);  // ab G2
  load(q, Ui, nu, c1, g.V);
  mul(D, t, q);  // ab G2 b^{-1}
  load(q, Ui, mu, s, g.V);
  mul_acc<+1>(Gh, D, q);
}

__device__ __forceinline__ void force_stage_b_df(mat<df64>& Gh, const Geo& g, int s, const int x[4], int p,
                                                 const float4* __restrict__ U, const float4* __restrict__ Ui,
                                                 const float4* __restrict__ Pq, const float4* __restrict__ Dq,
                                                 const float4* __restrict__ F, float4* C, df64 beta6) {
  const int mu = plane_mu(p), nu = plane_nu(p), pc = 5 - p;
  const unsigned long long m = (p == 1 || p == 4) ? 0x8000000000000000ull : 0ull;
  const int c3 = hop(g, s, x, nu, 1);
  Work<df64, 3> ws(1);  // slot 0 holds Gh
  mat<df64>&D = ws[0], &t = ws[1], &q = ws[2];
  // corner c3: G3r = u G3 u^{-1} (in q); slot 3 partial = [D, G3r] + (beta/6) D
  load_signed(q, F, pc, c3, g.V, m);
  load(D, U, nu, s, g.V);
  mul(t, D, q);
  load(D, Ui, nu, s, g.V);
  mul(q, t, D);
  load(D, Dq, p, s, g.V);
  scaled(t, beta6, D);
  commutator_acc(t, D, q);
  store(C, 4 * p + 3, s, g.V, t);
  // G^ += P G3r P^{-1}, P^{-1} = P - D; the plaquette's D then lives in q
  load(t, Pq, p, s, g.V);
  mul(D, t, q);  // P G3r
  load(q, Dq, p, s, g.V);
#pragma unroll
  for (int k = 0; k < 9; ++k) t.e[k] = csub(t.e[k], q.e[k]);  // P^{-1}
  mul_acc<+1>(Gh, D, t);
  // K = P^{-1} G^ + G^ P, in D
  mul(D, t, Gh);
#pragma unroll
  for (int k = 0; k < 9; ++k) t.e[k] = cadd(t.e[k], q.e[k]);  // P again
  mul_acc<+1>(D, Gh, t);
  // slot 1: -K + (beta/6) D
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    t.e[k].re = fma(beta6, q.e[k].re, -D.e[k].re);
    t.e[k].im = fma(beta6, q.e[k].im, -D.e[k].im);
  }
  store(C, 4 * p + 1, s, g.V, t);
  // slot 0: K + partial
  load_rw(t, C, 4 * p + 0, s, g.V);
#pragma unroll
  for (int k = 0; k < 9; ++k) t.e[k] = cadd(t.e[k], D.e[k]);
  store(C, 4 * p + 0, s, g.V, t);
  // slot 2: a^{-1} (K + partial) a
  load_rw(t, C, 4 * p + 2, s, g.V);
#pragma unroll
  for (int k = 0; k < 9; ++k) t.e[k] = cadd(t.e[k], D.e[k]);
  load(Gh, Ui, mu, s, g.V);
  mul(q, Gh, t);
  load(Gh, U, mu, s, g.V);
  mul(t, q, Gh);
  store(C, 4 * p + 2, s, g.V, t);
  // slot 3: u^{-1} (-K + partial) u
  load_rw(t, C, 4 * p + 3, s, g.V);
#pragma unroll
  for (int k = 0; k < 9; ++k) t.e[k] = csub(t.e[k], D.e[k]);
  load(Gh, Ui, nu, s, g.V);
  mul(q, Gh, t);
  load(Gh, U, nu, s, g.V);
  mul(t, q, Gh);
  store(C, 4 * p + 3, s, g.V, t);
}

__global__ void __launch_bounds__(DF_FORCE_BLOCK, 3) k_plaq_force_a_df(Geo g, const float4* __restrict__ U,
                                                                    const float4* __restrict__ Ui,
                                                                    const float4* __restrict__ Dq,
                                                                    const float4* __restrict__ F,
                                                                    float4* Gq, float4* C,
                                                                    df64 beta6) {
  const int p = blockIdx.x % 6;
  const int s = (blockIdx.x / 6) * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int x[4];
  site_coords(g, s, x);
  Work<df64, 1> wg(0);
  mat<df64>& Gh = wg[0];
  force_stage_a_df(Gh, g, s, x, p, U, Ui, Dq, F, C, beta6);
  store(Gq, GQ_PLANE * p, s, g.V, Gh);  // plane 4p + 1 of C (see k_plaq_force_a)
}
__global__ void __launch_bounds__(DF_FORCE_BLOCK, 3) k_plaq_force_b_df(Geo g, const float4* __restrict__ U,
                                                                    const float4* __restrict__ Ui,
                                                                    const float4* __restrict__ Pq,
                                                                    const float4* __restrict__ Dq,
                                                                    const float4* __restrict__ F,
                                                                    const float4* Gq, float4* C,
                                                                    df64 beta6) {
  const int p = blockIdx.x % 6;
  const int s = (blockIdx.x / 6) * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int x[4];
  site_coords(g, s, x);
  Work<df64, 1> wg(0);
  mat<df64>& Gh = wg[0];
  load_rw(Gh, Gq, GQ_PLANE * p, s, g.V);  // before stage b writes slot 1 of (p, s) over it
  force_stage_b_df(Gh, g, s, x, p, U, Ui, Pq, Dq, F, C, beta6);
}

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
  cudaError_t e = allow_ws(k_plaq_df, NSLOT_PLAQ);
  if (e == cudaSuccess) e = allow_ws(k_clover_rot_df, NSLOT_CLOVER);
  if (e == cudaSuccess) e = allow_ws(k_plaq_force_wilson<df64>, NSLOT_WILSON);
  if (e == cudaSuccess) e = allow_ws(k_plaq_force_a_df, NSLOT_FORCE);
  if (e == cudaSuccess) e = allow_ws(k_plaq_force_b_df, NSLOT_FORCE);
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
  k_plaq_df<<<grid(g.V, 6, bs), bs, ws_bytes(NSLOT_PLAQ, bs), st>>>(g, (const V2*)U, (const V2*)Ui, (V2*)Pq, (V2*)Dq);
  return cudaGetLastError();
}

cudaError_t launch_clover_rot_df64(const GeoH& h, const void* U, const void* Ui, const void* Dq,
                                 void* F, double sre, double sim, cudaStream_t st) {
  Geo g = make_geo(h.L, h.V);
  const int bs = block_of(h, TUNE_CLOVER);
  k_clover_rot_df<<<grid(g.V, 6, bs), bs, ws_bytes(NSLOT_CLOVER, bs), st>>>(g, (const V2*)U, (const V2*)Ui, (const V2*)Dq,
                                                                           (V2*)F, df_host(sre), df_host(sim));
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
  const int bf = bs < DF_FORCE_BLOCK ? bs : DF_FORCE_BLOCK;
  k_plaq_force_a_df<<<grid(g.V, 6, bf), bf, ws_bytes(NSLOT_FORCE, bf), st>>>(g, (const V2*)U, (const V2*)Ui, (const V2*)Dq,
                                                                            (const V2*)F, (V2*)Gq, (V2*)C, b6);
  k_plaq_force_b_df<<<grid(g.V, 6, bf), bf, ws_bytes(NSLOT_FORCE, bf), st>>>(g, (const V2*)U, (const V2*)Ui, (const V2*)Pq,
                                                                            (const V2*)Dq, (const V2*)F, (const V2*)Gq,
                                                                            (V2*)C, b6);
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

