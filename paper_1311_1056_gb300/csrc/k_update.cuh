// k_update.cuh -- the CL step: plaquettes, clover field, per-plaquette drift
// contributions, and the per-link gather + noise + FP64 exponential update
// with det re-projection.
//
// Action (Sec. 5, eq. "eq:st"): S = S_W - i theta sum_x q_L(x) with the
// Wilson action continued holomorphically (U^+ -> U^{-1}) and
//   q_L(x) = kappa [Tr F01 F23 - Tr F02 F13 + Tr F03 F12](x),  kappa = -1/(256 pi^2),
// where F_{mu nu}(x) = sum over the four clover leaves L at x of (L - L^{-1})
// (the paper's signed eps-tilde sum regrouped by plane).
//
// Drift matrix X_S of a link, D_a S = i Tr(lambda_a X_S), D_a the left
// derivative U -> exp(i a lambda_a) U.  Every term of S is a function of
// plaquettes, so X_S is a sum over the six plaquettes through the link, and
// each plaquette serves its four links at once.  For the plaquette based at x
// in plane (mu < nu), P = a b c d with a = U_mu(x), b = U_nu(x+mu),
// c = U_mu(x+nu)^{-1}, d = U_nu(x)^{-1} = u^{-1}, corners c0 = x, c1 = x+mu,
// c2 = x+mu+nu, c3 = x+nu, D = P - P^{-1}, and the dual fields
// G_k = s F^_{comp}(c_k) (F^ = -i theta kappa F, s = +1, -1, +1 for the pairs
// 01|23, 02|13, 03|12) carried to c0:
//   G1^ = a G1 a^{-1}, G2^ = (ab) G2 (ab)^{-1}, G3r = u G3 u^{-1}, G3^ = P G3r P^{-1},
//   G^ = G0 + G1^ + G2^ + G3^,   K = G^ P + P^{-1} G^,   [A, B] = AB - BA,
// the product rule over the four leaves of the plaquette (one per corner) and
// the Wilson term -(beta/6) Tr(P + P^{-1}) give, each in its own link's frame,
//   U_mu(x)    : K + [D, G0] - (beta/6) D
//   U_nu(x)    : -K + (beta/6) D
//   U_nu(x+mu) : a^{-1} (K + [D, G0] + [D, G1^] - (beta/6) D) a
//   U_mu(x+nu) : u^{-1} (-K + [D, G3r] + (beta/6) D) u
// (about 22 matrix products per plaquette for all four links).
//
// Update (the CL step of the method, Sec. 2 and its refs):
//   K_a = -D_a S,  A = i lambda_a (eps K_a + sqrt(eps) eta_a)
//     = 2 eps (X_S - Tr X_S / 3) + i sqrt(eps) eta_a lambda_a,  <eta_a eta_b> = 2 delta_ab,
//   U' = exp(A) U  (exp in FP64),  U' <- U' det(U')^{-1/3}  (FP64 factor).
#pragma once
#include <type_traits>

#include "expm.cuh"
#include "lattice.cuh"
#include "launch.h"
#include "philox.cuh"
#include "su3.cuh"

namespace clgc {

enum { MODE_UPDATE = 0, MODE_DRIFT = 1, MODE_DRIFTMAX = 2, MODE_UPDATE_X = 3 };

struct UpdArgs {
  double beta, eps, sqrt_eps;
  uint64_t seed;
  StepDev* sd;    // device-resident step state (graph-replayable)
  int adaptive;   // 1: the step size is sd->eps_n (set by the drift pass)
};

// Sign flip on the integer pipe (no floating-point instruction).
__device__ __forceinline__ double flip(double x, unsigned long long m) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)m);
}
__device__ __forceinline__ float flip(float x, unsigned long long m) {
  return __int_as_float(__float_as_int(x) ^ (int)(m >> 32));
}
__device__ __forceinline__ df64 flip(df64 x, unsigned long long m) {
  return df64(flip(x.hi, m), flip(x.lo, m));
}
template <typename T>
__device__ __forceinline__ void load_signed(mat<T>& G, const typename vec2_of<T>::type* F, int p,
                                            int s, int V, unsigned long long m) {
  load(G, F, p, s, V);
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    G.e[k].re = flip(G.e[k].re, m);
    G.e[k].im = flip(G.e[k].im, m);
  }
}

// Plain (coherent) loads, for data this kernel itself wrote.
template <typename T>
__device__ __forceinline__ void load_rw(mat<T>& a, const typename vec2_of<T>::type* f, int plane,
                                        int site, int V) {
  const typename vec2_of<T>::type* p = f + (size_t)plane * 9 * V + site;
#pragma unroll
  for (int k = 0; k < 9; ++k) a.e[k] = unpack(p[(size_t)k * V]);
}

// c += [a, b] = a b - b a
template <typename T>
__device__ __forceinline__ void commutator_acc(mat<T>& c, const mat<T>& a, const mat<T>& b) {
  mul_acc<+1>(c, a, b);
  mul_acc<-1>(c, b, a);
}

template <typename T>
__device__ __forceinline__ void scaled(mat<T>& r, T c, const mat<T>& a) {
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    r.e[k].re = c * a.e[k].re;
    r.e[k].im = c * a.e[k].im;
  }
}

// ---------------------------------------------------------------- inverses
// Ui = adj(U) = U^{-1} for every link (det U = 1 by the re-projection).
template <typename T>
__device__ __forceinline__ void k_link_inverse_body(Geo g, const typename vec2_of<T>::type* __restrict__ U,
                                                      typename vec2_of<T>::type* __restrict__ Ui, int vb) {
  const int mu = vb % 4;
  const int s = (vb / 4) * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  mat<T> u, ui;
  load(u, U, mu, s, g.V);
  adj(ui, u);
  store(Ui, mu, s, g.V, ui);
}
template <typename T>
__global__ void __launch_bounds__(TUNE_MAX_BLOCK) k_link_inverse(Geo g, const typename vec2_of<T>::type* __restrict__ U,
                                                      typename vec2_of<T>::type* __restrict__ Ui) {
  k_link_inverse_body<T>(g, U, Ui, blockIdx.x);
}

// The inverse of link (mu, site) as the plaquette, clover and force kernels
// use it.  FP64: loaded from the U^{-1} field the link-inverse pass wrote
// (forming it costs 126 flops on the FP64 pipe these kernels are bound by).
// FP32 storage: formed from the link (the same adjugate, so the same bits,
// on the FP32 pipe, which these memory- and latency-bound kernels leave
// idle); no link-inverse pass runs and the load usually hits a line of U the
// kernel reads anyway.
template <typename T>
__host__ __device__ constexpr bool inverse_on_the_fly() { return sizeof(T) == 4; }
template <typename T>
__device__ __forceinline__ void load_inv(mat<T>& ui, const typename vec2_of<T>::type* __restrict__ U,
                                         const typename vec2_of<T>::type* __restrict__ Ui, int mu, int site, int V) {
  if constexpr (inverse_on_the_fly<T>()) {
    mat<T> u;
    load(u, U, mu, site, V);
    adj(ui, u);
  } else {
    load(ui, Ui, mu, site, V);
  }
}

// ------------------------------------------------------------- plaquettes
// P_{mu nu}(x) = U_mu(x) U_nu(x+mu) U_mu(x+nu)^{-1} U_nu(x)^{-1} and
// D = P - P^{-1}, six planes per site.
template <typename T>
__device__ __forceinline__ void k_plaq_body(Geo g, const typename vec2_of<T>::type* __restrict__ U,
                                              const typename vec2_of<T>::type* __restrict__ Ui,
                                              typename vec2_of<T>::type* __restrict__ Pq,
                                              typename vec2_of<T>::type* __restrict__ Dq, int vb) {
  const int p = vb % 6, mu = plane_mu(p), nu = plane_nu(p);
  const int s = (vb / 6) * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int x[4];
  site_coords(g, s, x);
  Work<T, 5> ws(0);
  mat<T>&a = ws[0], &b = ws[1], &A = ws[2], &B = ws[3], &P = ws[4];
  load(a, U, mu, s, g.V);
  load(b, U, nu, hop(g, s, x, mu, 1), g.V);
  mul(A, a, b);
  load_inv(a, U, Ui, mu, hop(g, s, x, nu, 1), g.V);
  load_inv(b, U, Ui, nu, s, g.V);
  mul(B, a, b);
  mul(P, A, B);
  store(Pq, p, s, g.V, P);
  adj(A, P);
#pragma unroll
  for (int k = 0; k < 9; ++k) P.e[k] = csub(P.e[k], A.e[k]);
  store(Dq, p, s, g.V, P);
}
template <typename T>
__global__ void __launch_bounds__(TUNE_MAX_BLOCK) k_plaq(Geo g, const typename vec2_of<T>::type* __restrict__ U,
                                              const typename vec2_of<T>::type* __restrict__ Ui,
                                              typename vec2_of<T>::type* __restrict__ Pq,
                                              typename vec2_of<T>::type* __restrict__ Dq) {
  k_plaq_body<T>(g, U, Ui, Pq, Dq, blockIdx.x);
}

// ------------------------------------------------------------ clover field
// F_{mu nu}(x) = sum of (L - L^{-1}) over the four leaves at x; each leaf is a
// neighbouring plaquette carried to x:
//   L1 = P(x),  L2 = U_mu(x-mu)^{-1} P(x-mu) U_mu(x-mu),
//   L4 = U_nu(x-nu)^{-1} P(x-nu) U_nu(x-nu),
//   L3 = W^{-1} P(x-mu-nu) W with W = U_mu(x-mu-nu) U_nu(x-nu),
// so F = D(x) + the three carried D's.  Stored times a complex scale.
template <typename T>
__device__ __forceinline__ void k_clover_rot_body(Geo g, const typename vec2_of<T>::type* __restrict__ U,
                                                    const typename vec2_of<T>::type* __restrict__ Ui,
                                                    const typename vec2_of<T>::type* __restrict__ Dq,
                                                    typename vec2_of<T>::type* __restrict__ F,
                                                    double sre, double sim, int vb) {
  const int p = vb % 6, mu = plane_mu(p), nu = plane_nu(p);
  const int s = (vb / 6) * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int x[4];
  site_coords(g, s, x);
  const int xmm = hop(g, s, x, mu, -1), xmn = hop(g, s, x, nu, -1);
  const int xmm_mn = hop2(g, s, x, mu, -1, nu, -1);
  Work<T, 4> ws(0);
  mat<T>&acc = ws[0], &w = ws[1], &d = ws[2], &t = ws[3];
  load(acc, Dq, p, s, g.V);
  // L2 = U_mu(x-mu)^{-1} D(x-mu) U_mu(x-mu)
  load_inv(w, U, Ui, mu, xmm, g.V);
  load(d, Dq, p, xmm, g.V);
  mul(t, w, d);
  load(w, U, mu, xmm, g.V);
  mul_acc<+1>(acc, t, w);
  // L3 + L4 = U_nu(x-nu)^{-1} [D(x-nu) + U_mu(x-mu-nu)^{-1} D(x-mu-nu) U_mu(x-mu-nu)] U_nu(x-nu)
  load_inv(w, U, Ui, mu, xmm_mn, g.V);
  load(d, Dq, p, xmm_mn, g.V);
  mul(t, w, d);
  load(w, U, mu, xmm_mn, g.V);
  load(d, Dq, p, xmn, g.V);
  mul_acc<+1>(d, t, w);
  load_inv(w, U, Ui, nu, xmn, g.V);
  mul(t, w, d);
  load(w, U, nu, xmn, g.V);
  mul_acc<+1>(acc, t, w);
  cx<T> sc = {(T)sre, (T)sim};
#pragma unroll
  for (int k = 0; k < 9; ++k) acc.e[k] = cmul(acc.e[k], sc);
  store(F, p, s, g.V, acc);
}
template <typename T>
__global__ void __launch_bounds__(TUNE_MAX_BLOCK) k_clover_rot(Geo g, const typename vec2_of<T>::type* __restrict__ U,
                                                    const typename vec2_of<T>::type* __restrict__ Ui,
                                                    const typename vec2_of<T>::type* __restrict__ Dq,
                                                    typename vec2_of<T>::type* __restrict__ F,
                                                    double sre, double sim) {
  k_clover_rot_body<T>(g, U, Ui, Dq, F, sre, sim, blockIdx.x);
}

// ----------------------------------------------------- plaquette drift
// Contributions of the plaquette (x, p) to its four links, into
// C[4p + slot]: slot 0 U_mu(x), 1 U_nu(x), 2 U_nu(x+mu), 3 U_mu(x+nu).
// With theta the work has two stages: a handles corners c0..c2 (G0 + G1^ +
// G2^ and the slot 0 / slot 2 partials, parked in C); b adds corner c3, forms
// K and completes the four slots.  In FP64 (36 registers per matrix) the
// stages run as two kernels with the partial G^ parked in Gq, so neither
// spills; in FP32 one kernel runs both.
template <typename T>
__device__ __forceinline__ void k_plaq_force_wilson_body(Geo g, const typename vec2_of<T>::type* __restrict__ U,
                                                           const typename vec2_of<T>::type* __restrict__ Ui,
                                                           const typename vec2_of<T>::type* __restrict__ Dq,
                                                           typename vec2_of<T>::type* C, T beta6, int vb) {
  const int p = vb % 6, mu = plane_mu(p), nu = plane_nu(p);
  const int s = (vb / 6) * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  Work<T, 4> ws(0);
  mat<T>&D = ws[0], &M = ws[1], &t = ws[2], &a = ws[3];
  load(D, Dq, p, s, g.V);
  scaled(M, -beta6, D);
  store(C, 4 * p + 0, s, g.V, M);
  load_inv(a, U, Ui, mu, s, g.V);
  mul(t, a, M);
  load(a, U, mu, s, g.V);
  mul(M, t, a);
  store(C, 4 * p + 2, s, g.V, M);
  scaled(M, beta6, D);
  store(C, 4 * p + 1, s, g.V, M);
  load_inv(a, U, Ui, nu, s, g.V);
  mul(t, a, M);
  load(a, U, nu, s, g.V);
  mul(M, t, a);
  store(C, 4 * p + 3, s, g.V, M);
}
template <typename T>
__global__ void __launch_bounds__(TUNE_MAX_BLOCK) k_plaq_force_wilson(Geo g, const typename vec2_of<T>::type* __restrict__ U,
                                                           const typename vec2_of<T>::type* __restrict__ Ui,
                                                           const typename vec2_of<T>::type* __restrict__ Dq,
                                                           typename vec2_of<T>::type* C, T beta6) {
  k_plaq_force_wilson_body<T>(g, U, Ui, Dq, C, beta6, blockIdx.x);
}

// Corners c0..c2: G^ (partial) into Gh, slot 0 and slot 2 partials into C.
template <typename T>
__device__ __forceinline__ void force_stage_a(mat<T>& Gh, const Geo& g, int s, const int x[4], int p,
                                              const typename vec2_of<T>::type* __restrict__ U,
                                              const typename vec2_of<T>::type* __restrict__ Ui,
                                              const typename vec2_of<T>::type* __restrict__ Dq,
                                              const typename vec2_of<T>::type* __restrict__ F,
                                              typename vec2_of<T>::type* C, T beta6) {
  const int mu = plane_mu(p), nu = plane_nu(p), pc = 5 - p;
  const unsigned long long m = (p == 1 || p == 4) ? 0x8000000000000000ull : 0ull;
  const int c1 = hop(g, s, x, mu, 1);
  Work<T, 4> ws(1);  // slot 0 holds Gh
  mat<T>&D = ws[0], &M = ws[1], &t = ws[2], &q = ws[3];
  load(D, Dq, p, s, g.V);
  // corner c0: slot 0 partial = [D, G0] - (beta/6) D
  load_signed(Gh, F, pc, s, g.V, m);
  scaled(M, -beta6, D);
  commutator_acc(M, D, Gh);
  store(C, 4 * p + 0, s, g.V, M);
  // corner c1: G1^ = a G1 a^{-1}; slot 2 partial (c0 frame) = slot 0 partial + [D, G1^]
  load_signed(t, F, pc, c1, g.V, m);
  load(q, U, mu, s, g.V);
  mul(D, q, t);  // a G1 (D is re-read below)
  load_inv(q, U, Ui, mu, s, g.V);
  mul(t, D, q);  // G1^
#pragma unroll
  for (int k = 0; k < 9; ++k) Gh.e[k] = cadd(Gh.e[k], t.e[k]);
  load(D, Dq, p, s, g.V);
  commutator_acc(M, D, t);
  store(C, 4 * p + 2, s, g.V, M);
  // corner c2: G2^ = (ab) G2 (ab)^{-1}, with (ab)^{-1} = adj(ab) = adj(b) adj(a)
  // (the inverses used everywhere are adjugates: det U = 1 by the re-projection)
  load(M, U, mu, s, g.V);
  load(q, U, nu, c1, g.V);
  mul(D, M, q);  // ab
  load_signed(q, F, pc, hop(g, c1, x, nu, 1), g.V, m);
  mul(t, D, q);  // ab G2
  adj(M, D);     // (ab)^{-1}
  mul_acc<+1>(Gh, t, M);
}

// Corner c3, K, and the four slots completed; Gh holds the stage-a sum.
template <typename T>
__device__ __forceinline__ void force_stage_b(mat<T>& Gh, const Geo& g, int s, const int x[4], int p,
                                              const typename vec2_of<T>::type* __restrict__ U,
                                              const typename vec2_of<T>::type* __restrict__ Ui,
                                              const typename vec2_of<T>::type* __restrict__ Pq,
                                              const typename vec2_of<T>::type* __restrict__ Dq,
                                              const typename vec2_of<T>::type* __restrict__ F,
                                              typename vec2_of<T>::type* C, T beta6) {
  const int mu = plane_mu(p), nu = plane_nu(p), pc = 5 - p;
  const unsigned long long m = (p == 1 || p == 4) ? 0x8000000000000000ull : 0ull;
  const int c3 = hop(g, s, x, nu, 1);
  Work<T, 4> ws(1);  // slot 0 holds Gh
  mat<T>&D = ws[0], &M = ws[1], &t = ws[2], &q = ws[3];
  // corner c3: G3r = u G3 u^{-1}; slot 3 partial = [D, G3r] + (beta/6) D
  load_signed(q, F, pc, c3, g.V, m);
  load(M, U, nu, s, g.V);
  mul(t, M, q);
  load_inv(M, U, Ui, nu, s, g.V);
  mul(q, t, M);
  load(D, Dq, p, s, g.V);
  scaled(M, beta6, D);
  commutator_acc(M, D, q);
  store(C, 4 * p + 3, s, g.V, M);
  // G^ += P G3r P^{-1}, with P^{-1} = P - D formed in place
  mat<T>& P = M;
  load(P, Pq, p, s, g.V);
  mul(t, P, q);
#pragma unroll
  for (int k = 0; k < 9; ++k) P.e[k] = csub(P.e[k], D.e[k]);  // P^{-1}
  mul_acc<+1>(Gh, t, P);
  // K = P^{-1} G^ + G^ P
  mat<T>& K = q;
  mul(K, P, Gh);
#pragma unroll
  for (int k = 0; k < 9; ++k) P.e[k] = cadd(P.e[k], D.e[k]);  // P again
  mul_acc<+1>(K, Gh, P);
  // slot 1: -K + (beta/6) D
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    M.e[k].re = fma(beta6, D.e[k].re, -K.e[k].re);
    M.e[k].im = fma(beta6, D.e[k].im, -K.e[k].im);
  }
  store(C, 4 * p + 1, s, g.V, M);
  // slot 0: K + partial
  load_rw(M, C, 4 * p + 0, s, g.V);
#pragma unroll
  for (int k = 0; k < 9; ++k) M.e[k] = cadd(M.e[k], K.e[k]);
  store(C, 4 * p + 0, s, g.V, M);
  // slot 2: a^{-1} (K + partial) a
  load_rw(M, C, 4 * p + 2, s, g.V);
#pragma unroll
  for (int k = 0; k < 9; ++k) M.e[k] = cadd(M.e[k], K.e[k]);
  load_inv(Gh, U, Ui, mu, s, g.V);
  mul(t, Gh, M);
  load(Gh, U, mu, s, g.V);
  mul(M, t, Gh);
  store(C, 4 * p + 2, s, g.V, M);
  // slot 3: u^{-1} (-K + partial) u
  load_rw(M, C, 4 * p + 3, s, g.V);
#pragma unroll
  for (int k = 0; k < 9; ++k) M.e[k] = csub(M.e[k], K.e[k]);
  load_inv(Gh, U, Ui, nu, s, g.V);
  mul(t, Gh, M);
  load(Gh, U, nu, s, g.V);
  mul(M, t, Gh);
  store(C, 4 * p + 3, s, g.V, M);
}

// Split form (FP64): stage a, G^ parked in Gq, stage b.  Gq is not a buffer
// of its own: the partial of plaquette (p, s) sits in plane 4p + 1 of C (Gq
// points at plane 1 of C, so Gq plane GQ_PLANE * p is C plane 4p + 1), the
// slot-1 contribution of that same plaquette, which only stage b writes, and
// only after the same thread has read the partial back.  Gq and C may alias,
// so neither carries __restrict__ and stage b reads Gq with a plain load.
const int GQ_PLANE = 4;
template <typename T>
__device__ __forceinline__ void k_plaq_force_a_body(Geo g, const typename vec2_of<T>::type* __restrict__ U,
                                                      const typename vec2_of<T>::type* __restrict__ Ui,
                                                      const typename vec2_of<T>::type* __restrict__ Dq,
                                                      const typename vec2_of<T>::type* __restrict__ F,
                                                      typename vec2_of<T>::type* Gq,
                                                      typename vec2_of<T>::type* C, T beta6, int vb) {
  const int p = vb % 6;
  const int s = (vb / 6) * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int x[4];
  site_coords(g, s, x);
  Work<T, 1> wg(0);
  mat<T>& Gh = wg[0];
  force_stage_a(Gh, g, s, x, p, U, Ui, Dq, F, C, beta6);
  store(Gq, GQ_PLANE * p, s, g.V, Gh);
}
template <typename T>
__global__ void __launch_bounds__(TUNE_MAX_BLOCK) k_plaq_force_a(Geo g, const typename vec2_of<T>::type* __restrict__ U,
                                                      const typename vec2_of<T>::type* __restrict__ Ui,
                                                      const typename vec2_of<T>::type* __restrict__ Dq,
                                                      const typename vec2_of<T>::type* __restrict__ F,
                                                      typename vec2_of<T>::type* Gq,
                                                      typename vec2_of<T>::type* C, T beta6) {
  k_plaq_force_a_body<T>(g, U, Ui, Dq, F, Gq, C, beta6, blockIdx.x);
}
template <typename T>
__device__ __forceinline__ void k_plaq_force_b_body(Geo g, const typename vec2_of<T>::type* __restrict__ U,
                                                      const typename vec2_of<T>::type* __restrict__ Ui,
                                                      const typename vec2_of<T>::type* __restrict__ Pq,
                                                      const typename vec2_of<T>::type* __restrict__ Dq,
                                                      const typename vec2_of<T>::type* __restrict__ F,
                                                      const typename vec2_of<T>::type* Gq,
                                                      typename vec2_of<T>::type* C, T beta6, int vb) {
  const int p = vb % 6;
  const int s = (vb / 6) * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int x[4];
  site_coords(g, s, x);
  Work<T, 1> wg(0);
  mat<T>& Gh = wg[0];
  load_rw(Gh, Gq, GQ_PLANE * p, s, g.V);  // before stage b writes slot 1 of (p, s) over it
  force_stage_b(Gh, g, s, x, p, U, Ui, Pq, Dq, F, C, beta6);
}
template <typename T>
__global__ void __launch_bounds__(TUNE_MAX_BLOCK) k_plaq_force_b(Geo g, const typename vec2_of<T>::type* __restrict__ U,
                                                      const typename vec2_of<T>::type* __restrict__ Ui,
                                                      const typename vec2_of<T>::type* __restrict__ Pq,
                                                      const typename vec2_of<T>::type* __restrict__ Dq,
                                                      const typename vec2_of<T>::type* __restrict__ F,
                                                      const typename vec2_of<T>::type* Gq,
                                                      typename vec2_of<T>::type* C, T beta6) {
  k_plaq_force_b_body<T>(g, U, Ui, Pq, Dq, F, Gq, C, beta6, blockIdx.x);
}
// Fused form (FP32, which needs no split to stay in registers).
template <typename T>
__device__ __forceinline__ void k_plaq_force_ab_body(Geo g, const typename vec2_of<T>::type* __restrict__ U,
                                                       const typename vec2_of<T>::type* __restrict__ Ui,
                                                       const typename vec2_of<T>::type* __restrict__ Pq,
                                                       const typename vec2_of<T>::type* __restrict__ Dq,
                                                       const typename vec2_of<T>::type* __restrict__ F,
                                                       typename vec2_of<T>::type* C, T beta6, int vb) {
  const int p = vb % 6;
  const int s = (vb / 6) * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int x[4];
  site_coords(g, s, x);
  Work<T, 1> wg(0);
  mat<T>& Gh = wg[0];
  force_stage_a(Gh, g, s, x, p, U, Ui, Dq, F, C, beta6);
  force_stage_b(Gh, g, s, x, p, U, Ui, Pq, Dq, F, C, beta6);
}
// Left to itself the compiler gives the fused FP32 force 228 registers, two
// blocks of 128 per SM; capped at 160 it keeps three (a few hundred bytes of
// spills, served by L1): 1.27 -> 1.04 ms per 32^4 step on GB300 (caps of 152
// and 168: 1.08 and 1.10 ms; 128: 1.50 ms; the split a / b form in FP32:
// 1.57 ms).  __maxnreg__ excludes __launch_bounds__; at 160 registers every
// tuned block size up to TUNE_MAX_BLOCK still launches.
const int FORCE_AB_MAXNREG = 160;
template <typename T>
__global__ void __maxnreg__(FORCE_AB_MAXNREG) k_plaq_force_ab(Geo g, const typename vec2_of<T>::type* __restrict__ U,
                                                       const typename vec2_of<T>::type* __restrict__ Ui,
                                                       const typename vec2_of<T>::type* __restrict__ Pq,
                                                       const typename vec2_of<T>::type* __restrict__ Dq,
                                                       const typename vec2_of<T>::type* __restrict__ F,
                                                       typename vec2_of<T>::type* C, T beta6) {
  k_plaq_force_ab_body<T>(g, U, Ui, Pq, Dq, F, C, beta6, blockIdx.x);
}

// Noise matrix sum_a eta_a lambda_a (Hermitian) into the imaginary part of A,
// scaled by sqrt(eps): A += i sqrt(eps) H.
template <typename R>
__device__ __forceinline__ void add_noise(mat<R>& A, const R* e, R se) {
  const R r3 = (R)0.57735026918962576451;  // 1/sqrt(3)
  R h00 = e[2] + e[7] * r3, h11 = -e[2] + e[7] * r3, h22 = (R)-2 * e[7] * r3;
  // i * (hr + i hi) = -hi + i hr
  A.e[0].im = fma(se, h00, A.e[0].im);
  A.e[4].im = fma(se, h11, A.e[4].im);
  A.e[8].im = fma(se, h22, A.e[8].im);
  // H01 = e1 - i e2, H10 = e1 + i e2 ; H02 = e4 - i e5 ; H12 = e6 - i e7
  A.e[1].re = fma(se, e[1], A.e[1].re);  A.e[1].im = fma(se, e[0], A.e[1].im);
  A.e[3].re = fma(-se, e[1], A.e[3].re); A.e[3].im = fma(se, e[0], A.e[3].im);
  A.e[2].re = fma(se, e[4], A.e[2].re);  A.e[2].im = fma(se, e[3], A.e[2].im);
  A.e[6].re = fma(-se, e[4], A.e[6].re); A.e[6].im = fma(se, e[3], A.e[6].im);
  A.e[5].re = fma(se, e[6], A.e[5].re);  A.e[5].im = fma(se, e[5], A.e[5].im);
  A.e[7].re = fma(-se, e[6], A.e[7].re); A.e[7].im = fma(se, e[5], A.e[7].im);
}

// A = 2 eps (X - Tr X / 3) + i sqrt(eps) sqrt(2) g_a lambda_a in the real type R.
template <typename R>
__device__ __forceinline__ void exponent(mat<R>& A, const R* g, R eps, R sqrt_eps) {
  const R tr_re = (A.e[0].re + A.e[4].re + A.e[8].re) * (R)(1.0 / 3.0);
  const R tr_im = (A.e[0].im + A.e[4].im + A.e[8].im) * (R)(1.0 / 3.0);
  A.e[0].re -= tr_re; A.e[4].re -= tr_re; A.e[8].re -= tr_re;
  A.e[0].im -= tr_im; A.e[4].im -= tr_im; A.e[8].im -= tr_im;
  const R e2 = (R)2 * eps;
#pragma unroll
  for (int k = 0; k < 9; ++k) { A.e[k].re *= e2; A.e[k].im *= e2; }
  add_noise(A, g, sqrt_eps * (R)1.41421356237309504880);  // eta = sqrt(2) * normal
}

// ------------------------------------------------ gather + exponential update
// X of link (x, mu) = sum of its six plaquette contributions: for nu != mu,
// mu < nu: slot 0 of (x, p) and slot 3 of (x - nu, p); mu > nu: slot 1 of
// (x, p) and slot 2 of (x - nu, p), p the plane of (mu, nu).
template <typename T, int MODE>
__device__ __forceinline__ void k_update_gather_body(Geo g, const typename vec2_of<T>::type* __restrict__ U,
                                                       const typename vec2_of<T>::type* __restrict__ C,
                                                       typename vec2_of<T>::type* __restrict__ out,
                                                       UpdArgs a, int vb) {
  const int MU = vb % 4;
  const int s_raw = (vb / 4) * blockDim.x + threadIdx.x;
  if (MODE != MODE_DRIFTMAX && s_raw >= g.V) return;
  // the max pass keeps whole warps alive for its shuffle: lanes past the end
  // redo the last site (same value, so the max is unchanged)
  const int s = s_raw < g.V ? s_raw : g.V - 1;
  int x[4];
  site_coords(g, s, x);
  Work<T, 2> ws(0);
  mat<T>&X = ws[0], &t = ws[1];
  if (MODE == MODE_UPDATE_X) {
    load(X, C, MU, s, g.V);  // the drift stored by the MODE_DRIFTMAX pass
  } else {
    set_zero(X);
#pragma unroll
    for (int nu = 0; nu < 4; ++nu) {
      if (nu == MU) continue;
      const int p = MU < nu ? plane_index(MU, nu) : plane_index(nu, MU);
      const int sl_here = MU < nu ? 0 : 1, sl_back = MU < nu ? 3 : 2;
      load(t, C, 4 * p + sl_here, s, g.V);
#pragma unroll
      for (int k = 0; k < 9; ++k) X.e[k] = cadd(X.e[k], t.e[k]);
      load(t, C, 4 * p + sl_back, hop(g, s, x, nu, -1), g.V);
#pragma unroll
      for (int k = 0; k < 9; ++k) X.e[k] = cadd(X.e[k], t.e[k]);
    }
  }
  if (MODE == MODE_DRIFT) {
    store(out, MU, s, g.V, X);
    return;
  }
  if (MODE == MODE_DRIFTMAX) {
    if (s_raw < g.V) store(out, MU, s, g.V, X);
    // |K|^2 = sum_a |Tr(lambda_a X)|^2 = 2 |X - Tr X / 3|_F^2 (Tr l_a l_b = 2 delta_ab)
    mat<double> Xd;
    convert(Xd, X);
    const double tr_re = (Xd.e[0].re + Xd.e[4].re + Xd.e[8].re) * (1.0 / 3.0);
    const double tr_im = (Xd.e[0].im + Xd.e[4].im + Xd.e[8].im) * (1.0 / 3.0);
    Xd.e[0].re -= tr_re; Xd.e[4].re -= tr_re; Xd.e[8].re -= tr_re;
    Xd.e[0].im -= tr_im; Xd.e[4].im -= tr_im; Xd.e[8].im -= tr_im;
    unsigned long long k2 = (unsigned long long)__double_as_longlong(2.0 * norm2(Xd));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long v = __shfl_xor_sync(0xffffffffu, k2, o);
      k2 = v > k2 ? v : k2;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(&a.sd->kmax2_bits, k2);
    return;
  }
  // exponent A = 2 eps (X - Tr X/3) + i sqrt(eps) eta_a lambda_a; exp in FP64.
  // The FP64 form builds A in FP64; the FP32-storage form builds it in FP32
  // (X and the noise carry FP32 information only) and widens it for the exp.
  const uint32_t step = a.sd->step;
  const double eps = a.adaptive ? a.sd->eps_n : a.eps;
  const double sqrt_eps = a.adaptive ? a.sd->sqrt_eps_n : a.sqrt_eps;
  if constexpr (std::is_same<T, df64>::value) {
    // DF64: the noise, the exponent, the exponential (its scalar recurrences
    // too), the update and the re-projection in double-float; no FP64
    // instruction on the common path
    df64 eta[8];
    normals_df64<4>(eta, a.seed, step, (uint32_t)s, (uint32_t)MU, STREAM_CL);
    exponent<df64>(X, eta, df64(eps), df64(sqrt_eps));
    // three workspace slots: E overwrites X (entry by entry), the link U
    // takes the slot of X^2 once E is formed
    Work<df64, 1> wu(2);
    mat<df64>&E = X, &Ul = t, &Un = wu[0];
    expm_traceless_df(E, X, t);
    load(Ul, U, MU, s, g.V);
    mul_df_compact(Un, E, Ul);
    const cx<df64> z = det_inv_cuberoot_df(det(Un));
#pragma unroll 1
    for (int k = 0; k < 9; ++k) Un.e[k] = cmul(Un.e[k], z);  // rolled: Un is in the workspace; saves code
    store(out, MU, s, g.V, Un);
    return;
  }
  mat<double> A;
  float rA = -1.f;
  if (sizeof(T) == 8) {
    double eta[8];
    normals_f64<4>(eta, a.seed, step, (uint32_t)s, (uint32_t)MU, STREAM_CL);
    convert(A, X);
    exponent<double>(A, eta, eps, sqrt_eps);
  } else {
    float ef[8];
    normals_f32<4>(ef, a.seed, step, (uint32_t)s, (uint32_t)MU, STREAM_CL);
    mat<float> Af;
    convert(Af, X);
    exponent<float>(Af, ef, (float)eps, (float)sqrt_eps);
    rA = sqrtf(norm2(Af));
    convert(A, Af);
  }
  mat<double> E;
  expm_traceless(E, A, rA, taylor_tol<T>());
  mat<T> Et, Ul, Un;
  convert(Et, E);
  load(Ul, U, MU, s, g.V);
  mul(Un, Et, Ul);
  mat<double> Und;
  convert(Und, Un);
  cx<double> z = det_inv_cuberoot(det(Und));
  cx<T> zt = {cvt<T>(z.re), cvt<T>(z.im)};
#pragma unroll
  for (int k = 0; k < 9; ++k) Un.e[k] = cmul(Un.e[k], zt);
  store(out, MU, s, g.V, Un);
}
template <typename T, int MODE>
__global__ void __launch_bounds__(TUNE_MAX_BLOCK) k_update_gather(Geo g, const typename vec2_of<T>::type* __restrict__ U,
                                                       const typename vec2_of<T>::type* __restrict__ C,
                                                       typename vec2_of<T>::type* __restrict__ out,
                                                       UpdArgs a) {
  k_update_gather_body<T, MODE>(g, U, C, out, a, blockIdx.x);
}

}  // namespace clgc
