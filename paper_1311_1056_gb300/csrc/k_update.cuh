// k_update.cuh -- the CL step: Wilson staple drift + clover theta drift,
// Philox noise, FP64 exponential update and det re-projection, one thread
// per link.
//
// Action (Sec. 5, eq. "eq:st"): S = S_W - i theta sum_x q_L(x) with the
// Wilson action continued holomorphically (U^+ -> U^{-1}) and
//   q_L(x) = kappa [Tr F01 F23 - Tr F02 F13 + Tr F03 F12](x),  kappa = -1/(256 pi^2),
// where F_{mu nu}(x) = sum over the four clover leaves L at x of (L - L^{-1})
// (this is the paper's signed eps-tilde sum regrouped by plane).
//
// Drift matrix X_S of link l = (x, mu), defined by D_a S = i Tr(lambda_a X_S)
// with D_a the left derivative U -> exp(i a lambda_a) U.  For each of the six
// plaquettes through l written as P = U_l w1 w2 w3 (sgn = +1: the one based
// at x in the (mu, nu) plane, sgn = -1: the one based at x - nu), with corners
// c0 = x, c1 = x+mu, c2, c3 in the order of the loop:
//   Wilson:  X += -(beta/6) (U_l W - W^{-1} U_l^{-1}),  W = w1 w2 w3
//   theta :  X += sigma [U_l T1 + T2 U_l^{-1}] with G_k = F^(c_k) of the
//            complementary plane (F^ = -i theta kappa F, done by the clover
//            kernel) and
//     T1 = W G0 + G1 W + w1 G2 w2 w3 + w1 w2 G3 w3
//     T2 = G0 W^{-1} + W^{-1} G1 + (w2 w3)^{-1} G2 w1^{-1} + w3^{-1} G3 (w1 w2)^{-1}
//   sigma = sgn * (pair sign: +1, -1, +1 for 01|23, 02|13, 03|12)
//               * (+1 if mu < nu, else -1: F_{nu mu} = -F_{mu nu}).
// T1 and T2 are the product rule for the leaf (and its inverse) at each
// corner with the dual field inserted at that corner.
//
// Update (the CL step of the method, Sec. 2 and its refs):
//   K_a = -D_a S,  A = i lambda_a (eps K_a + sqrt(eps) eta_a)
//     = 2 eps (X_S - Tr X_S / 3) + i sqrt(eps) eta_a lambda_a,  <eta_a eta_b> = 2 delta_ab,
//   U' = exp(A) U  (exp in FP64),  U' <- U' det(U')^{-1/3}  (FP64 factor).
#pragma once
#include "expm.cuh"
#include "lattice.cuh"
#include "philox.cuh"
#include "su3.cuh"

namespace clgc {

enum { MODE_UPDATE = 0, MODE_DRIFT = 1 };

struct UpdArgs {
  double beta, eps, sqrt_eps;
  uint64_t seed;
  uint32_t step;
};

// Raw link or its inverse (adjugate), whichever the loop needs.
template <typename T>
__device__ __forceinline__ void load_link(mat<T>& m, const typename vec2_of<T>::type* U, int mu,
                                          int s, int V, bool inverse) {
  if (inverse) {
    mat<T> t;
    load(t, U, mu, s, V);
    adj(m, t);
  } else {
    load(m, U, mu, s, V);
  }
}

// Sign flip on the integer pipe (no FP64 instruction): every theta term
// contains exactly one factor G, so sigma = -1 is applied by negating G.
__device__ __forceinline__ double flip(double x, unsigned long long m) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)m);
}
__device__ __forceinline__ float flip(float x, unsigned long long m) {
  return __int_as_float(__float_as_int(x) ^ (int)(m >> 32));
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

// The products are regrouped to share factors (a23 = w2 w3, i23 = a23^{-1}):
//   T1 = w1 Y + G1 W,       Y = a23 G0 + G2 a23 + w2 (G3 w3)
//   T2 = Z w1^{-1} + W^{-1} G1,  Z = G0 i23 + i23 G2 + (w3^{-1} G3) w2^{-1}
// so that U_l T1 + T2 U_l^{-1} is accumulated as S1 += T1, S2 += T2 and
// X = U_l S1 + S2 U_l^{-1} at the end (14 matrix products per plaquette).
// The six plaquettes run as a loop (not unrolled): one body's working set
// fits the register file; unrolled, the FP64 form spills tens of KB.
template <typename T, bool THETA>
__device__ __forceinline__ void drift_matrix(mat<T>& X, mat<T>& Ul, const Geo& g, int s,
                                             const int x[4], const int mu,
                                             const typename vec2_of<T>::type* __restrict__ U,
                                             const typename vec2_of<T>::type* __restrict__ F,
                                             T beta6) {
  mat<T> S1, S2;
  set_zero(S1);
  set_zero(S2);
  const int c1 = hop(g, s, x, mu, +1);
#pragma unroll 1
  for (int pl = 0; pl < 6; ++pl) {
    const int nu = (pl >> 1) + ((pl >> 1) >= mu ? 1 : 0);
    const int sgn = (pl & 1) ? -1 : 1;
    const int p = mu < nu ? plane_index(mu, nu) : plane_index(nu, mu);
    const int pc = 5 - p;
    const int sigma = sgn * ((p == 1 || p == 4) ? -1 : 1) * (mu < nu ? 1 : -1);
    const unsigned long long m = sigma < 0 ? 0x8000000000000000ull : 0ull;
    const int c2 = hop(g, c1, x, nu, sgn);
    const int c3 = hop(g, s, x, nu, sgn);
    // loop from x: U_l, w1 to c2, w2 to c3, w3 back to x
    //   sgn = +1: w1 = U_nu(x+mu), w2 = U_mu(x+nu)^{-1}, w3 = U_nu(x)^{-1}
    //   sgn = -1: w1 = U_nu(x+mu-nu)^{-1}, w2 = U_mu(x-nu)^{-1}, w3 = U_nu(x-nu)
    const int w1site = sgn > 0 ? c1 : c2, w3site = sgn > 0 ? s : c3;
    mat<T> a23, i23, Y, G, t;
    {
      mat<T> w2, w3;
      load_link(w2, U, mu, c3, g.V, true);
      load_link(w3, U, nu, w3site, g.V, sgn > 0);
      mul(a23, w2, w3);
      if (THETA) {
        load_signed(G, F, pc, s, g.V, m);
        mul(Y, a23, G);
        load_signed(G, F, pc, c2, g.V, m);
        mul_acc<+1>(Y, G, a23);
        load_signed(G, F, pc, c3, g.V, m);
        mul(t, G, w3);
        mul_acc<+1>(Y, w2, t);
      }
    }
    {
      mat<T> w1, W, Wi;
      load_link(w1, U, nu, w1site, g.V, sgn < 0);
      mul(W, w1, a23);
      if (THETA) adj(i23, a23);
      if (THETA) mul_acc<+1>(S1, w1, Y);
      adj(Wi, W);
      axpy<-1>(S1, beta6, W);
      axpy<+1>(S2, beta6, Wi);
      if (THETA) {
        load_signed(G, F, pc, c1, g.V, m);
        mul_acc<+1>(S1, G, W);
        mul_acc<+1>(S2, Wi, G);
      }
    }
    if (THETA) {
      mat<T>& Z = Y;
      load_signed(G, F, pc, s, g.V, m);
      mul(Z, G, i23);
      load_signed(G, F, pc, c2, g.V, m);
      mul_acc<+1>(Z, i23, G);
      {
        mat<T> w3i;
        load_link(w3i, U, nu, w3site, g.V, sgn < 0);
        load_signed(G, F, pc, c3, g.V, m);
        mul(t, w3i, G);
      }
      {
        mat<T> w2i;
        load_link(w2i, U, mu, c3, g.V, false);
        mul_acc<+1>(Z, t, w2i);
      }
      mat<T>& w1i = t;
      load_link(w1i, U, nu, w1site, g.V, sgn > 0);
      mul_acc<+1>(S2, Z, w1i);
    }
  }
  load(Ul, U, mu, s, g.V);
  mat<T> Uli;
  adj(Uli, Ul);
  mul(X, Ul, S1);
  mul_acc<+1>(X, S2, Uli);
}

// Noise matrix sum_a eta_a lambda_a (Hermitian) into the imaginary part of A,
// scaled by sqrt(eps): A += i sqrt(eps) H.
__device__ __forceinline__ void add_noise(mat<double>& A, const double* e, double se) {
  const double r3 = 0.57735026918962576451;  // 1/sqrt(3)
  double h00 = e[2] + e[7] * r3, h11 = -e[2] + e[7] * r3, h22 = -2.0 * e[7] * r3;
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

template <typename T, bool THETA, int MODE>
__device__ __forceinline__ void cl_link(const Geo& g, int s, const int MU,
                                        const typename vec2_of<T>::type* U,
                                        const typename vec2_of<T>::type* F,
                                        typename vec2_of<T>::type* out, const UpdArgs& a) {
  int x[4];
  site_coords(g, s, x);
  mat<T> X, Ul;
  drift_matrix<T, THETA>(X, Ul, g, s, x, MU, U, F, (T)(a.beta / 6.0));
  if (MODE == MODE_DRIFT) {
    store(out, MU, s, g.V, X);
    return;
  }
  // exponent A = 2 eps (X - Tr X/3) + i sqrt(eps) eta_a lambda_a, in FP64
  mat<double> A;
  convert(A, X);
  {
    double tr_re = (A.e[0].re + A.e[4].re + A.e[8].re) * (1.0 / 3.0);
    double tr_im = (A.e[0].im + A.e[4].im + A.e[8].im) * (1.0 / 3.0);
    A.e[0].re -= tr_re; A.e[4].re -= tr_re; A.e[8].re -= tr_re;
    A.e[0].im -= tr_im; A.e[4].im -= tr_im; A.e[8].im -= tr_im;
    const double e2 = 2.0 * a.eps;
#pragma unroll
    for (int k = 0; k < 9; ++k) { A.e[k].re *= e2; A.e[k].im *= e2; }
  }
  double eta[8];
  if (sizeof(T) == 8) {
    normals_f64<4>(eta, a.seed, a.step, (uint32_t)s, (uint32_t)MU, STREAM_CL);
  } else {
    float ef[8];
    normals_f32<4>(ef, a.seed, a.step, (uint32_t)s, (uint32_t)MU, STREAM_CL);
#pragma unroll
    for (int k = 0; k < 8; ++k) eta[k] = (double)ef[k];
  }
  add_noise(A, eta, a.sqrt_eps * 1.41421356237309504880);  // eta = sqrt(2) * normal
  mat<double> E;
  expm_traceless(E, A);
  mat<T> Et, Un;
  convert(Et, E);
  mul(Un, Et, Ul);
  mat<double> Und;
  convert(Und, Un);
  cx<double> z = det_inv_cuberoot(det(Und));
  cx<T> zt = {(T)z.re, (T)z.im};
#pragma unroll
  for (int k = 0; k < 9; ++k) Un.e[k] = cmul(Un.e[k], zt);
  store(out, MU, s, g.V, Un);
}

template <typename T, bool THETA, int MODE>
__global__ void __launch_bounds__(128) k_cl_update(Geo g, const typename vec2_of<T>::type* __restrict__ U,
                                                   const typename vec2_of<T>::type* __restrict__ F,
                                                   typename vec2_of<T>::type* __restrict__ out,
                                                   UpdArgs a) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  cl_link<T, THETA, MODE>(g, s, (int)blockIdx.y, U, F, out, a);
}

}  // namespace clgc
