// pchain.cpp -- plain FP64 CPU oracle for the SU(2) Polyakov chain of
// arXiv:1311.1056 (Sec. 3 and Sec. 4): S = -(beta/2) Tr(U_1 U_2 ... U_N),
// complex beta, links in SL(2,C), complex Langevin with (adaptive) gauge
// cooling.
//
// TEST INFRASTRUCTURE ONLY: the independent checker of the CUDA chain
// kernel.  Only the tests, the smoke check and the CPU-baseline leg of the
// benchmark load it.  Nothing here is shared with the CUDA library.
//
// Literal on purpose: the drift of link k multiplies out the whole cyclic
// product U_k ... U_N U_1 ... U_{k-1} for every k and takes the three traces
// with the Pauli matrices one by one; exp is Taylor with scaling and
// squaring; the cooling gradient is the traced definition per generator.
// Pins: tests/test_oracle_pchain.py (finite differences of the action, the
// exact one-link cooling fixed point, gauge invariance, the exact answer
// I_2(beta)/I_1(beta) at real beta).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "oracle.h"

namespace {

using cd = std::complex<double>;
const cd I1(0.0, 1.0);

struct M2 {
  cd m[2][2];
};

M2 zero2() {
  M2 r;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) r.m[i][j] = 0.0;
  return r;
}
M2 ident2() {
  M2 r = zero2();
  r.m[0][0] = r.m[1][1] = 1.0;
  return r;
}
M2 mul(const M2& a, const M2& b) {
  M2 r;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) r.m[i][j] = a.m[i][0] * b.m[0][j] + a.m[i][1] * b.m[1][j];
  return r;
}
M2 add(const M2& a, const M2& b) {
  M2 r;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) r.m[i][j] = a.m[i][j] + b.m[i][j];
  return r;
}
M2 scale(const M2& a, cd s) {
  M2 r;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) r.m[i][j] = s * a.m[i][j];
  return r;
}
M2 dagger(const M2& a) {
  M2 r;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) r.m[i][j] = std::conj(a.m[j][i]);
  return r;
}
cd trace(const M2& a) { return a.m[0][0] + a.m[1][1]; }
cd det(const M2& a) { return a.m[0][0] * a.m[1][1] - a.m[0][1] * a.m[1][0]; }
M2 inverse(const M2& a) {  // adjugate / det
  cd d = det(a);
  M2 r;
  r.m[0][0] = a.m[1][1] / d;
  r.m[1][1] = a.m[0][0] / d;
  r.m[0][1] = -a.m[0][1] / d;
  r.m[1][0] = -a.m[1][0] / d;
  return r;
}
double normF(const M2& a) {
  double s = 0.0;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) s += std::norm(a.m[i][j]);
  return std::sqrt(s);
}

// Pauli matrices sigma_1..3 (Tr sigma_a sigma_b = 2 delta_ab).
M2 pauli(int a) {
  M2 r = zero2();
  if (a == 1) r.m[0][1] = r.m[1][0] = 1.0;
  if (a == 2) {
    r.m[0][1] = -I1;
    r.m[1][0] = I1;
  }
  if (a == 3) {
    r.m[0][0] = 1.0;
    r.m[1][1] = -1.0;
  }
  return r;
}

// exp by Taylor series with scaling and squaring.
M2 expm(const M2& a) {
  double n = normF(a);
  int sq = 0;
  while (n > 0.5 && sq < 1100) {  // the bound only stops an infinite norm
    n *= 0.5;
    ++sq;
  }
  M2 x = scale(a, std::ldexp(1.0, -sq));
  M2 term = ident2(), sum = ident2();
  for (int k = 1; k <= 30; ++k) {
    term = scale(mul(term, x), 1.0 / k);
    sum = add(sum, term);
  }
  for (int i = 0; i < sq; ++i) sum = mul(sum, sum);
  return sum;
}

M2 load(const double* p) {
  M2 r;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) r.m[i][j] = cd(p[4 * i + 2 * j], p[4 * i + 2 * j + 1]);
  return r;
}
void store(const M2& a, double* p) {
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      p[4 * i + 2 * j] = a.m[i][j].real();
      p[4 * i + 2 * j + 1] = a.m[i][j].imag();
    }
}

std::vector<M2> load_chain(int n, const double* U) {
  std::vector<M2> v(n);
  for (int k = 0; k < n; ++k) v[k] = load(U + 8 * k);
  return v;
}
void store_chain(const std::vector<M2>& v, double* U) {
  for (size_t k = 0; k < v.size(); ++k) store(v[k], U + 8 * k);
}

// U_k U_{k+1} ... U_{n-1} U_0 ... U_{k-1}
M2 cyclic_product(const std::vector<M2>& U, int k) {
  const int n = (int)U.size();
  M2 p = ident2();
  for (int j = 0; j < n; ++j) p = mul(p, U[(k + j) % n]);
  return p;
}

const uint32_t STREAM_PC_CL = 3, STREAM_PC_GAUGE = 4;

// K_a(k) = -D_a S, D_a S = d/dalpha S(e^{i alpha sigma_a} U_k) at alpha = 0
//        = -(beta/2) Tr(U_1..U_{k-1} i sigma_a U_k ... U_N) = -(i beta/2) Tr(sigma_a P_k).
void drift(const std::vector<M2>& U, cd beta, std::vector<cd>& K) {
  const int n = (int)U.size();
  K.assign(3 * (size_t)n, 0.0);
  for (int k = 0; k < n; ++k) {
    M2 P = cyclic_product(U, k);
    for (int a = 1; a <= 3; ++a) K[3 * k + a - 1] = I1 * beta / 2.0 * trace(mul(pauli(a), P));
  }
}

// f_ak = 2 Tr[sigma_a (U_k U_k^+ - U_{k-1}^+ U_{k-1})]  (eq. "eq:24" on the chain)
void gradient(const std::vector<M2>& U, std::vector<double>& f) {
  const int n = (int)U.size();
  f.assign(3 * (size_t)n, 0.0);
  for (int k = 0; k < n; ++k) {
    const M2& u = U[k];
    const M2& v = U[(k - 1 + n) % n];
    M2 G = add(mul(u, dagger(u)), scale(mul(dagger(v), v), -1.0));
    for (int a = 1; a <= 3; ++a) f[3 * k + a - 1] = (2.0 * trace(mul(pauli(a), G))).real();
  }
}

double unitarity_norm(const std::vector<M2>& U) {
  double s = 0.0;
  for (const M2& u : U) s += 0.5 * trace(mul(u, dagger(u))).real();
  return s / U.size();
}

// U_k <- Omega_k U_k Omega_{k+1}^{-1}, Omega_k = exp(-eps alpha_ad f_ak sigma_a)
void cool_sweep(std::vector<M2>& U, double eps, double alpha_ad) {
  const int n = (int)U.size();
  std::vector<double> f;
  gradient(U, f);
  std::vector<M2> Om(n);
  for (int k = 0; k < n; ++k) {
    M2 H = zero2();
    for (int a = 1; a <= 3; ++a) H = add(H, scale(pauli(a), -eps * alpha_ad * f[3 * k + a - 1]));
    Om[k] = expm(H);
  }
  std::vector<M2> V(n);
  for (int k = 0; k < n; ++k) V[k] = mul(mul(Om[k], U[k]), inverse(Om[(k + 1) % n]));
  U.swap(V);
}

// The stop rule of the SU(3) oracle (Sec. 4 reading), with D_1 = (1/2)<Tr U U^+>
// and D_2 = <|f_ak|>_{a,k} (or its RMS).
void cool(std::vector<M2>& U, const or_cool_params& p, or_cool_report& rep) {
  rep.sweeps = 0;
  rep.alpha_ad_last = 0.0;
  const int n = (int)U.size();
  double un_prev = 0.0;
  for (int k = 0;; ++k) {
    std::vector<double> f;
    gradient(U, f);
    double un = unitarity_norm(U);
    double sabs = 0.0, ssq = 0.0;
    for (double v : f) {
      sabs += std::fabs(v);
      ssq += v * v;
    }
    double D = 1.0;
    if (p.mode == OR_D1) D = un;
    if (p.mode == OR_D2_MEANABS) D = sabs / (3.0 * n);
    if (p.mode == OR_D2_RMS) D = std::sqrt(ssq / (3.0 * n));
    if (k == 0) rep.un_before = un;
    rep.un_after = un;
    bool stop;
    if (p.forced_sweeps >= 0) {
      stop = (k >= p.forced_sweeps);
    } else {
      stop = (k >= p.n_max);
      if (k >= p.n_min) {
        if (un - 1.0 < p.d_floor) stop = true;
        if (k >= 1 && (un_prev - un) < p.tol_rel * (un_prev - 1.0)) stop = true;
      }
    }
    if (D < p.d_guard) stop = true;
    if (stop) break;
    double alpha_ad = p.alpha / D;
    cool_sweep(U, p.eps, alpha_ad);
    rep.alpha_ad_last = alpha_ad;
    rep.sweeps++;
    un_prev = un;
  }
}

// One CL step, all links at once: U_k' = exp(i sigma_a (eps K_a + sqrt(eps) eta_a)) U_k,
// eta_a = sqrt(2) * normal (Philox stream 3, counter (k, step, 3 << 8, j)),
// then U' <- U' / det(U')^(1/2) (principal branch).
void cl_step(std::vector<M2>& U, cd beta, double eps, uint64_t seed, uint32_t step) {
  const int n = (int)U.size();
  std::vector<cd> K;
  drift(U, beta, K);
  std::vector<M2> V(n);
  for (int k = 0; k < n; ++k) {
    double g[4];
    or_normals(seed, step, (uint32_t)k, 0u, STREAM_PC_CL, 2, g);
    M2 A = zero2();
    for (int a = 1; a <= 3; ++a) {
      cd c = eps * K[3 * k + a - 1] + std::sqrt(eps) * std::sqrt(2.0) * g[a - 1];
      A = add(A, scale(pauli(a), I1 * c));
    }
    M2 W = mul(expm(A), U[k]);
    V[k] = scale(W, 1.0 / std::sqrt(det(W)));
  }
  U.swap(V);
}

}  // namespace

extern "C" {

void or_pauli(int a, double* out8) { store(pauli(a), out8); }

int or_pc_cold(int n, double* U) {
  if (n < 1 || !U) return -1;
  for (int k = 0; k < n; ++k) store(ident2(), U + 8 * k);
  return 0;
}

// U_k <- Om_k U_k Om_{k+1}^{-1}, Om_k = exp(i w_a sigma_a), w_a = i sigma g_a
// (g standard normal, Philox stream 4, counter (k, 0, 4 << 8, j)).
int or_pc_random_gauge(int n, uint64_t seed, double sigma, double* U) {
  if (n < 1 || !U) return -1;
  std::vector<M2> V = load_chain(n, U), Om(n);
  for (int k = 0; k < n; ++k) {
    double g[4];
    or_normals(seed, 0u, (uint32_t)k, 0u, STREAM_PC_GAUGE, 2, g);
    M2 A = zero2();
    for (int a = 1; a <= 3; ++a) A = add(A, scale(pauli(a), I1 * (I1 * sigma * g[a - 1])));
    Om[k] = expm(A);
  }
  for (int k = 0; k < n; ++k) V[k] = mul(mul(Om[k], V[k]), inverse(Om[(k + 1) % n]));
  store_chain(V, U);
  return 0;
}

int or_pc_action(int n, const double* U, double br, double bi, double* out2) {
  if (n < 1 || !U || !out2) return -1;
  std::vector<M2> V = load_chain(n, U);
  cd s = -cd(br, bi) / 2.0 * trace(cyclic_product(V, 0));
  out2[0] = s.real();
  out2[1] = s.imag();
  return 0;
}

int or_pc_drift(int n, const double* U, double br, double bi, double* K) {
  if (n < 1 || !U || !K) return -1;
  std::vector<cd> k;
  drift(load_chain(n, U), cd(br, bi), k);
  for (size_t i = 0; i < k.size(); ++i) {
    K[2 * i] = k[i].real();
    K[2 * i + 1] = k[i].imag();
  }
  return 0;
}

int or_pc_step(int n, double* U, double br, double bi, double eps, uint64_t seed, uint32_t step) {
  if (n < 1 || !U || !(eps >= 0.0)) return -1;
  std::vector<M2> V = load_chain(n, U);
  cl_step(V, cd(br, bi), eps, seed, step);
  store_chain(V, U);
  return 0;
}

int or_pc_cool_gradient(int n, const double* U, double* f) {
  if (n < 1 || !U || !f) return -1;
  std::vector<double> v;
  gradient(load_chain(n, U), v);
  std::copy(v.begin(), v.end(), f);
  return 0;
}

int or_pc_cool_sweep(int n, double* U, double eps, double alpha_ad) {
  if (n < 1 || !U) return -1;
  std::vector<M2> V = load_chain(n, U);
  cool_sweep(V, eps, alpha_ad);
  store_chain(V, U);
  return 0;
}

int or_pc_cool(int n, double* U, const or_cool_params* p, or_cool_report* rep) {
  if (n < 1 || !U || !p) return -1;
  std::vector<M2> V = load_chain(n, U);
  or_cool_report r;
  cool(V, *p, r);
  store_chain(V, U);
  if (rep) *rep = r;
  return 0;
}

// out4: (1/2) Tr(U_1 ... U_N) re, im; unitarity norm (1/N) sum (1/2) Tr U U^+;
// max |det U - 1|.
int or_pc_observables(int n, const double* U, double* out4) {
  if (n < 1 || !U || !out4) return -1;
  std::vector<M2> V = load_chain(n, U);
  cd t = 0.5 * trace(cyclic_product(V, 0));
  double md = 0.0;
  for (const M2& u : V) md = std::max(md, std::abs(det(u) - 1.0));
  out4[0] = t.real();
  out4[1] = t.imag();
  out4[2] = unitarity_norm(V);
  out4[3] = md;
  return 0;
}

// n_steps of [CL step, cooling (cool may be NULL)], recording after every
// step the 4 observables and the sweep count (5 doubles per step).
int or_pc_trajectory(int n, double* U, double br, double bi, double eps, uint64_t seed, uint32_t step0,
                     int n_steps, const or_cool_params* cool_p, double* rec) {
  if (n < 1 || !U || n_steps < 0) return -1;
  std::vector<M2> V = load_chain(n, U);
  for (int s = 0; s < n_steps; ++s) {
    cl_step(V, cd(br, bi), eps, seed, step0 + (uint32_t)s);
    or_cool_report r;
    r.sweeps = 0;
    if (cool_p) cool(V, *cool_p, r);
    if (rec) {
      store_chain(V, U);
      or_pc_observables(n, U, rec + 5 * s);
      rec[5 * s + 4] = r.sweeps;
    }
  }
  store_chain(V, U);
  return 0;
}

}  // extern "C"
