// pchain.cu -- the SU(2) Polyakov chain of Sec. 3-4, eq. "eq:s":
// S = -(beta/2) Tr(U_1 ... U_N), complex beta, links in SL(2,C), complex
// Langevin with (adaptive) gauge cooling (cl_pchain_*, include/cl.h).
//
// One CTA per chain and one thread per link; the chain lives in shared memory
// for a whole chunk of steps, so one launch runs [CL step, cooling sweeps,
// observables] many times with no HBM traffic but the records.  The drift of
// link k needs the cyclic product P_k = U_k ... U_N U_1 ... U_{k-1}; it is
// P_k = Suf_k Pre_{k-1} from an inclusive prefix and suffix product scan
// (Hillis-Steele, log2 N rounds).  With sum_a sigma_a Tr(sigma_a M) =
// 2 (M - Tr M / 2) the exponent of the update is
//   A = -eps beta (P_k - Tr P_k / 2) + i sqrt(eps) sqrt(2) g_a sigma_a,
// and exp of a traceless 2x2 matrix is cosh(s) + sinh(s)/s A with s^2 = -det A.
// Cooling: G_k = U_k U_k^+ - U_{k-1}^+ U_{k-1}, f_ak = 2 Tr(sigma_a G_k),
// Omega_k = exp(-eps alpha_ad f_ak sigma_a) (Hermitian: cosh r + sinh r / r H),
// U_k <- Omega_k U_k Omega_{k+1}^{-1}; the adaptive rule (alpha_ad = alpha / D,
// sweep-count stop rule) runs on the block's fixed-order reductions.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/cl.h"
#include "launch.h"
#include "philox.cuh"
#include "runtime.h"
#include "su3.cuh"

namespace clgc {
namespace {

const uint32_t STREAM_PC_CL = 3, STREAM_PC_GAUGE = 4;
const int PC_MAX_LINKS = 1024;
const int PC_CHUNK = 256;  // steps per launch

typedef cx<double> C;
struct M2 {
  C e[4];  // row-major [[e0 e1] [e2 e3]]
};

__device__ __forceinline__ M2 m2mul(const M2& x, const M2& y) {
  M2 r;
  r.e[0] = cfma(x.e[1], y.e[2], cmul(x.e[0], y.e[0]));
  r.e[1] = cfma(x.e[1], y.e[3], cmul(x.e[0], y.e[1]));
  r.e[2] = cfma(x.e[3], y.e[2], cmul(x.e[2], y.e[0]));
  r.e[3] = cfma(x.e[3], y.e[3], cmul(x.e[2], y.e[1]));
  return r;
}
__device__ __forceinline__ C cscale(C a, double s) { return C{a.re * s, a.im * s}; }
__device__ __forceinline__ C cconj(C a) { return C{a.re, -a.im}; }
__device__ __forceinline__ C m2det(const M2& x) { return cfms(x.e[1], x.e[2], cmul(x.e[0], x.e[3])); }

// Principal square root: Re >= 0.
__device__ __forceinline__ C csqrt_p(C z) {
  const double r = hypot(z.re, z.im);
  if (r == 0.0) return C{0.0, 0.0};
  if (z.re >= 0.0) {
    const double t = sqrt(0.5 * (r + z.re));
    return C{t, z.im / (2.0 * t)};
  }
  const double t = sqrt(0.5 * (r - z.re));
  return C{fabs(z.im) / (2.0 * t), copysign(t, z.im)};
}
__device__ __forceinline__ C cinv(C z) {
  const double d = 1.0 / (z.re * z.re + z.im * z.im);
  return C{z.re * d, -z.im * d};
}

// exp(A) for traceless A: cosh(s) I + sinh(s)/s A, s^2 = -det A; both
// coefficients are even in s, so they are power series in s^2 when s is small.
__device__ __forceinline__ M2 exp_traceless(const M2& A) {
  const C s2 = cfma(A.e[0], A.e[0], cmul(A.e[1], A.e[2]));
  C ch, sh;
  if (s2.re * s2.re + s2.im * s2.im < 0.25) {
    C t = C{1.0, 0.0};
    ch = t;
    sh = t;
    C ts = t;  // s^(2j) / (2j+1)!
    for (int j = 1; j <= 10; ++j) {
      t = cscale(cmul(t, s2), 1.0 / ((2.0 * j - 1.0) * (2.0 * j)));  // s^(2j) / (2j)!
      ch = cadd(ch, t);
      ts = cscale(cmul(ts, s2), 1.0 / ((2.0 * j) * (2.0 * j + 1.0)));
      sh = cadd(sh, ts);
    }
  } else {
    const C s = csqrt_p(s2);
    double sy, cy;
    sincos(s.im, &sy, &cy);
    const double chx = cosh(s.re), shx = sinh(s.re);
    ch = C{chx * cy, shx * sy};
    const C sinh_s = C{shx * cy, chx * sy};
    sh = cmul(sinh_s, cinv(s));
  }
  M2 r;
  r.e[0] = cfma(sh, A.e[0], ch);
  r.e[1] = cmul(sh, A.e[1]);
  r.e[2] = cmul(sh, A.e[2]);
  r.e[3] = cfma(sh, A.e[3], ch);
  return r;
}

// exp(+-H), H = h_a sigma_a with real h: cosh r I +- sinh(r)/r H.
__device__ __forceinline__ void exp_herm_pair(const double h[3], M2& ep, M2& em) {
  const double r2 = h[0] * h[0] + h[1] * h[1] + h[2] * h[2];
  const double r = sqrt(r2);
  double ch, sh;
  if (r < 1e-4) {
    ch = 1.0 + r2 * (0.5 + r2 * (1.0 / 24.0));
    sh = 1.0 + r2 * (1.0 / 6.0 + r2 * (1.0 / 120.0));
  } else {
    ch = cosh(r);
    sh = sinh(r) / r;
  }
  // H = [[h3, h1 - i h2], [h1 + i h2, -h3]]
  const double a = sh * h[2], b = sh * h[0], c = sh * h[1];
  ep.e[0] = C{ch + a, 0.0};
  ep.e[1] = C{b, -c};
  ep.e[2] = C{b, c};
  ep.e[3] = C{ch - a, 0.0};
  em.e[0] = C{ch - a, 0.0};
  em.e[1] = C{-b, c};
  em.e[2] = C{-b, -c};
  em.e[3] = C{ch + a, 0.0};
}

struct PcArgs {
  int n, n_chains;
  double2* U;             // [chain][k][4] complex entries
  const double* beta;     // [chain][re, im]
  const uint64_t* seed;   // [chain]
  uint32_t step0;         // Philox step word of the first step of this launch
  int n_steps;
  int done0;              // steps of this run call before this launch
  double eps;
  int cool;               // 0: no cooling
  CoolArgs ca;
  int obs_every;          // > 0: a record after every obs_every-th step of the run call
  double* obs;            // [record][chain][5]
};

// An array of n 2x2 complex matrices in shared memory, component-major
// (entry q of matrix k at p[q n + k]): consecutive threads touch consecutive
// doubles, so a warp's access is free of bank conflicts.
struct SM2 {
  double* p;
  int n;
  __device__ __forceinline__ M2 get(int k) const {
    M2 r;
#pragma unroll
    for (int q = 0; q < 4; ++q) r.e[q] = C{p[(2 * q) * n + k], p[(2 * q + 1) * n + k]};
    return r;
  }
  __device__ __forceinline__ void set(int k, const M2& m) const {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      p[(2 * q) * n + k] = m.e[q].re;
      p[(2 * q + 1) * n + k] = m.e[q].im;
    }
  }
};

// Fixed-order sum of three values and max of one over the block; every
// thread gets the totals.  red holds 32 * 4 doubles.
__device__ __forceinline__ void block_reduce4(double v[4], double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v[0] += __shfl_down_sync(0xffffffffu, v[0], o);
    v[1] += __shfl_down_sync(0xffffffffu, v[1], o);
    v[2] += __shfl_down_sync(0xffffffffu, v[2], o);
    v[3] = fmax(v[3], __shfl_down_sync(0xffffffffu, v[3], o));
  }
  __syncthreads();  // red may still be read from the previous call
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) red[4 * w + q] = v[q];
  }
  __syncthreads();
  double t[4] = {0.0, 0.0, 0.0, 0.0};
  for (int i = 0; i < nw; ++i) {
    t[0] += red[4 * i];
    t[1] += red[4 * i + 1];
    t[2] += red[4 * i + 2];
    t[3] = fmax(t[3], red[4 * i + 3]);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) v[q] = t[q];
}

// As[k] = U_0 ... U_k, Bs[k] = U_k ... U_{n-1}.
__device__ __forceinline__ void scan_products(const SM2& Us, const SM2& As, const SM2& Bs, int n) {
  const int k = threadIdx.x;
  const bool act = k < n;
  if (act) {
    const M2 u = Us.get(k);
    As.set(k, u);
    Bs.set(k, u);
  }
  __syncthreads();
  for (int off = 1; off < n; off <<= 1) {
    const bool da = act && k >= off, db = act && k + off < n;
    M2 pa, pb;
    if (da) pa = As.get(k - off);
    if (db) pb = Bs.get(k + off);
    __syncthreads();
    if (da) As.set(k, m2mul(pa, As.get(k)));
    if (db) Bs.set(k, m2mul(Bs.get(k), pb));
    __syncthreads();
  }
}

// MAXT = 512 for chains of up to 512 links (128 registers a thread, no
// spills); 1024 for longer ones (64 registers: some spilling to L1).
template <int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_pchain(PcArgs a) {
  extern __shared__ double smem[];
  const int n = a.n, c = blockIdx.x, k = threadIdx.x;
  const bool act = k < n;
  const SM2 Us{smem, n}, As{smem + 8 * n, n}, Bs{smem + 16 * n, n};
  double* red = smem + 24 * n;
  double2* Ug = a.U + (size_t)c * n * 4;
  if (act) {
    M2 u;
    for (int q = 0; q < 4; ++q) {
      const double2 v = Ug[4 * k + q];
      u.e[q] = C{v.x, v.y};
    }
    Us.set(k, u);
  }
  __syncthreads();
  const C beta = C{a.beta[2 * c], a.beta[2 * c + 1]};
  const uint64_t seed = a.seed[c];
  const double sq = sqrt(a.eps) * 1.41421356237309504880;  // sqrt(eps) * sqrt(2)
  for (int s = 0; s < a.n_steps; ++s) {
    // ---- CL step, all links at once
    scan_products(Us, As, Bs, n);
    // (each thread reads only its own link of Us, so it writes it in place)
    if (act) {
      const M2 P = k == 0 ? Bs.get(0) : m2mul(Bs.get(k), As.get(k - 1));
      double g[4];
      normals_f64<2>(g, seed, a.step0 + (uint32_t)s, (uint32_t)k, 0u, STREAM_PC_CL);
      const C htr = cscale(cadd(P.e[0], P.e[3]), 0.5);
      const C mb = C{-a.eps * beta.re, -a.eps * beta.im};  // -eps beta
      M2 A;
      A.e[0] = cmul(mb, csub(P.e[0], htr));
      A.e[3] = cmul(mb, csub(P.e[3], htr));
      A.e[1] = cmul(mb, P.e[1]);
      A.e[2] = cmul(mb, P.e[2]);
      // + i sq [[g3, g1 - i g2], [g1 + i g2, -g3]]
      A.e[0].im += sq * g[2];
      A.e[3].im -= sq * g[2];
      A.e[1].re += sq * g[1];
      A.e[1].im += sq * g[0];
      A.e[2].re -= sq * g[1];
      A.e[2].im += sq * g[0];
      M2 W = m2mul(exp_traceless(A), Us.get(k));
      const C z = cinv(csqrt_p(m2det(W)));
#pragma unroll
      for (int q = 0; q < 4; ++q) W.e[q] = cmul(W.e[q], z);
      Us.set(k, W);
    }
    __syncthreads();
    // ---- gauge cooling (the adaptive rule of the SU(3) path, per chain)
    int sweeps = 0;
    double un = 0.0, un_prev = 0.0;
    for (int it = 0;; ++it) {
      double v[4] = {0.0, 0.0, 0.0, 0.0}, f[3] = {0.0, 0.0, 0.0};
      if (act) {
        const M2 u = Us.get(k);
        const M2 w = Us.get(k == 0 ? n - 1 : k - 1);
        // G = u u^+ - w^+ w (Hermitian)
        C G00 = C{0.0, 0.0}, G01 = C{0.0, 0.0}, G10 = C{0.0, 0.0}, G11 = C{0.0, 0.0};
        G00 = cfma(u.e[0], cconj(u.e[0]), cfma(u.e[1], cconj(u.e[1]), G00));
        G01 = cfma(u.e[0], cconj(u.e[2]), cfma(u.e[1], cconj(u.e[3]), G01));
        G10 = cfma(u.e[2], cconj(u.e[0]), cfma(u.e[3], cconj(u.e[1]), G10));
        G11 = cfma(u.e[2], cconj(u.e[2]), cfma(u.e[3], cconj(u.e[3]), G11));
        G00 = cfms(cconj(w.e[0]), w.e[0], cfms(cconj(w.e[2]), w.e[2], G00));
        G01 = cfms(cconj(w.e[0]), w.e[1], cfms(cconj(w.e[2]), w.e[3], G01));
        G10 = cfms(cconj(w.e[1]), w.e[0], cfms(cconj(w.e[3]), w.e[2], G10));
        G11 = cfms(cconj(w.e[1]), w.e[1], cfms(cconj(w.e[3]), w.e[3], G11));
        f[0] = 2.0 * (G01.re + G10.re);
        f[1] = 2.0 * (G10.im - G01.im);
        f[2] = 2.0 * (G00.re - G11.re);
        const double tuu = u.e[0].re * u.e[0].re + u.e[0].im * u.e[0].im + u.e[1].re * u.e[1].re +
                           u.e[1].im * u.e[1].im + u.e[2].re * u.e[2].re + u.e[2].im * u.e[2].im +
                           u.e[3].re * u.e[3].re + u.e[3].im * u.e[3].im;
        v[0] = 0.5 * tuu;
        v[1] = fabs(f[0]) + fabs(f[1]) + fabs(f[2]);
        v[2] = f[0] * f[0] + f[1] * f[1] + f[2] * f[2];
      }
      block_reduce4(v, red);
      un = v[0] / n;
      if (!a.cool) break;
      double D = 1.0;
      if (a.ca.mode == CL_D1) D = un;
      if (a.ca.mode == CL_D2_MEANABS) D = v[1] / (3.0 * n);
      if (a.ca.mode == CL_D2_RMS) D = sqrt(v[2] / (3.0 * n));
      bool stop;
      if (a.ca.forced_sweeps >= 0) {
        stop = it >= a.ca.forced_sweeps;
      } else {
        stop = it >= a.ca.n_max;
        if (it >= a.ca.n_min) {
          if (un - 1.0 < a.ca.d_floor) stop = true;
          if (it >= 1 && (un_prev - un) < a.ca.tol_rel * (un_prev - 1.0)) stop = true;
        }
      }
      if (D < a.ca.d_guard) stop = true;
      if (stop) break;
      const double alpha_ad = a.ca.alpha / D;
      if (act) {
        const double ea = -a.ca.eps * alpha_ad;  // the cooling eps, not the Langevin one
        const double h[3] = {ea * f[0], ea * f[1], ea * f[2]};
        M2 om, omi;
        exp_herm_pair(h, om, omi);
        As.set(k, om);
        Bs.set(k, omi);
      }
      __syncthreads();
      if (act) Us.set(k, m2mul(m2mul(As.get(k), Us.get(k)), Bs.get(k + 1 == n ? 0 : k + 1)));
      __syncthreads();
      ++sweeps;
      un_prev = un;
    }
    // ---- records
    const int done = a.done0 + s + 1;
    if (a.obs_every > 0 && done % a.obs_every == 0) {
      scan_products(Us, As, Bs, n);
      double v[4] = {0.0, 0.0, 0.0, 0.0};
      if (act) {
        const C d = m2det(Us.get(k));
        v[3] = hypot(d.re - 1.0, d.im);
      }
      block_reduce4(v, red);
      if (k == 0) {
        double* o = a.obs + ((size_t)(done / a.obs_every - 1) * a.n_chains + c) * 5;
        const M2 tot = As.get(n - 1);
        o[0] = 0.5 * (tot.e[0].re + tot.e[3].re);
        o[1] = 0.5 * (tot.e[0].im + tot.e[3].im);
        o[2] = un;
        o[3] = v[3];
        o[4] = (double)sweeps;
      }
      __syncthreads();
    }
  }
  if (act) {
    const M2 u = Us.get(k);
    for (int q = 0; q < 4; ++q) Ug[4 * k + q] = make_double2(u.e[q].re, u.e[q].im);
  }
}

}  // namespace
}  // namespace clgc

namespace clgc {
namespace {

// Cold start then U_k <- Om_k U_k Om_{k+1}^{-1}, Om_k = exp(i w_a sigma_a),
// w_a = i sigma g_a: Om_k = exp(-sigma g_a sigma_a) (Hermitian), Philox stream 4.
__global__ void k_pchain_start(int n, int n_chains, double2* U, const uint64_t* seeds, double sigma) {
  const int c = blockIdx.y, k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n || c >= n_chains) return;
  const int k1 = k + 1 == n ? 0 : k + 1;
  double g0[4], g1[4];
  normals_f64<2>(g0, seeds[c], 0u, (uint32_t)k, 0u, STREAM_PC_GAUGE);
  normals_f64<2>(g1, seeds[c], 0u, (uint32_t)k1, 0u, STREAM_PC_GAUGE);
  const double h0[3] = {-sigma * g0[0], -sigma * g0[1], -sigma * g0[2]};
  const double h1[3] = {-sigma * g1[0], -sigma * g1[1], -sigma * g1[2]};
  M2 om, omi_unused, om1_unused, om1i;
  exp_herm_pair(h0, om, omi_unused);
  exp_herm_pair(h1, om1_unused, om1i);
  const M2 u = m2mul(om, om1i);
  double2* o = U + ((size_t)c * n + k) * 4;
  for (int q = 0; q < 4; ++q) o[q] = make_double2(u.e[q].re, u.e[q].im);
}

size_t pchain_smem(int n) { return (size_t)24 * n * sizeof(double) + 4 * 32 * sizeof(double); }

}  // namespace
}  // namespace clgc

using namespace clgc;
using namespace clrt;

struct cl_pchain {
  int n_chains, n;
  cudaStream_t st;
  double2* U;       // [chain][k][4]
  double* beta;     // [chain][2]
  uint64_t* seeds;  // [chain]
  uint64_t step;    // steps taken (the Philox step word of the next one)
};

extern "C" {

cl_status cl_pchain_create(int n_chains, int n_links, const double* beta, const uint64_t* seeds,
                           double gauge_sigma, void* cuda_stream, cl_pchain** out) {
  if (!out) return fail(CL_ERR_INVALID, "NULL argument");
  *out = nullptr;
  if (n_chains < 1 || n_chains > 65535 || n_links < 1 || n_links > PC_MAX_LINKS || !beta || !seeds)
    return fail(CL_ERR_INVALID, "need 1 <= n_links <= 1024, 1 <= n_chains <= 65535, beta and seeds");
  if (!(gauge_sigma >= 0.0)) return fail(CL_ERR_INVALID, "gauge_sigma must be >= 0");
  CK(cudaFuncSetAttribute(k_pchain<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pchain_smem(512)));
  CK(cudaFuncSetAttribute(k_pchain<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)pchain_smem(PC_MAX_LINKS)));
  cl_pchain* p = new cl_pchain();
  p->n_chains = n_chains;
  p->n = n_links;
  p->st = (cudaStream_t)cuda_stream;
  p->U = nullptr;
  p->beta = nullptr;
  p->seeds = nullptr;
  p->step = 0;
  cudaError_t e = cudaMalloc(&p->U, sizeof(double2) * 4 * (size_t)n_links * n_chains);
  if (e == cudaSuccess) e = cudaMalloc(&p->beta, sizeof(double) * 2 * n_chains);
  if (e == cudaSuccess) e = cudaMalloc(&p->seeds, sizeof(uint64_t) * n_chains);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->beta, beta, sizeof(double) * 2 * n_chains, cudaMemcpyHostToDevice, p->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->seeds, seeds, sizeof(uint64_t) * n_chains, cudaMemcpyHostToDevice, p->st);
  if (e == cudaSuccess) {
    dim3 grid((unsigned)((n_links + 127) / 128), (unsigned)n_chains);
    k_pchain_start<<<grid, 128, 0, p->st>>>(n_links, n_chains, p->U, p->seeds, gauge_sigma);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);  // beta and seeds were pageable
  if (e != cudaSuccess) {
    cl_pchain_free(p);
    return fail(e == cudaErrorMemoryAllocation ? CL_ERR_OOM : CL_ERR_CUDA,
                std::string("cl_pchain_create: ") + cudaGetErrorString(e));
  }
  *out = p;
  return CL_OK;
}

cl_status cl_pchain_run(cl_pchain* p, int n_steps, double eps, const cl_cool_params* cp, int obs_every,
                        double* obs_out) {
  if (!p || n_steps < 0 || !(eps >= 0.0)) return fail(CL_ERR_INVALID, "bad arguments");
  if (obs_every > 0 && !obs_out) return fail(CL_ERR_INVALID, "obs_out is NULL");
  if (cp) {
    cl_status s = check_cool(cp);
    if (s != CL_OK) return s;
  }
  const int nrec = obs_every > 0 ? n_steps / obs_every : 0;
  double* dobs = nullptr;
  if (nrec > 0) CK(cudaMalloc(&dobs, sizeof(double) * 5 * (size_t)nrec * p->n_chains));
  PcArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n = p->n;
  a.n_chains = p->n_chains;
  a.U = p->U;
  a.beta = p->beta;
  a.seed = p->seeds;
  a.eps = eps;
  a.cool = cp ? 1 : 0;
  if (cp) {
    a.ca.eps = cp->eps;
    a.ca.alpha = cp->alpha;
    a.ca.tol_rel = cp->tol_rel;
    a.ca.d_floor = cp->d_floor;
    a.ca.d_guard = cp->d_guard;
    a.ca.mode = (int)cp->mode;
    a.ca.n_min = cp->n_min;
    a.ca.n_max = cp->n_max;
    a.ca.forced_sweeps = cp->forced_sweeps;
  }
  a.obs_every = nrec > 0 ? obs_every : 0;
  a.obs = dobs;
  const int threads = ((p->n + 31) / 32) * 32;
  cudaError_t e = cudaSuccess;
  for (int done = 0; done < n_steps && e == cudaSuccess; done += PC_CHUNK) {
    a.step0 = (uint32_t)(p->step + done);
    a.done0 = done;
    a.n_steps = std::min(PC_CHUNK, n_steps - done);
    if (threads <= 512)
      k_pchain<512><<<p->n_chains, threads, pchain_smem(p->n), p->st>>>(a);
    else
      k_pchain<1024><<<p->n_chains, threads, pchain_smem(p->n), p->st>>>(a);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && nrec > 0)
    e = cudaMemcpyAsync(obs_out, dobs, sizeof(double) * 5 * (size_t)nrec * p->n_chains,
                        cudaMemcpyDeviceToHost, p->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
  if (dobs) cudaFree(dobs);
  if (e != cudaSuccess) return fail(CL_ERR_CUDA, std::string("cl_pchain_run: ") + cudaGetErrorString(e));
  p->step += (uint64_t)n_steps;
  return CL_OK;
}

cl_status cl_pchain_get_links(cl_pchain* p, double* host) {
  if (!p || !host) return fail(CL_ERR_INVALID, "NULL argument");
  CK(cudaMemcpyAsync(host, p->U, sizeof(double2) * 4 * (size_t)p->n * p->n_chains, cudaMemcpyDeviceToHost,
                     p->st));
  CK(cudaStreamSynchronize(p->st));
  return CL_OK;
}

cl_status cl_pchain_set_links(cl_pchain* p, const double* host) {
  if (!p || !host) return fail(CL_ERR_INVALID, "NULL argument");
  CK(cudaMemcpyAsync(p->U, host, sizeof(double2) * 4 * (size_t)p->n * p->n_chains, cudaMemcpyHostToDevice,
                     p->st));
  CK(cudaStreamSynchronize(p->st));
  return CL_OK;
}

cl_status cl_pchain_get_step(const cl_pchain* p, uint64_t* step) {
  if (!p || !step) return fail(CL_ERR_INVALID, "NULL argument");
  *step = p->step;
  return CL_OK;
}

void cl_pchain_free(cl_pchain* p) {
  if (!p) return;
  if (p->st) cudaStreamSynchronize(p->st);
  else cudaDeviceSynchronize();
  if (p->U) cudaFree(p->U);
  if (p->beta) cudaFree(p->beta);
  if (p->seeds) cudaFree(p->seeds);
  delete p;
}

}  // extern "C"
