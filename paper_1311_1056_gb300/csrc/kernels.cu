// kernels.cu -- starts, layout conversion, clover field, gauge cooling and
// observables.  The CL update kernel itself is in k_update.cuh
// (instantiated by k_update_f64.cu / k_update_f32.cu).
#include <type_traits>

#include "cvt.cuh"
#include "expm.cuh"
#include "launch.h"
#include "lattice.cuh"
#include "philox.cuh"
#include "su3.cuh"

namespace clgc {

namespace {

const double KAPPA_Q = -1.0 / (256.0 * 9.86960440108935861883);  // -1/(256 pi^2)

Geo to_geo(const GeoH& h) { return make_geo(h.L, h.V); }

inline dim3 grid_sites(int V, int planes = 1) {
  return dim3((unsigned)((V + RED_THREADS - 1) / RED_THREADS), (unsigned)planes);
}

// Fixed-order block reduction of NQ doubles (slot MAXSLOT takes the max)
// into the block's record rec[0 .. NQ-1].
template <int NQ, int MAXSLOT>
__device__ __forceinline__ void block_reduce_store(double* v, double* rec) {
  __shared__ double sm[RED_THREADS / 32][NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      double o = __shfl_down_sync(0xffffffffu, v[q], off);
      v[q] = (q == MAXSLOT) ? fmax(v[q], o) : v[q] + o;
    }
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NQ; ++q) sm[w][q] = v[q];
  __syncthreads();
  if (threadIdx.x < NQ) {
    int q = threadIdx.x;
    double s = sm[0][q];
    for (int k = 1; k < RED_THREADS / 32; ++k) s = (q == MAXSLOT) ? fmax(s, sm[k][q]) : s + sm[k][q];
    rec[q] = s;
  }
}

// Single-block fixed-order sum of nb records of NQ doubles.
template <int NQ, int MAXSLOT>
__device__ __forceinline__ void reduce_partials(const double* partials, int nb, double* out) {
  __shared__ double sm[256][NQ];
  double v[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) v[q] = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double x = partials[(size_t)b * NQ + q];
      v[q] = (q == MAXSLOT) ? fmax(v[q], x) : v[q] + x;
    }
#pragma unroll
  for (int q = 0; q < NQ; ++q) sm[threadIdx.x][q] = v[q];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
#pragma unroll
      for (int q = 0; q < NQ; ++q)
        sm[threadIdx.x][q] = (q == MAXSLOT) ? fmax(sm[threadIdx.x][q], sm[threadIdx.x + w][q])
                                            : sm[threadIdx.x][q] + sm[threadIdx.x + w][q];
    __syncthreads();
  }
  if (threadIdx.x == 0)
#pragma unroll
    for (int q = 0; q < NQ; ++q) out[q] = sm[0][q];
}

template <typename T>
__device__ __forceinline__ bool finite_mat(const mat<T>& a) {
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 9; ++k) ok = ok && isfinite(a.e[k].re) && isfinite(a.e[k].im);
  return ok;
}

// --------------------------------------------------------------- starts
template <typename T>
__global__ void k_cold(Geo g, typename vec2_of<T>::type* U) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  mat<T> I;
  set_ident(I);
  store(U, blockIdx.y, s, g.V, I);
}

// Haar SU(3): Gram-Schmidt on the rows of a complex Gaussian matrix (Philox
// stream 2) gives Haar U(3); the principal cube root of the determinant maps
// it to SU(3).
template <typename T>
__global__ void k_hot(Geo g, typename vec2_of<T>::type* U, uint64_t seed) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int mu = blockIdx.y;
  double z[18];
  normals_f64<9>(z, seed, 0u, (uint32_t)s, (uint32_t)mu, STREAM_HOT);
  mat<double> m;
#pragma unroll
  for (int k = 0; k < 9; ++k) m.e[k] = cx<double>{z[2 * k], z[2 * k + 1]};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int k = 0; k < i; ++k) {
      cx<double> ip = {0.0, 0.0};  // <row_k, row_i>
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        cx<double> ck = {m.e[3 * k + j].re, -m.e[3 * k + j].im};
        ip = cfma(ck, m.e[3 * i + j], ip);
      }
#pragma unroll
      for (int j = 0; j < 3; ++j) m.e[3 * i + j] = cfms(ip, m.e[3 * k + j], m.e[3 * i + j]);
    }
    double n = 0.0;
#pragma unroll
    for (int j = 0; j < 3; ++j) n = fma(m.e[3 * i + j].re, m.e[3 * i + j].re, fma(m.e[3 * i + j].im, m.e[3 * i + j].im, n));
    double inv = 1.0 / sqrt(n);
#pragma unroll
    for (int j = 0; j < 3; ++j) { m.e[3 * i + j].re *= inv; m.e[3 * i + j].im *= inv; }
  }
  cx<double> zf = det_inv_cuberoot(det(m));
#pragma unroll
  for (int k = 0; k < 9; ++k) m.e[k] = cmul(m.e[k], zf);
  mat<T> t;
  convert(t, m);
  store(U, mu, s, g.V, t);
}

// Read-only load of one real of a packed field.
__device__ __forceinline__ double ldg_real(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ldg_real(const float* p) { return __ldg(p); }
__device__ __forceinline__ df64 ldg_real(const df64* p) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return df64(v.x, v.y);
}

// Packed Hermitian field: planes d0, d1, d2, re01, im01, re02, im02, re12, im12.
template <typename T>
__device__ __forceinline__ void store_herm(T* P, int s, int V, const herm& h) {
  P[0 * (size_t)V + s] = cvt<T>(h.d0);
  P[1 * (size_t)V + s] = cvt<T>(h.d1);
  P[2 * (size_t)V + s] = cvt<T>(h.d2);
  P[3 * (size_t)V + s] = cvt<T>(h.o01.re);
  P[4 * (size_t)V + s] = cvt<T>(h.o01.im);
  P[5 * (size_t)V + s] = cvt<T>(h.o02.re);
  P[6 * (size_t)V + s] = cvt<T>(h.o02.im);
  P[7 * (size_t)V + s] = cvt<T>(h.o12.re);
  P[8 * (size_t)V + s] = cvt<T>(h.o12.im);
}
template <typename T>
__device__ __forceinline__ void load_herm_mat(mat<T>& m, const T* __restrict__ P, int s, int V) {
  T d0 = ldg_real(P + s), d1 = ldg_real(P + (size_t)V + s), d2 = ldg_real(P + 2 * (size_t)V + s);
  T a = ldg_real(P + 3 * (size_t)V + s), b = ldg_real(P + 4 * (size_t)V + s);
  T c = ldg_real(P + 5 * (size_t)V + s), d = ldg_real(P + 6 * (size_t)V + s);
  T e = ldg_real(P + 7 * (size_t)V + s), f = ldg_real(P + 8 * (size_t)V + s);
  m.e[0] = cx<T>{d0, T(0)};
  m.e[4] = cx<T>{d1, T(0)};
  m.e[8] = cx<T>{d2, T(0)};
  m.e[1] = cx<T>{a, b};
  m.e[3] = cx<T>{a, -b};
  m.e[2] = cx<T>{c, d};
  m.e[6] = cx<T>{c, -d};
  m.e[5] = cx<T>{e, f};
  m.e[7] = cx<T>{e, -f};
}

template <typename T>
__device__ __forceinline__ void store_herm_df(T* P, int s, int V, const herm_df& h) {
  if constexpr (std::is_same<T, df64>::value) {
    P[0 * (size_t)V + s] = h.d0;
    P[1 * (size_t)V + s] = h.d1;
    P[2 * (size_t)V + s] = h.d2;
    P[3 * (size_t)V + s] = h.o01.re;
    P[4 * (size_t)V + s] = h.o01.im;
    P[5 * (size_t)V + s] = h.o02.re;
    P[6 * (size_t)V + s] = h.o02.im;
    P[7 * (size_t)V + s] = h.o12.re;
    P[8 * (size_t)V + s] = h.o12.im;
  }
}
// H = c * sum_a g_a lambda_a in double-float.
__device__ __forceinline__ herm_df herm_from_algebra_df(const df64* g, df64 c) {
  const df64 r3 = df_const(0.57735026918962576451);
  herm_df h;
  h.d0 = c * (g[2] + g[7] * r3);
  h.d1 = c * (g[7] * r3 - g[2]);
  h.d2 = -(c * df_ldexp(g[7] * r3, 1));
  h.o01 = cx<df64>{c * g[0], -(c * g[1])};
  h.o02 = cx<df64>{c * g[3], -(c * g[4])};
  h.o12 = cx<df64>{c * g[5], -(c * g[6])};
  return h;
}

// H = c * sum_a g_a lambda_a (Hermitian, traceless), g real.
__device__ __forceinline__ herm herm_from_algebra(const double* g, double c) {
  const double r3 = 0.57735026918962576451;
  herm h;
  h.d0 = c * (g[2] + g[7] * r3);
  h.d1 = c * (-g[2] + g[7] * r3);
  h.d2 = c * (-2.0 * g[7] * r3);
  h.o01 = cx<double>{c * g[0], -c * g[1]};
  h.o02 = cx<double>{c * g[3], -c * g[4]};
  h.o12 = cx<double>{c * g[5], -c * g[6]};
  return h;
}

// Omega_x = exp(i w_a lambda_a) with w_a = i sigma g_a, i.e. exp(-sigma g_a lambda_a).
template <typename T>
__global__ void k_gauge_omega(Geo g, T* Om, T* Omi, uint64_t seed, double sigma) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  double r[8];
  normals_f64<4>(r, seed, 0u, (uint32_t)s, 0u, STREAM_GAUGE);
  herm h = herm_from_algebra(r, -sigma), om, omi;
  expm_hermitian_pair(om, omi, h, taylor_tol<T>());
  store_herm(Om, s, g.V, om);
  store_herm(Omi, s, g.V, omi);
}

// The CL noise of links (site0 + i, mu) as form T draws it (a diagnostic).
template <typename T>
__global__ void k_noise_sample(int site0, int n, uint64_t seed, uint32_t step, uint32_t mu, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t s = (uint32_t)(site0 + i);
  if constexpr (std::is_same<T, double>::value) {
    normals_f64<4>(out + 8 * (size_t)i, seed, step, s, mu, STREAM_CL);
  } else if constexpr (std::is_same<T, float>::value) {
    float e[8];
    normals_f32<4>(e, seed, step, s, mu, STREAM_CL);
#pragma unroll
    for (int j = 0; j < 8; ++j) out[8 * (size_t)i + j] = (double)e[j];
  } else {
    df64 e[8];
    normals_df64<4>(e, seed, step, s, mu, STREAM_CL);
#pragma unroll
    for (int j = 0; j < 8; ++j) out[8 * (size_t)i + j] = (double)e[j];
  }
}

// ------------------------------------------------------------ conversion
// AoS [site][plane][row][col]{re,im} doubles <-> SoA planes of T2, through a
// shared-memory transpose of CONV_SITES sites: the AoS side (often the host's
// page-locked memory, read or written over the host link) is one contiguous
// run per block, and the SoA side is CONV_SITES consecutive sites per row.
// The tile's pitch is odd in 16-byte units, so the column-wise accesses of a
// quarter warp hit distinct banks.
const int CONV_SITES = 32, CONV_MAX_ROWS = 54;  // up to 6 planes
__host__ __device__ constexpr int conv_pitch(int rows) { return rows + 1 + (rows & 1); }

template <typename T>
__global__ void __launch_bounds__(256) k_aos_to_soa(Geo g, const double* __restrict__ aos,
                                                    typename vec2_of<T>::type* U, int nplanes) {
  __shared__ double2 buf[CONV_SITES * conv_pitch(CONV_MAX_ROWS)];
  const int R = 9 * nplanes, pitch = conv_pitch(R);
  const int s0 = blockIdx.x * CONV_SITES;
  const int ns = min(CONV_SITES, g.V - s0);
  const double* src = aos + 2 * (size_t)s0 * R;
  for (int e = threadIdx.x; e < ns * R; e += blockDim.x) {
    const int j = e / R, r = e - j * R;
    buf[j * pitch + r] = make_double2(src[2 * e], src[2 * e + 1]);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < R * CONV_SITES; e += blockDim.x) {
    const int r = e / CONV_SITES, j = e - r * CONV_SITES;
    if (j < ns) {
      const double2 v = buf[j * pitch + r];
      U[(size_t)r * g.V + s0 + j] = pack(cx<T>{(T)v.x, (T)v.y});
    }
  }
}
template <typename T>
__global__ void __launch_bounds__(256) k_soa_to_aos(Geo g, const typename vec2_of<T>::type* __restrict__ U,
                                                    double* aos, int nplanes) {
  __shared__ double2 buf[CONV_SITES * conv_pitch(CONV_MAX_ROWS)];
  const int R = 9 * nplanes, pitch = conv_pitch(R);
  const int s0 = blockIdx.x * CONV_SITES;
  const int ns = min(CONV_SITES, g.V - s0);
  for (int e = threadIdx.x; e < R * CONV_SITES; e += blockDim.x) {
    const int r = e / CONV_SITES, j = e - r * CONV_SITES;
    if (j < ns) {
      const cx<T> c = unpack(U[(size_t)r * g.V + s0 + j]);
      buf[j * pitch + r] = make_double2((double)c.re, (double)c.im);
    }
  }
  __syncthreads();
  double* dst = aos + 2 * (size_t)s0 * R;
  for (int e = threadIdx.x; e < ns * R; e += blockDim.x) {
    const int j = e / R, r = e - j * R;
    const double2 v = buf[j * pitch + r];
    dst[2 * e] = v.x;
    dst[2 * e + 1] = v.y;
  }
}

// --------------------------------------------------------------- cooling
// The gradient of the DF64 form: G_x accumulated entry by entry in
// double-float (dacc, renormalised after every link), f stored as hi + lo
// float pairs, the rule's sums kept per thread in double-float and widened
// to FP64 once for the block reduction.
__device__ __forceinline__ void dacc_add_abs2(dacc& a, cx<df64> z, bool neg) {
  dacc_add(a, neg ? -z.re : z.re, z.re);
  dacc_add(a, neg ? -z.im : z.im, z.im);
}
// a += sign * x conj(y)
__device__ __forceinline__ void dacc_add_xcy(dacc& re, dacc& im, cx<df64> x, cx<df64> y, bool neg) {
  const df64 xr = neg ? -x.re : x.re, xi = neg ? -x.im : x.im;
  dacc_add(re, xr, y.re);
  dacc_add(re, xi, y.im);
  dacc_add(im, xi, y.re);
  dacc_add(im, -xr, y.im);
}
__device__ __forceinline__ void cool_grad_df(const Geo& g, const float4* __restrict__ U, float2* f,
                                             double* v) {
  df64 s_abs(0.0f, 0.0f), s_sq(0.0f, 0.0f), s_un(0.0f, 0.0f);
  int bad = 0;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += gridDim.x * blockDim.x) {
    int x[4];
    site_coords(g, s, x);
    dacc G[9];  // 00, 11, 22, 01re, 01im, 02re, 02im, 12re, 12im
#pragma unroll
    for (int q = 0; q < 9; ++q) G[q] = dacc{0.0f, 0.0f};
    bool ok = true;
    df64 un(0.0f, 0.0f);
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
#pragma unroll 1
      for (int mu = 0; mu < 4; ++mu) {  // rolled: unrolled, the code outgrows the instruction cache
        // entry e of the link at p[e V]; three entries at a time keep the
        // registers for one more resident block
        const float4* p = U + (size_t)mu * 9 * g.V + (dir == 0 ? s : hop(g, s, x, mu, -1));
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          // + U U^+: column k of the forward link; - U^+ U: row k of the backward link
          const int e0 = dir == 0 ? k : 3 * k, e1 = dir == 0 ? 3 + k : 3 * k + 1, e2 = dir == 0 ? 6 + k : 3 * k + 2;
          const cx<df64> r0 = unpack(__ldg(p + (size_t)e0 * g.V)), r1 = unpack(__ldg(p + (size_t)e1 * g.V)),
                         r2 = unpack(__ldg(p + (size_t)e2 * g.V));
          const bool neg = dir == 1;
          dacc_add_abs2(G[0], r0, neg);
          dacc_add_abs2(G[1], r1, neg);
          dacc_add_abs2(G[2], r2, neg);
          // + r_i conj(r_j) forward; - conj(c_i) c_j = - x conj(y) with x = conj(c_i),
          // y = conj(c_j) backward
          if (dir == 0) {
            dacc_add_xcy(G[3], G[4], r0, r1, false);
            dacc_add_xcy(G[5], G[6], r0, r2, false);
            dacc_add_xcy(G[7], G[8], r1, r2, false);
          } else {
            const cx<df64> q0 = {r0.re, -r0.im}, q1 = {r1.re, -r1.im}, q2 = {r2.re, -r2.im};
            dacc_add_xcy(G[3], G[4], q0, q1, true);
            dacc_add_xcy(G[5], G[6], q0, q2, true);
            dacc_add_xcy(G[7], G[8], q1, q2, true);
          }
        }
#pragma unroll
        for (int q = 0; q < 9; ++q) dacc_norm(G[q]);
      }
      if (dir == 0) un = dacc_get(G[0]) + dacc_get(G[1]) + dacc_get(G[2]);
    }
    const df64 g00 = dacc_get(G[0]), g11 = dacc_get(G[1]), g22 = dacc_get(G[2]);
    df64 fa[8];
    fa[0] = df_ldexp(dacc_get(G[3]), 2);
    fa[1] = -df_ldexp(dacc_get(G[4]), 2);
    fa[2] = df_ldexp(g00 - g11, 1);
    fa[3] = df_ldexp(dacc_get(G[5]), 2);
    fa[4] = -df_ldexp(dacc_get(G[6]), 2);
    fa[5] = df_ldexp(dacc_get(G[7]), 2);
    fa[6] = -df_ldexp(dacc_get(G[8]), 2);
    fa[7] = df_ldexp(df_const(0.57735026918962576451) * (g00 + g11 - df_ldexp(g22, 1)), 1);
    ok = ok && isfinite(un);
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      f[(size_t)a * g.V + s] = make_float2(fa[a].hi, fa[a].lo);
      s_abs = s_abs + (fa[a].hi < 0.0f ? -fa[a] : fa[a]);
      s_sq = fma(fa[a], fa[a], s_sq);
      ok = ok && isfinite(fa[a]);
    }
    s_un = s_un + un;
    bad += ok ? 0 : 1;
  }
  v[0] = (double)s_abs;
  v[1] = (double)s_sq;
  v[2] = (double)s_un * (1.0 / 3.0);
  v[3] = (double)bad;
}

// f_ax = 2 Tr[lambda_a G_x], G_x = sum_mu (U_{x,mu} U_{x,mu}^+ - U_{x-mu,mu}^+ U_{x-mu,mu})
// (Sec. 2, eq. "eq:24") at site s, in the link type; returns the sum over
// the four links at x of Tr U U^+.
template <typename T>
__device__ __forceinline__ T cool_grad_site(const Geo& g, const typename vec2_of<T>::type* __restrict__ U, int s,
                                            const int x[4], T fa[8]) {
  T g00 = T(0), g11 = T(0), g22 = T(0);
  cx<T> g01 = {T(0), T(0)}, g02 = {T(0), T(0)}, g12 = {T(0), T(0)};
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    mat<T> u;
    load(u, U, mu, s, g.V);
    // + U U^+ : (i,j) = sum_k U_ik conj(U_jk)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      cx<T> r0 = u.e[k], r1 = u.e[3 + k], r2 = u.e[6 + k];
      g00 = fma(r0.re, r0.re, fma(r0.im, r0.im, g00));
      g11 = fma(r1.re, r1.re, fma(r1.im, r1.im, g11));
      g22 = fma(r2.re, r2.re, fma(r2.im, r2.im, g22));
      g01 = cfma(r0, cx<T>{r1.re, -r1.im}, g01);
      g02 = cfma(r0, cx<T>{r2.re, -r2.im}, g02);
      g12 = cfma(r1, cx<T>{r2.re, -r2.im}, g12);
    }
  }
  // sum over the four links at x of Tr U U^+ = the diagonal accumulated so far
  const T un = g00 + g11 + g22;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    mat<T> u;
    load(u, U, mu, hop(g, s, x, mu, -1), g.V);
    // - U^+ U : (i,j) = sum_k conj(U_ki) U_kj
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      cx<T> c0 = u.e[3 * k], c1 = u.e[3 * k + 1], c2 = u.e[3 * k + 2];
      g00 = fma(-c0.re, c0.re, fma(-c0.im, c0.im, g00));
      g11 = fma(-c1.re, c1.re, fma(-c1.im, c1.im, g11));
      g22 = fma(-c2.re, c2.re, fma(-c2.im, c2.im, g22));
      g01 = cfms(cx<T>{c0.re, -c0.im}, c1, g01);
      g02 = cfms(cx<T>{c0.re, -c0.im}, c2, g02);
      g12 = cfms(cx<T>{c1.re, -c1.im}, c2, g12);
    }
  }
  const T r3 = (T)0.57735026918962576451;
  const T two = T(2), four = T(4);
  fa[0] = four * g01.re;
  fa[1] = -(four * g01.im);
  fa[2] = two * (g00 - g11);
  fa[3] = four * g02.re;
  fa[4] = -(four * g02.im);
  fa[5] = four * g12.re;
  fa[6] = -(four * g12.im);
  fa[7] = two * r3 * (g00 + g11 - two * g22);
  return un;
}

// The gradient f into [a][V] (FP64) with, per block, sum |f|, sum f^2,
// sum (1/3) Tr U U^+ of the links at x and the nonfinite count.
// Block vb of nvb (the grid-stride loop over sites and the record index).
template <typename T>
__device__ __forceinline__ void cool_grad_body(const Geo& g, const typename vec2_of<T>::type* __restrict__ U,
                                               double* __restrict__ f, double* partials, const CoolState* cs,
                                               int vb, int nvb) {
  if (cs && cs->done) return;
  double v[NQ_COOL] = {0.0, 0.0, 0.0, 0.0};
  for (int s = vb * blockDim.x + threadIdx.x; s < g.V; s += nvb * blockDim.x) {
    int x[4];
    site_coords(g, s, x);
    T fa[8];
    const T un = cool_grad_site<T>(g, U, s, x, fa);
    bool ok = isfinite(un);
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const double d = cvt<double>(fa[a]);
      f[(size_t)a * g.V + s] = d;
      v[0] += fabs(d);
      v[1] = fma(d, d, v[1]);
      ok = ok && isfinite(fa[a]);
    }
    v[2] += cvt<double>(un) * (1.0 / 3.0);
    v[3] += ok ? 0.0 : 1.0;
  }
  block_reduce_store<NQ_COOL, -1>(v, partials + (size_t)vb * NQ_COOL);
}
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_cool_grad(Geo g, const typename vec2_of<T>::type* __restrict__ U,
                                                          double* __restrict__ f, double* partials,
                                                          const CoolState* cs) {
  cool_grad_body<T>(g, U, f, partials, cs, blockIdx.x, gridDim.x);
}

// Single-pass sweep of the D_0 / D_1 rules, part 1: the strength alpha_ad of
// these rules needs only the unitarity norm, which the previous sweep's apply
// (k_cool_apply_tiles) summed, so the rule has decided before this kernel runs
// and the gradient never leaves the thread: f_ax at x, then Omega_x =
// exp(-eps alpha_ad f_ax lambda_a) and its inverse (FP64), stored packed.
template <typename T>
__device__ __forceinline__ void cool_grad_omega_body(const Geo& g, const typename vec2_of<T>::type* __restrict__ U,
                                                     T* __restrict__ Om, T* __restrict__ Omi, double eps,
                                                     const CoolState* cs, int vb, int nvb) {
  if (cs->done) return;
  const double c = -eps * cs->alpha_ad;
  for (int s = vb * blockDim.x + threadIdx.x; s < g.V; s += nvb * blockDim.x) {
    int x[4];
    site_coords(g, s, x);
    T fa[8];
    cool_grad_site<T>(g, U, s, x, fa);
    double fd[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) fd[a] = cvt<double>(fa[a]);
    herm h = herm_from_algebra(fd, c), om, omi;
    expm_hermitian_pair(om, omi, h, taylor_tol<T>());
    store_herm(Om, s, g.V, om);
    store_herm(Omi, s, g.V, omi);
  }
}
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_cool_grad_omega(Geo g,
                                                                const typename vec2_of<T>::type* __restrict__ U,
                                                                T* __restrict__ Om, T* __restrict__ Omi, double eps,
                                                                const CoolState* cs) {
  cool_grad_omega_body<T>(g, U, Om, Omi, eps, cs, blockIdx.x, gridDim.x);
}

// The adaptive rule (Sec. 4): alpha_ad = alpha / D with D_0 = 1,
// D_1 = (1/3)<Tr U U^+> (normalised unitarity norm), D_2 = <|f_ax|>_{a,x}
// (or its RMS).  Sweep count: at least n_min, at most n_max; stop once the
// norm decreases by less than tol_rel of its distance from 1 or that distance
// is below d_floor; no sweep when D < d_guard; forced_sweeps >= 0 fixes the count.
// tot: sum |f_ax|, sum f_ax^2, sum (1/3) Tr U U^+ over the links, nonfinite count.
__device__ __forceinline__ void cool_rule(const Geo& g, const double* tot, const CoolArgs& a, CoolState* cs,
                                          int first) {
  if (first) {
    cs->alpha_ad = 0.0;
    cs->alpha_ad_last = 0.0;
    cs->un_prev = 0.0;
    cs->sweeps = 0;
    cs->done = 0;
    cs->k = 0;
    cs->nonfinite = 0;
  }
  if (cs->done) return;
  const double V = (double)g.V;
  double un = tot[2] / (4.0 * V);
  double D = 1.0;
  if (a.mode == 1) D = un;
  if (a.mode == 2) D = tot[0] / (8.0 * V);
  if (a.mode == 3) D = sqrt(tot[1] / (8.0 * V));
  int k = cs->k;
  if (k == 0) cs->un_before = un;
  cs->un_after = un;
  cs->D = D;
  bool stop;
  if (a.forced_sweeps >= 0) {
    stop = k >= a.forced_sweeps;
  } else {
    stop = k >= a.n_max;
    if (k >= a.n_min) {
      if (un - 1.0 < a.d_floor) stop = true;
      if (k >= 1 && (cs->un_prev - un) < a.tol_rel * (cs->un_prev - 1.0)) stop = true;
    }
  }
  if (D < a.d_guard) stop = true;
  if (tot[3] != 0.0 || !isfinite(un)) {
    cs->nonfinite = 1;
    stop = true;
  }
  cs->k = k + 1;
  if (stop) {
    cs->done = 1;
    return;
  }
  cs->alpha_ad = a.alpha / D;
  cs->alpha_ad_last = cs->alpha_ad;
  cs->sweeps += 1;
  cs->un_prev = un;
}
__device__ __forceinline__ void cool_adapt_body(const Geo& g, const double* partials, int nb, const CoolArgs& a,
                                                CoolState* cs, int first) {
  __shared__ double tot[NQ_COOL];
  reduce_partials<NQ_COOL, -1>(partials, nb, tot);
  __syncthreads();
  if (threadIdx.x != 0) return;
  cool_rule(g, tot, a, cs, first);
}
__global__ void k_cool_adapt(Geo g, const double* partials, int nb, CoolArgs a, CoolState* cs, int first) {
  cool_adapt_body(g, partials, nb, a, cs, first);
}

// The DF64 gradient kernel: its own launch bound, so that the whole
// reduction grid (8 blocks per SM) is resident in one wave.
__global__ void __launch_bounds__(RED_THREADS, RED_MAX_BLOCKS / 152) k_cool_grad_df(Geo g, const float4* __restrict__ U,
                                                                             float2* __restrict__ f, double* partials,
                                                                             const CoolState* cs) {
  if (cs && cs->done) return;
  double v[NQ_COOL] = {0.0, 0.0, 0.0, 0.0};
  cool_grad_df(g, U, f, v);
  block_reduce_store<NQ_COOL, -1>(v, partials + (size_t)blockIdx.x * NQ_COOL);
}

// Omega_x = exp(-eps alpha_ad f_ax lambda_a) and its inverse: FP64, or
// double-float in the DF64 form.
template <typename T>
__device__ __forceinline__ void cool_omega_body(const Geo& g, const double* __restrict__ f, T* Om, T* Omi, double eps,
                                                const CoolState* cs, int vb) {
  if (cs->done) return;
  int s = vb * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  if constexpr (std::is_same<T, df64>::value) {
    // DF64: f as hi + lo pairs, the exponential pair in double-float
    const float2* fp = reinterpret_cast<const float2*>(f);
    df64 fa[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const float2 w = __ldg(fp + (size_t)a * g.V + s);
      fa[a] = df64(w.x, w.y);
    }
    herm_df h = herm_from_algebra_df(fa, df64(-eps * cs->alpha_ad)), om, omi;
    expm_hermitian_pair_df(om, omi, h);
    store_herm_df(Om, s, g.V, om);
    store_herm_df(Omi, s, g.V, omi);
  } else {
    double fa[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) fa[a] = __ldg(f + (size_t)a * g.V + s);
    herm h = herm_from_algebra(fa, -eps * cs->alpha_ad), om, omi;
    expm_hermitian_pair(om, omi, h, taylor_tol<T>());
    store_herm(Om, s, g.V, om);
    store_herm(Omi, s, g.V, omi);
  }
}
template <typename T>
__global__ void __launch_bounds__(TUNE_MAX_BLOCK) k_cool_omega(Geo g, const double* __restrict__ f, T* Om, T* Omi,
                                                           double eps, const CoolState* cs) {
  cool_omega_body<T>(g, f, Om, Omi, eps, cs, blockIdx.x);
}

// U_{x,mu} <- Omega_x U_{x,mu} Omega_{x+mu}^{-1}, all links at once (in place:
// every link is read and written by the same thread).
template <typename T>
__device__ __forceinline__ void cool_apply_body(const Geo& g, typename vec2_of<T>::type* U, const T* __restrict__ Om,
                                                const T* __restrict__ Omi, const CoolState* cs, int vb) {
  if (cs && cs->done) return;
  const int mu = vb % 4;
  const int s = (vb / 4) * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int x[4];
  site_coords(g, s, x);
  mat<T> o, oi, u, t;
  load_herm_mat(o, Om, s, g.V);
  load_herm_mat(oi, Omi, hop(g, s, x, mu, 1), g.V);
  load(u, U, mu, s, g.V);
  mul_herm_left(t, o, u);
  mul_herm_right(u, t, oi);
  store(U, mu, s, g.V, u);
}
template <typename T>
__global__ void __launch_bounds__(TUNE_MAX_BLOCK) k_cool_apply(Geo g, typename vec2_of<T>::type* U, const T* __restrict__ Om,
                                                           const T* __restrict__ Omi,
                                                           const CoolState* cs) {
  cool_apply_body<T>(g, U, Om, Omi, cs, blockIdx.x);
}

// Single-pass sweep of the D_0 / D_1 rules, part 2: the apply over tiles of
// COOL_TILE consecutive sites inside one x3 layer (tile `tile` of layer
// `layer`; the last tile of a layer may be short), one thread per site and
// its four links (Omega_x loaded once), with one record per tile of what the
// rule needs for the next sweep: the sum of (1/3) Tr U U^+ over the tile's
// updated links (FP64, summed in a fixed order) and their nonfinite count (a
// NaN or Inf entry makes a site's sum of squares NaN or +Inf).  A record per
// tile, not per block of a grid-stride loop, makes the records and the rule's
// sum independent of the launch shape: a fused batch, which runs the tiles of
// many chains in one launch, gives each chain the records of its lone run.
// Resident blocks of COOL_TILE threads the tile kernels are built for: 72
// registers a thread with FP32 links, 128 with FP64 ones (a few bytes of spills).
#define COOL_TILE_MIN_BLOCKS(T) (sizeof(T) == 4 ? 7 : 4)
__device__ __forceinline__ int layer_sites(const Geo& g) { return g.V / g.L[3]; }
__device__ __forceinline__ int tiles_per_layer(const Geo& g) { return (layer_sites(g) + COOL_TILE - 1) / COOL_TILE; }

template <typename T>
__device__ __forceinline__ void cool_apply_tile(const Geo& g, typename vec2_of<T>::type* U, const T* __restrict__ Om,
                                                const T* __restrict__ Omi, double2* rec, int layer, int tile) {
  const int V3 = layer_sites(g);
  const int s0 = layer * V3 + tile * COOL_TILE;
  const int s1 = min(s0 + COOL_TILE, (layer + 1) * V3);
  const int s = s0 + (int)threadIdx.x;
  double2 v = make_double2(0.0, 0.0);
  if (s < s1) {
    int x[4];
    site_coords(g, s, x);
    mat<T> o;
    load_herm_mat(o, Om, s, g.V);
    T un = T(0);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      mat<T> oi, u, t;
      load_herm_mat(oi, Omi, hop(g, s, x, mu, 1), g.V);
      load(u, U, mu, s, g.V);
      mul_herm_left(t, o, u);
      mul_herm_right(u, t, oi);
      store(U, mu, s, g.V, u);
      un += norm2(u);
    }
    v.x = cvt<double>(un) * (1.0 / 3.0);
    v.y = isfinite(un) ? 0.0 : 1.0;
  }
  // fixed-order tile sum: warp shuffles, then the warps' sums in order
  __shared__ double2 sm[COOL_TILE / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, off);
    v.y += __shfl_down_sync(0xffffffffu, v.y, off);
  }
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 t = sm[0];
#pragma unroll
    for (int w = 1; w < COOL_TILE / 32; ++w) {
      t.x += sm[w].x;
      t.y += sm[w].y;
    }
    rec[layer * tiles_per_layer(g) + tile] = t;
  }
}

// One block per tile (block b: layer b / tiles_per_layer, tile b % tiles_per_layer).
template <typename T>
__global__ void __launch_bounds__(COOL_TILE, COOL_TILE_MIN_BLOCKS(T))
    k_cool_apply_tiles(Geo g, typename vec2_of<T>::type* U, const T* __restrict__ Om, const T* __restrict__ Omi,
                       double2* rec, const CoolState* cs) {
  if (cs->done) return;
  const int tpl = tiles_per_layer(g);
  cool_apply_tile<T>(g, U, Om, Omi, rec, blockIdx.x / tpl, blockIdx.x % tpl);
}

// The rule from the tile records: a fixed-order sum over the nrec records by
// COOL_RULE_THREADS threads (thread t takes records t, t + COOL_RULE_THREADS,
// ..., then warp shuffles and the warps' sums in order), with the |f| slots
// of the record layout 0 (D_0 / D_1 do not use them).
enum { COOL_RULE_THREADS = 1024 };
__device__ __forceinline__ void cool_adapt_tiles_body(const Geo& g, const double2* __restrict__ rec, int nrec,
                                                      const CoolArgs& a, CoolState* cs) {
  __shared__ double2 sm[COOL_RULE_THREADS / 32];
  double2 v = make_double2(0.0, 0.0);
#pragma unroll 4
  for (int b = threadIdx.x; b < nrec; b += COOL_RULE_THREADS) {
    const double2 r = __ldg(rec + b);
    v.x += r.x;
    v.y += r.y;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, off);
    v.y += __shfl_down_sync(0xffffffffu, v.y, off);
  }
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x >= 32) return;
  v = sm[threadIdx.x];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, off);
    v.y += __shfl_down_sync(0xffffffffu, v.y, off);
  }
  if (threadIdx.x != 0 || cs->done) return;
  const double tot[NQ_COOL] = {0.0, 0.0, v.x, v.y};
  cool_rule(g, tot, a, cs, 0);
}
__global__ void __launch_bounds__(COOL_RULE_THREADS) k_cool_adapt_tiles(Geo g, const double2* rec, int nrec,
                                                                        CoolArgs a, CoolState* cs) {
  cool_adapt_tiles_body(g, rec, nrec, a, cs);
}

const int DF_APPLY_BLOCK = 128;  // the DF64 apply's largest block (its launch bound)

// The DF64 apply: row i of Omega U (five real terms per part of each entry,
// Dot2-accumulated), then row i of (Omega U) Omega'^{-1}, stored at once; the
// whole link is read before the first row is written.  (Capping it at 96
// registers for a fifth block per SM spills and gains nothing.)
__global__ void __launch_bounds__(DF_APPLY_BLOCK, 4) k_cool_apply_df(Geo g, float4* U, const df64* __restrict__ Om,
                                                                  const df64* __restrict__ Omi,
                                                                  const CoolState* cs) {
  if (cs && cs->done) return;
  const int mu = blockIdx.x % 4;
  const int s = (blockIdx.x / 4) * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int x[4];
  site_coords(g, s, x);
  mat<df64> o, oi, u;
  load_herm_mat(o, Om, s, g.V);
  load_herm_mat(oi, Omi, hop(g, s, x, mu, 1), g.V);
  load(u, U, mu, s, g.V);
  float4* p = U + (size_t)mu * 9 * g.V + s;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    cx<df64> t[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {  // t_j = (Omega U)_ij, Omega_ii real
      const df64 d = o.e[4 * i].re;
      dacc re = dacc_first(d, u.e[3 * i + j].re), im = dacc_first(d, u.e[3 * i + j].im);
#pragma unroll
      for (int k = 0; k < 3; ++k)
        if (k != i) {
          const cx<df64> a = o.e[3 * i + k], b = u.e[3 * k + j];
          dacc_add(re, a.re, b.re);
          dacc_add(re, -a.im, b.im);
          dacc_add(im, a.re, b.im);
          dacc_add(im, a.im, b.re);
        }
      t[j] = cx<df64>{dacc_get(re), dacc_get(im)};
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {  // (t Omega'^{-1})_j, Omega'^{-1}_jj real
      const df64 d = oi.e[4 * j].re;
      dacc re = dacc_first(t[j].re, d), im = dacc_first(t[j].im, d);
#pragma unroll
      for (int k = 0; k < 3; ++k)
        if (k != j) {
          const cx<df64> a = t[k], b = oi.e[3 * k + j];
          dacc_add(re, a.re, b.re);
          dacc_add(re, -a.im, b.im);
          dacc_add(im, a.re, b.im);
          dacc_add(im, a.im, b.re);
        }
      p[(size_t)(3 * i + j) * g.V] = pack(cx<df64>{dacc_get(re), dacc_get(im)});
    }
  }
}

// ----------------------------------------------------------- observables
// Per site: the six plaquettes P_{mu nu}(x) = U_mu(x) U_nu(x+mu) U_mu(x+nu)^{-1} U_nu(x)^{-1}
// (Tr P / 3 and Tr P + Tr P^{-1} for S_W), (1/3) Tr U U^+ of the four links,
// max |det U - 1| (FP64), nonfinite count and, with the clover field,
// q_L(x) = kappa [Tr F01 F23 - Tr F02 F13 + Tr F03 F12].
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_obs(Geo g, const typename vec2_of<T>::type* __restrict__ U,
                                                    const typename vec2_of<T>::type* __restrict__ F,
                                                    int with_q, double* partials, double* q_site) {
  double v[NQ_OBS];
#pragma unroll
  for (int q = 0; q < NQ_OBS; ++q) v[q] = 0.0;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += gridDim.x * blockDim.x) {
    int x[4];
    site_coords(g, s, x);
    bool ok = true;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      mat<T> u;
      load(u, U, mu, s, g.V);
      ok = ok && finite_mat(u);
      v[4] += (double)norm2(u) * (1.0 / 3.0);
      mat<double> ud;
      convert(ud, u);
      cx<double> d = det(ud);
      v[7] = fmax(v[7], hypot(d.re - 1.0, d.im));
    }
#pragma unroll
    for (int p = 0; p < 6; ++p) {
      const int mu = plane_mu(p), nu = plane_nu(p);
      mat<T> a, b, A, B, Ai, Bi;
      load(a, U, mu, s, g.V);
      load(b, U, nu, hop(g, s, x, mu, 1), g.V);
      mul(A, a, b);
      load(a, U, nu, s, g.V);
      load(b, U, mu, hop(g, s, x, nu, 1), g.V);
      mul(B, a, b);
      adj(Bi, B);
      adj(Ai, A);
      cx<T> tp = trace_mul(A, Bi);   // Tr P
      cx<T> tpi = trace_mul(B, Ai);  // Tr P^{-1}
      v[0] += (double)tp.re * (1.0 / 3.0);
      v[1] += (double)tp.im * (1.0 / 3.0);
      v[2] += (double)tp.re + (double)tpi.re;
      v[3] += (double)tp.im + (double)tpi.im;
    }
    if (with_q) {
      mat<T> F1, F2;
      cx<double> q = {0.0, 0.0};
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        load(F1, F, p, s, g.V);
        load(F2, F, 5 - p, s, g.V);
        cx<T> t = trace_mul(F1, F2);
        double sg = (p == 1) ? -1.0 : 1.0;
        q.re += sg * (double)t.re;
        q.im += sg * (double)t.im;
      }
      q.re *= KAPPA_Q;
      q.im *= KAPPA_Q;
      v[5] += q.re;
      v[6] += q.im;
      if (q_site) {
        q_site[2 * (size_t)s] = q.re;
        q_site[2 * (size_t)s + 1] = q.im;
      }
    }
    v[8] += ok ? 0.0 : 1.0;
  }
  block_reduce_store<NQ_OBS, 7>(v, partials + (size_t)blockIdx.x * NQ_OBS);
}

__global__ void k_obs_final(Geo g, const double* partials, int nb, double beta, double th_re,
                            double th_im, ObsOut* out) {
  __shared__ double tot[NQ_OBS];
  reduce_partials<NQ_OBS, 7>(partials, nb, tot);
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double V = (double)g.V, np = 6.0 * V;
  out->plaq_re = tot[0] / np;
  out->plaq_im = tot[1] / np;
  out->un = tot[4] / (4.0 * V);
  out->q_re = tot[5];
  out->q_im = tot[6];
  out->sw_re = beta * np - beta / 6.0 * tot[2];
  out->sw_im = -beta / 6.0 * tot[3];
  // S = S_W - i theta Q
  out->s_re = out->sw_re + th_re * tot[6] + th_im * tot[5];
  out->s_im = out->sw_im - th_re * tot[5] + th_im * tot[6];
  out->max_det_dev = tot[7];
  out->nonfinite = tot[8];
}

// Self-test of the integer-pipe conversions (cvt.cuh) against the hardware
// ones, bit for bit (NaN against NaN).  Case i draws 64 random bits by the
// SplitMix64 finaliser of seed + i: all 32-bit float patterns (every exponent,
// subnormals, infinities, NaNs) for f2d; for d2f doubles whose exponent spans
// the float range and both its ends (underflow to zero, overflow to inf),
// every fourth an exact rounding tie, every eighth a full random pattern.
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
__global__ void k_selftest_convert(uint64_t seed, long long n, unsigned long long* bad) {
  unsigned long long b0 = 0, b1 = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const uint64_t r = splitmix64(seed + (uint64_t)i), q = splitmix64(r);
    const float f = __uint_as_float((unsigned)r);
    const double a = f2d(f), b = (double)f;
    if (!(isnan(a) && isnan(b)) && __double_as_longlong(a) != __double_as_longlong(b)) ++b0;
    uint64_t bits;
    if ((i & 7) == 7) {
      bits = q;
    } else {
      const uint64_t e = 860u + (q >> 52) % 310u;  // float underflow .. overflow
      uint64_t m = q & 0xfffffffffffffull;
      if ((i & 3) == 0) m = (m & ~0x1fffffffull) | 0x10000000ull;  // exact tie
      bits = ((r >> 63) << 63) | (e << 52) | m;
    }
    const double d = __longlong_as_double((long long)bits);
    const float x = d2f(d), y = __double2float_rn(d);
    if (!(isnan(x) && isnan(y)) && __float_as_uint(x) != __float_as_uint(y)) ++b1;
  }
  if (b0) atomicAdd(bad, b0);
  if (b1) atomicAdd(bad + 1, b1);
}

// Distance in units in the last place of b (at least the spacing of the
// smallest normal, so exact zeros compare by absolute error).
__device__ __forceinline__ double ulps(double a, double b) {
  const double fb = fabs(b);
  const double up = __longlong_as_double(__double_as_longlong(fb) + 1);  // the next double above |b|
  const double u = fmax(up - fb, 2.2250738585072014e-308);
  return fabs(a - b) / u;
}
// The table-driven ln and sincospi of the FP64 Box-Muller (philox.cuh)
// against CUDA's log and sincospi on n uniforms (k + 1/2) 2^-52: k over its
// whole range, its smallest values, and values next to 2^52; the largest
// distances in ulp (rounded up) into worst[0] (ln) and worst[1] (sin, cos).
__global__ void k_selftest_box_muller(uint64_t seed, long long n, unsigned long long* worst) {
  double w0 = 0.0, w1 = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const uint64_t r = splitmix64(seed + (uint64_t)i);
    uint64_t k = r >> 12;                                        // 52 bits
    if ((i & 15) == 1) k >>= (r & 63) % 52;                      // small k: deep tail of ln
    if ((i & 15) == 2) k = ((1ull << 52) - 1) - (k >> 30);       // u next to 1
    if ((i & 15) == 3) k = (k >> 45) << 45 | ((r & 1) ? 0 : (1ull << 45) - 1);  // next to the sin grid
    const double u = u52_bits(k);
    w0 = fmax(w0, ulps(ln_unit(u), log(u)));
    double s, c, s0, c0;
    sincospi_2u52(k, &s, &c);
    sincospi(2.0 * u, &s0, &c0);
    w1 = fmax(w1, fmax(ulps(s, s0), ulps(c, c0)));
  }
  atomicMax(worst, (unsigned long long)ceil(w0));
  atomicMax(worst + 1, (unsigned long long)ceil(w1));
}

}  // namespace

// ------------------------------------------------------------ fused batch
// The cooling kernels of a fused batch: one launch over the blocks of every
// listed chain, each block running the body of the chain's own kernel with
// the chain's geometry, buffers and rule state (see ensemble.cuh).  Cooling
// follows the step's update, which wrote the chain's Un: that is the link
// field these kernels cool (the runtime swaps U and Un after the step).
namespace {

__device__ __forceinline__ Geo ens_geo(const ChainDesc& c) {
  Geo g;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    g.L[mu] = c.L[mu];
    g.stride[mu] = c.stride[mu];
  }
  g.V = c.V;
  return g;
}
__device__ __forceinline__ int ens_reduce_blocks(int V) {
  const int b = (V + RED_THREADS - 1) / RED_THREADS;
  return b < RED_MAX_BLOCKS ? b : RED_MAX_BLOCKS;
}

// first = 1: the call's first gradient, which always runs (as k_cool_grad with no state)
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_ens_cool_grad(const ChainDesc* __restrict__ cd,
                                                              const WorkItem* __restrict__ w, int first) {
  typedef typename vec2_of<T>::type V2;
  const WorkItem it = w[blockIdx.x];
  const ChainDesc& c = cd[it.chain];
  cool_grad_body<T>(ens_geo(c), (const V2*)c.Un, (double*)c.f, c.partials, first ? nullptr : c.cs, it.vb,
                    ens_reduce_blocks(c.V));
}
template <typename T>
__global__ void __launch_bounds__(TUNE_MAX_BLOCK) k_ens_cool_omega(const ChainDesc* __restrict__ cd,
                                                                  const WorkItem* __restrict__ w) {
  const WorkItem it = w[blockIdx.x];
  const ChainDesc& c = cd[it.chain];
  cool_omega_body<T>(ens_geo(c), (const double*)c.f, (T*)c.Om, (T*)c.Omi, c.ca.eps, c.cs, it.vb);
}
template <typename T>
__global__ void __launch_bounds__(TUNE_MAX_BLOCK) k_ens_cool_apply(const ChainDesc* __restrict__ cd,
                                                                  const WorkItem* __restrict__ w) {
  typedef typename vec2_of<T>::type V2;
  const WorkItem it = w[blockIdx.x];
  const ChainDesc& c = cd[it.chain];
  cool_apply_body<T>(ens_geo(c), (V2*)c.Un, (const T*)c.Om, (const T*)c.Omi, c.cs, it.vb);
}
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_ens_cool_grad_omega(const ChainDesc* __restrict__ cd,
                                                                    const WorkItem* __restrict__ w) {
  typedef typename vec2_of<T>::type V2;
  const WorkItem it = w[blockIdx.x];
  const ChainDesc& c = cd[it.chain];
  cool_grad_omega_body<T>(ens_geo(c), (const V2*)c.Un, (T*)c.Om, (T*)c.Omi, c.ca.eps, c.cs, it.vb,
                          ens_reduce_blocks(c.V));
}
template <typename T>
__global__ void __launch_bounds__(COOL_TILE, COOL_TILE_MIN_BLOCKS(T)) k_ens_cool_apply_tiles(const ChainDesc* __restrict__ cd,
                                                                   const WorkItem* __restrict__ w) {
  typedef typename vec2_of<T>::type V2;
  const WorkItem it = w[blockIdx.x];
  const ChainDesc& c = cd[it.chain];
  const Geo g = ens_geo(c);
  if (c.cs->done) return;
  const int tpl = tiles_per_layer(g);
  cool_apply_tile<T>(g, (V2*)c.Un, (const T*)c.Om, (const T*)c.Omi, (double2*)c.arec, it.vb / tpl, it.vb % tpl);
}
// the rule, one block of 256 threads per listed chain
__global__ void k_ens_cool_adapt(const ChainDesc* __restrict__ cd, const int* __restrict__ chains, int first) {
  const ChainDesc& c = cd[chains[blockIdx.x]];
  cool_adapt_body(ens_geo(c), c.partials, ens_reduce_blocks(c.V), c.ca, c.cs, first);
}
// the rule of single-pass chains from their tile records, one block per listed chain
__global__ void __launch_bounds__(COOL_RULE_THREADS) k_ens_cool_adapt_tiles(const ChainDesc* __restrict__ cd,
                                                               const int* __restrict__ chains) {
  const ChainDesc& c = cd[chains[blockIdx.x]];
  const Geo g = ens_geo(c);
  cool_adapt_tiles_body(g, (const double2*)c.arec, g.L[3] * tiles_per_layer(g), c.ca, c.cs);
}

template <typename T>
cudaError_t launch_ens_cool_family(int fam, const ChainDesc* cd, const WorkItem* w, int nw, int arg, cudaStream_t st) {
  const unsigned n = (unsigned)nw;
  switch (fam) {
    case ENS_COOL_GRAD: k_ens_cool_grad<T><<<n, RED_THREADS, 0, st>>>(cd, w, arg); break;
    case ENS_COOL_OMEGA: k_ens_cool_omega<T><<<n, ENS_BLOCK, 0, st>>>(cd, w); break;
    case ENS_COOL_APPLY: k_ens_cool_apply<T><<<n, ENS_BLOCK, 0, st>>>(cd, w); break;
    case ENS_COOL_GRAD_OMEGA: k_ens_cool_grad_omega<T><<<n, RED_THREADS, 0, st>>>(cd, w); break;
    case ENS_COOL_APPLY_UN: k_ens_cool_apply_tiles<T><<<n, COOL_TILE, 0, st>>>(cd, w); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_ens_step_f64(int fam, const ChainDesc* cd, const WorkItem* w, int nw, cudaStream_t st);
cudaError_t launch_ens_step_f32(int fam, const ChainDesc* cd, const WorkItem* w, int nw, cudaStream_t st);

cudaError_t launch_ens(int prec, int fam, const ChainDesc* cd, const WorkItem* w, int nw, int arg, cudaStream_t st) {
  if (nw <= 0) return cudaSuccess;
  if (prec != 0 && prec != 1) return cudaErrorInvalidValue;
  if (fam < ENS_COOL_GRAD)
    return prec == 0 ? launch_ens_step_f64(fam, cd, w, nw, st) : launch_ens_step_f32(fam, cd, w, nw, st);
  return prec == 0 ? launch_ens_cool_family<double>(fam, cd, w, nw, arg, st)
                   : launch_ens_cool_family<float>(fam, cd, w, nw, arg, st);
}

cudaError_t launch_ens_cool_adapt(const ChainDesc* cd, const int* chains, int n, int first, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_ens_cool_adapt<<<n, 256, 0, st>>>(cd, chains, first);
  return cudaGetLastError();
}

cudaError_t launch_ens_cool_adapt_tiles(const ChainDesc* cd, const int* chains, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_ens_cool_adapt_tiles<<<n, COOL_RULE_THREADS, 0, st>>>(cd, chains);
  return cudaGetLastError();
}

cudaError_t launch_selftest_convert(uint64_t seed, long long n, unsigned long long* bad, cudaStream_t st) {
  k_selftest_convert<<<RED_MAX_BLOCKS, RED_THREADS, 0, st>>>(seed, n, bad);
  return cudaGetLastError();
}

cudaError_t launch_selftest_box_muller(uint64_t seed, long long n, unsigned long long* worst, cudaStream_t st) {
  k_selftest_box_muller<<<RED_MAX_BLOCKS, RED_THREADS, 0, st>>>(seed, n, worst);
  return cudaGetLastError();
}

// Reduction kernels loop over sites with at most RED_MAX_BLOCKS blocks, so
// the one-block rule reads few records; the split depends on V only.
// Launch with the link type of precision prec (0 FP64, 1 FP32 storage, 2 DF64).
template <typename Fn>
cudaError_t by_prec(int prec, Fn fn) {
  if (prec == 0) fn(double());
  else if (prec == 1) fn(float());
  else fn(df64());
  return cudaGetLastError();
}

int reduce_blocks(int V) {
  int b = (V + RED_THREADS - 1) / RED_THREADS;
  return b < RED_MAX_BLOCKS ? b : RED_MAX_BLOCKS;
}

cudaError_t launch_cold(int prec, const GeoH& h, void* U, cudaStream_t st) {
  Geo g = to_geo(h);
  return by_prec(prec, [&](auto t) {
    using T = decltype(t);
    k_cold<T><<<grid_sites(g.V, 4), RED_THREADS, 0, st>>>(g, (typename vec2_of<T>::type*)U);
  });
}

cudaError_t launch_hot(int prec, const GeoH& h, void* U, uint64_t seed, cudaStream_t st) {
  Geo g = to_geo(h);
  return by_prec(prec, [&](auto t) {
    using T = decltype(t);
    k_hot<T><<<grid_sites(g.V, 4), RED_THREADS, 0, st>>>(g, (typename vec2_of<T>::type*)U, seed);
  });
}

cudaError_t launch_gauge_omega(int prec, const GeoH& h, void* Om, void* Omi, uint64_t seed,
                               double sigma, cudaStream_t st) {
  Geo g = to_geo(h);
  return by_prec(prec, [&](auto t) {
    using T = decltype(t);
    k_gauge_omega<T><<<grid_sites(g.V), RED_THREADS, 0, st>>>(g, (T*)Om, (T*)Omi, seed, sigma);
  });
}

cudaError_t launch_aos_to_soa(int prec, const GeoH& h, const double* aos, void* U, int nplanes,
                              cudaStream_t st) {
  Geo g = to_geo(h);
  if (nplanes < 1 || 9 * nplanes > CONV_MAX_ROWS) return cudaErrorInvalidValue;
  const unsigned blocks = (unsigned)((g.V + CONV_SITES - 1) / CONV_SITES);
  return by_prec(prec, [&](auto t) {
    using T = decltype(t);
    k_aos_to_soa<T><<<blocks, 256, 0, st>>>(g, aos, (typename vec2_of<T>::type*)U, nplanes);
  });
}

cudaError_t launch_soa_to_aos(int prec, const GeoH& h, const void* U, double* aos, int nplanes,
                              cudaStream_t st) {
  Geo g = to_geo(h);
  if (nplanes < 1 || 9 * nplanes > CONV_MAX_ROWS) return cudaErrorInvalidValue;
  const unsigned blocks = (unsigned)((g.V + CONV_SITES - 1) / CONV_SITES);
  return by_prec(prec, [&](auto t) {
    using T = decltype(t);
    k_soa_to_aos<T><<<blocks, 256, 0, st>>>(g, (const typename vec2_of<T>::type*)U, aos, nplanes);
  });
}

cudaError_t launch_noise_sample(int prec, int site0, int n, uint64_t seed, uint32_t step, int mu, double* out,
                                cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  return by_prec(prec, [&](auto t) {
    using T = decltype(t);
    k_noise_sample<T><<<(n + 127) / 128, 128, 0, st>>>(site0, n, seed, step, (uint32_t)mu, out);
  });
}

cudaError_t launch_cool_grad(int prec, const GeoH& h, const void* U, void* f, double* partials,
                             const CoolState* cs, cudaStream_t st) {
  Geo g = to_geo(h);
  return by_prec(prec, [&](auto t) {
    using T = decltype(t);
    if constexpr (std::is_same<T, df64>::value)
      k_cool_grad_df<<<reduce_blocks(g.V), RED_THREADS, 0, st>>>(g, (const float4*)U, (float2*)f, partials, cs);
    else
      k_cool_grad<T><<<reduce_blocks(g.V), RED_THREADS, 0, st>>>(g, (const typename vec2_of<T>::type*)U, (double*)f,
                                                                partials, cs);
  });
}

cudaError_t launch_cool_adapt(const GeoH& h, const double* partials, CoolArgs a, CoolState* cs,
                              int first, cudaStream_t st) {
  Geo g = to_geo(h);
  k_cool_adapt<<<1, 256, 0, st>>>(g, partials, reduce_blocks(g.V), a, cs, first);
  return cudaGetLastError();
}

cudaError_t launch_cool_omega(int prec, const GeoH& h, const void* f, void* Om, void* Omi, double eps,
                              const CoolState* cs, cudaStream_t st) {
  Geo g = to_geo(h);
  const int bs = block_of(h, TUNE_OMEGA);
  const dim3 grid((unsigned)((g.V + bs - 1) / bs));
  return by_prec(prec, [&](auto t) {
    using T = decltype(t);
    k_cool_omega<T><<<grid, bs, 0, st>>>(g, (const double*)f, (T*)Om, (T*)Omi, eps, cs);
  });
}

cudaError_t launch_cool_apply(int prec, const GeoH& h, void* U, const void* Om, const void* Omi,
                              const CoolState* cs, cudaStream_t st) {
  Geo g = to_geo(h);
  const int bs = block_of(h, TUNE_APPLY);
  const dim3 grid((unsigned)(((g.V + bs - 1) / bs) * 4));
  return by_prec(prec, [&](auto t) {
    using T = decltype(t);
    if constexpr (std::is_same<T, df64>::value) {
      const int b = bs < DF_APPLY_BLOCK ? bs : DF_APPLY_BLOCK;
      const dim3 gd((unsigned)(((g.V + b - 1) / b) * 4));
      k_cool_apply_df<<<gd, b, 0, st>>>(g, (float4*)U, (const df64*)Om, (const df64*)Omi, cs);
    } else
      k_cool_apply<T><<<grid, bs, 0, st>>>(g, (typename vec2_of<T>::type*)U, (const T*)Om, (const T*)Omi, cs);
  });
}

cudaError_t launch_cool_grad_omega(int prec, const GeoH& h, const void* U, void* Om, void* Omi, double eps,
                                   const CoolState* cs, cudaStream_t st) {
  Geo g = to_geo(h);
  if (prec == 0)
    k_cool_grad_omega<double><<<reduce_blocks(g.V), RED_THREADS, 0, st>>>(g, (const double2*)U, (double*)Om,
                                                                          (double*)Omi, eps, cs);
  else if (prec == 1)
    k_cool_grad_omega<float><<<reduce_blocks(g.V), RED_THREADS, 0, st>>>(g, (const float2*)U, (float*)Om,
                                                                         (float*)Omi, eps, cs);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

int cool_tiles(const GeoH& h) {
  const int V3 = h.V / h.L[3];
  return h.L[3] * ((V3 + COOL_TILE - 1) / COOL_TILE);
}

cudaError_t launch_cool_apply_tiles(int prec, const GeoH& h, void* U, const void* Om, const void* Omi, double* rec,
                                    const CoolState* cs, cudaStream_t st) {
  Geo g = to_geo(h);
  const unsigned n = (unsigned)cool_tiles(h);
  if (prec == 0)
    k_cool_apply_tiles<double><<<n, COOL_TILE, 0, st>>>(g, (double2*)U, (const double*)Om, (const double*)Omi,
                                                        (double2*)rec, cs);
  else if (prec == 1)
    k_cool_apply_tiles<float><<<n, COOL_TILE, 0, st>>>(g, (float2*)U, (const float*)Om, (const float*)Omi,
                                                       (double2*)rec, cs);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_cool_adapt_tiles(const GeoH& h, const double* rec, CoolArgs a, CoolState* cs, cudaStream_t st) {
  Geo g = to_geo(h);
  k_cool_adapt_tiles<<<1, COOL_RULE_THREADS, 0, st>>>(g, (const double2*)rec, cool_tiles(h), a, cs);
  return cudaGetLastError();
}

cudaError_t launch_obs(int prec, const GeoH& h, const void* U, const void* F, int with_q,
                       double* partials, double* q_site, cudaStream_t st) {
  Geo g = to_geo(h);
  return by_prec(prec, [&](auto t) {
    using T = decltype(t);
    k_obs<T><<<reduce_blocks(g.V), RED_THREADS, 0, st>>>(g, (const typename vec2_of<T>::type*)U,
                                                        (const typename vec2_of<T>::type*)F, with_q, partials,
                                                        q_site);
  });
}

cudaError_t launch_obs_final(const GeoH& h, const double* partials, double beta, double th_re,
                             double th_im, ObsOut* out, cudaStream_t st) {
  Geo g = to_geo(h);
  k_obs_final<<<1, 256, 0, st>>>(g, partials, reduce_blocks(g.V), beta, th_re, th_im, out);
  return cudaGetLastError();
}

}  // namespace clgc
