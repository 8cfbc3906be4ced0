// noalloc.cu -- observables of caller-owned device links without any device
// allocation (cl_observables_noalloc in include/cl.h).
//
// Who needs it: code that cannot call cudaMalloc/cudaFree -- a host program
// whose device memory is owned by its own pool or arena and must account for
// every byte, or a latency-critical loop that cannot pay for an allocation
// that may synchronise the device.  Such a caller passes the links and the
// output buffer; the per-block partial sums live in the fixed array below.
//
// The array is a file-scope __device__ variable, so every GPU that loads the
// library holds it (CL_NOALLOC_MAX_BLOCKS records of 9 doubles, 147,456 bytes)
// until the process exits.  Its device address is looked up once per device
// with cudaGetSymbolAddress; host code never uses the symbol itself, which on
// the host is only a stand-in.  Every call shares the array: each launch
// overwrites the records it reads, so nothing needs clearing, but calls that
// overlap on the GPU (different streams, or different host threads) race on it.
#include <climits>
#include <mutex>
#include <string>

#include "../../include/cl.h"
#include "expm.cuh"
#include "lattice.cuh"
#include "su3.cuh"

namespace clgc {
void set_last_error(const std::string& msg);  // capi.cu: text returned by cl_last_error()

// The fixed scratch: one record of 9 partial sums per block.
static __device__ __align__(256) double g_noalloc_partials[CL_NOALLOC_MAX_BLOCKS * 9];

namespace {

const int NA_THREADS = 128;
const int NA_NQ = 9;
const double NA_KAPPA_Q = -1.0 / (256.0 * 9.86960440108935861883);

std::mutex g_setup_mutex;
double* g_scratch_addr[CL_NOALLOC_MAX_DEVICES] = {nullptr};

// Link U_mu(s) from the AoS layout of cl.h.
__device__ __forceinline__ void load_aos(mat<double>& m, const double* __restrict__ aos, int s, int mu) {
  const double* p = aos + ((size_t)s * 4 + mu) * 18;
#pragma unroll
  for (int k = 0; k < 9; ++k) m.e[k] = cx<double>{__ldg(p + 2 * k), __ldg(p + 2 * k + 1)};
}

// F_{mu nu}(x) = sum of the four clover leaves L at x (oriented mu -> nu) of L - L^{-1}.
__device__ void clover_at(mat<double>& F, const Geo& g, const double* aos, int s, const int x[4],
                          int mu, int nu) {
  const int xpm = hop(g, s, x, mu, 1), xmm = hop(g, s, x, mu, -1);
  const int xpn = hop(g, s, x, nu, 1), xmn = hop(g, s, x, nu, -1);
  const int xmm_pn = hop2(g, s, x, mu, -1, nu, 1), xmm_mn = hop2(g, s, x, mu, -1, nu, -1);
  const int xpm_mn = hop2(g, s, x, mu, 1, nu, -1);
  mat<double> a, b, A, B, L, Li;
  set_zero(F);
  for (int leaf = 0; leaf < 4; ++leaf) {
    if (leaf == 0) {  // U_mu(x) U_nu(x+mu) [U_nu(x) U_mu(x+nu)]^{-1}
      load_aos(a, aos, s, mu); load_aos(b, aos, xpm, nu); mul(A, a, b);
      load_aos(a, aos, s, nu); load_aos(b, aos, xpn, mu); mul(B, a, b);
      adj(a, B); mul(L, A, a);
    } else if (leaf == 1) {  // U_nu(x) [U_nu(x-mu) U_mu(x-mu+nu)]^{-1} U_mu(x-mu)
      load_aos(a, aos, xmm, nu); load_aos(b, aos, xmm_pn, mu); mul(B, a, b); adj(A, B);
      load_aos(a, aos, s, nu); mul(B, a, A);
      load_aos(b, aos, xmm, mu); mul(L, B, b);
    } else if (leaf == 2) {  // [U_nu(x-mu-nu) U_mu(x-mu)]^{-1} U_mu(x-mu-nu) U_nu(x-nu)
      load_aos(a, aos, xmm_mn, nu); load_aos(b, aos, xmm, mu); mul(B, a, b); adj(A, B);
      load_aos(a, aos, xmm_mn, mu); load_aos(b, aos, xmn, nu); mul(B, a, b);
      mul(L, A, B);
    } else {  // U_nu(x-nu)^{-1} U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^{-1}
      load_aos(a, aos, xmn, mu); load_aos(b, aos, xpm_mn, nu); mul(B, a, b);
      load_aos(a, aos, xmn, nu); adj(A, a); mul(a, A, B);
      load_aos(b, aos, s, mu); adj(A, b); mul(L, a, A);
    }
    adj(Li, L);
#pragma unroll
    for (int k = 0; k < 9; ++k) F.e[k] = cadd(F.e[k], csub(L.e[k], Li.e[k]));
  }
}

// Per-site observables (plaquette traces, (1/3) Tr U U^+, max |det U - 1|,
// q_L with the clover field formed on the fly, nonfinite count), grid-stride
// over sites, one partial record per block into the fixed array.
__global__ void __launch_bounds__(NA_THREADS) k_obs_noalloc(Geo g, const double* __restrict__ aos,
                                                            double* __restrict__ partials) {
  double v[NA_NQ];
#pragma unroll
  for (int q = 0; q < NA_NQ; ++q) v[q] = 0.0;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += gridDim.x * blockDim.x) {
    int x[4];
    site_coords(g, s, x);
    bool ok = true;
    for (int mu = 0; mu < 4; ++mu) {
      mat<double> u;
      load_aos(u, aos, s, mu);
#pragma unroll
      for (int k = 0; k < 9; ++k) ok = ok && isfinite(u.e[k].re) && isfinite(u.e[k].im);
      v[4] += norm2(u) * (1.0 / 3.0);
      cx<double> d = det(u);
      v[7] = fmax(v[7], hypot(d.re - 1.0, d.im));
    }
    for (int p = 0; p < 6; ++p) {
      const int mu = plane_mu(p), nu = plane_nu(p);
      mat<double> a, b, A, B, Ai, Bi;
      load_aos(a, aos, s, mu);
      load_aos(b, aos, hop(g, s, x, mu, 1), nu);
      mul(A, a, b);
      load_aos(a, aos, s, nu);
      load_aos(b, aos, hop(g, s, x, nu, 1), mu);
      mul(B, a, b);
      adj(Bi, B);
      adj(Ai, A);
      cx<double> tp = trace_mul(A, Bi), tpi = trace_mul(B, Ai);
      v[0] += tp.re * (1.0 / 3.0);
      v[1] += tp.im * (1.0 / 3.0);
      v[2] += tp.re + tpi.re;
      v[3] += tp.im + tpi.im;
    }
    cx<double> q = {0.0, 0.0};
    for (int p = 0; p < 3; ++p) {
      mat<double> F1, F2;
      clover_at(F1, g, aos, s, x, plane_mu(p), plane_nu(p));
      clover_at(F2, g, aos, s, x, plane_mu(5 - p), plane_nu(5 - p));
      cx<double> t = trace_mul(F1, F2);
      const double sg = (p == 1) ? -1.0 : 1.0;
      q.re += sg * t.re;
      q.im += sg * t.im;
    }
    v[5] += NA_KAPPA_Q * q.re;
    v[6] += NA_KAPPA_Q * q.im;
    v[8] += ok ? 0.0 : 1.0;
  }
  __shared__ double sm[NA_THREADS / 32][NA_NQ];
#pragma unroll
  for (int q = 0; q < NA_NQ; ++q)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      double o = __shfl_down_sync(0xffffffffu, v[q], off);
      v[q] = (q == 7) ? fmax(v[q], o) : v[q] + o;
    }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NA_NQ; ++q) sm[w][q] = v[q];
  __syncthreads();
  if (threadIdx.x < NA_NQ) {
    const int q = threadIdx.x;
    double t = sm[0][q];
    for (int k = 1; k < NA_THREADS / 32; ++k) t = (q == 7) ? fmax(t, sm[k][q]) : t + sm[k][q];
    partials[(size_t)blockIdx.x * NA_NQ + q] = t;
  }
}

// Fixed-order sum of the nb records into the caller's 10 outputs (cl_obs order).
__global__ void k_obs_noalloc_final(Geo g, const double* __restrict__ partials, int nb, double beta,
                                    double th_re, double th_im, double* __restrict__ out) {
  __shared__ double sm[256][NA_NQ];
  double v[NA_NQ];
#pragma unroll
  for (int q = 0; q < NA_NQ; ++q) v[q] = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
#pragma unroll
    for (int q = 0; q < NA_NQ; ++q) {
      const double x = partials[(size_t)b * NA_NQ + q];
      v[q] = (q == 7) ? fmax(v[q], x) : v[q] + x;
    }
#pragma unroll
  for (int q = 0; q < NA_NQ; ++q) sm[threadIdx.x][q] = v[q];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
#pragma unroll
      for (int q = 0; q < NA_NQ; ++q)
        sm[threadIdx.x][q] = (q == 7) ? fmax(sm[threadIdx.x][q], sm[threadIdx.x + w][q])
                                      : sm[threadIdx.x][q] + sm[threadIdx.x + w][q];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const double V = (double)g.V, np = 6.0 * V;
  const double* t = sm[0];
  const double sw_re = beta * np - beta / 6.0 * t[2], sw_im = -beta / 6.0 * t[3];
  out[0] = t[0] / np;                       // plaq_re
  out[1] = t[1] / np;                       // plaq_im
  out[2] = t[4] / (4.0 * V);                // un
  out[3] = t[5];                            // q_re
  out[4] = t[6];                            // q_im
  out[5] = sw_re;                           // sw_re
  out[6] = sw_im;                           // sw_im
  out[7] = sw_re + th_re * t[6] + th_im * t[5];  // S = S_W - i theta Q
  out[8] = sw_im - th_re * t[5] + th_im * t[6];
  out[9] = (t[8] > 0.0) ? nan("") : t[7];   // max |det U - 1|; NaN if a link is not finite
}

cl_status na_fail(cl_status s, const std::string& m) {
  set_last_error(m);
  return s;
}

// Device address of the fixed array on the current device (looked up once).
cl_status scratch_address(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(CL_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= CL_NOALLOC_MAX_DEVICES) return na_fail(CL_ERR_INVALID, "device index beyond CL_NOALLOC_MAX_DEVICES");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess || !p)
      return na_fail(CL_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = (double*)p;
  }
  *out = g_scratch_addr[dev];
  return CL_OK;
}

}  // namespace
}  // namespace clgc

using namespace clgc;

extern "C" cl_status cl_observables_noalloc(const double* dev_links, const int L[4], double beta,
                                            double theta_re, double theta_im, double* dev_out,
                                            void* cuda_stream) {
  if (!dev_links || !L || !dev_out) return na_fail(CL_ERR_INVALID, "NULL argument");
  long long V = 1;
  for (int mu = 0; mu < 4; ++mu) {
    if (L[mu] < 1) return na_fail(CL_ERR_INVALID, "lattice extent < 1");
    V *= L[mu];
    if (V > CL_NOALLOC_MAX_SITES)
      return na_fail(CL_ERR_INVALID, "lattice volume beyond CL_NOALLOC_MAX_SITES");
  }
  double* scratch = nullptr;
  cl_status s = scratch_address(&scratch);
  if (s != CL_OK) return s;
  Geo g = make_geo(L, (int)V);
  long long want = (V + NA_THREADS - 1) / NA_THREADS;
  const int nb = (int)(want < CL_NOALLOC_MAX_BLOCKS ? want : CL_NOALLOC_MAX_BLOCKS);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  k_obs_noalloc<<<nb, NA_THREADS, 0, st>>>(g, dev_links, scratch);
  k_obs_noalloc_final<<<1, 256, 0, st>>>(g, scratch, nb, beta, theta_re, theta_im, dev_out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(CL_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  return CL_OK;
}
