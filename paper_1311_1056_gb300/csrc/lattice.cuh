// lattice.cuh -- periodic 4D lattice geometry shared by all kernels.
//
// Site index s = x0 + L0*(x1 + L1*(x2 + L2*x3)), direction mu = 0..3 along x_mu,
// periodic in every direction (any L_mu >= 1).  Link fields are SoA:
// element k (= 3*row + col) of U_mu(s) sits at ((mu*9 + k)*V + s), so a warp of
// consecutive sites reads 32 consecutive 16-byte (FP64) or 8-byte (FP32) words.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace clgc {

struct Geo {
  int L[4];
  int stride[4];
  int V;
};

inline Geo make_geo(const int L[4], int V) {
  Geo g;
  int st = 1;
  for (int mu = 0; mu < 4; ++mu) {
    g.L[mu] = L[mu];
    g.stride[mu] = st;
    st *= L[mu];
  }
  g.V = V;
  return g;
}

__device__ __forceinline__ void site_coords(const Geo& g, int s, int x[4]) {
  x[0] = s % g.L[0];
  int r = s / g.L[0];
  x[1] = r % g.L[1];
  r /= g.L[1];
  x[2] = r % g.L[2];
  x[3] = r / g.L[2];
}

// Site x + d e_mu, d in {-1, 0, +1}; x holds the coordinates of s in direction mu.
__device__ __forceinline__ int hop(const Geo& g, int s, const int x[4], int mu, int d) {
  int xm = x[mu] + d;
  int t = s + d * g.stride[mu];
  if (xm >= g.L[mu]) t -= g.L[mu] * g.stride[mu];
  if (xm < 0) t += g.L[mu] * g.stride[mu];
  return t;
}

// Site x + dm e_mu + dn e_nu (mu != nu): hops along different directions
// commute and leave the other coordinate unchanged.
__device__ __forceinline__ int hop2(const Geo& g, int s, const int x[4], int mu, int dm, int nu,
                                    int dn) {
  return hop(g, hop(g, s, x, mu, dm), x, nu, dn);
}

// Plane index of (a, b), a < b: (0,1)->0 (0,2)->1 (0,3)->2 (1,2)->3 (1,3)->4 (2,3)->5.
// The complementary plane of p is 5 - p.
__host__ __device__ constexpr int plane_index(int a, int b) {
  return a == 0 ? b - 1 : (a == 1 ? b + 1 : 5);
}
__host__ __device__ constexpr int plane_mu(int p) { return p < 3 ? 0 : (p < 5 ? 1 : 2); }
__host__ __device__ constexpr int plane_nu(int p) { return p < 3 ? p + 1 : (p < 5 ? p - 1 : 3); }

}  // namespace clgc
