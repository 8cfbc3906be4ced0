// oracle.cpp -- plain FP64 CPU oracle for complex Langevin (CL) with adaptive
// gauge cooling of SU(3) Yang-Mills with a theta-term (arXiv:1311.1056).
//
// TEST INFRASTRUCTURE ONLY: the independent checker of the CUDA path.  Only
// the tests, the smoke check and the CPU-baseline leg of the benchmark load
// it.  Nothing here is shared with the CUDA library.
//
// Every routine is written from the definitions, slow and literal:
//   * the action is a list of traced closed loops (Wilson plaquettes and the
//     384 signed eps-tilde terms of q_L per site, Sec. 5, eq. "eq:st"),
//   * the drift is the product rule applied occurrence by occurrence to every
//     loop that contains a link,
//   * exp is Taylor with scaling and squaring, inverse is Gauss-Jordan,
//     det is the Leibniz sum.
// Parity pins that tie each routine to the paper are in tests/test_oracle_*.py.
// Functions without such a pin: none (the sweep-count stop rule of or_cool is
// a reading of Sec. 4, pinned only by its stated invariants).
#include "oracle.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

using cd = std::complex<double>;
const cd I1(0.0, 1.0);
const double PI = 3.14159265358979323846264338327950288;

struct Mat {
  cd m[3][3];
};

Mat zero() {
  Mat r;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) r.m[i][j] = 0.0;
  return r;
}
Mat ident() {
  Mat r = zero();
  for (int i = 0; i < 3; ++i) r.m[i][i] = 1.0;
  return r;
}
Mat mul(const Mat& a, const Mat& b) {
  Mat r;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      cd s = 0.0;
      for (int k = 0; k < 3; ++k) s += a.m[i][k] * b.m[k][j];
      r.m[i][j] = s;
    }
  return r;
}
Mat add(const Mat& a, const Mat& b) {
  Mat r;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) r.m[i][j] = a.m[i][j] + b.m[i][j];
  return r;
}
Mat sub(const Mat& a, const Mat& b) {
  Mat r;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) r.m[i][j] = a.m[i][j] - b.m[i][j];
  return r;
}
Mat scale(const Mat& a, cd c) {
  Mat r;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) r.m[i][j] = c * a.m[i][j];
  return r;
}
Mat dagger(const Mat& a) {
  Mat r;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) r.m[i][j] = std::conj(a.m[j][i]);
  return r;
}
cd trace(const Mat& a) { return a.m[0][0] + a.m[1][1] + a.m[2][2]; }

double norm1(const Mat& a) {  // max column sum
  double best = 0.0;
  for (int j = 0; j < 3; ++j) {
    double s = 0.0;
    for (int i = 0; i < 3; ++i) s += std::abs(a.m[i][j]);
    best = std::max(best, s);
  }
  return best;
}
double normF(const Mat& a) {
  double s = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) s += std::norm(a.m[i][j]);
  return std::sqrt(s);
}

// Leibniz formula: det = sum over permutations of sign * prod a[i][p(i)].
cd det(const Mat& a) {
  static const int perm[6][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1},
                                 {0, 2, 1}, {2, 1, 0}, {1, 0, 2}};
  static const double sgn[6] = {1, 1, 1, -1, -1, -1};
  cd s = 0.0;
  for (int p = 0; p < 6; ++p)
    s += sgn[p] * a.m[0][perm[p][0]] * a.m[1][perm[p][1]] * a.m[2][perm[p][2]];
  return s;
}

// Gauss-Jordan elimination with partial pivoting.
Mat inverse(const Mat& a) {
  cd w[3][6];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      w[i][j] = a.m[i][j];
      w[i][j + 3] = (i == j) ? 1.0 : 0.0;
    }
  for (int c = 0; c < 3; ++c) {
    int piv = c;
    for (int r = c + 1; r < 3; ++r)
      if (std::abs(w[r][c]) > std::abs(w[piv][c])) piv = r;
    if (piv != c)
      for (int j = 0; j < 6; ++j) std::swap(w[c][j], w[piv][j]);
    cd d = w[c][c];
    for (int j = 0; j < 6; ++j) w[c][j] /= d;
    for (int r = 0; r < 3; ++r) {
      if (r == c) continue;
      cd f = w[r][c];
      for (int j = 0; j < 6; ++j) w[r][j] -= f * w[c][j];
    }
  }
  Mat r;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) r.m[i][j] = w[i][j + 3];
  return r;
}

// exp(A) by scaling and squaring of the Taylor series (Higham's classic
// scheme): A/2^s has 1-norm <= 1/2, the series runs until a term is below
// 1e-20 of the sum, and the result is squared s times.
Mat expm(const Mat& a) {
  int s = 0;
  double nrm = norm1(a);
  // (s < 1100 only stops the halving of an infinite norm; every finite
  // double is below 2^1024 and needs fewer halvings)
  while (nrm > 0.5 && s < 1100) {
    nrm *= 0.5;
    ++s;
  }
  Mat b = scale(a, std::ldexp(1.0, -s));
  Mat sum = ident(), term = ident();
  for (int k = 1; k < 60; ++k) {
    term = scale(mul(term, b), 1.0 / k);
    sum = add(sum, term);
    if (normF(term) < 1e-20 * normF(sum)) break;
  }
  for (int i = 0; i < s; ++i) sum = mul(sum, sum);
  return sum;
}

// Gell-Mann matrices lambda_1..lambda_8 (Tr lambda_a lambda_b = 2 delta_ab).
Mat gellmann(int a) {
  Mat r = zero();
  switch (a) {
    case 1: r.m[0][1] = 1.0; r.m[1][0] = 1.0; break;
    case 2: r.m[0][1] = -I1; r.m[1][0] = I1; break;
    case 3: r.m[0][0] = 1.0; r.m[1][1] = -1.0; break;
    case 4: r.m[0][2] = 1.0; r.m[2][0] = 1.0; break;
    case 5: r.m[0][2] = -I1; r.m[2][0] = I1; break;
    case 6: r.m[1][2] = 1.0; r.m[2][1] = 1.0; break;
    case 7: r.m[1][2] = -I1; r.m[2][1] = I1; break;
    case 8: {
      double c = 1.0 / std::sqrt(3.0);
      r.m[0][0] = c; r.m[1][1] = c; r.m[2][2] = -2.0 * c;
      break;
    }
    default: break;
  }
  return r;
}

Mat load(const double* p) {
  Mat r;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) r.m[i][j] = cd(p[2 * (3 * i + j)], p[2 * (3 * i + j) + 1]);
  return r;
}
void store(const Mat& a, double* p) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      p[2 * (3 * i + j)] = a.m[i][j].real();
      p[2 * (3 * i + j) + 1] = a.m[i][j].imag();
    }
}

// ---------------------------------------------------------------- geometry
struct Lat {
  int L[4];
  int64_t V;
  std::vector<int64_t> up, dn;  // up[s*4+mu] = s + e_mu, dn = s - e_mu
};

bool make_lat(const int L[4], Lat& g) {
  g.V = 1;
  for (int mu = 0; mu < 4; ++mu) {
    if (L[mu] < 1) return false;
    g.L[mu] = L[mu];
    g.V *= L[mu];
  }
  g.up.resize(4 * g.V);
  g.dn.resize(4 * g.V);
  for (int64_t s = 0; s < g.V; ++s) {
    int x[4];
    int64_t r = s;
    for (int mu = 0; mu < 4; ++mu) {
      x[mu] = (int)(r % g.L[mu]);
      r /= g.L[mu];
    }
    for (int mu = 0; mu < 4; ++mu) {
      int y[4] = {x[0], x[1], x[2], x[3]};
      y[mu] = (x[mu] + 1) % g.L[mu];
      g.up[4 * s + mu] = y[0] + (int64_t)g.L[0] * (y[1] + (int64_t)g.L[1] * (y[2] + (int64_t)g.L[2] * y[3]));
      y[mu] = (x[mu] - 1 + g.L[mu]) % g.L[mu];
      g.dn[4 * s + mu] = y[0] + (int64_t)g.L[0] * (y[1] + (int64_t)g.L[1] * (y[2] + (int64_t)g.L[2] * y[3]));
    }
  }
  return true;
}

// ------------------------------------------------------------------- Philox
void philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Uniform in (0,1) from two words: a 52-bit integer k plus one half, times 2^-52.
double uniform52(uint32_t hi, uint32_t lo) {
  double k = (double)(hi >> 6) * 67108864.0 + (double)(lo >> 6);
  return (k + 0.5) * (1.0 / 4503599627370496.0);
}

void normals(uint64_t seed, uint32_t step, uint32_t site, uint32_t slot, uint32_t stream,
             int n_pairs, double* out) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int j = 0; j < n_pairs; ++j) {
    uint32_t ctr[4] = {site, step, slot | (stream << 8), (uint32_t)j};
    uint32_t r[4];
    philox(ctr, key, r);
    double u1 = uniform52(r[0], r[1]);
    double u2 = uniform52(r[2], r[3]);
    double rad = std::sqrt(-2.0 * std::log(u1));
    out[2 * j] = rad * std::cos(2.0 * PI * u2);
    out[2 * j + 1] = rad * std::sin(2.0 * PI * u2);
  }
}

const uint32_t STREAM_CL = 0, STREAM_GAUGE = 1, STREAM_HOT = 2;

// ------------------------------------------------------- loops and actions
// One factor of a closed loop: U_mu(site) or its inverse.
struct Factor {
  int64_t site;
  int mu;
  bool inv;
};

// Walk from y along signed directions d (+(mu+1) forward, -(mu+1) backward).
// A forward step contributes U_mu(y) and moves to y+e_mu; a backward step
// moves to y-e_mu and contributes U_mu(y-e_mu)^{-1}.
void walk(const Lat& g, int64_t y, const int* d, int n, std::vector<Factor>& loop) {
  for (int k = 0; k < n; ++k) {
    int mu = std::abs(d[k]) - 1;
    if (d[k] > 0) {
      loop.push_back({y, mu, false});
      y = g.up[4 * y + mu];
    } else {
      y = g.dn[4 * y + mu];
      loop.push_back({y, mu, true});
    }
  }
}

int perm_sign(const int p[4]) {  // sign of a permutation of {0,1,2,3}
  int s = 1;
  for (int i = 0; i < 4; ++i)
    for (int j = i + 1; j < 4; ++j)
      if (p[i] > p[j]) s = -s;
  return s;
}

// All signed direction quadruples (d1,d2,d3,d4) with |d| a permutation of
// (1,2,3,4), with their eps-tilde value: eps-tilde is the Levi-Civita symbol
// of the unsigned directions times the product of the four signs.
struct Quad {
  int d[4];
  int eps;
};
std::vector<Quad> all_quads() {
  std::vector<Quad> q;
  int p[4] = {0, 1, 2, 3};
  do {
    int ps = perm_sign(p);
    for (int sgn = 0; sgn < 16; ++sgn) {
      Quad t;
      int prod = 1;
      for (int k = 0; k < 4; ++k) {
        int s = (sgn >> k) & 1 ? -1 : 1;
        t.d[k] = s * (p[k] + 1);
        prod *= s;
      }
      t.eps = ps * prod;
      q.push_back(t);
    }
  } while (std::next_permutation(p, p + 4));
  return q;
}

// One term of the action: coef * Tr(product of the loop).
struct Term {
  cd coef;
  std::vector<Factor> loop;
};

// The terms of S = S_W - i theta sum_x q_L(x) rooted at site y, minus the
// constant beta per plaquette.  S_W = beta sum_{x,mu<nu} [1 - (Tr P + Tr P^{-1})/6]
// (Wilson action with U^dagger continued to U^{-1});
// q_L(x) = -1/(2^4 32 pi^2) sum eps-tilde Tr[U_{mu nu}(x) U_{rho sigma}(x)]
// with U_{mu nu}(x) = U_mu(x) U_nu(x+mu) U_{-mu}(x+mu+nu) U_{-nu}(x+nu).
void terms_at(const Lat& g, int64_t y, double beta, cd theta, const std::vector<Quad>& quads,
              std::vector<Term>& out) {
  out.clear();
  if (beta != 0.0) {
    for (int mu = 0; mu < 4; ++mu)
      for (int nu = mu + 1; nu < 4; ++nu) {
        Term t;
        t.coef = -beta / 6.0;
        int dp[4] = {mu + 1, nu + 1, -(mu + 1), -(nu + 1)};  // P
        walk(g, y, dp, 4, t.loop);
        out.push_back(t);
        Term u;
        u.coef = -beta / 6.0;
        int dq[4] = {nu + 1, mu + 1, -(nu + 1), -(mu + 1)};  // P^{-1}
        walk(g, y, dq, 4, u.loop);
        out.push_back(u);
      }
  }
  if (theta != 0.0) {
    const double qnorm = -1.0 / (16.0 * 32.0 * PI * PI);
    for (const Quad& qd : quads) {
      Term t;
      t.coef = -I1 * theta * qnorm * (double)qd.eps;
      int a[4] = {qd.d[0], qd.d[1], -qd.d[0], -qd.d[1]};
      int b[4] = {qd.d[2], qd.d[3], -qd.d[2], -qd.d[3]};
      walk(g, y, a, 4, t.loop);
      walk(g, y, b, 4, t.loop);
      out.push_back(t);
    }
  }
}

const Mat& factor_matrix(const Factor& f, const std::vector<Mat>& U, const std::vector<Mat>& Uinv) {
  return f.inv ? Uinv[4 * f.site + f.mu] : U[4 * f.site + f.mu];
}

cd loop_trace(const Term& t, const std::vector<Mat>& U, const std::vector<Mat>& Uinv) {
  Mat p = ident();
  for (const Factor& f : t.loop) p = mul(p, factor_matrix(f, U, Uinv));
  return trace(p);
}

// Product rule for D_a [coef Tr(M_1..M_n)] at position k, D_a the left
// derivative U -> exp(i alpha lambda_a) U.  With R_k = M_{k+1}..M_n M_1..M_{k-1}:
// a factor U_l contributes +coef U_l R_k to X_l, a factor U_l^{-1}
// contributes -coef R_k U_l^{-1}; then D_a(term) = i Tr(lambda_a X_l).
Mat occurrence_contribution(const Term& t, size_t k, const std::vector<Mat>& U,
                            const std::vector<Mat>& Uinv) {
  size_t n = t.loop.size();
  Mat r = ident();
  for (size_t j = 1; j < n; ++j) r = mul(r, factor_matrix(t.loop[(k + j) % n], U, Uinv));
  const Factor& f = t.loop[k];
  if (!f.inv) return scale(mul(U[4 * f.site + f.mu], r), t.coef);
  return scale(mul(r, Uinv[4 * f.site + f.mu]), -t.coef);
}

bool load_links(const Lat& g, const double* p, std::vector<Mat>& U) {
  U.resize(4 * g.V);
  for (int64_t l = 0; l < 4 * g.V; ++l) U[l] = load(p + 18 * l);
  return true;
}
void store_links(const Lat& g, const std::vector<Mat>& U, double* p) {
  for (int64_t l = 0; l < 4 * g.V; ++l) store(U[l], p + 18 * l);
}
std::vector<Mat> inverses(const std::vector<Mat>& U) {
  std::vector<Mat> r(U.size());
#pragma omp parallel for schedule(static)
  for (int64_t l = 0; l < (int64_t)U.size(); ++l) r[l] = inverse(U[l]);
  return r;
}

// Drift X_S of every link: every term rooted at every site, every factor of
// it scattered into its link.  Each thread scatters into its own buffer; the
// buffers are summed in thread order.
void drift_all(const Lat& g, const std::vector<Mat>& U, double beta, cd theta, std::vector<Mat>& X) {
  std::vector<Mat> Uinv = inverses(U);
  std::vector<Quad> quads = all_quads();
  int nth = 1;
#ifdef _OPENMP
  nth = omp_get_max_threads();
#endif
  std::vector<std::vector<Mat>> part(nth);
#pragma omp parallel num_threads(nth)
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    std::vector<Mat>& Xl = part[tid];
    Xl.assign(4 * g.V, zero());
    std::vector<Term> terms;
#pragma omp for schedule(static)
    for (int64_t y = 0; y < g.V; ++y) {
      terms_at(g, y, beta, theta, quads, terms);
      for (const Term& t : terms)
        for (size_t k = 0; k < t.loop.size(); ++k) {
          const Factor& f = t.loop[k];
          int64_t l = 4 * f.site + f.mu;
          Xl[l] = add(Xl[l], occurrence_contribution(t, k, U, Uinv));
        }
    }
  }
  X.assign(4 * g.V, zero());
  for (int t = 0; t < nth; ++t)
    for (int64_t l = 0; l < 4 * g.V; ++l) X[l] = add(X[l], part[t][l]);
}

// Sites whose rooted terms can contain link (s0, mu): every loop of the
// action starts at its root y and stays within the union of two unit squares
// at y, so y = s0 - c where c is a corner offset with at most two nonzero
// components, each +-1.  Returned without duplicates (small lattices wrap).
std::vector<int64_t> candidate_roots(const Lat& g, int64_t s0) {
  std::vector<int64_t> r;
  for (int a = 0; a < 4; ++a)
    for (int sa = -1; sa <= 1; ++sa)
      for (int b = a + 1; b < 5; ++b)
        for (int sb = -1; sb <= 1; ++sb) {
          int64_t y = s0;
          if (sa == 1) y = g.up[4 * y + a];
          if (sa == -1) y = g.dn[4 * y + a];
          if (b < 4) {
            if (sb == 1) y = g.up[4 * y + b];
            if (sb == -1) y = g.dn[4 * y + b];
          }
          r.push_back(y);
        }
  std::sort(r.begin(), r.end());
  r.erase(std::unique(r.begin(), r.end()), r.end());
  return r;
}

// Drift X_S at one link by gathering every occurrence of it in the terms
// rooted at the candidate sites.
Mat drift_one(const Lat& g, const std::vector<Mat>& U, const std::vector<Mat>& Uinv, double beta,
              cd theta, const std::vector<Quad>& quads, int64_t link) {
  int64_t s0 = link / 4;
  int mu0 = (int)(link % 4);
  Mat X = zero();
  std::vector<Term> terms;
  for (int64_t y : candidate_roots(g, s0)) {
    terms_at(g, y, beta, theta, quads, terms);
    for (const Term& t : terms)
      for (size_t k = 0; k < t.loop.size(); ++k)
        if (t.loop[k].site == s0 && t.loop[k].mu == mu0)
          X = add(X, occurrence_contribution(t, k, U, Uinv));
  }
  return X;
}

// The CL update of one link given its drift matrix X_S:
// K_a = -D_a S = -i Tr(lambda_a X_S); A = sum_a i (eps K_a + sqrt(eps) eta_a) lambda_a;
// U' = exp(A) U; U' <- U' / det(U')^(1/3) (principal branch).
Mat cl_update_link(const Mat& Ul, const Mat& X, double eps, uint64_t seed, uint32_t step,
                   int64_t site, int mu) {
  double g[8];
  normals(seed, step, (uint32_t)site, (uint32_t)mu, STREAM_CL, 4, g);
  Mat A = zero();
  for (int a = 1; a <= 8; ++a) {
    Mat la = gellmann(a);
    cd K = -I1 * trace(mul(la, X));
    double eta = std::sqrt(2.0) * g[a - 1];
    A = add(A, scale(la, I1 * (eps * K + std::sqrt(eps) * eta)));
  }
  Mat Un = mul(expm(A), Ul);
  cd d = det(Un);
  return scale(Un, 1.0 / std::pow(d, 1.0 / 3.0));
}

// Gauge-cooling gradient at site x (Sec. 2, eq. "eq:24"):
// f_ax = 2 Tr[lambda_a sum_mu (U_{x,mu} U_{x,mu}^+ - U_{x-mu,mu}^+ U_{x-mu,mu})].
void cool_gradient_all(const Lat& g, const std::vector<Mat>& U, std::vector<double>& f) {
  f.assign(8 * g.V, 0.0);
#pragma omp parallel for schedule(static)
  for (int64_t x = 0; x < g.V; ++x) {
    Mat G = zero();
    for (int mu = 0; mu < 4; ++mu) {
      const Mat& Uf = U[4 * x + mu];
      const Mat& Ub = U[4 * g.dn[4 * x + mu] + mu];
      G = add(G, sub(mul(Uf, dagger(Uf)), mul(dagger(Ub), Ub)));
    }
    for (int a = 1; a <= 8; ++a) f[8 * x + a - 1] = (2.0 * trace(mul(gellmann(a), G))).real();
  }
}

// One sweep: Omega_x = exp(-eps alpha f_ax lambda_a) at every site, then
// U_{x,mu} <- Omega_x U_{x,mu} Omega_{x+mu}^{-1} for all links at once.
void cool_sweep_all(const Lat& g, std::vector<Mat>& U, double eps, double alpha) {
  std::vector<double> f;
  cool_gradient_all(g, U, f);
  std::vector<Mat> Om(g.V), Omi(g.V);
#pragma omp parallel for schedule(static)
  for (int64_t x = 0; x < g.V; ++x) {
    Mat H = zero();
    for (int a = 1; a <= 8; ++a) H = add(H, scale(gellmann(a), -eps * alpha * f[8 * x + a - 1]));
    Om[x] = expm(H);
    Omi[x] = inverse(Om[x]);
  }
  std::vector<Mat> Un(U.size());
#pragma omp parallel for schedule(static)
  for (int64_t x = 0; x < g.V; ++x)
    for (int mu = 0; mu < 4; ++mu)
      Un[4 * x + mu] = mul(mul(Om[x], U[4 * x + mu]), Omi[g.up[4 * x + mu]]);
  U.swap(Un);
}

// Unitarity norm averaged over links: (1/3) Tr U U^+.
double unitarity_norm(const Lat& g, const std::vector<Mat>& U) {
  double s = 0.0;
  for (int64_t l = 0; l < 4 * g.V; ++l) s += trace(mul(U[l], dagger(U[l]))).real() / 3.0;
  return s / (4.0 * g.V);
}

std::vector<cd> qdensity_all(const Lat& g, const std::vector<Mat>& U) {
  std::vector<Mat> Uinv = inverses(U);
  std::vector<Quad> quads = all_quads();
  std::vector<cd> q(g.V);
  const double qnorm = -1.0 / (16.0 * 32.0 * PI * PI);
#pragma omp parallel for schedule(static)
  for (int64_t y = 0; y < g.V; ++y) {
    std::vector<Term> terms;
    terms_at(g, y, 0.0, 1.0, quads, terms);  // theta = 1: coef = -i qnorm eps
    cd s = 0.0;
    for (size_t i = 0; i < terms.size(); ++i) s += (double)quads[i].eps * loop_trace(terms[i], U, Uinv);
    q[y] = qnorm * s;
  }
  return q;
}

void observables(const Lat& g, const std::vector<Mat>& U, double beta, cd theta, double* out) {
  std::vector<Mat> Uinv = inverses(U);
  cd plaq = 0.0, trP = 0.0;
  for (int64_t x = 0; x < g.V; ++x)
    for (int mu = 0; mu < 4; ++mu)
      for (int nu = mu + 1; nu < 4; ++nu) {
        Term t;
        int dp[4] = {mu + 1, nu + 1, -(mu + 1), -(nu + 1)};
        walk(g, x, dp, 4, t.loop);
        Term u;
        int dq[4] = {nu + 1, mu + 1, -(nu + 1), -(mu + 1)};
        walk(g, x, dq, 4, u.loop);
        cd tp = loop_trace(t, U, Uinv), tq = loop_trace(u, U, Uinv);
        plaq += tp / 3.0;
        trP += tp + tq;
      }
  double nplaq = 6.0 * g.V;
  cd SW = beta * nplaq - beta / 6.0 * trP;
  std::vector<cd> q = qdensity_all(g, U);
  cd Q = 0.0;
  for (cd v : q) Q += v;
  cd S = SW - I1 * theta * Q;
  double maxdev = 0.0;
  for (const Mat& m : U) maxdev = std::max(maxdev, std::abs(det(m) - 1.0));
  out[0] = plaq.real() / nplaq;
  out[1] = plaq.imag() / nplaq;
  out[2] = unitarity_norm(g, U);
  out[3] = Q.real();
  out[4] = Q.imag();
  out[5] = SW.real();
  out[6] = SW.imag();
  out[7] = S.real();
  out[8] = S.imag();
  out[9] = maxdev;
}

void cl_step_all(const Lat& g, std::vector<Mat>& U, double beta, cd theta, double eps,
                 uint64_t seed, uint32_t step) {
  std::vector<Mat> X;
  drift_all(g, U, beta, theta, X);
  std::vector<Mat> Un(U.size());
#pragma omp parallel for schedule(static)
  for (int64_t l = 0; l < 4 * g.V; ++l)
    Un[l] = cl_update_link(U[l], X[l], eps, seed, step, l / 4, (int)(l % 4));
  U.swap(Un);
}

// Sec. 4: alpha_ad = alpha / D with D_0 = 1, D_1 = (1/3)<Tr U U^+>,
// D_2 = <|f_ax|>_{a,x} (or its RMS variant).  Sweep-count rule: at least
// n_min and at most n_max sweeps; stop once the unitarity norm has stopped
// decreasing by more than tol_rel of its distance from 1, or once that
// distance is below d_floor; skip when D < d_guard.  forced_sweeps >= 0 makes
// the count exactly forced_sweeps.
int cool_all(const Lat& g, std::vector<Mat>& U, const or_cool_params& p, or_cool_report& rep) {
  rep.sweeps = 0;
  rep.alpha_ad_last = 0.0;
  double un_prev = 0.0;
  for (int k = 0;; ++k) {
    std::vector<double> f;
    cool_gradient_all(g, U, f);
    double un = unitarity_norm(g, U);
    double sabs = 0.0, ssq = 0.0;
    for (double v : f) {
      sabs += std::fabs(v);
      ssq += v * v;
    }
    double D = 1.0;
    if (p.mode == OR_D1) D = un;
    if (p.mode == OR_D2_MEANABS) D = sabs / (8.0 * g.V);
    if (p.mode == OR_D2_RMS) D = std::sqrt(ssq / (8.0 * g.V));
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
    cool_sweep_all(g, U, p.eps, alpha_ad);
    rep.alpha_ad_last = alpha_ad;
    rep.sweeps++;
    un_prev = un;
  }
  return 0;
}

}  // namespace

// ====================================================================== C API
extern "C" {

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  philox(ctr, key, out);
}

void or_normals(uint64_t seed, uint32_t step, uint32_t site, uint32_t slot, uint32_t stream,
                int n_pairs, double* out) {
  normals(seed, step, site, slot, stream, n_pairs, out);
}

void or_normals_sites(uint64_t seed, uint32_t step, uint32_t site0, int nsites, uint32_t slot,
                      uint32_t stream, int n_pairs, double* out) {
  for (int i = 0; i < nsites; ++i)
    normals(seed, step, site0 + (uint32_t)i, slot, stream, n_pairs, out + (size_t)i * 2 * n_pairs);
}

void or_gellmann(int a, double* out18) { store(gellmann(a), out18); }
void or_expm(const double* a18, double* out18) { store(expm(load(a18)), out18); }
void or_inverse(const double* a18, double* out18) { store(inverse(load(a18)), out18); }
void or_det(const double* a18, double* out2) {
  cd d = det(load(a18));
  out2[0] = d.real();
  out2[1] = d.imag();
}

int or_cold_start(const int L[4], double* U) {
  Lat g;
  if (!make_lat(L, g)) return -1;
  for (int64_t l = 0; l < 4 * g.V; ++l) store(ident(), U + 18 * l);
  return 0;
}

// Haar SU(3): Gram-Schmidt on the rows of a complex Gaussian matrix gives a
// Haar U(3) matrix; dividing by the principal cube root of its determinant
// maps it to SU(3) (left-invariance is kept, so the result is Haar on SU(3)).
int or_hot_start(const int L[4], uint64_t seed, double* U) {
  Lat g;
  if (!make_lat(L, g)) return -1;
#pragma omp parallel for schedule(static)
  for (int64_t l = 0; l < 4 * g.V; ++l) {
    double z[18];
    normals(seed, 0, (uint32_t)(l / 4), (uint32_t)(l % 4), STREAM_HOT, 9, z);
    cd row[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) row[i][j] = cd(z[2 * (3 * i + j)], z[2 * (3 * i + j) + 1]);
    for (int i = 0; i < 3; ++i) {
      for (int k = 0; k < i; ++k) {  // row_i -= <row_k, row_i> row_k
        cd ip = 0.0;
        for (int j = 0; j < 3; ++j) ip += std::conj(row[k][j]) * row[i][j];
        for (int j = 0; j < 3; ++j) row[i][j] -= ip * row[k][j];
      }
      double n = 0.0;
      for (int j = 0; j < 3; ++j) n += std::norm(row[i][j]);
      n = std::sqrt(n);
      for (int j = 0; j < 3; ++j) row[i][j] /= n;
    }
    Mat m;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) m.m[i][j] = row[i][j];
    cd d = det(m);
    store(scale(m, 1.0 / std::pow(d, 1.0 / 3.0)), U + 18 * l);
  }
  return 0;
}

int or_gauge_transform(const int L[4], const double* Om, double* U) {
  Lat g;
  if (!make_lat(L, g)) return -1;
  std::vector<Mat> O(g.V), Oi(g.V), Uv;
  for (int64_t x = 0; x < g.V; ++x) {
    O[x] = load(Om + 18 * x);
    Oi[x] = inverse(O[x]);
  }
  load_links(g, U, Uv);
  for (int64_t x = 0; x < g.V; ++x)
    for (int mu = 0; mu < 4; ++mu)
      store(mul(mul(O[x], Uv[4 * x + mu]), Oi[g.up[4 * x + mu]]), U + 18 * (4 * x + mu));
  return 0;
}

int or_random_gauge(const int L[4], uint64_t seed, double sigma, double* U) {
  Lat g;
  if (!make_lat(L, g)) return -1;
  std::vector<double> Om(18 * g.V);
  for (int64_t x = 0; x < g.V; ++x) {
    double r[8];
    normals(seed, 0, (uint32_t)x, 0, STREAM_GAUGE, 4, r);
    Mat A = zero();
    for (int a = 1; a <= 8; ++a) {
      cd w = I1 * sigma * r[a - 1];  // omega_a = i * sigma * g_a
      A = add(A, scale(gellmann(a), I1 * w));
    }
    store(expm(A), Om.data() + 18 * x);
  }
  return or_gauge_transform(L, Om.data(), U);
}

int or_observables(const int L[4], const double* U, double beta, double th_re, double th_im,
                   double* out10) {
  Lat g;
  if (!make_lat(L, g)) return -1;
  std::vector<Mat> Uv;
  load_links(g, U, Uv);
  observables(g, Uv, beta, cd(th_re, th_im), out10);
  return 0;
}

int or_qdensity(const int L[4], const double* U, double* q) {
  Lat g;
  if (!make_lat(L, g)) return -1;
  std::vector<Mat> Uv;
  load_links(g, U, Uv);
  std::vector<cd> qv = qdensity_all(g, Uv);
  for (int64_t x = 0; x < g.V; ++x) {
    q[2 * x] = qv[x].real();
    q[2 * x + 1] = qv[x].imag();
  }
  return 0;
}

int or_action(const int L[4], const double* U, double beta, double th_re, double th_im,
              double* out2) {
  double o[10];
  int r = or_observables(L, U, beta, th_re, th_im, o);
  out2[0] = o[7];
  out2[1] = o[8];
  return r;
}

int or_drift(const int L[4], const double* U, double beta, double th_re, double th_im, double* X) {
  Lat g;
  if (!make_lat(L, g)) return -1;
  std::vector<Mat> Uv, Xv;
  load_links(g, U, Uv);
  drift_all(g, Uv, beta, cd(th_re, th_im), Xv);
  store_links(g, Xv, X);
  return 0;
}

int or_drift_at(const int L[4], const double* U, double beta, double th_re, double th_im, int n,
                const int64_t* links, double* X) {
  Lat g;
  if (!make_lat(L, g) || n < 0) return -1;
  for (int i = 0; i < n; ++i)
    if (links[i] < 0 || links[i] >= 4 * g.V) return -2;
  std::vector<Mat> Uv;
  load_links(g, U, Uv);
  std::vector<Mat> Uinv = inverses(Uv);
  std::vector<Quad> quads = all_quads();
#pragma omp parallel for schedule(dynamic)
  for (int i = 0; i < n; ++i)
    store(drift_one(g, Uv, Uinv, beta, cd(th_re, th_im), quads, links[i]), X + 18 * i);
  return 0;
}

int or_cl_step(const int L[4], double* U, double beta, double th_re, double th_im, double eps,
               uint64_t seed, uint32_t step) {
  Lat g;
  if (!make_lat(L, g)) return -1;
  std::vector<Mat> Uv;
  load_links(g, U, Uv);
  cl_step_all(g, Uv, beta, cd(th_re, th_im), eps, seed, step);
  store_links(g, Uv, U);
  return 0;
}

// Adaptive Langevin step size (the runaway control that accompanies gauge
// cooling): with the drift K_a = -D_a S = -i Tr(lambda_a X_S) of every link,
// K_max = max over links of (sum_a |K_a|^2)^(1/2); the step runs with
// eps_n = eps * min(1, k_ref / K_max) in both the drift and the noise term
// (k_ref <= 0: eps_n = eps).
int or_cl_step_adaptive(const int L[4], double* U, double beta, double th_re, double th_im,
                        double eps, double k_ref, uint64_t seed, uint32_t step, double* eps_used,
                        double* k_max) {
  Lat g;
  if (!make_lat(L, g)) return -1;
  std::vector<Mat> Uv;
  load_links(g, U, Uv);
  std::vector<Mat> X;
  drift_all(g, Uv, beta, cd(th_re, th_im), X);
  double kmax = 0.0;
  for (const Mat& x : X) {
    double k2 = 0.0;
    for (int a = 1; a <= 8; ++a) k2 += std::norm(-I1 * trace(mul(gellmann(a), x)));
    kmax = std::max(kmax, std::sqrt(k2));
  }
  double e = eps;
  if (k_ref > 0.0 && kmax > k_ref) e = eps * (k_ref / kmax);
  cl_step_all(g, Uv, beta, cd(th_re, th_im), e, seed, step);
  store_links(g, Uv, U);
  if (eps_used) *eps_used = e;
  if (k_max) *k_max = kmax;
  return 0;
}

int or_cl_step_at(const int L[4], const double* U, double beta, double th_re, double th_im,
                  double eps, uint64_t seed, uint32_t step, int n, const int64_t* links,
                  double* Unew) {
  std::vector<double> X(18 * (size_t)std::max(n, 0));
  int r = or_drift_at(L, U, beta, th_re, th_im, n, links, X.data());
  if (r) return r;
  for (int i = 0; i < n; ++i) {
    Mat Ul = load(U + 18 * links[i]);
    store(cl_update_link(Ul, load(X.data() + 18 * i), eps, seed, step, links[i] / 4,
                         (int)(links[i] % 4)),
          Unew + 18 * i);
  }
  return 0;
}

// One CL step followed by one cooling sweep at fixed alpha_ad, evaluated
// only at the chosen links: the post-step links that the cooling
// transformations at x and x+mu need (the links at and into those sites)
// are built from their own drifts, then Omega_x U'_{x,mu} Omega_{x+mu}^{-1}.
int or_step_sweep_at(const int L[4], const double* U, double beta, double th_re, double th_im,
                     double eps, uint64_t seed, uint32_t step, double eps_cool, double alpha_ad,
                     int n, const int64_t* links, double* after_step, double* after_sweep) {
  Lat g;
  if (!make_lat(L, g) || n < 0) return -1;
  for (int i = 0; i < n; ++i)
    if (links[i] < 0 || links[i] >= 4 * g.V) return -2;
  std::vector<Mat> Uv;
  load_links(g, U, Uv);
  std::vector<Mat> Uinv = inverses(Uv);
  std::vector<Quad> quads = all_quads();
  cd theta(th_re, th_im);
  auto stepped = [&](int64_t l) {
    Mat X = drift_one(g, Uv, Uinv, beta, theta, quads, l);
    return cl_update_link(Uv[l], X, eps, seed, step, l / 4, (int)(l % 4));
  };
  auto omega = [&](int64_t y, bool inv) {
    Mat G = zero();
    for (int mu = 0; mu < 4; ++mu) {
      Mat Uf = stepped(4 * y + mu);
      Mat Ub = stepped(4 * g.dn[4 * y + mu] + mu);
      G = add(G, sub(mul(Uf, dagger(Uf)), mul(dagger(Ub), Ub)));
    }
    Mat H = zero();
    for (int a = 1; a <= 8; ++a) {
      double fa = (2.0 * trace(mul(gellmann(a), G))).real();
      H = add(H, scale(gellmann(a), -eps_cool * alpha_ad * fa));
    }
    Mat O = expm(H);
    return inv ? inverse(O) : O;
  };
#pragma omp parallel for schedule(dynamic)
  for (int i = 0; i < n; ++i) {
    int64_t l = links[i], x = l / 4;
    int mu = (int)(l % 4);
    Mat Us = stepped(l);
    store(Us, after_step + 18 * i);
    store(mul(mul(omega(x, false), Us), omega(g.up[4 * x + mu], true)), after_sweep + 18 * i);
  }
  return 0;
}

int or_cool_gradient(const int L[4], const double* U, double* f) {
  Lat g;
  if (!make_lat(L, g)) return -1;
  std::vector<Mat> Uv;
  load_links(g, U, Uv);
  std::vector<double> fv;
  cool_gradient_all(g, Uv, fv);
  std::memcpy(f, fv.data(), sizeof(double) * fv.size());
  return 0;
}

int or_cool_sweep(const int L[4], double* U, double eps, double alpha_ad) {
  Lat g;
  if (!make_lat(L, g)) return -1;
  std::vector<Mat> Uv;
  load_links(g, U, Uv);
  cool_sweep_all(g, Uv, eps, alpha_ad);
  store_links(g, Uv, U);
  return 0;
}

int or_cool(const int L[4], double* U, const or_cool_params* p, or_cool_report* rep) {
  Lat g;
  if (!make_lat(L, g) || !p) return -1;
  std::vector<Mat> Uv;
  load_links(g, U, Uv);
  or_cool_report r;
  cool_all(g, Uv, *p, r);
  store_links(g, Uv, U);
  if (rep) *rep = r;
  return 0;
}

int or_trajectory(const int L[4], double* U, double beta, double th_re, double th_im, double eps,
                  uint64_t seed, uint32_t step0, int n_steps, const or_cool_params* cool,
                  int obs_every, double* obs_out) {
  Lat g;
  if (!make_lat(L, g) || n_steps < 0) return -1;
  std::vector<Mat> Uv;
  load_links(g, U, Uv);
  cd theta(th_re, th_im);
  int rec = 0;
  for (int i = 0; i < n_steps; ++i) {
    cl_step_all(g, Uv, beta, theta, eps, seed, step0 + (uint32_t)i);
    or_cool_report r = {0, 0.0, 0.0, 0.0};
    if (cool) cool_all(g, Uv, *cool, r);
    if (obs_every > 0 && (i + 1) % obs_every == 0 && obs_out) {
      double* o = obs_out + 14 * rec++;
      observables(g, Uv, beta, theta, o);
      o[10] = r.sweeps;
      o[11] = r.alpha_ad_last;
      o[12] = r.un_before;
      o[13] = r.un_after;
    }
  }
  store_links(g, Uv, U);
  return 0;
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
