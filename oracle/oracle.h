/*
 * oracle.h -- plain FP64 CPU oracle for complex Langevin (CL) dynamics of
 * SU(3) Yang-Mills with a clover theta-term and adaptive gauge cooling
 * (Bongiovanni, Aarts, Seiler, Sexty, Stamatescu, "Adaptive gauge cooling for
 * complex Langevin dynamics", LATTICE 2013, arXiv:1311.1056).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the independent checker of the
 * CUDA path: only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark may load it.  It shares no code, header, table or constant
 * with the CUDA library and never calls it.
 *
 * Conventions (all arrays are caller-owned host memory, FP64):
 *   L[4]      lattice extents, periodic in every direction, each >= 1.
 *   site      s = x0 + L0*(x1 + L1*(x2 + L2*x3)); direction mu = 0..3 is x_mu.
 *   links     AoS [site][mu][row][col]{re,im}: V*4*18 doubles.
 *   matrices  one 3x3 complex matrix = 18 doubles, row-major {re,im}.
 *   Omega     one matrix per site: V*18 doubles.
 * Every function returns 0 on success and a negative value on bad arguments.
 */
#ifndef CL_ORACLE_H
#define CL_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

/* Philox4x32-10 of Salmon, Moraes, Dror, Shaw (SC'11): out = philox(ctr, key). */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* 2*n_pairs standard normal numbers for one (seed, step, site, slot, stream)
 * key: counter (site, step, slot | stream<<8, j), j = 0..n_pairs-1, each
 * counter giving one Box-Muller pair. */
void or_normals(uint64_t seed, uint32_t step, uint32_t site, uint32_t slot,
                uint32_t stream, int n_pairs, double* out);
/* The same for the sites site0 .. site0 + nsites - 1: out[(i * 2 * n_pairs) + k]. */
void or_normals_sites(uint64_t seed, uint32_t step, uint32_t site0, int nsites, uint32_t slot,
                      uint32_t stream, int n_pairs, double* out);

/* 3x3 primitives (used by the pins that check the oracle's own building blocks). */
void or_gellmann(int a /* 1..8 */, double* out18);
void or_expm(const double* a18, double* out18);
void or_inverse(const double* a18, double* out18);
void or_det(const double* a18, double* out2);

/* Starts.  cold: U = 1.  hot: Haar SU(3) per link (Philox stream 2).
 * random_gauge: U_{x,mu} <- Om_x U Om_{x+mu}^{-1} with Om_x = exp(i w_a lambda_a),
 * w_a = i*sigma*g_a (g standard normal, Philox stream 1). */
int or_cold_start(const int L[4], double* U);
int or_hot_start(const int L[4], uint64_t seed, double* U);
int or_random_gauge(const int L[4], uint64_t seed, double sigma, double* U);
/* U_{x,mu} <- Om_x U_{x,mu} Om_{x+mu}^{-1} for caller-given Om (V*18). */
int or_gauge_transform(const int L[4], const double* Om, double* U);

/* Observables (out[0..9]): plaquette re, im; unitarity norm; Q re, im;
 * S_W re, im; S = S_W - i theta Q re, im; max |det U - 1|. */
int or_observables(const int L[4], const double* U, double beta,
                   double theta_re, double theta_im, double* out10);
/* q_L(x) per site, complex (V*2), by the brute-force signed sum. */
int or_qdensity(const int L[4], const double* U, double* q);
/* The action S = S_W - i theta sum_x q_L(x) (out2 = re, im). */
int or_action(const int L[4], const double* U, double beta,
              double theta_re, double theta_im, double* out2);

/* Drift matrix X_S of every link, D_a S = i Tr(lambda_a X_S) (4V*18). */
int or_drift(const int L[4], const double* U, double beta,
             double theta_re, double theta_im, double* X);
/* The same matrix at n chosen links (link id = site*4 + mu), by gathering
 * the action terms that contain each link. */
int or_drift_at(const int L[4], const double* U, double beta,
                double theta_re, double theta_im, int n, const int64_t* links,
                double* X);

/* One CL step, all links at once (Euler):
 * U' = exp(i lambda_a (eps K_a + sqrt(eps) eta_a)) U, K_a = -D_a S,
 * eta_a = sqrt(2) * normal from Philox stream 0, then U' <- U' / det(U')^(1/3). */
int or_cl_step(const int L[4], double* U, double beta, double theta_re,
               double theta_im, double eps, uint64_t seed, uint32_t step);
/* The CL step with the adaptive step size: K_max = max over links of
 * (sum_a |K_a|^2)^(1/2), K_a = -i Tr(lambda_a X_S); the step uses
 * eps_n = eps * min(1, k_ref / K_max) (k_ref <= 0: eps).  eps_used, k_max
 * may be NULL. */
int or_cl_step_adaptive(const int L[4], double* U, double beta, double theta_re,
                        double theta_im, double eps, double k_ref, uint64_t seed, uint32_t step,
                        double* eps_used, double* k_max);
/* The updated matrices U' of n chosen links only (the input lattice is not
 * modified), for sampled checks on large lattices. */
int or_cl_step_at(const int L[4], const double* U, double beta,
                  double theta_re, double theta_im, double eps, uint64_t seed,
                  uint32_t step, int n, const int64_t* links, double* Unew);

/* One CL step then one cooling sweep with fixed alpha_ad, evaluated only at
 * n chosen links (for sampled checks on large lattices): after_step gets U'
 * and after_sweep Omega_x U' Omega_{x+mu}^{-1}, 18 doubles per link. */
int or_step_sweep_at(const int L[4], const double* U, double beta, double theta_re,
                     double theta_im, double eps, uint64_t seed, uint32_t step, double eps_cool,
                     double alpha_ad, int n, const int64_t* links, double* after_step,
                     double* after_sweep);

/* Gauge-cooling gradient f_ax = 2 Tr[lambda_a sum_mu (U U^+ - U^+_{x-mu} U_{x-mu})] (V*8). */
int or_cool_gradient(const int L[4], const double* U, double* f);
/* One cooling sweep with step eps*alpha_ad, all links at once. */
int or_cool_sweep(const int L[4], double* U, double eps, double alpha_ad);

enum { OR_D0 = 0, OR_D1 = 1, OR_D2_MEANABS = 2, OR_D2_RMS = 3 };
typedef struct {
  double eps, alpha;
  int mode;             /* OR_D0 .. OR_D2_RMS */
  int n_min, n_max;     /* sweep-count bounds of the adaptive stop rule */
  double tol_rel;       /* stop when (UN_prev - UN) < tol_rel * (UN_prev - 1) */
  double d_floor;       /* stop when UN - 1 < d_floor */
  double d_guard;       /* skip cooling when D < d_guard */
  int forced_sweeps;    /* >= 0: exactly this many sweeps (parity mode) */
} or_cool_params;
typedef struct {
  int sweeps;
  double alpha_ad_last, un_before, un_after;
} or_cool_report;
int or_cool(const int L[4], double* U, const or_cool_params* p, or_cool_report* rep);

/* n_steps of [CL step, cooling]; after every obs_every-th step the 10
 * observables of or_observables and 4 report entries (sweeps, alpha_ad_last,
 * un_before, un_after) are appended to obs_out (14 doubles per record).
 * cool may be NULL (no cooling).  The step counter starts at step0. */
int or_trajectory(const int L[4], double* U, double beta, double theta_re,
                  double theta_im, double eps, uint64_t seed, uint32_t step0,
                  int n_steps, const or_cool_params* cool, int obs_every,
                  double* obs_out);

/* ---- SU(2) Polyakov chain (Sec. 3, eq. "eq:s"): S = -(beta/2) Tr(U_1 ... U_N),
 * complex beta = (br, bi).  A chain is n links, each a 2x2 complex matrix,
 * row-major {re,im} (8 doubles).  Link k joins sites k and k+1 (periodic);
 * the gauge transformation at site k is U_k <- Om_k U_k, U_{k-1} <- U_{k-1} Om_k^{-1}. */
void or_pauli(int a /* 1..3 */, double* out8);
int or_pc_cold(int n, double* U);
/* U_k <- Om_k U_k Om_{k+1}^{-1}, Om_k = exp(i w_a sigma_a), w_a = i sigma g_a (Philox stream 4). */
int or_pc_random_gauge(int n, uint64_t seed, double sigma, double* U);
int or_pc_action(int n, const double* U, double br, double bi, double* out2);
/* K_a(k) = -D_a S (3 complex per link: 6n doubles). */
int or_pc_drift(int n, const double* U, double br, double bi, double* K);
/* U_k' = exp(i sigma_a (eps K_a + sqrt(eps) eta_a)) U_k, eta = sqrt(2) normal
 * (Philox stream 3, counter (k, step, 3 << 8, j)), then U' / det(U')^(1/2). */
int or_pc_step(int n, double* U, double br, double bi, double eps, uint64_t seed, uint32_t step);
/* f_ak = 2 Tr[sigma_a (U_k U_k^+ - U_{k-1}^+ U_{k-1})] (3n doubles). */
int or_pc_cool_gradient(int n, const double* U, double* f);
int or_pc_cool_sweep(int n, double* U, double eps, double alpha_ad);
/* The adaptive cooling call with the SU(3) stop rule; D_1 = (1/2)<Tr U U^+>, D_2 = <|f_ak|>. */
int or_pc_cool(int n, double* U, const or_cool_params* p, or_cool_report* rep);
/* (1/2) Tr(U_1 ... U_N) re, im; (1/N) sum (1/2) Tr U U^+; max |det U - 1|. */
int or_pc_observables(int n, const double* U, double* out4);
/* n_steps of [CL step, cooling (cool may be NULL)]; rec (may be NULL) gets
 * the 4 observables and the sweep count after every step (5 doubles). */
int or_pc_trajectory(int n, double* U, double br, double bi, double eps, uint64_t seed,
                     uint32_t step0, int n_steps, const or_cool_params* cool, double* rec);

/* Number of OpenMP threads the oracle uses. */
int or_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
