// launch.h -- host-side launchers of the CL / gauge-cooling kernels (internal
// interface between the C-ABI runtime and the kernel translation units).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace clgc {

// Launch families whose block size is tunable (cl_autotune).  Every thread
// of these kernels owns one site (or one link), so the block size changes
// neither the arithmetic nor its order; the reductions keep a fixed shape.
enum { TUNE_CLOVER = 0, TUNE_FORCE = 1, TUNE_UPDATE = 2, TUNE_OMEGA = 3, TUNE_APPLY = 4, NTUNE = 5 };
const int TUNE_DEFAULT_BLOCK = 128;
const int TUNE_MAX_BLOCK = 256;  // the launch bound of the tunable kernels

struct GeoH {
  int L[4];
  int V;
  int blk[NTUNE];  // threads per block per family; 0 = TUNE_DEFAULT_BLOCK
};

inline int block_of(const GeoH& h, int fam) { return h.blk[fam] > 0 ? h.blk[fam] : TUNE_DEFAULT_BLOCK; }

// Per-lattice step state, resident on the device so that captured graphs
// replay with fresh noise and the adaptive step size is decided on the GPU.
struct StepDev {
  uint32_t step;                 // Philox step counter (the noise key's step word)
  uint32_t pad;
  double eps_n, sqrt_eps_n;      // step size of the current step (adaptive mode)
  double t;                      // Langevin time: sum of the step sizes taken
  double kmax;                   // K_max of the last adaptive step
  unsigned long long kmax2_bits; // running max of |K|^2 (non-negative doubles order as integers)
};

// Packed results of the cooling rule, resident on the device.
struct CoolState {
  double alpha_ad;       // alpha / D of the sweep about to run
  double alpha_ad_last;  // of the last applied sweep
  double un_prev;        // unitarity norm before the last applied sweep
  double un_before, un_after, D;
  int sweeps, done, k, nonfinite;
};

struct CoolArgs {
  double eps, alpha, tol_rel, d_floor, d_guard;
  int mode, n_min, n_max, forced_sweeps;
};

// Observables accumulated on the device (FP64), one record per call.
struct ObsOut {
  double plaq_re, plaq_im, un, q_re, q_im, sw_re, sw_im, s_re, s_im, max_det_dev;
  double nonfinite;
};

enum { NQ_OBS = 9, NQ_COOL = 4, RED_THREADS = 128, RED_MAX_BLOCKS = 1216 };

// One chain of a fused batch (the ensemble kernels below): its geometry (the
// fields of lattice.cuh's Geo), device buffers and per-chain parameters.  U
// holds the links the step starts from; the update writes Un, and cooling
// then works on Un (the runtime swaps the two after the step).
struct ChainDesc {
  int L[4], stride[4], V;
  void *U, *Un, *Ui, *Pq, *Dq, *F, *C, *Gq, *f, *Om, *Omi;
  double* partials;
  double* arec;             // the single-pass apply's tile records
  CoolState* cs;
  StepDev* sd;
  double beta, sre, sim;    // coupling; clover scale -i theta kappa = sre + i sim
  double eps, sqrt_eps, k_ref;
  uint64_t seed;
  CoolArgs ca;
};
// One block of a fused launch: chain index and the block index that a
// launch for that chain alone would have had.
struct WorkItem {
  int chain, vb;
};
// Fused kernel families (one launch over the work list's blocks of every
// chain; block size ENS_BLOCK, the reductions' RED_THREADS).
enum {
  ENS_INVERSE = 0,      // link inverses, 4 directions
  ENS_PLAQ = 1,         // plaquettes, 6 planes
  ENS_CLOVER = 2,       // clover field (theta != 0 chains)
  ENS_FORCE_WILSON = 3, // drift contributions, theta = 0 chains
  ENS_FORCE_THETA = 4,  // drift contributions, theta != 0 chains (FP64: two kernels)
  ENS_UPDATE = 5,       // gather + update, fixed step size
  ENS_DRIFTMAX = 6,     // gather, drift into Ui, max |K|^2 (adaptive step size)
  ENS_UPDATE_X = 7,     // update from the drift in Ui (adaptive step size)
  ENS_COOL_GRAD = 8,    // gradient + rule sums (RED_THREADS blocks, grid-stride per chain)
  ENS_COOL_OMEGA = 9,   // Omega, Omega^{-1}
  ENS_COOL_APPLY = 10,  // apply, 4 directions
  ENS_COOL_GRAD_OMEGA = 11, // single-pass sweeps (D_0 / D_1): gradient + Omega
  ENS_COOL_APPLY_UN = 12,   // single-pass sweeps: apply per tile + norm sums (one item per tile)
  ENS_NFAM = 13
};
const int ENS_BLOCK = 128;

int reduce_blocks(int V);  // number of per-block partial records for V sites

// prec: 0 = FP64 links, 1 = FP32 links.  All pointers are device pointers;
// link fields are SoA (see lattice.cuh), `partials` holds reduce_blocks(V)
// records of NQ_* doubles.
cudaError_t launch_cold(int prec, const GeoH& g, void* U, cudaStream_t st);
cudaError_t launch_hot(int prec, const GeoH& g, void* U, uint64_t seed, cudaStream_t st);
// Omega_x = exp(-sigma g_a lambda_a) per site (Philox stream 1) into Om/Omi.
cudaError_t launch_gauge_omega(int prec, const GeoH& g, void* Om, void* Omi, uint64_t seed,
                               double sigma, cudaStream_t st);
cudaError_t launch_aos_to_soa(int prec, const GeoH& g, const double* aos, void* U, int nplanes,
                              cudaStream_t st);
cudaError_t launch_soa_to_aos(int prec, const GeoH& g, const void* U, double* aos, int nplanes,
                              cudaStream_t st);
// The CL step (k_update.cuh): link inverses Ui; plaquettes P and D = P - P^{-1}
// (six planes); the clover field F^ = scale * F_{mu nu}(x) built from the D's;
// the per-plaquette drift contributions C (24 planes: 4 links x 6 planes);
// then per link the gather of its six contributions followed by the update
// (mode 0) or by storing the drift matrix X_S (mode 1).
// Lets the double-float link-algebra kernels take their shared-memory matrix
// workspace (up to 5 x 144 B per thread); called before the first DF64 launch.
cudaError_t prepare_df64_kernels();
cudaError_t launch_noise_sample(int prec, int site0, int n, uint64_t seed, uint32_t step, int mu, double* out,
                                cudaStream_t st);
cudaError_t launch_link_inverse(int prec, const GeoH& g, const void* U, void* Ui, cudaStream_t st);
cudaError_t launch_plaq(int prec, const GeoH& g, const void* U, const void* Ui, void* Pq, void* Dq,
                        cudaStream_t st);
cudaError_t launch_clover_rot(int prec, const GeoH& g, const void* U, const void* Ui, const void* Dq,
                              void* F, double scale_re, double scale_im, cudaStream_t st);
// (theta != 0 runs two kernels, parking partial sums of the transported dual
// fields in Gq, six planes.)
cudaError_t launch_plaq_force(int prec, bool theta, const GeoH& g, const void* U, const void* Ui,
                              const void* Pq, const void* Dq, const void* F, void* Gq, void* C,
                              double beta, cudaStream_t st);
// mode 0: update from the gathered drift (eps, or the device step size when
// sd_adaptive); 1: write the drift X_S to out; 2: write X_S to out and fold
// max |K|^2 into sd->kmax2_bits; 3: update reading X_S from C (a mode-2 output).
cudaError_t launch_update_gather(int prec, int mode, const GeoH& g, const void* U, const void* C, void* out,
                                 double eps, uint64_t seed, StepDev* sd, bool sd_adaptive, cudaStream_t st);
// step += 1 on the device (the Philox step counter read by the update).
// After an update: step += 1 and t += the step size taken (eps, or the
// device step size when adaptive).
cudaError_t launch_step_bump(StepDev* sd, double eps, bool adaptive, cudaStream_t st);
// Adaptive step size from the drift pass: eps_n = eps min(1, k_ref / K_max).
cudaError_t launch_step_eps(StepDev* sd, double eps, double k_ref, cudaStream_t st);
// Cooling: gradient f (8 FP64 values per site, [a][V]) + partial sums; the
// rule; Omega; apply.
cudaError_t launch_cool_grad(int prec, const GeoH& g, const void* U, void* f, double* partials,
                             const CoolState* cs, cudaStream_t st);
cudaError_t launch_cool_adapt(const GeoH& g, const double* partials, CoolArgs a, CoolState* cs,
                              int first, cudaStream_t st);
cudaError_t launch_cool_omega(int prec, const GeoH& g, const void* f, void* Om, void* Omi,
                              double eps, const CoolState* cs, cudaStream_t st);
cudaError_t launch_cool_apply(int prec, const GeoH& g, void* U, const void* Om, const void* Omi,
                              const CoolState* cs, cudaStream_t st);
// Single-pass sweep of the D_0 / D_1 rules (FP64 and FP32 storage only):
// Omega and Omega^{-1} straight from the gradient with the strength the rule
// already set; the apply over tiles of COOL_TILE sites inside one x3 layer,
// one record per tile of the rule's inputs for the next sweep ((1/3) Tr U U^+
// and nonfinite count, 2 doubles; cool_tiles(g) records); the rule from
// those records.
enum { COOL_TILE = 128 };
int cool_tiles(const GeoH& g);
cudaError_t launch_cool_grad_omega(int prec, const GeoH& g, const void* U, void* Om, void* Omi, double eps,
                                   const CoolState* cs, cudaStream_t st);
cudaError_t launch_cool_apply_tiles(int prec, const GeoH& g, void* U, const void* Om, const void* Omi,
                                    double* rec, const CoolState* cs, cudaStream_t st);
cudaError_t launch_cool_adapt_tiles(const GeoH& g, const double* rec, CoolArgs a, CoolState* cs, cudaStream_t st);
// Observables: per-site pass (F must hold the unscaled clover field when
// with_q) then the final fixed-order reduction into *out.
cudaError_t launch_obs(int prec, const GeoH& g, const void* U, const void* F, int with_q,
                       double* partials, double* q_site, cudaStream_t st);
cudaError_t launch_obs_final(const GeoH& g, const double* partials, double beta, double th_re,
                             double th_im, ObsOut* out, cudaStream_t st);
// Fused batch: one launch of family fam (ENS_*) over nw work items (device
// arrays cd, w); FP64 and FP32 storage only.  Per-chain kernels (one thread
// or one block per chain): the adaptive step size, the step counter, and the
// cooling rule (first = the call's first sweep).
// arg: ENS_COOL_GRAD's `first` flag (the call's first gradient runs whatever the rule state).
cudaError_t launch_ens(int prec, int fam, const ChainDesc* cd, const WorkItem* w, int nw, int arg, cudaStream_t st);
cudaError_t launch_ens_step_eps(const ChainDesc* cd, const int* chains, int n, cudaStream_t st);
cudaError_t launch_ens_step_bump(const ChainDesc* cd, const int* chains, const int* adaptive, int n,
                                 cudaStream_t st);
cudaError_t launch_ens_cool_adapt(const ChainDesc* cd, const int* chains, int n, int first, cudaStream_t st);
// the rule of single-pass chains from their tile records (ChainDesc::arec)
cudaError_t launch_ens_cool_adapt_tiles(const ChainDesc* cd, const int* chains, int n, cudaStream_t st);
// Integer-pipe float <-> double conversions (cvt.cuh) against the hardware
// ones on n generated cases; mismatch counts added into bad[0] (float ->
// double) and bad[1] (double -> float).
cudaError_t launch_selftest_convert(uint64_t seed, long long n, unsigned long long* bad, cudaStream_t st);
// The FP64 Box-Muller's table-driven ln and sincospi against CUDA's log and
// sincospi on n generated uniforms; the largest distances in ulp (rounded
// up) into worst[0] (ln) and worst[1] (sin, cos).
cudaError_t launch_selftest_box_muller(uint64_t seed, long long n, unsigned long long* worst, cudaStream_t st);

}  // namespace clgc
