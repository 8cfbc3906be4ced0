/*
 * cl.h -- C-ABI of the GB300 complex-Langevin + adaptive gauge-cooling library
 * (libcl.so), following Bongiovanni, Aarts, Seiler, Sexty, Stamatescu,
 * "Adaptive gauge cooling for complex Langevin dynamics", LATTICE 2013
 * (arXiv:1311.1056).
 *
 * The method: SU(3) Yang-Mills with a theta-term, S = S_W - i theta sum_x q_L(x)
 * (Sec. 5, eq. "eq:st"), evolved by complex Langevin on SL(3,C) links
 * (Sec. 2), each step followed by gauge-cooling sweeps
 * Omega_x = exp(-eps alpha f_ax lambda_a) that lower the unitarity norm
 * (Sec. 2, eq. "eq:24"), with the adaptive strength alpha_ad = alpha / D
 * (Sec. 4).
 *
 * Conventions shared by every call:
 *  - Lattice: periodic, extents L[0..3] >= 1, V = L0 L1 L2 L3 sites,
 *    site s = x0 + L0 (x1 + L1 (x2 + L2 x3)), direction mu = 0..3 along x_mu.
 *  - Host link arrays ("AoS"): V*4*9 complex numbers as 2*V*4*9 doubles,
 *    index ((s*4 + mu)*9 + 3*row + col)*2 + {0: re, 1: im}.
 *  - Ownership: the library owns every device buffer it allocates; the
 *    caller owns every host buffer and every device pointer it passes in.
 *    Device pointers passed in must stay valid until the call's work on the
 *    lattice's stream has completed.
 *  - Streams: all device work of a lattice is enqueued on the CUDA stream
 *    given to cl_init_lattice (NULL = legacy default stream).  Calls that
 *    return host results (cl_observables, cl_get_*, cl_cool with a report,
 *    cl_trajectory, cl_drift, cl_cool_gradient, cl_qdensity) synchronise
 *    that stream; the others only enqueue.
 *  - Errors: every call returns a cl_status and never aborts.  A CUDA error
 *    gives CL_ERR_CUDA; its text is kept (per thread) for cl_last_error().
 *    A lattice is not thread-safe: one host thread per lattice at a time.
 *  - Precision (cl_precision): CL_FP64 keeps links and all arithmetic in
 *    FP64.  CL_FP32_STORAGE stores and multiplies links in FP32 and keeps in
 *    FP64 the matrix exponentials of the Langevin and cooling updates, the
 *    det U = 1 re-projection and every global reduction.  CL_DF64 stores
 *    links as double-float pairs (hi + lo floats, ~48 significant bits) and
 *    does the link algebra (products, inverses, plaquettes, clover, drift,
 *    cooling transformations), the noise, the exponentials and the
 *    re-projection in double-float arithmetic on the FP32 pipe, with only
 *    the reductions' final sums in FP64; its results agree with CL_FP64 to
 *    ~1e-14 per step.
 *  - Noise: Philox4x32-10 keyed by (seed, step, site, mu), so results do not
 *    depend on launch shape, and a run resumed from cl_get_links /
 *    cl_get_step reproduces the uninterrupted one.
 */
#ifndef CL_GAUGECOOL_H
#define CL_GAUGECOOL_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cl_lattice cl_lattice; /* opaque; owns its device memory */

typedef enum {
  CL_OK = 0,
  CL_ERR_INVALID = 1,   /* bad argument (NULL pointer, size, mode) */
  CL_ERR_OOM = 2,       /* device allocation failed */
  CL_ERR_CUDA = 3,      /* a CUDA runtime error; see cl_last_error() */
  CL_ERR_NONFINITE = 4, /* a NaN/Inf appeared in the links (CL runaway) */
  CL_ERR_RUNAWAY = 5,   /* unitarity norm above the caller's bound */
  CL_ERR_TIMEOUT = 6    /* a bounded wait for device work gave up (cl_wait, cl_batch_wait) */
} cl_status;

typedef enum { CL_FP64 = 0, CL_FP32_STORAGE = 1, CL_DF64 = 2 } cl_precision;
typedef enum { CL_START_COLD = 0, CL_START_HOT = 1 } cl_start;

/* Choice of D in alpha_ad = alpha / D (Sec. 4): D_0 = 1; D_1 = (1/3)<Tr U U^+>
 * (the normalised unitarity norm, >= 1); D_2 = <|f_ax|>_{a,x}; D_2 RMS =
 * sqrt(<f_ax^2>_{a,x}). */
typedef enum { CL_D0 = 0, CL_D1 = 1, CL_D2_MEANABS = 2, CL_D2_RMS = 3 } cl_adapt;

typedef struct {
  int L[4];             /* lattice extents, each >= 1 */
  double beta;          /* Wilson coupling beta = 6/g^2 */
  double theta_re;      /* theta_L, complex (real theta: complex action; */
  double theta_im;      /*   imaginary theta: real action, Sec. 5) */
  cl_precision prec;
  uint64_t seed;        /* Philox key of every random number of this lattice */
  cl_start start;       /* cold (U = 1) or Haar-random SU(3) (Philox stream 2) */
  double gauge_sigma;   /* > 0: then U_{x,mu} <- Om_x U Om_{x+mu}^{-1} with
                           Om_x = exp(i w_a lambda_a), w_a = i N(0, gauge_sigma^2)
                           (Philox stream 1); 0: no transformation */
} cl_params;

typedef struct {
  double eps;        /* epsilon in Omega_x = exp(-eps alpha_ad f_ax lambda_a) */
  double alpha;      /* alpha_gf (alpha of alpha_ad = alpha / D) */
  cl_adapt mode;     /* choice of D */
  int n_min, n_max;  /* sweep-count bounds of the adaptive stop rule */
  double tol_rel;    /* stop when UN_prev - UN < tol_rel (UN_prev - 1) */
  double d_floor;    /* stop when UN - 1 < d_floor */
  double d_guard;    /* no sweep when D < d_guard (gradient at rounding level) */
  int forced_sweeps; /* >= 0: exactly this many sweeps (reproducible counts) */
} cl_cool_params;

/* Observables: plaquette (1/3)<Tr U_P> (complex), unitarity norm
 * (1/3)<Tr U U^+> over links (Sec. 2; distance d = un - 1, Sec. 3),
 * topological charge Q_L = sum_x q_L(x) (complex, Sec. 5), Wilson action
 * S_W, full action S = S_W - i theta Q_L, and max |det U - 1|. */
typedef struct {
  double plaq_re, plaq_im, un, q_re, q_im, sw_re, sw_im, s_re, s_im, max_det_dev;
} cl_obs;

typedef struct {
  int sweeps;             /* cooling sweeps applied */
  double alpha_ad_last;   /* alpha_ad of the last applied sweep (0 if none) */
  double un_before;       /* unitarity norm before the first sweep */
  double un_after;        /* after the last sweep */
} cl_cool_report;

/* Create a lattice on the current CUDA device and initialise its links
 * (start, then the optional random gauge transformation).  cuda_stream is a
 * cudaStream_t (may be NULL).  On success *out owns the device memory
 * (per site: 54 complex 3x3 matrices in FP64 and DF64 -- links, a second
 * link buffer, inverses, plaquettes, their differences, the clover field and
 * the 24 drift contributions, whose planes also hold the theta force's
 * parked partial sums and, outside the CL step, the cooling fields: 7,776
 * bytes; 50 in FP32 storage, which forms the inverses where it uses them:
 * 3,600 bytes; cl_lattice_bytes gives the exact figure).
 * Errors: CL_ERR_INVALID (NULL, extents < 1, V*6*9 beyond int range),
 * CL_ERR_OOM, CL_ERR_CUDA. */
cl_status cl_init_lattice(const cl_params* params, void* cuda_stream, cl_lattice** out);

/* Re-initialise a lattice in place for a new chain with the same extents and
 * precision (reuses its device memory): start field, step counter and
 * cooling state from params, as cl_init_lattice; captured step graphs are
 * dropped, tuned block sizes kept.  Waits for the lattice's stream first.
 * Errors: CL_ERR_INVALID (other extents or precision), CL_ERR_CUDA. */
cl_status cl_reset_lattice(cl_lattice* lat, const cl_params* params);

/* Device bytes cl_init_lattice allocates for params (links, the second link
 * buffer, link inverses, plaquettes, drift slots -- which also hold the
 * cooling fields --, clover field and reduction records; the optional
 * staging buffer of the host link exchange is not included).
 * Errors: CL_ERR_INVALID. */
cl_status cl_lattice_bytes(const cl_params* params, size_t* bytes);

/* n_steps complex Langevin steps, no cooling (Sec. 2; the update
 * U' = exp(i lambda_a (eps K_a + sqrt(eps) eta_a)) U, K_a = -D_a S,
 * <eta_a eta_b> = 2 delta_ab, all links at once, then U' <- U' det(U')^{-1/3}).
 * The drift contains the Wilson staples and the clover theta-term (Sec. 5).
 * Enqueue only.  Errors: CL_ERR_INVALID (eps < 0, n_steps < 0), CL_ERR_CUDA. */
cl_status cl_step(cl_lattice* lat, double eps, int n_steps);

/* Gauge cooling with the adaptive rule (Sec. 2 eq. "eq:24", Sec. 4).  The
 * rule runs on the device; report may be NULL (then nothing is
 * synchronised).  With a report: CL_ERR_NONFINITE if the links hold a
 * NaN/Inf.  Errors: CL_ERR_INVALID (bad mode/bounds), CL_ERR_CUDA. */
cl_status cl_cool(cl_lattice* lat, const cl_cool_params* cp, cl_cool_report* report);
/* The report of the most recent cooling call on this lattice, whether it ran
 * through cl_cool, cl_trajectory, a replayed step graph or a batch (waits for
 * the lattice's stream).  Errors: CL_ERR_INVALID, CL_ERR_NONFINITE, CL_ERR_CUDA. */
cl_status cl_cool_last_report(cl_lattice* lat, cl_cool_report* report);

/* Observables of the current links (synchronises).  CL_ERR_NONFINITE when a
 * link holds a NaN/Inf (*out is still written). */
cl_status cl_observables(cl_lattice* lat, cl_obs* out);

/* The fused hot path: n_steps times [one CL step, cooling with cp (may be
 * NULL: no cooling)]; after every obs_every-th step (obs_every > 0) the
 * observables go to obs_out[k] and the cooling report to rep_out[k] (either
 * may be NULL), k = 0 .. n_steps/obs_every - 1.  Records are kept on the
 * device and copied once at the end (synchronises when obs_every > 0).
 * runaway_un > 0: CL_ERR_RUNAWAY if a recorded unitarity norm exceeds it. */
cl_status cl_trajectory(cl_lattice* lat, double eps, int n_steps, const cl_cool_params* cp,
                        int obs_every, cl_obs* obs_out, cl_cool_report* rep_out,
                        double runaway_un);

/* Launch shapes.  Five kernel families take a tunable block size (threads
 * per block; each thread owns one site or link, so the results do not depend
 * on it): CL_TUNE_CLOVER (link inverses, plaquettes, clover field),
 * CL_TUNE_FORCE (per-plaquette drift), CL_TUNE_UPDATE (noise + exponential
 * update), CL_TUNE_OMEGA (cooling transformation), CL_TUNE_APPLY (cooling
 * apply).  The reductions keep a fixed shape so that their summation order,
 * and hence every result, is the same under any tuning.
 * cl_set_blocks: blocks[CL_NTUNE], each 0 (default, 128) or a multiple of 32
 *   in [32, 256]; takes effect for later launches (graphs already captured
 *   keep the shape they were captured with).
 * cl_get_blocks: the block sizes in effect.
 * cl_autotune: times one CL step + 2 cooling sweeps (eps, cp with the sweep
 *   count forced to 2) reps times for every candidate block size in
 *   {32, 64, 128, 256}, sets the fastest per family and writes it to
 *   blocks_out (may be NULL).  ms_out (may be NULL) receives the mean
 *   per-step milliseconds, [4 candidates][CL_NTUNE].  The lattice is left as
 *   it was (links, step counter, cooling state; snapshot in a temporary
 *   device buffer of one link field).  With use_cache != 0 and ms_out NULL a
 *   shape tuned before in this process (same device, precision, extents and
 *   theta == 0 or not) is reused without timing.
 * Errors: CL_ERR_INVALID, CL_ERR_OOM, CL_ERR_CUDA. */
typedef enum { CL_TUNE_CLOVER = 0, CL_TUNE_FORCE = 1, CL_TUNE_UPDATE = 2, CL_TUNE_OMEGA = 3,
               CL_TUNE_APPLY = 4, CL_NTUNE = 5 } cl_tune_family;
cl_status cl_set_blocks(cl_lattice* lat, const int* blocks);
cl_status cl_get_blocks(cl_lattice* lat, int* blocks);
cl_status cl_autotune(cl_lattice* lat, double eps, const cl_cool_params* cp, int reps, int use_cache,
                      int* blocks_out, double* ms_out);

/* Checkpoint / resume.  The whole state of a chain in one host buffer of
 * cl_state_size bytes: a header (extents, precision, parameters, Philox step
 * word and Langevin time, last adaptive step size, cooling-rule state,
 * adaptive-step reference, tuned block sizes) followed by the link field in
 * its device storage form (copied verbatim, so the restore is exact in every
 * precision; FP64 and DF64 16 B, FP32 storage 8 B per complex entry).  The
 * noise is counter-based, so a lattice loaded from a checkpoint continues bit
 * for bit as the saved one would have.  cl_load_state needs a lattice of the
 * same extents and precision; it takes the saved parameters (beta, theta,
 * seed, ...) over and drops captured step graphs.  Both wait for the
 * lattice's stream.  Errors: CL_ERR_INVALID (NULL, short buffer, not a
 * checkpoint, other extents or precision), CL_ERR_CUDA. */
cl_status cl_state_size(const cl_lattice* lat, size_t* bytes);
cl_status cl_save_state(cl_lattice* lat, void* host, size_t bytes);
cl_status cl_load_state(cl_lattice* lat, const void* host, size_t bytes);

/* A non-blocking CUDA stream owned by the caller (for cl_init_lattice when
 * the caller has none of its own); destroy it after the lattices that use it
 * (cl_stream_destroy waits for its work first).  Errors: CL_ERR_INVALID,
 * CL_ERR_CUDA. */
cl_status cl_stream_create(void** stream);
cl_status cl_stream_destroy(void* stream);

/* One step of the hot path as a CUDA graph.  cl_capture_step records [CL
 * step, cooling with cp (NULL: none)] on the lattice's stream, which must not
 * be the legacy default stream; nothing runs at capture.  cl_replay enqueues
 * the recorded step n_steps times (one graph launch each; the Philox step
 * counter lives on the device, so every replay draws fresh noise).  The
 * cooling rule still decides on the device how many of the recorded n_max
 * sweeps run.  Replays and ordinary calls may be mixed.
 * Errors: CL_ERR_INVALID (NULL stream, bad eps/cp, nothing captured), CL_ERR_CUDA. */
cl_status cl_capture_step(cl_lattice* lat, double eps, const cl_cool_params* cp);
cl_status cl_replay(cl_lattice* lat, int n_steps);

/* An ensemble of independent chains advanced together: one graph launch
 * advances every chain by one step (eps[i], and cooling cps[i] when
 * with_cooling) -- fused launches over all chains' blocks (see
 * cl_batch_set_fused), or a graph that forks from an internal stream to every
 * lattice's own stream, records each chain's own kernels and joins back, so
 * that the GPU runs the chains' kernels concurrently.  The lattices stay owned by the caller and
 * must outlive the batch; while in a batch they are advanced with
 * cl_batch_run (a lattice stepped on its own is detected and refused with
 * CL_ERR_INVALID).  cl_batch_run orders itself after work already queued on
 * the lattices' streams, and later per-lattice calls (observables, links,
 * cooling report) order themselves after it; cl_batch_synchronize waits for
 * the batch on the host.
 * Errors: CL_ERR_INVALID (n < 1, NULL, shared lattices or streams, default
 * stream), CL_ERR_CUDA. */
typedef struct cl_batch cl_batch;
cl_status cl_batch_create(int n, cl_lattice* const* lats, const double* eps,
                          const cl_cool_params* cps, int with_cooling, cl_batch** out);
/* Add a lattice (with its eps and, for a cooling batch, its cooling
 * parameters) to / remove one from the batch; the batch graph is captured
 * again (waits for the batch's pending work).  A removed lattice is the
 * caller's again and may be stepped on its own.  An empty batch runs nothing.
 * Errors: CL_ERR_INVALID (already a member / not a member, shared stream,
 * default stream, bad eps or cp), CL_ERR_CUDA. */
cl_status cl_batch_add(cl_batch* batch, cl_lattice* lat, double eps, const cl_cool_params* cp);
cl_status cl_batch_remove(cl_batch* batch, cl_lattice* lat);
cl_status cl_batch_size(const cl_batch* batch, int* n);
/* Fused mode: instead of every chain's own kernels on its own stream, one
 * launch per kernel family runs the blocks of all chains (each block runs
 * its chain's kernel body with that chain's geometry, buffers and state, so
 * every chain's arithmetic, noise and cooling decisions are exactly those of
 * its own launches); the launches of one step are captured as one graph on
 * the batch's internal stream.  All members must have the same precision,
 * FP64 or FP32 storage (CL_ERR_INVALID otherwise; the batch then stays in
 * its previous mode).  cl_batch_create starts a batch fused when its
 * members allow it, else with per-chain graphs; cl_batch_add of a member of
 * another precision switches a fused batch to per-chain graphs.  Setting the
 * mode re-captures the batch (waits for its pending work).  The launches of
 * a fused step are counted on the first member's cl_launch_count (the others
 * share them).  cl_batch_get_fused returns the mode.  Errors:
 * CL_ERR_INVALID, CL_ERR_OOM, CL_ERR_CUDA. */
cl_status cl_batch_set_fused(cl_batch* batch, int fused);
cl_status cl_batch_get_fused(const cl_batch* batch, int* fused);
cl_status cl_batch_run(cl_batch* batch, int n_steps);
cl_status cl_batch_synchronize(cl_batch* batch);
cl_status cl_batch_wait(cl_batch* batch, double timeout_s);  /* as cl_wait, for the batch */
void cl_batch_free(cl_batch* batch);

/* ------------------------------------------------------ SU(2) Polyakov chain
 * The model of Sec. 3-4 (eq. "eq:s"): S = -(beta/2) Tr(U_1 U_2 ... U_N) with
 * complex beta and links in SL(2,C); many independent chains of the same
 * length N advanced together (one CTA per chain, the chain kept in shared
 * memory for up to 256 steps per launch).  The one-link model it reduces to
 * has <(1/2) Tr(U_1 ... U_N)> = I_2(beta) / I_1(beta).
 * Links: host arrays [chain][k][2][2] complex as {re,im} doubles (8 per link).
 * CL step: U_k <- exp(i sigma_a (eps K_a + sqrt(eps) eta_a)) U_k, K_a = -D_a S,
 * eta_a = sqrt(2) * normal (Philox key = the chain's seed, counter
 * (k, step, 3 << 8, j)), then U_k / det(U_k)^(1/2).  Cooling: f_ak =
 * 2 Tr[sigma_a (U_k U_k^+ - U_{k-1}^+ U_{k-1})], Omega_k = exp(-eps alpha_ad
 * f_ak sigma_a), U_k <- Omega_k U_k Omega_{k+1}^{-1}, with the stop rule of
 * cl_cool (D_1 = (1/2)<Tr U U^+>, D_2 = <|f_ak|>).
 * cl_pchain_create: beta [n_chains][2] (re, im), seeds [n_chains]; start U = 1
 *   transformed by Omega_k = exp(i w_a sigma_a), w_a = i gauge_sigma g_a
 *   (Philox stream 4, counter (k, 0, 4 << 8, j)).  1 <= n_links <= 1024,
 *   1 <= n_chains <= 65535.
 * cl_pchain_run: n_steps of [CL step (eps), cooling with cp (NULL: none)];
 *   with obs_every > 0, after every obs_every-th step of this call one record
 *   per chain is written to obs_out[record][chain][5]: (1/2) Tr(U_1...U_N)
 *   re, im; unitarity norm (1/N) sum (1/2) Tr U U^+; max |det U - 1|; sweeps.
 *   Waits for the stream at the end.
 * Errors: CL_ERR_INVALID, CL_ERR_OOM, CL_ERR_CUDA. */
typedef struct cl_pchain cl_pchain;
cl_status cl_pchain_create(int n_chains, int n_links, const double* beta, const uint64_t* seeds,
                           double gauge_sigma, void* cuda_stream, cl_pchain** out);
cl_status cl_pchain_run(cl_pchain* chains, int n_steps, double eps, const cl_cool_params* cp,
                        int obs_every, double* obs_out);
cl_status cl_pchain_get_links(cl_pchain* chains, double* host);
cl_status cl_pchain_set_links(cl_pchain* chains, const double* host);
cl_status cl_pchain_get_step(const cl_pchain* chains, uint64_t* step);
void cl_pchain_free(cl_pchain* chains);

/* ------------------------------------------------------------------ serving
 * A request server: complex-Langevin trajectories (one chain each) admitted
 * as they arrive and advanced concurrently on one GPU.  Every resident chain
 * keeps its links, Philox step counter and cooling state in HBM and has its
 * own stream with up to two chunks of chunk_steps steps queued ahead of the
 * host; a chain that finishes frees its slot and the next queued request is
 * admitted at once (continuous batching).  Admission is first come, first
 * served, limited by max_slots resident chains and by hbm_budget_bytes of
 * lattice memory (cl_lattice_bytes); idle lattices are kept for reuse by
 * requests of the same extents and dropped, oldest first, when a new one
 * needs the room.  A chain's result does not depend on what runs beside it:
 * its noise is keyed by its own seed and step, and its kernels and
 * reductions are the same as for a lone cl_step / cl_cool sequence.
 * The server is driven by the calling thread (no threads of its own); one
 * server must not be used from two threads at once. */
typedef struct {
  int L[4];
  double beta, theta_re, theta_im;
  double eps;          /* CL step size, also the cooling eps */
  int n_steps;         /* CL steps (each followed by the cooling call) */
  uint64_t seed;       /* Philox key of this chain */
  cl_start start;
  double gauge_sigma;  /* optional random SL(3,C) transformation of the start */
  int64_t tag;         /* caller's identifier, returned in the result */
} cl_request;

typedef struct {
  double hbm_budget_bytes;  /* admission limit on resident lattice memory */
  int max_slots;            /* chains resident at once */
  cl_precision prec;        /* storage form of every chain */
  int chunk_steps;          /* steps per queued chunk */
  int use_graphs;           /* 1: steps replay a captured graph; 0: eager launches */
  int cool_enabled;         /* 1: each step is followed by cooling with `cool` */
  cl_cool_params cool;      /* its eps is replaced by the request's eps */
  int blocks_from_autotune; /* 1: tune block sizes per lattice shape (cached) */
  double k_ref;             /* > 0: adaptive step size of every chain (cl_set_adaptive_step) */
  double runaway_un;        /* > 0 (with cooling): a chain whose unitarity norm after a
                               chunk's last cooling call exceeds this, or whose links
                               are non-finite, is stopped there with CL_ERR_RUNAWAY */
} cl_server_config;

typedef struct {
  int64_t tag;
  cl_status status;          /* CL_OK, CL_ERR_RUNAWAY (stopped early) or CL_ERR_NONFINITE */
  int n_steps;               /* steps run (fewer than requested after a runaway) */
  cl_obs obs;                /* observables after the last step */
  cl_cool_report last_cool;  /* report of the last step's cooling */
  double t_submit, t_admit, t_done;  /* server clock, seconds */
} cl_result;

typedef struct {
  int64_t submitted, admitted, completed, runaways;
  int active, queued, pooled, peak_active;
  uint64_t bytes_in_use, peak_bytes;
} cl_server_stats;

typedef struct cl_server cl_server;
/* Errors: CL_ERR_INVALID (bad configuration). */
cl_status cl_server_create(const cl_server_config* cfg, cl_server** out);
/* Seconds since cl_server_create (the clock of t_submit / t_admit / t_done). */
double cl_server_clock(const cl_server* srv);
/* Queue a request (nothing runs until the next poll).  t_submit < 0 stamps
 * the current server clock.  Errors: CL_ERR_INVALID (bad request, or one
 * larger than the whole budget). */
cl_status cl_server_submit(cl_server* srv, const cl_request* req, double t_submit);
/* Advance the server without blocking: retire finished chunks and chains,
 * queue further chunks, admit waiting requests; then hand out up to max_out
 * finished results (completion order) into out, their number in *n_out.
 * Errors: CL_ERR_INVALID, CL_ERR_OOM, CL_ERR_CUDA. */
cl_status cl_server_poll(cl_server* srv, cl_result* out, int max_out, int* n_out);
cl_status cl_server_stats_get(const cl_server* srv, cl_server_stats* out);
/* Replay a request trace in real time: request i is submitted when the
 * server clock reaches (start of the call) + arrival_s[i] (sorted), and the
 * call returns when all n have finished; results[] in completion order,
 * t_submit = the scheduled arrival, so host lag counts as latency. */
cl_status cl_server_run_trace(cl_server* srv, int n, const cl_request* reqs, const double* arrival_s,
                              cl_result* results);
void cl_server_free(cl_server* srv);

/* Links as host AoS doubles (layout above), any precision (FP32 links are
 * widened).  host_aos holds V*4*18 doubles.  Page-locked host memory that the
 * device can address (cudaHostAlloc, cudaHostRegister, a framework's pinned
 * tensor) is read or written in place by the layout kernel over the host
 * link; pageable memory goes through a device staging buffer (allocated on
 * first use).  Synchronises.  Errors: CL_ERR_INVALID (NULL), CL_ERR_OOM
 * (staging), CL_ERR_CUDA. */
cl_status cl_get_links(cl_lattice* lat, double* host_aos);
/* Replace the links from host AoS doubles (FP32 storage rounds them).
 * Enqueue only, but host_aos may be reused on return (the copy completes first). */
cl_status cl_set_links(cl_lattice* lat, const double* host_aos);
/* The same with a caller-owned device AoS buffer (e.g. a torch tensor). */
cl_status cl_get_links_device(cl_lattice* lat, double* dev_aos);
cl_status cl_set_links_device(cl_lattice* lat, const double* dev_aos);

/* Philox step counter (number of CL steps taken; keys the noise). */
cl_status cl_get_step(const cl_lattice* lat, uint64_t* step);
cl_status cl_set_step(cl_lattice* lat, uint64_t step);

/* Adaptive Langevin step size (the runaway control that goes with gauge
 * cooling): with k_ref > 0 every later CL step first gathers the drift of all
 * links and K_max = max over links of |K|, |K|^2 = sum_a |K_a|^2 =
 * 2 |X_S - Tr X_S / 3|_F^2, then runs with eps_n = eps min(1, k_ref / K_max)
 * in the drift and sqrt(eps_n) in the noise; the decision is taken on the
 * device (graph-replayable).  The cooling that follows keeps its own eps.
 * k_ref = 0 turns it off.  Errors: CL_ERR_INVALID (k_ref < 0 or NaN). */
cl_status cl_set_adaptive_step(cl_lattice* lat, double k_ref);
/* Langevin time t = sum of the step sizes taken since the start, and the
 * eps_n and K_max of the last adaptive step (0 before one).  Waits for the
 * lattice's stream; any pointer may be NULL.  Errors: CL_ERR_INVALID, CL_ERR_CUDA. */
cl_status cl_get_langevin_time(cl_lattice* lat, double* t, double* eps_last, double* kmax_last);

/* Drift matrix X_S of every link, D_a S = i Tr(lambda_a X_S) (Sec. 5 action),
 * as host AoS doubles (V*4*18).  Synchronises. */
cl_status cl_drift(cl_lattice* lat, double* host_aos);
/* Cooling gradient f_ax = 2 Tr[lambda_a sum_mu (U U^+ - U^+_{x-mu} U_{x-mu})]
 * (Sec. 2, eq. "eq:24"), host doubles, layout [a][site] (8*V).  Synchronises. */
cl_status cl_cool_gradient(cl_lattice* lat, double* host_f);

/* The standard normal numbers of the CL noise as the kernels of form prec
 * draw them (Philox4x32-10 stream 0, Box-Muller): for each of the nsites
 * sites site0 .. site0 + nsites - 1 and direction mu, the 8 numbers of link
 * (site, mu) at step `step` (the update's eta_a = sqrt(2) times them, a =
 * 1..8, so that <eta_a eta_b> = 2 delta_ab), host doubles [site][8].  FP64 draws them in FP64,
 * DF64 in double-float, FP32 storage in float.  A diagnostic: it uses the
 * current device and the legacy default stream, allocates and frees its own
 * device buffer, and synchronises.  Errors: CL_ERR_INVALID (NULL out, bad
 * precision, nsites < 0, site0 < 0, mu outside 0..3), CL_ERR_OOM, CL_ERR_CUDA. */
cl_status cl_noise_sample(cl_precision prec, uint64_t seed, uint32_t step, int mu, int site0, int nsites,
                          double* host_out);
/* Self-test of the float <-> double conversions the FP32-storage kernels
 * perform on the integer pipe (IEEE-754 field moves, round to nearest even):
 * on n generated cases (every float bit pattern class; doubles across the
 * float range, its underflow and overflow ends and exact rounding ties) it
 * compares each with the hardware conversion bit for bit and returns the
 * mismatch counts (both 0 when correct).  A diagnostic with no counterpart in
 * the paper: current device, legacy default stream, its own 16-byte device
 * buffer, synchronises.  Errors: CL_ERR_INVALID (NULL, n < 0), CL_ERR_OOM,
 * CL_ERR_CUDA. */
cl_status cl_selftest_convert(uint64_t seed, int64_t n, int64_t* bad_f2d, int64_t* bad_d2f);
/* Self-test of the FP64 noise's transcendentals: the table-driven ln and
 * sincospi that the FP64 Box-Muller uses for its uniforms (k + 1/2) 2^-52
 * (Sec. 2 noise), against CUDA's log and sincospi on n generated uniforms
 * (the whole range, the deep tail of ln, values next to 1 and next to the
 * sine table's grid).  Returns the largest distances in units in the last
 * place, rounded up.  A diagnostic with no counterpart in the paper: current
 * device, legacy default stream, its own 16-byte device buffer, synchronises.
 * Errors: CL_ERR_INVALID (NULL, n < 0), CL_ERR_OOM, CL_ERR_CUDA. */
cl_status cl_selftest_box_muller(uint64_t seed, int64_t n, int64_t* ulp_ln, int64_t* ulp_sincos);
/* Topological charge density q_L(x) (Sec. 5), host doubles [site]{re,im} (2*V). */
cl_status cl_qdensity(cl_lattice* lat, double* host_q);

/* Optional per-phase timing: with timing on, every kernel launch of the
 * lattice is bracketed by two CUDA events on the lattice's stream and its
 * duration is added to its phase.  cl_set_timing clears the totals (and
 * waits for pending events); cl_get_timing synchronises the stream and
 * returns, per phase, the summed milliseconds and the number of launches
 * (arrays of CL_NPHASE entries, either may be NULL).  Timing adds two event
 * records per launch and is off by default. */
enum {
  CL_PHASE_CLOVER = 0,     /* link inverses, plaquettes, clover field */
  CL_PHASE_UPDATE = 1,     /* drift gather + noise + exponential update */
  CL_PHASE_COOL_GRAD = 2,  /* cooling gradient f_ax + partial sums */
  CL_PHASE_COOL_RULE = 3,  /* adaptive rule (one block) */
  CL_PHASE_COOL_OMEGA = 4, /* Omega_x, Omega_x^{-1} */
  CL_PHASE_COOL_APPLY = 5, /* U <- Omega U Omega^{-1} */
  CL_PHASE_OBS = 6,        /* observables */
  CL_PHASE_FORCE = 7,      /* per-plaquette drift contributions (two kernels with theta) */
  CL_PHASE_COOL_GRAD_OMEGA = 8, /* single-pass D_0 / D_1 sweeps: gradient and Omega in one kernel */
  CL_NPHASE = 9
};
cl_status cl_set_timing(cl_lattice* lat, int on);
cl_status cl_get_timing(cl_lattice* lat, double* ms, int64_t* launches);

/* Number of kernels this lattice has launched so far. */
cl_status cl_launch_count(const cl_lattice* lat, int64_t* count);
/* Wait for the lattice's stream. */
cl_status cl_synchronize(cl_lattice* lat);
/* Bounded wait: returns CL_OK once all work queued on the lattice's stream
 * (or, for cl_batch_wait, the batch's) has finished, or CL_ERR_TIMEOUT when
 * timeout_s seconds pass first -- the work keeps running and may be waited
 * for again.  A caller (a server, a watchdog) uses it to detect a chain that
 * takes longer than it should without blocking on it.  The host polls the
 * stream; nothing waits on the device.  Errors: CL_ERR_INVALID (NULL,
 * timeout_s < 0 or NaN), CL_ERR_TIMEOUT, CL_ERR_CUDA. */
cl_status cl_wait(cl_lattice* lat, double timeout_s);
/* Release every device buffer of the lattice (NULL is ignored). */
void cl_free(cl_lattice* lat);

/* Observables of caller-owned device links with no device allocation.
 *
 * For callers that cannot allocate device memory: programs whose device
 * memory belongs to their own pool or arena (every byte accounted for), and
 * latency-critical loops that cannot afford cudaMalloc/cudaFree, which may
 * synchronise the device.  The paper has no counterpart: this is a systems
 * variant of cl_observables.
 *
 * dev_links: device AoS FP64 links (layout above, V*4*18 doubles), read only.
 * L: extents, each >= 1, with V <= CL_NOALLOC_MAX_SITES (else CL_ERR_INVALID).
 * dev_out: device, 10 doubles written in cl_obs field order (plaquette re/im,
 *   unitarity norm, Q re/im, S_W re/im, S re/im, max |det U - 1|).
 * cuda_stream: the stream to enqueue on (NULL = legacy default stream).
 * Nothing is synchronised.  A link with a NaN or Inf entry makes the
 * max |det U - 1| output NaN (the other outputs are then meaningless too).
 *
 * The per-block partial sums live in one fixed device array inside the
 * library (CL_NOALLOC_MAX_BLOCKS records of 9 doubles, 147,456 bytes), which
 * every GPU that loads the library holds until the process exits; launches
 * use at most that many blocks, whatever V.  The first call on each device
 * looks up the array's device address (cudaGetSymbolAddress), so make that
 * first call before any stream capture; the address is kept for the life
 * of the process, so calls after cudaDeviceReset() on that device are not
 * supported.  All calls share the array: calls that overlap on the GPU
 * (other streams or host threads) race on it.  Errors:
 * CL_ERR_INVALID (NULL, extents, volume, device index beyond
 * CL_NOALLOC_MAX_DEVICES), CL_ERR_CUDA; text in cl_last_error(). */
#define CL_NOALLOC_MAX_BLOCKS 2048
#define CL_NOALLOC_MAX_DEVICES 64
#define CL_NOALLOC_MAX_SITES (1LL << 30)
cl_status cl_observables_noalloc(const double* dev_links, const int L[4], double beta,
                                 double theta_re, double theta_im, double* dev_out,
                                 void* cuda_stream);

const char* cl_status_str(cl_status s);
/* Text of the last error on this host thread ("" if none). */
const char* cl_last_error(void);
int cl_version(void);

#ifdef __cplusplus
}
#endif
#endif
