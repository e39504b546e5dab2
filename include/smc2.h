/*
 * smc2.h -- C ABI of the GB300 SMC^2 library (libsmc2.so).
 *
 * The library runs the data-parallel hot path of SMC^2 (Rosato, Varsi,
 * Murphy, Maskell, "An O(log2 N) SMC^2 algorithm on distributed memory with
 * an approx. optimal L-kernel"): N parameter samples theta, each scored by a
 * bootstrap particle filter (Sec. II) of M particles over T observations,
 * importance-weighted with an L-kernel (Sec. IV-A, IV-D), resampled with
 * systematic resampling (Sec. IV-B) and recycled across iterations
 * (Sec. IV-C).  Every step runs in the library's own CUDA kernels on one
 * GPU (sm_103a); the host side only validates arguments, owns a small device
 * workspace and enqueues work.
 *
 * General conventions
 *  - Every call returns an smc2_status; no exception or signal crosses the
 *    ABI.  SMC2_EINVAL is returned before any GPU work is enqueued.
 *  - Pointers marked "device" must be device (or managed) memory of the
 *    current CUDA device; "host" pointers are plain host memory (pinned or
 *    pageable).  "host or device" pointers may be either (unified addressing).
 *  - All GPU work of a context is enqueued on the CUDA stream given to
 *    smc2_init (NULL = the legacy default stream) and is asynchronous unless
 *    the call says it synchronises.  Caller buffers must stay valid until the
 *    work that uses them has completed on that stream.
 *  - Device-side errors (an outer weight set that is zero or NaN throughout)
 *    are recorded in a device status word and reported by the next
 *    synchronising call; the first error is sticky until smc2_destroy or
 *    smc2_reset.  The kernels hold no spin-waits (their only waits are
 *    hardware barriers) and compute every index they use from exact integer
 *    arithmetic on validated sizes, so no device status exists for an expired
 *    wait or an index out of range.
 *  - Parameters theta are in unconstrained coordinates:
 *      SMC2_MODEL_LG_AR1: (phi, log sigma_x, log sigma_y), D = 3;
 *      SMC2_MODEL_SEIR:   (log beta0, log sigma_rw, log kappa, log gamma), D = 4.
 *    Device theta arrays are structure-of-arrays, theta[d * ld + i].
 *  - Random numbers come from Philox4x32-10 (Salmon et al., SC'11) keyed by
 *    the seed, with counters (c0, c1, i | dataset << 20, tag | k << 4), so a
 *    run is a deterministic function of its configuration and seed.
 */
#ifndef SMC2_H
#define SMC2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SMC2_OK = 0,
  SMC2_EINVAL = 1,     /* invalid argument or configuration */
  SMC2_ENOMEM = 2,     /* device or host allocation failed */
  SMC2_ECUDA = 3,      /* a CUDA runtime call failed */
  SMC2_ENONFINITE = 4, /* every outer importance weight is zero or NaN */
  SMC2_ECHOL = 5,      /* reserved: L-kernel factorisation failures fall back, see smc2_iter_stats */
  SMC2_ETIMEOUT = 6,   /* reserved, never returned: no kernel of this library spin-waits */
  SMC2_EBOUNDS = 7,    /* reserved, never returned: device indices are exact by construction */
  SMC2_ESTATE = 8      /* call not valid in the context's current state */
} smc2_status;

enum { SMC2_MODEL_LG_AR1 = 0, SMC2_MODEL_SEIR = 1, SMC2_MODEL_SIR = 2 };
enum { SMC2_PRIOR_GAUSS = 0, SMC2_PRIOR_UNIFORM = 1 };
enum { SMC2_PREC_FP64 = 0, SMC2_PREC_MIXED = 1 };   /* MIXED: FP32 particles, FP64 outer */
enum { SMC2_PROP_RW = 0, SMC2_PROP_MLP = 1 };
enum { SMC2_LK_FORWARD = 0, SMC2_LK_GAUSS_OPT = 1 };
enum { SMC2_PF_SYSTEMATIC = 0, SMC2_PF_MULTINOMIAL = 1 };
enum { SMC2_PF_ANY = 0, SMC2_PF_GROUPS = 1, SMC2_PF_FP32 = 2 };

#define SMC2_MAX_D 8
#define SMC2_MAX_M 4096     /* particles per filter (see M in smc2_config) */
#define SMC2_MAX_N 16384
#define SMC2_MAX_DATASETS 4096

typedef struct smc2_ctx smc2_ctx; /* opaque; owns its device workspace */

/* Sampler configuration (host memory, read during smc2_init only).
 * model, precision, proposal, lkernel: the enums above.
 * D: dimension of theta (3 for LG_AR1, 4 for SEIR, 2 for SIR).
 * N, M, T: theta samples, particles per filter, observations; used when
 *   n_datasets <= 1, otherwise taken per dataset from ds_N, ds_M, ds_T.
 *   M <= SMC2_MAX_M, and a filter's particles must fit one CTA's shared
 *   memory (227 KB): in FP64 the SEIR-type model takes M <= 2048.
 * K: iterations the context will run (sizes the statistics history).
 * rw_scale: standard deviation of the Gaussian random-walk proposal in every
 *   unconstrained coordinate (Sec. IV-A, Eq. 19: Sigma = rw_scale^2 I).
 * ess_frac: outer resampling when ESS < ess_frac * N (Sec. IV-B uses 1/2).
 * seed: key of the random stream.
 * prior_mean, prior_sd: independent Gaussian prior (= q_1 of Eq. 16) in the
 *   unconstrained coordinates, first D entries used.
 * prior_kind, prior_lo, prior_hi: SMC2_PRIOR_UNIFORM replaces the Gaussian
 *   prior by independent uniforms on [prior_lo, prior_hi] (the SIR experiment
 *   of Sec. V-A draws theta_1 from U[0, 1]); its log-density is -inf outside,
 *   so proposals there get zero weight.
 * npop, e0, i0, n_sub, lambda_floor: SEIR constants (population, initial
 *   exposed and infectious, Euler substeps per day, floor of the Poisson mean).
 *   The SIR model (Sec. V-A, theta = (beta, gamma) in natural units, state
 *   (S, I) with S_0 = npop - i0, I_0 = i0) uses npop (an integer <= 2^24) and
 *   i0; each day n(S->I) ~ Bin(S, 1 - exp(-beta I / npop)) and
 *   n(I->R) ~ Bin(I, 1 - exp(-gamma)), y_t ~ Poisson(I_t).  It runs with
 *   ppt <= 4 (M <= 2048).
 * ppt: particles per thread of the particle-filter kernel (0 = pick by the
 *   built-in tuner; otherwise 1, 2, 4, 8 or 16).
 * proposal = SMC2_PROP_MLP (learned proposal; not in the paper): once the
 *   network explains half the variance of its standardised targets (from
 *   k = 3 on) and the previous population has ESS >= 2 (D + 1) and a positive
 *   definite covariance Sigma = L L^T, theta_k = theta_{k-1} + h L (w + z),
 *   z ~ N(0, I), w = h/2 L^T grad log pi^(theta_{k-1}) clipped to [-3, 3]:
 *   a Langevin step preconditioned by Sigma (drift h^2/2 Sigma grad log pi^)
 *   with the gradient of a 64-wide two-layer tanh network trained in the run
 *   (tensor cores, bfloat16 operands, FP32 accumulation, Adam) on the
 *   (theta, log pi^) pairs of the last mlp_window iterations; otherwise the
 *   random walk above.  The network proposing at k was trained on the pairs
 *   of iterations up to k - 2 (its training overlaps iteration k - 1).  log q
 *   is the exact Gaussian density, so Eq. (20) with the Gaussian L-kernel
 *   keeps the weights valid.  Requires lkernel = SMC2_LK_GAUSS_OPT and one
 *   dataset.
 * pf_scheme, pf_ess_frac: particle-filter resampling (Sec. II).  The default
 *   (0, 0) resamples systematically after every step t < T.  pf_scheme =
 *   SMC2_PF_MULTINOMIAL draws every slot on its own; pf_ess_frac in (0, 1]
 *   resamples only when the ESS of the filter's weights (Eq. 12) is below
 *   pf_ess_frac * M, carrying the weights in between (Eq. 5) and resetting them
 *   to their mean on resampling (Eq. 13) -- the paper's filter is multinomial
 *   with pf_ess_frac = 1/2.  Either option needs ppt <= 4 (M <= 2048).
 * mlp_h, mlp_lr, mlp_steps, mlp_window: step h of the learned proposal, Adam
 *   learning rate, Adam steps per iteration, iterations of training pairs
 *   kept (0 selects 1.0, 5e-3, 16, 4; steps <= 256, window <= 16).
 * cta_threads: threads per particle-filter CTA (0 = pick by the tuner;
 *   otherwise a multiple of 32 up to 512 that holds whole filter groups).
 *   The tuner times every valid (ppt, cta_threads) pair on the context's own
 *   work list, prior draws of theta and min(T, 32) steps, then the shapes
 *   within 15 % of the fastest five times each over min(T, 64) steps, during
 *   smc2_init.
 * pf_family: the particle-filter kernel the tuner may pick: 0 either,
 *   SMC2_PF_GROUPS pf_kernel only (filter groups of any width, several per
 *   CTA), SMC2_PF_FP32 the register-resident FP32 filter with 2, 4 or 8
 *   particles per thread (mixed precision, LG or SEIR model, the default
 *   filter; one filter per CTA when every dataset's group has the same width,
 *   else groups of unequal width sharing a CTA).  Both compute the same filter;
 *   they differ in speed only.
 * n_datasets: number of independent datasets run together (<= 1: one).
 * ds_N, ds_M, ds_T: host arrays of n_datasets sizes (NULL when n_datasets <= 1). */
typedef struct {
  int model, precision, proposal, lkernel;
  int D, N, M, T, K;
  double rw_scale, ess_frac;
  uint64_t seed;
  double prior_mean[SMC2_MAX_D], prior_sd[SMC2_MAX_D];
  double npop, e0, i0, lambda_floor;
  int n_sub;
  int ppt;
  int cta_threads;
  int n_datasets;
  const int* ds_N;
  const int* ds_M;
  const int* ds_T;
  double mlp_h, mlp_lr;
  int mlp_steps, mlp_window;
  double pf_ess_frac;
  int pf_scheme;
  int prior_kind;
  double prior_lo[SMC2_MAX_D], prior_hi[SMC2_MAX_D];
  int pf_family;
} smc2_config;

/* Statistics of one iteration k of one dataset (Sec. IV-A, IV-B):
 * ess = N_eff of Eq. (25) = l_k of Eq. (24); lse = log sum_i w_k^i;
 * lse2 = log sum_i (w_k^i)^2; logz = lse - log N, the evidence estimate;
 * est = f~_k of Eq. (21) with f(theta) = theta (before resampling);
 * resampled = 1 when ESS < ess_frac N; lk_fallback = 1 when the Gaussian
 * L-kernel was numerically singular and the forward kernel (Eq. 30) was used.
 * mlp_used, mlp_loss: see SMC2_PROP_MLP in smc2_config. */
typedef struct {
  int k, resampled, lk_fallback, dataset;
  double ess, lse, lse2, logz;
  double est[SMC2_MAX_D];
  int mlp_used;        /* 1: theta_k came from the learned proposal */
  int pad;
  double mlp_loss;     /* training loss of the surrogate that proposed (learned proposal) */
  double cov[SMC2_MAX_D * SMC2_MAX_D]; /* weighted covariance of theta_k, entry (d, e) at
                                           d * SMC2_MAX_D + e (Eq. 21 with f = (theta - est)
                                           (theta - est)^T, before resampling) */
} smc2_iter_stats;

/* Create a context: validate cfg, allocate the device workspace, copy the
 * observations y (host or device, the concatenation over datasets of T_d
 * doubles; SEIR counts are non-negative integers stored as doubles) and
 * precompute the per-step observation terms on the device.  stream is a
 * cudaStream_t (NULL: legacy default stream).  Synchronises the stream.
 * Errors: EINVAL (bad configuration; *out untouched), ENOMEM, ECUDA. */
smc2_status smc2_init(const smc2_config* cfg, const double* y, void* stream, smc2_ctx** out);

/* Replace the observations of every dataset (same layout as smc2_init; host
 * or device) and recompute the observation terms.  Asynchronous on the
 * context stream: a host y must stay valid until the stream reaches it. */
smc2_status smc2_set_observations(smc2_ctx* ctx, const double* y);

/* Rewind the sampler to k = 0 with a new seed and clear the sticky error
 * and the statistics history.  Asynchronous. */
smc2_status smc2_reset(smc2_ctx* ctx, uint64_t seed);

/* Bootstrap particle filter log-likelihood estimates (Sec. II, Eq. 8):
 * loglik[i] = log p^(y_{1:T} | theta_i) for i < n, with theta_dev device SoA
 * [D][n], loglik_dev device [n], the random stream of filter i at iteration
 * `iteration` of dataset `dataset` (uses that dataset's M, T and y).  Every
 * step propagates with the state equation (Eq. 1), weights with the
 * observation density (Eq. 2, bootstrap form of Eq. 5), adds
 * log((1/M) sum w_t) and resamples systematically (Eqs. 26-27, Algorithm 1)
 * after every step t < T.  A filter whose weights all vanish returns -inf.
 * Asynchronous.  Errors: EINVAL (n < 1 or n > SMC2_MAX_N, bad dataset). */
smc2_status smc2_pf_loglik(smc2_ctx* ctx, const double* theta_dev, int n, int iteration,
                           int dataset, double* loglik_dev);

/* As smc2_pf_loglik, and also writes the per-step increments
 * delta_dev[i * T + t] = log p^(y_{1:t+1}) - log p^(y_{1:t}) and the
 * ancestors anc_dev[(i * (T-1) + t) * M + j] of slot j after step t+1
 * (either may be NULL).  Diagnostic path for checking the filter; on a
 * context whose filter is the FP32 one it runs that filter's traced
 * instantiation, whose arithmetic equals the untraced one's. */
smc2_status smc2_pf_trace(smc2_ctx* ctx, const double* theta_dev, int n, int iteration,
                          int dataset, double* loglik_dev, double* delta_dev, int32_t* anc_dev);

/* As smc2_pf_trace, and also the per-step quantities of the FP32 filter that a
 * stage-wise check needs (mixed precision, LG or SEIR model, the default
 * filter; the context's ppt must be 2, 4 or 8): after the propagation of
 * step t (0-based t < T), by particle j, at index (i T + t) M + j:
 * x_dev[.. * 5 + e] the state (LG: x in e = 0; SEIR: S, E, I, log beta and the
 * day's incidence lambda in e = 0..4), logw_dev the log-weight log g(y_t | x_t)
 * (Eq. 2; -inf for a NaN), q_dev the quantised weight floor(exp(logw - max)
 * 2^B) the resampling after step t used (Eqs. 26-27).  All outputs device
 * memory; delta_dev and anc_dev as in smc2_pf_trace (may be NULL).  It runs
 * the traced instantiation of the FP32 filter with one filter per CTA, whose
 * arithmetic equals the sampler's instantiations' (grouped or not).  Errors:
 * EINVAL (another precision, model or filter, a ppt outside 2, 4, 8, a NULL
 * trace pointer). */
smc2_status smc2_pf_trace_states(smc2_ctx* ctx, const double* theta_dev, int n, int iteration, int dataset,
                                 double* loglik_dev, double* delta_dev, int32_t* anc_dev, float* x_dev,
                                 float* logw_dev, uint64_t* q_dev);

/* One SMC^2 iteration of every dataset (Sec. IV):
 *  k = 1: draw theta ~ q_1 = prior (Eq. 16), weight w = pi / q_1 (Eq. 17);
 *  k > 1: propose theta_k ~ N(theta_{k-1}, rw_scale^2 I) (Eqs. 18-19),
 *         fit the L-kernel (Eqs. 32-35) and weight by Eq. (20);
 * then normalise (Eq. 22), estimate (Eq. 21), ESS and l_k (Eqs. 24-25),
 * evidence, and when ESS < ess_frac N resample (Eqs. 26-27), redistribute
 * (Algorithm 1's output order) and reset the weights (Sec. IV-B).
 * stats_host (host, n_datasets entries, may be NULL): if given, the call
 * synchronises and fills it.  Errors: ESTATE (K iterations already run),
 * ENONFINITE (reported when synchronising). */
smc2_status smc2_iterate(smc2_ctx* ctx, smc2_iter_stats* stats_host);

/* n_iter iterations back to back without host synchronisation (captured
 * once as a CUDA graph and replayed).  stats_host (may be NULL) receives
 * n_iter * n_datasets entries, iteration-major, and makes the call
 * synchronise.  Errors: ESTATE when fewer than n_iter iterations remain. */
smc2_status smc2_run(smc2_ctx* ctx, int n_iter, smc2_iter_stats* stats_host);

/* Recycled estimate after the iterations run so far (Sec. IV-C, Eq. 29 with
 * the constants of Eqs. 23-24): mean_host[D] = sum_k c_k f~_k; the latest
 * evidence estimate log Z_k; ess_sum = sum_k l_k, the ESS of the recycled
 * estimator; cov_host (row-major D x D) = sum_k c_k (C_k + f~_k f~_k^T) -
 * mean mean^T, the recycled posterior covariance, C_k the weighted
 * covariance of iteration k.  Any output pointer may be NULL.  Synchronises;
 * returns the sticky device status.  Errors: EINVAL (bad dataset), ESTATE
 * (no iteration run yet). */
smc2_status smc2_estimate(smc2_ctx* ctx, int dataset, double* mean_host,
                          double* log_evidence_host, double* ess_sum_host, double* cov_host);

/* Copy the statistics of iterations 1..k of a dataset to host (k entries;
 * *k_out receives k).  Synchronises. */
smc2_status smc2_get_history(smc2_ctx* ctx, int dataset, smc2_iter_stats* hist_host, int cap,
                             int* k_out);

/* The proposals theta_k of the latest iteration (host, row-major [N][D]) and
 * log q(theta_k | theta_{k-1}) (host, N; the prior's log density at k = 1),
 * the terms of Eq. (20) that the proposal contributes.  Either pointer may
 * be NULL.  Synchronises.  Errors: EINVAL (bad dataset). */
smc2_status smc2_get_proposals(smc2_ctx* ctx, int dataset, double* theta_host, double* logq_host);

/* The learned proposal's state that the next iteration uses
 * (proposal = SMC2_PROP_MLP, dataset 0): params_host (FP32, the layout of
 * smc2_mlp_loss_grad: 64 D + 4289 values), stdz_host (FP64, 2 D + 6 values:
 * input means mu[D], input sds sd[D], tau, zmean, zsd, target variance,
 * training loss, ymax; the score is d log pi^ / d theta_d = tau zsd (ds/dx)_d /
 * sd_d at x_d = (theta_d - mu_d) / sd_d), L_host (FP64, row-major D x D lower
 * Cholesky factor of the weighted population covariance) and *pop_ok (the
 * factor is usable).  Any pointer may be NULL.  Synchronises.  Errors:
 * EINVAL (no learned proposal in this context). */
smc2_status smc2_get_learned_state(smc2_ctx* ctx, float* params_host, double* stdz_host, double* L_host,
                                   int* pop_ok);

/* The learned proposal's training state after the latest training call (not
 * yet published; the call after iteration k trains on the ring holding the
 * pairs of iterations k - W + 1 .. k, and its result proposes at k + 2):
 * params_host, m_host, v_host (FP32, 64 D + 4289 values each: parameters and
 * Adam moments), *step_host (Adam steps taken), stdz_host (FP64, 2 D + 6
 * values in the layout of smc2_get_learned_state, from that call's
 * standardisation and its loss), ring_th_host (FP32, row-major
 * [mlp_window N][D]) and ring_lp_host (FP32, mlp_window N values: log prior
 * + PF log-likelihood) with *ring_rows_host rows filled (iteration k's pairs
 * in rows ((k - 1) mod W) N .. + N - 1).  Any pointer may be NULL.
 * Synchronises.  Errors: EINVAL (no learned proposal in this context). */
smc2_status smc2_get_learned_training(smc2_ctx* ctx, float* params_host, float* m_host, float* v_host,
                                      int* step_host, double* stdz_host, float* ring_th_host,
                                      float* ring_lp_host, int* ring_rows_host);

/* Checkpoint / resume of a dataset's population after iteration k: theta
 * (host, row-major [N][D]), log prior, PF log-likelihood estimate and
 * unnormalised log weight (host, N each).  get synchronises; set is
 * asynchronous and, for dataset 0, sets the context's iteration counter
 * to k (all datasets share it).  The recycling accumulators and history are
 * part of the state through smc2_get_history / smc2_set_history. */
smc2_status smc2_get_state(smc2_ctx* ctx, int dataset, int* k_out, double* theta_host,
                           double* logprior_host, double* loglik_host, double* logw_host);
smc2_status smc2_set_state(smc2_ctx* ctx, int dataset, int k, const double* theta_host,
                           const double* logprior_host, const double* loglik_host,
                           const double* logw_host);
smc2_status smc2_set_history(smc2_ctx* ctx, int dataset, const smc2_iter_stats* hist_host, int k);

/* Systematic resampling primitive (Sec. IV-B, Eqs. 26-27 and Algorithm 1's
 * output order) on quantised weights: q_dev (device, n unsigned 64-bit
 * integers with sum S, 0 < S < 2^64), U a 32-bit random word, u = (2U+1)/2^33.
 * anc_dev (device, n) receives a_j = min{i : C_i > floor((j + u) S / n)},
 * C the inclusive prefix sum of q.  Exact integer arithmetic.  Enqueued on
 * `stream`.  Errors: EINVAL (n < 1 or n > SMC2_MAX_N). */
smc2_status smc2_resample_systematic(const uint64_t* q_dev, int n, uint32_t U, int32_t* anc_dev,
                                     void* stream);

/* The library's random stream, for checking: for each of n counters
 * ctr_dev[4r .. 4r+3] (device), words_dev[4r..] (device, may be NULL)
 * receive Philox4x32-10 of (counter, seed) and z_dev[4r..] (device, may be
 * NULL) the four Box-Muller normals made from them, in double (precision
 * SMC2_PREC_FP64) or float arithmetic widened to double (SMC2_PREC_MIXED). */
smc2_status smc2_philox_normals(uint64_t seed, const uint32_t* ctr_dev, int n, int precision,
                                uint32_t* words_dev, double* z_dev, void* stream);

/* Particle-filter log-likelihoods that allocate no device memory (the paper
 * has no counterpart: this is a deployment variant of smc2_pf_loglik).
 * For callers that cannot allocate once running: a fixed device-memory
 * budget, a framework whose own pool owns the device memory, or a loop that
 * cannot afford the implicit synchronisation of cudaMalloc.  It computes
 * what smc2_pf_loglik computes for dataset 0 of a context made from cfg --
 * loglik_dev[i] for theta_dev (device SoA [D][n]) with y_dev (device, cfg->T
 * doubles), the random stream of `iteration` -- but needs no context.  Its
 * scratch (observation terms and the kernel's work-unit counter) is a 1 MiB
 * static device array that every GPU loading the library holds until exit.
 * Limits: cfg->T <= SMC2_NOALLOC_MAX_T and the usual n, M limits; larger
 * sizes return SMC2_EINVAL before any work is enqueued.  cfg->ppt selects
 * particles per thread (0: 2).  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) and should come before any
 * stream capture.  Every call reuses the same array and clears the counter
 * it needs, so calls that overlap on the GPU (other streams, other threads)
 * race on it.  Asynchronous on `stream`.  The filter kernel records no
 * device status: a filter whose weights all vanish returns -inf in
 * loglik_dev, and a non-finite theta gives a non-finite entry there, which the
 * caller reads.  Errors: EINVAL, ECUDA. */
#define SMC2_NOALLOC_MAX_T 32000
smc2_status smc2_pf_loglik_noalloc(const smc2_config* cfg, const double* y_dev,
                                   const double* theta_dev, int n, int iteration,
                                   double* loglik_dev, void* stream);

/* Diagnostic (the paper has no counterpart): the device's FP32 and FP64
 * fused multiply-add throughput in FLOP/s (host outputs, either may be NULL),
 * from kernels of independent FMA chains that fill every SM, timed with CUDA
 * events on `stream`.  These are the arithmetic rates the roofline of the
 * particle filter (FP32) and of the outer FP64 kernels is stated against.
 * Synchronises `stream`; allocates nothing.  Errors: ECUDA. */
smc2_status smc2_fma_rates(double* fp32_flops, double* fp64_flops, void* stream);

/* Surrogate network of the learned proposal (not in the paper; it proposes
 * theta_k in place of the random walk of Sec. IV-A, and the L-kernel weights
 * of Eq. (20) keep the estimator exact): s(x) = w3.h2 + b3, h2 = tanh(W2^T h1
 * + b2), h1 = tanh(W1^T x + b1), hidden width 64, x in R^D (D <= 8).
 * params_dev (device FP32) holds, in order, W1 [D][64], b1 [64], W2 [64][64]
 * (input-major), b2 [64], w3 [64], b3: 64 D + 4289 values, starting on a
 * 16-byte boundary (it is read as float4).  The products run
 * on tensor cores with bfloat16 operands (x, the weights W1, W2, w3, h1, h2
 * and the backward signals rounded to the nearest bfloat16; the biases stay
 * FP32) and FP32 accumulation.
 *
 * smc2_mlp_loss_grad: mean squared error L = (1/R) sum_r (s(x_r) - y_r)^2 of
 * R rows x_dev [R][D] (device FP32), y_dev [R], into *loss_dev and its
 * gradient grad_dev [params] (device FP32).  Allocates its partial sums on
 * `stream` (stream-ordered).  Errors: EINVAL (D outside 1..8, R < 1, a NULL
 * pointer, params_dev not 16-byte aligned).
 * smc2_mlp_input_grad: s(x_r) into s_dev [R] (may be NULL) and ds/dx into
 * dx_dev [R][D].
 * smc2_mlp_adam_step: one training step as the sampler takes it (the same
 * kernel, a thread-block cluster whose CTAs split the rows and reduce their
 * partial gradients over distributed shared memory): the gradient of L at
 * params_dev, then Adam (beta1 = 0.9, beta2 = 0.999, eps = 1e-8,
 * bias-corrected) with learning rate lr at step t = *step_dev + 1 (device
 * int, advanced in place), updating params_dev, m_dev, v_dev (device FP32, one
 * value per parameter); *loss_dev receives L before the update.  Allocates
 * nothing.
 * smc2_mlp_train_ring: the sampler's training call on caller buffers (the
 * same kernel).  From R rows of (theta, log pi^) -- ring_th_dev [R][D] and
 * ring_lp_dev [R], device FP32 -- it forms the training set: tau = max(2, D),
 * z = max((log pi^ - ymax) / tau, -8) with ymax the largest finite log pi^
 * (-8 for a non-finite one), target y = (z - mean z) / sd z over all rows
 * (sd 1 and target variance 0 when var z <= 1e-8), inputs x = (theta - mu) /
 * sd with the mean and standard deviation of the rows above the clip (of
 * every finite row when fewer than 2 D + 2 are; sd at least 1e-6), written
 * to x_dev [R][D] and y_dev [R]; then `steps` Adam steps as
 * smc2_mlp_adam_step takes them, continuing params, m, v and *step_dev.
 * stdz_dev (device FP64, 2 D + 6 values in the layout of
 * smc2_get_learned_state) receives the standardisation and the loss of the
 * last step before its update (0 when steps = 0).  Allocates a few hundred
 * bytes on `stream` (stream-ordered).  Errors: EINVAL (D outside 1..8, R < 1,
 * steps outside 0..256, a NULL pointer, params_dev not 16-byte aligned). */
smc2_status smc2_mlp_loss_grad(int D, const float* params_dev, const float* x_dev, const float* y_dev,
                               int R, float* grad_dev, float* loss_dev, void* stream);
smc2_status smc2_mlp_input_grad(int D, const float* params_dev, const float* x_dev, int R,
                                float* s_dev, float* dx_dev, void* stream);
smc2_status smc2_mlp_adam_step(int D, float* params_dev, float* m_dev, float* v_dev, int* step_dev,
                               const float* x_dev, const float* y_dev, int R, float lr, float* loss_dev,
                               void* stream);
smc2_status smc2_mlp_train_ring(int D, float* params_dev, float* m_dev, float* v_dev, int* step_dev,
                                const float* ring_th_dev, const float* ring_lp_dev, int R, int steps, float lr,
                                float* x_dev, float* y_dev, double* stdz_dev, void* stream);

/* Wait for the context stream and return the sticky device status. */
smc2_status smc2_sync(smc2_ctx* ctx);

/* Device timing of the particle-filter kernel: when enabled, CUDA events
 * bracket every particle-filter launch on the context stream; smc2_get_timing
 * synchronises and returns the summed milliseconds and launch count since
 * the last reset of the counters, plus the number of kernels this context
 * has launched (graph replays count their kernel nodes). */
smc2_status smc2_set_timing(smc2_ctx* ctx, int enable);
smc2_status smc2_get_timing(smc2_ctx* ctx, double* pf_ms, int64_t* pf_launches,
                            int64_t* kernel_launches, int reset);

/* The particle-filter launch shape in use: particles per thread, threads per
 * CTA, CTAs per launch, and the kernel family in *fp32_filter: 0 pf_kernel,
 * 1 the register-resident FP32 filter with one filter per CTA, 2 the same with
 * filter groups of unequal width sharing a CTA (host outputs, any may be
 * NULL). */
smc2_status smc2_get_launch_shape(smc2_ctx* ctx, int* ppt, int* cta_threads, int* grid, int* fp32_filter);

/* Release the context and its device workspace (synchronises its stream). */
void smc2_destroy(smc2_ctx* ctx);

/* The last CUDA runtime failure seen by this thread inside the library, as
 * "call: error name (description)", or "" (thread-local static storage).
 * Diagnostic companion of SMC2_ECUDA / SMC2_ENOMEM. */
const char* smc2_last_error_string(void);

/* Human-readable name of a status code (static storage). */
const char* smc2_status_string(smc2_status s);

#ifdef __cplusplus
}
#endif
#endif /* SMC2_H */
