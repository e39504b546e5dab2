/*
 * smc2_oracle.h -- plain, slow, FP64 CPU oracle of the SMC^2 hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load this code.  It shares no code,
 * header, table or helper with the CUDA library; the two meet only through
 * the seeded synthetic inputs and the random-number definition below, which
 * each side implements on its own from its published description.
 *
 * Conventions (the numerics definition both sides are written from):
 *
 *  Random numbers.  Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel
 *  random numbers: as easy as 1, 2, 3", SC'11), key = (seed low 32 bits,
 *  seed high 32 bits), counter = (c0, c1, c2, c3) with
 *     c2 = theta index i | dataset << 20,   c3 = tag | iteration k << 4.
 *  A 32-bit word w becomes the uniform u = ((w >> 9) + 0.5) * 2^-23 in (0,1)
 *  (exact in float and double);
 *  words (w0,w1) and (w2,w3) become two Box-Muller pairs
 *     r = sqrt(-2 ln u_a),  (r cos 2 pi u_b, r sin 2 pi u_b).
 *  Tags and the meaning of c0, c1:
 *     1 THETA_INIT   c0 = coordinate group g (coordinates 4g..4g+3), c1 = 0
 *     2 PROPOSE      same layout as THETA_INIT
 *     3 OUTER_RES    c0 = c1 = 0, c2 = dataset << 20; word 0 is U
 *     4 PF_INIT      c0 = particle j, c1 = 0; normal 0 is the initial draw
 *     5 PF_PROP      c0 = particle j, c1 = (t-1) >> 2; step t uses normal (t-1) & 3
 *     6 PF_RES       c0 = 0, c1 = t; word 0 is U for the resampling after step t
 *     8 PF_MULTI     c0 = slot j >> 2, c1 = t; word j & 3 is U_j for multinomial
 *                    resampling after step t (one call serves four slots)
 *     9 PF_BINOM     c0 = j + 4096 m, c1 = t: call m of particle j's word stream
 *                    at step t; the SIR model's S -> I draw reads the words of
 *                    calls m = 0, 1, ... in order (x, y, z, w), and its I -> R
 *                    draw continues from where the first stopped.
 *  A word w read by the binomial sampler becomes u = (2w + 1) 2^-33 (exact in
 *  double); a uniform prior draw uses the same form of the THETA_INIT words.
 *
 *  Systematic resampling in integers.  For log-weights l_0..l_{n-1} with
 *  maximum m, q_i = floor(exp(l_i - m) * 2^B) with B = min(52, 63 - ceil(log2 n)),
 *  C_i = q_0 + ... + q_i, S = C_{n-1}, u = (2U + 1) / 2^33, and
 *     cdf^i = n C_i / S,   ncopies^i = ceil(cdf^i - u) - ceil(cdf^{i-1} - u),
 *  evaluated exactly in 128-bit integers, then Algorithm 1 (sequential
 *  redistribution) lays the copies out in index order.
 */
#ifndef SMC2_ORACLE_H
#define SMC2_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORACLE_LG = 0, ORACLE_SEIR = 1, ORACLE_SIR = 2 };
enum { ORACLE_PRIOR_GAUSS = 0, ORACLE_PRIOR_UNIFORM = 1 };
enum { ORACLE_LK_FORWARD = 0, ORACLE_LK_GAUSS = 1 };
enum {
  ORACLE_TAG_THETA_INIT = 1, ORACLE_TAG_PROPOSE = 2, ORACLE_TAG_OUTER_RES = 3,
  ORACLE_TAG_PF_INIT = 4, ORACLE_TAG_PF_PROP = 5, ORACLE_TAG_PF_RES = 6,
  ORACLE_TAG_PF_MULTI = 8, ORACLE_TAG_PF_BINOM = 9
};
enum { ORACLE_PF_SYSTEMATIC = 0, ORACLE_PF_MULTINOMIAL = 1 };
#define ORACLE_MAX_D 8

typedef struct {
  int model;             /* ORACLE_LG, ORACLE_SEIR or ORACLE_SIR */
  int D, N, M, T;        /* dim theta, theta samples, PF particles, time steps */
  int lkernel;           /* ORACLE_LK_FORWARD or ORACLE_LK_GAUSS */
  int dataset;           /* dataset index (random-stream key only) */
  double rw_scale;       /* random-walk proposal standard deviation */
  double ess_frac;       /* outer resampling when ESS < ess_frac * N */
  uint64_t seed;
  double prior_mean[ORACLE_MAX_D], prior_sd[ORACLE_MAX_D];
  /* SEIR constants: population, E0, I0, Euler substeps per day, incidence floor;
   * the SIR model uses npop and i0 */
  double npop, e0, i0, lambda_floor;
  int n_sub;
  /* PF resampling (Sec. II): scheme, and the schedule -- every step t < T when
   * pf_ess_frac <= 0, otherwise when the ESS of the PF weights (Eq. 12) is
   * below pf_ess_frac * M (the paper's choice is multinomial below M/2). */
  int pf_scheme;
  double pf_ess_frac;
  /* Prior: independent Gaussians N(prior_mean, prior_sd^2), or with
   * ORACLE_PRIOR_UNIFORM independent uniforms on [prior_lo, prior_hi]. */
  int prior_kind;
  double prior_lo[ORACLE_MAX_D], prior_hi[ORACLE_MAX_D];
} oracle_cfg;

typedef struct {
  int k, resampled, lk_fallback, pad;
  double lse, lse2, ess, logz;   /* LSE(log w), LSE(2 log w), ESS = l_k, log Z_k */
  double est[ORACLE_MAX_D];      /* f~_k = sum_i w~_k^i theta_k^i */
  double cov[ORACLE_MAX_D * ORACLE_MAX_D];  /* sum_i w~_k^i (theta_k^i - f~_k)(theta_k^i - f~_k)^T, [D][D] */
} oracle_stats;

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double oracle_uniform23(uint32_t w);
void oracle_normals4(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, double z[4]);

double oracle_kalman_loglik(double phi, double sx, double sy, const double* y, int T);

int oracle_fixed_point_bits(int n);
int oracle_quantise(const double* logw, int n, uint64_t* q);
int oracle_systematic_from_q(const uint64_t* q, int n, uint32_t U, int32_t* ncopies, int32_t* anc);
/* Multinomial resampling on the same integer weights: slot j draws its own
 * u_j = (2 U_j + 1) / 2^33 and takes a_j = min{i : C_i > floor(u_j S)},
 * C the inclusive prefix of q.  Returns 0, or -1 when S = 0. */
int oracle_multinomial_from_q(const uint64_t* q, int n, const uint32_t* U, int32_t* anc);
/* ESS of the integer weights, S^2 / sum q^2 (Eq. 12), formed as
 * (double)S * (double)S / ((double)hi * 2^64 + (double)lo) from the exact
 * 128-bit sum of squares hi:lo: every operation correctly rounded, so any
 * machine forms the same value. */
double oracle_ess_from_q(const uint64_t* q, int n);

/* Binomial(n, p) variate from a fresh PF_BINOM-layout word stream with
 * counters (c0 + 4096 m, c1, c2, c3), m = 0, 1, ...  n a non-negative integer.
 * p <= 0 (or NaN) gives 0, p >= 1 gives n; p > 1/2 draws n - Bin(n, 1 - p).
 * n p < 10: inversion, a sequential search from 0 on the pmf recurrence
 * (a redraw if rounding carries the search past n).  Otherwise Hormann's
 * transformed rejection with squeeze (W. Hormann, "The generation of binomial
 * random variates", J. Statist. Comput. Simul. 46, 1993, algorithm BTRS).
 * After 64 calls (256 words; probability below 1e-40 for any n, p) the draw
 * returns floor((n + 1) p).  *words (if not NULL) receives the words read. */
double oracle_binomial(double n, double p, uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                       uint32_t c3, int* words);

double oracle_log_obs(const oracle_cfg* c, const double* theta, const double* x, double y);
/* The filter's step loop body (Sec. II), for stage-wise checks: initial states
 * (M x 5), one step's propagation (Eq. 1) and log-weights (Eq. 2) in place on
 * x, and the word U of the resampling after step t. */
void oracle_pf_initial(const oracle_cfg* c, const double* theta, uint32_t k, uint32_t i, double* x);
void oracle_pf_propagate(const oracle_cfg* c, const double* theta, uint32_t k, uint32_t i, int t, double y,
                         double* x, double* ell);
uint32_t oracle_pf_resample_word(const oracle_cfg* c, uint32_t k, uint32_t i, int t);
void oracle_pf_log_weights(const oracle_cfg* c, const double* theta, const double* x, double y, double* ell);
double oracle_pf_loglik(const oracle_cfg* c, const double* theta, const double* y, uint32_t k,
                        uint32_t i, double* delta_out, int32_t* anc_out);

double oracle_log_prior(const oracle_cfg* c, const double* theta);
int oracle_lkernel_fit(int D, int N, const double* theta_prev, const double* theta_new,
                       const double* wn_prev, double* mu, double* sigma, double* A,
                       double* Lc, double* logdet_c);
double oracle_gauss_lkernel_logpdf(int D, const double* mu, const double* A, const double* Lc,
                                   double logdet_c, const double* a, const double* b);

int oracle_smc2_step(const oracle_cfg* c, const double* y, int k, double* theta, double* logprior,
                     double* loglik, double* logw, oracle_stats* st);

/* Surrogate network of the learned proposal: s(x) = w3 . h2 + b3,
 * h2 = tanh(W2^T h1 + b2), h1 = tanh(W1^T x + b1), x in R^D, hidden width H.
 * Parameters, one vector: W1 [D][H], b1 [H], W2 [H][H] (input-major), b2 [H],
 * w3 [H], b3 -- D H + H H + 3 H + 1 values.  bf16 != 0 rounds, to the nearest
 * bfloat16 (ties to even), the values the tensor-core kernels feed to their
 * products: x, h1, h2 and the backward signals dz2 and dz1. */
double oracle_bf16(double v);
int oracle_mlp_nparams(int D, int H);
void oracle_mlp_forward(int D, int H, const double* params, const double* x, int R, int bf16, double* out);
double oracle_mlp_loss_grad(int D, int H, const double* params, const double* x, const double* y, int R,
                            int bf16, double* grad);
void oracle_mlp_input_grad(int D, int H, const double* params, const double* x, int R, int bf16,
                           double* s_out, double* dx);
void oracle_adam_step(int n, double* params, const double* grad, double* m, double* v, int t, double lr,
                      double beta1, double beta2, double eps);
/* The learned proposal's sampler-side steps (not in the paper; the builder's
 * choices L2-L4 of the learned proposal, written from their statement).  The
 * network proposing at iteration k was trained by the call after iteration
 * k - 2, which continued the parameters and Adam state of the call before it
 * on the (theta, log pi^) pairs of the last W iterations. */
typedef struct {
  double mu[ORACLE_MAX_D], sd[ORACLE_MAX_D]; /* input standardisation */
  double ymax, tau;                          /* z = max((log pi^ - ymax) / tau, -8) */
  double zmean, zsd;                         /* target y = (z - zmean) / zsd */
  double var_y;                              /* variance of the targets: 1, or 0 for constant z */
  int rows;                                  /* rows of the training set */
  int rows_moments;                          /* rows the input moments were taken over */
} oracle_mlp_norm;
void oracle_mlp_weights_bf16(int D, int H, const double* params, double* out);
int oracle_mlp_standardise(int D, int R, const double* th, const double* lp, double* x, double* y,
                           oracle_mlp_norm* nm);
double oracle_mlp_train(int D, int H, int R, const double* th, const double* lp, int steps, double lr,
                        int bf16, double* params, double* m, double* v, int* t, oracle_mlp_norm* nm,
                        double* x_out, double* y_out);
void oracle_mlp_score(int D, int H, const double* params, const oracle_mlp_norm* nm, const double* theta,
                      int R, int bf16, double* score);
int oracle_population_factor(int D, const double* cov, double ess, double* L);
int oracle_learned_decision(int k, double loss, double var_y, int pop_ok);
void oracle_langevin_propose(int D, double h, const double* L, const double* theta_prev, const double* g,
                             const double* z, double* theta_out, double* logq);

void oracle_recycle(int K, int D, const oracle_stats* st, double* est_out, double* c_out);
/* Recycled posterior covariance: Eq. (29) applied to f(theta) = theta theta^T,
 * minus the recycled mean's outer product; cov_out [D][D]. */
void oracle_recycle_cov(int K, int D, const oracle_stats* st, double* cov_out);

#ifdef __cplusplus
}
#endif
#endif
