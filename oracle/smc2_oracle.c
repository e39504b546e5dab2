/*
 * smc2_oracle.c -- plain, slow, FP64 CPU oracle of the SMC^2 hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the CUDA library never
 * does.  Every function follows the paper (Rosato, Varsi, Murphy, Maskell,
 * "An O(log2 N) SMC^2 algorithm on distributed memory with an approx.
 * optimal L-kernel") step by step, in its order and notation, with no
 * blocking, fusion or reordering.  Readings of passages that are garbled or
 * silent are stated where they are used.  The random-number and
 * fixed-point conventions are described in smc2_oracle.h.
 */
#include "smc2_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define LOG_2PI 1.8378770664093454835606594728112

typedef __int128 i128;
typedef unsigned __int128 u128;

/* ------------------------------------------------------------------ */
/* Random numbers                                                      */
/* ------------------------------------------------------------------ */

/* Philox4x32-10 as published by Salmon et al. (SC'11): ten rounds of the
 * Philox S-box on a 4-word counter; each round multiplies words 0 and 2 by
 * the two round multipliers, and the key is bumped by the two Weyl
 * constants between rounds. */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t mult0 = 0xD2511F53u, mult1 = 0xCD9E8D57u;
  const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += weyl0;
      k1 += weyl1;
    }
    uint64_t p0 = (uint64_t)mult0 * (uint64_t)x0;
    uint64_t p1 = (uint64_t)mult1 * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* The 23 high bits of a word, centred in their cell: a uniform on (0,1)
 * that float32 and float64 both hold exactly. */
double oracle_uniform23(uint32_t w) { return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0); }

/* Four standard normals by the Box-Muller transform of the four uniforms. */
void oracle_normals4(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, double z[4]) {
  uint32_t ctr[4] = {c0, c1, c2, c3};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  uint32_t w[4];
  oracle_philox4x32_10(ctr, key, w);
  for (int pair = 0; pair < 2; ++pair) {
    double ua = oracle_uniform23(w[2 * pair]);
    double ub = oracle_uniform23(w[2 * pair + 1]);
    double r = sqrt(-2.0 * log(ua));
    z[2 * pair] = r * cos(2.0 * M_PI * ub);
    z[2 * pair + 1] = r * sin(2.0 * M_PI * ub);
  }
}

static uint32_t oracle_word(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, int idx) {
  uint32_t ctr[4] = {c0, c1, c2, c3};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  uint32_t w[4];
  oracle_philox4x32_10(ctr, key, w);
  return w[idx];
}

static uint32_t oracle_word0(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3) {
  return oracle_word(seed, c0, c1, c2, c3, 0);
}

/* ------------------------------------------------------------------ */
/* Exact likelihood of the linear-Gaussian AR(1) model (Kalman filter)  */
/* ------------------------------------------------------------------ */

/* x_0 ~ N(0,1), x_t = phi x_{t-1} + sx e_t, y_t = x_t + sy n_t, t = 1..T.
 * Returns log p(y_{1:T}) by the prediction-error decomposition. */
double oracle_kalman_loglik(double phi, double sx, double sy, const double* y, int T) {
  double mean = 0.0, var = 1.0, ll = 0.0;
  for (int t = 0; t < T; ++t) {
    mean = phi * mean;
    var = phi * phi * var + sx * sx;
    double s = var + sy * sy;
    double v = y[t] - mean;
    ll += -0.5 * (LOG_2PI + log(s) + v * v / s);
    double gain = var / s;
    mean = mean + gain * v;
    var = (1.0 - gain) * var;
  }
  return ll;
}

/* ------------------------------------------------------------------ */
/* Systematic resampling: Sec. IV-B, Eqs. (26)-(28), Algorithm 1        */
/* ------------------------------------------------------------------ */

/* Fixed-point precision: the largest B <= 52 with n * 2^B < 2^64. */
int oracle_fixed_point_bits(int n) {
  int c = 0;
  while (((int64_t)1 << c) < (int64_t)n) ++c;
  int b = 63 - c;
  return b < 52 ? b : 52;
}

/* q_i = floor(exp(l_i - max l) 2^B): the normalised weights of Eq. (11) up
 * to the common factor 2^B / max w.  Non-finite log-weights get q = 0.
 * Returns B, or -1 when no weight is positive. */
int oracle_quantise(const double* logw, int n, uint64_t* q) {
  double m = -INFINITY;
  for (int i = 0; i < n; ++i)
    if (!isnan(logw[i]) && logw[i] > m) m = logw[i];
  if (!(m > -INFINITY) || isinf(m)) return -1;
  int B = oracle_fixed_point_bits(n);
  for (int i = 0; i < n; ++i) {
    if (isnan(logw[i]) || isinf(logw[i])) {
      q[i] = 0;
    } else {
      double e = ldexp(exp(logw[i] - m), B);
      q[i] = (uint64_t)floor(e);
    }
  }
  return B;
}

static i128 oracle_ceil_div(i128 x, i128 d) { /* d > 0 */
  if (x >= 0) return (x + d - 1) / d;
  return -((-x) / d);
}

/* Choice (Eqs. 26-27) and Redistribution (Algorithm 1).
 * cdf^i = n C_i / S is the cumulative sum of Eq. (26) on the quantised
 * weights; u = (2U+1)/2^33.  The printed Eq. (27) reads
 * ncopies^i = ceil(cdf^{i+1} - u) - ceil(cdf^i - u); with the inclusive
 * cdf of Eq. (26) its indices are one apart, so the oracle takes
 * ncopies^i = ceil(cdf^i - u) - ceil(cdf^{i-1} - u), cdf^{-1} = 0.
 * Each ceil is evaluated exactly as ceil((n C 2^33 - (2U+1) S) / (2^33 S)).
 * Returns 0, or -1 when S = 0 or the counts break Eq. (28). */
int oracle_systematic_from_q(const uint64_t* q, int n, uint32_t U, int32_t* ncopies, int32_t* anc) {
  uint64_t S = 0;
  for (int i = 0; i < n; ++i) S += q[i];
  if (S == 0) return -1;
  const i128 two33 = (i128)1 << 33;
  const i128 den = two33 * (i128)S;
  const i128 uS = (2 * (i128)U + 1) * (i128)S;
  uint64_t C = 0; /* C_{-1} = 0 */
  i128 prev = oracle_ceil_div((i128)n * (i128)C * two33 - uS, den);
  int total = 0;
  for (int i = 0; i < n; ++i) {
    C += q[i];
    i128 cur = oracle_ceil_div((i128)n * (i128)C * two33 - uS, den);
    int nc = (int)(cur - prev);
    if (nc < 0 || nc > n) return -1; /* Eq. (28a) */
    ncopies[i] = nc;
    total += nc;
    prev = cur;
  }
  if (total != n) return -1; /* Eq. (28b) */
  /* Algorithm 1 (S-R): copy item j ncopies^j times, in order of j. */
  int slot = 0;
  for (int j = 0; j < n; ++j)
    for (int copy = 1; copy <= ncopies[j]; ++copy) anc[slot++] = j;
  return 0;
}

/* ------------------------------------------------------------------ */
/* Binomial variates (the SIR flows of Sec. V-A)                        */
/* ------------------------------------------------------------------ */

/* The words of one draw, read in order from Philox calls m = 0, 1, ... */
typedef struct {
  uint32_t key[2], ctr[4], w[4];
  int used, calls, words;
} binom_words;

static void binom_words_init(binom_words* b, uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                             uint32_t c3) {
  b->key[0] = (uint32_t)seed;
  b->key[1] = (uint32_t)(seed >> 32);
  b->ctr[0] = c0;
  b->ctr[1] = c1;
  b->ctr[2] = c2;
  b->ctr[3] = c3;
  b->used = 4;
  b->calls = 0;
  b->words = 0;
}

/* Next uniform (2w + 1) 2^-33 in (0, 1); 0 when the 64 calls are spent. */
static double binom_next_u(binom_words* b) {
  if (b->used == 4) {
    if (b->calls == 64) return 0.0;
    uint32_t ctr[4] = {b->ctr[0] + 4096u * (uint32_t)b->calls, b->ctr[1], b->ctr[2], b->ctr[3]};
    oracle_philox4x32_10(ctr, b->key, b->w);
    b->calls++;
    b->used = 0;
  }
  b->words++;
  return (2.0 * (double)b->w[b->used++] + 1.0) * 0x1p-33;
}

/* log k! through the gamma function. */
static double log_factorial(double k) { return lgamma(k + 1.0); }

/* Bin(n, p) for 0 < p <= 1/2; returns -1 when the words run out. */
static double binom_half(double n, double p, binom_words* b) {
  const double q = 1.0 - p;
  if (n * p < 10.0) {
    /* inversion: P(0) = q^n, P(k) = P(k-1) ((n + 1) s / k - s) with s = p / q */
    const double s = p / q, a = (n + 1.0) * s, r0 = exp(n * log1p(-p));
    for (;;) {
      double u = binom_next_u(b);
      if (u == 0.0) return -1.0;
      double r = r0, k = 0.0;
      while (u > r) {
        u -= r;
        k += 1.0;
        if (k > n) break; /* rounding left u above the total mass: draw again */
        r *= a / k - s;
      }
      if (k <= n) return k;
    }
  }
  /* BTRS: a transformed-rejection proposal k = floor((2a/us + b) u + c) with a
   * squeeze accepting most draws outright; otherwise the exact test of the
   * log-pmf ratio to the mode m against log(v alpha / (a/us^2 + b)). */
  const double spq = sqrt(n * p * q);
  const double bb = 1.15 + 2.53 * spq;
  const double aa = -0.0873 + 0.0248 * bb + 0.01 * p;
  const double c = n * p + 0.5;
  const double vr = 0.92 - 4.2 / bb;
  for (;;) {
    const double u1 = binom_next_u(b);
    const double v1 = binom_next_u(b);
    if (u1 == 0.0 || v1 == 0.0) return -1.0;
    const double u = u1 - 0.5;
    const double us = 0.5 - fabs(u);
    const double k = floor((2.0 * aa / us + bb) * u + c);
    if (k < 0.0 || k > n) continue;
    if (us >= 0.07 && v1 <= vr) return k;
    const double alpha = (2.83 + 5.1 / bb) * spq;
    const double lpq = log(p / q);
    const double m = floor((n + 1.0) * p);
    const double h = log_factorial(m) + log_factorial(n - m);
    const double v = log(v1 * alpha / (aa / (us * us) + bb));
    if (v <= h - log_factorial(k) - log_factorial(n - k) + (k - m) * lpq) return k;
  }
}

/* Bin(n, p) reading the stream b from where it stands. */
static double binomial_from(double n, double p, binom_words* b) {
  if (!(p > 0.0) || n <= 0.0) return 0.0;
  if (!(p < 1.0)) return n;
  if (p > 0.5) {
    const double r = binom_half(n, 1.0 - p, b);
    return r < 0.0 ? floor((n + 1.0) * p) : n - r;
  }
  const double r = binom_half(n, p, b);
  return r < 0.0 ? floor((n + 1.0) * p) : r;
}

double oracle_binomial(double n, double p, uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                       uint32_t c3, int* words) {
  binom_words b;
  binom_words_init(&b, seed, c0, c1, c2, c3);
  const double k = binomial_from(n, p, &b);
  if (words) *words = b.words;
  return k;
}

/* ------------------------------------------------------------------ */
/* State-space models: Sec. II, Eqs. (1)-(2)                            */
/* ------------------------------------------------------------------ */

/* Linear-Gaussian AR(1): theta = (phi, log sx, log sy).
 * SEIR-type: theta = (log beta0, log sigma_rw, log kappa, log gamma); the
 * state is (S, E, I, log beta_t, lambda_t) with R = Npop - S - E - I and
 * lambda_t the day's incidence (the E -> I flow), observed as Poisson.
 * SIR (Sec. V-A): theta = (beta, gamma); the state is (S, I), integers, with
 * R = Npop - S - I, I_0 = i0, and each day the binomial flows
 *   n(S->I) ~ Bin(S, 1 - exp(-beta I / Npop)),  n(I->R) ~ Bin(I, 1 - exp(-gamma)),
 * observed as y_t ~ Poisson(I_t).  The printed S->I probability also carries
 * S_{t-1} in the exponent; the oracle takes the per-susceptible hazard
 * beta I / Npop of the chain-binomial SIR model the section cites. */

static void oracle_initial_state(const oracle_cfg* c, const double* theta, uint32_t k, uint32_t c2,
                                 int j, double* x) {
  if (c->model == ORACLE_LG) {
    double z[4];
    oracle_normals4(c->seed, (uint32_t)j, 0, c2, ORACLE_TAG_PF_INIT | (k << 4), z);
    x[0] = z[0];
  } else if (c->model == ORACLE_SIR) {
    x[0] = c->npop - c->i0;
    x[1] = c->i0;
  } else {
    x[0] = c->npop - c->e0 - c->i0;
    x[1] = c->e0;
    x[2] = c->i0;
    x[3] = theta[0];
    x[4] = 0.0;
  }
}

/* One draw of Eq. (1), the bootstrap proposal q = f. */
static void oracle_propagate(const oracle_cfg* c, const double* theta, double z, double* x) {
  if (c->model == ORACLE_LG) {
    x[0] = theta[0] * x[0] + exp(theta[1]) * z;
  } else {
    double logbeta = x[3] + exp(theta[1]) * z;
    double beta = exp(logbeta), kappa = exp(theta[2]), gamma = exp(theta[3]);
    double dt = 1.0 / (double)c->n_sub;
    double S = x[0], E = x[1], I = x[2], lambda = 0.0;
    for (int s = 0; s < c->n_sub; ++s) {
      double infection = beta * S * I / c->npop;
      double onset = kappa * E;
      double recovery = gamma * I;
      lambda += dt * onset;
      S = fmax(S - dt * infection, 0.0);
      E = fmax(E + dt * (infection - onset), 0.0);
      I = fmax(I + dt * (onset - recovery), 0.0);
    }
    x[0] = S; x[1] = E; x[2] = I; x[3] = logbeta;
    x[4] = fmax(lambda, c->lambda_floor);
  }
}

/* One day of the SIR model for particle j at step t: both flows from the
 * previous day's (S, I); probabilities 1 - exp(-h) formed as -expm1(-h).  The
 * two draws read one word stream, the I->R draw from where the S->I draw
 * stopped. */
static void oracle_propagate_sir(const oracle_cfg* c, const double* theta, uint32_t k, uint32_t c2,
                                 int j, int t, double* x) {
  const double S = x[0], I = x[1];
  const double p_si = -expm1(-(theta[0] * I / c->npop));
  const double p_ir = -expm1(-theta[1]);
  binom_words b;
  binom_words_init(&b, c->seed, (uint32_t)j, (uint32_t)t, c2, ORACLE_TAG_PF_BINOM | (k << 4));
  const double n_si = binomial_from(S, p_si, &b);
  const double n_ir = binomial_from(I, p_ir, &b);
  x[0] = S - n_si;
  x[1] = I + n_si - n_ir;
}

/* log g(y_t | x_t, theta), Eq. (2). */
double oracle_log_obs(const oracle_cfg* c, const double* theta, const double* x, double y) {
  if (c->model == ORACLE_SIR) { /* Poisson(y; I), a point mass at 0 when I = 0 */
    const double I = x[1];
    if (I > 0.0) return (y > 0.0 ? y * log(I) : 0.0) - I - lgamma(y + 1.0);
    return y > 0.0 ? -INFINITY : 0.0;
  }
  if (c->model == ORACLE_LG) {
    double sy = exp(theta[2]);
    double r = (y - x[0]) / sy;
    return -0.5 * LOG_2PI - log(sy) - 0.5 * r * r;
  } else {
    double lambda = x[4];
    return (y > 0.0 ? y * log(lambda) : 0.0) - lambda - lgamma(y + 1.0);
  }
}

/* ------------------------------------------------------------------ */
/* Bootstrap particle filter: Sec. II                                   */
/* ------------------------------------------------------------------ */

/* Multinomial resampling on integer weights q (Sec. II): slot j takes the
 * first index i whose cumulative weight C_i exceeds floor(u_j S), with
 * u_j = (2 U_j + 1) / 2^33 from its own word U_j.  Returns -1 when S = 0. */
int oracle_multinomial_from_q(const uint64_t* q, int n, const uint32_t* U, int32_t* anc) {
  uint64_t* C = (uint64_t*)malloc(sizeof(uint64_t) * n);
  uint64_t S = 0;
  for (int i = 0; i < n; ++i) {
    S += q[i];
    C[i] = S;
  }
  if (S == 0) {
    free(C);
    return -1;
  }
  for (int j = 0; j < n; ++j) {
    const unsigned __int128 num = (unsigned __int128)(2ull * U[j] + 1ull) * S;
    const uint64_t tau = (uint64_t)(num >> 33); /* floor(u_j S), u_j < 1 so tau < S */
    int lo = 0, hi = n - 1;                     /* smallest i with C_i > tau */
    while (lo < hi) {
      const int mid = (lo + hi) / 2;
      if (C[mid] > tau)
        hi = mid;
      else
        lo = mid + 1;
    }
    anc[j] = lo;
  }
  free(C);
  return 0;
}

double oracle_ess_from_q(const uint64_t* q, int n) {
  uint64_t S = 0;
  unsigned __int128 Q2 = 0;
  for (int i = 0; i < n; ++i) {
    S += q[i];
    Q2 += (unsigned __int128)q[i] * q[i];
  }
  const double q2 = (double)(uint64_t)(Q2 >> 64) * 0x1p64 + (double)(uint64_t)Q2;
  return (double)S * (double)S / q2;
}

/* The body of the filter's step loop, exposed for stage-wise checks: the
 * initial states of filter i at iteration k (M x 5, the layout below), and one
 * step t: every particle j propagated by Eq. (1) with the step's normal of slot
 * j (or its binomial flows), then ell[j] = log g(y_t | x_j) (Eq. 2; -inf for a
 * NaN).  oracle_pf_loglik runs the same two functions in its loop. */
void oracle_pf_initial(const oracle_cfg* c, const double* theta, uint32_t k, uint32_t i, double* x) {
  const uint32_t c2 = i | ((uint32_t)c->dataset << 20);
  for (int j = 0; j < c->M; ++j) oracle_initial_state(c, theta, k, c2, j, x + 5 * j);
}

void oracle_pf_propagate(const oracle_cfg* c, const double* theta, uint32_t k, uint32_t i, int t, double y,
                         double* x, double* ell) {
  const uint32_t c2 = i | ((uint32_t)c->dataset << 20);
  for (int j = 0; j < c->M; ++j) {
    double* xj = x + 5 * j;
    if (c->model == ORACLE_SIR) {
      oracle_propagate_sir(c, theta, k, c2, j, t, xj);
    } else {
      double z[4];
      oracle_normals4(c->seed, (uint32_t)j, (uint32_t)((t - 1) >> 2), c2, ORACLE_TAG_PF_PROP | (k << 4), z);
      oracle_propagate(c, theta, z[(t - 1) & 3], xj);
    }
    const double l = oracle_log_obs(c, theta, xj, y);
    ell[j] = isnan(l) ? -INFINITY : l;
  }
}

/* ell[j] = log g(y | x_j) (Eq. 2; -inf for a NaN) for the M states x (M x 5). */
void oracle_pf_log_weights(const oracle_cfg* c, const double* theta, const double* x, double y, double* ell) {
  for (int j = 0; j < c->M; ++j) {
    const double l = oracle_log_obs(c, theta, x + 5 * j, y);
    ell[j] = isnan(l) ? -INFINITY : l;
  }
}

/* The word U of the systematic resampling after step t of filter i at iteration k. */
uint32_t oracle_pf_resample_word(const oracle_cfg* c, uint32_t k, uint32_t i, int t) {
  const uint32_t c2 = i | ((uint32_t)c->dataset << 20);
  return oracle_word0(c->seed, 0, (uint32_t)t, c2, ORACLE_TAG_PF_RES | (k << 4));
}

/* Returns log p^(y_{1:T} | theta), Eq. (8), for filter i of iteration k.
 * The unnormalised weight of particle j is carried as exp(L + lw_j): L is
 * the log of the common weight given to every particle at the last reset
 * (Eq. 13), lw_j the log of the product of the Eq. (5) factors since then
 * (with q = f the factor is g(y_t | x_t)).  After step t < T the filter
 * resamples -- systematically, or multinomially with pf_scheme = 1 -- at
 * every step, or with pf_ess_frac > 0 only when the ESS of Eq. (12) is
 * below pf_ess_frac M.  delta_out (T entries) receives
 * log p^(y_{1:t}) - log p^(y_{1:t-1}); anc_out ((T-1) x M) the ancestors
 * (the identity on steps that keep every particle). */
double oracle_pf_loglik(const oracle_cfg* c, const double* theta, const double* y, uint32_t k,
                        uint32_t i, double* delta_out, int32_t* anc_out) {
  const int M = c->M, T = c->T, SD = 5;
  const uint32_t c2 = i | ((uint32_t)c->dataset << 20);
  double* x = (double*)malloc(sizeof(double) * M * SD);
  double* xn = (double*)malloc(sizeof(double) * M * SD);
  double* lw = (double*)malloc(sizeof(double) * M);
  uint64_t* q = (uint64_t*)malloc(sizeof(uint64_t) * M);
  int32_t* ncop = (int32_t*)malloc(sizeof(int32_t) * M);
  int32_t* anc = (int32_t*)malloc(sizeof(int32_t) * M);
  oracle_pf_initial(c, theta, k, i, x);
  for (int j = 0; j < M; ++j) lw[j] = 0.0;
  double L = 0.0;    /* log of the common weight: w_0 = 1 */
  double loglik = 0.0; /* log p^(y_{1:t}) */
  uint32_t* Um = (uint32_t*)malloc(sizeof(uint32_t) * M);
  double* ell = (double*)malloc(sizeof(double) * M);
  for (int t = 1; t <= T; ++t) {
    oracle_pf_propagate(c, theta, k, i, t, y[t - 1], x, ell);
    for (int j = 0; j < M; ++j) lw[j] = lw[j] + ell[j]; /* Eq. (5) in logs */
    double m = -INFINITY;
    for (int j = 0; j < M; ++j)
      if (lw[j] > m) m = lw[j];
    if (!(m > -INFINITY)) { /* every weight is zero: p^ = 0 */
      for (int s = t; s <= T; ++s)
        if (delta_out) delta_out[s - 1] = -INFINITY;
      loglik = -INFINITY;
      goto done;
    }
    double sum = 0.0;
    for (int j = 0; j < M; ++j) sum += exp(lw[j] - m);
    /* Eq. (8): log of (1/M) sum_j exp(L + lw_j). */
    double logp = L + m + log(sum) - log((double)M);
    if (delta_out) delta_out[t - 1] = logp - loglik;
    loglik = logp;
    if (t < T) {
      oracle_quantise(lw, M, q);
      /* the schedule: every step, or when the ESS (Eq. 12) is below pf_ess_frac M */
      const int resample = !(c->pf_ess_frac > 0.0) || oracle_ess_from_q(q, M) < c->pf_ess_frac * (double)M;
      if (resample) {
        if (c->pf_scheme == ORACLE_PF_MULTINOMIAL) {
          for (int j = 0; j < M; ++j)
            Um[j] = oracle_word(c->seed, (uint32_t)j >> 2, (uint32_t)t, c2, ORACLE_TAG_PF_MULTI | (k << 4), j & 3);
          oracle_multinomial_from_q(q, M, Um, anc);
        } else {
          oracle_systematic_from_q(q, M, oracle_pf_resample_word(c, k, i, t), ncop, anc);
        }
        for (int j = 0; j < M; ++j) memcpy(xn + SD * j, x + SD * anc[j], sizeof(double) * SD);
        double* tmp = x; x = xn; xn = tmp;
        /* Eq. (13): every particle now carries the mean weight. */
        L = logp;
        for (int j = 0; j < M; ++j) lw[j] = 0.0;
      } else {
        for (int j = 0; j < M; ++j) anc[j] = j; /* no resampling: each particle keeps its weight */
      }
      if (anc_out) memcpy(anc_out + (size_t)(t - 1) * M, anc, sizeof(int32_t) * M);
    }
  }
done:
  free(x); free(xn); free(lw); free(q); free(ncop); free(anc); free(Um); free(ell);
  return loglik;
}

/* ------------------------------------------------------------------ */
/* SMC^2 outer sampler: Sec. IV                                         */
/* ------------------------------------------------------------------ */

/* log p(theta): independent Gaussians in the unconstrained coordinates, or
 * independent uniforms on [lo, hi] (-inf outside). */
double oracle_log_prior(const oracle_cfg* c, const double* theta) {
  double lp = 0.0;
  if (c->prior_kind == ORACLE_PRIOR_UNIFORM) {
    for (int d = 0; d < c->D; ++d) {
      if (!(theta[d] >= c->prior_lo[d] && theta[d] <= c->prior_hi[d])) return -INFINITY;
      lp -= log(c->prior_hi[d] - c->prior_lo[d]);
    }
    return lp;
  }
  for (int d = 0; d < c->D; ++d) {
    double r = (theta[d] - c->prior_mean[d]) / c->prior_sd[d];
    lp += -0.5 * LOG_2PI - log(c->prior_sd[d]) - 0.5 * r * r;
  }
  return lp;
}

static double oracle_gauss_iso_logpdf(int D, const double* x, const double* mean, double sd) {
  double ss = 0.0;
  for (int d = 0; d < D; ++d) {
    double r = (x[d] - mean[d]) / sd;
    ss += r * r;
  }
  return -0.5 * D * LOG_2PI - D * log(sd) - 0.5 * ss;
}

/* Lower Cholesky factor of the n x n matrix a (row-major).  A pivot counts
 * as zero (return -1) unless it exceeds 1e-12 (a_jj + mean_j^2): below that
 * the fitted variance is rounding noise of the second moment. */
static int oracle_cholesky(int n, const double* a, const double* mean, double* l) {
  memset(l, 0, sizeof(double) * n * n);
  for (int j = 0; j < n; ++j) {
    double s = a[j * n + j];
    for (int p = 0; p < j; ++p) s -= l[j * n + p] * l[j * n + p];
    double floor_j = 1e-12 * (a[j * n + j] + mean[j] * mean[j]);
    if (!(s > floor_j) || !isfinite(s)) return -1;
    l[j * n + j] = sqrt(s);
    for (int r = j + 1; r < n; ++r) {
      double v = a[r * n + j];
      for (int p = 0; p < j; ++p) v -= l[r * n + p] * l[j * n + p];
      l[r * n + j] = v / l[j * n + j];
    }
  }
  return 0;
}

/* Approximately optimal L-kernel, Sec. IV-D, Eqs. (32)-(35).
 * a = theta_{k-1} (parents), b = theta_k (their proposals), weighted by the
 * normalised parent weights.  Eq. (32): fit a joint Gaussian to (a, b)
 * (weighted mean and covariance, normalised by the weight sum).
 * Eqs. (33)-(35) print the conditional with its factors transposed and the
 * density argument as theta_k; the oracle takes the Gaussian conditional of
 * a given b:
 *   mu_{a|b}(b) = mu_a + S_ab S_bb^{-1} (b - mu_b),
 *   S_{a|b}     = S_aa - S_ab S_bb^{-1} S_ba,
 *   L(a | b)    = N(a; mu_{a|b}(b), S_{a|b}).
 * Outputs: mu (2D), sigma (2D x 2D), A = S_ab S_bb^{-1} (D x D), Lc =
 * chol(S_{a|b}) and log det S_{a|b}.  Returns 0, or 1 when S_bb or S_{a|b}
 * is numerically singular (the caller then uses the forward kernel, Eq. 30). */
int oracle_lkernel_fit(int D, int N, const double* theta_prev, const double* theta_new,
                       const double* wn_prev, double* mu, double* sigma, double* A, double* Lc,
                       double* logdet_c) {
  const int D2 = 2 * D;
  double wsum = 0.0;
  for (int i = 0; i < N; ++i) wsum += wn_prev[i];
  for (int r = 0; r < D2; ++r) {
    double s = 0.0;
    for (int i = 0; i < N; ++i) {
      double z = r < D ? theta_prev[i * D + r] : theta_new[i * D + (r - D)];
      s += wn_prev[i] * z;
    }
    mu[r] = s / wsum;
  }
  for (int r = 0; r < D2; ++r) {
    for (int s = 0; s < D2; ++s) {
      double acc = 0.0;
      for (int i = 0; i < N; ++i) {
        double zr = r < D ? theta_prev[i * D + r] : theta_new[i * D + (r - D)];
        double zs = s < D ? theta_prev[i * D + s] : theta_new[i * D + (s - D)];
        acc += wn_prev[i] * (zr - mu[r]) * (zs - mu[s]);
      }
      sigma[r * D2 + s] = acc / wsum;
    }
  }
  double saa[ORACLE_MAX_D * ORACLE_MAX_D], sab[ORACLE_MAX_D * ORACLE_MAX_D];
  double sbb[ORACLE_MAX_D * ORACLE_MAX_D], lb[ORACLE_MAX_D * ORACLE_MAX_D];
  for (int r = 0; r < D; ++r)
    for (int s = 0; s < D; ++s) {
      saa[r * D + s] = sigma[r * D2 + s];
      sab[r * D + s] = sigma[r * D2 + (D + s)];
      sbb[r * D + s] = sigma[(D + r) * D2 + (D + s)];
    }
  if (oracle_cholesky(D, sbb, mu + D, lb) != 0) return 1;
  /* A = S_ab S_bb^{-1}: solve S_bb X = S_ba (= S_ab^T) column by column, A = X^T. */
  for (int col = 0; col < D; ++col) {
    double rhs[ORACLE_MAX_D], tmp[ORACLE_MAX_D], sol[ORACLE_MAX_D];
    for (int r = 0; r < D; ++r) rhs[r] = sab[col * D + r]; /* column col of S_ba */
    for (int r = 0; r < D; ++r) {                          /* forward: lb tmp = rhs */
      double v = rhs[r];
      for (int p = 0; p < r; ++p) v -= lb[r * D + p] * tmp[p];
      tmp[r] = v / lb[r * D + r];
    }
    for (int r = D - 1; r >= 0; --r) { /* backward: lb^T sol = tmp */
      double v = tmp[r];
      for (int p = r + 1; p < D; ++p) v -= lb[p * D + r] * sol[p];
      sol[r] = v / lb[r * D + r];
    }
    for (int r = 0; r < D; ++r) A[col * D + r] = sol[r]; /* row col of A */
  }
  double sc[ORACLE_MAX_D * ORACLE_MAX_D];
  for (int r = 0; r < D; ++r)
    for (int s = 0; s < D; ++s) {
      double v = saa[r * D + s];
      for (int p = 0; p < D; ++p) v -= A[r * D + p] * sab[s * D + p]; /* (A S_ba)_{rs} */
      sc[r * D + s] = v;
    }
  if (oracle_cholesky(D, sc, mu, Lc) != 0) return 1;
  double ld = 0.0;
  for (int r = 0; r < D; ++r) ld += 2.0 * log(Lc[r * D + r]);
  *logdet_c = ld;
  return 0;
}

/* log N(a; mu_a + A (b - mu_b), Lc Lc^T), Eq. (33) under the reading above. */
double oracle_gauss_lkernel_logpdf(int D, const double* mu, const double* A, const double* Lc,
                                   double logdet_c, const double* a, const double* b) {
  double r[ORACLE_MAX_D], v[ORACLE_MAX_D];
  for (int p = 0; p < D; ++p) {
    double m = mu[p];
    for (int s = 0; s < D; ++s) m += A[p * D + s] * (b[s] - mu[D + s]);
    r[p] = a[p] - m;
  }
  double ss = 0.0;
  for (int p = 0; p < D; ++p) {
    double s = r[p];
    for (int l = 0; l < p; ++l) s -= Lc[p * D + l] * v[l];
    v[p] = s / Lc[p * D + p];
    ss += v[p] * v[p];
  }
  return -0.5 * D * LOG_2PI - 0.5 * logdet_c - 0.5 * ss;
}

/* Eqs. (22), (21), (24), (25): normalise, estimate, recycling constant,
 * ESS, and the evidence estimate log Z_k = log((1/N) sum_i w_k^i). */
static int oracle_normalise(const oracle_cfg* c, const double* theta, const double* logw,
                            oracle_stats* st) {
  const int N = c->N, D = c->D;
  double m = -INFINITY;
  for (int i = 0; i < N; ++i)
    if (logw[i] > m) m = logw[i];
  if (!(m > -INFINITY) || isinf(m)) return 4;
  double sw = 0.0, sw2 = 0.0;
  for (int i = 0; i < N; ++i) {
    double w = exp(logw[i] - m);
    sw += w;
    sw2 += w * w;
  }
  st->lse = m + log(sw);
  st->lse2 = 2.0 * m + log(sw2);
  double sum_wn2 = 0.0;
  for (int d = 0; d < D; ++d) st->est[d] = 0.0;
  for (int i = 0; i < N; ++i) {
    double wn = exp(logw[i] - m) / sw; /* Eq. (22) */
    sum_wn2 += wn * wn;
    for (int d = 0; d < D; ++d) st->est[d] += wn * theta[i * D + d]; /* Eq. (21) */
  }
  /* Eq. (21) with f = (theta - f~)(theta - f~)^T: the weighted covariance, second pass */
  for (int d = 0; d < D * D; ++d) st->cov[d] = 0.0;
  for (int i = 0; i < N; ++i) {
    double wn = exp(logw[i] - m) / sw;
    for (int d = 0; d < D; ++d)
      for (int e = 0; e < D; ++e)
        st->cov[d * D + e] += wn * (theta[i * D + d] - st->est[d]) * (theta[i * D + e] - st->est[e]);
  }
  st->ess = 1.0 / sum_wn2; /* Eq. (25); equals l_k of Eq. (24) */
  st->logz = st->lse - log((double)N);
  return 0;
}

/* One SMC^2 iteration k (1-based) in place on the population (row-major
 * theta[N][D], logprior, loglik, logw).  On entry the arrays hold the
 * population after iteration k-1 (ignored for k = 1); on exit they hold
 * iteration k after the resampling decision.  Returns 0, or 4 when every
 * outer weight is zero. */
int oracle_smc2_step(const oracle_cfg* c, const double* y, int k, double* theta, double* logprior,
                     double* loglik, double* logw, oracle_stats* st) {
  const int N = c->N, D = c->D;
  const uint32_t ds = (uint32_t)c->dataset << 20;
  memset(st, 0, sizeof(*st));
  st->k = k;
  double* th_new = (double*)malloc(sizeof(double) * N * D);
  double* lp_new = (double*)malloc(sizeof(double) * N);
  double* ll_new = (double*)malloc(sizeof(double) * N);
  double* lw_new = (double*)malloc(sizeof(double) * N);
  int rc = 0;
  if (k == 1) {
    /* Eq. (16): theta_1^i ~ q_1 = prior; Eq. (17): w_1 = pi / q_1. */
    for (int i = 0; i < N; ++i) {
      for (int g = 0; g * 4 < D; ++g) {
        const uint32_t c3 = ORACLE_TAG_THETA_INIT | ((uint32_t)k << 4);
        if (c->prior_kind == ORACLE_PRIOR_UNIFORM) { /* theta_d = lo + (hi - lo) u, u = (2w + 1) 2^-33 */
          const uint32_t ctr[4] = {(uint32_t)g, 0u, (uint32_t)i | ds, c3};
          const uint32_t key[2] = {(uint32_t)c->seed, (uint32_t)(c->seed >> 32)};
          uint32_t w[4];
          oracle_philox4x32_10(ctr, key, w);
          for (int r = 0; r < 4 && 4 * g + r < D; ++r) {
            int d = 4 * g + r;
            double u = (2.0 * (double)w[r] + 1.0) * 0x1p-33;
            th_new[i * D + d] = c->prior_lo[d] + (c->prior_hi[d] - c->prior_lo[d]) * u;
          }
          continue;
        }
        double z[4];
        oracle_normals4(c->seed, (uint32_t)g, 0, (uint32_t)i | ds, c3, z);
        for (int r = 0; r < 4 && 4 * g + r < D; ++r) {
          int d = 4 * g + r;
          th_new[i * D + d] = c->prior_mean[d] + c->prior_sd[d] * z[r];
        }
      }
      lp_new[i] = oracle_log_prior(c, th_new + i * D);
      ll_new[i] = oracle_pf_loglik(c, th_new + i * D, y, (uint32_t)k, (uint32_t)i, NULL, NULL);
      double logq1 = oracle_log_prior(c, th_new + i * D);
      lw_new[i] = (lp_new[i] + ll_new[i]) - logq1;
    }
  } else {
    /* Normalised parent weights (Eq. 22 at k-1) for the L-kernel fit. */
    double m = -INFINITY, sw = 0.0;
    for (int i = 0; i < N; ++i)
      if (logw[i] > m) m = logw[i];
    double* wn = (double*)malloc(sizeof(double) * N);
    for (int i = 0; i < N; ++i) sw += exp(logw[i] - m);
    for (int i = 0; i < N; ++i) wn[i] = exp(logw[i] - m) / sw;
    /* Eqs. (18)-(19): theta_k^i ~ N(theta_{k-1}^i, rw_scale^2 I). */
    double* logq = (double*)malloc(sizeof(double) * N);
    for (int i = 0; i < N; ++i) {
      for (int g = 0; g * 4 < D; ++g) {
        double z[4];
        oracle_normals4(c->seed, (uint32_t)g, 0, (uint32_t)i | ds,
                        ORACLE_TAG_PROPOSE | ((uint32_t)k << 4), z);
        for (int r = 0; r < 4 && 4 * g + r < D; ++r) {
          int d = 4 * g + r;
          th_new[i * D + d] = theta[i * D + d] + c->rw_scale * z[r];
        }
      }
      logq[i] = oracle_gauss_iso_logpdf(D, th_new + i * D, theta + i * D, c->rw_scale);
      lp_new[i] = oracle_log_prior(c, th_new + i * D);
      ll_new[i] = oracle_pf_loglik(c, th_new + i * D, y, (uint32_t)k, (uint32_t)i, NULL, NULL);
    }
    /* L-kernel (Sec. IV-D). */
    double mu[2 * ORACLE_MAX_D], sigma[4 * ORACLE_MAX_D * ORACLE_MAX_D];
    double A[ORACLE_MAX_D * ORACLE_MAX_D], Lc[ORACLE_MAX_D * ORACLE_MAX_D], logdet_c = 0.0;
    int fallback = 1;
    if (c->lkernel == ORACLE_LK_GAUSS)
      fallback = oracle_lkernel_fit(D, N, theta, th_new, wn, mu, sigma, A, Lc, &logdet_c);
    st->lk_fallback = (c->lkernel == ORACLE_LK_GAUSS) ? fallback : 0;
    for (int i = 0; i < N; ++i) {
      double logL;
      if (fallback) /* Eq. (30): L(a | b) = q(a | b) */
        logL = oracle_gauss_iso_logpdf(D, theta + i * D, th_new + i * D, c->rw_scale);
      else
        logL = oracle_gauss_lkernel_logpdf(D, mu, A, Lc, logdet_c, theta + i * D, th_new + i * D);
      /* Eq. (20) in logs. */
      lw_new[i] = logw[i] + (lp_new[i] + ll_new[i]) - (logprior[i] + loglik[i]) + logL - logq[i];
      if (isnan(lw_new[i])) lw_new[i] = -INFINITY;
    }
    free(wn);
    free(logq);
  }
  memcpy(theta, th_new, sizeof(double) * N * D);
  memcpy(logprior, lp_new, sizeof(double) * N);
  memcpy(loglik, ll_new, sizeof(double) * N);
  memcpy(logw, lw_new, sizeof(double) * N);
  rc = oracle_normalise(c, theta, logw, st);
  if (rc != 0) goto out;
  /* Sec. IV-B: resample when N_eff < ess_frac N (the paper uses N/2). */
  if (st->ess < c->ess_frac * (double)N) {
    uint64_t* q = (uint64_t*)malloc(sizeof(uint64_t) * N);
    int32_t* ncop = (int32_t*)malloc(sizeof(int32_t) * N);
    int32_t* anc = (int32_t*)malloc(sizeof(int32_t) * N);
    uint32_t U = oracle_word0(c->seed, 0, 0, ds, ORACLE_TAG_OUTER_RES | ((uint32_t)k << 4));
    oracle_quantise(logw, N, q);
    oracle_systematic_from_q(q, N, U, ncop, anc);
    for (int j = 0; j < N; ++j) {
      memcpy(theta + j * D, th_new + anc[j] * D, sizeof(double) * D);
      logprior[j] = lp_new[anc[j]];
      loglik[j] = ll_new[anc[j]];
    }
    /* Reset: every normalised weight becomes 1/N; the unnormalised weight
     * is the mean (1/N) sum_i w_k^i, which keeps the evidence estimate. */
    for (int j = 0; j < N; ++j) logw[j] = st->lse - log((double)N);
    st->resampled = 1;
    free(q); free(ncop); free(anc);
  }
out:
  free(th_new); free(lp_new); free(ll_new); free(lw_new);
  return rc;
}

/* Recycling, Sec. IV-C and Eqs. (23)-(24), (29): c_k = l_k / sum_k l_k and
 * f~ = sum_k c_k f~_k, with l_k the ESS of iteration k. */
void oracle_recycle(int K, int D, const oracle_stats* st, double* est_out, double* c_out) {
  double lsum = 0.0;
  for (int k = 0; k < K; ++k) lsum += st[k].ess;
  for (int d = 0; d < D; ++d) est_out[d] = 0.0;
  for (int k = 0; k < K; ++k) {
    double ck = st[k].ess / lsum;
    if (c_out) c_out[k] = ck;
    for (int d = 0; d < D; ++d) est_out[d] += ck * st[k].est[d];
  }
}

void oracle_recycle_cov(int K, int D, const oracle_stats* st, double* cov_out) {
  double lsum = 0.0, mean[ORACLE_MAX_D] = {0.0};
  for (int k = 0; k < K; ++k) lsum += st[k].ess;
  for (int d = 0; d < D * D; ++d) cov_out[d] = 0.0;
  for (int k = 0; k < K; ++k) {
    const double ck = st[k].ess / lsum; /* Eqs. (23), (24) */
    for (int d = 0; d < D; ++d) {
      mean[d] += ck * st[k].est[d];
      for (int e = 0; e < D; ++e)  /* the recycled second moment E[theta_d theta_e] */
        cov_out[d * D + e] += ck * (st[k].cov[d * D + e] + st[k].est[d] * st[k].est[e]);
    }
  }
  for (int d = 0; d < D; ++d)
    for (int e = 0; e < D; ++e) cov_out[d * D + e] -= mean[d] * mean[e];
}

/* ------------------------------------------------------------------ */
/* Surrogate network of the learned proposal (not in the paper)         */
/* ------------------------------------------------------------------ */

/* Nearest bfloat16 (8 exponent bits, 7 fraction bits), ties to even,
 * returned as a double.  Finite inputs only. */
double oracle_bf16(double v) {
  float f = (float)v;
  uint32_t u;
  memcpy(&u, &f, sizeof(u));
  uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;
  u &= 0xffff0000u;
  memcpy(&f, &u, sizeof(f));
  return (double)f;
}

int oracle_mlp_nparams(int D, int H) { return D * H + H * H + 3 * H + 1; }

static double oracle_round(double v, int bf16) { return bf16 ? oracle_bf16(v) : v; }

/* One row: z1 = W1^T x + b1, h1 = tanh z1, z2 = W2^T h1 + b2, h2 = tanh z2,
 * s = w3 . h2 + b3.  h1r, h2r are the values fed to the next product. */
static double oracle_mlp_row(int D, int H, const double* p, const double* x, int bf16, double* h1,
                             double* h1r, double* h2, double* h2r) {
  const double *W1 = p, *b1 = W1 + D * H, *W2 = b1 + H, *b2 = W2 + H * H, *w3 = b2 + H, *b3 = w3 + H;
  for (int o = 0; o < H; ++o) {
    double z = b1[o];
    for (int d = 0; d < D; ++d) z += oracle_round(x[d], bf16) * W1[d * H + o];
    h1[o] = tanh(z);
    h1r[o] = oracle_round(h1[o], bf16);
  }
  for (int o = 0; o < H; ++o) {
    double z = b2[o];
    for (int i = 0; i < H; ++i) z += h1r[i] * W2[i * H + o];
    h2[o] = tanh(z);
    h2r[o] = oracle_round(h2[o], bf16);
  }
  double sv = b3[0];
  for (int i = 0; i < H; ++i) sv += h2r[i] * w3[i];
  return sv;
}

void oracle_mlp_forward(int D, int H, const double* params, const double* x, int R, int bf16, double* out) {
  double* buf = (double*)malloc(sizeof(double) * 4 * H);
  for (int r = 0; r < R; ++r)
    out[r] = oracle_mlp_row(D, H, params, x + (size_t)r * D, bf16, buf, buf + H, buf + 2 * H, buf + 3 * H);
  free(buf);
}

/* Back-propagation of a signal g (ds) through one row; adds the parameter
 * gradients scaled by g to grad (if not NULL) and writes ds/dx * g to dx
 * (if not NULL). */
static void oracle_mlp_back_row(int D, int H, const double* p, const double* x, const double* h1,
                                const double* h1r, const double* h2, const double* h2r, double g,
                                int bf16, double* grad, double* dx) {
  const double *W1 = p, *W2 = W1 + D * H + H, *w3 = W2 + H * H + H;
  double* dz2 = (double*)malloc(sizeof(double) * 2 * H);
  double* dz1 = dz2 + H;
  for (int o = 0; o < H; ++o) dz2[o] = oracle_round(g * w3[o] * (1.0 - h2[o] * h2[o]), bf16);
  for (int i = 0; i < H; ++i) {
    double dh = 0.0;
    for (int o = 0; o < H; ++o) dh += W2[i * H + o] * dz2[o];
    dz1[i] = oracle_round(dh * (1.0 - h1[i] * h1[i]), bf16);
  }
  if (grad) {
    double *gW1 = grad, *gb1 = gW1 + D * H, *gW2 = gb1 + H, *gb2 = gW2 + H * H, *gw3 = gb2 + H,
           *gb3 = gw3 + H;
    for (int d = 0; d < D; ++d)
      for (int o = 0; o < H; ++o) gW1[d * H + o] += oracle_round(x[d], bf16) * dz1[o];
    for (int o = 0; o < H; ++o) gb1[o] += dz1[o];
    for (int i = 0; i < H; ++i)
      for (int o = 0; o < H; ++o) gW2[i * H + o] += h1r[i] * dz2[o];
    for (int o = 0; o < H; ++o) gb2[o] += dz2[o];
    for (int i = 0; i < H; ++i) gw3[i] += h2r[i] * g;
    gb3[0] += g;
  }
  if (dx)
    for (int d = 0; d < D; ++d) {
      double v = 0.0;
      for (int o = 0; o < H; ++o) v += W1[d * H + o] * dz1[o];
      dx[d] = v;
    }
  free(dz2);
}

/* Mean squared error L = (1/R) sum_r (s(x_r) - y_r)^2 and its gradient. */
double oracle_mlp_loss_grad(int D, int H, const double* params, const double* x, const double* y, int R,
                            int bf16, double* grad) {
  const int P = oracle_mlp_nparams(D, H);
  double* buf = (double*)malloc(sizeof(double) * 4 * H);
  for (int q = 0; q < P; ++q) grad[q] = 0.0;
  double loss = 0.0;
  for (int r = 0; r < R; ++r) {
    const double* xr = x + (size_t)r * D;
    double sv = oracle_mlp_row(D, H, params, xr, bf16, buf, buf + H, buf + 2 * H, buf + 3 * H);
    double e = sv - y[r];
    loss += e * e;
    oracle_mlp_back_row(D, H, params, xr, buf, buf + H, buf + 2 * H, buf + 3 * H, 2.0 * e / R, bf16,
                        grad, NULL);
  }
  free(buf);
  return loss / R;
}

/* s(x_r) and ds/dx at every row. */
void oracle_mlp_input_grad(int D, int H, const double* params, const double* x, int R, int bf16,
                           double* s_out, double* dx) {
  double* buf = (double*)malloc(sizeof(double) * 4 * H);
  for (int r = 0; r < R; ++r) {
    const double* xr = x + (size_t)r * D;
    double sv = oracle_mlp_row(D, H, params, xr, bf16, buf, buf + H, buf + 2 * H, buf + 3 * H);
    if (s_out) s_out[r] = sv;
    oracle_mlp_back_row(D, H, params, xr, buf, buf + H, buf + 2 * H, buf + 3 * H, 1.0, bf16, NULL,
                        dx + (size_t)r * D);
  }
  free(buf);
}

/* Adam (Kingma and Ba, 2015): moments with bias correction at step t >= 1. */
void oracle_adam_step(int n, double* params, const double* grad, double* m, double* v, int t, double lr,
                      double beta1, double beta2, double eps) {
  const double c1 = 1.0 - pow(beta1, (double)t), c2 = 1.0 - pow(beta2, (double)t);
  for (int q = 0; q < n; ++q) {
    m[q] = beta1 * m[q] + (1.0 - beta1) * grad[q];
    v[q] = beta2 * v[q] + (1.0 - beta2) * grad[q] * grad[q];
    const double mh = m[q] / c1, vh = v[q] / c2;
    params[q] -= lr * mh / (sqrt(vh) + eps);
  }
}

/* ------------------------------------------------------------------ */
/* The learned proposal inside the sampler (not in the paper)           */
/* ------------------------------------------------------------------ */

/* The weights W1, W2 and w3 rounded to bfloat16 as the tensor-core kernels
 * use them; the biases b1, b2 and b3 unchanged. */
void oracle_mlp_weights_bf16(int D, int H, const double* params, double* out) {
  const int P = oracle_mlp_nparams(D, H);
  const int b1 = D * H, W2 = b1 + H, b2 = W2 + H * H, w3 = b2 + H, b3 = w3 + H;
  for (int q = 0; q < P; ++q) {
    const int weight = q < b1 || (q >= W2 && q < b2) || (q >= w3 && q < b3);
    out[q] = weight ? oracle_bf16(params[q]) : params[q];
  }
}

/* Training set of the surrogate (choice L2).  Rows r < R hold theta_r (R x D)
 * and the log target estimate lp_r = log p(theta_r) + log p^(y | theta_r).
 *   tau = max(2, D), ymax = the largest finite lp,
 *   z_r = max((lp_r - ymax) / tau, -8) (-8 for a non-finite lp_r),
 *   y_r = (z_r - mean z) / sd z over all R rows (population moments; when the
 *         variance of z is at most 1e-8 the sd is taken as 1 and var_y = 0,
 *         otherwise var_y = 1, the variance of the targets),
 *   x_r = (theta_r - mu) / sd, mu and sd the mean and population standard
 *         deviation of theta over the rows whose z lies above the clip -- or
 *         over every row with a finite lp when fewer than 2 D + 2 rows do;
 *         sd = 1 for fewer than two such rows, and at least 1e-6.  With no
 *         such row, mu = 0 and sd = 1.
 * Returns the number of rows the input moments were taken over. */
int oracle_mlp_standardise(int D, int R, const double* th, const double* lp, double* x, double* y,
                           oracle_mlp_norm* nm) {
  memset(nm, 0, sizeof(*nm));
  const double tau = D > 2 ? (double)D : 2.0;
  double ymax = -INFINITY;
  for (int r = 0; r < R; ++r)
    if (isfinite(lp[r]) && lp[r] > ymax) ymax = lp[r];
  double* z = (double*)malloc(sizeof(double) * (R > 0 ? R : 1));
  int above = 0;
  for (int r = 0; r < R; ++r) {
    if (isfinite(lp[r])) {
      const double v = (lp[r] - ymax) / tau;
      z[r] = v > -8.0 ? v : -8.0;
      if (v > -8.0) ++above;
    } else {
      z[r] = -8.0;
    }
  }
  /* input moments: the rows above the clip, else every row with a finite lp */
  const int use_all = above < 2 * D + 2;
  int cnt = 0;
  double mean[ORACLE_MAX_D] = {0.0}, var[ORACLE_MAX_D] = {0.0};
  for (int r = 0; r < R; ++r) {
    if (!isfinite(lp[r]) || (!use_all && !(z[r] > -8.0))) continue;
    ++cnt;
    for (int d = 0; d < D; ++d) mean[d] += th[(size_t)r * D + d];
  }
  for (int d = 0; d < D; ++d) mean[d] = cnt > 0 ? mean[d] / cnt : 0.0;
  for (int r = 0; r < R; ++r) {
    if (!isfinite(lp[r]) || (!use_all && !(z[r] > -8.0))) continue;
    for (int d = 0; d < D; ++d) {
      const double e = th[(size_t)r * D + d] - mean[d];
      var[d] += e * e;
    }
  }
  for (int d = 0; d < D; ++d) {
    double sd = cnt > 1 ? sqrt(var[d] / cnt) : 1.0;
    nm->mu[d] = mean[d];
    nm->sd[d] = sd > 1e-6 ? sd : 1e-6;
  }
  /* targets */
  double zm = 0.0, zv = 0.0;
  for (int r = 0; r < R; ++r) zm += z[r];
  zm = R > 0 ? zm / R : 0.0;
  for (int r = 0; r < R; ++r) zv += (z[r] - zm) * (z[r] - zm);
  zv = R > 0 ? zv / R : 0.0;
  nm->tau = tau;
  nm->ymax = ymax;
  nm->zmean = zm;
  nm->zsd = zv > 1e-8 ? sqrt(zv) : 1.0;
  nm->var_y = zv > 1e-8 ? 1.0 : 0.0;
  nm->rows = R;
  nm->rows_moments = cnt;
  for (int r = 0; r < R; ++r) {
    if (y) y[r] = (z[r] - zm) / nm->zsd;
    if (x)
      for (int d = 0; d < D; ++d) x[(size_t)r * D + d] = (th[(size_t)r * D + d] - nm->mu[d]) / nm->sd[d];
  }
  free(z);
  return cnt;
}

/* One training call of the surrogate (choices L1, L2): the training set of
 * oracle_mlp_standardise from the R rows (th, lp), then `steps` full-batch
 * Adam steps (beta = (0.9, 0.999), eps = 1e-8, learning rate lr) on the mean
 * squared error, continuing the step counter *t and the moments m, v.  With
 * bf16 != 0 every gradient is taken as the kernels take it: at the weights
 * rounded to bfloat16 (oracle_mlp_weights_bf16) with the bfloat16 rounding
 * points of oracle_mlp_loss_grad; the update applies to the unrounded
 * params.  nm, x, y (R x D and R values; either may be NULL) receive the
 * training set.  Returns the loss of the last step, before its update. */
double oracle_mlp_train(int D, int H, int R, const double* th, const double* lp, int steps, double lr,
                        int bf16, double* params, double* m, double* v, int* t, oracle_mlp_norm* nm,
                        double* x_out, double* y_out) {
  const int P = oracle_mlp_nparams(D, H);
  double* x = (double*)malloc(sizeof(double) * (size_t)(R > 0 ? R : 1) * D);
  double* y = (double*)malloc(sizeof(double) * (R > 0 ? R : 1));
  double* pw = (double*)malloc(sizeof(double) * P);
  double* g = (double*)malloc(sizeof(double) * P);
  oracle_mlp_norm local;
  oracle_mlp_standardise(D, R, th, lp, x, y, nm ? nm : &local);
  double loss = 0.0;
  for (int it = 0; it < steps; ++it) {
    if (bf16)
      oracle_mlp_weights_bf16(D, H, params, pw);
    else
      memcpy(pw, params, sizeof(double) * P);
    loss = R > 0 ? oracle_mlp_loss_grad(D, H, pw, x, y, R, bf16, g) : 0.0;
    if (R == 0)
      for (int q = 0; q < P; ++q) g[q] = 0.0;
    *t += 1;
    oracle_adam_step(P, params, g, m, v, *t, lr, 0.9, 0.999, 1e-8);
  }
  if (x_out) memcpy(x_out, x, sizeof(double) * (size_t)R * D);
  if (y_out) memcpy(y_out, y, sizeof(double) * R);
  free(x); free(y); free(pw); free(g);
  return loss;
}

/* Gradient of the surrogate's log target at theta (choice L3): with
 * x = (theta - mu) / sd, the fitted log target is ymax + tau (zmean + zsd s(x)),
 * so d log pi^ / d theta_d = tau zsd (ds/dx)_d / sd_d.  R rows of theta
 * (R x D) into score (R x D).  bf16 as in oracle_mlp_train. */
void oracle_mlp_score(int D, int H, const double* params, const oracle_mlp_norm* nm, const double* theta,
                      int R, int bf16, double* score) {
  const int P = oracle_mlp_nparams(D, H);
  double* pw = (double*)malloc(sizeof(double) * P);
  double* x = (double*)malloc(sizeof(double) * (size_t)(R > 0 ? R : 1) * D);
  if (bf16)
    oracle_mlp_weights_bf16(D, H, params, pw);
  else
    memcpy(pw, params, sizeof(double) * P);
  for (int r = 0; r < R; ++r)
    for (int d = 0; d < D; ++d) x[(size_t)r * D + d] = (theta[(size_t)r * D + d] - nm->mu[d]) / nm->sd[d];
  oracle_mlp_input_grad(D, H, pw, x, R, bf16, NULL, score);
  for (int r = 0; r < R; ++r)
    for (int d = 0; d < D; ++d) score[(size_t)r * D + d] *= nm->tau * nm->zsd / nm->sd[d];
  free(pw); free(x);
}

/* Lower Cholesky factor L of the population covariance (row-major D x D)
 * that the learned proposal scales its steps by (choice L4).  Returns 1 when
 * it is usable -- the population's ESS is at least 2 (D + 1) and every pivot
 * exceeds 1e-12 of its diagonal entry -- and 0 otherwise. */
int oracle_population_factor(int D, const double* cov, double ess, double* L) {
  const double zero[ORACLE_MAX_D] = {0.0};
  const int chol_ok = oracle_cholesky(D, cov, zero, L) == 0;
  return chol_ok && ess >= 2.0 * (D + 1);
}

/* Whether iteration k proposes with the network (choice L4): from k = 3 on,
 * while the published network's training loss is finite and below half the
 * variance of its targets, and the previous population's factor is usable;
 * otherwise the random walk of Eq. (19). */
int oracle_learned_decision(int k, double loss, double var_y, int pop_ok) {
  return k >= 3 && isfinite(loss) && var_y > 0.0 && loss < 0.5 * var_y && pop_ok;
}

/* The learned proposal (choice L3): a Langevin step preconditioned by the
 * population covariance Sigma = L L^T with the surrogate's score g:
 *   w = clip(h/2 L^T g, -3, 3) coordinatewise (the drift in whitened units),
 *   theta_k = theta_{k-1} + h L (w + z),  z ~ N(0, I),
 * so theta_k ~ N(theta_{k-1} + h L w, h^2 L L^T); *logq receives that
 * Gaussian density at theta_k, evaluated from its definition. */
void oracle_langevin_propose(int D, double h, const double* L, const double* theta_prev, const double* g,
                             const double* z, double* theta_out, double* logq) {
  double w[ORACLE_MAX_D], mean[ORACLE_MAX_D], u[ORACLE_MAX_D];
  for (int r = 0; r < D; ++r) { /* (L^T g)_r = sum_d L_dr g_d */
    double s = 0.0;
    for (int d = 0; d < D; ++d) s += L[d * D + r] * g[d];
    s *= 0.5 * h;
    w[r] = s < -3.0 ? -3.0 : (s > 3.0 ? 3.0 : s);
  }
  for (int d = 0; d < D; ++d) {
    double lw = 0.0, lz = 0.0;
    for (int c = 0; c <= d; ++c) {
      lw += L[d * D + c] * w[c];
      lz += L[d * D + c] * (w[c] + z[c]);
    }
    mean[d] = theta_prev[d] + h * lw;
    theta_out[d] = theta_prev[d] + h * lz;
  }
  /* log N(theta_k; mean, h^2 L L^T): solve L u = (theta_k - mean) / h */
  double logdet = 0.0, ss = 0.0;
  for (int d = 0; d < D; ++d) {
    double r = (theta_out[d] - mean[d]) / h;
    for (int c = 0; c < d; ++c) r -= L[d * D + c] * u[c];
    u[d] = r / L[d * D + d];
    ss += u[d] * u[d];
    logdet += log(h * L[d * D + d]);
  }
  *logq = -0.5 * D * LOG_2PI - logdet - 0.5 * ss;
}
