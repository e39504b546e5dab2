// pf_impl.cuh -- bootstrap particle filter kernel (Sec. II of the paper).
//
// One group of threads runs one filter over all T steps: each thread holds
// PPT consecutive particles in registers.  Per step:
//   1. propagate with the state equation (Eq. 1) using counter-based normals;
//   2. log-weight with the observation density (Eq. 2; bootstrap form of Eq. 5);
//   3. group max of the log-weights (warp shuffles, one barrier);
//   4. quantise q_j = floor(exp(l_j - max) 2^B), warp-local inclusive scan of q
//      in registers + shuffles, warp totals to shared memory (second barrier);
//   5. log-likelihood increment log((1/M) sum_j w_j) = max + log(S 2^-B) - log M
//      from the exact integer total S (Eq. 8, with the mean-weight reset of
//      Eq. 13 every step);
//   6. systematic resampling (Eqs. 26-27): slot j takes the first particle whose
//      cumulative weight exceeds tau_j = floor((j + u) S / M).  Equivalently
//      particle i fills the slots F(C_{i-1}) .. F(C_i) - 1, F(C) being the
//      number of thresholds below C; each thread computes F at its particles'
//      cumulative weights (a float estimate, settled by an exact 128-bit
//      comparison near integers).  A warp's particles fill one contiguous run
//      of slots, which the warp copies 32 slots at a time (each lane finds its
//      slot's particle by a shuffle search over the lanes' ranges), and after
//      a third barrier every thread reads the states of its own slots.
//      (Staged variants keep the prefix in shared memory and search it instead.)
// A work unit is `count` filters of one job (dataset); units are taken from an
// atomic queue so that jobs of uneven length balance over the SMs.
// With 8 or more particles per thread ("staged"), the log-weights and the
// thread-local prefixes pass through shared memory instead of registers, which
// lets a 512-particle filter run in a single warp: the group reductions become
// warp shuffles and the per-thread costs are shared by 16 particles.
#pragma once
#include <cfloat>
#include <cmath>
#include <type_traits>

#include "binomial.cuh"
#include "common.cuh"
#include "internal.h"

namespace smc2 {

template <typename R>
struct R4Of;
template <>
struct R4Of<float> {
  using type = float4;
};
struct __align__(32) Double4 {
  double x, y, z, w;
};
template <>
struct R4Of<double> {
  using type = Double4;
};

template <int MODEL>
struct ModelDims;
template <>
struct ModelDims<MODEL_LG> {
  static constexpr int D = 3, NS = 1;
};
template <>
struct ModelDims<MODEL_SEIR> {
  static constexpr int D = 4, NS = 4;
};
template <>
struct ModelDims<MODEL_SIR> {
  static constexpr int D = 2, NS = 2;
};

__host__ __device__ inline int group_threads_for(int ppt, int M) {
  const int t = (M + ppt - 1) / ppt;
  return (t + 31) & ~31;
}

// Shared memory of one filter group (Mp = particles incl. padding, nw warps):
//   P  u64 [Mp]      inclusive prefix of the quantised weights (staged: warp-local; variants:
//                    global, for multinomial slots; absent otherwise)
//   X  R   [Mp][ns]  particle states, one vector per particle (per slot after resampling)
//   Xo R   [Mp][ns]  states before resampling, by particle (register-resident variants)
//   Z  R   [4][Mp]   the four normals of the current Philox counter of every particle
//   L  R   [Mp]      log-weights (staged path only)
//   wsum u64 [nw], wmax 8 B [nw], wq2 u128 [nw] (variants: sums of q^2 for the ESS),
//   sU u32 [8] (resampling words of two groups of four steps)
__host__ __device__ constexpr bool is_staged(int ppt) { return ppt >= 8; }
__host__ __device__ inline size_t region_bytes(int Mp, int nw, int ns, int rsize, bool staged,
                                               bool general) {
  size_t b = (size_t)(staged ? 1 : 2) * ns * Mp * rsize + (size_t)4 * Mp * rsize + (size_t)nw * 16 + 32;
  if (staged || general) b += (size_t)Mp * 8;
  if (general) b += (size_t)nw * 16;
  if (staged) b += (size_t)Mp * rsize;
  return (b + 15) & ~(size_t)15;
}

// Register budget per variant (threads x registers must fit the SM at the
// shapes the tuner tries); beyond it the compiler spills to local memory.
template <typename R, int PPT>
struct RegCap {
  static constexpr int value =
      sizeof(R) == 4 ? (PPT <= 2 ? 64 : (PPT == 4 ? 96 : (PPT == 8 ? 128 : 168)))
                     : (PPT == 1 ? 80 : (PPT == 2 ? 96 : (PPT <= 8 ? 128 : 168)));
  static_assert(PPT == 1 || PPT == 2 || PPT == 4 || PPT == 8 || PPT == 16, "particles per thread");
};

template <typename R, int NS>
struct StateVec;
template <typename R>
struct StateVec<R, 1> {
  __device__ __forceinline__ static void store(R* X, int j, const R* x) { X[j] = x[0]; }
  __device__ __forceinline__ static void load(const R* X, int j, R* x) { x[0] = X[j]; }
};
template <>
struct StateVec<float, 2> {
  __device__ __forceinline__ static void store(float* X, int j, const float* x) {
    reinterpret_cast<float2*>(X)[j] = make_float2(x[0], x[1]);
  }
  __device__ __forceinline__ static void load(const float* X, int j, float* x) {
    const float2 v = reinterpret_cast<const float2*>(X)[j];
    x[0] = v.x;
    x[1] = v.y;
  }
};
template <>
struct StateVec<double, 2> {
  __device__ __forceinline__ static void store(double* X, int j, const double* x) {
    reinterpret_cast<double2*>(X)[j] = make_double2(x[0], x[1]);
  }
  __device__ __forceinline__ static void load(const double* X, int j, double* x) {
    const double2 v = reinterpret_cast<const double2*>(X)[j];
    x[0] = v.x;
    x[1] = v.y;
  }
};
template <>
struct StateVec<float, 4> {
  __device__ __forceinline__ static void store(float* X, int j, const float* x) {
    reinterpret_cast<float4*>(X)[j] = make_float4(x[0], x[1], x[2], x[3]);
  }
  __device__ __forceinline__ static void load(const float* X, int j, float* x) {
    const float4 v = reinterpret_cast<const float4*>(X)[j];
    x[0] = v.x;
    x[1] = v.y;
    x[2] = v.z;
    x[3] = v.w;
  }
};
template <>
struct StateVec<double, 4> {
  __device__ __forceinline__ static void store(double* X, int j, const double* x) {
    reinterpret_cast<double2*>(X)[2 * j] = make_double2(x[0], x[1]);
    reinterpret_cast<double2*>(X)[2 * j + 1] = make_double2(x[2], x[3]);
  }
  __device__ __forceinline__ static void load(const double* X, int j, double* x) {
    const double2 a = reinterpret_cast<const double2*>(X)[2 * j];
    const double2 b = reinterpret_cast<const double2*>(X)[2 * j + 1];
    x[0] = a.x;
    x[1] = a.y;
    x[2] = b.x;
    x[3] = b.y;
  }
};

template <typename R>
__device__ __forceinline__ R neg_inf();
template <>
__device__ __forceinline__ float neg_inf<float>() {
  return -INFINITY;
}
template <>
__device__ __forceinline__ double neg_inf<double>() {
  return -HUGE_VAL;
}

__device__ __forceinline__ uint64_t to_u64_rz(float v) { return __float2ull_rz(v); }
__device__ __forceinline__ uint64_t to_u64_rz(double v) { return __double2ull_rz(v); }

// u64 to float from its two 32-bit halves (relative error below 2^-23).
__device__ __forceinline__ float u64_to_float(uint64_t v) {
  return fmaf(__uint2float_rn((uint32_t)(v >> 32)), 0x1p32f, __uint2float_rn((uint32_t)v));
}

// Counting slot thresholds of systematic resampling (Eqs. 26-27) below a
// cumulative weight C: tau_j = floor((2^33 j + 2U + 1) S / (M 2^33)) < C holds
// exactly when (2^33 j + 2U + 1) S < C M 2^33 (both sides below 2^110).
struct SlotCount {
  uint64_t S, M33, U21;  // total, M 2^33, 2U + 1
  float scale, off;      // M / S and (2U + 1) 2^-33 for the float estimate
  float margin;          // bound on the error of the estimate
  int M;
};
__device__ __forceinline__ SlotCount slot_count_setup(uint32_t U, uint64_t S, int M) {
  SlotCount sc;
  sc.S = S;
  sc.M33 = (uint64_t)M << 33;
  sc.U21 = 2ull * U + 1ull;
  sc.scale = __fdividef((float)M, u64_to_float(S));
  sc.off = fmaf(2.f, (float)U, 1.f) * 0x1p-33f;
  sc.margin = fmaf((float)M, 0x1p-18f, 0x1p-16f);
  sc.M = M;
  return sc;
}
// F(C) = #{j in [0, M): tau_j < C} = ceil(C M / S - (2U+1) 2^-33) clamped to
// [0, M].  The crossing point is estimated in float: Cf approximates C to
// about 2^-22 relative, so the estimate is within M 2^-19 of it, inside
// `margin`.  Away from an integer the estimate's ceiling is F; within the
// margin of an integer n (clamped to [0, M - 1]), F is n or n + 1 and one exact
// comparison, tau_n < C, says which.
// Away from integers the estimate lies in (-1, M) (0 <= C <= S), so its ceiling is
// already in [0, M]; only the exact branch clamps.
__device__ __forceinline__ int slots_below(const SlotCount& sc, uint64_t C, float Cf) {
  const float est = fmaf(Cf, sc.scale, -sc.off);
  const float nf = rintf(est);
  if (fabsf(est - nf) > sc.margin) return (int)nf + (est > nf ? 1 : 0);
  int n = min(max((int)nf, 0), sc.M - 1);
  const uint64_t a = ((uint64_t)n << 33) + sc.U21;
  const uint64_t lh = __umul64hi(a, sc.S), ll = a * sc.S;
  const uint64_t rh = __umul64hi(C, sc.M33), rl = C * sc.M33;
  n += (lh < rh || (lh == rh && ll < rl)) ? 1 : 0;
  return n;
}

// exp in the working precision: the FP32 path uses the hardware exp2
// approximation (relative error about 2^-22), the FP64 path the full-precision exp.
__device__ __forceinline__ float fast_exp(float x) { return __expf(x); }
__device__ __forceinline__ double fast_exp(double x) { return exp(x); }

// Per-filter constants of the model in the working precision.
template <typename R, int MODEL>
struct FilterParams;

template <typename R>
struct FilterParams<R, MODEL_LG> {
  R phi, sx, inv_sy, c_obs;
  __device__ void load(const double* th, const PFModel&) {
    const double sy = exp(th[2]);
    phi = (R)th[0];
    sx = (R)exp(th[1]);
    inv_sy = (R)(1.0 / sy);
    c_obs = (R)(-0.5 * kLog2Pi - th[2]);
  }
  __device__ __forceinline__ void init(R* x, R z0, const double*) const { x[0] = z0; }
  __device__ __forceinline__ void propagate(R* x, R z) const { x[0] = phi * x[0] + sx * z; }
  template <typename R4>
  __device__ __forceinline__ R log_obs(const R* x, const R4& ob) const {
    const R r = (ob.x - x[0]) * inv_sy;
    return c_obs - (R)0.5 * r * r;
  }
};

template <typename R>
struct FilterParams<R, MODEL_SEIR> {
  R srw, kappa, gamma, inv_npop, dt, lam_floor, S0, E0, I0, lb0;
  int n_sub;
  __device__ void load(const double* th, const PFModel& m) {
    lb0 = (R)th[0];
    srw = (R)exp(th[1]);
    kappa = (R)exp(th[2]);
    gamma = (R)exp(th[3]);
    inv_npop = (R)(1.0 / m.npop);
    dt = (R)(1.0 / m.n_sub);
    n_sub = m.n_sub;
    lam_floor = (R)m.lambda_floor;
    S0 = (R)(m.npop - m.e0 - m.i0);
    E0 = (R)m.e0;
    I0 = (R)m.i0;
  }
  __device__ __forceinline__ void init(R* x, R, const double*) const {
    x[0] = S0;
    x[1] = E0;
    x[2] = I0;
    x[3] = lb0;
  }
  // x = (S, E, I, log beta); the day's incidence lambda is returned in x[4]'s place
  __device__ __forceinline__ void propagate(R* x, R z) const {
    x[3] = x[3] + srw * z;
  }
  __device__ __forceinline__ void substep(R beta, R& S, R& E, R& I, R& lam) const {
    const R infection = beta * S * I * inv_npop;
    const R onset = kappa * E;
    const R recovery = gamma * I;
    lam += dt * onset;
    S = fmax(S - dt * infection, (R)0);
    E = fmax(E + dt * (infection - onset), (R)0);
    I = fmax(I + dt * (onset - recovery), (R)0);
  }
  __device__ __forceinline__ R day(R* x) const {
    const R beta = fast_exp(x[3]);
    R S = x[0], E = x[1], I = x[2], lam = (R)0;
    if (n_sub == 2) {  // the common case, unrolled
      substep(beta, S, E, I, lam);
      substep(beta, S, E, I, lam);
    } else {
      for (int s = 0; s < n_sub; ++s) substep(beta, S, E, I, lam);
    }
    x[0] = S;
    x[1] = E;
    x[2] = I;
    return fmax(lam, lam_floor);
  }
  // Poisson log-pmf written as y (log1p(d) - d) + c_y with d = (lambda - y) / y and
  // c_y = y log y - y - log y! precomputed: no cancellation between y log lambda and lambda.
  template <typename R4>
  __device__ __forceinline__ R log_pois(R lam, const R4& ob) const {
    if (ob.x > (R)0) {
      const R d = (lam - ob.x) * ob.y;
      return ob.x * (log1p(d) - d) + ob.z;
    }
    return -lam;
  }
};

// Binomial SIR model (Sec. V-A): theta = (beta, gamma), state (S, I) integers
// held in the working precision (exact below 2^24).  Each day, from the previous
// day's compartments, n(S->I) ~ Bin(S, 1 - exp(-beta I / Npop)) and
// n(I->R) ~ Bin(I, 1 - exp(-gamma)); y_t ~ Poisson(I_t).  (The printed S->I
// probability also carries S_{t-1} in the exponent; this is the per-susceptible
// hazard of the chain-binomial model the section cites.)  Both flows are drawn
// by the binomial sampler of the working precision from particle j's one word
// stream of step t, the I->R draw reading from where the S->I draw stopped.
template <typename R>
struct FilterParams<R, MODEL_SIR> {
  R beta, npop, S0, I0, p_ir;
  __device__ void load(const double* th, const PFModel& m) {
    beta = (R)th[0];
    npop = (R)m.npop;
    p_ir = (R)(-expm1(-th[1]));
    S0 = (R)(m.npop - m.i0);
    I0 = (R)m.i0;
  }
  __device__ __forceinline__ void init(R* x, R, const double*) const {
    x[0] = S0;
    x[1] = I0;
  }
  __device__ __forceinline__ void day(R* x, uint32_t j, uint32_t t, uint32_t c2, uint32_t c3,
                                      uint2 key) const {
    const R S = x[0], I = x[1];
    const R h = beta * I / npop;
    const R p_si = -expm1(-h);
    typename std::conditional<sizeof(R) == 8, BinomWords, BinomWordsF>::type b(make_uint4(j, t, c2, c3), key);
    const R n_si = binomial_draw(S, p_si, b);
    const R n_ir = binomial_draw(I, p_ir, b);
    x[0] = S - n_si;
    x[1] = (I + n_si) - n_ir;  // integers: exact in either precision
  }
  // Poisson(y; I) as for the SEIR-type model, with a point mass at 0 when I = 0
  template <typename R4>
  __device__ __forceinline__ R log_obs(const R* x, const R4& ob) const {
    const R I = x[1];
    if (!(I > (R)0)) return ob.x > (R)0 ? neg_inf<R>() : (R)0;
    if (ob.x > (R)0) {
      const R d = (I - ob.x) * ob.y;
      return ob.x * (log1p(d) - d) + ob.z;
    }
    return -I;
  }
};

// NAMED: groups wider than a warp that share a CTA synchronise on named
// barriers 1..15 (ptxas then reserves all 16 barriers of the CTA, which limits
// residency to four CTAs per SM).  Otherwise a wide group is the whole CTA and
// uses __syncthreads, and a one-warp group uses __syncwarp.
template <typename R, int MODEL, int PPT, bool NAMED, bool GENERAL>
__device__ __forceinline__ void run_filter(const PFJob& J, const PFModel& mdl, int i, int g, int lt,
                                           int gt, unsigned char* region, uint2 key, uint32_t k,
                                           int t_cap) {
  constexpr int NS = ModelDims<MODEL>::NS;
  constexpr int D = ModelDims<MODEL>::D;
  using R4 = typename R4Of<R>::type;
  const int M = J.M, T = t_cap > 0 ? min(J.T, t_cap) : J.T;
  const int Mp = gt * PPT;
  const int nw = gt >> 5;
  const int lane = lt & 31, warp = lt >> 5;
  const int seg = 32 * PPT;  // particles per warp

  constexpr bool STAGED = is_staged(PPT);
  constexpr bool GEN = GENERAL && !STAGED;
  uint64_t* P = reinterpret_cast<uint64_t*>(region);   // [Mp] inclusive prefix of q (staged, variants)
  R* X = reinterpret_cast<R*>(P + (STAGED || GEN ? Mp : 0));  // [Mp][NS] particle states
  R* Xo = X + (size_t)NS * Mp;                          // [Mp][NS] states by particle (not staged)
  R* Z = X + (size_t)NS * Mp * (STAGED ? 1 : 2);       // [4][Mp] cached normals
  uint64_t* wsum = reinterpret_cast<uint64_t*>(Z + (size_t)4 * Mp);  // [nw] warp totals
  R* wmax = reinterpret_cast<R*>(wsum + nw);            // [nw] warp maxima (8-byte slots)
  unsigned __int128* wq2 = reinterpret_cast<unsigned __int128*>(wsum + 2 * nw);  // [nw] sums of q^2 (variants)
  uint32_t* sU = reinterpret_cast<uint32_t*>(wsum + (GEN ? 4 : 2) * nw);  // [8] resampling words
  R* Lw = reinterpret_cast<R*>(reinterpret_cast<unsigned char*>(sU) + 32);  // [Mp] staged log-weights

  auto group_sync = [&]() {
    if (nw == 1)
      __syncwarp();
    else if constexpr (NAMED)
      named_barrier(1 + g, gt);
    else
      __syncthreads();
  };

  double th[D];
#pragma unroll
  for (int d = 0; d < D; ++d) th[d] = J.theta[(size_t)d * J.ld + i];
  FilterParams<R, MODEL> fp;
  fp.load(th, mdl);

  const uint32_t c2 = counter_c2((uint32_t)i, J.c2hi);
  const uint32_t c3prop = counter_c3(TAG_PF_PROP, k);
  const uint32_t c3res = counter_c3(TAG_PF_RES, k);
  const uint32_t c3multi = counter_c3(TAG_PF_MULTI, k);
  const uint32_t c3binom = counter_c3(TAG_PF_BINOM, k);
  const int B = fixed_point_bits(M);
  const int log2M = ((M & (M - 1)) == 0) ? (__ffs(M) - 1) : -1;
  const R scaleB = (R)ldexp(1.0, B);
  const double log_norm = -(double)B * kLn2 - log((double)M);
  const R4* obs = reinterpret_cast<const R4*>(J.obs);

  R x[PPT][NS];
#pragma unroll
  for (int r = 0; r < PPT; ++r) {
    R z0 = (R)0;
    if constexpr (MODEL == MODEL_LG) {
      R z[4];
      normals4<R>(make_uint4((uint32_t)(lt * PPT + r), 0u, c2, counter_c3(TAG_PF_INIT, k)), key, z);
      z0 = z[0];
    }
    fp.init(x[r], z0, th);
  }

  // Weights (Eq. 5): exp(Lc + lwc_j), Lc the common log weight set by the last
  // resampling (Eq. 13), lwc_j the particle's log factor since (register-resident
  // variants; with resampling every step lwc stays zero).
  // (GENERAL instantiations only: the ESS schedule and multinomial slots; the default
  // instantiations resample systematically every step and keep no factors)
  const bool adaptive = GEN && mdl.pf_ess_frac > 0.0;
  const float ess_thr = (float)(mdl.pf_ess_frac * (double)M);  // mixed precision's ESS threshold
  const bool multinomial = GEN && mdl.pf_scheme == 1;
  R lwc[GEN ? PPT : 1];
#pragma unroll
  for (int r = 0; r < (GEN ? PPT : 1); ++r) lwc[r] = (R)0;
  double Lc = 0.0;
  double loglik = 0.0;  // log p^(y_{1:t}) (Eq. 8)
  for (int t = 1; t <= T; ++t) {
    const int tm = (t - 1) & 3;
    if (MODEL != MODEL_SIR && tm == 0) {  // one Philox call per particle every four steps; normals kept in shared memory
#pragma unroll
      for (int r = 0; r < PPT; ++r) {
        R z4[4];
        normals4<R>(make_uint4((uint32_t)(lt * PPT + r), (uint32_t)((t - 1) >> 2), c2, c3prop), key,
                    z4);
#pragma unroll
        for (int e = 0; e < 4; ++e) Z[e * Mp + lt * PPT + r] = z4[e];
      }
    }
    // resampling words of steps t..t+3, one lane each, double-buffered by step group
    uint32_t* sUg = sU + 4 * (((t - 1) >> 2) & 1);
    if (tm == 0 && lt < 4 && t + lt < T)
      sUg[lt] = philox4x32_10(make_uint4(0u, (uint32_t)(t + lt), c2, c3res), key).x;
    const R4 ob = obs[t - 1];
    R ell[STAGED ? 1 : PPT];
    R lmax = neg_inf<R>();
#pragma unroll
    for (int r = 0; r < PPT; ++r) {
      R l;
      if constexpr (MODEL == MODEL_SIR) {
        fp.day(x[r], (uint32_t)(lt * PPT + r), (uint32_t)t, c2, c3binom, key);
        l = fp.log_obs(x[r], ob);
      } else if constexpr (MODEL == MODEL_LG) {
        fp.propagate(x[r], Z[tm * Mp + lt * PPT + r]);
        l = fp.log_obs(x[r], ob);
      } else {
        fp.propagate(x[r], Z[tm * Mp + lt * PPT + r]);
        const R lam = fp.day(x[r]);
        l = fp.log_pois(lam, ob);
      }
      if (isnan(l) || lt * PPT + r >= M) l = neg_inf<R>();
      if constexpr (STAGED) {
        Lw[lt * PPT + r] = l;
      } else {
        if constexpr (GEN) l = lwc[GEN ? r : 0] + l;  // Eq. (5) in logs: the factor since the last resampling
        ell[r] = l;
        StateVec<R, NS>::store(Xo, lt * PPT + r, x[r]);
      }
      lmax = fmax(lmax, l);
    }
    // (3) group maximum
    lmax = warp_max(lmax);
    if (nw > 1 && lane == 0) wmax[warp] = lmax;
    group_sync();
    if (nw > 1) lmax = warp_max(lane < nw ? wmax[lane] : neg_inf<R>());
    const R m = lmax;
    if (!(m > neg_inf<R>())) {  // every weight vanished: the estimate is zero
      loglik = -HUGE_VAL;
      if (lt == 0 && J.delta)
        for (int s = t; s <= T; ++s) J.delta[(size_t)i * T + (s - 1)] = -HUGE_VAL;
      break;
    }
    // (4) quantise and scan (warp-local inclusive prefix in P, warp totals in wsum)
    uint64_t run = 0;
    if constexpr (STAGED) {
      // thread-local inclusive prefix into P, then the thread's offset added in place
#pragma unroll
      for (int r = 0; r < PPT; ++r) {
        const R l = Lw[lt * PPT + r];
        run += (l > neg_inf<R>()) ? to_u64_rz(fast_exp(l - m) * scaleB) : 0ull;
        P[lt * PPT + r] = run;
        StateVec<R, NS>::store(X, lt * PPT + r, x[r]);
      }
    }
    uint64_t c[STAGED ? 1 : PPT];  // thread-local inclusive prefix of q
    float cf[STAGED ? 1 : PPT];     // the same from the unfloored values, in float
    if constexpr (!STAGED) {
      float runf = 0.f;
#pragma unroll
      for (int r = 0; r < PPT; ++r) {
        const R v = (ell[r] > neg_inf<R>()) ? fast_exp(ell[r] - m) * scaleB : (R)0;
        run += to_u64_rz(v);
        runf += (float)v;
        c[r] = run;
        cf[r] = runf;
      }
    }
    const uint64_t incl = warp_incl_scan_u64(run, lane);
    const uint64_t excl = incl - run;
    if constexpr (STAGED) {
#pragma unroll
      for (int r = 0; r < PPT; ++r) P[lt * PPT + r] += excl;
    }
    if (lane == 31) wsum[warp] = incl;
    if (adaptive) {  // the warp's sum of q^2, exact in 128 bits
      unsigned __int128 q2 = 0;
      if constexpr (!STAGED) {
        uint64_t prev = 0;
#pragma unroll
        for (int r = 0; r < PPT; ++r) {
          const uint64_t qv = c[r] - prev;
          prev = c[r];
          q2 += (unsigned __int128)qv * qv;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const uint64_t lo = __shfl_xor_sync(0xffffffffu, (uint64_t)q2, o);
        const uint64_t hi = __shfl_xor_sync(0xffffffffu, (uint64_t)(q2 >> 64), o);
        q2 += ((unsigned __int128)hi << 64) | lo;
      }
      if (lane == 0) wq2[warp] = q2;
    }
    group_sync();
    // total S, and the weight `base` of the warps before this one: an inclusive
    // scan of the warp totals across the lanes
    uint64_t wpre = lane < nw ? wsum[lane] : 0ull;
    for (int o = 1; o < nw; o <<= 1) {
      const uint64_t n = __shfl_up_sync(0xffffffffu, wpre, o);
      if (lane >= o) wpre += n;
    }
    const uint64_t S = __shfl_sync(0xffffffffu, wpre, nw - 1);
    const uint64_t base_incl = __shfl_sync(0xffffffffu, wpre, warp > 0 ? warp - 1 : 0);
    const uint64_t base = warp > 0 ? base_incl : 0ull;
    // (5) log-likelihood increment: log S from its binary exponent and mantissa
    // log p^(y_{1:t}) = Lc + log((1/M) sum_j exp(lwc_j + l_j)) from the exact integer total
    // (thread 0 of the group carries Lc and the estimate)
    if (lt == 0) {
      const int e = 63 - __clzll((long long)S);
      const R mant = (R)(e >= 52 ? (S >> (e - 52)) : (S << (52 - e))) * (R)0x1p-52;
      const double lmean = (double)m + ((double)e * kLn2 + (double)log(mant)) + log_norm;
      double delta = lmean;
      if constexpr (GEN) {
        const double logp_prev = loglik;
        loglik = Lc + lmean;
        delta = loglik - logp_prev;
      } else {
        loglik += lmean;
      }
      if (J.delta) J.delta[(size_t)i * T + (t - 1)] = delta;
    }
    // the schedule: every step, or when the ESS of the integer weights (Eq. 12) is below
    // pf_ess_frac M, formed with the same correctly rounded operations as the oracle (by
    // lane 0 of every warp, from the same totals, so the whole group decides alike)
    bool resample = t < T;
    if (adaptive && resample) {
      int below = 0;
      if (lane == 0) {
        unsigned __int128 Q2 = 0;
        for (int w = 0; w < nw; ++w) Q2 += wq2[w];
        if constexpr (sizeof(R) == 8) {  // the oracle's operations, bit for bit
          const double q2 = (double)(uint64_t)(Q2 >> 64) * 0x1p64 + (double)(uint64_t)Q2;
          const double ess = __ddiv_rn((double)S * (double)S, q2);
          below = ess < mdl.pf_ess_frac * (double)M;
        } else {  // mixed precision: the same test in float, S^2 < threshold sum q^2
          const float q2 = fmaf(__ull2float_rn((uint64_t)(Q2 >> 64)), 0x1p64f, __ull2float_rn((uint64_t)Q2));
          const float Sf = u64_to_float(S);
          below = Sf * Sf < ess_thr * q2;
        }
      }
      resample = __shfl_sync(0xffffffffu, below, 0) != 0;
    }
    if constexpr (GEN) {
      if (resample) Lc = loglik;  // Eq. (13): every particle will carry the mean weight (thread 0)
      if (t < T && !resample) {  // every particle keeps its state and its factor
#pragma unroll
        for (int r = 0; r < (GEN ? PPT : 1); ++r) {
          lwc[r] = ell[STAGED ? 0 : r];
          const int j = lt * PPT + r;
          if (J.anc && j < M) J.anc[((size_t)i * (T - 1) + (t - 1)) * M + j] = j;
        }
        continue;
      }
#pragma unroll
      for (int r = 0; r < (GEN ? PPT : 1); ++r) lwc[r] = (R)0;
    }
    if (GEN && resample && multinomial) {
      // slot j draws u_j = (2 U_j + 1) / 2^33 (word j & 3 of call j >> 2) and takes the
      // first particle with C_i > floor(u_j S)
#pragma unroll
      for (int r = 0; r < PPT; ++r) P[lt * PPT + r] = base + excl + c[r];
      group_sync();
      uint4 wj = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
      for (int r = 0; r < PPT; ++r) {
        const int j = lt * PPT + r;
        if (r == 0 || (j & 3) == 0)  // a thread's consecutive slots share their calls
          wj = philox4x32_10(make_uint4((uint32_t)j >> 2, (uint32_t)t, c2, c3multi), key);
        if (j >= M) continue;
        const uint32_t Uj = (j & 2) ? ((j & 1) ? wj.w : wj.z) : ((j & 1) ? wj.y : wj.x);
        const uint64_t tau = (uint64_t)(((unsigned __int128)(2ull * Uj + 1ull) * S) >> 33);
        int lo = 0, hi = M - 1;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (P[mid] > tau)
            hi = mid;
          else
            lo = mid + 1;
        }
        StateVec<R, NS>::load(Xo, lo, x[r]);
        if (J.anc) J.anc[((size_t)i * (T - 1) + (t - 1)) * M + j] = lo;
      }
      group_sync();  // P and Xo free for the next step
      continue;
    }
    // (6) systematic resampling and ancestor gather.  The thread's slots are
    // consecutive and their ancestors non-decreasing: the first is found by a
    // search over the warp totals and a binary search inside one warp's prefix,
    // the others by galloping forward from the previous ancestor.
    if (!STAGED && t < T) {
      const SlotCount sc = slot_count_setup(sUg[tm], S, M);
      const uint64_t C0 = base + excl;  // cumulative weight before the thread's first particle
      const float C0f = u64_to_float(C0);
      int ends[PPT];
#pragma unroll
      for (int r = 0; r < PPT; ++r) ends[r] = slots_below(sc, C0 + c[r], C0f + cf[r]);
      // the warp's particles fill the slots [first, last), in particle order
      const int first = __shfl_sync(0xffffffffu, slots_below(sc, C0, C0f), 0);
      const int last = __shfl_sync(0xffffffffu, ends[PPT - 1], 31);
      const int pbase = warp * 32 * PPT;  // the warp's first particle
      __syncwarp();                       // the warp's states in Xo
      for (int j0 = first; j0 < last; j0 += 32) {
        const int j = j0 + lane;
        // the lane whose particles cover slot j: the lanes whose ranges end at or before j
        int src = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
          const int e = __shfl_sync(0xffffffffu, ends[PPT - 1], src + step - 1);
          if (e <= j) src += step;
        }
        src = min(src, 31);
        int rr = 0;
#pragma unroll
        for (int r = 0; r < PPT - 1; ++r) rr += __shfl_sync(0xffffffffu, ends[r], src) <= j ? 1 : 0;
        if (j < last) {
          const int a = pbase + src * PPT + rr;
          R v[NS];
          StateVec<R, NS>::load(Xo, a, v);
          StateVec<R, NS>::store(X, j, v);
          if (J.anc) J.anc[((size_t)i * (T - 1) + (t - 1)) * M + j] = a;
        }
      }
      group_sync();
#pragma unroll
      for (int r = 0; r < PPT; ++r)
        if (lt * PPT + r < M) StateVec<R, NS>::load(X, lt * PPT + r, x[r]);
    }
    if (STAGED && t < T) {
      const uint32_t U = sUg[tm];
      int w = 0, a = 0;
      uint64_t base = 0;
#pragma unroll
      for (int r = 0; r < PPT; ++r) {
        const int j = lt * PPT + r;
        if (j < M) {
          const uint64_t tau = slot_threshold((uint32_t)j, U, S, M, log2M);
          while (w < nw - 1 && base + wsum[w] <= tau) {  // answer lies in a later warp
            base += wsum[w];
            ++w;
            a = w * seg;
          }
          const uint64_t tl = tau - base;
          const int seg_end = w * seg + seg - 1;  // P[seg_end] = wsum[w] > tl
          if (r == 0) {
            int lo = w * seg, hi = seg_end;
            while (lo < hi) {
              const int mid = (lo + hi) >> 1;
              if (P[mid] > tl)
                hi = mid;
              else
                lo = mid + 1;
            }
            a = lo;
          } else if (P[a] <= tl) {
            int lo = a + 1, step = 1;
            while (lo + step - 1 < seg_end && P[lo + step - 1] <= tl) {
              lo += step;
              step <<= 1;
            }
            int hi = min(lo + step - 1, seg_end);
            while (lo < hi) {
              const int mid = (lo + hi) >> 1;
              if (P[mid] > tl)
                hi = mid;
              else
                lo = mid + 1;
            }
            a = lo;
          }
          StateVec<R, NS>::load(X, a, x[r]);
          if (J.anc) J.anc[((size_t)i * (T - 1) + (t - 1)) * M + j] = a;
        }
      }
    }
  }
  if (lt == 0) J.loglik[i] = loglik;
}

template <typename R, int MODEL, int PPT, bool NAMED, bool GENERAL>
__global__ void __maxnreg__((RegCap<R, PPT>::value)) pf_kernel(PFLaunch L) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_wu;
  constexpr int NS = ModelDims<MODEL>::NS;
  const uint32_t k = L.k_done ? (uint32_t)(*L.k_done + 1) : (uint32_t)L.k_imm;
  const uint2 key = seed_key(L.seed);
  for (int it = 0;; ++it) {
    int w;
    if (L.wu_counter) {
      __syncthreads();
      if (threadIdx.x == 0) s_wu = atomicAdd(L.wu_counter, 1);
      __syncthreads();
      w = s_wu;
    } else {
      w = blockIdx.x + it * gridDim.x;
    }
    if (w >= L.n_wu) break;
    int job, first, count;
    if (L.wus) {
      const int4 u = L.wus[w];
      job = u.x;
      first = u.y;
      count = u.z;
    } else {
      job = 0;
      first = w * L.fpc_single;
      count = min(L.fpc_single, L.job0.n - first);
    }
    const PFJob J = L.jobs ? L.jobs[job] : L.job0;
    const int gt = group_threads_for(PPT, J.M);
    const int g = threadIdx.x / gt, lt = threadIdx.x - g * gt;
    const size_t rb = region_bytes(gt * PPT, gt >> 5, NS, (int)sizeof(R), is_staged(PPT), GENERAL);
    if (g < count && (g + 1) * gt <= (int)blockDim.x)
      run_filter<R, MODEL, PPT, NAMED, GENERAL>(J, L.mdl, first + g, g, lt, gt, smem + g * rb, key, k,
                                                L.t_cap);
    if (!L.wu_counter) __syncthreads();
  }
}


template <typename R, int MODEL, int PPT, bool NAMED, bool GENERAL>
const void* pf_kernel_ptr() {
  return reinterpret_cast<const void*>(&pf_kernel<R, MODEL, PPT, NAMED, GENERAL>);
}

// The GENERAL instantiations exist for the register-resident shapes only.
template <typename R, int MODEL, bool NAMED, bool GENERAL>
const void* pf_select_ppt(int ppt) {
  switch (ppt) {
    case 1: return pf_kernel_ptr<R, MODEL, 1, NAMED, GENERAL>();
    case 2: return pf_kernel_ptr<R, MODEL, 2, NAMED, GENERAL>();
    case 4: return pf_kernel_ptr<R, MODEL, 4, NAMED, GENERAL>();
    case 8:  // the variants and the SIR model run in the register-resident shapes only
      if constexpr (GENERAL || MODEL == MODEL_SIR) return nullptr;
      else return pf_kernel_ptr<R, MODEL, 8, NAMED, false>();
    case 16:
      if constexpr (GENERAL || MODEL == MODEL_SIR) return nullptr;
      else return pf_kernel_ptr<R, MODEL, 16, NAMED, false>();
    default: return nullptr;
  }
}

template <typename R, bool GENERAL>
const void* pf_select_precision(int model, int ppt, bool named) {
  if (model == MODEL_LG)
    return named ? pf_select_ppt<R, MODEL_LG, true, GENERAL>(ppt) : pf_select_ppt<R, MODEL_LG, false, GENERAL>(ppt);
  return named ? pf_select_ppt<R, MODEL_SEIR, true, GENERAL>(ppt) : pf_select_ppt<R, MODEL_SEIR, false, GENERAL>(ppt);
}

template <typename R, bool GENERAL>
const void* pf_select_sir(int ppt, bool named) {
  return named ? pf_select_ppt<R, MODEL_SIR, true, GENERAL>(ppt) : pf_select_ppt<R, MODEL_SIR, false, GENERAL>(ppt);
}

const void* pf_select_f32(int model, int ppt, bool named);
const void* pf_select_f64(int model, int ppt, bool named);
const void* pf_select_general_f32(int model, int ppt, bool named);
const void* pf_select_general_f64(int model, int ppt, bool named);
// the SIR model's instantiations (pf_sir_f32.cu, pf_sir_f64.cu)
const void* pf_select_sir_f32(int ppt, bool named, bool general);
const void* pf_select_sir_f64(int ppt, bool named, bool general);

}  // namespace smc2
