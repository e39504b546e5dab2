// pf_fast.cuh -- the FP32 bootstrap particle filter (Sec. II) with one filter
// per thread group and the particles held in registers: the group is the whole
// CTA, or (the grouped instantiations, for datasets of unequal M) one of
// several groups of unequal width that share it.
//
// The same filter as pf_kernel's default (systematic resampling after every
// step t < T, Eqs. 26-27 with Algorithm 1's output order; the mean-weight reset
// of Eq. 13; the likelihood increment of Eq. 8), shaped for few instructions
// per particle: each of the group's T threads owns PPT consecutive particles
// (2, 4 or 8) and works on them in pairs with the packed two-wide FP32
// instructions, and no step has a loop whose length differs between lanes.
// Per step:
//   1. propagate and log-weight every particle in registers (Eqs. 1, 2, 5);
//   2. the group maximum of the log-weights (one warp reduction; one barrier
//      when the group has several warps);
//   3. q_j = floor(exp(l_j - max) 2^B) with the floor to u64 taken as two exact
//      32-bit conversions (a float-to-u64 conversion instruction would run on
//      the narrow FP64 pipe), a thread-local inclusive prefix, one warp scan and
//      (several warps) one more barrier for the warp totals;
//   4. the increment max + log(S 2^-B) - log M from the exact integer total S;
//   5. resampling by marks: particle j fills the slots F(C_{j-1}) .. F(C_j) - 1,
//      F(C) the number of thresholds tau_s = floor((s + u) S / M) below C (the
//      slot counting of pf_kernel).  Each particle with copies writes its index,
//      tagged with a step counter, at its first slot, and at the first slot of
//      every thread whose slots its range covers (the rare ranges that cover
//      more than one such slot after the loop, so that the loop has no branch);
//      after a barrier the ancestor of slot s is the largest current tag at or
//      before s within its thread's slots -- ancestors never decrease along the
//      slots -- and the thread reads that particle's state.
// Shared arrays indexed by a slot or a particle s keep it at row s % PPT, column
// s / PPT, so that a warp reading one entry per thread touches consecutive words.
#pragma once

#include "pf_impl.cuh"

namespace smc2 {

// floor(v) for a float 0 <= v <= 2^52 as its two 32-bit halves: hi = floor(v 2^-32)
// and lo = floor(v - hi 2^32).  Both steps are exact in float (v 2^-32 is a power-of-
// two scaling; v - hi 2^32 = v mod 2^32 holds at most v's 24 significant bits), and
// the two 32-bit conversions avoid the float-to-u64 one, which runs on the FP64 pipe.
__device__ __forceinline__ uint64_t floor_to_u64(float v) {
  const float hi = floorf(v * 0x1p-32f);
  const float lo = fmaf(-hi, 0x1p32f, v);
  return ((uint64_t)__float2uint_rz(hi) << 32) | (uint64_t)__float2uint_rz(lo);
}

// 2^x by the hardware approximation (relative error about 2^-22; 0 for -inf).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float rcp_approx(float x) {  // 1/x, hardware approximation (about 1 ulp)
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_approx(float x) {  // log2 x, hardware approximation
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 max2(float2 a, float b) { return make_float2(fmaxf(a.x, b), fmaxf(a.y, b)); }

// The models' per-filter constants for pairs of particles (the SEIR-type
// model's Euler day and Poisson log-weight, the AR(1) step and Gaussian
// log-weight), computed as FilterParams computes them for one particle.
template <int MODEL>
struct PairModel;

template <>
struct PairModel<MODEL_LG> {
  float2 phi, sx, inv_sy, c_obs;
  __device__ explicit PairModel(const FilterParams<float, MODEL_LG>& f)
      : phi(bc2(f.phi)), sx(bc2(f.sx)), inv_sy(bc2(f.inv_sy)), c_obs(bc2(f.c_obs)) {}
  // x = phi x + sx z; l = c - (1/2) ((y - x) / sy)^2 (no fix-up: far = 0)
  __device__ __forceinline__ static float2 fix_far(float2 l, float2, int, const float4&) { return l; }
  __device__ __forceinline__ float2 step(float2* x, float2 z, const float4& ob, float2& lam, float2& d,
                                         int& far) const {
    far = 0;
    d = bc2(0.f);
    x[0] = fma2(phi, x[0], mul2(sx, z));
    const float2 r = mul2(fma2(x[0], bc2(-1.f), bc2(ob.x)), inv_sy);
    lam = bc2(0.f);
    return fma2(mul2(bc2(-0.5f), r), r, c_obs);
  }
};

template <>
struct PairModel<MODEL_SEIR> {
  float2 srw, kappa, gamma, inv_npop, dt, ndt;
  float lam_floor;
  int n_sub;
  __device__ explicit PairModel(const FilterParams<float, MODEL_SEIR>& f)
      : srw(bc2(f.srw)), kappa(bc2(f.kappa)), gamma(bc2(f.gamma)), inv_npop(bc2(f.inv_npop)), dt(bc2(f.dt)),
        ndt(bc2(-f.dt)), lam_floor(f.lam_floor), n_sub(f.n_sub) {}
  __device__ __forceinline__ void substep(float2 beta, float2& S, float2& E, float2& I, float2& lam) const {
    const float2 inf = mul2(mul2(mul2(beta, S), I), inv_npop);
    const float2 onset = mul2(kappa, E);
    const float2 recovery = mul2(gamma, I);
    lam = fma2(dt, onset, lam);
    S = max2(fma2(ndt, inf, S), 0.f);
    E = max2(fma2(dt, fma2(onset, bc2(-1.f), inf), E), 0.f);       // E + dt (inf - onset)
    I = max2(fma2(dt, fma2(recovery, bc2(-1.f), onset), I), 0.f);  // I + dt (onset - recovery)
  }
  // x = (S, E, I, log beta) of two particles; returns their log-weights, and lam the day's incidence
  __device__ __forceinline__ float2 step(float2* x, float2 z, const float4& ob, float2& lam, float2& d,
                                         int& far) const {
    x[3] = fma2(srw, z, x[3]);
    const float2 beta = make_float2(__expf(x[3].x), __expf(x[3].y));
    float2 S = x[0], E = x[1], I = x[2];
    lam = bc2(0.f);
    if (n_sub == 2) {
      substep(beta, S, E, I, lam);
      substep(beta, S, E, I, lam);
    } else {
      for (int s = 0; s < n_sub; ++s) substep(beta, S, E, I, lam);
    }
    x[0] = S;
    x[1] = E;
    x[2] = I;
    lam = max2(lam, lam_floor);
    // Poisson log-pmf y (log1p(d) - d) + c_y, d = (lambda - y) / y (no cancellation near y);
    // d is returned for the fix-up of the pairs whose |s| > 1/3 (see log1p_minus)
    if (ob.x > 0.f) {
      d = mul2(add2(lam, bc2(-ob.x)), bc2(ob.y));
      return fma2(bc2(ob.x), log1p_minus(d, far), bc2(ob.z));
    }
    far = 0;
    return mul2(lam, bc2(-1.f));
  }
  // the Poisson log-weights of a pair whose log1p_minus took the series outside its range
  __device__ __forceinline__ static float2 fix_far(float2 l, float2 d, int far, const float4& ob) {
    const float2 u = add2(d, bc2(1.f));
    const float2 lg = make_float2(lg2_approx(u.x), lg2_approx(u.y));
    const float2 r2 = fma2(bc2(ob.x), fma2(lg, bc2(0.69314718055994531f), mul2(d, bc2(-1.f))), bc2(ob.z));
    return make_float2((far & 1) ? r2.x : l.x, (far & 2) ? r2.y : l.y);
  }
  // log1p(d) - d for two values.  With s = d / (2 + d), ln(1 + d) = 2 atanh s =
  // 2 (s + s^3/3 + s^5/5 + ...) (Abramowitz and Stegun 4.1.27), and 2s - d = -s d, so
  //   log1p(d) - d = -s d + 2 s^3 (1/3 + s^2/5 + s^4/7 + ... + s^10/13):
  // for d < 0 both terms have one sign, for d > 0 the second is at most 2 s^2 / 3 <= 0.08 of
  // the first, so no leading digits cancel.  For |s| <= 1/3 (-1/2 <= d <= 1) the omitted
  // terms are below 10^-7 of the result.  Outside, |log1p(d) - d| >= 0.19 and
  // ln(1 + d) from the hardware log2 (absolute error about 2^-22) serves; the warp takes
  // that path (fix_far) only when one of its lanes needs it.
  __device__ __forceinline__ static float2 log1p_minus(float2 d, int& far) {
    const float2 den = add2(d, bc2(2.f));
    const float2 sv = mul2(d, make_float2(rcp_approx(den.x), rcp_approx(den.y)));
    const float2 s2 = mul2(sv, sv);
    float2 p = fma2(s2, bc2(1.f / 13.f), bc2(1.f / 11.f));
    p = fma2(s2, p, bc2(1.f / 9.f));
    p = fma2(s2, p, bc2(1.f / 7.f));
    p = fma2(s2, p, bc2(1.f / 5.f));
    p = fma2(s2, p, bc2(1.f / 3.f));
    const float2 t = mul2(mul2(s2, sv), bc2(2.f));                      // 2 s^3
    far = (fabsf(sv.x) > (1.f / 3.f) ? 1 : 0) | (fabsf(sv.y) > (1.f / 3.f) ? 2 : 0);
    return fma2(sv, mul2(d, bc2(-1.f)), mul2(t, p));  // -s d + 2 s^3 P(s^2)
  }
};

// Four normals from one Philox call with the round keys of the kernel's
// parameter block (the same numbers as normals4 with the seed's key).
__device__ __forceinline__ void normals4_rk(uint4 c, const uint32_t (&rk)[20], float z[4]) {
  const uint4 w = philox4x32_10_rk(c, rk);
  box_muller<float>(w.x, w.y, z[0], z[1]);
  box_muller<float>(w.z, w.w, z[2], z[3]);
}

// Register budget per particles-per-thread shape of the FP32 filter (grouped
// instantiations hold the group's width, index and region in registers too).
// 64 at ppt 4 fits four 256-thread CTAs per SM without spills; at ppt 8, 96
// registers (five 128-thread CTAs per SM, no spills) measured slower than 128.
template <int PPT, bool GROUPED>
struct FastRegCap {
  static constexpr int value = GROUPED ? (PPT <= 2 ? 72 : (PPT == 4 ? 96 : 128))
                                       : (PPT <= 2 ? 64 : (PPT == 4 ? 64 : 128));
  static_assert(PPT == 2 || PPT == 4 || PPT == 8, "particles per thread");
};

// Shared memory of one filter group of T threads holding Mp = PPT T particles
// (the whole CTA's, or one of the grouped instantiation's regions):
//   Xo    float  [PPT][T][NS]   states after propagation, by particle
//   Z     float2 [4][PPT/2][T]  the four normals of the current Philox counter of each slot pair
//   mark  u32    [PPT][T]       step-tagged particle indices at the slots
//   carry u32    [T]            the tagged ancestor of each thread's first slot
//   wsum u64 [32], wmax float [32], sU u32 [8]
__host__ __device__ constexpr size_t fast_region_bytes(int Mp, int ns) {
  return (size_t)ns * Mp * 4 + (size_t)4 * Mp * 4 + (size_t)Mp * 4 + (size_t)(Mp / 2) * 4 + 32 * 8 + 32 * 4 + 32;
}

constexpr int kMarkBits = 12;  // particle index bits of a mark (M <= 4096)

// Maximum over the warp in one reduction instruction: a float maps to an int
// whose signed order is the float's (negative values have their magnitude bits
// flipped), -inf included; no NaN reaches it.
__device__ __forceinline__ float warp_max_redux(float v) {
  const int b = __float_as_int(v);
  const int key = b ^ ((b >> 31) & 0x7fffffff);
  const int m = __reduce_max_sync(0xffffffffu, key);
  return __int_as_float(m ^ ((m >> 31) & 0x7fffffff));
}

// slots_below split for a whole warp: the float estimate decides every crossing
// point away from an integer (slots_estimate, which flags the others), and the
// exact 128-bit comparison (slots_exact) settles the flagged ones.
__device__ __forceinline__ int slots_estimate(const SlotCount& sc, float Cf, bool& near) {
  const float est = fmaf(Cf, sc.scale, -sc.off);
  near = !(fabsf(est - rintf(est)) > sc.margin);
  return __float2int_ru(est);  // the ceiling, in one conversion
}
__device__ __forceinline__ int slots_exact(const SlotCount& sc, uint64_t C, float Cf) {
  const float est = fmaf(Cf, sc.scale, -sc.off);
  int n = min(max((int)rintf(est), 0), sc.M - 1);
  const uint64_t a = ((uint64_t)n << 33) + sc.U21;
  const uint64_t lh = __umul64hi(a, sc.S), ll = a * sc.S;
  const uint64_t rh = __umul64hi(C, sc.M33), rl = C * sc.M33;
  return n + ((lh < rh || (lh == rh && ll < rl)) ? 1 : 0);
}

// Barrier of one filter group of T threads (group g of its CTA).  Ungrouped
// instantiations run one group that is the whole CTA.  Grouped ones (datasets of
// unequal width in one launch) let a warp synchronise alone, a group that fills
// the CTA use the CTA barrier, and groups of several warps that share a CTA use
// named barrier 1 + g.
template <bool GROUPED>
__device__ __forceinline__ void fast_group_sync(int T, int g) {
  if (!GROUPED)
    __syncthreads();
  else if (T == 32)
    __syncwarp();
  else if (T != (int)blockDim.x)
    named_barrier(1 + g, T);
  else
    __syncthreads();
}

template <int MODEL, int PPT, bool TRACE, bool GROUPED>
__device__ __forceinline__ void fast_filter(const PFJob& J, const PFModel& mdl, int i, unsigned char* smem,
                                            const uint32_t (&rk)[20], uint32_t k, int t_cap, int lt, int T,
                                            int g) {
  constexpr int NS = ModelDims<MODEL>::NS;
  constexpr int D = ModelDims<MODEL>::D;
  constexpr int LOG2P = PPT == 2 ? 1 : (PPT == 4 ? 2 : 3);
  constexpr int NP = PPT / 2;  // pairs per thread
  const int nw = T >> 5;
  const int lane = lt & 31, warp = lt >> 5;
  const int M = J.M, TT = t_cap > 0 ? min(J.T, t_cap) : J.T;
  const int Mp = PPT * T;
  float* Xo = reinterpret_cast<float*>(smem);                           // [PPT][T][NS]
  float2* Z = reinterpret_cast<float2*>(Xo + (size_t)NS * Mp);          // [4][NP][T]
  uint32_t* mark = reinterpret_cast<uint32_t*>(Z + (size_t)2 * Mp);     // [PPT][T]
  uint32_t* carry = mark + Mp;                                          // [T]
  uint64_t* wsum = reinterpret_cast<uint64_t*>(carry + (Mp / 2));       // [32] (Mp / 2 >= T keeps 8-byte alignment)
  float* wmax = reinterpret_cast<float*>(wsum + 32);                    // [32]
  uint32_t* sU = reinterpret_cast<uint32_t*>(wmax + 32);                // [8]

  // the marks start untagged for every filter: the region may have held another
  // dataset's layout, and the step tag restarts at 1
  for (int s = lt; s < Mp; s += T) mark[s] = 0u;
  carry[lt] = 0u;  // threads whose slots are all padding keep this valid ancestor (particle 0)
  uint32_t tag = 0;
  fast_group_sync<GROUPED>(T, g);

  double th[D];
#pragma unroll
  for (int d = 0; d < D; ++d) th[d] = J.theta[(size_t)d * J.ld + i];
  FilterParams<float, MODEL> fp;
  fp.load(th, mdl);
  const PairModel<MODEL> pm(fp);

  const uint32_t c2 = counter_c2((uint32_t)i, J.c2hi);
  const uint32_t c3prop = counter_c3(TAG_PF_PROP, k);
  const uint32_t c3res = counter_c3(TAG_PF_RES, k);
  const int B = fixed_point_bits(M);
  const float2 scaleB = bc2(ldexpf(1.f, B));
  const float logM = logf((float)M);
  const float4* obs = reinterpret_cast<const float4*>(J.obs);

  float2 x[NP][NS];  // particles 2p and 2p + 1 of the thread in x[p] (.x, .y)
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    float a[NS], b[NS];
    float za = 0.f, zb = 0.f;
    if constexpr (MODEL == MODEL_LG) {
      float z[4];
      normals4_rk(make_uint4((uint32_t)(lt * PPT + 2 * p), 0u, c2, counter_c3(TAG_PF_INIT, k)), rk, z);
      za = z[0];
      normals4_rk(make_uint4((uint32_t)(lt * PPT + 2 * p + 1), 0u, c2, counter_c3(TAG_PF_INIT, k)), rk, z);
      zb = z[0];
    }
    fp.init(a, za, th);
    fp.init(b, zb, th);
#pragma unroll
    for (int e = 0; e < NS; ++e) x[p][e] = make_float2(a[e], b[e]);
  }

  // log p^(y_{1:t}) (Eq. 8) = lsum_m + lsum_hi + lsum_lo, carried by thread 0
  double lsum_m = 0.0;
  float lsum_hi = 0.f, lsum_lo = 0.f;
  bool dead = false;
  for (int t = 1; t <= TT; ++t) {
    const int tm = (t - 1) & 3;
    uint32_t* sUg = sU + 4 * (((t - 1) >> 2) & 1);
    if (tm == 0) {  // one Philox call per slot every four steps; the normals wait in shared memory
#pragma unroll 1
      for (int p = 0; p < NP; ++p) {
        float za[4], zb[4];
        normals4_rk(make_uint4((uint32_t)(lt * PPT + 2 * p), (uint32_t)((t - 1) >> 2), c2, c3prop), rk, za);
        normals4_rk(make_uint4((uint32_t)(lt * PPT + 2 * p + 1), (uint32_t)((t - 1) >> 2), c2, c3prop), rk, zb);
#pragma unroll
        for (int e = 0; e < 4; ++e) Z[(e * NP + p) * T + lt] = make_float2(za[e], zb[e]);
      }
      if (lt < 4 && t + lt < TT) sUg[lt] = philox4x32_10_rk(make_uint4(0u, (uint32_t)(t + lt), c2, c3res), rk).x;
      if (nw == 1) __syncwarp();  // the resampling words before the warp reads them (wider groups: barriers below)
    }
    const float4 ob = obs[t - 1];
    float ell[PPT];
    float lmax = -INFINITY;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      float2 lam, dp;
      int far;
      float2 l2 = pm.step(x[p], Z[(tm * NP + p) * T + lt], ob, lam, dp, far);
      if (__any_sync(0xffffffffu, far != 0)) l2 = PairModel<MODEL>::fix_far(l2, dp, far, ob);  // rare
      const int j = lt * PPT + 2 * p;
      const float la = (isnan(l2.x) || j >= M) ? -INFINITY : l2.x;
      const float lb = (isnan(l2.y) || j + 1 >= M) ? -INFINITY : l2.y;
      ell[2 * p] = la;
      ell[2 * p + 1] = lb;
      lmax = fmaxf(lmax, fmaxf(la, lb));
      if constexpr (TRACE) {
        if (J.xtr) {
          const size_t row = ((size_t)i * J.T + (t - 1)) * M + j;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            if (j + h >= M) continue;
            float* xt = J.xtr + (row + h) * kTraceState;
#pragma unroll
            for (int e = 0; e < NS; ++e) xt[e] = h ? x[p][e].y : x[p][e].x;
            if constexpr (MODEL == MODEL_SEIR) xt[NS] = h ? lam.y : lam.x;
            J.ltr[row + h] = h ? lb : la;
          }
        }
      }
    }
    // (2) group maximum
    lmax = warp_max_redux(lmax);
    if (nw > 1) {  // lane w reads warp w's maximum; one more reduction spreads the group's
      if (lane == 0) wmax[warp] = lmax;
      fast_group_sync<GROUPED>(T, g);
      lmax = warp_max_redux(lane < nw ? wmax[lane] : -INFINITY);
    }
    const float m = lmax;
    if (!(m > -INFINITY)) {  // every weight vanished: the estimate is zero
      dead = true;
      if constexpr (TRACE) {
        if (lt == 0 && J.delta)
          for (int s = t; s <= J.T; ++s) J.delta[(size_t)i * J.T + (s - 1)] = -HUGE_VAL;
      }
      break;
    }
    // (3) quantise: v = 2^((l - max) log2 e) 2^B (0 for l = -inf), q = floor(v); the
    // thread-local inclusive prefix (exact) and its float shadow
    uint64_t c[PPT];
    float cf[PPT];
    uint64_t run = 0;
    float runf = 0.f;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const float2 a = mul2(add2(make_float2(ell[2 * p], ell[2 * p + 1]), bc2(-m)), bc2(1.4426950408889634f));
      const float2 v = mul2(make_float2(ex2_approx(a.x), ex2_approx(a.y)), scaleB);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float vh = h ? v.y : v.x;
        const uint64_t q = floor_to_u64(vh);
        run += q;
        runf += vh;
        c[2 * p + h] = run;
        cf[2 * p + h] = runf;
        if constexpr (TRACE) {
          if (J.qtr && lt * PPT + 2 * p + h < M) J.qtr[((size_t)i * J.T + (t - 1)) * M + lt * PPT + 2 * p + h] = q;
        }
      }
    }
    const uint64_t incl = warp_incl_scan_u64(run, lane);
    const uint64_t excl = incl - run;
    uint64_t S, base = 0;
    if (nw > 1) {  // lane w reads warp w's total; an inclusive shuffle scan gives S and the warp's base
      if (lane == 31) wsum[warp] = incl;
      fast_group_sync<GROUPED>(T, g);
      uint64_t wp = lane < nw ? wsum[lane] : 0ull;
      for (int o = 1; o < nw; o <<= 1) {
        const uint64_t n = __shfl_up_sync(0xffffffffu, wp, o);
        if (lane >= o) wp += n;
      }
      S = __shfl_sync(0xffffffffu, wp, nw - 1);
      const uint64_t b = __shfl_sync(0xffffffffu, wp, warp > 0 ? warp - 1 : 0);
      base = warp > 0 ? b : 0ull;
    } else {
      S = __shfl_sync(0xffffffffu, incl, 31);
    }
    // (4) log-likelihood increment from the exact integer total (S >= 2^(B-1), B >= 51):
    // max + [(e - B) ln 2 + log(S 2^-e) - log M].  The maxima are summed in FP64 (exact for
    // floats); the bracket, a few units in size, as an unevaluated float pair (hi, lo) by
    // Knuth's TwoSum, which keeps the sum to about 2^-48, so that a step costs the narrow
    // FP64 pipe two instructions.
    if (lt == 0) {
      const int e = 63 - __clzll((long long)S);
      const float mant = __uint2float_rn((uint32_t)(S >> (e - 31))) * 0x1p-31f;  // S / 2^e in [1, 2]
      const float small = fmaf((float)(e - B), (float)kLn2, logf(mant)) - logM;
      lsum_m += (double)m;
      const float sh = lsum_hi + small, bv = sh - lsum_hi;  // TwoSum: sh + err = lsum_hi + small exactly
      lsum_lo += (lsum_hi - (sh - bv)) + (small - bv);
      lsum_hi = sh;
      if constexpr (TRACE) {
        if (J.delta) J.delta[(size_t)i * J.T + (t - 1)] = (double)m + (double)small;
      }
    }
    // (5) systematic resampling by marks
    if (t < TT) {
      if (++tag == (1u << (32 - kMarkBits))) {  // the tags are spent: clear every mark, start again
        for (int s = lt; s < Mp; s += T) mark[s] = 0u;
        tag = 1;
        fast_group_sync<GROUPED>(T, g);
      }
      const uint32_t tg = tag << kMarkBits;
      const SlotCount sc = slot_count_setup(sUg[tm], S, M);
      const uint64_t C0 = base + excl;  // cumulative weight before the thread's first particle
      const float C0f = u64_to_float(C0);
      int ends[PPT + 1];
      if constexpr (PPT < 8) {
        // Few particles per thread: every crossing from the float estimate, whose
        // error is under 17 M u + 2 u + 8 M / S (u = 2^-24): S and C0 each reach float
        // through two roundings (2 u), the approximate division M / S adds 2 ulp (4 u),
        // the thread's running float sum 7 u of its own share (at most M) and its
        // unfloored weights under 8 M / S, the sum C0 + share and the fma 1 u each, and
        // the offset 2 u absolute.  A margin of M 2^-19 + 2^-20 covers that 1.8 times.
        SlotCount sm = sc;
        sm.margin = fmaf((float)M, 0x1p-19f, 0x1p-20f);
        uint32_t near_mask = 0;
#pragma unroll
        for (int r = 0; r <= PPT; ++r) {
          bool nr;
          ends[r] = slots_estimate(sm, r == 0 ? C0f : C0f + cf[r - 1], nr);
          near_mask |= nr ? (1u << r) : 0u;
        }
        if (__any_sync(0xffffffffu, near_mask != 0)) {
#pragma unroll
          for (int r = 0; r <= PPT; ++r)
            if (near_mask & (1u << r))
              ends[r] = slots_exact(sm, r == 0 ? C0 : C0 + c[r - 1], r == 0 ? C0f : C0f + cf[r - 1]);
        }
      } else {
        // Eight particles per thread, where one exact test per thread costs less than
        // the near crossings' tests: the thread's first crossing exactly, n0 from the
        // float estimate (its error, under 17 M u, is far below 1/2), then
        // E = C0 M 2^33 - (2^33 n0 + 2U + 1) S, which is S 2^33 (x0 - n0) for the crossing
        // point x0 = C0 M / S - (2U + 1) 2^-33 of Eq. (27): F(C0) = n0 + [E > 0], and
        // e0 = x0 - n0 = E 2^-33 / S to about 9 u.  |x0 - n0| < 1 and S <= 2^63 keep
        // E 2^-33 inside 64 bits.
        const int n0 = min(max((int)rintf(fmaf(C0f, sc.scale, -sc.off)), 0), M - 1);
        const uint64_t a0 = ((uint64_t)n0 << 33) + sc.U21;
        const uint64_t p_lo = a0 * sc.S, p_hi = __umul64hi(a0, sc.S);
        const uint64_t q_lo = C0 * sc.M33, q_hi = __umul64hi(C0, sc.M33);
        const uint64_t e_lo = q_lo - p_lo, e_hi = q_hi - p_hi - (q_lo < p_lo ? 1ull : 0ull);
        const long long e33 = (long long)((e_hi << 31) | (e_lo >> 33));
        const float e0 = fmaf((float)(int)(e33 >> 32), 0x1p32f, (float)(uint32_t)e33) * sc.scale / (float)M;
        // The later crossings x0 + s_r M / S, s_r the thread's share of the weight
        // before particle r: its float sum errs by 7 u of itself, M / S by 6 u and the
        // product by 1 u, so y = e0 + s_r M / S errs by under 15 u s_r M / S + 10 u.  A
        // margin of 2^-19 (s_r M / S + 1) covers that twice; crossings inside it (rare:
        // the margin follows the share, not M) take the exact test.
        ends[0] = n0 + (((long long)e_hi > 0 || (e_hi == 0 && e_lo != 0)) ? 1 : 0);
        uint32_t near_mask = 0;
#pragma unroll
        for (int r = 1; r <= PPT; ++r) {
          const float inc = cf[r - 1] * sc.scale;
          const float y = e0 + inc;
          near_mask |= !(fabsf(y - rintf(y)) > fmaf(inc, 0x1p-19f, 0x1p-19f)) ? (1u << r) : 0u;
          ends[r] = n0 + __float2int_ru(y);
        }
        if (__any_sync(0xffffffffu, near_mask != 0)) {
#pragma unroll
          for (int r = 1; r <= PPT; ++r)
            if (near_mask & (1u << r)) ends[r] = slots_exact(sc, C0 + c[r - 1], C0f + cf[r - 1]);
        }
      }
      int start = ends[0];
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        float a[NS], b[NS];
#pragma unroll
        for (int e = 0; e < NS; ++e) {
          a[e] = x[p][e].x;
          b[e] = x[p][e].y;
        }
        StateVec<float, NS>::store(Xo + (size_t)((2 * p) * T + lt) * NS, 0, a);
        StateVec<float, NS>::store(Xo + (size_t)((2 * p + 1) * T + lt) * NS, 0, b);
      }
      uint32_t longmask = 0;  // particles whose slots reach past a second thread's first slot
#pragma unroll
      for (int r = 0; r < PPT; ++r) {
        const int end = ends[r + 1];
        const uint32_t mk = tg | (uint32_t)(lt * PPT + r);
        if (end > start) mark[(start & (PPT - 1)) * T + (start >> LOG2P)] = mk;
        // the first slot of every thread inside [start, end): usually none or one
        const int b0 = (start + PPT - 1) & ~(PPT - 1);
        if (b0 < end) carry[b0 >> LOG2P] = mk;
        longmask |= (end - b0 > PPT) ? (1u << r) : 0u;
        start = end;
      }
      if (__any_sync(0xffffffffu, longmask != 0)) {  // the further first slots, after the straight-line loop
        start = ends[0];
#pragma unroll
        for (int r = 0; r < PPT; ++r) {
          const int end = ends[r + 1];
          if ((longmask >> r) & 1u) {
            const uint32_t mk = tg | (uint32_t)(lt * PPT + r);
            for (int b = ((start + PPT - 1) & ~(PPT - 1)) + PPT; b < end; b += PPT) carry[b >> LOG2P] = mk;
          }
          start = end;
        }
      }
      fast_group_sync<GROUPED>(T, g);
      uint32_t a = carry[lt];
#pragma unroll
      for (int r = 0; r < PPT; ++r) {
        // Padding slots (j >= M) take the last real particle's mark, or the
        // cleared carry (particle 0): a valid state whose weight is never used.
        a = max(a, mark[r * T + lt]);
        const int src = (int)(a & ((1u << kMarkBits) - 1));
        if constexpr (TRACE) {
          if (J.anc && lt * PPT + r < M) J.anc[((size_t)i * (J.T - 1) + (t - 1)) * M + lt * PPT + r] = src;
        }
        const float* xs = Xo + ((size_t)(src & (PPT - 1)) * T + (src >> LOG2P)) * NS;
        float v[NS];
        StateVec<float, NS>::load(xs, 0, v);
#pragma unroll
        for (int e = 0; e < NS; ++e) {
          if (r & 1)
            x[r >> 1][e].y = v[e];
          else
            x[r >> 1][e].x = v[e];
        }
      }
      if (nw == 1) __syncwarp();  // every read done before the next step's writes
    }
  }
  if (lt == 0) J.loglik[i] = dead ? -HUGE_VAL : lsum_m + ((double)lsum_hi + (double)lsum_lo);
}

template <int MODEL, int PPT, bool TRACE, bool GROUPED>
__global__ void __maxnreg__((FastRegCap<PPT, GROUPED>::value)) pf_fast_kernel(PFLaunch L) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_wu;
  const uint32_t k = L.k_done ? (uint32_t)(*L.k_done + 1) : (uint32_t)L.k_imm;
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
    if (!GROUPED) {  // one group, the whole CTA: a unit's filters run in turn
      for (int f = 0; f < count; ++f) {
        if (f) __syncthreads();
        fast_filter<MODEL, PPT, TRACE, false>(J, L.mdl, first + f, smem, L.rk, k, L.t_cap, threadIdx.x, blockDim.x, 0);
      }
    } else {  // groups of T threads, one filter each: warps, or named-barrier groups
      const int T = group_threads_for(PPT, J.M);
      const int g = threadIdx.x / T, lt = threadIdx.x - g * T;
      const size_t rb = (fast_region_bytes(PPT * T, ModelDims<MODEL>::NS) + 15) & ~(size_t)15;
      if (g < count && (g + 1) * T <= (int)blockDim.x)
        fast_filter<MODEL, PPT, TRACE, true>(J, L.mdl, first + g, smem + g * rb, L.rk, k, L.t_cap, lt, T, g);
    }
    if (!L.wu_counter) __syncthreads();
  }
}

template <int MODEL, bool TRACE, bool GROUPED>
const void* pf_fast_select(int ppt) {
  switch (ppt) {
    case 2: return reinterpret_cast<const void*>(&pf_fast_kernel<MODEL, 2, TRACE, GROUPED>);
    case 4: return reinterpret_cast<const void*>(&pf_fast_kernel<MODEL, 4, TRACE, GROUPED>);
    case 8: return reinterpret_cast<const void*>(&pf_fast_kernel<MODEL, 8, TRACE, GROUPED>);
    default: return nullptr;
  }
}

// instantiated in pf_fast_lg.cu, pf_fast_seir.cu (one group per CTA) and
// pf_fast_grouped.cu (groups of unequal width sharing a CTA, untraced)
const void* pf_fast_select_lg(int ppt, bool trace);
const void* pf_fast_select_seir(int ppt, bool trace);
const void* pf_fast_select_grouped(int model, int ppt);

}  // namespace smc2
