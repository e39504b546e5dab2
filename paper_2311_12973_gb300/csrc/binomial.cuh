// Binomial variates for the SIR model's daily flows (Sec. V-A draws them as
// binomials; the paper names no sampler).
//
// Bin(n, p): p <= 0 (or NaN) gives 0, p >= 1 gives n, p > 1/2 gives
// n - Bin(n, 1 - p).  For 0 < p <= 1/2:
//  * n p < 10: inversion, a sequential search from 0 on the pmf recurrence
//    P(0) = (1-p)^n, P(k) = P(k-1) ((n+1) s / k - s), s = p / (1-p); a search
//    that rounding carries past n draws again;
//  * otherwise the transformed rejection with squeeze of W. Hormann, "The
//    generation of binomial random variates", J. Statist. Comput. Simul. 46
//    (1993), algorithm BTRS: k = floor((2a/us + b) u + c) from u uniform on
//    (-1/2, 1/2), us = 1/2 - |u|; the squeeze us >= 0.07, v <= v_r accepts most
//    proposals outright, the rest pass the exact test of log(v alpha / (a/us^2 + b))
//    against the log-pmf ratio to the mode m.
// Uniforms come from a Philox word stream: call m = 0, 1, ... of counter
// (c0 + 4096 m, c1, c2, c3), words read in order x, y, z, w, each word w giving
// u = (2w + 1) 2^-33 (exact in double).  Consecutive draws may share a stream,
// each reading from where the last stopped.  After 64 calls (probability far
// below 1e-40) a draw returns floor((n + 1) p).
//
// The FP64 form below does every step in double with explicitly rounded
// operations, so that its decisions follow the same roundings on any IEEE
// machine (only exp, log1p, log and lgamma round on their own); the FP32 form
// further down serves the mixed-precision filter.
#pragma once

#include "common.cuh"

namespace smc2 {

struct BinomWords {
  uint4 ctr;
  uint2 key;
  uint4 cur;  // unread words of the current call, next in .x
  int left, calls;

  __device__ __forceinline__ BinomWords(uint4 c, uint2 k) : ctr(c), key(k), cur(), left(0), calls(0) {}

  // next uniform in (0, 1), or 0 when the stream is spent
  __device__ __forceinline__ double next() {
    if (left == 0) {
      if (calls == 64) return 0.0;
      cur = philox4x32_10(make_uint4(ctr.x + 4096u * (uint32_t)calls, ctr.y, ctr.z, ctr.w), key);
      ++calls;
      left = 4;
    }
    const uint32_t w = cur.x;
    cur.x = cur.y;
    cur.y = cur.z;
    cur.z = cur.w;
    --left;
    return ((double)w * 2.0 + 1.0) * 0x1p-33;  // exact
  }
};

// 0 < p <= 1/2; -1 when the stream is spent
static __device__ __noinline__ double binomial_half(double n, double p, BinomWords& b) {
  const double q = __dsub_rn(1.0, p);
  if (__dmul_rn(n, p) < 10.0) {
    const double s = __ddiv_rn(p, q);
    const double a = __dmul_rn(__dadd_rn(n, 1.0), s);
    const double r0 = exp(__dmul_rn(n, log1p(-p)));
    for (;;) {
      double u = b.next();
      if (u == 0.0) return -1.0;
      double r = r0, k = 0.0;
      while (u > r) {
        u = __dsub_rn(u, r);
        k = __dadd_rn(k, 1.0);
        if (k > n) break;
        r = __dmul_rn(r, __dsub_rn(__ddiv_rn(a, k), s));
      }
      if (k <= n) return k;
    }
  }
  const double spq = __dsqrt_rn(__dmul_rn(__dmul_rn(n, p), q));
  const double bb = __dadd_rn(1.15, __dmul_rn(2.53, spq));
  const double aa = __dadd_rn(__dadd_rn(-0.0873, __dmul_rn(0.0248, bb)), __dmul_rn(0.01, p));
  const double c = __dadd_rn(__dmul_rn(n, p), 0.5);
  const double vr = __dsub_rn(0.92, __ddiv_rn(4.2, bb));
  for (;;) {
    const double u1 = b.next();
    const double v1 = b.next();
    if (u1 == 0.0 || v1 == 0.0) return -1.0;
    const double u = __dsub_rn(u1, 0.5);
    const double us = __dsub_rn(0.5, fabs(u));
    const double k = floor(__dadd_rn(__dmul_rn(__dadd_rn(__ddiv_rn(__dmul_rn(2.0, aa), us), bb), u), c));
    if (k < 0.0 || k > n) continue;
    if (us >= 0.07 && v1 <= vr) return k;
    const double alpha = __dmul_rn(__dadd_rn(2.83, __ddiv_rn(5.1, bb)), spq);
    const double lpq = log(__ddiv_rn(p, q));
    const double m = floor(__dmul_rn(__dadd_rn(n, 1.0), p));
    const double h = __dadd_rn(lgamma(__dadd_rn(m, 1.0)), lgamma(__dadd_rn(__dsub_rn(n, m), 1.0)));
    const double v = log(__ddiv_rn(__dmul_rn(v1, alpha), __dadd_rn(__ddiv_rn(aa, __dmul_rn(us, us)), bb)));
    const double rhs = __dadd_rn(__dsub_rn(__dsub_rn(h, lgamma(__dadd_rn(k, 1.0))),
                                           lgamma(__dadd_rn(__dsub_rn(n, k), 1.0))),
                                 __dmul_rn(__dsub_rn(k, m), lpq));
    if (v <= rhs) return k;
  }
}

// Bin(n, p) for an integer n >= 0, reading the stream b from where it stands.
__device__ __forceinline__ double binomial_draw(double n, double p, BinomWords& b) {
  if (!(p > 0.0) || n <= 0.0) return 0.0;
  if (!(p < 1.0)) return n;
  if (p > 0.5) {
    const double r = binomial_half(n, __dsub_rn(1.0, p), b);
    return r < 0.0 ? floor(__dmul_rn(__dadd_rn(n, 1.0), p)) : __dsub_rn(n, r);
  }
  const double r = binomial_half(n, p, b);
  return r < 0.0 ? floor(__dmul_rn(__dadd_rn(n, 1.0), p)) : r;
}

// ---------------------------------------------------------------------------
// FP32 form (mixed precision).  The same two methods in float, with float
// uniforms u = ((w >> 9) + 0.5) 2^-23 (exact) from the same word stream.  A
// warp pays for a branch any of its lanes takes, and a double instruction
// occupies the narrow FP64 unit for the whole warp, so the rare exact test is
// in float too, in a form without cancellation: with m the mode and Stirling's
// log j! = (j + 1/2) log(j + 1) - (j + 1) + log(2 pi)/2 + fc(j),
//   log f(k)/f(m) = (m + 1/2) log1p((m - k)/(k + 1))
//                 + (n - m + 1/2) log1p((k - m)/(n - k + 1))
//                 + (k - m) log1p(((n + 2) p - (k + 1)) / ((k + 1) q))
//                 + fc(m) + fc(n - m) - fc(k) - fc(n - k),
// every log of a ratio near 1 at the k the test sees; (n + 2) p - (k + 1)
// takes the product's exact rounding error from an FMA, so the difference of
// two nearby values keeps its accuracy.  The error is below 5e-5 for n <= 1e4
// (1.3e-3 at n = 2^24), against the exact log-pmf ratio.  BTRS's proposal adds the large
// offset c = n p + 1/2 as floor(c) + floor(t + frac(c)), so the float rounding
// of the sum is that of the small part.  This is the FP64 sampler up to float
// roundings, not bit for bit.
// ---------------------------------------------------------------------------

// fc(j) = log j! - [(j + 1/2) log(j + 1) - (j + 1) + log(2 pi)/2]: the series
// 1/(12 x) - 1/(360 x^3) + 1/(1260 x^5), x = j + 1, for j >= 10 (error below
// 1/(1680 x^7)); from the exact factorial below 10.
__device__ __forceinline__ float stirling_fc(float j) {
  const float x = j + 1.f;
  if (j < 10.f) {
    float f = 1.f;
    for (int i = 2; i <= (int)j; ++i) f *= (float)i;  // exact: 9! < 2^24
    return logf(f) - ((j + 0.5f) * logf(x) - x + 0.918938533f);
  }
  const float r = __fdividef(1.f, x), r2 = r * r;
  return r * (1.f / 12.f - r2 * (1.f / 360.f - r2 * (1.f / 1260.f)));
}

struct BinomWordsF {
  uint4 ctr;
  uint2 key;
  uint4 cur;
  int left, calls;

  __device__ __forceinline__ BinomWordsF(uint4 c, uint2 k) : ctr(c), key(k), cur(), left(0), calls(0) {}

  __device__ __forceinline__ float next() {
    if (left == 0) {
      if (calls == 64) return 0.f;
      cur = philox4x32_10(make_uint4(ctr.x + 4096u * (uint32_t)calls, ctr.y, ctr.z, ctr.w), key);
      ++calls;
      left = 4;
    }
    const uint32_t w = cur.x;
    cur.x = cur.y;
    cur.y = cur.z;
    cur.z = cur.w;
    --left;
    return ((float)(w >> 9) + 0.5f) * 0x1p-23f;
  }
};

static __device__ __noinline__ float binomial_half_f32(float n, float p, BinomWordsF& b) {
  const float q = 1.f - p;
  if (n * p < 10.f) {
    const float s = p / q;
    const float a = (n + 1.f) * s;
    const float r0 = expf(n * log1pf(-p));
    for (;;) {
      float u = b.next();
      if (u == 0.f) return -1.f;
      float r = r0, k = 0.f;
      while (u > r) {
        u -= r;
        k += 1.f;
        if (k > n) break;
        r *= __fdividef(a, k) - s;
      }
      if (k <= n) return k;
    }
  }
  const float spq = sqrtf(n * p * q);
  const float bb = 1.15f + 2.53f * spq;
  const float aa = -0.0873f + 0.0248f * bb + 0.01f * p;
  const float c = n * p + 0.5f;
  const float ci = floorf(c), cf = c - ci;
  const float vr = 0.92f - __fdividef(4.2f, bb);
  bool have_m = false;
  float m = 0.f, fcm = 0.f, alpha = 0.f, np2 = 0.f, np2_err = 0.f;
  for (;;) {
    const float u1 = b.next();
    const float v1 = b.next();
    if (u1 == 0.f || v1 == 0.f) return -1.f;
    const float u = u1 - 0.5f;
    const float us = 0.5f - fabsf(u);
    const float k = ci + floorf((__fdividef(2.f * aa, us) + bb) * u + cf);
    if (k < 0.f || k > n) continue;
    if (us >= 0.07f && v1 <= vr) return k;
    if (!have_m) {
      m = floorf(fmaf(n, p, p));  // floor((n + 1) p), one rounding
      fcm = stirling_fc(m) + stirling_fc(n - m);
      alpha = (2.83f + __fdividef(5.1f, bb)) * spq;
      const float n2 = n + 2.f;
      np2 = n2 * p;
      np2_err = fmaf(n2, p, -np2);  // (n + 2) p = np2 + np2_err exactly
      have_m = true;
    }
    const float d = ((np2 - (k + 1.f)) + np2_err);
    const float lr = (m + 0.5f) * log1pf(__fdividef(m - k, k + 1.f)) +
                     (n - m + 0.5f) * log1pf(__fdividef(k - m, n - k + 1.f)) +
                     (k - m) * log1pf(__fdividef(d, (k + 1.f) * q)) + fcm - stirling_fc(k) -
                     stirling_fc(n - k);
    const float v = logf(__fdividef(v1 * alpha, __fdividef(aa, us * us) + bb));
    if (v <= lr) return k;
  }
}

// Bin(n, p) in the FP32 form, for an integer n >= 0 below 2^24, reading the
// stream b from where it stands.
__device__ __forceinline__ float binomial_draw(float n, float p, BinomWordsF& b) {
  if (!(p > 0.f) || n <= 0.f) return 0.f;
  if (!(p < 1.f)) return n;
  if (p > 0.5f) {
    const float r = binomial_half_f32(n, 1.f - p, b);
    return r < 0.f ? floorf((n + 1.f) * p) : n - r;
  }
  const float r = binomial_half_f32(n, p, b);
  return r < 0.f ? floorf((n + 1.f) * p) : r;
}

}  // namespace smc2
