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
// Uniforms come from the draw's own Philox word stream: call m = 0, 1, ... of
// counter (c0 + 8192 m, c1, c2, c3), words read in order x, y, z, w, each word
// w giving u = (2w + 1) 2^-33 (exact in double).  After 64 calls (probability
// far below 1e-40 for any n, p) the draw returns floor((n + 1) p).
//
// The arithmetic is in double in both precisions (the log-pmf differences of
// the exact test cancel to a few units in float at n ~ 1e4), with explicitly
// rounded operations, so that the decisions follow the same roundings on any
// IEEE machine; only exp, log1p, log and lgamma round on their own.
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
      cur = philox4x32_10(make_uint4(ctr.x + 8192u * (uint32_t)calls, ctr.y, ctr.z, ctr.w), key);
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

// Bin(n, p) for an integer n >= 0 from the word stream of counter ctr.
__device__ __forceinline__ double binomial_draw(double n, double p, uint4 ctr, uint2 key) {
  if (!(p > 0.0) || n <= 0.0) return 0.0;
  if (!(p < 1.0)) return n;
  BinomWords b(ctr, key);
  if (p > 0.5) {
    const double r = binomial_half(n, __dsub_rn(1.0, p), b);
    return r < 0.0 ? floor(__dmul_rn(__dadd_rn(n, 1.0), p)) : __dsub_rn(n, r);
  }
  const double r = binomial_half(n, p, b);
  return r < 0.0 ? floor(__dmul_rn(__dadd_rn(n, 1.0), p)) : r;
}

}  // namespace smc2
