// common.cuh -- device building blocks shared by the SMC^2 kernels.
//
// Counter-based random numbers (Philox4x32-10 of Salmon, Moraes, Dror and
// Shaw, SC'11), uniforms that float and double hold exactly, Box-Muller
// normals, warp reductions and scans, and the device status word.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace smc2 {

// Random-stream tags (bits 0..3 of counter word 3; the iteration k fills bits 4..31).
enum : uint32_t {
  TAG_THETA_INIT = 1,  // c0 = coordinate group, c1 = 0
  TAG_PROPOSE = 2,     // c0 = coordinate group, c1 = 0
  TAG_OUTER_RES = 3,   // c0 = c1 = 0, c2 = dataset << 20; word 0
  TAG_PF_INIT = 4,     // c0 = particle, c1 = 0; normal 0
  TAG_PF_PROP = 5,     // c0 = particle, c1 = (t-1) >> 2; normal (t-1) & 3
  TAG_PF_RES = 6,      // c0 = 0, c1 = t; word 0
  TAG_MLP_INIT = 7,    // c0 = parameter index; word 0 (surrogate network initial weights)
  TAG_PF_MULTI = 8,    // c0 = slot >> 2, c1 = t; word slot & 3 (multinomial PF resampling)
  TAG_PF_BINOM = 9,    // c0 = particle + 4096 call, c1 = t (the SIR flows' shared word stream)
};

// Device status bits (sticky; mapped to smc2_status codes on the host).
enum : int { ST_NONFINITE = 1 };

enum : int { MODEL_LG = 0, MODEL_SEIR = 1, MODEL_SIR = 2 };
enum : int { LK_FORWARD = 0, LK_GAUSS = 1 };

constexpr int kMaxD = 8;
constexpr double kLog2Pi = 1.8378770664093454835606594728112;
constexpr double kLn2 = 0.69314718055994530941723212145818;

__device__ __forceinline__ uint32_t counter_c2(uint32_t i, uint32_t ds_hi) { return i | ds_hi; }
__device__ __forceinline__ uint32_t counter_c3(uint32_t tag, uint32_t k) { return tag | (k << 4); }

// Philox4x32-10: ten rounds; each multiplies words 0 and 2 by the round
// multipliers (keeping both halves of the products) and mixes in the key,
// which advances by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 key) {
  const uint32_t mult0 = 0xD2511F53u, mult1 = 0xCD9E8D57u;
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t k0 = key.x + (uint32_t)round * 0x9E3779B9u;
    const uint32_t k1 = key.y + (uint32_t)round * 0xBB67AE85u;
    const uint64_t p0 = (uint64_t)mult0 * c.x, p1 = (uint64_t)mult1 * c.z;  // one wide multiply each
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// The same generator with its round keys given: rk[2r] = key.x + r 0x9E3779B9,
// rk[2r + 1] = key.y + r 0xBB67AE85 (philox_round_keys), so that a kernel can keep
// them in its parameter block and fold them into the XORs as constants.
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const uint32_t (&rk)[20]) {
  const uint32_t mult0 = 0xD2511F53u, mult1 = 0xCD9E8D57u;
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint64_t p0 = (uint64_t)mult0 * c.x, p1 = (uint64_t)mult1 * c.z;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c = make_uint4(hi1 ^ c.y ^ rk[2 * round], lo1, hi0 ^ c.w ^ rk[2 * round + 1], lo0);
  }
  return c;
}

__host__ __device__ inline void philox_round_keys(uint64_t seed, uint32_t rk[20]) {
  const uint32_t k0 = (uint32_t)(seed & 0xffffffffull), k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    rk[2 * r] = k0 + (uint32_t)r * 0x9E3779B9u;
    rk[2 * r + 1] = k1 + (uint32_t)r * 0xBB67AE85u;
  }
}

__device__ __forceinline__ uint2 seed_key(uint64_t seed) {
  return make_uint2((uint32_t)(seed & 0xffffffffull), (uint32_t)(seed >> 32));
}

// u = ((w >> 9) + 1/2) 2^-23, built from the exponent bits of 1.0 so that no
// integer-to-float conversion is needed: (1 + k 2^-23) - (1 - 2^-24) is exact.
template <typename R>
__device__ __forceinline__ R uniform23(uint32_t w);
template <>
__device__ __forceinline__ float uniform23<float>(uint32_t w) {
  return __uint_as_float(0x3f800000u | (w >> 9)) - (1.0f - 0x1p-24f);
}
template <>
__device__ __forceinline__ double uniform23<double>(uint32_t w) {
  const uint64_t bits = 0x3ff0000000000000ull | ((uint64_t)(w >> 9) << 29);
  return __longlong_as_double((long long)bits) - (1.0 - 0x1p-24);
}

template <typename R>
__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, R& z0, R& z1);
// FP32: hardware approximations (lg2, rsqrt, sin, cos; absolute error about
// 2^-21 on [-pi, pi]).  The angle is taken as 2 pi (u_b - 1/2), inside that
// range, and the pair is negated back: (cos 2 pi u_b, sin 2 pi u_b).
template <>
__device__ __forceinline__ void box_muller<float>(uint32_t wa, uint32_t wb, float& z0, float& z1) {
  const float ua = uniform23<float>(wa), ub = uniform23<float>(wb);
  const float e = -2.0f * __logf(ua);
  const float r = e * rsqrtf(e);
  float s, c;
  __sincosf(6.28318530717958647692f * (ub - 0.5f), &s, &c);
  z0 = -r * c;
  z1 = -r * s;
}
template <>
__device__ __forceinline__ void box_muller<double>(uint32_t wa, uint32_t wb, double& z0, double& z1) {
  const double ua = uniform23<double>(wa), ub = uniform23<double>(wb);
  const double r = sqrt(-2.0 * log(ua));
  double s, c;
  sincospi(2.0 * ub, &s, &c);
  z0 = r * c;
  z1 = r * s;
}

// Four normals from one Philox call: (w0, w1) and (w2, w3) are two Box-Muller pairs.
template <typename R>
__device__ __forceinline__ void normals4(uint4 c, uint2 key, R z[4]) {
  const uint4 w = philox4x32_10(c, key);
  box_muller<R>(w.x, w.y, z[0], z[1]);
  box_muller<R>(w.z, w.w, z[2], z[3]);
}

__device__ __forceinline__ int fixed_point_bits(int n) {
  const int c = (n <= 1) ? 0 : 32 - __clz(n - 1);  // ceil(log2 n)
  const int b = 63 - c;
  return b < 52 ? b : 52;
}

// floor((2^33 j + 2U + 1) S / (n 2^33)): the threshold of slot j.
__device__ __forceinline__ uint64_t slot_threshold(uint32_t j, uint32_t U, uint64_t S, int n,
                                                   int log2n) {
  const unsigned __int128 num = (((unsigned __int128)j << 33) + 2ull * U + 1ull) * S;
  if (log2n >= 0) return (uint64_t)(num >> (33 + log2n));
  return (uint64_t)(num / ((unsigned __int128)n << 33));
}

template <typename R>
__device__ __forceinline__ R warp_max(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ uint64_t warp_incl_scan_u64(uint64_t v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

__device__ __forceinline__ void named_barrier(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ void raise_status(int* status, int bits) {
  if (status) atomicOr(status, bits);
}

}  // namespace smc2
