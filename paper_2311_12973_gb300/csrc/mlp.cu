// mlp.cu -- the surrogate network of the learned proposal on tensor cores.
//
// s(x) = w3 . tanh(W2^T tanh(W1^T x + b1) + b2) + b3, hidden width 64, with
// bfloat16 operands and FP32 accumulation (mma.sync m16n8k16).  A warp owns
// 16 rows; the accumulator fragments of one layer are re-packed in registers
// as the operand fragments of the next.  Training computes per-CTA partial
// gradients of the mean squared error (the weight gradient dW2 = h1^T dz2 is
// a second product over the CTA's 64 rows, staged transposed in shared
// memory), then one kernel sums them in a fixed order and takes an Adam step.
// The proposal uses the gradient with respect to the input.
#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"

namespace smc2 {

using bf16 = __nv_bfloat16;

constexpr int kRowsCta = 16 * kMlpWarps;  // rows per CTA
constexpr int kLd = kMlpH + 8;             // padded row of 64-wide bf16 tiles (conflict-free fragments)
constexpr int kLd1 = 24;                   // padded row of the 16-wide W1 tile

__host__ __device__ inline int mlp_nparams(int D) { return D * kMlpH + kMlpH * kMlpH + 3 * kMlpH + 1; }
__host__ __device__ inline int off_b1(int D) { return D * kMlpH; }
__host__ __device__ inline int off_W2(int D) { return D * kMlpH + kMlpH; }
__host__ __device__ inline int off_b2(int D) { return off_W2(D) + kMlpH * kMlpH; }
__host__ __device__ inline int off_w3(int D) { return off_b2(D) + kMlpH; }
__host__ __device__ inline int off_b3(int D) { return off_w3(D) + kMlpH; }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ float round_bf16(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
__device__ __forceinline__ uint32_t ld32(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }

// D = A B + D for a 16x16 (row) by 16x8 (column) bf16 product, FP32 accumulators.
__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Shared-memory copy of the operands, padded rows:
//   w1t [64][kLd1]  W1 transposed (k = input coordinate, zero beyond D)
//   w1b [8][kLd]    W1 input-major (rows beyond D zero)
//   w2t [64][kLd]   W2 transposed (output-major)
//   w2b [64][kLd]   W2 input-major
//   w3b [64], b1, b2, w3 in FP32
struct MlpSmemWeights {
  bf16 w1t[kMlpH * kLd1];
  bf16 w1b[8 * kLd];
  bf16 w2t[kMlpH * kLd];
  bf16 w2b[kMlpH * kLd];
  bf16 w3b[kMlpH];
  float b1[kMlpH], b2[kMlpH], w3f[kMlpH];
  float b3;
};

// Load the weights from the FP32 parameter vector (bf16-rounded copies).
__device__ void load_weights(MlpSmemWeights& W, const float* p, int D) {
  for (int e = threadIdx.x; e < kMlpH * kLd1; e += blockDim.x) {
    const int o = e / kLd1, d = e % kLd1;
    W.w1t[e] = __float2bfloat16_rn(d < D ? p[d * kMlpH + o] : 0.f);
  }
  for (int e = threadIdx.x; e < 8 * kLd; e += blockDim.x) {
    const int d = e / kLd, o = e % kLd;
    W.w1b[e] = __float2bfloat16_rn(d < D && o < kMlpH ? p[d * kMlpH + o] : 0.f);
  }
  const float* W2 = p + off_W2(D);
  for (int e = threadIdx.x; e < kMlpH * kLd; e += blockDim.x) {
    const int r = e / kLd, q = e % kLd;
    W.w2t[e] = __float2bfloat16_rn(q < kMlpH ? W2[q * kMlpH + r] : 0.f);  // [o][i]
    W.w2b[e] = __float2bfloat16_rn(q < kMlpH ? W2[r * kMlpH + q] : 0.f);  // [i][o]
  }
  for (int e = threadIdx.x; e < kMlpH; e += blockDim.x) {
    W.w3b[e] = __float2bfloat16_rn(p[off_w3(D) + e]);
    W.w3f[e] = p[off_w3(D) + e];
    W.b1[e] = p[off_b1(D) + e];
    W.b2[e] = p[off_b2(D) + e];
  }
  if (threadIdx.x == 0) W.b3 = p[off_b3(D)];
}

// Forward pass of one warp's 16 rows.  Lane (g, t) = (lane / 4, lane % 4)
// holds columns 8j + 2t + {0,1} of rows g and g+8 of every 16x8 tile j.
struct WarpForward {
  float h1[8][4], h2[8][4];  // tanh activations (FP32)
  float s_lo, s_hi;          // s of rows g and g+8 (every lane of the quad)
};

__device__ __forceinline__ void warp_forward(const MlpSmemWeights& W, const float* xa, const float* xb,
                                             WarpForward& F) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const uint32_t a0 = pack_bf16(xa[0], xa[1]), a1 = pack_bf16(xb[0], xb[1]);
  const uint32_t a2 = pack_bf16(xa[2], xa[3]), a3 = pack_bf16(xb[2], xb[3]);
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    const bf16* w = W.w1t + (8 * j + g) * kLd1 + 2 * t;
    mma_bf16(c, a0, a1, a2, a3, ld32(w), ld32(w + 8));
    const int col = 8 * j + 2 * t;
    F.h1[j][0] = tanhf(c[0] + W.b1[col]);
    F.h1[j][1] = tanhf(c[1] + W.b1[col + 1]);
    F.h1[j][2] = tanhf(c[2] + W.b1[col]);
    F.h1[j][3] = tanhf(c[3] + W.b1[col + 1]);
  }
  uint32_t hA[4][4];
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    hA[kk][0] = pack_bf16(F.h1[2 * kk][0], F.h1[2 * kk][1]);
    hA[kk][1] = pack_bf16(F.h1[2 * kk][2], F.h1[2 * kk][3]);
    hA[kk][2] = pack_bf16(F.h1[2 * kk + 1][0], F.h1[2 * kk + 1][1]);
    hA[kk][3] = pack_bf16(F.h1[2 * kk + 1][2], F.h1[2 * kk + 1][3]);
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const bf16* w = W.w2t + (8 * j + g) * kLd + 16 * kk + 2 * t;
      mma_bf16(c, hA[kk][0], hA[kk][1], hA[kk][2], hA[kk][3], ld32(w), ld32(w + 8));
    }
    const int col = 8 * j + 2 * t;
    F.h2[j][0] = tanhf(c[0] + W.b2[col]);
    F.h2[j][1] = tanhf(c[1] + W.b2[col + 1]);
    F.h2[j][2] = tanhf(c[2] + W.b2[col]);
    F.h2[j][3] = tanhf(c[3] + W.b2[col + 1]);
  }
  float c3[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    const uint32_t b0 = g == 0 ? ld32(W.w3b + 16 * kk + 2 * t) : 0u;
    const uint32_t b1 = g == 0 ? ld32(W.w3b + 16 * kk + 8 + 2 * t) : 0u;
    mma_bf16(c3, pack_bf16(F.h2[2 * kk][0], F.h2[2 * kk][1]), pack_bf16(F.h2[2 * kk][2], F.h2[2 * kk][3]),
             pack_bf16(F.h2[2 * kk + 1][0], F.h2[2 * kk + 1][1]),
             pack_bf16(F.h2[2 * kk + 1][2], F.h2[2 * kk + 1][3]), b0, b1);
  }
  // column 0 of the output tile sits in the lanes with t = 0
  F.s_lo = __shfl_sync(0xffffffffu, c3[0], lane & ~3) + W.b3;
  F.s_hi = __shfl_sync(0xffffffffu, c3[2], lane & ~3) + W.b3;
}

// Back-propagation of the row signals (ga, gb) to dz1 (bf16-rounded values),
// optionally keeping dz2 (bf16-rounded) for the weight gradients.
__device__ __forceinline__ void warp_backward(const MlpSmemWeights& W, const WarpForward& F, float ga,
                                              float gb, float (&dz2)[8][4], float (&dz1)[8][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int col = 8 * j + 2 * t;
    dz2[j][0] = round_bf16(ga * W.w3f[col] * (1.f - F.h2[j][0] * F.h2[j][0]));
    dz2[j][1] = round_bf16(ga * W.w3f[col + 1] * (1.f - F.h2[j][1] * F.h2[j][1]));
    dz2[j][2] = round_bf16(gb * W.w3f[col] * (1.f - F.h2[j][2] * F.h2[j][2]));
    dz2[j][3] = round_bf16(gb * W.w3f[col + 1] * (1.f - F.h2[j][3] * F.h2[j][3]));
  }
  uint32_t zA[4][4];
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    zA[kk][0] = pack_bf16(dz2[2 * kk][0], dz2[2 * kk][1]);
    zA[kk][1] = pack_bf16(dz2[2 * kk][2], dz2[2 * kk][3]);
    zA[kk][2] = pack_bf16(dz2[2 * kk + 1][0], dz2[2 * kk + 1][1]);
    zA[kk][3] = pack_bf16(dz2[2 * kk + 1][2], dz2[2 * kk + 1][3]);
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {  // dh1 = dz2 W2^T, tile j over the input units
    float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const bf16* w = W.w2b + (8 * j + g) * kLd + 16 * kk + 2 * t;
      mma_bf16(c, zA[kk][0], zA[kk][1], zA[kk][2], zA[kk][3], ld32(w), ld32(w + 8));
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) dz1[j][e] = round_bf16(c[e] * (1.f - F.h1[j][e] * F.h1[j][e]));
  }
}

// Sum over the eight row groups g of a warp (lanes with equal t).
__device__ __forceinline__ float sum_over_g(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 8);
  v += __shfl_xor_sync(0xffffffffu, v, 16);
  return v;
}

struct MlpGradSmem {
  MlpSmemWeights W;
  bf16 h1T[kMlpH * kLd];   // [i][row] h1 of the CTA's rows (bf16)
  bf16 dz2T[kMlpH * kLd];  // [o][row] dz2 of the CTA's rows (bf16)
  float col[kMlpWarps][3][kMlpH];        // per warp: db1, db2, dw3
  float w1g[kMlpWarps][kMlpMaxD][kMlpH]; // per warp: dW1
  float sc[kMlpWarps][2];                // per warp: sum e^2, db3
};

size_t mlp_grad_smem_bytes() { return sizeof(MlpGradSmem); }

// Per-CTA partial gradients of L = (1/R) sum (s(x_r) - y_r)^2 into
// part[blockIdx.x][0..P) and sum e^2 into part[blockIdx.x][P].
__global__ void __launch_bounds__(32 * kMlpWarps)
    mlp_grad_kernel(const float* __restrict__ p, int D, const float* __restrict__ x,
                    const float* __restrict__ y, int R, float* __restrict__ part, int* step) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MlpGradSmem& S = *reinterpret_cast<MlpGradSmem*>(smem_raw);
  load_weights(S.W, p, D);
  if (step && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(step, 1);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int ra = blockIdx.x * kRowsCta + warp * 16 + g, rb = ra + 8;
  const bool va = ra < R, vb = rb < R;
  float xa[4], xb[4];  // input columns 2t, 2t+1 (a0/a1) and 2t+8, 2t+9 (a2/a3)
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int k = 2 * t + (e & 1) + (e >> 1) * 8;
    xa[e] = (va && k < D) ? x[(size_t)ra * D + k] : 0.f;
    xb[e] = (vb && k < D) ? x[(size_t)rb * D + k] : 0.f;
  }
  WarpForward F;
  warp_forward(S.W, xa, xb, F);
  const float ea = va ? F.s_lo - y[ra] : 0.f, eb = vb ? F.s_hi - y[rb] : 0.f;
  const float ga = 2.f * ea / (float)R, gb = 2.f * eb / (float)R;
  float dz2[8][4], dz1[8][4];
  warp_backward(S.W, F, ga, gb, dz2, dz1);
  // loss and db3: rows counted once, in the t = 0 lanes
  const float l = warp_sum(t == 0 ? ea * ea + eb * eb : 0.f);
  const float d3 = warp_sum(t == 0 ? ga + gb : 0.f);
  if (lane == 0) {
    S.sc[warp][0] = l;
    S.sc[warp][1] = d3;
  }
  // column sums over the warp's rows: db2, dw3, db1, dW1
#pragma unroll
  for (int j = 0; j < 8; ++j) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int col = 8 * j + 2 * t + e;
      const float v_db2 = sum_over_g(dz2[j][e] + dz2[j][2 + e]);
      const float v_dw3 = sum_over_g(round_bf16(F.h2[j][e]) * ga + round_bf16(F.h2[j][2 + e]) * gb);
      const float v_db1 = sum_over_g(dz1[j][e] + dz1[j][2 + e]);
      if (g == 0) {
        S.col[warp][1][col] = v_db2;
        S.col[warp][2][col] = v_dw3;
        S.col[warp][0][col] = v_db1;
      }
      for (int d = 0; d < D; ++d) {
        const float xad = va ? round_bf16(x[(size_t)ra * D + d]) : 0.f;
        const float xbd = vb ? round_bf16(x[(size_t)rb * D + d]) : 0.f;
        const float v = sum_over_g(xad * dz1[j][e] + xbd * dz1[j][2 + e]);
        if (g == 0) S.w1g[warp][d][col] = v;
      }
    }
  }
  // stage h1 and dz2 transposed for dW2 = h1^T dz2 over the CTA's rows
  const int rl = warp * 16 + g;
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int c = 8 * j + 2 * t + e;
      S.h1T[c * kLd + rl] = __float2bfloat16_rn(F.h1[j][e]);
      S.h1T[c * kLd + rl + 8] = __float2bfloat16_rn(F.h1[j][2 + e]);
      S.dz2T[c * kLd + rl] = __float2bfloat16_rn(dz2[j][e]);
      S.dz2T[c * kLd + rl + 8] = __float2bfloat16_rn(dz2[j][2 + e]);
    }
  __syncthreads();
  float* out = part + (size_t)blockIdx.x * (mlp_nparams(D) + 1);
  {
    float acc[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {  // k = the CTA's rows 16kk..16kk+15
      const bf16* a = S.h1T + (16 * warp + g) * kLd + 16 * kk + 2 * t;
      const uint32_t a0 = ld32(a), a1 = ld32(a + 8 * kLd), a2 = ld32(a + 8), a3 = ld32(a + 8 * kLd + 8);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const bf16* b = S.dz2T + (8 * j + g) * kLd + 16 * kk + 2 * t;
        mma_bf16(acc[j], a0, a1, a2, a3, ld32(b), ld32(b + 8));
      }
    }
    float* gW2 = out + off_W2(D);
    const int i0 = 16 * warp + g;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int o = 8 * j + 2 * t;
      gW2[i0 * kMlpH + o] = acc[j][0];
      gW2[i0 * kMlpH + o + 1] = acc[j][1];
      gW2[(i0 + 8) * kMlpH + o] = acc[j][2];
      gW2[(i0 + 8) * kMlpH + o + 1] = acc[j][3];
    }
  }
  // the remaining partials: warp sums in warp order
  for (int e = threadIdx.x; e < kMlpH; e += blockDim.x) {
    float b1s = 0.f, b2s = 0.f, w3s = 0.f;
    for (int w = 0; w < kMlpWarps; ++w) {
      b1s += S.col[w][0][e];
      b2s += S.col[w][1][e];
      w3s += S.col[w][2][e];
    }
    out[off_b1(D) + e] = b1s;
    out[off_b2(D) + e] = b2s;
    out[off_w3(D) + e] = w3s;
    for (int d = 0; d < D; ++d) {
      float s1 = 0.f;
      for (int w = 0; w < kMlpWarps; ++w) s1 += S.w1g[w][d][e];
      out[d * kMlpH + e] = s1;
    }
  }
  if (threadIdx.x == 0) {
    float l2 = 0.f, b3s = 0.f;
    for (int w = 0; w < kMlpWarps; ++w) {
      l2 += S.sc[w][0];
      b3s += S.sc[w][1];
    }
    out[off_b3(D)] = b3s;
    out[mlp_nparams(D)] = l2;
  }
}

// Gradient (and mean loss) from the partials, summed over CTAs in order; with
// adam != 0 also one Adam step on p (moments m, v; step count *step).
__global__ void mlp_reduce_kernel(float* p, int D, const float* part, int n_cta, int R, float* grad,
                                  float* loss, int adam, float* m, float* v, const int* step,
                                  float lr, float beta1, float beta2, float eps) {
  const int P = mlp_nparams(D);
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q > P) return;
  float s = 0.f;
  for (int c = 0; c < n_cta; ++c) s += part[(size_t)c * (P + 1) + q];
  if (q == P) {
    if (loss) loss[0] = s / (float)R;
    return;
  }
  if (grad) grad[q] = s;
  if (!adam) return;
  const int tstep = *step;
  const float mq = beta1 * m[q] + (1.f - beta1) * s;
  const float vq = beta2 * v[q] + (1.f - beta2) * s * s;
  m[q] = mq;
  v[q] = vq;
  const float mh = mq / (1.f - powf(beta1, (float)tstep));
  const float vh = vq / (1.f - powf(beta2, (float)tstep));
  p[q] -= lr * mh / (sqrtf(vh) + eps);
}

// s(x) and ds/dx of R rows.
__global__ void __launch_bounds__(32 * kMlpWarps)
    mlp_input_grad_kernel(const float* __restrict__ p, int D, const float* __restrict__ x, int R,
                          float* __restrict__ s_out, float* __restrict__ dx) {
  __shared__ MlpSmemWeights W;
  load_weights(W, p, D);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int ra = blockIdx.x * kRowsCta + warp * 16 + g, rb = ra + 8;
  const bool va = ra < R, vb = rb < R;
  float xa[4], xb[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int k = 2 * t + (e & 1) + (e >> 1) * 8;
    xa[e] = (va && k < D) ? x[(size_t)ra * D + k] : 0.f;
    xb[e] = (vb && k < D) ? x[(size_t)rb * D + k] : 0.f;
  }
  WarpForward F;
  warp_forward(W, xa, xb, F);
  float dz2[8][4], dz1[8][4];
  warp_backward(W, F, 1.f, 1.f, dz2, dz1);
  // dx = dz1 W1^T: k over the hidden units, n over the input coordinates (padded to 8)
  float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    const bf16* w = W.w1b + g * kLd + 16 * kk + 2 * t;
    mma_bf16(c, pack_bf16(dz1[2 * kk][0], dz1[2 * kk][1]), pack_bf16(dz1[2 * kk][2], dz1[2 * kk][3]),
             pack_bf16(dz1[2 * kk + 1][0], dz1[2 * kk + 1][1]),
             pack_bf16(dz1[2 * kk + 1][2], dz1[2 * kk + 1][3]), ld32(w), ld32(w + 8));
  }
  if (t == 0) {
    if (va && s_out) s_out[ra] = F.s_lo;
    if (vb && s_out) s_out[rb] = F.s_hi;
  }
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int d = 2 * t + e;
    if (d < D) {
      if (va) dx[(size_t)ra * D + d] = c[e];
      if (vb) dx[(size_t)rb * D + d] = c[2 + e];
    }
  }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
int mlp_param_count(int D) { return mlp_nparams(D); }
int mlp_grad_ctas(int R) { return (R + kRowsCta - 1) / kRowsCta; }

cudaError_t mlp_grad_launch(const float* p, int D, const float* x, const float* y, int R, float* part,
                            int* step, cudaStream_t s) {
  const size_t smem = sizeof(MlpGradSmem);
  cudaError_t e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  mlp_grad_kernel<<<mlp_grad_ctas(R), 32 * kMlpWarps, smem, s>>>(p, D, x, y, R, part, step);
  return cudaGetLastError();
}

cudaError_t mlp_reduce_launch(float* p, int D, const float* part, int n_cta, int R, float* grad,
                              float* loss, int adam, float* m, float* v, const int* step, float lr,
                              cudaStream_t s) {
  const int P = mlp_nparams(D);
  mlp_reduce_kernel<<<(P + 1 + 255) / 256, 256, 0, s>>>(p, D, part, n_cta, R, grad, loss, adam, m, v,
                                                       step, lr, 0.9f, 0.999f, 1e-8f);
  return cudaGetLastError();
}

cudaError_t mlp_input_grad_launch(const float* p, int D, const float* x, int R, float* s_out, float* dx,
                                  cudaStream_t s) {
  mlp_input_grad_kernel<<<(R + kRowsCta - 1) / kRowsCta, 32 * kMlpWarps, 0, s>>>(p, D, x, R, s_out, dx);
  return cudaGetLastError();
}

}  // namespace smc2
