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
#include <cooperative_groups.h>
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

// tanh x = sign(x) (1 - e) / (1 + e) with e = exp(-2|x|) in (0, 1]: the
// hardware exp2 (relative error about 2^-22) and a fast division.  The
// absolute error stays near 2^-22, far below the half step (2^-9 relative) of
// the bfloat16 the activations are rounded to.
__device__ __forceinline__ float tanh_act(float x) {
  const float e = __expf(-2.f * fabsf(x));
  return copysignf(__fdividef(1.f - e, 1.f + e), x);
}
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
  float b1[kMlpH], b2[kMlpH], w3f[kMlpH];  // w3f: the bfloat16 w3 as FP32
  float b3;
};

// Load the weights from the FP32 parameter vector (bf16-rounded copies).
// Every thread issues its float4 loads before the first shared-memory store
// (the vector is 16-byte aligned and every block of it starts at a multiple
// of four floats), so a CTA waits for about one L2 round trip; the
// transposes happen in the shared-memory stores.
__device__ void load_weights(MlpSmemWeights& W, const float* p, int D) {
  constexpr int kV = 8;  // float4 loads in flight per thread and round
  const int nt = blockDim.x, tid = threadIdx.x;
  for (int e = tid; e < kMlpH * kLd1; e += nt) W.w1t[e] = __float2bfloat16_rn(0.f);
  for (int e = tid; e < 8 * kLd; e += nt) W.w1b[e] = __float2bfloat16_rn(0.f);
  __syncthreads();
  const int n4 = (mlp_nparams(D) - 1) / 4;  // float4 blocks before b3
  const float4* p4 = reinterpret_cast<const float4*>(p);
  for (int base = tid; base < n4; base += kV * nt) {
    float4 v[kV];
#pragma unroll
    for (int u = 0; u < kV; ++u) {
      const int q4 = base + u * nt;
      v[u] = q4 < n4 ? p4[q4] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < kV; ++u) {
      const int q4 = base + u * nt;
      if (q4 >= n4) break;
      const float vals[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int q = 4 * q4 + c;
        const float f = vals[c];
        if (q < off_b1(D)) {  // W1[d][o]
          const int d = q / kMlpH, o = q % kMlpH;
          const bf16 h = __float2bfloat16_rn(f);
          W.w1t[o * kLd1 + d] = h;
          W.w1b[d * kLd + o] = h;
        } else if (q < off_W2(D)) {
          W.b1[q - off_b1(D)] = f;
        } else if (q < off_b2(D)) {  // W2[i][o]
          const int r = q - off_W2(D), i = r / kMlpH, o = r % kMlpH;
          const bf16 h = __float2bfloat16_rn(f);
          W.w2b[i * kLd + o] = h;
          W.w2t[o * kLd + i] = h;
        } else if (q < off_w3(D)) {
          W.b2[q - off_b2(D)] = f;
        } else {
          const bf16 h = __float2bfloat16_rn(f);  // weights are used rounded, biases exact
          W.w3b[q - off_w3(D)] = h;
          W.w3f[q - off_w3(D)] = __bfloat162float(h);
        }
      }
    }
  }
  if (tid == 0) W.b3 = p[off_b3(D)];
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
    F.h1[j][0] = tanh_act(c[0] + W.b1[col]);
    F.h1[j][1] = tanh_act(c[1] + W.b1[col + 1]);
    F.h1[j][2] = tanh_act(c[2] + W.b1[col]);
    F.h1[j][3] = tanh_act(c[3] + W.b1[col + 1]);
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
    F.h2[j][0] = tanh_act(c[0] + W.b2[col]);
    F.h2[j][1] = tanh_act(c[1] + W.b2[col + 1]);
    F.h2[j][2] = tanh_act(c[2] + W.b2[col]);
    F.h2[j][3] = tanh_act(c[3] + W.b2[col + 1]);
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

constexpr int kGradWarps = 8;                            // warps of a training-step CTA
constexpr int kGradTiles = 1;                            // 16-row tiles per warp
constexpr int kRowsGrad = 16 * kGradWarps * kGradTiles;  // rows per CTA
constexpr int kLdR = kRowsGrad + 8;                      // padded row of the staged [unit][row] tiles

struct MlpGradSmem {
  MlpSmemWeights W;
  bf16 h1T[kMlpH * kLdR];                   // [i][row] h1 of the CTA's rows (bf16)
  bf16 dz2T[kMlpH * kLdR];                  // [o][row] dz2 of the CTA's rows (bf16)
  float col[kGradWarps][3][kMlpH];          // per warp: db1, db2, dw3
  float w1g[kGradWarps][kMlpMaxD][kMlpH];   // per warp: dW1
  float sc[kGradWarps][2];                  // per warp: sum e^2, db3
};

size_t mlp_grad_smem_bytes() { return sizeof(MlpGradSmem); }

// Partial gradients of L = (1/R) sum (s(x_r) - y_r)^2: CTA c writes the
// gradient over its rows (and their sum of e^2) to part[c][0..P].
__global__ void __launch_bounds__(32 * kGradWarps)
    mlp_grad_kernel(const float* __restrict__ p, int D, const float* __restrict__ x,
                    const float* __restrict__ y, int R_imm, const int* R_dev, float* __restrict__ part,
                    int* step) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int R = R_dev ? *R_dev : R_imm;
  const int n_active = (R + kRowsGrad - 1) / kRowsGrad;
  const int P = mlp_nparams(D);
  MlpGradSmem& S = *reinterpret_cast<MlpGradSmem*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  if (step && blockIdx.x == 0 && threadIdx.x == 0) *step += 1;  // the Adam step this gradient feeds
  if ((int)blockIdx.x < n_active) {
    load_weights(S.W, p, D);
    for (int e = threadIdx.x; e < kGradWarps * 3 * kMlpH; e += blockDim.x) (&S.col[0][0][0])[e] = 0.f;
    for (int e = threadIdx.x; e < kGradWarps * kMlpMaxD * kMlpH; e += blockDim.x) (&S.w1g[0][0][0])[e] = 0.f;
    __syncthreads();
    float l_acc = 0.f, d3_acc = 0.f;
    for (int tile = 0; tile < kGradTiles; ++tile) {
      const int rl = (warp * kGradTiles + tile) * 16 + g;  // row within the CTA
      const int ra = blockIdx.x * kRowsGrad + rl, rb = ra + 8;
      const bool va = ra < R, vb = rb < R;
      float xa[4], xb[4], xfa[kMlpMaxD], xfb[kMlpMaxD];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int k = 2 * t + (e & 1) + (e >> 1) * 8;
        xa[e] = (va && k < D) ? x[(size_t)ra * D + k] : 0.f;
        xb[e] = (vb && k < D) ? x[(size_t)rb * D + k] : 0.f;
      }
#pragma unroll
      for (int d = 0; d < kMlpMaxD; ++d) {
        xfa[d] = (va && d < D) ? round_bf16(x[(size_t)ra * D + d]) : 0.f;
        xfb[d] = (vb && d < D) ? round_bf16(x[(size_t)rb * D + d]) : 0.f;
      }
      WarpForward F;
      warp_forward(S.W, xa, xb, F);
      const float ea = va ? F.s_lo - y[ra] : 0.f, eb = vb ? F.s_hi - y[rb] : 0.f;
      const float ga = 2.f * ea / (float)R, gb = 2.f * eb / (float)R;
      float dz2[8][4], dz1[8][4];
      warp_backward(S.W, F, ga, gb, dz2, dz1);
      // loss and db3: rows counted once, in the t = 0 lanes
      l_acc += warp_sum(t == 0 ? ea * ea + eb * eb : 0.f);
      d3_acc += warp_sum(t == 0 ? ga + gb : 0.f);
      // column sums over the tile's rows: db2, dw3, db1, dW1 (the warp owns its slots)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int c = 8 * j + 2 * t + e;
          const float v_db2 = sum_over_g(dz2[j][e] + dz2[j][2 + e]);
          const float v_dw3 = sum_over_g(round_bf16(F.h2[j][e]) * ga + round_bf16(F.h2[j][2 + e]) * gb);
          const float v_db1 = sum_over_g(dz1[j][e] + dz1[j][2 + e]);
          if (g == 0) {
            S.col[warp][1][c] += v_db2;
            S.col[warp][2][c] += v_dw3;
            S.col[warp][0][c] += v_db1;
          }
#pragma unroll
          for (int d = 0; d < kMlpMaxD; ++d) {
            if (d >= D) break;
            const float w = sum_over_g(xfa[d] * dz1[j][e] + xfb[d] * dz1[j][2 + e]);
            if (g == 0) S.w1g[warp][d][c] += w;
          }
        }
      }
      // stage h1 and dz2 transposed for dW2 = h1^T dz2 over the CTA's rows
#pragma unroll
      for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int c = 8 * j + 2 * t + e;
          S.h1T[c * kLdR + rl] = __float2bfloat16_rn(F.h1[j][e]);
          S.h1T[c * kLdR + rl + 8] = __float2bfloat16_rn(F.h1[j][2 + e]);
          S.dz2T[c * kLdR + rl] = __float2bfloat16_rn(dz2[j][e]);
          S.dz2T[c * kLdR + rl + 8] = __float2bfloat16_rn(dz2[j][2 + e]);
        }
    }
    if (lane == 0) {
      S.sc[warp][0] = l_acc;
      S.sc[warp][1] = d3_acc;
    }
    __syncthreads();
    float* out = part + (size_t)blockIdx.x * (P + 1);
    {  // dW2: warp (mt, nh) computes units i of m-tile mt against o of n-tiles 4 nh .. 4 nh + 3
      const int mt = warp & 3, nh = warp >> 2;
      float acc[4][4];
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll 4
      for (int kk = 0; kk < kRowsGrad / 16; ++kk) {
        const bf16* a = S.h1T + (16 * mt + g) * kLdR + 16 * kk + 2 * t;
        const uint32_t a0 = ld32(a), a1 = ld32(a + 8 * kLdR), a2 = ld32(a + 8), a3 = ld32(a + 8 * kLdR + 8);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const bf16* b = S.dz2T + (8 * (4 * nh + j) + g) * kLdR + 16 * kk + 2 * t;
          mma_bf16(acc[j], a0, a1, a2, a3, ld32(b), ld32(b + 8));
        }
      }
      float* gW2 = out + off_W2(D);
      const int i0 = 16 * mt + g;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int o = 8 * (4 * nh + j) + 2 * t;
        gW2[i0 * kMlpH + o] = acc[j][0];
        gW2[i0 * kMlpH + o + 1] = acc[j][1];
        gW2[(i0 + 8) * kMlpH + o] = acc[j][2];
        gW2[(i0 + 8) * kMlpH + o + 1] = acc[j][3];
      }
    }
    // the remaining partials: warp sums in warp order
    for (int e = threadIdx.x; e < kMlpH; e += blockDim.x) {
      float b1s = 0.f, b2s = 0.f, w3s = 0.f;
      for (int w = 0; w < kGradWarps; ++w) {
        b1s += S.col[w][0][e];
        b2s += S.col[w][1][e];
        w3s += S.col[w][2][e];
      }
      out[off_b1(D) + e] = b1s;
      out[off_b2(D) + e] = b2s;
      out[off_w3(D) + e] = w3s;
      for (int d = 0; d < D; ++d) {
        float s1 = 0.f;
        for (int w = 0; w < kGradWarps; ++w) s1 += S.w1g[w][d][e];
        out[d * kMlpH + e] = s1;
      }
    }
    if (threadIdx.x == 0) {
      float l2 = 0.f, b3s = 0.f;
      for (int w = 0; w < kGradWarps; ++w) {
        l2 += S.sc[w][0];
        b3s += S.sc[w][1];
      }
      out[off_b3(D)] = b3s;
      out[P] = l2;
    }
  }
}

// Sum of the partials over the CTAs in order, then the loss (and the gradient
// when grad != nullptr) and, with adam != 0, one Adam step on p (moments m, v;
// *step, already advanced by the gradient kernel, is the step number).
__global__ void __launch_bounds__(128)
    mlp_reduce_kernel(float* p, int D, const float* __restrict__ part, int R_imm, const int* R_dev,
                      float* grad, float* loss, int adam, float* m, float* v, int* step, float lr) {
  const int P = mlp_nparams(D);
  const int R = R_dev ? *R_dev : R_imm;
  const int n = (R + kRowsGrad - 1) / kRowsGrad;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q > P) return;
  float sum = 0.f;
  for (int c0 = 0; c0 < n; c0 += 16) {
    float tv[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) tv[u] = c0 + u < n ? __ldcg(part + (size_t)(c0 + u) * (P + 1) + q) : 0.f;
#pragma unroll
    for (int u = 0; u < 16; ++u) sum += tv[u];
  }
  if (q == P) {
    if (loss) loss[0] = R > 0 ? sum / (float)R : 0.f;
    return;
  }
  if (grad) grad[q] = sum;
  if (!adam) return;
  const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
  const float mq = beta1 * m[q] + (1.f - beta1) * sum;
  const float vq = beta2 * v[q] + (1.f - beta2) * sum * sum;
  m[q] = mq;
  v[q] = vq;
  const float t_step = (float)*step;
  const float bc1 = 1.f - powf(beta1, t_step), bc2 = 1.f - powf(beta2, t_step);
  p[q] -= lr * (mq / bc1) / (sqrtf(vq / bc2) + eps);
}

// ---------------------------------------------------------------------------
// training: all Adam steps of one call in one launch of a thread-block cluster
// ---------------------------------------------------------------------------
// The cluster's CTAs split the rows; each keeps the FP32 parameters, their
// bfloat16 copies, its rows and its partial gradient in shared memory, so the
// kernel body, the weights and the data stay on the SMs for every step.  Per
// step: partial gradients over the CTA's rows; cluster barrier; CTA c sums
// parameter slice c over the cluster's CTAs in rank order (distributed shared
// memory), takes the Adam step on it and writes the new values into every
// CTA's parameter copy; cluster barrier.
constexpr int kTrainWarps = 8;
constexpr int kMaxCluster = 16;                    // CTAs of the training cluster, at most
constexpr int kTrainRows = 16 * 2 * kTrainWarps;  // rows per chunk: two 16-row tiles per warp
constexpr int kLdT = kTrainRows + 8;              // padded row of the staged [unit][row] tiles
constexpr int kMlpPmax = kMlpMaxD * kMlpH + kMlpH * kMlpH + 3 * kMlpH + 1;

struct MlpTrainSmem {
  MlpSmemWeights W;
  bf16 h1T[kMlpH * kLdT];                   // [i][row] h1 of the chunk's rows (bf16)
  bf16 dz2T[kMlpH * kLdT];                  // [o][row] dz2 of the chunk's rows (bf16)
  bf16 dz1T[kMlpH * kLdT];                  // [o][row] dz1 of the chunk's rows (bf16)
  bf16 xT[16 * kLdT];                       // [d][row] inputs (bf16), row D all ones, rest zero
  float col[kTrainWarps][3][kMlpH];         // per warp: dw3 (slot 2)
  float sc[kTrainWarps][2];                 // per warp: sum e^2, db3
  float pf[kMlpPmax];                       // FP32 parameters
  float gp[kMlpPmax + 1];                   // partial gradient over the CTA's rows, then sum e^2
  float xs[kTrainRows * kMlpMaxD];          // the chunk's inputs
  float ys[kTrainRows];                     // and targets
  float wred[kTrainWarps][2 * kMlpMaxD + 1];  // block reductions: per-warp values
  float cred[2 * kMlpMaxD + 1];               // the CTA's totals, read by the cluster
};

// Totals over the cluster of NV per-thread values (sums, or maxima), in a
// fixed order: warp shuffles, the warps in order, then the CTAs in rank order
// through distributed shared memory.  Every thread of every CTA gets them.
template <int NV>
__device__ void cluster_totals(float (&v)[NV], MlpTrainSmem& S, cooperative_groups::cluster_group& cluster,
                               bool is_max) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    const float r = is_max ? warp_max(v[i]) : warp_sum(v[i]);
    if (lane == 0) S.wred[warp][i] = r;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    float r = S.wred[0][threadIdx.x];
    for (int w = 1; w < kTrainWarps; ++w) r = is_max ? fmaxf(r, S.wred[w][threadIdx.x]) : r + S.wred[w][threadIdx.x];
    S.cred[threadIdx.x] = r;
  }
  cluster.sync();
  const int C = (int)cluster.num_blocks();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    float u[kMaxCluster];
#pragma unroll
    for (int q = 0; q < kMaxCluster; ++q) u[q] = q < C ? cluster.map_shared_rank(S.cred, q)[i] : 0.f;
    float r = u[0];
#pragma unroll
    for (int q = 1; q < kMaxCluster; ++q)
      if (q < C) r = is_max ? fmaxf(r, u[q]) : r + u[q];
    v[i] = r;
  }
  cluster.sync();  // cred free again
}

// bfloat16 operand copies from the FP32 parameters in shared memory.
__device__ void refresh_weights(MlpSmemWeights& W, const float* pf, int D) {
  const int nt = blockDim.x, tid = threadIdx.x;
  for (int e = tid; e < kMlpH * kLd1; e += nt) W.w1t[e] = __float2bfloat16_rn(0.f);
  for (int e = tid; e < 8 * kLd; e += nt) W.w1b[e] = __float2bfloat16_rn(0.f);
  __syncthreads();
  for (int q = tid; q < D * kMlpH; q += nt) {
    const int d = q / kMlpH, o = q % kMlpH;
    const bf16 h = __float2bfloat16_rn(pf[q]);
    W.w1t[o * kLd1 + d] = h;
    W.w1b[d * kLd + o] = h;
  }
  const float* W2 = pf + off_W2(D);
  for (int q = tid; q < kMlpH * kMlpH; q += nt) {
    const int i = q / kMlpH, o = q % kMlpH;
    const bf16 h = __float2bfloat16_rn(W2[q]);
    W.w2b[i * kLd + o] = h;
    W.w2t[o * kLd + i] = h;
  }
  for (int e = tid; e < kMlpH; e += nt) {
    const bf16 h = __float2bfloat16_rn(pf[off_w3(D) + e]);
    W.w3b[e] = h;
    W.w3f[e] = __bfloat162float(h);
    W.b1[e] = pf[off_b1(D) + e];
    W.b2[e] = pf[off_b2(D) + e];
  }
  if (tid == 0) W.b3 = pf[off_b3(D)];
  __syncthreads();
}

// Ring standardisation (the training set of the learned proposal), when ring
// is non-null: z = max((log pi - max log pi) / tau, -8), tau = max(2, D), the
// target y = (z - mean z) / sd z; inputs standardised by the mean and sd of
// the rows above the clip (all rows if fewer than 2D + 2), moments taken about
// ring row 0; results into x, y (global) and *norm.  Then `steps` Adam steps.
struct MlpRing {
  const float* th;   // [rows][D]
  const float* lp;   // [rows]
  const int* rows;
  MlpNorm* norm;
};

__global__ void __launch_bounds__(32 * kTrainWarps)
    mlp_train_kernel(float* p, float* m, float* v, int* step, float* x, float* y, int R_imm, const int* R_dev,
                     float* loss, int D, int steps, float lr, MlpRing ring) {
  namespace cg = cooperative_groups;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MlpTrainSmem& S = *reinterpret_cast<MlpTrainSmem*>(smem_raw);
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks(), c = (int)cluster.block_rank();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  const int P = mlp_nparams(D);
  const int R = ring.th ? *ring.rows : (R_dev ? *R_dev : R_imm);
  const int per = (R + C - 1) / C, r0 = min(c * per, R), r1 = min(r0 + per, R);
  if (ring.th) {
    const float tau = D > 2 ? (float)D : 2.f, inv_tau = 1.f / tau;
    float mx[1] = {-INFINITY};
    for (int r = r0 + tid; r < r1; r += blockDim.x) {
      const float l = ring.lp[r];
      if (isfinite(l)) mx[0] = fmaxf(mx[0], l);
    }
    cluster_totals<1>(mx, S, cluster, true);
    const float ymax = mx[0], cut = ymax - 8.f * tau;
    float ref[kMlpMaxD], mu[kMlpMaxD], sd[kMlpMaxD];
#pragma unroll
    for (int d = 0; d < kMlpMaxD; ++d) ref[d] = (R > 0 && d < D) ? ring.th[d] : 0.f;
    for (int pass = 0; pass < 2; ++pass) {  // pass 0: rows above the clip; pass 1: every finite row
      float acc[2 * kMlpMaxD + 1];
#pragma unroll
      for (int i = 0; i < 2 * kMlpMaxD + 1; ++i) acc[i] = 0.f;
      for (int r = r0 + tid; r < r1; r += blockDim.x) {
        const float l = ring.lp[r];
        if (!isfinite(l) || (pass == 0 && l <= cut)) continue;
        acc[2 * kMlpMaxD] += 1.f;
#pragma unroll
        for (int d = 0; d < kMlpMaxD; ++d) {
          if (d >= D) break;
          const float cdev = ring.th[(size_t)r * D + d] - ref[d];
          acc[d] += cdev;
          acc[kMlpMaxD + d] += cdev * cdev;
        }
      }
      cluster_totals<2 * kMlpMaxD + 1>(acc, S, cluster, false);
      const float cnt = acc[2 * kMlpMaxD];
#pragma unroll
      for (int d = 0; d < kMlpMaxD; ++d) {
        const float m1 = cnt > 0.f ? acc[d] / cnt : 0.f;
        const float m2 = cnt > 0.f ? acc[kMlpMaxD + d] / cnt : 0.f;
        mu[d] = ref[d] + m1;
        sd[d] = fmaxf(cnt > 1.f ? sqrtf(fmaxf(m2 - m1 * m1, 0.f)) : 1.f, 1e-6f);
      }
      if (cnt >= 2.f * D + 2.f) break;
    }
    auto z_of = [&](float l) { return isfinite(l) ? fmaxf((l - ymax) * inv_tau, -8.f) : -8.f; };
    float zs[2] = {0.f, 0.f};
    for (int r = r0 + tid; r < r1; r += blockDim.x) {
      const float z = z_of(ring.lp[r]);
      zs[0] += z;
      zs[1] += z * z;
    }
    cluster_totals<2>(zs, S, cluster, false);
    const float zmean = R > 0 ? zs[0] / (float)R : 0.f;
    const float zvar = R > 0 ? fmaxf(zs[1] / (float)R - zmean * zmean, 0.f) : 0.f;
    const float zsd = zvar > 1e-8f ? sqrtf(zvar) : 1.f, inv_zsd = 1.f / zsd;
    float inv_sd[kMlpMaxD];
#pragma unroll
    for (int d = 0; d < kMlpMaxD; ++d) inv_sd[d] = 1.f / sd[d];
    for (int r = r0 + tid; r < r1; r += blockDim.x) {
      y[r] = (z_of(ring.lp[r]) - zmean) * inv_zsd;
#pragma unroll
      for (int d = 0; d < kMlpMaxD; ++d) {
        if (d >= D) break;
        x[(size_t)r * D + d] = (ring.th[(size_t)r * D + d] - mu[d]) * inv_sd[d];
      }
    }
    if (c == 0 && tid == 0) {
      MlpNorm& nm = *ring.norm;
      for (int d = 0; d < D; ++d) {
        nm.mu[d] = mu[d];
        nm.sd[d] = 1.0 / (double)inv_sd[d];
      }
      nm.ymax = ymax;
      nm.tau = tau;
      nm.zmean = zmean;
      nm.zsd = zsd;
      nm.rows = R;
      nm.var_y = zvar > 1e-8f ? 1.f : 0.f;
    }
    __syncthreads();  // this CTA's rows of x, y written before it reads them back
  }
  const bool cached = r1 - r0 <= kTrainRows;  // one chunk: rows stay in shared memory
  const int slice = (P + C - 1) / C, q0 = min(c * slice, P), q1 = min(q0 + slice, P);
  const int t0 = *step;
  for (int q = tid; q < P; q += blockDim.x) S.pf[q] = p[q];
  __syncthreads();  // every parameter loaded before any thread reads another's (also with no step)
  const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
  for (int it = 0; it < steps; ++it) {
    refresh_weights(S.W, S.pf, D);  // ends with a barrier
    for (int e = tid; e < kTrainWarps * 3 * kMlpH; e += blockDim.x) (&S.col[0][0][0])[e] = 0.f;
    float acc[4][4];  // dW2 tile of this warp: units i of m-tile (warp & 3), o of n-tiles 4 (warp >> 2) + j
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    // rows d < D: dW1[d][o]; row D: db1[o] (from [x^T; 1] dz1) and db2[o] (from 1^T dz2),
    // for the units o = 8 warp .. 8 warp + 7
    float w1acc[4] = {0.f, 0.f, 0.f, 0.f}, b2acc[4] = {0.f, 0.f, 0.f, 0.f};
    float l_acc = 0.f, d3_acc = 0.f;
    for (int base = r0; base < r1 || (base == r0 && r0 == r1); base += kTrainRows) {
      const int n = min(kTrainRows, r1 - base);
      if (!cached || it == 0) {
        for (int e = tid; e < kTrainRows * D; e += blockDim.x) S.xs[e] = e < n * D ? x[(size_t)base * D + e] : 0.f;
        for (int e = tid; e < kTrainRows; e += blockDim.x) S.ys[e] = e < n ? y[base + e] : 0.f;
        __syncthreads();
        for (int e = tid; e < 16 * kTrainRows; e += blockDim.x) {
          const int d = e / kTrainRows, r = e % kTrainRows;
          S.xT[d * kLdT + r] = __float2bfloat16_rn(d < D ? S.xs[r * D + d] : (d == D ? 1.f : 0.f));
        }
      }
      __syncthreads();
#pragma unroll 1
      for (int tile = 0; tile < 2; ++tile) {
        const int rl = (warp * 2 + tile) * 16 + g;  // row within the chunk
        const bool va = rl < n, vb = rl + 8 < n;
        float xa[4], xb[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int k = 2 * t + (e & 1) + (e >> 1) * 8;
          xa[e] = k < D ? S.xs[rl * D + k] : 0.f;
          xb[e] = k < D ? S.xs[(rl + 8) * D + k] : 0.f;
        }
        WarpForward F;
        warp_forward(S.W, xa, xb, F);
        const float ea = va ? F.s_lo - S.ys[rl] : 0.f, eb = vb ? F.s_hi - S.ys[rl + 8] : 0.f;
        const float ga = 2.f * ea / (float)R, gb = 2.f * eb / (float)R;
        float dz2[8][4], dz1[8][4];
        warp_backward(S.W, F, ga, gb, dz2, dz1);
        l_acc += warp_sum(t == 0 ? ea * ea + eb * eb : 0.f);
        d3_acc += warp_sum(t == 0 ? ga + gb : 0.f);
        // dw3 = sum_r h2_r ga_r (FP32 row signal): a shuffle reduction per column
#pragma unroll
        for (int j = 0; j < 8; ++j) {
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int cc = 8 * j + 2 * t + e;
            const float v_dw3 = sum_over_g(round_bf16(F.h2[j][e]) * ga + round_bf16(F.h2[j][2 + e]) * gb);
            if (g == 0) S.col[warp][2][cc] += v_dw3;
          }
        }
        // stage h1, dz2, dz1 transposed: the weight gradients are products over rows
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int cc = 8 * j + 2 * t + e;
            S.h1T[cc * kLdT + rl] = __float2bfloat16_rn(F.h1[j][e]);
            S.h1T[cc * kLdT + rl + 8] = __float2bfloat16_rn(F.h1[j][2 + e]);
            S.dz2T[cc * kLdT + rl] = __float2bfloat16_rn(dz2[j][e]);
            S.dz2T[cc * kLdT + rl + 8] = __float2bfloat16_rn(dz2[j][2 + e]);
            S.dz1T[cc * kLdT + rl] = __float2bfloat16_rn(dz1[j][e]);
            S.dz1T[cc * kLdT + rl + 8] = __float2bfloat16_rn(dz1[j][2 + e]);
          }
      }
      __syncthreads();
      {  // dW2 += h1^T dz2, [dW1; db1] += [x^T; 1] dz1, db2 += 1^T dz2 over the chunk's rows
        const int mt = warp & 3, nh = warp >> 2;
#pragma unroll 2
        for (int kk = 0; kk < kTrainRows / 16; ++kk) {
          const bf16* a = S.h1T + (16 * mt + g) * kLdT + 16 * kk + 2 * t;
          const uint32_t a0 = ld32(a), a1 = ld32(a + 8 * kLdT), a2 = ld32(a + 8), a3 = ld32(a + 8 * kLdT + 8);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const bf16* b = S.dz2T + (8 * (4 * nh + j) + g) * kLdT + 16 * kk + 2 * t;
            mma_bf16(acc[j], a0, a1, a2, a3, ld32(b), ld32(b + 8));
          }
          const bf16* xa = S.xT + g * kLdT + 16 * kk + 2 * t;
          const uint32_t x0 = ld32(xa), x1 = ld32(xa + 8 * kLdT), x2 = ld32(xa + 8), x3 = ld32(xa + 8 * kLdT + 8);
          const bf16* b1p = S.dz1T + (8 * warp + g) * kLdT + 16 * kk + 2 * t;
          mma_bf16(w1acc, x0, x1, x2, x3, ld32(b1p), ld32(b1p + 8));
          const bf16* b2p = S.dz2T + (8 * warp + g) * kLdT + 16 * kk + 2 * t;
          mma_bf16(b2acc, x0, x1, x2, x3, ld32(b2p), ld32(b2p + 8));
        }
      }
      __syncthreads();  // staging free for the next chunk
      if (r0 == r1) break;
    }
    // the CTA's partial gradient into gp
    {
      float* gW2 = S.gp + off_W2(D);
      const int mt = warp & 3, nh = warp >> 2, i0 = 16 * mt + g;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int o = 8 * (4 * nh + j) + 2 * t;
        gW2[i0 * kMlpH + o] = acc[j][0];
        gW2[i0 * kMlpH + o + 1] = acc[j][1];
        gW2[(i0 + 8) * kMlpH + o] = acc[j][2];
        gW2[(i0 + 8) * kMlpH + o + 1] = acc[j][3];
      }
    }
    if (lane == 0) {
      S.sc[warp][0] = l_acc;
      S.sc[warp][1] = d3_acc;
    }
    __syncthreads();
    {  // rows g (c0, c1) and g + 8 (c2, c3) of the [x^T; 1] products, units 8 warp + 2t, + 1
      const int o = 8 * warp + 2 * t;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int row = g + 8 * h;
        if (row < D) {
          S.gp[row * kMlpH + o] = w1acc[2 * h];
          S.gp[row * kMlpH + o + 1] = w1acc[2 * h + 1];
        } else if (row == D) {
          S.gp[off_b1(D) + o] = w1acc[2 * h];
          S.gp[off_b1(D) + o + 1] = w1acc[2 * h + 1];
          S.gp[off_b2(D) + o] = b2acc[2 * h];
          S.gp[off_b2(D) + o + 1] = b2acc[2 * h + 1];
        }
      }
    }
    for (int e = tid; e < kMlpH; e += blockDim.x) {
      float w3s = 0.f;
      for (int w = 0; w < kTrainWarps; ++w) w3s += S.col[w][2][e];
      S.gp[off_w3(D) + e] = w3s;
    }
    if (tid == 0) {
      float l2 = 0.f, b3s = 0.f;
      for (int w = 0; w < kTrainWarps; ++w) {
        l2 += S.sc[w][0];
        b3s += S.sc[w][1];
      }
      S.gp[off_b3(D)] = b3s;
      S.gp[P] = l2;
    }
    cluster.sync();  // every CTA's partial gradient complete
    const int tstep = t0 + it + 1;
    const float bc1 = 1.f - powf(beta1, (float)tstep), bc2 = 1.f - powf(beta2, (float)tstep);
    for (int q = q0 + tid; q < q1; q += blockDim.x) {
      float part[kMaxCluster];  // every rank's partial in flight at once, summed in rank order
#pragma unroll
      for (int r = 0; r < kMaxCluster; ++r) part[r] = r < C ? cluster.map_shared_rank(S.gp, r)[q] : 0.f;
      float sum = 0.f;
#pragma unroll
      for (int r = 0; r < kMaxCluster; ++r) sum += part[r];
      const float mq = beta1 * m[q] + (1.f - beta1) * sum;
      const float vq = beta2 * v[q] + (1.f - beta2) * sum * sum;
      m[q] = mq;
      v[q] = vq;
      const float pn = S.pf[q] - lr * (mq / bc1) / (sqrtf(vq / bc2) + eps);
      for (int r = 0; r < C; ++r) cluster.map_shared_rank(S.pf, r)[q] = pn;
    }
    if (c == 0 && tid == 0) {
      float l2 = 0.f;
      for (int r = 0; r < C; ++r) l2 += cluster.map_shared_rank(S.gp, r)[P];
      *loss = R > 0 ? l2 / (float)R : 0.f;
    }
    cluster.sync();  // every parameter copy updated; partial gradients free again
  }
  for (int q = q0 + tid; q < q1; q += blockDim.x) p[q] = S.pf[q];
  if (c == 0 && tid == 0) *step = t0 + steps;
}

// s and ds/dx of a warp's rows g and g+8: lane (g, t) returns dx of
// coordinates 2t and 2t+1 (rows g: dx_lo, g+8: dx_hi).
__device__ __forceinline__ void warp_input_grad(const MlpSmemWeights& W, const float* xa, const float* xb,
                                                WarpForward& F, float (&dx_lo)[2], float (&dx_hi)[2]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
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
  dx_lo[0] = c[0];
  dx_lo[1] = c[1];
  dx_hi[0] = c[2];
  dx_hi[1] = c[3];
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
  float dlo[2], dhi[2];
  warp_input_grad(W, xa, xb, F, dlo, dhi);
  if (t == 0) {
    if (va && s_out) s_out[ra] = F.s_lo;
    if (vb && s_out) s_out[rb] = F.s_hi;
  }
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int d = 2 * t + e;
    if (d < D) {
      if (va) dx[(size_t)ra * D + d] = dlo[e];
      if (vb) dx[(size_t)rb * D + d] = dhi[e];
    }
  }
}

// ---------------------------------------------------------------------------
// the learned proposal inside the sampler (dataset 0)
// ---------------------------------------------------------------------------

// Xavier-uniform weights and zero biases from the random stream (tag MLP_INIT);
// Adam moments and step cleared.
__global__ void mlp_init_kernel(MlpDev M, int D, uint64_t seed) {
  const int P = mlp_nparams(D);
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q == 0) *M.step = 0;
  if (q >= P) return;
  const float u = 2.f * uniform23<float>(philox4x32_10(make_uint4((uint32_t)q, 0u, 0u, TAG_MLP_INIT),
                                                       seed_key(seed)).x) - 1.f;
  float a = 0.f;
  if (q < off_b1(D))
    a = sqrtf(6.f / (float)(D + kMlpH));
  else if (q >= off_W2(D) && q < off_b2(D))
    a = sqrtf(6.f / (float)(2 * kMlpH));
  else if (q >= off_w3(D) && q < off_b3(D))
    a = sqrtf(6.f / (float)(kMlpH + 1));
  M.p[q] = a * u;
  M.p_use[q] = a * u;
  M.m[q] = 0.f;
  M.v[q] = 0.f;
}

// (theta_k, log pi^(theta_k)) of this iteration's proposals into ring slot (k-1) mod W.
__global__ void mlp_append_kernel(OuterParams P) {
  const DSDev& S = P.ds[0];
  const int k = *P.k_done + 1, N = S.N, D = P.D;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const size_t row = (size_t)((k - 1) % P.mlp.W) * N + i;
  for (int d = 0; d < D; ++d) P.mlp.ring_th[row * D + d] = (float)S.thB[(size_t)d * N + i];
  P.mlp.ring_lp[row] = (float)(S.lpB[i] + S.llB[i]);
  if (i == 0) *P.mlp.ring_rows = min(k, P.mlp.W) * N;
}

// The trained state becomes the one the proposal reads.
__global__ void mlp_publish_kernel(MlpDev M, int n_par) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n_par) M.p_use[q] = M.p[q];
  if (q == 0) {
    *M.norm_use = *M.norm;
    *M.loss_use = *M.loss;
  }
}

// Score of the surrogate at the parents theta_{k-1}: through the input and
// target standardisations, d log pi^ / d theta_d = tau zsd (ds/dx)_d / sd_d.
// Decides whether iteration k proposes with it: from k = 3 on, while the
// published network explains half the variance of its targets and the
// population covariance has a usable Cholesky factor.
__global__ void __launch_bounds__(32 * kMlpWarps) mlp_score_kernel(OuterParams P) {
  __shared__ MlpSmemWeights W;
  const DSDev& S = P.ds[0];
  const int k = *P.k_done + 1, N = S.N, D = P.D;
  const MlpNorm& nm = *P.mlp.norm_use;
  const float loss = *P.mlp.loss_use;
  const bool use = k >= 3 && isfinite(loss) && nm.var_y > 0.f && loss < 0.5f * nm.var_y && S.cur->pop_ok;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S.cur->mlp_used = use ? 1 : 0;
    S.cur->mlp_loss = (double)loss;
  }
  if (!use) return;
  load_weights(W, P.mlp.p_use, D);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int ra = blockIdx.x * kRowsCta + warp * 16 + g, rb = ra + 8;
  const bool va = ra < N, vb = rb < N;
  float xa[4], xb[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int d = 2 * t + (e & 1) + (e >> 1) * 8;
    xa[e] = (va && d < D) ? (float)((S.thA[(size_t)d * N + ra] - nm.mu[d]) / nm.sd[d]) : 0.f;
    xb[e] = (vb && d < D) ? (float)((S.thA[(size_t)d * N + rb] - nm.mu[d]) / nm.sd[d]) : 0.f;
  }
  WarpForward F;
  float dlo[2], dhi[2];
  warp_input_grad(W, xa, xb, F, dlo, dhi);
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int d = 2 * t + e;
    if (d >= D) continue;
    const double scale = nm.tau * nm.zsd / nm.sd[d];
    if (va) P.mlp.score[(size_t)d * N + ra] = scale * dlo[e];
    if (vb) P.mlp.score[(size_t)d * N + rb] = scale * dhi[e];
  }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
int mlp_param_count(int D) { return mlp_nparams(D); }
int mlp_grad_ctas(int R) { return (R + kRowsGrad - 1) / kRowsGrad; }

// One gradient (and optionally Adam) step over R rows (R_dev, when given, holds
// the row count; R bounds it and sizes the grid).
cudaError_t mlp_step_launch(float* p, int D, const float* x, const float* y, int R, const int* R_dev,
                            float* part, float* grad, float* loss, int adam, float* m, float* v, int* step,
                            float lr, cudaStream_t s) {
  const size_t smem = sizeof(MlpGradSmem);
  cudaError_t e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  mlp_grad_kernel<<<mlp_grad_ctas(R), 32 * kGradWarps, smem, s>>>(p, D, x, y, R, R_dev, part,
                                                                  adam ? step : nullptr);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int P = mlp_nparams(D);
  mlp_reduce_kernel<<<(P + 1 + 127) / 128, 128, 0, s>>>(p, D, part, R, R_dev, grad, loss, adam, m, v, step,
                                                         lr);
  return cudaGetLastError();
}

size_t mlp_train_smem_bytes() { return sizeof(MlpTrainSmem); }

cudaError_t mlp_train_footprint(int* ctas, int* threads, int* regs, size_t* smem) {
  cudaFuncAttributes a{};
  const cudaError_t e = cudaFuncGetAttributes(&a, mlp_train_kernel);
  if (e != cudaSuccess) return e;
  *ctas = mlp_train_cluster_size();
  *threads = 32 * kTrainWarps;
  *regs = a.numRegs;
  *smem = sizeof(MlpTrainSmem) + a.sharedSizeBytes;
  return cudaSuccess;
}

// Largest cluster (16, 8, 4, 2 or 1 CTAs) that the device can co-schedule with
// this kernel's shared memory.
int mlp_train_cluster_size() {
  static int cached = 0;
  if (cached) return cached;
  const size_t smem = sizeof(MlpTrainSmem);
  if (cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    return 0;
  for (int C = 16; C >= 1; C >>= 1) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(32 * kTrainWarps);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, mlp_train_kernel, &cfg) == cudaSuccess && n > 0) {
      cached = C;
      return C;
    }
    cudaGetLastError();
  }
  return 0;
}

cudaError_t mlp_train_steps_launch(float* p, float* m, float* v, int* step, float* x, float* y, int R,
                                   const int* R_dev, float* loss, int D, int steps, float lr, cudaStream_t s,
                                   const MlpDev* ring_of) {
  const int C = mlp_train_cluster_size();
  if (C < 1) return cudaErrorInvalidConfiguration;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(32 * kTrainWarps);
  cfg.dynamicSmemBytes = sizeof(MlpTrainSmem);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  MlpRing ring{};
  if (ring_of) {
    ring.th = ring_of->ring_th;
    ring.lp = ring_of->ring_lp;
    ring.rows = ring_of->ring_rows;
    ring.norm = ring_of->norm;
  }
  return cudaLaunchKernelEx(&cfg, mlp_train_kernel, p, m, v, step, x, y, R, R_dev, loss, D, steps, lr, ring);
}

// The training call on caller buffers: the ring (th, lp) of *rows_dev rows is
// standardised into x, y and *norm, then `steps` Adam steps continue (p, m, v,
// *step); the same kernel and cluster shape as the sampler's own call.
cudaError_t mlp_train_ring_launch(float* p, float* m, float* v, int* step, const float* th, const float* lp,
                                  const int* rows_dev, int R, MlpNorm* norm, float* x, float* y, float* loss,
                                  int D, int steps, float lr, cudaStream_t s) {
  MlpDev M{};
  M.ring_th = const_cast<float*>(th);
  M.ring_lp = const_cast<float*>(lp);
  M.ring_rows = const_cast<int*>(rows_dev);
  M.norm = norm;
  return mlp_train_steps_launch(p, m, v, step, x, y, R, nullptr, loss, D, steps, lr, s, &M);
}

// The standardisation and training loss as FP64 values: mu[D], sd[D], tau, zmean,
// zsd, var_y, loss, ymax.
__global__ void mlp_norm_export_kernel(const MlpNorm* nm, const float* loss, int D, double* out) {
  const int e = threadIdx.x;
  if (e < D) {
    out[e] = nm->mu[e];
    out[D + e] = nm->sd[e];
  }
  if (e == 0) {
    out[2 * D] = nm->tau;
    out[2 * D + 1] = nm->zmean;
    out[2 * D + 2] = nm->zsd;
    out[2 * D + 3] = nm->var_y;
    out[2 * D + 4] = *loss;
    out[2 * D + 5] = nm->ymax;
  }
}

cudaError_t mlp_norm_export_launch(const MlpNorm* nm, const float* loss, int D, double* out, cudaStream_t s) {
  mlp_norm_export_kernel<<<1, 32, 0, s>>>(nm, loss, D, out);
  return cudaGetLastError();
}

cudaError_t mlp_init_launch(const MlpDev& M, int D, uint64_t seed, cudaStream_t s) {
  const int P = mlp_nparams(D);
  mlp_init_kernel<<<(P + 255) / 256, 256, 0, s>>>(M, D, seed);
  return cudaGetLastError();
}

// Store this iteration's rows (before resampling moves the population).
cudaError_t mlp_append_launch(const OuterParams& P, int N, cudaStream_t s) {
  mlp_append_kernel<<<(N + 127) / 128, 128, 0, s>>>(P);
  return cudaGetLastError();
}

// Standardise the ring and take `steps` Adam steps on it: one cluster launch.
cudaError_t mlp_train_launch(const OuterParams& P, int steps, float lr, cudaStream_t s) {
  const MlpDev& M = P.mlp;
  return mlp_train_steps_launch(M.p, M.m, M.v, M.step, M.xs, M.ys, M.W * P.ds_N0, nullptr, M.loss, P.D, steps, lr,
                                s, &M);
}

cudaError_t mlp_publish_launch(const OuterParams& P, cudaStream_t s) {
  const int n_par = mlp_nparams(P.D);
  mlp_publish_kernel<<<(n_par + 255) / 256, 256, 0, s>>>(P.mlp, n_par);
  return cudaGetLastError();
}

cudaError_t mlp_score_launch(const OuterParams& P, int N, cudaStream_t s) {
  mlp_score_kernel<<<(N + kRowsCta - 1) / kRowsCta, 32 * kMlpWarps, 0, s>>>(P);
  return cudaGetLastError();
}

cudaError_t mlp_input_grad_launch(const float* p, int D, const float* x, int R, float* s_out, float* dx,
                                  cudaStream_t s) {
  mlp_input_grad_kernel<<<(R + kRowsCta - 1) / kRowsCta, 32 * kMlpWarps, 0, s>>>(p, D, x, R, s_out, dx);
  return cudaGetLastError();
}

}  // namespace smc2
