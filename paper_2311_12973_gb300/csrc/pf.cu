// pf.cu -- bootstrap particle filter kernel (Sec. II of the paper).
//
// One group of threads runs one filter over all T steps: each thread holds
// PPT consecutive particles in registers.  Per step:
//   1. propagate with the state equation (Eq. 1) using counter-based normals;
//   2. log-weight with the observation density (Eq. 2; bootstrap form of Eq. 5);
//   3. group max of the log-weights (warp shuffles, one barrier);
//   4. quantise q_j = floor(exp(l_j - max) 2^B), warp-local inclusive scan of q
//      in registers + shuffles, warp totals and particle states to shared memory
//      (second barrier);
//   5. log-likelihood increment log((1/M) sum_j w_j) = max + log(S 2^-B) - log M
//      from the exact integer total S (Eq. 8, with the mean-weight reset of
//      Eq. 13 every step);
//   6. systematic resampling (Eqs. 26-27): slot j takes the first particle whose
//      cumulative weight exceeds floor((j + u) S / M), found by a search over
//      the warp totals and then a binary search inside one warp's prefix;
//      the slot's new state is gathered from shared memory.
// A work unit is `count` filters of one job (dataset); units are taken from an
// atomic queue so that jobs of uneven length balance over the SMs.
#include <cfloat>
#include <cmath>

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

__host__ __device__ inline int group_threads_for(int ppt, int M) {
  const int t = (M + ppt - 1) / ppt;
  return (t + 31) & ~31;
}

__host__ __device__ inline size_t region_bytes(int Mp, int nw, int ns, int rsize) {
  size_t b = (size_t)Mp * 8 + (size_t)ns * Mp * rsize + (size_t)nw * 8 + (size_t)nw * rsize + 8;
  return (b + 15) & ~(size_t)15;
}

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
  __device__ __forceinline__ R day(R* x) const {
    const R beta = exp(x[3]);
    R S = x[0], E = x[1], I = x[2], lam = (R)0;
    for (int s = 0; s < n_sub; ++s) {
      const R infection = beta * S * I * inv_npop;
      const R onset = kappa * E;
      const R recovery = gamma * I;
      lam += dt * onset;
      S = fmax(S - dt * infection, (R)0);
      E = fmax(E + dt * (infection - onset), (R)0);
      I = fmax(I + dt * (onset - recovery), (R)0);
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

template <typename R, int MODEL, int PPT>
__device__ __forceinline__ void run_filter(const PFJob& J, const PFModel& mdl, int i, int g, int lt,
                                           int gt, unsigned char* region, uint2 key, uint32_t k) {
  constexpr int NS = ModelDims<MODEL>::NS;
  constexpr int D = ModelDims<MODEL>::D;
  using R4 = typename R4Of<R>::type;
  const int M = J.M, T = J.T;
  const int Mp = gt * PPT;
  const int nw = gt >> 5;
  const int lane = lt & 31, warp = lt >> 5;
  const int seg = 32 * PPT;  // particles per warp

  uint64_t* P = reinterpret_cast<uint64_t*>(region);   // [Mp] warp-local inclusive prefix of q
  R* X = reinterpret_cast<R*>(P + Mp);                  // [NS][Mp] particle states
  uint64_t* wsum = reinterpret_cast<uint64_t*>(X + (size_t)NS * Mp);  // [nw] warp totals
  R* wmax = reinterpret_cast<R*>(wsum + nw);            // [nw] warp maxima
  uint32_t* sU = reinterpret_cast<uint32_t*>(wmax + nw);  // [2] resampling words, by step parity

  auto group_sync = [&]() {
    if (nw == 1)
      __syncwarp();
    else
      named_barrier(1 + g, gt);
  };

  double th[D];
#pragma unroll
  for (int d = 0; d < D; ++d) th[d] = J.theta[(size_t)d * J.ld + i];
  FilterParams<R, MODEL> fp;
  fp.load(th, mdl);

  const uint32_t c2 = counter_c2((uint32_t)i, J.c2hi);
  const uint32_t c3prop = counter_c3(TAG_PF_PROP, k);
  const uint32_t c3res = counter_c3(TAG_PF_RES, k);
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

  double loglik = 0.0;
  bool dead = false;
  for (int t0 = 1; t0 <= T && !dead; t0 += 4) {
    R zc[PPT][4];
#pragma unroll
    for (int r = 0; r < PPT; ++r)
      normals4<R>(make_uint4((uint32_t)(lt * PPT + r), (uint32_t)((t0 - 1) >> 2), c2, c3prop), key,
                  zc[r]);
#pragma unroll
    for (int tm = 0; tm < 4; ++tm) {
      const int t = t0 + tm;
      if (t > T || dead) break;
      if (lt == 0 && t < T) sU[t & 1] = philox4x32_10(make_uint4(0u, (uint32_t)t, c2, c3res), key).x;
      const R4 ob = obs[t - 1];
      R ell[PPT];
      R lmax = neg_inf<R>();
#pragma unroll
      for (int r = 0; r < PPT; ++r) {
        fp.propagate(x[r], zc[r][tm]);
        R l;
        if constexpr (MODEL == MODEL_LG) {
          l = fp.log_obs(x[r], ob);
        } else {
          const R lam = fp.day(x[r]);
          l = fp.log_pois(lam, ob);
        }
        if (isnan(l) || lt * PPT + r >= M) l = neg_inf<R>();
        ell[r] = l;
        lmax = fmax(lmax, l);
      }
      // (3) group maximum
      lmax = warp_max(lmax);
      if (nw > 1 && lane == 0) wmax[warp] = lmax;
      group_sync();
      if (nw > 1) {
        lmax = wmax[0];
        for (int w = 1; w < nw; ++w) lmax = fmax(lmax, wmax[w]);
      }
      const R m = lmax;
      if (!(m > neg_inf<R>())) {  // every weight vanished: the estimate is zero
        dead = true;
        loglik = -HUGE_VAL;
        if (lt == 0 && J.delta)
          for (int s = t; s <= T; ++s) J.delta[(size_t)i * T + (s - 1)] = -HUGE_VAL;
        break;
      }
      // (4) quantise and scan
      uint64_t run = 0, c[PPT];
#pragma unroll
      for (int r = 0; r < PPT; ++r) {
        const uint64_t qv = (ell[r] > neg_inf<R>()) ? to_u64_rz(exp(ell[r] - m) * scaleB) : 0ull;
        run += qv;
        c[r] = run;
      }
      const uint64_t incl = warp_incl_scan_u64(run, lane);
      const uint64_t excl = incl - run;
#pragma unroll
      for (int r = 0; r < PPT; ++r) {
        P[lt * PPT + r] = excl + c[r];
#pragma unroll
        for (int s = 0; s < NS; ++s) X[s * Mp + lt * PPT + r] = x[r][s];
      }
      if (lane == 31) wsum[warp] = incl;
      group_sync();
      uint64_t S = 0;
      for (int w = 0; w < nw; ++w) S += wsum[w];
      // (5) log-likelihood increment
      if (lt == 0) {
        const double delta = (double)m + log((double)S) + log_norm;
        loglik += delta;
        if (J.delta) J.delta[(size_t)i * T + (t - 1)] = delta;
      }
      // (6) systematic resampling and ancestor gather
      if (t < T) {
        const uint32_t U = sU[t & 1];
#pragma unroll
        for (int r = 0; r < PPT; ++r) {
          const int j = lt * PPT + r;
          if (j < M) {
            const uint64_t tau = slot_threshold((uint32_t)j, U, S, M, log2M);
            uint64_t base = 0;
            int w = 0;
            while (w < nw - 1 && base + wsum[w] <= tau) {
              base += wsum[w];
              ++w;
            }
            const uint64_t tl = tau - base;
            int lo = w * seg, hi = lo + seg - 1;
            while (lo < hi) {
              const int mid = (lo + hi) >> 1;
              if (P[mid] > tl)
                hi = mid;
              else
                lo = mid + 1;
            }
#pragma unroll
            for (int s = 0; s < NS; ++s) x[r][s] = X[s * Mp + lo];
            if (J.anc) J.anc[((size_t)i * (T - 1) + (t - 1)) * M + j] = lo;
          }
        }
      }
    }
  }
  if (lt == 0) J.loglik[i] = loglik;
}

template <typename R, int MODEL, int PPT>
__global__ void __launch_bounds__(kPfMaxBlock) pf_kernel(PFLaunch L) {
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
    const size_t rb = region_bytes(gt * PPT, gt >> 5, NS, (int)sizeof(R));
    if (g < count && (g + 1) * gt <= (int)blockDim.x)
      run_filter<R, MODEL, PPT>(J, L.mdl, first + g, g, lt, gt, smem + g * rb, key, k);
    if (!L.wu_counter) __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

int pf_group_threads(int ppt, int M) { return group_threads_for(ppt, M); }

size_t pf_smem_bytes(int precision, int model, int ppt, int block, int M) {
  const int gt = group_threads_for(ppt, M);
  const int fpc = block / gt;
  const int ns = model == MODEL_LG ? 1 : 4;
  const int rs = precision == SMC2_PREC_FP64 ? 8 : 4;
  return (size_t)fpc * region_bytes(gt * ppt, gt >> 5, ns, rs);
}

template <typename R, int MODEL, int PPT>
static const void* kernel_ptr() {
  return reinterpret_cast<const void*>(&pf_kernel<R, MODEL, PPT>);
}

static const void* select_kernel(int precision, int model, int ppt) {
#define SMC2_PF_CASE(R, MODEL)                 \
  switch (ppt) {                               \
    case 1: return kernel_ptr<R, MODEL, 1>();  \
    case 2: return kernel_ptr<R, MODEL, 2>();  \
    case 4: return kernel_ptr<R, MODEL, 4>();  \
    case 8: return kernel_ptr<R, MODEL, 8>();  \
    default: return nullptr;                   \
  }
  if (precision == SMC2_PREC_FP64) {
    if (model == MODEL_LG) SMC2_PF_CASE(double, MODEL_LG)
    SMC2_PF_CASE(double, MODEL_SEIR)
  }
  if (model == MODEL_LG) SMC2_PF_CASE(float, MODEL_LG)
  SMC2_PF_CASE(float, MODEL_SEIR)
#undef SMC2_PF_CASE
}

cudaError_t pf_configure(int precision, int model, int ppt, size_t smem) {
  const void* f = select_kernel(precision, model, ppt);
  if (!f) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

int pf_occupancy(int precision, int model, int ppt, int block, size_t smem) {
  const void* f = select_kernel(precision, model, ppt);
  int n = 0;
  if (!f || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, block, smem) != cudaSuccess) return 0;
  return n;
}

cudaError_t pf_launch(int precision, int model, int ppt, int grid, int block, size_t smem,
                      const PFLaunch& L, cudaStream_t s) {
  const void* f = select_kernel(precision, model, ppt);
  if (!f) return cudaErrorInvalidValue;
  void* args[] = {const_cast<PFLaunch*>(&L)};
  return cudaLaunchKernel(f, dim3(grid), dim3(block), args, smem, s);
}

}  // namespace smc2
