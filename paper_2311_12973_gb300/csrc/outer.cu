// outer.cu -- the SMC^2 outer step (Sec. IV of the paper), in FP64.
//
// One iteration is five launches (four over a (block, dataset) grid):
//   propose   k = 1: theta ~ q_1 = prior (Eq. 16); k > 1: Gaussian random walk
//             (Eqs. 18-19) and, for the Gaussian L-kernel, per-block weighted
//             moments of the pairs (theta_{k-1}, theta_k).
//   lkfit     one warp per dataset totals the moments, fits the joint Gaussian
//             and conditions it (Eqs. 32-35); it runs beside the particle filter.
//   weights   Eq. (17) at k = 1, Eq. (20) after; per-block max / sums; the last
//             block forms log sum w, log sum w^2, ESS (Eqs. 24-25), the estimate
//             (Eq. 21), the evidence and the recycling sums (Eqs. 23, 29).
//   quantise  q_i = floor(exp(log w_i - max) 2^B) when ESS < ess_frac N.
//   resample  every block scans all q into shared memory and redistributes its
//             own slots (Eq. 27 counts, Algorithm 1 order), or copies when no
//             resampling was triggered; weights reset to the mean (Sec. IV-B).
// The "last block" steps use an atomic ticket; their sums run in block order,
// so results do not depend on scheduling.
#include <cfloat>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace smc2 {

constexpr int kResWarps = kResBlock / 32;
static_assert(kOuterBlock == 32, "the per-sample outer kernels are one warp per block");

template <int D>
__device__ __forceinline__ double log_prior(const OuterParams& P, const double* th) {
  double lp = 0.0;
  if (P.prior_kind == 1) {  // independent uniforms on [lo, hi]
#pragma unroll
    for (int d = 0; d < D; ++d) {
      if (!(th[d] >= P.prior_lo[d] && th[d] <= P.prior_hi[d])) return -HUGE_VAL;
      lp -= P.log_prior_width[d];
    }
    return lp;
  }
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const double r = (th[d] - P.prior_mean[d]) * P.inv_prior_sd[d];
    lp += -0.5 * kLog2Pi - P.log_prior_sd[d] - 0.5 * r * r;
  }
  return lp;
}

// log N(x; mean, rw_scale^2 I)
template <int D>
__device__ __forceinline__ double rw_logpdf(const OuterParams& P, const double* x, const double* mean) {
  double ss = 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const double r = (x[d] - mean[d]) * P.inv_rw;
    ss += r * r;
  }
  return -0.5 * D * kLog2Pi - D * P.log_rw - 0.5 * ss;
}

// log N(a; mu_a + A (b - mu_b), Lc Lc^T)
template <int D>
__device__ __forceinline__ double lk_logpdf(const LKParams& L, const double* a, const double* b) {
  double r[D], v[D];
#pragma unroll
  for (int p = 0; p < D; ++p) {
    double m = L.mu[p];
#pragma unroll
    for (int s = 0; s < D; ++s) m += L.A[p * D + s] * (b[s] - L.mu[D + s]);
    r[p] = a[p] - m;
  }
  double ss = 0.0;
#pragma unroll
  for (int p = 0; p < D; ++p) {
    double s = r[p];
#pragma unroll
    for (int l = 0; l < p; ++l) s -= L.Lc[p * D + l] * v[l];
    v[p] = s * L.Lc_inv[p];
    ss += v[p] * v[p];
  }
  return -0.5 * D * kLog2Pi - 0.5 * L.logdet - 0.5 * ss;
}

// Warp-cooperative Cholesky of the n x n matrix a (shared, row-major) into l
// (shared), with the pivot floor 1e-12 (a_jj + mean_j^2): column by column,
// lane 0 forms the pivot and its reciprocal, lanes r > j update row r.
// Returns 0 on success (same value in every lane).
__device__ int warp_chol(int n, const double* a, const double* mean, double* l, double* inv_diag) {
  const int lane = threadIdx.x & 31;
  for (int e = lane; e < n * n; e += 32) l[e] = 0.0;
  __syncwarp();
  int ok = 1;
  for (int j = 0; j < n; ++j) {
    if (lane == 0) {
      double sj = a[j * n + j];
      for (int p = 0; p < j; ++p) sj -= l[j * n + p] * l[j * n + p];
      const double floor_j = 1e-12 * (a[j * n + j] + mean[j] * mean[j]);
      ok = (sj > floor_j) && isfinite(sj);
      const double d = ok ? sqrt(sj) : 1.0;
      l[j * n + j] = d;
      inv_diag[j] = 1.0 / d;
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) return -1;
    __syncwarp();
    const int r = j + 1 + lane;
    if (r < n) {
      double v = a[r * n + j];
      for (int p = 0; p < j; ++p) v -= l[r * n + p] * l[j * n + p];
      l[r * n + j] = v * inv_diag[j];
    }
    __syncwarp();
  }
  return 0;
}

// Moment slots: 0 = sum w; 1..2D = sum w z_r; then sum w z_r z_s for r <= s.
__device__ __forceinline__ int n_moments(int D) { return 1 + 2 * D + D * (2 * D + 1); }

struct FitScratch {
  double sig[4 * kMaxD * kMaxD], mu[2 * kMaxD], m1[2 * kMaxD];
  double saa[kMaxD * kMaxD], sab[kMaxD * kMaxD], sbb[kMaxD * kMaxD], lb[kMaxD * kMaxD];
  double sc[kMaxD * kMaxD], inv_b[kMaxD], tmp[kMaxD * kMaxD];
};

// Gaussian fit of (theta_{k-1}, theta_k) from the weighted moment totals and
// its conditional a | b (Eqs. 32-35 under the reading in the oracle), by one warp.
__device__ void lk_fit_warp(int D, const double* tot, const double* shift, FitScratch& F,
                            LKParams* out) {
  const int lane = threadIdx.x & 31, D2 = 2 * D;
  const double W = tot[0];
  const double invW = 1.0 / W;
  for (int r = lane; r < D2; r += 32) {
    F.m1[r] = tot[1 + r] * invW;
    F.mu[r] = shift[r] + F.m1[r];
  }
  __syncwarp();
  for (int e = lane; e < D2 * D2; e += 32) {
    const int r = e / D2, q = e % D2;
    const int lo = r < q ? r : q, hi = r < q ? q : r;
    const int slot = 1 + D2 + lo * D2 - lo * (lo - 1) / 2 + (hi - lo);
    F.sig[e] = tot[slot] * invW - F.m1[r] * F.m1[q];
  }
  __syncwarp();
  for (int e = lane; e < D * D; e += 32) {
    const int r = e / D, q = e % D;
    F.saa[e] = F.sig[r * D2 + q];
    F.sab[e] = F.sig[r * D2 + (D + q)];
    F.sbb[e] = F.sig[(D + r) * D2 + (D + q)];
  }
  for (int r = lane; r < D2; r += 32) out->mu[r] = F.mu[r];
  if (lane == 0) out->fallback = 1;
  __syncwarp();
  if (warp_chol(D, F.sbb, F.mu + D, F.lb, F.inv_b) != 0) return;
  // A = S_ab S_bb^{-1}: lane c solves S_bb x = (row c of S_ab)^T; A's row c = x
  if (lane < D) {
    const int c = lane;
    double* t = F.tmp + c * D;
    for (int r = 0; r < D; ++r) {
      double v = F.sab[c * D + r];
      for (int p = 0; p < r; ++p) v -= F.lb[r * D + p] * t[p];
      t[r] = v * F.inv_b[r];
    }
    for (int r = D - 1; r >= 0; --r) {
      double v = t[r];
      for (int p = r + 1; p < D; ++p) v -= F.lb[p * D + r] * out->A[c * D + p];
      out->A[c * D + r] = v * F.inv_b[r];
    }
  }
  __syncwarp();
  for (int e = lane; e < D * D; e += 32) {
    const int r = e / D, q = e % D;
    double v = F.saa[e];
    for (int p = 0; p < D; ++p) v -= out->A[r * D + p] * F.sab[q * D + p];
    F.sc[e] = v;
  }
  __syncwarp();
  if (warp_chol(D, F.sc, F.mu, F.tmp, out->Lc_inv) != 0) return;
  for (int e = lane; e < D * D; e += 32) out->Lc[e] = F.tmp[e];
  double ld = lane < D ? 2.0 * log(F.tmp[lane * D + lane]) : 0.0;
  for (int o = 16; o > 0; o >>= 1) ld += __shfl_xor_sync(0xffffffffu, ld, o);
  if (lane == 0) {
    out->logdet = ld;
    out->fallback = 0;
  }
}

// ---------------------------------------------------------------------------
// propose (+ L-kernel fit)
// ---------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(kOuterBlock) propose_kernel(OuterParams P) {
  const DSDev& S = P.ds[blockIdx.y];
  if ((int)blockIdx.x >= S.nblk) return;
  __shared__ double zs[kOuterBlock][2 * kMaxD];
  __shared__ double ws[kOuterBlock];
  const int N = S.N, lane = threadIdx.x;
  const int i = blockIdx.x * kOuterBlock + lane;
  const uint32_t k = (uint32_t)(*P.k_done + 1);
  const bool act = i < N;
  const uint2 key = seed_key(P.seed);
  double a[D], b[D];
  // random walk (Eqs. 18-19); learned proposal: theta_k = a + h L (w + z) with
  // L L^T the population covariance and w = h/2 L^T grad log pi^(a), clipped
  // at +-3, so that the drift is h^2/2 Sigma grad log pi^ in whitened units
  const bool mlp = k > 1 && P.mlp.on && S.cur->mlp_used;
  if (act) {
    const uint32_t c2 = counter_c2((uint32_t)i, S.c2hi);
    double z[D];
#pragma unroll
    for (int g = 0; g * 4 < D; ++g) {
      double z4[4];
      normals4<double>(make_uint4((uint32_t)g, 0u, c2,
                                  counter_c3(k == 1 ? TAG_THETA_INIT : TAG_PROPOSE, k)),
                       key, z4);
#pragma unroll
      for (int r = 0; r < 4 && 4 * g + r < D; ++r) z[4 * g + r] = z4[r];
    }
    if (k == 1 && P.prior_kind == 1) {
      // uniform prior: theta_d = lo + (hi - lo) u from the THETA_INIT words, u = (2w + 1) 2^-33
#pragma unroll
      for (int g = 0; g * 4 < D; ++g) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)g, 0u, c2, counter_c3(TAG_THETA_INIT, k)), key);
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int r = 0; r < 4 && 4 * g + r < D; ++r) {
          const double u = ((double)ws[r] * 2.0 + 1.0) * 0x1p-33;
          const int d = 4 * g + r;
          b[d] = __dadd_rn(P.prior_lo[d], __dmul_rn(__dsub_rn(P.prior_hi[d], P.prior_lo[d]), u));
        }
      }
    } else if (k == 1) {
#pragma unroll
      for (int d = 0; d < D; ++d) b[d] = P.prior_mean[d] + P.prior_sd[d] * z[d];
    } else {
#pragma unroll
      for (int d = 0; d < D; ++d) a[d] = S.thA[(size_t)d * N + i];
      if (!mlp) {
#pragma unroll
        for (int d = 0; d < D; ++d) b[d] = a[d] + P.rw_scale * z[d];
      } else {
        const double* L = S.cur->Lpop;
        const double h = P.mlp.h;
        double g[D], u[D];
#pragma unroll
        for (int d = 0; d < D; ++d) g[d] = P.mlp.score[(size_t)d * N + i];
#pragma unroll
        for (int r = 0; r < D; ++r) {
          double w = 0.0;
#pragma unroll
          for (int d = r; d < D; ++d) w += L[d * kMaxD + r] * g[d];
          w = fmin(fmax(0.5 * h * w, -3.0), 3.0);
          u[r] = w + z[r];
        }
#pragma unroll
        for (int r = 0; r < D; ++r) {
          double v = 0.0;
#pragma unroll
          for (int c = 0; c <= r; ++c) v += L[r * kMaxD + c] * u[c];
          b[r] = a[r] + h * v;
        }
      }
    }
#pragma unroll
    for (int d = 0; d < D; ++d) S.thB[(size_t)d * N + i] = b[d];
    const double lp = log_prior<D>(P, b);
    S.lpB[i] = lp;
    if (k == 1) {
      S.logq[i] = lp;
    } else if (mlp) {
      // N(b; a + h L w, h^2 L L^T) at b = a + h L (w + z)
      double lq = -0.5 * D * kLog2Pi - D * log(P.mlp.h);
#pragma unroll
      for (int d = 0; d < D; ++d) lq += -log(S.cur->Lpop[d * kMaxD + d]) - 0.5 * z[d] * z[d];
      S.logq[i] = lq;
    } else {
      S.logq[i] = rw_logpdf<D>(P, b, a);
    }
  }
  if (k == 1 || P.lkernel != LK_GAUSS) return;

  // weighted moments of z = (theta_{k-1}, theta_k) - shift over this block's samples;
  // the shift (sample 0's parent) keeps the one-pass covariance well conditioned
  double shift[D];
#pragma unroll
  for (int d = 0; d < D; ++d) shift[d] = S.thA[(size_t)d * N];
  ws[lane] = act ? exp(S.logw[i] - S.cur->m_par) : 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    zs[lane][d] = act ? a[d] - shift[d] : 0.0;
    zs[lane][D + d] = act ? b[d] - shift[d] : 0.0;
  }
  __syncwarp();
  const int NM = n_moments(D);
  for (int mo = lane; mo < NM; mo += 32) {
    int r = -1, q = -1;
    if (mo >= 1 && mo <= 2 * D) {
      r = mo - 1;
    } else if (mo > 2 * D) {
      int slot = mo - 1 - 2 * D;
      r = 0;
      while (slot >= 2 * D - r) {
        slot -= 2 * D - r;
        ++r;
      }
      q = r + slot;
    }
    double acc = 0.0;
    for (int e = 0; e < kOuterBlock; ++e) {
      double v = ws[e];
      if (r >= 0) v *= zs[e][r];
      if (q >= 0) v *= zs[e][q];
      acc += v;
    }
    S.part[(size_t)blockIdx.x * kPartStride + mo] = acc;
  }
}

// Totals of the block moments and the L-kernel fit of one dataset, by one warp.
// It needs only the proposal kernel's partial moments, so it runs beside the
// particle filter (a parallel branch of the iteration graph).
template <int D>
__global__ void __launch_bounds__(32) lkfit_kernel(OuterParams P) {
  const DSDev& S = P.ds[blockIdx.y];
  const uint32_t k = (uint32_t)(*P.k_done + 1);
  if (k == 1 || P.lkernel != LK_GAUSS) return;
  __shared__ double tot[kPartStride];
  __shared__ FitScratch fit;
  const int lane = threadIdx.x, N = S.N;
  const int NM = n_moments(D);
  // totals: lane l takes blocks l, l+32, ... in order, then a fixed shuffle tree
  for (int mo = 0; mo < NM; ++mo) {
    double t = 0.0;
    for (int bb = lane; bb < S.nblk; bb += 32) t += S.part[(size_t)bb * kPartStride + mo];
    t = warp_sum(t);
    if (lane == 0) tot[mo] = t;
  }
  __syncwarp();
  double sh2[2 * D];
#pragma unroll
  for (int r = 0; r < 2 * D; ++r) sh2[r] = S.thA[(size_t)(r % D) * N];
  lk_fit_warp(D, tot, sh2, fit, S.lk);
}

// ---------------------------------------------------------------------------
// weights + normalisation statistics
// ---------------------------------------------------------------------------
// Recycling sums (Eqs. 23-24, 29): rec = [sum l_k, sum l_k f~_k [D],
// sum l_k (C_k + f~_k f~_k^T) [D][D]], C_k the iteration's weighted covariance.
__device__ __forceinline__ void accumulate_recycling(double* rec, double* est_rec, double ess,
                                                     const double* est, const double* cov, int D) {
  rec[0] += ess;
  for (int d = 0; d < D; ++d) rec[1 + d] += ess * est[d];
  for (int d = 0; d < D; ++d)
    for (int e = 0; e < D; ++e) rec[1 + D + d * D + e] += ess * (cov[d * kMaxD + e] + est[d] * est[e]);
  for (int d = 0; d < D; ++d) est_rec[d] = rec[1 + d] / rec[0];
}

__host__ __device__ constexpr int tri(int d, int f) { return d * (d + 1) / 2 + f; }  // f <= d

// Learned proposal: the lower Cholesky factor of the weighted covariance of
// theta_k; usable when every pivot is positive and the population holds
// ESS >= 2 (D + 1).
template <int D>
__device__ void population_cholesky(const smc2_iter_stats& st, IterCur* cur) {
  double Lm[D][D];
  bool ok = st.ess >= 2.0 * (D + 1);
  for (int d = 0; d < D; ++d)
    for (int f = 0; f <= d; ++f) Lm[d][f] = st.cov[d * kMaxD + f];
  for (int j = 0; j < D; ++j) {
    double a = Lm[j][j];
    for (int c = 0; c < j; ++c) a -= Lm[j][c] * Lm[j][c];
    if (!(a > 1e-12 * fabs(Lm[j][j])) || !(a > 0.0)) {
      ok = false;
      a = 1.0;
    }
    const double ljj = sqrt(a);
    Lm[j][j] = ljj;
    for (int r = j + 1; r < D; ++r) {
      double v = Lm[r][j];
      for (int c = 0; c < j; ++c) v -= Lm[r][c] * Lm[j][c];
      Lm[r][j] = v / ljj;
    }
  }
  for (int d = 0; d < D; ++d)
    for (int f = 0; f < D; ++f) cur->Lpop[d * kMaxD + f] = f <= d ? Lm[d][f] : 0.0;
  cur->pop_ok = ok ? 1 : 0;
}

template <int D>
__global__ void __launch_bounds__(kOuterBlock) weights_kernel(OuterParams P) {
  const DSDev& S = P.ds[blockIdx.y];
  if ((int)blockIdx.x >= S.nblk) return;
  const int N = S.N, lane = threadIdx.x;
  const int i = blockIdx.x * kOuterBlock + lane;
  const uint32_t k = (uint32_t)(*P.k_done + 1);
  const bool act = i < N;
  double lw = -HUGE_VAL, b[D];
  if (act) {
#pragma unroll
    for (int d = 0; d < D; ++d) b[d] = S.thB[(size_t)d * N + i];
    const double lpB = S.lpB[i], llB = S.llB[i], lq = S.logq[i];
    if (k == 1) {
      lw = (lpB + llB) - lq;  // Eq. (17)
    } else {
      double a[D];
#pragma unroll
      for (int d = 0; d < D; ++d) a[d] = S.thA[(size_t)d * N + i];
      const bool gauss = P.lkernel == LK_GAUSS && !S.lk->fallback;
      const double logL = gauss ? lk_logpdf<D>(*S.lk, a, b) : rw_logpdf<D>(P, a, b);
      lw = S.logw[i] + (lpB + llB) - (S.lpA[i] + S.llA[i]) + logL - lq;  // Eq. (20)
    }
    if (isnan(lw)) lw = -HUGE_VAL;
    S.logw[i] = lw;
  }
  const double mb = warp_max(lw);
  const double e = (act && lw > -HUGE_VAL) ? exp(lw - mb) : 0.0;
  double* ps = S.part_st + (size_t)blockIdx.x * kStatStride;
  constexpr int NV = 2 + D + D * (D + 1) / 2;  // sums of e, e^2, e theta_d, e c_d c_f
  __shared__ double terms[NV][kOuterBlock + 1];
  __shared__ double totals[NV];
  {
    // the block's sums of e, e^2, e theta_d and e c_d c_f (second moments about the
    // dataset's first proposal, close to the population, so the covariance loses
    // little to cancellation): every lane writes its terms to a padded row, then
    // lane q adds column q over the lanes in order
    double c[D];
#pragma unroll
    for (int d = 0; d < D; ++d) c[d] = act ? b[d] - S.thB[(size_t)d * N] : 0.0;
    terms[0][lane] = e;
    terms[1][lane] = e * e;
#pragma unroll
    for (int d = 0; d < D; ++d) terms[2 + d][lane] = act ? e * b[d] : 0.0;
#pragma unroll
    for (int d = 0; d < D; ++d)
#pragma unroll
      for (int f = 0; f <= d; ++f) terms[2 + D + tri(d, f)][lane] = e * c[d] * c[f];
    __syncwarp();
    if (lane < NV) {
      double sum = 0.0;
      for (int l = 0; l < kOuterBlock; ++l) sum += terms[lane][l];
      ps[1 + lane] = sum;
    }
    if (lane == 0) ps[0] = mb;
  }
  __threadfence();
  __syncwarp();
  unsigned ticket = 0;
  if (lane == 0) ticket = atomicAdd(&S.tickets[1], 1u);
  ticket = __shfl_sync(0xffffffffu, ticket, 0);
  if (ticket != (unsigned)(S.nblk - 1)) return;
  __threadfence();
  // combine the block partials: lane l takes blocks l, l+32, ... in order, then a fixed shuffle tree
  double m = -HUGE_VAL;
  for (int bb = lane; bb < S.nblk; bb += 32) m = fmax(m, __ldcg(&S.part_st[(size_t)bb * kStatStride]));
  m = warp_max(m);
  smc2_iter_stats st;
  st.k = (int)k;
  st.dataset = (int)blockIdx.y;
  st.lk_fallback = (k > 1 && P.lkernel == LK_GAUSS) ? S.lk->fallback : 0;
  IterCur* cur = S.cur;
  if (!(m > -HUGE_VAL) || isinf(m) || isnan(m)) {
    if (lane == 0) {
      raise_status(P.status, ST_NONFINITE);
      st.resampled = 0;
      st.mlp_used = 0;
      st.pad = 0;
      st.mlp_loss = 0.0;
      st.ess = st.lse = st.lse2 = st.logz = NAN;
      for (int d = 0; d < kMaxD; ++d) st.est[d] = NAN;
      for (int q = 0; q < kMaxD * kMaxD; ++q) st.cov[q] = NAN;
      cur->resample = 0;
      if ((int)k <= P.K) S.hist[k - 1] = st;
      S.tickets[1] = 0;
    }
    return;
  }
  constexpr int NQ = D * (D + 1) / 2;
  static_assert(3 + D + NQ <= kStatStride, "statistics stride");
  // every lane rescales its blocks' sums to the common maximum; then lane q adds
  // statistic q over the lanes in order (a transpose through shared memory)
  double v[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = 0.0;
  for (int bb = lane; bb < S.nblk; bb += 32) {
    const double* pb = S.part_st + (size_t)bb * kStatStride;
    const double mbb = __ldcg(pb);
    if (!(mbb > -HUGE_VAL)) continue;
    const double f = exp(mbb - m);
    v[1] += __ldcg(pb + 2) * (f * f);
#pragma unroll
    for (int q = 0; q < NV; ++q)
      if (q != 1) v[q] += __ldcg(pb + 1 + q) * f;
  }
#pragma unroll
  for (int q = 0; q < NV; ++q) terms[q][lane] = v[q];
  __syncwarp();
  if (lane < NV) {
    double sum = 0.0;
    for (int l = 0; l < kOuterBlock; ++l) sum += terms[lane][l];
    totals[lane] = sum;
  }
  __syncwarp();
  const double s1 = totals[0], s2 = totals[1], inv_s1 = 1.0 / s1;
  double sth[D], sqq[NQ];
#pragma unroll
  for (int d = 0; d < D; ++d) sth[d] = totals[2 + d];
#pragma unroll
  for (int q = 0; q < NQ; ++q) sqq[q] = totals[2 + D + q];
  if (lane != 0) return;
  st.lse = m + log(s1);
  st.lse2 = 2.0 * m + log(s2);
  st.ess = (s1 * s1) / s2;
  st.logz = st.lse - S.logN;
  for (int d = 0; d < kMaxD; ++d) st.est[d] = d < D ? sth[d] * inv_s1 : 0.0;
  st.resampled = st.ess < P.ess_frac * (double)N;
  cur->m = m;
  cur->lse = st.lse;
  cur->resample = st.resampled;
  cur->m_par = st.resampled ? st.lse - S.logN : m;
  // weighted covariance of theta_k (Eq. 21 with f = (theta - f~)(theta - f~)^T)
  for (int q = 0; q < kMaxD * kMaxD; ++q) st.cov[q] = 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const double md = st.est[d] - S.thB[(size_t)d * N];
#pragma unroll
    for (int f = 0; f <= d; ++f) {
      const double mf = st.est[f] - S.thB[(size_t)f * N];
      const double v = sqq[tri(d, f)] * inv_s1 - md * mf;
      st.cov[d * kMaxD + f] = v;
      st.cov[f * kMaxD + d] = v;
    }
  }
  if (P.mlp.on) population_cholesky<D>(st, cur);
  st.mlp_used = (k > 1 && P.mlp.on) ? cur->mlp_used : 0;
  st.pad = 0;
  st.mlp_loss = (k > 1 && P.mlp.on) ? cur->mlp_loss : 0.0;
  accumulate_recycling(S.rec, S.est_rec, st.ess, st.est, st.cov, D);
  if ((int)k <= P.K) S.hist[k - 1] = st;
  S.tickets[1] = 0;
}

// ---------------------------------------------------------------------------
// quantise
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kOuterBlock) quantise_kernel(OuterParams P) {
  const DSDev& S = P.ds[blockIdx.y];
  if ((int)blockIdx.x >= S.nblk || !S.cur->resample) return;
  const int i = blockIdx.x * kOuterBlock + threadIdx.x;
  if (i >= S.N) return;
  const double lw = S.logw[i];
  const double scale = ldexp(1.0, fixed_point_bits(S.N));
  S.q[i] = (lw > -HUGE_VAL && !isnan(lw)) ? __double2ull_rz(exp(lw - S.cur->m) * scale) : 0ull;
}

// ---------------------------------------------------------------------------
// resample: block-wide inclusive scan of all q into shared memory, then the
// block's own slots; both this kernel and the standalone primitive use it.
// ---------------------------------------------------------------------------
__device__ uint64_t scan_all_to_smem(const uint64_t* q, int n, uint64_t* C) {
  __shared__ uint64_t wt[kResWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t carry = 0;
  for (int base = 0; base < n; base += kResBlock) {
    const int idx = base + threadIdx.x;
    const uint64_t v = idx < n ? q[idx] : 0ull;
    const uint64_t incl = warp_incl_scan_u64(v, lane);
    if (lane == 31) wt[warp] = incl;
    __syncthreads();
    uint64_t off = 0, total = 0;
    for (int w = 0; w < kResWarps; ++w) {
      const uint64_t tw = wt[w];
      if (w < warp) off += tw;
      total += tw;
    }
    if (idx < n) C[idx] = carry + off + incl;
    carry += total;
    __syncthreads();
  }
  return carry;
}

__device__ __forceinline__ int search_first_greater(const uint64_t* C, int n, uint64_t tau) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (C[mid] > tau)
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
}

__global__ void __launch_bounds__(kResBlock) resample_kernel(OuterParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* C = reinterpret_cast<uint64_t*>(smem_raw);
  const DSDev& S = P.ds[blockIdx.y];
  const int N = S.N, D = P.D, tid = threadIdx.x;
  const uint32_t k = (uint32_t)(*P.k_done + 1);
  if ((int)blockIdx.x < S.nblk_res) {
    const int j = blockIdx.x * kResBlock + tid;
    if (S.cur->resample) {
      const uint64_t total = scan_all_to_smem(S.q, N, C);
      const uint32_t U =
          philox4x32_10(make_uint4(0u, 0u, S.c2hi, counter_c3(TAG_OUTER_RES, k)), seed_key(P.seed)).x;
      const int log2n = ((N & (N - 1)) == 0) ? (__ffs(N) - 1) : -1;
      if (j < N) {
        const uint64_t tau = slot_threshold((uint32_t)j, U, total, N, log2n);
        const int a = search_first_greater(C, N, tau);
        for (int d = 0; d < D; ++d) S.thA[(size_t)d * N + j] = S.thB[(size_t)d * N + a];
        S.lpA[j] = S.lpB[a];
        S.llA[j] = S.llB[a];
        S.logw[j] = S.cur->lse - S.logN;
      }
    } else if (j < N) {
      for (int d = 0; d < D; ++d) S.thA[(size_t)d * N + j] = S.thB[(size_t)d * N + j];
      S.lpA[j] = S.lpB[j];
      S.llA[j] = S.llB[j];
    }
  }
  // the last block of the whole grid advances the iteration counter
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    const unsigned nb = gridDim.x * gridDim.y;
    if (atomicAdd(P.grid_ticket, 1u) == nb - 1) {
      *P.k_done = (int)k;
      *P.grid_ticket = 0;
    }
  }
}

__global__ void __launch_bounds__(kResBlock)
    resample_primitive_kernel(const uint64_t* q, int n, uint32_t U, int32_t* anc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* C = reinterpret_cast<uint64_t*>(smem_raw);
  const uint64_t total = scan_all_to_smem(q, n, C);
  const int log2n = ((n & (n - 1)) == 0) ? (__ffs(n) - 1) : -1;
  const int j = blockIdx.x * kResBlock + threadIdx.x;
  if (j < n && total > 0) anc[j] = search_first_greater(C, n, slot_threshold((uint32_t)j, U, total, n, log2n));
}

__global__ void philox_normals_kernel(uint64_t seed, const uint32_t* ctr, int n, int precision,
                                      uint32_t* words, double* z) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const uint4 c = make_uint4(ctr[4 * r], ctr[4 * r + 1], ctr[4 * r + 2], ctr[4 * r + 3]);
  const uint2 key = seed_key(seed);
  if (words) {
    const uint4 w = philox4x32_10(c, key);
    words[4 * r] = w.x;
    words[4 * r + 1] = w.y;
    words[4 * r + 2] = w.z;
    words[4 * r + 3] = w.w;
  }
  if (z) {
    if (precision == SMC2_PREC_FP64) {
      double v[4];
      normals4<double>(c, key, v);
      for (int a = 0; a < 4; ++a) z[4 * r + a] = v[a];
    } else {
      float v[4];
      normals4<float>(c, key, v);
      for (int a = 0; a < 4; ++a) z[4 * r + a] = (double)v[a];
    }
  }
}

template <typename R>
__global__ void obs_terms_kernel(int model, const double* y, int T, R* obs) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  const double v = y[t];
  double inv = 0.0, c = 0.0;
  if (model != MODEL_LG && v > 0.0) {  // Poisson terms (SEIR-type and SIR)
    inv = 1.0 / v;
    c = -lgamma(v + 1.0) + v * log(v) - v;
  }
  obs[4 * t] = (R)v;
  obs[4 * t + 1] = (R)inv;
  obs[4 * t + 2] = (R)c;
  obs[4 * t + 3] = (R)0;
}

// Parent reference after a restored state: m_par = max_i log w_i of one dataset.
__global__ void parent_reference_kernel(OuterParams P, int dataset) {
  const DSDev& S = P.ds[dataset];
  double m = -HUGE_VAL;
  for (int i = threadIdx.x; i < S.N; i += 32) m = fmax(m, S.logw[i]);
  m = warp_max(m);
  if (threadIdx.x == 0) S.cur->m_par = m;
}

// Recycling sums rebuilt from a restored history, in iteration order, with the
// same accumulation as the weights kernel.
__global__ void rebuild_recycling_kernel(OuterParams P, int dataset, int k) {
  const DSDev& S = P.ds[dataset];
  for (int a = 0; a <= P.D + P.D * P.D; ++a) S.rec[a] = 0.0;
  for (int d = 0; d < P.D; ++d) S.est_rec[d] = 0.0;
  for (int e = 0; e < k; ++e) {
    const smc2_iter_stats& st = S.hist[e];
    if (isfinite(st.ess)) accumulate_recycling(S.rec, S.est_rec, st.ess, st.est, st.cov, P.D);
  }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
cudaError_t outer_obs_terms(int precision, int model, const double* y, int T, void* obs,
                            cudaStream_t s) {
  const int blk = 128, grid = (T + blk - 1) / blk;
  if (precision == SMC2_PREC_FP64)
    obs_terms_kernel<double><<<grid, blk, 0, s>>>(model, y, T, static_cast<double*>(obs));
  else
    obs_terms_kernel<float><<<grid, blk, 0, s>>>(model, y, T, static_cast<float*>(obs));
  return cudaGetLastError();
}

cudaError_t outer_propose(const OuterParams& P, int max_nblk, cudaStream_t s) {
  const dim3 grid(max_nblk, P.n_ds);
  if (P.D == 2)
    propose_kernel<2><<<grid, kOuterBlock, 0, s>>>(P);
  else if (P.D == 3)
    propose_kernel<3><<<grid, kOuterBlock, 0, s>>>(P);
  else if (P.D == 4)
    propose_kernel<4><<<grid, kOuterBlock, 0, s>>>(P);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}
cudaError_t outer_lkfit(const OuterParams& P, cudaStream_t s) {
  const dim3 grid(1, P.n_ds);
  if (P.D == 2)
    lkfit_kernel<2><<<grid, 32, 0, s>>>(P);
  else if (P.D == 3)
    lkfit_kernel<3><<<grid, 32, 0, s>>>(P);
  else if (P.D == 4)
    lkfit_kernel<4><<<grid, 32, 0, s>>>(P);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}
cudaError_t outer_weights(const OuterParams& P, int max_nblk, cudaStream_t s) {
  const dim3 grid(max_nblk, P.n_ds);
  if (P.D == 2)
    weights_kernel<2><<<grid, kOuterBlock, 0, s>>>(P);
  else if (P.D == 3)
    weights_kernel<3><<<grid, kOuterBlock, 0, s>>>(P);
  else if (P.D == 4)
    weights_kernel<4><<<grid, kOuterBlock, 0, s>>>(P);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}
cudaError_t outer_quantise(const OuterParams& P, int max_nblk, cudaStream_t s) {
  quantise_kernel<<<dim3(max_nblk, P.n_ds), kOuterBlock, 0, s>>>(P);
  return cudaGetLastError();
}
cudaError_t outer_resample(const OuterParams& P, int max_nblk_res, int max_N, cudaStream_t s) {
  const size_t smem = (size_t)max_N * sizeof(uint64_t);
  cudaError_t e = cudaFuncSetAttribute(resample_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  resample_kernel<<<dim3(max_nblk_res, P.n_ds), kResBlock, smem, s>>>(P);
  return cudaGetLastError();
}
cudaError_t outer_parent_reference(const OuterParams& P, int dataset, cudaStream_t s) {
  parent_reference_kernel<<<1, 32, 0, s>>>(P, dataset);
  return cudaGetLastError();
}
cudaError_t outer_rebuild_recycling(const OuterParams& P, int dataset, int k, cudaStream_t s) {
  rebuild_recycling_kernel<<<1, 1, 0, s>>>(P, dataset, k);
  return cudaGetLastError();
}
cudaError_t resample_systematic_launch(const uint64_t* q, int n, uint32_t U, int32_t* anc,
                                       cudaStream_t s) {
  const size_t smem = (size_t)n * sizeof(uint64_t);
  cudaError_t e = cudaFuncSetAttribute(resample_primitive_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  resample_primitive_kernel<<<(n + kResBlock - 1) / kResBlock, kResBlock, smem, s>>>(q, n, U, anc);
  return cudaGetLastError();
}
cudaError_t philox_normals_launch(uint64_t seed, const uint32_t* ctr, int n, int precision,
                                  uint32_t* words, double* z, cudaStream_t s) {
  philox_normals_kernel<<<(n + 127) / 128, 128, 0, s>>>(seed, ctr, n, precision, words, z);
  return cudaGetLastError();
}

}  // namespace smc2
