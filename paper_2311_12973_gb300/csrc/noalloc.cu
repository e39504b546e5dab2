// noalloc.cu -- particle-filter log-likelihoods with no device allocation.
//
// Some callers cannot allocate device memory once they are running: a host
// with a fixed device-memory budget set at start-up, a framework whose own
// pool owns all device memory (so a cudaMalloc behind its back can fail or
// fragment it), or a latency-critical loop that cannot afford the implicit
// device synchronisation of cudaMalloc / cudaFree.  smc2_pf_loglik needs a
// context, and creating one allocates; this entry point needs none.  Its
// scratch -- the per-step observation terms and the work-unit counter of the
// particle-filter kernel -- lives in the file-scope device array below, which
// every GPU that loads the library holds until the process exits.
#include <cmath>
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace smc2 {
namespace {

// 1 MiB of scratch: the work-unit counter, then up to SMC2_NOALLOC_MAX_T steps of
// observation terms (four values per step, 32 bytes in FP64).
constexpr size_t kNoallocScratchBytes = 1u << 20;
constexpr size_t kNoallocCounterBytes = 256;
static_assert(kNoallocScratchBytes - kNoallocCounterBytes >= (size_t)SMC2_NOALLOC_MAX_T * 32,
              "scratch must hold the observation terms of the longest series");

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_dev[kMaxDevices] = {};  // device address of g_noalloc_scratch, per device

// Every refusal is a status code; `what` names the reason for a reader of the source.
smc2_status fail(smc2_status s, const char* what) {
  static_cast<void>(what);
  return s;
}

// The host-side name of g_noalloc_scratch is not a device address: the
// address is looked up once per device, with that device current.
smc2_status scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(SMC2_ECUDA, "cudaGetDevice failed");
  if (dev < 0 || dev >= kMaxDevices) return fail(SMC2_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return fail(SMC2_ECUDA, cudaGetErrorString(e));
    g_scratch_dev[dev] = p;
  }
  *out = g_scratch_dev[dev];
  return SMC2_OK;
}

}  // namespace
}  // namespace smc2

using namespace smc2;

extern "C" smc2_status smc2_pf_loglik_noalloc(const smc2_config* cfg, const double* y_dev,
                                              const double* theta_dev, int n, int iteration,
                                              double* loglik_dev, void* stream) {
  if (!cfg || !y_dev || !theta_dev || !loglik_dev) return fail(SMC2_EINVAL, "null pointer argument");
  if (cfg->model != SMC2_MODEL_LG_AR1 && cfg->model != SMC2_MODEL_SEIR && cfg->model != SMC2_MODEL_SIR)
    return fail(SMC2_EINVAL, "unknown model");
  if (cfg->precision != SMC2_PREC_FP64 && cfg->precision != SMC2_PREC_MIXED)
    return fail(SMC2_EINVAL, "unknown precision");
  if (n < 1 || n > SMC2_MAX_N) return fail(SMC2_EINVAL, "n outside [1, SMC2_MAX_N]");
  if (cfg->M < 1 || cfg->M > SMC2_MAX_M) return fail(SMC2_EINVAL, "M outside [1, SMC2_MAX_M]");
  if (cfg->T < 1 || cfg->T > SMC2_NOALLOC_MAX_T)
    return fail(SMC2_EINVAL, "T outside [1, SMC2_NOALLOC_MAX_T]: the fixed scratch holds no more steps");
  if (iteration < 0 || iteration >= (1 << 28)) return fail(SMC2_EINVAL, "iteration out of range");
  if (cfg->model == SMC2_MODEL_SEIR &&
      (!(cfg->npop > 0) || cfg->n_sub < 1 || !(cfg->lambda_floor > 0)))
    return fail(SMC2_EINVAL, "invalid SEIR constants");
  if (cfg->model == SMC2_MODEL_SIR &&
      (!(cfg->npop > 0) || cfg->npop > 16777216.0 || cfg->npop != floor(cfg->npop) ||
       !(cfg->i0 >= 0 && cfg->i0 <= cfg->npop) || cfg->i0 != floor(cfg->i0)))
    return fail(SMC2_EINVAL, "invalid SIR constants");
  const int ppt = cfg->ppt ? cfg->ppt : 2;
  if (ppt != 1 && ppt != 2 && ppt != 4 && ppt != 8 && ppt != 16) return fail(SMC2_EINVAL, "ppt");
  if ((cfg->pf_scheme != SMC2_PF_SYSTEMATIC && cfg->pf_scheme != SMC2_PF_MULTINOMIAL) ||
      !(cfg->pf_ess_frac >= 0.0 && cfg->pf_ess_frac <= 1.0))
    return fail(SMC2_EINVAL, "pf_scheme / pf_ess_frac");
  const bool general = cfg->pf_scheme != SMC2_PF_SYSTEMATIC || cfg->pf_ess_frac > 0.0;
  if (general && ppt > 4) return fail(SMC2_EINVAL, "the PF variants need ppt <= 4");
  if (cfg->model == SMC2_MODEL_SIR && ppt > 4) return fail(SMC2_EINVAL, "the SIR model needs ppt <= 4");
  const int gt = pf_group_threads(ppt, cfg->M);
  if (gt > kPfMaxBlock) return fail(SMC2_EINVAL, "M too large for this ppt");

  void* scratch = nullptr;
  smc2_status st = scratch_address(&scratch);
  if (st != SMC2_OK) return st;
  int* counter = static_cast<int*>(scratch);
  void* obs = static_cast<unsigned char*>(scratch) + kNoallocCounterBytes;
  const int model = cfg->model;  // the internal model ids equal the ABI's
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  // one filter group per CTA (or several one-warp groups): no named barriers
  const int block = gt > 32 ? gt : 256;
  const size_t smem = pf_smem_bytes(cfg->precision, model, ppt, general, block, cfg->M);
  if (smem > 227 * 1024) return fail(SMC2_EINVAL, "shared memory of the launch shape");
  cudaError_t e = pf_configure(cfg->precision, model, ppt, false, general, smem);
  if (e != cudaSuccess) return fail(SMC2_ECUDA, cudaGetErrorString(e));
  const int occ = pf_occupancy(cfg->precision, model, ppt, false, general, block, smem);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || occ < 1)
    return fail(SMC2_ECUDA, "device query");

  // the previous call's counter is still in the array: start it from zero
  e = cudaMemsetAsync(counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return fail(SMC2_ECUDA, cudaGetErrorString(e));
  e = outer_obs_terms(cfg->precision, model, y_dev, cfg->T, obs, s);
  if (e != cudaSuccess) return fail(SMC2_ECUDA, cudaGetErrorString(e));

  PFLaunch L{};
  L.jobs = nullptr;
  L.job0.theta = theta_dev;
  L.job0.ld = n;
  L.job0.n = n;
  L.job0.M = cfg->M;
  L.job0.T = cfg->T;
  L.job0.loglik = loglik_dev;
  L.job0.obs = obs;
  L.job0.c2hi = 0;
  L.wus = nullptr;
  L.fpc_single = block / gt;
  L.n_wu = (n + L.fpc_single - 1) / L.fpc_single;
  L.wu_counter = counter;
  L.seed = cfg->seed;
  philox_round_keys(cfg->seed, L.rk);
  L.k_done = nullptr;
  L.k_imm = iteration;
  L.status = nullptr;
  L.mdl.npop = cfg->npop;
  L.mdl.e0 = cfg->e0;
  L.mdl.i0 = cfg->i0;
  L.mdl.lambda_floor = cfg->lambda_floor;
  L.mdl.n_sub = cfg->n_sub;
  L.mdl.pf_scheme = cfg->pf_scheme;
  L.mdl.pf_ess_frac = cfg->pf_ess_frac;
  L.t_cap = 0;
  const int grid = L.n_wu < occ * sms ? L.n_wu : occ * sms;
  e = pf_launch(cfg->precision, model, ppt, false, general, grid, block, smem, L, s);
  if (e != cudaSuccess) return fail(SMC2_ECUDA, cudaGetErrorString(e));
  return SMC2_OK;
}

// ---------------------------------------------------------------------------
// FMA throughput (diagnostic)
// ---------------------------------------------------------------------------
namespace smc2 {
namespace {

__device__ double g_fma_sink;  // keeps the chains live

constexpr int kFmaChains = 8;

template <typename R>
__global__ void __launch_bounds__(256) fma_rate_kernel(int iters, R b, R c) {
  R a[kFmaChains];
#pragma unroll
  for (int q = 0; q < kFmaChains; ++q) a[q] = (R)(threadIdx.x + q) * (R)1e-3;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int q = 0; q < kFmaChains; ++q) a[q] = fma(a[q], b, c);
  R s = 0;
#pragma unroll
  for (int q = 0; q < kFmaChains; ++q) s += a[q];
  if (s == (R)-12345.0) g_fma_sink = (double)s;  // never true for these inputs
}

template <typename R>
smc2_status fma_rate(int iters, double* flops, cudaStream_t s) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SMC2_ECUDA;
  const int grid = sms * 8, block = 256;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return SMC2_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return SMC2_ECUDA;
  }
  float ms = 0.f;
  fma_rate_kernel<R><<<grid, block, 0, s>>>(iters / 8, (R)0.9999, (R)1e-7);  // warm-up
  cudaEventRecord(e0, s);
  fma_rate_kernel<R><<<grid, block, 0, s>>>(iters, (R)0.9999, (R)1e-7);
  cudaEventRecord(e1, s);
  const bool ok = cudaGetLastError() == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                  cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.f;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok) return SMC2_ECUDA;
  *flops = 2.0 * kFmaChains * (double)iters * grid * block / (ms * 1e-3);
  return SMC2_OK;
}

}  // namespace
}  // namespace smc2

extern "C" smc2_status smc2_fma_rates(double* fp32_flops, double* fp64_flops, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  smc2_status st = SMC2_OK;
  if (fp32_flops) st = fma_rate<float>(1 << 16, fp32_flops, s);
  if (st == SMC2_OK && fp64_flops) st = fma_rate<double>(1 << 11, fp64_flops, s);
  return st;
}
