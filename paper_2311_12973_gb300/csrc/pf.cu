// pf.cu -- host side of the particle-filter kernel: shapes, attributes, launches.
#include <algorithm>
#include <mutex>

#include "pf_fast.cuh"

namespace smc2 {

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

int pf_group_threads(int ppt, int M) { return group_threads_for(ppt, M); }

size_t pf_smem_bytes(int precision, int model, int ppt, bool general, int block, int M) {
  const int gt = group_threads_for(ppt, M);
  const int fpc = block / gt;
  const int ns = model == MODEL_LG ? 1 : model == MODEL_SIR ? 2 : 4;
  const int rs = precision == SMC2_PREC_FP64 ? 8 : 4;
  return (size_t)fpc * region_bytes(gt * ppt, gt >> 5, ns, rs, is_staged(ppt), general);
}

static const void* select_kernel(int precision, int model, int ppt, bool named, bool general) {
  if (model == MODEL_SIR)
    return precision == SMC2_PREC_FP64 ? pf_select_sir_f64(ppt, named, general)
                                       : pf_select_sir_f32(ppt, named, general);
  if (general)
    return precision == SMC2_PREC_FP64 ? pf_select_general_f64(model, ppt, named)
                                       : pf_select_general_f32(model, ppt, named);
  return precision == SMC2_PREC_FP64 ? pf_select_f64(model, ppt, named)
                                     : pf_select_f32(model, ppt, named);
}

// The dynamic shared-memory limit is an attribute of the kernel, shared by
// every context and by the allocation-free entry point that launch the same
// instantiation: it is only ever raised, so that one caller's smaller shape
// never refuses another's larger launch.
cudaError_t pf_configure(int precision, int model, int ppt, bool named, bool general, size_t smem) {
  const void* f = select_kernel(precision, model, ppt, named, general);
  if (!f) return cudaErrorInvalidValue;
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  cudaFuncAttributes a{};
  const cudaError_t e = cudaFuncGetAttributes(&a, f);
  if (e != cudaSuccess) return e;
  if ((size_t)a.maxDynamicSharedSizeBytes >= smem) return cudaSuccess;
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

int pf_occupancy(int precision, int model, int ppt, bool named, bool general, int block, size_t smem) {
  const void* f = select_kernel(precision, model, ppt, named, general);
  int n = 0;
  if (!f || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, block, smem) != cudaSuccess) return 0;
  return n;
}

cudaError_t pf_launch(int precision, int model, int ppt, bool named, bool general, int grid, int block,
                      size_t smem, const PFLaunch& L, cudaStream_t s) {
  const void* f = select_kernel(precision, model, ppt, named, general);
  if (!f) return cudaErrorInvalidValue;
  void* args[] = {const_cast<PFLaunch*>(&L)};
  return cudaLaunchKernel(f, dim3(grid), dim3(block), args, smem, s);
}

// ---------------------------------------------------------------------------
// the FP32 one-group-per-CTA filter (pf_fast.cuh)
// ---------------------------------------------------------------------------
bool pf_fast_eligible(int precision, int model, bool general, int ppt) {
  return precision == SMC2_PREC_MIXED && (model == MODEL_LG || model == MODEL_SEIR) && !general &&
         (ppt == 2 || ppt == 4 || ppt == 8);
}

size_t pf_fast_smem_bytes(int model, int ppt, int block, int M) {
  const int T = group_threads_for(ppt, M);
  const size_t rb = (fast_region_bytes(ppt * T, model == MODEL_LG ? 1 : 4) + 15) & ~(size_t)15;
  return (size_t)(block / T) * rb;
}

static const void* select_fast(int model, int ppt, bool trace, bool grouped) {
  if (grouped) return trace ? nullptr : pf_fast_select_grouped(model, ppt);
  if (model == MODEL_LG) return pf_fast_select_lg(ppt, trace);
  if (model == MODEL_SEIR) return pf_fast_select_seir(ppt, trace);
  return nullptr;
}

cudaError_t pf_fast_configure(int model, int ppt, bool trace, bool grouped, size_t smem) {
  const void* f = select_fast(model, ppt, trace, grouped);
  if (!f) return cudaErrorInvalidValue;
  static std::mutex mu;  // only ever raised, as for pf_kernel
  std::lock_guard<std::mutex> lock(mu);
  cudaFuncAttributes a{};
  const cudaError_t e = cudaFuncGetAttributes(&a, f);
  if (e != cudaSuccess) return e;
  if ((size_t)a.maxDynamicSharedSizeBytes >= smem) return cudaSuccess;
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

int pf_fast_occupancy(int model, int ppt, bool trace, bool grouped, int block, size_t smem) {
  const void* f = select_fast(model, ppt, trace, grouped);
  int n = 0;
  if (!f || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, block, smem) != cudaSuccess) return 0;
  return n;
}

cudaError_t pf_fast_launch(int model, int ppt, bool trace, bool grouped, int grid, int block, size_t smem,
                           const PFLaunch& L, cudaStream_t s) {
  const void* f = select_fast(model, ppt, trace, grouped);
  if (!f) return cudaErrorInvalidValue;
  void* args[] = {const_cast<PFLaunch*>(&L)};
  return cudaLaunchKernel(f, dim3(grid), dim3(block), args, smem, s);
}

// CTAs of kernel f (block threads, smem bytes of dynamic shared memory) that fit
// on one SM beside a resident CTA of another kernel (o_threads threads of o_regs
// registers, o_smem bytes of shared memory): registers are allocated per warp
// in units of 256, and every CTA reserves the device's per-block shared memory.
static int blocks_beside(const void* f, int block, size_t smem, int o_threads, int o_regs, size_t o_smem) {
  cudaFuncAttributes a{};
  int dev = 0, regs_sm = 0, smem_sm = 0, resv = 0, thr_sm = 0, blk_sm = 0;
  if (!f || cudaFuncGetAttributes(&a, f) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&blk_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev) != cudaSuccess)
    return 0;
  auto regs_of = [](int threads, int regs) {
    return ((threads + 31) / 32) * (((regs * 32) + 255) / 256 * 256);
  };
  const long r_free = (long)regs_sm - regs_of(o_threads, o_regs);
  const long s_free = (long)smem_sm - (long)(o_smem + resv);
  const long t_free = (long)thr_sm - o_threads;
  const long per_r = regs_of(block, a.numRegs), per_s = (long)(smem + a.sharedSizeBytes + resv);
  if (r_free < 0 || s_free < 0 || t_free < 0) return 0;
  long n = std::min<long>(blk_sm - 1, t_free / block);
  n = std::min(n, r_free / per_r);
  if (per_s > 0) n = std::min(n, s_free / per_s);
  return (int)std::max<long>(n, 0);
}

int pf_blocks_beside(int precision, int model, int ppt, bool named, bool general, int block, size_t smem,
                     int o_threads, int o_regs, size_t o_smem) {
  return blocks_beside(select_kernel(precision, model, ppt, named, general), block, smem, o_threads, o_regs,
                       o_smem);
}

int pf_fast_blocks_beside(int model, int ppt, bool grouped, int block, size_t smem, int o_threads, int o_regs,
                          size_t o_smem) {
  return blocks_beside(select_fast(model, ppt, false, grouped), block, smem, o_threads, o_regs, o_smem);
}

}  // namespace smc2
