// api.cu -- the C ABI declared in include/smc2.h.
//
// Host responsibilities only: validate, own one device arena per context,
// build the particle-filter work list, enqueue kernels on the context stream
// and capture iterations into CUDA graphs.  No step of the sampler runs here.
#include <algorithm>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "internal.h"

using namespace smc2;

namespace {

// Host-side trace ranges (NVTX) around the library's calls: a profiler that
// attaches (ncu --nvtx, nsys) sees them and the kernels launched inside; with
// none attached each range costs a few nanoseconds.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

// Learned proposal defaults: step h, Adam rate, Adam steps per iteration,
// iterations of training pairs kept.
constexpr double kMlpStep = 1.0;
constexpr double kMlpLr = 5e-3;
constexpr int kMlpSteps = 16;
constexpr int kMlpWindow = 4;

struct GraphKey {
  int n_iter, timing;
  bool operator<(const GraphKey& o) const {
    return n_iter != o.n_iter ? n_iter < o.n_iter : timing < o.timing;
  }
};

struct TimedGraph {
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaEvent_t> ev;  // pairs around each PF launch
};

}  // namespace

struct smc2_ctx {
  smc2_config cfg{};
  int n_ds = 1, D = 0, K = 0, precision = 0, model = 0;
  std::vector<int> N, M, T, nblk, nblk_res;
  std::vector<size_t> yoff;
  size_t ytot = 0;
  int max_N = 0, max_nblk = 0, max_nblk_res = 0;
  cudaStream_t stream = nullptr, cap_stream = nullptr, side_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaStream_t train_stream = nullptr;              // learned-proposal training branch
  cudaEvent_t ev_tfork = nullptr, ev_tjoin = nullptr;
  bool train_pending = false;                       // while capturing: branch not yet joined
  int device = 0, sms = 0;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  double* d_y = nullptr;
  std::vector<void*> d_obs;
  std::vector<DSDev> h_ds;
  DSDev* d_ds = nullptr;
  PFJob* d_jobs = nullptr;
  int4* d_wus = nullptr;
  int n_wus = 0;
  int* d_wu_counter = nullptr;
  int* d_k = nullptr;
  int* d_status = nullptr;
  unsigned* d_grid_ticket = nullptr;
  int ppt = 4, pf_block = 256, pf_grid = 1;
  bool pf_named = false;    // pf_kernel: named-barrier groups; the FP32 filter: grouped instantiation
  bool pf_general = false;  // the paper's PF variants: multinomial slots, ESS-triggered resampling
  bool pf_fast = false;     // the FP32 filter of pf_fast.cuh runs
  size_t pf_smem = 0;
  int k_host = 0;
  std::map<GraphKey, TimedGraph> graphs;
  bool timing = false;
  double pf_ms = 0.0;
  int64_t pf_launches = 0, kernel_launches = 0;
  OuterParams op{};
  PFLaunch pl{};
  MlpDev mlp{};
};

namespace {

smc2_status map_cuda(cudaError_t e) {
  if (e == cudaSuccess) return SMC2_OK;
  if (e == cudaErrorMemoryAllocation) return SMC2_ENOMEM;
  return SMC2_ECUDA;
}

thread_local char g_last_error[256] = "";

smc2_status record_cuda(cudaError_t e, const char* what) {
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s)", what, cudaGetErrorName(e),
           cudaGetErrorString(e));
  return map_cuda(e);
}

#define SMC2_TRY(expr)                                      \
  do {                                                      \
    cudaError_t _e = (expr);                                \
    if (_e != cudaSuccess) return record_cuda(_e, #expr);   \
  } while (0)

smc2_status status_from_bits(int bits) {
  if (bits & ST_NONFINITE) return SMC2_ENONFINITE;
  return SMC2_OK;
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

smc2_status validate(const smc2_config* c) {
  if (!c) return SMC2_EINVAL;
  if (c->model != SMC2_MODEL_LG_AR1 && c->model != SMC2_MODEL_SEIR && c->model != SMC2_MODEL_SIR)
    return SMC2_EINVAL;
  if (c->precision != SMC2_PREC_FP64 && c->precision != SMC2_PREC_MIXED) return SMC2_EINVAL;
  if (c->proposal != SMC2_PROP_RW && c->proposal != SMC2_PROP_MLP) return SMC2_EINVAL;
  if (c->proposal == SMC2_PROP_MLP &&
      (c->lkernel != SMC2_LK_GAUSS_OPT || c->n_datasets > 1 || c->D > kMlpMaxD))
    return SMC2_EINVAL;
  if (!(c->mlp_h >= 0.0 && c->mlp_h < 1e3) || !(c->mlp_lr >= 0.0 && c->mlp_lr < 1.0) ||
      c->mlp_steps < 0 || c->mlp_steps > 256 || c->mlp_window < 0 || c->mlp_window > 16)
    return SMC2_EINVAL;
  if (c->lkernel != SMC2_LK_FORWARD && c->lkernel != SMC2_LK_GAUSS_OPT) return SMC2_EINVAL;
  if (c->D != (c->model == SMC2_MODEL_LG_AR1 ? 3 : c->model == SMC2_MODEL_SIR ? 2 : 4)) return SMC2_EINVAL;
  if (c->K < 1 || c->K > (1 << 27)) return SMC2_EINVAL;
  if (!finite_pos(c->rw_scale) || !std::isfinite(c->ess_frac) || c->ess_frac < 0.0) return SMC2_EINVAL;
  if (c->prior_kind != SMC2_PRIOR_GAUSS && c->prior_kind != SMC2_PRIOR_UNIFORM) return SMC2_EINVAL;
  for (int d = 0; d < c->D; ++d) {
    if (c->prior_kind == SMC2_PRIOR_UNIFORM) {
      if (!std::isfinite(c->prior_lo[d]) || !std::isfinite(c->prior_hi[d]) ||
          !finite_pos(c->prior_hi[d] - c->prior_lo[d]))
        return SMC2_EINVAL;
    } else if (!std::isfinite(c->prior_mean[d]) || !finite_pos(c->prior_sd[d])) {
      return SMC2_EINVAL;
    }
  }
  if (c->model == SMC2_MODEL_SIR) {  // integer compartments, exact in float
    if (!finite_pos(c->npop) || c->npop > 16777216.0 || c->npop != std::floor(c->npop) ||
        !(c->i0 >= 0.0 && c->i0 <= c->npop) || c->i0 != std::floor(c->i0) || c->ppt > 4)
      return SMC2_EINVAL;
  }
  if (c->model == SMC2_MODEL_SEIR) {
    if (!finite_pos(c->npop) || !std::isfinite(c->e0) || !std::isfinite(c->i0) || c->e0 < 0 ||
        c->i0 < 0 || c->e0 + c->i0 > c->npop || c->n_sub < 1 || c->n_sub > 64 ||
        !finite_pos(c->lambda_floor))
      return SMC2_EINVAL;
  }
  if (c->ppt != 0 && c->ppt != 1 && c->ppt != 2 && c->ppt != 4 && c->ppt != 8 && c->ppt != 16)
    return SMC2_EINVAL;
  if (c->pf_family < SMC2_PF_ANY || c->pf_family > SMC2_PF_FP32) return SMC2_EINVAL;
  if ((c->pf_scheme != SMC2_PF_SYSTEMATIC && c->pf_scheme != SMC2_PF_MULTINOMIAL) ||
      !(c->pf_ess_frac >= 0.0 && c->pf_ess_frac <= 1.0))
    return SMC2_EINVAL;
  const bool general = c->pf_scheme != SMC2_PF_SYSTEMATIC || c->pf_ess_frac > 0.0;
  if (general && c->ppt > 4) return SMC2_EINVAL;  // the variants run in the register-resident shapes
  if (c->cta_threads != 0 && (c->cta_threads < 32 || c->cta_threads > kPfMaxBlock || c->cta_threads % 32))
    return SMC2_EINVAL;
  const int nd = c->n_datasets <= 1 ? 1 : c->n_datasets;
  if (nd > SMC2_MAX_DATASETS) return SMC2_EINVAL;
  if (c->n_datasets > 1 && (!c->ds_N || !c->ds_M || !c->ds_T)) return SMC2_EINVAL;
  for (int d = 0; d < nd; ++d) {
    const int n = c->n_datasets > 1 ? c->ds_N[d] : c->N;
    const int m = c->n_datasets > 1 ? c->ds_M[d] : c->M;
    const int t = c->n_datasets > 1 ? c->ds_T[d] : c->T;
    if (n < 1 || n > SMC2_MAX_N || m < 1 || m > SMC2_MAX_M || t < 1 || t > (1 << 24))
      return SMC2_EINVAL;
    const int gt = pf_group_threads(c->ppt ? c->ppt : 16, m);
    if (gt > (c->cta_threads ? c->cta_threads : kPfMaxBlock)) return SMC2_EINVAL;
    // a filter's particles live in one CTA's shared memory: some shape must fit
    const int model = c->model;  // the internal model ids equal the ABI's
    bool fits = false;
    for (int ppt : {1, 2, 4, 8, 16}) {
      if ((c->ppt && ppt != c->ppt) || ((general || model == MODEL_SIR) && ppt > 4)) continue;
      const int g = pf_group_threads(ppt, m);
      if (g <= kPfMaxBlock && pf_smem_bytes(c->precision, model, ppt, general, g, m) <= 227 * 1024) fits = true;
    }
    if (!fits) return SMC2_EINVAL;
  }
  return SMC2_OK;
}

template <typename Tp>
Tp* carve(char*& p, size_t count) {
  p = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(p) + 255) & ~uintptr_t(255));
  Tp* r = reinterpret_cast<Tp*>(p);
  p += count * sizeof(Tp);
  return r;
}

size_t obs_bytes(const smc2_ctx* c, int d) {
  return (size_t)c->T[d] * 4 * (c->precision == SMC2_PREC_FP64 ? 8 : 4);
}

// Lay out (or size, when base == nullptr) the arena.
size_t layout(smc2_ctx* c, char* base) {
  char* p = base ? base : reinterpret_cast<char*>(uintptr_t(256));
  char* start = p;
  const int D = c->D;
  c->d_y = carve<double>(p, c->ytot);
  c->d_k = carve<int>(p, 4);
  c->d_status = carve<int>(p, 4);
  c->d_grid_ticket = carve<unsigned>(p, 4);
  c->d_wu_counter = carve<int>(p, 4);
  c->d_obs.assign(c->n_ds, nullptr);
  c->h_ds.assign(c->n_ds, DSDev{});
  for (int d = 0; d < c->n_ds; ++d) {
    DSDev& s = c->h_ds[d];
    const int N = c->N[d];
    s.N = N;
    s.M = c->M[d];
    s.T = c->T[d];
    s.nblk = c->nblk[d];
    s.nblk_res = c->nblk_res[d];
    s.logN = std::log((double)N);
    s.thA = carve<double>(p, (size_t)D * N);
    s.thB = carve<double>(p, (size_t)D * N);
    s.lpA = carve<double>(p, N);
    s.lpB = carve<double>(p, N);
    s.llA = carve<double>(p, N);
    s.llB = carve<double>(p, N);
    s.logw = carve<double>(p, N);
    s.logq = carve<double>(p, N);
    s.q = carve<uint64_t>(p, N);
    s.part = carve<double>(p, (size_t)s.nblk * kPartStride);
    s.part_st = carve<double>(p, (size_t)s.nblk * kStatStride);
    s.tickets = carve<unsigned>(p, 4);
    s.lk = carve<LKParams>(p, 1);
    s.cur = carve<IterCur>(p, 1);
    s.hist = carve<smc2_iter_stats>(p, c->K);
    s.rec = carve<double>(p, 1 + D + D * D);
    s.est_rec = carve<double>(p, D);
    c->d_obs[d] = carve<char>(p, obs_bytes(c, d));
    s.obs = c->d_obs[d];
    s.c2hi = (uint32_t)d << 20;
  }
  MlpDev& M = c->mlp;
  M = MlpDev{};
  if (c->cfg.proposal == SMC2_PROP_MLP) {
    const int P = mlp_param_count(D), N0 = c->N[0];
    M.on = 1;
    M.W = c->cfg.mlp_window;
    M.h = c->cfg.mlp_h;
    const size_t rows = (size_t)M.W * N0;
    M.p = carve<float>(p, P);
    M.p_use = carve<float>(p, P);
    M.norm_use = carve<MlpNorm>(p, 1);
    M.loss_use = carve<float>(p, 4);
    M.ring_rows = carve<int>(p, 4);
    M.m = carve<float>(p, P);
    M.v = carve<float>(p, P);
    M.step = carve<int>(p, 4);
    M.loss = carve<float>(p, 4);
    M.ring_th = carve<float>(p, rows * D);
    M.ring_lp = carve<float>(p, rows);
    M.xs = carve<float>(p, rows * D);
    M.ys = carve<float>(p, rows);
    M.norm = carve<MlpNorm>(p, 1);
    M.score = carve<double>(p, (size_t)D * N0);
  }
  c->d_ds = carve<DSDev>(p, c->n_ds);
  c->d_jobs = carve<PFJob>(p, c->n_ds);
  size_t wu_cap = 0;
  for (int n : c->N) wu_cap += (size_t)n;
  c->d_wus = carve<int4>(p, wu_cap);
  return (size_t)(p - start) + 256;
}

// A launch shape is valid when every dataset's filter group fits the CTA and,
// for groups wider than a warp, at most 15 groups share it (named barriers 1..15).
bool shape_valid(const smc2_ctx* c, int ppt, int block, bool named) {
  for (int m : c->M) {
    const int gt = pf_group_threads(ppt, m);
    if (gt > block) return false;
    if (gt == 32) continue;                       // one-warp groups: __syncwarp
    if (!named && gt != block) return false;      // wide group = the whole CTA
    if (named && (block / gt > 15 || block % gt)) return false;
  }
  return true;
}

void build_work_units(smc2_ctx* c, std::vector<int4>& wus) {
  wus.clear();
  for (int d = 0; d < c->n_ds; ++d) {
    const int gt = pf_group_threads(c->ppt, c->M[d]);
    const int fpc = std::max(1, c->pf_block / gt);
    for (int f = 0; f < c->N[d]; f += fpc) wus.push_back(make_int4(d, f, std::min(fpc, c->N[d] - f), 0));
  }
  // longest processing time first: cost ~ T * M * filters
  std::stable_sort(wus.begin(), wus.end(), [&](const int4& a, const int4& b) {
    const double ca = (double)c->T[a.x] * c->M[a.x] * a.z, cb = (double)c->T[b.x] * c->M[b.x] * b.z;
    return ca > cb;
  });
}

// The particle-filter launch of the context's shape, either kernel family.
cudaError_t ctx_pf_launch(const smc2_ctx* c, int grid, const PFLaunch& L, cudaStream_t s, bool trace = false) {
  if (c->pf_fast) return pf_fast_launch(c->model, c->ppt, trace, c->pf_named, grid, c->pf_block, c->pf_smem, L, s);
  return pf_launch(c->precision, c->model, c->ppt, c->pf_named, c->pf_general, grid, c->pf_block, c->pf_smem, L, s);
}

int ctx_pf_occupancy(const smc2_ctx* c, bool trace = false) {
  if (c->pf_fast) return pf_fast_occupancy(c->model, c->ppt, trace, c->pf_named, c->pf_block, c->pf_smem);
  return pf_occupancy(c->precision, c->model, c->ppt, c->pf_named, c->pf_general, c->pf_block, c->pf_smem);
}

// The FP32 filter of pf_fast.cuh at ppt.  When every dataset's filter group
// has the same width, one group is the CTA; otherwise (grouped) the CTA is as
// wide as the widest group and narrower groups share it: warps, or groups of
// several warps on named barriers 1..15.
bool fast_shape_valid(const smc2_ctx* c, int ppt, int* block, bool* grouped) {
  if (!pf_fast_eligible(c->precision, c->model, c->pf_general, ppt)) return false;
  int b = 32;
  bool gr = false;
  for (int m : c->M) b = std::max(b, pf_group_threads(ppt, m));
  for (int m : c->M) {
    const int gt = pf_group_threads(ppt, m);
    if (gt != b) gr = true;
    if (b % gt || (gt > 32 && b / gt > 15)) return false;
    if (pf_fast_smem_bytes(c->model, ppt, b, m) > 227 * 1024) return false;
  }
  if (b > kPfMaxBlock || (c->cfg.cta_threads && b != c->cfg.cta_threads)) return false;
  *block = b;
  *grouped = gr;
  return true;
}

smc2_status apply_shape(smc2_ctx* c, int ppt, int block, bool named, bool upload, bool fast = false) {
  c->ppt = ppt;
  c->pf_block = block;
  c->pf_named = named;
  c->pf_fast = fast;
  size_t smem = 0;
  for (int m : c->M)
    smem = std::max(smem, fast ? pf_fast_smem_bytes(c->model, ppt, block, m)
                               : pf_smem_bytes(c->precision, c->model, ppt, c->pf_general, block, m));
  if (smem > 227 * 1024) return SMC2_EINVAL;
  c->pf_smem = smem;
  if (fast)
    SMC2_TRY(pf_fast_configure(c->model, ppt, false, named, smem));
  else
    SMC2_TRY(pf_configure(c->precision, c->model, ppt, named, c->pf_general, smem));
  std::vector<int4> wus;
  build_work_units(c, wus);
  c->n_wus = (int)wus.size();
  const int occ = ctx_pf_occupancy(c);
  if (occ < 1) return SMC2_EINVAL;
  c->pf_grid = std::min(c->n_wus, occ * c->sms);
  c->pl.n_wu = c->n_wus;
  if (upload)
    SMC2_TRY(cudaMemcpyAsync(c->d_wus, wus.data(), wus.size() * sizeof(int4), cudaMemcpyHostToDevice,
                             c->stream));
  return SMC2_OK;
}

// With the learned proposal, the training cluster runs beside the particle
// filter and holds part of its SMs (registers, shared memory and threads of one
// CTA each).  A shape whose work units fit in one wave of the whole GPU but not
// beside the cluster would run a second wave of whole filters every iteration,
// so the tuner weighs its time by the ratio of waves with and without the
// cluster.
float training_wave_factor(const smc2_ctx* c) {
  int ctas = 0, threads = 0, regs = 0;
  size_t smem = 0;
  if (mlp_train_footprint(&ctas, &threads, &regs, &smem) != cudaSuccess || ctas < 1) return 1.f;
  const int occ = ctx_pf_occupancy(c);
  const int beside = c->pf_fast ? pf_fast_blocks_beside(c->model, c->ppt, c->pf_named, c->pf_block, c->pf_smem,
                                                        threads, regs, smem)
                                : pf_blocks_beside(c->precision, c->model, c->ppt, c->pf_named, c->pf_general,
                                                   c->pf_block, c->pf_smem, threads, regs, smem);
  const long full = (long)occ * c->sms;
  const long with = (long)occ * (c->sms - ctas) + (long)std::min(occ, beside) * ctas;
  if (full < 1 || with < 1) return 1.f;
  const long w_full = (c->n_wus + full - 1) / full, w_with = (c->n_wus + with - 1) / with;
  return (float)w_with / (float)w_full;
}

// Launch-shape tuner: time every valid (particles per thread, CTA threads) pair
// on the context's own work list (prior draws of theta, min(T, 32) steps), then
// the few within 15 % of the fastest again, over min(T, 64) steps, in turn.
smc2_status choose_launch_shape(smc2_ctx* c) {
  const TraceRange range("smc2 launch-shape tuner");
  struct Shape {
    int ppt, block;
    bool named, fast;
  };
  std::vector<Shape> cand;
  for (int ppt : {2, 4, 8}) {  // the FP32 filter of pf_fast.cuh
    int block = 0;
    bool grouped = false;
    if (c->cfg.pf_family != SMC2_PF_GROUPS && (!c->cfg.ppt || ppt == c->cfg.ppt) &&
        fast_shape_valid(c, ppt, &block, &grouped))
      cand.push_back({ppt, block, grouped, true});
  }
  for (int ppt : {1, 2, 4, 8, 16}) {
    if (c->cfg.ppt && ppt != c->cfg.ppt) continue;
    if ((c->pf_general || c->model == MODEL_SIR) && ppt > 4) continue;  // register-resident shapes only
    if (c->cfg.pf_family == SMC2_PF_FP32) break;
    for (int block = 32; block <= kPfMaxBlock; block += 32) {
      if (c->cfg.cta_threads && block != c->cfg.cta_threads) continue;
      if (!c->cfg.cta_threads && (block & (block - 1))) continue;  // powers of two when tuning
      if (shape_valid(c, ppt, block, false))
        cand.push_back({ppt, block, false, false});
      else if (shape_valid(c, ppt, block, true))
        cand.push_back({ppt, block, true, false});
    }
  }
  if (cand.empty()) return SMC2_EINVAL;
  if (cand.size() == 1) return apply_shape(c, cand[0].ppt, cand[0].block, cand[0].named, true, cand[0].fast);
  cudaStream_t s = c->stream;
  SMC2_TRY(outer_propose(c->op, c->max_nblk, s));  // k = 1: prior draws into the proposal buffers
  cudaEvent_t e0, e1;
  SMC2_TRY(cudaEventCreate(&e0));
  SMC2_TRY(cudaEventCreate(&e1));
  // one launch of the applied shape over t_cap steps; < 0 on failure
  auto time_launch = [&](int t_cap) -> float {
    PFLaunch L = c->pl;
    L.t_cap = t_cap;
    float ms = 0.f;
    const bool ok = cudaMemsetAsync(c->d_wu_counter, 0, sizeof(int), s) == cudaSuccess &&
                    cudaEventRecord(e0, s) == cudaSuccess && ctx_pf_launch(c, c->pf_grid, L, s) == cudaSuccess &&
                    cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                    cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    c->kernel_launches++;
    cudaGetLastError();
    return ok ? ms : -1.f;
  };
  // first pass: one warm-up launch, then the best of two over 32 steps
  std::vector<std::pair<float, size_t>> timed;
  for (size_t ci = 0; ci < cand.size(); ++ci) {
    const auto& cb = cand[ci];
    if (apply_shape(c, cb.ppt, cb.block, cb.named, true, cb.fast) != SMC2_OK) continue;
    float cand_best = 1e30f;
    bool ok = time_launch(4) >= 0.f;
    for (int rep = 0; rep < 2 && ok; ++rep) {
      const float ms = time_launch(32);
      ok = ms >= 0.f;
      if (ok) cand_best = std::min(cand_best, ms);
    }
    if (!ok) continue;
    if (c->mlp.on) cand_best *= training_wave_factor(c);
    timed.push_back({cand_best, ci});
  }
  if (timed.empty()) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return SMC2_EINVAL;
  }
  std::sort(timed.begin(), timed.end());
  // second pass: the shapes within 15 % of the fastest, timed in turn over 64 steps
  // five times each (interleaved, so that a clock ramp touches them alike); the
  // smallest median wins
  std::vector<size_t> fin;
  for (const auto& tc : timed)
    if (fin.size() < 3 && tc.first <= 1.15f * timed[0].first) fin.push_back(tc.second);
  size_t pick_i = timed[0].second;
  if (fin.size() > 1) {
    std::vector<std::vector<float>> ts(fin.size());
    for (int rep = 0; rep < 5; ++rep)
      for (size_t f = 0; f < fin.size(); ++f) {
        const auto& cb = cand[fin[f]];
        if (apply_shape(c, cb.ppt, cb.block, cb.named, true, cb.fast) != SMC2_OK) continue;
        const float ms = time_launch(64);
        if (ms >= 0.f) ts[f].push_back(c->mlp.on ? ms * training_wave_factor(c) : ms);
      }
    float best = 1e30f;
    for (size_t f = 0; f < fin.size(); ++f) {
      if (ts[f].size() < 3) continue;
      std::sort(ts[f].begin(), ts[f].end());
      const float med = ts[f][ts[f].size() / 2];
      if (med < best) {
        best = med;
        pick_i = fin[f];
      }
    }
  }
  const Shape pick = cand[pick_i];
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return apply_shape(c, pick.ppt, pick.block, pick.named, true, pick.fast);
}

smc2_status clear_run_state(smc2_ctx* c) {
  cudaStream_t s = c->stream;
  SMC2_TRY(cudaMemsetAsync(c->d_k, 0, 4 * sizeof(int), s));
  SMC2_TRY(cudaMemsetAsync(c->d_status, 0, 4 * sizeof(int), s));
  SMC2_TRY(cudaMemsetAsync(c->d_grid_ticket, 0, 4 * sizeof(unsigned), s));
  for (int d = 0; d < c->n_ds; ++d) {
    const DSDev& ds = c->h_ds[d];
    SMC2_TRY(cudaMemsetAsync(ds.tickets, 0, 4 * sizeof(unsigned), s));
    SMC2_TRY(cudaMemsetAsync(ds.hist, 0, (size_t)c->K * sizeof(smc2_iter_stats), s));
    SMC2_TRY(cudaMemsetAsync(ds.rec, 0, (size_t)(1 + c->D + c->D * c->D) * sizeof(double), s));
    SMC2_TRY(cudaMemsetAsync(ds.est_rec, 0, (size_t)c->D * sizeof(double), s));
    SMC2_TRY(cudaMemsetAsync(ds.cur, 0, sizeof(IterCur), s));
    SMC2_TRY(cudaMemsetAsync(ds.lk, 0, sizeof(LKParams), s));
  }
  if (c->mlp.on) {
    SMC2_TRY(mlp_init_launch(c->mlp, c->D, c->cfg.seed, s));
    for (float* l : {c->mlp.loss, c->mlp.loss_use})  // NaN: no trained network yet
      SMC2_TRY(cudaMemsetAsync(l, 0xff, 4 * sizeof(float), s));
    for (MlpNorm* nm : {c->mlp.norm, c->mlp.norm_use}) SMC2_TRY(cudaMemsetAsync(nm, 0, sizeof(MlpNorm), s));
    SMC2_TRY(cudaMemsetAsync(c->mlp.ring_rows, 0, 4 * sizeof(int), s));
    c->kernel_launches++;
  }
  c->k_host = 0;
  return SMC2_OK;
}

smc2_status compute_obs(smc2_ctx* c, cudaStream_t s) {
  for (int d = 0; d < c->n_ds; ++d) {
    SMC2_TRY(outer_obs_terms(c->precision, c->model, c->d_y + c->yoff[d], c->T[d], c->d_obs[d], s));
    c->kernel_launches++;
  }
  return SMC2_OK;
}

void fill_params(smc2_ctx* c) {
  OuterParams& P = c->op;
  P.ds = c->d_ds;
  P.n_ds = c->n_ds;
  P.D = c->D;
  P.lkernel = c->cfg.lkernel == SMC2_LK_GAUSS_OPT ? LK_GAUSS : LK_FORWARD;
  P.K = c->K;
  P.rw_scale = c->cfg.rw_scale;
  P.ess_frac = c->cfg.ess_frac;
  for (int d = 0; d < 8; ++d) {
    P.prior_mean[d] = c->cfg.prior_mean[d];
    P.prior_sd[d] = c->cfg.prior_sd[d];
    P.inv_prior_sd[d] = d < c->D ? 1.0 / c->cfg.prior_sd[d] : 0.0;
    P.log_prior_sd[d] = d < c->D ? std::log(c->cfg.prior_sd[d]) : 0.0;
    P.prior_lo[d] = c->cfg.prior_lo[d];
    P.prior_hi[d] = c->cfg.prior_hi[d];
    P.log_prior_width[d] =
        (d < c->D && c->cfg.prior_kind == SMC2_PRIOR_UNIFORM) ? std::log(c->cfg.prior_hi[d] - c->cfg.prior_lo[d]) : 0.0;
  }
  P.prior_kind = c->cfg.prior_kind;
  P.inv_rw = 1.0 / c->cfg.rw_scale;
  P.log_rw = std::log(c->cfg.rw_scale);
  P.seed = c->cfg.seed;
  P.k_done = c->d_k;
  P.status = c->d_status;
  P.grid_ticket = c->d_grid_ticket;
  P.mlp = c->mlp;
  P.ds_N0 = c->N[0];

  PFLaunch& L = c->pl;
  L.jobs = c->d_jobs;
  L.wus = c->d_wus;
  L.n_wu = c->n_wus;
  L.fpc_single = 0;
  L.wu_counter = c->d_wu_counter;
  L.seed = c->cfg.seed;
  philox_round_keys(c->cfg.seed, L.rk);
  L.k_done = c->d_k;
  L.k_imm = 0;
  L.status = c->d_status;
  L.mdl.npop = c->cfg.npop;
  L.mdl.e0 = c->cfg.e0;
  L.mdl.i0 = c->cfg.i0;
  L.mdl.lambda_floor = c->cfg.lambda_floor;
  L.mdl.n_sub = c->cfg.n_sub;
  L.mdl.pf_scheme = c->cfg.pf_scheme;
  L.mdl.pf_ess_frac = c->cfg.pf_ess_frac;
}

// One iteration of every dataset, enqueued on s; the L-kernel fit runs on the
// side stream between a fork after the proposal and a join before the weights.
// With the learned proposal, the network is trained on the train stream from
// after this iteration's weights to after the next iteration's weights, beside
// the next proposal and particle filter; the trained state is then published
// for the iteration after that.  Every iteration therefore proposes with the
// network trained on the pairs of iterations up to k - 2, however the
// iterations are grouped into calls.
cudaError_t join_training(smc2_ctx* c, cudaStream_t s) {
  const bool pending = c->train_pending;
  c->train_pending = false;
  return pending ? cudaStreamWaitEvent(s, c->ev_tjoin, 0) : cudaSuccess;
}

smc2_status enqueue_iteration(smc2_ctx* c, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1) {
  if (c->mlp.on) SMC2_TRY(mlp_score_launch(c->op, c->N[0], s));
  SMC2_TRY(outer_propose(c->op, c->max_nblk, s));
  SMC2_TRY(cudaEventRecord(c->ev_fork, s));
  SMC2_TRY(cudaStreamWaitEvent(c->side_stream, c->ev_fork, 0));
  SMC2_TRY(outer_lkfit(c->op, c->side_stream));
  SMC2_TRY(cudaEventRecord(c->ev_join, c->side_stream));
  SMC2_TRY(cudaMemsetAsync(c->d_wu_counter, 0, sizeof(int), s));
  if (ev0) SMC2_TRY(cudaEventRecordWithFlags(ev0, s, cudaEventRecordExternal));
  SMC2_TRY(ctx_pf_launch(c, c->pf_grid, c->pl, s));
  if (ev1) SMC2_TRY(cudaEventRecordWithFlags(ev1, s, cudaEventRecordExternal));
  SMC2_TRY(cudaStreamWaitEvent(s, c->ev_join, 0));
  SMC2_TRY(outer_weights(c->op, c->max_nblk, s));
  if (c->mlp.on) {
    SMC2_TRY(join_training(c, s));
    SMC2_TRY(mlp_publish_launch(c->op, s));
    SMC2_TRY(mlp_append_launch(c->op, c->N[0], s));
    SMC2_TRY(cudaEventRecord(c->ev_tfork, s));
    SMC2_TRY(cudaStreamWaitEvent(c->train_stream, c->ev_tfork, 0));
    SMC2_TRY(mlp_train_launch(c->op, c->cfg.mlp_steps, (float)c->cfg.mlp_lr, c->train_stream));
    SMC2_TRY(cudaEventRecord(c->ev_tjoin, c->train_stream));
    c->train_pending = true;
  }
  SMC2_TRY(outer_quantise(c->op, c->max_nblk, s));
  SMC2_TRY(outer_resample(c->op, c->max_nblk_res, c->max_N, s));
  return SMC2_OK;
}

int launches_per_iteration(const smc2_ctx* c) {
  return 6 + (c->mlp.on ? 4 : 0);  // score, publish, append, training
}


smc2_status get_graph(smc2_ctx* c, int n_iter, TimedGraph** out) {
  const GraphKey key{n_iter, c->timing ? 1 : 0};
  auto it = c->graphs.find(key);
  if (it != c->graphs.end()) {
    *out = &it->second;
    return SMC2_OK;
  }
  TimedGraph g;
  if (c->timing) {
    g.ev.resize(2 * (size_t)n_iter);
    for (auto& e : g.ev) SMC2_TRY(cudaEventCreate(&e));
  }
  SMC2_TRY(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  smc2_status st = SMC2_OK;
  for (int it2 = 0; it2 < n_iter && st == SMC2_OK; ++it2)
    st = enqueue_iteration(c, c->cap_stream, c->timing ? g.ev[2 * it2] : nullptr,
                           c->timing ? g.ev[2 * it2 + 1] : nullptr);
  const cudaError_t ej = join_training(c, c->cap_stream);  // no branch outlives the graph
  if (st == SMC2_OK && ej != cudaSuccess) st = record_cuda(ej, "join_training");
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
  if (st != SMC2_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  SMC2_TRY(e);
  e = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  SMC2_TRY(e);
  auto ins = c->graphs.emplace(key, std::move(g));
  *out = &ins.first->second;
  return SMC2_OK;
}

void drop_graphs(smc2_ctx* c) {
  for (auto& kv : c->graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    for (auto e : kv.second.ev) cudaEventDestroy(e);
  }
  c->graphs.clear();
}

smc2_status sticky(smc2_ctx* c) {
  int bits = 0;
  SMC2_TRY(cudaMemcpyAsync(&bits, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  SMC2_TRY(cudaStreamSynchronize(c->stream));
  return status_from_bits(bits);
}

bool bad_ds(const smc2_ctx* c, int d) { return !c || d < 0 || d >= c->n_ds; }

}  // namespace

extern "C" {

const char* smc2_last_error_string(void) { return g_last_error; }

const char* smc2_status_string(smc2_status s) {
  switch (s) {
    case SMC2_OK: return "ok";
    case SMC2_EINVAL: return "invalid argument";
    case SMC2_ENOMEM: return "out of memory";
    case SMC2_ECUDA: return "CUDA runtime error";
    case SMC2_ENONFINITE: return "every importance weight is zero or not finite";
    case SMC2_ECHOL: return "covariance factorisation failed";
    case SMC2_ETIMEOUT: return "reserved (never returned)";
    case SMC2_EBOUNDS: return "reserved (never returned)";
    case SMC2_ESTATE: return "call not valid in the current state";
  }
  return "unknown status";
}

smc2_status smc2_init(const smc2_config* cfg, const double* y, void* stream, smc2_ctx** out) {
  const TraceRange range("smc2_init");
  if (!out || !y) return SMC2_EINVAL;
  smc2_status st = validate(cfg);
  if (st != SMC2_OK) return st;
  smc2_ctx* c = new (std::nothrow) smc2_ctx();
  if (!c) return SMC2_ENOMEM;
  c->cfg = *cfg;
  c->pf_general = cfg->pf_scheme != SMC2_PF_SYSTEMATIC || cfg->pf_ess_frac > 0.0;
  if (c->cfg.mlp_h == 0.0) c->cfg.mlp_h = kMlpStep;
  if (c->cfg.mlp_lr == 0.0) c->cfg.mlp_lr = kMlpLr;
  if (c->cfg.mlp_steps == 0) c->cfg.mlp_steps = kMlpSteps;
  if (c->cfg.mlp_window == 0) c->cfg.mlp_window = kMlpWindow;
  c->n_ds = cfg->n_datasets <= 1 ? 1 : cfg->n_datasets;
  c->D = cfg->D;
  c->K = cfg->K;
  c->precision = cfg->precision;
  c->model = cfg->model;  // the internal model ids equal the ABI's
  for (int d = 0; d < c->n_ds; ++d) {
    c->N.push_back(cfg->n_datasets > 1 ? cfg->ds_N[d] : cfg->N);
    c->M.push_back(cfg->n_datasets > 1 ? cfg->ds_M[d] : cfg->M);
    c->T.push_back(cfg->n_datasets > 1 ? cfg->ds_T[d] : cfg->T);
    c->nblk.push_back((c->N[d] + kOuterBlock - 1) / kOuterBlock);
    c->nblk_res.push_back((c->N[d] + kResBlock - 1) / kResBlock);
    c->max_nblk_res = std::max(c->max_nblk_res, c->nblk_res[d]);
    c->yoff.push_back(c->ytot);
    c->ytot += c->T[d];
    c->max_N = std::max(c->max_N, c->N[d]);
    c->max_nblk = std::max(c->max_nblk, c->nblk[d]);
  }
  c->cfg.ds_N = c->cfg.ds_M = c->cfg.ds_T = nullptr;
  c->stream = static_cast<cudaStream_t>(stream);
  auto fail = [&](smc2_status s) {
    smc2_destroy(c);
    return s;
  };
  if (cudaGetDevice(&c->device) != cudaSuccess) return fail(SMC2_ECUDA);
  if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
    return fail(SMC2_ECUDA);
  if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->train_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_tfork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_tjoin, cudaEventDisableTiming) != cudaSuccess)
    return fail(SMC2_ECUDA);

  c->arena_bytes = layout(c, nullptr);
  if (cudaMalloc(&c->arena, c->arena_bytes) != cudaSuccess) return fail(SMC2_ENOMEM);
  layout(c, c->arena);

  std::vector<PFJob> jobs(c->n_ds);
  c->n_wus = 0;
  for (int d = 0; d < c->n_ds; ++d) {
    PFJob& j = jobs[d];
    j.theta = c->h_ds[d].thB;
    j.ld = c->N[d];
    j.n = c->N[d];
    j.M = c->M[d];
    j.T = c->T[d];
    j.loglik = c->h_ds[d].llB;
    j.delta = nullptr;
    j.anc = nullptr;
    j.obs = c->d_obs[d];
    j.c2hi = c->h_ds[d].c2hi;
  }
  cudaStream_t s = c->stream;
  if (cudaMemcpyAsync(c->d_y, y, c->ytot * sizeof(double), cudaMemcpyDefault, s) != cudaSuccess ||
      cudaMemcpyAsync(c->d_ds, c->h_ds.data(), c->n_ds * sizeof(DSDev), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(c->d_jobs, jobs.data(), c->n_ds * sizeof(PFJob), cudaMemcpyHostToDevice, s) !=
          cudaSuccess)
    return fail(SMC2_ECUDA);
  if ((st = clear_run_state(c)) != SMC2_OK) return fail(st);
  if ((st = compute_obs(c, s)) != SMC2_OK) return fail(st);
  fill_params(c);
  if ((st = choose_launch_shape(c)) != SMC2_OK) return fail(st);
  if ((st = clear_run_state(c)) != SMC2_OK) return fail(st);
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail(SMC2_ECUDA);
  *out = c;
  return SMC2_OK;
}

smc2_status smc2_set_observations(smc2_ctx* c, const double* y) {
  if (!c || !y) return SMC2_EINVAL;
  SMC2_TRY(cudaMemcpyAsync(c->d_y, y, c->ytot * sizeof(double), cudaMemcpyDefault, c->stream));
  return compute_obs(c, c->stream);
}

smc2_status smc2_reset(smc2_ctx* c, uint64_t seed) {
  if (!c) return SMC2_EINVAL;
  if (seed != c->cfg.seed) {
    drop_graphs(c);
    c->cfg.seed = seed;
    fill_params(c);
  }
  return clear_run_state(c);
}

static smc2_status pf_standalone(smc2_ctx* c, const double* theta, int n, int iteration, int dataset,
                                 double* loglik, double* delta, int32_t* anc, float* xtr = nullptr,
                                 float* ltr = nullptr, uint64_t* qtr = nullptr) {
  const TraceRange range("smc2 particle filter");
  if (!c || !theta || !loglik || n < 1 || n > SMC2_MAX_N || bad_ds(c, dataset) || iteration < 0 ||
      iteration >= (1 << 28))
    return SMC2_EINVAL;
  const bool states = xtr || ltr || qtr;
  if (states) {
    if (!xtr || !ltr || !qtr) return SMC2_EINVAL;
    if (!pf_fast_eligible(c->precision, c->model, c->pf_general, c->ppt)) return SMC2_EINVAL;
  }
  // the FP32 filter writes increments and ancestors only in its traced instantiation
  const bool trace = states || (c->pf_fast && (delta || anc));
  PFJob job{};
  job.xtr = xtr;
  job.ltr = ltr;
  job.qtr = qtr;
  job.theta = theta;
  job.ld = n;
  job.n = n;
  job.M = c->M[dataset];
  job.T = c->T[dataset];
  job.loglik = loglik;
  job.delta = delta;
  job.anc = anc;
  job.obs = c->d_obs[dataset];
  job.c2hi = (uint32_t)dataset << 20;
  // the job travels inside the kernel's parameter block
  PFLaunch L = c->pl;
  L.jobs = nullptr;
  L.job0 = job;
  const int gt = pf_group_threads(c->ppt, job.M);
  L.fpc_single = std::max(1, c->pf_block / gt);
  L.wus = nullptr;
  L.n_wu = (n + L.fpc_single - 1) / L.fpc_single;
  L.wu_counter = nullptr;
  L.k_done = nullptr;
  L.k_imm = iteration;
  if (trace) {  // the traced FP32 filter at the context's ppt, one filter group per CTA
    const int block = pf_group_threads(c->ppt, job.M);
    const size_t smem = pf_fast_smem_bytes(c->model, c->ppt, block, job.M);
    SMC2_TRY(pf_fast_configure(c->model, c->ppt, true, false, smem));
    L.fpc_single = 1;
    L.n_wu = n;
    const int occ = std::max(1, pf_fast_occupancy(c->model, c->ppt, true, false, block, smem));
    SMC2_TRY(pf_fast_launch(c->model, c->ppt, true, false, std::min(n, occ * c->sms), block, smem, L, c->stream));
    c->kernel_launches++;
    return SMC2_OK;
  }
  const int occ = std::max(1, ctx_pf_occupancy(c, trace));
  const int grid = std::min(L.n_wu, occ * c->sms);
  SMC2_TRY(ctx_pf_launch(c, grid, L, c->stream, trace));
  c->kernel_launches++;
  return SMC2_OK;
}

smc2_status smc2_pf_loglik(smc2_ctx* c, const double* theta, int n, int iteration, int dataset,
                           double* loglik) {
  return pf_standalone(c, theta, n, iteration, dataset, loglik, nullptr, nullptr);
}

smc2_status smc2_pf_trace(smc2_ctx* c, const double* theta, int n, int iteration, int dataset,
                          double* loglik, double* delta, int32_t* anc) {
  return pf_standalone(c, theta, n, iteration, dataset, loglik, delta, anc);
}

smc2_status smc2_pf_trace_states(smc2_ctx* c, const double* theta, int n, int iteration, int dataset,
                                 double* loglik, double* delta, int32_t* anc, float* x, float* logw,
                                 uint64_t* q) {
  if (!x || !logw || !q) return SMC2_EINVAL;
  return pf_standalone(c, theta, n, iteration, dataset, loglik, delta, anc, x, logw, q);
}

smc2_status smc2_run(smc2_ctx* c, int n_iter, smc2_iter_stats* stats_host) {
  const TraceRange range("smc2_run");
  if (!c || n_iter < 1) return SMC2_EINVAL;
  if (c->k_host + n_iter > c->K) return SMC2_ESTATE;
  TimedGraph* g = nullptr;
  smc2_status st = get_graph(c, n_iter, &g);
  if (st != SMC2_OK) return st;
  SMC2_TRY(cudaGraphLaunch(g->exec, c->stream));
  const int k0 = c->k_host;
  c->k_host += n_iter;
  c->kernel_launches += (int64_t)launches_per_iteration(c) * n_iter;
  if (c->timing) {
    SMC2_TRY(cudaStreamSynchronize(c->stream));
    for (int i = 0; i < n_iter; ++i) {
      float ms = 0.f;
      SMC2_TRY(cudaEventElapsedTime(&ms, g->ev[2 * i], g->ev[2 * i + 1]));
      c->pf_ms += ms;
      c->pf_launches++;
    }
  }
  if (stats_host) {
    for (int d = 0; d < c->n_ds; ++d)
      for (int i = 0; i < n_iter; ++i)
        SMC2_TRY(cudaMemcpyAsync(stats_host + (size_t)i * c->n_ds + d, c->h_ds[d].hist + k0 + i,
                                 sizeof(smc2_iter_stats), cudaMemcpyDeviceToHost, c->stream));
    return sticky(c);
  }
  return SMC2_OK;
}

smc2_status smc2_iterate(smc2_ctx* c, smc2_iter_stats* stats_host) {
  return smc2_run(c, 1, stats_host);
}

smc2_status smc2_estimate(smc2_ctx* c, int dataset, double* mean_host, double* logz_host,
                          double* ess_sum_host, double* cov_host) {
  if (bad_ds(c, dataset)) return SMC2_EINVAL;
  if (c->k_host < 1) return SMC2_ESTATE;
  const DSDev& s = c->h_ds[dataset];
  const int D = c->D;
  smc2_iter_stats last;
  std::vector<double> rec((size_t)1 + D + D * D);
  SMC2_TRY(cudaMemcpyAsync(&last, s.hist + (c->k_host - 1), sizeof(last), cudaMemcpyDeviceToHost, c->stream));
  SMC2_TRY(cudaMemcpyAsync(rec.data(), s.rec, rec.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  const smc2_status st = sticky(c);
  const double l = rec[0];
  // recycled mean and covariance: the l_k-weighted first and second moments (Eq. 29)
  for (int d = 0; d < D; ++d) {
    const double md = rec[1 + d] / l;
    if (mean_host) mean_host[d] = md;
    if (cov_host)
      for (int e = 0; e < D; ++e) cov_host[d * D + e] = rec[1 + D + d * D + e] / l - md * (rec[1 + e] / l);
  }
  if (logz_host) *logz_host = last.logz;
  if (ess_sum_host) *ess_sum_host = l;
  return st;
}

smc2_status smc2_get_history(smc2_ctx* c, int dataset, smc2_iter_stats* hist, int cap, int* k_out) {
  if (bad_ds(c, dataset) || !hist || cap < 0) return SMC2_EINVAL;
  const int k = std::min(c->k_host, cap);
  if (k > 0)
    SMC2_TRY(cudaMemcpyAsync(hist, c->h_ds[dataset].hist, (size_t)k * sizeof(smc2_iter_stats),
                             cudaMemcpyDeviceToHost, c->stream));
  if (k_out) *k_out = c->k_host;
  return sticky(c);
}

smc2_status smc2_get_state(smc2_ctx* c, int dataset, int* k_out, double* theta, double* lp,
                           double* ll, double* lw) {
  if (bad_ds(c, dataset)) return SMC2_EINVAL;
  const DSDev& s = c->h_ds[dataset];
  const int N = s.N, D = c->D;
  std::vector<double> soa((size_t)D * N);
  SMC2_TRY(cudaMemcpyAsync(soa.data(), s.thA, soa.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (lp) SMC2_TRY(cudaMemcpyAsync(lp, s.lpA, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (ll) SMC2_TRY(cudaMemcpyAsync(ll, s.llA, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (lw) SMC2_TRY(cudaMemcpyAsync(lw, s.logw, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  smc2_status st = sticky(c);
  if (theta)
    for (int i = 0; i < N; ++i)
      for (int d = 0; d < D; ++d) theta[(size_t)i * D + d] = soa[(size_t)d * N + i];
  if (k_out) *k_out = c->k_host;
  return st;
}

smc2_status smc2_get_proposals(smc2_ctx* c, int dataset, double* theta, double* logq) {
  if (bad_ds(c, dataset)) return SMC2_EINVAL;
  const DSDev& s = c->h_ds[dataset];
  const int N = s.N, D = c->D;
  std::vector<double> soa((size_t)D * N);
  if (theta)
    SMC2_TRY(cudaMemcpyAsync(soa.data(), s.thB, soa.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (logq) SMC2_TRY(cudaMemcpyAsync(logq, s.logq, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  const smc2_status st = sticky(c);
  if (theta)
    for (int i = 0; i < N; ++i)
      for (int d = 0; d < D; ++d) theta[(size_t)i * D + d] = soa[(size_t)d * N + i];
  return st;
}

smc2_status smc2_get_learned_state(smc2_ctx* c, float* params, double* stdz, double* L, int* pop_ok) {
  if (!c || !c->mlp.on) return SMC2_EINVAL;
  const int D = c->D;
  MlpNorm nm{};
  float loss = 0.f;
  IterCur cur{};
  if (params)
    SMC2_TRY(cudaMemcpyAsync(params, c->mlp.p_use, (size_t)mlp_param_count(D) * sizeof(float),
                             cudaMemcpyDeviceToHost, c->stream));
  SMC2_TRY(cudaMemcpyAsync(&nm, c->mlp.norm_use, sizeof(MlpNorm), cudaMemcpyDeviceToHost, c->stream));
  SMC2_TRY(cudaMemcpyAsync(&loss, c->mlp.loss_use, sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  SMC2_TRY(cudaMemcpyAsync(&cur, c->h_ds[0].cur, sizeof(IterCur), cudaMemcpyDeviceToHost, c->stream));
  const smc2_status st = sticky(c);
  if (stdz) {
    for (int d = 0; d < D; ++d) {
      stdz[d] = nm.mu[d];
      stdz[D + d] = nm.sd[d];
    }
    stdz[2 * D] = nm.tau;
    stdz[2 * D + 1] = nm.zmean;
    stdz[2 * D + 2] = nm.zsd;
    stdz[2 * D + 3] = nm.var_y;
    stdz[2 * D + 4] = loss;
    stdz[2 * D + 5] = nm.ymax;
  }
  if (L)
    for (int d = 0; d < D; ++d)
      for (int f = 0; f < D; ++f) L[d * D + f] = cur.Lpop[d * kMaxD + f];
  if (pop_ok) *pop_ok = cur.pop_ok;
  return st;
}

smc2_status smc2_get_learned_training(smc2_ctx* c, float* params, float* m, float* v, int* step, double* stdz,
                                      float* ring_th, float* ring_lp, int* ring_rows) {
  if (!c || !c->mlp.on) return SMC2_EINVAL;
  const int D = c->D;
  const size_t P = (size_t)mlp_param_count(D), rows = (size_t)c->mlp.W * c->N[0];
  cudaStream_t s = c->stream;
  MlpNorm nm{};
  float loss = 0.f;
  int hs = 0, hr = 0;
  if (params) SMC2_TRY(cudaMemcpyAsync(params, c->mlp.p, P * sizeof(float), cudaMemcpyDeviceToHost, s));
  if (m) SMC2_TRY(cudaMemcpyAsync(m, c->mlp.m, P * sizeof(float), cudaMemcpyDeviceToHost, s));
  if (v) SMC2_TRY(cudaMemcpyAsync(v, c->mlp.v, P * sizeof(float), cudaMemcpyDeviceToHost, s));
  if (ring_th) SMC2_TRY(cudaMemcpyAsync(ring_th, c->mlp.ring_th, rows * D * sizeof(float), cudaMemcpyDeviceToHost, s));
  if (ring_lp) SMC2_TRY(cudaMemcpyAsync(ring_lp, c->mlp.ring_lp, rows * sizeof(float), cudaMemcpyDeviceToHost, s));
  SMC2_TRY(cudaMemcpyAsync(&hs, c->mlp.step, sizeof(int), cudaMemcpyDeviceToHost, s));
  SMC2_TRY(cudaMemcpyAsync(&hr, c->mlp.ring_rows, sizeof(int), cudaMemcpyDeviceToHost, s));
  SMC2_TRY(cudaMemcpyAsync(&nm, c->mlp.norm, sizeof(MlpNorm), cudaMemcpyDeviceToHost, s));
  SMC2_TRY(cudaMemcpyAsync(&loss, c->mlp.loss, sizeof(float), cudaMemcpyDeviceToHost, s));
  const smc2_status st = sticky(c);
  if (step) *step = hs;
  if (ring_rows) *ring_rows = hr;
  if (stdz) {
    for (int d = 0; d < D; ++d) {
      stdz[d] = nm.mu[d];
      stdz[D + d] = nm.sd[d];
    }
    stdz[2 * D] = nm.tau;
    stdz[2 * D + 1] = nm.zmean;
    stdz[2 * D + 2] = nm.zsd;
    stdz[2 * D + 3] = nm.var_y;
    stdz[2 * D + 4] = loss;
    stdz[2 * D + 5] = nm.ymax;
  }
  return st;
}

smc2_status smc2_set_state(smc2_ctx* c, int dataset, int k, const double* theta, const double* lp,
                           const double* ll, const double* lw) {
  if (bad_ds(c, dataset) || !theta || !lp || !ll || !lw || k < 0 || k > c->K) return SMC2_EINVAL;
  DSDev& s = c->h_ds[dataset];
  const int N = s.N, D = c->D;
  std::vector<double> soa((size_t)D * N);
  for (int i = 0; i < N; ++i)
    for (int d = 0; d < D; ++d) soa[(size_t)d * N + i] = theta[(size_t)i * D + d];
  cudaStream_t st = c->stream;
  SMC2_TRY(cudaMemcpyAsync(s.thA, soa.data(), soa.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  SMC2_TRY(cudaMemcpyAsync(s.lpA, lp, N * sizeof(double), cudaMemcpyHostToDevice, st));
  SMC2_TRY(cudaMemcpyAsync(s.llA, ll, N * sizeof(double), cudaMemcpyHostToDevice, st));
  SMC2_TRY(cudaMemcpyAsync(s.logw, lw, N * sizeof(double), cudaMemcpyHostToDevice, st));
  SMC2_TRY(outer_parent_reference(c->op, dataset, st));
  c->kernel_launches++;
  if (dataset == 0) {
    SMC2_TRY(cudaMemcpyAsync(c->d_k, &k, sizeof(int), cudaMemcpyHostToDevice, st));
    c->k_host = k;
  }
  return cudaStreamSynchronize(st) == cudaSuccess ? SMC2_OK : SMC2_ECUDA;
}

smc2_status smc2_set_history(smc2_ctx* c, int dataset, const smc2_iter_stats* hist, int k) {
  if (bad_ds(c, dataset) || k < 0 || k > c->K || (k > 0 && !hist)) return SMC2_EINVAL;
  const DSDev& s = c->h_ds[dataset];
  if (k > 0)
    SMC2_TRY(cudaMemcpyAsync(s.hist, hist, (size_t)k * sizeof(smc2_iter_stats), cudaMemcpyHostToDevice,
                             c->stream));
  SMC2_TRY(outer_rebuild_recycling(c->op, dataset, k, c->stream));
  c->kernel_launches++;
  return cudaStreamSynchronize(c->stream) == cudaSuccess ? SMC2_OK : SMC2_ECUDA;
}

smc2_status smc2_resample_systematic(const uint64_t* q, int n, uint32_t U, int32_t* anc, void* stream) {
  if (!q || !anc || n < 1 || n > SMC2_MAX_N) return SMC2_EINVAL;
  return map_cuda(resample_systematic_launch(q, n, U, anc, static_cast<cudaStream_t>(stream)));
}

smc2_status smc2_philox_normals(uint64_t seed, const uint32_t* ctr, int n, int precision,
                                uint32_t* words, double* z, void* stream) {
  if (!ctr || n < 1 || (precision != SMC2_PREC_FP64 && precision != SMC2_PREC_MIXED)) return SMC2_EINVAL;
  return map_cuda(philox_normals_launch(seed, ctr, n, precision, words, z, static_cast<cudaStream_t>(stream)));
}

smc2_status smc2_mlp_loss_grad(int D, const float* params, const float* x, const float* y, int R,
                               float* grad, float* loss, void* stream) {
  if (D < 1 || D > kMlpMaxD || R < 1 || !params || !x || !y || !grad || !loss) return SMC2_EINVAL;
  if (reinterpret_cast<uintptr_t>(params) % 16 != 0) return SMC2_EINVAL;  // read as float4
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int n_cta = mlp_grad_ctas(R);
  float* part = nullptr;
  SMC2_TRY(cudaMallocAsync(reinterpret_cast<void**>(&part),
                           (size_t)n_cta * (mlp_param_count(D) + 1) * sizeof(float), s));
  const cudaError_t e = mlp_step_launch(const_cast<float*>(params), D, x, y, R, nullptr, part, grad, loss, 0,
                                        nullptr, nullptr, nullptr, 0.f, s);
  cudaFreeAsync(part, s);
  SMC2_TRY(e);
  return SMC2_OK;
}

smc2_status smc2_mlp_adam_step(int D, float* params, float* m, float* v, int* step, const float* x,
                               const float* y, int R, float lr, float* loss, void* stream) {
  if (D < 1 || D > kMlpMaxD || R < 1 || !params || !m || !v || !step || !x || !y || !loss ||
      !(lr >= 0.f && lr < 1.f))
    return SMC2_EINVAL;
  if (reinterpret_cast<uintptr_t>(params) % 16 != 0) return SMC2_EINVAL;  // the documented layout
  SMC2_TRY(mlp_train_steps_launch(params, m, v, step, const_cast<float*>(x), const_cast<float*>(y), R, nullptr,
                                  loss, D, 1, lr, static_cast<cudaStream_t>(stream)));
  return SMC2_OK;
}

smc2_status smc2_mlp_train_ring(int D, float* params, float* m, float* v, int* step, const float* ring_th,
                                const float* ring_lp, int R, int steps, float lr, float* x, float* y,
                                double* stdz, void* stream) {
  if (D < 1 || D > kMlpMaxD || R < 1 || steps < 0 || steps > 256 || !params || !m || !v || !step || !ring_th ||
      !ring_lp || !x || !y || !stdz || !(lr >= 0.f && lr < 1.f))
    return SMC2_EINVAL;
  if (reinterpret_cast<uintptr_t>(params) % 16 != 0) return SMC2_EINVAL;  // the documented layout
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  struct Scratch {
    MlpNorm nm;
    float loss;
    int rows;
  };
  Scratch* w = nullptr;
  SMC2_TRY(cudaMallocAsync(reinterpret_cast<void**>(&w), sizeof(Scratch), s));
  cudaError_t e = cudaMemsetAsync(w, 0, sizeof(Scratch), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&w->rows, &R, sizeof(int), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = mlp_train_ring_launch(params, m, v, step, ring_th, ring_lp, &w->rows, R, &w->nm, x, y, &w->loss, D, steps,
                              lr, s);
  if (e == cudaSuccess) e = mlp_norm_export_launch(&w->nm, &w->loss, D, stdz, s);
  const cudaError_t ef = cudaFreeAsync(w, s);
  SMC2_TRY(e);
  SMC2_TRY(ef);
  return SMC2_OK;
}

smc2_status smc2_mlp_input_grad(int D, const float* params, const float* x, int R, float* s_out, float* dx,
                                void* stream) {
  if (D < 1 || D > kMlpMaxD || R < 1 || !params || !x || !dx) return SMC2_EINVAL;
  if (reinterpret_cast<uintptr_t>(params) % 16 != 0) return SMC2_EINVAL;  // read as float4
  SMC2_TRY(mlp_input_grad_launch(params, D, x, R, s_out, dx, static_cast<cudaStream_t>(stream)));
  return SMC2_OK;
}

smc2_status smc2_sync(smc2_ctx* c) {
  if (!c) return SMC2_EINVAL;
  return sticky(c);
}

smc2_status smc2_get_launch_shape(smc2_ctx* c, int* ppt, int* cta_threads, int* grid, int* fp32_filter) {
  if (!c) return SMC2_EINVAL;
  if (fp32_filter) *fp32_filter = c->pf_fast ? (c->pf_named ? 2 : 1) : 0;
  if (ppt) *ppt = c->ppt;
  if (cta_threads) *cta_threads = c->pf_block;
  if (grid) *grid = c->pf_grid;
  return SMC2_OK;
}

smc2_status smc2_set_timing(smc2_ctx* c, int enable) {
  if (!c) return SMC2_EINVAL;
  c->timing = enable != 0;
  return SMC2_OK;
}

smc2_status smc2_get_timing(smc2_ctx* c, double* pf_ms, int64_t* pf_launches, int64_t* kernel_launches,
                            int reset) {
  if (!c) return SMC2_EINVAL;
  SMC2_TRY(cudaStreamSynchronize(c->stream));
  if (pf_ms) *pf_ms = c->pf_ms;
  if (pf_launches) *pf_launches = c->pf_launches;
  if (kernel_launches) *kernel_launches = c->kernel_launches;
  if (reset) {
    c->pf_ms = 0.0;
    c->pf_launches = 0;
    c->kernel_launches = 0;
  }
  return SMC2_OK;
}

void smc2_destroy(smc2_ctx* c) {
  if (!c) return;
  if (c->stream || c->arena) cudaStreamSynchronize(c->stream);
  drop_graphs(c);
  if (c->arena) cudaFree(c->arena);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->side_stream) cudaStreamDestroy(c->side_stream);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->train_stream) cudaStreamDestroy(c->train_stream);
  if (c->ev_tfork) cudaEventDestroy(c->ev_tfork);
  if (c->ev_tjoin) cudaEventDestroy(c->ev_tjoin);
  delete c;
}

}  // extern "C"
