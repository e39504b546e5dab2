// internal.h -- descriptors shared by the library's translation units.
//
// Device memory layout (per dataset d, all arrays in one arena):
//   thA, thB   double SoA [D][N]  current population / proposals
//   lpA, lpB   double [N]         log prior of A / B
//   llA, llB   double [N]         PF log-likelihood estimate of A / B
//   logw       double [N]         unnormalised log weight (index-aligned with A and B)
//   logq       double [N]         log proposal density of B given A
//   q          uint64 [N]         quantised weights for outer resampling
//   part       double [nblk][kPartStride]  per-block partial sums
//   obs        R4 [T]             per-step observation terms in the PF precision
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/smc2.h"

namespace smc2 {

constexpr int kOuterBlock = 32;                        // threads of the per-sample outer kernels (one warp)
constexpr int kResBlock = 256;                         // threads of the resampling kernel
constexpr int kPfMaxBlock = 512;                       // threads of a particle-filter CTA, at most
constexpr int kMlpH = 64;                              // hidden width of the surrogate network
constexpr int kMlpWarps = 4;                           // warps (16 rows each) per network CTA
constexpr int kMlpMaxD = 8;                            // input dimension, at most
constexpr int kPartStride = 160;                       // >= 1 + 2D + 2D(2D+1)/2 for D <= 8
constexpr int kStatStride = 24;                        // >= 3 + D + D (D + 1) / 2

struct LKParams {
  double mu[2 * 8];    // (mu_a, mu_b)
  double A[8 * 8];     // S_ab S_bb^{-1}, row-major D x D
  double Lc[8 * 8];    // lower Cholesky factor of S_{a|b}
  double Lc_inv[8];    // reciprocals of its diagonal
  double logdet;       // log det S_{a|b}
  int fallback;        // 1: forward kernel used this iteration
  int pad;
};

struct IterCur {       // working scalars of the current iteration of one dataset
  double m;            // max log w (quantisation reference)
  double lse;          // log sum w
  double m_par;        // max parent log weight for the next iteration's L-kernel fit
  double Lpop[64];     // learned proposal: Cholesky factor of the weighted population covariance
  int pop_ok;          // Lpop usable (positive pivots, ESS >= 2 (D + 1))
  int resample;
  int mlp_used;        // 1: this iteration proposes with the learned drift
  double mlp_loss;     // training loss of the network that proposed
};

// Learned proposal: standardisation of the training set.
struct MlpNorm {
  double mu[8], sd[8];  // input standardisation
  double ymax, tau;     // z = max((log pi - ymax) / tau, -8)
  double zmean, zsd;    // y = (z - zmean) / zsd, the training target
  int rows;             // rows in the training set
  float var_y;          // variance of the targets (1, or 0 when they are constant)
};

// Learned proposal: device state (dataset 0 of a context).  Training writes
// p, norm and loss; the proposal reads the published copies p_use, norm_use,
// loss_use, so that training can run beside the next iteration.
struct MlpDev {
  int on, W;            // enabled; iterations kept in the training ring
  double h;             // proposal step
  float *p, *m, *v;     // parameters and Adam moments (FP32)
  int* step;            // Adam steps taken
  float* loss;          // latest training loss (mean squared error)
  float *ring_th, *ring_lp;   // [W N][D], [W N] (theta, log pi^)
  int* ring_rows;       // rows of the ring filled so far
  float *xs, *ys;       // standardised training set
  MlpNorm* norm;
  float* p_use;         // published parameters, standardisation and loss
  MlpNorm* norm_use;
  float* loss_use;
  double* score;        // [D][N] grad log pi^ at the parents (surrogate)
};

struct DSDev {
  int N, M, T, nblk;   // nblk: blocks of kOuterBlock samples
  int nblk_res;        // blocks of kResBlock slots
  double logN;
  double *thA, *thB, *lpA, *lpB, *llA, *llB, *logw, *logq;
  uint64_t* q;
  double* part;        // [nblk][kPartStride]
  double* part_st;     // [nblk][kStatStride]
  unsigned* tickets;   // [4]
  LKParams* lk;
  IterCur* cur;
  smc2_iter_stats* hist;  // [K]
  double* rec;         // [1 + D]: sum l_k, sum l_k f~_k
  double* est_rec;     // [D]: recycled estimate
  const void* obs;     // PF observation terms (R4 per step)
  uint32_t c2hi;       // dataset << 20
  int pad;
};

struct OuterParams {
  const DSDev* ds;
  int n_ds, D, lkernel, K;
  double rw_scale, ess_frac;
  double prior_mean[8], prior_sd[8];
  double inv_prior_sd[8], log_prior_sd[8];   // configuration constants
  double prior_lo[8], prior_hi[8], log_prior_width[8];  // uniform prior (prior_kind 1)
  int prior_kind;
  double inv_rw, log_rw;
  uint64_t seed;
  int* k_done;         // completed iterations; the running iteration is k_done + 1
  int* status;
  unsigned* grid_ticket;
  MlpDev mlp;
  int ds_N0;           // N of dataset 0
};

// One particle-filter job: n filters of one dataset.
struct PFJob {
  const double* theta; // SoA [D][ld]
  int ld, n, M, T;
  double* loglik;      // [n]
  double* delta;       // optional [n][T]
  int32_t* anc;        // optional [n][T-1][M]
  const void* obs;     // R4 per step
  uint32_t c2hi;
  int pad;
  // optional per-step trace of the FP32 filter (traced instantiations only): after the
  // propagation of step t, by particle j, at [(i T + t - 1) M + j]: the state (LG x;
  // SEIR S, E, I, log beta and the day's incidence) in xtr [..][kTraceState], the
  // log-weight in ltr and the quantised weight in qtr
  float* xtr;
  float* ltr;
  uint64_t* qtr;
};
constexpr int kTraceState = 5;  // floats per particle in a state trace

struct PFModel {
  double npop, e0, i0, lambda_floor;
  int n_sub;
  int pf_scheme;       // PF resampling: 0 systematic, 1 multinomial
  double pf_ess_frac;  // <= 0: every step; else when the ESS is below pf_ess_frac * M
};

struct PFLaunch {
  const PFJob* jobs;   // NULL: the single job job0
  const int4* wus;     // (job, first filter, count, -); NULL: one job, unit w = filters [w*fpc, ...)
  int n_wu;
  int fpc_single;      // filters per unit when wus == NULL
  int* wu_counter;     // dynamic scheduling when not NULL
  uint64_t seed;
  const int* k_done;   // iteration = *k_done + 1 when not NULL
  int k_imm;
  int* status;
  PFModel mdl;
  int t_cap;           // > 0: run at most t_cap steps (launch-shape tuning)
  int pad;
  uint32_t rk[20];     // Philox round keys of seed (philox_round_keys), read as constants
  PFJob job0;
};

// Launch-shape helpers (pf.cu).
size_t pf_smem_bytes(int precision, int model, int ppt, bool general, int block, int M);
int pf_group_threads(int ppt, int M);
cudaError_t pf_launch(int precision, int model, int ppt, bool named, bool general, int grid, int block,
                      size_t smem, const PFLaunch& L, cudaStream_t s);
cudaError_t pf_configure(int precision, int model, int ppt, bool named, bool general, size_t smem);
int pf_occupancy(int precision, int model, int ppt, bool named, bool general, int block, size_t smem);

// The register-resident FP32 filter of pf_fast.cuh: the default filter
// (systematic resampling after every step) of the LG and SEIR models in mixed
// precision, ppt 2, 4 or 8, one filter group per CTA or (grouped) groups of
// unequal width sharing a CTA.  trace selects the instantiation that writes the
// per-step trace of PFJob (states, log-weights, integer weights, increments and
// ancestors); the untraced ones write only the log-likelihoods.
bool pf_fast_eligible(int precision, int model, bool general, int ppt);
size_t pf_fast_smem_bytes(int model, int ppt, int block, int M);
cudaError_t pf_fast_launch(int model, int ppt, bool trace, bool grouped, int grid, int block, size_t smem,
                           const PFLaunch& L, cudaStream_t s);
cudaError_t pf_fast_configure(int model, int ppt, bool trace, bool grouped, size_t smem);
int pf_fast_occupancy(int model, int ppt, bool trace, bool grouped, int block, size_t smem);
// Particle-filter CTAs (the context's kernel, untraced) that fit on an SM beside
// one resident CTA of another kernel (o_threads threads of o_regs registers,
// o_smem bytes of shared memory).
int pf_blocks_beside(int precision, int model, int ppt, bool named, bool general, int block, size_t smem,
                     int o_threads, int o_regs, size_t o_smem);
int pf_fast_blocks_beside(int model, int ppt, bool grouped, int block, size_t smem, int o_threads, int o_regs,
                          size_t o_smem);

// Outer kernels (outer.cu).
cudaError_t outer_obs_terms(int precision, int model, const double* y, int T, void* obs,
                            cudaStream_t s);
cudaError_t outer_propose(const OuterParams& P, int max_nblk, cudaStream_t s);
cudaError_t outer_lkfit(const OuterParams& P, cudaStream_t s);
cudaError_t outer_weights(const OuterParams& P, int max_nblk, cudaStream_t s);
cudaError_t outer_quantise(const OuterParams& P, int max_nblk, cudaStream_t s);
cudaError_t outer_resample(const OuterParams& P, int max_nblk_res, int max_N, cudaStream_t s);
cudaError_t outer_parent_reference(const OuterParams& P, int dataset, cudaStream_t s);
cudaError_t outer_rebuild_recycling(const OuterParams& P, int dataset, int k, cudaStream_t s);
cudaError_t resample_systematic_launch(const uint64_t* q, int n, uint32_t U, int32_t* anc,
                                       cudaStream_t s);
// Surrogate network (mlp.cu).
int mlp_param_count(int D);
int mlp_grad_ctas(int R);  // CTAs (and partial-gradient rows) of one training step over R rows
size_t mlp_grad_smem_bytes();
cudaError_t mlp_step_launch(float* p, int D, const float* x, const float* y, int R, const int* R_dev,
                            float* part, float* grad, float* loss, int adam, float* m, float* v, int* step,
                            float lr, cudaStream_t s);
int mlp_train_cluster_size();  // CTAs of the training cluster (0: no cluster can be scheduled)
size_t mlp_train_smem_bytes();
// Per-SM footprint of the training cluster: its CTAs, and one CTA's threads,
// registers per thread and shared memory.
cudaError_t mlp_train_footprint(int* ctas, int* threads, int* regs, size_t* smem);
cudaError_t mlp_train_steps_launch(float* p, float* m, float* v, int* step, float* x, float* y, int R,
                                   const int* R_dev, float* loss, int D, int steps, float lr, cudaStream_t s,
                                   const MlpDev* ring_of = nullptr);
cudaError_t mlp_train_ring_launch(float* p, float* m, float* v, int* step, const float* th, const float* lp,
                                  const int* rows_dev, int R, MlpNorm* norm, float* x, float* y, float* loss,
                                  int D, int steps, float lr, cudaStream_t s);
cudaError_t mlp_norm_export_launch(const MlpNorm* nm, const float* loss, int D, double* out, cudaStream_t s);
cudaError_t mlp_init_launch(const MlpDev& M, int D, uint64_t seed, cudaStream_t s);
cudaError_t mlp_append_launch(const OuterParams& P, int N, cudaStream_t s);
cudaError_t mlp_train_launch(const OuterParams& P, int steps, float lr, cudaStream_t s);
cudaError_t mlp_publish_launch(const OuterParams& P, cudaStream_t s);
cudaError_t mlp_score_launch(const OuterParams& P, int N, cudaStream_t s);
cudaError_t mlp_input_grad_launch(const float* p, int D, const float* x, int R, float* s_out, float* dx,
                                  cudaStream_t s);

cudaError_t philox_normals_launch(uint64_t seed, const uint32_t* ctr, int n, int precision,
                                  uint32_t* words, double* z, cudaStream_t s);

}  // namespace smc2
