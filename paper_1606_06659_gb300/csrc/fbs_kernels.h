// fbs_kernels.h -- host-side launchers of the sweep, set-up, uniform and ESS
// kernels (fbs_kernels.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "fbs_common.cuh"

namespace fbs {

constexpr int kDefaultBlock = 128;

size_t gene_smem_bytes(int N, int block);
cudaError_t prepare_gene_kernel(int N, int block);
cudaError_t launch_gene(const ModelConst& mc, const DevPtrs& p, int block, cudaStream_t s);
cudaError_t launch_hyper(const ModelConst& mc, const DevPtrs& p, int nblk, cudaStream_t s);
cudaError_t launch_eps_f64(const ModelConst& mc, const DevPtrs& p, int seg_i, cudaStream_t s);
cudaError_t launch_gb_f64(const ModelConst& mc, const DevPtrs& p, int block, int seg_i,
                          cudaStream_t s);
cudaError_t launch_set_run(Hyper* hy, long long burnin, long long tune_start, long long thin,
                           cudaStream_t s);
cudaError_t launch_init(const ModelConst& mc, const DevPtrs& p, const int32_t* y_in,
                        int gene_major, const double* pinv, double w0, int set_state,
                        long long trace_cap, cudaStream_t s);
cudaError_t launch_zero_moments(const ModelConst& mc, const DevPtrs& p, cudaStream_t s);
cudaError_t launch_init_hyper(const ModelConst& mc, Hyper* hy, const double* beta_d,
                              const float* beta_f, double w0, int set_state, cudaStream_t s);
cudaError_t launch_init_run(Hyper* hy, long long trace_cap, cudaStream_t s);

// FP32 form (fbs_gene_f32.cu)
size_t gene_smem_bytes_f32(int N, int block);
cudaError_t prepare_gene_kernel_f32(int N, int block);
cudaError_t launch_eps_f32(const ModelConst& mc, const DevPtrsF32& p, int seg_i, cudaStream_t s);
// img: null, or the learned proposal's weight image, whose network the kernel
// then evaluates for its own genes first (block must be 128)
cudaError_t launch_gb_f32(const ModelConst& mc, const DevPtrsF32& p, int block, int seg_i,
                          cudaStream_t s, const void* img = nullptr);
cudaError_t launch_seg_begin(Hyper* hy, cudaStream_t s);
// A segment of n_sweeps sweeps of the plain FP32 form in one cooperative launch
// (persistent blocks, grid barriers; bit-identical to the separate launches).
// gsync: kPersistentSyncBytes of device memory, reset by the launch.
constexpr size_t kPersistentSyncBytes = 256;
cudaError_t launch_sweeps_f32(const ModelConst& mc, const DevPtrsF32& p, const DevPtrs& hp,
                              int n_sweeps, void* gsync, cudaStream_t s, int* grid_out);

cudaError_t launch_mh_step_f32(const ModelConst& mc, const DevPtrsF32& p, long long it,
                              cudaStream_t s);

// Gelman-Rubin factors of n parameters from C chains' moments (FP64 arrays, or
// FP32 Kahan planes [4][n] when f32)
struct RhatInput {
  int C, f32;
  long long M, n;
  const double* m[FBS_MAX_RHAT_CHAINS];
  const double* q[FBS_MAX_RHAT_CHAINS];
  const float* mf[FBS_MAX_RHAT_CHAINS];
};
cudaError_t launch_rhat(const RhatInput& in, double* out, cudaStream_t s);
// Pooled posterior mean, sd and the interval mean -/+ z sd of n parameters from
// the same inputs as launch_rhat (C >= 1): out [4][n] = mean, sd, lo, hi.
cudaError_t launch_estimates(const RhatInput& in, double z, double* out, cudaStream_t s);

// learned proposal (fbs_learned.cu)
// Training control block in device memory (one Adam step per captured replay).
struct TrainCtl {
  unsigned long long t;      // Adam steps done before the current step
  long long k, steps, epoch_steps;  // step within the call, steps of the call, of an epoch
  double lr, loss_sum;       // base step size; loss summed over the last epoch's steps
  float b1, b2;
  unsigned int done;         // blocks of the current step's reduction that finished
};
// One training step on the device: minibatch drawn for step t + 1, forward and
// backward on the tensor cores, gradient reduction, Adam, control-block update
// (two launches).  A tensor-core wait that gives up after `polls` polls sets
// kFlagTimeout in *flags, and the step then leaves the parameters unchanged.
// img: the step's weight image (train_image_bytes(L), zeroed when allocated,
// packed from params by launch_pack_train_image before the first step); the
// Adam update rewrites it for the next step.
cudaError_t launch_train_step(float* params, int L, int Bsz, const float* feat, const float* beta,
                              long long M, uint64_t seed, TrainCtl* ctl, const float* st,
                              float* part, float* grad, float* loss, float* adam_m, float* adam_v,
                              void* img, unsigned* flags, unsigned polls, cudaStream_t s);
size_t train_image_bytes(int L);
cudaError_t launch_pack_train_image(const float* params, int L, void* img, cudaStream_t s);
int mlp_param_count(int L);
cudaError_t launch_proposal_f32(const ModelConst& mc, const DevPtrsF32& p, const void* w_bf16,
                                float* out, cudaStream_t s);
cudaError_t launch_collect_f32(const ModelConst& mc, const DevPtrsF32& p, float* feat,
                               float* beta, long long row, cudaStream_t s);
cudaError_t launch_col_stats(const float* feat, const float* beta, long long M, int F, int L,
                             float* st, cudaStream_t s);
cudaError_t launch_fold(float* params, const float* st, int L, int to_raw, cudaStream_t s);
// one training step's gradient: fused forward/backward per block of 128 rows on
// the tensor cores, then the blocks' partial sums in block order (part:
// [train_blocks(Bsz)][np + 1]); flags and polls as for launch_train_step
size_t train_smem_bytes(int L);
int train_blocks(int Bsz);
cudaError_t prepare_train_kernel(int L);
cudaError_t launch_mlp_grad(const float* params, int L, int Bsz, const float* fb, const float* yb,
                            float* part, float* grad, float* loss, void* img, unsigned* flags,
                            unsigned polls, cudaStream_t s);
size_t tc_image_bytes(int L);
cudaError_t launch_pack_image(const float* params, void* img, int L, cudaStream_t s);

// batched FP32 kernels (fbs_gene_f32.cu)
cudaError_t prepare_batch_kernels(int max_N, int gb_block);
cudaError_t launch_eps_f32_batch(const ModelConst* mcs, const DevPtrsF32* ps, const int4* tab,
                                 int n_blocks, int block, int seg_i, cudaStream_t s);
cudaError_t launch_gb_f32_batch(const ModelConst* mcs, const DevPtrsF32* ps, const int2* tab,
                                int n_blocks, int block, int max_N, int seg_i, cudaStream_t s);
cudaError_t launch_hyper_batch(const ModelConst* mcs, const DevPtrsF32* ps, const int* nblk,
                               int C, cudaStream_t s);
cudaError_t launch_seg_begin_batch(const DevPtrsF32* ps, int C, cudaStream_t s);
cudaError_t launch_top_level(const ModelConst* mcs, const DevPtrsF32* ps, int C, TopLevel* top,
                             double* trace, cudaStream_t s);
cudaError_t launch_set_run_batch(const DevPtrsF32* ps, int C, long long burnin,
                                 long long tune_start, long long thin, cudaStream_t s);
constexpr int kEpsCounterCopiesHost = kCounterCopies;
cudaError_t launch_init_f32(const ModelConst& mc, const DevPtrsF32& p, const int32_t* y_in,
                            int gene_major, const double* pinv, double w0, int set_state,
                            cudaStream_t s);
cudaError_t launch_zero_moments_f32(const ModelConst& mc, const DevPtrsF32& p, cudaStream_t s);
cudaError_t launch_uniforms(uint64_t seed, uint32_t chain, uint32_t stream, uint32_t index0,
                            int n_index, uint32_t iter, uint32_t k0, int n_k, double* out,
                            cudaStream_t s);
// Sets the message fbs_last_error_string() returns on the calling thread.
void set_last_error(const std::string& msg);

cudaError_t launch_ess(const double* tr, long long rows, long long S, double* ess,
                       cudaStream_t s);

}  // namespace fbs
