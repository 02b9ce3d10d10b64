// fbs_common.cuh -- device-side data layout shared by the kernels and the host
// code of the GB300 Gibbs sampler (Landau & Niemi, arXiv 1606.06659).
//
// HBM layout: every per-gene array is stored sample- or column-major with the
// gene index fastest ([N][G], [L][G], [G]), so a warp of 32 consecutive genes
// reads 32 consecutive words of each plane.
#pragma once

#include <stdint.h>

#include "fbs.h"

namespace fbs {

constexpr int kMaxN = FBS_MAX_N;
constexpr int kMaxL = FBS_MAX_L;
constexpr int kMaxP = 2 * FBS_MAX_L + 2;     // nu, tau, theta[L], sigma2[L]
constexpr int kMaxCls = FBS_MAX_CLASSES;
constexpr int kMaxPat = 8;  // distinct rows of X the FP32 beta columns sum over
constexpr int kNumPart = 2 + 2 * FBS_MAX_L;  // S1, S2, B1'[L], B2'[L]
constexpr int kCounterCopies = 32;  // the eps kernels spread their counter atomics

// RNG stream identifiers: one per kind of random variable.
enum : uint32_t {
  kStreamEps = 1,
  kStreamGamma = 2,
  kStreamNu = 3,
  kStreamTau = 4,
  kStreamBeta = 5,
  kStreamTheta = 6,
  kStreamSigma = 7,
  kStreamMH = 8,      // learned-proposal move of beta_g
  kStreamTrain = 9,   // minibatch sampling when training the proposal
  kStreamPsi = 10,    // top level of the three-level model
};

// Default bound of every tensor-core wait (mbarrier try_wait polls) of the
// proposal network; a wait that reaches it gives up and sets kFlagTimeout.
constexpr unsigned kTcWaitPolls = 1u << 24;

// Proposals of the eta-preserving move: the network's, or centred on the prior.
enum : int { kMoveNet = 1, kMovePrior = 2 };

// Learned proposal: hidden width of the two layers, limits of the per-gene
// features (4L+1) and outputs (L + L(L+1)/2).
constexpr int kMlpHidden = 64;
constexpr int kMaxFeat = 4 * FBS_MAX_L + 1;
constexpr int kMaxOut = FBS_MAX_L + FBS_MAX_L * (FBS_MAX_L + 1) / 2;

// Class of a non-zero value of one column of X: +1, -1 or any other value.
enum : int8_t { kClsPlus = 1, kClsMinus = 2, kClsOther = 0 };

// Model constants, passed to every kernel by value (kernel-parameter space).
struct ModelConst {
  int N, G, L, P;
  int K, shrink_max;
  int moments_eps, trace_beta;
  uint32_t seed_lo, seed_hi, chain;
  int all_slice;                  // 1: gamma_g, tau, sigma_l by slice updates too
  double a, b, d;
  double c2[kMaxL];               // c_l^2
  double s2[kMaxL];               // s_l^2
  double s[kMaxL];                // s_l
  double h[kMaxN];
  double X[kMaxN * kMaxL];        // [N][L]
  // Column classes for the beta_gl conditional: the non-zero values of column
  // l are grouped; cls[l][n] = class of X_nl (-1 when X_nl == 0).
  int ncls[kMaxL];
  double cval[kMaxL][kMaxCls];
  int8_t ckind[kMaxL][kMaxCls];
  int8_t cls[kMaxL][kMaxN];
  // FP32 copies for the FP32 form (conversions from FP64 run on the slow FP64 pipe)
  float hf[kMaxN];
  float Xf[kMaxN * kMaxL];
  float cvalf[kMaxL][kMaxCls];
  // Distinct rows of X (patterns): pat[n] = pattern of sample n, pcls[l][r] =
  // class of pattern r in column l (-1 for a zero); npat = kMaxPat + 1 when X
  // has more distinct rows (the FP32 beta columns then sum over samples).
  int npat;
  int8_t pat[kMaxN];
  int8_t pcls[kMaxL][kMaxPat];
};

// Propositions of the contrast probabilities, in device memory: proposition q
// holds when v[q][k] . beta_g > b[q][k] for every k < terms[q].
struct Contrasts {
  int n;
  int terms[FBS_MAX_CONTRASTS];
  double v[FBS_MAX_CONTRASTS][FBS_MAX_CONTRAST_TERMS][kMaxL];
  double b[FBS_MAX_CONTRASTS][FBS_MAX_CONTRAST_TERMS];
  float vf[FBS_MAX_CONTRASTS][FBS_MAX_CONTRAST_TERMS][kMaxL];
  float bf[FBS_MAX_CONTRASTS][FBS_MAX_CONTRAST_TERMS];
};

// Hyperparameters, run parameters and chain bookkeeping, in device memory.
struct Hyper {
  double phi[kMaxP];
  double m_phi[kMaxP], q_phi[kMaxP];   // running mean / mean square
  double w_nu, waux_nu;
  long long it;          // iterations completed
  long long n_mom;       // draws folded into the running moments
  long long trace_rows;  // rows written to the trace
  long long burnin, tune_start, thin, trace_cap;
  unsigned int flags;
  unsigned int pad;
  // iteration count and moment count when the current run segment started
  // (kernels that may run concurrently with the hyperparameter kernel derive
  // their iteration from these instead of reading `it`)
  long long seg_it, seg_nmom;
  // slice widths and tuning sums of tau and sigma_1..sigma_L (all_slice only)
  double w_hyp[kMaxL + 1], waux_hyp[kMaxL + 1];
};

// Top level of the three-level model (Section 2.3) over a batch of K datasets,
// in device memory: psi = (b, m_1..m_L) with tau_k ~ Gamma(a_k, rate b) and
// theta_kl ~ N(m_l, c_kl^2); b ~ Gamma(a_b, rate b_b), m_l ~ N(0, e_l^2).
struct TopLevel {
  double psi[kMaxL + 1];
  double m_psi[kMaxL + 1], q_psi[kMaxL + 1];  // running mean / mean square
  long long n_mom, trace_rows, trace_cap;
  unsigned long long gamma_caps;             // b draws that ran out of attempts
  double a_b, b_b;
  double e2[kMaxL];                          // e_l^2
  uint32_t seed_lo, seed_hi;
  int L, K;
};

// Device pointers of one chain.
struct DevPtrs {
  const int32_t* y;   // [N][G]
  const double* T;    // [L][G] sum_n y_gn X_nl
  double* eps;        // [N][G]
  double* w_eps;      // [N][G]
  double* waux_eps;   // [N][G]
  double* beta;       // [L][G]
  double* w_beta;     // [L][G]
  double* waux_beta;  // [L][G]
  double* gam;        // [G]
  double* w_gam;      // [G] slice widths of gamma_g (all_slice only)
  double* waux_gam;   // [G]
  double* m_eps;      // [N][G] running mean
  double* q_eps;      // [N][G] running mean square
  double* m_beta;     // [L][G]
  double* q_beta;     // [L][G]
  double* m_gam;      // [G]
  double* q_gam;      // [G]
  double* partial;    // [n_blocks][kNumPart]
  Hyper* hyp;
  double* trace_phi;  // [trace_cap][P]
  double* trace_beta; // [trace_cap][L][G] or null
  unsigned long long* counters;  // [copies][FBS_NUM_COUNTERS]
  double* mu;         // [N][G] Poisson means at the new eps (split sweep kernels)
  const Contrasts* con;  // null: no contrast probabilities
  unsigned* con_count;   // [n][G]
  unsigned long long* ktime;  // kernel-time probe (fbs_profile only; see ktime_begin)
  int ktime_n;
};

// Device pointers of one chain in the FP32 form: per-gene state in FP32, each
// running moment a Kahan-compensated FP32 pair (value m, compensation c; the
// moment is m - c); partial sums, hyperparameters and traces in FP64.
struct DevPtrsF32 {
  const int32_t* y;   // [N][G]
  const double* T;    // [L][G] (exact count sums, kept for fbs_count_sums)
  float* eps;         // [N][G]
  float* w_eps;
  float* waux_eps;
  float* beta;        // [L][G]
  float* w_beta;
  float* waux_beta;
  float* gam;         // [G]
  float* mom_eps;     // [4][N][G]: mean, mean compensation, mean square, its compensation
  float* mom_beta;    // [4][L][G]
  float* mom_gam;     // [4][G]
  float* mu;          // [N][G] Poisson means at the new eps, from the eps kernel
  // learned proposal (null prop: plain slice updates only)
  float* prop;        // [n_out][G] proposal mean and Cholesky parameters per gene
  const uint8_t* use_mh;  // [G] the gene's proposal kind (0: slice updates only)
  unsigned* mh_acc;   // [2][G] accepted moves per kind (kind - 1)
  unsigned* mh_try;   // [2][G] attempted moves per kind
  int mh_all;         // 0: per-gene kind (use_mh); 1, 2: that kind for every gene;
                      // 3: every gene, network / prior on alternate iterations
  int mh_replace;     // 1: the move replaces the slice updates of beta_g; 0: both run
  unsigned tc_polls;  // bound of each tensor-core wait of the network pass
  double* partial;    // [n_blocks][kNumPart]
  Hyper* hyp;
  double* trace_phi;  // [trace_cap][P]
  double* trace_beta; // [trace_cap][L][G] or null
  unsigned long long* counters;
  const Contrasts* con;  // null: no contrast probabilities
  unsigned* con_count;   // [n][G]
  const double* psi;     // null, or the batch's TopLevel::psi (three-level model)
  unsigned long long* ktime;  // kernel-time probe (fbs_profile only; see ktime_begin)
  int ktime_n;
};

// Flag bits in Hyper::flags.
enum : unsigned int { kFlagNonfinite = 1u, kFlagTimeout = 2u };

#ifdef __CUDACC__
// Kernel-time probe of fbs_profile: with kt non-null (only in the graph that
// fbs_profile replays), the first thread of every block folds the global timer
// (ns) at the block's start into kt[slot] (minimum) and at its end into
// kt[n + slot] (maximum), so that kt[n + slot] - kt[slot] is the kernel's span
// from its first block's start to its last block's end.  Sweep kernels call
// ktime_begin first and ktime_end last, with every thread of the block.
__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void ktime_begin(unsigned long long* kt, int n, int slot) {
  if (kt != nullptr && threadIdx.x == 0 && slot >= 0 && slot < n)
    atomicMin(kt + slot, global_timer_ns());
}

__device__ __forceinline__ void ktime_end(unsigned long long* kt, int n, int slot) {
  if (kt != nullptr) {
    __syncthreads();
    if (threadIdx.x == 0 && slot >= 0 && slot < n) atomicMax(kt + n + slot, global_timer_ns());
  }
}
#endif

}  // namespace fbs
