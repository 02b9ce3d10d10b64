// fbs_noalloc.cu -- one Gibbs sweep on caller-owned device arrays that
// allocates nothing (fbs_sweep_noalloc in include/fbs.h).
//
// The sweep kernels need scratch memory between their two launches: per-block
// partial sums, the hyperparameter block and the counters.  Here that scratch
// is one file-scope __device__ array of fixed size, so the call itself needs no
// cudaMalloc, no workspace and no stream or event of its own.  Every call on a
// device shares the array; calls whose work overlaps on the GPU (for example
// on two streams at once) race on it.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <string>

#include "fbs.h"
#include "fbs_common.cuh"
#include "fbs_kernels.h"

using namespace fbs;

namespace {

constexpr int kNoAllocBlock = 128;
constexpr int kNoAllocMaxBlocks = FBS_NOALLOC_MAX_GENES / kNoAllocBlock;
constexpr size_t kPartDoubles = (size_t)kNoAllocMaxBlocks * kNumPart;
constexpr size_t kHyperDoubles = (sizeof(Hyper) + 255) / 256 * 256 / 8;
constexpr size_t kScratchDoubles = kPartDoubles + kHyperDoubles + FBS_NUM_COUNTERS;
constexpr int kMaxDevices = 64;

static_assert(kPartDoubles * 8 % 256 == 0, "Hyper must stay 256-byte aligned");

// partials [kNoAllocMaxBlocks][kNumPart], then Hyper, then the counters
static __device__ __align__(256) double g_sweep_scratch[kScratchDoubles];

std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};

int fail_na(int code, const std::string& msg) {
  set_last_error(msg);
  return code;
}

#define NA_CUDA(call)                                                                       \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return fail_na(FBS_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Device address of the scratch array on the current device, looked up once
// per device with that device current.
int scratch_address(double** out) {
  int dev = 0;
  NA_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail_na(FBS_E_CUDA, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    NA_CUDA(cudaGetSymbolAddress(&p, g_sweep_scratch));
    g_scratch_addr[dev] = (double*)p;
  }
  *out = g_scratch_addr[dev];
  return FBS_OK;
}

// Writes the call's whole hyperparameter block into the scratch (the array keeps
// the previous call's contents): zero, then phi, w_nu, waux_nu and the running
// phi moments from the caller's arrays and the run fields from the arguments,
// which a launch passes by value; clears the counters.  One block.
__global__ void k_noalloc_begin(Hyper* hy, unsigned long long* cnt, const double* __restrict__ hyp,
                                const double* __restrict__ m_phi, const double* __restrict__ q_phi,
                                int P, long long it, long long n_mom, long long burnin) {
  const int tid = threadIdx.x;
  unsigned long long* w = reinterpret_cast<unsigned long long*>(hy);
  for (int i = tid; i < (int)(sizeof(Hyper) / 8); i += blockDim.x) w[i] = 0ull;
  if (tid < FBS_NUM_COUNTERS) cnt[tid] = 0ull;
  __syncthreads();
  if (tid < P) {
    hy->phi[tid] = hyp[tid];
    if (m_phi) {
      hy->m_phi[tid] = m_phi[tid];
      hy->q_phi[tid] = q_phi[tid];
    }
  }
  if (tid == 0) {
    hy->w_nu = hyp[P];
    hy->waux_nu = hyp[P + 1];
    hy->it = it - 1;
    hy->n_mom = n_mom;
    hy->burnin = burnin;
    hy->tune_start = burnin / 2;
    hy->thin = 1;
    hy->trace_cap = 0;
  }
}

// Copies the new phi, w_nu, waux_nu (and the phi moments) back to the caller's
// arrays and, when status is not null, the flags word and this call's counters.
__global__ void k_noalloc_end(const Hyper* hy, const unsigned long long* cnt, double* hyp,
                              double* m_phi, double* q_phi, int P, unsigned long long* status) {
  const int tid = threadIdx.x;
  if (tid < P) {
    hyp[tid] = hy->phi[tid];
    if (m_phi) {
      m_phi[tid] = hy->m_phi[tid];
      q_phi[tid] = hy->q_phi[tid];
    }
  }
  if (tid == 0) {
    hyp[P] = hy->w_nu;
    hyp[P + 1] = hy->waux_nu;
    if (status) status[0] = hy->flags;
  }
  if (status && tid < FBS_NUM_COUNTERS) status[1 + tid] = cnt[tid];
}

}  // namespace

extern "C" {

int fbs_sweep_noalloc(const fbs_sweep_args* a) {
  set_last_error("");
  if (!a) return fail_na(FBS_E_ARG, "args is NULL");
  const int N = a->N, G = a->G, L = a->L;
  if (N < 1 || N > FBS_MAX_N || L < 1 || L > FBS_MAX_L || G < 2)
    return fail_na(FBS_E_ARG, "need 1 <= N <= FBS_MAX_N, 1 <= L <= FBS_MAX_L, G >= 2");
  if (G > FBS_NOALLOC_MAX_GENES)
    return fail_na(FBS_E_ARG, "G exceeds FBS_NOALLOC_MAX_GENES, the size of the static scratch");
  if (a->it < 1 || a->burnin < 0 || a->n_mom < 0)
    return fail_na(FBS_E_ARG, "need it >= 1, burnin >= 0, n_mom >= 0");
  // n_mom counts post-burn-in draws folded in before iteration it: at most
  // it - 1 - burnin of them exist
  if (a->n_mom > (a->it - 1 > a->burnin ? a->it - 1 - a->burnin : 0))
    return fail_na(FBS_E_ARG, "n_mom exceeds the post-burn-in iterations before it");
  if (a->step_out_max < 0 || a->shrink_max < 0)
    return fail_na(FBS_E_ARG, "step_out_max and shrink_max must be >= 0");
  if (!a->X || !a->h || !a->priors.c || !a->priors.s)
    return fail_na(FBS_E_ARG, "X, h, priors.c and priors.s must be non-NULL host arrays");
  if (!a->y || !a->T || !a->eps || !a->w_eps || !a->waux_eps || !a->beta || !a->w_beta ||
      !a->waux_beta || !a->gam || !a->hyp)
    return fail_na(FBS_E_ARG, "a state or data device pointer is NULL");
  const bool mom = a->it > a->burnin;
  if (mom && (!a->m_beta || !a->q_beta || !a->m_gam || !a->q_gam || !a->m_phi || !a->q_phi ||
              (a->m_eps != nullptr) != (a->q_eps != nullptr)))
    return fail_na(FBS_E_ARG, "post-burn-in sweeps need the moment arrays");
  auto pos = [](double v) { return isfinite(v) && v > 0.0; };
  if (!pos(a->priors.a) || !pos(a->priors.b) || !pos(a->priors.d))
    return fail_na(FBS_E_ARG, "prior constants must be finite and > 0");

  ModelConst mc;
  memset(&mc, 0, sizeof(mc));
  mc.N = N;
  mc.G = G;
  mc.L = L;
  mc.P = 2 * L + 2;
  mc.K = a->step_out_max;
  mc.shrink_max = a->shrink_max;
  mc.moments_eps = a->m_eps ? 1 : 0;
  mc.trace_beta = 0;
  mc.seed_lo = (uint32_t)(a->seed & 0xffffffffu);
  mc.seed_hi = (uint32_t)(a->seed >> 32);
  mc.chain = a->chain;
  mc.a = a->priors.a;
  mc.b = a->priors.b;
  mc.d = a->priors.d;
  for (int l = 0; l < L; ++l) {
    if (!pos(a->priors.c[l]) || !pos(a->priors.s[l]))
      return fail_na(FBS_E_ARG, "prior constants must be finite and > 0");
    mc.c2[l] = a->priors.c[l] * a->priors.c[l];
    mc.s2[l] = a->priors.s[l] * a->priors.s[l];
  }
  for (int n = 0; n < N; ++n) {
    if (!isfinite(a->h[n])) return fail_na(FBS_E_ARG, "h has a non-finite entry");
    mc.h[n] = a->h[n];
    for (int l = 0; l < L; ++l) {
      if (!isfinite(a->X[n * L + l])) return fail_na(FBS_E_ARG, "X has a non-finite entry");
      mc.X[n * kMaxL + l] = a->X[n * L + l];
    }
  }
  for (int l = 0; l < L; ++l) {
    int nc = 0;
    for (int n = 0; n < N; ++n) {
      const double v = a->X[n * L + l];
      if (v == 0.0) {
        mc.cls[l][n] = -1;
        continue;
      }
      int j = 0;
      while (j < nc && mc.cval[l][j] != v) ++j;
      if (j == nc) {
        if (nc == kMaxCls)
          return fail_na(FBS_E_ARG, "a column of X has more than FBS_MAX_CLASSES distinct values");
        mc.cval[l][nc] = v;
        mc.ckind[l][nc] = v == 1.0 ? kClsPlus : (v == -1.0 ? kClsMinus : kClsOther);
        ++nc;
      }
      mc.cls[l][n] = (int8_t)j;
    }
    mc.ncls[l] = nc;
  }

  double* base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  Hyper* d_hyp = (Hyper*)(base + kPartDoubles);
  unsigned long long* d_cnt = (unsigned long long*)(base + kPartDoubles + kHyperDoubles);

  DevPtrs p;
  memset(&p, 0, sizeof(p));
  p.y = a->y;
  p.T = a->T;
  p.eps = a->eps;
  p.w_eps = a->w_eps;
  p.waux_eps = a->waux_eps;
  p.beta = a->beta;
  p.w_beta = a->w_beta;
  p.waux_beta = a->waux_beta;
  p.gam = a->gam;
  p.m_eps = a->m_eps;
  p.q_eps = a->q_eps;
  p.m_beta = a->m_beta;
  p.q_beta = a->q_beta;
  p.m_gam = a->m_gam;
  p.q_gam = a->q_gam;
  p.partial = base;
  p.hyp = d_hyp;
  p.trace_phi = nullptr;
  p.trace_beta = nullptr;
  p.counters = d_cnt;

  cudaStream_t s = (cudaStream_t)a->stream;
  const int P = mc.P;
  double* m_phi = mom ? a->m_phi : nullptr;
  double* q_phi = mom ? a->q_phi : nullptr;
  k_noalloc_begin<<<1, 64, 0, s>>>(d_hyp, d_cnt, a->hyp, m_phi, q_phi, P, a->it, a->n_mom,
                                   a->burnin);
  NA_CUDA(cudaGetLastError());
  NA_CUDA(prepare_gene_kernel(N, kNoAllocBlock));
  NA_CUDA(launch_gene(mc, p, kNoAllocBlock, s));
  NA_CUDA(launch_hyper(mc, p, (G + kNoAllocBlock - 1) / kNoAllocBlock, s));
  k_noalloc_end<<<1, 64, 0, s>>>(d_hyp, d_cnt, a->hyp, m_phi, q_phi, P,
                                 reinterpret_cast<unsigned long long*>(a->status));
  NA_CUDA(cudaGetLastError());
  return FBS_OK;
}

}  // extern "C"
