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
  // The array keeps the previous call's contents: rewrite the hyperparameter
  // block and clear the counters before the kernels read them.
  Hyper hy;
  memset(&hy, 0, sizeof(hy));
  hy.it = a->it - 1;
  hy.n_mom = a->n_mom;
  hy.burnin = a->burnin;
  hy.tune_start = a->burnin / 2;
  hy.thin = 1;
  hy.trace_cap = 0;
  NA_CUDA(cudaMemcpyAsync(d_hyp, &hy, sizeof(Hyper), cudaMemcpyHostToDevice, s));
  NA_CUDA(cudaMemcpyAsync(d_hyp->phi, a->hyp, (size_t)P * 8, cudaMemcpyDeviceToDevice, s));
  NA_CUDA(cudaMemcpyAsync(&d_hyp->w_nu, a->hyp + P, 2 * 8, cudaMemcpyDeviceToDevice, s));
  if (mom) {
    NA_CUDA(cudaMemcpyAsync(d_hyp->m_phi, a->m_phi, (size_t)P * 8, cudaMemcpyDeviceToDevice, s));
    NA_CUDA(cudaMemcpyAsync(d_hyp->q_phi, a->q_phi, (size_t)P * 8, cudaMemcpyDeviceToDevice, s));
  }
  NA_CUDA(cudaMemsetAsync(d_cnt, 0, FBS_NUM_COUNTERS * sizeof(unsigned long long), s));

  NA_CUDA(prepare_gene_kernel(N, kNoAllocBlock));
  NA_CUDA(launch_gene(mc, p, kNoAllocBlock, s));
  NA_CUDA(launch_hyper(mc, p, (G + kNoAllocBlock - 1) / kNoAllocBlock, s));

  NA_CUDA(cudaMemcpyAsync(a->hyp, d_hyp->phi, (size_t)P * 8, cudaMemcpyDeviceToDevice, s));
  NA_CUDA(cudaMemcpyAsync(a->hyp + P, &d_hyp->w_nu, 2 * 8, cudaMemcpyDeviceToDevice, s));
  if (mom) {
    NA_CUDA(cudaMemcpyAsync(a->m_phi, d_hyp->m_phi, (size_t)P * 8, cudaMemcpyDeviceToDevice, s));
    NA_CUDA(cudaMemcpyAsync(a->q_phi, d_hyp->q_phi, (size_t)P * 8, cudaMemcpyDeviceToDevice, s));
  }
  return FBS_OK;
}

}  // extern "C"
