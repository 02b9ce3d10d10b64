// fbs_kernels.cu -- CUDA kernels of one Gibbs sweep (Algorithm 1 of Landau &
// Niemi, arXiv 1606.06659) for sm_103a, plus initialisation, trace and ESS
// kernels.
//
// A sweep is two launches:
//   gene kernel   one thread per gene g: slice updates of eps_g1..eps_gN
//                 (Algorithm 1 step 1), the conjugate gamma_g draw (step 2), slice
//                 updates of beta_g1..beta_gL in order (step 5), width tuning
//                 (Algorithm 2 step 7), Welford moments (Section 3.1) and the
//                 per-block FP64 partial sums that feed steps 3, 4, 6, 7;
//   hyper kernel  one block: fixed-order reduction of the partials, then nu (slice,
//                 step 3) and tau (step 4) on lane 0 while lanes 1..L draw
//                 theta_l (step 6) and sigma_l^2 (step 7).
// Drawing beta before nu and tau is exact: the beta_gl conditional involves
// neither, and theirs involve no beta (Figure 3); the counter-based generator
// gives every variable the same uniforms in either order.
// With ModelConst::all_slice the gamma_g draw (gene kernel), tau (warp 0 of the
// hyper kernel, after nu) and sigma_l (lane 32+l) are slice updates of the same
// full conditionals instead, each variable with its own tuned width, as
// Section 4.2 slice-samples every non-normal conditional.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fbs_common.cuh"
#include "fbs_kernels.h"
#include "fbs_rng.cuh"
#include "fbs_hyper.cuh"

namespace fbs {

// ---------------------------------------------------------------- densities

// log f(eps_gn = x | ...) = y x - exp(A + x) - x^2 hg, with A = h_n + X_n beta_g and
// hg = 1/(2 gamma_g).  aux = exp(A + x), the Poisson mean at x.
struct EpsDensity {
  double y, A, hg;
  __device__ __forceinline__ double operator()(double x, double* aux) const {
    const double e = exp(A + x);
    *aux = e;
    return y * x - e - x * x * hg;
  }
};

// log f(beta_gl = b | ...) = b T_gl - sum_j Q_j exp(v_j (b - b0)) - (b - theta_l)^2 hs,
// where Q_j sums exp(h_n + eps_gn + X_n beta_g) (current beta, beta_gl = b0) over
// the samples n whose X_nl equals the j-th distinct non-zero value v_j of
// column l.  Samples with X_nl = 0 only add a constant.  hs = 1/(2 sigma_l^2).
struct BetaDensity {
  double T, b0, theta, hs;
  int ncls;
  double Q[kMaxCls];
  double v[kMaxCls];
  int8_t kind[kMaxCls];
  __device__ __forceinline__ double operator()(double b, double* aux) const {
    const double dlt = b - b0;
    const double z = exp(dlt);
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kMaxCls; ++j) {
      if (j < ncls) {
        double e;
        if (kind[j] == kClsPlus) e = z;
        else if (kind[j] == kClsMinus) e = 1.0 / z;
        else e = exp(v[j] * dlt);
        s += Q[j] * e;
      }
    }
    *aux = z;
    const double dv = b - theta;
    return b * T - s - dv * dv * hs;
  }
};

// BetaDensity with the class count NC fixed at compile time (NC = kMaxCls keeps
// the runtime bound `ncls`); the same arithmetic over the classes a column has.
template <int NC>
struct BetaDensityT {
  double T, b0, theta, hs;
  int ncls;
  double Q[NC];
  double v[NC];
  int8_t kind[NC];
  __device__ __forceinline__ double operator()(double b, double* aux) const {
    const double dlt = b - b0;
    const double z = exp(dlt);
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      if (NC < kMaxCls || j < ncls) {
        double e;
        if (kind[j] == kClsPlus) e = z;
        else if (kind[j] == kClsMinus) e = 1.0 / z;
        else e = exp(v[j] * dlt);
        s += Q[j] * e;
      }
    }
    *aux = z;
    const double dv = b - theta;
    return b * T - s - dv * dv * hs;
  }
};

// FP32 filters of the FP64 slice updates (slice_update_filtered).  Each returns
// Delta(p) = log f(p) - log f(x0) in the relative form of the FP32 sweep, which
// needs no evaluation at x0, and a bound on |Delta32 - Delta| + |the FP64
// evaluation's error|.  FP32 part: 2^-20 (16 times the unit roundoff) times the
// sum of the terms' magnitudes and of the sensitivities of Delta to the FP32
// roundings of its inputs (x - x0, y or T, the rate mu0 from expf of the rounded
// log-rate, Q_j, 1/(2 gamma) or 1/(2 sigma^2)) and to the series or expf of
// e^z - 1 - z; FP64 part: 2^-46 (64 times the FP64 unit roundoff) times the
// magnitudes of the terms of log f(p), log f(x0) and the level.

// eps: Delta(x) = d (y - mu0) - mu0 (e^d - 1 - d) - d (d + 2 x0) hg, d = x - x0.
struct EpsFilter {
  double x0;
  float y, mu0, x0f, hg, amag, c64;  // amag = |log-rate at x0| + 8; c64: log f(x0) magnitude
  __device__ __forceinline__ float operator()(double pt, float* eb) const {
    const float d = (float)(pt - x0);
    const float ad = fabsf(d);
    const float e = em1mx(d);
    const float ed1 = d + e;             // e^d - 1
    const float mued = mu0 + mu0 * ed1;  // mu0 e^d, the rate at pt
    const float t1 = d * (y - mu0);
    const float t2 = mu0 * e;
    const float t3 = d * (d + 2.0f * x0f) * hg;
    const float b32 = fabsf(t1) + fabsf(t2) + fabsf(t3) +
                      ad * (y + mu0 + mued + (2.0f * fabsf(x0f) + 2.0f * ad) * hg) +
                      amag * mu0 * fabsf(ed1) + mu0 * (2.0f + fabsf(ed1) + ad);
    const float px = fabsf(x0f) + ad;
    const float b64 = c64 + y * px + mued * (amag + ad) + px * px * hg;
    *eb = 0x1p-20f * b32 + 0x1p-46f * b64;
    return t1 - t2 - t3;
  }
};

// beta_gl: Delta(b) = d T - sum_j Q_j (e^{v_j d} - 1) - d (d + 2 (b0 - theta)) hs.
template <int NC>
struct BetaFilterT {
  double b0;
  float T, bt, hs, b0f, c64;  // bt = b0 - theta; c64: log f(b0) magnitude
  int ncls;
  float Q[NC], v[NC];
  __device__ __forceinline__ float operator()(double b, float* eb) const {
    const float d = (float)(b - b0);
    const float ad = fabsf(d);
    float s = 0.0f, sa = 0.0f, sq = 0.0f, se = 0.0f;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      if (NC < kMaxCls || j < ncls) {
        const float z = v[j] * d;
        const float ej1 = z + em1mx(z);  // e^z - 1
        const float q = Q[j] * ej1;
        s += q;
        sa += fabsf(q);
        sq += Q[j] * ((fabsf(v[j]) * ad + 1.0f) * (2.0f + fabsf(ej1)) + fabsf(z));
        se += Q[j] * (2.0f + fabsf(ej1));
      }
    }
    const float t1 = d * T;
    const float t3 = d * (d + 2.0f * bt) * hs;
    const float b32 = fabsf(t1) + sa + fabsf(t3) +
                      ad * (fabsf(T) + (2.0f * fabsf(bt) + 2.0f * ad) * hs) + sq;
    const float pb = fabsf(b0f) + ad, pt = fabsf(bt) + ad;
    const float b64 = c64 + pb * fabsf(T) + se + pt * pt * hs;
    *eb = 0x1p-20f * b32 + 0x1p-46f * b64;
    return t1 - s - t3;
  }
};

// log f(gamma_g = x | ...) = -shape1 log x - B / x on x > 0, with shape1 = (N + nu)/2 + 1
// and B = (sum_n eps_gn^2 + nu tau)/2: the Inverse-Gamma full conditional of step 2,
// slice-sampled in the all-slice variant (Section 4.2).
struct GamDensity {
  double shape1, B;
  __device__ __forceinline__ double operator()(double x, double* aux) const {
    *aux = 0.0;
    if (!(x > 0.0)) return -INFINITY;
    return -shape1 * log(x) - B / x;
  }
};

// ---------------------------------------------------------------- block reduction

template <int NV>
__device__ __forceinline__ void block_sum_to(double (&v)[NV], double* out, double* smem) {
  // warp-shuffle tree, then one value per warp through shared memory
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double x = v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) smem[warp * NV + i] = x;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
    for (int w = 0; w < nwarp; ++w) s += smem[w * NV + threadIdx.x];
    out[threadIdx.x] = s;
  }
}

// ---------------------------------------------------------------- gene kernel (FP64)

__global__ void __launch_bounds__(128) k_gene_f64(ModelConst mc, DevPtrs p) {
  extern __shared__ double smem_dyn[];  // mu[n][blockDim] then reduction scratch
  const int G = mc.G, N = mc.N, L = mc.L;
  const Hyper* hy = p.hyp;
  const long long it = hy->it + 1;
  const uint32_t it32 = (uint32_t)it;
  const long long burnin = hy->burnin, tune_start = hy->tune_start;
  const bool mom = it > burnin;
  const double inv_k = mom ? 1.0 / (double)(hy->n_mom + 1) : 0.0;
  const double nu = hy->phi[0], tau = hy->phi[1];
  const bool trace_now = mom && mc.trace_beta && p.trace_beta != nullptr &&
                         ((it - burnin) % hy->thin == 0) && hy->trace_rows < hy->trace_cap;
  const long long trace_row = hy->trace_rows;

  double* mu = smem_dyn;  // mu[n * blockDim + tid]
  const int tid = threadIdx.x;
  const int g = blockIdx.x * blockDim.x + tid;
  const bool active = g < G;

  double part[kNumPart];
#pragma unroll
  for (int i = 0; i < kNumPart; ++i) part[i] = 0.0;
  unsigned evals_e = 0, evals_b = 0, caps = 0, gcaps = 0, nonfin = 0;

  if (active) {
    double beta[kMaxL];
#pragma unroll
    for (int l = 0; l < kMaxL; ++l) beta[l] = l < L ? p.beta[(size_t)l * G + g] : 0.0;
    double gam = p.gam[g];
    const double hg = 0.5 / gam;

    // ---- step 1: eps_gn, n = 1..N
    double ss = 0.0;
    for (int n = 0; n < N; ++n) {
      const size_t e = (size_t)n * G + g;
      double A = mc.h[n];
#pragma unroll
      for (int l = 0; l < kMaxL; ++l)
        if (l < L) A += mc.X[n * kMaxL + l] * beta[l];
      EpsDensity f{(double)p.y[e], A, hg};
      Rng r(mc.seed_lo, mc.seed_hi, mc.chain, kStreamEps, (uint32_t)((size_t)g * N + n), it32);
      const double x0 = p.eps[e];
      double w = p.w_eps[e], waux = p.waux_eps[e];
      SliceResult s = slice_update(x0, w, f, r, mc.K, mc.shrink_max);
      evals_e += s.evals;
      caps += s.capped;
      nonfin += s.nonfinite;
      mu[n * blockDim.x + tid] = s.aux;
      p.eps[e] = s.x;
      if (it <= burnin) {
        tune_width(w, waux, it, s.x, x0, burnin, tune_start);
        p.w_eps[e] = w;
        p.waux_eps[e] = waux;
      }
      ss += s.x * s.x;
      if (mom && mc.moments_eps) {
        const double m = p.m_eps[e], q = p.q_eps[e];
        p.m_eps[e] = m + (s.x - m) * inv_k;
        p.q_eps[e] = q + (s.x * s.x - q) * inv_k;
      }
    }

    // ---- step 2: gamma_g ~ IG((N + nu)/2, (sum eps^2 + nu tau)/2)
    {
      Rng r(mc.seed_lo, mc.seed_hi, mc.chain, kStreamGamma, (uint32_t)g, it32);
      bool gcap = false;
      const double shape = 0.5 * ((double)N + nu);
      const double scale = 0.5 * (ss + nu * tau);
      gam = scale / gamma_mt(shape, r, 0, &gcap);
      gcaps += gcap;
      p.gam[g] = gam;
      if (mom) {
        const double m = p.m_gam[g], q = p.q_gam[g];
        p.m_gam[g] = m + (gam - m) * inv_k;
        p.q_gam[g] = q + (gam * gam - q) * inv_k;
      }
      part[0] = log(gam);
      part[1] = 1.0 / gam;
    }

    // ---- step 5: beta_gl, l = 1..L in order
    for (int l = 0; l < L; ++l) {
      const size_t e = (size_t)l * G + g;
      const double theta = hy->phi[2 + l];
      const double sig2 = hy->phi[2 + L + l];
      BetaDensity f;
      f.T = p.T[e];
      f.b0 = beta[l];
      f.theta = theta;
      f.hs = 0.5 / sig2;
      f.ncls = mc.ncls[l];
#pragma unroll
      for (int j = 0; j < kMaxCls; ++j) {
        f.Q[j] = 0.0;
        f.v[j] = mc.cval[l][j];
        f.kind[j] = mc.ckind[l][j];
      }
      for (int n = 0; n < N; ++n) {
        const int c = mc.cls[l][n];
        const double m = mu[n * blockDim.x + tid];
#pragma unroll
        for (int j = 0; j < kMaxCls; ++j)
          if (j == c) f.Q[j] += m;
      }
      Rng r(mc.seed_lo, mc.seed_hi, mc.chain, kStreamBeta, (uint32_t)((size_t)g * L + l), it32);
      const double x0 = beta[l];
      double w = p.w_beta[e], waux = p.waux_beta[e];
      SliceResult s = slice_update(x0, w, f, r, mc.K, mc.shrink_max);
      evals_b += s.evals;
      caps += s.capped;
      nonfin += s.nonfinite;
      // carry exp(h_n + eps_gn + X_n beta_g) to the new beta_gl
      if (s.x != x0) {
        const double dlt = s.x - x0;
        double ej[kMaxCls];
        const double z = exp(dlt);
#pragma unroll
        for (int j = 0; j < kMaxCls; ++j) {
          ej[j] = 1.0;
          if (j < f.ncls) {
            if (f.kind[j] == kClsPlus) ej[j] = z;
            else if (f.kind[j] == kClsMinus) ej[j] = 1.0 / z;
            else ej[j] = exp(f.v[j] * dlt);
          }
        }
        for (int n = 0; n < N; ++n) {
          const int c = mc.cls[l][n];
          double fac = 1.0;
#pragma unroll
          for (int j = 0; j < kMaxCls; ++j)
            if (j == c) fac = ej[j];
          mu[n * blockDim.x + tid] *= fac;
        }
      }
      beta[l] = s.x;
      p.beta[e] = s.x;
      if (it <= burnin) {
        tune_width(w, waux, it, s.x, x0, burnin, tune_start);
        p.w_beta[e] = w;
        p.waux_beta[e] = waux;
      }
      if (mom) {
        const double m = p.m_beta[e], q = p.q_beta[e];
        p.m_beta[e] = m + (s.x - m) * inv_k;
        p.q_beta[e] = q + (s.x * s.x - q) * inv_k;
      }
      if (trace_now) p.trace_beta[(size_t)trace_row * L * G + e] = s.x;
      const double dv = s.x - theta;  // shifted by the current theta_l
      part[2 + l] = dv;
      part[2 + kMaxL + l] = dv * dv;
    }
  }

  // ---- per-block partial sums for steps 3, 4, 6, 7
  double* red = smem_dyn + (size_t)N * blockDim.x;
  block_sum_to<kNumPart>(part, p.partial + (size_t)blockIdx.x * kNumPart, red);

  // ---- counters
  unsigned long long c4[4] = {evals_e, evals_b, caps, gcaps};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    unsigned long long x = c4[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    c4[i] = x;
  }
  unsigned nf = nonfin;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nf += __shfl_down_sync(0xffffffffu, nf, o);
  if ((tid & 31) == 0) {
    if (c4[0]) atomicAdd(&p.counters[FBS_CNT_EVALS_EPS], c4[0]);
    if (c4[1]) atomicAdd(&p.counters[FBS_CNT_EVALS_BETA], c4[1]);
    if (c4[2]) atomicAdd(&p.counters[FBS_CNT_SLICE_CAPS], c4[2]);
    if (c4[3]) atomicAdd(&p.counters[FBS_CNT_GAMMA_CAPS], c4[3]);
    if (nf) {
      atomicAdd(&p.counters[FBS_CNT_NONFINITE], (unsigned long long)nf);
      atomicOr(&p.hyp->flags, kFlagNonfinite);
    }
  }
}

// ---------------------------------------------------------------- split sweep kernels (FP64)
//
// The same arithmetic as k_gene_f64 split in two launches so that every SM gets
// work at any G and the hyperparameter kernel of sweep m can run concurrently
// with the eps kernel of sweep m+1 (the eps conditionals involve no
// hyperparameter).  k_gene_f64 remains for fbs_sweep_noalloc.

__device__ __forceinline__ void add_counters_u(unsigned long long* base, unsigned evals_e,
                                               unsigned evals_b, unsigned caps, unsigned gcaps,
                                               unsigned nonfin, unsigned* flags,
                                               unsigned evals_g = 0) {
  unsigned v[6] = {evals_e, evals_b, caps, gcaps, nonfin, evals_g};
#pragma unroll
  for (int i = 0; i < 6; ++i) v[i] = __reduce_add_sync(0xffffffffu, v[i]);  // warp sum
  if ((threadIdx.x & 31) == 0) {
    if (v[0]) atomicAdd(&base[FBS_CNT_EVALS_EPS], (unsigned long long)v[0]);
    if (v[1]) atomicAdd(&base[FBS_CNT_EVALS_BETA], (unsigned long long)v[1]);
    if (v[2]) atomicAdd(&base[FBS_CNT_SLICE_CAPS], (unsigned long long)v[2]);
    if (v[3]) atomicAdd(&base[FBS_CNT_GAMMA_CAPS], (unsigned long long)v[3]);
    if (v[4]) {
      atomicAdd(&base[FBS_CNT_NONFINITE], (unsigned long long)v[4]);
      atomicOr(flags, kFlagNonfinite);
    }
    if (v[5]) atomicAdd(&base[FBS_CNT_EVALS_GAMMA], (unsigned long long)v[5]);
  }
}

// Step 1: one thread per eps_gn (element e = n*G + g of the [N][G] planes).
__global__ void __launch_bounds__(256) k_eps_f64(ModelConst mc, DevPtrs p, int seg_i) {
  ktime_begin(p.ktime, p.ktime_n, 3 * seg_i);
  const int G = mc.G, N = mc.N, L = mc.L;
  const Hyper* hy = p.hyp;
  const long long it = hy->seg_it + seg_i + 1;
  const long long burnin = hy->burnin, tune_start = hy->tune_start;
  const bool mom = it > burnin;
  long long before = (it - 1) - (hy->seg_it > burnin ? hy->seg_it : burnin);
  if (before < 0) before = 0;
  const double inv_k = mom ? 1.0 / (double)(hy->seg_nmom + before + 1) : 0.0;
  const int n = blockIdx.y;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t e = (size_t)n * G + g;
  unsigned evals = 0, caps = 0, nonfin = 0;
  if (g < G) {
    double A = mc.h[n];
#pragma unroll
    for (int l = 0; l < kMaxL; ++l)
      if (l < L) A += mc.X[n * kMaxL + l] * p.beta[(size_t)l * G + g];
    EpsDensity f{(double)p.y[e], A, 0.5 / p.gam[g]};
    Rng r(mc.seed_lo, mc.seed_hi, mc.chain, kStreamEps, (uint32_t)((size_t)g * N + n),
          (uint32_t)it);
    const double x0 = p.eps[e];
    double w = p.w_eps[e];
    // comparisons decided in FP32 where an error bound allows (the same result);
    // a start whose rate does not fit FP32 takes the FP64 comparisons throughout
    const float af = (float)(A + x0), hgf = (float)f.hg, yf = (float)f.y, x0f = (float)x0;
    const float mu0f = expf(af);
    SliceResult s;
    if (isfinite(mu0f) && isfinite(hgf) && isfinite(x0f) && af < 80.0f) {
      const float amag = fabsf(af) + 8.0f;
      EpsFilter ff{x0, yf, mu0f, x0f, hgf, amag,
                   yf * fabsf(x0f) + mu0f * amag + x0f * x0f * hgf + 64.0f};
      s = slice_update_filtered(x0, w, f, ff, r, mc.K, mc.shrink_max);
      s.aux = exp(A + s.x);  // the rate at the result, as the density computes it
    } else {
      s = slice_update(x0, w, f, r, mc.K, mc.shrink_max);
    }
    evals = s.evals;
    caps = s.capped;
    nonfin = s.nonfinite;
    p.mu[e] = s.aux;
    p.eps[e] = s.x;
    if (it <= burnin) {
      double waux = p.waux_eps[e];
      tune_width(w, waux, it, s.x, x0, burnin, tune_start);
      p.w_eps[e] = w;
      p.waux_eps[e] = waux;
    }
    if (mom && mc.moments_eps) {
      const double m = p.m_eps[e], q = p.q_eps[e];
      p.m_eps[e] = m + (s.x - m) * inv_k;
      p.q_eps[e] = q + (s.x * s.x - q) * inv_k;
    }
  }
  add_counters_u(p.counters + ((blockIdx.x + blockIdx.y) % kCounterCopies) * FBS_NUM_COUNTERS, evals, 0, caps,
                 0, nonfin, &p.hyp->flags);
  ktime_end(p.ktime, p.ktime_n, 3 * seg_i);
}

// Steps 2 and 5: one thread per gene, after the eps kernel of this sweep and the
// hyperparameter kernel of the previous one.
// One slice update of beta_gl (step 5) for a column with NC value classes, with
// the class sums of the rates in shared memory, the moments, trace and partials.
template <int NC>
__device__ __forceinline__ void beta_column_f64(const ModelConst& mc, const DevPtrs& p, int l,
                                                int g, double* mu, double* bs, double* ps, int B,
                                                int tid, const Hyper* hy, long long it,
                                                uint32_t it32, long long burnin,
                                                long long tune_start, bool mom, double inv_k,
                                                bool trace_now, long long trace_row,
                                                unsigned& evals_b, unsigned& caps,
                                                unsigned& nonfin) {
  const int G = mc.G, N = mc.N, L = mc.L;
  const size_t e = (size_t)l * G + g;
  const double theta = hy->phi[2 + l];
  const double sig2 = hy->phi[2 + L + l];
  BetaDensityT<NC> f;
  f.T = p.T[e];
  const double b_cur = bs[l * B + tid];
  f.b0 = b_cur;
  f.theta = theta;
  f.hs = 0.5 / sig2;
  f.ncls = mc.ncls[l];
#pragma unroll
  for (int j = 0; j < NC; ++j) {
    f.Q[j] = 0.0;
    f.v[j] = mc.cval[l][j];
    f.kind[j] = mc.ckind[l][j];
  }
  for (int n = 0; n < N; ++n) {
    const int c = mc.cls[l][n];
    const double m = mu[n * blockDim.x + tid];
#pragma unroll
    for (int j = 0; j < NC; ++j)
      if (j == c) f.Q[j] += m;
  }
  Rng r(mc.seed_lo, mc.seed_hi, mc.chain, kStreamBeta, (uint32_t)((size_t)g * L + l), it32);
  const double x0 = b_cur;
  double w = p.w_beta[e];
  // comparisons decided in FP32 where an error bound allows (the same result)
  BetaFilterT<NC> ff;
  ff.b0 = x0;
  ff.b0f = (float)x0;
  ff.T = (float)f.T;
  ff.bt = (float)(x0 - theta);
  ff.hs = (float)f.hs;
  ff.ncls = f.ncls;
  bool filt = isfinite(ff.T) && isfinite(ff.bt) && isfinite(ff.hs) && isfinite(ff.b0f);
  float qs = 0.0f;
#pragma unroll
  for (int j = 0; j < NC; ++j) {
    ff.Q[j] = (float)f.Q[j];
    ff.v[j] = (float)f.v[j];
    if (NC < kMaxCls || j < f.ncls) qs += ff.Q[j];
  }
  filt = filt && isfinite(qs);
  ff.c64 = fabsf(ff.b0f) * fabsf(ff.T) + qs + ff.bt * ff.bt * ff.hs + 64.0f;
  SliceResult s = filt && isfinite(ff.c64) ? slice_update_filtered(x0, w, f, ff, r, mc.K, mc.shrink_max)
                                           : slice_update(x0, w, f, r, mc.K, mc.shrink_max);
  evals_b += s.evals;
  caps += s.capped;
  nonfin += s.nonfinite;
  if (s.x != x0) {
    const double dlt = s.x - x0;
    double ej[NC];
    const double z = exp(dlt);
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      ej[j] = 1.0;
      if (NC < kMaxCls || j < f.ncls) {
        if (f.kind[j] == kClsPlus) ej[j] = z;
        else if (f.kind[j] == kClsMinus) ej[j] = 1.0 / z;
        else ej[j] = exp(f.v[j] * dlt);
      }
    }
    for (int n = 0; n < N; ++n) {
      const int c = mc.cls[l][n];
      double fac = 1.0;
#pragma unroll
      for (int j = 0; j < NC; ++j)
        if (j == c) fac = ej[j];
      mu[n * blockDim.x + tid] *= fac;
    }
  }
  bs[l * B + tid] = s.x;
  p.beta[e] = s.x;
  if (it <= burnin) {
    double waux = p.waux_beta[e];
    tune_width(w, waux, it, s.x, x0, burnin, tune_start);
    p.w_beta[e] = w;
    p.waux_beta[e] = waux;
  }
  if (mom) {
    const double m = p.m_beta[e], q = p.q_beta[e];
    p.m_beta[e] = m + (s.x - m) * inv_k;
    p.q_beta[e] = q + (s.x * s.x - q) * inv_k;
  }
  if (trace_now) p.trace_beta[(size_t)trace_row * L * G + e] = s.x;
  const double dv = s.x - theta;
  ps[(2 + l) * B + tid] = dv;
  ps[(2 + kMaxL + l) * B + tid] = dv * dv;
}

__global__ void __launch_bounds__(128) k_gb_f64(ModelConst mc, DevPtrs p, int seg_i) {
  // shared: mu[N][B], beta[L][B], partials[kNumPart][B] (values indexed by a runtime
  // l live here rather than in local memory), then the reduction scratch
  extern __shared__ double smem_dyn[];
  ktime_begin(p.ktime, p.ktime_n, 3 * seg_i + 1);
  const int G = mc.G, N = mc.N, L = mc.L;
  const Hyper* hy = p.hyp;
  const long long it = hy->seg_it + seg_i + 1;
  const uint32_t it32 = (uint32_t)it;
  const long long burnin = hy->burnin, tune_start = hy->tune_start;
  const bool mom = it > burnin;
  const double inv_k = mom ? 1.0 / (double)(hy->n_mom + 1) : 0.0;
  const double nu = hy->phi[0], tau = hy->phi[1];
  const bool trace_now = mom && mc.trace_beta && p.trace_beta != nullptr &&
                         ((it - burnin) % hy->thin == 0) && hy->trace_rows < hy->trace_cap;
  const long long trace_row = hy->trace_rows;

  const int B = blockDim.x;
  double* mu = smem_dyn;
  double* bs = mu + (size_t)N * B;
  double* ps = bs + (size_t)kMaxL * B;
  const int tid = threadIdx.x;
  const int g = blockIdx.x * B + tid;
  const bool active = g < G;

#pragma unroll
  for (int i = 0; i < kNumPart; ++i) ps[i * B + tid] = 0.0;
  unsigned evals_b = 0, evals_g = 0, caps = 0, gcaps = 0, nonfin = 0;

  if (active) {
    for (int l = 0; l < L; ++l) bs[l * B + tid] = p.beta[(size_t)l * G + g];
    double ss = 0.0;
#pragma unroll 4
    for (int n = 0; n < N; ++n) {
      const size_t e = (size_t)n * G + g;
      const double x = p.eps[e];
      ss += x * x;
      mu[n * blockDim.x + tid] = p.mu[e];
    }

    // ---- step 2: gamma_g ~ IG((N + nu)/2, (sum eps^2 + nu tau)/2), exactly or
    // (all_slice) by a slice update of that density with the gene's own width
    {
      Rng r(mc.seed_lo, mc.seed_hi, mc.chain, kStreamGamma, (uint32_t)g, it32);
      const double shape = 0.5 * ((double)N + nu);
      const double scale = 0.5 * (ss + nu * tau);
      double gam;
      if (mc.all_slice) {
        const double x0 = p.gam[g];
        double w = p.w_gam[g], waux = p.waux_gam[g];
        SliceResult s = slice_update(x0, w, GamDensity{shape + 1.0, scale}, r, mc.K, mc.shrink_max);
        evals_g += s.evals;
        caps += s.capped;
        nonfin += s.nonfinite;
        gam = s.x;
        if (it <= burnin) {
          tune_width(w, waux, it, s.x, x0, burnin, tune_start);
          p.w_gam[g] = w;
          p.waux_gam[g] = waux;
        }
      } else {
        bool gcap = false;
        gam = scale / gamma_mt(shape, r, 0, &gcap);
        gcaps += gcap;
      }
      p.gam[g] = gam;
      if (mom) {
        const double m = p.m_gam[g], q = p.q_gam[g];
        p.m_gam[g] = m + (gam - m) * inv_k;
        p.q_gam[g] = q + (gam * gam - q) * inv_k;
      }
      ps[0 * B + tid] = log(gam);
      ps[1 * B + tid] = 1.0 / gam;
    }

    // ---- step 5: beta_gl, l = 1..L in order
    for (int l = 0; l < L; ++l) {
      switch (mc.ncls[l]) {
        case 1:
          beta_column_f64<1>(mc, p, l, g, mu, bs, ps, B, tid, hy, it, it32, burnin, tune_start, mom, inv_k,
                               trace_now, trace_row, evals_b, caps, nonfin);
          break;
        case 2:
          beta_column_f64<2>(mc, p, l, g, mu, bs, ps, B, tid, hy, it, it32, burnin, tune_start, mom, inv_k,
                               trace_now, trace_row, evals_b, caps, nonfin);
          break;
        case 3:
          beta_column_f64<3>(mc, p, l, g, mu, bs, ps, B, tid, hy, it, it32, burnin, tune_start, mom, inv_k,
                               trace_now, trace_row, evals_b, caps, nonfin);
          break;
        default:
          beta_column_f64<kMaxCls>(mc, p, l, g, mu, bs, ps, B, tid, hy, it, it32, burnin, tune_start, mom, inv_k,
                               trace_now, trace_row, evals_b, caps, nonfin);
      }
    }
    // contrast probabilities (§3.1): count the iterations whose beta_g satisfies
    // each proposition
    if (mom && p.con != nullptr) {
      const Contrasts* cs = p.con;
      for (int q = 0; q < cs->n; ++q) {
        bool ok = true;
        for (int k = 0; k < cs->terms[q] && ok; ++k) {
          double sv = 0.0;
          for (int l = 0; l < L; ++l) sv = __dadd_rn(sv, __dmul_rn(cs->v[q][k][l], bs[l * B + tid]));
          ok = sv > cs->b[q][k];
        }
        if (ok) p.con_count[(size_t)q * G + g] += 1u;
      }
    }
  }

  double part[kNumPart];
#pragma unroll
  for (int i = 0; i < kNumPart; ++i) part[i] = ps[i * B + tid];
  double* red = ps + (size_t)kNumPart * B;
  block_sum_to<kNumPart>(part, p.partial + (size_t)blockIdx.x * kNumPart, red);
  add_counters_u(p.counters, 0, evals_b, caps, gcaps, nonfin, &p.hyp->flags, evals_g);
  ktime_end(p.ktime, p.ktime_n, 3 * seg_i + 1);
}

__global__ void __launch_bounds__(kHyperThreads) k_hyper(ModelConst mc, DevPtrs p, int nblk) {
  // the sweep of the segment this launch completes (probe slot only)
  const int slot = p.ktime ? 3 * (int)(p.hyp->it - p.hyp->seg_it) + 2 : 0;
  ktime_begin(p.ktime, p.ktime_n, slot);
  hyper_body(mc, p.partial, p.hyp, p.trace_phi, p.counters, nblk);
  ktime_end(p.ktime, p.ktime_n, slot);
}

// ---------------------------------------------------------------- convergence

// Gelman-Rubin potential scale reduction of parameter i (§3.1) from the chains'
// running means and mean squares over M draws each.
__global__ void k_rhat(RhatInput in, double* __restrict__ out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= in.n) return;
  const int C = in.C;
  const double M = (double)in.M;
  double mean[FBS_MAX_RHAT_CHAINS], msq[FBS_MAX_RHAT_CHAINS];
  double tot = 0.0;
  for (int c = 0; c < C; ++c) {
    if (in.f32) {
      const float* b = in.mf[c];
      mean[c] = (double)b[i] - (double)b[in.n + i];
      msq[c] = (double)b[2 * in.n + i] - (double)b[3 * in.n + i];
    } else {
      mean[c] = in.m[c][i];
      msq[c] = in.q[c][i];
    }
    tot += mean[c];
  }
  const double grand = tot / C;
  double bsum = 0.0, wsum = 0.0;
  for (int c = 0; c < C; ++c) {
    const double dm = mean[c] - grand;
    bsum += dm * dm;
    wsum += M / (M - 1.0) * (msq[c] - mean[c] * mean[c]);
  }
  const double B = M / (C - 1) * bsum;
  const double W = wsum / C;
  out[i] = W > 0.0 ? sqrt(1.0 + (B / W - 1.0) / M) : NAN;
}

// Posterior summaries of parameter i (§3.1) from C chains' running means and
// mean squares, pooled over the chains: mean = (1/C) sum_c mean_c, msq = (1/C)
// sum_c msq_c, sd = sqrt(msq - mean^2) (0 where rounding makes it negative), and
// the normal-approximation interval mean -/+ z sd.  out: [4][n] = mean, sd, lo, hi.
__global__ void k_estimates(RhatInput in, double z, double* __restrict__ out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= in.n) return;
  double mean = 0.0, msq = 0.0;
  for (int c = 0; c < in.C; ++c) {
    if (in.f32) {
      const float* b = in.mf[c];
      mean += (double)b[i] - (double)b[in.n + i];
      msq += (double)b[2 * in.n + i] - (double)b[3 * in.n + i];
    } else {
      mean += in.m[c][i];
      msq += in.q[c][i];
    }
  }
  mean /= in.C;
  msq /= in.C;
  const double var = msq - mean * mean;
  const double sd = var > 0.0 ? sqrt(var) : 0.0;
  out[i] = mean;
  out[in.n + i] = sd;
  out[2 * in.n + i] = mean - z * sd;
  out[3 * in.n + i] = mean + z * sd;
}

cudaError_t launch_estimates(const RhatInput& in, double z, double* out, cudaStream_t s) {
  if (in.n <= 0) return cudaSuccess;
  const int blk = 128;
  k_estimates<<<(unsigned)((in.n + blk - 1) / blk), blk, 0, s>>>(in, z, out);
  return cudaGetLastError();
}

cudaError_t launch_rhat(const RhatInput& in, double* out, cudaStream_t s) {
  if (in.n <= 0) return cudaSuccess;
  const int blk = 128;
  k_rhat<<<(unsigned)((in.n + blk - 1) / blk), blk, 0, s>>>(in, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- set-up kernels

__global__ void k_set_run(Hyper* hy, long long burnin, long long tune_start, long long thin) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    hy->burnin = burnin;
    hy->tune_start = tune_start;
    hy->thin = thin;
  }
}

__global__ void k_init_run(Hyper* hy, long long trace_cap) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    hy->burnin = 0;
    hy->tune_start = 0;
    hy->thin = 1;
    hy->trace_cap = trace_cap;
  }
}

// y to [N][G]; T[l][g] = sum_n y X_nl; default beta_g = P (log(y+1) - h); eps = 0;
// gamma = 1; widths w0; tuning sums and moments 0.
__global__ void k_init_genes(ModelConst mc, DevPtrs p, const int32_t* y_in, int gene_major,
                             const double* __restrict__ pinv, double w0, int set_state) {
  const int G = mc.G, N = mc.N, L = mc.L;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    double r[kMaxN];
    double T[kMaxL];
#pragma unroll
    for (int l = 0; l < kMaxL; ++l) T[l] = 0.0;
    for (int n = 0; n < N; ++n) {
      const int32_t yv = gene_major ? y_in[(size_t)g * N + n] : y_in[(size_t)n * G + g];
      const_cast<int32_t*>(p.y)[(size_t)n * G + g] = yv;
      r[n] = log((double)yv + 1.0) - mc.h[n];
#pragma unroll
      for (int l = 0; l < kMaxL; ++l)
        if (l < L) T[l] += (double)yv * mc.X[n * kMaxL + l];
    }
    for (int l = 0; l < L; ++l) {
      const_cast<double*>(p.T)[(size_t)l * G + g] = T[l];
      if (set_state) {
        double s = 0.0;
        for (int n = 0; n < N; ++n) s += pinv[l * kMaxN + n] * r[n];
        p.beta[(size_t)l * G + g] = s;
        p.w_beta[(size_t)l * G + g] = w0;
        p.waux_beta[(size_t)l * G + g] = 0.0;
      }
    }
    if (set_state) {
      for (int n = 0; n < N; ++n) {
        p.eps[(size_t)n * G + g] = 0.0;
        p.w_eps[(size_t)n * G + g] = w0;
        p.waux_eps[(size_t)n * G + g] = 0.0;
      }
      p.gam[g] = 1.0;
      if (p.w_gam) {
        p.w_gam[g] = w0;
        p.waux_gam[g] = 0.0;
      }
    }
  }
}

// Zero the running moments and the chain bookkeeping.
__global__ void k_zero_moments(ModelConst mc, DevPtrs p) {
  const int G = mc.G, N = mc.N, L = mc.L;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    if (p.m_eps)
      for (int n = 0; n < N; ++n) {
        p.m_eps[(size_t)n * G + g] = 0.0;
        p.q_eps[(size_t)n * G + g] = 0.0;
      }
    for (int l = 0; l < L; ++l) {
      p.m_beta[(size_t)l * G + g] = 0.0;
      p.q_beta[(size_t)l * G + g] = 0.0;
    }
    p.m_gam[g] = 0.0;
    p.q_gam[g] = 0.0;
  }
}

// Default hyperparameters from the starting beta: theta_l the mean, sigma_l^2 the
// variance clamped to [1e-6, s_l^2/4] (two passes, one block), nu = min(3, d/2),
// tau = 1.
__global__ void k_init_hyper(ModelConst mc, Hyper* hy, const double* beta_d,
                             const float* beta_f, double w0, int set_state) {
  __shared__ double red[1024 / 32][kMaxL];
  __shared__ double mean_s[kMaxL];
  const int G = mc.G, L = mc.L;
  if (set_state) {
    for (int pass = 0; pass < 2; ++pass) {
      double acc[kMaxL];
#pragma unroll
      for (int l = 0; l < kMaxL; ++l) acc[l] = 0.0;
      for (int g = threadIdx.x; g < G; g += blockDim.x) {
#pragma unroll
        for (int l = 0; l < kMaxL; ++l) {
          if (l < L) {
            const size_t e = (size_t)l * G + g;
            const double b = beta_d ? beta_d[e] : (double)beta_f[e];
            if (pass == 0) acc[l] += b;
            else {
              const double dv = b - mean_s[l];
              acc[l] += dv * dv;
            }
          }
        }
      }
#pragma unroll
      for (int l = 0; l < kMaxL; ++l) {
        double x = acc[l];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][l] = x;
      }
      __syncthreads();
      if (threadIdx.x < L) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][threadIdx.x];
        if (pass == 0) mean_s[threadIdx.x] = s / (double)G;
        else {
          const double var = s / (double)G;
          const double upper = 0.25 * mc.s2[threadIdx.x];
          hy->phi[2 + threadIdx.x] = mean_s[threadIdx.x];
          hy->phi[2 + L + threadIdx.x] = fmin(fmax(var, 1e-6), upper);
        }
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) {
    if (set_state) {
      hy->phi[0] = fmin(3.0, 0.5 * mc.d);
      hy->phi[1] = 1.0;
      hy->w_nu = w0;
      hy->waux_nu = 0.0;
      for (int i = 0; i <= kMaxL; ++i) {
        hy->w_hyp[i] = w0;
        hy->waux_hyp[i] = 0.0;
      }
      hy->it = 0;
    }
    for (int i = 0; i < kMaxP; ++i) {
      hy->m_phi[i] = 0.0;
      hy->q_phi[i] = 0.0;
    }
    hy->n_mom = 0;
    hy->trace_rows = 0;
    hy->flags = 0;
  }
}

// ---------------------------------------------------------------- uniforms, ESS

__global__ void k_uniforms(uint32_t seed_lo, uint32_t seed_hi, uint32_t chain, uint32_t stream,
                           uint32_t index0, int n_index, uint32_t iter, uint32_t k0, int n_k,
                           double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_index) return;
  Rng r(seed_lo, seed_hi, chain, stream, index0 + (uint32_t)i, iter);
  for (int k = 0; k < n_k; ++k) out[(size_t)i * n_k + k] = r.u(k0 + (uint32_t)k);
}

// Geyer initial-monotone-sequence ESS of every column of a [rows][S] trace:
// one thread per series, reading row by row (consecutive series are adjacent).
__global__ void k_ess(const double* __restrict__ tr, long long rows, long long S, double* ess) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const long long n = rows;
  double mean = 0.0;
  for (long long t = 0; t < n; ++t) mean += tr[t * S + s];
  mean /= (double)n;
  double c0 = 0.0;
  for (long long t = 0; t < n; ++t) {
    const double dv = tr[t * S + s] - mean;
    c0 += dv * dv;
  }
  c0 /= (double)n;
  if (!(c0 > 0.0)) {
    ess[s] = (double)n;
    return;
  }
  double sum = 0.0, prev = INFINITY;
  for (long long j = 0; 2 * j + 1 < n; ++j) {
    double pair = 0.0;
    for (long long k = 2 * j; k <= 2 * j + 1; ++k) {
      double ck = 0.0;
      for (long long t = 0; t + k < n; ++t)
        ck += (tr[t * S + s] - mean) * (tr[(t + k) * S + s] - mean);
      pair += ck / (double)n / c0;
    }
    if (!(pair > 0.0)) break;
    if (pair > prev) pair = prev;
    sum += pair;
    prev = pair;
  }
  double tau = -1.0 + 2.0 * sum;
  if (tau < 1.0 / (double)n) tau = 1.0 / (double)n;
  ess[s] = (double)n / tau;
}

// ---------------------------------------------------------------- launchers

size_t gene_smem_bytes(int N, int block) {
  return (size_t)N * block * sizeof(double) + (size_t)(block / 32) * kNumPart * sizeof(double);
}

cudaError_t launch_gene(const ModelConst& mc, const DevPtrs& p, int block, cudaStream_t s) {
  const int nblk = (mc.G + block - 1) / block;
  k_gene_f64<<<nblk, block, gene_smem_bytes(mc.N, block), s>>>(mc, p);
  return cudaGetLastError();
}

cudaError_t launch_hyper(const ModelConst& mc, const DevPtrs& p, int nblk, cudaStream_t s) {
  k_hyper<<<1, kHyperThreads, 0, s>>>(mc, p, nblk);
  return cudaGetLastError();
}

size_t gb_smem_bytes_f64(int N, int block) {
  return ((size_t)N + kMaxL + kNumPart) * block * sizeof(double) +
         (size_t)(block / 32) * kNumPart * sizeof(double);
}

cudaError_t prepare_gene_kernel(int N, int block) {
  const size_t smem = gene_smem_bytes(N, block);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_gene_f64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  const size_t smem_gb = gb_smem_bytes_f64(N, block);
  if (smem_gb > 48 * 1024)
    return cudaFuncSetAttribute(k_gb_f64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_gb);
  return cudaSuccess;
}

cudaError_t launch_eps_f64(const ModelConst& mc, const DevPtrs& p, int seg_i, cudaStream_t s) {
  const int blk = 256;
  const dim3 grid((unsigned)((mc.G + blk - 1) / blk), (unsigned)mc.N);
  k_eps_f64<<<grid, blk, 0, s>>>(mc, p, seg_i);
  return cudaGetLastError();
}

cudaError_t launch_gb_f64(const ModelConst& mc, const DevPtrs& p, int block, int seg_i,
                          cudaStream_t s) {
  const int nblk = (mc.G + block - 1) / block;
  k_gb_f64<<<nblk, block, gb_smem_bytes_f64(mc.N, block), s>>>(mc, p, seg_i);
  return cudaGetLastError();
}

cudaError_t launch_set_run(Hyper* hy, long long burnin, long long tune_start, long long thin,
                           cudaStream_t s) {
  k_set_run<<<1, 32, 0, s>>>(hy, burnin, tune_start, thin);
  return cudaGetLastError();
}

cudaError_t launch_init(const ModelConst& mc, const DevPtrs& p, const int32_t* y_in,
                        int gene_major, const double* pinv, double w0, int set_state,
                        long long trace_cap, cudaStream_t s) {
  const int blk = 256;
  const int grid = (mc.G + blk - 1) / blk;
  k_init_run<<<1, 32, 0, s>>>(p.hyp, trace_cap);
  k_init_genes<<<grid, blk, 0, s>>>(mc, p, y_in, gene_major, pinv, w0, set_state);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_zero_moments<<<grid, blk, 0, s>>>(mc, p);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_init_hyper<<<1, 1024, 0, s>>>(mc, p.hyp, p.beta, nullptr, w0, set_state);
  return cudaGetLastError();
}

cudaError_t launch_zero_moments(const ModelConst& mc, const DevPtrs& p, cudaStream_t s) {
  const int blk = 256;
  const int grid = (mc.G + blk - 1) / blk;
  k_zero_moments<<<grid, blk, 0, s>>>(mc, p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_init_hyper<<<1, 1024, 0, s>>>(mc, p.hyp, p.beta, nullptr, 0.0, 0);
  return cudaGetLastError();
}

cudaError_t launch_init_hyper(const ModelConst& mc, Hyper* hy, const double* beta_d,
                              const float* beta_f, double w0, int set_state, cudaStream_t s) {
  k_init_hyper<<<1, 1024, 0, s>>>(mc, hy, beta_d, beta_f, w0, set_state);
  return cudaGetLastError();
}

cudaError_t launch_init_run(Hyper* hy, long long trace_cap, cudaStream_t s) {
  k_init_run<<<1, 32, 0, s>>>(hy, trace_cap);
  return cudaGetLastError();
}

cudaError_t launch_uniforms(uint64_t seed, uint32_t chain, uint32_t stream, uint32_t index0,
                            int n_index, uint32_t iter, uint32_t k0, int n_k, double* out,
                            cudaStream_t s) {
  const int blk = 128;
  k_uniforms<<<(n_index + blk - 1) / blk, blk, 0, s>>>((uint32_t)seed, (uint32_t)(seed >> 32),
                                                        chain, stream, index0, n_index, iter, k0,
                                                        n_k, out);
  return cudaGetLastError();
}

cudaError_t launch_ess(const double* tr, long long rows, long long S, double* ess,
                       cudaStream_t s) {
  const int blk = 128;
  k_ess<<<(unsigned)((S + blk - 1) / blk), blk, 0, s>>>(tr, rows, S, ess);
  return cudaGetLastError();
}

}  // namespace fbs
