// fbs_hyper.cuh -- the hyperparameter steps of one Gibbs sweep (Algorithm 1
// steps 3, 4, 6, 7 of Landau & Niemi, arXiv 1606.06659) as a block-level device
// function, shared by the single-chain and the batched hyperparameter kernels.
// tau and sigma_l^2 are drawn exactly, or (ModelConst::all_slice) by slice
// updates of their conditionals: tau spread over warp 0, sigma_l on lane 32+l.
#pragma once

#include <math.h>
#include <stdint.h>

#include "fbs_common.cuh"
#include "fbs_rng.cuh"

namespace fbs {

// ---------------------------------------------------------------- hyper kernel

// log f(nu | ...) = -G lgamma(nu/2) + (G nu/2) log(nu tau/2) - (nu/2)(S1 + tau S2) on
// (0, d), S1 = sum_g log gamma_g, S2 = sum_g 1/gamma_g (Algorithm 1 step 3, the
// sum read as log gamma_g + tau/gamma_g, which the Inverse-Gamma(nu/2, nu tau/2)
// prior of the gamma_g gives).
struct NuDensity {
  double G, d, tau, S1, S2;
  // out of line: one copy of lgamma and log for every evaluation point (see
  // hyper_gamma below)
  __device__ __noinline__ double operator()(double nu, double* aux) const {
    *aux = 0.0;
    if (!(nu > 0.0 && nu < d)) return -INFINITY;
    return -G * lgamma(0.5 * nu) + 0.5 * G * nu * log(0.5 * nu * tau) -
           0.5 * nu * (S1 + tau * S2);
  }
};

// log f(tau | ...) = (shape - 1) log tau - rate tau on tau > 0, shape = a + G nu/2,
// rate = b + (nu/2) S2: the Gamma full conditional of step 4, slice-sampled in the
// all-slice variant (Section 4.2).
struct TauDensity {
  double shape, rate;
  __device__ __forceinline__ double operator()(double x, double* aux) const {
    *aux = 0.0;
    if (!(x > 0.0)) return -INFINITY;
    return (shape - 1.0) * log(x) - rate * x;
  }
};

// log f(sigma_l | ...) = -G log sigma_l - hS / sigma_l^2 on 0 < sigma_l < s_l, hS =
// sum_g (beta_gl - theta_l)^2 / 2: G Normal(theta_l, sigma_l^2) terms times the flat
// Uniform(0, s_l) prior, the step 7 conditional of sigma_l itself (all-slice variant).
struct SigDensity {
  double G, hS, s;
  __device__ __forceinline__ double operator()(double x, double* aux) const {
    *aux = 0.0;
    if (!(x > 0.0 && x < s)) return -INFINITY;
    return -G * log(x) - hS / (x * x);
  }
};

// Out-of-line copies of the transcendental-heavy steps (one copy each in the
// kernel's code instead of one per call site).
static __device__ __noinline__ double hyper_gamma(double shape, Rng& r, uint32_t k0, bool* capped) {
  return gamma_mt(shape, r, k0, capped);
}

static __device__ __noinline__ double hyper_normal(Rng& r, uint32_t k0) { return normal_bm(r, k0); }

// The first attempts of a Marsaglia-Tsang draw whose shape is not known yet:
// the normal x_j = normal_bm(r, k0 + 4j) and the uniform u_j = r.u(k0 + 4j + 2)
// of attempts j < kPreAttempts, with log u_j.  They depend only on the random
// numbers, so another warp computes them while the shape is being found.
constexpr int kPreAttempts = 2;
struct GammaPre {
  double x[kPreAttempts], u[kPreAttempts], logu[kPreAttempts];
};

static __device__ __noinline__ void gamma_pre(Rng& r, uint32_t k0, GammaPre* g) {
  for (int j = 0; j < kPreAttempts; ++j) {
    g->x[j] = normal_bm(r, k0 + 4u * (uint32_t)j);
    g->u[j] = r.u(k0 + 4u * (uint32_t)j + 2u);
    g->logu[j] = log(g->u[j]);
  }
}

// gamma_mt(shape, r, k0, capped) with the first attempts' random quantities
// taken from *g: the same operations on the same numbers, so the same result.
// A shape below 1 needs the boost uniform and takes gamma_mt itself.
static __device__ __noinline__ double gamma_mt_pre(double shape, const GammaPre* g, Rng& r,
                                                  uint32_t k0, bool* capped) {
  if (shape < 1.0) return gamma_mt(shape, r, k0, capped);
  const double dd = __dsub_rn(shape, 1.0 / 3.0);
  const double cc = 1.0 / sqrt(__dmul_rn(9.0, dd));
  for (uint32_t j = 0; j < (uint32_t)kGammaAttempts; ++j) {
    const bool pre = j < (uint32_t)kPreAttempts;
    const double x = pre ? g->x[j] : normal_bm(r, k0 + 4 * j);
    double v = __dadd_rn(1.0, __dmul_rn(cc, x));
    if (v <= 0.0) continue;
    v = __dmul_rn(__dmul_rn(v, v), v);
    const double u = pre ? g->u[j] : r.u(k0 + 4 * j + 2);
    const double x2 = __dmul_rn(x, x);
    if (u < __dsub_rn(1.0, __dmul_rn(__dmul_rn(0.0331, x2), x2)))
      return __dmul_rn(__dmul_rn(dd, v), 1.0);
    const double rhs = __dadd_rn(__dmul_rn(0.5, x2),
                                 __dmul_rn(dd, __dadd_rn(__dsub_rn(1.0, v), log(v))));
    if ((pre ? g->logu[j] : log(u)) < rhs) return __dmul_rn(__dmul_rn(dd, v), 1.0);
  }
  *capped = true;
  return shape;
}

// trunc_invgamma of fbs_rng.cuh whose first attempt's gamma draw gv0 (with its
// cap flag) was made beforehand; later attempts draw their own.
static __device__ __noinline__ double hyper_trunc_invgamma(double shape, double scale,
                                                           double upper, double keep, double gv0,
                                                           bool gcap0, Rng& r, bool* gcap,
                                                           bool* tcap) {
  *gcap = *gcap || gcap0;
  const double x0 = scale / gv0;
  if (x0 < upper) return x0;
  for (uint32_t t = 1; t < (uint32_t)kTruncAttempts; ++t) {
    const double gv = hyper_gamma(shape, r, kTruncStride * t, gcap);
    const double x = scale / gv;
    if (x < upper) return x;
  }
  *tcap = true;
  return keep;
}

// Four warps: warp 0 the nu slice update then tau, warp 1 theta_l then sigma_l^2
// (lane l), warp 2 the first gamma draw of every sigma_l^2 (its shape (G-1)/2 is
// known), warp 3 the random quantities of tau's first draw attempts; warps 2
// and 3 hand their results over through named barriers 1 and 2.
constexpr int kHyperThreads = 128;
// the partial sums are read by 7 threads per column (126 threads): thread t takes
// column t mod kNumPart and every 7th row from row t / kNumPart
constexpr int kRedRows = kHyperThreads / kNumPart;

__device__ __forceinline__ void named_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int count) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Steps 3, 4, 6, 7 for one chain, executed by one block of kHyperThreads threads:
// the chain's `nblk` per-block partial sums are folded in a fixed order.  psi:
// null, or the top level (b, m_1..m_L) of the three-level model, which replaces
// the rate b of the tau prior and the zero mean of the theta_l priors.
__device__ __forceinline__ void hyper_body(const ModelConst& mc, const double* partial, Hyper* hy,
                                           double* trace_phi, unsigned long long* counters,
                                           int nblk, const double* psi = nullptr) {
  __shared__ double red[kRedRows][kNumPart];
  __shared__ double tot[kNumPart];
  __shared__ double phi_new[kMaxP];
  __shared__ Hyper sh;  // a copy of the chain's Hyper block: one load instead of a
                        // chain of dependent global reads on the serial path
  __shared__ GammaPre tau_pre;           // from warp 3, for warp 0
  __shared__ double sig_g[kMaxL];        // from warp 2, for warp 1
  __shared__ int sig_gcap[kMaxL];
  static_assert(sizeof(Hyper) % 8 == 0, "Hyper is copied as 8-byte words");
  static_assert(kRedRows * kNumPart <= kHyperThreads && kHyperThreads == 128, "warp roles");
  const int L = mc.L, P = mc.P;
  const double G = (double)mc.G;
  const int tid = threadIdx.x;
  for (int i = tid; i < (int)(sizeof(Hyper) / 8); i += kHyperThreads)
    reinterpret_cast<unsigned long long*>(&sh)[i] = reinterpret_cast<const unsigned long long*>(hy)[i];
  const long long it = hy->it + 1;
  const uint32_t it32 = (uint32_t)it;

  // fixed-order reduction of the per-block partials: thread t sums column
  // t mod kNumPart over rows t / kNumPart + kRedRows k (two interleaved
  // accumulators, added at the end); consecutive threads read consecutive words
  if (tid < kRedRows * kNumPart) {
    const int col = tid % kNumPart, r0 = tid / kNumPart;
    double a0 = 0.0, a1 = 0.0;
    int b = r0;
    for (; b + kRedRows < nblk; b += 2 * kRedRows) {
      a0 += partial[(size_t)b * kNumPart + col];
      a1 += partial[(size_t)(b + kRedRows) * kNumPart + col];
    }
    if (b < nblk) a0 += partial[(size_t)b * kNumPart + col];
    red[r0][col] = a0 + a1;
  }
  __syncthreads();
  if (tid < kMaxP) phi_new[tid] = tid < P ? sh.phi[tid] : 0.0;
  if (tid < kNumPart) {
    double s = 0.0;
    for (int r = 0; r < kRedRows; ++r) s += red[r][tid];
    tot[tid] = s;
  }
  __syncthreads();

  const double S1 = tot[0], S2 = tot[1];
  if (tid < 32) {
    // step 3: nu, the slice update spread over warp 0
    const double tau_old = sh.phi[1];
    NuDensity f{G, mc.d, tau_old, S1, S2};
    Rng r(mc.seed_lo, mc.seed_hi, mc.chain, kStreamNu, 0u, it32);
    const double x0 = sh.phi[0];
    SliceResult s = slice_update_warp(x0, sh.w_nu, f, r, mc.K, mc.shrink_max);
    const double nu = s.x;
    if (!mc.all_slice) named_sync(2, 64);  // tau_pre from warp 3
    Rng rt(mc.seed_lo, mc.seed_hi, mc.chain, kStreamTau, 0u, it32);
    const double shape = mc.a + 0.5 * G * nu;
    const double rate = (psi ? psi[0] : mc.b) + 0.5 * nu * S2;
    SliceResult st;
    if (mc.all_slice)  // step 4 by a slice update of the Gamma conditional, on warp 0
      st = slice_update_warp(sh.phi[1], sh.w_hyp[0], TauDensity{shape, rate}, rt, mc.K,
                             mc.shrink_max);
    if (tid == 0) {
      if (it <= sh.burnin) {
        double w = sh.w_nu, waux = sh.waux_nu;
        tune_width(w, waux, it, nu, x0, sh.burnin, sh.tune_start);
        hy->w_nu = w;
        hy->waux_nu = waux;
      }
      atomicAdd(&counters[FBS_CNT_EVALS_NU], (unsigned long long)s.evals);
      if (s.capped) atomicAdd(&counters[FBS_CNT_SLICE_CAPS], 1ull);
      if (s.nonfinite) {
        atomicAdd(&counters[FBS_CNT_NONFINITE], 1ull);
        atomicOr(&hy->flags, kFlagNonfinite);
      }
      // step 4: tau ~ Gamma(a + G nu/2, rate b + nu S2 / 2)
      double tau;
      if (mc.all_slice) {
        tau = st.x;
        if (it <= sh.burnin) {
          double w = sh.w_hyp[0], waux = sh.waux_hyp[0];
          tune_width(w, waux, it, tau, sh.phi[1], sh.burnin, sh.tune_start);
          hy->w_hyp[0] = w;
          hy->waux_hyp[0] = waux;
        }
        atomicAdd(&counters[FBS_CNT_EVALS_HYPER], (unsigned long long)st.evals);
        if (st.capped) atomicAdd(&counters[FBS_CNT_SLICE_CAPS], 1ull);
        if (st.nonfinite) {
          atomicAdd(&counters[FBS_CNT_NONFINITE], 1ull);
          atomicOr(&hy->flags, kFlagNonfinite);
        }
      } else {
        bool gcap = false;
        tau = gamma_mt_pre(shape, &tau_pre, rt, 0, &gcap) / rate;
        if (gcap) atomicAdd(&counters[FBS_CNT_GAMMA_CAPS], 1ull);
      }
      phi_new[0] = nu;
      phi_new[1] = tau;
    }
  } else if (tid < 64) {
    const int l = tid - 32;
    const bool on = l < L;
    // step 6: theta_l ~ N(v B1 / sigma^2, v), v = 1/(G/sigma^2 + 1/c^2);
    // the partials hold B1' = sum (beta - theta_old), B2' = sum (beta - theta_old)^2
    double th = 0.0, th_old = 0.0, sig2 = 0.0, S = 0.0;
    if (on) {
      th_old = sh.phi[2 + l];
      sig2 = sh.phi[2 + L + l];
      const double B1s = tot[2 + l], B2s = tot[2 + kMaxL + l];
      const double B1 = B1s + G * th_old;
      const double v = 1.0 / (G / sig2 + 1.0 / mc.c2[l]);
      const double mean = psi ? v * (B1 / sig2 + psi[1 + l] / mc.c2[l]) : v * B1 / sig2;
      Rng r(mc.seed_lo, mc.seed_hi, mc.chain, kStreamTheta, (uint32_t)l, it32);
      th = mean + sqrt(v) * hyper_normal(r, 0);
      const double dl = th - th_old;
      S = B2s - 2.0 * dl * B1s + G * dl * dl;
    }
    if (!mc.all_slice) named_sync(1, 64);  // sig_g from warp 2
    if (on) {
      // step 7: sigma_l^2 ~ IG((G-1)/2, S/2) on (0, s_l^2), S = sum (beta - theta_new)^2
      Rng rs(mc.seed_lo, mc.seed_hi, mc.chain, kStreamSigma, (uint32_t)l, it32);
      double s2n;
      if (mc.all_slice) {
        // a slice update of sigma_l itself on (0, s_l); the state keeps sigma_l^2
        const double x0 = sqrt(sig2);
        SliceResult ss = slice_update(x0, sh.w_hyp[1 + l], SigDensity{G, 0.5 * S, mc.s[l]}, rs,
                                      mc.K, mc.shrink_max);
        s2n = ss.x * ss.x;
        if (it <= sh.burnin) {
          double w = sh.w_hyp[1 + l], waux = sh.waux_hyp[1 + l];
          tune_width(w, waux, it, ss.x, x0, sh.burnin, sh.tune_start);
          hy->w_hyp[1 + l] = w;
          hy->waux_hyp[1 + l] = waux;
        }
        atomicAdd(&counters[FBS_CNT_EVALS_HYPER], (unsigned long long)ss.evals);
        if (ss.capped) atomicAdd(&counters[FBS_CNT_SLICE_CAPS], 1ull);
        if (ss.nonfinite) {
          atomicAdd(&counters[FBS_CNT_NONFINITE], 1ull);
          atomicOr(&hy->flags, kFlagNonfinite);
        }
      } else {
        bool gcap = false, tcap = false;
        s2n = hyper_trunc_invgamma(0.5 * (G - 1.0), 0.5 * S, mc.s2[l], sig2, sig_g[l],
                                   sig_gcap[l] != 0, rs, &gcap, &tcap);
        if (gcap) atomicAdd(&counters[FBS_CNT_GAMMA_CAPS], 1ull);
        if (tcap) atomicAdd(&counters[FBS_CNT_TRUNC_CAPS], 1ull);
      }
      phi_new[2 + l] = th;
      phi_new[2 + L + l] = s2n;
    }
  } else if (tid < 96) {
    // the first truncated-draw attempt of every sigma_l^2: a Gamma((G-1)/2) draw
    if (!mc.all_slice) {
      const int l = tid - 64;
      if (l < L) {
        Rng rs(mc.seed_lo, mc.seed_hi, mc.chain, kStreamSigma, (uint32_t)l, it32);
        bool gcap = false;
        sig_g[l] = hyper_gamma(0.5 * (G - 1.0), rs, 0, &gcap);
        sig_gcap[l] = gcap ? 1 : 0;
      }
      named_arrive(1, 64);
    }
  } else {
    // the random quantities of tau's first draw attempts
    if (!mc.all_slice) {
      if (tid == 96) {
        Rng rt(mc.seed_lo, mc.seed_hi, mc.chain, kStreamTau, 0u, it32);
        gamma_pre(rt, 0, &tau_pre);
      }
      named_arrive(2, 64);
    }
  }
  __syncthreads();

  const bool mom = it > sh.burnin;
  if (tid < P) {
    const double x = phi_new[tid];
    hy->phi[tid] = x;
    if (mom) {
      const double inv_k = 1.0 / (double)(sh.n_mom + 1);
      const double m = sh.m_phi[tid], q = sh.q_phi[tid];
      hy->m_phi[tid] = m + (x - m) * inv_k;
      hy->q_phi[tid] = q + (x * x - q) * inv_k;
    }
    if (mom && ((it - sh.burnin) % sh.thin == 0) && sh.trace_rows < sh.trace_cap &&
        trace_phi != nullptr)
      trace_phi[(size_t)sh.trace_rows * P + tid] = x;
  }
  __syncthreads();
  if (tid == 0) {
    if (mom && ((it - sh.burnin) % sh.thin == 0) && sh.trace_rows < sh.trace_cap)
      hy->trace_rows = sh.trace_rows + 1;
    if (mom) hy->n_mom = sh.n_mom + 1;
    hy->it = it;
    atomicAdd(&counters[FBS_CNT_SWEEPS], 1ull);
  }
}

}  // namespace fbs
