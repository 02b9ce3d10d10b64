// fbs_gene_f32.cu -- the per-gene kernel of the Gibbs sweep in its FP32 form
// (Landau & Niemi, arXiv 1606.06659, Algorithm 1 steps 1, 2, 5 with Algorithm
// 2), plus its set-up kernels.
//
// Slice evaluations run in FP32 on the log density relative to the start
// point x0, Delta(x) = log f(x) - log f(x0), written so that no two large terms
// cancel:
//   eps:  Delta(x) = d (y - mu0) - mu0 (e^d - 1 - d) - d (d + 2 x0) / (2 gamma)
//   beta: Delta(b) = sum_j [v_j d (Y_j - Q_j) - Q_j (e^{v_j d} - 1 - v_j d)]
//                    - d (d + 2 (b0 - theta)) / (2 sigma^2)
// with d = x - x0, mu0 = exp(h + x0 + X beta) the Poisson mean at x0, Y_j and
// Q_j the counts and Poisson means summed over the samples whose X_nl is the
// j-th distinct value v_j of column l.  Since Delta(x0) = 0, the slice level is
// log U and no evaluation at x0 is needed.  Uniforms are 23-bit FP32 numbers,
// four per Philox block.  The partial sums for the hyperparameter steps are
// reduced exactly to FP64 (error-free FP32 pair sums within a warp, FP64
// across warps and blocks), and the running moments are Kahan-compensated
// FP32 pairs.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fbs_common.cuh"
#include "fbs_kernels.h"
#include "fbs_rng.cuh"
#include "fbs_hyper.cuh"
#include "fbs_tc.cuh"

namespace fbs {

// ---------------------------------------------------------------- FP32 random numbers

// The uniforms of one random variable in the FP32 form: uniform k is word k%4 of
// Philox block k/4, as ((w >> 9) + 1/2) / 2^23 (exact in FP32, inside (0,1)).
struct Rng4 {
  uint32_t key0, key1, index, sblk, iter, chain;
  uint32_t cached;
  uint4 w;

  __device__ __forceinline__ Rng4(uint32_t seed_lo, uint32_t seed_hi, uint32_t chain_,
                                  uint32_t stream, uint32_t index_, uint32_t iter_)
      : key0(seed_lo), key1(seed_hi), index(index_), sblk(stream << 24), iter(iter_),
        chain(chain_), cached(0xFFFFFFFFu), w(make_uint4(0, 0, 0, 0)) {}

  __device__ __forceinline__ float u(uint32_t k) {
    const uint32_t blk = k >> 2;
    if (blk != cached) {
      w = philox4x32_10(make_uint4(index, sblk | blk, iter, chain), key0, key1);
      cached = blk;
    }
    const uint32_t j = k & 3u;
    const uint32_t x = j == 0 ? w.x : (j == 1 ? w.y : (j == 2 ? w.z : w.w));
    return word(x);
  }

  // The uniform of Philox word x.
  static __device__ __forceinline__ float word(uint32_t x) {
    return __fmul_rn(__fadd_rn(__uint2float_rn(x >> 9), 0.5f), 0x1p-23f);
  }

  // Philox block blk (uniforms 4 blk .. 4 blk + 3), cached.
  __device__ __forceinline__ uint4 block(uint32_t blk) {
    if (blk != cached) {
      w = philox4x32_10(make_uint4(index, sblk | blk, iter, chain), key0, key1);
      cached = blk;
    }
    return w;
  }
};

__device__ __forceinline__ float normal_bm_f(Rng4& r, uint32_t k0) {
  const float u1 = r.u(k0), u2 = r.u(k0 + 1);
  return sqrtf(-2.0f * __logf(u1)) * __cosf(6.2831853071795865f * u2);
}

// Gamma(shape, 1), Marsaglia & Tsang (2000), uniform layout as in the FP64 form.
__device__ __forceinline__ float gamma_mt_f(float shape, Rng4& r, uint32_t k0, bool* capped) {
  const float alpha = shape < 1.0f ? shape + 1.0f : shape;
  const float dd = alpha - (1.0f / 3.0f);
  const float cc = rsqrtf(9.0f * dd);
  float boost = 1.0f;
  if (shape < 1.0f) boost = __powf(r.u(k0 + 3), 1.0f / shape);
  for (uint32_t j = 0; j < (uint32_t)kGammaAttempts; ++j) {
    const float x = normal_bm_f(r, k0 + 4 * j);
    float v = 1.0f + cc * x;
    if (v <= 0.0f) continue;
    v = v * v * v;
    const float u = r.u(k0 + 4 * j + 2);
    const float x2 = x * x;
    if (u < 1.0f - 0.0331f * x2 * x2) return dd * v * boost;
    if (__logf(u) < 0.5f * x2 + dd * (1.0f - v + __logf(v))) return dd * v * boost;
  }
  *capped = true;
  return shape;
}

// ---------------------------------------------------------------- densities

struct EpsDensityF {
  float D, mu0, x0, hg;  // D = y - mu0, hg = 1 / (2 gamma)
  __device__ __forceinline__ float operator()(float x, float* aux) const {
    const float d = x - x0;
    const float e = em1mx(d);
    *aux = mu0 + mu0 * (d + e);
    return d * D - mu0 * e - d * (d + 2.0f * x0) * hg;
  }
};

// Relative log density of beta_gl: with d = b - b0 and the column's value
// classes j (value v_j, rate sum Q_j and count sum Y_j at b0, D_j = Y_j - Q_j),
// Delta(b) = sum_j [v_j d D_j - Q_j em1mx(v_j d)] - d (d + 2 (b0 - theta)) / (2 sigma^2).
// The class count NC is fixed at compile time, so that the loops run over the
// classes a column has (NC = kMaxCls keeps the runtime bound `ncls`).
template <int NC>
struct BetaDensityFT {
  float bt, hs, b0;
  int ncls;
  float Q[NC], D[NC], v[NC];
  __device__ __forceinline__ float operator()(float b, float* aux) const {
    const float d = b - b0;
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      if (NC < kMaxCls || j < ncls) {
        const float z = v[j] * d;
        s += z * D[j] - Q[j] * em1mx(z);
      }
    }
    *aux = d;
    return s - d * (d + 2.0f * bt) * hs;
  }
};

struct SliceResultF {
  float x, aux;
  unsigned evals;
  bool capped, nonfinite;
};

// Algorithm 2, steps 1-6, on Delta (Delta(x0) = 0): level log U_0, interval from
// U_1, K_L from U_2, the j-th shrinkage proposal from U_{3+j}.
template <class F>
__device__ __forceinline__ SliceResultF slice_update_f(float x0, float aux0, float w, const F& f,
                                                       Rng4& r, int K, int shrink_max) {
  SliceResultF res;
  res.evals = 0;
  res.nonfinite = !(isfinite(x0) && isfinite(aux0));
  const float logu = __logf(r.u(0));
  const float v = __fmul_rn(w, r.u(1));
  float lo = __fsub_rn(x0, v);
  float hi = __fadd_rn(lo, w);
  int KL = (int)__fmul_rn((float)(K + 1), r.u(2));
  if (KL > K) KL = K;
  const int KR = K - KL;
  float aux;
  for (int k = 0; k < KL; ++k) {
    ++res.evals;
    if (logu < f(lo, &aux)) lo = __fsub_rn(lo, w); else break;
  }
  for (int k = 0; k < KR; ++k) {
    ++res.evals;
    if (logu < f(hi, &aux)) hi = __fadd_rn(hi, w); else break;
  }
  // shrinkage: proposal j takes uniform 3 + j (word 3 of block 0, then the four
  // words of block 1, 2, ..), so that the word is a compile-time choice
  auto propose = [&](float u) -> bool {
    const float xs = __fadd_rn(lo, __fmul_rn(__fsub_rn(hi, lo), u));
    ++res.evals;
    if (logu < f(xs, &aux)) {
      res.x = xs;
      res.aux = aux;
      res.capped = false;
      return true;
    }
    if (xs > x0) hi = xs; else lo = xs;
    return false;
  };
  if (shrink_max > 0 && propose(Rng4::word(r.block(0u).w))) return res;
  for (int j = 1, b = 1; j < shrink_max; ++b) {
    const uint4 q = r.block((uint32_t)b);
    if (propose(Rng4::word(q.x))) return res;
    if (++j >= shrink_max) break;
    if (propose(Rng4::word(q.y))) return res;
    if (++j >= shrink_max) break;
    if (propose(Rng4::word(q.z))) return res;
    if (++j >= shrink_max) break;
    if (propose(Rng4::word(q.w))) return res;
    ++j;
  }
  res.x = x0;
  res.aux = aux0;
  res.capped = true;
  return res;
}

__device__ __forceinline__ void tune_width_f(float& w, float& waux, long long it, float x_new,
                                             float x_old, long long burnin, long long tune_start) {
  if (it > burnin) return;
  waux += (float)it * fabsf(x_new - x_old);
  if (it > tune_start) {
    const float wn = waux / (0.5f * (float)it * (float)(it + 1));
    if (wn > 0.0f && isfinite(wn)) w = wn;
  }
}

// Welford update of a Kahan-compensated FP32 pair (m, c) representing m - c.
__device__ __forceinline__ void welford_kahan(float* base, size_t plane, size_t e, float x,
                                              float inv_k) {
  float m = base[e], c = base[plane + e];
  float q = base[2 * plane + e], cq = base[3 * plane + e];
  {
    const float inc = (x - (m - c)) * inv_k;
    const float y = inc - c;
    const float t = m + y;
    c = __fsub_rn(__fsub_rn(t, m), y);
    m = t;
  }
  {
    const float inc = (x * x - (q - cq)) * inv_k;
    const float y = inc - cq;
    const float t = q + y;
    cq = __fsub_rn(__fsub_rn(t, q), y);
    q = t;
  }
  base[e] = m;
  base[plane + e] = c;
  base[2 * plane + e] = q;
  base[3 * plane + e] = cq;
}

// Error-free FP32 pair addition (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

// ---------------------------------------------------------------- sweep kernels (FP32)


// Warp sums of the counters, one atomic per warp into one of several copies.
__device__ __forceinline__ void add_counters(unsigned long long* base, unsigned evals_e,
                                             unsigned evals_b, unsigned caps, unsigned gcaps,
                                             unsigned nonfin, unsigned* flags) {
  unsigned v[5] = {evals_e, evals_b, caps, gcaps, nonfin};
#pragma unroll
  for (int i = 0; i < 5; ++i) v[i] = __reduce_add_sync(0xffffffffu, v[i]);  // warp sum
  if ((threadIdx.x & 31) == 0) {
    if (v[0]) atomicAdd(&base[FBS_CNT_EVALS_EPS], (unsigned long long)v[0]);
    if (v[1]) atomicAdd(&base[FBS_CNT_EVALS_BETA], (unsigned long long)v[1]);
    if (v[2]) atomicAdd(&base[FBS_CNT_SLICE_CAPS], (unsigned long long)v[2]);
    if (v[3]) atomicAdd(&base[FBS_CNT_GAMMA_CAPS], (unsigned long long)v[3]);
    if (v[4]) {
      atomicAdd(&base[FBS_CNT_NONFINITE], (unsigned long long)v[4]);
      atomicOr(flags, kFlagNonfinite);
    }
  }
}

// Step 1 of Algorithm 1 in the FP32 form: one thread per eps_gn (element e of
// the [N][G] planes).  It reads beta_g and gamma_g of the previous iteration and
// writes the new eps_gn and mu_gn = exp(h_n + eps_gn + X_n beta_g) for the
// gamma/beta kernel.  It involves no hyperparameter, so within a captured
// segment it runs concurrently with the hyperparameter kernel of the previous
// iteration; its iteration number comes from the segment snapshot.
__device__ __forceinline__ void eps_f32_body(const ModelConst& mc, const DevPtrsF32& p, int seg_i,
                                             int n, int g, int copy) {
  const int G = mc.G, N = mc.N, L = mc.L;
  const Hyper* hy = p.hyp;
  const long long it = hy->seg_it + seg_i + 1;
  const long long burnin = hy->burnin, tune_start = hy->tune_start;
  const bool mom = it > burnin;
  long long before = (it - 1) - (hy->seg_it > burnin ? hy->seg_it : burnin);
  if (before < 0) before = 0;
  const float inv_k = mom ? 1.0f / (float)(hy->seg_nmom + before + 1) : 0.0f;
  const size_t NG = (size_t)N * G;
  const size_t e = (size_t)n * G + g;
  unsigned evals = 0, caps = 0, nonfin = 0;
  if (g < G) {
    float A = mc.hf[n];
#pragma unroll
    for (int l = 0; l < kMaxL; ++l)
      if (l < L) A += mc.Xf[n * kMaxL + l] * p.beta[(size_t)l * G + g];
    const float hg = 0.5f / p.gam[g];
    const float x0 = p.eps[e];
    const float mu0 = expf(A + x0);
    EpsDensityF f{(float)p.y[e] - mu0, mu0, x0, hg};
    Rng4 r(mc.seed_lo, mc.seed_hi, mc.chain, kStreamEps, (uint32_t)((size_t)g * N + n),
           (uint32_t)it);
    float w = p.w_eps[e];
    SliceResultF s = slice_update_f(x0, mu0, w, f, r, mc.K, mc.shrink_max);
    evals = s.evals;
    caps = s.capped;
    nonfin = s.nonfinite;
    p.mu[e] = s.aux;
    p.eps[e] = s.x;
    if (it <= burnin) {
      float waux = p.waux_eps[e];
      tune_width_f(w, waux, it, s.x, x0, burnin, tune_start);
      p.w_eps[e] = w;
      p.waux_eps[e] = waux;
    }
    if (mom && mc.moments_eps) welford_kahan(p.mom_eps, NG, e, s.x, inv_k);
  }
  add_counters(p.counters + copy * FBS_NUM_COUNTERS, evals, 0, caps, 0, nonfin, &p.hyp->flags);
}

// At least 5 blocks of 256 per SM (at most 51 registers, no spills): 5 rather
// than 4 resident blocks took the kernel from 24.1 to 22.9 us at N=16 G=40000
// (6 blocks: 23.2 us).
__global__ void __launch_bounds__(256, 5) k_eps_f32(ModelConst mc, DevPtrsF32 p, int seg_i) {
  ktime_begin(p.ktime, p.ktime_n, 3 * seg_i);
  eps_f32_body(mc, p, seg_i, blockIdx.y, blockIdx.x * blockDim.x + threadIdx.x,
               (blockIdx.x + blockIdx.y) % kCounterCopies);
  ktime_end(p.ktime, p.ktime_n, 3 * seg_i);
}

// Which proposal gene g uses at iteration it: 0 none, kMoveNet the network's,
// kMovePrior the prior-centred one.  p.mh_all = 0: the calibrated per-gene
// choice; 1 or 2: that kind for every gene; 3 (calibration): every gene, the
// network on even and the prior on odd iterations.
__device__ __forceinline__ int move_kind(const DevPtrsF32& p, int g, long long it) {
  if (p.mh_all == 3) return (it & 1) ? kMovePrior : kMoveNet;
  if (p.mh_all) return p.mh_all;
  return (int)p.use_mh[g];
}

// The learned-proposal move of gene g (FP32): beta* from the multivariate t
// distribution with kTDof degrees of freedom, centre mu and scale C C^T given by
// the proposal network (beta* = mu + s C xi, s = sqrt(kTDof / chi2)), and
// eps* = eps - X (beta* - beta), so that every log-rate h_n + eps_n + X_n beta is
// unchanged and the Poisson likelihood cancels; accepted with probability
// min(1, pi(eps*, beta*) q(beta) / (pi(eps, beta) q(beta*))), where pi holds the
// Normal(0, gamma) priors of eps and the Normal(theta, sigma^2) priors of beta.
// The proposal depends only on quantities the move leaves unchanged, so this is
// an exact Metropolis-Hastings step; the t tails dominate the target's Gaussian
// tails, which keeps the ratio target / proposal bounded (uniform ergodicity).
// Uniforms 0..2L-1 give the normals, uniform 2L the acceptance and uniforms
// 2L+1..2L+4 the chi-square variate chi2 = -2 log(U1 U2 U3 U4) (kTDof = 8).
// kind kMoveNet takes the centre and scale from the network; kind kMovePrior
// from the hyperparameters alone (centre theta, scale diag(sigma)), which suits
// genes whose conditional is close to the prior (very large gamma_g), where the
// network, trained mostly on typical genes, extrapolates poorly.  Either way
// the proposal depends only on quantities the move keeps.
// The network's outputs are read from prop[k pstride + pidx].  Returns true
// when accepted.
constexpr int kTDof = 8;

__device__ __forceinline__ bool mh_move_f32(const ModelConst& mc, const DevPtrsF32& p, int g,
                                            uint32_t it32, float* bs, int B, int tid,
                                            const Hyper* hy, float hg, int kind,
                                            const float* prop, size_t pstride, int pidx) {
  const int G = mc.G, N = mc.N, L = mc.L;
  float mu[kMaxL], C[kMaxL][kMaxL], xi[kMaxL], bn[kMaxL], d[kMaxL];
#pragma unroll
  for (int i = 0; i < kMaxL; ++i) {
    mu[i] = 0.0f;
#pragma unroll
    for (int j = 0; j < kMaxL; ++j) C[i][j] = 0.0f;
  }
  int k = 2 * L;
#pragma unroll
  for (int i = 0; i < kMaxL; ++i) {
    if (i < L) {
      if (kind == kMoveNet) {
        mu[i] = prop[(size_t)i * pstride + pidx];
        C[i][i] = expf(prop[(size_t)(L + i) * pstride + pidx]);
#pragma unroll
        for (int j = 0; j < kMaxL; ++j)
          if (j < i) C[i][j] = prop[(size_t)(k++) * pstride + pidx];
      } else {  // the prior's centre and scales
        mu[i] = (float)hy->phi[2 + i];
        C[i][i] = sqrtf((float)hy->phi[2 + L + i]);
      }
    }
  }
  Rng4 r(mc.seed_lo, mc.seed_hi, mc.chain, kStreamMH, (uint32_t)g, it32);
  float lp = 0.0f;  // log prior ratio of beta
  float xx = 0.0f;  // |xi|^2
#pragma unroll
  for (int i = 0; i < kMaxL; ++i) {
    xi[i] = 0.0f;
    if (i < L) xi[i] = normal_bm_f(r, 2 * i);
    xx += xi[i] * xi[i];
  }
  const float log_u = __logf(r.u(2u * (uint32_t)L));
  const uint32_t kc = 2u * (uint32_t)L + 1u;
  const float chi2 = -2.0f * (logf(r.u(kc)) + logf(r.u(kc + 1u)) + logf(r.u(kc + 2u)) +
                              logf(r.u(kc + 3u)));
  const float st = sqrtf((float)kTDof / chi2);
#pragma unroll
  for (int i = 0; i < kMaxL; ++i) {
    float v = 0.0f;
#pragma unroll
    for (int j = 0; j < kMaxL; ++j)
      if (j <= i) v += C[i][j] * xi[j];
    v = mu[i] + st * v;
    bn[i] = v;
    d[i] = i < L ? v - bs[i * B + tid] : 0.0f;
  }
  float u[kMaxL];
  float uu = 0.0f;  // |C^-1 (beta - mu)|^2
#pragma unroll
  for (int i = 0; i < kMaxL; ++i) {
    u[i] = 0.0f;
    if (i < L) {
      float v = bs[i * B + tid] - mu[i];
#pragma unroll
      for (int j = 0; j < kMaxL; ++j)
        if (j < i) v -= C[i][j] * u[j];
      u[i] = v / C[i][i];
      uu += u[i] * u[i];
      const float bt = bs[i * B + tid] - (float)hy->phi[2 + i];
      lp -= d[i] * (d[i] + 2.0f * bt) * (0.5f / (float)hy->phi[2 + L + i]);
    }
  }
  // log q(beta) - log q(beta*), with C^-1 (beta* - mu) = st xi
  const float inv_dof = 1.0f / (float)kTDof;
  const float lq = -0.5f * (float)(kTDof + L) *
                   (log1pf(uu * inv_dof) - log1pf(st * st * xx * inv_dof));
  // eps prior ratio: sum_n [eps_n^2 - (eps_n - X_n d)^2] / (2 gamma)
  float se = 0.0f;
  for (int n = 0; n < N; ++n) {
    float xd = 0.0f;
#pragma unroll
    for (int l = 0; l < kMaxL; ++l)
      if (l < L) xd += mc.Xf[n * kMaxL + l] * d[l];
    se += xd * (2.0f * p.eps[(size_t)n * G + g] - xd);
  }
  const float la = se * hg + lp + lq;
  const bool acc = log_u < la;
  if (acc) {
    for (int n = 0; n < N; ++n) {
      float xd = 0.0f;
#pragma unroll
      for (int l = 0; l < kMaxL; ++l)
        if (l < L) xd += mc.Xf[n * kMaxL + l] * d[l];
      p.eps[(size_t)n * G + g] -= xd;
    }
#pragma unroll
    for (int i = 0; i < kMaxL; ++i)
      if (i < L) bs[i * B + tid] = bn[i];
  }
  return acc;
}

// One slice update of beta_gl (step 5) for a column with NC value classes:
// class sums Q_j (rates) and Y_j (counts) from the per-thread rows in shared
// memory, the update, and the rates carried to the new value.
template <int NC>
__device__ __forceinline__ void beta_column_f32(const ModelConst& mc, const DevPtrsF32& p, int l,
                                                int g, float* mu, const float* ys, float* bs,
                                                int B, int tid, const Hyper* hy, long long it,
                                                uint32_t it32, long long burnin,
                                                long long tune_start, unsigned& evals_b,
                                                unsigned& caps, unsigned& nonfin, bool use_pat,
                                                float* E, const float* Yp) {
  const int G = mc.G, N = mc.N, L = mc.L;
  const size_t e = (size_t)l * G + g;
  const float theta = (float)hy->phi[2 + l];
  const float sig2 = (float)hy->phi[2 + L + l];
  BetaDensityFT<NC> f;
  const float b_cur = bs[l * B + tid];
  f.b0 = b_cur;
  f.bt = b_cur - theta;
  f.hs = 0.5f / sig2;
  f.ncls = mc.ncls[l];
  float Y[NC];
#pragma unroll
  for (int j = 0; j < NC; ++j) {
    f.Q[j] = 0.0f;
    Y[j] = 0.0f;
    f.v[j] = mc.cvalf[l][j];
  }
  if (use_pat) {
#pragma unroll
    for (int r = 0; r < kMaxPat; ++r)
      if (r < mc.npat) {
        const int c = mc.pcls[l][r];
#pragma unroll
        for (int j = 0; j < NC; ++j)
          if (j == c) {
            f.Q[j] += E[r];
            Y[j] += Yp[r];
          }
      }
  } else {
    for (int n = 0; n < N; ++n) {
      const int c = mc.cls[l][n];
      const float m = mu[n * B + tid];
      const float yv = ys[n * B + tid];
#pragma unroll
      for (int j = 0; j < NC; ++j)
        if (j == c) {
          f.Q[j] += m;
          Y[j] += yv;
        }
    }
  }
#pragma unroll
  for (int j = 0; j < NC; ++j) f.D[j] = Y[j] - f.Q[j];
  Rng4 r(mc.seed_lo, mc.seed_hi, mc.chain, kStreamBeta, (uint32_t)((size_t)g * L + l), it32);
  const float x0 = b_cur;
  float w = p.w_beta[e];
  SliceResultF s = slice_update_f(x0, 0.0f, w, f, r, mc.K, mc.shrink_max);
  evals_b += s.evals;
  caps += s.capped;
  nonfin += s.nonfinite;
  if (s.x != x0) {
    const float d = s.x - x0;
    float fac[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      const float z = f.v[j] * d;
      fac[j] = 1.0f + (z + em1mx(z));
    }
    if (use_pat) {
#pragma unroll
      for (int r = 0; r < kMaxPat; ++r)
        if (r < mc.npat) {
          const int c = mc.pcls[l][r];
          float fc = 1.0f;
#pragma unroll
          for (int j = 0; j < NC; ++j)
            if (j == c) fc = fac[j];
          E[r] *= fc;
        }
    } else {
      for (int n = 0; n < N; ++n) {
        const int c = mc.cls[l][n];
        float fc = 1.0f;
#pragma unroll
        for (int j = 0; j < NC; ++j)
          if (j == c) fc = fac[j];
        mu[n * B + tid] *= fc;
      }
    }
  }
  bs[l * B + tid] = s.x;
  if (it <= burnin) {
    float waux = p.waux_beta[e];
    tune_width_f(w, waux, it, s.x, x0, burnin, tune_start);
    p.w_beta[e] = w;
    p.waux_beta[e] = waux;
  }
}

// Shared memory of the gamma/beta updates for blocks of B threads: mu, y [N][B],
// beta [kMaxL][B], partials [kNumPart][B] (floats), then FP64 warp sums.
__host__ __device__ inline size_t gb_smem_bytes_f32(int N, int B) {
  return ((2 * (size_t)N + kMaxL + kNumPart) * B + 2) * sizeof(float) +
         (size_t)(B / 32) * kNumPart * sizeof(double);
}

// Steps 2 and 5 of Algorithm 1 in the FP32 form: one thread per gene.  The
// hyperparameter kernel of the previous iteration has finished when it runs.
// Genes marked for the learned proposal first make its move (which keeps every
// log-rate, so the rates mu stay valid); the slice updates of beta_g follow the
// gamma draw, for every gene unless the move replaces them (p.mh_replace).
// net_ok: false when this block's network pass gave up (its genes then skip the
// network's move); prop_s: the network's outputs of the block's genes in shared
// memory ([K][B]), or nullptr (the move reads p.prop, [K][G]).
__device__ __forceinline__ void gb_f32_body(const ModelConst& mc, const DevPtrsF32& p, int seg_i,
                                            int blk, bool net_ok = true,
                                            const float* prop_s = nullptr) {
  // shared: mu[N][B], y[N][B], beta[L][B], partials[kNumPart][B] (per-thread values
  // indexed by a runtime l live here rather than in local memory); then FP64 warp sums
  extern __shared__ float smem_f[];
  const int G = mc.G, N = mc.N, L = mc.L;
  const Hyper* hy = p.hyp;
  const long long it = hy->seg_it + seg_i + 1;
  const uint32_t it32 = (uint32_t)it;
  const long long burnin = hy->burnin, tune_start = hy->tune_start;
  const bool mom = it > burnin;
  const float inv_k = mom ? 1.0f / (float)(hy->n_mom + 1) : 0.0f;
  const float nu = (float)hy->phi[0], tau = (float)hy->phi[1];
  const bool trace_now = mom && mc.trace_beta && p.trace_beta != nullptr &&
                         ((it - burnin) % hy->thin == 0) && hy->trace_rows < hy->trace_cap;
  const long long trace_row = hy->trace_rows;
  const size_t LG = (size_t)L * G;

  const int B = blockDim.x;
  float* mu = smem_f;
  float* ys = mu + (size_t)N * B;
  float* bs = ys + (size_t)N * B;
  float* ps = bs + (size_t)kMaxL * B;
  const int tid = threadIdx.x;
  const int g = blk * B + tid;
  const bool active = g < G;

#pragma unroll
  for (int i = 0; i < kNumPart; ++i) ps[i * B + tid] = 0.0f;
  unsigned evals_b = 0, caps = 0, gcaps = 0, nonfin = 0;

  if (active) {
    for (int l = 0; l < L; ++l) bs[l * B + tid] = p.beta[(size_t)l * G + g];
    // 16 samples' loads in flight at a time (at N = 16 the whole gene; 8 or 4 lost
    // 0.3-1.4 us of the kernel at N=16 G=40000)
#pragma unroll 16
    for (int n = 0; n < N; ++n) {
      const size_t e = (size_t)n * G + g;
      mu[n * B + tid] = p.mu[e];
      ys[n * B + tid] = (float)p.y[e];
    }

    // per-pattern sums of the rates and counts, in registers, when X has at most
    // kMaxPat distinct rows (the move below keeps every rate)
    const bool use_pat = mc.npat <= kMaxPat;
    float E[kMaxPat], Yp[kMaxPat];
#pragma unroll
    for (int r = 0; r < kMaxPat; ++r) {
      E[r] = 0.0f;
      Yp[r] = 0.0f;
    }
    if (use_pat) {
      for (int n = 0; n < N; ++n) {
        const int pr = mc.pat[n];
        const float m = mu[n * B + tid], yv = ys[n * B + tid];
#pragma unroll
        for (int r = 0; r < kMaxPat; ++r)
          if (r == pr) {
            E[r] += m;
            Yp[r] += yv;
          }
      }
    }

    // ---- learned-proposal move (keeps every log-rate, so mu stays valid)
    int kind = p.prop != nullptr ? move_kind(p, g, it) : 0;
    if (kind == kMoveNet && !net_ok) kind = 0;
    const bool mh_gene = kind != 0;
    if (mh_gene) {
      const bool acc =
          prop_s != nullptr
              ? mh_move_f32(mc, p, g, it32, bs, B, tid, hy, 0.5f / p.gam[g], kind, prop_s,
                            (size_t)B, tid)
              : mh_move_f32(mc, p, g, it32, bs, B, tid, hy, 0.5f / p.gam[g], kind, p.prop,
                            (size_t)G, g);
      const size_t ci = (size_t)(kind - 1) * G + g;
      p.mh_try[ci] += 1u;
      p.mh_acc[ci] += acc ? 1u : 0u;
    }

    float ss = 0.0f;
#pragma unroll 16
    for (int n = 0; n < N; ++n) {
      const float x = p.eps[(size_t)n * G + g];
      ss += x * x;
    }

    // ---- step 2: gamma_g ~ IG((N + nu)/2, (sum eps^2 + nu tau)/2)
    {
      Rng4 r(mc.seed_lo, mc.seed_hi, mc.chain, kStreamGamma, (uint32_t)g, it32);
      bool gcap = false;
      const float shape = 0.5f * ((float)N + nu);
      const float scale = 0.5f * (ss + nu * tau);
      const float gam = scale / gamma_mt_f(shape, r, 0, &gcap);
      gcaps += gcap;
      p.gam[g] = gam;
      if (mom) welford_kahan(p.mom_gam, (size_t)G, (size_t)g, gam, inv_k);
      ps[0 * B + tid] = __logf(gam);
      ps[1 * B + tid] = 1.0f / gam;
    }

    // ---- step 5: beta_gl, l = 1..L in order (genes without the learned move)
    const bool skip_slices = mh_gene && p.mh_replace;
    for (int l = 0; l < L && !skip_slices; ++l) {
      switch (mc.ncls[l]) {
        case 1:
          beta_column_f32<1>(mc, p, l, g, mu, ys, bs, B, tid, hy, it, it32, burnin, tune_start,
                             evals_b, caps, nonfin, use_pat, E, Yp);
          break;
        case 2:
          beta_column_f32<2>(mc, p, l, g, mu, ys, bs, B, tid, hy, it, it32, burnin, tune_start,
                             evals_b, caps, nonfin, use_pat, E, Yp);
          break;
        case 3:
          beta_column_f32<3>(mc, p, l, g, mu, ys, bs, B, tid, hy, it, it32, burnin, tune_start,
                             evals_b, caps, nonfin, use_pat, E, Yp);
          break;
        default:
          beta_column_f32<kMaxCls>(mc, p, l, g, mu, ys, bs, B, tid, hy, it, it32, burnin,
                                   tune_start, evals_b, caps, nonfin, use_pat, E, Yp);
      }
    }

    // ---- the new beta_g: state, moments, trace, partial sums for steps 6-7
    for (int l = 0; l < L; ++l) {
      const size_t e = (size_t)l * G + g;
      const float b = bs[l * B + tid];
      p.beta[e] = b;
      if (mom) welford_kahan(p.mom_beta, LG, e, b, inv_k);
      if (trace_now) p.trace_beta[(size_t)trace_row * LG + e] = (double)b;
      const float dv = b - (float)hy->phi[2 + l];
      ps[(2 + l) * B + tid] = dv;
      ps[(2 + kMaxL + l) * B + tid] = dv * dv;
    }
    // contrast probabilities (§3.1), evaluated in FP32
    if (mom && p.con != nullptr) {
      const Contrasts* cs = p.con;
      for (int q = 0; q < cs->n; ++q) {
        bool ok = true;
        for (int k = 0; k < cs->terms[q] && ok; ++k) {
          float sv = 0.0f;
          for (int l = 0; l < L; ++l) sv = __fadd_rn(sv, __fmul_rn(cs->vf[q][k][l], bs[l * B + tid]));
          ok = sv > cs->bf[q][k];
        }
        if (ok) p.con_count[(size_t)q * G + g] += 1u;
      }
    }
  }

  // ---- partial sums: error-free FP32 pair sums within the warp, FP64 beyond.
  // Lane i < kNumPart sums row i of the warp's 32 values (read in an order
  // rotated by i, so that the lanes hit distinct shared-memory banks).
  const int lane = tid & 31, warp = tid >> 5, nwarp = B >> 5;
  double* red = reinterpret_cast<double*>(
      smem_f + (((2 * (size_t)N + kMaxL + kNumPart) * B + 1) & ~(size_t)1));
  __syncwarp();
  if (lane < kNumPart) {
    const float* row = ps + (size_t)lane * B + warp * 32;
    float sm = 0.0f, c = 0.0f;
    for (int j = 0; j < 32; ++j) {
      float t, e;
      two_sum(sm, row[(j + lane) & 31], t, e);
      sm = t;
      c += e;
    }
    red[warp * kNumPart + lane] = (double)sm + (double)c;
  }
  __syncthreads();
  if (tid < kNumPart) {
    double acc = 0.0;
    for (int w = 0; w < nwarp; ++w) acc += red[w * kNumPart + tid];
    p.partial[(size_t)blk * kNumPart + tid] = acc;
  }
  add_counters(p.counters, 0, evals_b, caps, gcaps, nonfin, &p.hyp->flags);
}

__global__ void __launch_bounds__(128) k_gb_f32(ModelConst mc, DevPtrsF32 p, int seg_i) {
  ktime_begin(p.ktime, p.ktime_n, 3 * seg_i + 1);
  gb_f32_body(mc, p, seg_i, blockIdx.x);
  ktime_end(p.ktime, p.ktime_n, 3 * seg_i + 1);
}

// Shared memory of the fused kernel: the network pass (its weight image; the A
// operands are in tensor memory) from offset 0, then the gamma/beta updates'
// arrays from offset 0, and
// the network's outputs of the block's genes ([K][128] floats) at
// gb_net_stash_offset, past both the weight image and those arrays.
__host__ __device__ inline size_t gb_net_stash_offset(int N, int L) {
  size_t off_a;
  tc_smem_layout(L, &off_a);
  const size_t gb = gb_smem_bytes_f32(N, 128);
  return ((off_a > gb ? off_a : gb) + 15) & ~(size_t)15;
}

size_t gb_net_smem_bytes(int N, int L) {
  const size_t tc = tc_smem_layout(L, nullptr);
  const size_t st = gb_net_stash_offset(N, L) + (size_t)tc_shape(L).K * 128 * sizeof(float);
  return tc > st ? tc : st;
}

// With the learned proposal (128 threads): the block first evaluates the network
// for its 128 genes on the tensor cores (outputs to shared memory, read by the
// same threads in the move: a round trip through global memory less), then frees
// the tensor memory and reuses the shared memory below the outputs for the
// gamma/beta updates.  A kernel of its own, so that the plain gamma/beta kernel
// keeps its own register allocation.
__global__ void __launch_bounds__(128) k_gb_net_f32(ModelConst mc, DevPtrsF32 p, int seg_i,
                                                    const uint8_t* __restrict__ img) {
  ktime_begin(p.ktime, p.ktime_n, 3 * seg_i + 1);
  bool net_ok;
  float* prop_s;
  {
    extern __shared__ __align__(1024) uint8_t sm_tc[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int s_abort;
    const TcShape t = tc_shape(mc.L);
    if (threadIdx.x == 0) s_abort = 0;
    TcBlock c;
    tc_begin(c, bars, &tmem_slot, img, sm_tc, t.bytes, p.tc_polls);
    if (!c.w_ok) s_abort = 1;
    __syncthreads();
    const int g = blockIdx.x * 128 + (int)threadIdx.x;
    prop_s = reinterpret_cast<float*>(sm_tc + gb_net_stash_offset(mc.N, mc.L));
    if (!s_abort)
      tc_tile(c, mc, p, t, sm_tc, g, net_gene(p, g, mc.G), prop_s, 128, (int)threadIdx.x,
              &s_abort);
    __syncthreads();
    net_ok = s_abort == 0;
    tc_end(c, !net_ok, &p.hyp->flags);
    fence_async_smem();
    __syncthreads();  // below the outputs, the shared memory is the gamma/beta updates' from here on
  }
  gb_f32_body(mc, p, seg_i, blockIdx.x, net_ok, prop_s);
  ktime_end(p.ktime, p.ktime_n, 3 * seg_i + 1);
}

// The learned move alone, at the current state, for the genes that use it (every
// gene when p.mh_all), with the random numbers of iteration `it`.
__global__ void __launch_bounds__(128) k_mh_step_f32(ModelConst mc, DevPtrsF32 p, long long it) {
  __shared__ float bs[kMaxL * 128];
  const int B = blockDim.x, tid = threadIdx.x;
  const int g = blockIdx.x * B + tid;
  if (g >= mc.G) return;
  const int kind = move_kind(p, g, it);
  if (kind == 0) return;
  const int G = mc.G, L = mc.L;
  for (int l = 0; l < L; ++l) bs[l * B + tid] = p.beta[(size_t)l * G + g];
  const bool acc = mh_move_f32(mc, p, g, (uint32_t)it, bs, B, tid, p.hyp, 0.5f / p.gam[g], kind,
                               p.prop, (size_t)G, g);
  const size_t ci = (size_t)(kind - 1) * G + g;
  p.mh_try[ci] += 1u;
  if (acc) {
    p.mh_acc[ci] += 1u;
    for (int l = 0; l < L; ++l) p.beta[(size_t)l * G + g] = bs[l * B + tid];
  }
}

__global__ void k_seg_begin(Hyper* hy) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    hy->seg_it = hy->it;
    hy->seg_nmom = hy->n_mom;
  }
}

// ---------------------------------------------------------------- persistent sweeps (FP32)
//
// A whole segment of sweeps of one chain (Algorithm 1, every step) in one
// cooperative launch whose blocks are all resident: per sweep, every block takes
// tiles of 128 eps_gn updates (step 1), a grid barrier, every block takes
// 128-gene blocks of gamma/beta updates (steps 2, 5), a grid barrier, then block 0
// runs the hyperparameter steps (3, 4, 6, 7) while the other blocks go on to the
// next sweep's eps updates, which involve no hyperparameter; the next barrier
// also waits for block 0.  The per-element, per-gene and hyperparameter device
// functions are those of k_eps_f32, k_gb_f32 and k_hyper, with the same Philox
// counters and the same per-gene-block partial sums, so the chain is
// bit-identical to the graph of separate launches.

// Sense-reversing grid barrier in device memory (zeroed before each launch).
struct GridSync {
  unsigned int count, gen;
};

// Polls of a barrier wait (each followed by a 64 ns sleep, about 4 s in all)
// before the wait gives up, sets kFlagTimeout and ends the launch.
constexpr unsigned kGridWaitLimit = 1u << 26;

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_gpu(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Every block of the grid arrives; the last one to arrive resets the count and
// opens the next generation.  Writes of every block before the barrier are
// visible to every block after it.  Returns false in every thread of a block
// whose wait gave up.
__device__ __forceinline__ bool grid_sync(GridSync* gs, unsigned* flags, volatile int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned gen = ld_acquire_gpu(&gs->gen);
    __threadfence();
    const unsigned arrived = atomicAdd(&gs->count, 1u) + 1u;
    int ok = 1;
    if (arrived == gridDim.x) {
      atomicExch(&gs->count, 0u);
      __threadfence();
      st_release_gpu(&gs->gen, gen + 1u);
    } else {
      unsigned polls = 0;
      while (ld_acquire_gpu(&gs->gen) == gen) {
        if (++polls >= kGridWaitLimit) {
          ok = 0;
          atomicOr(flags, kFlagTimeout);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

__global__ void __launch_bounds__(128, 4) k_sweeps_f32(ModelConst mc, DevPtrsF32 p, DevPtrs hp,
                                                   int n_sweeps, int nblk, GridSync* gs) {
  __shared__ int s_ok;
  const int tiles_g = (mc.G + 127) / 128;
  const int n_tiles = tiles_g * mc.N;
  for (int i = 0; i < n_sweeps; ++i) {
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
      const int n = t / tiles_g;
      eps_f32_body(mc, p, i, n, (t - n * tiles_g) * 128 + (int)threadIdx.x, t % kCounterCopies);
    }
    if (!grid_sync(gs, &p.hyp->flags, &s_ok)) return;
    for (int b = blockIdx.x; b < nblk; b += gridDim.x) {
      gb_f32_body(mc, p, i, b);
      __syncthreads();  // the next gene block reuses the shared memory
    }
    if (!grid_sync(gs, &p.hyp->flags, &s_ok)) return;
    if (blockIdx.x == 0) hyper_body(mc, hp.partial, hp.hyp, hp.trace_phi, hp.counters, nblk);
  }
}

cudaError_t launch_sweeps_f32(const ModelConst& mc, const DevPtrsF32& p, const DevPtrs& hp,
                              int n_sweeps, void* gsync, cudaStream_t s, int* grid_out) {
  const int block = 128;
  const int nblk = (mc.G + block - 1) / block;
  const size_t smem = gene_smem_bytes_f32(mc.N, block);
  cudaError_t e = cudaFuncSetAttribute(k_sweeps_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)gene_smem_bytes_f32(FBS_MAX_N, block));
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweeps_f32, block, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int grid = per_sm * sms;
  const int most = nblk > ((mc.G + 127) / 128) * mc.N ? nblk : ((mc.G + 127) / 128) * mc.N;
  if (grid > most) grid = most;
  if ((e = cudaMemsetAsync(gsync, 0, sizeof(GridSync), s)) != cudaSuccess) return e;
  ModelConst mc_ = mc;
  DevPtrsF32 p_ = p;
  DevPtrs hp_ = hp;
  int n_ = n_sweeps, nb_ = nblk;
  GridSync* gs_ = (GridSync*)gsync;
  void* args[] = {&mc_, &p_, &hp_, &n_, &nb_, &gs_};
  if (grid_out) *grid_out = grid;
  return cudaLaunchCooperativeKernel((const void*)k_sweeps_f32, dim3(grid), dim3(block), args, smem,
                                     s);
}

// ---------------------------------------------------------------- batched kernels (FP32)
//
// Many independent datasets / chains in one launch.  Each dataset keeps its own
// model constants and device pointers in global memory; a block table maps every
// block of a launch to one dataset (and to a sample row and gene block for the
// eps kernel), so a block never straddles two datasets and uneven N and G need no
// padding beyond the last block of each dataset.

// At most 51 registers (at least 5 blocks of 256 per SM, as k_eps_f32): 454 -> 511
// batch sweeps/s on the 64-dataset batch.
__global__ void __launch_bounds__(256, 5) k_eps_f32_batch(const ModelConst* __restrict__ mcs,
                                                       const DevPtrsF32* __restrict__ ps,
                                                       const int4* __restrict__ tab, int seg_i) {
  const int4 t = tab[blockIdx.x];  // dataset, sample row n, gene block, counter copy
  eps_f32_body(mcs[t.x], ps[t.x], seg_i, t.y, t.z * blockDim.x + threadIdx.x, t.w);
}

__global__ void __launch_bounds__(128) k_gb_f32_batch(const ModelConst* __restrict__ mcs,
                                                      const DevPtrsF32* __restrict__ ps,
                                                      const int2* __restrict__ tab, int seg_i) {
  const int2 t = tab[blockIdx.x];  // dataset, gene block within the dataset
  gb_f32_body(mcs[t.x], ps[t.x], seg_i, t.y);
}

// One block per dataset.
__global__ void __launch_bounds__(kHyperThreads) k_hyper_batch(const ModelConst* __restrict__ mcs,
                                                               const DevPtrsF32* __restrict__ ps,
                                                               const int* __restrict__ nblk) {
  const int c = blockIdx.x;
  const DevPtrsF32& p = ps[c];
  hyper_body(mcs[c], p.partial, p.hyp, p.trace_phi, p.counters, nblk[c], p.psi);
}

// Top level of the three-level model, one warp, after the datasets' hyper
// steps of the same sweep: lane 0 draws b ~ Gamma(a_b + sum_k a_k, rate b_b +
// sum_k tau_k), lane 1+l draws m_l ~ N(w sum_k theta_kl / c_kl^2, w) with
// w = 1 / (sum_k 1/c_kl^2 + 1/e_l^2); the sums over k run in dataset order.
// Moments and trace follow dataset 0's iteration, burn-in and thinning.
__global__ void __launch_bounds__(32) k_top_level(const ModelConst* __restrict__ mcs,
                                                  const DevPtrsF32* __restrict__ ps, int C,
                                                  TopLevel* __restrict__ top,
                                                  double* __restrict__ trace) {
  const int lane = threadIdx.x;
  const int L = top->L;
  const Hyper* h0 = ps[0].hyp;
  const long long it = h0->it;
  const uint32_t it32 = (uint32_t)it;
  double x = 0.0;
  if (lane == 0) {
    double sa = 0.0, st = 0.0;
    for (int k = 0; k < C; ++k) {
      sa += mcs[k].a;
      st += ps[k].hyp->phi[1];
    }
    Rng r(top->seed_lo, top->seed_hi, 0u, kStreamPsi, 0u, it32);
    bool cap = false;
    x = gamma_mt(top->a_b + sa, r, 0, &cap) / (top->b_b + st);
    if (cap) atomicAdd(&top->gamma_caps, 1ull);
  } else if (lane <= L) {
    const int l = lane - 1;
    double prec = 0.0, s = 0.0;
    for (int k = 0; k < C; ++k) {
      const double c2 = mcs[k].c2[l];
      prec += 1.0 / c2;
      s += ps[k].hyp->phi[2 + l] / c2;
    }
    const double w = 1.0 / (prec + 1.0 / top->e2[l]);
    Rng r(top->seed_lo, top->seed_hi, 0u, kStreamPsi, (uint32_t)lane, it32);
    x = __dadd_rn(__dmul_rn(w, s), __dmul_rn(sqrt(w), normal_bm(r, 0)));
  }
  const bool mom = it > h0->burnin;
  const bool tr = mom && ((it - h0->burnin) % h0->thin == 0) && top->trace_rows < top->trace_cap &&
                  trace != nullptr;
  if (lane <= L) {
    top->psi[lane] = x;
    if (mom) {
      const double inv_k = 1.0 / (double)(top->n_mom + 1);
      const double m = top->m_psi[lane], q = top->q_psi[lane];
      top->m_psi[lane] = m + (x - m) * inv_k;
      top->q_psi[lane] = q + (x * x - q) * inv_k;
    }
    if (tr) trace[(size_t)top->trace_rows * (L + 1) + lane] = x;
  }
  __syncwarp();
  if (lane == 0) {
    if (mom) top->n_mom += 1;
    if (tr) top->trace_rows += 1;
  }
}

__global__ void k_seg_begin_batch(const DevPtrsF32* __restrict__ ps, int C) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < C) {
    Hyper* hy = ps[c].hyp;
    hy->seg_it = hy->it;
    hy->seg_nmom = hy->n_mom;
  }
}

__global__ void k_set_run_batch(const DevPtrsF32* __restrict__ ps, int C, long long burnin,
                                long long tune_start, long long thin) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < C) {
    Hyper* hy = ps[c].hyp;
    hy->burnin = burnin;
    hy->tune_start = tune_start;
    hy->thin = thin;
  }
}

cudaError_t prepare_batch_kernels(int max_N, int gb_block) {
  const size_t smem = gene_smem_bytes_f32(max_N, gb_block);
  if (smem > 48 * 1024)
    return cudaFuncSetAttribute(k_gb_f32_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
  return cudaSuccess;
}

cudaError_t launch_eps_f32_batch(const ModelConst* mcs, const DevPtrsF32* ps, const int4* tab,
                                 int n_blocks, int block, int seg_i, cudaStream_t s) {
  k_eps_f32_batch<<<n_blocks, block, 0, s>>>(mcs, ps, tab, seg_i);
  return cudaGetLastError();
}

cudaError_t launch_gb_f32_batch(const ModelConst* mcs, const DevPtrsF32* ps, const int2* tab,
                                int n_blocks, int block, int max_N, int seg_i, cudaStream_t s) {
  k_gb_f32_batch<<<n_blocks, block, gene_smem_bytes_f32(max_N, block), s>>>(mcs, ps, tab, seg_i);
  return cudaGetLastError();
}

cudaError_t launch_hyper_batch(const ModelConst* mcs, const DevPtrsF32* ps, const int* nblk,
                               int C, cudaStream_t s) {
  k_hyper_batch<<<C, kHyperThreads, 0, s>>>(mcs, ps, nblk);
  return cudaGetLastError();
}

cudaError_t launch_top_level(const ModelConst* mcs, const DevPtrsF32* ps, int C, TopLevel* top,
                             double* trace, cudaStream_t s) {
  k_top_level<<<1, 32, 0, s>>>(mcs, ps, C, top, trace);
  return cudaGetLastError();
}

cudaError_t launch_seg_begin_batch(const DevPtrsF32* ps, int C, cudaStream_t s) {
  k_seg_begin_batch<<<(C + 127) / 128, 128, 0, s>>>(ps, C);
  return cudaGetLastError();
}

cudaError_t launch_set_run_batch(const DevPtrsF32* ps, int C, long long burnin,
                                 long long tune_start, long long thin, cudaStream_t s) {
  k_set_run_batch<<<(C + 127) / 128, 128, 0, s>>>(ps, C, burnin, tune_start, thin);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- set-up kernels (FP32)

// Same starting values as the FP64 form, computed in FP64 and stored in FP32.
__global__ void k_init_genes_f32(ModelConst mc, DevPtrsF32 p, const int32_t* y_in,
                                 int gene_major, const double* __restrict__ pinv, double w0,
                                 int set_state) {
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
        p.beta[(size_t)l * G + g] = (float)s;
        p.w_beta[(size_t)l * G + g] = (float)w0;
        p.waux_beta[(size_t)l * G + g] = 0.0f;
      }
    }
    if (set_state) {
      for (int n = 0; n < N; ++n) {
        p.eps[(size_t)n * G + g] = 0.0f;
        p.w_eps[(size_t)n * G + g] = (float)w0;
        p.waux_eps[(size_t)n * G + g] = 0.0f;
      }
      p.gam[g] = 1.0f;
    }
  }
}

__global__ void k_zero_moments_f32(ModelConst mc, DevPtrsF32 p) {
  const size_t NG = (size_t)mc.N * mc.G, LG = (size_t)mc.L * mc.G, G = mc.G;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < 4 * NG;
       i += (size_t)gridDim.x * blockDim.x) {
    p.mom_eps[i] = 0.0f;
    if (i < 4 * LG) p.mom_beta[i] = 0.0f;
    if (i < 4 * G) p.mom_gam[i] = 0.0f;
  }
}

cudaError_t prepare_gene_kernel_f32(int N, int block) {
  const size_t smem = gene_smem_bytes_f32(N, block);
  if (smem > 48 * 1024)
    return cudaFuncSetAttribute(k_gb_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
  return cudaSuccess;
}

size_t gene_smem_bytes_f32(int N, int block) { return gb_smem_bytes_f32(N, block); }

cudaError_t launch_eps_f32(const ModelConst& mc, const DevPtrsF32& p, int seg_i,
                           cudaStream_t s) {
  const int blk = 256;
  const dim3 grid((unsigned)((mc.G + blk - 1) / blk), (unsigned)mc.N);
  k_eps_f32<<<grid, blk, 0, s>>>(mc, p, seg_i);
  return cudaGetLastError();
}

cudaError_t launch_gb_f32(const ModelConst& mc, const DevPtrsF32& p, int block, int seg_i,
                          cudaStream_t s, const void* img) {
  const int nblk = (mc.G + block - 1) / block;
  size_t smem = gene_smem_bytes_f32(mc.N, block);
  if (img != nullptr) {
    if (block != 128) return cudaErrorInvalidValue;  // one thread per gene of a 128-gene tile
    smem = gb_net_smem_bytes(mc.N, mc.L);
    size_t most = 0;
    for (int L = 1; L <= FBS_MAX_L; ++L) {
      const size_t b = gb_net_smem_bytes(FBS_MAX_N, L);
      if (b > most) most = b;
    }
    cudaError_t e = cudaFuncSetAttribute(k_gb_net_f32,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
    if (e != cudaSuccess) return e;
  }
  if (img != nullptr) k_gb_net_f32<<<nblk, block, smem, s>>>(mc, p, seg_i, (const uint8_t*)img);
  else k_gb_f32<<<nblk, block, smem, s>>>(mc, p, seg_i);
  return cudaGetLastError();
}

cudaError_t launch_mh_step_f32(const ModelConst& mc, const DevPtrsF32& p, long long it,
                              cudaStream_t s) {
  const int block = 128;
  k_mh_step_f32<<<(mc.G + block - 1) / block, block, 0, s>>>(mc, p, it);
  return cudaGetLastError();
}

cudaError_t launch_seg_begin(Hyper* hy, cudaStream_t s) {
  k_seg_begin<<<1, 32, 0, s>>>(hy);
  return cudaGetLastError();
}

cudaError_t launch_init_f32(const ModelConst& mc, const DevPtrsF32& p, const int32_t* y_in,
                            int gene_major, const double* pinv, double w0, int set_state,
                            cudaStream_t s) {
  const int blk = 256;
  const int grid = (mc.G + blk - 1) / blk;
  k_init_genes_f32<<<grid, blk, 0, s>>>(mc, p, y_in, gene_major, pinv, w0, set_state);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_zero_moments_f32(mc, p, s);
}

cudaError_t launch_zero_moments_f32(const ModelConst& mc, const DevPtrsF32& p, cudaStream_t s) {
  const size_t n = 4 * (size_t)mc.N * mc.G;
  const int blk = 256;
  const unsigned grid = (unsigned)((n + blk - 1) / blk);
  k_zero_moments_f32<<<grid, blk, 0, s>>>(mc, p);
  return cudaGetLastError();
}

}  // namespace fbs
