// fbs_rng.cuh -- counter-based random numbers, variate generators and the
// stepping-out slice sampler, as device functions.
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC 2011) in
// place of the CURAND generator the paper used (Section 4.2).  A variable is
// addressed by (stream, index, iteration, chain) and its k-th uniform comes
// from counter block k/2, so any thread can draw any variable's numbers in any
// order and the CPU oracle, which implements the same definition, consumes the
// identical uniforms.
#pragma once

#include <stdint.h>

namespace fbs {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr int kGammaAttempts = 64;
constexpr int kTruncAttempts = 16;
constexpr uint32_t kTruncStride = 256;  // uniforms reserved per truncated-draw attempt

// e^z - 1 - z without cancellation: Taylor series to z^9 for |z| < 1/2 (relative
// truncation error below 3e-9), expf otherwise.
__device__ __forceinline__ float em1mx(float z) {
  if (fabsf(z) < 0.5f) {
    float p = 1.0f / 362880.0f;
    p = fmaf(p, z, 1.0f / 40320.0f);
    p = fmaf(p, z, 1.0f / 5040.0f);
    p = fmaf(p, z, 1.0f / 720.0f);
    p = fmaf(p, z, 1.0f / 120.0f);
    p = fmaf(p, z, 1.0f / 24.0f);
    p = fmaf(p, z, 1.0f / 6.0f);
    p = fmaf(p, z, 0.5f);
    return z * z * p;
  }
  return expf(z) - 1.0f - z;
}

// Ten Philox rounds: two 32x32->64 multiplies per round, key bumped by the
// Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// The uniforms of one random variable.  u(k) returns uniform k; consecutive k
// share a Philox block, which is cached.
struct Rng {
  uint32_t key0, key1, index, sblk, iter, chain;
  uint32_t cached;
  uint4 w;

  __device__ __forceinline__ Rng(uint32_t seed_lo, uint32_t seed_hi, uint32_t chain_,
                                 uint32_t stream, uint32_t index_, uint32_t iter_)
      : key0(seed_lo), key1(seed_hi), index(index_), sblk(stream << 24), iter(iter_),
        chain(chain_), cached(0xFFFFFFFFu), w(make_uint4(0, 0, 0, 0)) {}

  __device__ __forceinline__ double u(uint32_t k) {
    const uint32_t blk = k >> 1;
    if (blk != cached) {
      w = philox4x32_10(make_uint4(index, sblk | blk, iter, chain), key0, key1);
      cached = blk;
    }
    const unsigned long long x = (k & 1u)
                                     ? ((unsigned long long)w.w << 32 | w.z)
                                     : ((unsigned long long)w.y << 32 | w.x);
    // (floor(x / 2^12) + 1/2) / 2^52 = v / 2^53 with v = 2 floor(x / 2^12) + 1, an odd
    // integer below 2^53, so the double is assembled from integer operations: the
    // leading bit of v moved to bit 52 gives the mantissa, its position the exponent
    const unsigned long long v = ((x >> 12) << 1) | 1ull;
    const int sh = __clzll((long long)v) - 11;
    const unsigned long long bits =
        ((unsigned long long)(1022 - sh) << 52) | ((v << sh) & 0xFFFFFFFFFFFFFull);
    return __longlong_as_double((long long)bits);
  }
};

// Box-Muller normal from uniforms k0, k0+1 (cosine branch).
__device__ __forceinline__ double normal_bm(Rng& r, uint32_t k0) {
  const double u1 = r.u(k0), u2 = r.u(k0 + 1);
  return __dmul_rn(sqrt(__dmul_rn(-2.0, log(u1))), cos(__dmul_rn(kTwoPi, u2)));
}

// Gamma(shape, 1) by Marsaglia & Tsang (2000): attempt j takes uniforms
// k0+4j, k0+4j+1 (normal) and k0+4j+2 (acceptance); uniform k0+3 is the
// U^(1/shape) factor for shape < 1.  After 64 failed attempts the shape is
// returned and *capped is set.
__device__ __forceinline__ double gamma_mt(double shape, Rng& r, uint32_t k0, bool* capped) {
  const double alpha = shape < 1.0 ? __dadd_rn(shape, 1.0) : shape;
  const double dd = __dsub_rn(alpha, 1.0 / 3.0);
  const double cc = 1.0 / sqrt(__dmul_rn(9.0, dd));
  double boost = 1.0;
  if (shape < 1.0) boost = pow(r.u(k0 + 3), 1.0 / shape);
  for (uint32_t j = 0; j < (uint32_t)kGammaAttempts; ++j) {
    const double x = normal_bm(r, k0 + 4 * j);
    double v = __dadd_rn(1.0, __dmul_rn(cc, x));
    if (v <= 0.0) continue;
    v = __dmul_rn(__dmul_rn(v, v), v);
    const double u = r.u(k0 + 4 * j + 2);
    const double x2 = __dmul_rn(x, x);
    if (u < __dsub_rn(1.0, __dmul_rn(__dmul_rn(0.0331, x2), x2)))
      return __dmul_rn(__dmul_rn(dd, v), boost);
    const double rhs = __dadd_rn(__dmul_rn(0.5, x2),
                                 __dmul_rn(dd, __dadd_rn(__dsub_rn(1.0, v), log(v))));
    if (log(u) < rhs) return __dmul_rn(__dmul_rn(dd, v), boost);
  }
  *capped = true;
  return shape;
}

// Inverse-Gamma(shape, scale) truncated to (0, upper) by rejection; attempt t
// uses the gamma uniforms starting at 256 t.  After 16 failures `keep` is
// returned and *capped is set: keeping the current value leaves the target
// unchanged because the failure probability does not depend on it.
__device__ __forceinline__ double trunc_invgamma(double shape, double scale, double upper,
                                                 double keep, Rng& r, bool* gcap, bool* tcap) {
  for (uint32_t t = 0; t < (uint32_t)kTruncAttempts; ++t) {
    const double gv = gamma_mt(shape, r, kTruncStride * t, gcap);
    const double x = scale / gv;
    if (x < upper) return x;
  }
  *tcap = true;
  return keep;
}

struct SliceResult {
  double x;         // new value
  double aux;       // the density functor's auxiliary value at x
  unsigned evals;   // log-density evaluations
  bool capped;      // shrinkage ran out of proposals; x is the start value
  bool nonfinite;   // log density at the start value was not finite
};

// One update of the univariate stepping-out slice sampler (Algorithm 2,
// steps 1-6) from x0 with width w and stepping-out bound K.  Uniform 0 sets
// the level log u = log f(x0) + log U, uniform 1 places the interval, uniform
// 2 splits K into K_L + K_R, uniform 3+j is the j-th shrinkage proposal.
// f(x, &aux) returns log f(x) (up to a constant) and an auxiliary value that is
// kept for the accepted point.  The interval arithmetic is rounded step by
// step (no fused multiply-add) so that it matches a plain IEEE evaluation.
template <class F>
__device__ __forceinline__ SliceResult slice_update(double x0, double w, const F& f, Rng& r,
                                                    int K, int shrink_max) {
  SliceResult res;
  double aux0;
  const double f0 = f(x0, &aux0);
  res.evals = 1;
  res.nonfinite = !isfinite(f0);
  const double logu = __dadd_rn(f0, log(r.u(0)));
  const double v = __dmul_rn(w, r.u(1));
  double lo = __dsub_rn(x0, v);
  double hi = __dadd_rn(lo, w);
  int KL = (int)__dmul_rn((double)(K + 1), r.u(2));
  if (KL > K) KL = K;
  const int KR = K - KL;
  double aux;
  for (int k = 0; k < KL; ++k) {
    ++res.evals;
    if (logu < f(lo, &aux)) lo = __dsub_rn(lo, w); else break;
  }
  for (int k = 0; k < KR; ++k) {
    ++res.evals;
    if (logu < f(hi, &aux)) hi = __dadd_rn(hi, w); else break;
  }
  for (int j = 0; j < shrink_max; ++j) {
    const double xs = __dadd_rn(lo, __dmul_rn(__dsub_rn(hi, lo), r.u(3u + (uint32_t)j)));
    ++res.evals;
    if (logu < f(xs, &aux)) {
      res.x = xs;
      res.aux = aux;
      res.capped = false;
      return res;
    }
    if (xs > x0) hi = xs; else lo = xs;
  }
  res.x = x0;
  res.aux = aux0;
  res.capped = true;
  return res;
}

// slice_update (Algorithm 2, steps 1-6) with every comparison "log u < log f(p)"
// first decided in FP32.  ff(p, &bound) returns Delta(p) = log f(p) - log f(x0)
// in FP32 and a bound on the sum of its error and of the error with which the
// FP64 evaluation (f) of the same comparison is made; with the FP32 level
// log U_0, a gap beyond the two bounds decides the comparison exactly as the
// FP64 arithmetic would, and only a gap inside them evaluates f in FP64 (the
// level log f(x0) + log U_0 is then computed once).  The uniforms, the interval
// arithmetic (FP64, rounded step by step), the evaluation count, the result and
// its flags are those of slice_update; the caller computes the auxiliary value
// at the result.  ff must be usable only where f(x0) is finite (the caller
// checks this and otherwise calls slice_update), so nonfinite is false.
template <class F, class FF>
__device__ __forceinline__ SliceResult slice_update_filtered(double x0, double w, const F& f,
                                                             const FF& ff, Rng& r, int K,
                                                             int shrink_max) {
  SliceResult res;
  res.evals = 1;
  res.nonfinite = false;
  res.aux = 0.0;
  const double u0 = r.u(0);
  const float lu = logf((float)u0);
  // error of lu: the rounding of u0 to FP32 and logf's (ulp) error, with margin
  const float lu_err = 0x1p-20f * (fabsf(lu) + 1.0f);
  double logu = 0.0;
  bool have_level = false;
  auto above = [&](double pt) -> bool {  // the FP64 comparison logu < f(pt)
    float eb;
    const float gap = ff(pt, &eb) - lu;
    const float tol = eb + lu_err;
    if (gap > tol) return true;
    if (gap < -tol) return false;
    if (!have_level) {
      double a0;
      logu = __dadd_rn(f(x0, &a0), log(u0));
      have_level = true;
    }
    double a;
    return logu < f(pt, &a);
  };
  const double v = __dmul_rn(w, r.u(1));
  double lo = __dsub_rn(x0, v);
  double hi = __dadd_rn(lo, w);
  int KL = (int)__dmul_rn((double)(K + 1), r.u(2));
  if (KL > K) KL = K;
  const int KR = K - KL;
  for (int k = 0; k < KL; ++k) {
    ++res.evals;
    if (above(lo)) lo = __dsub_rn(lo, w); else break;
  }
  for (int k = 0; k < KR; ++k) {
    ++res.evals;
    if (above(hi)) hi = __dadd_rn(hi, w); else break;
  }
  for (int j = 0; j < shrink_max; ++j) {
    const double xs = __dadd_rn(lo, __dmul_rn(__dsub_rn(hi, lo), r.u(3u + (uint32_t)j)));
    ++res.evals;
    if (above(xs)) {
      res.x = xs;
      res.capped = false;
      return res;
    }
    if (xs > x0) hi = xs; else lo = xs;
  }
  res.x = x0;
  res.capped = true;
  return res;
}

// slice_update executed by the 32 lanes of a warp, with the same result (value,
// evaluation count, flags) as the sequential form: the stepping-out points
// (lo - k w and hi + k w, each rounded step by step as in the sequential loop)
// and the shrinkage proposals (the chain of brackets that follows when every
// earlier proposal was rejected; a bracket depends only on which side of x0 the
// rejected proposals fell) are known before any density is evaluated, so each
// round evaluates up to 32 of them at once and keeps the outcome of the first
// one the sequential loop would stop at.  Round 1: lane 0 evaluates f(x0),
// lanes 1..15 the first 15 left points, lanes 16..31 the first 16 right points;
// later rounds take 16 points per side, then 32 shrinkage proposals.  Every lane
// returns the result.
template <class F>
__device__ __forceinline__ SliceResult slice_update_warp(double x0, double w, const F& f, Rng& r,
                                                         int K, int shrink_max) {
  const int lane = threadIdx.x & 31;
  SliceResult res;
  const double lu0 = log(r.u(0));
  const double v = __dmul_rn(w, r.u(1));
  const double lo0 = __dsub_rn(x0, v);
  const double hi0 = __dadd_rn(lo0, w);
  int KL = (int)__dmul_rn((double)(K + 1), r.u(2));
  if (KL > K) KL = K;
  const int KR = K - KL;

  // round 1: f(x0) and the first stepping-out points
  double aux, aux0 = 0.0;
  double pt;
  int side, k;  // side 0: left, 1: right, -1: none
  if (lane == 0) {
    pt = x0, side = -1, k = 0;
  } else if (lane < 16) {
    side = 0, k = lane - 1;
  } else {
    side = 1, k = lane - 16;
  }
  if (side == 0) {
    pt = lo0;
    for (int i = 0; i < k; ++i) pt = __dsub_rn(pt, w);
  } else if (side == 1) {
    pt = hi0;
    for (int i = 0; i < k; ++i) pt = __dadd_rn(pt, w);
  }
  const bool need = side < 0 || (side == 0 ? k < KL : k < KR);
  double fv = need ? f(pt, &aux) : 0.0;
  if (lane == 0) aux0 = aux;
  const double f0 = __shfl_sync(0xffffffffu, fv, 0);
  aux0 = __shfl_sync(0xffffffffu, aux0, 0);
  res.nonfinite = !isfinite(f0);
  const double logu = __dadd_rn(f0, lu0);
  res.evals = 1;

  // stepping out: a side stops at its first failing point or after K_side points
  double lo = lo0, hi = hi0;
  bool open_l = KL > 0, open_r = KR > 0;
  int base_l = 0, base_r = 0;     // index of this round's first point per side
  int nl = 15, nr = 16;           // points per side in this round
  double start_l = lo0, start_r = hi0;
  for (int round = 0; open_l || open_r; ++round) {
    if (round > 0) {
      // points base + (lane & 15) for lanes 0..15 (left), 16..31 (right)
      side = lane < 16 ? 0 : 1;
      k = lane & 15;
      nl = nr = 16;
      pt = side == 0 ? start_l : start_r;
      for (int i = 0; i < k; ++i) pt = side == 0 ? __dsub_rn(pt, w) : __dadd_rn(pt, w);
      const bool act = side == 0 ? (open_l && base_l + k < KL) : (open_r && base_r + k < KR);
      fv = act ? f(pt, &aux) : 0.0;
    }
    // lane index of point j of each side in this round
    const int off_l = round == 0 ? 1 : 0, off_r = 16;
    const bool pass = logu < fv;
    const unsigned bal = __ballot_sync(0xffffffffu, pass);
    if (open_l) {
      const int m = min(nl, KL - base_l);  // points of this round the loop would reach
      int j = 0;
      while (j < m && ((bal >> (off_l + j)) & 1u)) ++j;
      // j passes, then (if j < m) one failure
      res.evals += (unsigned)(j < m ? j + 1 : m);
      for (int i = 0; i < j; ++i) lo = __dsub_rn(lo, w);
      base_l += m;
      if (j < m || base_l >= KL) open_l = false;
      else start_l = lo;
    }
    if (open_r) {
      const int m = min(nr, KR - base_r);
      int j = 0;
      while (j < m && ((bal >> (off_r + j)) & 1u)) ++j;
      res.evals += (unsigned)(j < m ? j + 1 : m);
      for (int i = 0; i < j; ++i) hi = __dadd_rn(hi, w);
      base_r += m;
      if (j < m || base_r >= KR) open_r = false;
      else start_r = hi;
    }
  }

  // shrinkage: lane j proposes the (base + j)-th point of the rejection chain;
  // the first round takes 8 proposals (most updates accept within a few), later
  // rounds 32.  Lane j draws only the uniform of proposal base + j (one Philox
  // block per lane, in parallel); every lane then walks the chain with the
  // uniforms broadcast from their lanes, keeping its own point, and ends with
  // the bracket left after rejecting all m points.
  for (int base = 0, width = 8; base < shrink_max; base += width, width = 32) {
    const int m = min(width, shrink_max - base);
    const double u_mine = lane < m ? r.u(3u + (uint32_t)(base + lane)) : 0.0;
    double l2 = lo, h2 = hi, xs = 0.0;
    for (int i = 0; i < m; ++i) {
      const double ui = __shfl_sync(0xffffffffu, u_mine, i);
      const double xi = __dadd_rn(l2, __dmul_rn(__dsub_rn(h2, l2), ui));
      if (i == lane) xs = xi;
      if (xi > x0) h2 = xi; else l2 = xi;
    }
    const bool act = lane < m;
    fv = act ? f(xs, &aux) : -INFINITY;
    const unsigned bal = __ballot_sync(0xffffffffu, act && logu < fv);
    if (bal) {
      const int j = __ffs(bal) - 1;
      res.evals += (unsigned)(j + 1);
      res.x = __shfl_sync(0xffffffffu, xs, j);
      res.aux = __shfl_sync(0xffffffffu, aux, j);
      res.capped = false;
      return res;
    }
    res.evals += (unsigned)m;
    lo = l2;  // the bracket after the m rejections (the same in every lane)
    hi = h2;
  }
  res.x = x0;
  res.aux = aux0;
  res.capped = true;
  return res;
}

// Width tuning, Algorithm 2 step 7: while it <= M_B add it*|x_new - x_old| to
// w_aux; once it > M_C set w = w_aux / (it (it+1) / 2) when that is positive and
// finite.
__device__ __forceinline__ void tune_width(double& w, double& waux, long long it, double x_new,
                                           double x_old, long long burnin, long long tune_start) {
  if (it > burnin) return;
  waux = __dadd_rn(waux, __dmul_rn((double)it, fabs(__dsub_rn(x_new, x_old))));
  if (it > tune_start) {
    const double wn = __ddiv_rn(waux, __dmul_rn(__dmul_rn(0.5, (double)it), (double)(it + 1)));
    if (wn > 0.0 && isfinite(wn)) w = wn;
  }
}

}  // namespace fbs
