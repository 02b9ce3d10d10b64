/*
 * fbs_oracle.c -- plain FP64 CPU oracle for one Gibbs sweep of the RNA-seq
 * hierarchical model of Landau & Niemi (arXiv 1606.06659).
 *
 * TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg load this file; the GPU library never does.  It is written
 * to be read against the paper, not to be fast: one Philox block per uniform,
 * one exp per sample and per evaluation, sums in index order.
 *
 * What each part follows:
 *   model and full conditionals ........ Section 4.1, Figure 3
 *   sweep order ........................ Algorithm 1 (Section 4.2), steps 1-7
 *   nu conditional ..................... Algorithm 1 step 3, with the sum read as
 *                                        log(gamma_g) + tau/gamma_g (the printed
 *                                        nu/gamma_g does not follow from the model)
 *   tau conditional .................... Algorithm 1 step 4
 *   slice sampler and width tuning ..... Algorithm 2 (Appendix A), steps 1-7
 *   running means / mean squares ....... Section 3.1 (Welford's one-pass update)
 *   gamma_g, theta_l, sigma_l^2 ........ conjugate draws derived from Figure 3
 *   random numbers ..................... Philox4x32-10 (Salmon et al., SC 2011)
 *                                        in place of CURAND (Section 4.2)
 *   gamma variates ..................... Marsaglia & Tsang (2000)
 *   normal variates .................... Box & Muller (1958), cosine branch
 *   effective sample size .............. Geyer (1992) initial monotone sequence
 *
 * Parity status of every function is recorded beside it ("pinned by").
 */
#include "fbs_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TWO_PI 6.283185307179586476925286766559
#define ORC_GAMMA_ATTEMPTS 64
#define ORC_TRUNC_ATTEMPTS 16
#define ORC_TRUNC_STRIDE 256 /* uniforms reserved per truncated-draw attempt */

/* ------------------------------------------------------------------------ */
/* Random numbers                                                            */
/* ------------------------------------------------------------------------ */

/* Philox4x32-10 block function, Salmon, Moraes, Dror & Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3" (SC 2011): ten rounds of the 4x32 S-box with
 * multipliers 0xD2511F53 / 0xCD9E8D57 and Weyl key increments 0x9E3779B9 /
 * 0xBB67AE85.  Pinned by the published known-answer vectors. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0;
    x1 = y1;
    x2 = y2;
    x3 = y3;
  }
  out[0] = x0;
  out[1] = x1;
  out[2] = x2;
  out[3] = x3;
}

/* The k-th uniform of random variable `index` of kind `stream` at iteration
 * `iter` of chain `chain`.  Counter = (index, stream<<24 | k>>1, iter, chain),
 * key = (low, high) 32 bits of the seed; uniform k takes output words
 * (1,0) when k is even and (3,2) when odd as a 64-bit integer x, and returns
 * (floor(x / 2^12) + 1/2) / 2^52, which is exact in double and lies in (0, 1).
 * Pinned by the Philox known-answer vectors and by exact integer arithmetic. */
double orc_uniform(uint64_t seed, uint32_t chain, uint32_t stream, uint32_t index,
                   uint32_t iter, uint32_t k) {
  uint32_t ctr[4] = {index, (stream << 24) | (k >> 1), iter, chain};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  uint32_t o[4];
  orc_philox4x32_10(ctr, key, o);
  uint64_t x = (k & 1u) ? (((uint64_t)o[3] << 32) | o[2]) : (((uint64_t)o[1] << 32) | o[0]);
  return ((double)(x >> 12) + 0.5) * 0x1p-52;
}

/* Standard normal from uniforms k0, k0+1 (Box-Muller, cosine branch).
 * Pinned by a Kolmogorov-Smirnov test against the normal CDF. */
double orc_normal(uint64_t seed, uint32_t chain, uint32_t stream, uint32_t index,
                  uint32_t iter, uint32_t k0) {
  double u1 = orc_uniform(seed, chain, stream, index, iter, k0);
  double u2 = orc_uniform(seed, chain, stream, index, iter, k0 + 1);
  return sqrt(-2.0 * log(u1)) * cos(ORC_TWO_PI * u2);
}

/* Gamma(shape, rate 1) by Marsaglia & Tsang (2000).  Attempt j (j < 64) uses
 * uniforms k0+4j, k0+4j+1 for its normal and k0+4j+2 for its acceptance test;
 * uniform k0+3 is the U^(1/shape) boost used when shape < 1.  After 64 failed
 * attempts the shape itself is returned and *caps is incremented.
 * Pinned by Kolmogorov-Smirnov tests against the gamma CDF. */
double orc_gamma(double shape, uint64_t seed, uint32_t chain, uint32_t stream,
                 uint32_t index, uint32_t iter, uint32_t k0, int64_t* caps) {
  double alpha = shape < 1.0 ? shape + 1.0 : shape;
  double dd = alpha - 1.0 / 3.0;
  double cc = 1.0 / sqrt(9.0 * dd);
  double boost = 1.0;
  if (shape < 1.0) {
    double ub = orc_uniform(seed, chain, stream, index, iter, k0 + 3);
    boost = pow(ub, 1.0 / shape);
  }
  for (uint32_t j = 0; j < ORC_GAMMA_ATTEMPTS; ++j) {
    double x = orc_normal(seed, chain, stream, index, iter, k0 + 4 * j);
    double v = 1.0 + cc * x;
    if (v <= 0.0) continue;
    v = v * v * v;
    double u = orc_uniform(seed, chain, stream, index, iter, k0 + 4 * j + 2);
    double x2 = x * x;
    if (u < 1.0 - 0.0331 * x2 * x2) return dd * v * boost;
    if (log(u) < 0.5 * x2 + dd * (1.0 - v + log(v))) return dd * v * boost;
  }
  if (caps) ++*caps;
  return shape;
}

void orc_fill_uniforms(uint64_t seed, uint32_t chain, uint32_t stream, uint32_t index0,
                       int n_index, uint32_t iter, uint32_t k0, int n_k, double* out) {
  for (int i = 0; i < n_index; ++i)
    for (int k = 0; k < n_k; ++k)
      out[(size_t)i * n_k + k] =
          orc_uniform(seed, chain, stream, index0 + (uint32_t)i, iter, k0 + (uint32_t)k);
}

void orc_fill_gamma(double shape, uint64_t seed, uint32_t chain, uint32_t stream,
                    uint32_t index0, int n, uint32_t iter, double* out) {
  for (int i = 0; i < n; ++i)
    out[i] = orc_gamma(shape, seed, chain, stream, index0 + (uint32_t)i, iter, 0, NULL);
}

void orc_fill_normal(uint64_t seed, uint32_t chain, uint32_t stream, uint32_t index0, int n,
                     uint32_t iter, double* out) {
  for (int i = 0; i < n; ++i) out[i] = orc_normal(seed, chain, stream, index0 + (uint32_t)i, iter, 0);
}

/* Inverse-gamma(shape, scale) truncated to (0, upper) by rejection: attempt t
 * draws 1/Gamma with its uniforms starting at 256*t.  After 16 failures the
 * value `keep` is returned and *caps is incremented. */
static double orc_trunc_invgamma(double shape, double scale, double upper, double keep,
                                 uint64_t seed, uint32_t chain, uint32_t stream, uint32_t index,
                                 uint32_t iter, int64_t* gcaps, int64_t* tcaps) {
  for (uint32_t t = 0; t < ORC_TRUNC_ATTEMPTS; ++t) {
    double gv = orc_gamma(shape, seed, chain, stream, index, iter, ORC_TRUNC_STRIDE * t, gcaps);
    double x = scale / gv;
    if (x < upper) return x;
  }
  if (tcaps) ++*tcaps;
  return keep;
}

/* ------------------------------------------------------------------------ */
/* Full conditionals (Section 4.1, Figure 3); constants in the variable are  */
/* dropped.                                                                  */
/* ------------------------------------------------------------------------ */

/* log p(eps_gn | ...) = y_gn*x - exp(h_n + x + X_n beta_g) - x^2 / (2 gamma_g):
 * Poisson likelihood of y_gn times the Normal(0, gamma_g) prior of eps_gn.
 * Pinned by quadrature of the model density and Kolmogorov-Smirnov tests. */
double orc_logf_eps(const orc_model* m, const orc_state* st, int g, int n, double x) {
  const int L = m->L;
  double xb = 0.0;
  for (int l = 0; l < L; ++l) xb += m->X[n * L + l] * st->beta[(size_t)g * L + l];
  double eta = m->h[n] + x + xb;
  double y = (double)m->y[(size_t)g * m->N + n];
  return y * x - exp(eta) - x * x / (2.0 * st->gam[g]);
}

/* log p(beta_gl | ...) = b * sum_n y_gn X_nl - sum_n exp(h_n + eps_gn + X_n beta_g)
 * - (b - theta_l)^2 / (2 sigma_l^2), with beta_gl = b inside X_n beta_g.
 * Pinned by quadrature of the model density and Kolmogorov-Smirnov tests. */
double orc_logf_beta(const orc_model* m, const orc_state* st, int g, int l, double b) {
  const int N = m->N, L = m->L;
  double T = 0.0, rate = 0.0;
  for (int n = 0; n < N; ++n) {
    double xb = 0.0;
    for (int k = 0; k < L; ++k) {
      double bk = (k == l) ? b : st->beta[(size_t)g * L + k];
      xb += m->X[n * L + k] * bk;
    }
    T += (double)m->y[(size_t)g * N + n] * m->X[n * L + l];
    rate += exp(m->h[n] + st->eps[(size_t)g * N + n] + xb);
  }
  double theta = st->phi[2 + l], sig2 = st->phi[2 + L + l];
  double dv = b - theta;
  return b * T - rate - dv * dv / (2.0 * sig2);
}

typedef struct {
  double G, d, tau, S1, S2;
} orc_nu_ctx;

static double orc_logf_nu_ctx(double nu, const orc_nu_ctx* c) {
  if (!(nu > 0.0 && nu < c->d)) return -INFINITY;
  return -c->G * lgamma(0.5 * nu) + 0.5 * c->G * nu * log(0.5 * nu * c->tau) -
         0.5 * nu * (c->S1 + c->tau * c->S2);
}

static void orc_gamma_sums(const orc_model* m, const orc_state* st, double* S1, double* S2) {
  double s1 = 0.0, s2 = 0.0;
  for (int g = 0; g < m->G; ++g) {
    s1 += log(st->gam[g]);
    s2 += 1.0 / st->gam[g];
  }
  *S1 = s1;
  *S2 = s2;
}

/* log p(nu | ...) = -G lgamma(nu/2) + (G nu / 2) log(nu tau / 2)
 *                   - (nu/2) sum_g [log gamma_g + tau / gamma_g],  0 < nu < d
 * (Algorithm 1 step 3; the product of Inverse-Gamma(nu/2, nu tau/2) densities of
 * the gamma_g with the Uniform(0, d) prior).  Pinned by quadrature of the sum of
 * inverse-gamma log densities and a Kolmogorov-Smirnov test. */
double orc_logf_nu(const orc_model* m, const orc_state* st, double nu) {
  orc_nu_ctx c;
  c.G = (double)m->G;
  c.d = m->d;
  c.tau = st->phi[1];
  orc_gamma_sums(m, st, &c.S1, &c.S2);
  return orc_logf_nu_ctx(nu, &c);
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2: univariate stepping-out slice sampler                        */
/* ------------------------------------------------------------------------ */

typedef double (*orc_logf_fn)(double x, const void* ctx);

typedef struct {
  uint64_t seed;
  uint32_t chain, stream, index, iter;
} orc_rng;

static double orc_u(const orc_rng* r, uint32_t k) {
  return orc_uniform(r->seed, r->chain, r->stream, r->index, r->iter, k);
}

/* Steps 1-6 of Algorithm 2 from x0 with width w and stepping-out bound K.
 * Uniform 0 places the level u under f(x0) (on the log scale), uniform 1 places
 * the initial interval, uniform 2 splits K into K_L and K_R, and uniform 3+j is
 * the j-th proposal of the shrinkage loop, which gives up after shrink_max
 * proposals and then keeps x0.  Comparisons are strict, as printed. */
static double orc_slice(double x0, orc_logf_fn f, const void* ctx, double w, int K,
                        int shrink_max, const orc_rng* r, int64_t* evals, orc_counters* cnt) {
  double f0 = f(x0, ctx);
  ++*evals;
  if (!isfinite(f0) && cnt) ++cnt->nonfinite;
  double logu = f0 + log(orc_u(r, 0));       /* step 1: u ~ U(0, f(x0)) */
  double v = w * orc_u(r, 1);                /* step 2a */
  double lo = x0 - v;                        /* step 2b */
  double hi = lo + w;                        /* step 2c */
  int KL = (int)((double)(K + 1) * orc_u(r, 2)); /* step 3a: uniform on {0..K} */
  if (KL > K) KL = K;
  int KR = K - KL;                           /* step 3b */
  for (int k = 0; k < KL; ++k) {             /* step 4a */
    ++*evals;
    if (logu < f(lo, ctx)) lo -= w; else break;
  }
  for (int k = 0; k < KR; ++k) {             /* step 4b */
    ++*evals;
    if (logu < f(hi, ctx)) hi += w; else break;
  }
  for (int j = 0; j < shrink_max; ++j) {     /* steps 5-6 */
    double xs = lo + (hi - lo) * orc_u(r, 3u + (uint32_t)j);
    ++*evals;
    if (logu < f(xs, ctx)) return xs;
    if (xs > x0) hi = xs; else lo = xs;
  }
  if (cnt) ++cnt->slice_caps;
  return x0;
}

/* Step 7 of Algorithm 2: during burn-in (it <= M_B) add it*|x_new - x_old| to
 * w_aux; after M_C iterations set w = w_aux / (it (it+1) / 2).  A width that
 * would not be positive and finite leaves w unchanged. */
static void orc_tune(double* w, double* waux, int64_t it, double x_new, double x_old,
                     const orc_opts* o) {
  if (it > o->burnin) return;
  *waux += (double)it * fabs(x_new - x_old);
  if (it > o->tune_start) {
    double wn = *waux / (0.5 * (double)it * (double)(it + 1));
    if (wn > 0.0 && isfinite(wn)) *w = wn;
  }
}

/* Full conditionals that the all-slice variant (Section 4.2: every non-normal
 * conditional is slice-sampled) hands to Algorithm 2.  Pinned in the tests
 * against the exact Inverse-Gamma, Gamma and truncated square-root
 * Inverse-Gamma laws of the conjugate steps below. */
typedef struct {
  double shape1; /* (N + nu)/2 + 1 */
  double B;      /* (sum_n eps_gn^2 + nu tau)/2 */
} orc_gam_ctx;

/* log f(gamma_g) = -((N + nu)/2 + 1) log gamma_g - B / gamma_g on gamma_g > 0 */
static double orc_f_gam(double x, const void* vctx) {
  const orc_gam_ctx* c = (const orc_gam_ctx*)vctx;
  if (!(x > 0.0)) return -INFINITY;
  return -c->shape1 * log(x) - c->B / x;
}

typedef struct {
  double shape;  /* a + G nu / 2 */
  double rate;   /* b + (nu/2) sum_g 1/gamma_g */
} orc_tau_ctx;

/* log f(tau) = (shape - 1) log tau - rate tau on tau > 0 */
static double orc_f_tau(double x, const void* vctx) {
  const orc_tau_ctx* c = (const orc_tau_ctx*)vctx;
  if (!(x > 0.0)) return -INFINITY;
  return (c->shape - 1.0) * log(x) - c->rate * x;
}

typedef struct {
  double G;      /* number of genes */
  double hS;     /* sum_g (beta_gl - theta_l)^2 / 2 */
  double s;      /* upper end s_l of the Uniform(0, s_l) prior */
} orc_sig_ctx;

/* log f(sigma_l) = -G log sigma_l - hS / sigma_l^2 on 0 < sigma_l < s_l: G
 * Normal(theta_l, sigma_l^2) terms times the flat prior density of sigma_l */
static double orc_f_sig(double x, const void* vctx) {
  const orc_sig_ctx* c = (const orc_sig_ctx*)vctx;
  if (!(x > 0.0 && x < c->s)) return -INFINITY;
  return -c->G * log(x) - c->hS / (x * x);
}

typedef struct {
  int kind;
  double p0, p1;
} orc_textbook_ctx;

static double orc_logf_textbook(double x, const void* vctx) {
  const orc_textbook_ctx* c = (const orc_textbook_ctx*)vctx;
  if (c->kind == 0) {
    double dv = x - c->p0;
    return -dv * dv / (2.0 * c->p1);
  }
  if (!(x > 0.0)) return -INFINITY;
  return (c->p0 - 1.0) * log(x) - c->p1 * x;
}

void orc_slice_textbook(int kind, double p0, double p1, int n, const double* x0, double w,
                        int step_out_max, int shrink_max, uint64_t seed, uint32_t iter,
                        double* out, int64_t* evals) {
  orc_textbook_ctx c = {kind, p0, p1};
  int64_t ev = 0;
  for (int i = 0; i < n; ++i) {
    orc_rng r = {seed, 0, ORC_STREAM_TEST, (uint32_t)i, iter};
    out[i] = orc_slice(x0[i], orc_logf_textbook, &c, w, step_out_max, shrink_max, &r, &ev, NULL);
  }
  if (evals) *evals = ev;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1                                                               */
/* ------------------------------------------------------------------------ */

typedef struct {
  const orc_model* m;
  const orc_state* st;
  int g, j;
} orc_gene_ctx;

static double orc_f_eps(double x, const void* vctx) {
  const orc_gene_ctx* c = (const orc_gene_ctx*)vctx;
  return orc_logf_eps(c->m, c->st, c->g, c->j, x);
}

static double orc_f_beta(double b, const void* vctx) {
  const orc_gene_ctx* c = (const orc_gene_ctx*)vctx;
  return orc_logf_beta(c->m, c->st, c->g, c->j, b);
}

static double orc_f_nu(double nu, const void* vctx) {
  return orc_logf_nu_ctx(nu, (const orc_nu_ctx*)vctx);
}

/* Host threads of the per-gene loops of steps 1, 2 and 5 (OpenMP, when the
 * oracle is compiled with it; 1 by default).  Every gene's update reads only
 * its own state and its own Philox counters, so the states do not depend on
 * the thread count; each thread counts into its own counters, which are added
 * up at the end of the loop. */
static int orc_threads = 1;

void orc_set_threads(int n) { orc_threads = n > 0 ? n : 1; }

int orc_get_threads(void) { return orc_threads; }

static void orc_add_counters(orc_counters* to, const orc_counters* from) {
  int64_t* a = (int64_t*)to;
  const int64_t* b = (const int64_t*)from;
  for (size_t i = 0; i < sizeof(orc_counters) / sizeof(int64_t); ++i) a[i] += b[i];
}

/* Step 1: in parallel over (g, n), a slice update of every eps_gn. */
void orc_step_eps(const orc_model* m, orc_state* st, const orc_opts* o, int64_t it,
                  orc_counters* cnt) {
  const int N = m->N;
#pragma omp parallel num_threads(orc_threads) if (orc_threads > 1)
  {
    orc_counters loc;
    memset(&loc, 0, sizeof(loc));
#pragma omp for schedule(static)
    for (int g = 0; g < m->G; ++g) {
      for (int n = 0; n < N; ++n) {
        size_t e = (size_t)g * N + n;
        orc_gene_ctx c = {m, st, g, n};
        orc_rng r = {o->seed, o->chain, ORC_STREAM_EPS, (uint32_t)e, (uint32_t)it};
        double x_old = st->eps[e];
        double x_new = orc_slice(x_old, orc_f_eps, &c, st->w_eps[e], o->step_out_max,
                                 o->shrink_max, &r, &loc.evals_eps, &loc);
        st->eps[e] = x_new;
        orc_tune(&st->w_eps[e], &st->waux_eps[e], it, x_new, x_old, o);
      }
    }
#pragma omp critical
    orc_add_counters(cnt, &loc);
  }
}

/* Step 2: in parallel over g, gamma_g from its full conditional
 * Inverse-Gamma((N + nu)/2, (sum_n eps_gn^2 + nu tau)/2), the conjugate update
 * of the Inverse-Gamma(nu/2, nu tau/2) prior by N Normal(0, gamma_g) terms:
 * drawn exactly, or (all_slice) by a slice update of that density. */
void orc_step_gamma(const orc_model* m, orc_state* st, const orc_opts* o, int64_t it,
                    orc_counters* cnt) {
  const int N = m->N;
  const double nu = st->phi[0], tau = st->phi[1];
#pragma omp parallel num_threads(orc_threads) if (orc_threads > 1)
  {
    orc_counters loc;
    memset(&loc, 0, sizeof(loc));
#pragma omp for schedule(static)
    for (int g = 0; g < m->G; ++g) {
      double ss = 0.0;
      for (int n = 0; n < N; ++n) {
        double e = st->eps[(size_t)g * N + n];
        ss += e * e;
      }
      double shape = 0.5 * ((double)N + nu);
      double scale = 0.5 * (ss + nu * tau);
      if (o->all_slice) {
        orc_gam_ctx c = {shape + 1.0, scale};
        orc_rng r = {o->seed, o->chain, ORC_STREAM_GAMMA, (uint32_t)g, (uint32_t)it};
        double x_old = st->gam[g];
        double x_new = orc_slice(x_old, orc_f_gam, &c, st->w_gam[g], o->step_out_max,
                                 o->shrink_max, &r, &loc.evals_gam, &loc);
        st->gam[g] = x_new;
        orc_tune(&st->w_gam[g], &st->waux_gam[g], it, x_new, x_old, o);
        continue;
      }
      double gv = orc_gamma(shape, o->seed, o->chain, ORC_STREAM_GAMMA, (uint32_t)g,
                            (uint32_t)it, 0, &loc.gamma_caps);
      st->gam[g] = scale / gv;
    }
#pragma omp critical
    orc_add_counters(cnt, &loc);
  }
}

/* Step 3: reduction to S1 = sum log gamma_g and S2 = sum 1/gamma_g, then a slice
 * update of nu on (0, d). */
void orc_step_nu(const orc_model* m, orc_state* st, const orc_opts* o, int64_t it,
                 orc_counters* cnt) {
  orc_nu_ctx c;
  c.G = (double)m->G;
  c.d = m->d;
  c.tau = st->phi[1];
  orc_gamma_sums(m, st, &c.S1, &c.S2);
  orc_rng r = {o->seed, o->chain, ORC_STREAM_NU, 0u, (uint32_t)it};
  double x_old = st->phi[0];
  double x_new = orc_slice(x_old, orc_f_nu, &c, st->w_nu[0], o->step_out_max, o->shrink_max,
                           &r, &cnt->evals_nu, cnt);
  st->phi[0] = x_new;
  orc_tune(st->w_nu, st->waux_nu, it, x_new, x_old, o);
}

/* Step 4: reduction to S2 = sum 1/gamma_g, then
 * tau ~ Gamma(a + G nu / 2, rate = b + (nu/2) S2): drawn exactly, or (all_slice)
 * by a slice update of that density. */
void orc_step_tau(const orc_model* m, orc_state* st, const orc_opts* o, int64_t it,
                  orc_counters* cnt) {
  double S1, S2;
  orc_gamma_sums(m, st, &S1, &S2);
  const double nu = st->phi[0];
  double shape = m->a + 0.5 * (double)m->G * nu;
  double rate = m->b + 0.5 * nu * S2;
  if (o->all_slice) {
    orc_tau_ctx c = {shape, rate};
    orc_rng r = {o->seed, o->chain, ORC_STREAM_TAU, 0u, (uint32_t)it};
    double x_old = st->phi[1];
    double x_new = orc_slice(x_old, orc_f_tau, &c, st->w_hyp[0], o->step_out_max,
                             o->shrink_max, &r, &cnt->evals_hyp, cnt);
    st->phi[1] = x_new;
    orc_tune(&st->w_hyp[0], &st->waux_hyp[0], it, x_new, x_old, o);
    return;
  }
  double gv = orc_gamma(shape, o->seed, o->chain, ORC_STREAM_TAU, 0u, (uint32_t)it, 0,
                        &cnt->gamma_caps);
  st->phi[1] = gv / rate;
}

/* Step 5 for one column l: in parallel over g, a slice update of beta_gl. */
void orc_step_beta_l(const orc_model* m, orc_state* st, const orc_opts* o, int64_t it, int l,
                     orc_counters* cnt) {
  const int L = m->L;
#pragma omp parallel num_threads(orc_threads) if (orc_threads > 1)
  {
    orc_counters loc;
    memset(&loc, 0, sizeof(loc));
#pragma omp for schedule(static)
    for (int g = 0; g < m->G; ++g) {
      size_t e = (size_t)g * L + l;
      orc_gene_ctx c = {m, st, g, l};
      orc_rng r = {o->seed, o->chain, ORC_STREAM_BETA, (uint32_t)e, (uint32_t)it};
      double x_old = st->beta[e];
      double x_new = orc_slice(x_old, orc_f_beta, &c, st->w_beta[e], o->step_out_max,
                               o->shrink_max, &r, &loc.evals_beta, &loc);
      st->beta[e] = x_new;
      orc_tune(&st->w_beta[e], &st->waux_beta[e], it, x_new, x_old, o);
    }
#pragma omp critical
    orc_add_counters(cnt, &loc);
  }
}

/* Step 5: for l = 1..L in sequence. */
void orc_step_beta(const orc_model* m, orc_state* st, const orc_opts* o, int64_t it,
                   orc_counters* cnt) {
  for (int l = 0; l < m->L; ++l) orc_step_beta_l(m, st, o, it, l, cnt);
}

/* Step 6: reduction to sum_g beta_gl, then theta_l ~ Normal(v sum_g beta_gl /
 * sigma_l^2, v) with v = 1 / (G / sigma_l^2 + 1 / c_l^2): the normal-normal
 * update of the Normal(0, c_l^2) prior. */
void orc_step_theta(const orc_model* m, orc_state* st, const orc_opts* o, int64_t it,
                    orc_counters* cnt) {
  (void)cnt;
  const int L = m->L;
  for (int l = 0; l < L; ++l) {
    double B1 = 0.0;
    for (int g = 0; g < m->G; ++g) B1 += st->beta[(size_t)g * L + l];
    double sig2 = st->phi[2 + L + l];
    double v = 1.0 / ((double)m->G / sig2 + 1.0 / (m->c[l] * m->c[l]));
    double mean = m->theta_mean ? v * (B1 / sig2 + m->theta_mean[l] / (m->c[l] * m->c[l]))
                                : v * B1 / sig2;
    double z = orc_normal(o->seed, o->chain, ORC_STREAM_THETA, (uint32_t)l, (uint32_t)it, 0);
    st->phi[2 + l] = mean + sqrt(v) * z;
  }
}

/* Step 7: reduction to S_l = sum_g (beta_gl - theta_l)^2, then sigma_l^2 ~
 * Inverse-Gamma((G-1)/2, S_l/2) truncated to (0, s_l^2): the Uniform(0, s_l)
 * prior on sigma_l carries the Jacobian 1/(2 sigma_l) onto sigma_l^2.  With
 * all_slice, sigma_l is slice-sampled on (0, s_l) instead. */
void orc_step_sigma(const orc_model* m, orc_state* st, const orc_opts* o, int64_t it,
                    orc_counters* cnt) {
  const int L = m->L;
  for (int l = 0; l < L; ++l) {
    double theta = st->phi[2 + l];
    double S = 0.0;
    for (int g = 0; g < m->G; ++g) {
      double dv = st->beta[(size_t)g * L + l] - theta;
      S += dv * dv;
    }
    if (o->all_slice) {
      /* the slice variable is sigma_l itself; the state keeps sigma_l^2 */
      orc_sig_ctx c = {(double)m->G, 0.5 * S, m->s[l]};
      orc_rng r = {o->seed, o->chain, ORC_STREAM_SIGMA, (uint32_t)l, (uint32_t)it};
      double x_old = sqrt(st->phi[2 + L + l]);
      double x_new = orc_slice(x_old, orc_f_sig, &c, st->w_hyp[1 + l], o->step_out_max,
                               o->shrink_max, &r, &cnt->evals_hyp, cnt);
      st->phi[2 + L + l] = x_new * x_new;
      orc_tune(&st->w_hyp[1 + l], &st->waux_hyp[1 + l], it, x_new, x_old, o);
      continue;
    }
    double shape = 0.5 * ((double)m->G - 1.0);
    double upper = m->s[l] * m->s[l];
    st->phi[2 + L + l] =
        orc_trunc_invgamma(shape, 0.5 * S, upper, st->phi[2 + L + l], o->seed, o->chain,
                           ORC_STREAM_SIGMA, (uint32_t)l, (uint32_t)it, &cnt->gamma_caps,
                           &cnt->trunc_caps);
  }
}

/* The top-level step of the three-level model: psi given the K datasets'
 * hyperparameters.  The theta_kl are Normal(m_l, c_kl^2) terms of m_l and the
 * tau_k Gamma(a_k, rate b) terms of b, so both updates are conjugate: a
 * reduction over k to sum_k tau_k and sum_k a_k (b), and to sum_k theta_kl /
 * c_kl^2 and sum_k 1/c_kl^2 (m_l). */
void orc_step_psi(int K, int L, const double* phi, const double* a, const double* c,
                  const double* e, double a_b, double b_b, uint64_t seed, int64_t it,
                  double* psi, int64_t* gamma_caps) {
  const int P = 2 * L + 2;
  double sa = 0.0, st = 0.0;
  for (int k = 0; k < K; ++k) {
    sa += a[k];
    st += phi[(size_t)k * P + 1];
  }
  double gv = orc_gamma(a_b + sa, seed, 0u, ORC_STREAM_PSI, 0u, (uint32_t)it, 0, gamma_caps);
  psi[0] = gv / (b_b + st);
  for (int l = 0; l < L; ++l) {
    double prec = 0.0, s = 0.0;
    for (int k = 0; k < K; ++k) {
      double c2 = c[(size_t)k * L + l] * c[(size_t)k * L + l];
      prec += 1.0 / c2;
      s += phi[(size_t)k * P + 2 + l] / c2;
    }
    double w = 1.0 / (prec + 1.0 / (e[l] * e[l]));
    double z = orc_normal(seed, 0u, ORC_STREAM_PSI, 1u + (uint32_t)l, (uint32_t)it, 0);
    psi[1 + l] = w * s + sqrt(w) * z;
  }
}

/* Welford's update (Section 3.1) of a running mean and mean square with the
 * k-th draw x. */
static void orc_welford(double* mean, double* msq, double x, int64_t k) {
  *mean += (x - *mean) / (double)k;
  *msq += (x * x - *msq) / (double)k;
}

static void orc_update_moments(const orc_model* m, const orc_state* st, orc_moments* mom) {
  const int64_t k = mom->count + 1;
  const size_t GN = (size_t)m->G * m->N, GL = (size_t)m->G * m->L;
  for (size_t i = 0; i < GN; ++i) orc_welford(&mom->mean_eps[i], &mom->msq_eps[i], st->eps[i], k);
  for (size_t i = 0; i < GL; ++i)
    orc_welford(&mom->mean_beta[i], &mom->msq_beta[i], st->beta[i], k);
  for (int g = 0; g < m->G; ++g) orc_welford(&mom->mean_gam[g], &mom->msq_gam[g], st->gam[g], k);
  for (int p = 0; p < 2 * m->L + 2; ++p)
    orc_welford(&mom->mean_phi[p], &mom->msq_phi[p], st->phi[p], k);
  mom->count = k;
}

void orc_sweep(const orc_model* m, orc_state* st, const orc_opts* o, int64_t it,
               orc_moments* mom, orc_counters* cnt) {
  orc_step_eps(m, st, o, it, cnt);   /* step 1 */
  orc_step_gamma(m, st, o, it, cnt); /* step 2 */
  orc_step_nu(m, st, o, it, cnt);    /* step 3 */
  orc_step_tau(m, st, o, it, cnt);   /* step 4 */
  orc_step_beta(m, st, o, it, cnt);  /* step 5 */
  orc_step_theta(m, st, o, it, cnt); /* step 6 */
  orc_step_sigma(m, st, o, it, cnt); /* step 7 */
  if (mom && it > o->burnin) orc_update_moments(m, st, mom);
}

int64_t orc_run(const orc_model* m, orc_state* st, const orc_opts* o, int64_t it0,
                int64_t n_iter, int64_t thin, orc_moments* mom, orc_counters* cnt,
                double* trace_phi, double* trace_beta, int64_t trace_cap) {
  const int P = 2 * m->L + 2;
  const size_t GL = (size_t)m->G * m->L;
  int64_t rows = 0;
  for (int64_t it = it0 + 1; it <= it0 + n_iter; ++it) {
    orc_sweep(m, st, o, it, mom, cnt);
    if (it > o->burnin && thin > 0 && (it - o->burnin) % thin == 0 && rows < trace_cap) {
      if (trace_phi) memcpy(trace_phi + (size_t)rows * P, st->phi, sizeof(double) * P);
      if (trace_beta) memcpy(trace_beta + (size_t)rows * GL, st->beta, sizeof(double) * GL);
      ++rows;
    }
  }
  return rows;
}

/* ------------------------------------------------------------------------ */
/* Starting values and count sums                                            */
/* ------------------------------------------------------------------------ */

/* Default starting values (the paper leaves them open): eps = 0; beta_g the
 * least-squares fit of log(y_gn + 1) - h_n on X; gamma_g = 1; theta_l and
 * sigma_l^2 the mean and variance of the beta_gl over g, the variance clamped to
 * [1e-6, s_l^2 / 4]; nu = min(3, d/2); tau = 1; every width w0, every w_aux 0. */
int orc_init_state(const orc_model* m, orc_state* st, const orc_opts* o) {
  const int N = m->N, G = m->G, L = m->L;
  double* A = (double*)calloc((size_t)L * 2 * L, sizeof(double)); /* [X^T X | I] */
  double* P = (double*)calloc((size_t)L * N, sizeof(double));     /* (X^T X)^-1 X^T */
  if (!A || !P) {
    free(A);
    free(P);
    return -1;
  }
  for (int i = 0; i < L; ++i) {
    for (int j = 0; j < L; ++j) {
      double s = 0.0;
      for (int n = 0; n < N; ++n) s += m->X[n * L + i] * m->X[n * L + j];
      A[i * 2 * L + j] = s;
    }
    A[i * 2 * L + L + i] = 1.0;
  }
  double scale = 0.0;
  for (int i = 0; i < L; ++i) scale = fmax(scale, fabs(A[i * 2 * L + i]));
  /* Gauss-Jordan elimination with partial pivoting */
  for (int col = 0; col < L; ++col) {
    int piv = col;
    for (int r = col + 1; r < L; ++r)
      if (fabs(A[r * 2 * L + col]) > fabs(A[piv * 2 * L + col])) piv = r;
    if (!(fabs(A[piv * 2 * L + col]) > 1e-10 * scale)) {
      free(A);
      free(P);
      return -1;
    }
    if (piv != col)
      for (int j = 0; j < 2 * L; ++j) {
        double t = A[col * 2 * L + j];
        A[col * 2 * L + j] = A[piv * 2 * L + j];
        A[piv * 2 * L + j] = t;
      }
    double p = A[col * 2 * L + col];
    for (int j = 0; j < 2 * L; ++j) A[col * 2 * L + j] /= p;
    for (int r = 0; r < L; ++r) {
      if (r == col) continue;
      double f = A[r * 2 * L + col];
      for (int j = 0; j < 2 * L; ++j) A[r * 2 * L + j] -= f * A[col * 2 * L + j];
    }
  }
  for (int l = 0; l < L; ++l)
    for (int n = 0; n < N; ++n) {
      double s = 0.0;
      for (int k = 0; k < L; ++k) s += A[l * 2 * L + L + k] * m->X[n * L + k];
      P[l * N + n] = s;
    }
  for (int g = 0; g < G; ++g) {
    for (int l = 0; l < L; ++l) {
      double s = 0.0;
      for (int n = 0; n < N; ++n)
        s += P[l * N + n] * (log((double)m->y[(size_t)g * N + n] + 1.0) - m->h[n]);
      st->beta[(size_t)g * L + l] = s;
    }
    for (int n = 0; n < N; ++n) st->eps[(size_t)g * N + n] = 0.0;
    st->gam[g] = 1.0;
  }
  st->phi[0] = fmin(3.0, 0.5 * m->d);
  st->phi[1] = 1.0;
  for (int l = 0; l < L; ++l) {
    double mean = 0.0;
    for (int g = 0; g < G; ++g) mean += st->beta[(size_t)g * L + l];
    mean /= (double)G;
    double var = 0.0;
    for (int g = 0; g < G; ++g) {
      double dv = st->beta[(size_t)g * L + l] - mean;
      var += dv * dv;
    }
    var /= (double)G;
    double upper = 0.25 * m->s[l] * m->s[l];
    st->phi[2 + l] = mean;
    st->phi[2 + L + l] = fmin(fmax(var, 1e-6), upper);
  }
  for (size_t i = 0; i < (size_t)G * N; ++i) {
    st->w_eps[i] = o->w0;
    st->waux_eps[i] = 0.0;
  }
  for (size_t i = 0; i < (size_t)G * L; ++i) {
    st->w_beta[i] = o->w0;
    st->waux_beta[i] = 0.0;
  }
  st->w_nu[0] = o->w0;
  st->waux_nu[0] = 0.0;
  for (int g = 0; g < G; ++g) {
    st->w_gam[g] = o->w0;
    st->waux_gam[g] = 0.0;
  }
  for (int i = 0; i <= L; ++i) {
    st->w_hyp[i] = o->w0;
    st->waux_hyp[i] = 0.0;
  }
  free(A);
  free(P);
  return 0;
}

void orc_count_sums(const orc_model* m, int64_t* T) {
  const int N = m->N, L = m->L;
  for (int g = 0; g < m->G; ++g)
    for (int l = 0; l < L; ++l) {
      int64_t s = 0;
      for (int n = 0; n < N; ++n)
        s += (int64_t)m->y[(size_t)g * N + n] * (int64_t)llround(m->X[n * L + l]);
      T[(size_t)g * L + l] = s;
    }
}

/* ------------------------------------------------------------------------ */
/* Effective sample size                                                     */
/* ------------------------------------------------------------------------ */

/* Geyer's initial monotone sequence estimator: autocorrelations rho_k from the
 * biased autocovariance, pair sums Gamma_j = rho_2j + rho_2j+1 taken while
 * positive and made non-increasing, tau = -1 + 2 sum_j Gamma_j, ESS = n / tau.
 * A constant series returns n.  Pinned by AR(1) closed forms. */
double orc_ess(const double* x, int64_t n) {
  if (n < 4) return (double)n;
  double mean = 0.0;
  for (int64_t t = 0; t < n; ++t) mean += x[t];
  mean /= (double)n;
  double c0 = 0.0;
  for (int64_t t = 0; t < n; ++t) c0 += (x[t] - mean) * (x[t] - mean);
  c0 /= (double)n;
  if (!(c0 > 0.0)) return (double)n;
  double sum = 0.0, prev = INFINITY;
  for (int64_t j = 0; 2 * j + 1 < n; ++j) {
    double pair = 0.0;
    for (int64_t k = 2 * j; k <= 2 * j + 1; ++k) {
      double ck = 0.0;
      for (int64_t t = 0; t + k < n; ++t) ck += (x[t] - mean) * (x[t + k] - mean);
      pair += ck / (double)n / c0;
    }
    if (!(pair > 0.0)) break;
    if (pair > prev) pair = prev;
    sum += pair;
    prev = pair;
  }
  double tau = -1.0 + 2.0 * sum;
  if (tau < 1.0 / (double)n) tau = 1.0 / (double)n;
  return (double)n / tau;
}
