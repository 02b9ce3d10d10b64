/*
 * fbs_oracle.h -- plain FP64 CPU oracle for the Gibbs sweep of the RNA-seq
 * hierarchical model (Landau & Niemi, arXiv 1606.06659).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the GPU library includes, links or
 * calls this code; only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg load it.  It shares no code with the CUDA path: its
 * Philox generator, samplers, densities and reductions are written here
 * from their published definitions.
 *
 * Layouts (host memory, caller-owned, row-major):
 *   y      int32 [G][N]      counts, gene-major
 *   X      double [N][L]     model matrix
 *   h      double [N]        sample offsets
 *   eps    double [G][N]     epsilon_{gn}
 *   beta   double [G][L]     beta_{gl}
 *   gam    double [G]        gamma_g
 *   phi    double [2L+2]     (nu, tau, theta_1..theta_L, sigma^2_1..sigma^2_L)
 */
#ifndef FBS_ORACLE_H
#define FBS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* RNG stream identifiers: one per kind of random variable. */
enum {
  ORC_STREAM_EPS = 1,
  ORC_STREAM_GAMMA = 2,
  ORC_STREAM_NU = 3,
  ORC_STREAM_TAU = 4,
  ORC_STREAM_BETA = 5,
  ORC_STREAM_THETA = 6,
  ORC_STREAM_SIGMA = 7,
  ORC_STREAM_PSI = 10,
  ORC_STREAM_TEST = 200
};

typedef struct {
  int N, G, L;
  const int32_t* y; /* [G][N] */
  const double* X;  /* [N][L] */
  const double* h;  /* [N] */
  double a, b;      /* tau ~ Gamma(a, rate b) */
  double d;         /* nu ~ Uniform(0, d) */
  const double* c;  /* [L] theta_l ~ Normal(0, c_l^2) */
  const double* s;  /* [L] sigma_l ~ Uniform(0, s_l) */
  const double* theta_mean; /* [L] prior mean of theta_l (NULL: 0); the three-level
                               model sets it to the top-level m_l */
} orc_model;

typedef struct {
  double* eps;       /* [G][N] */
  double* beta;      /* [G][L] */
  double* gam;       /* [G] */
  double* phi;       /* [2L+2]: nu, tau, theta[L], sigma2[L] */
  double* w_eps;     /* [G][N] slice widths */
  double* waux_eps;  /* [G][N] tuning accumulators */
  double* w_beta;    /* [G][L] */
  double* waux_beta; /* [G][L] */
  double* w_nu;      /* [1] */
  double* waux_nu;   /* [1] */
  /* widths of the variables that only the all-slice variant slice-samples */
  double* w_gam;     /* [G] gamma_g */
  double* waux_gam;  /* [G] */
  double* w_hyp;     /* [1+L]: tau, then sigma_1..sigma_L */
  double* waux_hyp;  /* [1+L] */
} orc_state;

typedef struct {
  uint64_t seed;
  uint32_t chain;
  int step_out_max;   /* K of Algorithm 2 */
  int shrink_max;     /* cap on shrinkage draws per slice update */
  int64_t burnin;     /* M_B */
  int64_t tune_start; /* M_C */
  double w0;          /* initial slice width */
  int all_slice;      /* 1: slice-sample gamma_g, tau and sigma_l as well (Section 4.2:
                         every non-normal full conditional); 0: draw them exactly */
} orc_opts;

typedef struct {
  /* Welford running means / mean squares, Section 3.1 */
  double* mean_eps;  /* [G][N] */
  double* msq_eps;
  double* mean_beta; /* [G][L] */
  double* msq_beta;
  double* mean_gam;  /* [G] */
  double* msq_gam;
  double* mean_phi;  /* [2L+2] */
  double* msq_phi;
  int64_t count;     /* number of post-burn-in draws folded in */
} orc_moments;

typedef struct {
  int64_t evals_eps, evals_beta, evals_nu; /* log-density evaluations */
  int64_t slice_caps;                      /* slice updates that hit shrink_max */
  int64_t gamma_caps;                      /* gamma draws that ran out of attempts */
  int64_t trunc_caps;                      /* truncated draws that ran out of attempts */
  int64_t nonfinite;                       /* slice updates started at a non-finite density */
  int64_t evals_gam, evals_hyp;            /* all-slice variant: gamma_g; tau and sigma_l */
} orc_counters;

/* ---- host threads of the per-gene loops (OpenMP; default 1) ---- */
void orc_set_threads(int n);
int orc_get_threads(void);

/* ---- random numbers ---- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_uniform(uint64_t seed, uint32_t chain, uint32_t stream, uint32_t index,
                   uint32_t iter, uint32_t k);
double orc_normal(uint64_t seed, uint32_t chain, uint32_t stream, uint32_t index,
                  uint32_t iter, uint32_t k0);
double orc_gamma(double shape, uint64_t seed, uint32_t chain, uint32_t stream,
                 uint32_t index, uint32_t iter, uint32_t k0, int64_t* caps);
void orc_fill_uniforms(uint64_t seed, uint32_t chain, uint32_t stream, uint32_t index0,
                       int n_index, uint32_t iter, uint32_t k0, int n_k, double* out);
void orc_fill_gamma(double shape, uint64_t seed, uint32_t chain, uint32_t stream,
                    uint32_t index0, int n, uint32_t iter, double* out);
void orc_fill_normal(uint64_t seed, uint32_t chain, uint32_t stream, uint32_t index0,
                     int n, uint32_t iter, double* out);

/* ---- full-conditional log densities (additive constants dropped) ---- */
double orc_logf_eps(const orc_model* m, const orc_state* st, int g, int n, double x);
double orc_logf_beta(const orc_model* m, const orc_state* st, int g, int l, double b);
double orc_logf_nu(const orc_model* m, const orc_state* st, double nu);

/* ---- one slice update on a textbook target, for testing the sampler ---- */
/* kind 0: Normal(p0, variance p1); kind 1: Gamma(shape p0, rate p1) on x > 0 */
void orc_slice_textbook(int kind, double p0, double p1, int n, const double* x0, double w,
                        int step_out_max, int shrink_max, uint64_t seed, uint32_t iter,
                        double* out, int64_t* evals);

/* ---- Algorithm 1 steps, iteration m (1-based) ---- */
void orc_step_eps(const orc_model* m, orc_state* st, const orc_opts* o, int64_t it,
                  orc_counters* cnt);
void orc_step_gamma(const orc_model* m, orc_state* st, const orc_opts* o, int64_t it,
                    orc_counters* cnt);
void orc_step_nu(const orc_model* m, orc_state* st, const orc_opts* o, int64_t it,
                 orc_counters* cnt);
void orc_step_tau(const orc_model* m, orc_state* st, const orc_opts* o, int64_t it,
                  orc_counters* cnt);
void orc_step_beta_l(const orc_model* m, orc_state* st, const orc_opts* o, int64_t it, int l,
                     orc_counters* cnt);
void orc_step_beta(const orc_model* m, orc_state* st, const orc_opts* o, int64_t it,
                   orc_counters* cnt);
void orc_step_theta(const orc_model* m, orc_state* st, const orc_opts* o, int64_t it,
                    orc_counters* cnt);
void orc_step_sigma(const orc_model* m, orc_state* st, const orc_opts* o, int64_t it,
                    orc_counters* cnt);

/* Top level of the three-level model (Section 2.3, Figure 2) for K datasets of
 * this model whose hyperparameters share psi = (b, m_1..m_L):
 *   tau_k ~ Gamma(a_k, rate b), theta_kl ~ N(m_l, c_kl^2),
 *   b ~ Gamma(a_b, rate b_b), m_l ~ N(0, e_l^2).
 * Given phi_1..phi_K (phi [K][2L+2]), draws
 *   b ~ Gamma(a_b + sum_k a_k, rate b_b + sum_k tau_k),
 *   m_l ~ N(w sum_k theta_kl / c_kl^2, w), w = 1 / (sum_k 1/c_kl^2 + 1/e_l^2)
 * into psi [1+L] = (b, m_1..m_L).  a [K], c [K][L], e [L].  Random numbers:
 * stream ORC_STREAM_PSI, chain 0, index 0 for b and 1+l for m_l. */
void orc_step_psi(int K, int L, const double* phi, const double* a, const double* c,
                  const double* e, double a_b, double b_b, uint64_t seed, int64_t it,
                  double* psi, int64_t* gamma_caps);

/* one full sweep (Algorithm 1 steps 1-7), then Welford moments when it > burnin */
void orc_sweep(const orc_model* m, orc_state* st, const orc_opts* o, int64_t it,
               orc_moments* mom, orc_counters* cnt);

/* iterations it0+1 .. it0+n_iter; hyperparameters are written to trace_phi
 * ([n_trace][2L+2]) every `thin` post-burn-in iterations while room remains, and
 * beta to trace_beta ([n_trace][G][L]) if it is not NULL.  Returns rows written. */
int64_t orc_run(const orc_model* m, orc_state* st, const orc_opts* o, int64_t it0,
                int64_t n_iter, int64_t thin, orc_moments* mom, orc_counters* cnt,
                double* trace_phi, double* trace_beta, int64_t trace_cap);

/* default starting values; returns 0, or -1 when X^T X is singular */
int orc_init_state(const orc_model* m, orc_state* st, const orc_opts* o);

/* exact integer T_{gl} = sum_n y_{gn} X_{nl} for integer-valued X (int64 [G][L]) */
void orc_count_sums(const orc_model* m, int64_t* T);

/* Geyer initial-monotone-sequence effective sample size of one series */
double orc_ess(const double* x, int64_t n);

#ifdef __cplusplus
}
#endif
#endif
