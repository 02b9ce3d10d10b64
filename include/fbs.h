/*
 * fbs.h -- C ABI of the GB300 Gibbs sampler for the fully Bayesian RNA-seq
 * hierarchical model of Landau & Niemi, "A fully Bayesian strategy for
 * high-dimensional hierarchical modeling using massively parallel computing"
 * (arXiv 1606.06659).
 *
 * Model (Section 4.1, Figure 3), for genes g = 1..G, samples n = 1..N,
 * columns l = 1..L of the N x L model matrix X:
 *   y_gn      ~ Poisson(exp(h_n + eps_gn + X_n beta_g))
 *   eps_gn    ~ Normal(0, gamma_g)
 *   gamma_g   ~ Inverse-Gamma(nu/2, nu tau/2)
 *   nu        ~ Uniform(0, d),   tau ~ Gamma(a, rate b)
 *   beta_gl   ~ Normal(theta_l, sigma_l^2)
 *   theta_l   ~ Normal(0, c_l^2), sigma_l ~ Uniform(0, s_l)
 *
 * One iteration ("sweep") is Algorithm 1 (Section 4.2): slice updates of
 * every eps_gn and beta_gl (Algorithm 2, Appendix A, with its width tuning),
 * conjugate draws of gamma_g, tau, theta_l and sigma_l^2 (truncated
 * inverse-gamma), a slice update of nu, and post-burn-in running means and
 * mean squares of every parameter (Section 3.1).  All of it runs in this
 * library's CUDA kernels on one GPU; the host only launches them.
 *
 * Hyperparameter vector phi (length 2L+2) is ordered
 *   (nu, tau, theta_1..theta_L, sigma_1^2..sigma_L^2).
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC 2011) keyed by the 64-bit
 * seed, with counter (index, stream<<24 | block, iteration, chain); uniform k
 * of a variable is ((x >> 12) + 1/2) / 2^52 for the 64-bit word pair x of
 * block k/2.  The same definition, written independently, drives the CPU
 * oracle, so both consume identical uniforms.
 *
 * Errors: every int-returning call returns FBS_OK (0) or a negative FBS_E_*
 * code and sets a thread-local message readable with fbs_last_error_string().
 * No call throws across the ABI.  Calls on one handle must not run
 * concurrently from several host threads.
 */
#ifndef FBS_H
#define FBS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FBS_OK 0
#define FBS_E_ARG (-1)       /* invalid argument (sizes, non-finite inputs, singular X ...) */
#define FBS_E_CUDA (-2)      /* a CUDA runtime call failed */
#define FBS_E_OOM (-3)       /* device memory could not be obtained */
#define FBS_E_SLICE_CAP (-4) /* a slice update ran out of shrinkage proposals (kept its value) */
#define FBS_E_NONFINITE (-5) /* a slice update started from a non-finite log density */

#define FBS_MAX_N 64 /* samples */
#define FBS_MAX_L 8  /* columns of X */
#define FBS_MAX_CLASSES 8 /* distinct non-zero values in one column of X */

#define FBS_F64 0 /* all arithmetic in FP64 */
#define FBS_F32 1 /* slice log densities in FP32; reductions, hyperparameters, moments FP64 */

/* Counter slots returned by fbs_counters(). */
#define FBS_CNT_EVALS_EPS 0   /* log-density evaluations, eps updates */
#define FBS_CNT_EVALS_BETA 1  /* log-density evaluations, beta updates */
#define FBS_CNT_EVALS_NU 2    /* log-density evaluations, nu updates */
#define FBS_CNT_SLICE_CAPS 3  /* slice updates that ran out of shrinkage proposals */
#define FBS_CNT_GAMMA_CAPS 4  /* gamma draws that ran out of attempts */
#define FBS_CNT_TRUNC_CAPS 5  /* truncated sigma^2 draws that kept their value */
#define FBS_CNT_NONFINITE 6   /* slice updates started at a non-finite log density */
#define FBS_CNT_SWEEPS 7      /* completed iterations */
#define FBS_CNT_EVALS_GAMMA 8 /* log-density evaluations, gamma_g slice updates (all_slice) */
#define FBS_CNT_EVALS_HYPER 9 /* log-density evaluations, tau and sigma_l slice updates (all_slice) */
#define FBS_NUM_COUNTERS 10

typedef struct fbs_handle fbs_handle;

/* Prior constants (Section 4.1): tau ~ Gamma(a, rate b), nu ~ U(0, d),
 * theta_l ~ N(0, c_l^2), sigma_l ~ U(0, s_l).  c and s point to L host
 * doubles, read during fbs_init only.  All must be finite and > 0. */
typedef struct {
  double a, b, d;
  const double* c;
  const double* s;
} fbs_priors;

typedef struct {
  int precision;         /* FBS_F64 or FBS_F32 */
  double w0;             /* initial slice width of every slice variable (Algorithm 2) */
  int step_out_max;      /* K of Algorithm 2: stepping-out bound, split into K_L + K_R */
  int shrink_max;        /* shrinkage proposals per update before the update keeps x0 */
  uint32_t chain;        /* chain number, the fourth Philox counter word */
  int moments_eps;       /* 1: keep running moments of every eps_gn (default 1) */
  int64_t trace_cap;     /* rows of the thinned trace (phi, and beta if trace_beta) */
  int trace_beta;        /* 1: the trace also stores all G*L beta per row */
  int block;             /* threads per block of the per-gene kernel (0: library choice) */
  int graph_segment;     /* iterations per captured CUDA graph (0: library choice, 100) */
  int all_slice;         /* 1: slice-sample gamma_g, tau and sigma_l too, each with its own
                            width (Section 4.2 slice-samples every non-normal full
                            conditional); 0 (default): draw them exactly from their
                            Inverse-Gamma, Gamma and truncated laws.  FBS_F64 only. */
  int persistent;        /* 1: fbs_run sweeps each segment of graph_segment iterations in
                            one cooperative launch of resident blocks with grid barriers
                            (every step of Algorithm 1 inside; the same chain as the graph
                            of separate launches); 0 (default): a CUDA graph of three
                            launches per iteration.  FBS_F32 only; while the learned
                            proposal is in use the graph path runs. */
} fbs_options;

/* Fill *o with the defaults: FP64, w0 = 1, K = 100, shrink_max = 100, chain 0,
 * eps moments on, no trace, library-chosen block and graph segment. */
void fbs_default_options(fbs_options* o);

/* Device bytes fbs_init needs for these sizes and options (*bytes), so that a
 * caller can provide the memory itself (for example from the PyTorch caching
 * allocator).  Returns FBS_E_ARG for sizes outside the limits. */
int fbs_workspace_bytes(int N, int G, int L, const fbs_options* opt, size_t* bytes);

/* Create a sampler.  y: N*G host int32 counts, gene-major ([G][N]) when
 * gene_major != 0, else sample-major ([N][G]); X: host [N][L] row-major;
 * h: host [N] offsets.  All host arrays are copied during the call and stay
 * owned by the caller.  workspace: NULL (the library allocates and frees its
 * device memory) or a device pointer to >= fbs_workspace_bytes() bytes,
 * 256-byte aligned, owned by the caller and not touched after fbs_free.
 * stream: the cudaStream_t on which all work of this handle is ordered
 * (NULL = legacy default stream).
 * The starting state is the library default (eps = 0; beta_g least squares of
 * log(y_gn + 1) - h_n on X; gamma_g = 1; theta_l, sigma_l^2 the mean and variance
 * of beta_gl over genes, the variance clamped to [1e-6, s_l^2/4]; nu = min(3, d/2);
 * tau = 1; widths w0), at iteration 0.
 * Errors: FBS_E_ARG when N < 1, N > FBS_MAX_N, G < 2, L < 1, L > FBS_MAX_L,
 * a column of X has more than FBS_MAX_CLASSES distinct non-zero values, X^T X is
 * singular, y < 0, a non-finite X or h, a prior constant <= 0 or non-finite, or a
 * too-small workspace; FBS_E_OOM / FBS_E_CUDA from device allocation or copies. */
int fbs_init(fbs_handle** out, const int32_t* y, int N, int G, int gene_major, const double* X,
             int L, const double* h, const fbs_priors* pri, const fbs_options* opt,
             uint64_t seed, void* workspace, size_t workspace_bytes, void* stream);

/* Run iterations m = it+1 .. it+n_iter (it = iterations done so far) of
 * Algorithm 1.  burnin is M_B: slice widths are tuned while m <= M_B (after
 * M_C = burnin/2 iterations, Algorithm 2 step 7) and running moments and the
 * trace take the draws with m > M_B.  Every thin-th post-burn-in draw
 * ((m - M_B) % thin == 0) is appended to the trace while rows remain.
 * Asynchronous on the handle's stream; returns after enqueueing. Resumable:
 * a later call continues the same chain (keep burnin and thin the same).
 * Errors: FBS_E_ARG for n_iter < 0, burnin < 0 or thin < 1; FBS_E_CUDA. */
int fbs_run(fbs_handle* h, int64_t n_iter, int64_t burnin, int64_t thin);

/* Wait for the handle's work.  Returns FBS_E_CUDA on a CUDA error (or when a
 * bounded tensor-core wait of the proposal network gave up), else
 * FBS_E_NONFINITE if any slice update so far started from a non-finite log
 * density, else FBS_E_SLICE_CAP if any slice update so far used up its
 * shrink_max shrinkage proposals without accepting one, else FBS_OK.
 * Algorithm 2 (Appendix A) puts no bound on its shrinkage loop; here an
 * update that reaches the bound keeps its current value, so the chain goes on,
 * and FBS_CNT_SLICE_CAPS counts such updates.  Both conditions are
 * sticky: they are reported by every later fbs_sync of the handle. */
int fbs_sync(fbs_handle* h);

/* Running moments (Section 3.1) copied to caller-allocated host arrays, in
 * gene-major layout: eps [G][N], beta [G][L], gamma [G], phi [2L+2].  Any
 * pointer may be NULL to skip that array.  *count receives the number of
 * draws folded in.  Posterior sd = sqrt(msq - mean^2).  Synchronous. */
int fbs_moments(fbs_handle* h, double* mean_eps, double* msq_eps, double* mean_beta,
                double* msq_beta, double* mean_gam, double* msq_gam, double* mean_phi,
                double* msq_phi, int64_t* count);

/* ---- Posterior summaries (Section 3.1) ------------------------------------
 *
 * From the running means and mean squares of C >= 1 chains of the same model,
 * pooled as Section 3.1 pools them (mean = (1/C) sum_c mean_c, msq = (1/C)
 * sum_c msq_c): the posterior mean, the posterior standard deviation
 * sd = sqrt(msq - mean^2) (0 where rounding makes msq - mean^2 negative), and
 * the normal-approximation equal-tail interval mean -/+ z * sd, whose level is
 * 1 - 2 (1 - Phi(z)) (z = 1.959963984540054 gives 95%).  The arithmetic runs on
 * the device of chains[0]; the results are copied to the caller's host arrays.
 * Every output pointer may be NULL to skip it.  Layouts are gene-major, as in
 * fbs_moments: eps [G][N], beta [G][L], gamma [G], phi [2L+2]. */
typedef struct {
  double z;                                       /* interval half-width in sds, > 0 */
  double *mean_eps, *sd_eps, *lo_eps, *hi_eps;    /* [G][N]; need eps moments */
  double *mean_beta, *sd_beta, *lo_beta, *hi_beta;  /* [G][L] */
  double *mean_gam, *sd_gam, *lo_gam, *hi_gam;    /* [G] */
  double *mean_phi, *sd_phi, *lo_phi, *hi_phi;    /* [2L+2] */
  double* trace_phi;     /* [trace_rows_max][2L+2] thinned phi draws of chains[0], or NULL */
  int64_t trace_rows_max;
  int64_t trace_rows;    /* out: rows copied to trace_phi */
  int64_t count;         /* out: draws per chain folded into the moments (M) */
  int64_t counters[FBS_NUM_COUNTERS];  /* out: FBS_CNT_* summed over the chains */
  int64_t mh_accepted, mh_tried;       /* out: learned-proposal moves, summed (0 without) */
} fbs_estimates_out;

/* Summaries of one chain (fbs_estimates) or of C chains pooled
 * (fbs_estimates_pooled, 1 <= C <= FBS_MAX_RHAT_CHAINS; batch views allowed;
 * equal N, G, L, precision and draw counts M >= 1).  FBS_E_ARG for a
 * mismatch, z <= 0, M = 0, or eps outputs requested from a chain without eps
 * moments.  Synchronous (waits for every chain). */
int fbs_estimates(fbs_handle* h, fbs_estimates_out* out);
int fbs_estimates_pooled(int C, fbs_handle* const* chains, fbs_estimates_out* out);

/* Current state to / from host arrays (gene-major, as in fbs_moments), with
 * slice widths w and tuning sums w_aux: eps, w_eps, waux_eps [G][N]; beta,
 * w_beta, waux_beta [G][L]; gamma [G]; phi [2L+2]; w_nu, waux_nu [1]; *it the
 * iteration count.  NULL pointers are skipped.  fbs_set_state also resets
 * the running moments and the trace.  Synchronous. */
int fbs_get_state(fbs_handle* h, double* eps, double* beta, double* gam, double* phi,
                  double* w_eps, double* waux_eps, double* w_beta, double* waux_beta,
                  double* w_nu, double* waux_nu, int64_t* it);
int fbs_set_state(fbs_handle* h, const double* eps, const double* beta, const double* gam,
                  const double* phi, const double* w_eps, const double* waux_eps,
                  const double* w_beta, const double* waux_beta, const double* w_nu,
                  const double* waux_nu, int64_t it);

/* Slice widths and tuning sums of the variables that only all_slice samples
 * by slice updates: w_gam, waux_gam [G] (gamma_g); w_hyp, waux_hyp [1+L]
 * (tau, then sigma_1..sigma_L; the slice variable is sigma_l, not sigma_l^2).
 * fbs_init sets every width to w0 and every sum to 0 in either mode.  NULL
 * pointers are skipped; FBS_E_ARG for an FBS_F32 handle.  Synchronous. */
int fbs_get_slice_widths(fbs_handle* h, double* w_gam, double* waux_gam, double* w_hyp,
                         double* waux_hyp);
int fbs_set_slice_widths(fbs_handle* h, const double* w_gam, const double* waux_gam,
                         const double* w_hyp, const double* waux_hyp);

/* Thinned trace: up to max_rows rows copied to host: phi rows [rows][2L+2] and,
 * when the handle keeps it and beta != NULL, beta rows [rows][G][L].
 * *rows receives the number of rows copied.  Synchronous. */
int fbs_trace(fbs_handle* h, int64_t max_rows, double* phi, double* beta, int64_t* rows);

/* Effective sample size (Geyer's initial monotone sequence) of every column
 * of the device beta trace: ess [G][L] host array.  Runs in this library's
 * kernel on the stored trace rows.  FBS_E_ARG if the handle keeps no beta
 * trace or it holds fewer than 4 rows. Synchronous. */
int fbs_beta_ess(fbs_handle* h, double* ess);

/* Exact integer sums T_gl = sum_n y_gn X_nl computed on the device, for
 * integer-valued X: T [G][L] host int64.  FBS_E_ARG if X is not integral. */
int fbs_count_sums(fbs_handle* h, int64_t* T);

/* Counters (FBS_CNT_* slots, FBS_NUM_COUNTERS values) to a host array. */
int fbs_counters(fbs_handle* h, int64_t* out);

/* Runs n_iter (1..4096) iterations as one captured CUDA graph, the same launches
 * on the same two streams as the graph segments fbs_run replays (the
 * hyperparameter kernel overlapping the next iteration's eps kernel), with the
 * sweep kernels' timing probe on: the first thread of every block records the
 * device's global timer at the block's start and end, so each kernel's time is
 * the span from its first block's start to its last block's end inside the
 * replay.  Writes the means in milliseconds to ms[0..4]: the eps kernel, the
 * gamma/beta kernel (with the learned proposal and 128-thread blocks it
 * includes the network pass for its genes), the hyperparameter kernel, the
 * learned proposal's network pass launched alone afterwards (CUDA events around
 * direct launches; 0 when the handle does not use the proposal), and the
 * replay's time per iteration (first kernel start to last kernel end over
 * n_iter).  The chain advances by n_iter iterations exactly as with fbs_run.
 * Synchronous. */
int fbs_profile(fbs_handle* h, int64_t n_iter, int64_t burnin, int64_t thin, double* ms);

/* Throughput of the arithmetic pipes the sweep kernels use, measured on the
 * current device by this library's own kernels (every SM full, 8 independent
 * dependency chains per thread, best of 3 launches timed with CUDA events):
 * out[0] FP32 fused multiply-adds/s, out[1] ex2.approx/s and out[2] lg2.approx/s
 * (the MUFU base-2 exponential and logarithm), out[3] 32-bit integer
 * multiply-high/s (the Philox rounds), out[4] FP64 fused multiply-adds/s, each
 * counted per lane.  Takes a few milliseconds; changes no clock or other device
 * setting.  These are the denominators of the sweep's arithmetic roofline. */
int fbs_measure_peaks(double* out);

/* Philox uniforms exactly as the sampler draws them: out[i*n_k + k] is uniform
 * k0+k of variable index0+i of `stream` at iteration `iter` of chain `chain`,
 * generated on the device.  out is a host array of n_index*n_k doubles. */
int fbs_uniforms(uint64_t seed, uint32_t chain, uint32_t stream, uint32_t index0, int n_index,
                 uint32_t iter, uint32_t k0, int n_k, double* out);

/* ---- Posterior probabilities of contrasts (§3.1) ---------------------------
 *
 * For every gene the running mean over the post-burn-in iterations of the
 * indicator  v_1^T beta_g > b_1 and ... and v_K^T beta_g > b_K,  for up to
 * FBS_MAX_CONTRASTS propositions of up to FBS_MAX_CONTRAST_TERMS inequalities
 * each (the paper's estimator of gene-wise posterior probabilities of
 * contrasts; a disjunction follows from conjunctions by inclusion-exclusion).
 * The device keeps exact integer counts of the iterations whose beta_g (after
 * the sweep) satisfies each proposition; the FP64 form evaluates v^T beta in
 * FP64, the FP32 form in FP32, both as sum_l v_l beta_l in order l = 1..L
 * without fused multiply-add. */
#define FBS_MAX_CONTRASTS 8
#define FBS_MAX_CONTRAST_TERMS 4

/* Set (n >= 1) or clear (n = 0) the propositions and zero their counts.
 * n_terms[p] in [1, FBS_MAX_CONTRAST_TERMS] inequalities for proposition p;
 * v host [n][FBS_MAX_CONTRAST_TERMS][L] (row-major, L of the handle), b host
 * [n][FBS_MAX_CONTRAST_TERMS]; entries beyond n_terms[p] are ignored.  Counting
 * starts with the next post-burn-in iteration.  FBS_E_ARG for batch views, n or
 * n_terms out of range, or non-finite v or b.  Synchronous. */
int fbs_set_contrasts(fbs_handle* h, int n, const int* n_terms, const double* v, const double* b);

/* prob host [G][n]: count / M for each gene and proposition, M = the number of
 * post-burn-in iterations since fbs_set_contrasts (written to *m if m is not
 * NULL; prob is 0 while M = 0).  FBS_E_ARG if no propositions are set.
 * Synchronous. */
int fbs_contrast_probs(fbs_handle* h, double* prob, int64_t* m);

/* ---- Gelman-Rubin potential scale reduction (§3.1) ------------------------
 *
 * From the running means and mean squares of C chains of the same model
 * (each the mean over the same number M of post-burn-in draws):
 *   B = M/(C-1) sum_c (mean_c - mean)^2,  S_c^2 = M/(M-1) (msq_c - mean_c^2),
 *   W = (1/C) sum_c S_c^2,                Rhat = sqrt(1 + (B/W - 1)/M);
 * NaN where W is not positive.  Computed on the device of chains[0]. */
#define FBS_MAX_RHAT_CHAINS 64

/* chains: C handles (2 <= C <= FBS_MAX_RHAT_CHAINS; batch views allowed) with
 * equal N, G, L and precision and equal moment counts M >= 2.  Outputs (host,
 * each may be NULL): rhat_phi [2L+2], rhat_beta [G][L], rhat_gam [G],
 * rhat_eps [G][N] (needs the eps moments on every chain).  FBS_E_ARG on a
 * mismatch.  Synchronous (waits for every chain). */
int fbs_rhat(int C, fbs_handle* const* chains, double* rhat_phi, double* rhat_beta,
             double* rhat_gam, double* rhat_eps);

/* ---- Learned proposal for the beta_g block (FP32 handles) -------------------
 *
 * A multilayer perceptron (features -> 64 -> GELU -> 64 -> GELU -> Gaussian)
 * trained on the GPU from draws of the plain sampler proposes beta_g* ~
 * N(mu, C C^T) together with eps_g* = eps_g - X (beta_g* - beta_g), a move that
 * keeps every log-rate h_n + eps_gn + X_n beta_g: the Poisson likelihood cancels
 * and the move is accepted with probability
 *   min(1, N(eps*; 0, gamma) N(beta*; theta, sigma^2) q(beta) /
 *          (N(eps; 0, gamma) N(beta; theta, sigma^2) q(beta*))).
 * The features are X^T (eta_g - h)/N, asinh(X^T y_g), log gamma_g, theta and
 * log sigma, all unchanged by the move, so the step is an exact
 * Metropolis-Hastings update, made after the eps updates and before the gamma
 * draw by the genes that use it, with or without the slice updates of beta_g
 * (fbs_proposal_mode).  Genes whose acceptance rate falls below a threshold
 * during calibration keep only the slice updates; the per-gene choice is then
 * fixed.  Parameters: one flat
 * FP32 array W1 [64][F], b1 [64], W2 [64][64], b2 [64], W3 [K][64], b3 [K], with
 * F = 4L+1 and K = L + L(L+1)/2.  Inference runs on the tensor cores (tcgen05)
 * with every FP32 operand split into two BF16 numbers (hi + lo) and FP32
 * accumulation, about 16 significant bits per operand.  These calls return FBS_E_ARG for FP64 handles and batch views. */

/* Number of network parameters for L columns (-1 if L is out of range). */
int fbs_proposal_param_count(int L);

/* Run n_sweeps x thin plain sweeps (fbs_run with `burnin`), and after every thin
 * sweeps append (features, beta_g) of every gene to the device training set. */
int fbs_proposal_collect(fbs_handle* h, int64_t n_sweeps, int64_t burnin, int64_t thin);

/* Train the network on the collected pairs with Adam (Kingma & Ba) on minibatches
 * of `batch` pairs drawn with replacement, for `epochs` passes; every forward and
 * backward pass runs in this library's kernels (tcgen05 tensor cores, split-BF16
 * operands, 128 pairs per block).  The tensor-core waits of a step are bounded
 * by fbs_proposal_wait_limit's poll count: a step whose wait gives up leaves the
 * parameters unchanged, and the call returns FBS_E_CUDA with the parameters of
 * the last completed step.  Training works in standardised
 * coordinates (each feature and each beta column shifted by its mean over the
 * pairs and divided by its standard deviation); the parameters are mapped back
 * to raw coordinates afterwards, so inference and fbs_proposal_params see the
 * network on raw features.  The step size decays from lr to lr/20 along a
 * cosine over the call.  *final_loss: mean Gaussian negative log-likelihood of
 * the raw beta (without the L/2 log 2 pi constant) over the last epoch. */
int fbs_proposal_train(fbs_handle* h, int epochs, int batch, double lr, uint64_t seed,
                       double* final_loss);

/* Run n_sweeps sweeps in which every gene attempts the move, with the network's
 * proposal on even and the prior-centred proposal (centre theta, scale
 * diag(sigma), the same t family) on odd sweeps; then fix for every gene the
 * proposal with the higher acceptance rate if that rate reaches min_accept,
 * else only the slice updates, and set mode 1.  The prior-centred proposal suits
 * genes whose conditional is close to the prior (very large gamma_g), where the
 * network, trained mostly on typical genes, extrapolates poorly. */
int fbs_proposal_calibrate(fbs_handle* h, int64_t n_sweeps, int64_t burnin, double min_accept);

/* 0: plain slice updates for every gene; 1: the genes the calibration selected
 * make the learned move and then the slice updates of beta_g; 2: those genes make
 * the learned move instead of the slice updates.  The move keeps every log-rate
 * and the slice updates of beta_g keep eps, so mode 1 alternates between the two
 * parameterisations of the gene's log-rates. */
int fbs_proposal_mode(fbs_handle* h, int mode);

/* 1 (default): with 128-thread gamma/beta blocks (the FP32 default) that kernel
 * evaluates the network for its own 128 genes on the tensor cores before their
 * move; 0: a separate network kernel runs before it.  Both evaluate the same
 * tile code, so the chains are identical. */
int fbs_proposal_fused(fbs_handle* h, int on);

/* Bound of every wait of the tensor-core network pass (mbarrier polls; default
 * 2^24).  A wait that reaches it gives up: the block sets a flag, waits up to
 * 2^24 polls for its copies and matrix products still in flight, frees its tensor
 * memory, and its genes skip the network's move in that sweep; fbs_sync then
 * returns FBS_E_CUDA.  The training steps of fbs_proposal_train use the same
 * bound (a step that gives up is skipped and the call returns FBS_E_CUDA).  0
 * makes every pass give up at its first wait (which exercises that path).
 * FBS_E_ARG for FP64 handles and batch views. */
int fbs_proposal_wait_limit(fbs_handle* h, uint32_t polls);

/* Copy the FP32 parameters out (get != NULL) and/or in (set != NULL); n must equal
 * fbs_proposal_param_count(L). */
int fbs_proposal_params(fbs_handle* h, float* get, const float* set, int n);

/* The network's outputs for every gene at the current state (host [G][K]), as
 * the move reads them: mu (L), log of the Cholesky diagonal (L), sub-diagonal
 * entries in row order.  Synchronous. */
int fbs_proposal_outputs(fbs_handle* h, float* out);

/* One move at the current state, without the other updates of a sweep: the
 * genes the calibration selected with their proposals (all_genes = 0), or every
 * gene with the network's (1) or the prior-centred (2) proposal, propose and
 * accept or reject with the random numbers of iteration `it` (1 <= it < 2^32),
 * counting into fbs_proposal_stats.  The state keeps every log-rate.  Synchronous. */
int fbs_proposal_step(fbs_handle* h, int64_t it, int all_genes);

/* The proposal each gene uses (host [G]): 0 only the slice updates, 1 the
 * network's, 2 the prior-centred one (all 0 before a calibration). */
int fbs_proposal_kinds(fbs_handle* h, uint8_t* kinds);

/* Accepted and attempted moves since the calibration, the number of genes that
 * make the move and how many of them use the prior-centred proposal (each
 * output may be NULL). */
int fbs_proposal_stats(fbs_handle* h, int64_t* accepted, int64_t* tried, int* n_mh_genes,
                       int* n_prior_genes);

/* One forward and backward pass of the network on a host batch (features [B][F],
 * beta [B][L]) through the training kernels: *loss = mean negative
 * log-likelihood, grad = its gradient (host, fbs_proposal_param_count floats). */
int fbs_proposal_loss_grad(const float* params, int L, int B, const float* feat,
                           const float* beta, double* loss, float* grad);

/* ---- Batches: many datasets and chains in one launch -----------------------
 *
 * The conditionally independent updates of Algorithm 1 are independent across
 * datasets too, so C datasets of different N, G and L (and C chains, each with
 * its own seed and chain number) sweep together: one eps launch, one
 * gamma/beta launch and one hyperparameter launch (one block per dataset) per
 * iteration, replayed from a captured CUDA graph.  Batches run the FP32 form. */

typedef struct fbs_batch fbs_batch;

/* One dataset of a batch: y host [G][N] int32 gene-major; X host [N][L]; h host
 * [N]; priors; Philox seed and chain number.  Read during fbs_batch_init only. */
typedef struct {
  int N, G, L;
  const int32_t* y;
  const double* X;
  const double* h;
  fbs_priors priors;
  uint64_t seed;
  uint32_t chain;
} fbs_dataset;

/* Create a batch of C >= 1 datasets.  opt: precision must be FBS_F32; w0, K,
 * shrink_max, moments_eps, trace_cap and trace_beta apply to every dataset.
 * The library allocates the device memory.  Every dataset starts from the
 * default state of fbs_init.  Errors as fbs_init, naming the dataset. */
int fbs_batch_init(fbs_batch** out, int C, const fbs_dataset* sets, const fbs_options* opt,
                   void* stream);

/* fbs_run for every dataset of the batch at once (same n_iter, burnin, thin). */
int fbs_batch_run(fbs_batch* b, int64_t n_iter, int64_t burnin, int64_t thin);

/* Wait for the batch; FBS_E_NONFINITE if any dataset saw a non-finite start. */
int fbs_batch_sync(fbs_batch* b);

/* A handle viewing dataset c of the batch, owned by the batch: fbs_sync,
 * fbs_moments, fbs_get_state, fbs_set_state, fbs_trace, fbs_beta_ess,
 * fbs_count_sums and fbs_counters work on it; fbs_run and fbs_profile return
 * FBS_E_ARG; fbs_free ignores it.  NULL if c is out of range. */
fbs_handle* fbs_batch_chain(fbs_batch* b, int c);

/* Launch schedule: threads per block of the eps kernel (128 or 256) and of the
 * gamma/beta kernel (32, 64 or 128). */
int fbs_batch_set_schedule(fbs_batch* b, int eps_block, int gb_block);

/* Autotuner: times `sweeps` sweeps (direct launches, CUDA events) under every
 * schedule, keeps the fastest and returns it with its time per sweep.  The
 * trial sweeps are ordinary iterations of every chain, run with `burnin` as
 * M_B, so call it before fbs_batch_run with the burn-in that run will use. */
int fbs_batch_autotune(fbs_batch* b, int sweeps, int64_t burnin, int* eps_block, int* gb_block,
                       double* ms_per_sweep);

/* ---- Three-level model over a batch (Section 2.3, Figure 2) ---------------
 *
 * The batch's K = C datasets become the groups of a three-level model: dataset
 * k keeps its own hyperparameters phi_k = (nu_k, tau_k, theta_k, sigma^2_k), and
 * the phi_k share a top level psi = (b, m_1..m_L) through
 *   tau_k ~ Gamma(a_k, rate b),  theta_kl ~ N(m_l, c_kl^2),
 *   b ~ Gamma(a_b, rate b_b),    m_l ~ N(0, e_l^2)
 * (a_k, c_kl, and the other priors are dataset k's fbs_priors; its b is then
 * unused).  Every sweep runs the datasets' steps given psi, then draws psi
 * given the phi_k: b ~ Gamma(a_b + sum_k a_k, rate b_b + sum_k tau_k) and
 * m_l ~ N(w sum_k theta_kl / c_kl^2, w), w = 1/(sum_k 1/c_kl^2 + 1/e_l^2),
 * reductions over k in dataset order on one warp; Philox stream 10 with
 * key `seed`, chain word 0, index 0 for b and 1+l for m_l. */
typedef struct {
  double a_b, b_b;   /* b ~ Gamma(a_b, rate b_b); both finite and > 0 */
  const double* e;   /* [L] host, m_l ~ N(0, e_l^2); finite and > 0 */
  uint64_t seed;     /* Philox key of the psi draws */
} fbs_top_prior;

/* Switch the batch to the three-level model (pri != NULL) or back to K
 * independent datasets (pri == NULL).  psi0: host [1+L] = (b, m_1..m_L)
 * starting values, or NULL for (a_b / b_b, 0, .., 0).  Resets the psi moments
 * and trace; the psi trace keeps up to opt.trace_cap rows (same thinning as
 * the datasets' traces).  FBS_E_ARG if the datasets' L differ or a value is
 * out of range.  Synchronous. */
int fbs_batch_three_level(fbs_batch* b, const fbs_top_prior* pri, const double* psi0);

/* Top-level state to host: any pointer may be NULL.  psi, mean, msq [1+L]
 * (running mean and mean square over the post-burn-in iterations, count of
 * them in *count); trace [max_rows][1+L] (*rows copied); *gamma_caps = b draws
 * that ran out of attempts.  FBS_E_ARG if the batch is not three-level.
 * Synchronous. */
int fbs_batch_top_level(fbs_batch* b, double* psi, double* mean, double* msq, int64_t* count,
                        int64_t max_rows, double* trace, int64_t* rows, int64_t* gamma_caps);

void fbs_batch_free(fbs_batch* b);

/* ---- One sweep without any allocation ------------------------------------
 *
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory at the time they want to sweep: code that
 * runs while the host program forbids cudaMalloc (inside a region where the
 * allocator must not be called, or where all device memory has been handed to
 * another pool beforehand), or that already holds the chain's arrays in memory
 * it owns.  fbs_init needs device memory (its own or a caller workspace) and
 * creates a stream and events; fbs_sweep_noalloc needs neither.
 *
 * It runs iteration `it` of Algorithm 1 (the same kernels as fbs_run) on the
 * caller's device arrays, in the handle's device layout (genes fastest):
 *   y [N][G] int32, T [L][G] with T_lg = sum_n y_gn X_nl (inputs);
 *   eps, w_eps, waux_eps [N][G]; beta, w_beta, waux_beta [L][G]; gamma [G];
 *   hyp [2L+4] = (nu, tau, theta_1..L, sigma^2_1..L, w_nu, waux_nu)  (in/out);
 *   running moments m_* / q_* (mean / mean square): eps [N][G] (both may be
 *   NULL to skip), beta [L][G], gamma [G], phi [2L+2] -- updated, with n_mom
 *   draws already folded in, when it > burnin and otherwise untouched;
 *   n_mom may not exceed it - 1 - burnin (the post-burn-in iterations before
 *   this one), else FBS_E_ARG;
 *   status: NULL, or a device array of 1 + FBS_NUM_COUNTERS uint64 that
 *   receives this call's flags word (bit 0: a slice update started from a
 *   non-finite log density, which this call does not check for in the caller's
 *   state) and its FBS_CNT_* counters (FBS_CNT_SWEEPS = 1).
 * X, h and the priors are host arrays read during the call.  Slice widths are
 * tuned while it <= burnin (M_C = burnin/2).  No trace is written.
 *
 * Scratch: the per-block partial sums, the hyperparameter block and the
 * counters live in one file-scope static __device__ array of about 290 KiB
 * (FBS_NOALLOC_MAX_GENES / 128 blocks), which every GPU that loads the library
 * holds until the process exits.  G above FBS_NOALLOC_MAX_GENES returns
 * FBS_E_ARG.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current.  The address is kept for
 * the life of the process, so the entry point must not be used on a device
 * after cudaDeviceReset.  All calls share the array and every call rewrites what
 * it reads from it, so calls whose work overlaps on the GPU (different streams
 * at the same time) race; calls on one stream are ordered.  The call is
 * asynchronous on `stream` (NULL = legacy default stream): the outputs are
 * ready when the stream reaches them.  It calls no cudaMalloc, cudaFree or
 * other allocating routine.  Errors: FBS_E_ARG (sizes, NULL pointers, moment
 * arrays missing after burn-in, priors, X with too many distinct values),
 * FBS_E_CUDA. */
#define FBS_NOALLOC_MAX_GENES (2048 * 128)

typedef struct {
  int N, G, L;
  const double* X;      /* host [N][L] */
  const double* h;      /* host [N] */
  fbs_priors priors;    /* host */
  uint64_t seed;
  uint32_t chain;
  int step_out_max, shrink_max;
  int64_t it;           /* iteration to run, >= 1 */
  int64_t burnin;       /* M_B */
  int64_t n_mom;        /* draws already in the moments */
  const int32_t* y;
  const double* T;
  double *eps, *w_eps, *waux_eps;
  double *beta, *w_beta, *waux_beta;
  double* gam;
  double* hyp;
  double *m_eps, *q_eps, *m_beta, *q_beta, *m_gam, *q_gam, *m_phi, *q_phi;
  void* stream;
  uint64_t* status;     /* device [1 + FBS_NUM_COUNTERS] or NULL: see above */
} fbs_sweep_args;

int fbs_sweep_noalloc(const fbs_sweep_args* a);

/* Release the handle and any memory the library allocated for it. */
void fbs_free(fbs_handle* h);

/* Message describing the last error on the calling thread ("" if none). */
const char* fbs_last_error_string(void);

#ifdef __cplusplus
}
#endif
#endif /* FBS_H */
