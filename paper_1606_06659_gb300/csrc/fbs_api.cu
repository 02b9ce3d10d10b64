// fbs_api.cu -- the extern "C" entry points declared in include/fbs.h: input
// validation, device memory layout, CUDA-graph capture of sweep segments and
// the host side of every copy.  All sampling arithmetic is in fbs_kernels.cu.
#include <cuda_runtime.h>
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "fbs.h"
#include "fbs_common.cuh"
#include "fbs_kernels.h"

using namespace fbs;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define FBS_CUDA(call)                                                                    \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(e_ == cudaErrorMemoryAllocation ? FBS_E_OOM : FBS_E_CUDA,               \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                    \
  } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Byte offsets of every device buffer inside one workspace.
struct Layout {
  size_t y, T, eps, w_eps, waux_eps, m_eps, q_eps, mu, beta, w_beta, waux_beta, m_beta, q_beta;
  size_t gam, w_gam, waux_gam, m_gam, q_gam, partial, hyp, trace_phi, trace_beta, counters, pinv;
  size_t total;
};

Layout make_layout(int N, int G, int L, int nblk, long long trace_cap, int trace_beta) {
  Layout o;
  size_t at = 0;
  auto take = [&](size_t bytes) {
    size_t here = at;
    at = align256(at + bytes);
    return here;
  };
  const size_t NG = (size_t)N * G, LG = (size_t)L * G, P = 2 * (size_t)L + 2;
  o.y = take(NG * sizeof(int32_t));
  o.T = take(LG * 8);
  o.eps = take(NG * 8);
  o.w_eps = take(NG * 8);
  o.waux_eps = take(NG * 8);
  o.m_eps = take(NG * 8);
  o.q_eps = take(NG * 8);
  o.mu = take(NG * 8);
  o.beta = take(LG * 8);
  o.w_beta = take(LG * 8);
  o.waux_beta = take(LG * 8);
  o.m_beta = take(LG * 8);
  o.q_beta = take(LG * 8);
  o.gam = take((size_t)G * 8);
  o.w_gam = take((size_t)G * 8);
  o.waux_gam = take((size_t)G * 8);
  o.m_gam = take((size_t)G * 8);
  o.q_gam = take((size_t)G * 8);
  o.partial = take((size_t)nblk * kNumPart * 8);
  o.hyp = take(sizeof(Hyper));
  o.trace_phi = take((size_t)(trace_cap > 0 ? trace_cap : 1) * P * 8);
  o.trace_beta = trace_beta && trace_cap > 0 ? take((size_t)trace_cap * LG * 8) : 0;
  o.counters = take(kCounterCopies * FBS_NUM_COUNTERS * sizeof(unsigned long long));
  o.pinv = take((size_t)kMaxL * kMaxN * 8);
  o.total = at + 256;  // slack for aligning an unaligned base
  return o;
}

// FP32 form: per-gene state in FP32, four FP32 moment planes per parameter.
struct LayoutF32 {
  size_t y, T, eps, w_eps, waux_eps, mom_eps, mu, beta, w_beta, waux_beta, mom_beta, gam, mom_gam;
  size_t partial, hyp, trace_phi, trace_beta, counters, pinv, gsync, total;
};

LayoutF32 make_layout_f32(int N, int G, int L, int nblk, long long trace_cap, int trace_beta) {
  LayoutF32 o;
  size_t at = 0;
  auto take = [&](size_t bytes) {
    size_t here = at;
    at = align256(at + bytes);
    return here;
  };
  const size_t NG = (size_t)N * G, LG = (size_t)L * G, P = 2 * (size_t)L + 2;
  o.y = take(NG * sizeof(int32_t));
  o.T = take(LG * 8);
  o.eps = take(NG * 4);
  o.w_eps = take(NG * 4);
  o.waux_eps = take(NG * 4);
  o.mom_eps = take(4 * NG * 4);
  o.mu = take(NG * 4);
  o.beta = take(LG * 4);
  o.w_beta = take(LG * 4);
  o.waux_beta = take(LG * 4);
  o.mom_beta = take(4 * LG * 4);
  o.gam = take((size_t)G * 4);
  o.mom_gam = take(4 * (size_t)G * 4);
  o.partial = take((size_t)nblk * kNumPart * 8);
  o.hyp = take(sizeof(Hyper));
  o.trace_phi = take((size_t)(trace_cap > 0 ? trace_cap : 1) * P * 8);
  o.trace_beta = trace_beta && trace_cap > 0 ? take((size_t)trace_cap * LG * 8) : 0;
  o.counters = take(kEpsCounterCopiesHost * FBS_NUM_COUNTERS * sizeof(unsigned long long));
  o.pinv = take((size_t)kMaxL * kMaxN * 8);
  o.gsync = take(kPersistentSyncBytes);
  o.total = at + 256;
  return o;
}

// Threads per block of the gamma/beta kernel: FP64 work is bound by the FP64
// pipe, so small blocks spread it evenly over the SMs; the FP32 form is bound by
// latency and prefers more warps per block.
int block_of(const fbs_options* o) {
  if (o && o->block > 0) return o->block;
  return (o && o->precision == FBS_F32) ? 128 : 32;
}

}  // namespace

void fbs::set_last_error(const std::string& msg) { g_err = msg; }

// Learned beta_g proposal of one FP32 handle.
struct LearnedState {
  int L = 0, F = 0, K = 0, np = 0;
  float* params = nullptr;     // FP32 master parameters (flat)
  void* w_image = nullptr;     // inference weights: split BF16 operands + FP32 biases
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  long long adam_t = 0;
  float* prop = nullptr;       // [K][G] proposal outputs
  uint8_t* use_mh = nullptr;   // [G]
  unsigned* mh_acc = nullptr;  // [G]
  unsigned* mh_try = nullptr;  // [G]
  float* stats = nullptr;      // column means and scales of the pairs [2F + 2L]
  float* pair_feat = nullptr;  // [cap][F]
  float* pair_beta = nullptr;  // [cap][L]
  long long pair_cap = 0, pairs = 0;
  int mode = 0;                // 1: genes with use_mh take the learned move
  bool trained = false;
  bool fused = true;           // the gamma/beta kernel runs the network pass itself
};

struct fbs_handle {
  ModelConst mc;
  DevPtrs p;        // FP64 state; in the FP32 form only the shared fields are set
  DevPtrsF32 pf;    // FP32 state (FP32 form only)
  int prec = FBS_F64;
  fbs_options opt;
  Layout lay;
  LayoutF32 lay32;
  int block = kDefaultBlock, nblk = 0, seg = 100;
  bool x_integral = false;
  void* ws = nullptr;
  bool own_ws = false;
  cudaStream_t user = nullptr;  // caller's stream (ordering only)
  cudaStream_t s = nullptr;     // handle's own stream (all work, graph capture)
  cudaStream_t s2 = nullptr;    // hyperparameter branch of the FP32 graph
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaEvent_t ev_g = nullptr, ev_h = nullptr;  // gamma/beta done, hyperparameters done
  cudaGraphExec_t seg_exec = nullptr;
  long long trace_cap = 0;
  bool is_view = false;  // a dataset of a batch: state access only, owned by the batch
  LearnedState* learned = nullptr;
  Contrasts* con = nullptr;        // device propositions (null until set)
  unsigned* con_count = nullptr;   // device counts [FBS_MAX_CONTRASTS][G]
  int ncon = 0;
  long long con_nmom0 = 0;         // moment count when the propositions were set
};

namespace {

int enter(fbs_handle* h) {
  FBS_CUDA(cudaEventRecord(h->ev_in, h->user));
  FBS_CUDA(cudaStreamWaitEvent(h->s, h->ev_in, 0));
  return FBS_OK;
}

int leave(fbs_handle* h) {
  FBS_CUDA(cudaEventRecord(h->ev_out, h->s));
  FBS_CUDA(cudaStreamWaitEvent(h->user, h->ev_out, 0));
  return FBS_OK;
}

int check_opts(const fbs_options* o) {
  if (!o) return FBS_OK;
  if (o->precision != FBS_F64 && o->precision != FBS_F32)
    return fail(FBS_E_ARG, "precision must be FBS_F64 or FBS_F32");
  if (!(o->w0 > 0.0) || !isfinite(o->w0)) return fail(FBS_E_ARG, "w0 must be finite and > 0");
  if (o->step_out_max < 0 || o->step_out_max > (1 << 20))
    return fail(FBS_E_ARG, "step_out_max out of range");
  if (o->shrink_max < 0 || o->shrink_max > (1 << 20))
    return fail(FBS_E_ARG, "shrink_max out of range");
  if (o->trace_cap < 0) return fail(FBS_E_ARG, "trace_cap must be >= 0");
  if (o->block < 0 || o->block > 128 || (o->block % 32) != 0)
    return fail(FBS_E_ARG, "block must be 0 or a multiple of 32 up to 128");
  if (o->graph_segment < 0) return fail(FBS_E_ARG, "graph_segment must be >= 0");
  if (o->all_slice != 0 && o->all_slice != 1) return fail(FBS_E_ARG, "all_slice must be 0 or 1");
  if (o->all_slice && o->precision != FBS_F64)
    return fail(FBS_E_ARG, "all_slice runs in the FBS_F64 form");
  if (o->persistent != 0 && o->persistent != 1) return fail(FBS_E_ARG, "persistent must be 0 or 1");
  if (o->persistent && o->precision != FBS_F32)
    return fail(FBS_E_ARG, "the persistent sweep runs in the FBS_F32 form");
  return FBS_OK;
}

int check_sizes(int N, int G, int L) {
  if (N < 1 || N > FBS_MAX_N) return fail(FBS_E_ARG, "N must be in [1, FBS_MAX_N]");
  if (G < 2) return fail(FBS_E_ARG, "G must be >= 2");
  if (L < 1 || L > FBS_MAX_L) return fail(FBS_E_ARG, "L must be in [1, FBS_MAX_L]");
  return FBS_OK;
}

// (X^T X)^-1 X^T by Gauss-Jordan elimination with partial pivoting; false if singular.
bool pseudo_inverse(const double* X, int N, int L, double* pinv /* [kMaxL][kMaxN] */) {
  std::vector<double> A((size_t)L * 2 * L, 0.0);
  for (int i = 0; i < L; ++i) {
    for (int j = 0; j < L; ++j) {
      double s = 0.0;
      for (int n = 0; n < N; ++n) s += X[n * L + i] * X[n * L + j];
      A[i * 2 * L + j] = s;
    }
    A[i * 2 * L + L + i] = 1.0;
  }
  double scale = 0.0;
  for (int i = 0; i < L; ++i) scale = fmax(scale, fabs(A[i * 2 * L + i]));
  for (int col = 0; col < L; ++col) {
    int piv = col;
    for (int r = col + 1; r < L; ++r)
      if (fabs(A[r * 2 * L + col]) > fabs(A[piv * 2 * L + col])) piv = r;
    if (!(fabs(A[piv * 2 * L + col]) > 1e-10 * scale)) return false;
    if (piv != col)
      for (int j = 0; j < 2 * L; ++j) std::swap(A[col * 2 * L + j], A[piv * 2 * L + j]);
    const double pv = A[col * 2 * L + col];
    for (int j = 0; j < 2 * L; ++j) A[col * 2 * L + j] /= pv;
    for (int r = 0; r < L; ++r) {
      if (r == col) continue;
      const double f = A[r * 2 * L + col];
      for (int j = 0; j < 2 * L; ++j) A[r * 2 * L + j] -= f * A[col * 2 * L + j];
    }
  }
  for (int i = 0; i < kMaxL * kMaxN; ++i) pinv[i] = 0.0;
  for (int l = 0; l < L; ++l)
    for (int n = 0; n < N; ++n) {
      double s = 0.0;
      for (int k = 0; k < L; ++k) s += A[l * 2 * L + L + k] * X[n * L + k];
      pinv[l * kMaxN + n] = s;
    }
  return true;
}

DevPtrs carve(char* base, const Layout& o, int trace_beta) {
  DevPtrs p;
  memset(&p, 0, sizeof(p));  // no contrasts until they are set
  p.y = (const int32_t*)(base + o.y);
  p.T = (const double*)(base + o.T);
  p.eps = (double*)(base + o.eps);
  p.w_eps = (double*)(base + o.w_eps);
  p.waux_eps = (double*)(base + o.waux_eps);
  p.m_eps = (double*)(base + o.m_eps);
  p.q_eps = (double*)(base + o.q_eps);
  p.mu = (double*)(base + o.mu);
  p.beta = (double*)(base + o.beta);
  p.w_beta = (double*)(base + o.w_beta);
  p.waux_beta = (double*)(base + o.waux_beta);
  p.m_beta = (double*)(base + o.m_beta);
  p.q_beta = (double*)(base + o.q_beta);
  p.gam = (double*)(base + o.gam);
  p.w_gam = (double*)(base + o.w_gam);
  p.waux_gam = (double*)(base + o.waux_gam);
  p.m_gam = (double*)(base + o.m_gam);
  p.q_gam = (double*)(base + o.q_gam);
  p.partial = (double*)(base + o.partial);
  p.hyp = (Hyper*)(base + o.hyp);
  p.trace_phi = (double*)(base + o.trace_phi);
  p.trace_beta = trace_beta ? (double*)(base + o.trace_beta) : nullptr;
  p.counters = (unsigned long long*)(base + o.counters);
  return p;
}

DevPtrsF32 carve_f32_ptrs(char* base, const LayoutF32& o32, int trace_beta) {
  DevPtrsF32 f;
  memset(&f, 0, sizeof(f));  // no learned proposal until one is set up
  f.tc_polls = kTcWaitPolls;
  f.y = (const int32_t*)(base + o32.y);
  f.T = (const double*)(base + o32.T);
  f.eps = (float*)(base + o32.eps);
  f.w_eps = (float*)(base + o32.w_eps);
  f.waux_eps = (float*)(base + o32.waux_eps);
  f.mom_eps = (float*)(base + o32.mom_eps);
  f.mu = (float*)(base + o32.mu);
  f.beta = (float*)(base + o32.beta);
  f.w_beta = (float*)(base + o32.w_beta);
  f.waux_beta = (float*)(base + o32.waux_beta);
  f.mom_beta = (float*)(base + o32.mom_beta);
  f.gam = (float*)(base + o32.gam);
  f.mom_gam = (float*)(base + o32.mom_gam);
  f.partial = (double*)(base + o32.partial);
  f.hyp = (Hyper*)(base + o32.hyp);
  f.trace_phi = (double*)(base + o32.trace_phi);
  f.trace_beta = trace_beta ? (double*)(base + o32.trace_beta) : nullptr;
  f.counters = (unsigned long long*)(base + o32.counters);
  return f;
}

// FP32 pointers of one chain, and the FP64-struct fields the shared kernels and
// copies use (everything else null).
void carve_f32(char* base, const LayoutF32& o32, int trace_beta, DevPtrsF32& f, DevPtrs& p) {
  f = carve_f32_ptrs(base, o32, trace_beta);
  memset(&p, 0, sizeof(p));
  p.y = f.y;
  p.T = f.T;
  p.partial = f.partial;
  p.hyp = f.hyp;
  p.trace_phi = f.trace_phi;
  p.trace_beta = f.trace_beta;
  p.counters = f.counters;
}

// Copy a device [R][G] plane set (double or float) to a host [G][R] double array.
template <class T>
int to_host_gene_major(fbs_handle* h, const T* dev, int R, double* host) {
  const int G = h->mc.G;
  std::vector<T> tmp((size_t)R * G);
  FBS_CUDA(cudaMemcpyAsync(tmp.data(), dev, tmp.size() * sizeof(T), cudaMemcpyDeviceToHost, h->s));
  FBS_CUDA(cudaStreamSynchronize(h->s));
  for (int r = 0; r < R; ++r)
    for (int g = 0; g < G; ++g) host[(size_t)g * R + r] = (double)tmp[(size_t)r * G + g];
  return FBS_OK;
}

template <class T>
int from_host_gene_major(fbs_handle* h, T* dev, int R, const double* host) {
  const int G = h->mc.G;
  std::vector<T> tmp((size_t)R * G);
  for (int r = 0; r < R; ++r)
    for (int g = 0; g < G; ++g) tmp[(size_t)r * G + g] = (T)host[(size_t)g * R + r];
  FBS_CUDA(cudaMemcpyAsync(dev, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice, h->s));
  FBS_CUDA(cudaStreamSynchronize(h->s));
  return FBS_OK;
}

// A Kahan-compensated FP32 moment: planes value m and compensation c of
// [R][G] each, starting at `base + plane_offset`; the moment is m - c.
int kahan_to_host(fbs_handle* h, const float* base, int R, double* host) {
  const int G = h->mc.G;
  const size_t n = (size_t)R * G;
  std::vector<float> tmp(2 * n);
  FBS_CUDA(cudaMemcpyAsync(tmp.data(), base, 2 * n * 4, cudaMemcpyDeviceToHost, h->s));
  FBS_CUDA(cudaStreamSynchronize(h->s));
  for (int r = 0; r < R; ++r)
    for (int g = 0; g < G; ++g)
      host[(size_t)g * R + r] =
          (double)tmp[(size_t)r * G + g] - (double)tmp[n + (size_t)r * G + g];
  return FBS_OK;
}

int read_hyper(fbs_handle* h, Hyper* out) {
  FBS_CUDA(cudaMemcpyAsync(out, h->p.hyp, sizeof(Hyper), cudaMemcpyDeviceToHost, h->s));
  FBS_CUDA(cudaStreamSynchronize(h->s));
  return FBS_OK;
}

// The FP32 gamma/beta step of sweep i.  With the learned proposal and 128-thread
// blocks the kernel evaluates the network itself (tensor cores, its own 128
// genes); with other block sizes the stand-alone network pass runs first.
cudaError_t gb_f32_step(fbs_handle* h, int i, cudaStream_t s) {
  if (h->pf.prop == nullptr) return launch_gb_f32(h->mc, h->pf, h->block, i, s);
  if (h->block == 128 && h->learned->fused)
    return launch_gb_f32(h->mc, h->pf, 128, i, s, h->learned->w_image);
  cudaError_t e = launch_proposal_f32(h->mc, h->pf, h->learned->w_image, h->learned->prop, s);
  return e != cudaSuccess ? e : launch_gb_f32(h->mc, h->pf, h->block, i, s);
}

// n_iter sweeps launched one kernel at a time on the handle's stream.
int sweeps_direct(fbs_handle* h, int64_t n_iter) {
  if (h->prec == FBS_F32) {
    FBS_CUDA(launch_seg_begin(h->p.hyp, h->s));
    for (int64_t i = 0; i < n_iter; ++i) {
      FBS_CUDA(launch_eps_f32(h->mc, h->pf, (int)i, h->s));
      FBS_CUDA(gb_f32_step(h, (int)i, h->s));
      FBS_CUDA(launch_hyper(h->mc, h->p, h->nblk, h->s));
    }
    return FBS_OK;
  }
  FBS_CUDA(launch_seg_begin(h->p.hyp, h->s));
  for (int64_t i = 0; i < n_iter; ++i) {
    FBS_CUDA(launch_eps_f64(h->mc, h->p, (int)i, h->s));
    FBS_CUDA(launch_gb_f64(h->mc, h->p, h->block, (int)i, h->s));
    FBS_CUDA(launch_hyper(h->mc, h->p, h->nblk, h->s));
  }
  return FBS_OK;
}

// Enqueue one graph segment's work on the capturing stream.  In the FP32 form
// the hyperparameter kernel of sweep i runs on a second stream, concurrently
// with the eps kernel of sweep i+1 (whose conditionals involve no
// hyperparameter); the gamma/beta kernel of sweep i+1 waits for both.
cudaError_t capture_sweeps(fbs_handle* h, int n) {
  cudaError_t e = cudaSuccess;
  const bool f32 = h->prec == FBS_F32;
  if ((e = launch_seg_begin(h->p.hyp, h->s)) != cudaSuccess) return e;
  for (int i = 0; i < n; ++i) {
    e = f32 ? launch_eps_f32(h->mc, h->pf, i, h->s) : launch_eps_f64(h->mc, h->p, i, h->s);
    if (e != cudaSuccess) return e;
    if (i > 0 && (e = cudaStreamWaitEvent(h->s, h->ev_h, 0)) != cudaSuccess) return e;
    e = f32 ? gb_f32_step(h, i, h->s) : launch_gb_f64(h->mc, h->p, h->block, i, h->s);
    if (e != cudaSuccess) return e;
    if ((e = cudaEventRecord(h->ev_g, h->s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(h->s2, h->ev_g, 0)) != cudaSuccess) return e;
    if ((e = launch_hyper(h->mc, h->p, h->nblk, h->s2)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(h->ev_h, h->s2)) != cudaSuccess) return e;
  }
  return cudaStreamWaitEvent(h->s, h->ev_h, 0);
}

cudaError_t capture_segment(fbs_handle* h) { return capture_sweeps(h, h->seg); }

int ensure_graph(fbs_handle* h) {
  if (h->seg_exec) return FBS_OK;
  cudaGraph_t graph;
  FBS_CUDA(cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal));
  cudaError_t ce = capture_segment(h);
  if (ce != cudaSuccess) {
    graph = nullptr;
    cudaStreamEndCapture(h->s, &graph);
    if (graph) cudaGraphDestroy(graph);
    return fail(FBS_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
  }
  FBS_CUDA(cudaStreamEndCapture(h->s, &graph));
  cudaError_t e = cudaGraphInstantiate(&h->seg_exec, graph, 0);
  cudaGraphDestroy(graph);
  FBS_CUDA(e);
  return FBS_OK;
}

}  // namespace

namespace {

// Validates one dataset and builds its model constants and (X^T X)^-1 X^T.
int build_model(const int32_t* y, int N, int G, const double* X, int L, const double* hoff,
                const fbs_priors* pri, const fbs_options* o, uint64_t seed, uint32_t chain,
                ModelConst& mc, double* pinv, bool* integral_out) {
  int rc = check_sizes(N, G, L);
  if (rc) return rc;
  rc = check_opts(o);
  if (rc) return rc;
  if (!y || !X || !hoff || !pri || !pri->c || !pri->s)
    return fail(FBS_E_ARG, "y, X, h, priors, priors->c and priors->s must be non-NULL");
  auto pos = [](double v) { return isfinite(v) && v > 0.0; };
  if (!pos(pri->a) || !pos(pri->b) || !pos(pri->d))
    return fail(FBS_E_ARG, "prior constants a, b, d must be finite and > 0");
  for (int l = 0; l < L; ++l)
    if (!pos(pri->c[l]) || !pos(pri->s[l]))
      return fail(FBS_E_ARG, "prior constants c_l, s_l must be finite and > 0");
  for (int i = 0; i < N * L; ++i)
    if (!isfinite(X[i])) return fail(FBS_E_ARG, "X has a non-finite entry");
  for (int n = 0; n < N; ++n)
    if (!isfinite(hoff[n])) return fail(FBS_E_ARG, "h has a non-finite entry");
  for (size_t i = 0; i < (size_t)N * G; ++i)
    if (y[i] < 0) return fail(FBS_E_ARG, "y has a negative count");

  memset(&mc, 0, sizeof(mc));
  mc.N = N;
  mc.G = G;
  mc.L = L;
  mc.P = 2 * L + 2;
  mc.K = o->step_out_max;
  mc.shrink_max = o->shrink_max;
  mc.moments_eps = o->moments_eps ? 1 : 0;
  mc.trace_beta = (o->trace_beta && o->trace_cap > 0) ? 1 : 0;
  mc.seed_lo = (uint32_t)(seed & 0xffffffffu);
  mc.seed_hi = (uint32_t)(seed >> 32);
  mc.chain = chain;
  mc.all_slice = o->all_slice;
  mc.a = pri->a;
  mc.b = pri->b;
  mc.d = pri->d;
  for (int l = 0; l < L; ++l) {
    mc.c2[l] = pri->c[l] * pri->c[l];
    mc.s2[l] = pri->s[l] * pri->s[l];
    mc.s[l] = pri->s[l];
  }
  bool integral = true;
  for (int n = 0; n < N; ++n) {
    mc.h[n] = hoff[n];
    for (int l = 0; l < L; ++l) {
      mc.X[n * kMaxL + l] = X[n * L + l];
      if (X[n * L + l] != floor(X[n * L + l])) integral = false;
    }
  }
  *integral_out = integral;
  for (int n = 0; n < N; ++n) {
    mc.hf[n] = (float)mc.h[n];
    for (int l = 0; l < L; ++l) mc.Xf[n * kMaxL + l] = (float)mc.X[n * kMaxL + l];
  }
  for (int l = 0; l < L; ++l) {
    int nc = 0;
    for (int n = 0; n < N; ++n) {
      const double v = X[n * L + l];
      if (v == 0.0) {
        mc.cls[l][n] = -1;
        continue;
      }
      int j = 0;
      while (j < nc && mc.cval[l][j] != v) ++j;
      if (j == nc) {
        if (nc == kMaxCls)
          return fail(FBS_E_ARG, "a column of X has more than FBS_MAX_CLASSES distinct values");
        mc.cval[l][nc] = v;
        mc.cvalf[l][nc] = (float)v;
        mc.ckind[l][nc] = v == 1.0 ? kClsPlus : (v == -1.0 ? kClsMinus : kClsOther);
        ++nc;
      }
      mc.cls[l][n] = (int8_t)j;
    }
    mc.ncls[l] = nc;
  }
  // distinct rows of X, for the FP32 beta columns' per-pattern rate sums
  {
    int rep[kMaxPat];
    mc.npat = 0;
    for (int n = 0; n < N && mc.npat <= kMaxPat; ++n) {
      int r = 0;
      while (r < mc.npat && memcmp(&X[n * L], &X[rep[r] * L], sizeof(double) * L) != 0) ++r;
      if (r == mc.npat) {
        if (mc.npat == kMaxPat) {
          mc.npat = kMaxPat + 1;
          break;
        }
        rep[mc.npat++] = n;
      }
      mc.pat[n] = (int8_t)r;
    }
    for (int l = 0; l < kMaxL; ++l)
      for (int r = 0; r < kMaxPat; ++r)
        mc.pcls[l][r] = (l < L && r < mc.npat && mc.npat <= kMaxPat) ? mc.cls[l][rep[r]] : -1;
  }
  if (!pseudo_inverse(X, N, L, pinv)) return fail(FBS_E_ARG, "X^T X is singular");
  return FBS_OK;

}

}  // namespace

extern "C" {

void fbs_default_options(fbs_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->precision = FBS_F64;
  o->w0 = 1.0;
  o->step_out_max = 100;
  o->shrink_max = 100;
  o->chain = 0;
  o->moments_eps = 1;
  o->trace_cap = 0;
  o->trace_beta = 0;
  o->block = 0;
  o->graph_segment = 0;
}

int fbs_workspace_bytes(int N, int G, int L, const fbs_options* opt, size_t* bytes) {
  fbs_options d;
  fbs_default_options(&d);
  const fbs_options* o = opt ? opt : &d;
  int rc = check_sizes(N, G, L);
  if (rc) return rc;
  rc = check_opts(o);
  if (rc) return rc;
  if (!bytes) return fail(FBS_E_ARG, "bytes is NULL");
  const int block = block_of(o);
  const int nblk = (G + block - 1) / block;
  *bytes = o->precision == FBS_F32
               ? make_layout_f32(N, G, L, nblk, o->trace_cap, o->trace_beta).total
               : make_layout(N, G, L, nblk, o->trace_cap, o->trace_beta).total;
  return FBS_OK;
}

int fbs_init(fbs_handle** out, const int32_t* y, int N, int G, int gene_major, const double* X,
             int L, const double* hoff, const fbs_priors* pri, const fbs_options* opt,
             uint64_t seed, void* workspace, size_t workspace_bytes, void* stream) {
  g_err.clear();
  if (!out) return fail(FBS_E_ARG, "out is NULL");
  *out = nullptr;
  fbs_options d;
  fbs_default_options(&d);
  const fbs_options* o = opt ? opt : &d;
  ModelConst mc0;
  double pinv[kMaxL * kMaxN];
  bool integral = false;
  int rc = build_model(y, N, G, X, L, hoff, pri, o, seed, o->chain, mc0, pinv, &integral);
  if (rc) return rc;
  fbs_handle* h = new fbs_handle();
  h->mc = mc0;
  ModelConst& mc = h->mc;
  h->x_integral = integral;

  h->opt = *o;
  h->block = block_of(o);
  h->nblk = (G + h->block - 1) / h->block;
  h->seg = o->graph_segment > 0 ? o->graph_segment : 100;
  h->trace_cap = o->trace_cap;
  h->prec = o->precision;
  h->lay = make_layout(N, G, L, h->nblk, o->trace_cap, mc.trace_beta);
  h->lay32 = make_layout_f32(N, G, L, h->nblk, o->trace_cap, mc.trace_beta);
  const size_t need = h->prec == FBS_F32 ? h->lay32.total : h->lay.total;
  h->user = (cudaStream_t)stream;

  auto bail = [&](int code, const std::string& msg) {
    if (h->s) cudaStreamDestroy(h->s);
    if (h->s2) cudaStreamDestroy(h->s2);
    if (h->ev_g) cudaEventDestroy(h->ev_g);
    if (h->ev_h) cudaEventDestroy(h->ev_h);
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    if (h->own_ws && h->ws) cudaFree(h->ws);
    delete h;
    return fail(code, msg);
  };
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&h->s2, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&h->ev_g, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&h->ev_h, cudaEventDisableTiming)) != cudaSuccess)
    return bail(FBS_E_CUDA, std::string("stream/event creation: ") + cudaGetErrorString(e));
  if (workspace) {
    if (workspace_bytes < need) return bail(FBS_E_ARG, "workspace is too small");
    h->ws = workspace;
  } else {
    e = cudaMalloc(&h->ws, need);
    if (e != cudaSuccess) return bail(FBS_E_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    h->own_ws = true;
  }
  char* base = (char*)(((uintptr_t)h->ws + 255) & ~(uintptr_t)255);
  int32_t* y_raw = nullptr;  // raw counts, in a moment plane that is zeroed afterwards
  double* d_pinv = nullptr;
  if (h->prec == FBS_F32) {
    carve_f32(base, h->lay32, mc.trace_beta, h->pf, h->p);
    DevPtrsF32& f = h->pf;
    const LayoutF32& o32 = h->lay32;
    y_raw = (int32_t*)f.mom_eps;
    d_pinv = (double*)(base + o32.pinv);
    if ((e = prepare_gene_kernel_f32(N, h->block)) != cudaSuccess)
      return bail(FBS_E_CUDA, std::string("kernel attribute: ") + cudaGetErrorString(e));
  } else {
    h->p = carve(base, h->lay, mc.trace_beta);
    y_raw = (int32_t*)h->p.q_eps;
    d_pinv = (double*)(base + h->lay.pinv);
    if ((e = prepare_gene_kernel(N, h->block)) != cudaSuccess)
      return bail(FBS_E_CUDA, std::string("kernel attribute: ") + cudaGetErrorString(e));
  }

  if (enter(h) != FBS_OK) return bail(FBS_E_CUDA, g_err);
  if ((e = cudaMemcpyAsync(y_raw, y, (size_t)N * G * sizeof(int32_t), cudaMemcpyHostToDevice,
                           h->s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_pinv, pinv, sizeof(pinv), cudaMemcpyHostToDevice, h->s)) !=
          cudaSuccess ||
      (e = cudaMemsetAsync(h->p.counters, 0,
                           kCounterCopies * FBS_NUM_COUNTERS *
                               sizeof(unsigned long long),
                           h->s)) != cudaSuccess ||
      (e = cudaMemsetAsync(h->p.hyp, 0, sizeof(Hyper), h->s)) != cudaSuccess)
    return bail(FBS_E_CUDA, std::string("initialisation: ") + cudaGetErrorString(e));
  if (h->prec == FBS_F32) {
    if ((e = launch_init_run(h->p.hyp, o->trace_cap, h->s)) != cudaSuccess ||
        (e = launch_init_f32(mc, h->pf, y_raw, gene_major, d_pinv, o->w0, 1, h->s)) !=
            cudaSuccess ||
        (e = launch_init_hyper(mc, h->p.hyp, nullptr, h->pf.beta, o->w0, 1, h->s)) !=
            cudaSuccess)
      return bail(FBS_E_CUDA, std::string("initialisation: ") + cudaGetErrorString(e));
  } else {
    if ((e = launch_init(mc, h->p, y_raw, gene_major, d_pinv, o->w0, 1, o->trace_cap, h->s)) !=
        cudaSuccess)
      return bail(FBS_E_CUDA, std::string("initialisation: ") + cudaGetErrorString(e));
  }
  if ((e = cudaStreamSynchronize(h->s)) != cudaSuccess)
    return bail(FBS_E_CUDA, std::string("initialisation: ") + cudaGetErrorString(e));
  if (leave(h) != FBS_OK) return bail(FBS_E_CUDA, g_err);
  *out = h;
  return FBS_OK;
}

namespace {

// The handle's counters summed over their copies (synchronous).
int sum_counters(fbs_handle* h, int64_t* out) {
  const int copies = kCounterCopies;
  std::vector<unsigned long long> c((size_t)copies * FBS_NUM_COUNTERS);
  FBS_CUDA(cudaMemcpyAsync(c.data(), h->p.counters, c.size() * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, h->s));
  FBS_CUDA(cudaStreamSynchronize(h->s));
  for (int i = 0; i < FBS_NUM_COUNTERS; ++i) {
    unsigned long long t = 0;
    for (int k = 0; k < copies; ++k) t += c[(size_t)k * FBS_NUM_COUNTERS + i];
    out[i] = (int64_t)t;
  }
  return FBS_OK;
}

// FBS_E_SLICE_CAP once any slice update of the handle has used up its shrinkage
// proposals (Algorithm 2 has no bound; the update kept its value).
int slice_cap_status(fbs_handle* h) {
  int64_t c[FBS_NUM_COUNTERS];
  int rc = sum_counters(h, c);
  if (rc) return rc;
  if (c[FBS_CNT_SLICE_CAPS] > 0)
    return fail(FBS_E_SLICE_CAP, std::to_string(c[FBS_CNT_SLICE_CAPS]) +
                                     " slice update(s) ran out of shrinkage proposals and kept "
                                     "their value");
  return FBS_OK;
}

}  // namespace

int fbs_run(fbs_handle* h, int64_t n_iter, int64_t burnin, int64_t thin) {
  if (!h) return fail(FBS_E_ARG, "handle is NULL");
  if (h->is_view) return fail(FBS_E_ARG, "a batch dataset runs with fbs_batch_run");
  if (n_iter < 0 || burnin < 0 || thin < 1)
    return fail(FBS_E_ARG, "need n_iter >= 0, burnin >= 0, thin >= 1");
  if (n_iter == 0) return FBS_OK;
  int rc = enter(h);
  if (rc) return rc;
  FBS_CUDA(launch_set_run(h->p.hyp, burnin, burnin / 2, thin, h->s));
  int64_t left = n_iter;
  if (h->opt.persistent && h->pf.prop == nullptr) {
    // one cooperative launch per segment (the learned move takes the graph path)
    void* gsync = (char*)(((uintptr_t)h->ws + 255) & ~(uintptr_t)255) + h->lay32.gsync;
    while (left > 0) {
      const int n = (int)(left < h->seg ? left : h->seg);
      FBS_CUDA(launch_seg_begin(h->p.hyp, h->s));
      FBS_CUDA(launch_sweeps_f32(h->mc, h->pf, h->p, n, gsync, h->s, nullptr));
      left -= n;
    }
    return leave(h);
  }
  if (left >= h->seg) {
    rc = ensure_graph(h);
    if (rc) return rc;
    while (left >= h->seg) {
      FBS_CUDA(cudaGraphLaunch(h->seg_exec, h->s));
      left -= h->seg;
    }
  }
  if (left > 0) {
    rc = sweeps_direct(h, left);
    if (rc) return rc;
  }
  return leave(h);
}

int fbs_sync(fbs_handle* h) {
  if (!h) return fail(FBS_E_ARG, "handle is NULL");
  FBS_CUDA(cudaStreamSynchronize(h->s));
  FBS_CUDA(cudaGetLastError());
  Hyper hy;
  int rc = read_hyper(h, &hy);
  if (rc) return rc;
  if (hy.flags & kFlagTimeout)
    return fail(FBS_E_CUDA, "a bounded wait gave up (a tensor-core wait of the proposal network "
                            "or a grid barrier of the persistent sweep)");
  if (hy.flags & kFlagNonfinite)
    return fail(FBS_E_NONFINITE, "a slice update started from a non-finite log density");
  return slice_cap_status(h);
}

int fbs_moments(fbs_handle* h, double* mean_eps, double* msq_eps, double* mean_beta,
                double* msq_beta, double* mean_gam, double* msq_gam, double* mean_phi,
                double* msq_phi, int64_t* count) {
  if (!h) return fail(FBS_E_ARG, "handle is NULL");
  int rc = enter(h);
  if (rc) return rc;
  const int N = h->mc.N, L = h->mc.L, G = h->mc.G, P = h->mc.P;
  if (h->prec == FBS_F32) {
    const size_t NG = (size_t)N * G, LG = (size_t)L * G;
    const DevPtrsF32& f = h->pf;
    if (mean_eps && (rc = kahan_to_host(h, f.mom_eps, N, mean_eps))) return rc;
    if (msq_eps && (rc = kahan_to_host(h, f.mom_eps + 2 * NG, N, msq_eps))) return rc;
    if (mean_beta && (rc = kahan_to_host(h, f.mom_beta, L, mean_beta))) return rc;
    if (msq_beta && (rc = kahan_to_host(h, f.mom_beta + 2 * LG, L, msq_beta))) return rc;
    if (mean_gam && (rc = kahan_to_host(h, f.mom_gam, 1, mean_gam))) return rc;
    if (msq_gam && (rc = kahan_to_host(h, f.mom_gam + 2 * (size_t)G, 1, msq_gam))) return rc;
  } else {
    if (mean_eps && (rc = to_host_gene_major(h, h->p.m_eps, N, mean_eps))) return rc;
    if (msq_eps && (rc = to_host_gene_major(h, h->p.q_eps, N, msq_eps))) return rc;
    if (mean_beta && (rc = to_host_gene_major(h, h->p.m_beta, L, mean_beta))) return rc;
    if (msq_beta && (rc = to_host_gene_major(h, h->p.q_beta, L, msq_beta))) return rc;
    if (mean_gam) FBS_CUDA(cudaMemcpyAsync(mean_gam, h->p.m_gam, (size_t)G * 8, cudaMemcpyDeviceToHost, h->s));
    if (msq_gam) FBS_CUDA(cudaMemcpyAsync(msq_gam, h->p.q_gam, (size_t)G * 8, cudaMemcpyDeviceToHost, h->s));
  }
  Hyper hy;
  if ((rc = read_hyper(h, &hy))) return rc;
  if (mean_phi) memcpy(mean_phi, hy.m_phi, (size_t)P * 8);
  if (msq_phi) memcpy(msq_phi, hy.q_phi, (size_t)P * 8);
  if (count) *count = hy.n_mom;
  return leave(h);
}

int fbs_get_state(fbs_handle* h, double* eps, double* beta, double* gam, double* phi,
                  double* w_eps, double* waux_eps, double* w_beta, double* waux_beta,
                  double* w_nu, double* waux_nu, int64_t* it) {
  if (!h) return fail(FBS_E_ARG, "handle is NULL");
  int rc = enter(h);
  if (rc) return rc;
  const int N = h->mc.N, L = h->mc.L, G = h->mc.G, P = h->mc.P;
  if (h->prec == FBS_F32) {
    const DevPtrsF32& f = h->pf;
    if (eps && (rc = to_host_gene_major(h, (const float*)f.eps, N, eps))) return rc;
    if (w_eps && (rc = to_host_gene_major(h, (const float*)f.w_eps, N, w_eps))) return rc;
    if (waux_eps && (rc = to_host_gene_major(h, (const float*)f.waux_eps, N, waux_eps))) return rc;
    if (beta && (rc = to_host_gene_major(h, (const float*)f.beta, L, beta))) return rc;
    if (w_beta && (rc = to_host_gene_major(h, (const float*)f.w_beta, L, w_beta))) return rc;
    if (waux_beta && (rc = to_host_gene_major(h, (const float*)f.waux_beta, L, waux_beta))) return rc;
    if (gam && (rc = to_host_gene_major(h, (const float*)f.gam, 1, gam))) return rc;
  } else {
    if (eps && (rc = to_host_gene_major(h, (const double*)h->p.eps, N, eps))) return rc;
    if (w_eps && (rc = to_host_gene_major(h, (const double*)h->p.w_eps, N, w_eps))) return rc;
    if (waux_eps && (rc = to_host_gene_major(h, (const double*)h->p.waux_eps, N, waux_eps))) return rc;
    if (beta && (rc = to_host_gene_major(h, (const double*)h->p.beta, L, beta))) return rc;
    if (w_beta && (rc = to_host_gene_major(h, (const double*)h->p.w_beta, L, w_beta))) return rc;
    if (waux_beta && (rc = to_host_gene_major(h, (const double*)h->p.waux_beta, L, waux_beta))) return rc;
    if (gam) FBS_CUDA(cudaMemcpyAsync(gam, h->p.gam, (size_t)G * 8, cudaMemcpyDeviceToHost, h->s));
  }
  Hyper hy;
  if ((rc = read_hyper(h, &hy))) return rc;
  if (phi) memcpy(phi, hy.phi, (size_t)P * 8);
  if (w_nu) *w_nu = hy.w_nu;
  if (waux_nu) *waux_nu = hy.waux_nu;
  if (it) *it = hy.it;
  return leave(h);
}

int fbs_set_state(fbs_handle* h, const double* eps, const double* beta, const double* gam,
                  const double* phi, const double* w_eps, const double* waux_eps,
                  const double* w_beta, const double* waux_beta, const double* w_nu,
                  const double* waux_nu, int64_t it) {
  if (!h) return fail(FBS_E_ARG, "handle is NULL");
  if (it < 0) return fail(FBS_E_ARG, "it must be >= 0");
  int rc = enter(h);
  if (rc) return rc;
  const int N = h->mc.N, L = h->mc.L, G = h->mc.G, P = h->mc.P;
  (void)G;
  if (h->prec == FBS_F32) {
    const DevPtrsF32& f = h->pf;
    if (eps && (rc = from_host_gene_major(h, f.eps, N, eps))) return rc;
    if (w_eps && (rc = from_host_gene_major(h, f.w_eps, N, w_eps))) return rc;
    if (waux_eps && (rc = from_host_gene_major(h, f.waux_eps, N, waux_eps))) return rc;
    if (beta && (rc = from_host_gene_major(h, f.beta, L, beta))) return rc;
    if (w_beta && (rc = from_host_gene_major(h, f.w_beta, L, w_beta))) return rc;
    if (waux_beta && (rc = from_host_gene_major(h, f.waux_beta, L, waux_beta))) return rc;
    if (gam && (rc = from_host_gene_major(h, f.gam, 1, gam))) return rc;
    FBS_CUDA(launch_zero_moments_f32(h->mc, h->pf, h->s));
    FBS_CUDA(launch_init_hyper(h->mc, h->p.hyp, nullptr, f.beta, 0.0, 0, h->s));
  } else {
    if (eps && (rc = from_host_gene_major(h, h->p.eps, N, eps))) return rc;
    if (w_eps && (rc = from_host_gene_major(h, h->p.w_eps, N, w_eps))) return rc;
    if (waux_eps && (rc = from_host_gene_major(h, h->p.waux_eps, N, waux_eps))) return rc;
    if (beta && (rc = from_host_gene_major(h, h->p.beta, L, beta))) return rc;
    if (w_beta && (rc = from_host_gene_major(h, h->p.w_beta, L, w_beta))) return rc;
    if (waux_beta && (rc = from_host_gene_major(h, h->p.waux_beta, L, waux_beta))) return rc;
    if (gam && (rc = from_host_gene_major(h, h->p.gam, 1, gam))) return rc;
    FBS_CUDA(launch_zero_moments(h->mc, h->p, h->s));
  }
  Hyper hy;
  if ((rc = read_hyper(h, &hy))) return rc;
  if (phi) memcpy(hy.phi, phi, (size_t)P * 8);
  if (w_nu) hy.w_nu = *w_nu;
  if (waux_nu) hy.waux_nu = *waux_nu;
  hy.it = it;
  FBS_CUDA(cudaMemcpyAsync(h->p.hyp, &hy, sizeof(Hyper), cudaMemcpyHostToDevice, h->s));
  FBS_CUDA(cudaStreamSynchronize(h->s));
  return leave(h);
}

int fbs_get_slice_widths(fbs_handle* h, double* w_gam, double* waux_gam, double* w_hyp,
                         double* waux_hyp) {
  if (!h) return fail(FBS_E_ARG, "handle is NULL");
  if (h->prec != FBS_F64) return fail(FBS_E_ARG, "the FBS_F32 form keeps no gamma, tau or sigma widths");
  int rc = enter(h);
  if (rc) return rc;
  const size_t G = (size_t)h->mc.G, L = (size_t)h->mc.L;
  if (w_gam) FBS_CUDA(cudaMemcpyAsync(w_gam, h->p.w_gam, G * 8, cudaMemcpyDeviceToHost, h->s));
  if (waux_gam)
    FBS_CUDA(cudaMemcpyAsync(waux_gam, h->p.waux_gam, G * 8, cudaMemcpyDeviceToHost, h->s));
  Hyper hy;
  if ((rc = read_hyper(h, &hy))) return rc;
  if (w_hyp) memcpy(w_hyp, hy.w_hyp, (L + 1) * 8);
  if (waux_hyp) memcpy(waux_hyp, hy.waux_hyp, (L + 1) * 8);
  return leave(h);
}

int fbs_set_slice_widths(fbs_handle* h, const double* w_gam, const double* waux_gam,
                         const double* w_hyp, const double* waux_hyp) {
  if (!h) return fail(FBS_E_ARG, "handle is NULL");
  if (h->prec != FBS_F64) return fail(FBS_E_ARG, "the FBS_F32 form keeps no gamma, tau or sigma widths");
  int rc = enter(h);
  if (rc) return rc;
  const size_t G = (size_t)h->mc.G, L = (size_t)h->mc.L;
  if (w_gam) FBS_CUDA(cudaMemcpyAsync(h->p.w_gam, w_gam, G * 8, cudaMemcpyHostToDevice, h->s));
  if (waux_gam)
    FBS_CUDA(cudaMemcpyAsync(h->p.waux_gam, waux_gam, G * 8, cudaMemcpyHostToDevice, h->s));
  Hyper hy;
  if ((rc = read_hyper(h, &hy))) return rc;
  if (w_hyp) memcpy(hy.w_hyp, w_hyp, (L + 1) * 8);
  if (waux_hyp) memcpy(hy.waux_hyp, waux_hyp, (L + 1) * 8);
  FBS_CUDA(cudaMemcpyAsync(h->p.hyp, &hy, sizeof(Hyper), cudaMemcpyHostToDevice, h->s));
  FBS_CUDA(cudaStreamSynchronize(h->s));
  return leave(h);
}

int fbs_trace(fbs_handle* h, int64_t max_rows, double* phi, double* beta, int64_t* rows) {
  if (!h) return fail(FBS_E_ARG, "handle is NULL");
  if (max_rows < 0) return fail(FBS_E_ARG, "max_rows must be >= 0");
  int rc = enter(h);
  if (rc) return rc;
  Hyper hy;
  if ((rc = read_hyper(h, &hy))) return rc;
  const long long n = hy.trace_rows < max_rows ? hy.trace_rows : max_rows;
  const int P = h->mc.P, L = h->mc.L, G = h->mc.G;
  if (phi && n > 0)
    FBS_CUDA(cudaMemcpyAsync(phi, h->p.trace_phi, (size_t)n * P * 8, cudaMemcpyDeviceToHost, h->s));
  if (beta && n > 0) {
    if (!h->p.trace_beta) return fail(FBS_E_ARG, "this handle keeps no beta trace");
    std::vector<double> tmp((size_t)L * G);
    for (long long r = 0; r < n; ++r) {
      FBS_CUDA(cudaMemcpyAsync(tmp.data(), h->p.trace_beta + (size_t)r * L * G, tmp.size() * 8,
                               cudaMemcpyDeviceToHost, h->s));
      FBS_CUDA(cudaStreamSynchronize(h->s));
      double* dst = beta + (size_t)r * G * L;
      for (int l = 0; l < L; ++l)
        for (int g = 0; g < G; ++g) dst[(size_t)g * L + l] = tmp[(size_t)l * G + g];
    }
  }
  FBS_CUDA(cudaStreamSynchronize(h->s));
  if (rows) *rows = n;
  return leave(h);
}

int fbs_beta_ess(fbs_handle* h, double* ess) {
  if (!h || !ess) return fail(FBS_E_ARG, "handle or ess is NULL");
  if (!h->p.trace_beta) return fail(FBS_E_ARG, "this handle keeps no beta trace");
  int rc = enter(h);
  if (rc) return rc;
  Hyper hy;
  if ((rc = read_hyper(h, &hy))) return rc;
  if (hy.trace_rows < 4) return fail(FBS_E_ARG, "the beta trace holds fewer than 4 rows");
  const int L = h->mc.L, G = h->mc.G;
  const long long S = (long long)L * G;
  double* d_ess = nullptr;
  FBS_CUDA(cudaMallocAsync((void**)&d_ess, (size_t)S * 8, h->s));
  cudaError_t e = launch_ess(h->p.trace_beta, hy.trace_rows, S, d_ess, h->s);
  std::vector<double> tmp((size_t)S);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(tmp.data(), d_ess, (size_t)S * 8, cudaMemcpyDeviceToHost, h->s);
  cudaFreeAsync(d_ess, h->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
  FBS_CUDA(e);
  for (int l = 0; l < L; ++l)
    for (int g = 0; g < G; ++g) ess[(size_t)g * L + l] = tmp[(size_t)l * G + g];
  return leave(h);
}

int fbs_count_sums(fbs_handle* h, int64_t* T) {
  if (!h || !T) return fail(FBS_E_ARG, "handle or T is NULL");
  if (!h->x_integral) return fail(FBS_E_ARG, "X is not integer-valued");
  int rc = enter(h);
  if (rc) return rc;
  const int L = h->mc.L, G = h->mc.G;
  std::vector<double> tmp((size_t)L * G);
  FBS_CUDA(cudaMemcpyAsync(tmp.data(), h->p.T, tmp.size() * 8, cudaMemcpyDeviceToHost, h->s));
  FBS_CUDA(cudaStreamSynchronize(h->s));
  for (int l = 0; l < L; ++l)
    for (int g = 0; g < G; ++g) T[(size_t)g * L + l] = (int64_t)tmp[(size_t)l * G + g];
  return leave(h);
}

int fbs_counters(fbs_handle* h, int64_t* out) {
  if (!h || !out) return fail(FBS_E_ARG, "handle or out is NULL");
  int rc = enter(h);
  if (rc) return rc;
  if ((rc = sum_counters(h, out))) return rc;
  return leave(h);
}

int fbs_profile(fbs_handle* h, int64_t n_iter, int64_t burnin, int64_t thin, double* ms) {
  if (!h || !ms) return fail(FBS_E_ARG, "handle or ms is NULL");
  if (h->is_view) return fail(FBS_E_ARG, "a batch dataset runs with fbs_batch_run");
  if (n_iter < 1 || n_iter > 4096 || burnin < 0 || thin < 1)
    return fail(FBS_E_ARG, "need 1 <= n_iter <= 4096, burnin >= 0, thin >= 1");
  int rc = enter(h);
  if (rc) return rc;
  FBS_CUDA(launch_set_run(h->p.hyp, burnin, burnin / 2, thin, h->s));
  const bool learned = h->prec == FBS_F32 && h->pf.prop != nullptr;
  // probe slots: 3 kernels per sweep; starts [0, n), ends [n, 2n)
  const int n = (int)(3 * n_iter);
  unsigned long long* kt = nullptr;
  FBS_CUDA(cudaMalloc((void**)&kt, sizeof(unsigned long long) * 2 * (size_t)n));
  cudaError_t e = cudaMemsetAsync(kt, 0xFF, sizeof(unsigned long long) * n, h->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(kt + n, 0, sizeof(unsigned long long) * n, h->s);
  // the sweeps captured exactly as fbs_run's segments, with the probe on
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (e == cudaSuccess) e = cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    h->p.ktime = h->pf.ktime = kt;
    h->p.ktime_n = h->pf.ktime_n = n;
    e = capture_sweeps(h, (int)n_iter);
    h->p.ktime = h->pf.ktime = nullptr;
    h->p.ktime_n = h->pf.ktime_n = 0;
    cudaError_t e2 = cudaStreamEndCapture(h->s, &graph);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(exec, h->s);
  std::vector<unsigned long long> t((size_t)2 * n);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(t.data(), kt, sizeof(unsigned long long) * 2 * n, cudaMemcpyDeviceToHost,
                        h->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  cudaFree(kt);
  double span[3] = {0.0, 0.0, 0.0};  // eps, gamma/beta, hyperparameters (ns)
  unsigned long long first = ~0ull, last = 0ull;
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    if (t[i] == ~0ull || t[n + i] < t[i]) {
      e = cudaErrorUnknown;  // a probed kernel did not run
      break;
    }
    span[i % 3] += (double)(t[n + i] - t[i]);
    first = std::min(first, t[i]);
    last = std::max(last, t[n + i]);
  }
  // the network pass alone (the sweep runs it inside the gamma/beta kernel
  // when blocks have 128 threads): direct launches with CUDA events, timed for
  // reference; its outputs are recomputed by the next sweep
  double t_net = 0.0;
  if (e == cudaSuccess && learned) {
    cudaEvent_t a = nullptr, b = nullptr;
    e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    for (int64_t i = 0; i < n_iter && e == cudaSuccess; ++i) {
      cudaEventRecord(a, h->s);
      e = launch_proposal_f32(h->mc, h->pf, h->learned->w_image, h->learned->prop, h->s);
      cudaEventRecord(b, h->s);
      if (e == cudaSuccess) e = cudaEventSynchronize(b);
      float ms1 = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms1, a, b);
      t_net += ms1;
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
  if (e == cudaErrorUnknown) return fail(FBS_E_CUDA, "fbs_profile: a probed kernel left no time");
  FBS_CUDA(e);
  ms[0] = span[0] * 1e-6 / (double)n_iter;
  ms[1] = span[1] * 1e-6 / (double)n_iter;
  ms[2] = span[2] * 1e-6 / (double)n_iter;
  ms[3] = t_net / (double)n_iter;
  ms[4] = (double)(last - first) * 1e-6 / (double)n_iter;
  return leave(h);
}

int fbs_uniforms(uint64_t seed, uint32_t chain, uint32_t stream, uint32_t index0, int n_index,
                 uint32_t iter, uint32_t k0, int n_k, double* out) {
  if (n_index < 0 || n_k < 0 || !out) return fail(FBS_E_ARG, "bad sizes or NULL out");
  if (n_index == 0 || n_k == 0) return FBS_OK;
  double* d = nullptr;
  const size_t bytes = (size_t)n_index * n_k * 8;
  FBS_CUDA(cudaMalloc((void**)&d, bytes));
  cudaError_t e = launch_uniforms(seed, chain, stream, index0, n_index, iter, k0, n_k, d, 0);
  if (e == cudaSuccess) e = cudaMemcpy(out, d, bytes, cudaMemcpyDeviceToHost);
  cudaFree(d);
  FBS_CUDA(e);
  return FBS_OK;
}

void fbs_free(fbs_handle* h) {
  if (!h || h->is_view) return;
  if (h->s) cudaStreamSynchronize(h->s);
  cudaFree(h->con);
  cudaFree(h->con_count);
  if (LearnedState* ls = h->learned) {
    cudaFree(ls->params);
    cudaFree(ls->w_image);
    cudaFree(ls->adam_m);
    cudaFree(ls->adam_v);
    cudaFree(ls->prop);
    cudaFree(ls->use_mh);
    cudaFree(ls->mh_acc);
    cudaFree(ls->mh_try);
    cudaFree(ls->stats);
    cudaFree(ls->pair_feat);
    cudaFree(ls->pair_beta);
    delete ls;
  }
  if (h->seg_exec) cudaGraphExecDestroy(h->seg_exec);
  if (h->own_ws && h->ws) cudaFree(h->ws);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  if (h->ev_g) cudaEventDestroy(h->ev_g);
  if (h->ev_h) cudaEventDestroy(h->ev_h);
  if (h->s2) cudaStreamDestroy(h->s2);
  if (h->s) cudaStreamDestroy(h->s);
  delete h;
}

const char* fbs_last_error_string(void) { return g_err.c_str(); }



// ---------------------------------------------------------------- learned proposal

}  // extern "C"

namespace {

int learned_setup(fbs_handle* h) {
  if (!h) return fail(FBS_E_ARG, "handle is NULL");
  if (h->is_view) return fail(FBS_E_ARG, "the learned proposal needs a single-chain handle");
  if (h->prec != FBS_F32) return fail(FBS_E_ARG, "the learned proposal runs in the FBS_F32 form");
  if (h->learned) return FBS_OK;
  LearnedState* ls = new LearnedState();
  const int L = h->mc.L, G = h->mc.G;
  ls->L = L;
  ls->F = 4 * L + 1;
  ls->K = L + L * (L + 1) / 2;
  ls->np = mlp_param_count(L);
  h->learned = ls;
  FBS_CUDA(cudaMalloc((void**)&ls->params, sizeof(float) * ls->np));
  FBS_CUDA(cudaMalloc(&ls->w_image, tc_image_bytes(L)));
  FBS_CUDA(cudaMalloc((void**)&ls->adam_m, sizeof(float) * ls->np));
  FBS_CUDA(cudaMalloc((void**)&ls->adam_v, sizeof(float) * ls->np));
  FBS_CUDA(cudaMalloc((void**)&ls->prop, sizeof(float) * ls->K * (size_t)G));
  FBS_CUDA(cudaMalloc((void**)&ls->use_mh, (size_t)G));
  FBS_CUDA(cudaMalloc((void**)&ls->mh_acc, sizeof(unsigned) * 2 * (size_t)G));
  FBS_CUDA(cudaMalloc((void**)&ls->mh_try, sizeof(unsigned) * 2 * (size_t)G));
  FBS_CUDA(cudaMalloc((void**)&ls->stats, sizeof(float) * (size_t)(2 * ls->F + 2 * L)));
  FBS_CUDA(cudaMemsetAsync(ls->use_mh, 0, (size_t)G, h->s));
  FBS_CUDA(cudaMemsetAsync(ls->mh_acc, 0, sizeof(unsigned) * 2 * (size_t)G, h->s));
  FBS_CUDA(cudaMemsetAsync(ls->mh_try, 0, sizeof(unsigned) * 2 * (size_t)G, h->s));
  FBS_CUDA(cudaMemsetAsync(ls->adam_m, 0, sizeof(float) * ls->np, h->s));
  FBS_CUDA(cudaMemsetAsync(ls->adam_v, 0, sizeof(float) * ls->np, h->s));
  // He-style initialisation from Philox normals on the host (deterministic).
  std::vector<float> w(ls->np, 0.0f);
  uint64_t state = 0x9E3779B97F4A7C15ull;
  auto nrm = [&]() {  // Box-Muller on a splitmix64 stream
    auto next = [&]() {
      uint64_t z = (state += 0x9E3779B97F4A7C15ull);
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      return ((double)((z ^ (z >> 31)) >> 11) + 0.5) * 0x1p-53;
    };
    const double u1 = next(), u2 = next();
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
  };
  const int H = kMlpHidden, F = ls->F, K = ls->K;
  size_t o = 0;
  for (int i = 0; i < H * F; ++i) w[o++] = (float)(nrm() * sqrt(2.0 / F));
  o += H;
  for (int i = 0; i < H * H; ++i) w[o++] = (float)(nrm() * sqrt(2.0 / H));
  o += H;
  for (int i = 0; i < K * H; ++i) w[o++] = (float)(nrm() * 0.1 * sqrt(1.0 / H));
  FBS_CUDA(cudaMemcpyAsync(ls->params, w.data(), sizeof(float) * ls->np, cudaMemcpyHostToDevice,
                           h->s));
  FBS_CUDA(launch_pack_image(ls->params, ls->w_image, ls->L, h->s));
  FBS_CUDA(cudaStreamSynchronize(h->s));
  return FBS_OK;
}

void learned_apply(fbs_handle* h, int mode, int mh_all) {
  LearnedState* ls = h->learned;
  ls->mode = mode;
  h->pf.prop = mode ? ls->prop : nullptr;
  h->pf.mh_replace = mode == 2 ? 1 : 0;
  h->pf.use_mh = ls->use_mh;
  h->pf.mh_acc = ls->mh_acc;
  h->pf.mh_try = ls->mh_try;
  h->pf.mh_all = mh_all;
  if (h->seg_exec) {
    cudaGraphExecDestroy(h->seg_exec);
    h->seg_exec = nullptr;
  }
}

constexpr int kTrainGraphSteps = 8;  // training steps per replayed graph

// Scratch of one training step for batch size B; flags: the tensor-core wait
// flag word of the step's kernels (zeroed here).
struct TrainBufs {
  float *fb, *yb, *part, *grad, *loss;
  unsigned* flags;
  void* img;  // the training kernel's weight image (zeroed)
};

void train_bufs_free(TrainBufs& t) {
  cudaFree(t.fb);
  cudaFree(t.img);
  t.fb = nullptr;
  t.img = nullptr;
}

// Gradient and summed loss of the minibatch in t.fb / t.yb at params.
int mlp_step(const float* params, int L, int B, TrainBufs& t, cudaStream_t s) {
  FBS_CUDA(launch_mlp_grad(params, L, B, t.fb, t.yb, t.part, t.grad, t.loss, t.img, t.flags,
                           kTcWaitPolls, s));
  return FBS_OK;
}

int train_bufs_alloc(TrainBufs& t, int L, int B) {
  const int F = 4 * L + 1, np = mlp_param_count(L);
  memset(&t, 0, sizeof(t));
  const size_t n = (size_t)B * (F + L) + (size_t)train_blocks(B) * (np + 1) + np + 2;
  FBS_CUDA(prepare_train_kernel(L));
  float* base = nullptr;
  FBS_CUDA(cudaMalloc((void**)&base, n * sizeof(float)));
  float* q = base;
  t.fb = q; q += (size_t)B * F;
  t.yb = q; q += (size_t)B * L;
  t.part = q; q += (size_t)train_blocks(B) * (np + 1);
  t.grad = q; q += np;
  t.loss = q; q += 1;
  t.flags = reinterpret_cast<unsigned*>(q);
  t.img = nullptr;
  cudaError_t e = cudaMemset(t.flags, 0, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMalloc(&t.img, train_image_bytes(L));
  if (e == cudaSuccess) e = cudaMemset(t.img, 0, train_image_bytes(L));
  if (e != cudaSuccess) train_bufs_free(t);
  FBS_CUDA(e);
  return FBS_OK;
}

// Whether a tensor-core wait of the training kernels gave up (*flags, read
// after the stream's work finished).
int train_flags_ok(const TrainBufs& t, cudaStream_t s) {
  unsigned f = 0;
  FBS_CUDA(cudaMemcpyAsync(&f, t.flags, sizeof(f), cudaMemcpyDeviceToHost, s));
  FBS_CUDA(cudaStreamSynchronize(s));
  if (f & kFlagTimeout)
    return fail(FBS_E_CUDA, "a tensor-core wait of the training step gave up");
  return FBS_OK;
}

}  // namespace

extern "C" {

int fbs_proposal_collect(fbs_handle* h, int64_t n_pairs_sweeps, int64_t burnin, int64_t thin) {
  int rc = learned_setup(h);
  if (rc) return rc;
  if (n_pairs_sweeps < 1 || burnin < 0 || thin < 1)
    return fail(FBS_E_ARG, "need n_pairs_sweeps >= 1, burnin >= 0, thin >= 1");
  LearnedState* ls = h->learned;
  const long long need = ls->pairs + n_pairs_sweeps * (long long)h->mc.G;
  if (need > ls->pair_cap) {
    float *f = nullptr, *b = nullptr;
    FBS_CUDA(cudaMalloc((void**)&f, sizeof(float) * (size_t)need * ls->F));
    FBS_CUDA(cudaMalloc((void**)&b, sizeof(float) * (size_t)need * ls->L));
    if (ls->pairs > 0) {
      FBS_CUDA(cudaMemcpyAsync(f, ls->pair_feat, sizeof(float) * (size_t)ls->pairs * ls->F,
                               cudaMemcpyDeviceToDevice, h->s));
      FBS_CUDA(cudaMemcpyAsync(b, ls->pair_beta, sizeof(float) * (size_t)ls->pairs * ls->L,
                               cudaMemcpyDeviceToDevice, h->s));
      FBS_CUDA(cudaStreamSynchronize(h->s));
    }
    cudaFree(ls->pair_feat);
    cudaFree(ls->pair_beta);
    ls->pair_feat = f;
    ls->pair_beta = b;
    ls->pair_cap = need;
  }
  for (int64_t k = 0; k < n_pairs_sweeps; ++k) {
    rc = fbs_run(h, thin, burnin, 1);
    if (rc) return rc;
    FBS_CUDA(launch_collect_f32(h->mc, h->pf, ls->pair_feat, ls->pair_beta, ls->pairs, h->s));
    ls->pairs += h->mc.G;
  }
  FBS_CUDA(cudaStreamSynchronize(h->s));
  return FBS_OK;
}

int fbs_proposal_train(fbs_handle* h, int epochs, int batch, double lr, uint64_t seed,
                       double* final_loss) {
  int rc = learned_setup(h);
  if (rc) return rc;
  LearnedState* ls = h->learned;
  if (ls->pairs < 1) return fail(FBS_E_ARG, "no training pairs: call fbs_proposal_collect first");
  if (epochs < 1 || batch < 32 || !(lr > 0.0)) return fail(FBS_E_ARG, "bad epochs, batch or lr");
  TrainBufs t;
  rc = train_bufs_alloc(t, ls->L, batch);
  if (rc) return rc;
  const long long steps_per_epoch = (ls->pairs + batch - 1) / batch;
  const long long steps = steps_per_epoch * epochs;
  const int F = ls->F, L = ls->L;
  // Standardise features and beta by the pairs' column statistics; parameters
  // already trained (or set) move to those coordinates first, the initial ones
  // are drawn for them.
  std::vector<float> st_h(2 * F + 2 * L);
  cudaError_t e = launch_col_stats(ls->pair_feat, ls->pair_beta, ls->pairs, F, L, ls->stats, h->s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(st_h.data(), ls->stats, sizeof(float) * st_h.size(),
                        cudaMemcpyDeviceToHost, h->s);
  if (e == cudaSuccess && ls->trained) e = launch_fold(ls->params, ls->stats, L, 0, h->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
  double log_scale = 0.0;  // NLL of raw beta = NLL of standardised beta + sum log s_beta
  for (int l = 0; l < L; ++l) log_scale += log((double)st_h[2 * F + L + l]);
  // Training steps (minibatch gather, forward, backward, Adam, bookkeeping) are
  // captured once, kTrainGraphSteps of them in one graph and one alone, and
  // replayed to make `steps`; the step counter, the Adam scalars and the loss
  // sum live in a device control block.
  TrainCtl ctl;
  memset(&ctl, 0, sizeof(ctl));
  ctl.t = (unsigned long long)ls->adam_t;
  ctl.steps = steps;
  ctl.epoch_steps = steps_per_epoch;
  ctl.lr = lr;
  ctl.b1 = 0.9f;
  ctl.b2 = 0.999f;
  TrainCtl* d_ctl = nullptr;
  cudaGraphExec_t exec[2] = {nullptr, nullptr};  // kTrainGraphSteps steps, one step
  if (e == cudaSuccess) e = cudaMalloc((void**)&d_ctl, sizeof(TrainCtl));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_ctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice, h->s);
  if (e == cudaSuccess) e = launch_pack_train_image(ls->params, L, t.img, h->s);
  for (int gi = 0; gi < 2 && e == cudaSuccess; ++gi) {
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t ce = cudaSuccess;
      for (int k = 0; k < (gi == 0 ? kTrainGraphSteps : 1) && ce == cudaSuccess; ++k)
        ce = launch_train_step(ls->params, L, batch, ls->pair_feat, ls->pair_beta, ls->pairs,
                               seed, d_ctl, ls->stats, t.part, t.grad, t.loss, ls->adam_m,
                               ls->adam_v, t.img, t.flags, h->pf.tc_polls, h->s);
      e = cudaStreamEndCapture(h->s, &graph);
      if (e == cudaSuccess) e = ce;
    }
    if (e == cudaSuccess && rc == FBS_OK) e = cudaGraphInstantiate(&exec[gi], graph, 0);
    if (graph) cudaGraphDestroy(graph);
  }
  for (long long st = 0; st < steps / kTrainGraphSteps && rc == FBS_OK && e == cudaSuccess; ++st)
    e = cudaGraphLaunch(exec[0], h->s);
  for (long long st = 0; st < steps % kTrainGraphSteps && rc == FBS_OK && e == cudaSuccess; ++st)
    e = cudaGraphLaunch(exec[1], h->s);
  if (e == cudaSuccess && rc == FBS_OK)
    e = cudaMemcpyAsync(&ctl, d_ctl, sizeof(ctl), cudaMemcpyDeviceToHost, h->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
  for (cudaGraphExec_t x : exec)
    if (x) cudaGraphExecDestroy(x);
  cudaFree(d_ctl);
  // a step whose tensor-core wait gave up left the parameters as they were; the
  // parameters still go back to raw coordinates before the error is returned
  int rc_wait = FBS_OK;
  if (e == cudaSuccess && rc == FBS_OK) rc_wait = train_flags_ok(t, h->s);
  if (e == cudaSuccess && rc == FBS_OK) ls->adam_t = (long long)ctl.t;
  const double loss_epoch = ctl.loss_sum;
  if (e == cudaSuccess && rc == FBS_OK) e = launch_fold(ls->params, ls->stats, L, 1, h->s);
  if (e == cudaSuccess && rc == FBS_OK) e = launch_pack_image(ls->params, ls->w_image, ls->L, h->s);
  if (e == cudaSuccess && rc == FBS_OK) e = cudaStreamSynchronize(h->s);
  train_bufs_free(t);
  if (rc) return rc;
  FBS_CUDA(e);
  ls->trained = true;  // raw coordinates from here on, even after a failed wait
  if (rc_wait) return rc_wait;
  if (final_loss) *final_loss = loss_epoch / (double)steps_per_epoch + log_scale;
  if (h->seg_exec) {
    cudaGraphExecDestroy(h->seg_exec);
    h->seg_exec = nullptr;
  }
  return FBS_OK;
}

int fbs_proposal_calibrate(fbs_handle* h, int64_t n_sweeps, int64_t burnin, double min_accept) {
  int rc = learned_setup(h);
  if (rc) return rc;
  if (n_sweeps < 1 || burnin < 0 || !(min_accept >= 0.0 && min_accept <= 1.0))
    return fail(FBS_E_ARG, "need n_sweeps >= 1, burnin >= 0, 0 <= min_accept <= 1");
  LearnedState* ls = h->learned;
  const int G = h->mc.G;
  const size_t n2 = 2 * (size_t)G;
  FBS_CUDA(cudaMemsetAsync(ls->mh_acc, 0, sizeof(unsigned) * n2, h->s));
  FBS_CUDA(cudaMemsetAsync(ls->mh_try, 0, sizeof(unsigned) * n2, h->s));
  learned_apply(h, 1, 3);  // every gene, the two proposals on alternate sweeps
  rc = fbs_run(h, n_sweeps, burnin, 1);
  if (rc) return rc;
  std::vector<unsigned> acc(n2), tr(n2);
  FBS_CUDA(cudaMemcpyAsync(acc.data(), ls->mh_acc, sizeof(unsigned) * n2, cudaMemcpyDeviceToHost,
                           h->s));
  FBS_CUDA(cudaMemcpyAsync(tr.data(), ls->mh_try, sizeof(unsigned) * n2, cudaMemcpyDeviceToHost,
                           h->s));
  FBS_CUDA(cudaStreamSynchronize(h->s));
  // per gene: the proposal with the higher acceptance rate, if it reaches min_accept
  std::vector<uint8_t> use(G);
  for (int g = 0; g < G; ++g) {
    uint8_t best = 0;
    double best_rate = -1.0;
    for (int k = 0; k < 2; ++k) {
      const unsigned t = tr[(size_t)k * G + g], a = acc[(size_t)k * G + g];
      const double rate = t > 0 ? (double)a / (double)t : -1.0;
      if (t > 0 && a >= min_accept * t && rate > best_rate) {
        best_rate = rate;
        best = (uint8_t)(k + 1);
      }
    }
    use[g] = best;
  }
  FBS_CUDA(cudaMemcpyAsync(ls->use_mh, use.data(), (size_t)G, cudaMemcpyHostToDevice, h->s));
  FBS_CUDA(cudaMemsetAsync(ls->mh_acc, 0, sizeof(unsigned) * n2, h->s));
  FBS_CUDA(cudaMemsetAsync(ls->mh_try, 0, sizeof(unsigned) * n2, h->s));
  FBS_CUDA(cudaStreamSynchronize(h->s));
  learned_apply(h, 1, 0);
  return FBS_OK;
}

int fbs_proposal_mode(fbs_handle* h, int mode) {
  int rc = learned_setup(h);
  if (rc) return rc;
  if (mode < 0 || mode > 2) return fail(FBS_E_ARG, "mode must be 0, 1 or 2");
  FBS_CUDA(cudaStreamSynchronize(h->s));
  learned_apply(h, mode, 0);
  return FBS_OK;
}

int fbs_proposal_fused(fbs_handle* h, int on) {
  int rc = learned_setup(h);
  if (rc) return rc;
  if (on != 0 && on != 1) return fail(FBS_E_ARG, "on must be 0 or 1");
  FBS_CUDA(cudaStreamSynchronize(h->s));
  h->learned->fused = on != 0;
  if (h->seg_exec) {  // the captured segment changes
    cudaGraphExecDestroy(h->seg_exec);
    h->seg_exec = nullptr;
  }
  return FBS_OK;
}

int fbs_proposal_wait_limit(fbs_handle* h, uint32_t polls) {
  if (!h) return fail(FBS_E_ARG, "handle is NULL");
  if (h->prec != FBS_F32 || h->is_view)
    return fail(FBS_E_ARG, "the learned proposal needs a single-chain FBS_F32 handle");
  h->pf.tc_polls = polls;
  if (h->seg_exec) {  // captured kernels hold the old value
    cudaGraphExecDestroy(h->seg_exec);
    h->seg_exec = nullptr;
  }
  return FBS_OK;
}

int fbs_proposal_params(fbs_handle* h, float* get, const float* set, int n) {
  int rc = learned_setup(h);
  if (rc) return rc;
  LearnedState* ls = h->learned;
  if (n != ls->np) return fail(FBS_E_ARG, "n must equal the parameter count");
  FBS_CUDA(cudaStreamSynchronize(h->s));
  if (get)
    FBS_CUDA(cudaMemcpy(get, ls->params, sizeof(float) * n, cudaMemcpyDeviceToHost));
  if (set) {
    FBS_CUDA(cudaMemcpy(ls->params, set, sizeof(float) * n, cudaMemcpyHostToDevice));
    FBS_CUDA(launch_pack_image(ls->params, ls->w_image, ls->L, h->s));
    FBS_CUDA(cudaStreamSynchronize(h->s));
    ls->trained = true;
  }
  return FBS_OK;
}

int fbs_proposal_stats(fbs_handle* h, int64_t* accepted, int64_t* tried, int* n_mh_genes,
                       int* n_prior_genes) {
  if (!h || !h->learned) return fail(FBS_E_ARG, "the handle has no learned proposal");
  LearnedState* ls = h->learned;
  const int G = h->mc.G;
  const size_t n2 = 2 * (size_t)G;
  std::vector<unsigned> acc(n2), tr(n2);
  std::vector<uint8_t> use(G);
  FBS_CUDA(cudaStreamSynchronize(h->s));
  FBS_CUDA(cudaMemcpy(acc.data(), ls->mh_acc, sizeof(unsigned) * n2, cudaMemcpyDeviceToHost));
  FBS_CUDA(cudaMemcpy(tr.data(), ls->mh_try, sizeof(unsigned) * n2, cudaMemcpyDeviceToHost));
  FBS_CUDA(cudaMemcpy(use.data(), ls->use_mh, (size_t)G, cudaMemcpyDeviceToHost));
  int64_t a = 0, t = 0;
  int u = 0, up = 0;
  for (size_t i = 0; i < n2; ++i) {
    a += acc[i];
    t += tr[i];
  }
  for (int g = 0; g < G; ++g) {
    u += use[g] != 0;
    up += use[g] == kMovePrior;
  }
  if (accepted) *accepted = a;
  if (tried) *tried = t;
  if (n_mh_genes) *n_mh_genes = u;
  if (n_prior_genes) *n_prior_genes = up;
  return FBS_OK;
}

int fbs_rhat(int C, fbs_handle* const* chains, double* rhat_phi, double* rhat_beta,
             double* rhat_gam, double* rhat_eps) {
  if (C < 2 || C > FBS_MAX_RHAT_CHAINS || !chains)
    return fail(FBS_E_ARG, "need 2 <= C <= FBS_MAX_RHAT_CHAINS chains");
  for (int c = 0; c < C; ++c)
    if (!chains[c]) return fail(FBS_E_ARG, "a chain handle is NULL");
  const fbs_handle* h0 = chains[0];
  const int N = h0->mc.N, G = h0->mc.G, L = h0->mc.L, P = h0->mc.P;
  long long M = -1;
  for (int c = 0; c < C; ++c) {
    fbs_handle* h = chains[c];
    if (h->mc.N != N || h->mc.G != G || h->mc.L != L || h->prec != h0->prec)
      return fail(FBS_E_ARG, "chains differ in N, G, L or precision");
    if (rhat_eps && !h->mc.moments_eps) return fail(FBS_E_ARG, "a chain has no eps moments");
    FBS_CUDA(cudaStreamSynchronize(h->s));
    Hyper hy;
    int rc = read_hyper(h, &hy);
    if (rc) return rc;
    if (M < 0) M = hy.n_mom;
    if (hy.n_mom != M) return fail(FBS_E_ARG, "chains hold different numbers of draws");
  }
  if (M < 2) return fail(FBS_E_ARG, "need at least 2 post-burn-in draws per chain");
  const bool f32 = h0->prec == FBS_F32;
  const size_t NG = (size_t)N * G, LG = (size_t)L * G;
  double* d_out = nullptr;
  FBS_CUDA(cudaMalloc((void**)&d_out, sizeof(double) * std::max(NG, std::max(LG, (size_t)P))));
  cudaStream_t s = h0->s;
  auto run = [&](int which, long long n, double* host, int R) -> int {
    RhatInput in;
    memset(&in, 0, sizeof(in));
    in.C = C;
    in.M = M;
    in.n = n;
    in.f32 = f32 && which != 3;
    for (int c = 0; c < C; ++c) {
      const fbs_handle* h = chains[c];
      if (which == 3) {  // phi: FP64 moments in the Hyper block of either form
        in.m[c] = (const double*)((const char*)h->p.hyp + offsetof(Hyper, m_phi));
        in.q[c] = (const double*)((const char*)h->p.hyp + offsetof(Hyper, q_phi));
      } else if (f32) {
        in.mf[c] = which == 0 ? h->pf.mom_beta : (which == 1 ? h->pf.mom_gam : h->pf.mom_eps);
      } else {
        in.m[c] = which == 0 ? h->p.m_beta : (which == 1 ? h->p.m_gam : h->p.m_eps);
        in.q[c] = which == 0 ? h->p.q_beta : (which == 1 ? h->p.q_gam : h->p.q_eps);
      }
    }
    cudaError_t e = launch_rhat(in, d_out, s);
    std::vector<double> tmp((size_t)n);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(tmp.data(), d_out, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(FBS_E_CUDA, std::string("rhat: ") + cudaGetErrorString(e));
    if (which == 3) {
      for (int k = 0; k < P; ++k) host[k] = tmp[k];
    } else {
      for (int r = 0; r < R; ++r)
        for (int g = 0; g < G; ++g) host[(size_t)g * R + r] = tmp[(size_t)r * G + g];
    }
    return FBS_OK;
  };
  int rc = FBS_OK;
  if (!rc && rhat_beta) rc = run(0, (long long)LG, rhat_beta, L);
  if (!rc && rhat_gam) rc = run(1, (long long)G, rhat_gam, 1);
  if (!rc && rhat_eps) rc = run(2, (long long)NG, rhat_eps, N);
  if (!rc && rhat_phi) rc = run(3, (long long)P, rhat_phi, 1);
  cudaFree(d_out);
  return rc;
}

int fbs_estimates_pooled(int C, fbs_handle* const* chains, fbs_estimates_out* out) {
  if (C < 1 || C > FBS_MAX_RHAT_CHAINS || !chains || !out)
    return fail(FBS_E_ARG, "need 1 <= C <= FBS_MAX_RHAT_CHAINS chains and an output struct");
  if (!(out->z > 0.0) || !isfinite(out->z)) return fail(FBS_E_ARG, "z must be finite and > 0");
  if (out->trace_phi && out->trace_rows_max < 0)
    return fail(FBS_E_ARG, "trace_rows_max must be >= 0");
  for (int c = 0; c < C; ++c)
    if (!chains[c]) return fail(FBS_E_ARG, "a chain handle is NULL");
  fbs_handle* h0 = chains[0];
  const int N = h0->mc.N, G = h0->mc.G, L = h0->mc.L, P = h0->mc.P;
  const bool want_eps = out->mean_eps || out->sd_eps || out->lo_eps || out->hi_eps;
  long long M = -1;
  for (int k = 0; k < FBS_NUM_COUNTERS; ++k) out->counters[k] = 0;
  out->mh_accepted = out->mh_tried = 0;
  for (int c = 0; c < C; ++c) {
    fbs_handle* h = chains[c];
    if (h->mc.N != N || h->mc.G != G || h->mc.L != L || h->prec != h0->prec)
      return fail(FBS_E_ARG, "chains differ in N, G, L or precision");
    if (want_eps && !h->mc.moments_eps) return fail(FBS_E_ARG, "a chain has no eps moments");
    FBS_CUDA(cudaStreamSynchronize(h->s));
    Hyper hy;
    int rc = read_hyper(h, &hy);
    if (rc) return rc;
    if (M < 0) M = hy.n_mom;
    if (hy.n_mom != M) return fail(FBS_E_ARG, "chains hold different numbers of draws");
    int64_t cnt[FBS_NUM_COUNTERS];
    if ((rc = sum_counters(h, cnt))) return rc;
    for (int k = 0; k < FBS_NUM_COUNTERS; ++k) out->counters[k] += cnt[k];
    if (h->learned) {
      int64_t a = 0, t = 0;
      if ((rc = fbs_proposal_stats(h, &a, &t, nullptr, nullptr))) return rc;
      out->mh_accepted += a;
      out->mh_tried += t;
    }
  }
  if (M < 1) return fail(FBS_E_ARG, "the chains hold no post-burn-in draws");
  out->count = M;
  const bool f32 = h0->prec == FBS_F32;
  const size_t NG = (size_t)N * G, LG = (size_t)L * G;
  const size_t nmax = std::max(NG, std::max(LG, (size_t)P));
  double* d_out = nullptr;
  FBS_CUDA(cudaMalloc((void**)&d_out, sizeof(double) * 4 * nmax));
  cudaStream_t s = h0->s;
  // which: 0 beta, 1 gamma, 2 eps, 3 phi; dst = mean, sd, lo, hi (each may be NULL)
  auto run = [&](int which, long long n, int R, double* const* dst) -> int {
    if (!dst[0] && !dst[1] && !dst[2] && !dst[3]) return FBS_OK;
    RhatInput in;
    memset(&in, 0, sizeof(in));
    in.C = C;
    in.M = M;
    in.n = n;
    in.f32 = f32 && which != 3;
    for (int c = 0; c < C; ++c) {
      const fbs_handle* h = chains[c];
      if (which == 3) {  // phi: FP64 moments in the Hyper block of either form
        in.m[c] = (const double*)((const char*)h->p.hyp + offsetof(Hyper, m_phi));
        in.q[c] = (const double*)((const char*)h->p.hyp + offsetof(Hyper, q_phi));
      } else if (f32) {
        in.mf[c] = which == 0 ? h->pf.mom_beta : (which == 1 ? h->pf.mom_gam : h->pf.mom_eps);
      } else {
        in.m[c] = which == 0 ? h->p.m_beta : (which == 1 ? h->p.m_gam : h->p.m_eps);
        in.q[c] = which == 0 ? h->p.q_beta : (which == 1 ? h->p.q_gam : h->p.q_eps);
      }
    }
    cudaError_t e = launch_estimates(in, out->z, d_out, s);
    std::vector<double> tmp(4 * (size_t)n);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(tmp.data(), d_out, sizeof(double) * 4 * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(FBS_E_CUDA, std::string("estimates: ") + cudaGetErrorString(e));
    for (int k = 0; k < 4; ++k) {
      double* host = dst[k];
      if (!host) continue;
      const double* src = tmp.data() + (size_t)k * n;
      for (int r = 0; r < R; ++r)
        for (long long g = 0; g < n / R; ++g) host[(size_t)g * R + r] = src[(size_t)r * (n / R) + g];
    }
    return FBS_OK;
  };
  double* const beta_d[4] = {out->mean_beta, out->sd_beta, out->lo_beta, out->hi_beta};
  double* const gam_d[4] = {out->mean_gam, out->sd_gam, out->lo_gam, out->hi_gam};
  double* const eps_d[4] = {out->mean_eps, out->sd_eps, out->lo_eps, out->hi_eps};
  double* const phi_d[4] = {out->mean_phi, out->sd_phi, out->lo_phi, out->hi_phi};
  int rc = run(0, (long long)LG, L, beta_d);
  if (!rc) rc = run(1, (long long)G, 1, gam_d);
  if (!rc) rc = run(2, (long long)NG, N, eps_d);
  if (!rc) rc = run(3, (long long)P, 1, phi_d);
  cudaFree(d_out);
  if (rc) return rc;
  out->trace_rows = 0;
  if (out->trace_phi && out->trace_rows_max > 0)
    return fbs_trace(h0, out->trace_rows_max, out->trace_phi, nullptr, &out->trace_rows);
  return FBS_OK;
}

int fbs_estimates(fbs_handle* h, fbs_estimates_out* out) {
  fbs_handle* one[1] = {h};
  return fbs_estimates_pooled(1, one, out);
}

int fbs_set_contrasts(fbs_handle* h, int n, const int* n_terms, const double* v, const double* b) {
  if (!h) return fail(FBS_E_ARG, "handle is NULL");
  if (h->is_view) return fail(FBS_E_ARG, "contrast probabilities need a single-chain handle");
  if (n < 0 || n > FBS_MAX_CONTRASTS) return fail(FBS_E_ARG, "n must be in [0, FBS_MAX_CONTRASTS]");
  const int L = h->mc.L, G = h->mc.G;
  Contrasts hc;
  memset(&hc, 0, sizeof(hc));
  hc.n = n;
  if (n > 0 && (!n_terms || !v || !b)) return fail(FBS_E_ARG, "n_terms, v or b is NULL");
  for (int q = 0; q < n; ++q) {
    if (n_terms[q] < 1 || n_terms[q] > FBS_MAX_CONTRAST_TERMS)
      return fail(FBS_E_ARG, "n_terms must be in [1, FBS_MAX_CONTRAST_TERMS]");
    hc.terms[q] = n_terms[q];
    for (int k = 0; k < n_terms[q]; ++k) {
      const double bk = b[q * FBS_MAX_CONTRAST_TERMS + k];
      if (!isfinite(bk)) return fail(FBS_E_ARG, "b must be finite");
      hc.b[q][k] = bk;
      hc.bf[q][k] = (float)bk;
      for (int l = 0; l < L; ++l) {
        const double vl = v[((size_t)q * FBS_MAX_CONTRAST_TERMS + k) * L + l];
        if (!isfinite(vl)) return fail(FBS_E_ARG, "v must be finite");
        hc.v[q][k][l] = vl;
        hc.vf[q][k][l] = (float)vl;
      }
    }
  }
  FBS_CUDA(cudaStreamSynchronize(h->s));
  if (n > 0 && !h->con) {
    FBS_CUDA(cudaMalloc((void**)&h->con, sizeof(Contrasts)));
    FBS_CUDA(cudaMalloc((void**)&h->con_count, sizeof(unsigned) * FBS_MAX_CONTRASTS * (size_t)G));
  }
  if (n > 0) {
    FBS_CUDA(cudaMemcpy(h->con, &hc, sizeof(hc), cudaMemcpyHostToDevice));
    FBS_CUDA(cudaMemset(h->con_count, 0, sizeof(unsigned) * FBS_MAX_CONTRASTS * (size_t)G));
  }
  Hyper hy;
  int rc = read_hyper(h, &hy);
  if (rc) return rc;
  h->ncon = n;
  h->con_nmom0 = hy.n_mom;
  const Contrasts* dc = n > 0 ? h->con : nullptr;
  unsigned* dn = n > 0 ? h->con_count : nullptr;
  h->p.con = dc;
  h->p.con_count = dn;
  h->pf.con = dc;
  h->pf.con_count = dn;
  if (h->seg_exec) {  // the captured kernels hold the old pointers
    cudaGraphExecDestroy(h->seg_exec);
    h->seg_exec = nullptr;
  }
  return FBS_OK;
}

int fbs_contrast_probs(fbs_handle* h, double* prob, int64_t* m) {
  if (!h) return fail(FBS_E_ARG, "handle is NULL");
  if (h->ncon < 1) return fail(FBS_E_ARG, "no contrast propositions are set");
  if (!prob) return fail(FBS_E_ARG, "prob is NULL");
  Hyper hy;
  int rc = read_hyper(h, &hy);
  if (rc) return rc;
  const long long M = hy.n_mom - h->con_nmom0;
  const int G = h->mc.G, n = h->ncon;
  std::vector<unsigned> cnt((size_t)n * G);
  FBS_CUDA(cudaMemcpy(cnt.data(), h->con_count, sizeof(unsigned) * cnt.size(),
                      cudaMemcpyDeviceToHost));
  for (int g = 0; g < G; ++g)
    for (int q = 0; q < n; ++q)
      prob[(size_t)g * n + q] = M > 0 ? (double)cnt[(size_t)q * G + g] / (double)M : 0.0;
  if (m) *m = M;
  return FBS_OK;
}

int fbs_proposal_kinds(fbs_handle* h, uint8_t* kinds) {
  if (!h || !h->learned) return fail(FBS_E_ARG, "the handle has no learned proposal");
  if (!kinds) return fail(FBS_E_ARG, "kinds is NULL");
  FBS_CUDA(cudaStreamSynchronize(h->s));
  FBS_CUDA(cudaMemcpy(kinds, h->learned->use_mh, (size_t)h->mc.G, cudaMemcpyDeviceToHost));
  return FBS_OK;
}

int fbs_proposal_param_count(int L) { return (L < 1 || L > FBS_MAX_L) ? -1 : mlp_param_count(L); }

int fbs_proposal_outputs(fbs_handle* h, float* out) {
  int rc = learned_setup(h);
  if (rc) return rc;
  if (!out) return fail(FBS_E_ARG, "out is NULL");
  LearnedState* ls = h->learned;
  rc = enter(h);
  if (rc) return rc;
  DevPtrsF32 pf = h->pf;
  pf.use_mh = ls->use_mh;
  pf.mh_all = 1;
  FBS_CUDA(launch_proposal_f32(h->mc, pf, ls->w_image, ls->prop, h->s));
  const int G = h->mc.G, K = ls->K;
  std::vector<float> tmp((size_t)K * G);
  FBS_CUDA(cudaMemcpyAsync(tmp.data(), ls->prop, tmp.size() * sizeof(float),
                           cudaMemcpyDeviceToHost, h->s));
  FBS_CUDA(cudaStreamSynchronize(h->s));
  for (int k = 0; k < K; ++k)
    for (int g = 0; g < G; ++g) out[(size_t)g * K + k] = tmp[(size_t)k * G + g];
  return leave(h);
}

int fbs_proposal_step(fbs_handle* h, int64_t it, int all_genes) {
  int rc = learned_setup(h);
  if (rc) return rc;
  if (it < 1 || it > 0xFFFFFFFFll) return fail(FBS_E_ARG, "it must be in [1, 2^32)");
  if (all_genes < 0 || all_genes > 2) return fail(FBS_E_ARG, "all_genes must be 0, 1 or 2");
  LearnedState* ls = h->learned;
  rc = enter(h);
  if (rc) return rc;
  DevPtrsF32 pf = h->pf;
  pf.prop = ls->prop;
  pf.use_mh = ls->use_mh;
  pf.mh_acc = ls->mh_acc;
  pf.mh_try = ls->mh_try;
  pf.mh_all = all_genes;
  FBS_CUDA(launch_proposal_f32(h->mc, pf, ls->w_image, ls->prop, h->s));
  FBS_CUDA(launch_mh_step_f32(h->mc, pf, it, h->s));
  FBS_CUDA(cudaStreamSynchronize(h->s));
  return leave(h);
}

int fbs_proposal_loss_grad(const float* params, int L, int B, const float* feat,
                           const float* beta, double* loss, float* grad) {
  if (!params || !feat || !beta || L < 1 || L > FBS_MAX_L || B < 1)
    return fail(FBS_E_ARG, "bad arguments");
  const int F = 4 * L + 1, np = mlp_param_count(L);
  TrainBufs t;
  int rc = train_bufs_alloc(t, L, B);
  if (rc) return rc;
  float* dp = nullptr;
  cudaError_t e = cudaMalloc((void**)&dp, sizeof(float) * np);
  if (e == cudaSuccess) e = cudaMemcpy(dp, params, sizeof(float) * np, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(t.fb, feat, sizeof(float) * (size_t)B * F, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(t.yb, beta, sizeof(float) * (size_t)B * L, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) rc = mlp_step(dp, L, B, t, 0);
  if (e == cudaSuccess && rc == FBS_OK) rc = train_flags_ok(t, 0);
  float l = 0.f;
  if (e == cudaSuccess && rc == FBS_OK) e = cudaMemcpy(&l, t.loss, sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && rc == FBS_OK && grad)
    e = cudaMemcpy(grad, t.grad, sizeof(float) * np, cudaMemcpyDeviceToHost);
  cudaFree(dp);
  train_bufs_free(t);
  if (rc) return rc;
  FBS_CUDA(e);
  if (loss) *loss = (double)l / B;
  return FBS_OK;
}

// ---------------------------------------------------------------- batches

}  // extern "C"

struct fbs_batch {
  int C = 0;
  fbs_options opt;
  std::vector<fbs_handle*> views;
  std::vector<ModelConst> mcs;
  std::vector<DevPtrsF32> pfs;
  std::vector<int> G, N;
  char* ws = nullptr;            // all datasets' regions
  ModelConst* d_mc = nullptr;    // [C]
  DevPtrsF32* d_pf = nullptr;    // [C]
  int* d_nblk = nullptr;         // [C] gamma/beta blocks per dataset
  int4* d_eps_tab = nullptr;
  int2* d_gb_tab = nullptr;
  int n_eps = 0, n_gb = 0, eps_block = 256, gb_block = 128, max_N = 0, seg = 100;
  size_t eps_cap = 0, gb_cap = 0;
  cudaStream_t user = nullptr, s = nullptr, s2 = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_g = nullptr, ev_h = nullptr;
  cudaGraphExec_t exec = nullptr;
  TopLevel* d_top = nullptr;       // three-level model: the top level, or null
  double* d_top_trace = nullptr;   // [trace_cap][1+L]
  bool three_level = false;
};

namespace {

void batch_release(fbs_batch* b) {
  if (!b) return;
  if (b->s) cudaStreamSynchronize(b->s);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (fbs_handle* v : b->views) {
    if (v->ev_in) cudaEventDestroy(v->ev_in);
    if (v->ev_out) cudaEventDestroy(v->ev_out);
    delete v;
  }
  cudaFree(b->ws);
  cudaFree(b->d_mc);
  cudaFree(b->d_pf);
  cudaFree(b->d_nblk);
  cudaFree(b->d_eps_tab);
  cudaFree(b->d_gb_tab);
  cudaFree(b->d_top);
  cudaFree(b->d_top_trace);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->ev_g) cudaEventDestroy(b->ev_g);
  if (b->ev_h) cudaEventDestroy(b->ev_h);
  if (b->s2) cudaStreamDestroy(b->s2);
  if (b->s) cudaStreamDestroy(b->s);
  delete b;
}

// Block tables for a schedule: every eps block covers one sample row and up to
// eps_block genes of one dataset; every gamma/beta block covers up to gb_block
// genes of one dataset.
int batch_tables(fbs_batch* b, int eps_block, int gb_block) {
  std::vector<int4> et;
  std::vector<int2> gt;
  std::vector<int> nblk(b->C);
  for (int c = 0; c < b->C; ++c) {
    const int ge = (b->G[c] + eps_block - 1) / eps_block;
    for (int n = 0; n < b->N[c]; ++n)
      for (int k = 0; k < ge; ++k)
        et.push_back(make_int4(c, n, k, (int)((n + k) % kCounterCopies)));
    nblk[c] = (b->G[c] + gb_block - 1) / gb_block;
    for (int k = 0; k < nblk[c]; ++k) gt.push_back(make_int2(c, k));
  }
  if (et.size() > b->eps_cap || gt.size() > b->gb_cap)
    return fail(FBS_E_ARG, "schedule needs more blocks than the batch reserved");
  FBS_CUDA(cudaMemcpyAsync(b->d_eps_tab, et.data(), et.size() * sizeof(int4),
                           cudaMemcpyHostToDevice, b->s));
  FBS_CUDA(cudaMemcpyAsync(b->d_gb_tab, gt.data(), gt.size() * sizeof(int2),
                           cudaMemcpyHostToDevice, b->s));
  FBS_CUDA(cudaMemcpyAsync(b->d_nblk, nblk.data(), nblk.size() * sizeof(int),
                           cudaMemcpyHostToDevice, b->s));
  FBS_CUDA(cudaStreamSynchronize(b->s));
  FBS_CUDA(prepare_batch_kernels(b->max_N, gb_block));
  b->n_eps = (int)et.size();
  b->n_gb = (int)gt.size();
  b->eps_block = eps_block;
  b->gb_block = gb_block;
  for (int c = 0; c < b->C; ++c) b->views[c]->nblk = nblk[c];
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  return FBS_OK;
}

cudaError_t batch_sweeps_direct(fbs_batch* b, int64_t n_iter) {
  cudaError_t e = launch_seg_begin_batch(b->d_pf, b->C, b->s);
  for (int64_t i = 0; i < n_iter && e == cudaSuccess; ++i) {
    e = launch_eps_f32_batch(b->d_mc, b->d_pf, b->d_eps_tab, b->n_eps, b->eps_block, (int)i, b->s);
    if (e == cudaSuccess)
      e = launch_gb_f32_batch(b->d_mc, b->d_pf, b->d_gb_tab, b->n_gb, b->gb_block, b->max_N,
                              (int)i, b->s);
    if (e == cudaSuccess) e = launch_hyper_batch(b->d_mc, b->d_pf, b->d_nblk, b->C, b->s);
    if (e == cudaSuccess && b->three_level)
      e = launch_top_level(b->d_mc, b->d_pf, b->C, b->d_top, b->d_top_trace, b->s);
  }
  return e;
}

cudaError_t batch_capture(fbs_batch* b) {
  cudaError_t e;
  if ((e = launch_seg_begin_batch(b->d_pf, b->C, b->s)) != cudaSuccess) return e;
  for (int i = 0; i < b->seg; ++i) {
    e = launch_eps_f32_batch(b->d_mc, b->d_pf, b->d_eps_tab, b->n_eps, b->eps_block, i, b->s);
    if (e != cudaSuccess) return e;
    if (i > 0 && (e = cudaStreamWaitEvent(b->s, b->ev_h, 0)) != cudaSuccess) return e;
    e = launch_gb_f32_batch(b->d_mc, b->d_pf, b->d_gb_tab, b->n_gb, b->gb_block, b->max_N, i,
                            b->s);
    if (e != cudaSuccess) return e;
    if ((e = cudaEventRecord(b->ev_g, b->s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(b->s2, b->ev_g, 0)) != cudaSuccess) return e;
    if ((e = launch_hyper_batch(b->d_mc, b->d_pf, b->d_nblk, b->C, b->s2)) != cudaSuccess)
      return e;
    // the top level of sweep i follows the datasets' hyperparameters on the same
    // stream; the next hyper launch reads it
    if (b->three_level &&
        (e = launch_top_level(b->d_mc, b->d_pf, b->C, b->d_top, b->d_top_trace, b->s2)) !=
            cudaSuccess)
      return e;
    if ((e = cudaEventRecord(b->ev_h, b->s2)) != cudaSuccess) return e;
  }
  return cudaStreamWaitEvent(b->s, b->ev_h, 0);
}

}  // namespace

extern "C" {

int fbs_batch_init(fbs_batch** out, int C, const fbs_dataset* sets, const fbs_options* opt,
                   void* stream) {
  g_err.clear();
  if (!out) return fail(FBS_E_ARG, "out is NULL");
  *out = nullptr;
  if (C < 1 || !sets) return fail(FBS_E_ARG, "need C >= 1 datasets");
  fbs_options d;
  fbs_default_options(&d);
  d.precision = FBS_F32;
  const fbs_options* o = opt ? opt : &d;
  int rc = check_opts(o);
  if (rc) return rc;
  if (o->precision != FBS_F32) return fail(FBS_E_ARG, "batches run the FBS_F32 form");
  fbs_batch* b = new fbs_batch();
  b->C = C;
  b->opt = *o;
  b->user = (cudaStream_t)stream;
  b->seg = o->graph_segment > 0 ? o->graph_segment : 100;
  b->mcs.resize(C);
  b->pfs.resize(C);
  b->G.resize(C);
  b->N.resize(C);
  std::vector<double> pinv((size_t)C * kMaxL * kMaxN);
  std::vector<LayoutF32> lay(C);
  std::vector<size_t> off(C);
  std::vector<char> integral(C);
  size_t total = 0;
  for (int c = 0; c < C; ++c) {
    const fbs_dataset& ds = sets[c];
    bool integ = false;
    rc = build_model(ds.y, ds.N, ds.G, ds.X, ds.L, ds.h, &ds.priors, o, ds.seed, ds.chain,
                     b->mcs[c], pinv.data() + (size_t)c * kMaxL * kMaxN, &integ);
    if (rc) {
      g_err = "dataset " + std::to_string(c) + ": " + g_err;
      batch_release(b);
      return rc;
    }
    integral[c] = integ;
    b->G[c] = ds.G;
    b->N[c] = ds.N;
    b->max_N = std::max(b->max_N, ds.N);
    lay[c] = make_layout_f32(ds.N, ds.G, ds.L, (ds.G + 31) / 32, o->trace_cap,
                             b->mcs[c].trace_beta);
    off[c] = total;
    total += align256(lay[c].total);
    b->eps_cap += (size_t)ds.N * ((ds.G + 127) / 128);
    b->gb_cap += (size_t)((ds.G + 31) / 32);
  }
  cudaError_t e;
  auto bail = [&](int code, const std::string& msg) {
    batch_release(b);
    return fail(code, msg);
  };
  if ((e = cudaStreamCreateWithFlags(&b->s, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&b->s2, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&b->ev_g, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&b->ev_h, cudaEventDisableTiming)) != cudaSuccess)
    return bail(FBS_E_CUDA, std::string("stream/event creation: ") + cudaGetErrorString(e));
  if ((e = cudaMalloc((void**)&b->ws, total + 256)) != cudaSuccess ||
      (e = cudaMalloc((void**)&b->d_mc, sizeof(ModelConst) * C)) != cudaSuccess ||
      (e = cudaMalloc((void**)&b->d_pf, sizeof(DevPtrsF32) * C)) != cudaSuccess ||
      (e = cudaMalloc((void**)&b->d_nblk, sizeof(int) * C)) != cudaSuccess ||
      (e = cudaMalloc((void**)&b->d_eps_tab, sizeof(int4) * b->eps_cap)) != cudaSuccess ||
      (e = cudaMalloc((void**)&b->d_gb_tab, sizeof(int2) * b->gb_cap)) != cudaSuccess)
    return bail(e == cudaErrorMemoryAllocation ? FBS_E_OOM : FBS_E_CUDA,
                std::string("cudaMalloc: ") + cudaGetErrorString(e));
  if ((e = cudaEventRecord(b->ev_in, b->user)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(b->s, b->ev_in, 0)) != cudaSuccess)
    return bail(FBS_E_CUDA, cudaGetErrorString(e));
  if ((e = prepare_gene_kernel_f32(b->max_N, 128)) != cudaSuccess)
    return bail(FBS_E_CUDA, cudaGetErrorString(e));
  for (int c = 0; c < C; ++c) {
    const fbs_dataset& ds = sets[c];
    char* base = b->ws + off[c];
    fbs_handle* v = new fbs_handle();
    b->views.push_back(v);
    v->is_view = true;
    v->mc = b->mcs[c];
    v->prec = FBS_F32;
    v->opt = *o;
    v->lay32 = lay[c];
    v->trace_cap = o->trace_cap;
    v->x_integral = integral[c];
    v->user = b->user;
    v->s = b->s;
    carve_f32(base, lay[c], b->mcs[c].trace_beta, v->pf, v->p);
    b->pfs[c] = v->pf;
    if ((e = cudaEventCreateWithFlags(&v->ev_in, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&v->ev_out, cudaEventDisableTiming)) != cudaSuccess)
      return bail(FBS_E_CUDA, cudaGetErrorString(e));
    int32_t* y_raw = (int32_t*)v->pf.mom_eps;
    double* d_pinv = (double*)(base + lay[c].pinv);
    if ((e = cudaMemcpyAsync(y_raw, ds.y, (size_t)ds.N * ds.G * sizeof(int32_t),
                             cudaMemcpyHostToDevice, b->s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d_pinv, pinv.data() + (size_t)c * kMaxL * kMaxN,
                             sizeof(double) * kMaxL * kMaxN, cudaMemcpyHostToDevice, b->s)) !=
            cudaSuccess ||
        (e = cudaMemsetAsync(v->p.counters, 0,
                             kCounterCopies * FBS_NUM_COUNTERS * sizeof(unsigned long long),
                             b->s)) != cudaSuccess ||
        (e = cudaMemsetAsync(v->p.hyp, 0, sizeof(Hyper), b->s)) != cudaSuccess ||
        (e = launch_init_run(v->p.hyp, o->trace_cap, b->s)) != cudaSuccess ||
        (e = launch_init_f32(v->mc, v->pf, y_raw, 1, d_pinv, o->w0, 1, b->s)) != cudaSuccess ||
        (e = launch_init_hyper(v->mc, v->p.hyp, nullptr, v->pf.beta, o->w0, 1, b->s)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(b->s)) != cudaSuccess)
      return bail(FBS_E_CUDA, "dataset " + std::to_string(c) + " initialisation: " +
                                  cudaGetErrorString(e));
  }
  if ((e = cudaMemcpyAsync(b->d_mc, b->mcs.data(), sizeof(ModelConst) * C,
                           cudaMemcpyHostToDevice, b->s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(b->d_pf, b->pfs.data(), sizeof(DevPtrsF32) * C,
                           cudaMemcpyHostToDevice, b->s)) != cudaSuccess)
    return bail(FBS_E_CUDA, cudaGetErrorString(e));
  rc = batch_tables(b, 256, 128);
  if (rc) {
    std::string m = g_err;
    return bail(rc, m);
  }
  if ((e = cudaEventRecord(b->ev_out, b->s)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(b->user, b->ev_out, 0)) != cudaSuccess)
    return bail(FBS_E_CUDA, cudaGetErrorString(e));
  *out = b;
  return FBS_OK;
}

int fbs_batch_run(fbs_batch* b, int64_t n_iter, int64_t burnin, int64_t thin) {
  if (!b) return fail(FBS_E_ARG, "batch is NULL");
  if (n_iter < 0 || burnin < 0 || thin < 1)
    return fail(FBS_E_ARG, "need n_iter >= 0, burnin >= 0, thin >= 1");
  if (n_iter == 0) return FBS_OK;
  FBS_CUDA(cudaEventRecord(b->ev_in, b->user));
  FBS_CUDA(cudaStreamWaitEvent(b->s, b->ev_in, 0));
  FBS_CUDA(launch_set_run_batch(b->d_pf, b->C, burnin, burnin / 2, thin, b->s));
  int64_t left = n_iter;
  if (left >= b->seg) {
    if (!b->exec) {
      cudaGraph_t graph = nullptr;
      FBS_CUDA(cudaStreamBeginCapture(b->s, cudaStreamCaptureModeThreadLocal));
      cudaError_t ce = batch_capture(b);
      if (ce != cudaSuccess) {
        cudaStreamEndCapture(b->s, &graph);
        if (graph) cudaGraphDestroy(graph);
        return fail(FBS_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
      }
      FBS_CUDA(cudaStreamEndCapture(b->s, &graph));
      cudaError_t ie = cudaGraphInstantiate(&b->exec, graph, 0);
      cudaGraphDestroy(graph);
      FBS_CUDA(ie);
    }
    while (left >= b->seg) {
      FBS_CUDA(cudaGraphLaunch(b->exec, b->s));
      left -= b->seg;
    }
  }
  if (left > 0) FBS_CUDA(batch_sweeps_direct(b, left));
  FBS_CUDA(cudaEventRecord(b->ev_out, b->s));
  FBS_CUDA(cudaStreamWaitEvent(b->user, b->ev_out, 0));
  return FBS_OK;
}

int fbs_batch_sync(fbs_batch* b) {
  if (!b) return fail(FBS_E_ARG, "batch is NULL");
  FBS_CUDA(cudaStreamSynchronize(b->s));
  for (fbs_handle* v : b->views) {
    Hyper hy;
    int rc = read_hyper(v, &hy);
    if (rc) return rc;
    if (hy.flags & kFlagNonfinite)
      return fail(FBS_E_NONFINITE, "a slice update started from a non-finite log density");
  }
  for (fbs_handle* v : b->views) {
    int rc = slice_cap_status(v);
    if (rc) return rc;
  }
  return FBS_OK;
}

fbs_handle* fbs_batch_chain(fbs_batch* b, int c) {
  if (!b || c < 0 || c >= b->C) return nullptr;
  return b->views[c];
}

int fbs_batch_set_schedule(fbs_batch* b, int eps_block, int gb_block) {
  if (!b) return fail(FBS_E_ARG, "batch is NULL");
  if ((eps_block != 128 && eps_block != 256) ||
      (gb_block != 32 && gb_block != 64 && gb_block != 128))
    return fail(FBS_E_ARG, "eps_block must be 128 or 256 and gb_block 32, 64 or 128");
  FBS_CUDA(cudaStreamSynchronize(b->s));
  return batch_tables(b, eps_block, gb_block);
}

int fbs_batch_autotune(fbs_batch* b, int sweeps, int64_t burnin, int* eps_block, int* gb_block,
                       double* ms_per_sweep) {
  if (!b || sweeps < 1 || burnin < 0) return fail(FBS_E_ARG, "need a batch, sweeps >= 1, burnin >= 0");
  const int eb[2] = {128, 256}, gbv[3] = {32, 64, 128};
  double best = 1e300;
  int be = b->eps_block, bg = b->gb_block;
  cudaEvent_t t0, t1;
  FBS_CUDA(cudaEventCreate(&t0));
  FBS_CUDA(cudaEventCreate(&t1));
  int rc = FBS_OK;
  for (int i = 0; i < 2 && rc == FBS_OK; ++i)
    for (int j = 0; j < 3 && rc == FBS_OK; ++j) {
      rc = fbs_batch_set_schedule(b, eb[i], gbv[j]);
      if (rc) break;
      cudaError_t e = launch_set_run_batch(b->d_pf, b->C, burnin, burnin / 2, 1, b->s);
      if (e == cudaSuccess) e = batch_sweeps_direct(b, 1);  // warm-up
      if (e == cudaSuccess) e = cudaEventRecord(t0, b->s);
      if (e == cudaSuccess) e = batch_sweeps_direct(b, sweeps);
      if (e == cudaSuccess) e = cudaEventRecord(t1, b->s);
      if (e == cudaSuccess) e = cudaEventSynchronize(t1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
      if (e != cudaSuccess) {
        rc = fail(FBS_E_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
        break;
      }
      if (ms / sweeps < best) {
        best = ms / sweeps;
        be = eb[i];
        bg = gbv[j];
      }
    }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if (rc) return rc;
  rc = fbs_batch_set_schedule(b, be, bg);
  if (rc) return rc;
  if (eps_block) *eps_block = be;
  if (gb_block) *gb_block = bg;
  if (ms_per_sweep) *ms_per_sweep = best;
  return FBS_OK;
}

int fbs_batch_three_level(fbs_batch* b, const fbs_top_prior* pri, const double* psi0) {
  if (!b) return fail(FBS_E_ARG, "batch is NULL");
  const int L = b->mcs[0].L;
  auto pos = [](double v) { return isfinite(v) && v > 0.0; };
  if (pri) {
    for (int c = 1; c < b->C; ++c)
      if (b->mcs[c].L != L) return fail(FBS_E_ARG, "a three-level model needs the same L in every dataset");
    if (!pos(pri->a_b) || !pos(pri->b_b)) return fail(FBS_E_ARG, "a_b and b_b must be finite and > 0");
    if (!pri->e) return fail(FBS_E_ARG, "e is NULL");
    for (int l = 0; l < L; ++l)
      if (!pos(pri->e[l])) return fail(FBS_E_ARG, "e_l must be finite and > 0");
    if (psi0) {
      if (!pos(psi0[0])) return fail(FBS_E_ARG, "psi0[0] (b) must be finite and > 0");
      for (int l = 0; l < L; ++l)
        if (!isfinite(psi0[1 + l])) return fail(FBS_E_ARG, "psi0 has a non-finite m_l");
    }
  }
  FBS_CUDA(cudaStreamSynchronize(b->s));
  if (pri) {
    const long long cap = b->opt.trace_cap;
    if (!b->d_top) FBS_CUDA(cudaMalloc((void**)&b->d_top, sizeof(TopLevel)));
    if (cap > 0 && !b->d_top_trace)
      FBS_CUDA(cudaMalloc((void**)&b->d_top_trace, (size_t)cap * (L + 1) * sizeof(double)));
    TopLevel t;
    memset(&t, 0, sizeof(t));
    t.psi[0] = psi0 ? psi0[0] : pri->a_b / pri->b_b;
    for (int l = 0; l < L; ++l) {
      t.psi[1 + l] = psi0 ? psi0[1 + l] : 0.0;
      t.e2[l] = pri->e[l] * pri->e[l];
    }
    t.trace_cap = cap > 0 ? cap : 0;
    t.a_b = pri->a_b;
    t.b_b = pri->b_b;
    t.seed_lo = (uint32_t)(pri->seed & 0xffffffffu);
    t.seed_hi = (uint32_t)(pri->seed >> 32);
    t.L = L;
    t.K = b->C;
    FBS_CUDA(cudaMemcpyAsync(b->d_top, &t, sizeof(t), cudaMemcpyHostToDevice, b->s));
  }
  b->three_level = pri != nullptr;
  double* d_psi = pri ? reinterpret_cast<double*>(reinterpret_cast<char*>(b->d_top) +
                                                   offsetof(TopLevel, psi))
                     : nullptr;
  for (int c = 0; c < b->C; ++c) b->pfs[c].psi = d_psi;
  FBS_CUDA(cudaMemcpyAsync(b->d_pf, b->pfs.data(), sizeof(DevPtrsF32) * b->C,
                           cudaMemcpyHostToDevice, b->s));
  FBS_CUDA(cudaStreamSynchronize(b->s));
  if (b->exec) {  // the captured segment changes
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  return FBS_OK;
}

int fbs_batch_top_level(fbs_batch* b, double* psi, double* mean, double* msq, int64_t* count,
                        int64_t max_rows, double* trace, int64_t* rows, int64_t* gamma_caps) {
  if (!b) return fail(FBS_E_ARG, "batch is NULL");
  if (!b->three_level) return fail(FBS_E_ARG, "the batch is not a three-level model");
  if (max_rows < 0) return fail(FBS_E_ARG, "max_rows must be >= 0");
  FBS_CUDA(cudaStreamSynchronize(b->s));
  TopLevel t;
  FBS_CUDA(cudaMemcpy(&t, b->d_top, sizeof(t), cudaMemcpyDeviceToHost));
  const int n = t.L + 1;
  if (psi) memcpy(psi, t.psi, n * sizeof(double));
  if (mean) memcpy(mean, t.m_psi, n * sizeof(double));
  if (msq) memcpy(msq, t.q_psi, n * sizeof(double));
  if (count) *count = t.n_mom;
  if (gamma_caps) *gamma_caps = (int64_t)t.gamma_caps;
  const long long r = t.trace_rows < max_rows ? t.trace_rows : max_rows;
  if (trace && r > 0)
    FBS_CUDA(cudaMemcpy(trace, b->d_top_trace, (size_t)r * n * sizeof(double),
                        cudaMemcpyDeviceToHost));
  if (rows) *rows = trace ? r : 0;
  return FBS_OK;
}

void fbs_batch_free(fbs_batch* b) { batch_release(b); }

}  // extern "C"
