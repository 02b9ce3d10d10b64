// fbs_learned.cu -- the learned proposal for the beta_g block: the weight
// image and the stand-alone pass of the multilayer perceptron that maps the
// per-gene features to a Gaussian (the tensor-core code is in fbs_tc.cuh), the
// collection of training pairs from the plain sampler, and the training
// kernels (a fused per-block minibatch forward/backward pass with the Gaussian
// negative log-likelihood head, then the gradient reduction with Adam).  The
// move that uses the proposal, and the in-sweep network pass fused into the
// gamma/beta kernel, are in fbs_gene_f32.cu.
//
// Network: features (4L+1) -> 64 -> GELU -> 64 -> GELU -> L + L(L+1)/2 outputs:
// mean mu (L), log of the Cholesky diagonal (L), sub-diagonal entries in row
// order.  GELU is the tanh form of Hendrycks & Gimpel (2016).  Parameters are
// one flat FP32 array W1 [64][F], b1 [64], W2 [64][64], b2 [64], W3 [K][64],
// b3 [K]; inference (tensor cores) reads them as split BF16 operands.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fbs_common.cuh"
#include "fbs_kernels.h"
#include "fbs_rng.cuh"
#include "fbs_tc.cuh"

namespace fbs {

// GELU (tanh form) and its derivative at x from one tanh:
// a = x (1 + t) / 2, gd = (1 + t) / 2 + x (1 - t^2) u'(x) / 2, t = tanh(u(x)),
// u(x) = sqrt(2/pi) (x + 0.044715 x^3).  t = 1 - 2 / (1 + e^{2u}) from the fast
// exponential and division, as inference evaluates GELU (absolute error of t
// about 1e-7; |u| is clamped at 15, where tanh is 1 in FP32).
__device__ __forceinline__ void gelu_and_grad_f(float x, float* a, float* gd) {
  const float u = fminf(fmaxf(kSqrt2OverPi * (x + 0.044715f * x * x * x), -15.0f), 15.0f);
  const float t = 1.0f - __fdividef(2.0f, 1.0f + __expf(2.0f * u));
  const float du = kSqrt2OverPi * (1.0f + 3.0f * 0.044715f * x * x);
  *a = 0.5f * x * (1.0f + t);
  *gd = 0.5f * (1.0f + t) + 0.5f * x * (1.0f - t * t) * du;
}

__host__ __device__ inline int mlp_n_params(int F, int K) {
  return kMlpHidden * F + kMlpHidden + kMlpHidden * kMlpHidden + kMlpHidden + K * kMlpHidden + K;
}


// The weight image the kernel copies into shared memory: W1 [64][2 k1],
// W2 [64][128], W3 [n3][128] as split canonical operands (zero padding), then
// the biases b1, b2, b3 (n3, zero padded) in FP32.
__global__ void k_pack_image(const float* __restrict__ w, int L, uint8_t* __restrict__ img) {
  const TcShape t = tc_shape(L);
  const int H = kMlpHidden, F = t.F, K = t.K;
  const float* W1 = w;
  const float* b1 = W1 + H * F;
  const float* W2 = b1 + H;
  const float* b2 = W2 + H * H;
  const float* W3 = b2 + H;
  const float* b3 = W3 + K * H;
  const int n1 = H * t.k1, n2 = H * H, n3 = t.n3 * H, nb = 2 * H + t.n3;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n1 + n2 + n3 + nb;
       i += gridDim.x * blockDim.x) {
    uint8_t* base;
    int r, c, kin;
    float v;
    if (i < n1) {
      r = i / t.k1, c = i % t.k1, kin = t.k1, base = img;
      v = c < F ? W1[r * F + c] : 0.0f;
    } else if (i < n1 + n2) {
      const int j = i - n1;
      r = j / H, c = j % H, kin = H, base = img + t.off_w2;
      v = W2[r * H + c];
    } else if (i < n1 + n2 + n3) {
      const int j = i - n1 - n2;
      r = j / H, c = j % H, kin = H, base = img + t.off_w3;
      v = r < K ? W3[r * H + c] : 0.0f;
    } else {
      const int j = i - n1 - n2 - n3;
      float* bb = (float*)(img + t.off_b);
      bb[j] = j < H ? b1[j] : (j < 2 * H ? b2[j - H] : (j - 2 * H < K ? b3[j - 2 * H] : 0.0f));
      continue;
    }
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    *(__nv_bfloat16*)(base + canon_off(r, c, 2 * kin)) = hi;
    *(__nv_bfloat16*)(base + canon_off(r, kin + c, 2 * kin)) = lo;
  }
}

constexpr int kTcThreads = 128;  // one thread per gene of a tile (= TMEM lane)

// Stand-alone network pass (fbs_proposal_outputs, fbs_proposal_step): persistent
// over tiles of 128 genes, writes the outputs [K][G] of the genes that may use
// the network's proposal.  A wait that gives up sets kFlagTimeout, and the
// block frees its tensor memory and returns.
__global__ void __launch_bounds__(kTcThreads) k_proposal_tc(ModelConst mc, DevPtrsF32 p,
                                                           const uint8_t* __restrict__ img_g,
                                                           float* __restrict__ out, int ntiles) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_abort;
  const TcShape t = tc_shape(mc.L);
  if (threadIdx.x == 0) s_abort = 0;
  TcBlock c;
  tc_begin(c, bars, &tmem_slot, img_g, sm, t.bytes, p.tc_polls);
  if (!c.w_ok) s_abort = 1;
  __syncthreads();
  for (int tile = blockIdx.x; tile < ntiles && !s_abort; tile += gridDim.x) {
    const int g = tile * 128 + (int)threadIdx.x;
    if (!tc_tile(c, mc, p, t, sm, g, net_gene(p, g, mc.G), out, (size_t)mc.G, g, &s_abort))
      break;
  }
  tc_end(c, s_abort != 0, &p.hyp->flags);
}

// Training pairs from the current state of every gene: features [M][F] and
// beta [M][L] rows starting at `row`.
__global__ void k_collect_f32(ModelConst mc, DevPtrsF32 p, float* __restrict__ feat,
                              float* __restrict__ beta, long long row) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= mc.G) return;
  const int F = 4 * mc.L + 1, L = mc.L;
  float f[kMaxFeat];
  gene_features(mc, p, g, p.hyp, f);
  const size_t r = (size_t)(row + g);
  for (int i = 0; i < F; ++i) feat[r * F + i] = f[i];
  for (int l = 0; l < L; ++l) beta[r * L + l] = p.beta[(size_t)l * mc.G + g];
}

// ---------------------------------------------------------------- training

// Column means and scales of the training pairs, in FP64: block c < F takes
// feature column c, block F + l takes beta column l.  A beta column's scale is
// its standard deviation, or 1 when it is constant to within 1e-6 of its size.
// A feature column's scale is its standard deviation but at least
// kFeatScaleFloor: theta and log sigma, the same for every gene of a sweep, vary
// across the collected sweeps only by their posterior spread (~1e-3), and
// dividing by that would let the network fit noise with weights that, in raw
// coordinates, react strongly to the small moves of theta and sigma during
// sampling.  st = [mean_f (F), scale_f (F), mean_beta (L), scale_beta (L)].
constexpr double kFeatScaleFloor = 0.1;

__global__ void k_col_stats(const float* __restrict__ feat, const float* __restrict__ beta,
                            long long M, int F, int L, float* __restrict__ st) {
  const int c = blockIdx.x;
  const float* a = c < F ? feat + c : beta + (c - F);
  const int stride = c < F ? F : L;
  double s1 = 0.0, s2 = 0.0;
  for (long long m = threadIdx.x; m < M; m += blockDim.x) {
    const double x = a[(size_t)m * stride];
    s1 += x;
    s2 += x * x;
  }
  __shared__ double r1[32], r2[32];
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_down_sync(0xffffffffu, s1, o);
    s2 += __shfl_down_sync(0xffffffffu, s2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    r1[threadIdx.x >> 5] = s1;
    r2[threadIdx.x >> 5] = s2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t1 = 0.0, t2 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      t1 += r1[w];
      t2 += r2[w];
    }
    const double mean = t1 / (double)M;
    const double var = fmax(t2 / (double)M - mean * mean, 0.0);
    const double tol = 1e-6 * (1.0 + fabs(mean));
    const double sc = c < F ? fmax(sqrt(var), kFeatScaleFloor) : (var > tol * tol ? sqrt(var) : 1.0);
    if (c < F) {
      st[c] = (float)mean;
      st[F + c] = (float)sc;
    } else {
      st[2 * F + (c - F)] = (float)mean;
      st[2 * F + L + (c - F)] = (float)sc;
    }
  }
}

// Moves the parameters between the standardised coordinates training uses and
// the raw coordinates of features and beta that inference reads; the network's
// function is unchanged.  With f = m_f + s_f f', beta = m_b + S beta' (S =
// diag s_b): the first layer takes W1 / s_f and b1 - W1 m_f / s_f; the mean rows
// of the last layer scale by s_b,i and their bias adds m_b,i; the log-diagonal
// rows add log s_b,i to their bias; the sub-diagonal row (i, j) scales by s_b,i,
// so that the Cholesky factor becomes S C.  to_raw = 0 applies the inverse.
// One block: thread j < 64 takes row j of W1, thread 64 + k row k of W3.
__global__ void k_fold(float* __restrict__ w, const float* __restrict__ st, int L, int to_raw) {
  const int F = 4 * L + 1, K = L + L * (L + 1) / 2, H = kMlpHidden;
  float* W1 = w;
  float* b1 = W1 + H * F;
  float* W3 = b1 + H + H * H + H;
  float* b3 = W3 + K * H;
  const float* mf = st;
  const float* sf = st + F;
  const float* mb = st + 2 * F;
  const float* sb = st + 2 * F + L;
  const int t = threadIdx.x;
  if (t < H) {
    float acc = 0.0f;
    for (int i = 0; i < F; ++i) {
      float& a = W1[t * F + i];
      if (to_raw) {
        a = a / sf[i];
        acc += a * mf[i];
      } else {
        acc += a * mf[i];
        a = a * sf[i];
      }
    }
    b1[t] = to_raw ? b1[t] - acc : b1[t] + acc;
  } else if (t < H + K) {
    const int k = t - H;
    int row = -1;  // beta index whose scale multiplies this output
    float add = 0.0f;
    if (k < L) {
      row = k;
      add = mb[k];
    } else if (k < 2 * L) {
      add = logf(sb[k - L]);
    } else {
      int q = 2 * L;
      for (int i = 1; i < L && row < 0; ++i)
        for (int j = 0; j < i; ++j, ++q)
          if (q == k) {
            row = i;
            break;
          }
    }
    const float sc = row >= 0 ? sb[row] : 1.0f;
    if (to_raw) {
      for (int j = 0; j < H; ++j) W3[k * H + j] *= sc;
      b3[k] = b3[k] * sc + add;
    } else {
      for (int j = 0; j < H; ++j) W3[k * H + j] /= sc;
      b3[k] = (b3[k] - add) / sc;
    }
  }
}

// ---------------------------------------------------------------- training step (tensor cores)
//
// One training step's forward and backward pass for 128 minibatch rows per
// block (thread t = row t = tensor-memory lane t), every matrix product on the
// tensor cores (tcgen05, BF16 operands split as x = hi + lo, hi*hi + lo*hi +
// hi*lo accumulated in FP32, about 16 significant bits per operand):
//   forward   Z1 = X W1^T, A1 = gelu(Z1 + b1); Z2 = A1 W2^T, A2 = gelu(Z2 + b2);
//             O = A2 W3^T + b3; the Gaussian head gives the loss and dO = dL/dO
//   backward  G2 = (dO W3) . gelu'(Z2 + b2); G1 = (G2 W2) . gelu'(Z1 + b1)
//   weights   one product of [G2 | A2]^T (128 rows) with [A1 | X, 1 | dO] over
//             the block's rows gives dW2, db2 (the column of ones appended to
//             X) and dW3^T; a second, of [X, 1 | ..]^T with G1, gives dW1^T and
//             db1; db3 is a warp sum of dO.
// The forward and backward products read K-major operands (one row per
// thread); the weight-gradient products read the same bytes as MN-major
// operands (K = the block's rows), and the backward products read the weight
// images as MN-major operands, so nothing is transposed.  The block's sums
// over its rows of every parameter gradient and of the loss go to
// part[block][np + 1] in parameter order (the loss last); rows past Bsz take
// no part.  Every wait on the tensor cores is bounded by `polls`; a wait that
// gives up sets kFlagTimeout in *flags and the block returns after draining.
//
// Shared memory, in 16-byte chunks of 8 BF16 values, each operand row a hi
// half then a lo half:
//   W1 [64][k1], W2 [64][64], W3 [n3][64]    weight images (K-major)
//   b1 [64], b2 [64], b3 [n3]                FP32
//     (the image: one bulk copy of img, which the previous step's Adam update
//     or k_pack_train_image wrote)
//   bufF rows  [A1 (64) | X, 1 (k1) | dO (n3)]
//   bufG rows  [G2 (64) | A2 (64)]
//   bufG1 rows [G1 (64)]
// Tensor memory (512 columns): Z1 at 0 and Z2 at 64 (each replaced by GELU's
// derivative at Z + b in its forward epilogue, for the backward pass), O 128,
// dO W3 192, G2 W2 256, the first weight-gradient product 320 (64 + k1 + n3
// columns), the second 128.
struct TrainTc {
  int F, K, k1, n3, cx, co, half;  // half: chunks in a half row of bufF
  uint32_t sbo_w1, sbo_f;          // 8-row group strides of W1 and bufF
  uint32_t off_w2, off_w3, off_b, img_bytes, off_f, off_g, off_g1, bytes;
};

__host__ __device__ inline TrainTc train_tc_shape(int L) {
  TrainTc t;
  t.F = 4 * L + 1;
  t.K = L + L * (L + 1) / 2;
  t.k1 = (t.F + 1 + 15) & ~15;  // the features and the column of ones
  t.n3 = (t.K + 15) & ~15;
  t.cx = t.k1 / 8;
  t.co = t.n3 / 8;
  t.half = 8 + t.cx + t.co;
  t.sbo_w1 = (uint32_t)(2 * t.cx * 128);
  t.sbo_f = (uint32_t)(2 * t.half * 128);
  t.off_w2 = 8 * t.sbo_w1;
  t.off_w3 = t.off_w2 + 8 * 2048;
  t.off_b = t.off_w3 + (uint32_t)(t.n3 / 8) * 2048;
  t.img_bytes = t.off_b + (uint32_t)(128 + t.n3) * 4;  // a multiple of 16
  t.off_f = (t.img_bytes + 1023) & ~1023u;
  t.off_g = t.off_f + 16 * t.sbo_f;  // the second weight-gradient product reads up to
  t.off_g1 = t.off_g + 16 * 4096;    // 24 - half chunks past bufF, inside bufG
  t.bytes = t.off_g1 + 16 * 2048;
  return t;
}

// Parameter p (value w) into the training kernel's weight image (the bytes
// [0, img_bytes) of its shared memory): weights as split BF16 at their
// canonical positions, biases in FP32.  The padding (W1 columns from F, W3 rows
// and b3 entries from K) is zero from the image's allocation.
__device__ __forceinline__ void train_img_put(uint8_t* img, const TrainTc& t, int p, float w) {
  constexpr int H = kMlpHidden;
  const int F = t.F, K = t.K;
  const int ob1 = H * F, oW2 = ob1 + H, ob2 = oW2 + H * H, oW3 = ob2 + H, ob3 = oW3 + K * H;
  float* bias = reinterpret_cast<float*>(img + t.off_b);
  int r, c, lo;  // row, column, chunk offset of the lo half
  uint32_t base, sbo;
  if (p < ob1) {
    r = p / F, c = p % F, base = 0, sbo = t.sbo_w1, lo = t.cx;
  } else if (p < oW2) {
    bias[p - ob1] = w;
    return;
  } else if (p < ob2) {
    r = (p - oW2) / H, c = (p - oW2) % H, base = t.off_w2, sbo = 2048, lo = 8;
  } else if (p < oW3) {
    bias[H + p - ob2] = w;
    return;
  } else if (p < ob3) {
    r = (p - oW3) / H, c = (p - oW3) % H, base = t.off_w3, sbo = 2048, lo = 8;
  } else {
    bias[2 * H + p - ob3] = w;
    return;
  }
  const __nv_bfloat16 hi = __float2bfloat16_rn(w);
  const __nv_bfloat16 lw = __float2bfloat16_rn(w - __bfloat162float(hi));
  uint8_t* row = img + base + (size_t)(r >> 3) * sbo + (r & 7) * 16 + (c & 7) * 2;
  *(__nv_bfloat16*)(row + (c >> 3) * 128) = hi;
  *(__nv_bfloat16*)(row + ((c >> 3) + lo) * 128) = lw;
}

__global__ void k_pack_train_image(const float* __restrict__ w, int L, uint8_t* __restrict__ img) {
  const TrainTc t = train_tc_shape(L);
  const int np = mlp_n_params(t.F, t.K);
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x)
    train_img_put(img, t, p, w[p]);
}

constexpr uint32_t kTrainTmemCols = 512;
constexpr int kTrainOutPad = (kMaxOut + 15) & ~15;

// Writes 32 FP32 columns of this thread's tensor-memory lane and waits for the
// store.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
      "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
      "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]),
      "f"(v[8]), "f"(v[9]), "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]),
      "f"(v[15]), "f"(v[16]), "f"(v[17]), "f"(v[18]), "f"(v[19]), "f"(v[20]), "f"(v[21]),
      "f"(v[22]), "f"(v[23]), "f"(v[24]), "f"(v[25]), "f"(v[26]), "f"(v[27]), "f"(v[28]),
      "f"(v[29]), "f"(v[30]), "f"(v[31])
      : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Gaussian head, per row: loss = |u|^2 / 2 + sum log C_ll with C u = beta - mu;
// dL/dout (scaled by sc = 1/Bsz): d mu = -v, d logC_ii = 1 - v_i u_i C_ii,
// d C_ij = -v_i u_j (i > j), where C^T v = u.  o holds the outputs on entry and
// dL/dout on return.
// LL columns, every index a compile-time constant (registers only).
template <int LL>
__device__ __forceinline__ void nll_row_t(float* o, const float* y, float sc, float* loss) {
  float C[LL][LL], u[LL], v[LL];
#pragma unroll
  for (int i = 0; i < LL; ++i) {
#pragma unroll
    for (int j = 0; j < LL; ++j) C[i][j] = 0.0f;
  }
  int k = 2 * LL;
#pragma unroll
  for (int i = 0; i < LL; ++i) {
    C[i][i] = expf(o[LL + i]);
#pragma unroll
    for (int j = 0; j < i; ++j) C[i][j] = o[k++];
  }
  float ls = 0.0f;
#pragma unroll
  for (int i = 0; i < LL; ++i) {
    float s = y[i] - o[i];
#pragma unroll
    for (int j = 0; j < i; ++j) s -= C[i][j] * u[j];
    u[i] = s / C[i][i];
    ls += 0.5f * u[i] * u[i] + o[LL + i];
  }
#pragma unroll
  for (int i = LL - 1; i >= 0; --i) {
    float s = u[i];
#pragma unroll
    for (int j = i + 1; j < LL; ++j) s -= C[j][i] * v[j];
    v[i] = s / C[i][i];
  }
  k = 2 * LL;
#pragma unroll
  for (int i = 0; i < LL; ++i) {
#pragma unroll
    for (int j = 0; j < i; ++j) o[k++] = -v[i] * u[j] * sc;
  }
#pragma unroll
  for (int i = 0; i < LL; ++i) {
    o[LL + i] = (1.0f - v[i] * u[i] * C[i][i]) * sc;
    o[i] = -v[i] * sc;
  }
  *loss = ls;
}

// The head of the training step for LL columns: the outputs O + b3 from tensor
// memory, the loss and dO (zero for rows past the batch and columns past K),
// dO split into bufF, and the warp sums of dO (s_db3[warp]) and of the loss.
template <int LL>
__device__ __forceinline__ void train_head(uint32_t taddr, const float* b3, const float* y,
                                           bool row_ok, float sc, uint8_t* bF, uint32_t sbo_f,
                                           int ch_hi, int ch_lo, float* db3w, float* lossw) {
  constexpr int K = LL + LL * (LL + 1) / 2;
  constexpr int n3 = (K + 15) & ~15;
  const int tid = threadIdx.x, lane = tid & 31;
  float o[n3];
#pragma unroll
  for (int c0 = 0; c0 < n3; c0 += 16) {
    float v[16];
    tmem_ld16(taddr + (uint32_t)c0, v);
#pragma unroll
    for (int i = 0; i < 16; ++i) o[c0 + i] = v[i] + b3[c0 + i];
  }
  float loss = 0.0f;
  if (row_ok) nll_row_t<LL>(o, y, sc, &loss);
#pragma unroll
  for (int k = 0; k < n3; ++k)
    if (!row_ok || k >= K) o[k] = 0.0f;
#pragma unroll
  for (int q = 0; q < n3 / 8; ++q) store_split8_ch(bF, sbo_f, tid, ch_hi + q, ch_lo + q, o + 8 * q);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    float v = o[k];
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) v += __shfl_xor_sync(0xffffffffu, v, sh);
    if (lane == 0) db3w[k] = v;
  }
#pragma unroll
  for (int sh = 16; sh > 0; sh >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, sh);
  if (lane == 0) *lossw = loss;
}

// D (+)= A B^T over 16 ksteps rows of K for the three split products hi*hi,
// lo*hi, hi*lo.  Each operand: start addresses of its hi and lo halves, the
// address step per 16 rows of K, and its descriptor's leading and stride byte
// offsets.
__device__ __forceinline__ void issue_split(uint32_t d, uint32_t idesc, int ksteps, uint32_t a_hi,
                                            uint32_t a_lo, uint32_t a_step, uint32_t a_lbo,
                                            uint32_t a_sbo, uint32_t b_hi, uint32_t b_lo,
                                            uint32_t b_step, uint32_t b_lbo, uint32_t b_sbo) {
  const uint32_t pa[3] = {a_hi, a_lo, a_hi}, pb[3] = {b_hi, b_hi, b_lo};
  uint32_t acc = 0u;
#pragma unroll
  for (int q = 0; q < 3; ++q)
    for (int k = 0; k < ksteps; ++k) {
      umma_bf16(d, umma_desc_ls(pa[q] + k * a_step, a_lbo, a_sbo),
                umma_desc_ls(pb[q] + k * b_step, b_lbo, b_sbo), idesc, acc);
      acc = 1u;
    }
}

// Block barrier, then (thread 0) the products `issue` describes and a commit;
// every thread waits for their completion, and a second block barrier makes
// the outcome the same for every thread: false once any wait gave up.
template <class Issue>
__device__ __forceinline__ bool tc_run(TcBlock& c, volatile int* s_abort, Issue issue) {
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  if (*s_abort) return false;
  if (threadIdx.x == 0) {
    tc_fence_after();
    issue();
    umma_commit(c.bar_m);
  }
  c.pending = true;
  if (!mbar_wait(c.bar_m, c.ph, c.polls)) *s_abort = 1;
  else c.pending = false;
  c.ph ^= 1u;
  tc_fence_after();
  __syncthreads();
  return *s_abort == 0;
}

__global__ void __launch_bounds__(128) k_mlp_tc(
    int L, int Bsz, const float* __restrict__ fb,
    const float* __restrict__ yb, const float* __restrict__ feat,
    const float* __restrict__ beta, long long M, uint32_t seed_lo, uint32_t seed_hi,
    const TrainCtl* __restrict__ ctl, const float* __restrict__ st, float* __restrict__ part,
    const uint8_t* __restrict__ img, unsigned* __restrict__ flags, unsigned polls) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_abort;
  __shared__ float s_db3[4][kTrainOutPad];
  __shared__ float s_loss[4];
  constexpr int H = kMlpHidden;
  const TrainTc t = train_tc_shape(L);
  const int F = t.F, K = t.K, half = t.half;
  const int np = mlp_n_params(F, K);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int r0 = blockIdx.x * 128;
  const bool row_ok = tid < Bsz - r0;
  uint8_t* w1s = sm;
  uint8_t* w2s = sm + t.off_w2;
  uint8_t* w3s = sm + t.off_w3;
  float* bsm = reinterpret_cast<float*>(sm + t.off_b);
  uint8_t* bF = sm + t.off_f;
  uint8_t* bG = sm + t.off_g;
  uint8_t* bG1 = sm + t.off_g1;
  TcBlock c;
  c.polls = polls;
  c.cols = kTrainTmemCols;  // what the dealloc of tc_end frees
  c.bar_w = smem_u32(&bars[0]);
  c.bar_m = smem_u32(&bars[1]);
  c.ph = 0;
  c.pending = false;
  c.w_ok = false;
  if (tid == 0) {
    s_abort = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(c.bar_w) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(c.bar_m) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // the weight image (written by the previous step's Adam update, or packed
    // before the first step): one bulk copy, waited for before the first product
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(c.bar_w),
                 "r"(t.img_bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(sm)),
        "l"(img), "r"(t.img_bytes), "r"(c.bar_w)
        : "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(kTrainTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }

  // this thread's row: features and the column of ones (split into bufF), beta
  long long srow = 0;
  if (feat != nullptr && row_ok) {
    Rng rg(seed_lo, seed_hi, 0u, kStreamTrain, (uint32_t)(r0 + tid), (uint32_t)(ctl->t + 1));
    const long long m = (long long)(rg.u(0) * (double)M);
    srow = m >= M ? M - 1 : m;
  }
  // every load of the row first (one round of latency), then the arithmetic
  constexpr int kX = (kMaxFeat + 1 + 15) & ~15;
  float x[kX], y[kMaxL];
  {
    const float* xr = feat != nullptr ? feat + (size_t)srow * F : fb + (size_t)(r0 + tid) * F;
    const float* yr = feat != nullptr ? beta + (size_t)srow * L : yb + (size_t)(r0 + tid) * L;
#pragma unroll
    for (int f = 0; f < kX; ++f) x[f] = row_ok && f < F ? xr[f] : 0.0f;
#pragma unroll
    for (int l = 0; l < kMaxL; ++l) y[l] = row_ok && l < L ? yr[l] : 0.0f;
    if (feat != nullptr) {
#pragma unroll
      for (int f = 0; f < kX; ++f)
        if (f < F) x[f] = (x[f] - st[f]) / st[F + f];
#pragma unroll
      for (int l = 0; l < kMaxL; ++l)
        if (l < L) y[l] = (y[l] - st[2 * F + l]) / st[2 * F + L + l];
    }
#pragma unroll
    for (int f = 0; f < kX; ++f)
      if (f == F && row_ok) x[f] = 1.0f;
#pragma unroll
    for (int q = 0; q < kX / 8; ++q)
      if (q < t.cx) store_split8_ch(bF, t.sbo_f, tid, 8 + q, 8 + q + half, x + 8 * q);
  }

  c.w_ok = mbar_wait(c.bar_w, 0, c.polls);
  if (!c.w_ok) s_abort = 1;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  c.tmem = tmem_slot;
  const uint32_t tm = c.tmem, la = (uint32_t)(warp * 32) << 16;
  const uint32_t sF = smem_u32(bF), sG = smem_u32(bG), sG1 = smem_u32(bG1);
  const uint32_t sW1 = smem_u32(w1s), sW2 = smem_u32(w2s), sW3 = smem_u32(w3s);
  const uint32_t sbo_f = t.sbo_f, hb = (uint32_t)half * 128;
  const int cx = t.cx, k1 = t.k1, n3 = t.n3;
  bool ok = true;

  // ---- forward
  ok = tc_run(c, &s_abort, [&] {  // Z1 = X W1^T
    issue_split(tm, umma_idesc_bf16(128, H), k1 / 16, sF + 8 * 128, sF + 8 * 128 + hb, 256, 128,
                sbo_f, sW1, sW1 + cx * 128, 256, 128, t.sbo_w1);
  });
  if (ok) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float v[32];
      float gd[32];
      tmem_ld32(tm + la + 32 * h, v);
#pragma unroll
      for (int i = 0; i < 32; ++i) gelu_and_grad_f(v[i] + bsm[32 * h + i], &v[i], &gd[i]);
      tmem_st32(tm + la + 32 * h, gd);  // Z1 becomes gelu'(Z1 + b1)
#pragma unroll
      for (int q = 0; q < 4; ++q) store_split8_ch(bF, sbo_f, tid, 4 * h + q, 4 * h + q + half, v + 8 * q);
    }
    ok = tc_run(c, &s_abort, [&] {  // Z2 = A1 W2^T
      issue_split(tm + 64, umma_idesc_bf16(128, H), 4, sF, sF + hb, 256, 128, sbo_f, sW2,
                  sW2 + 8 * 128, 256, 128, 2048);
    });
  }
  if (ok) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float v[32];
      float gd[32];
      tmem_ld32(tm + la + 64 + 32 * h, v);
#pragma unroll
      for (int i = 0; i < 32; ++i) gelu_and_grad_f(v[i] + bsm[H + 32 * h + i], &v[i], &gd[i]);
      tmem_st32(tm + la + 64 + 32 * h, gd);  // Z2 becomes gelu'(Z2 + b2)
#pragma unroll
      for (int q = 0; q < 4; ++q) store_split8_ch(bG, 4096, tid, 8 + 4 * h + q, 24 + 4 * h + q, v + 8 * q);
    }
    ok = tc_run(c, &s_abort, [&] {  // O = A2 W3^T
      issue_split(tm + 128, umma_idesc_bf16(128, n3), 4, sG + 8 * 128, sG + 24 * 128, 256, 128,
                  4096, sW3, sW3 + 8 * 128, 256, 128, 2048);
    });
  }
  // ---- head: loss and dO (rows past Bsz: zero), dO into bufF, warp sums of dO
  if (ok) {
    static_assert(kMaxL == 8, "one case per number of columns");
    const float sc = 1.0f / (float)Bsz;
    const uint32_t ta = tm + la + 128;
    float* db3w = s_db3[warp];
    float* lw = &s_loss[warp];
    const int chh = 8 + cx, chl = 8 + cx + half;
    switch (L) {
      case 1: train_head<1>(ta, bsm + 2 * H, y, row_ok, sc, bF, sbo_f, chh, chl, db3w, lw); break;
      case 2: train_head<2>(ta, bsm + 2 * H, y, row_ok, sc, bF, sbo_f, chh, chl, db3w, lw); break;
      case 3: train_head<3>(ta, bsm + 2 * H, y, row_ok, sc, bF, sbo_f, chh, chl, db3w, lw); break;
      case 4: train_head<4>(ta, bsm + 2 * H, y, row_ok, sc, bF, sbo_f, chh, chl, db3w, lw); break;
      case 5: train_head<5>(ta, bsm + 2 * H, y, row_ok, sc, bF, sbo_f, chh, chl, db3w, lw); break;
      case 6: train_head<6>(ta, bsm + 2 * H, y, row_ok, sc, bF, sbo_f, chh, chl, db3w, lw); break;
      case 7: train_head<7>(ta, bsm + 2 * H, y, row_ok, sc, bF, sbo_f, chh, chl, db3w, lw); break;
      default: train_head<8>(ta, bsm + 2 * H, y, row_ok, sc, bF, sbo_f, chh, chl, db3w, lw); break;
    }
    ok = tc_run(c, &s_abort, [&] {  // dO W3 (W3 read as an MN-major B)
      issue_split(tm + 192, umma_idesc_bf16_mn(128, H, 0, 1), n3 / 16, sF + (8 + cx) * 128,
                  sF + (8 + cx) * 128 + hb, 256, 128, sbo_f, sW3, sW3 + 8 * 128, 4096, 2048, 128);
    });
  }
  // ---- backward
  if (ok) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float d[32], z[32];
      tmem_ld32(tm + la + 192 + 32 * h, d);
      tmem_ld32(tm + la + 64 + 32 * h, z);  // gelu'(Z2 + b2)
#pragma unroll
      for (int i = 0; i < 32; ++i) d[i] *= z[i];
#pragma unroll
      for (int q = 0; q < 4; ++q) store_split8_ch(bG, 4096, tid, 4 * h + q, 16 + 4 * h + q, d + 8 * q);
    }
    ok = tc_run(c, &s_abort, [&] {  // G2 W2 (W2 read as an MN-major B)
      issue_split(tm + 256, umma_idesc_bf16_mn(128, H, 0, 1), 4, sG, sG + 16 * 128, 256, 128,
                  4096, sW2, sW2 + 8 * 128, 4096, 2048, 128);
    });
  }
  if (ok) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float d[32], z[32];
      tmem_ld32(tm + la + 256 + 32 * h, d);
      tmem_ld32(tm + la + 32 * h, z);  // gelu'(Z1 + b1)
#pragma unroll
      for (int i = 0; i < 32; ++i) d[i] *= z[i];
#pragma unroll
      for (int q = 0; q < 4; ++q) store_split8_ch(bG1, 2048, tid, 4 * h + q, 8 + 4 * h + q, d + 8 * q);
    }
    // the weight gradients: K = the block's 128 rows, both operands MN-major
    ok = tc_run(c, &s_abort, [&] {
      issue_split(tm + 320, umma_idesc_bf16_mn(128, H + k1 + n3, 1, 1), 8, sG, sG + 16 * 128,
                  2 * 4096, 4096, 128, sF, sF + hb, 2 * sbo_f, sbo_f, 128);
      issue_split(tm + 128, umma_idesc_bf16_mn(128, H, 1, 1), 8, sF + 8 * 128,
                  sF + 8 * 128 + hb, 2 * sbo_f, sbo_f, 128, sG1, sG1 + 8 * 128, 2 * 2048, 2048,
                  128);
    });
  }
  // ---- this block's sums, in parameter order: W1 [64][F], b1, W2 [64][64], b2,
  // W3 [K][64], b3, loss
  if (ok) {
    float* out = part + (size_t)blockIdx.x * (np + 1);
    const int oW1 = 0, ob1 = H * F, oW2 = ob1 + H, ob2 = oW2 + H * H, oW3 = ob2 + H,
              ob3 = oW3 + K * H;
    if (warp < 2) {
      // first product, rows 0..63 (unit of G2): dW2 in columns 0..63, db2 in column 64 + F
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float v[32];
        tmem_ld32(tm + la + 320 + 32 * h, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) out[oW2 + tid * H + 32 * h + i] = v[i];
      }
      {
        float v[16];
        const int cb = H + (F / 16) * 16;
        tmem_ld16(tm + la + 320 + (uint32_t)cb, v);
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (cb + i == H + F) out[ob2 + tid] = v[i];
      }
      // second product, rows 0..63 (feature m of X, then the ones at m = F):
      // dW1^T and db1 in columns 0..63
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float v[32];
        tmem_ld32(tm + la + 128 + 32 * h, v);
        if (tid < F) {
#pragma unroll
          for (int i = 0; i < 32; ++i) out[oW1 + (32 * h + i) * F + tid] = v[i];
        } else if (tid == F) {
#pragma unroll
          for (int i = 0; i < 32; ++i) out[ob1 + 32 * h + i] = v[i];
        }
      }
    } else {
      // first product, rows 64..127 (unit of A2): dW3^T in columns 64 + k1 + k
      const int u = tid - H;
#pragma unroll
      for (int c0 = 0; c0 < kTrainOutPad; c0 += 16)
        if (c0 < n3) {
          float v[16];
          tmem_ld16(tm + la + 320 + (uint32_t)(H + k1 + c0), v);
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (c0 + i < K) out[oW3 + (c0 + i) * H + u] = v[i];
        }
    }
    __syncthreads();  // s_db3, s_loss (written before the last products)
    if (tid < K) out[ob3 + tid] = s_db3[0][tid] + s_db3[1][tid] + s_db3[2][tid] + s_db3[3][tid];
    if (tid == 0) out[np] = s_loss[0] + s_loss[1] + s_loss[2] + s_loss[3];
  }
  tc_end(c, s_abort != 0, flags);
}

// Adam (Kingma & Ba 2015) step sizes of the step the control block describes:
// t is the Adam step count before the step, k the step within the training
// call; the base step size decays along a cosine over the call to 5%.
__device__ __forceinline__ void adam_scalars(const TrainCtl* c, float* c1, float* c2,
                                             float* lr_t) {
  const float t1 = (float)(c->t + 1);
  *c1 = 1.0f - powf(c->b1, t1);
  *c2 = 1.0f - powf(c->b2, t1);
  *lr_t = (float)c->lr *
          (0.05f + 0.475f * (1.0f + cosf(3.14159265f * (float)c->k / (float)c->steps)));
}

// Gradient and summed loss of the whole minibatch from the blocks' partials
// (part [nblk][np + 1]), added in block order so that a step is deterministic:
// block b takes parameters 32b..32b+31, warp w the partial rows w, w + 8, ..,
// and warp 0 adds the eight warp sums in order.  With a control block it also
// applies Adam to w, m, v, writes the new w into the training kernel's weight
// image img and, in the last block to finish (ticket counter, no waiting), adds
// the loss to the last epoch's sum and advances t and k.  Does
// nothing once *flags is set (a tensor-core wait of the forward and backward
// pass gave up, so the partials are incomplete).
__global__ void __launch_bounds__(256) k_reduce_adam(const float* __restrict__ part, int nblk,
                                                     int np, float* __restrict__ grad,
                                                     float* __restrict__ loss, float* w, float* m,
                                                     float* v, TrainCtl* ctl, int B, float eps,
                                                     const unsigned* __restrict__ flags,
                                                     uint8_t* __restrict__ img, int L) {
  if (*(volatile const unsigned*)flags != 0u) return;
  __shared__ float red[8][33];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int p = blockIdx.x * 32 + lane;
  float s = 0.0f;
  if (p <= np) {
#pragma unroll 4
    for (int c = wp; c < nblk; c += 8) s += part[(size_t)c * (np + 1) + p];
  }
  red[wp][lane] = s;
  __syncthreads();
  if (wp == 0 && p <= np) {
    float g = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) g += red[i][lane];
    if (p == np) {
      *loss = g;
    } else {
      grad[p] = g;
      if (ctl != nullptr) {
        float c1, c2, lr_t;
        adam_scalars(ctl, &c1, &c2, &lr_t);
        const float b1 = ctl->b1, b2 = ctl->b2;
        const float mt = b1 * m[p] + (1.0f - b1) * g;
        const float vt = b2 * v[p] + (1.0f - b2) * g * g;
        m[p] = mt;
        v[p] = vt;
        const float wn = w[p] - lr_t * (mt / c1) / (sqrtf(vt / c2) + eps);
        w[p] = wn;
        train_img_put(img, train_tc_shape(L), p, wn);
      }
    }
  }
  if (ctl == nullptr) return;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(&ctl->done, 1u);
    if (prev == gridDim.x - 1) {
      __threadfence();
      const float lv = *(volatile const float*)loss;
      if (ctl->k >= ctl->steps - ctl->epoch_steps) ctl->loss_sum += (double)lv / (double)B;
      ctl->t += 1;
      ctl->k += 1;
      ctl->done = 0;
    }
  }
}

// ---------------------------------------------------------------- launchers

int mlp_param_count(int L) { return mlp_n_params(4 * L + 1, L + L * (L + 1) / 2); }

size_t tc_image_bytes(int L) { return (size_t)tc_shape(L).bytes; }

cudaError_t launch_pack_image(const float* params, void* img, int L, cudaStream_t s) {
  k_pack_image<<<64, 256, 0, s>>>(params, L, (uint8_t*)img);
  return cudaGetLastError();
}

cudaError_t launch_proposal_f32(const ModelConst& mc, const DevPtrsF32& p, const void* img,
                                float* out, cudaStream_t s) {
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const size_t smem = tc_smem_layout(mc.L, nullptr);
  e = cudaFuncSetAttribute(k_proposal_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)tc_smem_layout(FBS_MAX_L, nullptr));
  if (e != cudaSuccess) return e;
  // Up to four blocks per SM: 128 of the SM's 512 TMEM columns each.
  const int ntiles = (mc.G + 127) / 128;
  const int grid = ntiles < 4 * nsm ? ntiles : 4 * nsm;
  k_proposal_tc<<<grid, kTcThreads, smem, s>>>(mc, p, (const uint8_t*)img, out, ntiles);
  return cudaGetLastError();
}

cudaError_t launch_collect_f32(const ModelConst& mc, const DevPtrsF32& p, float* feat,
                               float* beta, long long row, cudaStream_t s) {
  const int blk = 128;
  k_collect_f32<<<(mc.G + blk - 1) / blk, blk, 0, s>>>(mc, p, feat, beta, row);
  return cudaGetLastError();
}

cudaError_t launch_col_stats(const float* feat, const float* beta, long long M, int F, int L,
                             float* st, cudaStream_t s) {
  k_col_stats<<<F + L, 256, 0, s>>>(feat, beta, M, F, L, st);
  return cudaGetLastError();
}

cudaError_t launch_fold(float* params, const float* st, int L, int to_raw, cudaStream_t s) {
  const int K = L + L * (L + 1) / 2;
  k_fold<<<1, ((kMlpHidden + K + 31) / 32) * 32, 0, s>>>(params, st, L, to_raw);
  return cudaGetLastError();
}

size_t train_smem_bytes(int L) { return (size_t)train_tc_shape(L).bytes; }

int train_blocks(int Bsz) { return (Bsz + 127) / 128; }

cudaError_t prepare_train_kernel(int L) {
  return cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)train_smem_bytes(L));
}

size_t train_image_bytes(int L) { return (size_t)train_tc_shape(L).img_bytes; }

cudaError_t launch_pack_train_image(const float* params, int L, void* img, cudaStream_t s) {
  k_pack_train_image<<<32, 256, 0, s>>>(params, L, (uint8_t*)img);
  return cudaGetLastError();
}

cudaError_t launch_mlp_grad(const float* params, int L, int Bsz, const float* fb, const float* yb,
                            float* part, float* grad, float* loss, void* img, unsigned* flags,
                            unsigned polls, cudaStream_t s) {
  const int nblk = train_blocks(Bsz);
  const int np = mlp_param_count(L);
  k_pack_train_image<<<32, 256, 0, s>>>(params, L, (uint8_t*)img);
  k_mlp_tc<<<nblk, 128, train_smem_bytes(L), s>>>(L, Bsz, fb, yb, nullptr, nullptr, 0,
                                                  0u, 0u, nullptr, nullptr, part,
                                                  (const uint8_t*)img, flags, polls);
  k_reduce_adam<<<(np + 1 + 31) / 32, 256, 0, s>>>(part, nblk, np, grad, loss, nullptr, nullptr,
                                                   nullptr, nullptr, Bsz, 0.0f, flags, nullptr, L);
  return cudaGetLastError();
}

cudaError_t launch_train_step(float* params, int L, int Bsz, const float* feat, const float* beta,
                              long long M, uint64_t seed, TrainCtl* ctl, const float* st,
                              float* part, float* grad, float* loss, float* adam_m, float* adam_v,
                              void* img, unsigned* flags, unsigned polls, cudaStream_t s) {
  const int nblk = train_blocks(Bsz);
  const int np = mlp_param_count(L);
  k_mlp_tc<<<nblk, 128, train_smem_bytes(L), s>>>(L, Bsz, nullptr, nullptr, feat, beta, M,
                                                  (uint32_t)seed, (uint32_t)(seed >> 32), ctl, st,
                                                  part, (const uint8_t*)img, flags, polls);
  k_reduce_adam<<<(np + 1 + 31) / 32, 256, 0, s>>>(part, nblk, np, grad, loss, params, adam_m,
                                                   adam_v, ctl, Bsz, 1e-8f, flags,
                                                   (uint8_t*)img, L);
  return cudaGetLastError();
}

}  // namespace fbs
