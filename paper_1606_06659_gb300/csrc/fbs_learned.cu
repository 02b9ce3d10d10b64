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

__device__ __forceinline__ float gelu_f(float x) {
  return 0.5f * x * (1.0f + tanhf(kSqrt2OverPi * (x + 0.044715f * x * x * x)));
}

__device__ __forceinline__ float gelu_grad_f(float x) {
  const float t = tanhf(kSqrt2OverPi * (x + 0.044715f * x * x * x));
  const float du = kSqrt2OverPi * (1.0f + 3.0f * 0.044715f * x * x);
  return 0.5f * (1.0f + t) + 0.5f * x * (1.0f - t * t) * du;
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
  size_t off_a;
  tc_smem_layout(mc.L, &off_a);
  if (threadIdx.x == 0) s_abort = 0;
  TcBlock c;
  tc_begin(c, bars, &tmem_slot, img_g, sm, t.bytes, p.tc_polls);
  if (!c.w_ok) s_abort = 1;
  __syncthreads();
  for (int tile = blockIdx.x; tile < ntiles && !s_abort; tile += gridDim.x) {
    const int g = tile * 128 + (int)threadIdx.x;
    if (!tc_tile(c, mc, p, t, sm, sm + off_a, g, net_gene(p, g, mc.G), out, &s_abort)) break;
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

// One training step's forward and backward pass of the network for
// kTrainRows rows per block, entirely in shared memory (weights, the rows'
// features and beta, both layers' pre-activations and activations, the
// outputs and the back-propagated gradients), then this block's sum over its
// rows of every parameter gradient and of the loss, written in parameter order
// to part[block][np + 1] (the loss last).  Rows past Bsz take no part.
//
// Gaussian head, per row: loss = |u|^2 / 2 + sum log C_ll with C u = beta - mu;
// dL/dout (scaled by 1/Bsz): d mu = -v, d logC_ii = 1 - v_i u_i C_ii,
// d C_ij = -v_i u_j (i > j), where C^T v = u.
constexpr int kTrainRows = 32;
constexpr int kTrainThreads = 256;
constexpr int kRowGroups = kTrainThreads / kMlpHidden;       // 4
constexpr int kRowsPerThread = kTrainRows / kRowGroups;      // 8

__host__ __device__ inline int train_smem_floats(int L) {
  const int H = kMlpHidden, HP = H + 1, F = 4 * L + 1, K = L + L * (L + 1) / 2, R = kTrainRows;
  return H * F + H * HP + K * HP + 2 * H + K + R * F + R * L + 6 * R * H + R * K + 32;
}

__device__ __forceinline__ void nll_row(float* o, const float* y, int L, float sc, float* loss) {
  float C[kMaxL][kMaxL], u[kMaxL], v[kMaxL];
  for (int i = 0; i < L; ++i)
    for (int j = 0; j < L; ++j) C[i][j] = 0.0f;
  int k = 2 * L;
  for (int i = 0; i < L; ++i) {
    C[i][i] = expf(o[L + i]);
    for (int j = 0; j < i; ++j) C[i][j] = o[k++];
  }
  float ls = 0.0f;
  for (int i = 0; i < L; ++i) {
    float s = y[i] - o[i];
    for (int j = 0; j < i; ++j) s -= C[i][j] * u[j];
    u[i] = s / C[i][i];
    ls += 0.5f * u[i] * u[i] + o[L + i];
  }
  for (int i = L - 1; i >= 0; --i) {
    float s = u[i];
    for (int j = i + 1; j < L; ++j) s -= C[j][i] * v[j];
    v[i] = s / C[i][i];
  }
  // o becomes dL/do
  k = 2 * L;
  for (int i = 0; i < L; ++i)
    for (int j = 0; j < i; ++j) o[k++] = -v[i] * u[j] * sc;
  for (int i = 0; i < L; ++i) {
    o[L + i] = (1.0f - v[i] * u[i] * C[i][i]) * sc;
    o[i] = -v[i] * sc;
  }
  *loss = ls;
}

// Rows: fb / yb [Bsz][F], [Bsz][L] as given, or (feat != null) a minibatch drawn
// with replacement from the M pairs feat [M][F], beta [M][L] for the step the
// control block describes (Philox stream kStreamTrain, index = row, iteration
// t + 1), standardised with st = (feature means, feature scales, beta means,
// beta scales).
__global__ void __launch_bounds__(kTrainThreads) k_mlp_fwd_bwd(
    const float* __restrict__ params, int L, int Bsz, const float* __restrict__ fb,
    const float* __restrict__ yb, const float* __restrict__ feat,
    const float* __restrict__ beta, long long M, uint32_t seed_lo, uint32_t seed_hi,
    const TrainCtl* __restrict__ ctl, const float* __restrict__ st, float* __restrict__ part) {
  extern __shared__ __align__(1024) uint8_t sm_raw[];
  float* sm = reinterpret_cast<float*>(sm_raw);
  constexpr int H = kMlpHidden, HP = kMlpHidden + 1, R = kTrainRows, T = kTrainThreads;
  const int F = 4 * L + 1, K = L + L * (L + 1) / 2;
  const int np = mlp_n_params(F, K);
  // weights: W1 [H][F]; W2 and W3 padded to H+1 columns (conflict-free reads by
  // output row and by input column)
  float* sW1 = sm;
  float* sW2 = sW1 + H * F;
  float* sW3 = sW2 + H * HP;
  float* sb1 = sW3 + K * HP;
  float* sb2 = sb1 + H;
  float* sb3 = sb2 + H;
  float* sX = sb3 + K;        // [R][F]
  float* sY = sX + R * F;     // [R][L]
  float* sZ1 = sY + R * L;    // [R][H] pre-activations and activations
  float* sA1 = sZ1 + R * H;
  float* sZ2 = sA1 + R * H;
  float* sA2 = sZ2 + R * H;
  float* sG2 = sA2 + R * H;   // dL/dz2
  float* sG1 = sG2 + R * H;   // dL/dz1
  float* sD = sG1 + R * H;    // [R][K] outputs, then dL/dout
  float* sred = sD + R * K;   // [32]
  const float* W1 = params;
  const float* b1 = W1 + H * F;
  const float* W2 = b1 + H;
  const float* b2 = W2 + H * H;
  const float* W3 = b2 + H;
  const float* b3 = W3 + K * H;
  const int tid = threadIdx.x;
  const int r0 = blockIdx.x * R;
  const int nr = min(R, Bsz - r0);
  __shared__ long long srow[R];
  if (feat != nullptr && tid < nr) {
    Rng rg(seed_lo, seed_hi, 0u, kStreamTrain, (uint32_t)(r0 + tid), (uint32_t)(ctl->t + 1));
    long long m = (long long)(rg.u(0) * (double)M);
    srow[tid] = m >= M ? M - 1 : m;
  }
#pragma unroll 4
  for (int i = tid; i < H * F; i += T) sW1[i] = W1[i];
#pragma unroll 4
  for (int i = tid; i < H * H; i += T) sW2[(i / H) * HP + i % H] = W2[i];
#pragma unroll 4
  for (int i = tid; i < K * H; i += T) sW3[(i / H) * HP + i % H] = W3[i];
  for (int i = tid; i < H; i += T) {
    sb1[i] = b1[i];
    sb2[i] = b2[i];
  }
  for (int i = tid; i < K; i += T) sb3[i] = b3[i];
  if (feat != nullptr) {
    __syncthreads();  // srow
    const float* mf = st;
    const float* sf = st + F;
    const float* mb = st + 2 * F;
    const float* sb = st + 2 * F + L;
    for (int i = tid; i < R * F; i += T) {
      const int r = i / F, f = i % F;
      sX[i] = r < nr ? (feat[(size_t)srow[r] * F + f] - mf[f]) / sf[f] : 0.0f;
    }
    for (int i = tid; i < R * L; i += T) {
      const int r = i / L, l = i % L;
      sY[i] = r < nr ? (beta[(size_t)srow[r] * L + l] - mb[l]) / sb[l] : 0.0f;
    }
  } else {
    for (int i = tid; i < R * F; i += T)
      sX[i] = i / F < nr ? fb[(size_t)r0 * F + i] : 0.0f;
    for (int i = tid; i < R * L; i += T)
      sY[i] = i / L < nr ? yb[(size_t)r0 * L + i] : 0.0f;
  }
  __syncthreads();

  // thread: unit h of a layer for rows rq, rq + 4, ..
  const int h = tid % H, rq = tid / H;
  float acc[kRowsPerThread];
  // layer 1
#pragma unroll
  for (int i = 0; i < kRowsPerThread; ++i) acc[i] = sb1[h];
  for (int f = 0; f < F; ++f) {
    const float w = sW1[h * F + f];
#pragma unroll
    for (int i = 0; i < kRowsPerThread; ++i) acc[i] += w * sX[(rq + kRowGroups * i) * F + f];
  }
#pragma unroll
  for (int i = 0; i < kRowsPerThread; ++i) {
    const int r = rq + kRowGroups * i;
    sZ1[r * H + h] = acc[i];
    sA1[r * H + h] = gelu_f(acc[i]);
  }
  __syncthreads();
  // layer 2
#pragma unroll
  for (int i = 0; i < kRowsPerThread; ++i) acc[i] = sb2[h];
  for (int k = 0; k < H; ++k) {
    const float w = sW2[h * HP + k];
#pragma unroll
    for (int i = 0; i < kRowsPerThread; ++i) acc[i] += w * sA1[(rq + kRowGroups * i) * H + k];
  }
#pragma unroll
  for (int i = 0; i < kRowsPerThread; ++i) {
    const int r = rq + kRowGroups * i;
    sZ2[r * H + h] = acc[i];
    sA2[r * H + h] = gelu_f(acc[i]);
  }
  __syncthreads();
  // output layer
  for (int e = tid; e < R * K; e += T) {
    const int r = e / K, j = e % K;
    float a = sb3[j];
    for (int k = 0; k < H; ++k) a += sW3[j * HP + k] * sA2[r * H + k];
    sD[e] = a;
  }
  __syncthreads();
  // head: one thread per row
  float loss = 0.0f;
  if (tid < R) {
    if (tid < nr) {
      nll_row(sD + tid * K, sY + tid * L, L, 1.0f / (float)Bsz, &loss);
    } else {
      for (int j = 0; j < K; ++j) sD[tid * K + j] = 0.0f;
    }
  }
  if (tid < 32) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_down_sync(0xffffffffu, loss, o);
    if (tid == 0) sred[0] = loss;
  }
  __syncthreads();
  // dL/dz2 = (dL/dout W3) * gelu'(z2)
#pragma unroll
  for (int i = 0; i < kRowsPerThread; ++i) acc[i] = 0.0f;
  for (int j = 0; j < K; ++j) {
    const float w = sW3[j * HP + h];
#pragma unroll
    for (int i = 0; i < kRowsPerThread; ++i) acc[i] += sD[(rq + kRowGroups * i) * K + j] * w;
  }
#pragma unroll
  for (int i = 0; i < kRowsPerThread; ++i) {
    const int r = rq + kRowGroups * i;
    sG2[r * H + h] = acc[i] * gelu_grad_f(sZ2[r * H + h]);
  }
  __syncthreads();
  // dL/dz1 = (dL/dz2 W2) * gelu'(z1)
#pragma unroll
  for (int i = 0; i < kRowsPerThread; ++i) acc[i] = 0.0f;
  for (int k = 0; k < H; ++k) {
    const float w = sW2[k * HP + h];
#pragma unroll
    for (int i = 0; i < kRowsPerThread; ++i) acc[i] += sG2[(rq + kRowGroups * i) * H + k] * w;
  }
#pragma unroll
  for (int i = 0; i < kRowsPerThread; ++i) {
    const int r = rq + kRowGroups * i;
    sG1[r * H + h] = acc[i] * gelu_grad_f(sZ1[r * H + h]);
  }
  __syncthreads();
  // this block's gradient sums over its rows, in parameter order
  float* out = part + (size_t)blockIdx.x * (np + 1);
  // offsets: W1 at 0, then b1, W2, b2, W3, b3
  const int ob1 = H * F, oW2 = ob1 + H, ob2 = oW2 + H * H, oW3 = ob2 + H, ob3 = oW3 + K * H;
  for (int p = tid; p < np; p += T) {
    float g = 0.0f;
    if (p < ob1) {
      const int u = p / F, f = p % F;
      for (int r = 0; r < R; ++r) g += sG1[r * H + u] * sX[r * F + f];
    } else if (p < oW2) {
      const int u = p - ob1;
      for (int r = 0; r < R; ++r) g += sG1[r * H + u];
    } else if (p < ob2) {
      const int q = p - oW2, u = q / H, k = q % H;
      for (int r = 0; r < R; ++r) g += sG2[r * H + u] * sA1[r * H + k];
    } else if (p < oW3) {
      const int u = p - ob2;
      for (int r = 0; r < R; ++r) g += sG2[r * H + u];
    } else if (p < ob3) {
      const int q = p - oW3, j = q / H, k = q % H;
      for (int r = 0; r < R; ++r) g += sD[r * K + j] * sA2[r * H + k];
    } else {
      const int j = p - ob3;
      for (int r = 0; r < R; ++r) g += sD[r * K + j];
    }
    out[p] = g;
  }
  if (tid == 0) out[np] = sred[0];
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
// applies Adam to w, m, v and, in the last block to finish (ticket counter, no
// waiting), adds the loss to the last epoch's sum and advances t and k.
__global__ void __launch_bounds__(256) k_reduce_adam(const float* __restrict__ part, int nblk,
                                                     int np, float* __restrict__ grad,
                                                     float* __restrict__ loss, float* w, float* m,
                                                     float* v, TrainCtl* ctl, int B, float eps) {
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
        w[p] -= lr_t * (mt / c1) / (sqrtf(vt / c2) + eps);
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
  // Up to three blocks per SM (shared memory), 128 TMEM columns each.
  const int ntiles = (mc.G + 127) / 128;
  const int grid = ntiles < 3 * nsm ? ntiles : 3 * nsm;
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

size_t train_smem_bytes(int L) { return (size_t)train_smem_floats(L) * sizeof(float); }

int train_blocks(int Bsz) { return (Bsz + kTrainRows - 1) / kTrainRows; }

cudaError_t prepare_train_kernel(int L) {
  return cudaFuncSetAttribute(k_mlp_fwd_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)train_smem_bytes(L));
}

cudaError_t launch_mlp_grad(const float* params, int L, int Bsz, const float* fb, const float* yb,
                            float* part, float* grad, float* loss, cudaStream_t s) {
  const int nblk = train_blocks(Bsz);
  const int np = mlp_param_count(L);
  k_mlp_fwd_bwd<<<nblk, kTrainThreads, train_smem_bytes(L), s>>>(
      params, L, Bsz, fb, yb, nullptr, nullptr, 0, 0u, 0u, nullptr, nullptr, part);
  k_reduce_adam<<<(np + 1 + 31) / 32, 256, 0, s>>>(part, nblk, np, grad, loss, nullptr, nullptr,
                                                   nullptr, nullptr, Bsz, 0.0f);
  return cudaGetLastError();
}

cudaError_t launch_train_step(float* params, int L, int Bsz, const float* feat, const float* beta,
                              long long M, uint64_t seed, TrainCtl* ctl, const float* st,
                              float* part, float* grad, float* loss, float* adam_m, float* adam_v,
                              cudaStream_t s) {
  const int nblk = train_blocks(Bsz);
  const int np = mlp_param_count(L);
  k_mlp_fwd_bwd<<<nblk, kTrainThreads, train_smem_bytes(L), s>>>(
      params, L, Bsz, nullptr, nullptr, feat, beta, M, (uint32_t)seed, (uint32_t)(seed >> 32),
      ctl, st, part);
  k_reduce_adam<<<(np + 1 + 31) / 32, 256, 0, s>>>(part, nblk, np, grad, loss, params, adam_m,
                                                   adam_v, ctl, Bsz, 1e-8f);
  return cudaGetLastError();
}

}  // namespace fbs
