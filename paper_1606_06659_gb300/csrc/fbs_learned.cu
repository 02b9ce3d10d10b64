// fbs_learned.cu -- the learned proposal for the beta_g block: per-gene
// features, the multilayer perceptron that maps them to a Gaussian, the
// collection of training pairs from the plain sampler, and the training
// kernels (minibatch gather, GEMMs, GELU, Gaussian negative log-likelihood
// head, Adam).  The move that uses the proposal is in fbs_gene_f32.cu.
//
// Network: features (4L+1) -> 64 -> GELU -> 64 -> GELU -> L + L(L+1)/2 outputs:
// mean mu (L), log of the Cholesky diagonal (L), sub-diagonal entries in row
// order.  GELU is the tanh form of Hendrycks & Gimpel (2016).  Parameters are
// one flat FP32 array W1 [64][F], b1 [64], W2 [64][64], b2 [64], W3 [K][64],
// b3 [K]; inference reads a BF16 copy with FP32 accumulation.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fbs_common.cuh"
#include "fbs_kernels.h"
#include "fbs_rng.cuh"

namespace fbs {

constexpr float kSqrt2OverPi = 0.7978845608028654f;

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

// Features of gene g, invariant under the move (which keeps eta = h + eps + X beta):
// X^T (eta_g - h) / N, asinh(X^T y_g), log gamma_g, theta, log sigma.
__device__ __forceinline__ void gene_features(const ModelConst& mc, const DevPtrsF32& p, int g,
                                              const Hyper* hy, float* f) {
  const int G = mc.G, N = mc.N, L = mc.L;
  float a[kMaxL];
#pragma unroll
  for (int l = 0; l < kMaxL; ++l) a[l] = 0.0f;
  float b[kMaxL];
#pragma unroll
  for (int l = 0; l < kMaxL; ++l) b[l] = l < L ? p.beta[(size_t)l * G + g] : 0.0f;
  for (int n = 0; n < N; ++n) {
    float lin = p.eps[(size_t)n * G + g];
#pragma unroll
    for (int l = 0; l < kMaxL; ++l)
      if (l < L) lin += mc.Xf[n * kMaxL + l] * b[l];
#pragma unroll
    for (int l = 0; l < kMaxL; ++l)
      if (l < L) a[l] += mc.Xf[n * kMaxL + l] * lin;
  }
  const float invN = 1.0f / (float)N;
  for (int l = 0; l < L; ++l) {
    f[l] = a[l] * invN;
    f[L + l] = asinhf((float)p.T[(size_t)l * G + g]);
    f[2 * L + 1 + l] = (float)hy->phi[2 + l];
    f[3 * L + 1 + l] = 0.5f * logf((float)hy->phi[2 + L + l]);
  }
  f[2 * L] = logf(p.gam[g]);
}

// One thread per gene: features, then the network with its BF16 weights staged in
// shared memory as FP32; writes the proposal parameters [K][G].  Genes that keep
// the slice updates are skipped unless every gene is being calibrated.
__global__ void __launch_bounds__(128) k_proposal_f32(ModelConst mc, DevPtrsF32 p,
                                                     const __nv_bfloat16* __restrict__ w,
                                                     float* __restrict__ out) {
  extern __shared__ float ws[];  // weights as FP32, then h2[64][blockDim]
  const int F = 4 * mc.L + 1, K = mc.L + mc.L * (mc.L + 1) / 2, H = kMlpHidden;
  const int np = mlp_n_params(F, K);
  for (int i = threadIdx.x; i < np; i += blockDim.x) ws[i] = __bfloat162float(w[i]);
  __syncthreads();
  const float* W1 = ws;
  const float* b1 = W1 + H * F;
  const float* W2 = b1 + H;
  const float* b2 = W2 + H * H;
  const float* W3 = b2 + H;
  const float* b3 = W3 + K * H;
  float* h2s = ws + ((np + 31) & ~31);
  const int B = blockDim.x, tid = threadIdx.x;
  const int g = blockIdx.x * B + tid;
  if (g >= mc.G) return;
  if (!(p.mh_all || p.use_mh[g])) return;
  float f[kMaxFeat];
  gene_features(mc, p, g, p.hyp, f);
  float h1[kMlpHidden];
#pragma unroll
  for (int j = 0; j < kMlpHidden; ++j) {
    float acc = b1[j];
    for (int i = 0; i < F; ++i) acc += W1[j * F + i] * f[i];
    h1[j] = gelu_f(acc);
  }
  for (int j = 0; j < H; ++j) {
    float acc = b2[j];
#pragma unroll
    for (int i = 0; i < kMlpHidden; ++i) acc += W2[j * H + i] * h1[i];
    h2s[j * B + tid] = gelu_f(acc);
  }
  for (int k = 0; k < K; ++k) {
    float acc = b3[k];
    for (int j = 0; j < H; ++j) acc += W3[k * H + j] * h2s[j * B + tid];
    out[(size_t)k * mc.G + g] = acc;
  }
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

// Minibatch: row i of the batch is pair floor(U * M) for a Philox uniform U,
// standardised with the column means and scales of `st` (see k_col_stats).
__global__ void k_gather_rows(const float* __restrict__ feat, const float* __restrict__ beta,
                              long long M, int F, int L, int Bsz, uint32_t seed_lo,
                              uint32_t seed_hi, uint32_t step, const float* __restrict__ st,
                              float* __restrict__ fb, float* __restrict__ yb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Bsz) return;
  Rng r(seed_lo, seed_hi, 0u, kStreamTrain, (uint32_t)i, step);
  long long m = (long long)(r.u(0) * (double)M);
  if (m >= M) m = M - 1;
  const float* mf = st;
  const float* sf = st + F;
  const float* mb = st + 2 * F;
  const float* sb = st + 2 * F + L;
  for (int k = 0; k < F; ++k) fb[(size_t)i * F + k] = (feat[(size_t)m * F + k] - mf[k]) / sf[k];
  for (int l = 0; l < L; ++l) yb[(size_t)i * L + l] = (beta[(size_t)m * L + l] - mb[l]) / sb[l];
}

// Column means and scales of the training pairs, in FP64: block c < F takes
// feature column c, block F + l takes beta column l.  The scale is the standard
// deviation, or 1 for a column that is constant to within 1e-6 of its size.
// st = [mean_f (F), scale_f (F), mean_beta (L), scale_beta (L)].
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
    const double sc = var > tol * tol ? sqrt(var) : 1.0;
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

// C[i][j] (+)= sum_k A(i,k) B(k,j) with A(i,k) = A[i*sai + k*sak] and
// B(k,j) = B[k*sbk + j*sbj]; 16x16 output tiles, the k range split over
// gridDim.z (partial sums added atomically when split).
constexpr int kTile = 16;

__global__ void k_gemm(int M, int Nn, int Kk, const float* __restrict__ A, long long sai,
                       long long sak, const float* __restrict__ Bm, long long sbk, long long sbj,
                       float* __restrict__ Cm, long long ldc, int accumulate) {
  __shared__ float As[kTile][kTile + 1];
  __shared__ float Bs[kTile][kTile + 1];
  const int ti = threadIdx.y, tj = threadIdx.x;
  const int i = blockIdx.y * kTile + ti, j = blockIdx.x * kTile + tj;
  const int kchunk = (Kk + gridDim.z - 1) / gridDim.z;
  const int k0 = blockIdx.z * kchunk, k1 = min(Kk, k0 + kchunk);
  float acc = 0.0f;
  for (int kb = k0; kb < k1; kb += kTile) {
    const int ka = kb + tj, kbb = kb + ti;
    As[ti][tj] = (i < M && ka < k1) ? A[(long long)i * sai + (long long)ka * sak] : 0.0f;
    const int jj = blockIdx.x * kTile + tj;
    Bs[ti][tj] = (jj < Nn && kbb < k1) ? Bm[(long long)kbb * sbk + (long long)jj * sbj] : 0.0f;
    __syncthreads();
#pragma unroll
    for (int t = 0; t < kTile; ++t) acc += As[ti][t] * Bs[t][tj];
    __syncthreads();
  }
  if (i < M && j < Nn) {
    float* c = Cm + (long long)i * ldc + j;
    if (gridDim.z > 1) atomicAdd(c, acc);
    else *c = accumulate ? *c + acc : acc;
  }
}

// Z += b (broadcast over rows), H = gelu(Z).
__global__ void k_bias_gelu(float* Z, float* Hh, const float* b, int rows, int cols, int act) {
  const long long n = (long long)rows * cols;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const float z = Z[t] + b[t % cols];
    Z[t] = z;
    if (act) Hh[t] = gelu_f(z);
  }
}

// dZ = dH * gelu'(Z)
__global__ void k_gelu_back(const float* Z, const float* dH, float* dZ, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    dZ[t] = dH[t] * gelu_grad_f(Z[t]);
}

// Gaussian head: per row, loss = |u|^2 / 2 + sum log C_ll with C u = beta - mu, and
// dL/dout (scaled by 1/B): d mu = -v, d logC_ii = 1 - v_i u_i C_ii,
// d C_ij = -v_i u_j (i > j), where C^T v = u.
__global__ void k_nll_head(const float* __restrict__ O, const float* __restrict__ Y, int Bsz,
                           int L, float* __restrict__ dO, float* __restrict__ loss_sum) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int K = L + L * (L + 1) / 2;
  float loss = 0.0f;
  if (r < Bsz) {
    const float* o = O + (size_t)r * K;
    float C[kMaxL][kMaxL], u[kMaxL], v[kMaxL];
    for (int i = 0; i < L; ++i)
      for (int j = 0; j < L; ++j) C[i][j] = 0.0f;
    int k = 2 * L;
    for (int i = 0; i < L; ++i) {
      C[i][i] = expf(o[L + i]);
      for (int j = 0; j < i; ++j) C[i][j] = o[k++];
    }
    for (int i = 0; i < L; ++i) {
      float s = Y[(size_t)r * L + i] - o[i];
      for (int j = 0; j < i; ++j) s -= C[i][j] * u[j];
      u[i] = s / C[i][i];
      loss += 0.5f * u[i] * u[i] + o[L + i];
    }
    for (int i = L - 1; i >= 0; --i) {
      float s = u[i];
      for (int j = i + 1; j < L; ++j) s -= C[j][i] * v[j];
      v[i] = s / C[i][i];
    }
    const float sc = 1.0f / (float)Bsz;
    float* d = dO + (size_t)r * K;
    for (int i = 0; i < L; ++i) {
      d[i] = -v[i] * sc;
      d[L + i] = (1.0f - v[i] * u[i] * C[i][i]) * sc;
    }
    k = 2 * L;
    for (int i = 0; i < L; ++i)
      for (int j = 0; j < i; ++j) d[k++] = -v[i] * u[j] * sc;
  }
  for (int o = 16; o > 0; o >>= 1) loss += __shfl_down_sync(0xffffffffu, loss, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss_sum, loss);
}

// Column sums: g[j] = sum_i D[i][j].
__global__ void k_colsum(const float* D, int rows, int cols, float* g) {
  const int j = blockIdx.x;
  float s = 0.0f;
  for (int i = threadIdx.x; i < rows; i += blockDim.x) s += D[(size_t)i * cols + j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __shared__ float red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    g[j] = t;
  }
}

// Adam (Kingma & Ba 2015) with bias correction.
__global__ void k_adam(float* w, const float* g, float* m, float* v, int n, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const float gt = g[t];
  const float mt = b1 * m[t] + (1.0f - b1) * gt;
  const float vt = b2 * v[t] + (1.0f - b2) * gt * gt;
  m[t] = mt;
  v[t] = vt;
  w[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
}

__global__ void k_to_bf16(const float* a, __nv_bfloat16* b, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) b[t] = __float2bfloat16_rn(a[t]);
}

// ---------------------------------------------------------------- launchers

int mlp_param_count(int L) { return mlp_n_params(4 * L + 1, L + L * (L + 1) / 2); }

size_t proposal_smem_bytes(int L, int block) {
  const int np = mlp_param_count(L);
  return ((size_t)((np + 31) & ~31) + (size_t)kMlpHidden * block) * sizeof(float);
}

cudaError_t launch_proposal_f32(const ModelConst& mc, const DevPtrsF32& p, const void* wv,
                                float* out, cudaStream_t s) {
  const __nv_bfloat16* w = (const __nv_bfloat16*)wv;
  const int blk = 128;
  const size_t smem = proposal_smem_bytes(mc.L, blk);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_proposal_f32,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  k_proposal_f32<<<(mc.G + blk - 1) / blk, blk, smem, s>>>(mc, p, w, out);
  return cudaGetLastError();
}

cudaError_t launch_collect_f32(const ModelConst& mc, const DevPtrsF32& p, float* feat,
                               float* beta, long long row, cudaStream_t s) {
  const int blk = 128;
  k_collect_f32<<<(mc.G + blk - 1) / blk, blk, 0, s>>>(mc, p, feat, beta, row);
  return cudaGetLastError();
}

cudaError_t launch_gather_rows(const float* feat, const float* beta, long long M, int F, int L,
                               int Bsz, uint64_t seed, uint32_t step, const float* st, float* fb,
                               float* yb, cudaStream_t s) {
  k_gather_rows<<<(Bsz + 127) / 128, 128, 0, s>>>(feat, beta, M, F, L, Bsz, (uint32_t)seed,
                                                  (uint32_t)(seed >> 32), step, st, fb, yb);
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

cudaError_t launch_gemm(int M, int Nn, int Kk, const float* A, long long sai, long long sak,
                        const float* B, long long sbk, long long sbj, float* C, long long ldc,
                        int split_k, int accumulate, cudaStream_t s) {
  dim3 grid((Nn + kTile - 1) / kTile, (M + kTile - 1) / kTile, split_k), block(kTile, kTile);
  k_gemm<<<grid, block, 0, s>>>(M, Nn, Kk, A, sai, sak, B, sbk, sbj, C, ldc, accumulate);
  return cudaGetLastError();
}

cudaError_t launch_bias_gelu(float* Z, float* H, const float* b, int rows, int cols, int act,
                             cudaStream_t s) {
  k_bias_gelu<<<256, 256, 0, s>>>(Z, H, b, rows, cols, act);
  return cudaGetLastError();
}

cudaError_t launch_gelu_back(const float* Z, const float* dH, float* dZ, long long n,
                             cudaStream_t s) {
  k_gelu_back<<<256, 256, 0, s>>>(Z, dH, dZ, n);
  return cudaGetLastError();
}

cudaError_t launch_nll_head(const float* O, const float* Y, int Bsz, int L, float* dO,
                            float* loss_sum, cudaStream_t s) {
  k_nll_head<<<(Bsz + 127) / 128, 128, 0, s>>>(O, Y, Bsz, L, dO, loss_sum);
  return cudaGetLastError();
}

cudaError_t launch_colsum(const float* D, int rows, int cols, float* g, cudaStream_t s) {
  k_colsum<<<cols, 256, 0, s>>>(D, rows, cols, g);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* w, const float* g, float* m, float* v, int n, float lr, float b1,
                        float b2, float eps, float c1, float c2, cudaStream_t s) {
  k_adam<<<(n + 255) / 256, 256, 0, s>>>(w, g, m, v, n, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float* a, void* b, int n, cudaStream_t s) {
  k_to_bf16<<<(n + 255) / 256, 256, 0, s>>>(a, (__nv_bfloat16*)b, n);
  return cudaGetLastError();
}

}  // namespace fbs
