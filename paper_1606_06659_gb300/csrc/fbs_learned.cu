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
// b3 [K]; inference (tensor cores) reads them as split BF16 operands.
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

// Part of X^T (eta_g - h) over the samples n0 <= n < n1 (eta - h = eps + X beta).
__device__ __forceinline__ void feature_sums(const ModelConst& mc, const DevPtrsF32& p, int g,
                                             int n0, int n1, float* a) {
  const int G = mc.G, L = mc.L;
  float b[kMaxL];
#pragma unroll
  for (int l = 0; l < kMaxL; ++l) {
    a[l] = 0.0f;
    b[l] = l < L ? p.beta[(size_t)l * G + g] : 0.0f;
  }
#pragma unroll 4
  for (int n = n0; n < n1; ++n) {
    float lin = p.eps[(size_t)n * G + g];
#pragma unroll
    for (int l = 0; l < kMaxL; ++l)
      if (l < L) lin += mc.Xf[n * kMaxL + l] * b[l];
#pragma unroll
    for (int l = 0; l < kMaxL; ++l)
      if (l < L) a[l] += mc.Xf[n * kMaxL + l] * lin;
  }
}

// The features of gene g from the sums a = X^T (eta_g - h): a / N, asinh(X^T y_g),
// log gamma_g, theta, log sigma; all unchanged by the move, which keeps eta.
__device__ __forceinline__ void finish_features(const ModelConst& mc, const DevPtrsF32& p, int g,
                                                const Hyper* hy, const float* a, float* f) {
  const int G = mc.G, L = mc.L;
  const float invN = 1.0f / (float)mc.N;
  for (int l = 0; l < L; ++l) {
    f[l] = a[l] * invN;
    f[L + l] = asinhf((float)p.T[(size_t)l * G + g]);
    f[2 * L + 1 + l] = (float)hy->phi[2 + l];
    f[3 * L + 1 + l] = 0.5f * logf((float)hy->phi[2 + L + l]);
  }
  f[2 * L] = logf(p.gam[g]);
}

__device__ __forceinline__ void gene_features(const ModelConst& mc, const DevPtrsF32& p, int g,
                                              const Hyper* hy, float* f) {
  float a[kMaxL];
  feature_sums(mc, p, g, 0, mc.N, a);
  finish_features(mc, p, g, hy, a, f);
}

// ---------------------------------------------------------------- tensor-core inference
//
// The network runs on the tensor cores (tcgen05): per tile of 128 genes (one
// thread per gene, four warps) three GEMMs D = A W^T with BF16 operands read
// from shared memory and FP32 accumulators in tensor memory, M = 128 and
// N = 64, 64, n3.  Every FP32 operand x (weights, features, activations) enters
// as a BF16 pair x = hi + lo, hi = bf16(x), lo = bf16(x - hi); each layer
// accumulates hi*hi + lo*hi + hi*lo, which keeps about 16 significant bits per
// operand (the lo*lo term is below that).  GELU, the biases and the split of
// the next layer's input run in the epilogue, one thread per TMEM lane (= gene).
//
// Operands use the canonical K-major layout without swizzle: 8 x 16-byte core
// matrices of 128 contiguous bytes, the core matrices of one 8-row group
// consecutive along K (leading byte offset 128), the groups `sbo` bytes apart.
// An operand with kw columns holds [hi (kw/2) | lo (kw/2)].

struct TcShape {
  int F, K;      // features, outputs
  int k1;        // input columns of the first layer per half (F rounded up to 16)
  int n3;        // rows of the last layer (K rounded up to 16)
  int off_w2, off_w3, off_b, bytes;  // weight image: W1, W2, W3, biases (FP32)
};

__host__ __device__ inline TcShape tc_shape(int L) {
  TcShape t;
  t.F = 4 * L + 1;
  t.K = L + L * (L + 1) / 2;
  t.k1 = (t.F + 15) & ~15;
  t.n3 = (t.K + 15) & ~15;
  t.off_w2 = kMlpHidden * 2 * t.k1 * 2;
  t.off_w3 = t.off_w2 + kMlpHidden * 2 * kMlpHidden * 2;
  t.off_b = t.off_w3 + t.n3 * 2 * kMlpHidden * 2;
  t.bytes = t.off_b + (2 * kMlpHidden + t.n3) * 4;
  return t;
}

constexpr int kMaxK1 = (kMaxFeat + 15) & ~15;

// Shared memory: the weight image, then one A operand buffer of 128 rows that
// holds in turn the split features (2 k1 columns) and the split activations of
// the two hidden layers (128 columns); each is dead once its GEMM completed.
__host__ __device__ inline size_t tc_smem_layout(int L, size_t* off_a, size_t* off_stage = nullptr) {
  const TcShape t = tc_shape(L);
  const size_t a = ((size_t)t.bytes + 1023) & ~(size_t)1023;
  const size_t cols = 2 * t.k1 > 2 * kMlpHidden ? 2 * t.k1 : 2 * kMlpHidden;
  const size_t stage = a + (size_t)128 * cols * 2;  // [128][kMaxL] floats
  if (off_a) *off_a = a;
  if (off_stage) *off_stage = stage;
  return stage + (size_t)128 * kMaxL * 4;
}

// Byte offset of element (r, c) of a canonical operand with kw columns.
__host__ __device__ inline uint32_t canon_off(int r, int c, int kw) {
  return (uint32_t)(((r >> 3) * (kw >> 3) + (c >> 3)) * 128 + (r & 7) * 16 + (c & 7) * 2);
}

// Row r, columns c0..c0+7 of an operand with kw = 2 kin columns: hi parts at
// c0.., lo parts at kin + c0.. (16-byte stores; pairs converted together).
__device__ __forceinline__ void store_split8(uint8_t* base, int kin, int r, int c0,
                                             const float* v) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 hb = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    const float2 hf = __bfloat1622float2(hb);
    const __nv_bfloat162 lb = __floats2bfloat162_rn(v[2 * i] - hf.x, v[2 * i + 1] - hf.y);
    h[i] = *reinterpret_cast<const uint32_t*>(&hb);
    l[i] = *reinterpret_cast<const uint32_t*>(&lb);
  }
  *(uint4*)(base + canon_off(r, c0, 2 * kin)) = make_uint4(h[0], h[1], h[2], h[3]);
  *(uint4*)(base + canon_off(r, kin + c0, 2 * kin)) = make_uint4(l[0], l[1], l[2], l[3]);
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

constexpr unsigned kTcWaitLimit = 1u << 24;  // try_wait polls before a wait gives up

__device__ __forceinline__ uint32_t smem_u32(const void* ptr) {
  return (uint32_t)__cvta_generic_to_shared(ptr);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (unsigned i = 0; i < kTcWaitLimit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, P;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Shared-memory matrix descriptor: start address, leading byte offset 128,
// stride byte offset `sbo` (all >> 4), descriptor version 1 (bit 46), no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and
// B BF16 (bits 7-9 and 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
      :
      : "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// D (+)= A B^T over kin columns for the three hi/lo products; a and b are the
// operands' shared addresses, both with 2 kin columns.
__device__ __forceinline__ void issue_layer(uint32_t d, uint32_t a, uint32_t b, int kin,
                                            uint32_t idesc) {
  const uint32_t sbo = (uint32_t)(2 * kin / 8) * 128;
  const uint32_t lo = (uint32_t)(kin / 8) * 128;
  const uint32_t pa[3] = {0u, lo, 0u}, pb[3] = {0u, 0u, lo};
  uint32_t acc = 0u;
#pragma unroll
  for (int q = 0; q < 3; ++q)
    for (int k = 0; k < kin; k += 16) {
      const uint32_t ko = (uint32_t)(k / 8) * 128;
      umma_bf16(d, umma_desc(a + pa[q] + ko, sbo), umma_desc(b + pb[q] + ko, sbo), idesc, acc);
      acc = 1u;
    }
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// GELU (tanh form) for inference: x (1 + tanh u) / 2 = x / (1 + e^{-2u}), from the
// fast exponential and division: about 1e-6 relative error, far below what the
// proposal needs.
__device__ __forceinline__ float gelu_fast(float x) {
  const float u = kSqrt2OverPi * (x + 0.044715f * x * x * x);
  return __fdividef(x, 1.0f + __expf(-2.0f * u));
}

// 32 consecutive FP32 columns of this thread's TMEM lane (one load, one wait).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Bias, GELU and the split store of this thread's 32 columns c0.. of a hidden layer.
__device__ __forceinline__ void hidden_epilogue(uint32_t taddr, const float* bias, uint8_t* abuf,
                                                int row, int c0) {
  float v[32];
  tmem_ld32(taddr, v);
#pragma unroll
  for (int i = 0; i < 32; i += 4) {
    const float4 bb = *reinterpret_cast<const float4*>(bias + c0 + i);
    v[i] = gelu_fast(v[i] + bb.x);
    v[i + 1] = gelu_fast(v[i + 1] + bb.y);
    v[i + 2] = gelu_fast(v[i + 2] + bb.z);
    v[i + 3] = gelu_fast(v[i + 3] + bb.w);
  }
#pragma unroll
  for (int i = 0; i < 32; i += 8) store_split8(abuf, kMlpHidden, row, c0 + i, v + i);
}

constexpr uint32_t kTmemCols = 128;  // D1 at columns 0..63, D2 at 64..127, D3 at 0..n3-1
constexpr int kTcThreads = 256;      // two warps per TMEM lane quadrant


// Persistent over tiles of 128 genes; writes the proposal parameters [K][G] of
// the genes that may use the network's proposal.  Threads t and
// t + 128 sum the features of gene row t over the two halves of the samples and
// thread t writes its split row of the first operand (row = TMEM lane); in the
// epilogues warp w reads lane quadrant w % 4 and column half w / 4.  A wait that gives up sets
// kFlagTimeout, and the CTA frees its tensor memory and returns.
__global__ void __launch_bounds__(kTcThreads) k_proposal_tc(ModelConst mc, DevPtrsF32 p,
                                                           const uint8_t* __restrict__ img_g,
                                                           float* __restrict__ out, int ntiles) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_abort;
  const TcShape t = tc_shape(mc.L);
  size_t off_a, off_stage;
  tc_smem_layout(mc.L, &off_a, &off_stage);
  uint8_t* abuf = sm + off_a;
  float* stage = (float*)(sm + off_stage);
  const float* bias = (const float*)(sm + t.off_b);
  const int tid = threadIdx.x, warp = tid >> 5, lane_id = tid & 31;
  const int quad = warp & 3, half = warp >> 2;
  const int row = quad * 32 + lane_id;  // the gene (TMEM lane) this thread reads back
  const uint32_t bar_w = smem_u32(&bars[0]), bar_m = smem_u32(&bars[1]);
  if (tid == 0) {
    s_abort = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_w) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_m) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  if (tid == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_w),
                 "r"((uint32_t)t.bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(sm)),
        "l"(img_g), "r"((uint32_t)t.bytes), "r"(bar_w)
        : "memory");
  }
  bool w_ok = mbar_wait(bar_w, 0);
  if (!w_ok) s_abort = 1;
  __syncthreads();

  const uint32_t id64 = umma_idesc_bf16(128, 64), id3 = umma_idesc_bf16(128, t.n3);
  const uint32_t lane_addr = (uint32_t)(quad * 32) << 16;
  const uint32_t sa = smem_u32(abuf), sw = smem_u32(sm);
  uint32_t ph = 0;
  bool pending = false;  // an MMA batch whose completion was not seen
  const int G = mc.G;

  for (int tile = blockIdx.x; tile < ntiles && !s_abort; tile += gridDim.x) {
    const int g = tile * 128 + row;
    // genes that may use the network's proposal in this sweep
    const bool act = g < G && (p.mh_all == kMoveNet || p.mh_all == 3 ||
                               (p.mh_all == 0 && p.use_mh[g] == kMoveNet));
    // features: threads 0..127 sum X^T (eta - h) over the first half of the
    // samples, threads 128..255 over the second half (same gene: row = tid % 128)
    {
      float a[kMaxL];
      const int nh = mc.N / 2;
      if (act) {
        if (half == 0) feature_sums(mc, p, g, 0, nh, a);
        else feature_sums(mc, p, g, nh, mc.N, a);
      }
      if (half == 1 && act) {
#pragma unroll
        for (int l = 0; l < kMaxL; ++l) stage[row * kMaxL + l] = a[l];
      }
      __syncthreads();
      if (half == 0) {
        float f[kMaxK1];
#pragma unroll
        for (int i = 0; i < kMaxK1; ++i) f[i] = 0.0f;
        if (act) {
#pragma unroll
          for (int l = 0; l < kMaxL; ++l) a[l] += stage[row * kMaxL + l];
          finish_features(mc, p, g, p.hyp, a, f);
        }
#pragma unroll
        for (int c0 = 0; c0 < kMaxK1; c0 += 8)
          if (c0 < t.k1) store_split8(abuf, t.k1, row, c0, f + c0);
      }
    }

    // ---- layer 1: D1 = A1 W1^T
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      issue_layer(tmem, sa, sw, t.k1, id64);
      umma_commit(bar_m);
    }
    pending = true;
    if (!mbar_wait(bar_m, ph)) s_abort = 1;
    else pending = false;
    ph ^= 1u;
    tc_fence_after();
    hidden_epilogue(tmem + lane_addr + (uint32_t)(half * 32), bias, abuf, row, half * 32);

    // ---- layer 2: D2 = A2 W2^T (A2 overwrote A1 after GEMM 1 completed)
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (s_abort) break;
    if (tid == 0) {
      tc_fence_after();
      issue_layer(tmem + kMlpHidden, sa, sw + (uint32_t)t.off_w2, kMlpHidden, id64);
      umma_commit(bar_m);
    }
    pending = true;
    if (!mbar_wait(bar_m, ph)) s_abort = 1;
    else pending = false;
    ph ^= 1u;
    tc_fence_after();
    hidden_epilogue(tmem + lane_addr + (uint32_t)(kMlpHidden + half * 32), bias + kMlpHidden, abuf,
                    row, half * 32);

    // ---- layer 3: D3 = A3 W3^T (D3 reuses D1's columns)
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (s_abort) break;
    if (tid == 0) {
      tc_fence_after();
      issue_layer(tmem, sa, sw + (uint32_t)t.off_w3, kMlpHidden, id3);
      umma_commit(bar_m);
    }
    pending = true;
    if (!mbar_wait(bar_m, ph)) s_abort = 1;
    else pending = false;
    ph ^= 1u;
    tc_fence_after();
    for (int c0 = half * 16; c0 < t.n3; c0 += 32) {
      float v[16];
      tmem_ld16(tmem + lane_addr + (uint32_t)c0, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int k = c0 + i;
        if (act && k < t.K) out[(size_t)k * G + g] = v[i] + bias[2 * kMlpHidden + k];
      }
    }
    tc_fence_before();
    __syncthreads();
  }

  if (s_abort) {
    if (tid == 0) atomicOr(&p.hyp->flags, kFlagTimeout);
    if (!w_ok) mbar_wait(bar_w, 0);
    if (pending) mbar_wait(bar_m, ph ^ 1u);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
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
  // Up to three CTAs per SM (shared memory), 128 TMEM columns each.
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
