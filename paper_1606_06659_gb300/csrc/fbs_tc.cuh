// fbs_tc.cuh -- the learned proposal network's inference on the tcgen05 tensor
// cores, as block-level device functions: per-gene features, split-BF16
// operands in shared memory, the three GEMMs with tensor-memory accumulators and
// their epilogues.  Used by the stand-alone proposal kernel and by the
// gamma/beta kernel, which evaluates the network for its own 128 genes before
// their move (Landau & Niemi, arXiv 1606.06659, with the learned proposal of
// this library; the network itself is not in the paper).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fbs_common.cuh"

namespace fbs {

constexpr float kSqrt2OverPi = 0.7978845608028654f;

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
// thread per gene, four warps) three GEMMs D = A W^T with FP32 accumulators in
// tensor memory, M = 128 and N = 64, 64, n3.  Every FP32 operand x (weights,
// features, activations) enters as a BF16 pair x = hi + lo, hi = bf16(x),
// lo = bf16(x - hi); each layer accumulates hi*hi + lo*hi + hi*lo, which keeps
// about 16 significant bits per operand (the lo*lo term is below that).  GELU,
// the biases and the split of the next layer's input run in the epilogue, one
// thread per TMEM lane (= gene).
//
// The weights (B operands) sit in shared memory in the canonical K-major
// layout without swizzle: 8 x 16-byte core matrices of 128 contiguous bytes,
// the core matrices of one 8-row group consecutive along K (leading byte
// offset 128), the groups `sbo` bytes apart; an operand with kw columns holds
// [hi (kw/2) | lo (kw/2)].  The features and activations (A operands) sit in
// tensor memory next to the accumulators: row m in lane m, BF16 values packed
// two per 32-bit column (element 2c in the low half of column c), hi columns
// then lo columns, so the epilogue writes the next layer's input with
// tcgen05.st and no shared memory is involved.

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

// Shared memory of the network pass: the weight image alone (the A operands are
// in tensor memory); *off_a = its size rounded to 1 KB, where a caller's own
// shared data may start.
__host__ __device__ inline size_t tc_smem_layout(int L, size_t* off_a) {
  const TcShape t = tc_shape(L);
  const size_t a = ((size_t)t.bytes + 1023) & ~(size_t)1023;
  if (off_a) *off_a = a;
  return a;
}

// Byte offset of element (r, c) of a canonical K-major operand with kw columns.
__host__ __device__ inline uint32_t canon_off(int r, int c, int kw) {
  return (uint32_t)(((r >> 3) * (kw >> 3) + (c >> 3)) * 128 + (r & 7) * 16 + (c & 7) * 2);
}

// Row r, 8 consecutive values v of an operand whose 8-row groups are sbo bytes
// apart: the BF16 hi parts into 16-byte chunk ch_hi of the row, the lo parts
// into chunk ch_lo (K-major: the chunk is 8 consecutive K columns; read as an
// MN-major operand, 8 consecutive M or N elements of K row r).
__device__ __forceinline__ void store_split8_ch(uint8_t* base, uint32_t sbo, int r, int ch_hi,
                                                int ch_lo, const float* v) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 hb = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    const float2 hf = __bfloat1622float2(hb);
    const __nv_bfloat162 lb = __floats2bfloat162_rn(v[2 * i] - hf.x, v[2 * i + 1] - hf.y);
    h[i] = *reinterpret_cast<const uint32_t*>(&hb);
    l[i] = *reinterpret_cast<const uint32_t*>(&lb);
  }
  uint8_t* row = base + (size_t)(r >> 3) * sbo + (r & 7) * 16;
  *(uint4*)(row + ch_hi * 128) = make_uint4(h[0], h[1], h[2], h[3]);
  *(uint4*)(row + ch_lo * 128) = make_uint4(l[0], l[1], l[2], l[3]);
}

constexpr unsigned kTcWaitLimit = kTcWaitPolls;  // polls of a drain wait before it gives up

__device__ __forceinline__ uint32_t smem_u32(const void* ptr) {
  return (uint32_t)__cvta_generic_to_shared(ptr);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          unsigned limit = kTcWaitLimit) {
  for (unsigned i = 0; i < limit; ++i) {
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

// The same with A (bit 15) and/or B (bit 16) MN-major: for such an operand the
// descriptor's leading byte offset is the stride between groups of 8 rows
// along K and the stride byte offset the stride between 16-byte chunks (8
// elements) along M or N; a core matrix holds 8 K rows of 16 bytes.
__host__ __device__ constexpr uint32_t umma_idesc_bf16_mn(int M, int N, int a_mn, int b_mn) {
  return umma_idesc_bf16(M, N) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16);
}

// Shared-memory matrix descriptor with explicit leading and stride byte offsets
// (no swizzle, descriptor version 1).
__device__ __forceinline__ uint64_t umma_desc_ls(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
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



// Tensor-memory A operands: 16-bit elements packed two per 32-bit column (element
// 2c in the low half of column c), row m in lane m.
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t* r) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
               "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* r) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
               "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
               "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
               : "memory");
}
// 2n values split into BF16 hi / lo parts packed in pairs: hi[i], lo[i] hold elements 2i, 2i+1.
template <int NW>
__device__ __forceinline__ void pack_split(const float* v, uint32_t* hi, uint32_t* lo) {
#pragma unroll
  for (int i = 0; i < NW; ++i) {
    const __nv_bfloat162 hb = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    const float2 hf = __bfloat1622float2(hb);
    const __nv_bfloat162 lb = __floats2bfloat162_rn(v[2 * i] - hf.x, v[2 * i + 1] - hf.y);
    hi[i] = *reinterpret_cast<const uint32_t*>(&hb);
    lo[i] = *reinterpret_cast<const uint32_t*>(&lb);
  }
}
__device__ __forceinline__ void umma_bf16_ta(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                             uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n"
      :
      : "r"(d), "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
// D (+)= A B^T over kin columns for the three hi/lo products, A in tensor memory
// (hi at column a, lo at a + kin / 2), B in shared memory with 2 kin columns.
__device__ __forceinline__ void issue_layer_ta(uint32_t d, uint32_t a, uint32_t b, int kin,
                                               uint32_t idesc) {
  const uint32_t sbo = (uint32_t)(2 * kin / 8) * 128;
  const uint32_t lo = (uint32_t)(kin / 8) * 128;
  const uint32_t pa[3] = {0u, (uint32_t)(kin / 2), 0u}, pb[3] = {0u, 0u, lo};
  uint32_t acc = 0u;
#pragma unroll
  for (int q = 0; q < 3; ++q)
    for (int k = 0; k < kin; k += 16) {
      umma_bf16_ta(d, a + pa[q] + (uint32_t)(k / 2), umma_desc(b + pb[q] + (uint32_t)(k / 8) * 128, sbo),
                   idesc, acc);
      acc = 1u;
    }
}
// Bias, GELU and the split tensor-memory store of this thread's 32 columns c0.. of a
// hidden layer (D at taddr_d, the next layer's A at a_hi / a_hi + 32).
__device__ __forceinline__ void hidden_epilogue_ta(uint32_t taddr_d, const float* bias,
                                                   uint32_t a_hi, int c0) {
  float v[32];
  tmem_ld32(taddr_d, v);
#pragma unroll
  for (int i = 0; i < 32; i += 4) {
    const float4 bb = *reinterpret_cast<const float4*>(bias + c0 + i);
    v[i] = gelu_fast(v[i] + bb.x);
    v[i + 1] = gelu_fast(v[i + 1] + bb.y);
    v[i + 2] = gelu_fast(v[i + 2] + bb.z);
    v[i + 3] = gelu_fast(v[i + 3] + bb.w);
  }
  uint32_t hi[16], lo[16];
  pack_split<16>(v, hi, lo);
  tmem_st16(a_hi + (uint32_t)(c0 / 2), hi);
  tmem_st16(a_hi + 32u + (uint32_t)(c0 / 2), lo);
}

constexpr uint32_t kTmemCols = 128;  // accumulators at columns 0..63, A operands at 64..127

// Per-block state of the network: tensor-memory base, the two mbarriers (weight
// image, MMA completion), the completion phase and the wait outcomes.
struct TcBlock {
  uint32_t tmem, cols, bar_w, bar_m, ph;  // cols: tensor-memory columns allocated
  unsigned polls;  // polls of each wait of the pass before it gives up
  bool w_ok, pending;
};

// Barriers, 128 tensor-memory columns and the weight image (one bulk copy of
// img_bytes into sm), by a block of 128 threads.  bars, tmem_slot: the block's
// static shared words; polls: the bound of every wait of the pass (the drain
// waits of tc_end always allow kTcWaitLimit polls).  Every thread returns with
// c.w_ok = its wait for the image succeeded.
__device__ __forceinline__ void tc_begin(TcBlock& c, uint64_t* bars, uint32_t* tmem_slot,
                                         const uint8_t* img_g, uint8_t* sm, int img_bytes,
                                         unsigned polls) {
  const int tid = threadIdx.x;
  c.polls = polls;
  c.cols = kTmemCols;
  c.bar_w = smem_u32(&bars[0]);
  c.bar_m = smem_u32(&bars[1]);
  c.ph = 0;
  c.pending = false;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(c.bar_w) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(c.bar_m) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  c.tmem = *tmem_slot;
  if (tid == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(c.bar_w),
                 "r"((uint32_t)img_bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(sm)),
        "l"(img_g), "r"((uint32_t)img_bytes), "r"(c.bar_w)
        : "memory");
  }
  c.w_ok = mbar_wait(c.bar_w, 0, c.polls);
}

// Frees the block's c.cols tensor-memory columns.  After a wait that gave up (aborted) it first sets
// kFlagTimeout in *flags and waits again, up to kTcWaitLimit polls, for the copy
// and the MMAs still in flight, so that none of them outlives the block.
__device__ __forceinline__ void tc_end(TcBlock& c, bool aborted, unsigned* flags) {
  if (aborted) {
    if (threadIdx.x == 0) atomicOr(flags, kFlagTimeout);
    if (!c.w_ok) mbar_wait(c.bar_w, 0);
    if (c.pending) mbar_wait(c.bar_m, c.ph ^ 1u);
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(c.tmem),
                 "r"(c.cols)
                 : "memory");
  }
}

// The network for one tile of 128 genes by the block's 128 threads: thread t
// holds gene g (its TMEM lane, row t of the A operands and accumulators), warp
// w reads and writes lane quadrant w.  The weight image is at sm.  Genes with
// act write their K outputs to out[k ostride + oidx] (global [K][G] with
// ostride = G, oidx = g, or a block's shared [K][128] with ostride = 128,
// oidx = t, outside the weight image).  Every wait is bounded; one that gives
// up sets *s_abort (block-shared), and the function returns false once every
// thread has seen it.  Ends with a block barrier.
__device__ __forceinline__ bool tc_tile(TcBlock& c, const ModelConst& mc, const DevPtrsF32& p,
                                        const TcShape& t, uint8_t* sm, int g, bool act,
                                        float* out, size_t ostride, int oidx,
                                        volatile int* s_abort) {
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t lane_addr = (uint32_t)(warp * 32) << 16;
  const uint32_t id64 = umma_idesc_bf16(128, 64), id3 = umma_idesc_bf16(128, t.n3);
  const uint32_t sw = smem_u32(sm);
  const float* bias = (const float*)(sm + t.off_b);
  // tensor memory: D at columns 0..63 (0..n3-1 for the last layer), the A
  // operand of the next product at 64..127 (hi, then lo)
  const uint32_t a_col = c.tmem + lane_addr + 64u;
  // features of this thread's gene, split into the first operand
  {
    float f[kMaxK1];
#pragma unroll
    for (int i = 0; i < kMaxK1; ++i) f[i] = 0.0f;
    if (act) {
      float a[kMaxL];
      feature_sums(mc, p, g, 0, mc.N, a);
      finish_features(mc, p, g, p.hyp, a, f);
    }
#pragma unroll
    for (int c0 = 0; c0 < kMaxK1; c0 += 16)
      if (c0 < t.k1) {
        uint32_t hi[8], lo[8];
        pack_split<8>(f + c0, hi, lo);
        tmem_st8(a_col + (uint32_t)(c0 / 2), hi);
        tmem_st8(a_col + (uint32_t)(t.k1 / 2 + c0 / 2), lo);
      }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  // three layers: D1 = A1 W1^T, D2 = A2 W2^T, D3 = A3 W3^T, each D at columns 0..;
  // A2, A3 overwrite the A columns once the product before them has completed
  const uint32_t ta = c.tmem + 64u;
  for (int layer = 0; layer < 3; ++layer) {
    tc_fence_before();
    __syncthreads();
    if (*s_abort) return false;
    const uint32_t d = c.tmem;
    if (tid == 0) {
      tc_fence_after();
      if (layer == 0) issue_layer_ta(d, ta, sw, t.k1, id64);
      else if (layer == 1) issue_layer_ta(d, ta, sw + (uint32_t)t.off_w2, kMlpHidden, id64);
      else issue_layer_ta(d, ta, sw + (uint32_t)t.off_w3, kMlpHidden, id3);
      umma_commit(c.bar_m);
    }
    c.pending = true;
    if (!mbar_wait(c.bar_m, c.ph, c.polls)) *s_abort = 1;
    else c.pending = false;
    c.ph ^= 1u;
    tc_fence_after();
    if (layer < 2) {
      const float* bl = bias + layer * kMlpHidden;
      hidden_epilogue_ta(c.tmem + lane_addr, bl, a_col, 0);
      hidden_epilogue_ta(c.tmem + lane_addr + 32u, bl, a_col, 32);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    } else {
      for (int c0 = 0; c0 < t.n3; c0 += 16) {
        float v[16];
        tmem_ld16(c.tmem + lane_addr + (uint32_t)c0, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int k = c0 + i;
          if (act && k < t.K) out[(size_t)k * ostride + oidx] = v[i] + bias[2 * kMlpHidden + k];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  return *s_abort == 0;
}

// Genes that may use the network's proposal in this sweep.
__device__ __forceinline__ bool net_gene(const DevPtrsF32& p, int g, int G) {
  return g < G && (p.mh_all == kMoveNet || p.mh_all == 3 ||
                   (p.mh_all == 0 && p.use_mh[g] == kMoveNet));
}

}  // namespace fbs
