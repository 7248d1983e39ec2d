// Learned certification surrogate: a 48 -> 128 -> 128 -> 128 -> 2 ReLU MLP that
// predicts, from 48 trajectory features of a candidate goal plan, the collision
// and localisation failure probabilities that Monte Carlo certification (Alg. 1
// step 4) would measure.  BF16 weights and activations, FP32 accumulation, FP32
// master weights trained with Adam on binary cross-entropy against MC hit rates.
//
// Every matrix product runs on the 5th-generation tensor cores: k_gemm_tc stages
// 128 x 64 (A) and N x 64 (B) BF16 tiles in shared memory in the no-swizzle
// K-major core-matrix layout (8 rows x 16 bytes per core matrix), one thread
// issues tcgen05.mma (M = 128, N <= 256, K = 16) into an FP32 accumulator in
// tensor memory, completion is signalled through an mbarrier (tcgen05.commit),
// and the four warps read their 32 accumulator lanes with tcgen05.ld for a fused
// epilogue.  Waits are bounded; a timeout sets an error word instead of hanging.
//
// Activation layout for a padded batch Bt (multiple of 128): X [Bt x 64] bf16
// (features 48..63 zero) and its transpose [64 x Bt]; H1..H3 [Bt x 128] bf16 and
// their transposes; logits [Bt x 16] fp32 (columns 2..15 unused).  Transposed
// copies feed the weight-gradient products dW = dZ^T X (K = batch).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"
#include "profile.h"

namespace mpap {

constexpr int kIn = 48, kInPad = 64, kHid = 128, kOut = 2, kOutPad = 16;
// packed parameter layout (also the ABI's): W1[128][48] b1[128] W2[128][128] b2
// W3[128][128] b3 W4[2][128] b4[2]
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kHid * kIn;
constexpr int kOffW2 = kOffB1 + kHid;
constexpr int kOffB2 = kOffW2 + kHid * kHid;
constexpr int kOffW3 = kOffB2 + kHid;
constexpr int kOffB3 = kOffW3 + kHid * kHid;
constexpr int kOffW4 = kOffB3 + kHid;
constexpr int kOffB4 = kOffW4 + kOut * kHid;
constexpr int kParams = kOffB4 + kOut;

typedef __nv_bfloat16 bf16;

// ---------------------------------------------------------------------------
// tcgen05 GEMM: C[M x N] = A[M x K] B[N x K]^T, A and B bf16 row-major with K
// contiguous (K-major).  One CTA (4 warps) per 128-row tile and K split.
// ---------------------------------------------------------------------------
enum { kEpiReluBf16 = 0, kEpiF32 = 1, kEpiF32Atomic = 2, kEpiMaskBf16 = 3 };

struct GemmArgs {
  const bf16* A;
  int lda;
  const bf16* B;
  int ldb;
  int M, N, K;       // M % 128 == 0, N % 16 == 0 and N <= 256, K % 64 == 0
  int k_split;       // K per CTA along gridDim.y (multiple of 64)
  int epi;
  const float* bias;    // [N] (optional)
  const bf16* mask;     // [M x N] (kEpiMaskBf16)
  bf16* out_bf;         // [M x N]
  bf16* out_bf_t;       // [N x M] (optional)
  float* out_f;         // [M x ldo]
  int ldo;
  uint32_t* err;
};

constexpr int kGemmThreads = 128;
constexpr uint32_t kTileBytesA = 128 * 64 * 2;   // 16 KB
constexpr uint32_t kGemmSmem = kTileBytesA + 256 * 64 * 2 + 1024;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start address, leading (K-direction) and
// stride (row-group direction) byte offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1u << 46;
  return d;
}

// Instruction descriptor for kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, shape M x N.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t tmem_cols_for(int N) {
  uint32_t c = 32;
  while (c < (uint32_t)N) c <<= 1;
  return c;
}

__global__ void __launch_bounds__(kGemmThreads) k_gemm_tc(GemmArgs g) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) unsigned long long s_mbar;
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t pad = ((raw + 1023u) & ~1023u) - raw;
  unsigned char* sA = smem_raw + pad;
  unsigned char* sB = sA + kTileBytesA;
  const uint32_t aA = smem_u32(sA), aB = smem_u32(sB);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * 128;
  const int kb = blockIdx.y * g.k_split;
  const int ke = min(g.K, kb + g.k_split);
  const uint32_t ncols = tmem_cols_for(g.N);
  const uint32_t mb = smem_u32(&s_mbar);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = s_tmem;
  const uint32_t idesc = umma_idesc_bf16(128, g.N);
  uint32_t phase = 0;
  bool timed_out = false;
  bool any = false;
  for (int k0 = kb; k0 < ke && !timed_out; k0 += 64) {
    // stage the A (128 x 64) and B (N x 64) tiles: core matrix (row group r/8,
    // k group kg) at byte (8 (r/8) + kg) * 128, row r%8 at +16 (r%8)
    for (int c = tid; c < 128 * 8; c += kGemmThreads) {
      const int r = c >> 3, kg = c & 7;
      const uint4 v = *reinterpret_cast<const uint4*>(g.A + (size_t)(m0 + r) * g.lda + k0 + kg * 8);
      *reinterpret_cast<uint4*>(sA + ((r >> 3) * 8 + kg) * 128 + (r & 7) * 16) = v;
    }
    for (int c = tid; c < g.N * 8; c += kGemmThreads) {
      const int r = c >> 3, kg = c & 7;
      const uint4 v = *reinterpret_cast<const uint4*>(g.B + (size_t)r * g.ldb + k0 + kg * 8);
      *reinterpret_cast<uint4*>(sB + ((r >> 3) * 8 + kg) * 128 + (r & 7) * 16) = v;
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const uint64_t ad = umma_desc(aA + s * 256, 128, 1024);
        const uint64_t bd = umma_desc(aB + s * 256, 128, 1024);
        const uint32_t acc = (any || s > 0) ? 1u : 0u;
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
                tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb));
    }
    any = true;
    // bounded wait for the tile's MMAs (shared-memory reuse and the result):
    // one second of GPU timer time, far beyond any healthy tile, so that it
    // only ends a kernel whose MMAs never complete.  This is a last resort: the
    // teardown below then frees tensor memory that MMAs still in flight may
    // write, so it reports MPAP_ERR_TIMEOUT rather than recovering.
    uint32_t done = 0;
    unsigned long long t0 = 0, t = 0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    while (!done) {
      asm volatile(
          "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
          : "=r"(done)
          : "r"(mb), "r"(phase));
      if (done) break;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (t - t0 > 1000000000ull) break;
    }
    phase ^= 1u;
    // one decision for the whole CTA, so every thread leaves the loop together
    if (__syncthreads_or(!done)) {
      timed_out = true;
      if (tid == 0) atomicOr(g.err, 1u);
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (any && !timed_out) {
    const int row = m0 + warp * 32 + lane;
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    for (int c0 = 0; c0 < g.N; c0 += 16) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr + (uint32_t)c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int col = c0 + j;
        float v = __uint_as_float(r[j]);
        if (g.epi == kEpiReluBf16) {
          if (g.bias) v += g.bias[col];
          v = fmaxf(v, 0.0f);
          const bf16 b = __float2bfloat16_rn(v);
          g.out_bf[(size_t)row * g.N + col] = b;
          if (g.out_bf_t) g.out_bf_t[(size_t)col * g.M + row] = b;
        } else if (g.epi == kEpiF32) {
          if (g.bias) v += g.bias[col];
          g.out_f[(size_t)row * g.ldo + col] = v;
        } else if (g.epi == kEpiF32Atomic) {
          atomicAdd(&g.out_f[(size_t)row * g.ldo + col], v);
        } else {
          const float mk = __bfloat162float(g.mask[(size_t)row * g.N + col]);
          const bf16 b = __float2bfloat16_rn(mk > 0.0f ? v : 0.0f);
          g.out_bf[(size_t)row * g.N + col] = b;
          if (g.out_bf_t) g.out_bf_t[(size_t)col * g.M + row] = b;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// ---------------------------------------------------------------------------
// Elementwise and reduction kernels
// ---------------------------------------------------------------------------
__global__ void k_mlp_prep_x(const float* __restrict__ x, uint32_t n, uint32_t Bt, bf16* __restrict__ xb,
                             bf16* __restrict__ xbt) {
  const uint32_t total = Bt * kInPad;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const uint32_t r = i / kInPad, c = i % kInPad;
    const float v = (r < n && c < (uint32_t)kIn) ? x[(size_t)r * kIn + c] : 0.0f;
    const bf16 b = __float2bfloat16_rn(v);
    xb[i] = b;
    xbt[(size_t)c * Bt + r] = b;
  }
}

// logits -> probabilities; loss and dL/dz for binary cross-entropy averaged over
// the n samples and the two outputs (dz = 0 on padded rows).
__global__ void k_mlp_loss(const float* __restrict__ logits, const float* __restrict__ y, uint32_t n, uint32_t Bt,
                           float* __restrict__ prob, float* __restrict__ dz, double* loss) {
  double local = 0.0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < Bt * kOut; i += gridDim.x * blockDim.x) {
    const uint32_t r = i / kOut, o = i % kOut;
    const float z = logits[(size_t)r * kOutPad + o];
    const float p = 1.0f / (1.0f + expf(-z));
    if (r < n) {
      if (prob) prob[(size_t)r * kOut + o] = p;
      if (y) {
        const float t = y[(size_t)r * kOut + o];
        dz[i] = (p - t) / (float)(2 * n);
        const float sp = z > 0.0f ? z + log1pf(expf(-z)) : log1pf(expf(z));
        local += (double)(sp - t * z);
      }
    } else if (dz) {
      dz[i] = 0.0f;
    }
  }
  if (loss) {
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xFFFFFFFFu, local, o);
    if ((threadIdx.x & 31) == 0 && local != 0.0) atomicAdd(loss, local / (double)(2 * n));
  }
}

// Output layer backward: dH3 = dz W4 (bf16 weights), masked by ReLU(H3) and
// rounded to bf16 (row-major and transposed); the 2 x 128 weight gradient and
// bias gradient of the output layer.
__global__ void k_mlp_out_back(const float* __restrict__ dz, const bf16* __restrict__ w4b,
                               const bf16* __restrict__ h3, uint32_t Bt, bf16* __restrict__ dz3,
                               bf16* __restrict__ dz3t) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < Bt * kHid; i += gridDim.x * blockDim.x) {
    const uint32_t r = i / kHid, k = i % kHid;
    float v = dz[(size_t)r * kOut + 0] * __bfloat162float(w4b[0 * kHid + k]);
    v += dz[(size_t)r * kOut + 1] * __bfloat162float(w4b[1 * kHid + k]);
    const bf16 b = __float2bfloat16_rn(__bfloat162float(h3[i]) > 0.0f ? v : 0.0f);
    dz3[i] = b;
    dz3t[(size_t)k * Bt + r] = b;
  }
}

// Row sums of a [rows x Bt] transposed bf16 matrix (bias gradients), one block
// per row, and the output layer's gradient from dz (fp32) and H3 (transposed).
__global__ void k_mlp_rowsum(const bf16* __restrict__ mt, uint32_t Bt, float* __restrict__ out) {
  float s = 0.0f;
  for (uint32_t c = threadIdx.x; c < Bt; c += blockDim.x) s += __bfloat162float(mt[(size_t)blockIdx.x * Bt + c]);
  __shared__ float red[32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    float t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
    if (threadIdx.x == 0) out[blockIdx.x] = t;
  }
}

__global__ void k_mlp_out_grad(const float* __restrict__ dz, const bf16* __restrict__ h3t, uint32_t Bt,
                               float* __restrict__ gw4, float* __restrict__ gb4) {
  // block k in [0, 128] (k = 128: bias), both outputs
  const uint32_t k = blockIdx.x;
  float s0 = 0.0f, s1 = 0.0f;
  for (uint32_t r = threadIdx.x; r < Bt; r += blockDim.x) {
    const float h = (k < (uint32_t)kHid) ? __bfloat162float(h3t[(size_t)k * Bt + r]) : 1.0f;
    s0 += dz[(size_t)r * kOut + 0] * h;
    s1 += dz[(size_t)r * kOut + 1] * h;
  }
  __shared__ float red[2][32];
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xFFFFFFFFu, s0, o);
    s1 += __shfl_xor_sync(0xFFFFFFFFu, s1, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = s0;
    red[1][threadIdx.x >> 5] = s1;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    float t0 = threadIdx.x < (blockDim.x >> 5) ? red[0][threadIdx.x] : 0.0f;
    float t1 = threadIdx.x < (blockDim.x >> 5) ? red[1][threadIdx.x] : 0.0f;
    for (int o = 16; o > 0; o >>= 1) {
      t0 += __shfl_xor_sync(0xFFFFFFFFu, t0, o);
      t1 += __shfl_xor_sync(0xFFFFFFFFu, t1, o);
    }
    if (threadIdx.x == 0) {
      if (k < (uint32_t)kHid) {
        gw4[0 * kHid + k] = t0;
        gw4[1 * kHid + k] = t1;
      } else {
        gb4[0] = t0;
        gb4[1] = t1;
      }
    }
  }
}

// First-layer weight gradient [128 x 64] -> packed [128 x 48].
__global__ void k_mlp_pack_gw1(const float* __restrict__ g64, float* __restrict__ g48) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < (uint32_t)(kHid * kIn)) g48[i] = g64[(i / kIn) * kInPad + (i % kIn)];
}

// Adam on the packed FP32 parameters.
__global__ void k_mlp_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < (uint32_t)kParams; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// BF16 operand copies of the FP32 master weights: W1 [128 x 64] (zero-padded),
// W2, W3 and their transposes, W4 [16 x 128] (rows 2..15 zero), bias b4 padded to 16.
struct MlpBf {
  bf16 *w1, *w2, *w3, *w4, *w2t, *w3t;
  float* b4p;
};

__global__ void k_mlp_refresh(const float* __restrict__ p, MlpBf o) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < (uint32_t)(kHid * kInPad)) {
    const uint32_t r = i / kInPad, c = i % kInPad;
    o.w1[i] = __float2bfloat16_rn(c < (uint32_t)kIn ? p[kOffW1 + r * kIn + c] : 0.0f);
  }
  if (i < (uint32_t)(kHid * kHid)) {
    const uint32_t r = i / kHid, c = i % kHid;
    o.w2[i] = __float2bfloat16_rn(p[kOffW2 + i]);
    o.w3[i] = __float2bfloat16_rn(p[kOffW3 + i]);
    o.w2t[i] = __float2bfloat16_rn(p[kOffW2 + c * kHid + r]);
    o.w3t[i] = __float2bfloat16_rn(p[kOffW3 + c * kHid + r]);
  }
  if (i < (uint32_t)(kOutPad * kHid)) {
    const uint32_t r = i / kHid;
    o.w4[i] = __float2bfloat16_rn(r < (uint32_t)kOut ? p[kOffW4 + i] : 0.0f);
  }
  if (i < (uint32_t)kOutPad) o.b4p[i] = i < (uint32_t)kOut ? p[kOffB4 + i] : 0.0f;
}

// Deterministic initialisation: U(-1/sqrt(fan_in), 1/sqrt(fan_in)) for weights,
// zero biases, from Philox4x32-10 (counter = parameter index, key = seed).
__global__ void k_mlp_init(float* __restrict__ p, uint32_t key0, uint32_t key1) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (uint32_t)kParams) return;
  int fan = 0;
  if (i < (uint32_t)kOffB1) fan = kIn;
  else if (i >= (uint32_t)kOffW2 && i < (uint32_t)kOffB2) fan = kHid;
  else if (i >= (uint32_t)kOffW3 && i < (uint32_t)kOffB3) fan = kHid;
  else if (i >= (uint32_t)kOffW4 && i < (uint32_t)kOffB4) fan = kHid;
  if (!fan) {
    p[i] = 0.0f;
    return;
  }
  uint32_t w0 = i, w1 = 0x4D4C50u, w2 = 0, w3 = 0;
  philox4x32_10(w0, w1, w2, w3, key0, key1);
  const float u = unit24(w0);
  p[i] = (2.0f * u - 1.0f) / sqrtf((float)fan);
}

}  // namespace mpap

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct mpap_mlp {
  uint32_t max_batch = 0;   // padded to a multiple of 128
  uint32_t step = 0;
  float* p = nullptr;       // [kParams] fp32 master weights
  float* g = nullptr;       // [kParams] gradients
  float* m = nullptr;       // Adam moments
  float* v = nullptr;
  float* gw1 = nullptr;     // [128 x 64] first-layer gradient before packing
  mpap::MlpBf bf{};
  // activations
  mpap::bf16 *xb = nullptr, *xbt = nullptr, *h[3] = {nullptr, nullptr, nullptr}, *ht[3] = {nullptr, nullptr, nullptr};
  mpap::bf16 *dzb[3] = {nullptr, nullptr, nullptr}, *dzt[3] = {nullptr, nullptr, nullptr};
  float* logits = nullptr;  // [Bt x 16]
  float* dz4 = nullptr;     // [Bt x 2]
  float* x_in = nullptr;    // [Bt x 48] staging for host inputs
  float* y_in = nullptr;    // [Bt x 2]
  float* prob = nullptr;    // [Bt x 2]
  double* loss = nullptr;
  uint32_t* err = nullptr;
};

namespace mpap {

namespace {

void mlp_release(mpap_mlp* n) {
  void* ptrs[] = {n->p, n->g, n->m, n->v, n->gw1, n->bf.w1, n->bf.w2, n->bf.w3, n->bf.w4, n->bf.w2t, n->bf.w3t,
                  n->bf.b4p, n->xb, n->xbt, n->h[0], n->h[1], n->h[2], n->ht[0], n->ht[1], n->ht[2],
                  n->dzb[0], n->dzb[1], n->dzb[2], n->dzt[0], n->dzt[1], n->dzt[2], n->logits, n->dz4,
                  n->x_in, n->y_in, n->prob, n->loss, n->err};
  for (void* q : ptrs) cudaFree(q);
  delete n;
}

template <typename T>
bool dev(T** p, size_t n) {
  return cuda_ok(cudaMalloc((void**)p, (n ? n : 1) * sizeof(T)), "cudaMalloc(mlp)");
}

int32_t gemm(cudaStream_t st, const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int K, int epi,
             const float* bias, const bf16* mask, bf16* out_bf, bf16* out_bf_t, float* out_f, int ldo, uint32_t* err,
             int splits = 1) {
  GemmArgs a;
  a.A = A;
  a.lda = lda;
  a.B = B;
  a.ldb = ldb;
  a.M = M;
  a.N = N;
  a.K = K;
  int ks = ((K / splits + 63) / 64) * 64;
  if (ks <= 0) ks = 64;
  a.k_split = ks;
  a.epi = epi;
  a.bias = bias;
  a.mask = mask;
  a.out_bf = out_bf;
  a.out_bf_t = out_bf_t;
  a.out_f = out_f;
  a.ldo = ldo;
  a.err = err;
  const dim3 grid(M / 128, (K + ks - 1) / ks);
  LaunchScope ls(st, "k_gemm_tc");
  k_gemm_tc<<<grid, kGemmThreads, kGemmSmem, st>>>(a);
  MPAP_CK(cudaGetLastError());
  return MPAP_OK;
}

void refresh(mpap_mlp* n, cudaStream_t st) {
  LaunchScope ls(st, "k_mlp_refresh");
  k_mlp_refresh<<<(kHid * kHid + 255) / 256, 256, 0, st>>>(n->p, n->bf);
}

// Forward pass on the staged inputs (x_in, n rows): H1..H3 and logits.
int32_t forward(mpap_mlp* nt, uint32_t n, uint32_t Bt, cudaStream_t st) {
  {
    LaunchScope ls(st, "k_mlp_prep_x");
    k_mlp_prep_x<<<(Bt * kInPad + 255) / 256, 256, 0, st>>>(nt->x_in, n, Bt, nt->xb, nt->xbt);
  }
  int32_t rc;
  if ((rc = gemm(st, nt->xb, kInPad, nt->bf.w1, kInPad, Bt, kHid, kInPad, kEpiReluBf16, nt->p + kOffB1, nullptr,
                 nt->h[0], nt->ht[0], nullptr, 0, nt->err)))
    return rc;
  if ((rc = gemm(st, nt->h[0], kHid, nt->bf.w2, kHid, Bt, kHid, kHid, kEpiReluBf16, nt->p + kOffB2, nullptr,
                 nt->h[1], nt->ht[1], nullptr, 0, nt->err)))
    return rc;
  if ((rc = gemm(st, nt->h[1], kHid, nt->bf.w3, kHid, Bt, kHid, kHid, kEpiReluBf16, nt->p + kOffB3, nullptr,
                 nt->h[2], nt->ht[2], nullptr, 0, nt->err)))
    return rc;
  return gemm(st, nt->h[2], kHid, nt->bf.w4, kHid, Bt, kOutPad, kHid, kEpiF32, nt->bf.b4p, nullptr, nullptr,
              nullptr, nt->logits, kOutPad, nt->err);
}

}  // namespace

int32_t mlp_create(uint64_t seed, uint32_t max_batch, mpap_mlp** out) {
  if (!out || max_batch == 0 || max_batch > (1u << 22)) {
    set_error("mlp: max_batch must be in [1, 2^22]");
    return MPAP_ERR_INVALID_ARG;
  }
  mpap_mlp* n = new mpap_mlp();
  const uint32_t Bt = (max_batch + 127) / 128 * 128;
  n->max_batch = Bt;
  bool ok = dev(&n->p, kParams) && dev(&n->g, kParams) && dev(&n->m, kParams) && dev(&n->v, kParams) &&
            dev(&n->gw1, kHid * kInPad) && dev(&n->bf.w1, kHid * kInPad) && dev(&n->bf.w2, kHid * kHid) &&
            dev(&n->bf.w3, kHid * kHid) && dev(&n->bf.w4, kOutPad * kHid) && dev(&n->bf.w2t, kHid * kHid) &&
            dev(&n->bf.w3t, kHid * kHid) && dev(&n->bf.b4p, kOutPad) && dev(&n->xb, (size_t)Bt * kInPad) &&
            dev(&n->xbt, (size_t)Bt * kInPad) && dev(&n->logits, (size_t)Bt * kOutPad) &&
            dev(&n->dz4, (size_t)Bt * kOut) && dev(&n->x_in, (size_t)Bt * kIn) && dev(&n->y_in, (size_t)Bt * kOut) &&
            dev(&n->prob, (size_t)Bt * kOut) && dev(&n->loss, 1) && dev(&n->err, 1);
  for (int l = 0; l < 3 && ok; ++l)
    ok = dev(&n->h[l], (size_t)Bt * kHid) && dev(&n->ht[l], (size_t)Bt * kHid) && dev(&n->dzb[l], (size_t)Bt * kHid) &&
         dev(&n->dzt[l], (size_t)Bt * kHid);
  if (!ok) {
    mlp_release(n);
    return MPAP_ERR_CUDA;
  }
  cudaStream_t st = 0;
  cudaMemsetAsync(n->m, 0, sizeof(float) * kParams, st);
  cudaMemsetAsync(n->v, 0, sizeof(float) * kParams, st);
  cudaMemsetAsync(n->err, 0, sizeof(uint32_t), st);
  {
    LaunchScope ls(st, "k_mlp_init");
    k_mlp_init<<<(kParams + 255) / 256, 256, 0, st>>>(n->p, (uint32_t)seed, (uint32_t)(seed >> 32));
  }
  refresh(n, st);
  if (!cuda_ok(cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem),
               "cudaFuncSetAttribute") ||
      !cuda_ok(cudaStreamSynchronize(st), "mlp init")) {
    mlp_release(n);
    return MPAP_ERR_CUDA;
  }
  *out = n;
  return MPAP_OK;
}

void mlp_free(mpap_mlp* n) {
  if (n) mlp_release(n);
}

int32_t mlp_get_params(mpap_mlp* n, float* params, cudaStream_t st) {
  MPAP_CK(cudaMemcpyAsync(params, n->p, sizeof(float) * kParams, cudaMemcpyDeviceToHost, st));
  MPAP_CK(cudaStreamSynchronize(st));
  return MPAP_OK;
}

int32_t mlp_set_params(mpap_mlp* n, const float* params, cudaStream_t st) {
  MPAP_CK(cudaMemcpyAsync(n->p, params, sizeof(float) * kParams, cudaMemcpyHostToDevice, st));
  MPAP_CK(cudaMemsetAsync(n->m, 0, sizeof(float) * kParams, st));
  MPAP_CK(cudaMemsetAsync(n->v, 0, sizeof(float) * kParams, st));
  n->step = 0;
  refresh(n, st);
  MPAP_CK(cudaStreamSynchronize(st));
  return MPAP_OK;
}

static int32_t stage(void* dst, const void* src, size_t bytes, int32_t mem, cudaStream_t st) {
  MPAP_CK(cudaMemcpyAsync(dst, src, bytes, mem == MPAP_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          st));
  return MPAP_OK;
}

static int32_t check_err(mpap_mlp* n, cudaStream_t st) {
  uint32_t e = 0;
  MPAP_CK(cudaMemcpyAsync(&e, n->err, 4, cudaMemcpyDeviceToHost, st));
  MPAP_CK(cudaStreamSynchronize(st));
  if (e) {
    cudaMemsetAsync(n->err, 0, 4, st);
    set_error("mlp: a tensor-core wait timed out");
    return MPAP_ERR_TIMEOUT;
  }
  return MPAP_OK;
}

uint32_t mlp_max_batch(const mpap_mlp* nt) { return nt->max_batch; }

int32_t mlp_forward(mpap_mlp* nt, const float* x, uint32_t n, float* prob, int32_t mem, cudaStream_t st) {
  if (n == 0) return MPAP_OK;
  if (n > nt->max_batch) {
    set_error("mlp_forward: batch %u exceeds max_batch %u", n, nt->max_batch);
    return MPAP_ERR_INVALID_ARG;
  }
  const uint32_t Bt = (n + 127) / 128 * 128;
  int32_t rc;
  if ((rc = stage(nt->x_in, x, sizeof(float) * n * kIn, mem, st))) return rc;
  if ((rc = forward(nt, n, Bt, st))) return rc;
  {
    LaunchScope ls(st, "k_mlp_loss");
    k_mlp_loss<<<(Bt * kOut + 255) / 256, 256, 0, st>>>(nt->logits, nullptr, n, Bt, nt->prob, nullptr, nullptr);
  }
  MPAP_CK(cudaMemcpyAsync(prob, nt->prob, sizeof(float) * n * kOut,
                          mem == MPAP_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  return check_err(nt, st);
}

int32_t mlp_train_step(mpap_mlp* nt, const float* x, const float* y, uint32_t n, float lr, int32_t apply,
                       float* loss_out, float* grads_out, int32_t mem, cudaStream_t st) {
  if (n == 0 || n > nt->max_batch) {
    set_error("mlp_train_step: batch %u not in [1, max_batch %u]", n, nt->max_batch);
    return MPAP_ERR_INVALID_ARG;
  }
  const uint32_t Bt = (n + 127) / 128 * 128;
  int32_t rc;
  if ((rc = stage(nt->x_in, x, sizeof(float) * n * kIn, mem, st)) ||
      (rc = stage(nt->y_in, y, sizeof(float) * n * kOut, mem, st)))
    return rc;
  if ((rc = forward(nt, n, Bt, st))) return rc;
  MPAP_CK(cudaMemsetAsync(nt->loss, 0, sizeof(double), st));
  {
    LaunchScope ls(st, "k_mlp_loss");
    k_mlp_loss<<<(Bt * kOut + 255) / 256, 256, 0, st>>>(nt->logits, nt->y_in, n, Bt, nullptr, nt->dz4, nt->loss);
  }
  float* G = nt->g;
  MPAP_CK(cudaMemsetAsync(G, 0, sizeof(float) * kParams, st));
  MPAP_CK(cudaMemsetAsync(nt->gw1, 0, sizeof(float) * kHid * kInPad, st));
  {
    LaunchScope ls(st, "k_mlp_out_back");
    k_mlp_out_back<<<(Bt * kHid + 255) / 256, 256, 0, st>>>(nt->dz4, nt->bf.w4, nt->h[2], Bt, nt->dzb[2], nt->dzt[2]);
  }
  {
    LaunchScope ls(st, "k_mlp_out_grad");
    k_mlp_out_grad<<<kHid + 1, 256, 0, st>>>(nt->dz4, nt->ht[2], Bt, G + kOffW4, G + kOffB4);
  }
  const int splits = (int)std::max<uint32_t>(1, std::min<uint32_t>(Bt / 256, 64));
  // layer 3: dW3 = dZ3^T H2, db3, dZ2 = (dZ3 W3) masked by H2
  if ((rc = gemm(st, nt->dzt[2], Bt, nt->ht[1], Bt, kHid, kHid, Bt, kEpiF32Atomic, nullptr, nullptr, nullptr, nullptr,
                 G + kOffW3, kHid, nt->err, splits)))
    return rc;
  {
    LaunchScope ls(st, "k_mlp_rowsum");
    k_mlp_rowsum<<<kHid, 256, 0, st>>>(nt->dzt[2], Bt, G + kOffB3);
  }
  if ((rc = gemm(st, nt->dzb[2], kHid, nt->bf.w3t, kHid, Bt, kHid, kHid, kEpiMaskBf16, nullptr, nt->h[1], nt->dzb[1],
                 nt->dzt[1], nullptr, 0, nt->err)))
    return rc;
  // layer 2
  if ((rc = gemm(st, nt->dzt[1], Bt, nt->ht[0], Bt, kHid, kHid, Bt, kEpiF32Atomic, nullptr, nullptr, nullptr, nullptr,
                 G + kOffW2, kHid, nt->err, splits)))
    return rc;
  {
    LaunchScope ls(st, "k_mlp_rowsum");
    k_mlp_rowsum<<<kHid, 256, 0, st>>>(nt->dzt[1], Bt, G + kOffB2);
  }
  if ((rc = gemm(st, nt->dzb[1], kHid, nt->bf.w2t, kHid, Bt, kHid, kHid, kEpiMaskBf16, nullptr, nt->h[0], nt->dzb[0],
                 nt->dzt[0], nullptr, 0, nt->err)))
    return rc;
  // layer 1: dW1 = dZ1^T X (128 x 64, packed to 128 x 48 afterwards)
  if ((rc = gemm(st, nt->dzt[0], Bt, nt->xbt, Bt, kHid, kInPad, Bt, kEpiF32Atomic, nullptr, nullptr, nullptr, nullptr,
                 nt->gw1, kInPad, nt->err, splits)))
    return rc;
  {
    LaunchScope ls(st, "k_mlp_rowsum");
    k_mlp_rowsum<<<kHid, 256, 0, st>>>(nt->dzt[0], Bt, G + kOffB1);
  }
  {
    LaunchScope ls(st, "k_mlp_pack_gw1");
    k_mlp_pack_gw1<<<(kHid * kIn + 255) / 256, 256, 0, st>>>(nt->gw1, G + kOffW1);
  }
  if (apply) {
    nt->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - (float)std::pow((double)b1, (double)nt->step);
    const float c2 = 1.0f - (float)std::pow((double)b2, (double)nt->step);
    {
      LaunchScope ls(st, "k_mlp_adam");
      k_mlp_adam<<<(kParams + 255) / 256, 256, 0, st>>>(nt->p, G, nt->m, nt->v, lr, b1, b2, 1e-8f, c1, c2);
    }
    refresh(nt, st);
  }
  if (loss_out) {
    double l = 0.0;
    MPAP_CK(cudaMemcpyAsync(&l, nt->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    MPAP_CK(cudaStreamSynchronize(st));
    *loss_out = (float)l;
  }
  if (grads_out)
    MPAP_CK(cudaMemcpyAsync(grads_out, G, sizeof(float) * kParams,
                            mem == MPAP_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  return check_err(nt, st);
}

}  // namespace mpap
