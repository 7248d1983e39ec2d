// Learned error-rate heuristic (Sec. 5.1): a feedforward network with two
// hidden layers of eight ReLU units maps the vehicle's linear and angular
// velocities and its visible-feature count to the mean and standard deviation
// of the Gaussian rate of the position-error magnitude, fitted by maximum
// likelihood; its values over mapped states are interpolated by weighted
// nearest neighbours over position, velocity and yaw.
//
//   z = W3 relu(W2 relu(W1 x + b1) + b2) + b3,  mean = z0,
//   std = softplus(z1) + 1e-3,  loss = mean(log std + (r - mean)^2 / (2 std^2))
//
// The network is tiny (154 parameters): one thread per sample on the CUDA
// cores, parameters in shared memory.  The gradient of a batch is summed per
// block in a fixed order (warp shuffles, then warps in order) and the blocks'
// partial sums are added in block order by the kernel that also takes the Adam
// step, so training is deterministic.
//
// Kernels:
//   k_err_forward   sample -> (mean, std)
//   k_err_grad      per-block partial gradient and loss of a batch
//   k_err_adam      sum of the partials (fixed order) and the Adam step
//   k_err_knn       weighted k nearest mapped states of every query state
//                   (map staged through shared memory in tiles)
//   k_err_levels    the same at the centres of a quality grid, quantised to
//                   the grid form of the heuristic
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"
#include "profile.h"

namespace mpap {

constexpr int kEIn = 7, kEHid = 8, kEOut = 2;
constexpr int kEParams = kEHid * kEIn + kEHid + kEHid * kEHid + kEHid + kEOut * kEHid + kEOut;   // 154
constexpr int oW1 = 0, oB1 = oW1 + kEHid * kEIn, oW2 = oB1 + kEHid, oB2 = oW2 + kEHid * kEHid,
              oW3 = oB2 + kEHid, oB3 = oW3 + kEOut * kEHid;
constexpr float kSigmaMin = 1e-3f;
constexpr int kEThreads = 256;
constexpr int kMaxK = 16;          // neighbours of the map interpolation
constexpr int kKnnTile = 256;      // mapped states per shared-memory tile
static_assert(kEParams == 154, "parameter layout");

}  // namespace mpap

struct mpap_errnet {
  uint32_t max_batch = 0;
  uint32_t step = 0;
  uint32_t max_blocks = 0;
  float* p = nullptr;        // [154] parameters
  float* m = nullptr;        // Adam moments
  float* v = nullptr;
  float* g = nullptr;        // [154] gradient of the last batch
  float* part = nullptr;     // [max_blocks][154] per-block partial gradients
  double* lpart = nullptr;   // [max_blocks] per-block partial losses
  double* loss = nullptr;    // [1]
  float* x_in = nullptr;     // [max_batch][7] host-input staging
  float* r_in = nullptr;     // [max_batch]
  float* out = nullptr;      // [max_batch][2]
};

namespace mpap {

namespace {

__device__ __forceinline__ float softplus_f(float z) { return fmaxf(z, 0.0f) + log1pf(expf(-fabsf(z))); }
__device__ __forceinline__ float sigmoid_f(float z) { return 1.0f / (1.0f + expf(-z)); }

// The forward pass of one sample from parameters P (shared memory): hidden
// pre-activations a1, a2 and outputs z.
__device__ __forceinline__ void err_fwd(const float* P, const float* x, float* a1, float* a2, float* z) {
  for (int j = 0; j < kEHid; ++j) {
    float s = P[oB1 + j];
    for (int i = 0; i < kEIn; ++i) s += P[oW1 + j * kEIn + i] * x[i];
    a1[j] = s;
  }
  for (int j = 0; j < kEHid; ++j) {
    float s = P[oB2 + j];
    for (int i = 0; i < kEHid; ++i) s += P[oW2 + j * kEHid + i] * fmaxf(a1[i], 0.0f);
    a2[j] = s;
  }
  for (int j = 0; j < kEOut; ++j) {
    float s = P[oB3 + j];
    for (int i = 0; i < kEHid; ++i) s += P[oW3 + j * kEHid + i] * fmaxf(a2[i], 0.0f);
    z[j] = s;
  }
}

__global__ void __launch_bounds__(kEThreads) k_err_forward(const float* __restrict__ p, const float* __restrict__ X,
                                                          uint32_t n, float* __restrict__ out) {
  __shared__ float P[kEParams];
  for (int i = threadIdx.x; i < kEParams; i += blockDim.x) P[i] = p[i];
  __syncthreads();
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    float x[kEIn], a1[kEHid], a2[kEHid], z[kEOut];
    for (int i = 0; i < kEIn; ++i) x[i] = X[(size_t)s * kEIn + i];
    err_fwd(P, x, a1, a2, z);
    out[2 * (size_t)s] = z[0];
    out[2 * (size_t)s + 1] = softplus_f(z[1]) + kSigmaMin;
  }
}

// Adds v over the warp; lane 0 holds the sum.
__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
  return v;
}

// One sample per thread (samples beyond n contribute zero); every parameter's
// contribution is summed over the warp, then over the block's warps in order,
// into part[block][*]; the loss likewise into lpart[block].
__global__ void __launch_bounds__(kEThreads) k_err_grad(const float* __restrict__ p, const float* __restrict__ X,
                                                       const float* __restrict__ R, uint32_t n,
                                                       float* __restrict__ part, double* __restrict__ lpart) {
  __shared__ float P[kEParams];
  __shared__ float W[kEThreads / 32][kEParams + 1];   // per-warp sums of the parameters, then the loss
  for (int i = threadIdx.x; i < kEParams; i += blockDim.x) P[i] = p[i];
  __syncthreads();
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool valid = s < n;
  float x[kEIn] = {0, 0, 0, 0, 0, 0, 0}, a1[kEHid], a2[kEHid], z[kEOut];
  float r = 0.0f;
  if (valid) {
    for (int i = 0; i < kEIn; ++i) x[i] = X[(size_t)s * kEIn + i];
    r = R[s];
  }
  err_fwd(P, x, a1, a2, z);
  const float inv_n = 1.0f / (float)n;
  const float sd = softplus_f(z[1]) + kSigmaMin;
  const float e = r - z[0];
  const float lo = valid ? (logf(sd) + e * e / (2.0f * sd * sd)) * inv_n : 0.0f;
  const float dmu = valid ? -e / (sd * sd) * inv_n : 0.0f;
  const float dsd = valid ? (1.0f / sd - e * e / (sd * sd * sd)) * inv_n : 0.0f;
  float dz[kEOut] = {dmu, dsd * sigmoid_f(z[1])};
  // back-propagation, every parameter's contribution reduced on the spot
  auto put = [&](int idx, float v) {
    const float t = warp_sum(v);
    if (lane == 0) W[warp][idx] = t;
  };
  float dh2[kEHid];
  for (int i = 0; i < kEHid; ++i) dh2[i] = 0.0f;
  for (int j = 0; j < kEOut; ++j) {
    for (int i = 0; i < kEHid; ++i) {
      put(oW3 + j * kEHid + i, dz[j] * fmaxf(a2[i], 0.0f));
      dh2[i] += dz[j] * P[oW3 + j * kEHid + i];
    }
    put(oB3 + j, dz[j]);
  }
  float dh1[kEHid];
  for (int i = 0; i < kEHid; ++i) dh1[i] = 0.0f;
  for (int j = 0; j < kEHid; ++j) {
    const float da = a2[j] > 0.0f ? dh2[j] : 0.0f;
    for (int i = 0; i < kEHid; ++i) {
      put(oW2 + j * kEHid + i, da * fmaxf(a1[i], 0.0f));
      dh1[i] += da * P[oW2 + j * kEHid + i];
    }
    put(oB2 + j, da);
  }
  for (int j = 0; j < kEHid; ++j) {
    const float da = a1[j] > 0.0f ? dh1[j] : 0.0f;
    for (int i = 0; i < kEIn; ++i) put(oW1 + j * kEIn + i, da * x[i]);
    put(oB1 + j, da);
  }
  put(kEParams, lo);
  __syncthreads();
  for (int idx = threadIdx.x; idx <= kEParams; idx += blockDim.x) {
    float t = 0.0f;
    for (int wi = 0; wi < kEThreads / 32; ++wi) t += W[wi][idx];
    if (idx < kEParams) part[(size_t)blockIdx.x * kEParams + idx] = t;
    else lpart[blockIdx.x] = (double)t;
  }
}

// Sums the blocks' partial gradients in block order (one thread per
// parameter), then, if apply, one Adam step (bias corrections c1, c2 from the
// host).  Thread kEParams sums the loss.
__global__ void k_err_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v, float* __restrict__ g,
                           const float* __restrict__ part, const double* __restrict__ lpart, uint32_t nblocks,
                           double* __restrict__ loss, float lr, float c1, float c2, int apply) {
  const int i = threadIdx.x;
  if (i == kEParams) {
    double t = 0.0;
    for (uint32_t b = 0; b < nblocks; ++b) t += lpart[b];
    *loss = t;
    return;
  }
  if (i > kEParams) return;
  float t = 0.0f;
  for (uint32_t b = 0; b < nblocks; ++b) t += part[(size_t)b * kEParams + i];
  g[i] = t;
  if (!apply) return;
  const float mi = 0.9f * m[i] + 0.1f * t;
  const float vi = 0.999f * v[i] + 0.001f * t * t;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + 1e-8f);
}

}  // namespace
}  // namespace mpap

namespace mpap {
namespace {

struct KnnArgs {
  const float* ms;    // [N][7] mapped states: position, velocity, yaw
  const float* mv;    // [N][2] mapped (mean, std)
  uint32_t N;
  uint32_t k;
  float wp, wv, wy;   // weights of position, velocity and yaw in the squared distance
};

__device__ __forceinline__ float wrap_pi(float a) {
  const float tau = 6.2831853071795864769f;
  return a - tau * rintf(a / tau);
}

// Weighted k-nearest-neighbour interpolation at state q (when `valid`): the
// map passes through shared memory in tiles, every thread keeps its k best
// (squared distance, index) pairs in increasing order (ties to the lower
// index); weights 1 / (d + 1e-6).  Every thread of the block must call it.
__device__ void knn_one(const KnnArgs& A, const float* q, bool valid, float* ts, float& o_mean, float& o_std) {
  float bd[kMaxK];
  uint32_t bi[kMaxK];
  for (int j = 0; j < kMaxK; ++j) {
    bd[j] = INFINITY;
    bi[j] = 0xFFFFFFFFu;
  }
  const int k = (int)A.k;
  for (uint32_t t0 = 0; t0 < A.N; t0 += kKnnTile) {
    const uint32_t nt = min((uint32_t)kKnnTile, A.N - t0);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nt * kEIn; i += blockDim.x) ts[i] = A.ms[(size_t)t0 * kEIn + i];
    __syncthreads();
    if (!valid) continue;
    for (uint32_t j = 0; j < nt; ++j) {
      const float* s = ts + j * kEIn;
      const float dx = q[0] - s[0], dy = q[1] - s[1], dz = q[2] - s[2];
      const float ex = q[3] - s[3], ey = q[4] - s[4], ez = q[5] - s[5];
      const float dw = wrap_pi(q[6] - s[6]);
      const float d2 = A.wp * (dx * dx + dy * dy + dz * dz) + A.wv * (ex * ex + ey * ey + ez * ez) + A.wy * (dw * dw);
      const uint32_t idx = t0 + j;
      if (d2 < bd[k - 1] || (d2 == bd[k - 1] && idx < bi[k - 1])) {
        int pos = k - 1;
        while (pos > 0 && (d2 < bd[pos - 1] || (d2 == bd[pos - 1] && idx < bi[pos - 1]))) {
          bd[pos] = bd[pos - 1];
          bi[pos] = bi[pos - 1];
          --pos;
        }
        bd[pos] = d2;
        bi[pos] = idx;
      }
    }
  }
  if (!valid) return;
  float sw = 0.0f, sm = 0.0f, ss = 0.0f;
  for (int j = 0; j < k; ++j) {
    const float wt = 1.0f / (sqrtf(bd[j]) + 1e-6f);
    sw += wt;
    sm += wt * A.mv[2 * (size_t)bi[j]];
    ss += wt * A.mv[2 * (size_t)bi[j] + 1];
  }
  o_mean = sm / sw;
  o_std = ss / sw;
}

__global__ void __launch_bounds__(kEThreads) k_err_knn(KnnArgs A, const float* __restrict__ Q, uint32_t nq,
                                                      float* __restrict__ out) {
  __shared__ float ts[kKnnTile * kEIn];
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < nq;
  float q[kEIn];
  for (int c = 0; c < kEIn; ++c) q[c] = valid ? Q[(size_t)i * kEIn + c] : 0.0f;
  float a = 0.0f, b = 0.0f;
  knn_one(A, q, valid, ts, a, b);
  if (valid) {
    out[2 * (size_t)i] = a;
    out[2 * (size_t)i + 1] = b;
  }
}

// The interpolated mean rate at every cell centre ((2 i + 1) / (2 G), ...) of a
// G^dp grid (x fastest; z = 0 in 2D), for one velocity and yaw, as a level of
// the grid form of the heuristic: clamp(floor(n_f (1 - mean / mu_ref) + 1/2), 0, K).
__global__ void __launch_bounds__(kEThreads) k_err_levels(KnnArgs A, int G, int dp, float vx, float vy, float vz,
                                                         float yaw, float mu_ref, int n_f, int K,
                                                         uint8_t* __restrict__ levels) {
  __shared__ float ts[kKnnTile * kEIn];
  const uint32_t cells = dp == 2 ? (uint32_t)(G * G) : (uint32_t)(G * G * G);
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = c < cells;
  const uint32_t ix = c % G, iy = (c / G) % G, iz = dp == 2 ? 0u : c / (uint32_t)(G * G);
  const float inv = 1.0f / (2.0f * (float)G);
  float q[kEIn] = {(2.0f * ix + 1.0f) * inv, (2.0f * iy + 1.0f) * inv, dp == 2 ? 0.0f : (2.0f * iz + 1.0f) * inv,
                   vx, vy, vz, yaw};
  float mean = 0.0f, sd = 0.0f;
  knn_one(A, q, valid, ts, mean, sd);
  if (valid) {
    const float x = floorf((float)n_f * (1.0f - mean / mu_ref) + 0.5f);
    levels[c] = (uint8_t)fminf(fmaxf(x, 0.0f), (float)K);
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
void errnet_free(mpap_errnet* n) {
  if (!n) return;
  void* ptrs[] = {n->p, n->m, n->v, n->g, n->part, n->lpart, n->loss, n->x_in, n->r_in, n->out};
  for (void* q : ptrs) cudaFree(q);
  delete n;
}

}  // namespace mpap

#include <random>

namespace {

cudaStream_t Se(void* s) { return static_cast<cudaStream_t>(s); }

template <typename T>
bool ealloc(T** p, size_t n) {
  return mpap::cuda_ok(cudaMalloc((void**)p, (n ? n : 1) * sizeof(T)), "cudaMalloc(errnet)");
}

uint32_t grid_for(uint32_t n) { return std::max(1u, (n + mpap::kEThreads - 1) / mpap::kEThreads); }

}  // namespace

extern "C" {

int32_t mpap_errnet_create(uint64_t seed, uint32_t max_batch, mpap_errnet** out) {
  using namespace mpap;
  if (!out || max_batch == 0 || max_batch > (1u << 24)) {
    set_error("errnet_create: max_batch must be in [1, 2^24]");
    return MPAP_ERR_INVALID_ARG;
  }
  mpap_errnet* n = new mpap_errnet();
  n->max_batch = max_batch;
  n->max_blocks = grid_for(max_batch);
  if (!(ealloc(&n->p, kEParams) && ealloc(&n->m, kEParams) && ealloc(&n->v, kEParams) && ealloc(&n->g, kEParams) &&
        ealloc(&n->part, (size_t)n->max_blocks * kEParams) && ealloc(&n->lpart, n->max_blocks) &&
        ealloc(&n->loss, 1) && ealloc(&n->x_in, (size_t)max_batch * kEIn) && ealloc(&n->r_in, max_batch) &&
        ealloc(&n->out, (size_t)max_batch * 2))) {
    errnet_free(n);
    return MPAP_ERR_CUDA;
  }
  // weights uniform in +-1/sqrt(fan in), biases zero
  std::vector<float> p(kEParams, 0.0f);
  std::mt19937_64 rng(seed);
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  auto fill = [&](int off, int rows, int cols) {
    const double s = 1.0 / std::sqrt((double)cols);
    for (int i = 0; i < rows * cols; ++i) p[off + i] = (float)(s * u(rng));
  };
  fill(oW1, kEHid, kEIn);
  fill(oW2, kEHid, kEHid);
  fill(oW3, kEOut, kEHid);
  if (!cuda_ok(cudaMemcpy(n->p, p.data(), sizeof(float) * kEParams, cudaMemcpyHostToDevice), "errnet params") ||
      !cuda_ok(cudaMemset(n->m, 0, sizeof(float) * kEParams), "errnet m") ||
      !cuda_ok(cudaMemset(n->v, 0, sizeof(float) * kEParams), "errnet v")) {
    errnet_free(n);
    return MPAP_ERR_CUDA;
  }
  *out = n;
  return MPAP_OK;
}

void mpap_errnet_free(mpap_errnet* n) { mpap::errnet_free(n); }

int32_t mpap_errnet_get_params(mpap_errnet* n, float* params, void* stream) {
  if (!n || !params) {
    mpap::set_error("errnet_get_params: null argument");
    return MPAP_ERR_INVALID_ARG;
  }
  MPAP_CK(cudaMemcpyAsync(params, n->p, sizeof(float) * mpap::kEParams, cudaMemcpyDeviceToHost, Se(stream)));
  MPAP_CK(cudaStreamSynchronize(Se(stream)));
  return MPAP_OK;
}

int32_t mpap_errnet_set_params(mpap_errnet* n, const float* params, void* stream) {
  if (!n || !params) {
    mpap::set_error("errnet_set_params: null argument");
    return MPAP_ERR_INVALID_ARG;
  }
  const cudaStream_t st = Se(stream);
  MPAP_CK(cudaMemcpyAsync(n->p, params, sizeof(float) * mpap::kEParams, cudaMemcpyHostToDevice, st));
  MPAP_CK(cudaMemsetAsync(n->m, 0, sizeof(float) * mpap::kEParams, st));
  MPAP_CK(cudaMemsetAsync(n->v, 0, sizeof(float) * mpap::kEParams, st));
  MPAP_CK(cudaStreamSynchronize(st));
  n->step = 0;
  return MPAP_OK;
}

int32_t mpap_errnet_forward(mpap_errnet* n, const float* x, uint32_t cnt, float* out, int32_t mem, void* stream) {
  using namespace mpap;
  if (!n || !x || !out || cnt > n->max_batch) {
    set_error("errnet_forward: null argument or more than max_batch samples");
    return MPAP_ERR_INVALID_ARG;
  }
  if (cnt == 0) return MPAP_OK;
  const cudaStream_t st = Se(stream);
  const bool dev = mem == MPAP_MEM_DEVICE;
  const float* dx = x;
  float* dout = dev ? out : n->out;
  if (!dev) {
    MPAP_CK(cudaMemcpyAsync(n->x_in, x, sizeof(float) * kEIn * (size_t)cnt, cudaMemcpyHostToDevice, st));
    dx = n->x_in;
  }
  {
    LaunchScope ls(st, "k_err_forward");
    k_err_forward<<<grid_for(cnt), kEThreads, 0, st>>>(n->p, dx, cnt, dout);
  }
  MPAP_CK(cudaGetLastError());
  if (!dev) {
    MPAP_CK(cudaMemcpyAsync(out, n->out, sizeof(float) * 2 * (size_t)cnt, cudaMemcpyDeviceToHost, st));
    MPAP_CK(cudaStreamSynchronize(st));
  }
  return MPAP_OK;
}

int32_t mpap_errnet_train_step(mpap_errnet* n, const float* x, const float* r, uint32_t cnt, float lr, int32_t apply,
                               float* loss, float* grads, int32_t mem, void* stream) {
  using namespace mpap;
  if (!n || !x || !r || cnt == 0 || cnt > n->max_batch) {
    set_error("errnet_train_step: null argument or a batch outside [1, max_batch]");
    return MPAP_ERR_INVALID_ARG;
  }
  const cudaStream_t st = Se(stream);
  const bool dev = mem == MPAP_MEM_DEVICE;
  const float* dx = x;
  const float* dr = r;
  if (!dev) {
    MPAP_CK(cudaMemcpyAsync(n->x_in, x, sizeof(float) * kEIn * (size_t)cnt, cudaMemcpyHostToDevice, st));
    MPAP_CK(cudaMemcpyAsync(n->r_in, r, sizeof(float) * (size_t)cnt, cudaMemcpyHostToDevice, st));
    dx = n->x_in;
    dr = n->r_in;
  }
  const uint32_t nb = grid_for(cnt);
  if (apply) n->step += 1;
  const double c1 = 1.0 / (1.0 - std::pow(0.9, (double)std::max(1u, n->step)));
  const double c2 = 1.0 / (1.0 - std::pow(0.999, (double)std::max(1u, n->step)));
  {
    LaunchScope ls(st, "k_err_grad");
    k_err_grad<<<nb, kEThreads, 0, st>>>(n->p, dx, dr, cnt, n->part, n->lpart);
  }
  {
    LaunchScope ls(st, "k_err_adam");
    k_err_adam<<<1, 160, 0, st>>>(n->p, n->m, n->v, n->g, n->part, n->lpart, nb, n->loss, lr, (float)c1, (float)c2,
                                  apply ? 1 : 0);
  }
  MPAP_CK(cudaGetLastError());
  if (grads)
    MPAP_CK(cudaMemcpyAsync(grads, n->g, sizeof(float) * kEParams, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            st));
  if (loss) {
    double l = 0.0;
    MPAP_CK(cudaMemcpyAsync(&l, n->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    MPAP_CK(cudaStreamSynchronize(st));
    *loss = (float)l;
  } else if (!dev && grads) {
    MPAP_CK(cudaStreamSynchronize(st));
  }
  return MPAP_OK;
}

}  // extern "C"

namespace {

// Device copies of the map (and optional extra blocks) for host inputs; a
// no-op for device inputs.  Frees its scratch on destruction.
struct MapStage {
  char* blk = nullptr;
  cudaStream_t st;
  explicit MapStage(cudaStream_t s) : st(s) {}
  ~MapStage() {
    if (blk) mpap::scratch_free(blk, st);
  }
};

int32_t map_args(const float* ms, const float* mv, uint32_t N, uint32_t k, const float* w, mpap::KnnArgs* A) {
  if (!ms || !mv || !w || N == 0 || k == 0 || k > (uint32_t)mpap::kMaxK) {
    mpap::set_error("errmap: null arrays, an empty map or k outside [1, 16]");
    return MPAP_ERR_INVALID_ARG;
  }
  if (!(w[0] >= 0.0f) || !(w[1] >= 0.0f) || !(w[2] >= 0.0f)) {
    mpap::set_error("errmap: distance weights must be non-negative");
    return MPAP_ERR_INVALID_ARG;
  }
  A->ms = ms;
  A->mv = mv;
  A->N = N;
  A->k = std::min(k, N);
  A->wp = w[0];
  A->wv = w[1];
  A->wy = w[2];
  return MPAP_OK;
}

}  // namespace

extern "C" {

int32_t mpap_errmap_query(const float* map_state, const float* map_val, uint32_t n_map, const float* q, uint32_t n_q,
                          uint32_t k, const float* w, float* out, int32_t mem, void* stream) {
  using namespace mpap;
  KnnArgs A;
  float wh[3] = {0, 0, 0};
  if (w) std::memcpy(wh, w, sizeof(wh));
  int32_t rc = map_args(map_state, map_val, n_map, k, w ? wh : nullptr, &A);
  if (rc) return rc;
  if (!q || !out) {
    set_error("errmap_query: null queries or output");
    return MPAP_ERR_INVALID_ARG;
  }
  if (n_q == 0) return MPAP_OK;
  const cudaStream_t st = Se(stream);
  MapStage stage(st);
  const float* dq = q;
  float* dout = out;
  if (mem != MPAP_MEM_DEVICE) {
    const size_t bs = ((size_t)n_map * kEIn * 4 + 255) & ~(size_t)255, bv = ((size_t)n_map * 8 + 255) & ~(size_t)255,
                 bq = ((size_t)n_q * kEIn * 4 + 255) & ~(size_t)255;
    MPAP_CK(scratch_alloc((void**)&stage.blk, bs + bv + bq + (size_t)n_q * 8, st));
    float* ds = reinterpret_cast<float*>(stage.blk);
    float* dv = reinterpret_cast<float*>(stage.blk + bs);
    float* dqq = reinterpret_cast<float*>(stage.blk + bs + bv);
    dout = reinterpret_cast<float*>(stage.blk + bs + bv + bq);
    MPAP_CK(cudaMemcpyAsync(ds, map_state, (size_t)n_map * kEIn * 4, cudaMemcpyHostToDevice, st));
    MPAP_CK(cudaMemcpyAsync(dv, map_val, (size_t)n_map * 8, cudaMemcpyHostToDevice, st));
    MPAP_CK(cudaMemcpyAsync(dqq, q, (size_t)n_q * kEIn * 4, cudaMemcpyHostToDevice, st));
    A.ms = ds;
    A.mv = dv;
    dq = dqq;
  }
  {
    LaunchScope ls(st, "k_err_knn");
    k_err_knn<<<grid_for(n_q), kEThreads, 0, st>>>(A, dq, n_q, dout);
  }
  MPAP_CK(cudaGetLastError());
  if (mem != MPAP_MEM_DEVICE) {
    MPAP_CK(cudaMemcpyAsync(out, dout, (size_t)n_q * 8, cudaMemcpyDeviceToHost, st));
    MPAP_CK(cudaStreamSynchronize(st));
  }
  return MPAP_OK;
}

int32_t mpap_errmap_levels(const float* map_state, const float* map_val, uint32_t n_map, uint32_t k, const float* w,
                           int32_t dim_kind, int32_t grid_G, const float* vel, float yaw, float mu_ref, int32_t n_f,
                           int32_t K, uint8_t* levels, int32_t mem, void* stream) {
  using namespace mpap;
  KnnArgs A;
  float wh[3] = {0, 0, 0};
  if (w) std::memcpy(wh, w, sizeof(wh));
  int32_t rc = map_args(map_state, map_val, n_map, k, w ? wh : nullptr, &A);
  if (rc) return rc;
  if ((dim_kind != MPAP_DIM_2D && dim_kind != MPAP_DIM_3D && dim_kind != MPAP_DIM_DI6) || grid_G < 1 ||
      grid_G > 1024 || (grid_G & (grid_G - 1)) || !vel || !levels || !(mu_ref > 0.0f) || n_f < 0 || K < 0 || K > 255) {
    set_error("errmap_levels: bad dimension, grid size (a power of two in [1, 1024]), velocity, output, mu_ref > 0 "
              "or levels");
    return MPAP_ERR_INVALID_ARG;
  }
  const int dp = dim_kind == MPAP_DIM_2D ? 2 : 3;
  const uint64_t cells = dp == 2 ? (uint64_t)grid_G * grid_G : (uint64_t)grid_G * grid_G * grid_G;
  if (cells > (1ull << 31)) {
    set_error("errmap_levels: grid too large");
    return MPAP_ERR_INVALID_ARG;
  }
  const cudaStream_t st = Se(stream);
  MapStage stage(st);
  uint8_t* dl = levels;
  if (mem != MPAP_MEM_DEVICE) {
    const size_t bs = ((size_t)n_map * kEIn * 4 + 255) & ~(size_t)255, bv = ((size_t)n_map * 8 + 255) & ~(size_t)255;
    MPAP_CK(scratch_alloc((void**)&stage.blk, bs + bv + cells, st));
    float* ds = reinterpret_cast<float*>(stage.blk);
    float* dv = reinterpret_cast<float*>(stage.blk + bs);
    dl = reinterpret_cast<uint8_t*>(stage.blk + bs + bv);
    MPAP_CK(cudaMemcpyAsync(ds, map_state, (size_t)n_map * kEIn * 4, cudaMemcpyHostToDevice, st));
    MPAP_CK(cudaMemcpyAsync(dv, map_val, (size_t)n_map * 8, cudaMemcpyHostToDevice, st));
    A.ms = ds;
    A.mv = dv;
  }
  {
    LaunchScope ls(st, "k_err_levels");
    k_err_levels<<<grid_for((uint32_t)cells), kEThreads, 0, st>>>(A, grid_G, dp, vel[0], vel[1], vel[2], yaw, mu_ref,
                                                                  n_f, K, dl);
  }
  MPAP_CK(cudaGetLastError());
  if (mem != MPAP_MEM_DEVICE) {
    MPAP_CK(cudaMemcpyAsync(levels, dl, cells, cudaMemcpyDeviceToHost, st));
    MPAP_CK(cudaStreamSynchronize(st));
  }
  return MPAP_OK;
}

}  // extern "C"
