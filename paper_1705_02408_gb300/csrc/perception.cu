// Perception quality levels from mapped features: the visible-feature count
// behind the Sec. 4.1 heuristic (a feature counts when it lies in range, inside
// the camera's horizontal field of view and unoccluded by the obstacles),
// evaluated at the centre of every cell of the quality grid for each of Y yaw
// headings, capped at the top level K.  The all-direction table (one heading,
// field of view off) serves as a scene's quality grid.
//
// One thread per (heading, cell); features are staged through shared memory in
// tiles and the boxes are staged whole; each sight line runs the closed-segment
// slab test against every box.  Every float operation is one IEEE operation in
// the order written, so the levels are exact against a sequential restatement.
#include <algorithm>
#include <cmath>

#include "internal.h"
#include "profile.h"

namespace mpap {

namespace {

struct FeatLevelJob {
  int dp, nb, nf, Y, K;
  unsigned long long cells;
  float half;                // half a cell: 0.5 / G
  float cos_half, range2;
  uint32_t G;
  const float* lo;           // [nb][3]
  const float* hi;
  const float* feat;         // [nf][3]
  const float* head;         // [Y][2]
  uint8_t* out;              // [Y][cells], x fastest
};

constexpr int kFeatTile = 512;

template <int DP>
__global__ void __launch_bounds__(256) k_feature_levels(FeatLevelJob J) {
  extern __shared__ float sm[];
  float* s_lo = sm;
  float* s_hi = sm + 3 * J.nb;
  float* s_f = sm + 6 * J.nb;   // [kFeatTile][3]
  for (int i = threadIdx.x; i < 3 * J.nb; i += blockDim.x) {
    s_lo[i] = J.lo[i];
    s_hi[i] = J.hi[i];
  }
  const unsigned long long total = (unsigned long long)J.Y * J.cells;
  const unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = t < total;
  float c[3] = {0.0f, 0.0f, 0.0f};
  float hx = 0.0f, hy = 0.0f;
  if (live) {
    const unsigned long long y = t / J.cells, cell = t % J.cells;
    const unsigned long long i = cell % J.G, j = (cell / J.G) % J.G;
    c[0] = __fmul_rn((float)(2 * i + 1), J.half);
    c[1] = __fmul_rn((float)(2 * j + 1), J.half);
    if (DP == 3) c[2] = __fmul_rn((float)(2 * (cell / ((unsigned long long)J.G * J.G)) + 1), J.half);
    hx = J.head[2 * y];
    hy = J.head[2 * y + 1];
  }
  int count = 0;
  for (int f0 = 0; f0 < J.nf; f0 += kFeatTile) {
    const int nt = min(kFeatTile, J.nf - f0);
    __syncthreads();   // the previous tile is done (the first time: the boxes are in)
    for (int i = threadIdx.x; i < 3 * nt; i += blockDim.x) s_f[i] = J.feat[3 * (size_t)f0 + i];
    __syncthreads();
    if (!live) continue;
    for (int f = 0; f < nt; ++f) {
      float d[3];
      d[0] = __fsub_rn(s_f[3 * f], c[0]);
      d[1] = __fsub_rn(s_f[3 * f + 1], c[1]);
      d[2] = (DP == 3) ? __fsub_rn(s_f[3 * f + 2], c[2]) : 0.0f;
      const float dxy2 = __fadd_rn(__fmul_rn(d[0], d[0]), __fmul_rn(d[1], d[1]));
      const float r2 = (DP == 3) ? __fadd_rn(dxy2, __fmul_rn(d[2], d[2])) : dxy2;
      if (r2 > J.range2) continue;
      const float dot = __fadd_rn(__fmul_rn(hx, d[0]), __fmul_rn(hy, d[1]));
      if (dot < __fmul_rn(J.cos_half, __fsqrt_rn(dxy2))) continue;
      bool blocked = false;
      for (int b = 0; b < J.nb && !blocked; ++b) blocked = seg_hits_box<DP>(c, d, s_lo + 3 * b, s_hi + 3 * b);
      count += blocked ? 0 : 1;
    }
  }
  if (live) J.out[t] = (uint8_t)(count < J.K ? count : J.K);
}

}  // namespace

int32_t feature_levels_impl(int dp, int nb, const float* lo, const float* hi, uint32_t nf, const float* feat,
                            uint32_t G, uint32_t Y, const float* head, float cos_half, float range, int K,
                            uint8_t* out, bool device, cudaStream_t st) {
  const unsigned long long cells = (unsigned long long)G * G * (dp == 3 ? G : 1u);
  const unsigned long long total = (unsigned long long)Y * cells;
  FeatLevelJob J;
  J.dp = dp;
  J.nb = nb;
  J.nf = (int)nf;
  J.Y = (int)Y;
  J.K = K;
  J.cells = cells;
  J.G = G;
  J.half = 0.5f / (float)G;
  J.cos_half = cos_half;
  J.range2 = range * range;
  char* blk = nullptr;
  if (device) {
    J.lo = lo;
    J.hi = hi;
    J.feat = feat;
    J.head = head;
    J.out = out;
  } else {
    // host arrays: one scratch block from the library pool, copied in and out
    const size_t b_box = sizeof(float) * 3 * (size_t)nb, b_feat = sizeof(float) * 3 * (size_t)nf,
                 b_head = sizeof(float) * 2 * (size_t)Y;
    auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
    MPAP_CK(scratch_alloc((void**)&blk, 2 * up(b_box) + up(b_feat) + up(b_head) + up(total) + 256, st));
    float* d_lo = (float*)blk;
    float* d_hi = (float*)(blk + up(b_box));
    float* d_feat = (float*)(blk + 2 * up(b_box));
    float* d_head = (float*)(blk + 2 * up(b_box) + up(b_feat));
    uint8_t* d_out = (uint8_t*)(blk + 2 * up(b_box) + up(b_feat) + up(b_head));
    const bool ok = (!nb || (cuda_ok(cudaMemcpyAsync(d_lo, lo, b_box, cudaMemcpyHostToDevice, st), "copy") &&
                             cuda_ok(cudaMemcpyAsync(d_hi, hi, b_box, cudaMemcpyHostToDevice, st), "copy"))) &&
                    (!nf || cuda_ok(cudaMemcpyAsync(d_feat, feat, b_feat, cudaMemcpyHostToDevice, st), "copy")) &&
                    cuda_ok(cudaMemcpyAsync(d_head, head, b_head, cudaMemcpyHostToDevice, st), "copy");
    if (!ok) {
      scratch_free(blk, st);
      return MPAP_ERR_CUDA;
    }
    J.lo = d_lo;
    J.hi = d_hi;
    J.feat = d_feat;
    J.head = d_head;
    J.out = d_out;
  }
  const size_t smem = sizeof(float) * (6 * (size_t)nb + 3 * (size_t)kFeatTile);
  const unsigned long long blocks = (total + 255) / 256;
  {
    LaunchScope ls(st, "k_feature_levels");
    if (dp == 3) k_feature_levels<3><<<(unsigned)blocks, 256, smem, st>>>(J);
    else k_feature_levels<2><<<(unsigned)blocks, 256, smem, st>>>(J);
  }
  bool ok = cuda_ok(cudaGetLastError(), "k_feature_levels");
  if (!device) {
    ok = ok && cuda_ok(cudaMemcpyAsync(out, J.out, total, cudaMemcpyDeviceToHost, st), "copy");
    scratch_free(blk, st);
    ok = cuda_ok(cudaStreamSynchronize(st), "sync") && ok;
  }
  return ok ? MPAP_OK : MPAP_ERR_CUDA;
}

}  // namespace mpap
