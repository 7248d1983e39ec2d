// Monte Carlo certification of a plan: Alg. 1 step 4 and the final phase of
// Sec. 3 (probability of meeting the localisation bound of Eq. 1 and the
// deviation bound of the robust motion planning problem, by rollouts).
//
// Two kernels per batch of plans:
//   k_mc_checkpoints  one thread per (plan edge, sub-step): the nominal state at
//                     the end of every sub-interval, in 2^-20 fixed point, with its
//                     perception quality level (same connection model and
//                     evaluation order as the roadmap build).
//   k_mc_rollouts     one thread per rollout: an integer error random walk over the
//                     checkpoints (relocalisation contraction, Irwin-Hall(12)
//                     noise from Philox4x32-10), counting localisation and
//                     collision/leave-map failures.
// and, for the closed-loop VIO model of Sec. 4.1 (mpap_certify_vio_batch),
//   k_vio_gains       one thread per plan: the Kalman gains of every checkpoint
//                     step from the covariance recursion (double, then Q16);
//   k_vio_rollouts    one thread per rollout: LQR tracking from the estimate,
//                     inertial prediction and Kalman position fixes per axis in
//                     integer arithmetic, the same failure events.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.h"
#include "profile.h"

namespace mpap {

// A CUDA check after a scratch block `blk` was taken on stream `st`: on failure
// the block goes back before the error is returned.
#define MPAP_CK_FREE(call)                                   \
  do {                                                       \
    if (!::mpap::cuda_ok((call), #call)) {                   \
      scratch_free(blk, st);                                 \
      return MPAP_ERR_CUDA;                                  \
    }                                                        \
  } while (0)

struct McJob {
  Geom g;
  const float* x;          // roadmap node states [6][V]
  uint32_t V;
  const uint32_t* path;    // device copy of the plan
  uint32_t path_len;
  int4* ckpt;              // [steps] {x, y, z (2^-20 units), level}
  uint32_t steps;
  uint32_t rollouts;
  uint32_t call_id;
  int K;                   // table size - 1 (levels are clamped to [0, K])
  uint32_t key0, key1;
  long long delta2;
  const int32_t* sigma;    // [K+1]
  const int32_t* shift;    // [K+1]
  uint32_t* hits;          // [3] loc, coll, any
};

__global__ void k_mc_checkpoints(const McJob* jobs) {
  const McJob& J = jobs[blockIdx.y];
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < J.steps; t += gridDim.x * blockDim.x) {
    const uint32_t j = t / (uint32_t)J.g.M;
    const int m = (int)(t % (uint32_t)J.g.M) + 1;
    const uint32_t a = J.path[j], b = J.path[j + 1];
    float xa[6], xb[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      xa[c] = J.x[(size_t)c * J.V + a];
      xb[c] = J.x[(size_t)c * J.V + b];
    }
    Conn cn;
    conn_setup(J.g, xa, xb, cn);
    conn_yaw(J.g, cn, a, b);
    float p[3];
    conn_point(J.g, cn, m, p);
    const float yaw_c[2] = {cn.psi0, cn.dpsi};
    int lev = J.g.dp == 2 ? level_ck_t<2>(J.g, yaw_c, m, p) : level_ck_t<3>(J.g, yaw_c, m, p);
    lev = lev > J.K ? J.K : lev;
    J.ckpt[t] = make_int4((int)__float2ll_rn(__fmul_rn(p[0], kTwo20)), (int)__float2ll_rn(__fmul_rn(p[1], kTwo20)),
                          (int)__float2ll_rn(__fmul_rn(p[2], kTwo20)), lev);
  }
}

constexpr int kMcMaxBoxes = 512;

// Point-in-box prefilter of the rollouts (scenes of at most 32 boxes): the unit
// interval in 2^-20 units is cut into 64 bins of 2^14; per axis a and bin i,
// bins[(2a) 64 + i] holds the boxes whose low face is at most the bin's largest
// coordinate and bins[(2a + 1) 64 + i] those whose high face is at least its
// smallest, so a box holding a point of bin i is in both: their AND over the
// axes is a superset of the boxes holding the point, checked exactly after.
constexpr int kMcBins = 64;
constexpr int kMcBinShift = 14;

__global__ void __launch_bounds__(256) k_mc_rollouts(const McJob* jobs) {
  const McJob& J = jobs[blockIdx.y];
  __shared__ int s_lo[3 * kMcMaxBoxes], s_hi[3 * kMcMaxBoxes];
  __shared__ uint32_t s_bins[6 * kMcBins];
  const int nb = J.g.nb < kMcMaxBoxes ? J.g.nb : kMcMaxBoxes;
  for (int i = threadIdx.x; i < 3 * nb; i += blockDim.x) {
    s_lo[i] = (int)__float2ll_rn(__fmul_rn(J.g.box_lo[i], kTwo20));
    s_hi[i] = (int)__float2ll_rn(__fmul_rn(J.g.box_hi[i], kTwo20));
  }
  __syncthreads();
  const bool binned = nb <= 32;
  if (binned) {
    for (int t = threadIdx.x; t < 6 * kMcBins; t += blockDim.x) {
      const int a = t / (2 * kMcBins), side = (t / kMcBins) & 1, i = t % kMcBins;
      const int bmin = i << kMcBinShift;
      const int bmax = (i == kMcBins - 1) ? (1 << 20) : ((i + 1) << kMcBinShift) - 1;
      uint32_t m = 0;
      for (int b = 0; b < nb; ++b) {
        const bool in = (side == 0) ? (s_lo[3 * b + a] <= bmax) : (s_hi[3 * b + a] >= bmin);
        m |= in ? (1u << b) : 0u;
      }
      s_bins[t] = m;
    }
    __syncthreads();
  }
  const int dp = J.g.dp;
  const uint32_t ro = blockIdx.x * blockDim.x + threadIdx.x;
  bool loc = false, coll = false;
  if (ro < J.rollouts) {
    long long e[3] = {0, 0, 0};
    const long long lim = 1ll << 30, one = 1ll << 20;
    const int calls = (12 * dp + 7) / 8;   // Philox calls needed for dp axes of noise
    for (uint32_t s = 0; s < J.steps && !(loc && coll); ++s) {
      const int4 ck = J.ckpt[s];
      const int k = ck.w;
      const int sh = __ldg(J.shift + k);
      if (sh > 0) {
#pragma unroll
        for (int i = 0; i < 3; ++i)
          if (i < dp) e[i] -= (e[i] >> sh);
      }
      uint32_t wd[20];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        if (c < calls) {
          uint32_t w0 = ro, w1 = s, w2 = (uint32_t)c, w3 = J.call_id;
          philox4x32_10(w0, w1, w2, w3, J.key0, J.key1);
          wd[4 * c + 0] = w0;
          wd[4 * c + 1] = w1;
          wd[4 * c + 2] = w2;
          wd[4 * c + 3] = w3;
        }
      }
      const long long sig = (long long)__ldg(J.sigma + k);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        if (i < dp) {
          long long xi = 0;
#pragma unroll
          for (int jj = 0; jj < 6; ++jj) {   // 12 draws = 6 words, low then high half
            const uint32_t w = wd[6 * i + jj];
            xi += (long long)(w & 0xFFFFu) + (long long)(w >> 16);
          }
          xi -= 6ll * 65536ll;
          long long v = e[i] + ((sig * xi) >> 16);
          v = v > lim ? lim : v;
          v = v < -lim ? -lim : v;
          e[i] = v;
        }
      }
      long long ee = 0;
#pragma unroll
      for (int i = 0; i < 3; ++i)
        if (i < dp) ee += e[i] * e[i];
      if (ee >= J.delta2) loc = true;
      const long long qx = (long long)ck.x + e[0], qy = (long long)ck.y + e[1], qz = (long long)ck.z + e[2];
      bool bad = qx < 0 || qx > one || qy < 0 || qy > one || (dp == 3 && (qz < 0 || qz > one));
      if (!bad && binned) {
        // inside the unit box: every coordinate lies in [0, 2^20]
        const int bx = min((int)(qx >> kMcBinShift), kMcBins - 1);
        const int by = min((int)(qy >> kMcBinShift), kMcBins - 1);
        uint32_t cand = s_bins[bx] & s_bins[kMcBins + bx] & s_bins[2 * kMcBins + by] & s_bins[3 * kMcBins + by];
        if (dp == 3) {
          const int bz = min((int)(qz >> kMcBinShift), kMcBins - 1);
          cand &= s_bins[4 * kMcBins + bz] & s_bins[5 * kMcBins + bz];
        }
        for (uint32_t mm = cand; mm && !bad; mm &= mm - 1) {
          const int b = __ffs(mm) - 1;
          bool in = qx >= s_lo[3 * b] && qx <= s_hi[3 * b] && qy >= s_lo[3 * b + 1] && qy <= s_hi[3 * b + 1];
          if (dp == 3) in = in && qz >= s_lo[3 * b + 2] && qz <= s_hi[3 * b + 2];
          bad = in;
        }
      }
      for (int b = 0; b < nb && !bad && !binned; ++b) {
        bool in = qx >= s_lo[3 * b] && qx <= s_hi[3 * b] && qy >= s_lo[3 * b + 1] && qy <= s_hi[3 * b + 1];
        if (dp == 3) in = in && qz >= s_lo[3 * b + 2] && qz <= s_hi[3 * b + 2];
        bad = in;
      }
      if (bad) coll = true;
    }
  }
  const unsigned nl = __reduce_add_sync(0xFFFFFFFFu, loc ? 1u : 0u);
  const unsigned nc = __reduce_add_sync(0xFFFFFFFFu, coll ? 1u : 0u);
  const unsigned na = __reduce_add_sync(0xFFFFFFFFu, (loc || coll) ? 1u : 0u);
  if ((threadIdx.x & 31) == 0) {
    if (nl) atomicAdd(J.hits + 0, nl);
    if (nc) atomicAdd(J.hits + 1, nc);
    if (na) atomicAdd(J.hits + 2, na);
  }
}

int32_t certify_batch_impl(mpap_roadmap* const* rms, const uint32_t* const* paths, const uint32_t* path_lens,
                           const mpap_mc_params* mcs, uint32_t n, mpap_cert* outs, cudaStream_t st) {
  if (n == 0) return MPAP_OK;
  std::vector<McJob> jobs(n);
  size_t total_steps = 0, total_path = 0, total_tab = 0;
  uint32_t max_ro = 0;
  for (uint32_t i = 0; i < n; ++i) {
    const mpap_roadmap* rm = rms[i];
    if (!rm || !rm->has_geometry) {
      set_error("certify: roadmap %u has no geometry", i);
      return MPAP_ERR_INVALID_ARG;
    }
    if (rm->nb > kMcMaxBoxes) {
      set_error("certify: at most %d boxes", kMcMaxBoxes);
      return MPAP_ERR_INVALID_ARG;
    }
    if (!mcs[i].sigma_fx || !mcs[i].shift || (path_lens[i] && !paths[i])) {
      set_error("certify: null table or path");
      return MPAP_ERR_INVALID_ARG;
    }
    for (uint32_t j = 0; j < path_lens[i]; ++j)
      if (paths[i][j] >= rm->V) {
        set_error("certify: path node %u out of range", paths[i][j]);
        return MPAP_ERR_INVALID_ARG;
      }
    for (int k = 0; k <= rm->K; ++k)
      if (mcs[i].shift[k] < 0 || mcs[i].shift[k] > 62) {
        set_error("certify: shift table entries must be in [0, 62]");
        return MPAP_ERR_INVALID_ARG;
      }
    const uint32_t steps = path_lens[i] >= 2 ? (path_lens[i] - 1) * (uint32_t)rm->M : 0u;
    McJob& J = jobs[i];
    J.g = rm->geom;
    J.x = rm->x;
    J.V = rm->V;
    J.path_len = path_lens[i];
    J.steps = steps;
    J.rollouts = mcs[i].rollouts;
    J.call_id = mcs[i].call_id;
    J.K = rm->K;
    J.key0 = (uint32_t)mcs[i].seed;
    J.key1 = (uint32_t)(mcs[i].seed >> 32);
    J.delta2 = (long long)mcs[i].delta_fx * (long long)mcs[i].delta_fx;
    total_steps += steps;
    total_path += path_lens[i];
    total_tab += 2 * (size_t)(rm->K + 1);
    max_ro = max_ro > mcs[i].rollouts ? max_ro : mcs[i].rollouts;
  }
  // one device scratch block: jobs | hits | paths | tables | checkpoints
  const size_t b_jobs = sizeof(McJob) * n;
  const size_t b_hits = sizeof(uint32_t) * 3 * n;
  const size_t b_path = sizeof(uint32_t) * (total_path + 1);
  const size_t b_tab = sizeof(int32_t) * (total_tab + 1);
  const size_t b_ck = sizeof(int4) * (total_steps + 1);
  auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t bytes = up(b_jobs) + up(b_hits) + up(b_path) + up(b_tab) + up(b_ck);
  char* blk = nullptr;
  MPAP_CK(scratch_alloc((void**)&blk, bytes, st));
  const size_t o_hits = up(b_jobs), o_path = o_hits + up(b_hits), o_tab = o_path + up(b_path);
  const size_t o_ck = o_tab + up(b_tab);
  McJob* d_jobs = (McJob*)blk;
  uint32_t* d_hits = (uint32_t*)(blk + o_hits);
  uint32_t* d_path = (uint32_t*)(blk + o_path);
  int32_t* d_tab = (int32_t*)(blk + o_tab);
  int4* d_ck = (int4*)(blk + o_ck);
  // host image of jobs | zeroed hit counters | paths | tables: one upload
  std::vector<char> himg(o_ck, 0);
  uint32_t* hpath = (uint32_t*)(himg.data() + o_path);
  int32_t* htab = (int32_t*)(himg.data() + o_tab);
  size_t po = 0, to = 0, co = 0;
  for (uint32_t i = 0; i < n; ++i) {
    const int K1 = rms[i]->K + 1;
    for (uint32_t j = 0; j < path_lens[i]; ++j) hpath[po + j] = paths[i][j];
    for (int k = 0; k < K1; ++k) {
      htab[to + k] = mcs[i].sigma_fx[k];
      htab[to + K1 + k] = mcs[i].shift[k];
    }
    jobs[i].path = d_path + po;
    jobs[i].sigma = d_tab + to;
    jobs[i].shift = d_tab + to + K1;
    jobs[i].ckpt = d_ck + co;
    jobs[i].hits = d_hits + 3 * i;
    po += path_lens[i];
    to += 2 * (size_t)K1;
    co += jobs[i].steps;
  }
  std::memcpy(himg.data(), jobs.data(), b_jobs);
  MPAP_CK_FREE(cudaMemcpyAsync(blk, himg.data(), o_ck, cudaMemcpyHostToDevice, st));
  uint32_t max_steps = 0;
  for (auto& J : jobs) max_steps = max_steps > J.steps ? max_steps : J.steps;
  if (max_steps) {
    dim3 gck((max_steps + 255) / 256, n);
    {
      ::mpap::LaunchScope ls_(st, "k_mc_checkpoints");
      k_mc_checkpoints<<<gck, 256, 0, st>>>(d_jobs);
    }
  }
  if (max_ro && max_steps) {
    dim3 gro((max_ro + 255) / 256, n);
    {
      ::mpap::LaunchScope ls_(st, "k_mc_rollouts");
      k_mc_rollouts<<<gro, 256, 0, st>>>(d_jobs);
    }
  }
  MPAP_CK_FREE(cudaGetLastError());
  std::vector<uint32_t> hh(3 * n);
  MPAP_CK_FREE(cudaMemcpyAsync(hh.data(), d_hits, b_hits, cudaMemcpyDeviceToHost, st));
  scratch_free(blk, st);
  MPAP_CK(cudaStreamSynchronize(st));
  for (uint32_t i = 0; i < n; ++i) {
    outs[i].hits_loc = hh[3 * i];
    outs[i].hits_coll = hh[3 * i + 1];
    outs[i].hits_any = hh[3 * i + 2];
    outs[i].rollouts = mcs[i].rollouts;
  }
  return MPAP_OK;
}

// ---------------------------------------------------------------------------
// Closed-loop VIO model (Sec. 4.1: LQR tracking of the nominal from the state
// estimate, inertial prediction, Kalman position fixes; the recurrences are
// stated with mpap_certify_vio_batch).  Three kernels per batch: the
// checkpoints (k_mc_checkpoints, shared with the error walk), the Kalman gains
// of every step (k_vio_gains: one thread per plan walks the covariance recursion
// in double, rounded to Q16 as the rollouts use them) and the rollouts
// (k_vio_rollouts: one thread per rollout, the three axes' integer states).
// ---------------------------------------------------------------------------
struct VioJob {
  McJob mc;                // checkpoints, rollouts, keys, delta, hit counters (sigma/shift unused)
  int32_t q_a, kp, kv;
  const int32_t* r;        // [K+1] position-fix noise per level
  int2* gains;             // [steps] {Lp, Lw} in Q16
};

__global__ void k_vio_gains(const VioJob* jobs, uint32_t n) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const VioJob& J = jobs[j];
  double p00 = 0.0, p01 = 0.0, p11 = 0.0;
  const double q2 = (double)J.q_a * (double)J.q_a;
  for (uint32_t s = 0; s < J.mc.steps; ++s) {
    const double a00 = p00 + 2.0 * p01 + p11 + 0.25 * q2;
    const double a01 = p01 + p11 + 0.5 * q2;
    const double a11 = p11 + q2;
    const int32_t r = J.r[J.mc.ckpt[s].w];
    double lp = 0.0, lw = 0.0;
    if (r > 0) {
      const double S = a00 + (double)r * (double)r;
      lp = a00 / S;
      lw = a01 / S;
      p00 = (1.0 - lp) * a00;
      p01 = (1.0 - lp) * a01;
      p11 = a11 - lw * a01;
    } else {
      p00 = a00;
      p01 = a01;
      p11 = a11;
    }
    J.gains[s] = make_int2((int)__double2ll_rn(lp * 65536.0), (int)__double2ll_rn(lw * 65536.0));
  }
}

__device__ __forceinline__ long long vio_clamp(long long x) {
  const long long lim = 1ll << 30;
  return x > lim ? lim : (x < -lim ? -lim : x);
}

__device__ __forceinline__ long long vio_round16(long long x) { return (x + 32768ll) >> 16; }

// Irwin-Hall normal from six Philox words (both 16-bit halves of each).
__device__ __forceinline__ long long vio_normal(const uint32_t* w) {
  long long xi = 0;
#pragma unroll
  for (int j = 0; j < 6; ++j) xi += (long long)(w[j] & 0xFFFFu) + (long long)(w[j] >> 16);
  return xi - 6ll * 65536ll;
}

__global__ void __launch_bounds__(256) k_vio_rollouts(const VioJob* jobs) {
  const VioJob& V = jobs[blockIdx.y];
  const McJob& J = V.mc;
  __shared__ int s_lo[3 * kMcMaxBoxes], s_hi[3 * kMcMaxBoxes];
  const int nb = J.g.nb < kMcMaxBoxes ? J.g.nb : kMcMaxBoxes;
  for (int i = threadIdx.x; i < 3 * nb; i += blockDim.x) {
    s_lo[i] = (int)__float2ll_rn(__fmul_rn(J.g.box_lo[i], kTwo20));
    s_hi[i] = (int)__float2ll_rn(__fmul_rn(J.g.box_hi[i], kTwo20));
  }
  __syncthreads();
  const int dp = J.g.dp;
  const uint32_t ro = blockIdx.x * blockDim.x + threadIdx.x;
  bool loc = false, coll = false;
  if (ro < J.rollouts) {
    long long p[3] = {0, 0, 0}, w[3] = {0, 0, 0}, ep[3] = {0, 0, 0}, ew[3] = {0, 0, 0};
    const long long one = 1ll << 20;
    const long long kp = V.kp, kv = V.kv, qa = V.q_a;
    for (uint32_t s = 0; s < J.steps; ++s) {
      const int4 ck = J.ckpt[s];
      const long long r = (long long)__ldg(V.r + ck.w);
      const int2 L = V.gains[s];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        if (i < dp) {
          uint32_t wd[12];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            uint32_t w0 = ro, w1 = s, w2 = (uint32_t)(3 * i + c), w3 = J.call_id;
            philox4x32_10(w0, w1, w2, w3, J.key0, J.key1);
            wd[4 * c + 0] = w0;
            wd[4 * c + 1] = w1;
            wd[4 * c + 2] = w2;
            wd[4 * c + 3] = w3;
          }
          const long long a = -vio_round16(kp * (p[i] + ep[i]) + kv * (w[i] + ew[i]));
          p[i] = vio_clamp(p[i] + w[i] + (a >> 1));
          w[i] = vio_clamp(w[i] + a);
          const long long na = (qa * vio_normal(wd)) >> 16;
          ep[i] = vio_clamp(ep[i] + ew[i] + (na >> 1));
          ew[i] = vio_clamp(ew[i] + na);
          if (r > 0) {
            const long long nu = (r * vio_normal(wd + 6)) >> 16;
            const long long t = nu - ep[i];
            ep[i] = vio_clamp(ep[i] + vio_round16((long long)L.x * t));
            ew[i] = vio_clamp(ew[i] + vio_round16((long long)L.y * t));
          }
        }
      }
      long long ee = 0;
#pragma unroll
      for (int i = 0; i < 3; ++i)
        if (i < dp) ee += ep[i] * ep[i];
      if (ee >= J.delta2) loc = true;
      const long long qx = (long long)ck.x + p[0], qy = (long long)ck.y + p[1], qz = (long long)ck.z + p[2];
      bool bad = qx < 0 || qx > one || qy < 0 || qy > one || (dp == 3 && (qz < 0 || qz > one));
      for (int b = 0; b < nb && !bad; ++b) {
        bool in = qx >= s_lo[3 * b] && qx <= s_hi[3 * b] && qy >= s_lo[3 * b + 1] && qy <= s_hi[3 * b + 1];
        if (dp == 3) in = in && qz >= s_lo[3 * b + 2] && qz <= s_hi[3 * b + 2];
        bad = in;
      }
      if (bad) coll = true;
    }
  }
  const unsigned nl = __reduce_add_sync(0xFFFFFFFFu, loc ? 1u : 0u);
  const unsigned nc = __reduce_add_sync(0xFFFFFFFFu, coll ? 1u : 0u);
  const unsigned na = __reduce_add_sync(0xFFFFFFFFu, (loc || coll) ? 1u : 0u);
  if ((threadIdx.x & 31) == 0) {
    if (nl) atomicAdd(J.hits + 0, nl);
    if (nc) atomicAdd(J.hits + 1, nc);
    if (na) atomicAdd(J.hits + 2, na);
  }
}

int32_t certify_vio_batch_impl(mpap_roadmap* const* rms, const uint32_t* const* paths, const uint32_t* path_lens,
                               const mpap_mc_params* mcs, const mpap_vio_params* vps, uint32_t n, mpap_cert* outs,
                               cudaStream_t st) {
  if (n == 0) return MPAP_OK;
  std::vector<VioJob> jobs(n);
  size_t total_steps = 0, total_path = 0, total_tab = 0;
  uint32_t max_ro = 0, max_steps = 0;
  for (uint32_t i = 0; i < n; ++i) {
    const mpap_roadmap* rm = rms[i];
    if (!rm || !rm->has_geometry) {
      set_error("certify_vio: roadmap %u has no geometry", i);
      return MPAP_ERR_INVALID_ARG;
    }
    if (rm->nb > kMcMaxBoxes) {
      set_error("certify_vio: at most %d boxes", kMcMaxBoxes);
      return MPAP_ERR_INVALID_ARG;
    }
    if (!vps[i].r_fx || (path_lens[i] && !paths[i])) {
      set_error("certify_vio: null table or path");
      return MPAP_ERR_INVALID_ARG;
    }
    for (uint32_t j = 0; j < path_lens[i]; ++j)
      if (paths[i][j] >= rm->V) {
        set_error("certify_vio: path node %u out of range", paths[i][j]);
        return MPAP_ERR_INVALID_ARG;
      }
    const uint32_t steps = path_lens[i] >= 2 ? (path_lens[i] - 1) * (uint32_t)rm->M : 0u;
    VioJob& V = jobs[i];
    std::memset(&V, 0, sizeof(V));
    McJob& J = V.mc;
    J.g = rm->geom;
    J.x = rm->x;
    J.V = rm->V;
    J.path_len = path_lens[i];
    J.steps = steps;
    J.rollouts = mcs[i].rollouts;
    J.call_id = mcs[i].call_id;
    J.K = rm->K;
    J.key0 = (uint32_t)mcs[i].seed;
    J.key1 = (uint32_t)(mcs[i].seed >> 32);
    J.delta2 = (long long)mcs[i].delta_fx * (long long)mcs[i].delta_fx;
    V.q_a = vps[i].q_a;
    V.kp = vps[i].kp_q16;
    V.kv = vps[i].kv_q16;
    total_steps += steps;
    total_path += path_lens[i];
    total_tab += (size_t)(rm->K + 1);
    max_ro = std::max(max_ro, mcs[i].rollouts);
    max_steps = std::max(max_steps, steps);
  }
  // one device scratch block: jobs | hits | paths | r tables | checkpoints | gains
  const size_t b_jobs = sizeof(VioJob) * n;
  const size_t b_hits = sizeof(uint32_t) * 3 * n;
  const size_t b_path = sizeof(uint32_t) * (total_path + 1);
  const size_t b_tab = sizeof(int32_t) * (total_tab + 1);
  const size_t b_ck = sizeof(int4) * (total_steps + 1);
  const size_t b_gain = sizeof(int2) * (total_steps + 1);
  auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t o_hits = up(b_jobs), o_path = o_hits + up(b_hits), o_tab = o_path + up(b_path);
  const size_t o_ck = o_tab + up(b_tab), o_gain = o_ck + up(b_ck);
  const size_t bytes = o_gain + up(b_gain);
  char* blk = nullptr;
  MPAP_CK(scratch_alloc((void**)&blk, bytes, st));
  VioJob* d_jobs = (VioJob*)blk;
  uint32_t* d_hits = (uint32_t*)(blk + o_hits);
  uint32_t* d_path = (uint32_t*)(blk + o_path);
  int32_t* d_tab = (int32_t*)(blk + o_tab);
  int4* d_ck = (int4*)(blk + o_ck);
  int2* d_gain = (int2*)(blk + o_gain);
  // host image of jobs | zeroed hit counters | paths | tables: one upload
  std::vector<char> himg(o_ck, 0);
  uint32_t* hpath = (uint32_t*)(himg.data() + o_path);
  int32_t* htab = (int32_t*)(himg.data() + o_tab);
  size_t po = 0, to = 0, co = 0;
  for (uint32_t i = 0; i < n; ++i) {
    const int K1 = rms[i]->K + 1;
    for (uint32_t j = 0; j < path_lens[i]; ++j) hpath[po + j] = paths[i][j];
    for (int k = 0; k < K1; ++k) htab[to + k] = vps[i].r_fx[k];
    McJob& J = jobs[i].mc;
    J.path = d_path + po;
    J.ckpt = d_ck + co;
    J.hits = d_hits + 3 * i;
    jobs[i].r = d_tab + to;
    jobs[i].gains = d_gain + co;
    po += path_lens[i];
    to += (size_t)K1;
    co += J.steps;
  }
  std::memcpy(himg.data(), jobs.data(), b_jobs);
  MPAP_CK_FREE(cudaMemcpyAsync(blk, himg.data(), o_ck, cudaMemcpyHostToDevice, st));
  // k_mc_checkpoints takes an array of McJob: a compact copy of the jobs'
  // checkpoint parts
  if (max_steps) {
    std::vector<McJob> mj(n);
    for (uint32_t i = 0; i < n; ++i) mj[i] = jobs[i].mc;
    McJob* d_mj = nullptr;
    if (scratch_alloc((void**)&d_mj, sizeof(McJob) * n, st) != cudaSuccess) {
      scratch_free(blk, st);
      set_error("certify_vio: scratch allocation failed");
      return MPAP_ERR_CUDA;
    }
    if (!cuda_ok(cudaMemcpyAsync(d_mj, mj.data(), sizeof(McJob) * n, cudaMemcpyHostToDevice, st), "copy")) {
      scratch_free(d_mj, st);
      scratch_free(blk, st);
      return MPAP_ERR_CUDA;
    }
    {
      ::mpap::LaunchScope ls_(st, "k_mc_checkpoints");
      k_mc_checkpoints<<<dim3((max_steps + 255) / 256, n), 256, 0, st>>>(d_mj);
    }
    scratch_free(d_mj, st);
    {
      ::mpap::LaunchScope ls_(st, "k_vio_gains");
      k_vio_gains<<<(n + 127) / 128, 128, 0, st>>>(d_jobs, n);
    }
    if (max_ro) {
      ::mpap::LaunchScope ls_(st, "k_vio_rollouts");
      k_vio_rollouts<<<dim3((max_ro + 255) / 256, n), 256, 0, st>>>(d_jobs);
    }
  }
  MPAP_CK_FREE(cudaGetLastError());
  std::vector<uint32_t> hh(3 * n);
  MPAP_CK_FREE(cudaMemcpyAsync(hh.data(), d_hits, b_hits, cudaMemcpyDeviceToHost, st));
  scratch_free(blk, st);
  MPAP_CK(cudaStreamSynchronize(st));
  for (uint32_t i = 0; i < n; ++i) {
    outs[i].hits_loc = hh[3 * i];
    outs[i].hits_coll = hh[3 * i + 1];
    outs[i].hits_any = hh[3 * i + 2];
    outs[i].rollouts = mcs[i].rollouts;
  }
  return MPAP_OK;
}

// ---------------------------------------------------------------------------
// Certification without any device allocation.
//
// Some callers cannot allocate device memory once they are running: a planner
// inside a robot's real-time control loop, where an allocation may block or
// fragment a fixed memory budget, or a host program whose device memory is all
// reserved by another framework's caching allocator.  For them the scratch that
// the certification kernels need (the job descriptor, a copy of the plan, the
// noise tables, the hit counters and the per-checkpoint nominal states) lives in
// one file-scope device array of fixed size instead of a stream-ordered
// allocation.  The array is part of the library image: every GPU that loads the
// library holds it (kNoAllocBytes) until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr uint32_t kNoAllocMaxPath = 4096;     // plan nodes
constexpr uint32_t kNoAllocMaxSteps = 65536;   // checkpoints, (path_len - 1) * M
constexpr uint32_t kNoAllocMaxLevels = 256;    // quality levels K + 1
constexpr size_t kNoAllocJob = 0;
constexpr size_t kNoAllocHits = 1024;
constexpr size_t kNoAllocPath = 2048;
constexpr size_t kNoAllocTables = kNoAllocPath + 4 * (size_t)kNoAllocMaxPath;
constexpr size_t kNoAllocCkpt = kNoAllocTables + 2 * 4 * (size_t)kNoAllocMaxLevels;
constexpr size_t kNoAllocBytes = kNoAllocCkpt + sizeof(int4) * (size_t)kNoAllocMaxSteps;
static_assert(sizeof(McJob) <= kNoAllocHits, "job descriptor does not fit its slot");

}  // namespace

static __device__ __align__(256) unsigned char g_certify_scratch[kNoAllocBytes];

namespace {

// Device address of g_certify_scratch on the current device.
int32_t noalloc_scratch(char** out) {
  // Looked up on every call (a host-side table lookup): after a device reset,
  // or a primary-context reset by another framework, the library's module is
  // loaded again and the array may sit at another address.
  void* p = nullptr;
  MPAP_CK(cudaGetSymbolAddress(&p, g_certify_scratch));
  *out = static_cast<char*>(p);
  return MPAP_OK;
}

}  // namespace

int32_t certify_noalloc_impl(const mpap_roadmap* rm, const uint32_t* path, uint32_t path_len,
                             const mpap_mc_params* mc, mpap_cert* out, cudaStream_t st) {
  if (!rm->has_geometry) {
    set_error("certify_noalloc: the roadmap has no geometry");
    return MPAP_ERR_INVALID_ARG;
  }
  if (rm->nb > kMcMaxBoxes) {
    set_error("certify_noalloc: at most %d boxes", kMcMaxBoxes);
    return MPAP_ERR_INVALID_ARG;
  }
  if (path_len > kNoAllocMaxPath) {
    set_error("certify_noalloc: plan of %u nodes exceeds the fixed maximum of %u", path_len, kNoAllocMaxPath);
    return MPAP_ERR_INVALID_ARG;
  }
  const uint64_t steps64 = path_len >= 2 ? (uint64_t)(path_len - 1) * (uint64_t)rm->M : 0ull;
  if (steps64 > kNoAllocMaxSteps) {
    set_error("certify_noalloc: %llu checkpoints exceed the fixed maximum of %u", (unsigned long long)steps64,
              kNoAllocMaxSteps);
    return MPAP_ERR_INVALID_ARG;
  }
  if ((uint32_t)rm->K + 1u > kNoAllocMaxLevels) {
    set_error("certify_noalloc: at most %u quality levels", kNoAllocMaxLevels);
    return MPAP_ERR_INVALID_ARG;
  }
  for (uint32_t j = 0; j < path_len; ++j)
    if (path[j] >= rm->V) {
      set_error("certify_noalloc: path node %u out of range", path[j]);
      return MPAP_ERR_INVALID_ARG;
    }
  for (int k = 0; k <= rm->K; ++k)
    if (mc->shift[k] < 0 || mc->shift[k] > 62) {
      set_error("certify_noalloc: shift table entries must be in [0, 62]");
      return MPAP_ERR_INVALID_ARG;
    }
  char* base = nullptr;
  int32_t rc = noalloc_scratch(&base);
  if (rc) return rc;
  const int K1 = rm->K + 1;
  McJob J;
  std::memset(&J, 0, sizeof(J));
  J.g = rm->geom;
  J.x = rm->x;
  J.V = rm->V;
  J.path = reinterpret_cast<const uint32_t*>(base + kNoAllocPath);
  J.path_len = path_len;
  J.ckpt = reinterpret_cast<int4*>(base + kNoAllocCkpt);
  J.steps = (uint32_t)steps64;
  J.rollouts = mc->rollouts;
  J.call_id = mc->call_id;
  J.K = rm->K;
  J.key0 = (uint32_t)mc->seed;
  J.key1 = (uint32_t)(mc->seed >> 32);
  J.delta2 = (long long)mc->delta_fx * (long long)mc->delta_fx;
  J.sigma = reinterpret_cast<const int32_t*>(base + kNoAllocTables);
  J.shift = reinterpret_cast<const int32_t*>(base + kNoAllocTables) + K1;
  J.hits = reinterpret_cast<uint32_t*>(base + kNoAllocHits);
  MPAP_CK(cudaMemcpyAsync(base + kNoAllocJob, &J, sizeof(J), cudaMemcpyHostToDevice, st));
  if (path_len)
    MPAP_CK(cudaMemcpyAsync(base + kNoAllocPath, path, 4 * (size_t)path_len, cudaMemcpyHostToDevice, st));
  MPAP_CK(cudaMemcpyAsync(base + kNoAllocTables, mc->sigma_fx, 4 * (size_t)K1, cudaMemcpyHostToDevice, st));
  MPAP_CK(cudaMemcpyAsync(base + kNoAllocTables + 4 * (size_t)K1, mc->shift, 4 * (size_t)K1,
                          cudaMemcpyHostToDevice, st));
  // the array keeps the previous call's contents: the counters restart at zero
  MPAP_CK(cudaMemsetAsync(base + kNoAllocHits, 0, 3 * sizeof(uint32_t), st));
  const McJob* d_job = reinterpret_cast<const McJob*>(base + kNoAllocJob);
  if (J.steps) {
    LaunchScope ls(st, "k_mc_checkpoints");
    k_mc_checkpoints<<<dim3((J.steps + 255) / 256, 1), 256, 0, st>>>(d_job);
  }
  if (J.steps && J.rollouts) {
    LaunchScope ls(st, "k_mc_rollouts");
    k_mc_rollouts<<<dim3((J.rollouts + 255) / 256, 1), 256, 0, st>>>(d_job);
  }
  MPAP_CK(cudaGetLastError());
  uint32_t hh[3] = {0, 0, 0};
  MPAP_CK(cudaMemcpyAsync(hh, base + kNoAllocHits, sizeof(hh), cudaMemcpyDeviceToHost, st));
  MPAP_CK(cudaStreamSynchronize(st));
  out->hits_loc = hh[0];
  out->hits_coll = hh[1];
  out->hits_any = hh[2];
  out->rollouts = mc->rollouts;
  return MPAP_OK;
}

// ---------------------------------------------------------------------------
// Trajectory features of candidate plans (input of the certification
// surrogate): one thread per (plan, bin).  A plan's Monte Carlo checkpoints
// s = 0 .. steps-1 (the M sub-steps of each edge, as k_mc_checkpoints) fall into
// 16 bins, s going to floor(16 s / steps); per bin the maximum and the sum of the
// quality levels and the minimum clearance (signed box distance in the max norm,
// and the distance to the walls of the unit map).  Every float operation is one
// IEEE operation, so the features are reproducible bit for bit.
// ---------------------------------------------------------------------------
struct FeatJob {
  Geom g;
  const float* x;
  uint32_t V;
  int K;
  uint32_t p0, n;          // plans p0 .. p0 + n - 1 lie on this roadmap
  const uint32_t* ptr;     // [plans + 1] offsets into path
  const uint32_t* path;
  float* feat;             // [plans][48]
};

__global__ void k_plan_features(const FeatJob* __restrict__ jobs) {
  const FeatJob& J = jobs[blockIdx.y];
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= J.n * 16u) return;
  const uint32_t i = J.p0 + (t >> 4), j = t & 15u;
  const uint32_t p0 = J.ptr[i], len = J.ptr[i + 1] - p0;
  const uint32_t M = (uint32_t)J.g.M;
  const uint32_t steps = len >= 2 ? (len - 1) * M : 0u;
  const uint32_t s_lo = (j * steps + 15u) / 16u, s_hi = ((j + 1) * steps + 15u) / 16u;
  int lmax = 0;
  uint32_t lsum = 0;
  float clr = INFINITY;
  const int dp = J.g.dp;
  uint32_t cur_e = 0xFFFFFFFFu;
  Conn cn;
  for (uint32_t s = s_lo; s < s_hi; ++s) {
    const uint32_t e = s / M;
    if (e != cur_e) {
      cur_e = e;
      const uint32_t a = J.path[p0 + e], b = J.path[p0 + e + 1];
      float xa[6], xb[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        xa[c] = J.x[(size_t)c * J.V + a];
        xb[c] = J.x[(size_t)c * J.V + b];
      }
      conn_setup(J.g, xa, xb, cn);
      conn_yaw(J.g, cn, a, b);
    }
    float p[3];
    conn_point(J.g, cn, (int)(s % M) + 1, p);
    const float yaw_c[2] = {cn.psi0, cn.dpsi};
    int lev = dp == 2 ? level_ck_t<2>(J.g, yaw_c, (int)(s % M) + 1, p) : level_ck_t<3>(J.g, yaw_c, (int)(s % M) + 1, p);
    lev = lev > J.K ? J.K : lev;
    lmax = lev > lmax ? lev : lmax;
    lsum += (uint32_t)lev;
    float c = INFINITY;
    for (int k = 0; k < dp; ++k) c = fminf(c, fminf(p[k], __fsub_rn(1.0f, p[k])));
    for (int b = 0; b < J.g.nb; ++b) {
      float d = -INFINITY;
      for (int k = 0; k < dp; ++k) {
        d = fmaxf(d, fmaxf(__fsub_rn(J.g.box_lo[3 * b + k], p[k]), __fsub_rn(p[k], J.g.box_hi[3 * b + k])));
      }
      c = fminf(c, d);
    }
    clr = fminf(clr, c);
  }
  float* f = J.feat + (size_t)i * 48;
  const float Kf = (float)(J.K > 0 ? J.K : 1);
  if (s_hi > s_lo) {
    f[j] = __fdiv_rn((float)lmax, Kf);
    f[16 + j] = __fdiv_rn((float)lsum, __fmul_rn(64.0f, Kf));
    f[32 + j] = __fmul_rn(4.0f, fminf(0.25f, clr));
  } else {
    f[j] = 0.0f;
    f[16 + j] = 0.0f;
    f[32 + j] = 1.0f;
  }
}

// Features of plans on n_rm roadmaps in one launch: the plans of roadmap r are
// plan_ptr[r] .. plan_ptr[r+1] - 1, plan i is path[path_ptr[i] .. path_ptr[i+1]).
int32_t plan_features_batch_impl(mpap_roadmap* const* rms, uint32_t n_rm, const uint32_t* plan_ptr,
                                 const uint32_t* path_ptr, const uint32_t* path, float* feat, cudaStream_t st) {
  if (!rms || !plan_ptr || (plan_ptr[n_rm] > plan_ptr[0] && (!path_ptr || !path || !feat))) {
    set_error("plan_features: null array");
    return MPAP_ERR_INVALID_ARG;
  }
  const uint32_t P0 = plan_ptr[0], n = plan_ptr[n_rm] - P0;
  if (n == 0) return MPAP_OK;
  uint32_t max_plans = 0;
  for (uint32_t r = 0; r < n_rm; ++r) {
    const mpap_roadmap* rm = rms[r];
    if (plan_ptr[r + 1] < plan_ptr[r]) {
      set_error("plan_features: plan_ptr must not decrease");
      return MPAP_ERR_INVALID_ARG;
    }
    if (plan_ptr[r + 1] == plan_ptr[r]) continue;
    if (!rm || !rm->has_geometry) {
      set_error("plan_features: roadmap %u has no geometry", r);
      return MPAP_ERR_INVALID_ARG;
    }
    max_plans = std::max(max_plans, plan_ptr[r + 1] - plan_ptr[r]);
    for (uint32_t i = plan_ptr[r]; i < plan_ptr[r + 1]; ++i) {
      if (path_ptr[i + 1] < path_ptr[i] + 2) {
        set_error("plan_features: plan %u has fewer than 2 nodes", i);
        return MPAP_ERR_INVALID_ARG;
      }
      for (uint32_t k = path_ptr[i]; k < path_ptr[i + 1]; ++k)
        if (path[k] >= rm->V) {
          set_error("plan_features: node %u out of range on roadmap %u", path[k], r);
          return MPAP_ERR_INVALID_ARG;
        }
    }
  }
  const uint32_t base = path_ptr[P0], total = path_ptr[P0 + n] - base;
  std::vector<uint32_t> ptr(n + 1);
  for (uint32_t i = 0; i <= n; ++i) ptr[i] = path_ptr[P0 + i] - base;
  std::vector<FeatJob> jobs;
  auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t b_jobs = up(sizeof(FeatJob) * n_rm), b_ptr = up(4 * ((size_t)n + 1)), b_path = up(4 * (size_t)total),
               b_feat = 4 * 48 * (size_t)n;
  char* blk = nullptr;
  MPAP_CK(scratch_alloc((void**)&blk, b_jobs + b_ptr + b_path + b_feat, st));
  const uint32_t* d_ptr = (const uint32_t*)(blk + b_jobs);
  const uint32_t* d_path = (const uint32_t*)(blk + b_jobs + b_ptr);
  float* d_feat = (float*)(blk + b_jobs + b_ptr + b_path);
  for (uint32_t r = 0; r < n_rm; ++r) {
    if (plan_ptr[r + 1] == plan_ptr[r]) continue;
    FeatJob J;
    J.g = rms[r]->geom;
    J.x = rms[r]->x;
    J.V = rms[r]->V;
    J.K = rms[r]->K;
    J.p0 = plan_ptr[r] - P0;
    J.n = plan_ptr[r + 1] - plan_ptr[r];
    J.ptr = d_ptr;
    J.path = d_path;
    J.feat = d_feat;
    jobs.push_back(J);
  }
  int32_t rc = MPAP_OK;
  if (!cuda_ok(cudaMemcpyAsync(blk, jobs.data(), sizeof(FeatJob) * jobs.size(), cudaMemcpyHostToDevice, st),
               "features jobs") ||
      !cuda_ok(cudaMemcpyAsync((void*)d_ptr, ptr.data(), 4 * ((size_t)n + 1), cudaMemcpyHostToDevice, st),
               "features ptr") ||
      !cuda_ok(cudaMemcpyAsync((void*)d_path, path + base, 4 * (size_t)total, cudaMemcpyHostToDevice, st),
               "features path"))
    rc = MPAP_ERR_CUDA;
  if (rc == MPAP_OK) {
    LaunchScope ls(st, "k_plan_features");
    const dim3 grid((max_plans * 16 + 255) / 256, (uint32_t)jobs.size());
    k_plan_features<<<grid, 256, 0, st>>>((const FeatJob*)blk);
    if (!cuda_ok(cudaGetLastError(), "k_plan_features")) rc = MPAP_ERR_CUDA;
  }
  if (rc == MPAP_OK && !cuda_ok(cudaMemcpyAsync(feat, d_feat, b_feat, cudaMemcpyDeviceToHost, st), "features out"))
    rc = MPAP_ERR_CUDA;
  scratch_free(blk, st);
  if (!cuda_ok(cudaStreamSynchronize(st), "plan_features")) rc = MPAP_ERR_CUDA;
  return rc;
}

int32_t plan_features_impl(mpap_roadmap* rm, uint32_t n, const uint32_t* path_ptr, const uint32_t* path, float* feat,
                           cudaStream_t st) {
  if (!rm || !rm->has_geometry) {
    set_error("plan_features: roadmap has no geometry");
    return MPAP_ERR_INVALID_ARG;
  }
  const uint32_t plan_ptr[2] = {0, n};
  return plan_features_batch_impl(&rm, 1, plan_ptr, path_ptr, path, feat, st);
}

}  // namespace mpap
