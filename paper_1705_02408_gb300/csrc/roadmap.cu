// Roadmap construction on the GPU: Alg. 1 steps 1-2 and Alg. 2 (BuildGraph) of
// Ichter et al., "Perception-Aware Motion Planning via Multiobjective Search on
// GPUs" -- SampleFree, Near, Collision and the per-edge perception transfer.
//
// Layout in HBM (one roadmap):
//   x        float [6][V]      node states, SoA (p0 p1 p2 v0 v1 v2)
//   fwd_ptr  u32   [V+1]       out-edge CSR, neighbours ascending
//   fwd_edge int4  [E]         {dst, cost_q, S, C}
//   rev_ptr  u32   [V+1]       in-edge CSR, sources ascending
//   rev_edge int4  [E]         {src, cost_q, S, C}
//   is_goal  u8    [V], goal_list u32 [n_goal]
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "internal.h"

namespace mpap {

namespace {
thread_local char g_last_error[512] = "";
}

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
}

const char* last_error() { return g_last_error; }

bool cuda_ok(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return true;
  set_error("%s: %s", what, cudaGetErrorString(e));
  return false;
}

void fill_geom_constants(Geom& g, int dim, int nb, int G, int n_f, int M, float r, float T) {
  g.dim = dim;
  g.dp = (dim == 2) ? 2 : 3;
  g.nb = nb;
  g.G = G;
  g.n_f = n_f;
  g.M = M;
  g.r = r;
  g.T = T;
  const double Td = (double)T;
  g.c1 = (float)(12.0 / (Td * Td * Td));
  g.c2 = (float)(12.0 / (Td * Td));
  g.c3 = (float)(4.0 / Td);
  g.e1 = (float)(6.0 / (Td * Td));
  g.e2 = (float)(2.0 / Td);
  g.inv6 = (float)(1.0 / 6.0);
  g.dtm = (float)(Td / (double)M);
  g.invM = 1.0f / (float)M;
  g.Tq = (int64_t)llrintf(T * 16777216.0f);
}

// ---------------------------------------------------------------------------
// Single-block exclusive scan (used for CSR row pointers and sample compaction).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_exclusive_scan(const uint32_t* __restrict__ in,
                                                         uint32_t* __restrict__ out, uint32_t n,
                                                         uint32_t* overflow) {
  __shared__ uint32_t warp_sums[32];
  __shared__ unsigned long long carry;
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0ull;
  __syncthreads();
  for (uint32_t base = 0; base < n; base += 1024u) {
    const uint32_t i = base + threadIdx.x;
    const uint32_t v = (i < n) ? in[i] : 0u;
    const uint32_t incl = warp_incl_scan(v);
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) warp_sums[lane] = warp_incl_scan(warp_sums[lane]);
    __syncthreads();
    const unsigned long long excl =
        carry + (warp ? warp_sums[warp - 1] : 0u) + (unsigned long long)(incl - v);
    if (i < n) {
      if (excl > 0xFFFFFFFFull) {
        out[i] = 0xFFFFFFFFu;
        if (overflow) *overflow = 1u;
      } else {
        out[i] = (uint32_t)excl;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_sums[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (carry > 0xFFFFFFFFull) {
      out[n] = 0xFFFFFFFFu;
      if (overflow) *overflow = 1u;
    } else {
      out[n] = (uint32_t)carry;
    }
  }
}

void launch_exclusive_scan(const uint32_t* in, uint32_t* out, uint32_t n, uint32_t* overflow,
                           cudaStream_t st) {
  k_exclusive_scan<<<1, 1024, 0, st>>>(in, out, n, overflow);
}

// ---------------------------------------------------------------------------
// SampleFree: candidate `att` is drawn from Philox4x32-10 with counter
// (att, 0, query_id, 0) (position) and (att, 1, query_id, 0) (velocity, 6D),
// key = seed; it is free iff outside every closed box (and |v| <= 1 in 6D).
// ---------------------------------------------------------------------------
__global__ void k_sample_candidates(Geom g, uint32_t key0, uint32_t key1, uint32_t qid,
                                    uint32_t a0, uint32_t count, float* __restrict__ cand,
                                    uint32_t* __restrict__ ok) {
  extern __shared__ float s_box[];
  float* s_lo = s_box;
  float* s_hi = s_box + 3 * g.nb;
  for (int i = threadIdx.x; i < 3 * g.nb; i += blockDim.x) {
    s_lo[i] = g.box_lo[i];
    s_hi[i] = g.box_hi[i];
  }
  __syncthreads();
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x) {
    const uint32_t att = a0 + t;
    uint32_t w0 = att, w1 = 0u, w2 = qid, w3 = 0u;
    philox4x32_10(w0, w1, w2, w3, key0, key1);
    float p[3] = {unit24(w0), unit24(w1), g.dp == 3 ? unit24(w2) : 0.0f};
    bool free = true;
    for (int b = 0; b < g.nb && free; ++b) free = !in_box(s_lo + 3 * b, s_hi + 3 * b, g.dp, p);
    float v[3] = {0.0f, 0.0f, 0.0f};
    if (free && g.dim == 6) {
      uint32_t u0 = att, u1 = 1u, u2 = qid, u3 = 0u;
      philox4x32_10(u0, u1, u2, u3, key0, key1);
      v[0] = __fsub_rn(__fmul_rn(2.0f, unit24(u0)), 1.0f);
      v[1] = __fsub_rn(__fmul_rn(2.0f, unit24(u1)), 1.0f);
      v[2] = __fsub_rn(__fmul_rn(2.0f, unit24(u2)), 1.0f);
      float vv = __fmul_rn(v[0], v[0]);
      vv = __fadd_rn(vv, __fmul_rn(v[1], v[1]));
      vv = __fadd_rn(vv, __fmul_rn(v[2], v[2]));
      free = (vv <= 1.0f);
    }
    cand[0 * count + t] = p[0];
    cand[1 * count + t] = p[1];
    cand[2 * count + t] = p[2];
    cand[3 * count + t] = v[0];
    cand[4 * count + t] = v[1];
    cand[5 * count + t] = v[2];
    ok[t] = free ? 1u : 0u;
  }
}

// Keeps the first `need` free candidates (in attempt order) as nodes 2+kept+...
__global__ void k_take_samples(const float* __restrict__ cand, const uint32_t* __restrict__ ok,
                               const uint32_t* __restrict__ rank, uint32_t count, uint32_t need,
                               uint32_t first, float* __restrict__ x, uint32_t V) {
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x) {
    if (!ok[t] || rank[t] >= need) continue;
    const uint32_t id = first + rank[t];
#pragma unroll
    for (int a = 0; a < 6; ++a) x[(size_t)a * V + id] = cand[(size_t)a * count + t];
  }
}

__global__ void k_set_endpoints(float* x, uint32_t V, float i0, float i1, float i2, float i3,
                                float i4, float i5, float g0, float g1, float g2, float g3,
                                float g4, float g5) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const float xi[6] = {i0, i1, i2, i3, i4, i5};
    const float xg[6] = {g0, g1, g2, g3, g4, g5};
    for (int a = 0; a < 6; ++a) {
      x[(size_t)a * V + 0] = xi[a];
      x[(size_t)a * V + 1] = xg[a];
    }
  }
}

// X_goal: nodes within goal_radius (position) of node 1.
__global__ void k_mark_goal(const float* __restrict__ x, uint32_t V, int dp, float r2,
                            uint8_t* __restrict__ is_goal, uint32_t* goal_list, uint32_t* n_goal) {
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int i = 0; i < dp; ++i) {
      float d = __fsub_rn(x[(size_t)i * V + v], x[(size_t)i * V + 1]);
      s = __fadd_rn(s, __fmul_rn(d, d));
    }
    const bool goal = (s <= r2);
    is_goal[v] = goal ? 1 : 0;
    if (goal) goal_list[atomicAdd(n_goal, 1u)] = v;
  }
}

// ---------------------------------------------------------------------------
// Near + Collision + transfer.  One warp per source node v; the CTA stages
// tiles of candidate neighbours u in shared memory and every lane tests one u
// per round.  The connections that pass (Cost < r, no collision) are counted
// (FILL = false) or written in ascending u order via ballot ranks (FILL = true),
// together with their quantised cost and the max-plus transfer (S, C).
// ---------------------------------------------------------------------------
constexpr int kEdgeWarps = 8;
constexpr int kEdgeTile = 256;

template <bool FILL>
__global__ void __launch_bounds__(kEdgeWarps * 32) k_edges(Geom g, const float* __restrict__ x,
                                                           uint32_t V, uint32_t* counts,
                                                           const uint32_t* __restrict__ row_ptr,
                                                           int4* __restrict__ edges, uint32_t* err) {
  extern __shared__ float smem[];
  float* s_lo = smem;
  float* s_hi = smem + 3 * g.nb;
  float* s_tile = smem + 6 * g.nb;   // [6][kEdgeTile]
  const int nc = (g.dim == 6) ? 6 : g.dp;
  const unsigned lane = lane_id();
  const uint32_t warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < 3 * g.nb; i += blockDim.x) {
    s_lo[i] = g.box_lo[i];
    s_hi[i] = g.box_hi[i];
  }
  const uint32_t v = blockIdx.x * kEdgeWarps + warp;
  const bool have_v = v < V;
  float a[6] = {0, 0, 0, 0, 0, 0};
  if (have_v)
    for (int c = 0; c < nc; ++c) a[c] = x[(size_t)c * V + v];
  uint32_t running = 0;
  const uint32_t out_base = (FILL && have_v) ? row_ptr[v] : 0u;
  for (uint32_t tb = 0; tb < V; tb += kEdgeTile) {
    __syncthreads();
    for (int i = threadIdx.x; i < kEdgeTile * nc; i += blockDim.x) {
      const int c = i / kEdgeTile, k = i % kEdgeTile;
      const uint32_t u = tb + k;
      s_tile[c * kEdgeTile + k] = (u < V) ? x[(size_t)c * V + u] : 0.0f;
    }
    __syncthreads();
    if (!have_v) continue;
    for (int sub = 0; sub < kEdgeTile; sub += 32) {
      const uint32_t u = tb + sub + lane;
      const bool valid = (u < V) && (u != v);
      float b[6] = {0, 0, 0, 0, 0, 0};
      for (int c = 0; c < nc; ++c) b[c] = s_tile[c * kEdgeTile + sub + lane];
      Conn cn;
      conn_setup(g, a, b, cn);
      bool ok = valid && (cn.cost < g.r);
      if (ok) ok = !conn_collides(g, cn, s_lo, s_hi);
      const unsigned bal = __ballot_sync(0xFFFFFFFFu, ok);
      if (FILL && ok) {
        const int64_t cq = quantise_cost(cn.cost);
        int64_t S, C;
        conn_transfer(g, cn, cq, S, C);
        if (cq > INT32_MAX || S > INT32_MAX || S < INT32_MIN || C > INT32_MAX) atomicOr(err, kErrEdge);
        const uint32_t pos = out_base + running + __popc(bal & ((1u << lane) - 1u));
        edges[pos] = make_int4((int)u, (int)cq, (int)S, (int)C);
      }
      running += __popc(bal);
    }
  }
  if (!FILL && have_v && lane == 0) counts[v] = running;
}

// In-degree count and reverse fill (one warp per source), then per-row sort.
__global__ void k_indegree(const uint32_t* __restrict__ fwd_ptr, const int4* __restrict__ fe,
                           uint32_t V, uint32_t* indeg) {
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < V; v += warps)
    for (uint32_t e = fwd_ptr[v] + lane_id(); e < fwd_ptr[v + 1]; e += 32) atomicAdd(&indeg[fe[e].x], 1u);
}

__global__ void k_reverse_fill(const uint32_t* __restrict__ fwd_ptr, const int4* __restrict__ fe,
                               uint32_t V, const uint32_t* __restrict__ rev_ptr, uint32_t* fill,
                               int4* __restrict__ re) {
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < V; v += warps)
    for (uint32_t e = fwd_ptr[v] + lane_id(); e < fwd_ptr[v + 1]; e += 32) {
      const int4 ed = fe[e];
      const uint32_t pos = rev_ptr[ed.x] + atomicAdd(&fill[ed.x], 1u);
      re[pos] = make_int4((int)v, ed.y, ed.z, ed.w);
    }
}

__global__ void k_sort_rows(const uint32_t* __restrict__ ptr, int4* __restrict__ rows, uint32_t V) {
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
    const uint32_t b = ptr[v], e = ptr[v + 1];
    for (uint32_t i = b + 1; i < e; ++i) {
      const int4 key = rows[i];
      uint32_t j = i;
      while (j > b && rows[j - 1].x > key.x) {
        rows[j] = rows[j - 1];
        --j;
      }
      rows[j] = key;
    }
  }
}

namespace {

template <typename T>
int32_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  MPAP_CK(cudaMalloc((void**)p, count * sizeof(T)));
  return MPAP_OK;
}

int32_t copy_in(void* dst, const void* src, size_t bytes, bool device_src, cudaStream_t st) {
  if (bytes == 0) return MPAP_OK;
  MPAP_CK(cudaMemcpyAsync(dst, src, bytes, device_src ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  return MPAP_OK;
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

#define MPAP_TRY(x)                  \
  do {                               \
    int32_t rc_ = (x);               \
    if (rc_ != MPAP_OK) {            \
      roadmap_free_impl(rm);         \
      return rc_;                    \
    }                                \
  } while (0)

// Builds the reverse CSR and the forward/reverse consistency from a filled
// forward CSR (fwd_ptr, fwd_edge).
int32_t finish_reverse(mpap_roadmap* rm, cudaStream_t st) {
  uint32_t* indeg = nullptr;
  MPAP_CK(cudaMallocAsync((void**)&indeg, sizeof(uint32_t) * (rm->V + 1), st));
  MPAP_CK(cudaMemsetAsync(indeg, 0, sizeof(uint32_t) * (rm->V + 1), st));
  const int blocks = 4 * sm_count();
  if (rm->E) k_indegree<<<blocks, 256, 0, st>>>(rm->fwd_ptr, rm->fwd_edge, rm->V, indeg);
  launch_exclusive_scan(indeg, rm->rev_ptr, rm->V, nullptr, st);
  MPAP_CK(cudaMemsetAsync(indeg, 0, sizeof(uint32_t) * (rm->V + 1), st));
  if (rm->E) {
    k_reverse_fill<<<blocks, 256, 0, st>>>(rm->fwd_ptr, rm->fwd_edge, rm->V, rm->rev_ptr, indeg, rm->rev_edge);
    k_sort_rows<<<(rm->V + 255) / 256, 256, 0, st>>>(rm->rev_ptr, rm->rev_edge, rm->V);
  }
  MPAP_CK(cudaFreeAsync(indeg, st));
  MPAP_CK(cudaGetLastError());
  return MPAP_OK;
}

}  // namespace

void roadmap_free_impl(mpap_roadmap* rm) {
  if (!rm) return;
  cudaFree(rm->x);
  cudaFree(rm->is_goal);
  cudaFree(rm->goal_list);
  cudaFree(rm->fwd_ptr);
  cudaFree(rm->fwd_edge);
  cudaFree(rm->rev_ptr);
  cudaFree(rm->rev_edge);
  cudaFree(rm->box_lo);
  cudaFree(rm->box_hi);
  cudaFree(rm->grid);
  delete rm;
}

int32_t build_roadmap_impl(const mpap_scene* sc, const mpap_roadmap_params* prm, const float* host_x,
                           uint32_t V_given, float r, float T, int M, float goal_radius,
                           mpap_roadmap** out, cudaStream_t st) {
  mpap_roadmap* rm = new mpap_roadmap();
  rm->dim = sc->dim_kind;
  rm->nb = sc->nb;
  rm->G = sc->grid_G;
  rm->n_f = sc->n_f;
  rm->K = sc->K;
  rm->M = M;
  rm->r = r;
  rm->T = T;
  rm->goal_radius = goal_radius;
  rm->has_geometry = true;
  rm->V = host_x ? V_given : prm->n + 2u;
  const uint32_t V = rm->V;
  const int dp = (rm->dim == 2) ? 2 : 3;
  size_t cells = (size_t)rm->G * rm->G * (dp == 3 ? rm->G : 1);
  const bool dev = (sc->mem == MPAP_MEM_DEVICE);

  MPAP_TRY(dalloc(&rm->box_lo, 3 * (size_t)rm->nb));
  MPAP_TRY(dalloc(&rm->box_hi, 3 * (size_t)rm->nb));
  MPAP_TRY(dalloc(&rm->grid, cells));
  MPAP_TRY(copy_in(rm->box_lo, sc->box_lo, 12 * (size_t)rm->nb, dev, st));
  MPAP_TRY(copy_in(rm->box_hi, sc->box_hi, 12 * (size_t)rm->nb, dev, st));
  MPAP_TRY(copy_in(rm->grid, sc->grid_level, cells, dev, st));
  fill_geom_constants(rm->geom, rm->dim, rm->nb, rm->G, rm->n_f, M, r, T);
  rm->geom.box_lo = rm->box_lo;
  rm->geom.box_hi = rm->box_hi;
  rm->geom.grid = rm->grid;
  const Geom& g = rm->geom;

  MPAP_TRY(dalloc(&rm->x, 6 * (size_t)V));
  MPAP_TRY(dalloc(&rm->is_goal, V));
  MPAP_TRY(dalloc(&rm->goal_list, V));
  MPAP_TRY(dalloc(&rm->fwd_ptr, (size_t)V + 1));
  MPAP_TRY(dalloc(&rm->rev_ptr, (size_t)V + 1));

  // small device scratch: [0] error bits, [1] n_goal, [2] scan overflow
  uint32_t* scratch = nullptr;
  if (!cuda_ok(cudaMallocAsync((void**)&scratch, 16, st), "cudaMallocAsync")) {
    roadmap_free_impl(rm);
    return MPAP_ERR_CUDA;
  }
  cudaMemsetAsync(scratch, 0, 16, st);
  const int sms = sm_count();
  const size_t box_smem = sizeof(float) * 6 * (size_t)rm->nb;

  if (host_x) {
    MPAP_TRY(copy_in(rm->x, host_x, sizeof(float) * 6 * (size_t)V, false, st));
  } else {
    k_set_endpoints<<<1, 32, 0, st>>>(rm->x, V, prm->x_init[0], prm->x_init[1], prm->x_init[2],
                                       prm->x_init[3], prm->x_init[4], prm->x_init[5], prm->x_goal[0],
                                       prm->x_goal[1], prm->x_goal[2], prm->x_goal[3], prm->x_goal[4],
                                       prm->x_goal[5]);
    // SampleFree in batches until n samples are kept (attempt budget 64 n + 4096).
    const uint64_t max_att = (uint64_t)prm->n * 64ull + 4096ull;
    const uint32_t key0 = (uint32_t)prm->seed, key1 = (uint32_t)(prm->seed >> 32);
    uint32_t kept = 0;
    uint64_t a0 = 0;
    float* cand = nullptr;
    uint32_t *ok = nullptr, *rank = nullptr;
    const uint32_t cap = 1u << 22;
    MPAP_CK(cudaMallocAsync((void**)&cand, sizeof(float) * 6 * cap, st));
    MPAP_CK(cudaMallocAsync((void**)&ok, sizeof(uint32_t) * cap, st));
    MPAP_CK(cudaMallocAsync((void**)&rank, sizeof(uint32_t) * (cap + 1), st));
    while (kept < prm->n) {
      if (a0 >= max_att || a0 > 0xFFFFFFFFull) break;
      uint64_t want = (uint64_t)(prm->n - kept) * 2ull + 8192ull;
      uint64_t count64 = want < cap ? want : cap;
      if (count64 > max_att - a0) count64 = max_att - a0;
      const uint32_t count = (uint32_t)count64;
      const int blocks = (int)((count + 255) / 256 < (uint32_t)(8 * sms) ? (count + 255) / 256 : 8 * sms);
      k_sample_candidates<<<blocks, 256, box_smem, st>>>(g, key0, key1, prm->query_id, (uint32_t)a0,
                                                         count, cand, ok);
      launch_exclusive_scan(ok, rank, count, nullptr, st);
      k_take_samples<<<blocks, 256, 0, st>>>(cand, ok, rank, count, prm->n - kept, 2u + kept, rm->x, V);
      uint32_t total = 0;
      MPAP_CK(cudaMemcpyAsync(&total, rank + count, 4, cudaMemcpyDeviceToHost, st));
      MPAP_CK(cudaStreamSynchronize(st));
      kept += (total < prm->n - kept) ? total : (prm->n - kept);
      a0 += count;
    }
    cudaFreeAsync(cand, st);
    cudaFreeAsync(ok, st);
    cudaFreeAsync(rank, st);
    if (kept < prm->n) {
      cudaFreeAsync(scratch, st);
      set_error("SampleFree: only %u of %u free samples in %llu attempts", kept, prm->n,
                (unsigned long long)max_att);
      roadmap_free_impl(rm);
      return MPAP_ERR_SAMPLING;
    }
  }

  k_mark_goal<<<(V + 255) / 256, 256, 0, st>>>(rm->x, V, dp, goal_radius * goal_radius, rm->is_goal,
                                               rm->goal_list, scratch + 1);

  // Near + Collision: count pass, scan, fill pass.
  uint32_t* counts = nullptr;
  MPAP_CK(cudaMallocAsync((void**)&counts, sizeof(uint32_t) * (V + 1), st));
  const int nc = (rm->dim == 6) ? 6 : dp;
  const size_t esmem = box_smem + sizeof(float) * nc * kEdgeTile;
  const int eblocks = (int)((V + kEdgeWarps - 1) / kEdgeWarps);
  k_edges<false><<<eblocks, kEdgeWarps * 32, esmem, st>>>(g, rm->x, V, counts, nullptr, nullptr, scratch);
  launch_exclusive_scan(counts, rm->fwd_ptr, V, scratch + 2, st);
  uint32_t hs[4] = {0, 0, 0, 0};
  uint32_t E32 = 0;
  MPAP_CK(cudaMemcpyAsync(&E32, rm->fwd_ptr + V, 4, cudaMemcpyDeviceToHost, st));
  MPAP_CK(cudaMemcpyAsync(hs, scratch, 12, cudaMemcpyDeviceToHost, st));
  MPAP_CK(cudaStreamSynchronize(st));
  if (hs[2]) {
    set_error("roadmap: more than 2^32 - 1 edges");
    cudaFreeAsync(counts, st);
    cudaFreeAsync(scratch, st);
    roadmap_free_impl(rm);
    return MPAP_ERR_CAPACITY;
  }
  rm->E = E32;
  rm->n_goal = hs[1];
  MPAP_TRY(dalloc(&rm->fwd_edge, rm->E));
  MPAP_TRY(dalloc(&rm->rev_edge, rm->E));
  k_edges<true><<<eblocks, kEdgeWarps * 32, esmem, st>>>(g, rm->x, V, nullptr, rm->fwd_ptr, rm->fwd_edge,
                                                         scratch);
  MPAP_CK(cudaGetLastError());
  cudaFreeAsync(counts, st);
  MPAP_TRY(finish_reverse(rm, st));
  MPAP_CK(cudaMemcpyAsync(hs, scratch, 4, cudaMemcpyDeviceToHost, st));
  MPAP_CK(cudaStreamSynchronize(st));
  cudaFreeAsync(scratch, st);
  if (hs[0]) {
    set_error("roadmap: an edge cost or transfer does not fit int32");
    roadmap_free_impl(rm);
    return MPAP_ERR_CAPACITY;
  }
  *out = rm;
  return MPAP_OK;
}

int32_t roadmap_from_csr_impl(uint32_t V, const uint32_t* row_ptr, const uint32_t* dst,
                              const int32_t* cost_q, const int32_t* S, const int32_t* C,
                              const uint8_t* is_goal, mpap_roadmap** out, cudaStream_t st) {
  mpap_roadmap* rm = new mpap_roadmap();
  rm->V = V;
  rm->E = row_ptr[V];
  rm->has_geometry = false;
  std::vector<int4> fe(rm->E);
  for (uint64_t e = 0; e < rm->E; ++e) fe[e] = make_int4((int)dst[e], cost_q[e], S[e], C[e]);
  std::vector<uint32_t> goals;
  for (uint32_t v = 0; v < V; ++v)
    if (is_goal[v]) goals.push_back(v);
  rm->n_goal = (uint32_t)goals.size();
  MPAP_TRY(dalloc(&rm->x, 6 * (size_t)V));
  MPAP_TRY(dalloc(&rm->is_goal, V));
  MPAP_TRY(dalloc(&rm->goal_list, V));
  MPAP_TRY(dalloc(&rm->fwd_ptr, (size_t)V + 1));
  MPAP_TRY(dalloc(&rm->rev_ptr, (size_t)V + 1));
  MPAP_TRY(dalloc(&rm->fwd_edge, rm->E));
  MPAP_TRY(dalloc(&rm->rev_edge, rm->E));
  MPAP_CK(cudaMemsetAsync(rm->x, 0, sizeof(float) * 6 * (size_t)V, st));
  MPAP_TRY(copy_in(rm->is_goal, is_goal, V, false, st));
  MPAP_TRY(copy_in(rm->goal_list, goals.data(), 4 * goals.size(), false, st));
  MPAP_TRY(copy_in(rm->fwd_ptr, row_ptr, 4 * ((size_t)V + 1), false, st));
  MPAP_TRY(copy_in(rm->fwd_edge, fe.data(), sizeof(int4) * rm->E, false, st));
  MPAP_TRY(finish_reverse(rm, st));
  MPAP_CK(cudaStreamSynchronize(st));
  *out = rm;
  return MPAP_OK;
}

}  // namespace mpap
