// Roadmap construction on the GPU: Alg. 1 steps 1-2 and Alg. 2 (BuildGraph) of
// Ichter et al., "Perception-Aware Motion Planning via Multiobjective Search on
// GPUs" -- SampleFree, Near, Collision and the per-edge perception transfer.
//
// Every kernel covers all roadmaps of one call (blockIdx.y = roadmap), so a
// batch of B roadmaps costs the same number of launches and host round trips
// (three) as a single one.
//
// Layout in HBM (one roadmap):
//   x        float [6][V]      node states, SoA (p0 p1 p2 v0 v1 v2)
//   fwd_ptr  u32   [V+1]       out-edge CSR, neighbours ascending
//   fwd_edge int4  [E]         {dst, cost_q, S, C}
//   rev_ptr  u32   [V+1]       in-edge CSR, sources ascending
//   rev_edge int4  [E]         {src, cost_q, S, C}
//   is_goal  u8    [V], goal_list u32 [n_goal]
//
// Near (Cost < r) is evaluated only for pairs whose target lies in grid cells
// that meet a ball known to contain every neighbour: radius r around the source
// in 2D/3D; in 6D radius sqrt((r - T) T^3 / 3) around p0 + v0 T, because the
// control energy satisfies J >= 3 |p1 - p0 - v0 T|^2 / T^3 (its minimum over the
// velocity difference).  Both radii carry a generous margin over the binary32
// rounding of the cost, so the edge set is exactly that of the all-pairs test;
// rows are sorted by neighbour afterwards.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "internal.h"
#include "profile.h"

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

// The camera-heading part of a roadmap's geometry (after fill_geom_constants).
void set_heading_geom(mpap_roadmap* rm) {
  rm->geom.n_head = rm->n_head;
  rm->geom.head_levels = rm->head;
  rm->geom.yaw = rm->yaw;
  rm->geom.cbin = (float)((double)rm->n_head / (2.0 * 3.14159265358979323846));
}

// Per-roadmap descriptor read by every build kernel.
struct BuildJob {
  Geom g;
  float* x;                // [6][V]
  uint32_t V;
  uint32_t n;              // samples to draw (0: node states given)
  uint32_t key0, key1, qid;
  uint32_t a0;             // first attempt of the current sampling round
  uint32_t cand_count;     // candidates in the current round (0: nothing to do)
  uint32_t kept;           // samples kept before the current round
  float xi[6], xg[6];      // x_init, x_goal
  float* cand;             // [6][C]
  uint32_t* ok;            // [C]
  uint32_t* rank;          // [C+1]
  float goal_r2;
  uint8_t* is_goal;
  uint32_t* goal_list;
  int GC;                  // grid cells per axis for the Near scan
  float R;                 // conservative neighbour radius (grid units: the grid spans [0, 1))
  // grid coordinate of a node: (p + bin_shift v - bin_lo) * bin_inv per axis (6D:
  // the backward point p - T v / 2); a source queries around p - bin_shift v
  float bin_shift, bin_lo, bin_inv;
  uint32_t* cell_cnt;      // [NC+1]
  uint32_t* cell_start;    // [NC+1]
  uint32_t* cell_of;       // [V]
  uint32_t* sorted;        // [V] node ids in cell order
  uint32_t* pos_of;        // [V] position of each node in cell order
  unsigned long long* near_tests;  // evaluated Cost(v, u) < r tests
  float* sx;               // [6][V] states in cell order
  uint32_t* counts;        // [V+1] out-degrees, counted by the row pass
  uint32_t* indeg;         // [V+1] in-degrees, counted by the one-pass edge build
  uint32_t* fill;          // [V+1] reverse-row cursors
  int4* rows;              // [V][kRowCap] per-source edge rows of the one-pass build
  int2* rows_peak;         // [V][kRowCap] their transfer peaks {Smax, Cmax}
  uint32_t* ovf;           // [V] sources with more than kRowCap edges (count in status[3])
  uint32_t* fwd_ptr;
  int4* fwd_edge;
  uint32_t* fwd_dst;
  uint32_t* rev_ptr;
  int4* rev_edge;
  int2* fwd_peak;
  int2* rev_peak;
  uint32_t* status;        // [4]: error bits, n_goal, scan overflow, overflowing sources
  int K;                   // top quality level
};

struct ScanSeg {
  const uint32_t* in;
  uint32_t* out;
  uint32_t n;
  uint32_t* overflow;
};

// ---------------------------------------------------------------------------
// Exclusive scans, one block per segment: out[0..n] with out[n] = total
// (saturating at 0xFFFFFFFF and flagging *overflow).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_scan_segments(const ScanSeg* __restrict__ segs) {
  const ScanSeg sg = segs[blockIdx.x];
  __shared__ uint32_t warp_sums[32];
  __shared__ unsigned long long carry;
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0ull;
  __syncthreads();
  for (uint32_t base = 0; base < sg.n; base += 1024u) {
    const uint32_t i = base + threadIdx.x;
    const uint32_t v = (i < sg.n) ? sg.in[i] : 0u;
    const uint32_t incl = warp_incl_scan(v);
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) warp_sums[lane] = warp_incl_scan(warp_sums[lane]);
    __syncthreads();
    const unsigned long long excl = carry + (warp ? warp_sums[warp - 1] : 0u) + (unsigned long long)(incl - v);
    if (i < sg.n) {
      if (excl > 0xFFFFFFFFull) {
        sg.out[i] = 0xFFFFFFFFu;
        if (sg.overflow) *sg.overflow = 1u;
      } else {
        sg.out[i] = (uint32_t)excl;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_sums[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (carry > 0xFFFFFFFFull) {
      sg.out[sg.n] = 0xFFFFFFFFu;
      if (sg.overflow) *sg.overflow = 1u;
    } else {
      sg.out[sg.n] = (uint32_t)carry;
    }
  }
}

// ---------------------------------------------------------------------------
// SampleFree: candidate `att` is drawn from Philox4x32-10 with counter
// (att, 0, query_id, 0) (position) and (att, 1, query_id, 0) (velocity, 6D),
// key = seed; it is free iff outside every closed box (and |v| <= 1 in 6D).
// ---------------------------------------------------------------------------
__global__ void k_sample_candidates(const BuildJob* __restrict__ jobs) {
  const BuildJob& J = jobs[blockIdx.y];
  if (J.cand_count == 0) return;
  const Geom& g = J.g;
  extern __shared__ float s_box[];
  float* s_lo = s_box;
  float* s_hi = s_box + 3 * g.nb;
  for (int i = threadIdx.x; i < 3 * g.nb; i += blockDim.x) {
    s_lo[i] = g.box_lo[i];
    s_hi[i] = g.box_hi[i];
  }
  __syncthreads();
  const uint32_t C = J.cand_count;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < C; t += gridDim.x * blockDim.x) {
    const uint32_t att = J.a0 + t;
    uint32_t w0 = att, w1 = 0u, w2 = J.qid, w3 = 0u;
    philox4x32_10(w0, w1, w2, w3, J.key0, J.key1);
    float p[3] = {unit24(w0), unit24(w1), g.dp == 3 ? unit24(w2) : 0.0f};
    bool free = true;
    for (int b = 0; b < g.nb && free; ++b) free = !in_box(s_lo + 3 * b, s_hi + 3 * b, g.dp, p);
    float v[3] = {0.0f, 0.0f, 0.0f};
    if (free && g.dim == 6) {
      uint32_t u0 = att, u1 = 1u, u2 = J.qid, u3 = 0u;
      philox4x32_10(u0, u1, u2, u3, J.key0, J.key1);
      v[0] = __fsub_rn(__fmul_rn(2.0f, unit24(u0)), 1.0f);
      v[1] = __fsub_rn(__fmul_rn(2.0f, unit24(u1)), 1.0f);
      v[2] = __fsub_rn(__fmul_rn(2.0f, unit24(u2)), 1.0f);
      float vv = __fmul_rn(v[0], v[0]);
      vv = __fadd_rn(vv, __fmul_rn(v[1], v[1]));
      vv = __fadd_rn(vv, __fmul_rn(v[2], v[2]));
      free = (vv <= 1.0f);
    }
    J.cand[0 * (size_t)C + t] = p[0];
    J.cand[1 * (size_t)C + t] = p[1];
    J.cand[2 * (size_t)C + t] = p[2];
    J.cand[3 * (size_t)C + t] = v[0];
    J.cand[4 * (size_t)C + t] = v[1];
    J.cand[5 * (size_t)C + t] = v[2];
    J.ok[t] = free ? 1u : 0u;
  }
}

// Keeps the first n - kept free candidates of this round, in attempt order, as
// nodes 2 + kept + rank.
__global__ void k_take_samples(const BuildJob* __restrict__ jobs) {
  const BuildJob& J = jobs[blockIdx.y];
  const uint32_t C = J.cand_count;
  if (C == 0) return;
  const uint32_t need = J.n - J.kept;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < C; t += gridDim.x * blockDim.x) {
    if (!J.ok[t] || J.rank[t] >= need) continue;
    const uint32_t id = 2u + J.kept + J.rank[t];
#pragma unroll
    for (int a = 0; a < 6; ++a) J.x[(size_t)a * J.V + id] = J.cand[(size_t)a * C + t];
  }
}

__global__ void k_set_endpoints(const BuildJob* __restrict__ jobs, uint32_t njobs) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= njobs || jobs[j].n == 0) return;
  const BuildJob& J = jobs[j];
  for (int a = 0; a < 6; ++a) {
    J.x[(size_t)a * J.V + 0] = J.xi[a];
    J.x[(size_t)a * J.V + 1] = J.xg[a];
  }
}

// Per-job counters for the host: accepted candidates of the round, edge count,
// error bits, goal count, scan overflow.
__global__ void k_gather_status(const BuildJob* __restrict__ jobs, uint32_t njobs, uint32_t* out) {
  const uint32_t n_jobs_pad = njobs;
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= njobs) return;
  const BuildJob& J = jobs[j];
  out[6 * j + 0] = J.cand_count ? J.rank[J.cand_count] : 0u;
  out[6 * j + 1] = J.fwd_ptr[J.V];
  out[6 * j + 2] = J.status[0];
  out[6 * j + 3] = J.status[1];
  out[6 * j + 4] = J.status[2];
  out[6 * j + 5] = J.status[3];
  out[6 * n_jobs_pad + 2 * j] = (uint32_t)(*J.near_tests);
  out[6 * n_jobs_pad + 2 * j + 1] = (uint32_t)(*J.near_tests >> 32);
}

// Quality levels must lie in 0..K (Sec. 4.1 heuristic; the certification tables
// have K + 1 entries): a larger level sets an error bit.
__global__ void k_check_levels(const BuildJob* __restrict__ jobs) {
  const BuildJob& J = jobs[blockIdx.y];
  const uint32_t G = (uint32_t)J.g.G;
  const uint32_t cells = (J.g.dp == 2) ? G * G : G * G * G;
  bool bad = false;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cells; i += gridDim.x * blockDim.x)
    bad = bad || (int)J.g.grid[i] > J.K;
  // and every table of the camera-heading form
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cells * (uint32_t)J.g.n_head;
       i += gridDim.x * blockDim.x)
    bad = bad || (int)J.g.head_levels[i] > J.K;
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&J.status[0], kErrLevel);
}

// Node yaws of the camera-heading form (Sec. 4.1, a single-integrator yaw):
// node v's yaw is uniform in [-pi, pi) from Philox4x32-10 with counter
// (v, 2, query_id, 0), key = seed (sampled roadmaps; given node states keep 0).
__global__ void k_node_yaw(const BuildJob* __restrict__ jobs) {
  const BuildJob& J = jobs[blockIdx.y];
  if (J.g.n_head == 0 || J.n == 0) return;
  float* yaw = const_cast<float*>(J.g.yaw);
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < J.V; v += gridDim.x * blockDim.x) {
    uint32_t w0 = v, w1 = 2u, w2 = J.qid, w3 = 0u;
    philox4x32_10(w0, w1, w2, w3, J.key0, J.key1);
    const float u = __fmul_rn((float)(w0 >> 8), 1.0f / 16777216.0f);
    yaw[v] = __fsub_rn(__fmul_rn(u, kTwoPiF), kPiF);
  }
}

// X_goal: nodes within goal_radius (position) of node 1.
__global__ void k_mark_goal(const BuildJob* __restrict__ jobs) {
  const BuildJob& J = jobs[blockIdx.y];
  const int dp = J.g.dp;
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < J.V; v += gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int i = 0; i < dp; ++i) {
      const float d = __fsub_rn(J.x[(size_t)i * J.V + v], J.x[(size_t)i * J.V + 1]);
      s = __fadd_rn(s, __fmul_rn(d, d));
    }
    const bool goal = (s <= J.goal_r2);
    J.is_goal[v] = goal ? 1 : 0;
    if (goal) J.goal_list[atomicAdd(&J.status[1], 1u)] = v;
  }
}

// ---------------------------------------------------------------------------
// Spatial binning of node positions for the Near scan.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int cell_coord(float p, int GC) {
  int c = (int)floorf(p * (float)GC);
  return c < 0 ? 0 : (c > GC - 1 ? GC - 1 : c);
}

// Grid coordinate of position p with velocity w along one axis.
__device__ __forceinline__ float bin_q(const BuildJob& J, float p, float w, float shift) {
  if (J.g.dim == 6) p = __fadd_rn(p, __fmul_rn(shift, w));
  return __fmul_rn(__fsub_rn(p, J.bin_lo), J.bin_inv);
}

__global__ void k_bin_count(const BuildJob* __restrict__ jobs) {
  const BuildJob& J = jobs[blockIdx.y];
  const int GC = J.GC;
  const bool six = J.g.dim == 6;
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < J.V; v += gridDim.x * blockDim.x) {
    uint32_t cell = 0;
    for (int i = J.g.dp - 1; i >= 0; --i) {
      const float w = six ? J.x[(size_t)(3 + i) * J.V + v] : 0.0f;
      cell = cell * GC + cell_coord(bin_q(J, J.x[(size_t)i * J.V + v], w, J.bin_shift), GC);
    }
    J.cell_of[v] = cell;
    atomicAdd(&J.cell_cnt[cell], 1u);
  }
}

__global__ void k_bin_scatter(const BuildJob* __restrict__ jobs) {
  const BuildJob& J = jobs[blockIdx.y];
  const int nc = (J.g.dim == 6) ? 6 : J.g.dp;
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < J.V; v += gridDim.x * blockDim.x) {
    const uint32_t cell = J.cell_of[v];
    const uint32_t pos = J.cell_start[cell] + atomicAdd(&J.cell_cnt[cell], 1u);
    J.sorted[pos] = v;
    J.pos_of[v] = pos;
    for (int c = 0; c < nc; ++c) J.sx[(size_t)c * J.V + pos] = J.x[(size_t)c * J.V + v];
  }
}

// ---------------------------------------------------------------------------
// Near + Collision + transfer.  For a source node v a warp walks the runs of grid
// cells (contiguous x-ranges) that meet the source's neighbour ball, flattened
// across up to 32 runs at a time, one candidate per lane, and evaluates
// Cost(v, u) exactly.  Pairs with Cost < r are queued in shared memory; every 32
// queued pairs are checked for collision and given their quantised cost and
// max-plus transfer (S, C) one per lane, so the expensive tests run 32-wide.
// ---------------------------------------------------------------------------
constexpr int kQueue = 64;
constexpr uint32_t kRowCap = 128;   // edges per source in the one-pass build

// Edge pass modes: one pass writing each source's edges into its own scratch row
// (kRow), and a second pass over only the sources whose rows overflowed, which
// writes straight into the CSR (kFillCsr, after the row pointers are known).
enum EdgeMode { kFillCsr = 1, kRow = 2 };

// Overflow pass: one flush of source v's queue, written straight into the CSR
// (forward row from out_base in discovery order, reverse records by cursor).
template <int DIM, bool HEAD>
__device__ __forceinline__ void edge_flush_csr(const BuildJob& J, uint32_t v, const float a[6], const uint32_t* q,
                                               int k, const float* s_lo, const float* s_hi, const uint32_t* s_bins,
                                               uint32_t out_base, uint32_t& running) {
  const Geom& g = J.g;
  const unsigned lane = lane_id();
  constexpr int nc = (DIM == 6) ? 6 : DIM;
  bool ok = false;
  Conn cn;
  uint32_t u = 0;
  if ((int)lane < k) {
    u = q[lane];
    float b[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int c = 0; c < nc; ++c) b[c] = J.x[(size_t)c * J.V + u];
    conn_setup_t<DIM>(g, a, b, cn);
    ok = !conn_collides_t<DIM>(g, cn, s_lo, s_hi, s_bins);
  }
  const unsigned bal = __ballot_sync(0xFFFFFFFFu, ok);
  if (ok) {
    const uint32_t rank = running + __popc(bal & ((1u << lane) - 1u));
    const int64_t cq = quantise_cost(cn.cost);
    int64_t S, C, Smax, Cmax;
    if constexpr (HEAD) conn_yaw(g, cn, v, u);
    conn_transfer_t<DIM, HEAD>(g, cn, cq, S, C, Smax, Cmax);
    if (cq > INT32_MAX || S > INT32_MAX || S < INT32_MIN || C > INT32_MAX || Smax > INT32_MAX || Cmax > INT32_MAX)
      atomicOr(&J.status[0], kErrEdge);
    const int4 rec = make_int4((int)u, (int)cq, (int)S, (int)C);
    const int2 pk = make_int2((int)Smax, (int)Cmax);
    J.fwd_edge[out_base + rank] = rec;
    J.fwd_dst[out_base + rank] = u;
    J.fwd_peak[out_base + rank] = pk;
    const uint32_t pos = J.rev_ptr[u] + atomicAdd(&J.fill[u], 1u);
    J.rev_edge[pos] = make_int4((int)v, rec.y, rec.z, rec.w);
    J.rev_peak[pos] = pk;
  }
  running += __popc(bal);
}

// Run rr of a source's neighbour ball: the x-range of one (y, z) row of cells,
// clipped to the ball's cross-section at the row's nearest point (conservative),
// as a range [rs, rs + rl) of cell-ordered nodes.
template <int DP>
__device__ __forceinline__ void neighbour_run(const BuildJob& J, uint32_t rr, uint32_t ny, const int clo[3],
                                              const int chi[3], const float ctr[3], float R, float cs, int GC,
                                              uint32_t& rs, uint32_t& rl) {
  const uint32_t yy = (uint32_t)clo[1] + rr % ny;
  const uint32_t zz = (DP == 3) ? (uint32_t)clo[2] + rr / ny : 0u;
  const float y0 = (float)yy * cs, y1 = (float)(yy + 1) * cs;
  const float dy = fmaxf(0.0f, fmaxf(y0 - ctr[1], ctr[1] - y1));
  float d2 = dy * dy;
  if (DP == 3) {
    const float z0 = (float)zz * cs, z1 = (float)(zz + 1) * cs;
    const float dz = fmaxf(0.0f, fmaxf(z0 - ctr[2], ctr[2] - z1));
    d2 += dz * dz;
  }
  // rows at the clamped grid border may hold nodes outside [0, 1]: keep the
  // full x-range there
  const bool border = (yy == 0 || yy == (uint32_t)GC - 1) || (DP == 3 && (zz == 0 || zz == (uint32_t)GC - 1));
  const float rem = R * R - d2;
  rs = 0;
  rl = 0;
  if (rem >= 0.0f || border) {
    int xlo = clo[0], xhi = chi[0];
    if (!border) {
      const float rx = sqrtf(rem) * 1.0001f + 1e-6f;
      xlo = cell_coord(ctr[0] - rx, GC);
      xhi = cell_coord(ctr[0] + rx, GC);
    }
    const uint32_t row = (zz * (uint32_t)GC + yy) * (uint32_t)GC;
    rs = J.cell_start[row + (uint32_t)xlo];
    rl = J.cell_start[row + (uint32_t)xhi + 1u] - rs;
  }
}

// Row pass: collision test, ranks and transfers of one queue flush whose lanes
// may belong to different sources (each lane carries its own source v).  The
// lanes of one source are contiguous and in discovery order, so one atomic add on
// the source's edge count per group hands out its ranks; the group that carries
// the count past kRowCap puts the source on the overflow list.
template <int DIM, bool HEAD>
__device__ __forceinline__ void edge_flush_rows(const BuildJob& J, const uint32_t* qu, const uint32_t* qv, int k,
                                                const float* s_lo, const float* s_hi, const uint32_t* s_bins) {
  const Geom& g = J.g;
  const unsigned lane = lane_id();
  constexpr int nc = (DIM == 6) ? 6 : DIM;
  bool ok = false;
  Conn cn;
  uint32_t u = 0, v = 0xFFFFFFFFu;
  if ((int)lane < k) {
    u = qu[lane];
    v = qv[lane];
    float a[6] = {0, 0, 0, 0, 0, 0}, b[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int c = 0; c < nc; ++c) {
      a[c] = J.x[(size_t)c * J.V + v];
      b[c] = J.x[(size_t)c * J.V + u];
    }
    conn_setup_t<DIM>(g, a, b, cn);
    ok = !conn_collides_t<DIM>(g, cn, s_lo, s_hi, s_bins);
  }
  const unsigned okb = __ballot_sync(0xFFFFFFFFu, ok);
  const unsigned same = __match_any_sync(0xFFFFFFFFu, v);
  const unsigned grp_ok = same & okb;
  const int leader = __ffs(same) - 1;
  uint32_t base = 0;
  if ((int)lane == leader && (int)lane < k && grp_ok) {
    const uint32_t n = (uint32_t)__popc(grp_ok);
    base = atomicAdd(&J.counts[v], n);
    if (base <= kRowCap && base + n > kRowCap) J.ovf[atomicAdd(&J.status[3], 1u)] = v;
  }
  base = __shfl_sync(0xFFFFFFFFu, base, leader);
  if (ok) {
    atomicAdd(&J.indeg[u], 1u);
    const uint32_t rank = base + (uint32_t)__popc(grp_ok & ((1u << lane) - 1u));
    if (rank < kRowCap) {
      const int64_t cq = quantise_cost(cn.cost);
      int64_t S, C, Smax, Cmax;
      if constexpr (HEAD) conn_yaw(g, cn, v, u);
      conn_transfer_t<DIM, HEAD>(g, cn, cq, S, C, Smax, Cmax);
      if (cq > INT32_MAX || S > INT32_MAX || S < INT32_MIN || C > INT32_MAX || Smax > INT32_MAX || Cmax > INT32_MAX)
        atomicOr(&J.status[0], kErrEdge);
      J.rows[(size_t)v * kRowCap + rank] = make_int4((int)u, (int)cq, (int)S, (int)C);
      J.rows_peak[(size_t)v * kRowCap + rank] = make_int2((int)Smax, (int)Cmax);
    }
  }
}

constexpr uint32_t kSourcesPerWarp = 8;

// Near + CollisionFree for every source, writing each source's edges to its
// scratch row with exact counts (sources beyond kRowCap edges go to the overflow
// pass).  A warp takes kSourcesPerWarp consecutive sources in cell order and
// feeds their Near candidates through one queue, so collision tests and
// transfers run on full warps across source boundaries.
template <int DIM, int WARPS, bool HEAD>
__global__ void __launch_bounds__(WARPS * 32, 32 / WARPS) k_edges_rows(const BuildJob* __restrict__ jobs,
                                                                    const uint32_t* __restrict__ job_ids) {
  const BuildJob& J = jobs[job_ids[blockIdx.y]];
  const Geom& g = J.g;
  extern __shared__ float smem[];
  float* s_lo = smem;
  float* s_hi = smem + 3 * g.nb;
  uint32_t* s_bins = reinterpret_cast<uint32_t*>(smem + 6 * g.nb);            // [dp][2][kBoxBins]
  uint32_t* s_queue = s_bins + 6 * kBoxBins;   // [warps][2][kQueue]
  constexpr int DP = (DIM == 2) ? 2 : 3;
  constexpr int nc = (DIM == 6) ? 6 : DIM;
  const unsigned lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t warp = threadIdx.x >> 5;
  uint32_t* qu = s_queue + warp * 2 * kQueue;
  uint32_t* qv = qu + kQueue;
  for (int i = threadIdx.x; i < 3 * g.nb; i += blockDim.x) {
    s_lo[i] = g.box_lo[i];
    s_hi[i] = g.box_hi[i];
  }
  __syncthreads();
  const bool binned = g.nb <= kBinMaxBoxes;
  if (binned) {
    build_box_bins(g.nb, DP, s_lo, s_hi, s_bins);
    __syncthreads();
  }
  const uint32_t V = J.V;
  const uint32_t first = (blockIdx.x * WARPS + warp) * kSourcesPerWarp;
  if (first >= V) return;
  const uint32_t last = min(first + kSourcesPerWarp, V);
  const int GC = J.GC;
  const float R = J.R;
  const float cs = 1.0f / (float)GC;
  uint32_t tests = 0;
  int qn = 0;
  for (uint32_t my_pos = first; my_pos < last; ++my_pos) {
    const uint32_t v = J.sorted[my_pos];
    float a[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int c = 0; c < nc; ++c) a[c] = J.sx[(size_t)c * V + my_pos];
    // centre and cell range of the neighbour ball
    float ctr[3] = {0, 0, 0};
    int clo[3] = {0, 0, 0}, chi[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < DP; ++i) {
      ctr[i] = bin_q(J, a[i], a[3 + i], -J.bin_shift);
      clo[i] = cell_coord(ctr[i] - R, GC);
      chi[i] = cell_coord(ctr[i] + R, GC);
    }
    const uint32_t ny = (uint32_t)(chi[1] - clo[1] + 1);
    const uint32_t nruns = ny * (DP == 3 ? (uint32_t)(chi[2] - clo[2] + 1) : 1u);
    for (uint32_t r0 = 0; r0 < nruns; r0 += 32) {
      uint32_t rs = 0, rl = 0;
      const uint32_t rr = r0 + lane;
      if (rr < nruns) neighbour_run<DP>(J, rr, ny, clo, chi, ctr, R, cs, GC, rs, rl);
      const uint32_t incl = warp_incl_scan(rl);
      const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
      const uint32_t excl = incl - rl;
      tests += total;
      for (uint32_t c0 = 0; c0 < total; c0 += 32) {
        const uint32_t c = c0 + lane;
        uint32_t owner = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const uint32_t probe = owner + step;
          if (__shfl_sync(0xFFFFFFFFu, excl, probe) <= c) owner = probe;
        }
        const uint32_t o_rs = __shfl_sync(0xFFFFFFFFu, rs, owner);
        const uint32_t o_ex = __shfl_sync(0xFFFFFFFFu, excl, owner);
        bool near = false;
        uint32_t sidx = 0;
        if (c < total) {
          sidx = o_rs + (c - o_ex);
          float b[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
          for (int k = 0; k < nc; ++k) b[k] = J.sx[(size_t)k * V + sidx];
          near = (sidx != my_pos) && (conn_cost_t<DIM>(g, a, b) < g.r);
        }
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, near);
        if (near) {
          const int at = qn + __popc(bal & lt);
          qu[at] = J.sorted[sidx];
          qv[at] = v;
        }
        qn += __popc(bal);
        if (qn >= 32) {
          __syncwarp();
          edge_flush_rows<DIM, HEAD>(J, qu, qv, 32, s_lo, s_hi, binned ? s_bins : nullptr);
          const bool mv = 32 + (int)lane < qn;
          const uint32_t ru = mv ? qu[32 + lane] : 0u, rv = mv ? qv[32 + lane] : 0u;
          __syncwarp();
          if (mv) {
            qu[lane] = ru;
            qv[lane] = rv;
          }
          qn -= 32;
          __syncwarp();
        }
      }
    }
  }
  __syncwarp();
  if (qn > 0) edge_flush_rows<DIM, HEAD>(J, qu, qv, qn, s_lo, s_hi, binned ? s_bins : nullptr);
  if (lane == 0) atomicAdd(J.near_tests, (unsigned long long)tests);
}

// Overflow pass: the sources whose rows outgrew kRowCap, one warp per source,
// edges written straight into the CSR at the source's row pointer.
template <int DIM, int WARPS, bool HEAD>
__global__ void __launch_bounds__(WARPS * 32, 32 / WARPS) k_edges_csr(const BuildJob* __restrict__ jobs,
                                                                   const uint32_t* __restrict__ job_ids) {
  const BuildJob& J = jobs[job_ids[blockIdx.y]];
  const Geom& g = J.g;
  extern __shared__ float smem[];
  float* s_lo = smem;
  float* s_hi = smem + 3 * g.nb;
  uint32_t* s_bins = reinterpret_cast<uint32_t*>(smem + 6 * g.nb);            // [dp][2][kBoxBins]
  uint32_t* s_queue = s_bins + 6 * kBoxBins;   // [warps][kQueue]
  constexpr int DP = (DIM == 2) ? 2 : 3;
  constexpr int nc = (DIM == 6) ? 6 : DIM;
  const unsigned lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t warp = threadIdx.x >> 5;
  uint32_t* q = s_queue + warp * kQueue;
  for (int i = threadIdx.x; i < 3 * g.nb; i += blockDim.x) {
    s_lo[i] = g.box_lo[i];
    s_hi[i] = g.box_hi[i];
  }
  __syncthreads();
  const bool binned = g.nb <= kBinMaxBoxes;
  if (binned) {
    build_box_bins(g.nb, DP, s_lo, s_hi, s_bins);
    __syncthreads();
  }
  const uint32_t slot = blockIdx.x * WARPS + warp;
  if (slot >= J.status[3]) return;
  const uint32_t v = J.ovf[slot];
  const uint32_t V = J.V;
  float a[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
  for (int c = 0; c < nc; ++c) a[c] = J.x[(size_t)c * V + v];
  // centre and cell range of the neighbour ball
  const int GC = J.GC;
  const float R = J.R;
  const float cs = 1.0f / (float)GC;
  float ctr[3] = {0, 0, 0};
  int clo[3] = {0, 0, 0}, chi[3] = {0, 0, 0};
#pragma unroll
  for (int i = 0; i < DP; ++i) {
    ctr[i] = bin_q(J, a[i], a[3 + i], -J.bin_shift);
    clo[i] = cell_coord(ctr[i] - R, GC);
    chi[i] = cell_coord(ctr[i] + R, GC);
  }
  const uint32_t ny = (uint32_t)(chi[1] - clo[1] + 1);
  const uint32_t nruns = ny * (DP == 3 ? (uint32_t)(chi[2] - clo[2] + 1) : 1u);
  const uint32_t my_pos = J.pos_of[v];
  uint32_t running = 0;
  uint32_t tests = 0;
  int qn = 0;
  const uint32_t out_base = J.fwd_ptr[v];
  for (uint32_t r0 = 0; r0 < nruns; r0 += 32) {
    // lane j describes run r0 + j: the x-range of one (y, z) row of cells, clipped
    // to the ball's cross-section at the row's nearest point (conservative)
    uint32_t rs = 0, rl = 0;
    const uint32_t rr = r0 + lane;
    if (rr < nruns) neighbour_run<DP>(J, rr, ny, clo, chi, ctr, R, cs, GC, rs, rl);
    const uint32_t incl = warp_incl_scan(rl);
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    const uint32_t excl = incl - rl;
    tests += total;
    for (uint32_t c0 = 0; c0 < total; c0 += 32) {
      const uint32_t c = c0 + lane;
      uint32_t owner = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const uint32_t probe = owner + step;
        if (__shfl_sync(0xFFFFFFFFu, excl, probe) <= c) owner = probe;
      }
      const uint32_t o_rs = __shfl_sync(0xFFFFFFFFu, rs, owner);
      const uint32_t o_ex = __shfl_sync(0xFFFFFFFFu, excl, owner);
      bool near = false;
      uint32_t sidx = 0;
      if (c < total) {
        sidx = o_rs + (c - o_ex);
        float b[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int k = 0; k < nc; ++k) b[k] = J.sx[(size_t)k * V + sidx];
        near = (sidx != my_pos) && (conn_cost_t<DIM>(g, a, b) < g.r);
      }
      const unsigned bal = __ballot_sync(0xFFFFFFFFu, near);
      if (near) q[qn + __popc(bal & lt)] = J.sorted[sidx];
      qn += __popc(bal);
      if (qn >= 32) {
        __syncwarp();
        edge_flush_csr<DIM, HEAD>(J, v, a, q, 32, s_lo, s_hi, binned ? s_bins : nullptr, out_base, running);
        const uint32_t rest = (32 + (int)lane < qn) ? q[32 + lane] : 0u;
        __syncwarp();
        if (32 + (int)lane < qn) q[lane] = rest;
        qn -= 32;
        __syncwarp();
      }
    }
  }
  __syncwarp();
  if (qn > 0) edge_flush_csr<DIM, HEAD>(J, v, a, q, qn, s_lo, s_hi, binned ? s_bins : nullptr, out_base, running);
  (void)tests;   // counted by the row pass
}

// One-pass build: copy each source's scratch row (at most kRowCap edges) into
// the forward CSR and scatter its edges into the reverse CSR (row pointers from
// the in-degrees the edge pass counted), one warp per source.  Rows stay in
// discovery (forward) or arrival (reverse) order: no kernel depends on the order
// of a row, and mpap_roadmap_export returns rows sorted by neighbour.
__global__ void k_compact_rows(const BuildJob* __restrict__ jobs) {
  const BuildJob& J = jobs[blockIdx.y];
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < J.V; v += warps) {
    const uint32_t b = J.fwd_ptr[v], len = J.fwd_ptr[v + 1] - b;
    if (len > kRowCap) continue;   // written by the overflow pass
    const int4* src = J.rows + (size_t)v * kRowCap;
    const int2* srcp = J.rows_peak + (size_t)v * kRowCap;
    for (uint32_t i = lane_id(); i < len; i += 32) {
      const int4 e = src[i];
      const int2 pk = srcp[i];
      J.fwd_edge[b + i] = e;
      J.fwd_dst[b + i] = (uint32_t)e.x;
      J.fwd_peak[b + i] = pk;
      const uint32_t pos = J.rev_ptr[e.x] + atomicAdd(&J.fill[e.x], 1u);
      J.rev_edge[pos] = make_int4((int)v, e.y, e.z, e.w);
      J.rev_peak[pos] = pk;
    }
  }
}

// In-degree count and reverse fill (one warp per source).
__global__ void k_indegree(const BuildJob* __restrict__ jobs) {
  const BuildJob& J = jobs[blockIdx.y];
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < J.V; v += warps)
    for (uint32_t e = J.fwd_ptr[v] + lane_id(); e < J.fwd_ptr[v + 1]; e += 32)
      atomicAdd(&J.counts[J.fwd_edge[e].x], 1u);
}

__global__ void k_reverse_fill(const BuildJob* __restrict__ jobs) {
  const BuildJob& J = jobs[blockIdx.y];
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < J.V; v += warps)
    for (uint32_t e = J.fwd_ptr[v] + lane_id(); e < J.fwd_ptr[v + 1]; e += 32) {
      const int4 ed = J.fwd_edge[e];
      const uint32_t pos = J.rev_ptr[ed.x] + atomicAdd(&J.fill[ed.x], 1u);
      J.rev_edge[pos] = make_int4((int)v, ed.y, ed.z, ed.w);
      J.rev_peak[pos] = J.fwd_peak[e];
    }
}

// ---------------------------------------------------------------------------
// Online update of a built roadmap (the map changes, the nodes stay): boxes are
// added and the quality grid may be replaced.  An added box can only remove
// edges, so an edge is tested against the added boxes alone, and only when a
// box of a bound on the edge's checkpoints meets one of them; its transfer is
// recomputed only when that bound meets a cell whose level the new grid
// changed.  The result is the roadmap the build would make from the same nodes
// on the updated scene.
//
// The bound.  2D/3D: the segment's bounding box.  6D: every position of the
// fixed-time double-integrator connection satisfies
//   |p(t) - (p0 + v0 t)| = |int_0^t (t - s) u(s) ds| <= sqrt(t^3 / 3) sqrt(J)
// (Cauchy-Schwarz, J = int |u|^2 = cost - T), so the connection stays within
// sqrt(T^3 J / 3) of the segment from p0 to p0 + v0 T; J comes from the edge's
// own quantised cost.  Both are grown by a margin far above the rounding of the
// floating-point checkpoints, so skipping an edge outside every added box and
// every changed cell changes no result.
// ---------------------------------------------------------------------------
constexpr float kReachMargin = 1e-3f;

template <int DIM>
__device__ __forceinline__ void edge_reach_box(const Geom& g, const float a[6], const float b[6], int cost_q,
                                               float lo[3], float hi[3]) {
  if (DIM != 6) {
    constexpr int DP = (DIM == 2) ? 2 : 3;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      lo[i] = (i < DP) ? fminf(a[i], b[i]) - kReachMargin : -INFINITY;
      hi[i] = (i < DP) ? fmaxf(a[i], b[i]) + kReachMargin : INFINITY;
    }
    return;
  }
  const float J = fmaxf(0.0f, (float)cost_q * (1.0f / 16777216.0f) - g.T) * 1.001f + 1e-3f;
  const float rho = sqrtf(g.T * g.T * g.T * J * (1.0f / 3.0f)) * 1.001f + kReachMargin;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float e = a[i] + a[3 + i] * g.T;
    lo[i] = fminf(a[i], e) - rho;
    hi[i] = fmaxf(a[i], e) + rho;
  }
}

struct UpdateJob {
  Geom g;                  // the updated scene (all boxes, the current grid)
  Geom g_add;              // the added boxes only
  const float* x;          // [6][V]
  uint32_t V;
  const uint32_t* ptr;     // [V+1] row pointers before the update
  const int4* edge;        // [E] records before the update
  const int2* peak;        // [E]
  int4* edge_upd;          // [E] records with the new transfers
  int2* peak_upd;          // [E]
  uint8_t* keep;           // [E]
  uint32_t* kept;          // [V+1] edges kept per source
  const uint32_t* ptr_new; // [V+1] row pointers after the update
  int4* edge_out;          // compacted forward CSR
  uint32_t* dst_out;
  int2* peak_out;
  uint32_t* status;        // [4] error bits, edges after the update, scan overflow, -
  int retransfer;          // the grid was replaced
  const int* creg;         // [6] index range of the cells whose level changed {min x, y, z, max x, y, z}
  float* box_lo_dst;       // where the added boxes go in the roadmap's box arrays
  float* box_hi_dst;
  uint32_t* ptr_out;       // [V+1] the roadmap's row pointers (ptr until the compaction, then ptr_new)
};

// Index range per axis of the cells whose level the new grid changes (one
// roadmap per blockIdx.y; creg starts at {INT_MAX x3, INT_MIN x3}).
// The roadmap's grid takes the new levels in the same pass (each cell is read
// and written by one thread only).
struct GridDiffJob {
  uint8_t* old_g;
  const uint8_t* new_g;
  int G, dp;
  int* creg;
};

__global__ void k_grid_diff(const GridDiffJob* __restrict__ jobs) {
  const GridDiffJob J = jobs[blockIdx.y];
  const size_t cells = (size_t)J.G * J.G * (J.dp == 3 ? J.G : 1);
  int mn[3] = {INT_MAX, INT_MAX, INT_MAX}, mx[3] = {INT_MIN, INT_MIN, INT_MIN};
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < cells; i += (size_t)gridDim.x * blockDim.x) {
    const uint8_t nv = J.new_g[i];
    if (J.old_g[i] != nv) {
      J.old_g[i] = nv;
      const int c[3] = {(int)(i % J.G), (int)((i / J.G) % J.G), J.dp == 3 ? (int)(i / ((size_t)J.G * J.G)) : 0};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        mn[k] = min(mn[k], c[k]);
        mx[k] = max(mx[k], c[k]);
      }
    }
  }
  if (mn[0] != INT_MAX) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      atomicMin(&J.creg[k], mn[k]);
      atomicMax(&J.creg[3 + k], mx[k]);
    }
  }
}

// One warp per source: collision of each out-edge against the added boxes and,
// when the grid changed, the edge's transfer on the new grid.  blockIdx.y picks
// the roadmap among those of this dimension.
template <int DIM>
__global__ void k_update_edges(const UpdateJob* __restrict__ jobs, const uint32_t* __restrict__ ids) {
  const UpdateJob& J = jobs[ids[blockIdx.y]];
  extern __shared__ float smem[];
  float* s_lo = smem;
  float* s_hi = smem + 3 * J.g_add.nb;
  for (int i = threadIdx.x; i < 3 * J.g_add.nb; i += blockDim.x) {
    s_lo[i] = J.g_add.box_lo[i];
    s_hi[i] = J.g_add.box_hi[i];
    if (blockIdx.x == 0) {
      // the added boxes join the roadmap's obstacles (read from their source here)
      J.box_lo_dst[i] = s_lo[i];
      J.box_hi_dst[i] = s_hi[i];
    }
  }
  __syncthreads();
  constexpr int nc = (DIM == 6) ? 6 : DIM;
  constexpr int DP = (DIM == 2) ? 2 : 3;
  // the changed cells as a closed region of positions (open towards a grid
  // border: positions beyond it fall into the border cells), grown by the margin
  float rlo[3] = {0, 0, 0}, rhi[3] = {0, 0, 0};
  bool any_changed = false;
  if (J.retransfer) {
    any_changed = J.creg[0] <= J.creg[3];
    const float Gf = (float)J.g.G;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int cmin = J.creg[i], cmax = J.creg[3 + i];
      rlo[i] = (i >= DP || cmin <= 0) ? -INFINITY : (float)cmin / Gf - kReachMargin;
      rhi[i] = (i >= DP || cmax >= J.g.G - 1) ? INFINITY : (float)(cmax + 1) / Gf + kReachMargin;
    }
  }
  const unsigned lane = lane_id();
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < J.V; v += warps) {
    float a[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int c = 0; c < nc; ++c) a[c] = J.x[(size_t)c * J.V + v];
    const uint32_t b0 = J.ptr[v], b1 = J.ptr[v + 1];
    uint32_t kept = 0;
    for (uint32_t e0 = b0; e0 < b1; e0 += 32) {
      const uint32_t e = e0 + lane;
      bool ok = false;
      if (e < b1) {
        int4 rec = J.edge[e];
        int2 pk = J.peak[e];
        float b[6] = {0, 0, 0, 0, 0, 0};
        if (DIM != 6) {
#pragma unroll
          for (int c = 0; c < nc; ++c) b[c] = J.x[(size_t)c * J.V + (uint32_t)rec.x];
        }
        float blo[3], bhi[3];
        edge_reach_box<DIM>(J.g, a, b, rec.y, blo, bhi);
        bool hit_box = false;
        for (int k = 0; k < J.g_add.nb && !hit_box; ++k)
          hit_box = blo[0] <= s_hi[3 * k] && bhi[0] >= s_lo[3 * k] && blo[1] <= s_hi[3 * k + 1] &&
                    bhi[1] >= s_lo[3 * k + 1] && blo[2] <= s_hi[3 * k + 2] && bhi[2] >= s_lo[3 * k + 2];
        const bool hit_cells = any_changed && blo[0] <= rhi[0] && bhi[0] >= rlo[0] && blo[1] <= rhi[1] &&
                               bhi[1] >= rlo[1] && blo[2] <= rhi[2] && bhi[2] >= rlo[2];
        ok = true;
        if (hit_box || hit_cells) {
          if (DIM == 6) {
#pragma unroll
            for (int c = 0; c < nc; ++c) b[c] = J.x[(size_t)c * J.V + (uint32_t)rec.x];
          }
          Conn cn;
          conn_setup_t<DIM>(J.g, a, b, cn);
          conn_yaw(J.g, cn, v, (uint32_t)rec.x);
          if (hit_box) ok = !conn_collides_t<DIM>(J.g_add, cn, s_lo, s_hi, nullptr);
          if (ok && hit_cells) {
            int64_t S, C, Smax, Cmax;
            if (J.g.n_head) conn_transfer_t<DIM, true>(J.g, cn, (int64_t)rec.y, S, C, Smax, Cmax);
            else conn_transfer_t<DIM, false>(J.g, cn, (int64_t)rec.y, S, C, Smax, Cmax);
            if (S > INT32_MAX || S < INT32_MIN || C > INT32_MAX || Smax > INT32_MAX || Cmax > INT32_MAX)
              atomicOr(&J.status[0], kErrEdge);
            rec.z = (int)S;
            rec.w = (int)C;
            pk = make_int2((int)Smax, (int)Cmax);
          }
        }
        J.edge_upd[e] = rec;
        J.peak_upd[e] = pk;
        J.keep[e] = ok ? 1 : 0;
      }
      kept += __popc(__ballot_sync(0xFFFFFFFFu, ok));
    }
    if (lane == 0) J.kept[v] = kept;
  }
}

// One warp per source: the kept edges, in their order, at the new row pointers
// (blockIdx.y: roadmap).
__global__ void k_update_compact(const UpdateJob* __restrict__ jobs) {
  const UpdateJob& J = jobs[blockIdx.y];
  const unsigned lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < J.V; v += warps) {
    const uint32_t b0 = J.ptr[v], b1 = J.ptr[v + 1];
    uint32_t out = J.ptr_new[v];
    for (uint32_t e0 = b0; e0 < b1; e0 += 32) {
      const uint32_t e = e0 + lane;
      const bool k = e < b1 && J.keep[e];
      const unsigned bal = __ballot_sync(0xFFFFFFFFu, k);
      if (k) {
        const uint32_t o = out + __popc(bal & lt);
        const int4 rec = J.edge_upd[e];
        J.edge_out[o] = rec;
        J.dst_out[o] = (uint32_t)rec.x;
        J.peak_out[o] = J.peak_upd[e];
      }
      out += __popc(bal);
    }
  }
}

// After the compaction: the new row pointers become the roadmap's, and the new
// edge count goes to the job's status word 1 (blockIdx.y: roadmap).
__global__ void k_update_ptrs(const UpdateJob* __restrict__ jobs) {
  const UpdateJob& J = jobs[blockIdx.y];
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v <= J.V; v += gridDim.x * blockDim.x) {
    const uint32_t p = J.ptr_new[v];
    J.ptr_out[v] = p;
    if (v == J.V) J.status[1] = p;
  }
}

template <int MODE, int WARPS, bool HEAD>
void launch_edges_h(int dim, dim3 grid, size_t smem, cudaStream_t st, const BuildJob* jobs, const uint32_t* ids) {
  const dim3 block(WARPS * 32);
  if (MODE == kRow) {
    if (dim == 6) k_edges_rows<6, WARPS, HEAD><<<grid, block, smem, st>>>(jobs, ids);
    else if (dim == 3) k_edges_rows<3, WARPS, HEAD><<<grid, block, smem, st>>>(jobs, ids);
    else k_edges_rows<2, WARPS, HEAD><<<grid, block, smem, st>>>(jobs, ids);
  } else {
    if (dim == 6) k_edges_csr<6, WARPS, HEAD><<<grid, block, smem, st>>>(jobs, ids);
    else if (dim == 3) k_edges_csr<3, WARPS, HEAD><<<grid, block, smem, st>>>(jobs, ids);
    else k_edges_csr<2, WARPS, HEAD><<<grid, block, smem, st>>>(jobs, ids);
  }
}

// dim: 2, 3, 6 for the grid form, plus kHeadDim for the camera-heading form
constexpr int kHeadDim = 100;

template <int MODE, int WARPS>
void launch_edges_w(int dim, dim3 grid, size_t smem, cudaStream_t st, const BuildJob* jobs, const uint32_t* ids) {
  if (dim > kHeadDim) launch_edges_h<MODE, WARPS, true>(dim - kHeadDim, grid, smem, st, jobs, ids);
  else launch_edges_h<MODE, WARPS, false>(dim, grid, smem, st, jobs, ids);
}

// One launch per dimension group; `warps` (4 or 8 warps per block) comes from
// the tuning table.
template <int MODE>
void launch_edges(int dim, uint32_t warps, uint32_t vmax, uint32_t njobs, size_t box_smem, cudaStream_t st,
                  const BuildJob* jobs, const uint32_t* ids) {
  LaunchScope ls(st, MODE == kRow ? "k_edges" : "k_edges_overflow");
  // row pass: kSourcesPerWarp sources per warp, queue of (target, source) pairs;
  // overflow pass: one source per warp
  const uint32_t per_block = (MODE == kRow) ? warps * kSourcesPerWarp : warps;
  const dim3 grid((vmax + per_block - 1) / per_block, njobs);
  const size_t smem = box_smem + sizeof(uint32_t) * 6 * kBoxBins +
                      sizeof(uint32_t) * warps * kQueue * (MODE == kRow ? 2 : 1);
  if (warps == 4) launch_edges_w<MODE, 4>(dim, grid, smem, st, jobs, ids);
  else launch_edges_w<MODE, 8>(dim, grid, smem, st, jobs, ids);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {

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

// (Re)allocates *p to hold `need` elements unless `cap` already suffices.
template <typename T>
int32_t grow(T** p, size_t& cap, size_t need) {
  if (need == 0) need = 1;
  if (*p && cap >= need) return MPAP_OK;
  cudaFree(*p);
  *p = nullptr;
  cap = 0;
  MPAP_CK(cudaMalloc((void**)p, need * sizeof(T)));
  cap = need;
  return MPAP_OK;
}

int32_t copy_in(void* dst, const void* src, size_t bytes, bool device_src, cudaStream_t st) {
  if (bytes == 0) return MPAP_OK;
  MPAP_CK(cudaMemcpyAsync(dst, src, bytes, device_src ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  return MPAP_OK;
}

}  // namespace

// Stream-ordered scratch from a library-owned memory pool that keeps freed
// memory mapped, so repeated calls of the same size do not map pages again.
cudaError_t scratch_alloc(void** p, size_t bytes, cudaStream_t st) {
  static cudaMemPool_t pools[64] = {};
  static std::mutex mu;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaMallocAsync(p, bytes, st);
  std::lock_guard<std::mutex> g(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool;
    e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[dev] = pool;
  }
  return cudaMallocFromPoolAsync(p, bytes, pools[dev], st);
}

void scratch_free(void* p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}

namespace {

// Scratch block carved into 256-byte aligned regions.
struct Carve {
  char* base = nullptr;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T* p = reinterpret_cast<T*>(base + off);
    off += count * sizeof(T);
    return p;
  }
};

// Conservative neighbour ball of the Near scan and the grid it runs on.  6D:
// per axis the minimum control energy of the fixed-time double-integrator
// connection splits into two non-negative parts,
//   J = 12 |(p1 - T v1 / 2) - (p0 + T v0 / 2)|^2 / T^3 + |v1 - v0|^2 / T,
// so Cost < r implies that the backward point p1 - T v1 / 2 of the target lies
// within sqrt((r - T) T^3 / 12) of the forward point p0 + T v0 / 2 of the source.
// Nodes are binned by their backward points, which lie in [-T/2, 1 + T/2] for
// |v| <= 1 (others are clamped into the border cells); the grid spans that range.
// The budget carries a margin far above binary32 rounding of the exact test.
void neighbour_ball(int dim, float r, float T, int dp, float& R, int& GC, float& shift, float& lo, float& inv) {
  if (dim == 6) {
    const double budget = std::max(0.0, ((double)r - (double)T) * 1.01 + 0.01);
    const double Td = (double)T;
    const double span = 1.0 + Td;
    shift = (float)(-0.5 * Td);
    lo = (float)(-0.5 * Td);
    inv = (float)(1.0 / span);
    R = (float)((std::sqrt(budget * Td * Td * Td / 12.0) * 1.001 + 1e-6) / span * 1.0001 + 1e-6);
    GC = (int)std::floor(4.0 / std::max((double)R, 1e-3));
    GC = std::min(std::max(GC, 1), 64);
  } else {
    shift = 0.0f;
    lo = 0.0f;
    inv = 1.0f;
    R = (float)((double)r * 1.001 + 1e-6);
    GC = (int)std::floor(2.0 / std::max((double)R, 1e-4));
    GC = std::min(std::max(GC, 1), dp == 2 ? 256 : 64);
  }
}

int32_t upload(void* d, const void* h, size_t bytes, cudaStream_t st) {
  MPAP_CK(cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, st));
  return MPAP_OK;
}

// Reverse CSR of the jobs' forward graphs (counts and fill are zeroed scratch).
int32_t build_reverse(uint32_t n, const std::vector<BuildJob>& hj, const BuildJob* d_jobs, ScanSeg* d_seg,
                      uint32_t Vmax, cudaStream_t st) {
  const int sms = sm_count();
  const dim3 gridw(std::min<uint32_t>((Vmax + 7) / 8, 4u * sms), n);
  {
    LaunchScope ls(st, "k_indegree");
    k_indegree<<<gridw, 256, 0, st>>>(d_jobs);
  }
  std::vector<ScanSeg> segs(n);
  for (uint32_t j = 0; j < n; ++j) segs[j] = ScanSeg{hj[j].counts, hj[j].rev_ptr, hj[j].V, nullptr};
  int32_t rc = upload(d_seg, segs.data(), sizeof(ScanSeg) * n, st);
  if (rc) return rc;
  {
    LaunchScope ls(st, "k_scan_segments");
    k_scan_segments<<<n, 1024, 0, st>>>(d_seg);
  }
  {
    LaunchScope ls(st, "k_reverse_fill");
    k_reverse_fill<<<gridw, 256, 0, st>>>(d_jobs);
  }
  MPAP_CK(cudaGetLastError());
  return MPAP_OK;
}

// Device buffers of one roadmap sized for V nodes (reused when large enough).
int32_t ensure_nodes(mpap_roadmap* rm, uint32_t V) {
  if (rm->x && rm->cap_V >= V) return MPAP_OK;
  cudaFree(rm->x);
  cudaFree(rm->is_goal);
  cudaFree(rm->goal_list);
  cudaFree(rm->fwd_ptr);
  cudaFree(rm->rev_ptr);
  rm->x = nullptr;
  rm->is_goal = nullptr;
  rm->goal_list = nullptr;
  rm->fwd_ptr = nullptr;
  rm->rev_ptr = nullptr;
  rm->cap_V = 0;
  MPAP_CK(cudaMalloc((void**)&rm->x, sizeof(float) * 6 * (size_t)V));
  MPAP_CK(cudaMalloc((void**)&rm->is_goal, V));
  MPAP_CK(cudaMalloc((void**)&rm->goal_list, sizeof(uint32_t) * (size_t)V));
  MPAP_CK(cudaMalloc((void**)&rm->fwd_ptr, sizeof(uint32_t) * ((size_t)V + 1)));
  MPAP_CK(cudaMalloc((void**)&rm->rev_ptr, sizeof(uint32_t) * ((size_t)V + 1)));
  rm->cap_V = V;
  return MPAP_OK;
}

int32_t ensure_edges(mpap_roadmap* rm, uint64_t E) {
  const size_t need = E ? (size_t)E : 1;
  if (rm->fwd_edge && rm->rev_edge && rm->fwd_dst && rm->fwd_peak && rm->rev_peak && rm->cap_E >= need)
    return MPAP_OK;
  cudaFree(rm->fwd_edge);
  cudaFree(rm->rev_edge);
  cudaFree(rm->fwd_dst);
  cudaFree(rm->fwd_peak);
  cudaFree(rm->rev_peak);
  rm->fwd_edge = nullptr;
  rm->rev_edge = nullptr;
  rm->fwd_dst = nullptr;
  rm->fwd_peak = nullptr;
  rm->rev_peak = nullptr;
  rm->cap_E = 0;
  MPAP_CK(cudaMalloc((void**)&rm->fwd_edge, sizeof(int4) * need));
  MPAP_CK(cudaMalloc((void**)&rm->rev_edge, sizeof(int4) * need));
  MPAP_CK(cudaMalloc((void**)&rm->fwd_dst, sizeof(uint32_t) * need));
  MPAP_CK(cudaMalloc((void**)&rm->fwd_peak, sizeof(int2) * need));
  MPAP_CK(cudaMalloc((void**)&rm->rev_peak, sizeof(int2) * need));
  rm->cap_E = need;
  return MPAP_OK;
}

// Box arrays hold room for kBoxRoom boxes beyond the scene's, so that an online
// update that adds a few needs no new allocation.
constexpr size_t kBoxRoom = 64;

int32_t ensure_scene(mpap_roadmap* rm, size_t nb, size_t cells) {
  if (!rm->box_lo || rm->cap_nb < 3 * nb + 3) {
    cudaFree(rm->box_lo);
    cudaFree(rm->box_hi);
    rm->box_lo = nullptr;
    rm->box_hi = nullptr;
    rm->cap_nb = 0;
    const size_t cap = 3 * (nb + kBoxRoom) + 3;
    MPAP_CK(cudaMalloc((void**)&rm->box_lo, sizeof(float) * cap));
    MPAP_CK(cudaMalloc((void**)&rm->box_hi, sizeof(float) * cap));
    rm->cap_nb = cap;
  }
  size_t c = rm->cap_cells;
  int32_t rc = grow(&rm->grid, c, cells);
  rm->cap_cells = c;
  return rc;
}

// Box arrays with room for nb boxes that keep the first nb_old (grown with room
// to spare; the old arrays are freed once the stream has copied them).
int32_t ensure_boxes_kept(mpap_roadmap* rm, size_t nb_old, size_t nb, cudaStream_t st) {
  if (rm->box_lo && rm->cap_nb >= 3 * nb + 3) return MPAP_OK;
  const size_t cap = 3 * (nb + kBoxRoom) + 3;
  float* lo = nullptr;
  float* hi = nullptr;
  if (cudaMalloc((void**)&lo, sizeof(float) * cap) != cudaSuccess ||
      cudaMalloc((void**)&hi, sizeof(float) * cap) != cudaSuccess) {
    cudaFree(lo);
    cudaFree(hi);
    set_error("roadmap_update: cudaMalloc of the box arrays failed");
    return MPAP_ERR_CUDA;
  }
  if (nb_old && rm->box_lo) {
    MPAP_CK(cudaMemcpyAsync(lo, rm->box_lo, sizeof(float) * 3 * nb_old, cudaMemcpyDeviceToDevice, st));
    MPAP_CK(cudaMemcpyAsync(hi, rm->box_hi, sizeof(float) * 3 * nb_old, cudaMemcpyDeviceToDevice, st));
  }
  MPAP_CK(cudaStreamSynchronize(st));
  cudaFree(rm->box_lo);
  cudaFree(rm->box_hi);
  rm->box_lo = lo;
  rm->box_hi = hi;
  rm->cap_nb = cap;
  return MPAP_OK;
}

}  // namespace

void roadmap_free_impl(mpap_roadmap* rm) {
  if (!rm) return;
  cudaFree(rm->head);
  cudaFree(rm->yaw);
  cudaFree(rm->x);
  cudaFree(rm->is_goal);
  cudaFree(rm->goal_list);
  cudaFree(rm->fwd_ptr);
  cudaFree(rm->fwd_edge);
  cudaFree(rm->fwd_dst);
  cudaFree(rm->fwd_peak);
  cudaFree(rm->rev_peak);
  cudaFree(rm->rev_ptr);
  cudaFree(rm->rev_edge);
  cudaFree(rm->box_lo);
  cudaFree(rm->box_hi);
  cudaFree(rm->grid);
  delete rm;
}

int32_t build_roadmaps_impl(uint32_t n, const BuildSpec* specs, mpap_roadmap** rms, cudaStream_t st) {
  if (n == 0) return MPAP_OK;
  std::vector<char> created(n, 0);
  char* blk = nullptr;
  auto fail = [&](int32_t rc) {
    if (blk) scratch_free(blk, st);
    for (uint32_t j = 0; j < n; ++j)
      if (created[j]) {
        roadmap_free_impl(rms[j]);
        rms[j] = nullptr;
      }
    return rc;
  };
#define MPAP_BTRY(x)                 \
  do {                               \
    const int32_t rc_ = (x);         \
    if (rc_ != MPAP_OK) return fail(rc_); \
  } while (0)
  std::vector<BuildJob> hj(n);
  std::vector<size_t> cand_cap(n), ncells(n);
  uint32_t Vmax = 0;
  int max_nb = 0;
  size_t max_qcells = 0;
  // 1. handles, buffers, scene copies, job constants
  for (uint32_t j = 0; j < n; ++j) {
    const BuildSpec& sp = specs[j];
    const mpap_scene* sc = sp.scene;
    if (!rms[j]) {
      rms[j] = new mpap_roadmap();
      created[j] = 1;
    }
    mpap_roadmap* rm = rms[j];
    rm->dim = sc->dim_kind;
    rm->nb = sc->nb;
    rm->G = sc->grid_G;
    rm->n_f = sc->n_f;
    rm->K = sc->K;
    rm->M = sp.M;
    rm->r = sp.r;
    rm->T = sp.T;
    rm->goal_radius = sp.goal_radius;
    rm->has_geometry = true;
    rm->V = sp.points ? sp.V_points : sp.params->n + 2u;
    rm->E = 0;
    rm->n_goal = 0;
    const uint32_t V = rm->V;
    const int dp = (rm->dim == 2) ? 2 : 3;
    const size_t cells = (size_t)rm->G * rm->G * (dp == 3 ? rm->G : 1);
    const bool dev = (sc->mem == MPAP_MEM_DEVICE);
    MPAP_BTRY(ensure_scene(rm, (size_t)rm->nb, cells));
    MPAP_BTRY(ensure_nodes(rm, V));
    MPAP_BTRY(copy_in(rm->box_lo, sc->box_lo, 12 * (size_t)rm->nb, dev, st));
    MPAP_BTRY(copy_in(rm->box_hi, sc->box_hi, 12 * (size_t)rm->nb, dev, st));
    MPAP_BTRY(copy_in(rm->grid, sc->grid_level, cells, dev, st));
    if (sp.points) MPAP_BTRY(copy_in(rm->x, sp.points, sizeof(float) * 6 * (size_t)V, false, st));
    rm->n_head = (sc->n_heading > 0 && sc->heading_levels) ? sc->n_heading : 0;
    if (rm->n_head) {
      size_t ch = rm->cap_head, cy = rm->cap_yaw;
      MPAP_BTRY(grow(&rm->head, ch, (size_t)rm->n_head * cells));
      rm->cap_head = ch;
      MPAP_BTRY(grow(&rm->yaw, cy, (size_t)V));
      rm->cap_yaw = cy;
      MPAP_BTRY(copy_in(rm->head, sc->heading_levels, (size_t)rm->n_head * cells, dev, st));
      if (sp.points)
        MPAP_BTRY(cuda_ok(cudaMemsetAsync(rm->yaw, 0, sizeof(float) * (size_t)V, st), "memset") ? MPAP_OK
                                                                                               : MPAP_ERR_CUDA);
    }
    fill_geom_constants(rm->geom, rm->dim, rm->nb, rm->G, rm->n_f, sp.M, sp.r, sp.T);
    set_heading_geom(rm);
    rm->geom.box_lo = rm->box_lo;
    rm->geom.box_hi = rm->box_hi;
    rm->geom.grid = rm->grid;
    {
      // 32-bit transfer sums are exact when M inc max(n_f, K - n_f) < 2^31, inc
      // = Tq (6D) or an edge's quantised cost (< r 2^24, 2D/3D)
      const double lmax = std::max((double)rm->n_f, (double)rm->K - (double)rm->n_f);
      const double inc_max = (rm->dim == 6) ? (double)rm->geom.Tq : std::ceil((double)sp.r * 16777216.0) + 1.0;
      rm->geom.narrow = ((double)sp.M * inc_max * lmax < 2147483647.0) ? 1 : 0;
    }
    max_qcells = std::max(max_qcells, cells);
    BuildJob& J = hj[j];
    std::memset(&J, 0, sizeof(J));
    J.g = rm->geom;
    J.K = rm->K;
    J.x = rm->x;
    J.V = V;
    J.n = sp.points ? 0u : sp.params->n;
    if (!sp.points) {
      J.key0 = (uint32_t)sp.params->seed;
      J.key1 = (uint32_t)(sp.params->seed >> 32);
      J.qid = sp.params->query_id;
      for (int a = 0; a < 6; ++a) {
        J.xi[a] = sp.params->x_init[a];
        J.xg[a] = sp.params->x_goal[a];
      }
    }
    J.goal_r2 = sp.goal_radius * sp.goal_radius;
    J.is_goal = rm->is_goal;
    J.goal_list = rm->goal_list;
    neighbour_ball(rm->dim, sp.r, sp.T, dp, J.R, J.GC, J.bin_shift, J.bin_lo, J.bin_inv);
    ncells[j] = dp == 2 ? (size_t)J.GC * J.GC : (size_t)J.GC * J.GC * J.GC;
    J.fwd_ptr = rm->fwd_ptr;
    J.rev_ptr = rm->rev_ptr;
    cand_cap[j] = J.n ? std::min<size_t>((size_t)J.n * 2 + 8192, (size_t)1 << 22) : 0;
    Vmax = std::max(Vmax, V);
    max_nb = std::max(max_nb, rm->nb);
  }
  // 2. one scratch block; the regions that must start at zero come first
  size_t bytes = 256 * 8 + (2 * sizeof(ScanSeg) + sizeof(BuildJob) + 48) * (size_t)n + 256 * (size_t)n;
  for (uint32_t j = 0; j < n; ++j)
    bytes += 256 * 13 + 4 * (ncells[j] + 1) + 16 + 32 * (cand_cap[j] + 1) + 4 * (ncells[j] + 1) +
             52 * ((size_t)hj[j].V + 1) + (sizeof(int4) + sizeof(int2)) * kRowCap * (size_t)hj[j].V + 1024;
  MPAP_CK(scratch_alloc((void**)&blk, bytes, st));
  Carve cv{blk, 0};
  for (uint32_t j = 0; j < n; ++j) hj[j].cell_cnt = cv.take<uint32_t>(ncells[j] + 1);
  for (uint32_t j = 0; j < n; ++j) hj[j].status = cv.take<uint32_t>(4);
  for (uint32_t j = 0; j < n; ++j) hj[j].near_tests = cv.take<unsigned long long>(1);
  for (uint32_t j = 0; j < n; ++j) {
    hj[j].counts = cv.take<uint32_t>((size_t)hj[j].V + 1);
    hj[j].indeg = cv.take<uint32_t>((size_t)hj[j].V + 1);
    hj[j].fill = cv.take<uint32_t>((size_t)hj[j].V + 1);
  }
  const size_t zero_bytes = cv.off;
  BuildJob* d_jobs = cv.take<BuildJob>(n);
  ScanSeg* d_seg = cv.take<ScanSeg>(2 * (size_t)n);
  uint32_t* d_gather = cv.take<uint32_t>(8 * (size_t)n);
  uint32_t* d_ids = cv.take<uint32_t>(n);
  for (uint32_t j = 0; j < n; ++j) {
    BuildJob& J = hj[j];
    J.cand = cv.take<float>(6 * cand_cap[j]);
    J.ok = cv.take<uint32_t>(cand_cap[j] + 1);
    J.rank = cv.take<uint32_t>(cand_cap[j] + 1);
    J.cell_start = cv.take<uint32_t>(ncells[j] + 1);
    J.cell_of = cv.take<uint32_t>(J.V);
    J.sorted = cv.take<uint32_t>(J.V);
    J.sx = cv.take<float>(6 * (size_t)J.V);
    J.rows = cv.take<int4>(kRowCap * (size_t)J.V);
    J.rows_peak = cv.take<int2>(kRowCap * (size_t)J.V);
    J.ovf = cv.take<uint32_t>((size_t)J.V);
    J.pos_of = cv.take<uint32_t>((size_t)J.V);
  }
  if (cv.off > bytes) {
    set_error("roadmap: scratch layout overflow");
    return fail(MPAP_ERR_CUDA);
  }
  MPAP_CK(cudaMemsetAsync(blk, 0, zero_bytes, st));
  const int sms = sm_count();
  std::vector<uint32_t> hg(8 * (size_t)n);
  auto gather = [&]() -> int32_t {
    {
      LaunchScope ls(st, "k_gather_status");
      k_gather_status<<<(n + 127) / 128, 128, 0, st>>>(d_jobs, n, d_gather);
    }
    MPAP_CK(cudaMemcpyAsync(hg.data(), d_gather, sizeof(uint32_t) * 8 * n, cudaMemcpyDeviceToHost, st));
    MPAP_CK(cudaStreamSynchronize(st));
    return MPAP_OK;
  };
  std::vector<ScanSeg> segs(n);

  // 3. SampleFree rounds (all sampling jobs together)
  bool any_sampling = false;
  for (uint32_t j = 0; j < n; ++j) any_sampling = any_sampling || hj[j].n > 0;
  if (any_sampling) {
    std::vector<uint64_t> att(n, 0);
    for (uint32_t round = 0;; ++round) {
      uint32_t maxc = 0;
      for (uint32_t j = 0; j < n; ++j) {
        BuildJob& J = hj[j];
        J.cand_count = 0;
        if (J.n == 0 || J.kept >= J.n) continue;
        const uint64_t max_att = (uint64_t)J.n * 64ull + 4096ull;
        if (att[j] >= max_att || att[j] > 0xFFFFFFFFull) {
          set_error("SampleFree: only %u of %u free samples in %llu attempts (roadmap %u)", J.kept, J.n,
                    (unsigned long long)max_att, j);
          return fail(MPAP_ERR_SAMPLING);
        }
        J.a0 = (uint32_t)att[j];
        J.cand_count = (uint32_t)std::min<uint64_t>(cand_cap[j], max_att - att[j]);
        maxc = std::max(maxc, J.cand_count);
      }
      if (maxc == 0) break;
      MPAP_BTRY(upload(d_jobs, hj.data(), sizeof(BuildJob) * n, st));
      if (round == 0) {
        LaunchScope ls(st, "k_set_endpoints");
        k_set_endpoints<<<(n + 127) / 128, 128, 0, st>>>(d_jobs, n);
      }
      const dim3 grid(std::min<uint32_t>((maxc + 255) / 256, 2u * sms), n);
      {
        LaunchScope ls(st, "k_sample_candidates");
        k_sample_candidates<<<grid, 256, sizeof(float) * 6 * max_nb, st>>>(d_jobs);
      }
      for (uint32_t j = 0; j < n; ++j) segs[j] = ScanSeg{hj[j].ok, hj[j].rank, hj[j].cand_count, nullptr};
      MPAP_BTRY(upload(d_seg, segs.data(), sizeof(ScanSeg) * n, st));
      {
        LaunchScope ls(st, "k_scan_segments");
        k_scan_segments<<<n, 1024, 0, st>>>(d_seg);
      }
      {
        LaunchScope ls(st, "k_take_samples");
        k_take_samples<<<grid, 256, 0, st>>>(d_jobs);
      }
      MPAP_BTRY(gather());
      for (uint32_t j = 0; j < n; ++j) {
        BuildJob& J = hj[j];
        if (J.cand_count == 0) continue;
        const uint32_t need = J.n - J.kept;
        J.kept += std::min(hg[6 * j + 0], need);
        att[j] += J.cand_count;
      }
    }
    for (uint32_t j = 0; j < n; ++j) hj[j].cand_count = 0;
  }
  MPAP_BTRY(upload(d_jobs, hj.data(), sizeof(BuildJob) * n, st));

  // 4. node yaws (camera-heading form), level check, goal region and spatial binning
  {
    bool any_head = false;
    for (uint32_t j = 0; j < n; ++j) any_head = any_head || (hj[j].g.n_head > 0 && hj[j].n > 0);
    if (any_head) {
      LaunchScope ls(st, "k_node_yaw");
      k_node_yaw<<<dim3(std::min<uint32_t>((Vmax + 255) / 256, 2u * sms), n), 256, 0, st>>>(d_jobs);
    }
  }
  {
    LaunchScope ls(st, "k_check_levels");
    k_check_levels<<<dim3((uint32_t)std::min<size_t>((max_qcells + 255) / 256, 2u * sms), n), 256, 0, st>>>(d_jobs);
  }
  const dim3 gridv(std::min<uint32_t>((Vmax + 255) / 256, 2u * sms), n);
  {
    LaunchScope ls(st, "k_mark_goal");
    k_mark_goal<<<gridv, 256, 0, st>>>(d_jobs);
  }
  {
    LaunchScope ls(st, "k_bin_count");
    k_bin_count<<<gridv, 256, 0, st>>>(d_jobs);
  }
  for (uint32_t j = 0; j < n; ++j) segs[j] = ScanSeg{hj[j].cell_cnt, hj[j].cell_start, (uint32_t)ncells[j], nullptr};
  MPAP_BTRY(upload(d_seg, segs.data(), sizeof(ScanSeg) * n, st));
  {
    LaunchScope ls(st, "k_scan_segments");
    k_scan_segments<<<n, 1024, 0, st>>>(d_seg);
  }
  // cell counts become scatter cursors (the count region precedes the status words)
  MPAP_CK(cudaMemsetAsync(blk, 0, (size_t)((char*)hj[0].status - blk), st));
  {
    LaunchScope ls(st, "k_bin_scatter");
    k_bin_scatter<<<gridv, 256, 0, st>>>(d_jobs);
  }

  // 5. Near + Collision: count pass, row pointers, fill pass (one launch per
  //    dimension and form: grid, or camera heading)
  std::vector<uint32_t> ids;
  const int dims[6] = {2, 3, 6, kHeadDim + 2, kHeadDim + 3, kHeadDim + 6};
  uint32_t id_off[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int di = 0; di < 6; ++di) {
    id_off[di] = (uint32_t)ids.size();
    for (uint32_t j = 0; j < n; ++j)
      if (hj[j].g.dim + (hj[j].g.n_head ? kHeadDim : 0) == dims[di]) ids.push_back(j);
  }
  id_off[6] = (uint32_t)ids.size();
  MPAP_BTRY(upload(d_ids, ids.data(), sizeof(uint32_t) * n, st));
  const size_t box_smem = sizeof(float) * 6 * max_nb;
  auto edges_pass = [&](int mode) {
    for (int di = 0; di < 6; ++di) {
      const uint32_t cnt = id_off[di + 1] - id_off[di];
      if (!cnt) continue;
      uint32_t vmax = 0;
      for (uint32_t k = id_off[di]; k < id_off[di + 1]; ++k) vmax = std::max(vmax, hj[ids[k]].V);
      const uint32_t warps = tuning_for(dims[di] % kHeadDim, vmax).edge_warps;
      if (mode == kFillCsr) {
        vmax = 0;
        for (uint32_t k = id_off[di]; k < id_off[di + 1]; ++k) vmax = std::max(vmax, hg[6 * ids[k] + 5]);
        if (vmax == 0) continue;
      }
      if (mode == kRow) launch_edges<kRow>(dims[di], warps, vmax, cnt, box_smem, st, d_jobs, d_ids + id_off[di]);
      else launch_edges<kFillCsr>(dims[di], warps, vmax, cnt, box_smem, st, d_jobs, d_ids + id_off[di]);
    }
  };
  // one pass: every source's edges into its scratch row, with exact out- and
  // in-degrees; forward and reverse row pointers in one scan launch
  edges_pass(kRow);
  segs.resize(2 * (size_t)n);
  for (uint32_t j = 0; j < n; ++j) {
    segs[j] = ScanSeg{hj[j].counts, hj[j].fwd_ptr, hj[j].V, hj[j].status + 2};
    segs[n + j] = ScanSeg{hj[j].indeg, hj[j].rev_ptr, hj[j].V, hj[j].status + 2};
  }
  MPAP_BTRY(upload(d_seg, segs.data(), sizeof(ScanSeg) * 2 * n, st));
  {
    LaunchScope ls(st, "k_scan_segments");
    k_scan_segments<<<2 * n, 1024, 0, st>>>(d_seg);
  }
  MPAP_BTRY(gather());
  bool row_overflow = false;
  for (uint32_t j = 0; j < n; ++j) {
    if (hg[6 * j + 4]) {
      set_error("roadmap %u: more than 2^32 - 1 edges", j);
      return fail(MPAP_ERR_CAPACITY);
    }
    mpap_roadmap* rm = rms[j];
    rm->E = hg[6 * j + 1];
    MPAP_BTRY(ensure_edges(rm, rm->E));
    hj[j].fwd_edge = rm->fwd_edge;
    hj[j].fwd_dst = rm->fwd_dst;
    hj[j].rev_edge = rm->rev_edge;
    hj[j].fwd_peak = rm->fwd_peak;
    hj[j].rev_peak = rm->rev_peak;
    row_overflow = row_overflow || hg[6 * j + 5] > 0;
  }
  MPAP_BTRY(upload(d_jobs, hj.data(), sizeof(BuildJob) * n, st));
  const dim3 gridw(std::min<uint32_t>((Vmax + 7) / 8, 4u * sms), n);
  {
    LaunchScope ls(st, "k_compact_rows");
    k_compact_rows<<<gridw, 256, 0, st>>>(d_jobs);
  }
  // sources with more than kRowCap neighbours: second pass over those only
  // (forward and reverse records)
  if (row_overflow) edges_pass(kFillCsr);
  MPAP_BTRY(gather());
  scratch_free(blk, st);
  blk = nullptr;
  for (uint32_t j = 0; j < n; ++j) {
    rms[j]->n_goal = hg[6 * j + 3];
    rms[j]->near_tests = (uint64_t)hg[6 * n + 2 * j] | ((uint64_t)hg[6 * n + 2 * j + 1] << 32);
    if (hg[6 * j + 2] & kErrLevel) {
      set_error("roadmap %u: a quality level of the grid exceeds K = %d", j, rms[j]->K);
      return fail(MPAP_ERR_INVALID_ARG);
    }
    if (hg[6 * j + 2]) {
      set_error("roadmap %u: an edge cost or transfer does not fit int32", j);
      return fail(MPAP_ERR_CAPACITY);
    }
  }
#undef MPAP_BTRY
  return MPAP_OK;
}

int32_t roadmap_from_csr_impl(uint32_t V, const uint32_t* row_ptr, const uint32_t* dst, const int32_t* cost_q,
                              const int32_t* S, const int32_t* C, const int32_t* Smax, const int32_t* Cmax,
                              const uint8_t* is_goal, mpap_roadmap** out, cudaStream_t st) {
  mpap_roadmap* rm = new mpap_roadmap();
  rm->V = V;
  rm->E = row_ptr[V];
  rm->has_geometry = false;
  std::vector<int4> fe(rm->E);
  std::vector<int2> fp(rm->E);
  for (uint64_t e = 0; e < rm->E; ++e) {
    fe[e] = make_int4((int)dst[e], cost_q[e], S[e], C[e]);
    fp[e] = (Smax && Cmax) ? make_int2(Smax[e], Cmax[e]) : make_int2(S[e], C[e]);
  }
  std::vector<uint32_t> goals;
  for (uint32_t v = 0; v < V; ++v)
    if (is_goal[v]) goals.push_back(v);
  rm->n_goal = (uint32_t)goals.size();
  int32_t rc;
  auto bail = [&](int32_t r) {
    roadmap_free_impl(rm);
    return r;
  };
  if ((rc = ensure_nodes(rm, V)) || (rc = ensure_edges(rm, rm->E))) return bail(rc);
  if (!cuda_ok(cudaMemsetAsync(rm->x, 0, sizeof(float) * 6 * (size_t)V, st), "memset")) return bail(MPAP_ERR_CUDA);
  if ((rc = copy_in(rm->is_goal, is_goal, V, false, st)) ||
      (rc = copy_in(rm->goal_list, goals.data(), 4 * goals.size(), false, st)) ||
      (rc = copy_in(rm->fwd_ptr, row_ptr, 4 * ((size_t)V + 1), false, st)) ||
      (rc = copy_in(rm->fwd_edge, fe.data(), sizeof(int4) * rm->E, false, st)) ||
      (rc = copy_in(rm->fwd_dst, dst, 4 * (size_t)rm->E, false, st)) ||
      (rc = copy_in(rm->fwd_peak, fp.data(), sizeof(int2) * rm->E, false, st)))
    return bail(rc);
  // reverse CSR with the build kernels (one job)
  BuildJob J;
  std::memset(&J, 0, sizeof(J));
  J.V = V;
  J.fwd_ptr = rm->fwd_ptr;
  J.fwd_edge = rm->fwd_edge;
  J.rev_ptr = rm->rev_ptr;
  J.rev_edge = rm->rev_edge;
  J.fwd_peak = rm->fwd_peak;
  J.rev_peak = rm->rev_peak;
  char* blk = nullptr;
  const size_t bytes = 4096 + 8 * ((size_t)V + 1) + 1024;
  if (!cuda_ok(scratch_alloc((void**)&blk, bytes, st), "scratch_alloc")) return bail(MPAP_ERR_CUDA);
  Carve cv{blk, 0};
  BuildJob* d_job = cv.take<BuildJob>(1);
  ScanSeg* d_seg = cv.take<ScanSeg>(1);
  J.counts = cv.take<uint32_t>((size_t)V + 1);
  J.fill = cv.take<uint32_t>((size_t)V + 1);
  std::vector<BuildJob> hj(1, J);
  if (!cuda_ok(cudaMemsetAsync(J.counts, 0, 4 * ((size_t)V + 1), st), "memset") ||
      !cuda_ok(cudaMemsetAsync(J.fill, 0, 4 * ((size_t)V + 1), st), "memset") ||
      (rc = upload(d_job, &J, sizeof(J), st)) || (rc = build_reverse(1, hj, d_job, d_seg, V, st))) {
    scratch_free(blk, st);
    return bail(rc ? rc : MPAP_ERR_CUDA);
  }
  scratch_free(blk, st);
  if (!cuda_ok(cudaStreamSynchronize(st), "sync")) return bail(MPAP_ERR_CUDA);
  *out = rm;
  return MPAP_OK;
}

int32_t roadmap_update_batch_impl(uint32_t n, mpap_roadmap* const* rms, const int32_t* nb_add,
                                  const float* const* add_lo, const float* const* add_hi,
                                  const uint8_t* const* grids, bool device, cudaStream_t st) {
  if (n == 0) return MPAP_OK;
  for (uint32_t j = 0; j < n; ++j) {
    if (!rms[j]->has_geometry) {
      set_error("roadmap_update: roadmap %u has no geometry", j);
      return MPAP_ERR_INVALID_ARG;
    }
    if (rms[j]->nb + nb_add[j] > 1024) {
      set_error("roadmap_update: roadmap %u would have more than 1024 boxes", j);
      return MPAP_ERR_INVALID_ARG;
    }
    if (rms[j]->n_head && grids && grids[j]) {
      set_error("roadmap_update: roadmap %u is in the camera-heading form; its levels cannot be replaced", j);
      return MPAP_ERR_INVALID_ARG;
    }
  }
  auto cells_of = [](const mpap_roadmap* rm) { return (size_t)rm->G * rm->G * (rm->dim == 2 ? 1 : rm->G); };
  // 1. box capacity (the old boxes stay where they are; the added ones are
  //    appended on the device), the updated geometry constants, sizes
  std::vector<int> nb_old(n);
  uint64_t E_sum = 0, V_sum = 0, add_sum = 0, cell_sum = 0;
  uint32_t Vmax = 0, n_grid = 0;
  int max_add = 0;
  for (uint32_t j = 0; j < n; ++j) {
    mpap_roadmap* rm = rms[j];
    nb_old[j] = rm->nb;
    const int nb = rm->nb + nb_add[j];
    int32_t rc = ensure_boxes_kept(rm, (size_t)rm->nb, (size_t)nb, st);
    if (rc) return rc;
    rm->nb = nb;
    fill_geom_constants(rm->geom, rm->dim, rm->nb, rm->G, rm->n_f, rm->M, rm->r, rm->T);
    set_heading_geom(rm);
    rm->geom.box_lo = rm->box_lo;
    rm->geom.box_hi = rm->box_hi;
    rm->geom.grid = rm->grid;
    const double lmax = std::max((double)rm->n_f, (double)rm->K - (double)rm->n_f);
    const double inc_max = (rm->dim == 6) ? (double)rm->geom.Tq : std::ceil((double)rm->r * 16777216.0) + 1.0;
    rm->geom.narrow = ((double)rm->M * inc_max * lmax < 2147483647.0) ? 1 : 0;
    E_sum += rm->E;
    V_sum += (uint64_t)rm->V + 1;
    Vmax = std::max(Vmax, rm->V);
    max_add = std::max(max_add, nb_add[j]);
    add_sum += (uint64_t)nb_add[j];
    if (grids && grids[j]) {
      ++n_grid;
      cell_sum += cells_of(rm);
    }
  }
  // 2. one scratch block: job tables, status words, changed-cell ranges, the
  //    host inputs staged in one upload, and per roadmap the updated records,
  //    keep flags, kept counts, new row pointers and reverse counters
  const size_t stage_bytes = device ? 0 : (2 * 12 * (size_t)add_sum + cell_sum);
  const size_t bytes = 256 * (8 * (size_t)n + 16) + 16 * (size_t)n + 24 * (size_t)n + stage_bytes +
                       16 * V_sum + (sizeof(int4) + sizeof(int2) + 1) * (size_t)E_sum +
                       (sizeof(UpdateJob) + sizeof(BuildJob) + sizeof(ScanSeg) + sizeof(GridDiffJob) + 4) * (size_t)n;
  char* blk = nullptr;
  MPAP_CK(scratch_alloc((void**)&blk, bytes, st));
  auto bail = [&](int32_t r) {
    scratch_free(blk, st);
    return r;
  };
  Carve cv{blk, 0};
  uint32_t* d_status = cv.take<uint32_t>(4 * (size_t)n);
  int* d_creg = cv.take<int>(6 * (size_t)n);
  UpdateJob* d_uj = cv.take<UpdateJob>(n);
  BuildJob* d_bj = cv.take<BuildJob>(n);
  ScanSeg* d_seg = cv.take<ScanSeg>(n);
  uint32_t* d_ids = cv.take<uint32_t>(n);
  GridDiffJob* d_gd = cv.take<GridDiffJob>(n);
  uint32_t* d_counts = cv.take<uint32_t>(2 * V_sum);     // reverse counters and fill cursors, all roadmaps
  uint8_t* d_stage = stage_bytes ? cv.take<uint8_t>(stage_bytes) : nullptr;
  std::vector<uint8_t> stage(stage_bytes);
  size_t st_box = 0, st_grid = 2 * 12 * (size_t)add_sum;
  std::vector<GridDiffJob> gd;
  std::vector<int> creg_init(6 * (size_t)n);
  std::vector<UpdateJob> uj(n);
  std::vector<BuildJob> bj(n);
  std::vector<ScanSeg> segs(n);
  size_t cnt_off = 0;
  for (uint32_t j = 0; j < n; ++j) {
    mpap_roadmap* rm = rms[j];
    const uint32_t V = rm->V;
    const uint64_t E = rm->E;
    UpdateJob& J = uj[j];
    std::memset(&J, 0, sizeof(J));
    J.g = rm->geom;
    J.g_add = rm->geom;
    J.g_add.nb = nb_add[j];
    if (nb_add[j]) {
      const size_t nbytes = 12 * (size_t)nb_add[j];
      if (device) {
        J.g_add.box_lo = add_lo[j];
        J.g_add.box_hi = add_hi[j];
      } else {
        std::memcpy(stage.data() + st_box, add_lo[j], nbytes);
        std::memcpy(stage.data() + st_box + nbytes, add_hi[j], nbytes);
        J.g_add.box_lo = reinterpret_cast<const float*>(d_stage + st_box);
        J.g_add.box_hi = reinterpret_cast<const float*>(d_stage + st_box + nbytes);
        st_box += 2 * nbytes;
      }
    }
    J.box_lo_dst = rm->box_lo + 3 * nb_old[j];
    J.box_hi_dst = rm->box_hi + 3 * nb_old[j];
    J.x = rm->x;
    J.V = V;
    J.ptr = rm->fwd_ptr;
    J.ptr_out = rm->fwd_ptr;
    J.edge = rm->fwd_edge;
    J.peak = rm->fwd_peak;
    J.edge_upd = cv.take<int4>(E);
    J.peak_upd = cv.take<int2>(E);
    J.keep = cv.take<uint8_t>(E);
    J.kept = cv.take<uint32_t>((size_t)V + 1);
    uint32_t* ptr_new = cv.take<uint32_t>((size_t)V + 1);
    J.ptr_new = ptr_new;
    J.edge_out = rm->fwd_edge;
    J.dst_out = rm->fwd_dst;
    J.peak_out = rm->fwd_peak;
    J.status = d_status + 4 * j;
    J.retransfer = (grids && grids[j]) ? 1 : 0;
    int* cr = d_creg + 6 * (size_t)j;
    for (int k = 0; k < 3; ++k) {
      creg_init[6 * (size_t)j + k] = INT_MAX;
      creg_init[6 * (size_t)j + 3 + k] = INT_MIN;
    }
    if (J.retransfer) {
      const size_t cells = cells_of(rm);
      const uint8_t* src = grids[j];
      if (!device) {
        std::memcpy(stage.data() + st_grid, grids[j], cells);
        src = d_stage + st_grid;
        st_grid += cells;
      }
      J.creg = cr;
      gd.push_back(GridDiffJob{rm->grid, src, (int)rm->G, rm->dim == 2 ? 2 : 3, cr});
    }
    segs[j] = ScanSeg{J.kept, ptr_new, V, d_status + 4 * j + 2};
    BuildJob& B = bj[j];
    std::memset(&B, 0, sizeof(B));
    B.V = V;
    B.fwd_ptr = rm->fwd_ptr;
    B.fwd_edge = rm->fwd_edge;
    B.rev_ptr = rm->rev_ptr;
    B.rev_edge = rm->rev_edge;
    B.fwd_peak = rm->fwd_peak;
    B.rev_peak = rm->rev_peak;
    B.counts = d_counts + cnt_off;
    B.fill = d_counts + V_sum + cnt_off;
    cnt_off += (size_t)V + 1;
  }
  if (cv.off > bytes) {
    set_error("roadmap_update: scratch layout overflow");
    return bail(MPAP_ERR_CUDA);
  }
  std::vector<uint32_t> ids;
  const int dims[3] = {2, 3, 6};
  uint32_t off[4] = {0, 0, 0, 0};
  for (int di = 0; di < 3; ++di) {
    off[di] = (uint32_t)ids.size();
    for (uint32_t j = 0; j < n; ++j)
      if (rms[j]->dim == dims[di]) ids.push_back(j);
  }
  off[3] = (uint32_t)ids.size();
  int32_t rc = MPAP_OK;
  if (!cuda_ok(cudaMemsetAsync(d_status, 0, 16 * (size_t)n, st), "memset") ||
      !cuda_ok(cudaMemsetAsync(d_counts, 0, sizeof(uint32_t) * 2 * V_sum, st), "memset"))
    return bail(MPAP_ERR_CUDA);
  if ((stage_bytes && (rc = upload(d_stage, stage.data(), stage_bytes, st))) ||
      (rc = upload(d_creg, creg_init.data(), sizeof(int) * 6 * (size_t)n, st)) ||
      (rc = upload(d_uj, uj.data(), sizeof(UpdateJob) * n, st)) ||
      (rc = upload(d_bj, bj.data(), sizeof(BuildJob) * n, st)) ||
      (rc = upload(d_seg, segs.data(), sizeof(ScanSeg) * n, st)) ||
      (rc = upload(d_ids, ids.data(), sizeof(uint32_t) * n, st)) ||
      (!gd.empty() && (rc = upload(d_gd, gd.data(), sizeof(GridDiffJob) * gd.size(), st))))
    return bail(rc);
  const int sms = sm_count();
  // 3. new grids: the cells whose level changes (their index range bounds the
  //    edges whose transfers are recomputed), written into the roadmaps' grids
  if (!gd.empty()) {
    uint32_t gmax = 0;
    for (const GridDiffJob& d : gd)
      gmax = std::max<uint32_t>(gmax, (uint32_t)(((size_t)d.G * d.G * (d.dp == 3 ? d.G : 1) + 255) / 256));
    LaunchScope ls(st, "k_grid_diff");
    k_grid_diff<<<dim3(std::min<uint32_t>(gmax, 64u), (uint32_t)gd.size()), 256, 0, st>>>(d_gd);
  }
  // 4. edges near the changes (one launch per dimension), new row pointers,
  //    compaction into the CSR, the row pointers and edge counts in place
  const uint32_t gx = std::min<uint32_t>((Vmax + 7) / 8, 4u * sms);
  const size_t sm = sizeof(float) * 6 * (size_t)max_add;
  {
    LaunchScope ls(st, "k_update_edges");
    for (int di = 0; di < 3; ++di) {
      const uint32_t cnt = off[di + 1] - off[di];
      if (!cnt) continue;
      const dim3 grid(gx, cnt);
      if (dims[di] == 6) k_update_edges<6><<<grid, 256, sm, st>>>(d_uj, d_ids + off[di]);
      else if (dims[di] == 3) k_update_edges<3><<<grid, 256, sm, st>>>(d_uj, d_ids + off[di]);
      else k_update_edges<2><<<grid, 256, sm, st>>>(d_uj, d_ids + off[di]);
    }
  }
  {
    LaunchScope ls(st, "k_scan_segments");
    k_scan_segments<<<n, 1024, 0, st>>>(d_seg);
  }
  {
    LaunchScope ls(st, "k_update_compact");
    k_update_compact<<<dim3(gx, n), 256, 0, st>>>(d_uj);
  }
  {
    LaunchScope ls(st, "k_update_ptrs");
    k_update_ptrs<<<dim3(std::min<uint32_t>((Vmax + 256) / 256, 4u * sms), n), 256, 0, st>>>(d_uj);
  }
  if (!cuda_ok(cudaGetLastError(), "update kernels")) return bail(MPAP_ERR_CUDA);
  // 5. the reverse CSR of every updated roadmap, then the status words back
  if ((rc = build_reverse(n, bj, d_bj, d_seg, Vmax, st))) return bail(rc);
  std::vector<uint32_t> hs(4 * (size_t)n);
  if (!cuda_ok(cudaMemcpyAsync(hs.data(), d_status, 16 * (size_t)n, cudaMemcpyDeviceToHost, st), "copy"))
    return bail(MPAP_ERR_CUDA);
  scratch_free(blk, st);
  if (!cuda_ok(cudaStreamSynchronize(st), "sync")) return MPAP_ERR_CUDA;
  for (uint32_t j = 0; j < n; ++j) rms[j]->E = hs[4 * j + 1];
  for (uint32_t j = 0; j < n; ++j)
    if (hs[4 * j]) {
      set_error("roadmap_update: an edge transfer of roadmap %u does not fit int32", j);
      return MPAP_ERR_CAPACITY;
    }
  return MPAP_OK;
}

}  // namespace mpap
