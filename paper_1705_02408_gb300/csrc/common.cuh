// Device-side building blocks shared by the MPAP kernels (sm_103a).
//
// Floating-point convention: every geometric quantity is evaluated with explicit
// round-to-nearest binary32 intrinsics (__fadd_rn, __fmul_rn, __fdiv_rn,
// __fsqrt_rn) in a fixed operation order, so no multiply-add contraction can occur
// and results are bit-reproducible against a plain IEEE-754 evaluation of the
// same expressions.  Floats become integers only through exact power-of-two
// scalings followed by round-half-even (__float2ll_rn) or floor.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mpap {

// Front entry flags, stored in the high bits of the 32-bit plan reference.
constexpr uint32_t kOpen = 0x80000000u;     // plan is in P_open
constexpr uint32_t kNew = 0x40000000u;      // candidate of the current wavefront
constexpr uint32_t kPidMask = 0x3FFFFFFFu;  // arena index (or parent index if kNew)
constexpr uint32_t kNone = 0xFFFFFFFFu;

// Device error bits (MPAP_ERR_CAPACITY unless noted).
constexpr uint32_t kErrFront = 1u;
constexpr uint32_t kErrArena = 2u;
constexpr uint32_t kErrGroup = 4u;
constexpr uint32_t kErrList = 8u;
constexpr uint32_t kErrEdge = 16u;
constexpr uint32_t kErrPath = 32u;
constexpr uint32_t kErrLevel = 64u;     // a quality level above K (MPAP_ERR_INVALID_ARG)

constexpr float kTwo24 = 16777216.0f;
constexpr float kTwo20 = 1048576.0f;

// Environment and connection model, passed by value to kernels.
struct Geom {
  int dim;        // 2, 3, or 6 (double integrator)
  int dp;         // position axes (2 or 3)
  int nb;         // number of boxes
  int G;          // grid cells per axis
  int n_f;
  int M;          // sub-steps per connection
  const float* box_lo;    // [nb][3]
  const float* box_hi;
  const uint8_t* grid;    // [G^dp], x fastest
  float r;
  float T;
  // double-integrator constants (rounded once from double on the host)
  float c1, c2, c3, e1, e2, inv6, dtm;
  float invM;             // 1 / M
  int64_t Tq;             // round(T 2^24)
  // 1 when M inc max(n_f, K - n_f) < 2^31 for every edge's increment inc (levels
  // 0..K): the transfer's partial sums then fit 32-bit integers exactly
  int narrow;
  // camera-heading form (Sec. 4.1, features in the field of view of the yaw):
  // n_head level tables [n_head][G^dp], table y for the heading 2 pi y / n_head,
  // node yaws [V]; n_head = 0: the one grid above
  int n_head;
  const uint8_t* head_levels;
  const float* yaw;
  float cbin;             // n_head / (2 pi), rounded once from double
};

// Yaw constants, rounded once from double.
constexpr float kTwoPiF = (float)(2.0 * 3.14159265358979323846);
constexpr float kPiF = (float)3.14159265358979323846;
constexpr float kInvTwoPiF = (float)(1.0 / (2.0 * 3.14159265358979323846));

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64
// multiplies with the published multipliers, the key advanced by the published
// Weyl constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox4x32_10(uint32_t& x0, uint32_t& x1, uint32_t& x2,
                                              uint32_t& x3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
    uint32_t lo_a = m0 * x0, hi_a = __umulhi(m0, x0);
    uint32_t lo_b = m1 * x2, hi_b = __umulhi(m1, x2);
    uint32_t y0 = hi_b ^ x1 ^ k0;
    uint32_t y2 = hi_a ^ x3 ^ k1;
    x0 = y0;
    x1 = lo_b;
    x2 = y2;
    x3 = lo_a;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

__device__ __forceinline__ float unit24(uint32_t w) {
  return __fmul_rn((float)(w >> 8), 5.9604644775390625e-8f);  // 2^-24, exact
}

// ---------------------------------------------------------------------------
// Geometry
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool in_box(const float* lo, const float* hi, int dp, const float p[3]) {
  bool in = true;
#pragma unroll
  for (int i = 0; i < 3; ++i)
    if (i < dp) in = in && (p[i] >= lo[i]) && (p[i] <= hi[i]);
  return in;
}

template <int DP>
__device__ __forceinline__ int level_at_t(const Geom& g, const float p[3]) {
  int c[3] = {0, 0, 0};
  const float Gf = (float)g.G;
#pragma unroll
  for (int i = 0; i < DP; ++i) {
    int ci = (int)floorf(__fmul_rn(p[i], Gf));
    ci = ci < 0 ? 0 : ci;
    ci = ci > g.G - 1 ? g.G - 1 : ci;
    c[i] = ci;
  }
  size_t idx = (DP == 2) ? ((size_t)c[1] * g.G + c[0]) : (((size_t)c[2] * g.G + c[1]) * g.G + c[0]);
  return (int)__ldg(g.grid + idx);
}

__device__ __forceinline__ int level_at(const Geom& g, const float p[3]) {
  return g.dp == 2 ? level_at_t<2>(g, p) : level_at_t<3>(g, p);
}

// Quality level at checkpoint m (position p) of connection c: the grid's level of
// p's cell, or in the heading form the level of p's cell in the table of the
// heading nearest to the checkpoint's yaw.
template <int DP>
__device__ __forceinline__ int level_ck_t(const Geom& g, const float* yaw_c, int m, const float p[3]) {
  if (g.n_head == 0) return level_at_t<DP>(g, p);
  const float t = __fmul_rn((float)m, g.invM);
  const float psi = __fadd_rn(yaw_c[0], __fmul_rn(t, yaw_c[1]));
  int y = __float2int_rn(__fmul_rn(psi, g.cbin));
  y = ((y % g.n_head) + g.n_head) % g.n_head;
  int c[3] = {0, 0, 0};
  const float Gf = (float)g.G;
#pragma unroll
  for (int i = 0; i < DP; ++i) {
    int ci = (int)floorf(__fmul_rn(p[i], Gf));
    ci = ci < 0 ? 0 : ci;
    ci = ci > g.G - 1 ? g.G - 1 : ci;
    c[i] = ci;
  }
  const size_t cells = (size_t)g.G * g.G * (DP == 3 ? g.G : 1);
  const size_t idx = (DP == 2) ? ((size_t)c[1] * g.G + c[0]) : (((size_t)c[2] * g.G + c[1]) * g.G + c[0]);
  return (int)__ldg(g.head_levels + (size_t)y * cells + idx);
}

// The optimal connection from state a to state b.
//   2D/3D: straight segment a + t d, t in [0, 1] (unit speed); cost = |d|.
//   6D:    p(t) = p0 + t (v0 + t (a0/2 + t j/6)) with a0 = 6 dp/T^2 - 2 dv/T and
//          j = 6 dv/T^2 - 12 dp/T^3 (dp = p1 - p0 - v0 T, dv = v1 - v0);
//          cost = T + sum_axes (12 dp^2/T^3 - 12 dp dv/T^2 + 4 dv^2/T).
struct Conn {
  float p0[3], v0[3], q2[3], q3[3];   // 6D cubic (q2 = a0/2, q3 = j/6)
  float d[3];                         // 2D/3D direction (p0 holds the start)
  float cost;
  float psi0, dpsi;                   // yaw at the start and its wrapped change (heading form)
};

// The yaw of the connection from node va to node vb (heading form): a constant
// rate along the shorter way round, psi(t) = psi0 + t dpsi, t = m / M.
__device__ __forceinline__ void conn_yaw(const Geom& g, Conn& c, uint32_t va, uint32_t vb) {
  c.psi0 = 0.0f;
  c.dpsi = 0.0f;
  if (g.n_head > 0) {
    const float ya = g.yaw[va], yb = g.yaw[vb];
    const float d = __fsub_rn(yb, ya);
    const float turns = rintf(__fmul_rn(d, kInvTwoPiF));
    c.psi0 = ya;
    c.dpsi = __fsub_rn(d, __fmul_rn(turns, kTwoPiF));
  }
}

// Cost only (the Near test), same operations and order as conn_setup.
template <int DIM>
__device__ __forceinline__ float conn_cost_t(const Geom& g, const float a[6], const float b[6]) {
  if (DIM != 6) {
    constexpr int DP = (DIM == 2) ? 2 : 3;
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < DP; ++i) {
      const float d = __fsub_rn(b[i], a[i]);
      const float sq = __fmul_rn(d, d);
      s = (i == 0) ? sq : __fadd_rn(s, sq);
    }
    return __fsqrt_rn(s);
  }
  float jsum = 0.0f;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float dpos = __fsub_rn(__fsub_rn(b[i], a[i]), __fmul_rn(a[3 + i], g.T));
    const float dvel = __fsub_rn(b[3 + i], a[3 + i]);
    const float t1 = __fmul_rn(__fmul_rn(g.c1, dpos), dpos);
    const float t2 = __fmul_rn(__fmul_rn(g.c2, dpos), dvel);
    const float t3 = __fmul_rn(__fmul_rn(g.c3, dvel), dvel);
    const float ji = __fadd_rn(__fsub_rn(t1, t2), t3);
    jsum = (i == 0) ? ji : __fadd_rn(jsum, ji);
  }
  return __fadd_rn(g.T, jsum);
}

template <int DIM>
__device__ __forceinline__ void conn_setup_t(const Geom& g, const float a[6], const float b[6], Conn& c) {
  if (DIM != 6) {
    constexpr int DP = (DIM == 2) ? 2 : 3;
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      if (i < DP) {
        c.p0[i] = a[i];
        c.d[i] = __fsub_rn(b[i], a[i]);
        const float sq = __fmul_rn(c.d[i], c.d[i]);
        s = (i == 0) ? sq : __fadd_rn(s, sq);
      } else {
        c.p0[i] = 0.0f;
        c.d[i] = 0.0f;
      }
    }
    c.cost = __fsqrt_rn(s);
    c.psi0 = 0.0f;
    c.dpsi = 0.0f;
    return;
  }
  float jsum = 0.0f;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float dpos = __fsub_rn(__fsub_rn(b[i], a[i]), __fmul_rn(a[3 + i], g.T));
    const float dvel = __fsub_rn(b[3 + i], a[3 + i]);
    const float t1 = __fmul_rn(__fmul_rn(g.c1, dpos), dpos);
    const float t2 = __fmul_rn(__fmul_rn(g.c2, dpos), dvel);
    const float t3 = __fmul_rn(__fmul_rn(g.c3, dvel), dvel);
    const float ji = __fadd_rn(__fsub_rn(t1, t2), t3);
    jsum = (i == 0) ? ji : __fadd_rn(jsum, ji);
    const float a0 = __fsub_rn(__fmul_rn(g.e1, dpos), __fmul_rn(g.e2, dvel));
    const float jk = __fsub_rn(__fmul_rn(g.e1, dvel), __fmul_rn(g.c1, dpos));
    c.p0[i] = a[i];
    c.v0[i] = a[3 + i];
    c.q2[i] = __fmul_rn(a0, 0.5f);
    c.q3[i] = __fmul_rn(jk, g.inv6);
  }
  c.cost = __fadd_rn(g.T, jsum);
  c.psi0 = 0.0f;
  c.dpsi = 0.0f;
}

__device__ __forceinline__ void conn_setup(const Geom& g, const float a[6], const float b[6], Conn& c) {
  if (g.dim == 6) conn_setup_t<6>(g, a, b, c);
  else if (g.dim == 3) conn_setup_t<3>(g, a, b, c);
  else conn_setup_t<2>(g, a, b, c);
}

// Position at the end of sub-interval m (m = 1..M).
template <int DIM>
__device__ __forceinline__ void conn_point_t(const Geom& g, const Conn& c, int m, float p[3]) {
  if (DIM != 6) {
    constexpr int DP = (DIM == 2) ? 2 : 3;
    const float t = __fmul_rn((float)m, g.invM);
#pragma unroll
    for (int i = 0; i < 3; ++i) p[i] = (i < DP) ? __fadd_rn(c.p0[i], __fmul_rn(t, c.d[i])) : 0.0f;
    return;
  }
  const float t = __fmul_rn((float)m, g.dtm);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float in = __fadd_rn(c.q2[i], __fmul_rn(t, c.q3[i]));
    const float mid = __fadd_rn(c.v0[i], __fmul_rn(t, in));
    p[i] = __fadd_rn(c.p0[i], __fmul_rn(t, mid));
  }
}

__device__ __forceinline__ void conn_point(const Geom& g, const Conn& c, int m, float p[3]) {
  if (g.dim == 6) conn_point_t<6>(g, c, m, p);
  else if (g.dim == 3) conn_point_t<3>(g, c, m, p);
  else conn_point_t<2>(g, c, m, p);
}

// Closed segment (2D/3D) against one closed box: slab clipping with IEEE division.
template <int DP>
__device__ __forceinline__ bool seg_hits_box(const float a[3], const float d[3], const float* lo,
                                             const float* hi) {
  float t0 = -INFINITY, t1 = INFINITY;
  bool miss = false;
#pragma unroll
  for (int i = 0; i < DP; ++i) {
    if (d[i] == 0.0f) {
      miss = miss || (a[i] < lo[i]) || (a[i] > hi[i]);
    } else {
      const float ta = __fdiv_rn(__fsub_rn(lo[i], a[i]), d[i]);
      const float tb = __fdiv_rn(__fsub_rn(hi[i], a[i]), d[i]);
      t0 = fmaxf(t0, fminf(ta, tb));
      t1 = fminf(t1, fmaxf(ta, tb));
    }
  }
  return !miss && (t0 <= t1) && (t1 >= 0.0f) && (t0 <= 1.0f);
}

// Box prefilter for scenes of at most 32 boxes: per axis a and bin i of a
// 64-bin grid over [0, 1), bins[(2a) 64 + i] holds the boxes whose low face lies
// below the top of bin i (every box at the last bin) and bins[(2a + 1) 64 + i]
// the boxes whose high face lies at or above the bottom of bin i (every box at
// bin 0).  A box meets the interval [l, h] on axis a only if it is in both
// bins[(2a) 64 + bin(h)] and bins[(2a + 1) 64 + bin(l)] (bins clamped to the
// grid; the 64x scaling is exact), so the AND over the axes is a superset of the
// boxes that a bounding box overlaps.
constexpr int kBoxBins = 64;
constexpr int kBinMaxBoxes = 32;

__device__ __forceinline__ int box_bin(float x) {
  const float f = floorf(x * (float)kBoxBins);
  return (f >= 0.0f) ? (f <= (float)(kBoxBins - 1) ? (int)f : kBoxBins - 1) : 0;
}

// Fills the prefilter table (dp axes) from the boxes in shared memory; all
// threads of the block take part.
__device__ __forceinline__ void build_box_bins(int nb, int dp, const float* s_lo, const float* s_hi,
                                               uint32_t* s_bins) {
  for (int t = threadIdx.x; t < dp * 2 * kBoxBins; t += blockDim.x) {
    const int a = t / (2 * kBoxBins), side = (t / kBoxBins) & 1, i = t % kBoxBins;
    uint32_t m = 0;
    for (int b = 0; b < nb; ++b) {
      const bool in = (side == 0) ? (i == kBoxBins - 1 || s_lo[3 * b + a] < (float)(i + 1) / (float)kBoxBins)
                                  : (i == 0 || s_hi[3 * b + a] >= (float)i / (float)kBoxBins);
      m |= in ? (1u << b) : 0u;
    }
    s_bins[t] = m;
  }
}

// Boxes (bit b = box b) that the bounding box [lo, hi] overlaps, exactly: the
// prefilter's candidates checked face by face.
template <int DP>
__device__ __forceinline__ uint32_t boxes_overlapping(const float lo[3], const float hi[3], const float* s_lo,
                                                      const float* s_hi, const uint32_t* s_bins) {
  uint32_t cand = 0xFFFFFFFFu;
#pragma unroll
  for (int a = 0; a < DP; ++a)
    cand &= s_bins[(2 * a) * kBoxBins + box_bin(hi[a])] & s_bins[(2 * a + 1) * kBoxBins + box_bin(lo[a])];
  uint32_t mask = 0;
  for (uint32_t mm = cand; mm; mm &= mm - 1) {
    const int b = __ffs(mm) - 1;
    const float* bl = s_lo + 3 * b;
    const float* bh = s_hi + 3 * b;
    bool overlap = true;
#pragma unroll
    for (int i = 0; i < DP; ++i) overlap = overlap && bl[i] <= hi[i] && bh[i] >= lo[i];
    mask |= overlap ? (1u << b) : 0u;
  }
  return mask;
}

// Collision of a connection against the boxes (box data in shared memory):
// 2D/3D exact slab test; 6D point tests at the M-1 interior checkpoints, where
// leaving the unit workspace also counts.
//
// Both forms first intersect the boxes with a bounding box of the connection and
// run the exact test only against boxes that overlap it.  6D: the bounding box of
// the checkpoints themselves (a closed box holds a checkpoint only if it overlaps
// their bounding box).  2D/3D: the segment's bounding box grown by 1e-5, which
// exceeds the rounding of the slab arithmetic by orders of magnitude, so a box
// outside it is also reported clear by the floating-point slab test.  With
// s_bins (at most 32 boxes) the overlapping boxes come from the prefilter table
// instead of a pass over every box; the set is the same.
template <int DIM>
__device__ __forceinline__ bool conn_collides_t(const Geom& g, const Conn& c, const float* s_lo,
                                                const float* s_hi, const uint32_t* s_bins) {
  if (DIM != 6) {
    constexpr int DP = (DIM == 2) ? 2 : 3;
    float lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < DP; ++i) {
      const float e = __fadd_rn(c.p0[i], c.d[i]);
      lo[i] = fminf(c.p0[i], e) - 1e-5f;
      hi[i] = fmaxf(c.p0[i], e) + 1e-5f;
    }
    if (s_bins) {
      for (uint32_t mm = boxes_overlapping<DP>(lo, hi, s_lo, s_hi, s_bins); mm; mm &= mm - 1) {
        const int b = __ffs(mm) - 1;
        if (seg_hits_box<DP>(c.p0, c.d, s_lo + 3 * b, s_hi + 3 * b)) return true;
      }
      return false;
    }
    for (int b = 0; b < g.nb; ++b) {
      const float* bl = s_lo + 3 * b;
      const float* bh = s_hi + 3 * b;
      bool overlap = true;
#pragma unroll
      for (int i = 0; i < DP; ++i) overlap = overlap && bl[i] <= hi[i] && bh[i] >= lo[i];
      if (overlap && seg_hits_box<DP>(c.p0, c.d, bl, bh)) return true;
    }
    return false;
  }
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int m = 1; m < g.M; ++m) {
    float p[3];
    conn_point_t<6>(g, c, m, p);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      lo[i] = fminf(lo[i], p[i]);
      hi[i] = fmaxf(hi[i], p[i]);
    }
  }
  if (g.M > 1 && (lo[0] < 0.0f || hi[0] > 1.0f || lo[1] < 0.0f || hi[1] > 1.0f || lo[2] < 0.0f || hi[2] > 1.0f))
    return true;
  for (int b0 = 0; b0 < g.nb; b0 += 32) {
    uint32_t mask = 0;
    if (s_bins) {
      mask = boxes_overlapping<3>(lo, hi, s_lo, s_hi, s_bins);
    } else {
      const int nbb = (g.nb - b0) < 32 ? (g.nb - b0) : 32;
      for (int j = 0; j < nbb; ++j) {
        const float* bl = s_lo + 3 * (b0 + j);
        const float* bh = s_hi + 3 * (b0 + j);
        const bool overlap = bl[0] <= hi[0] && bh[0] >= lo[0] && bl[1] <= hi[1] && bh[1] >= lo[1] &&
                             bl[2] <= hi[2] && bh[2] >= lo[2];
        mask |= overlap ? (1u << j) : 0u;
      }
    }
    if (!mask) continue;
    for (int m = 1; m < g.M; ++m) {
      float p[3];
      conn_point_t<6>(g, c, m, p);
      for (uint32_t mm = mask; mm; mm &= mm - 1) {
        const int b = b0 + __ffs(mm) - 1;
        if (in_box(s_lo + 3 * b, s_hi + 3 * b, 3, p)) return true;
      }
    }
  }
  return false;
}

__device__ __forceinline__ int64_t quantise_cost(float cost) {
  long long q = __float2ll_rn(__fmul_rn(cost, kTwo24));
  return q < 1 ? 1 : (int64_t)q;
}

// Per-edge perception transfer F_e(h) = max(C, h + S) from the M sub-steps
// (Sec. 4.1 heuristic on the quality grid): step m adds inc (n_f - k_m).  After m
// steps the heuristic is max(C_m, h + S_m), so its peak along the edge (the "for
// all t" form of Eq. 2) is max(Cmax, h + Smax) with Smax = max_m S_m and
// Cmax = max_m C_m.
template <typename I, int DIM, bool HEAD>
__device__ __forceinline__ void conn_transfer_i(const Geom& g, const Conn& c, int64_t cost_q, int64_t& S,
                                                int64_t& C, int64_t& Smax, int64_t& Cmax) {
  constexpr int DP = (DIM == 2) ? 2 : 3;
  const I inc = (I)((DIM == 6) ? g.Tq : cost_q);
  I s = 0, h = 0, smax = (sizeof(I) == 4) ? (I)INT32_MIN : (I)INT64_MIN, cmax = 0;
  const float yaw_c[2] = {c.psi0, c.dpsi};
  for (int m = 1; m <= g.M; ++m) {
    float p[3];
    conn_point_t<DIM>(g, c, m, p);
    const int lev = HEAD ? level_ck_t<DP>(g, yaw_c, m, p) : level_at_t<DP>(g, p);
    const I dm = inc * (I)(g.n_f - lev);
    s += dm;
    h += dm;
    h = h < 0 ? 0 : h;
    smax = s > smax ? s : smax;
    cmax = h > cmax ? h : cmax;
  }
  S = s;
  C = h;
  Smax = g.M > 0 ? (int64_t)smax : 0;
  Cmax = cmax;
}

// 32-bit partial sums where Geom::narrow proves them exact, 64-bit otherwise
// (the same values either way).  HEAD: the camera-heading form (levels from the
// table of the checkpoint's yaw; the caller has set the yaw with conn_yaw).
template <int DIM, bool HEAD = false>
__device__ __forceinline__ void conn_transfer_t(const Geom& g, const Conn& c, int64_t cost_q, int64_t& S,
                                                int64_t& C, int64_t& Smax, int64_t& Cmax) {
  if (g.narrow) conn_transfer_i<int32_t, DIM, HEAD>(g, c, cost_q, S, C, Smax, Cmax);
  else conn_transfer_i<int64_t, DIM, HEAD>(g, c, cost_q, S, C, Smax, Cmax);
}

// ---------------------------------------------------------------------------
// Warp helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  const unsigned l = lane_id();
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if (l >= (unsigned)o) v += t;
  }
  return v;
}

__device__ __forceinline__ int64_t shfl_i64(int64_t v, int src) {
  return (int64_t)__shfl_sync(0xFFFFFFFFu, (long long)v, src);
}
__device__ __forceinline__ int64_t shfl_xor_i64(int64_t v, int m) {
  return (int64_t)__shfl_xor_sync(0xFFFFFFFFu, (long long)v, m);
}
__device__ __forceinline__ int64_t shfl_up_i64(int64_t v, int o) {
  return (int64_t)__shfl_up_sync(0xFFFFFFFFu, (long long)v, o);
}

}  // namespace mpap
