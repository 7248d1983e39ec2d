// MPAP CPU oracle -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, single-threaded restatement of the method of Ichter, Landry,
// Schmerling and Pavone, "Perception-Aware Motion Planning via Multiobjective
// Search on GPUs" (arXiv 1705.02408).  Only the tests, the smoke check and the
// CPU-baseline leg of the benchmark load this library.  It shares no code with the
// CUDA library: everything below is written from the paper and from the readings
// of it listed in the project's design notes (dominance tie rule, grid form of the
// heuristic, Monte Carlo error model, floating-point evaluation order).
//
// Built with -O2 -ffp-contract=off so that every float operation is one IEEE-754
// binary32 operation in the order written (no fused multiply-add).
//
// Contents
//   philox4x32_10        Salmon et al., SC'11 (counter-based RNG)
//   sample_free          SampleFree(n) (Sec. 3 primitives; Alg. 2 first step)
//   edge_eval            Cost / Near / Collision (Sec. 3 primitives) and the
//                        per-edge perception transfer (Alg. 1 step 2, Sec. 4.1)
//   build_graph          Alg. 2 (BuildGraph)
//   explore              Alg. 3 (Explore), RemoveDominated (Sec. 3)
//   certify              Monte Carlo verification (Sec. 3 final phase, Eq. 1)
//   plan_features        trajectory features of candidate plans (the project's
//                        certification surrogate; not in the paper)
//
// Parity is pinned by the -m "not gpu" tests (brute-force label enumeration,
// Dijkstra special cases, closed forms, exact slab-test truth, 6D steering
// optimality, Philox known answers, exact one-step Monte Carlo tail).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <set>
#include <vector>

namespace {

// ----------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As Easy as
// 1, 2, 3", SC'11).  Multipliers and Weyl key increments are the published ones.
// ----------------------------------------------------------------------------
const uint32_t kPhiloxM0 = 0xD2511F53u;
const uint32_t kPhiloxM1 = 0xCD9E8D57u;
const uint32_t kPhiloxW0 = 0x9E3779B9u;
const uint32_t kPhiloxW1 = 0xBB67AE85u;

void philox4x32_10(const uint32_t in_ctr[4], const uint32_t in_key[2], uint32_t out[4]) {
  uint32_t c0 = in_ctr[0], c1 = in_ctr[1], c2 = in_ctr[2], c3 = in_ctr[3];
  uint32_t k0 = in_key[0], k1 = in_key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += kPhiloxW0;
      k1 += kPhiloxW1;
    }
    uint64_t prod0 = (uint64_t)kPhiloxM0 * (uint64_t)c0;
    uint64_t prod1 = (uint64_t)kPhiloxM1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// A 32-bit word to a float uniform in [0, 1): the top 24 bits times 2^-24 (exact).
float word_to_unit(uint32_t w) { return (float)(w >> 8) * (1.0f / 16777216.0f); }

// Yaw (Sec. 4.1: a single-integrator yaw state tracked exactly).  Constants are
// rounded once from double.
const float kTwoPiF = (float)(2.0 * 3.14159265358979323846);
const float kPiF = (float)3.14159265358979323846;
const float kInvTwoPiF = (float)(1.0 / (2.0 * 3.14159265358979323846));

// Node v's yaw, uniform in [-pi, pi): Philox counter (v, 2, query_id, 0), key seed.
float node_yaw(uint64_t seed, uint32_t query_id, uint32_t v) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t ctr[4] = {v, 2u, query_id, 0u};
  uint32_t w[4];
  philox4x32_10(ctr, key, w);
  float t = word_to_unit(w[0]) * kTwoPiF;
  return t - kPiF;
}

const float kTwo24 = 16777216.0f;   // cost quantum is 2^-24
const float kTwo20 = 1048576.0f;    // Monte Carlo fixed point is 2^-20

// ----------------------------------------------------------------------------
// Scene and roadmap containers.
// ----------------------------------------------------------------------------
struct Scene {
  int dim = 2;               // 2, 3 or 6 (6 = 3D double integrator)
  int nb = 0;
  std::vector<float> lo, hi; // [nb][3]
  int G = 1;
  std::vector<uint8_t> level;// [G^Dp], x fastest
  int n_f = 12, K = 24;
  // camera-heading form (Sec. 4.1: features in the field of view of the yaw):
  // Y level tables, table y for the heading 2 pi y / Y; 0 = one table (level)
  int Y = 0;
  std::vector<uint8_t> head;  // [Y][G^Dp]
  int dp() const { return dim == 2 ? 2 : 3; }
};

struct Roadmap {
  Scene sc;
  float r = 0, T = 0, goal_radius = 0;
  int M = 16;
  uint32_t V = 0;
  std::vector<float> x[6];            // node coordinates, SoA (p0..p2, v0..v2)
  std::vector<uint8_t> is_goal;
  std::vector<uint32_t> row_ptr;      // forward CSR, neighbours in ascending order
  std::vector<uint32_t> dst;
  std::vector<int32_t> cost_q, S, C;  // per edge: quantised cost, max-plus transfer
  std::vector<int32_t> Smax, Cmax;    // per edge: peak of the transfer over its sub-steps
  std::vector<float> yaw;             // [V] node yaw (camera-heading form only)
  // 6D steering constants, computed once in double and rounded to float.
  float c1 = 0, c2 = 0, c3 = 0, e1 = 0, e2 = 0, inv6 = 0, dtm = 0, Tq_f = 0;
  int64_t Tq = 0;
};

void set_di6_constants(Roadmap& rm) {
  double Td = (double)rm.T;
  rm.c1 = (float)(12.0 / (Td * Td * Td));
  rm.c2 = (float)(12.0 / (Td * Td));
  rm.c3 = (float)(4.0 / Td);
  rm.e1 = (float)(6.0 / (Td * Td));
  rm.e2 = (float)(2.0 / Td);
  rm.inv6 = (float)(1.0 / 6.0);
  rm.dtm = (float)(Td / (double)rm.M);
  rm.Tq = (int64_t)llrintf(rm.T * kTwo24);
}

// Closed-box point test over the position axes.
bool point_in_box(const Scene& sc, int b, const float p[3]) {
  for (int i = 0; i < sc.dp(); ++i) {
    if (p[i] < sc.lo[3 * b + i] || p[i] > sc.hi[3 * b + i]) return false;
  }
  return true;
}

bool point_in_any_box(const Scene& sc, const float p[3]) {
  for (int b = 0; b < sc.nb; ++b)
    if (point_in_box(sc, b, p)) return true;
  return false;
}

// Grid cell of a position: clamp(floor(x * G), 0, G - 1) per axis (G a power of two,
// so x * G is exact).
int level_at(const Scene& sc, const float p[3]) {
  int c[3] = {0, 0, 0};
  for (int i = 0; i < sc.dp(); ++i) {
    float s = p[i] * (float)sc.G;
    int ci = (int)std::floor(s);
    if (ci < 0) ci = 0;
    if (ci > sc.G - 1) ci = sc.G - 1;
    c[i] = ci;
  }
  size_t idx = (sc.dp() == 2) ? ((size_t)c[1] * sc.G + c[0])
                              : (((size_t)c[2] * sc.G + c[1]) * sc.G + c[0]);
  return sc.level[idx];
}

// Grid cell index of a position (as level_at).
size_t cell_index(const Scene& sc, const float p[3]) {
  int c[3] = {0, 0, 0};
  for (int i = 0; i < sc.dp(); ++i) {
    float s = p[i] * (float)sc.G;
    int ci = (int)std::floor(s);
    if (ci < 0) ci = 0;
    if (ci > sc.G - 1) ci = sc.G - 1;
    c[i] = ci;
  }
  return (sc.dp() == 2) ? ((size_t)c[1] * sc.G + c[0]) : (((size_t)c[2] * sc.G + c[1]) * sc.G + c[0]);
}

// ----------------------------------------------------------------------------
// SampleFree(n) (Sec. 3): candidates come from Philox with counter
// (attempt, 0|1, query_id, 0) and key = seed; a candidate is kept iff it is in free
// space (outside every closed box; for the double integrator also |v| <= 1).  The
// first n kept candidates, in attempt order, are the samples.
// ----------------------------------------------------------------------------
bool sample_free(Roadmap& rm, uint32_t n, uint64_t seed, uint32_t query_id,
                 const float x_init[6], const float x_goal[6]) {
  const Scene& sc = rm.sc;
  const int dp = sc.dp();
  rm.V = n + 2;
  for (int a = 0; a < 6; ++a) rm.x[a].assign(rm.V, 0.0f);
  for (int a = 0; a < 6; ++a) {
    rm.x[a][0] = x_init[a];
    rm.x[a][1] = x_goal[a];
  }
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t kept = 0;
  const uint64_t max_attempts = (uint64_t)n * 64u + 4096u;
  for (uint64_t att = 0; kept < n; ++att) {
    if (att >= max_attempts || att > 0xFFFFFFFFull) return false;
    uint32_t ctr0[4] = {(uint32_t)att, 0u, query_id, 0u};
    uint32_t w[4];
    philox4x32_10(ctr0, key, w);
    float p[3] = {0.0f, 0.0f, 0.0f};
    for (int i = 0; i < dp; ++i) p[i] = word_to_unit(w[i]);
    float v[3] = {0.0f, 0.0f, 0.0f};
    bool ok = !point_in_any_box(sc, p);
    if (ok && sc.dim == 6) {
      uint32_t ctr1[4] = {(uint32_t)att, 1u, query_id, 0u};
      uint32_t wv[4];
      philox4x32_10(ctr1, key, wv);
      for (int i = 0; i < 3; ++i) v[i] = 2.0f * word_to_unit(wv[i]) - 1.0f;
      float vv = v[0] * v[0];
      vv = vv + v[1] * v[1];
      vv = vv + v[2] * v[2];
      ok = (vv <= 1.0f);
    }
    if (!ok) continue;
    uint32_t id = 2 + kept;
    for (int i = 0; i < 3; ++i) rm.x[i][id] = p[i];
    for (int i = 0; i < 3; ++i) rm.x[3 + i][id] = v[i];
    ++kept;
  }
  if (sc.Y > 0) {
    rm.yaw.assign(rm.V, 0.0f);
    for (uint32_t v = 0; v < rm.V; ++v) rm.yaw[v] = node_yaw(seed, query_id, v);
  }
  return true;
}

// Goal region X_goal: a ball of radius goal_radius around x_goal's position
// (any velocity).  Node 1 is x_goal itself, so X_goal always holds a sample (Sec. 3).
void mark_goal(Roadmap& rm) {
  const int dp = rm.sc.dp();
  rm.is_goal.assign(rm.V, 0);
  float r2 = rm.goal_radius * rm.goal_radius;
  for (uint32_t v = 0; v < rm.V; ++v) {
    float s = 0.0f;
    for (int i = 0; i < dp; ++i) {
      float d = rm.x[i][v] - rm.x[i][1];
      s = s + d * d;
    }
    rm.is_goal[v] = (s <= r2) ? 1 : 0;
  }
}

// ----------------------------------------------------------------------------
// The optimal connection u -> v (Sec. 3 primitives Cost and Collision).
//   2D / 3D kinematic: the straight segment, traversed at unit speed; cost is its
//     Euclidean length.
//   6D double integrator (Sec. 4.1, x'' = u): fixed duration T, minimum-energy
//     control a(t) = a0 + j t, cost = T + integral |a|^2 dt.
// Checkpoint m (m = 1..M) is the state at the end of the m-th of M equal
// sub-intervals.
// ----------------------------------------------------------------------------
struct EdgeGeom {
  float cost = 0;
  float a[3] = {0, 0, 0}, d[3] = {0, 0, 0};      // segment start and direction
  float v0[3] = {0, 0, 0}, q2[3] = {0, 0, 0}, q3[3] = {0, 0, 0};
  float J = 0;
  float a0[3] = {0, 0, 0}, jk[3] = {0, 0, 0};
  float psi0 = 0, dpsi = 0;                      // yaw at the start and its wrapped change
};

EdgeGeom edge_geom(const Roadmap& rm, uint32_t u, uint32_t v) {
  EdgeGeom g;
  if (rm.sc.Y > 0) {
    // yaw moves at a constant rate along the shorter way round
    const float d = rm.yaw[v] - rm.yaw[u];
    const float turns = std::nearbyint(d * kInvTwoPiF);
    g.psi0 = rm.yaw[u];
    g.dpsi = d - turns * kTwoPiF;
  }
  if (rm.sc.dim != 6) {
    const int dp = rm.sc.dp();
    float s = 0.0f;
    for (int i = 0; i < dp; ++i) {
      g.a[i] = rm.x[i][u];
      g.d[i] = rm.x[i][v] - rm.x[i][u];
      float sq = g.d[i] * g.d[i];
      s = (i == 0) ? sq : (s + sq);
    }
    g.cost = std::sqrt(s);
    return g;
  }
  float jsum = 0.0f;
  for (int i = 0; i < 3; ++i) {
    float p0 = rm.x[i][u], p1 = rm.x[i][v];
    float w0 = rm.x[3 + i][u], w1 = rm.x[3 + i][v];
    float dpos = (p1 - p0) - w0 * rm.T;      // delta p = p1 - p0 - v0 T
    float dvel = w1 - w0;                      // delta v = v1 - v0
    // Gramian form of the minimum control energy per axis:
    // 12 dp^2 / T^3 - 12 dp dv / T^2 + 4 dv^2 / T.
    float ji = ((rm.c1 * dpos) * dpos - (rm.c2 * dpos) * dvel) + (rm.c3 * dvel) * dvel;
    jsum = (i == 0) ? ji : (jsum + ji);
    g.a0[i] = (rm.e1 * dpos) - (rm.e2 * dvel);  // a0 = 6 dp / T^2 - 2 dv / T
    g.jk[i] = (rm.e1 * dvel) - (rm.c1 * dpos);  // j  = 6 dv / T^2 - 12 dp / T^3
    g.a[i] = p0;
    g.v0[i] = w0;
    g.q2[i] = g.a0[i] * 0.5f;
    g.q3[i] = g.jk[i] * rm.inv6;
  }
  g.J = jsum;
  g.cost = rm.T + jsum;
  return g;
}

void checkpoint(const Roadmap& rm, const EdgeGeom& g, int m, float p[3]) {
  p[0] = p[1] = p[2] = 0.0f;
  if (rm.sc.dim != 6) {
    float t = (float)m * (1.0f / (float)rm.M);
    for (int i = 0; i < rm.sc.dp(); ++i) p[i] = g.a[i] + t * g.d[i];
    return;
  }
  float t = (float)m * rm.dtm;
  for (int i = 0; i < 3; ++i) {
    // Horner: p0 + t (v0 + t (a0 / 2 + t j / 6))
    float in = g.q2[i] + t * g.q3[i];
    float mid = g.v0[i] + t * in;
    p[i] = g.a[i] + t * mid;
  }
}

// Quality level at checkpoint m of an edge (position p).  Grid form: the level of
// p's cell.  Camera-heading form: the yaw at the checkpoint, psi0 + (m / M) dpsi,
// picks the nearest of the Y headings 2 pi y / Y, whose table gives the level
// of p's cell.
int checkpoint_level(const Roadmap& rm, const EdgeGeom& g, int m, const float p[3]) {
  const Scene& sc = rm.sc;
  if (sc.Y == 0) return level_at(sc, p);
  const float t = (float)m * (1.0f / (float)rm.M);
  const float psi = g.psi0 + t * g.dpsi;
  const float cbin = (float)((double)sc.Y / (2.0 * 3.14159265358979323846));
  int y = (int)std::nearbyint(psi * cbin);
  y = ((y % sc.Y) + sc.Y) % sc.Y;
  const size_t cells = (sc.dim == 2) ? (size_t)sc.G * sc.G : (size_t)sc.G * sc.G * sc.G;
  return sc.head[(size_t)y * cells + cell_index(sc, p)];
}

// Exact-in-FP32 slab test of the closed segment a + t d, t in [0, 1], against a
// closed box.
bool segment_hits_box(const Scene& sc, int b, const float a[3], const float d[3]) {
  float t0 = -INFINITY, t1 = INFINITY;
  for (int i = 0; i < sc.dp(); ++i) {
    float lo = sc.lo[3 * b + i], hi = sc.hi[3 * b + i];
    if (d[i] == 0.0f) {
      if (a[i] < lo || a[i] > hi) return false;
      continue;
    }
    float ta = (lo - a[i]) / d[i];
    float tb = (hi - a[i]) / d[i];
    t0 = std::fmax(t0, std::fmin(ta, tb));
    t1 = std::fmin(t1, std::fmax(ta, tb));
  }
  return t0 <= t1 && t1 >= 0.0f && t0 <= 1.0f;
}

bool edge_collides(const Roadmap& rm, const EdgeGeom& g) {
  const Scene& sc = rm.sc;
  if (sc.dim != 6) {
    for (int b = 0; b < sc.nb; ++b)
      if (segment_hits_box(sc, b, g.a, g.d)) return true;
    return false;
  }
  // 15 interior checkpoints (the endpoints are free samples); a checkpoint outside
  // the unit workspace counts as a collision.
  for (int m = 1; m < rm.M; ++m) {
    float p[3];
    checkpoint(rm, g, m, p);
    for (int i = 0; i < 3; ++i)
      if (p[i] < 0.0f || p[i] > 1.0f) return true;
    if (point_in_any_box(sc, p)) return true;
  }
  return false;
}

int64_t quantise_cost(float cost) {
  int64_t q = (int64_t)llrintf(cost * kTwo24);
  return q < 1 ? 1 : q;
}

// Per-step heuristic increments along an edge (Sec. 4.1 heuristic in grid form):
// each sub-step of duration dt adds dt and removes dt / n_f per visible feature,
// here k = the quality level at the checkpoint.  In units of 2^-24 / (M n_f)
// drift-time the increment is inc * (n_f - k) with inc = cost_q (unit speed) or
// round(T 2^24) (double integrator).
void edge_steps(const Roadmap& rm, const EdgeGeom& g, int64_t cost_q, std::vector<int64_t>& d) {
  d.resize(rm.M);
  int64_t inc = (rm.sc.dim == 6) ? rm.Tq : cost_q;
  for (int m = 1; m <= rm.M; ++m) {
    float p[3];
    checkpoint(rm, g, m, p);
    int k = checkpoint_level(rm, g, m, p);
    d[m - 1] = inc * (int64_t)(rm.sc.n_f - k);
  }
}

// Each step maps h to max(0, h + d_m) (drift is clamped at zero: fully localised).
// Composing the M steps gives F_e(h) = max(C_e, h + S_e) for h >= 0, where
// S_e = sum d_m and C_e = F_e(0).  C_e is obtained here by literally stepping h = 0.
// After m steps the heuristic is max(C_m, h + S_m) with the partial sums S_m and
// the stepped C_m, so its largest value along the edge (the "for all t" form of
// Eq. 2) is max(Cmax, h + Smax) with Smax = max_m S_m and Cmax = max_m C_m.
void transfer_from_steps(const std::vector<int64_t>& d, int64_t& S, int64_t& Cv, int64_t& Smax,
                         int64_t& Cmax) {
  S = 0;
  int64_t h = 0;
  Smax = INT64_MIN;
  Cmax = 0;
  for (int64_t dm : d) {
    S += dm;
    h = h + dm;
    if (h < 0) h = 0;
    Smax = std::max(Smax, S);
    Cmax = std::max(Cmax, h);
  }
  Cv = h;
  if (d.empty()) Smax = 0;
}

void transfer_from_steps(const std::vector<int64_t>& d, int64_t& S, int64_t& Cv) {
  int64_t a, b;
  transfer_from_steps(d, S, Cv, a, b);
}

// ----------------------------------------------------------------------------
// Alg. 2 BuildGraph: N(v) = Near(V \ {v}, v, r_n) minus colliding connections.
// Near uses the strict test Cost(v, u) < r_n.  Edge records are kept in ascending
// neighbour order.
// ----------------------------------------------------------------------------
bool build_graph(Roadmap& rm) {
  rm.row_ptr.assign(rm.V + 1, 0);
  rm.dst.clear(); rm.cost_q.clear(); rm.S.clear(); rm.C.clear(); rm.Smax.clear(); rm.Cmax.clear();
  std::vector<int64_t> d;
  for (uint32_t v = 0; v < rm.V; ++v) {
    for (uint32_t u = 0; u < rm.V; ++u) {
      if (u == v) continue;
      EdgeGeom g = edge_geom(rm, v, u);
      if (!(g.cost < rm.r)) continue;
      if (edge_collides(rm, g)) continue;
      int64_t cq = quantise_cost(g.cost);
      edge_steps(rm, g, cq, d);
      int64_t S, Cv, Smax, Cmax;
      transfer_from_steps(d, S, Cv, Smax, Cmax);
      if (cq > INT32_MAX || S > INT32_MAX || S < INT32_MIN || Cv > INT32_MAX || Smax > INT32_MAX ||
          Cmax > INT32_MAX)
        return false;
      rm.dst.push_back(u);
      rm.cost_q.push_back((int32_t)cq);
      rm.S.push_back((int32_t)S);
      rm.C.push_back((int32_t)Cv);
      rm.Smax.push_back((int32_t)Smax);
      rm.Cmax.push_back((int32_t)Cmax);
    }
    rm.row_ptr[v + 1] = (uint32_t)rm.dst.size();
  }
  return true;
}

// ----------------------------------------------------------------------------
// Alg. 3 Explore.
// ----------------------------------------------------------------------------
struct Plan {
  uint32_t head;
  int64_t parent;        // arena index of the plan this one extends (-1 for the root)
  int64_t cost, h;
  uint32_t iter;         // iteration in which the plan was created
  uint32_t parent_head;  // head of the parent plan (0xFFFFFFFF for the root)
  int64_t parent_cost;
  bool open, alive;
};

// Tie key: plans with identical (cost, h) at one head are ordered by creation
// iteration, then the parent's head, then the parent's cost (older first).
bool key_less(const Plan& a, const Plan& b) {
  if (a.iter != b.iter) return a.iter < b.iter;
  if (a.parent_head != b.parent_head) return a.parent_head < b.parent_head;
  return a.parent_cost < b.parent_cost;
}

// b dominates a (weak Pareto order with a total tie-break).  The paper's literal
// rule is (a.cost > b.cost) and (a.h >= b.h); the weak form additionally removes
// equal-cost plans with a worse or equal h, which keeps every front strictly
// monotone without changing the optimal cost (every transfer F_e is monotone and
// costs add).
bool dominates(const Plan& b, const Plan& a) {
  if (!(b.cost <= a.cost && b.h <= a.h)) return false;
  if (b.cost < a.cost || b.h < a.h) return true;
  return key_less(b, a);
}

struct ExploreOut {
  int status = 0;          // 0 ok, 1 no solution, -4 iteration limit, -2 capacity
  int64_t cost = 0, h = 0;
  std::vector<uint32_t> path;
  uint32_t wavefronts = 0;
  uint64_t expansions = 0;
  uint64_t plans_created = 0;
  std::vector<uint32_t> front_ptr;   // final per-node fronts, sorted by cost
  std::vector<int64_t> front_cost, front_h;
  // P_candidates in solution order, with their node sequences
  std::vector<int64_t> cand_cost, cand_h;
  std::vector<uint32_t> cand_ptr, cand_path;
};

void explore(const Roadmap& rm, int64_t beta, int64_t Lambda, uint32_t max_iters,
             bool goal_termination, uint64_t max_plans, bool check_interior, ExploreOut& out) {
  std::vector<Plan> plans;
  std::vector<std::vector<uint32_t>> P(rm.V);     // P(v): plans with head v
  std::set<uint32_t> open;                        // P_open (arena indices)
  plans.push_back(Plan{0u, -1, 0, 0, 0u, 0xFFFFFFFFu, 0, true, true});
  P[0].push_back(0);
  open.insert(0);
  std::vector<uint32_t> G = {0};                  // B, the group to expand
  int64_t i = 0;
  out.status = 0;
  out.wavefronts = 0;
  out.expansions = 0;

  auto goal_in_group = [&]() {
    for (uint32_t g : G)
      if (rm.is_goal[plans[g].head] && plans[g].h <= beta) return true;
    return false;
  };

  while (!open.empty() && !(goal_termination && goal_in_group())) {
    if (out.wavefronts >= max_iters) { out.status = -4; break; }
    out.wavefronts++;
    std::vector<uint32_t> touched;
    // Expand every plan of the group along every neighbour edge (in parallel in
    // the paper; sequential here).
    for (uint32_t gi : G) {
      const Plan p = plans[gi];
      for (uint32_t e = rm.row_ptr[p.head]; e < rm.row_ptr[p.head + 1]; ++e) {
        out.expansions++;
        uint32_t x = rm.dst[e];
        int64_t qcost = p.cost + (int64_t)rm.cost_q[e];
        // PH(x, p): the transfer of edge p.head -> x applied to p.h.
        int64_t qh = std::max((int64_t)rm.C[e], p.h + (int64_t)rm.S[e]);
        // perception-heuristic cutoff at the new head (Alg. 3), or at every
        // sub-step of the edge (the "for all t" form of Eq. 2)
        const int64_t peak = check_interior ? std::max((int64_t)rm.Cmax[e], p.h + (int64_t)rm.Smax[e]) : qh;
        if (peak <= beta) {
          if (plans.size() >= max_plans) { out.status = -2; return; }
          Plan q{x, (int64_t)gi, qcost, qh, (uint32_t)out.wavefronts, p.head, p.cost,
                 true, true};
          uint32_t qi = (uint32_t)plans.size();
          plans.push_back(q);
          P[x].push_back(qi);
          open.insert(qi);
          touched.push_back(x);
        }
      }
    }
    // RemoveDominated(P, P_open): drop every plan dominated by another plan with
    // the same head, from P_open and from P (closed dominated plans also leave the
    // stored front; their records stay in the arena for back-tracing).
    std::sort(touched.begin(), touched.end());
    touched.erase(std::unique(touched.begin(), touched.end()), touched.end());
    for (uint32_t x : touched) {
      std::vector<uint32_t>& px = P[x];
      std::vector<char> dead(px.size(), 0);
      for (size_t a = 0; a < px.size(); ++a)
        for (size_t b = 0; b < px.size(); ++b)
          if (a != b && dominates(plans[px[b]], plans[px[a]])) { dead[a] = 1; break; }
      std::vector<uint32_t> keep;
      for (size_t a = 0; a < px.size(); ++a) {
        if (dead[a]) {
          plans[px[a]].alive = false;
          plans[px[a]].open = false;
          open.erase(px[a]);
        } else {
          keep.push_back(px[a]);
        }
      }
      px.swap(keep);
    }
    // P_open <- P_open \ B
    for (uint32_t gi : G) {
      plans[gi].open = false;
      open.erase(gi);
    }
    i++;
    // B <- {p in P_open : p.cost <= i lambda r_n}
    G.clear();
    for (uint32_t pi : open)
      if (plans[pi].cost <= i * Lambda) G.push_back(pi);
  }
  out.plans_created = plans.size();

  // Final fronts, per node, sorted by cost.
  out.front_ptr.assign(rm.V + 1, 0);
  out.front_cost.clear(); out.front_h.clear();
  for (uint32_t v = 0; v < rm.V; ++v) {
    std::vector<uint32_t> px = P[v];
    std::sort(px.begin(), px.end(), [&](uint32_t a, uint32_t b) {
      if (plans[a].cost != plans[b].cost) return plans[a].cost < plans[b].cost;
      return plans[a].h < plans[b].h;
    });
    for (uint32_t pi : px) {
      out.front_cost.push_back(plans[pi].cost);
      out.front_h.push_back(plans[pi].h);
    }
    out.front_ptr[v + 1] = (uint32_t)out.front_cost.size();
  }
  if (out.status < 0) return;

  // P_candidates = {p in P(v) : v in X_goal}; return the minimum-cost one (ties:
  // lower h, then the tie key, then the lower head index).
  int64_t best = -1;
  for (uint32_t v = 0; v < rm.V; ++v) {
    if (!rm.is_goal[v]) continue;
    for (uint32_t pi : P[v]) {
      if (best < 0) { best = pi; continue; }
      const Plan& a = plans[pi];
      const Plan& b = plans[best];
      bool better = false;
      if (a.cost != b.cost) better = a.cost < b.cost;
      else if (a.h != b.h) better = a.h < b.h;
      else if (key_less(a, b)) better = true;
      else if (!key_less(b, a)) better = a.head < b.head;
      if (better) best = pi;
    }
  }
  if (best < 0) { out.status = 1; return; }
  // the whole candidate set, sorted by the same rule
  std::vector<uint32_t> cand;
  for (uint32_t v = 0; v < rm.V; ++v)
    if (rm.is_goal[v])
      for (uint32_t pi : P[v]) cand.push_back(pi);
  std::sort(cand.begin(), cand.end(), [&](uint32_t ia, uint32_t ib) {
    const Plan& a = plans[ia];
    const Plan& b = plans[ib];
    if (a.cost != b.cost) return a.cost < b.cost;
    if (a.h != b.h) return a.h < b.h;
    if (key_less(a, b)) return true;
    if (key_less(b, a)) return false;
    return a.head < b.head;
  });
  out.cand_ptr.assign(1, 0);
  for (uint32_t pi : cand) {
    out.cand_cost.push_back(plans[pi].cost);
    out.cand_h.push_back(plans[pi].h);
    std::vector<uint32_t> seq;
    for (int64_t a = pi; a >= 0; a = plans[a].parent) seq.push_back(plans[a].head);
    out.cand_path.insert(out.cand_path.end(), seq.rbegin(), seq.rend());
    out.cand_ptr.push_back((uint32_t)out.cand_path.size());
  }
  out.cost = plans[best].cost;
  out.h = plans[best].h;
  out.path.clear();
  for (int64_t pi = best; pi >= 0; pi = plans[pi].parent) out.path.push_back(plans[pi].head);
  std::reverse(out.path.begin(), out.path.end());
}

// ----------------------------------------------------------------------------
// Monte Carlo certification (Sec. 3 final phase; failure events of Eq. 1 and of
// the robust motion planning statement).  Error model (integer, in 2^-20 units):
// at every checkpoint of the plan, with k the quality level at the nominal state,
//   e <- e - (e >> s_k)          relocalisation contraction (skipped if s_k = 0)
//   e <- e + (sigma_k xi) >> 16  xi = sum of 12 uniform u16 - 6 * 2^16
// clamped to |e_i| <= 2^30.  A rollout fails localisation if e.e >= delta^2 and
// fails robustness (collision) if x_nom + e leaves the unit workspace or enters a
// closed box, at any checkpoint.  Noise comes from Philox with counter
// (rollout, step, call, call_id) and key = seed.
// ----------------------------------------------------------------------------
struct CertOut { uint32_t hits_loc = 0, hits_coll = 0, hits_any = 0, rollouts = 0; };

int certify(const Roadmap& rm, const uint32_t* path, uint32_t path_len, uint32_t rollouts,
            uint64_t seed, uint32_t call_id, int64_t delta_fx, const int32_t* sigma_fx,
            const int32_t* shift, CertOut& out) {
  const Scene& sc = rm.sc;
  const int dp = sc.dp();
  out = CertOut{};
  out.rollouts = rollouts;
  if (path_len < 2) return 0;
  // Nominal checkpoints and their quality levels.
  std::vector<int64_t> nom;     // [steps][3]
  std::vector<int> lev;
  for (uint32_t j = 0; j + 1 < path_len; ++j) {
    EdgeGeom g = edge_geom(rm, path[j], path[j + 1]);
    for (int m = 1; m <= rm.M; ++m) {
      float p[3];
      checkpoint(rm, g, m, p);
      for (int i = 0; i < 3; ++i) nom.push_back((int64_t)llrintf(p[i] * kTwo20));
      lev.push_back(checkpoint_level(rm, g, m, p));
    }
  }
  const uint32_t steps = (uint32_t)lev.size();
  std::vector<int64_t> blo(3 * sc.nb), bhi(3 * sc.nb);
  for (int b = 0; b < 3 * sc.nb; ++b) {
    blo[b] = (int64_t)llrintf(sc.lo[b] * kTwo20);
    bhi[b] = (int64_t)llrintf(sc.hi[b] * kTwo20);
  }
  const int64_t lim = (int64_t)1 << 30;
  const int64_t one = (int64_t)1 << 20;
  const int64_t delta2 = delta_fx * delta_fx;
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (uint32_t ro = 0; ro < rollouts; ++ro) {
    int64_t e[3] = {0, 0, 0};
    bool loc = false, coll = false;
    for (uint32_t s = 0; s < steps && !(loc && coll); ++s) {
      int k = lev[s];
      if (shift[k] > 0)
        for (int i = 0; i < dp; ++i) e[i] -= (e[i] >> shift[k]);
      uint32_t words[20];
      for (uint32_t c = 0; c < 5; ++c) {
        uint32_t ctr[4] = {ro, s, c, call_id};
        philox4x32_10(ctr, key, words + 4 * c);
      }
      for (int i = 0; i < dp; ++i) {
        int64_t xi = 0;
        for (int j = 0; j < 12; ++j) {
          int idx = 12 * i + j;                        // u16 index: low half first
          uint32_t w = words[idx >> 1];
          xi += (idx & 1) ? (int64_t)(w >> 16) : (int64_t)(w & 0xFFFFu);
        }
        xi -= 6 * 65536;
        e[i] += ((int64_t)sigma_fx[k] * xi) >> 16;
        if (e[i] > lim) e[i] = lim;
        if (e[i] < -lim) e[i] = -lim;
      }
      int64_t ee = 0;
      for (int i = 0; i < dp; ++i) ee += e[i] * e[i];
      if (ee >= delta2) loc = true;
      int64_t q[3];
      bool out_ws = false;
      for (int i = 0; i < dp; ++i) {
        q[i] = nom[3 * s + i] + e[i];
        if (q[i] < 0 || q[i] > one) out_ws = true;
      }
      bool in_box = false;
      for (int b = 0; b < sc.nb && !in_box; ++b) {
        bool inside = true;
        for (int i = 0; i < dp; ++i)
          if (q[i] < blo[3 * b + i] || q[i] > bhi[3 * b + i]) { inside = false; break; }
        in_box = inside;
      }
      if (out_ws || in_box) coll = true;
    }
    out.hits_loc += loc;
    out.hits_coll += coll;
    out.hits_any += (loc || coll);
  }
  return 0;
}

// ----------------------------------------------------------------------------
// Closed-loop VIO Monte Carlo model (Sec. 4.1: the nominal trajectory is tracked
// by an LQR controller; the state estimate fuses an inertial prediction from a
// noisy accelerometer with position fixes from the features in view through a
// Kalman filter).  The paper gives no parameters; every quantity below is this
// build's reading.  Per position axis, in 2^-20 units and per checkpoint step:
// true deviation (p, w) from the nominal (w = velocity x step) and estimation
// error (ep, ew) = estimate - truth.  At checkpoint s with quality level k:
//   a  = -round((kp (p + ep) + kv (w + ew)) / 2^16)   LQR control from the estimate
//   p += w + (a >> 1);  w += a                          the executed deviation
//   na = (q_a xi1) >> 16;  ep += ew + (na >> 1);  ew += na     inertial prediction
//   if r_k > 0:  nu = (r_k xi2) >> 16;  t = nu - ep;
//                ep += round(Lp_s t / 2^16);  ew += round(Lw_s t / 2^16)   position fix
// all clamped to |x| <= 2^30; round(x / 2^16) = (x + 2^15) >> 16.  (Lp_s, Lw_s)
// are the Kalman gains of step s from the covariance recursion in double (P_0 = 0;
// prediction A P A^T + q_a^2 B B^T with A = [1 1; 0 1], B = (1/2, 1); update
// with measurement noise r_k^2 when r_k > 0), quantised to Q16.  xi1, xi2 are
// the Irwin-Hall normals of certify(): axis i takes u16 words 24 i .. 24 i + 11
// and 24 i + 12 .. 24 i + 23 of Philox with counter (rollout, step, call, call_id),
// calls 0 .. ceil(3 dp) - 1.  Failures as in certify(): |ep| >= delta
// (localisation, Eq. 1) and the executed position nom + p outside the map or in a
// closed box (the robust problem).
// ----------------------------------------------------------------------------
void vio_gains(const std::vector<int>& lev, int32_t q_a, const int32_t* r_fx, std::vector<int32_t>& Lp,
               std::vector<int32_t>& Lw, std::vector<double>& P00) {
  double p00 = 0.0, p01 = 0.0, p11 = 0.0;
  const double q2 = (double)q_a * (double)q_a;
  const size_t n = lev.size();
  Lp.assign(n, 0);
  Lw.assign(n, 0);
  P00.assign(n, 0.0);
  for (size_t s = 0; s < n; ++s) {
    const double a00 = p00 + 2.0 * p01 + p11 + 0.25 * q2;
    const double a01 = p01 + p11 + 0.5 * q2;
    const double a11 = p11 + q2;
    const int32_t r = r_fx[lev[s]];
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
    Lp[s] = (int32_t)llrint(lp * 65536.0);
    Lw[s] = (int32_t)llrint(lw * 65536.0);
    P00[s] = p00;
  }
}

static inline int64_t clamp30(int64_t x) {
  const int64_t lim = (int64_t)1 << 30;
  return x > lim ? lim : (x < -lim ? -lim : x);
}

static inline int64_t round16(int64_t x) { return (x + 32768) >> 16; }

int certify_vio(const Roadmap& rm, const uint32_t* path, uint32_t path_len, uint32_t rollouts, uint64_t seed,
                uint32_t call_id, int64_t delta_fx, int32_t q_a, int32_t kp, int32_t kv, const int32_t* r_fx,
                CertOut& out, int64_t* ep_last, int32_t* gains, double* p00_out) {
  const Scene& sc = rm.sc;
  const int dp = sc.dp();
  out = CertOut{};
  out.rollouts = rollouts;
  if (path_len < 2) return 0;
  std::vector<int64_t> nom;
  std::vector<int> lev;
  for (uint32_t j = 0; j + 1 < path_len; ++j) {
    EdgeGeom g = edge_geom(rm, path[j], path[j + 1]);
    for (int m = 1; m <= rm.M; ++m) {
      float p[3];
      checkpoint(rm, g, m, p);
      for (int i = 0; i < 3; ++i) nom.push_back((int64_t)llrintf(p[i] * kTwo20));
      lev.push_back(checkpoint_level(rm, g, m, p));
    }
  }
  const uint32_t steps = (uint32_t)lev.size();
  std::vector<int32_t> Lp, Lw;
  std::vector<double> P00;
  vio_gains(lev, q_a, r_fx, Lp, Lw, P00);
  if (gains)
    for (uint32_t s = 0; s < steps; ++s) {
      gains[2 * s] = Lp[s];
      gains[2 * s + 1] = Lw[s];
    }
  if (p00_out)
    for (uint32_t s = 0; s < steps; ++s) p00_out[s] = P00[s];
  std::vector<int64_t> blo(3 * sc.nb), bhi(3 * sc.nb);
  for (int b = 0; b < 3 * sc.nb; ++b) {
    blo[b] = (int64_t)llrintf(sc.lo[b] * kTwo20);
    bhi[b] = (int64_t)llrintf(sc.hi[b] * kTwo20);
  }
  const int64_t one = (int64_t)1 << 20;
  const int64_t delta2 = delta_fx * delta_fx;
  const uint32_t ncalls = (uint32_t)(24 * dp + 7) / 8;
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (uint32_t ro = 0; ro < rollouts; ++ro) {
    int64_t p[3] = {0, 0, 0}, w[3] = {0, 0, 0}, ep[3] = {0, 0, 0}, ew[3] = {0, 0, 0};
    bool loc = false, coll = false;
    for (uint32_t s = 0; s < steps; ++s) {
      const int k = lev[s];
      uint32_t words[36];
      for (uint32_t c = 0; c < ncalls; ++c) {
        uint32_t ctr[4] = {ro, s, c, call_id};
        philox4x32_10(ctr, key, words + 4 * c);
      }
      auto normal = [&](int first) {
        int64_t xi = 0;
        for (int j = 0; j < 12; ++j) {
          const int idx = first + j;
          const uint32_t wd = words[idx >> 1];
          xi += (idx & 1) ? (int64_t)(wd >> 16) : (int64_t)(wd & 0xFFFFu);
        }
        return xi - 6 * 65536;
      };
      for (int i = 0; i < dp; ++i) {
        const int64_t a = -round16((int64_t)kp * (p[i] + ep[i]) + (int64_t)kv * (w[i] + ew[i]));
        p[i] = clamp30(p[i] + w[i] + (a >> 1));
        w[i] = clamp30(w[i] + a);
        const int64_t na = ((int64_t)q_a * normal(24 * i)) >> 16;
        ep[i] = clamp30(ep[i] + ew[i] + (na >> 1));
        ew[i] = clamp30(ew[i] + na);
        if (r_fx[k] > 0) {
          const int64_t nu = ((int64_t)r_fx[k] * normal(24 * i + 12)) >> 16;
          const int64_t t = nu - ep[i];
          ep[i] = clamp30(ep[i] + round16((int64_t)Lp[s] * t));
          ew[i] = clamp30(ew[i] + round16((int64_t)Lw[s] * t));
        }
      }
      int64_t ee = 0;
      for (int i = 0; i < dp; ++i) ee += ep[i] * ep[i];
      if (ee >= delta2) loc = true;
      int64_t q[3];
      bool out_ws = false;
      for (int i = 0; i < dp; ++i) {
        q[i] = nom[3 * s + i] + p[i];
        if (q[i] < 0 || q[i] > one) out_ws = true;
      }
      bool in_box = false;
      for (int b = 0; b < sc.nb && !in_box; ++b) {
        bool inside = true;
        for (int i = 0; i < dp; ++i)
          if (q[i] < blo[3 * b + i] || q[i] > bhi[3 * b + i]) { inside = false; break; }
        in_box = inside;
      }
      if (out_ws || in_box) coll = true;
    }
    if (ep_last) {
      ep_last[2 * (size_t)ro] = ep[0];
      ep_last[2 * (size_t)ro + 1] = p[0];
    }
    out.hits_loc += loc;
    out.hits_coll += coll;
    out.hits_any += (loc || coll);
  }
  return 0;
}

// ----------------------------------------------------------------------------
// Trajectory features of a plan (input of the certification surrogate, which is
// not in the paper).  The plan's Monte Carlo checkpoints s = 0 .. steps-1 (the M
// sub-steps of every edge, exactly as certify() visits them) are split into 16
// bins, s going to bin floor(16 s / steps).  For bin j: the maximum quality level
// / K, the sum of levels / (64 K), and 4 min(0.25, clearance), where the clearance
// of p is the smallest of the signed max-norm distances to the boxes
// (max_i max(lo_i - p_i, p_i - hi_i), negative inside) and of the distances to the
// walls of the unit map (min_i min(p_i, 1 - p_i)).  An empty bin gives 0, 0, 1.
// ----------------------------------------------------------------------------
void plan_features(const Roadmap& rm, const uint32_t* path, uint32_t len, float* f) {
  const Scene& sc = rm.sc;
  const int dp = sc.dp();
  std::vector<int> lev;
  std::vector<float> clr;
  for (uint32_t j = 0; j + 1 < len; ++j) {
    EdgeGeom g = edge_geom(rm, path[j], path[j + 1]);
    for (int m = 1; m <= rm.M; ++m) {
      float p[3];
      checkpoint(rm, g, m, p);
      int k = checkpoint_level(rm, g, m, p);
      lev.push_back(k > sc.K ? sc.K : k);
      float c = INFINITY;
      for (int i = 0; i < dp; ++i) c = std::fmin(c, std::fmin(p[i], 1.0f - p[i]));
      for (int b = 0; b < sc.nb; ++b) {
        float d = -INFINITY;
        for (int i = 0; i < dp; ++i)
          d = std::fmax(d, std::fmax(sc.lo[3 * b + i] - p[i], p[i] - sc.hi[3 * b + i]));
        c = std::fmin(c, d);
      }
      clr.push_back(c);
    }
  }
  const uint64_t steps = lev.size();
  const float Kf = (float)(sc.K > 0 ? sc.K : 1);
  for (int j = 0; j < 16; ++j) {
    int lmax = 0;
    uint32_t lsum = 0;
    float cmin = INFINITY;
    bool any = false;
    for (uint64_t s = 0; s < steps; ++s) {
      if ((16 * s) / steps != (uint64_t)j) continue;
      any = true;
      lmax = std::max(lmax, lev[s]);
      lsum += (uint32_t)lev[s];
      cmin = std::fmin(cmin, clr[s]);
    }
    f[j] = any ? (float)lmax / Kf : 0.0f;
    f[16 + j] = any ? (float)lsum / (64.0f * Kf) : 0.0f;
    f[32 + j] = any ? 4.0f * std::fmin(0.25f, cmin) : 1.0f;
  }
}

void set_heading(Scene& sc, int Y, const uint8_t* head) {
  sc.Y = Y > 0 ? Y : 0;
  if (sc.Y) {
    const size_t cells = (sc.dim == 2) ? (size_t)sc.G * sc.G : (size_t)sc.G * sc.G * sc.G;
    sc.head.assign(head, head + (size_t)sc.Y * cells);
  }
}

Scene make_scene(int dim, int nb, const float* lo, const float* hi, int G,
                 const uint8_t* level, int n_f, int K) {
  Scene sc;
  sc.dim = dim;
  sc.nb = nb;
  sc.lo.assign(lo, lo + 3 * nb);
  sc.hi.assign(hi, hi + 3 * nb);
  sc.G = G;
  size_t cells = (dim == 2) ? (size_t)G * G : (size_t)G * G * G;
  sc.level.assign(level, level + cells);
  sc.n_f = n_f;
  sc.K = K;
  return sc;
}

}  // namespace

// ============================================================================
// C interface used by the Python test harness (ctypes).
// ============================================================================
extern "C" {

struct orc_roadmap { Roadmap rm; };
struct orc_result { ExploreOut out; };

void orc_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  philox4x32_10(ctr, key, out);
}

// Build V = {x_init, x_goal} + SampleFree(n) and the r-disc graph (Alg. 2).
// Returns null on failure (sampling budget exhausted or an edge field overflowing
// int32).
orc_roadmap* orc_build_roadmap_heading(int dim, int nb, const float* lo, const float* hi, int G,
                                       const uint8_t* level, int n_f, int K, uint32_t n,
                                       uint64_t seed, uint32_t query_id, float r, float T, int M,
                                       const float* x_init, const float* x_goal, float goal_radius,
                                       int Y, const uint8_t* head) {
  orc_roadmap* h = new orc_roadmap();
  Roadmap& rm = h->rm;
  rm.sc = make_scene(dim, nb, lo, hi, G, level, n_f, K);
  set_heading(rm.sc, Y, head);
  rm.r = r; rm.T = T; rm.M = M; rm.goal_radius = goal_radius;
  set_di6_constants(rm);
  if (!sample_free(rm, n, seed, query_id, x_init, x_goal)) { delete h; return nullptr; }
  mark_goal(rm);
  if (!build_graph(rm)) { delete h; return nullptr; }
  return h;
}

orc_roadmap* orc_build_roadmap(int dim, int nb, const float* lo, const float* hi, int G,
                               const uint8_t* level, int n_f, int K, uint32_t n,
                               uint64_t seed, uint32_t query_id, float r, float T, int M,
                               const float* x_init, const float* x_goal, float goal_radius) {
  orc_roadmap* h = new orc_roadmap();
  Roadmap& rm = h->rm;
  rm.sc = make_scene(dim, nb, lo, hi, G, level, n_f, K);
  rm.r = r; rm.T = T; rm.M = M; rm.goal_radius = goal_radius;
  set_di6_constants(rm);
  if (!sample_free(rm, n, seed, query_id, x_init, x_goal)) { delete h; return nullptr; }
  mark_goal(rm);
  if (!build_graph(rm)) { delete h; return nullptr; }
  return h;
}

// Same graph construction on caller-given node states (x: [6][V] SoA) and, in the
// camera-heading form, yaws (yaw: [V], NULL for all zero).
orc_roadmap* orc_build_roadmap_from_points_heading(int dim, int nb, const float* lo, const float* hi,
                                                   int G, const uint8_t* level, int n_f, int K,
                                                   uint32_t V, const float* x, float r, float T, int M,
                                                   float goal_radius, int Y, const uint8_t* head,
                                                   const float* yaw) {
  orc_roadmap* h = new orc_roadmap();
  Roadmap& rm = h->rm;
  rm.sc = make_scene(dim, nb, lo, hi, G, level, n_f, K);
  set_heading(rm.sc, Y, head);
  rm.r = r; rm.T = T; rm.M = M; rm.goal_radius = goal_radius;
  set_di6_constants(rm);
  rm.V = V;
  for (int a = 0; a < 6; ++a) rm.x[a].assign(x + (size_t)a * V, x + (size_t)(a + 1) * V);
  if (Y > 0) {
    if (yaw) rm.yaw.assign(yaw, yaw + V);
    else rm.yaw.assign(V, 0.0f);
  }
  mark_goal(rm);
  if (!build_graph(rm)) { delete h; return nullptr; }
  return h;
}

orc_roadmap* orc_build_roadmap_from_points(int dim, int nb, const float* lo, const float* hi,
                                           int G, const uint8_t* level, int n_f, int K,
                                           uint32_t V, const float* x, float r, float T, int M,
                                           float goal_radius) {
  orc_roadmap* h = new orc_roadmap();
  Roadmap& rm = h->rm;
  rm.sc = make_scene(dim, nb, lo, hi, G, level, n_f, K);
  rm.r = r; rm.T = T; rm.M = M; rm.goal_radius = goal_radius;
  set_di6_constants(rm);
  rm.V = V;
  for (int a = 0; a < 6; ++a) rm.x[a].assign(x + (size_t)a * V, x + (size_t)(a + 1) * V);
  mark_goal(rm);
  if (!build_graph(rm)) { delete h; return nullptr; }
  return h;
}

// A roadmap given directly as a CSR graph (for hand-made search cases); no geometry.
orc_roadmap* orc_roadmap_from_csr(uint32_t V, const uint32_t* row_ptr, const uint32_t* dst,
                                  const int32_t* cost_q, const int32_t* S, const int32_t* C,
                                  const uint8_t* is_goal) {
  orc_roadmap* h = new orc_roadmap();
  Roadmap& rm = h->rm;
  rm.V = V;
  rm.row_ptr.assign(row_ptr, row_ptr + V + 1);
  uint32_t E = row_ptr[V];
  rm.dst.assign(dst, dst + E);
  rm.cost_q.assign(cost_q, cost_q + E);
  rm.S.assign(S, S + E);
  rm.C.assign(C, C + E);
  // without peaks an edge is one step: its peak is its end value
  rm.Smax.assign(S, S + E);
  rm.Cmax.assign(C, C + E);
  rm.is_goal.assign(is_goal, is_goal + V);
  for (int a = 0; a < 6; ++a) rm.x[a].assign(V, 0.0f);
  return h;
}

// The same with the per-edge peaks (Smax, Cmax) of the transfers.
orc_roadmap* orc_roadmap_from_csr_peaks(uint32_t V, const uint32_t* row_ptr, const uint32_t* dst,
                                        const int32_t* cost_q, const int32_t* S, const int32_t* C,
                                        const int32_t* Smax, const int32_t* Cmax, const uint8_t* is_goal) {
  orc_roadmap* h = orc_roadmap_from_csr(V, row_ptr, dst, cost_q, S, C, is_goal);
  const uint32_t E = row_ptr[V];
  h->rm.Smax.assign(Smax, Smax + E);
  h->rm.Cmax.assign(Cmax, Cmax + E);
  return h;
}

void orc_roadmap_get_peaks(const orc_roadmap* h, int32_t* Smax, int32_t* Cmax) {
  const Roadmap& rm = h->rm;
  if (Smax) std::memcpy(Smax, rm.Smax.data(), rm.Smax.size() * 4);
  if (Cmax) std::memcpy(Cmax, rm.Cmax.data(), rm.Cmax.size() * 4);
}

void orc_roadmap_free(orc_roadmap* h) { delete h; }
uint32_t orc_roadmap_V(const orc_roadmap* h) { return h->rm.V; }
uint32_t orc_roadmap_E(const orc_roadmap* h) { return (uint32_t)h->rm.dst.size(); }

void orc_roadmap_get(const orc_roadmap* h, float* x, uint8_t* is_goal, uint32_t* row_ptr,
                     uint32_t* dst, int32_t* cost_q, int32_t* S, int32_t* C) {
  const Roadmap& rm = h->rm;
  if (x) for (int a = 0; a < 6; ++a) std::memcpy(x + (size_t)a * rm.V, rm.x[a].data(), rm.V * 4);
  if (is_goal) std::memcpy(is_goal, rm.is_goal.data(), rm.V);
  if (row_ptr) std::memcpy(row_ptr, rm.row_ptr.data(), (rm.V + 1) * 4);
  size_t E = rm.dst.size();
  if (dst) std::memcpy(dst, rm.dst.data(), E * 4);
  if (cost_q) std::memcpy(cost_q, rm.cost_q.data(), E * 4);
  if (S) std::memcpy(S, rm.S.data(), E * 4);
  if (C) std::memcpy(C, rm.C.data(), E * 4);
}

// Geometry of one connection u -> v: cost, control energy J (6D), the M checkpoint
// positions [M][3], the per-step heuristic increments [M], and (6D) the
// coefficients a0[3], jerk[3].  Returns 1 if the connection collides.
int orc_edge_eval(const orc_roadmap* h, uint32_t u, uint32_t v, float* cost, float* J,
                  float* ckpt, int64_t* d, float* a0, float* jerk) {
  const Roadmap& rm = h->rm;
  EdgeGeom g = edge_geom(rm, u, v);
  if (cost) *cost = g.cost;
  if (J) *J = g.J;
  if (ckpt)
    for (int m = 1; m <= rm.M; ++m) checkpoint(rm, g, m, ckpt + 3 * (m - 1));
  if (d) {
    std::vector<int64_t> dd;
    edge_steps(rm, g, quantise_cost(g.cost), dd);
    for (int m = 0; m < rm.M; ++m) d[m] = dd[m];
  }
  if (a0) for (int i = 0; i < 3; ++i) a0[i] = g.a0[i];
  if (jerk) for (int i = 0; i < 3; ++i) jerk[i] = g.jk[i];
  return edge_collides(rm, g) ? 1 : 0;
}

// Segment-vs-box test on explicit float data (for the slab-test pins).
int orc_segment_hits_box(int dp, const float* a, const float* b, const float* lo,
                         const float* hi) {
  Scene sc;
  sc.dim = dp;
  sc.nb = 1;
  sc.lo.assign(lo, lo + 3);
  sc.hi.assign(hi, hi + 3);
  float aa[3] = {a[0], a[1], dp == 3 ? a[2] : 0.0f};
  float d[3] = {b[0] - a[0], b[1] - a[1], dp == 3 ? b[2] - a[2] : 0.0f};
  return segment_hits_box(sc, 0, aa, d) ? 1 : 0;
}

// Perception levels from mapped features (the visible-feature count behind the
// Sec. 4.1 heuristic).  For yaw bin y with horizontal heading (hx, hy) and the
// centre c = ((2i + 1) / (2G), ...) of grid cell (i, j[, k]), the level is the
// number of features f, capped at K, with
//   |f - c|^2 <= range^2                      (in range),
//   hx dx + hy dy >= cos_half sqrt(dx^2 + dy^2)   (inside the horizontal field of
//                                              view; d = f - c),
//   and the closed segment c -> f meeting no closed box (unoccluded).
// Every float operation is written out in order; division and square root are
// the IEEE ones.  out: [Y][G^Dp] (x fastest).
void orc_feature_levels(int dp, int nb, const float* lo, const float* hi, int nf, const float* feat, int G,
                        int Y, const float* head, float cos_half, float range, int K, uint8_t* out) {
  Scene sc;
  sc.dim = dp;
  sc.nb = nb;
  sc.lo.assign(lo, lo + 3 * nb);
  sc.hi.assign(hi, hi + 3 * nb);
  const float half = 0.5f / (float)G;
  const float range2 = range * range;
  const size_t cells = (size_t)G * G * (dp == 3 ? G : 1);
  for (int y = 0; y < Y; ++y) {
    const float hx = head[2 * y], hy = head[2 * y + 1];
    for (size_t cell = 0; cell < cells; ++cell) {
      const size_t i = cell % G, j = (cell / G) % G, k = (dp == 3) ? cell / ((size_t)G * G) : 0;
      const float c[3] = {(float)(2 * i + 1) * half, (float)(2 * j + 1) * half,
                          dp == 3 ? (float)(2 * k + 1) * half : 0.0f};
      int count = 0;
      for (int f = 0; f < nf; ++f) {
        float d[3];
        d[0] = feat[3 * f] - c[0];
        d[1] = feat[3 * f + 1] - c[1];
        d[2] = (dp == 3) ? feat[3 * f + 2] - c[2] : 0.0f;
        float dxy2 = d[0] * d[0];
        dxy2 = dxy2 + d[1] * d[1];
        float r2 = dxy2;
        if (dp == 3) r2 = r2 + d[2] * d[2];
        if (r2 > range2) continue;
        float dot = hx * d[0];
        dot = dot + hy * d[1];
        if (dot < cos_half * std::sqrt(dxy2)) continue;
        bool blocked = false;
        for (int b = 0; b < nb && !blocked; ++b) blocked = segment_hits_box(sc, b, c, d);
        if (!blocked) ++count;
      }
      out[(size_t)y * cells + cell] = (uint8_t)(count < K ? count : K);
    }
  }
}

orc_result* orc_explore(const orc_roadmap* h, int64_t beta, int64_t Lambda, uint32_t max_iters,
                        int goal_termination, uint64_t max_plans, int check_interior) {
  orc_result* r = new orc_result();
  explore(h->rm, beta, Lambda, max_iters, goal_termination != 0, max_plans, check_interior != 0, r->out);
  return r;
}

void orc_result_free(orc_result* r) { delete r; }

void orc_result_summary(const orc_result* r, int* status, int64_t* cost, int64_t* hval,
                        uint32_t* path_len, uint32_t* wavefronts, uint64_t* expansions,
                        uint64_t* plans_created, uint32_t* front_total) {
  const ExploreOut& o = r->out;
  *status = o.status;
  *cost = o.cost;
  *hval = o.h;
  *path_len = (uint32_t)o.path.size();
  *wavefronts = o.wavefronts;
  *expansions = o.expansions;
  *plans_created = o.plans_created;
  *front_total = (uint32_t)o.front_cost.size();
}

void orc_result_get(const orc_result* r, uint32_t* path, uint32_t* front_ptr,
                    int64_t* front_cost, int64_t* front_h) {
  const ExploreOut& o = r->out;
  if (path) std::memcpy(path, o.path.data(), o.path.size() * 4);
  if (front_ptr) std::memcpy(front_ptr, o.front_ptr.data(), o.front_ptr.size() * 4);
  if (front_cost) std::memcpy(front_cost, o.front_cost.data(), o.front_cost.size() * 8);
  if (front_h) std::memcpy(front_h, o.front_h.data(), o.front_h.size() * 8);
}

// P_candidates of an explore result: up to cap candidates (cost, h, node
// sequences packed as path[ptr[i] .. ptr[i+1])); returns the total count, or -1 if
// the paths need more than path_cap entries.
int orc_result_candidates(const orc_result* r, uint32_t cap, int64_t* cost, int64_t* hval,
                          uint32_t* ptr, uint32_t* path, uint32_t path_cap, uint32_t* n) {
  const ExploreOut& o = r->out;
  const uint32_t total = (uint32_t)o.cand_cost.size();
  const uint32_t k = std::min(cap, total);
  *n = k;
  if (k == 0) return (int)total;
  if (o.cand_ptr[k] > path_cap) return -1;
  for (uint32_t i = 0; i < k; ++i) {
    cost[i] = o.cand_cost[i];
    hval[i] = o.cand_h[i];
  }
  std::memcpy(ptr, o.cand_ptr.data(), 4 * ((size_t)k + 1));
  std::memcpy(path, o.cand_path.data(), 4 * (size_t)o.cand_ptr[k]);
  return (int)total;
}

void orc_plan_features(const orc_roadmap* h, uint32_t n, const uint32_t* ptr, const uint32_t* path,
                       float* feat) {
  for (uint32_t i = 0; i < n; ++i)
    plan_features(h->rm, path + ptr[i], ptr[i + 1] - ptr[i], feat + 48 * (size_t)i);
}

int orc_certify(const orc_roadmap* h, const uint32_t* path, uint32_t path_len, uint32_t rollouts,
                uint64_t seed, uint32_t call_id, int64_t delta_fx, const int32_t* sigma_fx,
                const int32_t* shift, uint32_t* hits /* loc, coll, any, rollouts */) {
  CertOut c;
  int rc = certify(h->rm, path, path_len, rollouts, seed, call_id, delta_fx, sigma_fx, shift, c);
  hits[0] = c.hits_loc;
  hits[1] = c.hits_coll;
  hits[2] = c.hits_any;
  hits[3] = c.rollouts;
  return rc;
}

int orc_certify_vio(const orc_roadmap* h, const uint32_t* path, uint32_t path_len, uint32_t rollouts,
                    uint64_t seed, uint32_t call_id, int64_t delta_fx, int32_t q_a, int32_t kp, int32_t kv,
                    const int32_t* r_fx, uint32_t* hits, int64_t* ep_last, int32_t* gains, double* p00) {
  CertOut c;
  int rc = certify_vio(h->rm, path, path_len, rollouts, seed, call_id, delta_fx, q_a, kp, kv, r_fx, c, ep_last,
                       gains, p00);
  hits[0] = c.hits_loc;
  hits[1] = c.hits_coll;
  hits[2] = c.hits_any;
  hits[3] = c.rollouts;
  return rc;
}

void orc_roadmap_yaw(const orc_roadmap* h, float* out) {
  const Roadmap& rm = h->rm;
  for (uint32_t v = 0; v < rm.V; ++v) out[v] = rm.yaw.empty() ? 0.0f : rm.yaw[v];
}

// Straight-line heuristic from node 0 to every node: F_{x_init -> v}(0) for the
// straight segment at unit speed with M checkpoints (positions only).  Used to set
// the perception bound beta as a percentile.
void orc_straight_line_h(const orc_roadmap* h, int64_t* out) {
  const Roadmap& rm = h->rm;
  Roadmap lin = rm;
  lin.sc.dim = (rm.sc.dim == 2) ? 2 : 3;
  std::vector<int64_t> d;
  for (uint32_t v = 0; v < rm.V; ++v) {
    if (v == 0) { out[v] = 0; continue; }
    EdgeGeom g = edge_geom(lin, 0, v);
    edge_steps(lin, g, quantise_cost(g.cost), d);
    int64_t S, Cv;
    transfer_from_steps(d, S, Cv);
    out[v] = Cv;
  }
}

}  // extern "C"
