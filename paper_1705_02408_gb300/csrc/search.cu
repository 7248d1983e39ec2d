// Wavefront multiobjective search: Alg. 3 (Explore) of Ichter et al., with
// RemoveDominated (Sec. 3) and the perception-heuristic cutoff h <= beta.
//
// The whole loop of Alg. 3 is one persistent kernel, k_wave, launched
// cooperatively (every block resident) over all queries of a batch.  Per
// wavefront i it runs two phases separated by grid barriers:
//   expand  one warp per node u with open plans: the group B_i of u (its open
//           plans with cost <= i Lambda, a cost-ordered part of its front) is
//           closed (P_open <- P_open \ B) and expanded along every out-edge
//           u -> x: q = (cost + cost_q, max(C, h + S)) (PH(x, p) of Sec. 3), cut
//           at beta.  A candidate that the stored front of x, or the previous
//           candidate of the same source along the same edge, already dominates
//           is dropped here (the front of x does not change during this phase);
//           the rest go to the candidate slots of x.  Small groups put the lanes
//           on the out-edges, large ones on the group plans.
//   merge   one warp per node x that received candidates: an exact skyline merge
//           of the candidates into the stored front under the weak Pareto order
//           with the total tie key (creation iteration, parent head): old plans
//           win ties, candidates tie-break by parent head.  Candidates are merged
//           in chunks of 32 (warp bitonic sort, prefix minimum, rank merge);
//           fronts of up to 32 entries stay in registers, larger ones are merged
//           between the node's two pool blocks.  New plans get arena records.
// The last block to reach the barrier after the merge ends the wavefront: per
// query it applies the loop condition of Alg. 3 (a goal plan in the next group,
// P_open empty, the iteration cap) and advances the iteration.  Every barrier
// wait is bounded in %globaltimer time; a wait that runs out ends the kernel
// with MPAP_ERR_TIMEOUT instead of hanging.
//
// HBM layout (NV = nodes summed over the batch):
//   fronts   a pool of {cost i64, h i64, ref u32 (arena | open | new), aux u32}
//            entries; every node owns two blocks of it (live front, merge
//            target), of power-of-two sizes from 16 up, taken from the pool with
//            one atomic add and replaced by a block twice the needed size when
//            too small (the old block is abandoned: at most as much again)
//   fdesc    [NV] {live block, count, other block, log2 sizes}
//   slots    [NV][64] candidates of the current wavefront {cost, h, parent, tie}
//            (32 B), count per node; more than 64 go to an overflow area in
//            arrival order and are regrouped per node before the merge
//   group    [cap] {cost, h, ref}: groups of more than 32 plans
//   arena    [cap] {head u32, parent u32, iter u32, cost i64} for back-tracing
#include <algorithm>
#include <climits>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "internal.h"
#include "profile.h"

namespace mpap {

constexpr uint32_t kSlots = 64;          // inline candidate slots per node and wavefront
constexpr uint32_t kDefaultWaitUs = 20000000;  // barrier wait limit when no query sets one
constexpr uint32_t kHugeMax = 8192;       // grid-wide merges per wavefront (further nodes: one warp each)
constexpr uint32_t kTile = 1024;          // cost buckets per warp tile of the grid-wide merge

struct QueryDev {
  const uint32_t* fwd_ptr;
  const int4* fwd_edge;     // per out-edge {dst, cost_q, S, C}
  const int2* fwd_peak;     // per out-edge {Smax, Cmax} (interior check)
  const uint8_t* is_goal;
  const uint32_t* goal_list;
  uint32_t n_goal;
  uint32_t V;
  uint32_t base;
  uint32_t max_iters;
  uint32_t flags;
  uint32_t pad;
  int64_t beta;
  int64_t Lambda;
  uint64_t pool_base;       // this query's share of the front pool: [base, base + cap)
  uint64_t pool_cap;
  uint64_t ov_base;         // and of the candidate overflow areas
  uint64_t ov_cap;
  uint64_t arena_base;      // and of the plan arena
  uint64_t arena_cap;
};

struct QueryState {
  long long open_cnt;
  unsigned long long expansions;
  unsigned long long plans;
  uint32_t wavefronts;
  uint32_t goal_hit;
  uint32_t done;
  int32_t status;
  uint32_t err;          // capacity error bits of this query (pool, arena, group, overflow)
  uint32_t goal_next;    // a goal node holds an open plan of the next group
  unsigned long long pool_n;  // entries of its pool share handed out
  uint32_t ov_n;         // candidates in its overflow share this wavefront
  uint32_t seg_n;        // entries of its regrouped overflow share handed out
  unsigned long long arena_n;  // records of its arena share handed out
};

struct ResultDev {
  long long cost;
  long long h;
  uint32_t path_len;
  int32_t status;
};

// A candidate in a slot (32 B): the plan it would be and, in the overflow area,
// its node and its index among the node's candidates.
struct __align__(16) Cand {
  long long cost;
  long long h;
  uint32_t pp;    // parent plan (arena index)
  uint32_t tb;    // tie key: 1 + parent head
  uint32_t g;     // node (overflow records)
  uint32_t i;     // index - kSlots among the node's candidates (overflow records)
};

// A node's front descriptor (32 B, one sector): its live block, count, other
// block and block sizes, and a copy of its last entry (highest cost, lowest h),
// which alone dominates most candidates that reach the node.
struct __align__(32) FDesc {
  uint4 d;          // {live block, count, other block, lg live | lg other << 8}
  longlong2 last;   // {cost, h} of entry count - 1 (count > 0)
};

struct Ctl {
  uint32_t oh_n[2];
  uint32_t m_n;          // nodes with candidates this wavefront
  uint32_t g_n;          // group array entries handed out this wavefront
  uint32_t err;
  uint32_t n_done;
  uint32_t it;           // current wavefront
  uint32_t nq;
  uint32_t iter_cap;     // loop bound (max over queries of max_iters, plus 2)
  uint32_t max_front;    // largest front committed by any node
  uint32_t lanes_from;   // group size from which the expansion puts lanes on plans
  uint32_t huge_from;    // front + candidates from which a node's merge is grid-wide
  uint32_t ov_any;       // some query overflowed its slots this wavefront
  // grid barrier
  uint32_t bar_count;
  uint32_t bar_gen;
  uint32_t timeout;      // a barrier wait ran out
  uint32_t pad;
  unsigned long long wait_ns;  // limit of one barrier wait
  unsigned long long t_mark;   // %globaltimer at the last barrier release
  unsigned long long ph_ns[4]; // expand, overflow regrouping, merge, end of wavefront
  unsigned long long idle_ns;  // block time spent waiting at grid barriers, summed over blocks
  uint32_t waves;
  uint32_t grab[2];      // work counters of the expansion and the merge (nodes handed out)
  uint32_t ovl_n;        // nodes with overflow records this wavefront
  uint32_t ov_total;     // overflow records of all queries this wavefront
  unsigned long long arena_common_n;   // records of the arena's common half handed out
  unsigned long long pool_common_n;    // entries of the front pool's common half handed out
  unsigned long long tmp_n;            // bulk-merge scratch entries handed out this wavefront
  // grid-wide merges of huge nodes (this wavefront)
  uint32_t hg_n;         // huge nodes handed to the grid-wide merge
  uint32_t hg_live;      // the grid-wide merge runs before the end of this wavefront
  uint32_t hg_nm;        // their members (front entries and candidates), flat
  uint32_t hg_nt;        // their bucket tiles, flat
  unsigned long long hg_ents;   // members reserved (bounds the flat index space)
};

// A node merged by the whole grid (see the grid-wide merge below).
struct HugeDesc {
  uint32_t g, q, n, nc;        // node, query, front entries, candidates
  uint32_t off, so;            // live front block; regrouped overflow segment (kNone: none)
  uint32_t lg_old;             // lg of the live block's size
  uint32_t out, lg_out;        // block the merged front goes to, lg of its size (0: none yet)
  uint32_t nb, shift;          // cost buckets (a power of two, at least kTile) and cost shift
  uint32_t ent0, tile0;        // first flat member and tile index
  uint32_t ok;                 // 0: skipped (its query failed for capacity)
  unsigned long long mem;      // scratch: members [mem, mem + n + nc)
  unsigned long long bkt;      //          buckets [bkt, bkt + nb)
  long long lo, hi;            // cost range of the members
  uint32_t n_out, n_new, removed_open, pad;
};

struct WS {
  uint64_t NV;
  uint32_t fcap;           // front pool entries per node (pool = NV fcap)
  uint64_t pcap;           // front pool entries
  uint64_t acap, gcap, ocap, tcap;
  uint64_t arena_common_base, arena_common_cap;   // the arena's half that all queries share
  uint64_t pool_common_base, pool_common_cap;     // the front pool's half that all queries share
  long long* f_cost;       // [pcap] front pool
  long long* f_h;
  uint32_t* f_pid;
  uint32_t* f_aux;
  FDesc* fdesc;            // [NV]
  Cand* slot;              // [NV * kSlots] candidates of this wavefront
  uint32_t* cand_n;        // [NV] candidates per node this wavefront (0 between wavefronts)
  Cand* ov;                // [ocap] overflow candidates in arrival order (per-query shares)
  Cand* ov2;               // [ocap] the same regrouped per node
  uint32_t* segoff;        // [NV] start of a node's regrouped overflow
  long long* t_cost;       // [tcap] bulk-merge scratch (reset every wavefront): candidate
  long long* t_h;          //   skylines {cost, h, parent, tie key} and insertion indices
  uint32_t* t_pp;
  uint32_t* t_tb;
  uint32_t* t_m;
  uint2* ovl;              // [NV] {node, query} with overflow records this wavefront
  uint32_t* ov_pref;       // [max_q + 1] exclusive prefix of the queries' overflow records
  uint32_t* oh_stamp;
  long long* g_cost;       // [gcap] groups of more than 32 plans
  long long* g_h;
  uint32_t* g_pid;
  uint2* oh_list;          // [2][NV] {node, query} with open plans (this / next wavefront)
  uint2* m_list;           // [NV] {node, query} with candidates this wavefront
  HugeDesc* hg;             // [kHugeMax] huge nodes of this wavefront
  uint32_t* a_head;
  uint32_t* a_parent;
  uint32_t* a_iter;
  long long* a_cost;
  Ctl* ctl;
  QueryDev* qd;
  QueryState* qs;
  ResultDev* res;
  uint32_t* path;
  uint32_t path_cap;
};

}  // namespace mpap

struct mpap_workspace {
  mpap::WS w{};
  uint32_t max_q = 0;
  // host record of the last search (for front export and tuning)
  std::vector<uint32_t> last_V, last_base;
  uint32_t last_max_front = 0;
  unsigned long long last_pool_used = 0;
  // pinned host staging of the results (grown on demand): per-query results,
  // states and the loop control block; the plans' node lists
  char* h_hdr = nullptr;
  size_t h_hdr_bytes = 0;
  char* h_path = nullptr;
  size_t h_path_bytes = 0;
};

namespace mpap {

constexpr int kWarpsPerBlock = 8;
constexpr unsigned kFull = 0xFFFFFFFFu;

void workspace_free(mpap_workspace* ws);
void profile_add(const char* name, uint64_t launches, double ms);
bool profile_enabled();
void launch_count_add(uint64_t n);

// Signed 64-bit atomic add through the unsigned overload (two's complement).
__device__ __forceinline__ void atomic_add_i64(long long* p, long long v) {
  atomicAdd(reinterpret_cast<unsigned long long*>(p), static_cast<unsigned long long>(v));
}

constexpr uint32_t kMinLg = 4;          // smallest pool block: 16 entries
constexpr uint32_t kNoBlock = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t ceil_lg(uint32_t n) {
  return n <= 1 ? 0u : 32u - (uint32_t)__clz(n - 1u);
}

// One block of 2^lg entries for query q (call from one lane): from the query's
// own pool share while it lasts, then from the pool's common half, which every
// query of the batch draws on (a query whose fronts outgrow its share borrows
// what the others leave); kNoBlock when both are used up.  Where a block lies
// does not change any result.
__device__ __forceinline__ uint32_t pool_alloc(const WS& w, uint32_t q, uint32_t lg) {
  const unsigned long long sz = 1ull << lg;
  const unsigned long long o = atomicAdd(&w.qs[q].pool_n, sz);
  const QueryDev& Q = w.qd[q];
  if (o + sz <= Q.pool_cap) return (uint32_t)(Q.pool_base + o);
  if (Q.flags & MPAP_QUERY_OWN_SHARE) return kNoBlock;
  const unsigned long long c = atomicAdd(&w.ctl->pool_common_n, sz);
  return (c + sz <= w.pool_common_cap) ? (uint32_t)(w.pool_common_base + c) : kNoBlock;
}

// Records a capacity error of query q (it ends at the end of the wavefront).
__device__ __forceinline__ void query_error(const WS& w, uint32_t q, uint32_t bit) {
  atomicOr(&w.qs[q].err, bit);
  atomicOr(&w.ctl->err, bit);
}

__device__ __forceinline__ unsigned long long global_timer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t ld_vol(const uint32_t* p) { return *(const volatile uint32_t*)p; }

// ---------------------------------------------------------------------------
// Grid barrier of the persistent loop.  The launch is cooperative, so every
// block is resident and the barrier cannot deadlock on scheduling.  Arrival is
// an atomic count behind a fence; the last block to arrive runs `epi` with all
// its threads, then releases the others by advancing the generation.  A block
// that waits longer than ctl->wait_ns (%globaltimer time), or sees that another
// block gave up, sets ctl->timeout and returns false: its caller leaves the
// kernel, and so, within one wait limit, does every other block.
// ---------------------------------------------------------------------------
template <class Epi>
__device__ __forceinline__ bool grid_barrier(const WS& w, Epi epi) {
  __shared__ uint32_t s_last, s_ok;
  Ctl* c = w.ctl;
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t gen = ld_vol(&c->bar_gen);
    __threadfence();
    const uint32_t arrived = atomicAdd(&c->bar_count, 1u) + 1u;
    s_last = arrived == gridDim.x ? 1u : 0u;
    s_ok = 1u;
    if (!s_last) {
      const unsigned long long t0 = global_timer();
      const unsigned long long lim = c->wait_ns;
      unsigned long long t = t0;
      while (ld_vol(&c->bar_gen) == gen) {
        t = global_timer();
        if (ld_vol(&c->timeout) || t - t0 > lim) {
          atomicExch(&c->timeout, 1u);
          s_ok = 0u;
          break;
        }
        __nanosleep(64);
      }
      atomicAdd(&c->idle_ns, t - t0);
    }
    __threadfence();
  }
  __syncthreads();
  if (s_last) {
    epi();
    __syncthreads();
    if (threadIdx.x == 0) {
      c->bar_count = 0;
      __threadfence();
      atomicAdd(&c->bar_gen, 1u);
    }
  }
  return s_ok != 0u;
}

// Phase time between the last release and now, charged to slot k (last block).
__device__ __forceinline__ void phase_mark(const WS& w, int k) {
  if (threadIdx.x == 0) {
    const unsigned long long now = global_timer();
    w.ctl->ph_ns[k] += now - w.ctl->t_mark;
    w.ctl->t_mark = now;
  }
}

// ---------------------------------------------------------------------------
__global__ void k_init(WS w, uint32_t nq, uint32_t iter_cap, uint32_t lanes_from, uint32_t huge_from,
                       unsigned long long wait_ns) {
  const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q == 0) {
    Ctl& c = *w.ctl;
    c.oh_n[0] = nq;
    c.oh_n[1] = 0;
    c.m_n = 0;
    c.g_n = 0;
    c.err = 0;
    c.it = 0;
    c.nq = nq;
    c.iter_cap = iter_cap;
    c.max_front = 1;
    c.lanes_from = lanes_from;
    c.huge_from = huge_from;
    c.ov_any = 0;
    c.bar_count = 0;
    c.bar_gen = 0;
    c.timeout = 0;
    c.wait_ns = wait_ns;
    c.t_mark = 0;
    for (int k = 0; k < 4; ++k) c.ph_ns[k] = 0;
    c.idle_ns = 0;
    c.waves = 0;
    c.grab[0] = 0;
    c.grab[1] = 0;
    c.ovl_n = 0;
    c.ov_total = 0;
    c.arena_common_n = 0;
    c.pool_common_n = 0;
    c.tmp_n = 0;
    c.hg_n = 0;
    c.hg_live = 0;
    c.hg_nm = 0;
    c.hg_nt = 0;
    c.hg_ents = 0;
  }
  if (q >= nq) return;
  const QueryDev& Q = w.qd[q];
  const uint32_t g = Q.base;   // x_init is node 0 of every roadmap
  QueryState s;
  s.open_cnt = 1;
  s.expansions = 0;
  s.plans = 0;
  s.wavefronts = 0;
  s.goal_hit = 0;
  s.done = 0;
  s.status = 0;
  s.err = 0;
  s.goal_next = 0;
  s.pool_n = 1u << kMinLg;          // the root's block opens the query's share
  s.ov_n = 0;
  s.seg_n = 0;
  s.arena_n = 1;                     // the root plan opens the query's arena share
  // the first group is {root}: a root inside X_goal ends the query before any
  // expansion (the loop condition of Alg. 3 is tested first)
  if (Q.is_goal[0] && !(Q.flags & MPAP_QUERY_NO_GOAL_STOP)) {
    s.done = 1;
    s.goal_hit = 1;
  }
  w.qs[q] = s;
  const uint32_t o = (uint32_t)Q.pool_base;
  const uint32_t a = (uint32_t)Q.arena_base;
  w.f_cost[o] = 0;
  w.f_h[o] = 0;
  w.f_pid[o] = a | kOpen;      // the root plan (x_init, {}, 0, 0) opens the arena share
  w.f_aux[o] = 0;
  FDesc fd0;
  fd0.d = make_uint4(o, 1u, 0u, kMinLg);
  fd0.last = make_longlong2(0, 0);
  w.fdesc[g] = fd0;
  w.a_head[a] = 0;
  w.a_parent[a] = kNone;
  w.a_iter[a] = 0;
  w.a_cost[a] = 0;
  w.oh_list[q] = make_uint2(g, q);
  w.oh_stamp[g] = 0;
}

// Counts the queries k_init ended at once (root in X_goal).
__global__ void k_init_done(WS w, uint32_t nq) {
  __shared__ uint32_t s_n;
  if (threadIdx.x == 0) s_n = 0;
  __syncthreads();
  for (uint32_t q = threadIdx.x; q < nq; q += blockDim.x)
    if (w.qs[q].done) atomicAdd(&s_n, 1u);
  __syncthreads();
  if (threadIdx.x == 0) w.ctl->n_done = s_n;
}
// ---------------------------------------------------------------------------
// Skyline merge of candidates into a front, 32 candidates at a time (warp per
// node).
// ---------------------------------------------------------------------------
struct WarpSmem {
  long long s_cost[32];    // chunk survivors, sorted
  long long s_h[32];
  uint32_t s_tb[32];
  uint32_t s_pp[32];
  uint32_t bins[33];
  long long st_cost[64];   // merged register front staging
  long long st_h[64];
  uint32_t st_pid[64];
  uint32_t st_aux[64];
};

__device__ __forceinline__ bool key_less(long long c1, long long h1, uint32_t t1, long long c2,
                                         long long h2, uint32_t t2) {
  if (c1 != c2) return c1 < c2;
  if (h1 != h2) return h1 < h2;
  return t1 < t2;
}

// Front of one node during the merge: in registers (lane j holds entry j, n <= 32)
// or in the node's live pool block.
struct FrontCursor {
  bool reg;
  bool err;          // a pool block could not be had: stop merging this node
  uint32_t off, lg;  // live block (lg = log2 size, 0: none)
  uint32_t off2, lg2;  // the other block (merge target)
  uint32_t n;        // live count
  uint32_t removed_open;
  bool any_new;
  long long rc, rh;  // register entry of this lane (reg mode)
  uint32_t rp, ra;
};

// Makes the other block hold at least `need` entries (warp-uniform); false when
// the pool is exhausted (the query is marked failed).
__device__ __forceinline__ bool ensure_other(const WS& w, uint32_t q, FrontCursor& fc, uint32_t need) {
  if (fc.lg2 != 0 && (1u << fc.lg2) >= need) return true;
  const uint32_t lg = max(kMinLg, ceil_lg(need) + 1u);
  uint32_t o = 0;
  if (lane_id() == 0) o = pool_alloc(w, q, lg);
  o = __shfl_sync(kFull, o, 0);
  if (o == kNoBlock) {
    if (lane_id() == 0) query_error(w, q, kErrFront);
    fc.err = true;
    return false;
  }
  fc.off2 = o;
  fc.lg2 = lg;
  return true;
}

__device__ __forceinline__ void swap_blocks(FrontCursor& fc) {
  const uint32_t o = fc.off, l = fc.lg;
  fc.off = fc.off2;
  fc.lg = fc.lg2;
  fc.off2 = o;
  fc.lg2 = l;
}

// Sort the chunk (one candidate per lane; padding lanes last) by (cost, h, tb)
// and keep its skyline: survivors are written to sm.s_* in order; returns their
// count.
__device__ __forceinline__ uint32_t chunk_skyline(WarpSmem& sm, bool ok, long long cc, long long ch,
                                                  uint32_t ctb, uint32_t cpp) {
  const unsigned lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  const long long vh = ok ? ch : LLONG_MAX;
  const uint32_t vt = ok ? ctb : 0xFFFFFFFFu;
  // 1. sort (cost, source lane) only -- two shuffles of key and index per
  //    step -- then gather the rest of each candidate from its source lane
  long long kc = ok ? cc : LLONG_MAX;
  uint32_t ks = lane;
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const long long oc = shfl_xor_i64(kc, j);
      const uint32_t os = __shfl_xor_sync(kFull, ks, j);
      const bool up = (lane & k) == 0;
      const bool lower = (lane & j) == 0;
      const bool o_less = oc < kc || (oc == kc && os < ks);
      const bool take = (lower == up) ? o_less : !o_less;
      if (take) {
        kc = oc;
        ks = os;
      }
    }
  }
  long long kh = shfl_i64(vh, (int)ks);
  uint32_t kt = __shfl_sync(kFull, vt, (int)ks), kp = __shfl_sync(kFull, cpp, (int)ks);
  // 2. equal costs among real candidates must be ordered by (h, tie key) too:
  //    then sort the chunk again on the full key (rare)
  {
    const long long pc = shfl_up_i64(kc, 1);
    const bool tie = lane > 0 && kt != 0xFFFFFFFFu && pc == kc;
    if (__any_sync(kFull, tie)) {
#pragma unroll
      for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
          const long long oc = shfl_xor_i64(kc, j), oh = shfl_xor_i64(kh, j);
          const uint32_t ot = __shfl_xor_sync(kFull, kt, j), op = __shfl_xor_sync(kFull, kp, j);
          const bool up = (lane & k) == 0;
          const bool lower = (lane & j) == 0;
          const bool o_less = key_less(oc, oh, ot, kc, kh, kt);
          const bool m_less = key_less(kc, kh, kt, oc, oh, ot);
          const bool take = (lower == up) ? o_less : m_less;
          if (take) {
            kc = oc;
            kh = oh;
            kt = ot;
            kp = op;
          }
        }
      }
    }
  }
  // exclusive prefix minimum of h in sorted order
  long long pm = kh;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long t = shfl_up_i64(pm, o);
    if (lane >= (unsigned)o) pm = t < pm ? t : pm;
  }
  long long excl = shfl_up_i64(pm, 1);
  if (lane == 0) excl = LLONG_MAX;
  const bool surv = (kt != 0xFFFFFFFFu) && kh < excl;
  const unsigned sb = __ballot_sync(kFull, surv);
  if (surv) {
    const uint32_t r = __popc(sb & lt);
    sm.s_cost[r] = kc;
    sm.s_h[r] = kh;
    sm.s_tb[r] = kt;
    sm.s_pp[r] = kp;
  }
  __syncwarp();
  return __popc(sb);
}

// Block-mode merge of up to 32 candidates into the live front of a node: the
// merged front is written to the node's other block, which then becomes live.
// Candidate tie key tb = 1 + parent head (old plans have tie key 0, i.e. they win
// exact (cost, h) ties).
__device__ __forceinline__ void merge_chunk_slab(const WS& w, uint32_t q, FrontCursor& fc, WarpSmem& sm, bool ok,
                                 long long cc, long long ch, uint32_t ctb, uint32_t cpp) {
  const unsigned lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  // 1. drop candidates dominated by the live front (last entry with cost <= cc)
  {
    const size_t o = fc.off;
    if (ok && fc.n > 0) {
      uint32_t L = 0, R = fc.n;
      while (L < R) {
        const uint32_t mid = (L + R) >> 1;
        if (w.f_cost[o + mid] <= cc) L = mid + 1; else R = mid;
      }
      if (L > 0) {
        const uint32_t j = L - 1;
        const long long fcost = w.f_cost[o + j], fh = w.f_h[o + j];
        const uint32_t fpid = w.f_pid[o + j];
        const uint32_t ftb = (fpid & kNew) ? w.f_aux[o + j] : 0u;
        if (fh <= ch && (fcost < cc || fh < ch || ftb < ctb)) ok = false;
      }
    }
  }
  if (!__any_sync(kFull, ok)) return;
  // 2. skyline of the chunk
  const uint32_t m = chunk_skyline(sm, ok, cc, ch, ctb, cpp);
  if (!ensure_other(w, q, fc, fc.n + m)) return;
  sm.bins[lane] = 0;
  if (lane == 0) sm.bins[32] = 0;
  __syncwarp();
  // 3. one pass over the live front: drop entries dominated by a survivor, write
  //    the kept ones to the other block at (kept rank + survivors before them)
  const size_t o = fc.off, on = fc.off2;
  uint32_t kept = 0;
  uint32_t rem_open = 0;
  for (uint32_t j0 = 0; j0 < fc.n; j0 += 32) {
    const uint32_t j = j0 + lane;
    const bool valid = j < fc.n;
    long long fcost = 0, fh = 0;
    uint32_t fpid = 0, faux = 0;
    if (valid) {
      fcost = w.f_cost[o + j];
      fh = w.f_h[o + j];
      fpid = w.f_pid[o + j];
      faux = w.f_aux[o + j];
    }
    const uint32_t ftb = (fpid & kNew) ? faux : 0u;
    uint32_t L = 0, R = m;
    while (L < R) {
      const uint32_t mid = (L + R) >> 1;
      if (sm.s_cost[mid] <= fcost) L = mid + 1; else R = mid;
    }
    bool dom = false;
    if (valid && L > 0) {
      const uint32_t s = L - 1;
      const long long scost = sm.s_cost[s], sh = sm.s_h[s];
      dom = sh <= fh && (scost < fcost || sh < fh || sm.s_tb[s] < ftb);
    }
    const bool keep = valid && !dom;
    if (dom && (fpid & kOpen) && !(fpid & kNew)) rem_open++;
    const unsigned kb = __ballot_sync(kFull, keep);
    if (keep) {
      const uint32_t pos = kept + __popc(kb & lt) + L;
      w.f_cost[on + pos] = fcost;
      w.f_h[on + pos] = fh;
      w.f_pid[on + pos] = fpid;
      w.f_aux[on + pos] = faux;
      atomicAdd(&sm.bins[L], 1u);
    }
    kept += __popc(kb);
  }
  __syncwarp();
  const uint32_t before = warp_incl_scan(lane < m ? sm.bins[lane] : 0u);
  if (lane < m) {
    const uint32_t pos = lane + before;
    w.f_cost[on + pos] = sm.s_cost[lane];
    w.f_h[on + pos] = sm.s_h[lane];
    w.f_pid[on + pos] = sm.s_pp[lane] | kNew;
    w.f_aux[on + pos] = sm.s_tb[lane];
  }
  for (int s = 16; s > 0; s >>= 1) rem_open += __shfl_xor_sync(kFull, rem_open, s);
  fc.removed_open += rem_open;
  swap_blocks(fc);
  fc.n = kept + m;
  fc.any_new = true;
  __syncwarp();
}
// Register-mode merge: the front (n <= 32) is held one entry per lane; all
// dominance tests are broadcasts over lanes.  If the merged front exceeds 32
// entries it is written to the node's other block and the node continues in
// block mode.
__device__ __forceinline__ void merge_chunk_reg(const WS& w, uint32_t q, FrontCursor& fc, WarpSmem& sm, bool ok,
                                long long cc, long long ch, uint32_t ctb, uint32_t cpp) {
  const unsigned lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t n = fc.n;
  const uint32_t rtb = (fc.rp & kNew) ? fc.ra : 0u;
  // 1. candidates dominated by any front entry
  if (__any_sync(kFull, ok)) {
    for (uint32_t j = 0; j < n; ++j) {
      const long long fcj = shfl_i64(fc.rc, (int)j), fhj = shfl_i64(fc.rh, (int)j);
      const uint32_t ftj = __shfl_sync(kFull, rtb, (int)j);
      if (ok && fcj <= cc && fhj <= ch && (fcj < cc || fhj < ch || ftj < ctb)) ok = false;
    }
  }
  if (!__any_sync(kFull, ok)) return;
  // 2. skyline of the chunk
  const uint32_t m = chunk_skyline(sm, ok, cc, ch, ctb, cpp);
  // 3. front entries dominated by a survivor; ranks of the merged order
  const bool valid = lane < n;
  bool dom = false;
  uint32_t below = 0;   // survivors with smaller cost
  for (uint32_t s = 0; s < m; ++s) {
    const long long scost = sm.s_cost[s], sh = sm.s_h[s];
    if (valid && scost <= fc.rc && sh <= fc.rh && (scost < fc.rc || sh < fc.rh || sm.s_tb[s] < rtb)) dom = true;
    below += (scost < fc.rc) ? 1u : 0u;
  }
  const bool keep = valid && !dom;
  const unsigned kb = __ballot_sync(kFull, keep);
  const uint32_t kept = __popc(kb);
  const uint32_t rem_open = __popc(__ballot_sync(kFull, dom && valid && (fc.rp & kOpen) && !(fc.rp & kNew)));
  if (keep) {
    const uint32_t pos = __popc(kb & lt) + below;
    sm.st_cost[pos] = fc.rc;
    sm.st_h[pos] = fc.rh;
    sm.st_pid[pos] = fc.rp;
    sm.st_aux[pos] = fc.ra;
  }
  // survivor lane s: kept front entries with smaller cost come first
  uint32_t before = 0;
  const long long my_scost = lane < m ? sm.s_cost[lane] : 0;
  for (uint32_t j = 0; j < n; ++j) {
    const long long fcj = shfl_i64(fc.rc, (int)j);
    const bool kj = (kb >> j) & 1u;
    before += (kj && fcj < my_scost) ? 1u : 0u;
  }
  if (lane < m) {
    const uint32_t pos = lane + before;
    sm.st_cost[pos] = sm.s_cost[lane];
    sm.st_h[pos] = sm.s_h[lane];
    sm.st_pid[pos] = sm.s_pp[lane] | kNew;
    sm.st_aux[pos] = sm.s_tb[lane];
  }
  __syncwarp();
  const uint32_t n_new = kept + m;
  if (n_new <= 32) {
    if (lane < n_new) {
      fc.rc = sm.st_cost[lane];
      fc.rh = sm.st_h[lane];
      fc.rp = sm.st_pid[lane];
      fc.ra = sm.st_aux[lane];
    }
    fc.n = n_new;
  } else {
    // spill to the other block and continue in block mode
    if (!ensure_other(w, q, fc, n_new)) return;
    const size_t on = fc.off2;
    for (uint32_t i = lane; i < n_new; i += 32) {
      w.f_cost[on + i] = sm.st_cost[i];
      w.f_h[on + i] = sm.st_h[i];
      w.f_pid[on + i] = sm.st_pid[i];
      w.f_aux[on + i] = sm.st_aux[i];
    }
    swap_blocks(fc);
    fc.reg = false;
    fc.n = n_new;
  }
  fc.removed_open += rem_open;
  fc.any_new = true;
  __syncwarp();
}

// r arena records for query q (call from one lane): from the query's own share
// while it lasts, then from the arena's common half, which every query of the
// batch draws on; kNone when both are used up (the query then fails).
__device__ __forceinline__ uint32_t arena_take(const WS& w, uint32_t q, uint32_t r) {
  const unsigned long long o = atomicAdd(&w.qs[q].arena_n, (unsigned long long)r);
  const QueryDev& Q = w.qd[q];
  if (o + r <= Q.arena_cap) return (uint32_t)(Q.arena_base + o);
  if (Q.flags & MPAP_QUERY_OWN_SHARE) {
    query_error(w, q, kErrArena);
    return kNone;
  }
  const unsigned long long c = atomicAdd(&w.ctl->arena_common_n, (unsigned long long)r);
  if (c + r <= w.arena_common_cap) return (uint32_t)(w.arena_common_base + c);
  query_error(w, q, kErrArena);
  return kNone;
}

// Per-block shared state of the wavefront kernel: per-query counter
// increments accumulated in shared memory (flushed to the query states once per
// phase, so the per-node updates never contend on one global address; batches
// of more than kAccQ queries add to the states directly), and per-warp buffers
// of nodes bound for the next open list.
constexpr uint32_t kAccQ = 256;
struct WaveSmem {
  long long open[kAccQ];
  unsigned long long plans[kAccQ];
  unsigned long long exps[kAccQ];
  uint2 lbuf[kWarpsPerBlock][32];   // bound for the next open list
  uint2 mbuf[kWarpsPerBlock][32];   // bound for this wavefront's merge list
};

struct WarpCtx {
  WaveSmem* s;
  uint2* next;        // open list of the next wavefront
  uint32_t lb_n;      // nodes in this warp's open-list buffer (warp-uniform)
  uint32_t mb_n;      // nodes in this warp's merge-list buffer (warp-uniform)
  uint32_t nq;
  uint32_t it;
  uint32_t huge_from;  // front + candidates from which a node's merge is grid-wide
};

__device__ __forceinline__ void acc_open(const WS& w, WarpCtx& cx, uint32_t q, long long v) {
  if (!v) return;
  if (cx.nq <= kAccQ) atomicAdd(reinterpret_cast<unsigned long long*>(&cx.s->open[q]), (unsigned long long)v);
  else atomic_add_i64(&w.qs[q].open_cnt, v);
}
__device__ __forceinline__ void acc_plans(const WS& w, WarpCtx& cx, uint32_t q, unsigned long long v) {
  if (!v) return;
  if (cx.nq <= kAccQ) atomicAdd(&cx.s->plans[q], v);
  else atomicAdd(&w.qs[q].plans, v);
}
__device__ __forceinline__ void acc_exps(const WS& w, WarpCtx& cx, uint32_t q, unsigned long long v) {
  if (!v) return;
  if (cx.nq <= kAccQ) atomicAdd(&cx.s->exps[q], v);
  else atomicAdd(&w.qs[q].expansions, v);
}

// Adds the block's accumulated increments to the query states (whole block).
__device__ __forceinline__ void flush_acc(const WS& w, WaveSmem& s, uint32_t nq) {
  __syncthreads();
  if (nq <= kAccQ) {
    for (uint32_t q = threadIdx.x; q < nq; q += blockDim.x) {
      if (s.open[q]) atomic_add_i64(&w.qs[q].open_cnt, s.open[q]);
      if (s.plans[q]) atomicAdd(&w.qs[q].plans, s.plans[q]);
      if (s.exps[q]) atomicAdd(&w.qs[q].expansions, s.exps[q]);
      s.open[q] = 0;
      s.plans[q] = 0;
      s.exps[q] = 0;
    }
  }
}

// Moves this warp's buffered nodes to the next open list (one atomic).
__device__ __forceinline__ void flush_next(const WS& w, WarpCtx& cx) {
  if (!cx.lb_n) return;
  const unsigned lane = lane_id();
  __syncwarp();
  uint32_t b = 0;
  if (lane == 0) b = atomicAdd(&w.ctl->oh_n[(cx.it + 1) & 1], cx.lb_n);
  b = __shfl_sync(kFull, b, 0);
  if (lane < cx.lb_n) cx.next[b + lane] = cx.s->lbuf[threadIdx.x >> 5][lane];
  __syncwarp();
  cx.lb_n = 0;
}

// Puts node g of query q on the next open list (warp-uniform arguments).  A
// node gets there at most once per wavefront: the expansion, which visits every
// listed node once, stamps the nodes it keeps on the list, and the merge, which
// visits every node once, skips stamped ones (no atomics needed).
__device__ __forceinline__ void push_next(const WS& w, WarpCtx& cx, uint32_t g, uint32_t q) {
  if (lane_id() == 0) cx.s->lbuf[threadIdx.x >> 5][cx.lb_n] = make_uint2(g, q);
  if (++cx.lb_n == 32) flush_next(w, cx);
}

// Moves this warp's buffered nodes to the merge list (one atomic).
__device__ __forceinline__ void flush_merge(const WS& w, WarpCtx& cx) {
  if (!cx.mb_n) return;
  const unsigned lane = lane_id();
  __syncwarp();
  uint32_t b = 0;
  if (lane == 0) b = atomicAdd(&w.ctl->m_n, cx.mb_n);
  b = __shfl_sync(kFull, b, 0);
  if (lane < cx.mb_n) w.m_list[b + lane] = cx.s->mbuf[threadIdx.x >> 5][lane];
  __syncwarp();
  cx.mb_n = 0;
}

// Arena records for the new entries of a block-mode front (marked open);
// returns their number.
__device__ __forceinline__ uint32_t arena_block(const WS& w, uint32_t q, uint32_t x, uint32_t it,
                                                const FrontCursor& fc) {
  const unsigned lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  uint32_t n_new = 0;
  const size_t o = fc.off;
  for (uint32_t j0 = 0; j0 < fc.n; j0 += 32) {
    const uint32_t j = j0 + lane;
    uint32_t pid = 0;
    if (j < fc.n) pid = w.f_pid[o + j];
    const bool isnew = (j < fc.n) && (pid & kNew);
    const unsigned bal = __ballot_sync(kFull, isnew);
    if (!bal) continue;
    uint32_t a0 = 0;
    if (lane == 0) a0 = arena_take(w, q, (uint32_t)__popc(bal));
    a0 = __shfl_sync(kFull, a0, 0);
    if (isnew) {
      if (a0 != kNone) {
        const uint32_t a = a0 + (uint32_t)__popc(bal & lt);
        w.a_head[a] = x;
        w.a_parent[a] = pid & kPidMask;
        w.a_iter[a] = it + 1;
        w.a_cost[a] = w.f_cost[o + j];
        w.f_pid[o + j] = a | kOpen;
      } else {
        w.f_pid[o + j] = kOpen;
      }
      w.f_aux[o + j] = 0;
    }
    n_new += __popc(bal);
  }
  return n_new;
}

// The node's new descriptor and counters, and its place in the next open list.
__device__ __forceinline__ void commit_tail(const WS& w, WarpCtx& cx, uint32_t q, uint32_t g, const FrontCursor& fc,
                                            uint32_t n_new, long long last_c, long long last_h, bool listed) {
  if (lane_id() == 0) {
    FDesc fd;
    fd.d = make_uint4(fc.off, fc.n, fc.off2, fc.lg | (fc.lg2 << 8));
    fd.last = make_longlong2(last_c, last_h);
    w.fdesc[g] = fd;
    acc_open(w, cx, q, (long long)n_new - (long long)fc.removed_open);
    acc_plans(w, cx, q, n_new);
    if (fc.n > ld_vol(&w.ctl->max_front)) atomicMax(&w.ctl->max_front, fc.n);
  }
  if (!listed) push_next(w, cx, g, q);
}

// ---------------------------------------------------------------------------
// Expansion (Alg. 3: every group plan along every out-edge of its head, the
// beta cutoff, and the part of RemoveDominated that the stored front of the
// target decides on its own).
// ---------------------------------------------------------------------------

// Group plans of one node staged per warp (groups of at most 32 plans).
struct GroupSmem {
  long long c[32];
  long long h[32];
  uint32_t p[32];
};

// First index in the cost-sorted front [o, o + n) whose cost exceeds c,
// searching from index i (fronts are strictly increasing in cost).
__device__ __forceinline__ uint32_t front_upper(const WS& w, size_t o, uint32_t n, uint32_t i, long long c) {
  if (n - i > 16) {
    uint32_t lo = i, hi = n;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (w.f_cost[o + mid] <= c) lo = mid + 1; else hi = mid;
    }
    return lo;
  }
  while (i < n && w.f_cost[o + i] <= c) ++i;
  return i;
}

// Slot bookkeeping after the atomic add that gave a lane its first slot s for r
// new candidates of node gx: the lane that opened gx this wavefront puts it on
// the merge list; slots from kSlots on are overflow records, whose indices in
// query q's overflow share come back in *ov (warp-aggregated).  Warp-collective.
__device__ __forceinline__ void slot_book(const WS& w, WarpCtx& cx, uint32_t q, uint32_t gx, uint32_t r, uint32_t s,
                                          uint32_t* ov) {
  const unsigned lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  const bool first = r && s == 0;
  const unsigned fb = __ballot_sync(kFull, first);
  if (fb) {
    const uint32_t nf = (uint32_t)__popc(fb);
    if (cx.mb_n + nf > 32) flush_merge(w, cx);
    if (first) cx.s->mbuf[threadIdx.x >> 5][cx.mb_n + __popc(fb & lt)] = make_uint2(gx, q);
    cx.mb_n += nf;
  }
  const uint32_t nov = (s + r > kSlots) ? s + r - max(s, kSlots) : 0u;
  *ov = 0;
  if (!__any_sync(kFull, nov != 0u)) return;    // the common case: every record fits its slots
  const uint32_t incl = warp_incl_scan(nov);
  const uint32_t tot = __shfl_sync(kFull, incl, 31);
  uint32_t b = 0;
  if (lane == 0) b = atomicAdd(&w.qs[q].ov_n, tot);
  b = __shfl_sync(kFull, b, 0);
  *ov = b + incl - nov;
}

// Stores candidate cd as candidate s of node gx (a slot, or overflow record oi
// of query q's share).
__device__ __forceinline__ void put_cand(const WS& w, const QueryDev& Q, uint32_t q, uint32_t gx, uint32_t s,
                                         uint32_t& oi, Cand cd) {
  if (s < kSlots) {
    w.slot[(size_t)gx * kSlots + s] = cd;
  } else {
    // the first overflow record of a node lists it for the regrouping
    if (s == kSlots) w.ovl[atomicAdd(&w.ctl->ovl_n, 1u)] = make_uint2(gx, q);
    if (oi < Q.ov_cap) {
      cd.g = gx;
      cd.i = s - kSlots;
      w.ov[Q.ov_base + oi] = cd;
    } else {
      query_error(w, q, kErrList);
    }
    ++oi;
  }
}

// Is candidate (c, h) dominated by the stored front of a node (descriptor xd)?
// The last entry decides most cases; otherwise the last entry of cost <= c (the
// one of lowest h among them: fronts are strictly monotone), found from index *i
// on (candidates of one run come in increasing cost).  Old plans win ties.
__device__ __forceinline__ bool front_dominates(const WS& w, const FDesc& xd, uint32_t* i, long long c, long long h) {
  const uint32_t n = xd.d.y;
  if (n == 0) return false;
  if (c >= xd.last.x && h >= xd.last.y) return true;
  *i = front_upper(w, xd.d.x, n, *i, c);
  return *i > 0 && w.f_h[(size_t)xd.d.x + *i - 1] <= h;
}

// Bit j set: group plan j extended along edge ed survives the beta cutoff, its
// run predecessor and the target's stored front.
__device__ __forceinline__ uint32_t filter_run(const WS& w, const QueryDev& Q, const GroupSmem& gs, uint32_t cnt,
                                               const int4& ed, const int2& pk, bool interior, const FDesc& xd) {
  uint32_t mask = 0, i = 0;
  long long prev_h = LLONG_MAX;
  for (uint32_t j = 0; j < cnt; ++j) {
    const long long gh = gs.h[j];
    const long long c = gs.c[j] + (long long)ed.y;
    const long long hh = gh + (long long)ed.z;
    const long long h = hh > (long long)ed.w ? hh : (long long)ed.w;
    long long peak = h;
    if (interior) {
      const long long hp = gh + (long long)pk.x;
      peak = hp > (long long)pk.y ? hp : (long long)pk.y;
    }
    if (peak > Q.beta) continue;
    // the previous plan of the run (lower cost) dominates unless h drops
    if (h >= prev_h) continue;
    prev_h = h;
    if (front_dominates(w, xd, &i, c, h)) continue;
    mask |= 1u << j;
  }
  return mask;
}

__device__ __forceinline__ void write_run(const WS& w, const QueryDev& Q, uint32_t q, uint32_t u, const GroupSmem& gs,
                                          uint32_t mask, const int4& ed, uint32_t gx, uint32_t s, uint32_t oi) {
  for (uint32_t m = mask; m; m &= m - 1u) {
    const uint32_t j = (uint32_t)__ffs(m) - 1u;
    Cand cd;
    cd.cost = gs.c[j] + (long long)ed.y;
    const long long hh = gs.h[j] + (long long)ed.z;
    cd.h = hh > (long long)ed.w ? hh : (long long)ed.w;
    cd.pp = gs.p[j];
    cd.tb = 1u + u;
    cd.g = 0;
    cd.i = 0;
    put_cand(w, Q, q, gx, s++, oi, cd);
  }
}

// Small groups: lanes on the out-edges of u (two edges per lane per step, all
// their loads in flight together), each lane walking the group plans (cost
// order) and the target's front together.
__device__ __forceinline__ void expand_edges(const WS& w, WarpCtx& cx, const QueryDev& Q, uint32_t q, uint32_t u, uint32_t e_beg,
                                             uint32_t e_end, const GroupSmem& gs, uint32_t cnt, bool interior) {
  const unsigned lane = lane_id();
  for (uint32_t e0 = e_beg; e0 < e_end; e0 += 64) {
    const uint32_t ea = e0 + lane, eb = ea + 32;
    const bool va = ea < e_end, vb = eb < e_end;
    int4 eda = make_int4(0, 0, 0, 0), edb = make_int4(0, 0, 0, 0);
    int2 pka = make_int2(0, 0), pkb = make_int2(0, 0);
    if (va) eda = __ldg(&Q.fwd_edge[ea]);
    if (vb) edb = __ldg(&Q.fwd_edge[eb]);
    if (interior) {
      if (va) pka = __ldg(&Q.fwd_peak[ea]);
      if (vb) pkb = __ldg(&Q.fwd_peak[eb]);
    }
    const uint32_t gxa = Q.base + (uint32_t)eda.x, gxb = Q.base + (uint32_t)edb.x;
    FDesc xa, xb;
    xa.d = make_uint4(0, 0, 0, 0);
    xa.last = make_longlong2(0, 0);
    xb = xa;
    if (va) xa = w.fdesc[gxa];
    if (vb) xb = w.fdesc[gxb];
    const uint32_t ma = va ? filter_run(w, Q, gs, cnt, eda, pka, interior, xa) : 0u;
    const uint32_t mb = vb ? filter_run(w, Q, gs, cnt, edb, pkb, interior, xb) : 0u;
    const uint32_t ra = (uint32_t)__popc(ma), rb = (uint32_t)__popc(mb);
    const uint32_t sa = ra ? atomicAdd(&w.cand_n[gxa], ra) : 0u;
    const uint32_t sb = rb ? atomicAdd(&w.cand_n[gxb], rb) : 0u;
    uint32_t oa = 0, ob = 0;
    slot_book(w, cx, q, gxa, ra, sa, &oa);
    if (__any_sync(kFull, vb)) slot_book(w, cx, q, gxb, rb, sb, &ob);
    write_run(w, Q, q, u, gs, ma, eda, gxa, sa, oa);
    write_run(w, Q, q, u, gs, mb, edb, gxb, sb, ob);
  }
}

// Large groups: one out-edge at a time, lanes on the group plans (a cost-sorted
// run of candidates per edge).
__device__ __forceinline__ void expand_plans(const WS& w, WarpCtx& cx, const QueryDev& Q, uint32_t q, uint32_t u, uint32_t e_beg,
                                             uint32_t e_end, const long long* gc, const long long* gh,
                                             const uint32_t* gp, uint32_t cnt, bool interior) {
  const unsigned lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  for (uint32_t e = e_beg; e < e_end; ++e) {
    const int4 ed = __ldg(&Q.fwd_edge[e]);
    int2 pk = make_int2(0, 0);
    if (interior) pk = __ldg(&Q.fwd_peak[e]);
    const uint32_t gx = Q.base + (uint32_t)ed.x;
    const FDesc xd = w.fdesc[gx];
    long long carry_h = 0;
    bool carry_ok = false;
    for (uint32_t j0 = 0; j0 < cnt; j0 += 32) {
      const uint32_t j = j0 + lane;
      bool ok = false;
      long long c = 0, h = 0;
      uint32_t pp = 0;
      if (j < cnt) {
        const long long ghj = gh[j];
        c = gc[j] + (long long)ed.y;
        const long long hh = ghj + (long long)ed.z;
        h = hh > (long long)ed.w ? hh : (long long)ed.w;
        pp = gp[j];
        long long peak = h;
        if (interior) {
          const long long hp = ghj + (long long)pk.x;
          peak = hp > (long long)pk.y ? hp : (long long)pk.y;
        }
        ok = peak <= Q.beta;
      }
      // run predecessor (the previous plan of the group along this edge)
      long long ph = shfl_up_i64(h, 1);
      bool pok = __shfl_up_sync(kFull, ok, 1);
      if (lane == 0) {
        ph = carry_h;
        pok = carry_ok;
      }
      carry_h = shfl_i64(h, 31);
      carry_ok = __shfl_sync(kFull, ok, 31);
      if (ok && pok && ph <= h) ok = false;
      uint32_t i0 = 0;
      if (ok && front_dominates(w, xd, &i0, c, h)) ok = false;
      const unsigned bal = __ballot_sync(kFull, ok);
      if (!bal) continue;
      const uint32_t r = (uint32_t)__popc(bal);
      // lane 0 takes the run's slots; the others follow it
      uint32_t s = 0, oi = 0;
      if (lane == 0) s = atomicAdd(&w.cand_n[gx], r);
      slot_book(w, cx, q, gx, lane == 0 ? r : 0u, s, &oi);
      s = __shfl_sync(kFull, s, 0);
      oi = __shfl_sync(kFull, oi, 0);
      if (ok) {
        const uint32_t k = (uint32_t)__popc(bal & lt);
        const uint32_t sk = s + k;
        // overflow index: the run's records before this one that overflowed
        uint32_t ok_i = oi + (sk >= kSlots ? sk - max(s, kSlots) : 0u);
        Cand cd;
        cd.cost = c;
        cd.h = h;
        cd.pp = pp;
        cd.tb = 1u + u;
        cd.g = 0;
        cd.i = 0;
        put_cand(w, Q, q, gx, sk, ok_i, cd);
      }
    }
  }
}

// Dynamic distribution of a phase's nodes over warps: a warp takes the next
// `chunk` list entries from the phase's counter (about 16 grabs per warp and
// phase), so warps that drew heavy nodes take fewer.
__device__ __forceinline__ uint32_t grab_chunk(uint32_t n_list, uint32_t warps) {
  return max(1u, n_list / (warps * 16u));
}
__device__ __forceinline__ uint32_t grab(uint32_t* ctr, uint32_t chunk) {
  uint32_t k = 0;
  if (lane_id() == 0) k = atomicAdd(ctr, chunk);
  return __shfl_sync(kFull, k, 0);
}

__device__ void phase_expand(const WS& w, WarpCtx& cx, GroupSmem& gs) {
  const unsigned lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t it = cx.it;
  const uint32_t n_list = ld_vol(&w.ctl->oh_n[it & 1]);
  const uint32_t lanes_from = w.ctl->lanes_from;
  const uint2* list = w.oh_list + (size_t)(it & 1) * w.NV;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t chunk = max(grab_chunk(n_list, warps), n_list / (warps * 4u));
  for (uint32_t k0 = grab(&w.ctl->grab[0], chunk); k0 < n_list; k0 = grab(&w.ctl->grab[0], chunk))
  for (uint32_t k = k0; k < min(k0 + chunk, n_list); ++k) {
    const uint2 gq = list[k];
    const uint32_t g = gq.x, q = gq.y;
    // the node's loads go out together, before the test of its query's state
    const QueryDev& Q = w.qd[q];
    const uint4 fd = w.fdesc[g].d;
    const uint32_t q_done = w.qs[q].done;
    const uint32_t u = g - Q.base;
    const uint32_t e_beg = __ldg(&Q.fwd_ptr[u]), e_end = __ldg(&Q.fwd_ptr[u + 1]);
    if (q_done) continue;
    const uint32_t n = fd.y;
    const size_t o = fd.x;
    const long long thr = (long long)it * Q.Lambda, thr2 = thr + Q.Lambda;
    uint32_t cnt = 0;
    bool rest = false, rgoal = false, global_group = false;
    uint32_t goff = 0;
    if (n <= 32) {
      uint32_t pid = 0;
      long long c = 0, hv = 0;
      if (lane < n) {
        pid = w.f_pid[o + lane];
        c = w.f_cost[o + lane];
        hv = w.f_h[o + lane];
      }
      const bool open = lane < n && (pid & kOpen);
      const bool isg = open && c <= thr;
      const unsigned gb = __ballot_sync(kFull, isg);
      cnt = (uint32_t)__popc(gb);
      rest = __any_sync(kFull, open && !isg);
      rgoal = __any_sync(kFull, open && !isg && c <= thr2);
      if (isg) {
        const uint32_t r = (uint32_t)__popc(gb & lt);
        gs.c[r] = c;
        gs.h[r] = hv;
        gs.p[r] = pid & kPidMask;
        w.f_pid[o + lane] = pid & ~kOpen;
      }
    } else {
      for (uint32_t j0 = 0; j0 < n; j0 += 32) {
        const uint32_t j = j0 + lane;
        uint32_t pid = 0;
        long long c = 0;
        if (j < n) {
          pid = w.f_pid[o + j];
          c = w.f_cost[o + j];
        }
        const bool open = j < n && (pid & kOpen);
        cnt += (uint32_t)__popc(__ballot_sync(kFull, open && c <= thr));
        rest = rest || __any_sync(kFull, open && c > thr);
        rgoal = rgoal || __any_sync(kFull, open && c > thr && c <= thr2);
      }
      if (cnt > 32) {
        if (lane == 0) goff = atomicAdd(&w.ctl->g_n, cnt);
        goff = __shfl_sync(kFull, goff, 0);
        global_group = true;
        if ((uint64_t)goff + cnt > w.gcap) {
          if (lane == 0) query_error(w, q, kErrGroup);
          cnt = 0;
        }
      }
      if (cnt) {
        uint32_t r0 = 0;
        for (uint32_t j0 = 0; j0 < n; j0 += 32) {
          const uint32_t j = j0 + lane;
          uint32_t pid = 0;
          long long c = 0;
          if (j < n) {
            pid = w.f_pid[o + j];
            c = w.f_cost[o + j];
          }
          const bool isg = j < n && (pid & kOpen) && c <= thr;
          const unsigned gb = __ballot_sync(kFull, isg);
          if (isg) {
            const uint32_t r = r0 + (uint32_t)__popc(gb & lt);
            if (global_group) {
              w.g_cost[goff + r] = c;
              w.g_h[goff + r] = w.f_h[o + j];
              w.g_pid[goff + r] = pid & kPidMask;
            } else {
              gs.c[r] = c;
              gs.h[r] = w.f_h[o + j];
              gs.p[r] = pid & kPidMask;
            }
            w.f_pid[o + j] = pid & ~kOpen;
          }
          r0 += (uint32_t)__popc(gb);
        }
      }
    }
    __syncwarp();
    if (lane == 0) {
      acc_open(w, cx, q, -(long long)cnt);
      acc_exps(w, cx, q, (unsigned long long)cnt * (e_end - e_beg));
      // one of the plans left open may be in the next group at a goal node
      // (the loop condition of the next iteration)
      if (rgoal && Q.is_goal[u]) w.qs[q].goal_next = 1u;
    }
    // plans left open keep the node on the open list (stamped: the merge of
    // this wavefront will not list it again)
    if (rest) {
      if (lane == 0) w.oh_stamp[g] = it + 1;
      push_next(w, cx, g, q);
    }
    if (cnt) {
      const bool interior = (Q.flags & MPAP_QUERY_CHECK_INTERIOR) != 0;
      if (!global_group && cnt < lanes_from)
        expand_edges(w, cx, Q, q, u, e_beg, e_end, gs, cnt, interior);
      else if (global_group)
        expand_plans(w, cx, Q, q, u, e_beg, e_end, w.g_cost + goff, w.g_h + goff, w.g_pid + goff, cnt, interior);
      else
        expand_plans(w, cx, Q, q, u, e_beg, e_end, gs.c, gs.h, gs.p, cnt, interior);
    }
    __syncwarp();
  }
  flush_next(w, cx);
  flush_merge(w, cx);
}

// ---------------------------------------------------------------------------
// Overflow regrouping (only in wavefronts where a node got more than kSlots
// candidates): every such node takes a contiguous segment of its query's
// second overflow share, then every overflow record moves to its node's
// segment.  The order inside a segment does not matter: the merge is a set
// function.
// ---------------------------------------------------------------------------
__device__ void phase_segments(const WS& w) {
  const uint32_t n_o = ld_vol(&w.ctl->ovl_n);
  const uint32_t nt = gridDim.x * blockDim.x;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n_o; k += nt) {
    const uint2 gq = w.ovl[k];
    const uint32_t nc = w.cand_n[gq.x];
    if (nc <= kSlots) continue;
    const QueryDev& Q = w.qd[gq.y];
    const uint32_t need = nc - kSlots;
    const uint32_t off = atomicAdd(&w.qs[gq.y].seg_n, need);
    if ((uint64_t)off + need > Q.ov_cap) {
      w.segoff[gq.x] = kNone;
      query_error(w, gq.y, kErrList);
    } else {
      w.segoff[gq.x] = (uint32_t)(Q.ov_base + off);
    }
  }
}

__device__ void phase_scatter(const WS& w) {
  const uint32_t nq = w.ctl->nq;
  const uint32_t total = ld_vol(&w.ctl->ov_total);
  const uint32_t nt = gridDim.x * blockDim.x;
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < total; r += nt) {
    // the query of record r: last q with ov_pref[q] <= r
    uint32_t lo = 0, hi = nq;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (w.ov_pref[mid] <= r) lo = mid; else hi = mid;
    }
    const QueryDev& Q = w.qd[lo];
    const Cand cd = w.ov[Q.ov_base + (r - w.ov_pref[lo])];
    const uint32_t so = w.segoff[cd.g];
    if (so != kNone) w.ov2[(size_t)so + cd.i] = cd;
  }
}

// One-pass merge of a register front with few candidates (front + candidates
// <= 32): the front's entries (lanes 0..n-1, tie key 0: older than any
// candidate) and the candidates (lanes n..n+nc-1, cc/ch/ctb/cpp of this lane)
// are sorted together by (cost, h, tie key) over the smallest power-of-two
// width that holds them; an item survives iff its h is below every h before it
// (the weak Pareto order with the tie key).  The new front is left in
// registers, lane j holding entry j.
__device__ __forceinline__ void merge_small(FrontCursor& fc, WarpSmem& sm, uint32_t nc, long long cc, long long ch,
                                            uint32_t ctb, uint32_t cpp) {
  const unsigned lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t n = fc.n, t = n + nc;
  const bool isf = lane < n, isc = lane >= n && lane < t;
  long long kc = isf ? fc.rc : (isc ? cc : LLONG_MAX);
  const long long vh = isf ? fc.rh : (isc ? ch : LLONG_MAX);
  const uint32_t vt = isf ? 0u : (isc ? ctb : 0xFFFFFFFFu);
  const uint32_t vp = isf ? fc.rp : (isc ? (cpp | kNew) : 0u);
  const uint32_t va = isf ? fc.ra : (isc ? ctb : 0u);
  uint32_t W = 2;
  while (W < t) W <<= 1;
  // 1. sort on (cost, source lane) within segments of W lanes
  uint32_t ks = lane;
  for (uint32_t k = 2; k <= W; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      const long long oc = shfl_xor_i64(kc, (int)j);
      const uint32_t os = __shfl_xor_sync(kFull, ks, (int)j);
      const bool up = (lane & k) == 0;
      const bool lower = (lane & j) == 0;
      const bool o_less = oc < kc || (oc == kc && os < ks);
      if ((lower == up) ? o_less : !o_less) {
        kc = oc;
        ks = os;
      }
    }
  }
  long long kh = shfl_i64(vh, (int)ks);
  uint32_t kt = __shfl_sync(kFull, vt, (int)ks);
  uint32_t kp = __shfl_sync(kFull, vp, (int)ks);
  uint32_t ka = __shfl_sync(kFull, va, (int)ks);
  // 2. equal costs must be ordered by (h, tie key) too (rare): sort again on the full key
  {
    const long long pc = shfl_up_i64(kc, 1);
    if (__any_sync(kFull, lane > 0 && kt != 0xFFFFFFFFu && pc == kc)) {
      for (uint32_t k = 2; k <= W; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
          const long long oc = shfl_xor_i64(kc, (int)j), oh = shfl_xor_i64(kh, (int)j);
          const uint32_t ot = __shfl_xor_sync(kFull, kt, (int)j), op = __shfl_xor_sync(kFull, kp, (int)j);
          const uint32_t oa = __shfl_xor_sync(kFull, ka, (int)j);
          const bool up = (lane & k) == 0;
          const bool lower = (lane & j) == 0;
          const bool o_less = key_less(oc, oh, ot, kc, kh, kt);
          const bool m_less = key_less(kc, kh, kt, oc, oh, ot);
          if ((lower == up) ? o_less : m_less) {
            kc = oc;
            kh = oh;
            kt = ot;
            kp = op;
            ka = oa;
          }
        }
      }
    }
  }
  // 3. skyline: exclusive prefix minimum of h in sorted order
  long long pm = kh;
  for (uint32_t o = 1; o < W; o <<= 1) {
    const long long x = shfl_up_i64(pm, (int)o);
    if (lane >= o && x < pm) pm = x;
  }
  long long excl = shfl_up_i64(pm, 1);
  if (lane == 0) excl = LLONG_MAX;
  const bool valid = lane < W && kt != 0xFFFFFFFFu;
  const bool surv = valid && kh < excl;
  const unsigned sb = __ballot_sync(kFull, surv);
  fc.removed_open += (uint32_t)__popc(__ballot_sync(kFull, valid && !surv && kt == 0u && (kp & kOpen)));
  fc.any_new = fc.any_new || __any_sync(kFull, surv && (kp & kNew));
  if (surv) {
    const uint32_t r = (uint32_t)__popc(sb & lt);
    sm.st_cost[r] = kc;
    sm.st_h[r] = kh;
    sm.st_pid[r] = kp;
    sm.st_aux[r] = ka;
  }
  __syncwarp();
  fc.n = (uint32_t)__popc(sb);
  if (lane < fc.n) {
    fc.rc = sm.st_cost[lane];
    fc.rh = sm.st_h[lane];
    fc.rp = sm.st_pid[lane];
    fc.ra = sm.st_aux[lane];
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// Merge (RemoveDominated, Sec. 3, for every node that received candidates).
// ---------------------------------------------------------------------------
// Bulk merge of a node's nc candidates (many) into its front, linear in the
// front's size: the candidates' own skyline S is built in this wavefront's
// scratch, 32 candidates at a time (each chunk filtered against S, reduced to
// its skyline and merged into S between two scratch regions); then one sweep
// over the front keeps the entries no survivor dominates and interleaves the
// survivors (no survivor is dominated by the front: the expansion dropped those).
// O(nc / 32 |S| / 32 + n / 32 + |S| log n / 32) warp steps instead of
// O(nc / 32 n / 32).  Returns false, changing nothing, when the scratch is
// used up; the caller then merges in chunks.
template <class Load>
__device__ bool merge_bulk(const WS& w, uint32_t q, FrontCursor& fc, WarpSmem& sm, uint32_t nc, Load load) {
  const unsigned lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  unsigned long long T = 0;
  if (lane == 0) T = atomicAdd(&w.ctl->tmp_n, 2ull * nc);
  T = __shfl_sync(kFull, T, 0);
  if (T + 2ull * nc > w.tcap) return false;
  size_t A = T, B = T + nc;
  uint32_t sn = 0;
  for (uint32_t c0 = 0; c0 < nc; c0 += 32) {
    long long cc = 0, ch = 0;
    uint32_t tb = 0, pp = 0;
    bool ok = c0 + lane < nc && load(c0 + lane, cc, ch, tb, pp);
    // 1. candidates dominated by the skyline so far (its last entry of cost <= cc)
    if (ok && sn) {
      uint32_t L = 0, R = sn;
      while (L < R) {
        const uint32_t mid = (L + R) >> 1;
        if (w.t_cost[A + mid] <= cc) L = mid + 1; else R = mid;
      }
      if (L > 0) {
        const long long sc = w.t_cost[A + L - 1], sh = w.t_h[A + L - 1];
        if (sh <= ch && (sc < cc || sh < ch || w.t_tb[A + L - 1] < tb)) ok = false;
      }
    }
    if (!__any_sync(kFull, ok)) continue;
    // 2. skyline of the chunk (sorted, in sm.s_*)
    const uint32_t m = chunk_skyline(sm, ok, cc, ch, tb, pp);
    sm.bins[lane] = 0;
    if (lane == 0) sm.bins[32] = 0;
    __syncwarp();
    // 3. S entries dominated by a chunk survivor drop out; the rest go to B at
    //    (kept rank + chunk survivors before them)
    uint32_t kept = 0;
    for (uint32_t j0 = 0; j0 < sn; j0 += 32) {
      const uint32_t j = j0 + lane;
      const bool valid = j < sn;
      long long fcost = 0, fh = 0;
      uint32_t fpp = 0, ftb = 0;
      if (valid) {
        fcost = w.t_cost[A + j];
        fh = w.t_h[A + j];
        fpp = w.t_pp[A + j];
        ftb = w.t_tb[A + j];
      }
      uint32_t L = 0, R = m;
      while (L < R) {
        const uint32_t mid = (L + R) >> 1;
        if (sm.s_cost[mid] <= fcost) L = mid + 1; else R = mid;
      }
      bool dom = false;
      if (valid && L > 0) {
        const long long scost = sm.s_cost[L - 1], sh = sm.s_h[L - 1];
        dom = sh <= fh && (scost < fcost || sh < fh || sm.s_tb[L - 1] < ftb);
      }
      const bool keep = valid && !dom;
      const unsigned kb = __ballot_sync(kFull, keep);
      if (keep) {
        const size_t pos = B + kept + __popc(kb & lt) + L;
        w.t_cost[pos] = fcost;
        w.t_h[pos] = fh;
        w.t_pp[pos] = fpp;
        w.t_tb[pos] = ftb;
        atomicAdd(&sm.bins[L], 1u);
      }
      kept += __popc(kb);
    }
    __syncwarp();
    const uint32_t before = warp_incl_scan(lane < m ? sm.bins[lane] : 0u);
    if (lane < m) {
      const size_t pos = B + lane + before;
      w.t_cost[pos] = sm.s_cost[lane];
      w.t_h[pos] = sm.s_h[lane];
      w.t_pp[pos] = sm.s_pp[lane];
      w.t_tb[pos] = sm.s_tb[lane];
    }
    __syncwarp();
    const size_t t = A;
    A = B;
    B = t;
    sn = kept + m;
  }
  if (sn == 0) return true;
  const size_t o = fc.off;
  const uint32_t n = fc.n;
  // 4. insertion index of every survivor: front entries of lower or equal cost
  for (uint32_t s0 = 0; s0 < sn; s0 += 32) {
    const uint32_t s = s0 + lane;
    if (s < sn) {
      const long long sc = w.t_cost[A + s];
      uint32_t L = 0, R = n;
      while (L < R) {
        const uint32_t mid = (L + R) >> 1;
        if (w.f_cost[o + mid] <= sc) L = mid + 1; else R = mid;
      }
      w.t_m[A + s] = L;
    }
  }
  if (!ensure_other(w, q, fc, n + sn)) return true;
  __syncwarp();
  // 5. one sweep over the front
  const size_t on = fc.off2;
  uint32_t K = 0, sp = 0, rem_open = 0;
  for (uint32_t j0 = 0; j0 < n; j0 += 32) {
    const uint32_t j = j0 + lane;
    const bool valid = j < n;
    long long fcost = 0, fh = 0;
    uint32_t fpid = 0, faux = 0;
    if (valid) {
      fcost = w.f_cost[o + j];
      fh = w.f_h[o + j];
      fpid = w.f_pid[o + j];
      faux = w.f_aux[o + j];
    }
    // survivors of lower or equal cost; the last of them alone can dominate (old plans win ties)
    uint32_t lo = 0, hi = sn;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (w.t_cost[A + mid] <= fcost) lo = mid + 1; else hi = mid;
    }
    bool dom = false;
    if (valid && lo > 0) {
      const long long sc = w.t_cost[A + lo - 1], sh = w.t_h[A + lo - 1];
      dom = sh <= fh && (sc < fcost || sh < fh);
    }
    const bool keep = valid && !dom;
    if (dom && (fpid & kOpen)) rem_open++;
    const unsigned kb = __ballot_sync(kFull, keep);
    if (keep) {
      const size_t pos = on + K + __popc(kb & lt) + lo;
      w.f_cost[pos] = fcost;
      w.f_h[pos] = fh;
      w.f_pid[pos] = fpid;
      w.f_aux[pos] = faux;
    }
    // survivors that go before a front entry of this chunk
    const uint32_t jend = min(j0 + 32u, n);
    for (;;) {
      const uint32_t s = sp + lane;
      bool emit = false;
      uint32_t mm = 0;
      if (s < sn) {
        mm = w.t_m[A + s];
        emit = mm < jend;
      }
      const unsigned eb = __ballot_sync(kFull, emit);
      if (emit) {
        const uint32_t d = mm - j0;   // 0 .. 31: earlier chunks emitted every index below j0
        const size_t pos = on + s + K + __popc(kb & ((1u << d) - 1u));
        w.f_cost[pos] = w.t_cost[A + s];
        w.f_h[pos] = w.t_h[A + s];
        w.f_pid[pos] = w.t_pp[A + s] | kNew;
        w.f_aux[pos] = w.t_tb[A + s];
      }
      const uint32_t c = __popc(eb);
      sp += c;
      if (c < 32) break;
    }
    K += __popc(kb);
  }
  // survivors after every front entry
  for (uint32_t s0 = sp; s0 < sn; s0 += 32) {
    const uint32_t s = s0 + lane;
    if (s < sn) {
      const size_t pos = on + s + K;
      w.f_cost[pos] = w.t_cost[A + s];
      w.f_h[pos] = w.t_h[A + s];
      w.f_pid[pos] = w.t_pp[A + s] | kNew;
      w.f_aux[pos] = w.t_tb[A + s];
    }
  }
  for (int sft = 16; sft > 0; sft >>= 1) rem_open += __shfl_xor_sync(kFull, rem_open, sft);
  fc.removed_open += rem_open;
  swap_blocks(fc);
  fc.n = K + sn;
  fc.reg = false;
  fc.any_new = true;
  __syncwarp();
  return true;
}

// ---------------------------------------------------------------------------
// Grid-wide merge of huge nodes (RemoveDominated for a node whose front and
// candidates together hold at least ctl->huge_from entries, 2048 by default).  One warp would take time
// linear in the front, or worse, and hold every other block at the next
// barrier; instead every warp of the grid takes part.  The node's members
// (front entries, tie key 0, and candidates) are bucketed by cost into nb
// buckets of equal width.  A member is dominated by a member of a lower bucket
// (strictly lower cost) iff the minimum h over all lower buckets is at most its
// own, which an exclusive prefix minimum over the buckets gives; and by a member
// of its own bucket iff one before it in the (cost, h, tie key) order has an h
// at most its own.  Domination is transitive, so testing against every member,
// dominated or not, is exact.  The survivors of each bucket are counted, and an
// exclusive prefix sum over the buckets places them in the new front in cost
// order.  Every step is a grid-stride loop over members or over tiles of kTile
// buckets (a warp each); grid barriers separate the steps.
// ---------------------------------------------------------------------------

// Hands node g to this wavefront's grid-wide merge (warp-collective).  False,
// with nothing changed that the caller relies on, when the merge has no room
// left: the caller then merges the node itself.
__device__ __forceinline__ bool defer_huge(const WS& w, uint32_t g, uint32_t q, const FrontCursor& fc,
                                           uint32_t nc, uint32_t so) {
  uint32_t ok = 0;
  if (lane_id() == 0) {
    const uint32_t N = fc.n + nc;
    const uint32_t nb = max(kTile, 1u << ceil_lg(N));
    Ctl* c = w.ctl;
    uint32_t idx = kNone;
    unsigned long long T = 0;
    if (atomicAdd(&c->hg_ents, (unsigned long long)N) + N <= (1ull << 31)) {
      T = atomicAdd(&c->tmp_n, (unsigned long long)N + nb);
      if (T + N + nb <= w.tcap) {
        idx = atomicAdd(&c->hg_n, 1u);
        if (idx >= kHugeMax) idx = kNone;
      }
    }
    if (idx != kNone) {
      HugeDesc d;
      d.g = g;
      d.q = q;
      d.n = fc.n;
      d.nc = nc;
      d.off = fc.off;
      d.so = so;
      d.lg_old = fc.lg;
      d.out = fc.off2;      // the merged front goes to the node's other block, grown
      d.lg_out = fc.lg2;    // once the survivors are counted if it is too small
      d.ok = 1;
      d.nb = nb;
      d.shift = 0;
      d.ent0 = 0;
      d.tile0 = 0;
      d.mem = T;
      d.bkt = T + N;
      d.lo = fc.n ? w.f_cost[fc.off] : LLONG_MAX;
      d.hi = fc.n ? w.f_cost[(size_t)fc.off + fc.n - 1] : LLONG_MIN;
      d.n_out = 0;
      d.n_new = 0;
      d.removed_open = 0;
      d.pad = 0;
      w.hg[idx] = d;
      ok = 1;
    }
  }
  return __shfl_sync(kFull, ok, 0) != 0;
}

// One node's merge with the whole warp (any front and candidate count).
__device__ __forceinline__ void merge_node(const WS& w, WarpCtx& cx, WarpSmem& sm, const uint2 gq) {
  const unsigned lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t it = cx.it;
  {
    const uint32_t g = gq.x, q = gq.y;
    const QueryDev& Q = w.qd[q];
    const uint32_t x = g - Q.base;
    const uint32_t nc = w.cand_n[g];
    const uint32_t so = nc > kSlots ? w.segoff[g] : 0u;
    const bool listed = w.oh_stamp[g] == it + 1;   // kept on the open list by the expansion
    FrontCursor fc;
    {
      const uint4 fd = w.fdesc[g].d;
      fc.off = fd.x;
      fc.n = fd.y;
      fc.off2 = fd.z;
      fc.lg = fd.w & 0xFFu;
      fc.lg2 = (fd.w >> 8) & 0xFFu;
    }
    // huge nodes are merged by the whole grid after this phase
    if (nc && fc.n + nc >= cx.huge_from && fc.n + nc <= (1u << 30) && defer_huge(w, g, q, fc, nc, so)) return;
    fc.err = false;
    fc.removed_open = 0;
    fc.any_new = false;
    fc.reg = fc.n <= 32;
    fc.rc = fc.rh = 0;
    fc.rp = fc.ra = 0;
    if (fc.reg && lane < fc.n) {
      const size_t o = fc.off;
      fc.rc = w.f_cost[o + lane];
      fc.rh = w.f_h[o + lane];
      fc.rp = w.f_pid[o + lane];
      fc.ra = w.f_aux[o + lane];
    }
    // candidate i of this node: an inline slot or its regrouped overflow
    auto load = [&](uint32_t i, long long& cc, long long& ch, uint32_t& tb, uint32_t& pp) -> bool {
      const Cand* src = nullptr;
      if (i < kSlots) src = &w.slot[(size_t)g * kSlots + i];
      else if (so != kNone) src = &w.ov2[(size_t)so + (i - kSlots)];
      if (!src) return false;
      const Cand cd = *src;
      cc = cd.cost;
      ch = cd.h;
      tb = cd.tb;
      pp = cd.pp;
      return true;
    };
    if (fc.reg && fc.n + nc <= 32) {
      long long cc = 0, ch = 0;
      uint32_t tb = 0, pp = 0;
      if (lane >= fc.n && lane < fc.n + nc) load(lane - fc.n, cc, ch, tb, pp);
      merge_small(fc, sm, nc, cc, ch, tb, pp);
    } else {
      // many candidates into a front that does not fit a warp: linear bulk merge
      // (chunks of 32 against the whole front when its scratch is used up)
      const bool bulk = nc > 32 && fc.n + nc > 64 && merge_bulk(w, q, fc, sm, nc, load);
      for (uint32_t c0 = 0; !bulk && c0 < nc && !fc.err; c0 += 32) {
        const uint32_t i = c0 + lane;
        bool ok = false;
        long long cc = 0, ch = 0;
        uint32_t tb = 0, pp = 0;
        if (i < nc) ok = load(i, cc, ch, tb, pp);
        if (fc.reg) merge_chunk_reg(w, q, fc, sm, ok, cc, ch, tb, pp);
        else merge_chunk_slab(w, q, fc, sm, ok, cc, ch, tb, pp);
      }
    }
    if (fc.any_new && !fc.err && fc.reg && (fc.lg == 0 || (1u << fc.lg) < fc.n)) {
      // the register front needs a (larger) live block to be written back to
      const uint32_t lg = max(kMinLg, ceil_lg(fc.n));
      uint32_t o = 0;
      if (lane == 0) o = pool_alloc(w, q, lg);
      o = __shfl_sync(kFull, o, 0);
      if (o == kNoBlock) {
        if (lane == 0) query_error(w, q, kErrFront);
        fc.err = true;
      } else {
        fc.off = o;
        fc.lg = lg;
      }
    }
    if (fc.any_new && !fc.err) {
      // give every new front entry an arena record and mark it open
      uint32_t n_new = 0;
      const long long thr2 = (long long)(it + 1) * Q.Lambda;
      bool gnext = false;
      if (fc.reg) {
        const bool isnew = lane < fc.n && (fc.rp & kNew);
        const unsigned bal = __ballot_sync(kFull, isnew);
        uint32_t a0 = kNone;
        if (lane == 0 && bal) a0 = arena_take(w, q, (uint32_t)__popc(bal));
        a0 = __shfl_sync(kFull, a0, 0);
        if (isnew) {
          if (a0 != kNone) {
            const uint32_t a = a0 + (uint32_t)__popc(bal & lt);
            w.a_head[a] = x;
            w.a_parent[a] = fc.rp & kPidMask;
            w.a_iter[a] = it + 1;
            w.a_cost[a] = fc.rc;
            fc.rp = a | kOpen;
          } else {
            fc.rp = kOpen;
          }
          fc.ra = 0;
        }
        n_new = (uint32_t)__popc(bal);
        // write the register front to the live block
        const size_t o = fc.off;
        if (lane < fc.n) {
          w.f_cost[o + lane] = fc.rc;
          w.f_h[o + lane] = fc.rh;
          w.f_pid[o + lane] = fc.rp;
          w.f_aux[o + lane] = fc.ra;
        }
        gnext = __any_sync(kFull, lane < fc.n && (fc.rp & kOpen) && fc.rc <= thr2);
      } else {
        n_new = arena_block(w, q, x, it, fc);
        for (uint32_t j0 = 0; j0 < fc.n; j0 += 32) {
          const uint32_t j = j0 + lane;
          const bool hit = j < fc.n && (w.f_pid[(size_t)fc.off + j] & kOpen) && w.f_cost[(size_t)fc.off + j] <= thr2;
          gnext = gnext || __any_sync(kFull, hit);
        }
      }
      long long lc, lh;
      if (fc.reg) {
        lc = shfl_i64(fc.rc, (int)fc.n - 1);
        lh = shfl_i64(fc.rh, (int)fc.n - 1);
      } else {
        lc = w.f_cost[(size_t)fc.off + fc.n - 1];
        lh = w.f_h[(size_t)fc.off + fc.n - 1];
      }
      commit_tail(w, cx, q, g, fc, n_new, lc, lh, listed);
      // an open plan of the next group at a goal node ends the query at the
      // top of the next iteration (the loop condition of Alg. 3)
      if (lane == 0 && gnext && Q.is_goal[x]) w.qs[q].goal_next = 1u;
    }
    if (lane == 0) w.cand_n[g] = 0;
  }
}

__device__ __forceinline__ long long shfl16_i64(long long v, uint32_t src) {
  return __shfl_sync(kFull, v, (int)src, 16);
}

// Two small merges at once, one per half-warp: lanes 16 s .. 16 s + 15 serve
// node gq of half s, whose front (n entries) and candidates (nc) fit 16 lanes
// together.  Within each half the one-pass merge of merge_small: sort (cost, h,
// tie key), keep the strict prefix minimum of h; then each half commits its
// node (pool block, arena records, descriptor, counters, next open list).
__device__ __forceinline__ void merge_pair16(const WS& w, WarpCtx& cx, WarpSmem& sm, const uint2 gq, const uint4 fd,
                                             uint32_t nc) {
  const unsigned lane = lane_id();
  const unsigned sl = lane & 15u, hb = lane & 16u;
  const unsigned llt = (1u << sl) - 1u;
  const uint32_t it = cx.it;
  const uint32_t g = gq.x, q = gq.y;
  const QueryDev& Q = w.qd[q];
  const uint32_t x = g - Q.base;
  const uint32_t n = fd.y, t = n + nc;
  const bool listed = w.oh_stamp[g] == it + 1;   // kept on the open list by the expansion
  const bool isf = sl < n, isc = sl >= n && sl < t;
  long long kc = LLONG_MAX, vh = LLONG_MAX;
  uint32_t vt = 0xFFFFFFFFu, vp = 0u, va = 0u;
  if (isf) {
    const size_t o = (size_t)fd.x + sl;
    kc = w.f_cost[o];
    vh = w.f_h[o];
    vp = w.f_pid[o];
    va = w.f_aux[o];
    vt = 0u;
  } else if (isc) {
    const Cand cd = w.slot[(size_t)g * kSlots + (sl - n)];
    kc = cd.cost;
    vh = cd.h;
    vt = cd.tb;
    vp = cd.pp | kNew;
    va = cd.tb;
  }
  uint32_t W = 2;
  const uint32_t tm = max(t, (uint32_t)__shfl_xor_sync(kFull, t, 16));
  while (W < tm) W <<= 1;
  // 1. sort on (cost, source lane) within each half (W <= 16 keeps every
  //    exchange inside its half)
  uint32_t ks = sl;
  for (uint32_t k = 2; k <= W; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      const long long oc = shfl_xor_i64(kc, (int)j);
      const uint32_t os = __shfl_xor_sync(kFull, ks, (int)j);
      const bool up = (sl & k) == 0;
      const bool lower = (sl & j) == 0;
      const bool o_less = oc < kc || (oc == kc && os < ks);
      if ((lower == up) ? o_less : !o_less) {
        kc = oc;
        ks = os;
      }
    }
  }
  long long kh = shfl16_i64(vh, ks);
  uint32_t kt = __shfl_sync(kFull, vt, (int)ks, 16);
  uint32_t kp = __shfl_sync(kFull, vp, (int)ks, 16);
  uint32_t ka = __shfl_sync(kFull, va, (int)ks, 16);
  // 2. equal costs: sort again on the full key (rare)
  {
    const long long pc = __shfl_up_sync(kFull, kc, 1, 16);
    if (__any_sync(kFull, sl > 0 && kt != 0xFFFFFFFFu && pc == kc)) {
      for (uint32_t k = 2; k <= W; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
          const long long oc = shfl_xor_i64(kc, (int)j), oh = shfl_xor_i64(kh, (int)j);
          const uint32_t ot = __shfl_xor_sync(kFull, kt, (int)j), op = __shfl_xor_sync(kFull, kp, (int)j);
          const uint32_t oa = __shfl_xor_sync(kFull, ka, (int)j);
          const bool up = (sl & k) == 0;
          const bool lower = (sl & j) == 0;
          const bool o_less = key_less(oc, oh, ot, kc, kh, kt);
          const bool m_less = key_less(kc, kh, kt, oc, oh, ot);
          if ((lower == up) ? o_less : m_less) {
            kc = oc;
            kh = oh;
            kt = ot;
            kp = op;
            ka = oa;
          }
        }
      }
    }
  }
  // 3. skyline within the half
  long long pm = kh;
  for (uint32_t o = 1; o < W; o <<= 1) {
    const long long y = __shfl_up_sync(kFull, pm, o, 16);
    if (sl >= o && y < pm) pm = y;
  }
  long long excl = __shfl_up_sync(kFull, pm, 1, 16);
  if (sl == 0) excl = LLONG_MAX;
  const bool valid = sl < W && kt != 0xFFFFFFFFu;
  const bool surv = valid && kh < excl;
  const uint32_t my = (__ballot_sync(kFull, surv) >> hb) & 0xFFFFu;
  const uint32_t removed =
      (uint32_t)__popc((__ballot_sync(kFull, valid && !surv && kt == 0u && (kp & kOpen)) >> hb) & 0xFFFFu);
  const bool any_new = ((__ballot_sync(kFull, surv && (kp & kNew)) >> hb) & 0xFFFFu) != 0u;
  if (surv) {
    const uint32_t r = hb + (uint32_t)__popc(my & llt);
    sm.st_cost[r] = kc;
    sm.st_h[r] = kh;
    sm.st_pid[r] = kp;
    sm.st_aux[r] = ka;
  }
  __syncwarp();
  const uint32_t nn = (uint32_t)__popc(my);
  long long rc = 0, rh = 0;
  uint32_t rp = 0;
  if (sl < nn) {
    rc = sm.st_cost[hb + sl];
    rh = sm.st_h[hb + sl];
    rp = sm.st_pid[hb + sl];
  }
  __syncwarp();
  // 4. commit, per half
  uint32_t off = fd.x, lg = fd.w & 0xFFu;
  const uint32_t off2 = fd.z, lg2 = (fd.w >> 8) & 0xFFu;
  bool ok = any_new;
  {
    const bool need = ok && (lg == 0 || (1u << lg) < nn);
    const uint32_t nlg = max(kMinLg, ceil_lg(nn));
    uint32_t o = 0;
    if (need && sl == 0) o = pool_alloc(w, q, nlg);
    o = __shfl_sync(kFull, o, (int)hb);
    if (need) {
      if (o == kNoBlock) {
        if (sl == 0) query_error(w, q, kErrFront);
        ok = false;
      } else {
        off = o;
        lg = nlg;
      }
    }
  }
  const bool isnew = ok && sl < nn && (rp & kNew);
  const uint32_t bal = (__ballot_sync(kFull, isnew) >> hb) & 0xFFFFu;
  uint32_t a0 = kNone;
  if (sl == 0 && bal) a0 = arena_take(w, q, (uint32_t)__popc(bal));
  a0 = __shfl_sync(kFull, a0, (int)hb);
  if (isnew) {
    if (a0 != kNone) {
      const uint32_t a = a0 + (uint32_t)__popc(bal & llt);
      w.a_head[a] = x;
      w.a_parent[a] = rp & kPidMask;
      w.a_iter[a] = it + 1;
      w.a_cost[a] = rc;
      rp = a | kOpen;
    } else {
      rp = kOpen;
    }
  }
  if (ok && sl < nn) {
    const size_t o = (size_t)off + sl;
    w.f_cost[o] = rc;
    w.f_h[o] = rh;
    w.f_pid[o] = rp;
    w.f_aux[o] = 0u;
  }
  const long long thr2 = (long long)(it + 1) * Q.Lambda;
  const bool gnext = ((__ballot_sync(kFull, ok && sl < nn && (rp & kOpen) && rc <= thr2) >> hb) & 0xFFFFu) != 0u;
  const long long lc = __shfl_sync(kFull, rc, (int)(hb + (nn ? nn - 1 : 0)));
  const long long lh = __shfl_sync(kFull, rh, (int)(hb + (nn ? nn - 1 : 0)));
  if (sl == 0) {
    if (ok) {
      FDesc d;
      d.d = make_uint4(off, nn, off2, lg | (lg2 << 8));
      d.last = make_longlong2(lc, lh);
      w.fdesc[g] = d;
      const uint32_t n_new = (uint32_t)__popc(bal);
      acc_open(w, cx, q, (long long)n_new - (long long)removed);
      acc_plans(w, cx, q, n_new);
      if (nn > ld_vol(&w.ctl->max_front)) atomicMax(&w.ctl->max_front, nn);
      if (gnext && Q.is_goal[x]) w.qs[q].goal_next = 1u;
    }
    w.cand_n[g] = 0;
  }
  // both halves' nodes to the next open list (warp-uniform calls)
  for (uint32_t h = 0; h < 32; h += 16) {
    const bool pk = __shfl_sync(kFull, ok && !listed, (int)h);
    const uint32_t pg = __shfl_sync(kFull, g, (int)h), pq = __shfl_sync(kFull, q, (int)h);
    if (pk) push_next(w, cx, pg, pq);
  }
}

__device__ void phase_merge(const WS& w, WarpCtx& cx, WarpSmem& sm) {
  const uint32_t n_m = ld_vol(&w.ctl->m_n);
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t chunk = max(2u, grab_chunk(n_m, warps));
  const unsigned half = lane_id() >> 4;
  for (uint32_t k0 = grab(&w.ctl->grab[1], chunk); k0 < n_m; k0 = grab(&w.ctl->grab[1], chunk)) {
    const uint32_t k1 = min(k0 + chunk, n_m);
    uint32_t k = k0;
    while (k < k1) {
      if (k + 1 < k1) {
        // two nodes whose fronts and candidates fit half a warp each go together
        const uint2 gq = w.m_list[k + half];
        const uint32_t nc = w.cand_n[gq.x];
        const uint4 fd = w.fdesc[gq.x].d;
        if (__all_sync(kFull, fd.y <= 16u && fd.y + nc <= 16u)) {
          merge_pair16(w, cx, sm, gq, fd, nc);
          k += 2;
          continue;
        }
      }
      merge_node(w, cx, sm, w.m_list[k]);
      ++k;
    }
  }
  flush_next(w, cx);
}

// Steps of the grid-wide merge (whole grid unless noted).
constexpr uint32_t kSurv = 0x80000000u;   // survivor mark on a placed member's tie key

__device__ __forceinline__ uint32_t gwarp() { return (blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ uint32_t nwarps() { return (gridDim.x * blockDim.x) >> 5; }

// The huge node holding flat member (tiles: tile) index x: the last one whose
// first index is <= x (skipped nodes hold no index).
__device__ __forceinline__ uint32_t huge_find(const WS& w, uint32_t nh, uint32_t x, bool tiles) {
  uint32_t lo = 0, hi = nh;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if ((tiles ? w.hg[mid].tile0 : w.hg[mid].ent0) <= x) lo = mid; else hi = mid;
  }
  return lo;
}

struct Member {
  long long c, h;
  uint32_t p, tb;   // pid (front entries) or parent plan (candidates); tie key
};

// Member i of huge node d: front entry i (tie key 0: older than any candidate)
// or candidate i - n; false when the candidate's record was lost to a full
// overflow share (its query has failed).
__device__ __forceinline__ bool huge_member(const WS& w, const HugeDesc& d, uint32_t i, Member& m) {
  if (i < d.n) {
    const size_t o = (size_t)d.off + i;
    m.c = w.f_cost[o];
    m.h = w.f_h[o];
    m.p = w.f_pid[o];
    m.tb = 0;
    return true;
  }
  const uint32_t k = i - d.n;
  const Cand* src;
  if (k < kSlots) src = &w.slot[(size_t)d.g * kSlots + k];
  else if (d.so != kNone) src = &w.ov2[(size_t)d.so + (k - kSlots)];
  else return false;
  const Cand cd = *src;
  m.c = cd.cost;
  m.h = cd.h;
  m.p = cd.pp;
  m.tb = cd.tb;
  return true;
}

__device__ __forceinline__ size_t huge_bucket(const HugeDesc& d, long long c) {
  return (size_t)d.bkt + (size_t)((unsigned long long)(c - d.lo) >> d.shift);
}

// Barrier after the merges, last block (all its threads): flat member and tile
// numbering of the huge nodes, an exclusive prefix sum over them (each thread
// sums a contiguous run of nodes, the runs' totals are scanned in order).
__device__ void huge_setup(const WS& w) {
  __shared__ uint32_t s_m[kWarpsPerBlock * 32], s_t[kWarpsPerBlock * 32];
  Ctl* c = w.ctl;
  const uint32_t nh = min(c->hg_n, kHugeMax);
  const uint32_t nt_ = blockDim.x;
  const uint32_t per = (nh + nt_ - 1) / nt_;
  const uint32_t k0 = min(nh, threadIdx.x * per), k1 = min(nh, k0 + per);
  uint32_t m = 0, t = 0;
  for (uint32_t k = k0; k < k1; ++k) {
    const HugeDesc& d = w.hg[k];
    if (d.ok) {
      m += d.n + d.nc;
      t += d.nb / kTile;
    }
  }
  s_m[threadIdx.x] = m;
  s_t[threadIdx.x] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t am = 0, at = 0;
    for (uint32_t i = 0; i < nt_; ++i) {
      const uint32_t a = s_m[i], b = s_t[i];
      s_m[i] = am;
      s_t[i] = at;
      am += a;
      at += b;
    }
    c->hg_nm = am;
    c->hg_nt = at;
    c->hg_live = 1;
  }
  __syncthreads();
  m = s_m[threadIdx.x];
  t = s_t[threadIdx.x];
  for (uint32_t k = k0; k < k1; ++k) {
    HugeDesc& d = w.hg[k];
    d.ent0 = m;
    d.tile0 = t;
    if (d.ok) {
      m += d.n + d.nc;
      t += d.nb / kTile;
    }
  }
}

// 1. Cost range of the candidates (the front's is its first and last entry);
//    bucket counters and cursors to 0, bucket minima to +infinity.
__device__ void huge_range(const WS& w) {
  const unsigned lane = lane_id();
  const uint32_t nh = min(ld_vol(&w.ctl->hg_n), kHugeMax), nm = ld_vol(&w.ctl->hg_nm), nt = ld_vol(&w.ctl->hg_nt);
  for (uint32_t b0 = gwarp() * 32u; b0 < nm; b0 += nwarps() * 32u) {
    const uint32_t x = b0 + lane;
    uint32_t k = kNone;
    bool v = false;
    long long c = 0;
    if (x < nm) {
      k = huge_find(w, nh, x, false);
      const HugeDesc& d = w.hg[k];
      const uint32_t i = x - d.ent0;
      Member m;
      if (i >= d.n && huge_member(w, d, i, m)) {
        v = true;
        c = m.c;
      }
    }
    const uint32_t k0 = __shfl_sync(kFull, k, 0);
    if (__all_sync(kFull, !v || k == k0)) {
      long long mn = v ? c : LLONG_MAX, mx = v ? c : LLONG_MIN;
      for (int s = 16; s > 0; s >>= 1) {
        mn = min(mn, (long long)shfl_xor_i64(mn, s));
        mx = max(mx, (long long)shfl_xor_i64(mx, s));
      }
      if (lane == 0 && mn <= mx) {
        atomicMin(&w.hg[k0].lo, mn);
        atomicMax(&w.hg[k0].hi, mx);
      }
    } else if (v) {
      atomicMin(&w.hg[k].lo, c);
      atomicMax(&w.hg[k].hi, c);
    }
  }
  for (uint32_t t = gwarp(); t < nt; t += nwarps()) {
    const HugeDesc& d = w.hg[huge_find(w, nh, t, true)];
    const size_t b0 = d.bkt + (size_t)(t - d.tile0) * kTile;
    for (uint32_t j = lane; j < kTile; j += 32) {
      w.t_m[b0 + j] = 0;
      w.t_tb[b0 + j] = 0;
      w.t_cost[b0 + j] = LLONG_MAX;
    }
  }
}

// Last block: the cost shift that maps each node's range onto its nb buckets.
__device__ void huge_shift(const WS& w) {
  const uint32_t nh = min(w.ctl->hg_n, kHugeMax);
  for (uint32_t k = threadIdx.x; k < nh; k += blockDim.x) {
    HugeDesc& d = w.hg[k];
    if (!d.ok || d.lo > d.hi) continue;
    const unsigned long long range = (unsigned long long)(d.hi - d.lo);
    uint32_t s = 0;
    while ((range >> s) >= d.nb) ++s;
    d.shift = s;
  }
}

// 2. Members per bucket and each bucket's minimum h.
__device__ void huge_count(const WS& w) {
  const unsigned lane = lane_id();
  const uint32_t nh = min(ld_vol(&w.ctl->hg_n), kHugeMax), nm = ld_vol(&w.ctl->hg_nm);
  for (uint32_t b0 = gwarp() * 32u; b0 < nm; b0 += nwarps() * 32u) {
    const uint32_t x = b0 + lane;
    if (x >= nm) continue;
    const HugeDesc& d = w.hg[huge_find(w, nh, x, false)];
    Member m;
    if (!huge_member(w, d, x - d.ent0, m)) continue;
    const size_t b = huge_bucket(d, m.c);
    atomicAdd(&w.t_m[b], 1u);
    atomicMin(&w.t_cost[b], m.h);
  }
}

// 3. Per tile (a warp each): its member count and minimum h, kept in the
//    bucket area's h column (minima at [0, ntl), counts at [ntl, 2 ntl)).
__device__ void huge_tile_agg(const WS& w) {
  const unsigned lane = lane_id();
  const uint32_t nh = min(ld_vol(&w.ctl->hg_n), kHugeMax), nt = ld_vol(&w.ctl->hg_nt);
  for (uint32_t t = gwarp(); t < nt; t += nwarps()) {
    const HugeDesc& d = w.hg[huge_find(w, nh, t, true)];
    const uint32_t tl = t - d.tile0, ntl = d.nb / kTile;
    const size_t b0 = d.bkt + (size_t)tl * kTile;
    long long mn = LLONG_MAX;
    uint32_t sum = 0;
    for (uint32_t j = lane; j < kTile; j += 32) {
      sum += w.t_m[b0 + j];
      mn = min(mn, w.t_cost[b0 + j]);
    }
    for (int s = 16; s > 0; s >>= 1) {
      sum += __shfl_xor_sync(kFull, sum, s);
      mn = min(mn, (long long)shfl_xor_i64(mn, s));
    }
    if (lane == 0) {
      w.t_h[d.bkt + tl] = mn;
      w.t_h[d.bkt + ntl + tl] = (long long)sum;
    }
  }
}

// Exclusive scan (minimum, or sum) of a[0, n) in place by the whole block;
// returns the total.
template <bool kMin>
__device__ long long block_scan_excl(long long* a, uint32_t n) {
  __shared__ long long s_w[kWarpsPerBlock];
  __shared__ long long s_carry;
  const long long id = kMin ? LLONG_MAX : 0;
  const unsigned lane = lane_id(), wid = threadIdx.x >> 5;
  __syncthreads();   // every thread has read the previous call's total
  if (threadIdx.x == 0) s_carry = id;
  __syncthreads();
  for (uint32_t i0 = 0; i0 < n; i0 += blockDim.x) {
    const uint32_t i = i0 + threadIdx.x;
    long long x = i < n ? a[i] : id;
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = shfl_up_i64(x, o);
      if (lane >= (unsigned)o) x = kMin ? min(x, y) : x + y;
    }
    if (lane == 31) s_w[wid] = x;
    __syncthreads();
    long long pre = s_carry;
    for (unsigned k = 0; k < wid; ++k) pre = kMin ? min(pre, s_w[k]) : pre + s_w[k];
    long long ex = shfl_up_i64(x, 1);
    if (lane == 0) ex = id;
    if (i < n) a[i] = kMin ? min(pre, ex) : pre + ex;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) s_carry = kMin ? min(pre, x) : pre + x;
    __syncthreads();
  }
  return s_carry;
}

// Last block: exclusive prefixes over each node's tiles, of the minima and
// counts (counts = true), or of the survivor counts, whose total is the size of
// the merged front; its block is then grown if needed (a node whose query's
// pool share is used up is skipped: the query fails).
__device__ void huge_tile_scan(const WS& w, bool counts) {
  const uint32_t nh = min(w.ctl->hg_n, kHugeMax);
  for (uint32_t k = 0; k < nh; ++k) {
    HugeDesc& d = w.hg[k];
    if (!d.ok) continue;
    const uint32_t ntl = d.nb / kTile;
    if (counts) block_scan_excl<true>(w.t_h + d.bkt, ntl);
    const long long tot = block_scan_excl<false>(w.t_h + d.bkt + ntl, ntl);
    if (!counts && threadIdx.x == 0) {
      d.n_out = (uint32_t)tot;
      if (d.lg_out == 0 || (1u << d.lg_out) < d.n_out) {
        d.lg_out = max(kMinLg, ceil_lg(d.n_out) + 1u);
        d.out = pool_alloc(w, d.q, d.lg_out);
        if (d.out == kNoBlock) {
          query_error(w, d.q, kErrFront);
          d.ok = 0;
        }
      }
    }
  }
  __syncthreads();
}

// 4. Per tile: each bucket's first member slot (exclusive prefix of the counts)
//    and the minimum h of all lower buckets (exclusive prefix minimum).
__device__ void huge_bucket_scan(const WS& w) {
  const unsigned lane = lane_id();
  const uint32_t nh = min(ld_vol(&w.ctl->hg_n), kHugeMax), nt = ld_vol(&w.ctl->hg_nt);
  for (uint32_t t = gwarp(); t < nt; t += nwarps()) {
    const HugeDesc& d = w.hg[huge_find(w, nh, t, true)];
    const uint32_t tl = t - d.tile0, ntl = d.nb / kTile;
    const size_t b0 = d.bkt + (size_t)tl * kTile;
    uint32_t cs = (uint32_t)w.t_h[d.bkt + ntl + tl];
    long long cm = w.t_h[d.bkt + tl];
    for (uint32_t j0 = 0; j0 < kTile; j0 += 32) {
      const size_t b = b0 + j0 + lane;
      const uint32_t cnt = w.t_m[b];
      long long im = w.t_cost[b];
      const uint32_t incl = warp_incl_scan(cnt);
      for (int o = 1; o < 32; o <<= 1) {
        const long long y = shfl_up_i64(im, o);
        if (lane >= (unsigned)o) im = min(im, y);
      }
      long long em = shfl_up_i64(im, 1);
      if (lane == 0) em = LLONG_MAX;
      w.t_m[b] = cs + incl - cnt;
      w.t_cost[b] = min(cm, em);
      cs += __shfl_sync(kFull, incl, 31);
      cm = min(cm, (long long)shfl_i64(im, 31));
    }
  }
}

// 5. Members dominated through a lower bucket drop out (open front entries
//    among them leave P_open); the rest are placed in their bucket's slots.
__device__ void huge_place(const WS& w) {
  const unsigned lane = lane_id();
  const uint32_t nh = min(ld_vol(&w.ctl->hg_n), kHugeMax), nm = ld_vol(&w.ctl->hg_nm);
  for (uint32_t b0 = gwarp() * 32u; b0 < nm; b0 += nwarps() * 32u) {
    const uint32_t x = b0 + lane;
    uint32_t k = kNone;
    bool rem = false;
    if (x < nm) {
      k = huge_find(w, nh, x, false);
      const HugeDesc& d = w.hg[k];
      const uint32_t i = x - d.ent0;
      Member m;
      if (huge_member(w, d, i, m)) {
        const size_t b = huge_bucket(d, m.c);
        if (w.t_cost[b] <= m.h) {
          rem = i < d.n && (m.p & kOpen);
        } else {
          const size_t pos = d.mem + w.t_m[b] + atomicAdd(&w.t_tb[b], 1u);
          w.t_cost[pos] = m.c;
          w.t_h[pos] = m.h;
          w.t_pp[pos] = m.p;
          w.t_tb[pos] = m.tb;
        }
      }
    }
    const uint32_t k0 = __shfl_sync(kFull, k, 0);
    if (__all_sync(kFull, x >= nm || k == k0)) {
      const uint32_t r = (uint32_t)__popc(__ballot_sync(kFull, rem));
      if (lane == 0 && r) atomicAdd(&w.hg[k0].removed_open, r);
    } else if (rem) {
      atomicAdd(&w.hg[k].removed_open, 1u);
    }
  }
}

// Is placed member i of a bucket at s dominated by another of the same bucket?
__device__ __forceinline__ bool bucket_dominated(const WS& w, size_t s, uint32_t k, uint32_t i, long long c,
                                                 long long h, uint32_t tb) {
  for (uint32_t j = 0; j < k; ++j) {
    if (j == i) continue;
    const long long hj = w.t_h[s + j];
    if (hj > h) continue;
    if (key_less(w.t_cost[s + j], hj, w.t_tb[s + j] & ~kSurv, c, h, tb)) return true;
  }
  return false;
}

// 6. Per tile: the survivors of each bucket (marked on their tie keys) and
//    their count; open front entries dominated inside their bucket leave
//    P_open.  Buckets of more than 32 members take the whole warp.
__device__ void huge_resolve(const WS& w) {
  const unsigned lane = lane_id();
  const uint32_t nh = min(ld_vol(&w.ctl->hg_n), kHugeMax), nt = ld_vol(&w.ctl->hg_nt);
  for (uint32_t t = gwarp(); t < nt; t += nwarps()) {
    const uint32_t hk = huge_find(w, nh, t, true);
    const HugeDesc& d = w.hg[hk];
    const uint32_t tl = t - d.tile0, ntl = d.nb / kTile;
    const size_t b0 = d.bkt + (size_t)tl * kTile;
    uint32_t tile_sv = 0, tile_rem = 0;
    for (uint32_t j0 = 0; j0 < kTile; j0 += 32) {
      const size_t b = b0 + j0 + lane;
      const uint32_t k = w.t_tb[b];
      const size_t s = d.mem + w.t_m[b];
      uint32_t sv = 0;
      const bool big = k > 32;
      if (!big) {
        for (uint32_t i = 0; i < k; ++i) {
          const long long c = w.t_cost[s + i], h = w.t_h[s + i];
          const uint32_t tb = w.t_tb[s + i] & ~kSurv;
          if (!bucket_dominated(w, s, k, i, c, h, tb)) {
            w.t_tb[s + i] = tb | kSurv;
            ++sv;
          } else if (tb == 0 && (w.t_pp[s + i] & kOpen)) {
            ++tile_rem;
          }
        }
      }
      for (unsigned bb = __ballot_sync(kFull, big); bb; bb &= bb - 1u) {
        const int L = __ffs(bb) - 1;
        const size_t sL = (size_t)__shfl_sync(kFull, (unsigned long long)s, L);
        const uint32_t kL = __shfl_sync(kFull, k, L);
        uint32_t cnt = 0;
        for (uint32_t i0 = 0; i0 < kL; i0 += 32) {
          const uint32_t i = i0 + lane;
          bool keep = false;
          uint32_t tb = 0;
          if (i < kL) {
            const long long c = w.t_cost[sL + i], h = w.t_h[sL + i];
            tb = w.t_tb[sL + i] & ~kSurv;
            keep = !bucket_dominated(w, sL, kL, i, c, h, tb);
          }
          __syncwarp();
          if (keep) w.t_tb[sL + i] = tb | kSurv;
          else if (i < kL && tb == 0 && (w.t_pp[sL + i] & kOpen)) ++tile_rem;
          cnt += (uint32_t)__popc(__ballot_sync(kFull, keep));
        }
        if (lane == (unsigned)L) sv = cnt;
      }
      w.t_pp[b] = sv;
      tile_sv += sv;
    }
    for (int o = 16; o > 0; o >>= 1) {
      tile_sv += __shfl_xor_sync(kFull, tile_sv, o);
      tile_rem += __shfl_xor_sync(kFull, tile_rem, o);
    }
    if (lane == 0) {
      w.t_h[d.bkt + ntl + tl] = (long long)tile_sv;
      if (tile_rem) atomicAdd(&w.hg[hk].removed_open, tile_rem);
    }
  }
}

// Rank of survivor i among the survivors of its bucket (cost order: survivors
// of one bucket have distinct costs).
__device__ __forceinline__ uint32_t survivor_rank(const WS& w, size_t s, uint32_t k, long long c) {
  uint32_t r = 0;
  for (uint32_t j = 0; j < k; ++j)
    if ((w.t_tb[s + j] & kSurv) && w.t_cost[s + j] < c) ++r;
  return r;
}

// Writes one survivor to the merged front; a new plan gets arena record a
// (kNone: none left) and is open.  Returns its pid.
__device__ __forceinline__ uint32_t huge_emit(const WS& w, size_t pos, uint32_t x, uint32_t it, long long c,
                                              long long h, uint32_t p, bool isnew, uint32_t a) {
  uint32_t pid = p;
  if (isnew) {
    pid = kOpen;
    if (a != kNone) {
      w.a_head[a] = x;
      w.a_parent[a] = p & kPidMask;
      w.a_iter[a] = it + 1;
      w.a_cost[a] = c;
      pid = a | kOpen;
    }
  }
  w.f_cost[pos] = c;
  w.f_h[pos] = h;
  w.f_pid[pos] = pid;
  w.f_aux[pos] = 0;
  return pid;
}

// 7. Per tile: survivors to their places in the merged front (exclusive prefix
//    of the survivor counts; cost order inside a bucket), new plans to arena
//    records (one range per 32 buckets), and the goal test of the next group.
__device__ void huge_write(const WS& w) {
  const unsigned lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t nh = min(ld_vol(&w.ctl->hg_n), kHugeMax), nt = ld_vol(&w.ctl->hg_nt), it = ld_vol(&w.ctl->it);
  for (uint32_t t = gwarp(); t < nt; t += nwarps()) {
    const uint32_t hk = huge_find(w, nh, t, true);
    const HugeDesc& d = w.hg[hk];
    if (!d.ok) continue;   // no block for the merged front: the query failed
    const QueryDev& Q = w.qd[d.q];
    const uint32_t x = d.g - Q.base;
    const long long thr2 = (long long)(it + 1) * Q.Lambda;
    const bool goal = Q.is_goal[x] != 0;
    const uint32_t tl = t - d.tile0, ntl = d.nb / kTile;
    const size_t b0 = d.bkt + (size_t)tl * kTile;
    uint32_t carry = (uint32_t)w.t_h[d.bkt + ntl + tl];
    uint32_t tile_new = 0;
    bool gnext = false;
    for (uint32_t j0 = 0; j0 < kTile; j0 += 32) {
      const size_t b = b0 + j0 + lane;
      const uint32_t k = w.t_tb[b];
      const size_t s = d.mem + w.t_m[b];
      const uint32_t sv = w.t_pp[b];
      const uint32_t incl = warp_incl_scan(sv);
      const uint32_t o0 = carry + incl - sv;
      carry += __shfl_sync(kFull, incl, 31);
      if (!__any_sync(kFull, sv != 0u)) continue;
      // new survivors of this lane's bucket, then one arena range for the step
      uint32_t nn = 0;
      for (uint32_t i = 0; i < k; ++i) {
        const uint32_t tb = w.t_tb[s + i];
        if ((tb & kSurv) && (tb & ~kSurv)) ++nn;
      }
      const uint32_t nincl = warp_incl_scan(nn);
      const uint32_t ntot = __shfl_sync(kFull, nincl, 31);
      uint32_t a0 = kNone;
      if (lane == 0 && ntot) a0 = arena_take(w, d.q, ntot);
      a0 = __shfl_sync(kFull, a0, 0);
      tile_new += ntot;
      uint32_t an = nincl - nn;   // this bucket's first record within the range
      const bool big = k > 32;
      if (!big) {
        for (uint32_t i = 0; i < k; ++i) {
          const uint32_t tb = w.t_tb[s + i];
          if (!(tb & kSurv)) continue;
          const long long c = w.t_cost[s + i], h = w.t_h[s + i];
          const bool isnew = (tb & ~kSurv) != 0;
          const size_t pos = (size_t)d.out + o0 + survivor_rank(w, s, k, c);
          const uint32_t pid = huge_emit(w, pos, x, it, c, h, w.t_pp[s + i], isnew,
                                         (isnew && a0 != kNone) ? a0 + an : kNone);
          if (isnew) ++an;
          gnext = gnext || ((pid & kOpen) && c <= thr2);
        }
      }
      for (unsigned bb = __ballot_sync(kFull, big); bb; bb &= bb - 1u) {
        const int L = __ffs(bb) - 1;
        const size_t sL = (size_t)__shfl_sync(kFull, (unsigned long long)s, L);
        const uint32_t kL = __shfl_sync(kFull, k, L);
        const uint32_t oL = __shfl_sync(kFull, o0, L);
        uint32_t aL = __shfl_sync(kFull, an, L);
        for (uint32_t i0 = 0; i0 < kL; i0 += 32) {
          const uint32_t i = i0 + lane;
          uint32_t tb = 0;
          if (i < kL) tb = w.t_tb[sL + i];
          const bool surv = (tb & kSurv) != 0;
          const bool isnew = surv && (tb & ~kSurv) != 0;
          const unsigned nb_ = __ballot_sync(kFull, isnew);
          if (surv) {
            const long long c = w.t_cost[sL + i], h = w.t_h[sL + i];
            const size_t pos = (size_t)d.out + oL + survivor_rank(w, sL, kL, c);
            const uint32_t pid = huge_emit(w, pos, x, it, c, h, w.t_pp[sL + i], isnew,
                                           (isnew && a0 != kNone) ? a0 + aL + (uint32_t)__popc(nb_ & lt) : kNone);
            gnext = gnext || ((pid & kOpen) && c <= thr2);
          }
          aL += (uint32_t)__popc(nb_);
        }
      }
    }
    if (lane == 0 && tile_new) atomicAdd(&w.hg[hk].n_new, tile_new);   // warp-uniform
    // an open plan of the next group at a goal node ends the query at the top of
    // the next iteration (the loop condition of Alg. 3)
    if (goal && __any_sync(kFull, gnext) && lane == 0) w.qs[d.q].goal_next = 1u;
  }
}

// Last block, after step 7: each node's new descriptor (the merged front is
// live, the old block becomes the other), its query's counters and its place in
// the next open list; then the grid-wide merge is closed for this wavefront.
__device__ void huge_finish(const WS& w) {
  Ctl* c = w.ctl;
  const uint32_t nh = min(c->hg_n, kHugeMax), it = c->it;
  for (uint32_t k = threadIdx.x; k < nh; k += blockDim.x) {
    const HugeDesc& d = w.hg[k];
    if (d.ok) {
      FDesc fd;
      fd.d = make_uint4(d.out, d.n_out, d.off, d.lg_out | (d.lg_old << 8));
      const size_t l = (size_t)d.out + d.n_out - 1;
      fd.last = d.n_out ? make_longlong2(w.f_cost[l], w.f_h[l]) : make_longlong2(0, 0);
      w.fdesc[d.g] = fd;
      atomic_add_i64(&w.qs[d.q].open_cnt, (long long)d.n_new - (long long)d.removed_open);
      atomicAdd(&w.qs[d.q].plans, (unsigned long long)d.n_new);
      atomicMax(&c->max_front, d.n_out);
      if (d.n_new && w.oh_stamp[d.g] != it + 1) {
        const uint32_t slot = atomicAdd(&c->oh_n[(it + 1) & 1], 1u);
        w.oh_list[(size_t)((it + 1) & 1) * w.NV + slot] = make_uint2(d.g, d.q);
      }
    }
    w.cand_n[d.g] = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    c->hg_n = 0;
    c->hg_live = 0;
    c->hg_nm = 0;
    c->hg_nt = 0;
    c->hg_ents = 0;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Work of the last block at the barriers.
// ---------------------------------------------------------------------------
// After the expansion: does any query need its overflow regrouped?  The
// exclusive prefix of the queries' overflow records (kept within each share)
// maps a flat record index to its query.
__device__ void epi_mid(const WS& w) {
  if (threadIdx.x == 0) {
    const uint32_t nq = w.ctl->nq;
    uint32_t acc = 0;
    for (uint32_t q = 0; q < nq; ++q) {
      w.ov_pref[q] = acc;
      acc += (uint32_t)min((uint64_t)w.qs[q].ov_n, w.qd[q].ov_cap);
    }
    w.ov_pref[nq] = acc;
    w.ctl->ov_total = acc;
    w.ctl->ov_any = acc ? 1u : 0u;
  }
  phase_mark(w, 0);
}

// End of wavefront i: the loop condition of Alg. 3 per query (tested in the
// order of the algorithm: P_open empty, a goal plan in the next group, then the
// iteration cap), then the next iteration.
__device__ void epi_end(const WS& w) {
  __shared__ uint32_t s_newly;
  if (threadIdx.x == 0) s_newly = 0;
  __syncthreads();
  Ctl* c = w.ctl;
  const uint32_t it = c->it, nq = c->nq;
  for (uint32_t q = threadIdx.x; q < nq; q += blockDim.x) {
    QueryState& s = w.qs[q];
    const QueryDev& Q = w.qd[q];
    if (s.done) continue;
    if (s.err) {
      s.done = 1;
      s.status = MPAP_ERR_CAPACITY;
    } else {
      s.wavefronts += 1;
      if (s.open_cnt == 0) {
        s.done = 1;
      } else if (s.goal_next && !(Q.flags & MPAP_QUERY_NO_GOAL_STOP)) {
        s.done = 1;
        s.goal_hit = 1;
      } else if (s.wavefronts >= Q.max_iters) {
        s.done = 1;
        s.status = MPAP_ERR_ITER_LIMIT;
      }
    }
    s.goal_next = 0;
    s.ov_n = 0;
    s.seg_n = 0;
    if (s.done) atomicAdd(&s_newly, 1u);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    c->n_done += s_newly;
    // the list consumed in this iteration becomes the append target of the next
    c->oh_n[it & 1] = 0;
    c->m_n = 0;
    c->g_n = 0;
    c->ov_any = 0;
    c->grab[0] = 0;
    c->grab[1] = 0;
    c->ovl_n = 0;
    c->tmp_n = 0;
    c->it = it + 1;
    c->waves += 1;
  }
  phase_mark(w, 3);
}

// The persistent wavefront loop (Alg. 3): one cooperative launch per search.
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 4) k_wave(WS w) {
  __shared__ WarpSmem smem[kWarpsPerBlock];
  __shared__ GroupSmem gsm[kWarpsPerBlock];
  __shared__ WaveSmem ws;
  WarpSmem& sm = smem[threadIdx.x >> 5];
  GroupSmem& gs = gsm[threadIdx.x >> 5];
  const uint32_t nq = w.ctl->nq;
  for (uint32_t q = threadIdx.x; q < kAccQ; q += blockDim.x) {
    ws.open[q] = 0;
    ws.plans[q] = 0;
    ws.exps[q] = 0;
  }
  __syncthreads();
  WarpCtx cx;
  cx.s = &ws;
  cx.lb_n = 0;
  cx.mb_n = 0;
  cx.nq = nq;
  cx.huge_from = w.ctl->huge_from;
  if (blockIdx.x == 0 && threadIdx.x == 0) w.ctl->t_mark = global_timer();
  for (;;) {
    const uint32_t it = ld_vol(&w.ctl->it);
    if (ld_vol(&w.ctl->n_done) >= nq || it >= w.ctl->iter_cap) break;
    cx.it = it;
    cx.next = w.oh_list + (size_t)((it + 1) & 1) * w.NV;
    phase_expand(w, cx, gs);
    flush_acc(w, ws, nq);
    if (!grid_barrier(w, [&] { epi_mid(w); })) return;
    if (ld_vol(&w.ctl->ov_any)) {
      phase_segments(w);
      if (!grid_barrier(w, [] {})) return;
      phase_scatter(w);
      if (!grid_barrier(w, [&] { phase_mark(w, 1); })) return;
    }
    phase_merge(w, cx, sm);
    flush_acc(w, ws, nq);
    if (!grid_barrier(w, [&] {
          if (ld_vol(&w.ctl->hg_n)) {
            huge_setup(w);
          } else {
            phase_mark(w, 2);
            epi_end(w);
          }
        }))
      return;
    if (ld_vol(&w.ctl->hg_live)) {
      // grid-wide merge of the huge nodes, then the end of the wavefront
      huge_range(w);
      if (!grid_barrier(w, [&] { huge_shift(w); })) return;
      huge_count(w);
      if (!grid_barrier(w, [] {})) return;
      huge_tile_agg(w);
      if (!grid_barrier(w, [&] { huge_tile_scan(w, true); })) return;
      huge_bucket_scan(w);
      if (!grid_barrier(w, [] {})) return;
      huge_place(w);
      if (!grid_barrier(w, [] {})) return;
      huge_resolve(w);
      if (!grid_barrier(w, [&] { huge_tile_scan(w, false); })) return;
      huge_write(w);
      if (!grid_barrier(w, [&] {
            huge_finish(w);
            phase_mark(w, 2);
            epi_end(w);
          }))
        return;
    }
  }
}

// ---------------------------------------------------------------------------
// Solution selection (Alg. 3 final lines) and back-tracing (block per query).
// Among all stored plans at goal nodes: minimum cost, then h, then the tie key
// (creation iteration, parent head, parent cost), then head index.
// ---------------------------------------------------------------------------
struct Best {
  long long cost, h, pcost;
  uint32_t iter, phead, head, ref;
};

__device__ __forceinline__ bool better(const Best& a, const Best& b) {
  if (a.cost != b.cost) return a.cost < b.cost;
  if (a.h != b.h) return a.h < b.h;
  if (a.iter != b.iter) return a.iter < b.iter;
  if (a.phead != b.phead) return a.phead < b.phead;
  if (a.pcost != b.pcost) return a.pcost < b.pcost;
  return a.head < b.head;
}

__global__ void k_finalize(WS w, uint32_t nq) {
  const uint32_t q = blockIdx.x;
  if (q >= nq) return;
  const QueryDev& Q = w.qd[q];
  const QueryState& s = w.qs[q];
  __shared__ Best sb[256];
  Best best;
  best.cost = LLONG_MAX;
  best.ref = kNone;
  if (s.status == 0) {
    for (uint32_t i = threadIdx.x; i < Q.n_goal; i += blockDim.x) {
      const uint32_t v = Q.goal_list[i];
      const uint32_t g = Q.base + v;
      const uint4 fd = w.fdesc[g].d;
      const uint32_t n = fd.y;
      const size_t o = fd.x;
      for (uint32_t j = 0; j < n; ++j) {
        Best c;
        c.cost = w.f_cost[o + j];
        c.h = w.f_h[o + j];
        c.ref = w.f_pid[o + j] & kPidMask;
        c.iter = w.a_iter[c.ref];
        const uint32_t par = w.a_parent[c.ref];
        c.phead = (par == kNone) ? kNone : w.a_head[par];
        c.pcost = (par == kNone) ? 0 : w.a_cost[par];
        c.head = v;
        if (best.ref == kNone || better(c, best)) best = c;
      }
    }
  }
  sb[threadIdx.x] = best;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) {
      const Best& o = sb[threadIdx.x + st];
      if (o.ref != kNone && (sb[threadIdx.x].ref == kNone || better(o, sb[threadIdx.x]))) sb[threadIdx.x] = o;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    ResultDev r;
    r.status = s.done ? s.status : (w.ctl->timeout ? MPAP_ERR_TIMEOUT : MPAP_ERR_ITER_LIMIT);
    r.cost = 0;
    r.h = 0;
    r.path_len = 0;
    if (r.status == 0) {
      const Best b = sb[0];
      if (b.ref == kNone) {
        r.status = MPAP_NO_SOLUTION;
      } else {
        r.cost = b.cost;
        r.h = b.h;
        uint32_t* path = w.path + (size_t)q * w.path_cap;
        uint32_t len = 0;
        uint32_t a = b.ref;
        while (a != kNone && len <= w.path_cap) {
          if (len < w.path_cap) path[len] = w.a_head[a];
          ++len;
          a = w.a_parent[a];
        }
        if (len > w.path_cap) {
          r.status = MPAP_ERR_CAPACITY;
        } else {
          for (uint32_t i = 0; i < len / 2; ++i) {
            const uint32_t t = path[i];
            path[i] = path[len - 1 - i];
            path[len - 1 - i] = t;
          }
        }
        r.path_len = len;
      }
    }
    w.res[q] = r;
  }
}

// ---------------------------------------------------------------------------
// Candidate export (Alg. 3 final lines: P_candidates, every plan stored at a goal
// node).  One block for one query: `cap` rounds, each picking the best plan that
// is strictly worse (in the solution order) than the previous pick, so the
// candidates come out in the order k_finalize uses; then each thread back-traces
// one candidate into the packed path array.
// ---------------------------------------------------------------------------
struct CandOut {
  long long* cost;
  long long* h;
  uint32_t* ref;
  uint32_t* ptr;       // [cap + 1]
  uint32_t* path;      // [path_cap]
  uint32_t path_cap;
  uint32_t* counts;    // [0] candidates written, [1] |P_candidates|, [2] path overflow
};

__device__ __forceinline__ Best goal_plan(const WS& w, uint32_t v, uint32_t ref, long long cost, long long h) {
  Best c;
  c.cost = cost;
  c.h = h;
  c.ref = ref;
  c.iter = w.a_iter[ref];
  const uint32_t par = w.a_parent[ref];
  c.phead = (par == kNone) ? kNone : w.a_head[par];
  c.pcost = (par == kNone) ? 0 : w.a_cost[par];
  c.head = v;
  return c;
}

// One block per query q0 + blockIdx.x; block b writes slice b of every output
// (cap candidates, cap + 1 offsets, path_cap path entries, 4 counters).  A query
// that did not finish with MPAP_OK gets zero counts.
__global__ void __launch_bounds__(256) k_candidates(WS w, uint32_t q0, uint32_t cap, CandOut ob) {
  const uint32_t b = blockIdx.x, q = q0 + b;
  CandOut o = ob;
  o.cost += (size_t)b * cap;
  o.h += (size_t)b * cap;
  o.ref += (size_t)b * cap;
  o.ptr += (size_t)b * (cap + 1);
  o.path += (size_t)b * o.path_cap;
  o.counts += (size_t)b * 4;
  if (w.res[q].status != MPAP_OK) {
    if (threadIdx.x == 0) {
      o.ptr[0] = 0;
      o.counts[0] = o.counts[1] = o.counts[2] = 0;
    }
    return;
  }
  const QueryDev& Q = w.qd[q];
  __shared__ Best sb[256];
  __shared__ Best prev;
  __shared__ uint32_t s_total, s_n;
  if (threadIdx.x == 0) {
    s_total = 0;
    s_n = 0;
  }
  __syncthreads();
  uint32_t mine = 0;
  for (uint32_t r = 0; r < cap; ++r) {
    Best best;
    best.cost = LLONG_MAX;
    best.ref = kNone;
    for (uint32_t i = threadIdx.x; i < Q.n_goal; i += blockDim.x) {
      const uint32_t v = Q.goal_list[i];
      const uint32_t g = Q.base + v;
      const uint4 fd = w.fdesc[g].d;
      const uint32_t n = fd.y;
      const size_t off = fd.x;
      if (r == 0) mine += n;
      for (uint32_t j = 0; j < n; ++j) {
        const Best c = goal_plan(w, v, w.f_pid[off + j] & kPidMask, w.f_cost[off + j], w.f_h[off + j]);
        if (r > 0 && !better(prev, c)) continue;
        if (best.ref == kNone || better(c, best)) best = c;
      }
    }
    sb[threadIdx.x] = best;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
      if ((int)threadIdx.x < st) {
        const Best& x = sb[threadIdx.x + st];
        if (x.ref != kNone && (sb[threadIdx.x].ref == kNone || better(x, sb[threadIdx.x]))) sb[threadIdx.x] = x;
      }
      __syncthreads();
    }
    const bool none = sb[0].ref == kNone;
    if (threadIdx.x == 0 && !none) {
      prev = sb[0];
      o.cost[r] = sb[0].cost;
      o.h[r] = sb[0].h;
      o.ref[r] = sb[0].ref;
      s_n = r + 1;
    }
    if (r == 0 && mine) atomicAdd(&s_total, mine);
    __syncthreads();
    if (none) break;
  }
  // path lengths, offsets (serial over at most cap candidates), then the paths
  const uint32_t nc = s_n;
  for (uint32_t i = threadIdx.x; i < nc; i += blockDim.x) {
    uint32_t len = 0;
    for (uint32_t a = o.ref[i]; a != kNone; a = w.a_parent[a]) ++len;
    o.ptr[i + 1] = len;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    o.ptr[0] = 0;
    for (uint32_t i = 0; i < nc; ++i) o.ptr[i + 1] += o.ptr[i];
    o.counts[0] = nc;
    o.counts[1] = s_total;
    o.counts[2] = o.ptr[nc] > o.path_cap ? 1u : 0u;
  }
  __syncthreads();
  if (o.ptr[nc] > o.path_cap) return;
  for (uint32_t i = threadIdx.x; i < nc; i += blockDim.x) {
    uint32_t k = o.ptr[i + 1];
    for (uint32_t a = o.ref[i]; a != kNone; a = w.a_parent[a]) o.path[--k] = w.a_head[a];
  }
}

// Packs the final fronts of one query (nodes base .. base+V-1) into [ptr[v],
// ptr[v+1]) of oc/oh (warp per node; front export for parity checks).
__global__ void k_gather_fronts(WS w, uint32_t base, uint32_t V, const uint32_t* __restrict__ ptr,
                                long long* __restrict__ oc, long long* __restrict__ oh) {
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < V; v += warps) {
    const uint4 fd = w.fdesc[base + v].d;
    for (uint32_t j = lane_id(); j < fd.y; j += 32) {
      oc[ptr[v] + j] = w.f_cost[(size_t)fd.x + j];
      oh[ptr[v] + j] = w.f_h[(size_t)fd.x + j];
    }
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {

int sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// Resident blocks per SM of k_wave (all of them must fit: cooperative launch).
int wave_occupancy() {
  static int occ = 0;
  if (!occ) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_wave, kWarpsPerBlock * 32, 0) != cudaSuccess ||
        occ < 1) {
      cudaGetLastError();
      occ = 1;
    }
  }
  return occ;
}

template <typename T>
bool walloc(T** p, size_t n) {
  return cuda_ok(cudaMalloc((void**)p, (n ? n : 1) * sizeof(T)), "cudaMalloc(workspace)");
}

}  // namespace

int32_t workspace_create(uint64_t total_nodes, uint32_t front_cap, uint64_t max_plans, uint32_t max_q,
                         mpap_workspace** out) {
  if (!out || total_nodes == 0 || total_nodes > 0xFFFFFFF0ull || front_cap == 0 || max_plans == 0 ||
      max_plans > (uint64_t)kPidMask) {
    set_error("mpap_workspace_create: invalid sizes");
    return MPAP_ERR_INVALID_ARG;
  }
  if (total_nodes * kSlots > 0xFFFFFFFFFFull) {
    set_error("mpap_workspace_create: too many nodes");
    return MPAP_ERR_INVALID_ARG;
  }
  mpap_workspace* ws = new mpap_workspace();
  WS& w = ws->w;
  w.NV = total_nodes;
  w.fcap = front_cap;
  w.pcap = (uint64_t)total_nodes * front_cap;
  if (w.pcap > 0xFFFFFFF0ull || w.pcap < 16) {
    delete ws;
    set_error("mpap_workspace_create: total_nodes x front_cap must lie in [16, 2^32 - 16]");
    return MPAP_ERR_INVALID_ARG;
  }
  w.acap = max_plans;
  w.gcap = max_plans;
  w.ocap = max_plans;
  w.tcap = max_plans;
  w.path_cap = 4096;
  ws->max_q = max_q;
  const size_t slots = (size_t)w.pcap;
  bool ok = walloc(&w.f_cost, slots) && walloc(&w.f_h, slots) && walloc(&w.f_pid, slots) &&
            walloc(&w.f_aux, slots) && walloc(&w.fdesc, w.NV) && walloc(&w.slot, w.NV * kSlots) &&
            walloc(&w.cand_n, w.NV) && walloc(&w.ov, w.ocap) && walloc(&w.ov2, w.ocap) &&
            walloc(&w.segoff, w.NV) && walloc(&w.t_cost, w.tcap) && walloc(&w.t_h, w.tcap) &&
            walloc(&w.t_pp, w.tcap) && walloc(&w.t_tb, w.tcap) && walloc(&w.t_m, w.tcap) && walloc(&w.ovl, w.NV) && walloc(&w.ov_pref, (size_t)max_q + 1) &&
            walloc(&w.oh_stamp, w.NV) && walloc(&w.g_cost, w.gcap) &&
            walloc(&w.g_h, w.gcap) && walloc(&w.g_pid, w.gcap) && walloc(&w.oh_list, 2 * w.NV) &&
            walloc(&w.m_list, w.NV) && walloc(&w.a_head, w.acap) && walloc(&w.a_parent, w.acap) &&
            walloc(&w.a_iter, w.acap) && walloc(&w.a_cost, w.acap) && walloc(&w.hg, kHugeMax) && walloc(&w.ctl, 1) && walloc(&w.qd, max_q) &&
            walloc(&w.qs, max_q) && walloc(&w.res, max_q) && walloc(&w.path, (size_t)max_q * w.path_cap);
  if (!ok) {
    workspace_free(ws);
    return MPAP_ERR_CUDA;
  }
  *out = ws;
  return MPAP_OK;
}

void workspace_free(mpap_workspace* ws) {
  if (!ws) return;
  WS& w = ws->w;
  void* ptrs[] = {w.f_cost, w.f_h,     w.f_pid,  w.f_aux,  w.fdesc,  w.slot,     w.cand_n, w.ov,
                  w.ov2,    w.segoff,  w.t_cost, w.t_h,    w.t_pp,   w.t_tb,    w.t_m,    w.ovl,    w.ov_pref, w.oh_stamp, w.g_cost, w.g_h,  w.g_pid,    w.oh_list, w.m_list,
                  w.a_head, w.a_parent, w.a_iter, w.a_cost, w.hg,     w.ctl,    w.qd,       w.qs,     w.res,
                  w.path};
  for (void* p : ptrs) cudaFree(p);
  if (ws->h_hdr) cudaFreeHost(ws->h_hdr);
  if (ws->h_path) cudaFreeHost(ws->h_path);
  delete ws;
}

namespace {

// Pinned host buffer of at least `bytes`, reallocated (contents dropped) when it
// is too small.  Called only when no copy into it is in flight.
int32_t host_stage(char** buf, size_t* have, size_t bytes) {
  if (*have >= bytes) return MPAP_OK;
  if (*buf) cudaFreeHost(*buf);
  *buf = nullptr;
  *have = 0;
  const size_t want = std::max<size_t>(bytes, 64u << 10);
  if (!cuda_ok(cudaMallocHost(reinterpret_cast<void**>(buf), want), "cudaMallocHost")) {
    *buf = nullptr;
    return MPAP_ERR_CUDA;
  }
  *have = want;
  return MPAP_OK;
}

constexpr size_t align64(size_t b) { return (b + 63) & ~(size_t)63; }

}  // namespace

// Tuning key of a batch: the common dimension (0 if mixed) and the largest V.
void batch_key(mpap_roadmap* const* rms, uint32_t nq, int& dim, uint32_t& V) {
  dim = -1;
  V = 0;
  for (uint32_t i = 0; i < nq; ++i) {
    if (!rms[i]) continue;
    dim = (dim < 0 || dim == rms[i]->dim) ? rms[i]->dim : 0;
    V = std::max(V, rms[i]->V);
  }
  if (dim < 0) dim = 0;
}

uint32_t workspace_last_max_front(const mpap_workspace* ws) { return ws->last_max_front; }
unsigned long long workspace_last_pool_used(const mpap_workspace* ws) { return ws->last_pool_used; }
uint64_t workspace_nodes(const mpap_workspace* ws) { return ws->w.NV; }

int32_t search_batch_impl(mpap_workspace* ws, mpap_roadmap* const* rms, const mpap_query* qs, uint32_t nq,
                          mpap_result* outs, cudaStream_t st) {
  WS& w = ws->w;
  if (nq == 0) return MPAP_OK;
  if (nq > ws->max_q) {
    set_error("search: %u queries exceed the workspace's %u", nq, ws->max_q);
    return MPAP_ERR_INVALID_ARG;
  }
  std::vector<QueryDev> qd(nq);
  uint64_t total = 0;
  uint32_t max_iters = 0;
  uint32_t wait_us = 0;
  for (uint32_t i = 0; i < nq; ++i) {
    const mpap_roadmap* rm = rms[i];
    if (!rm || rm->V < 1) {
      set_error("search: null or empty roadmap %u", i);
      return MPAP_ERR_INVALID_ARG;
    }
    if ((qs[i].group_width_q <= 0 && (!(qs[i].lambda > 0.0f) || !(qs[i].lambda <= 1.0f))) || qs[i].beta < 0 ||
        qs[i].max_iters == 0 || qs[i].max_iters > 0x7FFFFFF0u) {
      set_error("search: query %u needs lambda in (0, 1] (or group_width_q > 0), beta >= 0, 0 < max_iters < 2^31",
                i);
      return MPAP_ERR_INVALID_ARG;
    }
    QueryDev d{};
    d.fwd_ptr = rm->fwd_ptr;
    d.fwd_edge = rm->fwd_edge;
    d.fwd_peak = rm->fwd_peak;
    d.is_goal = rm->is_goal;
    d.goal_list = rm->goal_list;
    d.n_goal = rm->n_goal;
    d.V = rm->V;
    d.base = (uint32_t)total;
    d.max_iters = qs[i].max_iters;
    d.flags = qs[i].flags;
    d.beta = qs[i].beta;
    // Lambda = round(lambda r_n 2^24), the group threshold quantum (or the
    // caller's explicit width in cost quanta).
    d.Lambda = qs[i].group_width_q > 0 ? qs[i].group_width_q
                                       : (int64_t)llrint((double)qs[i].lambda * (double)rm->r * 16777216.0);
    if (d.Lambda < 1) d.Lambda = 1;
    total += rm->V;
    max_iters = std::max(max_iters, qs[i].max_iters);
    if (qs[i].wait_us && (wait_us == 0 || qs[i].wait_us < wait_us)) wait_us = qs[i].wait_us;
    qd[i] = d;
  }
  if (total > w.NV) {
    set_error("search: %llu nodes exceed the workspace's %llu", (unsigned long long)total,
              (unsigned long long)w.NV);
    return MPAP_ERR_INVALID_ARG;
  }
  // every query gets a share of the candidate overflow areas, of one half of
  // the front pool and of one half of the plan arena in proportion to its
  // nodes; the other halves of the pool and the arena are common to the batch
  const uint64_t a_shared = w.acap - w.acap / 2;
  w.arena_common_base = a_shared;
  w.arena_common_cap = w.acap / 2;
  const uint64_t p_shared = w.pcap - w.pcap / 2;
  w.pool_common_base = p_shared;
  w.pool_common_cap = w.pcap / 2;
  {
    uint64_t acc = 0, acc_o = 0, acc_a = 0;
    for (uint32_t i = 0; i < nq; ++i) {
      const bool last = i + 1 == nq;
      const double f = (double)qd[i].V / (double)total;
      const uint64_t cap = last ? p_shared - acc : (uint64_t)((double)p_shared * f);
      const uint64_t ocap = last ? w.ocap - acc_o : (uint64_t)((double)w.ocap * f);
      const uint64_t acap = last ? a_shared - acc_a : (uint64_t)((double)a_shared * f);
      if (cap < 16 || acap < 1) {
        set_error("search: query %u's share of the front pool (below 16 entries) or of the plan arena is too small",
                  i);
        return MPAP_ERR_CAPACITY;
      }
      qd[i].pool_base = acc;
      qd[i].pool_cap = cap;
      qd[i].ov_base = acc_o;
      qd[i].ov_cap = ocap;
      qd[i].arena_base = acc_a;
      qd[i].arena_cap = acap;
      acc += cap;
      acc_o += ocap;
      acc_a += acap;
    }
  }
  int kdim = -1;
  uint32_t kV = 0;
  batch_key(rms, nq, kdim, kV);
  const mpap_tuning tun = tuning_for(kdim, kV);
  ws->last_V.resize(nq);
  ws->last_base.resize(nq);
  for (uint32_t i = 0; i < nq; ++i) {
    ws->last_V[i] = qd[i].V;
    ws->last_base[i] = qd[i].base;
  }
  const size_t NVu = (size_t)total;
  const bool prof = profile_enabled();
  const unsigned long long wait_ns = (unsigned long long)(wait_us ? wait_us : kDefaultWaitUs) * 1000ull;
  MPAP_CK(cudaMemcpyAsync(w.qd, qd.data(), sizeof(QueryDev) * nq, cudaMemcpyHostToDevice, st));
  MPAP_CK(cudaMemsetAsync(w.fdesc, 0, sizeof(FDesc) * NVu, st));
  MPAP_CK(cudaMemsetAsync(w.cand_n, 0, sizeof(uint32_t) * NVu, st));
  MPAP_CK(cudaMemsetAsync(w.oh_stamp, 0xFF, sizeof(uint32_t) * NVu, st));
  {
    LaunchScope ls(st, "k_init");
    k_init<<<(nq + 127) / 128, 128, 0, st>>>(w, nq, max_iters + 2u, tun.plan_lanes_from, tun.grid_merge_from,
                                             wait_ns);
    k_init_done<<<1, 256, 0, st>>>(w, nq);
  }
  MPAP_CK(cudaGetLastError());
  const int grid = std::max(1, std::min<int>((int)tun.wave_blocks_per_sm, wave_occupancy())) * sms();
  {
    // the whole wavefront loop: one cooperative launch, every block resident
    void* args[] = {&w};
    LaunchScope ls(st, "k_wave");
    MPAP_CK(cudaLaunchCooperativeKernel((const void*)k_wave, dim3(grid), dim3(kWarpsPerBlock * 32), args, 0, st));
  }
  {
    LaunchScope ls(st, "k_finalize");
    k_finalize<<<nq, 256, 0, st>>>(w, nq);
  }
  MPAP_CK(cudaGetLastError());
  // results, query states and the control block: three copies into pinned staging
  const size_t o_qs = align64(sizeof(ResultDev) * nq), o_ctl = o_qs + align64(sizeof(QueryState) * nq);
  int32_t rc = host_stage(&ws->h_hdr, &ws->h_hdr_bytes, o_ctl + sizeof(Ctl));
  if (rc) return rc;
  const ResultDev* res = reinterpret_cast<const ResultDev*>(ws->h_hdr);
  const QueryState* qsh = reinterpret_cast<const QueryState*>(ws->h_hdr + o_qs);
  const Ctl& hc = *reinterpret_cast<const Ctl*>(ws->h_hdr + o_ctl);
  MPAP_CK(cudaMemcpyAsync(ws->h_hdr, w.res, sizeof(ResultDev) * nq, cudaMemcpyDeviceToHost, st));
  MPAP_CK(cudaMemcpyAsync(ws->h_hdr + o_qs, w.qs, sizeof(QueryState) * nq, cudaMemcpyDeviceToHost, st));
  MPAP_CK(cudaMemcpyAsync(ws->h_hdr + o_ctl, w.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  MPAP_CK(cudaStreamSynchronize(st));
  ws->last_max_front = hc.max_front;
  launch_count_add(1);   // k_init_done (k_init, k_wave and k_finalize count through their scopes)
  if (prof) {
    const char* names[4] = {"k_wave.expand", "k_wave.regroup", "k_wave.merge", "k_wave.end"};
    for (int k = 0; k < 4; ++k) profile_add(names[k], hc.waves, (double)hc.ph_ns[k] * 1e-6);
    // mean time a block of the grid spent waiting at barriers
    profile_add("k_wave.idle", hc.waves, (double)hc.idle_ns * 1e-6 / (double)grid);
  }
  rc = MPAP_OK;
  uint32_t lmax = 0;     // longest plan to return
  for (uint32_t i = 0; i < nq; ++i) {
    mpap_result& o = outs[i];
    o.status = res[i].status;
    o.cost = res[i].cost;
    o.h = res[i].h;
    o.wavefronts = qsh[i].wavefronts;
    o.expansions = qsh[i].expansions;
    o.plans = qsh[i].plans;
    o.path_len = res[i].path_len;
    if (o.status == MPAP_OK) {
      if (o.path && o.path_cap >= o.path_len) {
        lmax = std::max(lmax, o.path_len);
      } else if (o.path_cap < o.path_len) {
        o.status = MPAP_ERR_INVALID_ARG;
      }
    }
    if (o.status < 0 && rc == MPAP_OK) rc = o.status;
  }
  if (lmax) {
    // the first lmax entries of every query's plan row in one strided copy
    const int32_t r2 = host_stage(&ws->h_path, &ws->h_path_bytes, 4 * (size_t)nq * lmax);
    if (r2) return r2;
    MPAP_CK(cudaMemcpy2DAsync(ws->h_path, 4 * (size_t)lmax, w.path, 4 * (size_t)w.path_cap, 4 * (size_t)lmax, nq,
                              cudaMemcpyDeviceToHost, st));
    MPAP_CK(cudaStreamSynchronize(st));
    const uint32_t* hp = reinterpret_cast<const uint32_t*>(ws->h_path);
    for (uint32_t i = 0; i < nq; ++i) {
      mpap_result& o = outs[i];
      if (o.status == MPAP_OK && o.path && o.path_len)
        std::memcpy(o.path, hp + (size_t)i * lmax, 4 * (size_t)o.path_len);
    }
  }
  {
    unsigned long long used = 0;
    for (uint32_t i = 0; i < nq; ++i) used += std::min<unsigned long long>(qsh[i].pool_n, qd[i].pool_cap);
    used += std::min<unsigned long long>(hc.pool_common_n, w.pool_common_cap);
    ws->last_pool_used = used;
  }
  if (hc.timeout) {
    set_error("search: a grid barrier wait of the wavefront loop ran past its limit (%u us); unfinished queries "
              "report MPAP_ERR_TIMEOUT", wait_us ? wait_us : kDefaultWaitUs);
    rc = MPAP_ERR_TIMEOUT;
  } else if (hc.err) {
    set_error("search: capacity exceeded in at least one query (flags 0x%x: 1 front pool, 2 plan arena, "
              "4 group array, 8 candidate overflow); its status says so, the other queries' results stand", hc.err);
    rc = MPAP_ERR_CAPACITY;
  } else if (hc.n_done < nq) {
    set_error("search: wavefront loop stopped at its iteration bound");
    rc = MPAP_ERR_ITER_LIMIT;
  }
  return rc;
}

int32_t search_fronts_impl(mpap_workspace* ws, uint32_t index, uint32_t* front_ptr, int64_t* cost,
                           int64_t* h, uint64_t cap, uint64_t* total, cudaStream_t st) {
  const WS& w = ws->w;
  if (index >= ws->last_V.size()) {
    set_error("search_fronts: no query %u in the last search", index);
    return MPAP_ERR_INVALID_ARG;
  }
  const uint32_t V = ws->last_V[index], base = ws->last_base[index];
  std::vector<FDesc> fd(V);
  MPAP_CK(cudaMemcpyAsync(fd.data(), w.fdesc + base, sizeof(FDesc) * V, cudaMemcpyDeviceToHost, st));
  MPAP_CK(cudaStreamSynchronize(st));
  std::vector<uint32_t> ptr(V + 1);
  uint64_t t = 0;
  for (uint32_t v = 0; v < V; ++v) {
    ptr[v] = (uint32_t)t;
    t += fd[v].d.y;
  }
  ptr[V] = (uint32_t)t;
  if (front_ptr) std::memcpy(front_ptr, ptr.data(), 4 * ((size_t)V + 1));
  if (total) *total = t;
  if (t > cap) return MPAP_ERR_INVALID_ARG;
  if (t == 0 || (!cost && !h)) return MPAP_OK;
  // gather the fronts on the device into one packed block, then copy it out
  const size_t b_ptr = (4 * ((size_t)V + 1) + 255) & ~(size_t)255;
  char* blk = nullptr;
  MPAP_CK(scratch_alloc((void**)&blk, b_ptr + 16 * t, st));
  uint32_t* d_ptr = reinterpret_cast<uint32_t*>(blk);
  long long* d_c = reinterpret_cast<long long*>(blk + b_ptr);
  long long* d_h = d_c + t;
  int32_t rc = MPAP_OK;
  if (!cuda_ok(cudaMemcpyAsync(d_ptr, ptr.data(), 4 * ((size_t)V + 1), cudaMemcpyHostToDevice, st), "fronts ptr"))
    rc = MPAP_ERR_CUDA;
  if (rc == MPAP_OK) {
    LaunchScope ls(st, "k_gather_fronts");
    k_gather_fronts<<<std::min<uint32_t>((V + 7) / 8, 4096u), 256, 0, st>>>(w, base, V, d_ptr, d_c, d_h);
    if (!cuda_ok(cudaGetLastError(), "k_gather_fronts")) rc = MPAP_ERR_CUDA;
  }
  if (rc == MPAP_OK && cost &&
      !cuda_ok(cudaMemcpyAsync(cost, d_c, 8 * t, cudaMemcpyDeviceToHost, st), "fronts cost"))
    rc = MPAP_ERR_CUDA;
  if (rc == MPAP_OK && h && !cuda_ok(cudaMemcpyAsync(h, d_h, 8 * t, cudaMemcpyDeviceToHost, st), "fronts h"))
    rc = MPAP_ERR_CUDA;
  scratch_free(blk, st);
  if (!cuda_ok(cudaStreamSynchronize(st), "search_fronts")) rc = MPAP_ERR_CUDA;
  return rc;
}


namespace {

// Candidates of queries q0 .. q0 + nq - 1 into host arrays laid out in slices:
// cost/h [nq][cap], path_ptr [nq][cap + 1], path [nq][path_cap], n/total/ovf [nq].
int32_t candidates_run(mpap_workspace* ws, uint32_t q0, uint32_t nq, uint32_t cap, uint32_t path_cap,
                       int64_t* cost, int64_t* h, uint32_t* path_ptr, uint32_t* path, uint32_t* n_out,
                       uint32_t* total_out, uint32_t* ovf_out, cudaStream_t st) {
  const WS& w = ws->w;
  auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t b_cost = up(8 * (size_t)nq * cap), b_ref = up(4 * (size_t)nq * cap),
               b_ptr = up(4 * (size_t)nq * (cap + 1)), b_cnt = up(16 * (size_t)nq),
               b_path = up(4 * (size_t)nq * path_cap + 4);
  char* buf = nullptr;
  MPAP_CK(scratch_alloc((void**)&buf, 2 * b_cost + b_ref + b_ptr + b_cnt + b_path, st));
  CandOut o;
  o.cost = reinterpret_cast<long long*>(buf);
  o.h = reinterpret_cast<long long*>(buf + b_cost);
  o.ref = reinterpret_cast<uint32_t*>(buf + 2 * b_cost);
  o.ptr = reinterpret_cast<uint32_t*>(buf + 2 * b_cost + b_ref);
  o.counts = reinterpret_cast<uint32_t*>(buf + 2 * b_cost + b_ref + b_ptr);
  o.path = reinterpret_cast<uint32_t*>(buf + 2 * b_cost + b_ref + b_ptr + b_cnt);
  o.path_cap = path_cap;
  {
    LaunchScope ls(st, "k_candidates");
    k_candidates<<<nq, 256, 0, st>>>(w, q0, cap, o);
  }
  int32_t rc = cuda_ok(cudaGetLastError(), "k_candidates") ? MPAP_OK : MPAP_ERR_CUDA;
  std::vector<uint32_t> counts(4 * (size_t)nq);
  if (rc == MPAP_OK &&
      (!cuda_ok(cudaMemcpyAsync(counts.data(), o.counts, 16 * (size_t)nq, cudaMemcpyDeviceToHost, st), "counts") ||
       (cost && !cuda_ok(cudaMemcpyAsync(cost, o.cost, 8 * (size_t)nq * cap, cudaMemcpyDeviceToHost, st), "cost")) ||
       (h && !cuda_ok(cudaMemcpyAsync(h, o.h, 8 * (size_t)nq * cap, cudaMemcpyDeviceToHost, st), "h")) ||
       (path_ptr && !cuda_ok(cudaMemcpyAsync(path_ptr, o.ptr, 4 * (size_t)nq * (cap + 1), cudaMemcpyDeviceToHost, st),
                             "path_ptr")) ||
       (path && !cuda_ok(cudaMemcpyAsync(path, o.path, 4 * (size_t)nq * path_cap, cudaMemcpyDeviceToHost, st),
                         "path"))))
    rc = MPAP_ERR_CUDA;
  scratch_free(buf, st);
  if (!cuda_ok(cudaStreamSynchronize(st), "candidates")) rc = MPAP_ERR_CUDA;
  if (rc == MPAP_OK) {
    for (uint32_t i = 0; i < nq; ++i) {
      if (n_out) n_out[i] = counts[4 * i];
      if (total_out) total_out[i] = counts[4 * i + 1];
      if (ovf_out) ovf_out[i] = counts[4 * i + 2];
    }
  }
  return rc;
}

}  // namespace

int32_t search_candidates_impl(mpap_workspace* ws, uint32_t index, uint32_t cap, int64_t* cost, int64_t* h,
                               uint32_t* path_ptr, uint32_t* path, uint32_t path_cap, uint32_t* n_out,
                               uint32_t* total_out, cudaStream_t st) {
  const WS& w = ws->w;
  if (index >= ws->last_V.size()) {
    set_error("search_candidates: no query %u in the last search", index);
    return MPAP_ERR_INVALID_ARG;
  }
  ResultDev r;
  MPAP_CK(cudaMemcpyAsync(&r, w.res + index, sizeof(ResultDev), cudaMemcpyDeviceToHost, st));
  MPAP_CK(cudaStreamSynchronize(st));
  if (r.status != MPAP_OK) {
    set_error("search_candidates: query %u finished with status %d", index, r.status);
    return MPAP_ERR_INVALID_ARG;
  }
  if (cap == 0) {
    if (n_out) *n_out = 0;
    return MPAP_OK;
  }
  std::vector<int64_t> c(cap), hh(cap);
  std::vector<uint32_t> p(cap + 1), pa(path_cap ? path_cap : 1);
  uint32_t n = 0, total = 0, ovf = 0;
  int32_t rc = candidates_run(ws, index, 1, cap, path_cap, c.data(), hh.data(), p.data(), pa.data(), &n, &total,
                              &ovf, st);
  if (rc) return rc;
  if (n_out) *n_out = n;
  if (total_out) *total_out = total;
  if (ovf) {
    set_error("search_candidates: paths need more than path_cap = %u entries", path_cap);
    return MPAP_ERR_CAPACITY;
  }
  if (cost) std::memcpy(cost, c.data(), 8 * (size_t)n);
  if (h) std::memcpy(h, hh.data(), 8 * (size_t)n);
  if (path_ptr) std::memcpy(path_ptr, p.data(), 4 * ((size_t)n + 1));
  if (path && n) std::memcpy(path, pa.data(), 4 * (size_t)p[n]);
  return MPAP_OK;
}

int32_t search_candidates_batch_impl(mpap_workspace* ws, uint32_t nq, uint32_t cap, int64_t* cost, int64_t* h,
                                     uint32_t* path_ptr, uint32_t* path, uint32_t path_cap, uint32_t* n_out,
                                     uint32_t* total_out, cudaStream_t st) {
  if (nq > ws->last_V.size()) {
    set_error("search_candidates_batch: the last search had %zu queries", ws->last_V.size());
    return MPAP_ERR_INVALID_ARG;
  }
  if (nq == 0 || cap == 0) {
    for (uint32_t i = 0; i < nq; ++i) {
      if (n_out) n_out[i] = 0;
      if (total_out) total_out[i] = 0;
    }
    return MPAP_OK;
  }
  std::vector<uint32_t> ovf(nq);
  int32_t rc = candidates_run(ws, 0, nq, cap, path_cap, cost, h, path_ptr, path, n_out, total_out, ovf.data(), st);
  if (rc) return rc;
  for (uint32_t i = 0; i < nq; ++i)
    if (ovf[i]) {
      set_error("search_candidates_batch: query %u needs more than path_cap = %u path entries", i, path_cap);
      return MPAP_ERR_CAPACITY;
    }
  return MPAP_OK;
}


}  // namespace mpap
