// Wavefront multiobjective search: Alg. 3 (Explore) of Ichter et al., with
// RemoveDominated (Sec. 3) and the perception-heuristic cutoff h <= beta.
//
// Per wavefront (iteration i) three kernels run over all queries of a batch:
//   select  one warp per node with open plans: the group B_i of that node (its
//           open plans with cost <= i Lambda) is copied to the group array and
//           closed (P_open <- P_open \ B); every out-neighbour is marked touched.
//           A group plan at a goal node ends its query before expansion.
//   prune   one warp per touched node x ("pull"): each in-edge u -> x whose source
//           holds group plans yields candidates q = (cost + cost_q, max(C, h + S))
//           (PH(x, p) of Sec. 3), cut at beta, and merged into the stored front of
//           x.  The merge is an exact skyline under the weak Pareto order with the
//           total tie key (creation iteration, parent head): old plans win ties,
//           candidates tie-break by parent head.  Candidates are consumed in
//           chunks of 32: filter against the front, warp bitonic sort, warp
//           prefix-min, then a rank merge.  Fronts of up to 32 entries live in
//           registers (one entry per lane) for the whole merge; larger fronts are
//           merged between the node's two pool blocks in global memory.
//           Surviving candidates get arena records at the end.
//   end     one block: termination per query (goal in group, P_open empty,
//           iteration cap), list swap, loop condition.
// The loop runs on the device: the three kernels form the body of a CUDA graph
// conditional WHILE node, which `end` clears once every query has finished (or
// the iteration caps are reached), so a search is one graph launch.
//
// HBM layout (NV = nodes summed over the batch):
//   fronts   a pool of {cost i64, h i64, ref u32 (arena | open | new), aux u32}
//            entries; every node owns two blocks of it (live front, merge
//            target), of power-of-two sizes from 16 up, taken from the pool with
//            one atomic add and replaced by a block twice the needed size when
//            too small (the old block is abandoned: at most as much again)
//   fdesc    [NV] {live block, count, other block, log2 sizes}
//   group    [cap] {cost, h, ref}, per node offset/count, stamps [NV]
//   arena    [cap] {head u32, parent u32, iter u32, cost i64} for back-tracing
#include <algorithm>
#include <climits>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "internal.h"
#include "profile.h"

namespace mpap {

struct QueryDev {
  const uint32_t* rev_ptr;
  const int4* rev_edge;
  const int2* rev_peak;     // per reverse edge {Smax, Cmax} (interior check)
  const uint32_t* fwd_ptr;
  const uint32_t* fwd_dst;
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
};

struct QueryState {
  long long open_cnt;
  unsigned long long expansions;
  unsigned long long plans;
  uint32_t wavefronts;
  uint32_t goal_hit;
  uint32_t done;
  int32_t status;
  uint32_t err;          // capacity error bits of this query (pool, arena, group)
  uint32_t pad;
  unsigned long long pool_n;  // entries of its pool share handed out
};

struct ResultDev {
  long long cost;
  long long h;
  uint32_t path_len;
  int32_t status;
};

// Device-side launch timing of the loop kernels (first block start to last
// block end, %globaltimer nanoseconds).
struct KTime {
  unsigned long long start;
  unsigned long long total_ns;
  uint32_t blocks;
  uint32_t launches;
};

struct Ctl {
  uint32_t oh_n[2];
  uint32_t t_n;
  uint32_t g_n;
  unsigned long long arena_n;
  uint32_t err;
  uint32_t n_done;
  uint32_t it;          // current wavefront
  uint32_t nq;
  uint32_t iter_cap;    // loop bound (max over queries of max_iters, plus 2)
  uint32_t prof;        // record KTime
  uint32_t max_front;   // largest front committed by any node
  unsigned long long pool_n;  // front pool entries handed out
  unsigned long long tmp_n;   // bulk-merge scratch entries handed out this wavefront
  uint32_t b_n;         // nodes queued for the bulk prune this wavefront
  KTime kt[4];          // select, prune, bulk prune, end
};

struct WS {
  uint64_t NV;
  uint32_t fcap;           // front pool entries per node (pool = NV fcap)
  uint64_t pcap;           // front pool entries
  uint64_t acap, gcap;
  long long* f_cost;       // [pcap] front pool
  long long* f_h;
  uint32_t* f_pid;
  uint32_t* f_aux;
  uint4* fdesc;            // [NV] {live block, count, other block, lg live | lg other << 8}
  uint64_t tcap;           // bulk-merge scratch entries (reused every wavefront)
  long long* t_cost;       // [tcap] survivors of one run: cost, h, parent ref, insertion index
  long long* t_h;
  uint32_t* t_pp;
  uint32_t* t_m;
  uint4* gdesc;            // per node {iteration stamp, group count, group offset, 0}
  uint32_t* touch_stamp;
  uint32_t* oh_stamp;
  long long* g_cost;
  long long* g_h;
  uint32_t* g_pid;
  uint2* oh_list;           // [2][NV] {node, query} with open plans (this / next wavefront)
  uint2* t_list;            // [NV] {node, query} touched this wavefront
  uint2* b_list;            // [NV] {node, query} left to the bulk prune this wavefront
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
  // the device-side wavefront loop (built on first use)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap_stream = nullptr;
  uint32_t graph_sel = 0, graph_pru = 0;   // grids captured in the graph (blocks per SM)
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
// Resident blocks per SM the prune kernel is compiled for (register budget).
#ifndef MPAP_PRUNE_MIN_BLOCKS
#define MPAP_PRUNE_MIN_BLOCKS 4
#endif
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

// One block of 2^lg entries of query q's pool share (call from one lane);
// kNoBlock when the share is used up.  Shares are disjoint, so a query that
// runs out fails alone, whatever the others do.
__device__ __forceinline__ uint32_t pool_alloc(const WS& w, uint32_t q, uint32_t lg) {
  const unsigned long long sz = 1ull << lg;
  const unsigned long long o = atomicAdd(&w.qs[q].pool_n, sz);
  const QueryDev& Q = w.qd[q];
  return (o + sz <= Q.pool_cap) ? (uint32_t)(Q.pool_base + o) : kNoBlock;
}

// Records a capacity error of query q (it ends at the next end-of-wavefront).
__device__ __forceinline__ void query_error(const WS& w, uint32_t q, uint32_t bit) {
  atomicOr(&w.qs[q].err, bit);
  atomicOr(&w.ctl->err, bit);
}

__device__ __forceinline__ unsigned long long global_timer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void ktime_begin(const WS& w, int k) {
  if (w.ctl->prof && threadIdx.x == 0) atomicMin(&w.ctl->kt[k].start, global_timer());
}

// Every warp reports completion; the last one closes the launch (no block
// barrier, so early-finishing warps leave the SM immediately).
__device__ __forceinline__ void ktime_end(const WS& w, int k) {
  if (w.ctl->prof && (threadIdx.x & 31) == 0) {
    KTime& t = w.ctl->kt[k];
    __threadfence();
    const uint32_t total = gridDim.x * gridDim.y * ((blockDim.x + 31) >> 5);
    const uint32_t done = atomicAdd(&t.blocks, 1u);
    if (done == total - 1) {
      const unsigned long long now = global_timer();
      const unsigned long long s = atomicAdd(&t.start, 0ull);
      t.total_ns += now - s;
      t.launches += 1;
      t.start = ULLONG_MAX;
      t.blocks = 0;
      __threadfence();
    }
  }
}

// ---------------------------------------------------------------------------
__global__ void k_init(WS w, uint32_t nq, uint32_t iter_cap, uint32_t prof) {
  const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q == 0) {
    Ctl& c = *w.ctl;
    c.oh_n[0] = nq;
    c.oh_n[1] = 0;
    c.t_n = 0;
    c.g_n = 0;
    c.arena_n = nq;
    c.err = 0;
    c.n_done = 0;
    c.it = 0;
    c.nq = nq;
    c.iter_cap = iter_cap;
    c.prof = prof;
    c.max_front = 1;
    c.pool_n = 0;
    c.tmp_n = 0;
    c.b_n = 0;
    for (int k = 0; k < 4; ++k) {
      c.kt[k].start = ULLONG_MAX;
      c.kt[k].total_ns = 0;
      c.kt[k].blocks = 0;
      c.kt[k].launches = 0;
    }
  }
  if (q >= nq) return;
  const uint32_t g = w.qd[q].base;   // x_init is node 0 of every roadmap
  QueryState s;
  s.open_cnt = 1;
  s.expansions = 0;
  s.plans = 0;
  s.wavefronts = 0;
  s.goal_hit = 0;
  s.done = 0;
  s.status = 0;
  s.err = 0;
  s.pad = 0;
  s.pool_n = 1u << kMinLg;          // the root's block opens the query's share
  w.qs[q] = s;
  const uint32_t o = (uint32_t)w.qd[q].pool_base;
  w.f_cost[o] = 0;
  w.f_h[o] = 0;
  w.f_pid[o] = q | kOpen;      // the root plan (x_init, {}, 0, 0) is arena record q
  w.f_aux[o] = 0;
  w.fdesc[g] = make_uint4(o, 1u, 0u, kMinLg);
  w.a_head[q] = 0;
  w.a_parent[q] = kNone;
  w.a_iter[q] = 0;
  w.a_cost[q] = 0;
  w.oh_list[q] = make_uint2(g, q);
  w.oh_stamp[g] = 0;
}

// ---------------------------------------------------------------------------
// select: group formation, closing, goal test and marking (warp per node).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_select(WS w) {
  ktime_begin(w, 0);
  const uint32_t it = w.ctl->it;
  const unsigned lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t n_list = (w.ctl->n_done < w.ctl->nq) ? w.ctl->oh_n[it & 1] : 0u;
  const uint2* list = w.oh_list + (size_t)(it & 1) * w.NV;
  uint2* next = w.oh_list + (size_t)((it + 1) & 1) * w.NV;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n_list; k += warps) {
    const uint2 gq = list[k];
    const uint32_t g = gq.x, q = gq.y;
    if (w.qs[q].done) continue;
    const QueryDev& Q = w.qd[q];
    const uint4 fd = w.fdesc[g];
    // the out-edge range does not depend on the front: its loads go out now
    const uint32_t u = g - Q.base;
    const uint32_t e_beg = Q.fwd_ptr[u], e_end = Q.fwd_ptr[u + 1];
    const uint32_t n = fd.y;
    const size_t o = fd.x;
    const long long thr = (long long)it * Q.Lambda;
    uint32_t cnt = 0;
    bool rest = false;
    // a front of at most 32 entries stays in registers for the second pass
    uint32_t pid0 = 0;
    long long c0 = 0;
    for (uint32_t j0 = 0; j0 < n; j0 += 32) {
      const uint32_t j = j0 + lane;
      uint32_t pid = 0;
      long long c = 0;
      if (j < n) {
        pid = w.f_pid[o + j];
        c = w.f_cost[o + j];
      }
      if (j0 == 0) {
        pid0 = pid;
        c0 = c;
      }
      const bool open = (j < n) && (pid & kOpen);
      cnt += __popc(__ballot_sync(kFull, open && c <= thr));
      rest = rest || __any_sync(kFull, open && c > thr);
    }
    if (cnt) {
      uint32_t off = 0;
      if (lane == 0) off = atomicAdd(&w.ctl->g_n, cnt);
      off = __shfl_sync(kFull, off, 0);
      const bool fits = (uint64_t)off + cnt <= w.gcap;
      if (!fits) {
        if (lane == 0) query_error(w, q, kErrGroup);
      } else {
        uint32_t r0 = 0;
        for (uint32_t j0 = 0; j0 < n; j0 += 32) {
          const uint32_t j = j0 + lane;
          uint32_t pid = pid0;
          long long c = c0;
          if (j0 > 0 && j < n) {
            pid = w.f_pid[o + j];
            c = w.f_cost[o + j];
          }
          const bool isg = (j < n) && (pid & kOpen) && c <= thr;
          const unsigned bal = __ballot_sync(kFull, isg);
          if (isg) {
            const uint32_t r = off + r0 + __popc(bal & lt);
            w.g_cost[r] = c;
            w.g_h[r] = w.f_h[o + j];
            w.g_pid[r] = pid & kPidMask;
            w.f_pid[o + j] = pid & ~kOpen;
          }
          r0 += __popc(bal);
        }
        if (lane == 0) {
          w.gdesc[g] = make_uint4(it, cnt, off, 0u);
          atomic_add_i64(&w.qs[q].open_cnt, -(long long)cnt);
          if (Q.is_goal[u]) w.qs[q].goal_hit = 1u;
        }
        // mark the out-neighbours of this node as touched (deduplicated by stamp;
        // a plain read first skips the atomic for nodes already marked), 64 edges
        // per step with the loads of both halves in flight together
        for (uint32_t e0 = e_beg; e0 < e_end; e0 += 64) {
          const uint32_t ea = e0 + lane, eb = e0 + 32 + lane;
          const bool va = ea < e_end, vb = eb < e_end;
          const uint32_t ga = va ? Q.base + __ldg(&Q.fwd_dst[ea]) : 0u;
          const uint32_t gb = vb ? Q.base + __ldg(&Q.fwd_dst[eb]) : 0u;
          const uint32_t sa = va ? w.touch_stamp[ga] : it;
          const uint32_t sb = vb ? w.touch_stamp[gb] : it;
          bool fa = false, fb = false;
          if (sa != it) fa = atomicExch(&w.touch_stamp[ga], it) != it;
          if (sb != it) fb = atomicExch(&w.touch_stamp[gb], it) != it;
          const unsigned bala = __ballot_sync(kFull, fa), balb = __ballot_sync(kFull, fb);
          if (bala | balb) {
            uint32_t pos = 0;
            if (lane == 0) pos = atomicAdd(&w.ctl->t_n, __popc(bala) + __popc(balb));
            pos = __shfl_sync(kFull, pos, 0);
            if (fa) w.t_list[pos + __popc(bala & lt)] = make_uint2(ga, q);
            if (fb) w.t_list[pos + __popc(bala) + __popc(balb & lt)] = make_uint2(gb, q);
          }
        }
      }
    }
    if (rest && lane == 0) {
      if (atomicExch(&w.oh_stamp[g], it + 1) != it + 1) next[atomicAdd(&w.ctl->oh_n[(it + 1) & 1], 1u)] = make_uint2(g, q);
    }
  }
  ktime_end(w, 0);
}

// ---------------------------------------------------------------------------
// prune: pull candidates into the front of each touched node (warp per node).
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

// Bulk merge of one in-edge's candidate run into a block-mode front.  The run is
// the source's group (a contiguous part of its front: costs increasing, h
// decreasing) shifted along one edge, so its costs increase and its h do not
// increase: it is its own skyline once entries whose h equals their
// predecessor's are dropped.  Pass 1 keeps the run entries that pass the beta
// cutoff and survive the live front, compacting them into a temporary pool block
// with their insertion index m (front entries of lower or equal cost); pass 2
// sweeps the front once, dropping the entries a survivor dominates and
// interleaving the survivors.  O(n/32 + L log n / 32) warp steps per run, against
// O(L/32 * n/32) for chunked merging.
// Returns false (and changes nothing) when this wavefront's scratch is used up;
// the caller then merges the run in chunks.
__device__ __forceinline__ bool merge_run_bulk(const WS& w, uint32_t q, FrontCursor& fc, long long beta, uint32_t goff,
                                               uint32_t L, int cq, int S, int C, int Sm, int Cm, bool interior,
                                               uint32_t tb) {
  const unsigned lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  const size_t o = fc.off;
  const uint32_t n = fc.n;
  // run entry r: candidate, and whether it passes the cutoff, its run
  // predecessor and the live front (m = front entries of lower or equal cost)
  auto entry = [&](uint32_t r, long long& cc, long long& ch, uint32_t& pp, uint32_t& m) -> bool {
    const uint32_t gi = goff + r;
    const long long gh = w.g_h[gi];
    cc = w.g_cost[gi] + (long long)cq;
    const long long hh = gh + (long long)S;
    ch = hh > (long long)C ? hh : (long long)C;
    pp = w.g_pid[gi];
    long long peak = ch;
    if (interior) {
      const long long hp = gh + (long long)Sm;
      peak = hp > (long long)Cm ? hp : (long long)Cm;
    }
    if (peak > beta) return false;
    if (r > 0) {
      // the run predecessor (lower cost, h never lower) dominates iff its h is equal
      const long long ph = w.g_h[gi - 1] + (long long)S;
      const long long pch = ph > (long long)C ? ph : (long long)C;
      if (pch <= ch) return false;
    }
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (w.f_cost[o + mid] <= cc) lo = mid + 1; else hi = mid;
    }
    m = lo;
    if (lo > 0) {
      const uint32_t j = lo - 1;
      const long long fcost = w.f_cost[o + j], fh = w.f_h[o + j];
      const uint32_t fpid = w.f_pid[o + j];
      const uint32_t ftb = (fpid & kNew) ? w.f_aux[o + j] : 0u;
      if (fh <= ch && (fcost < cc || fh < ch || ftb < tb)) return false;
    }
    return true;
  };
  // pass 1a: count the survivors, then take exactly that much scratch
  uint32_t ns = 0;
  for (uint32_t r0 = 0; r0 < L; r0 += 32) {
    const uint32_t r = r0 + lane;
    long long cc, ch;
    uint32_t pp, m;
    ns += __popc(__ballot_sync(kFull, r < L && entry(r, cc, ch, pp, m)));
  }
  if (ns == 0) return true;
  unsigned long long T = 0;
  if (lane == 0) T = atomicAdd(&w.ctl->tmp_n, (unsigned long long)ns);
  T = __shfl_sync(kFull, T, 0);
  if (T + ns > w.tcap) return false;
  // pass 1b: the survivors, in run order, with their insertion index m
  uint32_t k = 0;
  for (uint32_t r0 = 0; r0 < L; r0 += 32) {
    const uint32_t r = r0 + lane;
    long long cc = 0, ch = 0;
    uint32_t pp = 0, m = 0;
    const bool ok = r < L && entry(r, cc, ch, pp, m);
    const unsigned sb = __ballot_sync(kFull, ok);
    if (ok) {
      const size_t t = (size_t)T + k + __popc(sb & lt);
      w.t_cost[t] = cc;
      w.t_h[t] = ch;
      w.t_pp[t] = pp;
      w.t_m[t] = m;
    }
    k += __popc(sb);
  }
  if (!ensure_other(w, q, fc, n + ns)) return true;
  __syncwarp();
  // pass 2: one sweep over the front
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
    const uint32_t ftb = (fpid & kNew) ? faux : 0u;
    // survivors of lower or equal cost; the last of them is the only one that can dominate
    uint32_t lo = 0, hi = ns;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (w.t_cost[(size_t)T + mid] <= fcost) lo = mid + 1; else hi = mid;
    }
    bool dom = false;
    if (valid && lo > 0) {
      const long long sc = w.t_cost[(size_t)T + lo - 1], sh = w.t_h[(size_t)T + lo - 1];
      dom = sh <= fh && (sc < fcost || sh < fh || tb < ftb);
    }
    const bool keep = valid && !dom;
    if (dom && (fpid & kOpen) && !(fpid & kNew)) rem_open++;
    const unsigned kb = __ballot_sync(kFull, keep);
    if (keep) {
      const size_t pos = on + K + __popc(kb & lt) + lo;
      w.f_cost[pos] = fcost;
      w.f_h[pos] = fh;
      w.f_pid[pos] = fpid;
      w.f_aux[pos] = faux;
    }
    // survivors inserted before a front entry of this chunk (m < end of chunk)
    const uint32_t jend = min(j0 + 32u, n);
    for (;;) {
      const uint32_t s = sp + lane;
      bool emit = false;
      uint32_t m = 0;
      if (s < ns) {
        m = w.t_m[(size_t)T + s];
        emit = m < jend;
      }
      const unsigned eb = __ballot_sync(kFull, emit);
      if (emit) {
        const uint32_t d = m - j0;   // 0 .. 31: earlier chunks emitted every m < j0
        const size_t pos = on + s + K + __popc(kb & ((1u << d) - 1u));
        w.f_cost[pos] = w.t_cost[(size_t)T + s];
        w.f_h[pos] = w.t_h[(size_t)T + s];
        w.f_pid[pos] = w.t_pp[(size_t)T + s] | kNew;
        w.f_aux[pos] = tb;
      }
      const uint32_t c = __popc(eb);
      sp += c;
      if (c < 32) break;
    }
    K += __popc(kb);
  }
  // survivors after every front entry
  for (uint32_t s0 = sp; s0 < ns; s0 += 32) {
    const uint32_t s = s0 + lane;
    if (s < ns) {
      const size_t pos = on + s + K;
      w.f_cost[pos] = w.t_cost[(size_t)T + s];
      w.f_h[pos] = w.t_h[(size_t)T + s];
      w.f_pid[pos] = w.t_pp[(size_t)T + s] | kNew;
      w.f_aux[pos] = tb;
    }
  }
  for (int sft = 16; sft > 0; sft >>= 1) rem_open += __shfl_xor_sync(kFull, rem_open, sft);
  fc.removed_open += rem_open;
  swap_blocks(fc);
  fc.n = K + ns;
  fc.any_new = true;
  __syncwarp();
  return true;
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
    unsigned long long a0 = 0;
    if (lane == 0) a0 = atomicAdd(&w.ctl->arena_n, (unsigned long long)__popc(bal));
    a0 = __shfl_sync(kFull, a0, 0);
    if (isnew) {
      const unsigned long long a = a0 + __popc(bal & lt);
      if (a < w.acap) {
        w.a_head[a] = x;
        w.a_parent[a] = pid & kPidMask;
        w.a_iter[a] = it + 1;
        w.a_cost[a] = w.f_cost[o + j];
        w.f_pid[o + j] = (uint32_t)a | kOpen;
      } else {
        query_error(w, q, kErrArena);
        w.f_pid[o + j] = kOpen;
      }
      w.f_aux[o + j] = 0;
    }
    n_new += __popc(bal);
  }
  return n_new;
}

// The node's new descriptor and counters, and its place in the next open list.
__device__ __forceinline__ void commit_tail(const WS& w, uint32_t q, uint32_t g, uint32_t it, const FrontCursor& fc,
                                            uint32_t n_new, uint2* next) {
  if (lane_id() == 0) {
    w.fdesc[g] = make_uint4(fc.off, fc.n, fc.off2, fc.lg | (fc.lg2 << 8));
    atomic_add_i64(&w.qs[q].open_cnt, (long long)n_new - (long long)fc.removed_open);
    atomicAdd(&w.qs[q].plans, (unsigned long long)n_new);
    atomicMax(&w.ctl->max_front, fc.n);
    if (atomicExch(&w.oh_stamp[g], it + 1) != it + 1) next[atomicAdd(&w.ctl->oh_n[(it + 1) & 1], 1u)] = make_uint2(g, q);
  }
}

// One node whose front is in block mode (more than 32 plans) at the start of the
// wavefront: if its in-edge runs are long on average every run is merged in
// bulk, otherwise its candidates are merged in chunks of 32; then the front is
// committed.
__device__ __forceinline__ void prune_node_bulk(const WS& w, WarpSmem& sm, uint32_t q, uint32_t g, uint32_t x,
                                             const QueryDev& Q, uint32_t it, uint32_t e_beg, uint32_t e_end,
                                             bool interior, uint2* next) {
  const unsigned lane = lane_id();
  FrontCursor fc;
  {
    const uint4 fd = w.fdesc[g];
    fc.off = fd.x;
    fc.n = fd.y;
    fc.off2 = fd.z;
    fc.lg = fd.w & 0xFFu;
    fc.lg2 = (fd.w >> 8) & 0xFFu;
  }
  fc.reg = false;
  fc.err = false;
  fc.removed_open = 0;
  fc.any_new = false;
  fc.rc = fc.rh = 0;
  fc.rp = fc.ra = 0;
  unsigned long long exps = 0;
  // runs long on average (more than 32 candidates per run): bulk merges; else
  // all candidates in chunks of 32
  uint32_t ctot = 0, runs = 0;
  for (uint32_t e0 = e_beg; e0 < e_end; e0 += 32) {
    const uint32_t e = e0 + lane;
    uint32_t cnt = 0;
    if (e < e_end) {
      const uint4 gd = w.gdesc[Q.base + (uint32_t)__ldg(&Q.rev_edge[e]).x];
      if (gd.x == it) cnt = gd.y;
    }
    ctot += __reduce_add_sync(kFull, cnt);
    runs += __popc(__ballot_sync(kFull, cnt > 0));
  }
  const bool bulk = ctot > 32u * runs;
  for (uint32_t e0 = e_beg; e0 < e_end; e0 += 32) {
    const uint32_t e = e0 + lane;
    int4 ed = make_int4(0, 0, 0, 0);
    int2 pk = make_int2(0, 0);
    uint32_t cnt = 0, goff = 0;
    if (e < e_end) {
      ed = __ldg(&Q.rev_edge[e]);
      if (interior) pk = __ldg(&Q.rev_peak[e]);
      const uint4 gd = w.gdesc[Q.base + (uint32_t)ed.x];
      if (gd.x == it) {
        cnt = gd.y;
        goff = gd.z;
      }
    }
    exps += __reduce_add_sync(kFull, cnt);
    if (!bulk) {
      // chunked: candidates of all runs of this chunk of in-edges, 32 at a time
      const uint32_t incl = warp_incl_scan(cnt);
      const uint32_t total = __shfl_sync(kFull, incl, 31);
      const uint32_t excl = incl - cnt;
      for (uint32_t c0 = 0; c0 < total && !fc.err; c0 += 32) {
        const uint32_t c = c0 + lane;
        uint32_t owner = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const uint32_t probe = owner + step;
          if (__shfl_sync(kFull, excl, probe) <= c) owner = probe;
        }
        const uint32_t o_excl = __shfl_sync(kFull, excl, owner), o_goff = __shfl_sync(kFull, goff, owner);
        const int o_src = __shfl_sync(kFull, ed.x, owner), o_cq = __shfl_sync(kFull, ed.y, owner);
        const int o_S = __shfl_sync(kFull, ed.z, owner), o_C = __shfl_sync(kFull, ed.w, owner);
        const int o_Sm = __shfl_sync(kFull, pk.x, owner), o_Cm = __shfl_sync(kFull, pk.y, owner);
        bool ok = false;
        long long cc = 0, ch = 0;
        uint32_t pp = 0;
        if (c < total) {
          const uint32_t gi = o_goff + (c - o_excl);
          const long long gh = w.g_h[gi];
          cc = w.g_cost[gi] + (long long)o_cq;
          const long long hh = gh + (long long)o_S;
          ch = hh > (long long)o_C ? hh : (long long)o_C;
          pp = w.g_pid[gi];
          long long peak = ch;
          if (interior) {
            const long long hp = gh + (long long)o_Sm;
            peak = hp > (long long)o_Cm ? hp : (long long)o_Cm;
          }
          ok = peak <= Q.beta;
        }
        merge_chunk_slab(w, q, fc, sm, ok, cc, ch, 1u + (uint32_t)o_src, pp);
      }
      continue;
    }
    for (unsigned rb = __ballot_sync(kFull, cnt > 0); rb; rb &= rb - 1) {
      const int l = __ffs(rb) - 1;
      const uint32_t r_goff = __shfl_sync(kFull, goff, l), r_cnt = __shfl_sync(kFull, cnt, l);
      const int r_src = __shfl_sync(kFull, ed.x, l), r_cq = __shfl_sync(kFull, ed.y, l);
      const int r_S = __shfl_sync(kFull, ed.z, l), r_C = __shfl_sync(kFull, ed.w, l);
      const int r_Sm = __shfl_sync(kFull, pk.x, l), r_Cm = __shfl_sync(kFull, pk.y, l);
      if (fc.err) continue;
      if (merge_run_bulk(w, q, fc, Q.beta, r_goff, r_cnt, r_cq, r_S, r_C, r_Sm, r_Cm, interior, 1u + (uint32_t)r_src))
        continue;
      // scratch used up this wavefront: merge the run in chunks of 32
      for (uint32_t r0 = 0; r0 < r_cnt && !fc.err; r0 += 32) {
        const uint32_t r = r0 + lane;
        bool ok = false;
        long long cc = 0, ch = 0;
        uint32_t pp = 0;
        if (r < r_cnt) {
          const uint32_t gi = r_goff + r;
          const long long gh = w.g_h[gi];
          cc = w.g_cost[gi] + (long long)r_cq;
          const long long hh = gh + (long long)r_S;
          ch = hh > (long long)r_C ? hh : (long long)r_C;
          pp = w.g_pid[gi];
          long long peak = ch;
          if (interior) {
            const long long hp = gh + (long long)r_Sm;
            peak = hp > (long long)r_Cm ? hp : (long long)r_Cm;
          }
          ok = peak <= Q.beta;
        }
        merge_chunk_slab(w, q, fc, sm, ok, cc, ch, 1u + (uint32_t)r_src, pp);
      }
    }
  }
  if (fc.any_new && !fc.err) commit_tail(w, q, g, it, fc, arena_block(w, q, x, it, fc), next);
  if (lane == 0 && exps) atomicAdd(&w.qs[q].expansions, exps);
}

__global__ void __launch_bounds__(kWarpsPerBlock * 32, MPAP_PRUNE_MIN_BLOCKS) k_prune(WS w) {
  ktime_begin(w, 1);
  __shared__ WarpSmem smem[kWarpsPerBlock];
  WarpSmem& sm = smem[threadIdx.x >> 5];
  const uint32_t it = w.ctl->it;
  const unsigned lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t n_list = (w.ctl->n_done < w.ctl->nq) ? w.ctl->t_n : 0u;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  uint2* next = w.oh_list + (size_t)((it + 1) & 1) * w.NV;
  for (uint32_t k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n_list; k += warps) {
    const uint2 gq = w.t_list[k];
    const uint32_t g = gq.x, q = gq.y;
    const QueryDev& Q = w.qd[q];
    {
      const QueryState& s = w.qs[q];
      if (s.done || (s.goal_hit && !(Q.flags & MPAP_QUERY_NO_GOAL_STOP)) || s.wavefronts >= Q.max_iters)
        continue;
    }
    const uint32_t x = g - Q.base;
    FrontCursor fc;
    {
      const uint4 fd = w.fdesc[g];
      fc.off = fd.x;
      fc.n = fd.y;
      fc.off2 = fd.z;
      fc.lg = fd.w & 0xFFu;
      fc.lg2 = (fd.w >> 8) & 0xFFu;
    }
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
    unsigned long long exps = 0;
    const uint32_t e_end = Q.rev_ptr[x + 1];
    const bool interior = (Q.flags & MPAP_QUERY_CHECK_INTERIOR) != 0;
    // a front in block mode from the start goes to the bulk prune kernel
    const bool to_bulk = !fc.reg;
    for (uint32_t e0 = to_bulk ? e_end : Q.rev_ptr[x]; e0 < e_end; e0 += 32) {
      const uint32_t e = e0 + lane;
      int4 ed = make_int4(0, 0, 0, 0);
      int2 pk = make_int2(0, 0);
      uint32_t cnt = 0, goff = 0;
      if (e < e_end) {
        ed = __ldg(&Q.rev_edge[e]);
        if (interior) pk = __ldg(&Q.rev_peak[e]);
        const uint4 gd = w.gdesc[Q.base + (uint32_t)ed.x];
        if (gd.x == it) {
          cnt = gd.y;
          goff = gd.z;
        }
      }
      const uint32_t incl = warp_incl_scan(cnt);
      const uint32_t total = __shfl_sync(kFull, incl, 31);
      const uint32_t excl = incl - cnt;
      exps += total;
      for (uint32_t c0 = 0; c0 < total; c0 += 32) {
        const uint32_t c = c0 + lane;
        // owner lane: the last lane whose exclusive offset is <= c
        uint32_t owner = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const uint32_t probe = owner + step;
          const uint32_t ev = __shfl_sync(kFull, excl, probe);
          if (ev <= c) owner = probe;
        }
        const uint32_t o_excl = __shfl_sync(kFull, excl, owner);
        const uint32_t o_goff = __shfl_sync(kFull, goff, owner);
        const int o_src = __shfl_sync(kFull, ed.x, owner);
        const int o_cq = __shfl_sync(kFull, ed.y, owner);
        const int o_S = __shfl_sync(kFull, ed.z, owner);
        const int o_C = __shfl_sync(kFull, ed.w, owner);
        const int o_Sm = __shfl_sync(kFull, pk.x, owner);
        const int o_Cm = __shfl_sync(kFull, pk.y, owner);
        bool ok = false;
        long long cc = 0, ch = 0;
        uint32_t pp = 0;
        if (c < total) {
          const uint32_t gi = o_goff + (c - o_excl);
          cc = w.g_cost[gi] + (long long)o_cq;
          const long long hh = w.g_h[gi] + (long long)o_S;
          ch = hh > (long long)o_C ? hh : (long long)o_C;
          pp = w.g_pid[gi];
          // perception-heuristic cutoff: at the new head (Alg. 3), or at every
          // sub-step of the edge (Eq. 2 for all t)
          long long peak = ch;
          if (interior) {
            const long long hp = w.g_h[gi] + (long long)o_Sm;
            peak = hp > (long long)o_Cm ? hp : (long long)o_Cm;
          }
          ok = peak <= Q.beta;
        }
        if (fc.err) continue;
        if (fc.reg) merge_chunk_reg(w, q, fc, sm, ok, cc, ch, 1u + (uint32_t)o_src, pp);
        else merge_chunk_slab(w, q, fc, sm, ok, cc, ch, 1u + (uint32_t)o_src, pp);
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
      if (fc.reg) {
        const bool isnew = lane < fc.n && (fc.rp & kNew);
        const unsigned bal = __ballot_sync(kFull, isnew);
        unsigned long long a0 = 0;
        if (lane == 0 && bal) a0 = atomicAdd(&w.ctl->arena_n, (unsigned long long)__popc(bal));
        a0 = __shfl_sync(kFull, a0, 0);
        if (isnew) {
          const unsigned long long a = a0 + __popc(bal & lt);
          if (a < w.acap) {
            w.a_head[a] = x;
            w.a_parent[a] = fc.rp & kPidMask;
            w.a_iter[a] = it + 1;
            w.a_cost[a] = fc.rc;
            fc.rp = (uint32_t)a | kOpen;
          } else {
            query_error(w, q, kErrArena);
            fc.rp = kOpen;
          }
          fc.ra = 0;
        }
        n_new = __popc(bal);
        // write the register front to the live block
        const size_t o = fc.off;
        if (lane < fc.n) {
          w.f_cost[o + lane] = fc.rc;
          w.f_h[o + lane] = fc.rh;
          w.f_pid[o + lane] = fc.rp;
          w.f_aux[o + lane] = fc.ra;
        }
      } else {
        n_new = arena_block(w, q, x, it, fc);
      }
      commit_tail(w, q, g, it, fc, n_new, next);
    }
    if (lane == 0 && exps) atomicAdd(&w.qs[q].expansions, exps);
    if (to_bulk && lane == 0) w.b_list[atomicAdd(&w.ctl->b_n, 1u)] = make_uint2(g, q);
  }
  ktime_end(w, 1);
}

// ---------------------------------------------------------------------------
// bulk prune: the nodes k_prune queued (fronts in block mode at the start of
// the wavefront), warp per node.  A kernel of its own, so that the
// register-mode path of k_prune keeps its registers.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 2) k_prune_bulk(WS w) {
  ktime_begin(w, 2);
  __shared__ WarpSmem smem[kWarpsPerBlock];
  WarpSmem& sm = smem[threadIdx.x >> 5];
  const uint32_t it = w.ctl->it;
  const uint32_t n_list = (w.ctl->n_done < w.ctl->nq) ? w.ctl->b_n : 0u;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  uint2* next = w.oh_list + (size_t)((it + 1) & 1) * w.NV;
  for (uint32_t k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n_list; k += warps) {
    const uint2 gq = w.b_list[k];
    const uint32_t g = gq.x, q = gq.y;
    const QueryDev& Q = w.qd[q];
    const uint32_t x = g - Q.base;
    prune_node_bulk(w, sm, q, g, x, Q, it, Q.rev_ptr[x], Q.rev_ptr[x + 1], (Q.flags & MPAP_QUERY_CHECK_INTERIOR) != 0,
                    next);
  }
  ktime_end(w, 2);
}

// ---------------------------------------------------------------------------
// end of wavefront (one block): termination per query, list swap, loop control.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_end(WS w, cudaGraphConditionalHandle cond, uint32_t in_graph) {
  ktime_begin(w, 3);
  __shared__ uint32_t s_newly;
  const uint32_t it = w.ctl->it, nq = w.ctl->nq;
  if (threadIdx.x == 0) s_newly = 0;
  __syncthreads();
  for (uint32_t q = threadIdx.x; q < nq; q += blockDim.x) {
    QueryState& s = w.qs[q];
    const QueryDev& Q = w.qd[q];
    if (s.done) continue;
    if (s.err) {
      s.done = 1;
      s.status = MPAP_ERR_CAPACITY;
    } else if (s.goal_hit && !(Q.flags & MPAP_QUERY_NO_GOAL_STOP)) {
      s.done = 1;
    } else if (s.wavefronts >= Q.max_iters) {
      s.done = 1;
      s.status = MPAP_ERR_ITER_LIMIT;
    } else {
      s.wavefronts += 1;
      if (s.open_cnt == 0) s.done = 1;
    }
    if (s.done) atomicAdd(&s_newly, 1u);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t done = w.ctl->n_done + s_newly;
    w.ctl->n_done = done;
    // the list consumed in this iteration becomes the append target of the next
    w.ctl->oh_n[it & 1] = 0;
    w.ctl->t_n = 0;
    w.ctl->g_n = 0;
    w.ctl->tmp_n = 0;
    w.ctl->b_n = 0;
    w.ctl->it = it + 1;
    if (in_graph) cudaGraphSetConditional(cond, (done < nq && it + 1 < w.ctl->iter_cap) ? 1u : 0u);
  }
  ktime_end(w, 3);
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
      const uint4 fd = w.fdesc[g];
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
    r.status = s.done ? s.status : MPAP_ERR_ITER_LIMIT;
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
      const uint4 fd = w.fdesc[g];
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
    const uint4 fd = w.fdesc[base + v];
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

template <typename T>
bool walloc(T** p, size_t n) {
  return cuda_ok(cudaMalloc((void**)p, (n ? n : 1) * sizeof(T)), "cudaMalloc(workspace)");
}

// Builds the device-side wavefront loop: a graph whose conditional WHILE node
// runs {select, prune, end} until `end` clears the condition.
int32_t build_loop_graph(mpap_workspace* ws, uint32_t sel, uint32_t pru) {
  if (ws->exec && ws->graph_sel == sel && ws->graph_pru == pru) return MPAP_OK;
  if (ws->exec) {
    cudaGraphExecDestroy(ws->exec);
    ws->exec = nullptr;
  }
  if (ws->graph) {
    cudaGraphDestroy(ws->graph);
    ws->graph = nullptr;
  }
  if (!ws->cap_stream) MPAP_CK(cudaStreamCreateWithFlags(&ws->cap_stream, cudaStreamNonBlocking));
  MPAP_CK(cudaGraphCreate(&ws->graph, 0));
  cudaGraphConditionalHandle cond;
  MPAP_CK(cudaGraphConditionalHandleCreate(&cond, ws->graph, 1u, cudaGraphCondAssignDefault));
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = cond;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  MPAP_CK(cudaGraphAddNode(&node, ws->graph, nullptr, nullptr, 0, &p));
  cudaGraph_t body = p.conditional.phGraph_out[0];
  MPAP_CK(cudaStreamBeginCaptureToGraph(ws->cap_stream, body, nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal));
  const int n = sms();
  k_select<<<sel * n, kWarpsPerBlock * 32, 0, ws->cap_stream>>>(ws->w);
  k_prune<<<pru * n, kWarpsPerBlock * 32, 0, ws->cap_stream>>>(ws->w);
  k_prune_bulk<<<2 * n, kWarpsPerBlock * 32, 0, ws->cap_stream>>>(ws->w);
  k_end<<<1, 1024, 0, ws->cap_stream>>>(ws->w, cond, 1u);
  cudaGraph_t captured = nullptr;
  MPAP_CK(cudaStreamEndCapture(ws->cap_stream, &captured));
  MPAP_CK(cudaGraphInstantiate(&ws->exec, ws->graph, 0));
  ws->graph_sel = sel;
  ws->graph_pru = pru;
  return MPAP_OK;
}

}  // namespace

bool host_stepped_loop() {
  static const bool host = [] {
    const char* e = getenv("MPAP_SEARCH_LOOP");
    return e && std::strcmp(e, "host") == 0;
  }();
  return host;
}

int32_t workspace_create(uint64_t total_nodes, uint32_t front_cap, uint64_t max_plans, uint32_t max_q,
                         mpap_workspace** out) {
  if (!out || total_nodes == 0 || total_nodes > 0xFFFFFFF0ull || front_cap == 0 || max_plans == 0 ||
      max_plans > (uint64_t)kPidMask) {
    set_error("mpap_workspace_create: invalid sizes");
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
  w.tcap = max_plans;
  w.path_cap = 4096;
  ws->max_q = max_q;
  const size_t slots = (size_t)w.pcap;
  bool ok = walloc(&w.f_cost, slots) && walloc(&w.f_h, slots) && walloc(&w.f_pid, slots) &&
            walloc(&w.f_aux, slots) && walloc(&w.fdesc, w.NV) && walloc(&w.t_cost, w.tcap) && walloc(&w.t_h, w.tcap) &&
            walloc(&w.t_pp, w.tcap) && walloc(&w.t_m, w.tcap) &&
            walloc(&w.gdesc, w.NV) && walloc(&w.touch_stamp, w.NV) &&
            walloc(&w.oh_stamp, w.NV) &&
            walloc(&w.g_cost, w.gcap) && walloc(&w.g_h, w.gcap) && walloc(&w.g_pid, w.gcap) &&
            walloc(&w.oh_list, 2 * w.NV) && walloc(&w.t_list, w.NV) && walloc(&w.b_list, w.NV) && walloc(&w.a_head, w.acap) &&
            walloc(&w.a_parent, w.acap) && walloc(&w.a_iter, w.acap) && walloc(&w.a_cost, w.acap) &&
            walloc(&w.ctl, 1) && walloc(&w.qd, max_q) && walloc(&w.qs, max_q) && walloc(&w.res, max_q) &&
            walloc(&w.path, (size_t)max_q * w.path_cap);
  if (!ok) {
    workspace_free(ws);
    return MPAP_ERR_CUDA;
  }
  *out = ws;
  return MPAP_OK;
}

void workspace_free(mpap_workspace* ws) {
  if (!ws) return;
  if (ws->exec) cudaGraphExecDestroy(ws->exec);
  if (ws->graph) cudaGraphDestroy(ws->graph);
  if (ws->cap_stream) cudaStreamDestroy(ws->cap_stream);
  WS& w = ws->w;
  void* ptrs[] = {w.f_cost, w.f_h, w.f_pid, w.f_aux, w.fdesc, w.t_cost, w.t_h, w.t_pp, w.t_m, w.gdesc, w.touch_stamp,
                  w.oh_stamp, w.g_cost, w.g_h, w.g_pid, w.oh_list, w.t_list, w.b_list,
                  w.a_head, w.a_parent, w.a_iter, w.a_cost, w.ctl, w.qd, w.qs, w.res, w.path};
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
    d.rev_ptr = rm->rev_ptr;
    d.rev_edge = rm->rev_edge;
    d.fwd_ptr = rm->fwd_ptr;
    d.fwd_dst = rm->fwd_dst;
    d.is_goal = rm->is_goal;
    d.goal_list = rm->goal_list;
    d.n_goal = rm->n_goal;
    d.V = rm->V;
    d.base = (uint32_t)total;
    d.max_iters = qs[i].max_iters;
    d.flags = qs[i].flags;
    d.beta = qs[i].beta;
    d.rev_peak = rm->rev_peak;
    // Lambda = round(lambda r_n 2^24), the group threshold quantum (or the
    // caller's explicit width in cost quanta).
    d.Lambda = qs[i].group_width_q > 0 ? qs[i].group_width_q
                                       : (int64_t)llrint((double)qs[i].lambda * (double)rm->r * 16777216.0);
    if (d.Lambda < 1) d.Lambda = 1;
    total += rm->V;
    max_iters = std::max(max_iters, qs[i].max_iters);
    qd[i] = d;
  }
  if (total > w.NV) {
    set_error("search: %llu nodes exceed the workspace's %llu", (unsigned long long)total,
              (unsigned long long)w.NV);
    return MPAP_ERR_INVALID_ARG;
  }
  // every query gets a share of the front pool in proportion to its nodes
  {
    uint64_t acc = 0;
    for (uint32_t i = 0; i < nq; ++i) {
      const uint64_t cap = (i + 1 == nq) ? w.pcap - acc : (uint64_t)((double)w.pcap * qd[i].V / (double)total);
      if (cap < 16) {
        set_error("search: query %u's share of the front pool is below 16 entries", i);
        return MPAP_ERR_CAPACITY;
      }
      qd[i].pool_base = acc;
      qd[i].pool_cap = cap;
      acc += cap;
    }
  }
  int kdim = -1;
  uint32_t kV = 0;
  batch_key(rms, nq, kdim, kV);
  const mpap_tuning tun = tuning_for(kdim, kV);
  int32_t rc = build_loop_graph(ws, tun.select_blocks_per_sm, tun.prune_blocks_per_sm);
  if (rc) return rc;
  ws->last_V.resize(nq);
  ws->last_base.resize(nq);
  for (uint32_t i = 0; i < nq; ++i) {
    ws->last_V[i] = qd[i].V;
    ws->last_base[i] = qd[i].base;
  }
  const size_t NVu = (size_t)total;
  const bool prof = profile_enabled();
  MPAP_CK(cudaMemcpyAsync(w.qd, qd.data(), sizeof(QueryDev) * nq, cudaMemcpyHostToDevice, st));
  MPAP_CK(cudaMemsetAsync(w.fdesc, 0, sizeof(uint4) * NVu, st));
  MPAP_CK(cudaMemsetAsync(w.gdesc, 0xFF, sizeof(uint4) * NVu, st));
  MPAP_CK(cudaMemsetAsync(w.touch_stamp, 0xFF, sizeof(uint32_t) * NVu, st));
  MPAP_CK(cudaMemsetAsync(w.oh_stamp, 0xFF, sizeof(uint32_t) * NVu, st));
  {
    LaunchScope ls(st, "k_init");
    k_init<<<(nq + 127) / 128, 128, 0, st>>>(w, nq, max_iters + 2u, prof ? 1u : 0u);
  }
  MPAP_CK(cudaGetLastError());
  if (!host_stepped_loop()) {
    // the whole wavefront loop: one graph launch
    MPAP_CK(cudaGraphLaunch(ws->exec, st));
  } else {
    // Host-stepped form of the same loop (MPAP_SEARCH_LOOP=host): identical
    // kernels launched one wavefront at a time, for per-kernel profilers that do
    // not see inside conditional graph nodes.
    const int n = sms();
    Ctl probe;
    for (uint32_t it = 0;; it += 2) {
      for (int r = 0; r < 2; ++r) {
        k_select<<<tun.select_blocks_per_sm * n, kWarpsPerBlock * 32, 0, st>>>(w);
        k_prune<<<tun.prune_blocks_per_sm * n, kWarpsPerBlock * 32, 0, st>>>(w);
        k_prune_bulk<<<2 * n, kWarpsPerBlock * 32, 0, st>>>(w);
        k_end<<<1, 1024, 0, st>>>(w, 0ull, 0u);
      }
      MPAP_CK(cudaGetLastError());
      MPAP_CK(cudaMemcpyAsync(&probe, w.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
      MPAP_CK(cudaStreamSynchronize(st));
      if (probe.n_done >= nq || probe.it >= max_iters + 2u) break;
    }
  }
  {
    LaunchScope ls(st, "k_finalize");
    k_finalize<<<nq, 256, 0, st>>>(w, nq);
  }
  MPAP_CK(cudaGetLastError());
  // results, query states and the control block: three copies into pinned staging
  const size_t o_qs = align64(sizeof(ResultDev) * nq), o_ctl = o_qs + align64(sizeof(QueryState) * nq);
  rc = host_stage(&ws->h_hdr, &ws->h_hdr_bytes, o_ctl + sizeof(Ctl));
  if (rc) return rc;
  const ResultDev* res = reinterpret_cast<const ResultDev*>(ws->h_hdr);
  const QueryState* qsh = reinterpret_cast<const QueryState*>(ws->h_hdr + o_qs);
  const Ctl& hc = *reinterpret_cast<const Ctl*>(ws->h_hdr + o_ctl);
  MPAP_CK(cudaMemcpyAsync(ws->h_hdr, w.res, sizeof(ResultDev) * nq, cudaMemcpyDeviceToHost, st));
  MPAP_CK(cudaMemcpyAsync(ws->h_hdr + o_qs, w.qs, sizeof(QueryState) * nq, cudaMemcpyDeviceToHost, st));
  MPAP_CK(cudaMemcpyAsync(ws->h_hdr + o_ctl, w.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  MPAP_CK(cudaStreamSynchronize(st));
  ws->last_max_front = hc.max_front;
  launch_count_add(4ull * hc.it);
  if (prof) {
    const char* names[4] = {"k_select", "k_prune", "k_prune_bulk", "k_end"};
    for (int k = 0; k < 4; ++k) profile_add(names[k], hc.kt[k].launches, (double)hc.kt[k].total_ns * 1e-6);
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
    ws->last_pool_used = used;
  }
  if (hc.err) {
    set_error("search: capacity exceeded in at least one query (flags 0x%x: 1 front pool, 2 plan arena, "
              "4 group array); its status says so, the other queries' results stand", hc.err);
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
  std::vector<uint4> fd(V);
  MPAP_CK(cudaMemcpyAsync(fd.data(), w.fdesc + base, sizeof(uint4) * V, cudaMemcpyDeviceToHost, st));
  MPAP_CK(cudaStreamSynchronize(st));
  std::vector<uint32_t> ptr(V + 1);
  uint64_t t = 0;
  for (uint32_t v = 0; v < V; ++v) {
    ptr[v] = (uint32_t)t;
    t += fd[v].y;
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
