/*
 * mpap.h -- C ABI of the GB300 (sm_103a) MPAP hot-path library (libmpap.so).
 *
 * MPAP is the Multiobjective Perception-Aware Planning method of Ichter, Landry,
 * Schmerling and Pavone (arXiv 1705.02408).  Given an obstacle set X_obs, dynamics,
 * an initial state x_init, a goal region X_goal, a cost c and a perception
 * heuristic h with bound beta (Sec. 2, Eq. 1 and Eq. 2), the library
 *   1. builds an r_n-disc roadmap with per-edge perception transfers
 *      (Alg. 1 steps 1-2, Alg. 2 BuildGraph),
 *   2. runs the wavefront multiobjective search (Alg. 1 step 3, Alg. 3 Explore),
 *   3. certifies the returned plan by Monte Carlo rollouts (Alg. 1 step 4).
 * Every step runs in this library's CUDA kernels; there is no CPU fallback.
 *
 * Conventions shared by all entry points
 *   - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it; calls that return host results synchronise
 *     that stream before returning.
 *   - Host input arrays are copied; the caller keeps ownership.  Arrays flagged
 *     MPAP_MEM_DEVICE are read in place (device pointers, 16-byte aligned) and must
 *     stay valid until the call returns.
 *   - Opaque handles (mpap_roadmap, mpap_workspace) own device memory and are
 *     released by their *_free function.  A handle must not be used by two calls
 *     that overlap in time.
 *   - Errors are returned as negative mpap_status values; mpap_last_error() gives
 *     a one-line description (thread-local).  Device-side failures (capacity
 *     overflow, iteration cap) are detected on the device and returned as status
 *     codes; no kernel traps.  The search loop's grid barriers wait a bounded
 *     time (mpap_query.wait_us) and report MPAP_ERR_TIMEOUT when it runs out.
 *
 * Units.  Costs are int64 multiples of 2^-24 (cost quantum).  Perception heuristic
 * values are int64 multiples of 2^-24 / (M n_f) units of drift time, where M is
 * the number of sub-steps per edge and n_f the number of features that cancels
 * drift (Sec. 4.1).  Monte Carlo positions are integers in units of 2^-20.
 */
#ifndef MPAP_H_
#define MPAP_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MPAP_OK = 0,
  MPAP_NO_SOLUTION = 1,       /* P_open became empty without a goal plan (Alg. 3) */
  MPAP_ERR_INVALID_ARG = -1,  /* null pointer, bad size, too-small output buffer */
  MPAP_ERR_CAPACITY = -2,     /* a front, the plan arena or a work list overflowed */
  MPAP_ERR_TIMEOUT = -3,      /* a bounded device wait gave up */
  MPAP_ERR_ITER_LIMIT = -4,   /* the search hit max_iters wavefronts */
  MPAP_ERR_CUDA = -5,         /* a CUDA runtime call failed */
  MPAP_ERR_SAMPLING = -6      /* SampleFree could not find n free samples */
} mpap_status;

typedef enum { MPAP_DIM_2D = 2, MPAP_DIM_3D = 3, MPAP_DIM_DI6 = 6 } mpap_dim_kind;
typedef enum { MPAP_MEM_HOST = 0, MPAP_MEM_DEVICE = 1 } mpap_mem;

typedef struct mpap_roadmap mpap_roadmap;
typedef struct mpap_workspace mpap_workspace;

/* The mapped environment (Sec. 2: X, X_obs; Sec. 4.1: the perception field).
 *   dim_kind    2 (unit square, kinematic), 3 (unit cube, kinematic) or
 *               6 (3D double integrator x'' = u with |v| <= 1, Sec. 4.1).
 *   nb, box_lo, box_hi   axis-aligned closed boxes, float[nb][3] (z ignored in 2D);
 *               nb may be 0 (the pointers may then be NULL).
 *   grid_G, grid_level   perception quality levels 0..K on a G^Dp grid over the
 *               unit square/cube (Dp = 2 or 3), uint8, x fastest; G a power of two
 *               in [1, 1024].  A level k stands for the number of visible features
 *               in the Sec. 4.1 heuristic.
 *   n_f, K      features that cancel drift (the paper uses 12) and the top level.
 *   mem         MPAP_MEM_HOST or MPAP_MEM_DEVICE for box_lo, box_hi, grid_level. */
typedef struct {
  int32_t dim_kind;
  int32_t nb;
  const float* box_lo;
  const float* box_hi;
  int32_t grid_G;
  const uint8_t* grid_level;
  int32_t n_f;
  int32_t K;
  int32_t mem;
  int32_t n_heading;               /* 0, or Y tables for the camera-heading form */
  const uint8_t* heading_levels;   /* [Y][G^Dp] (same memory kind as the grid) */
} mpap_scene;
/* The camera-heading form of the perception heuristic (Sec. 4.1: features count
 * only in the field of view of the yaw, a single-integrator state tracked
 * exactly).  With n_heading = Y > 0 every node carries a yaw (see
 * mpap_roadmap_export_yaw), the yaw moves at a constant rate along each edge the
 * shorter way round (psi(t) = psi_a + (m / M) wrap(psi_b - psi_a) at checkpoint m,
 * wrap(d) = d - 2 pi rint(d / (2 pi)), binary32), and checkpoint m reads its level
 * from table y = rint(psi n_heading / (2 pi)) mod Y (the heading 2 pi y / Y
 * nearest to the yaw; mpap_feature_levels computes such tables) instead of
 * grid_level, in the edge transfers, the certification and the plan features.
 * Levels must lie in 0..K as for the grid.  Such a roadmap's levels cannot be
 * replaced by mpap_roadmap_update (boxes can be added). */

/* Roadmap construction parameters (Alg. 2).
 *   n           free samples drawn by SampleFree; V = n + 2 nodes with
 *               node 0 = x_init and node 1 = x_goal.
 *   seed, query_id   key and third counter word of the Philox4x32-10 sampler.
 *   r           connection radius r_n in cost units (Near uses Cost < r).
 *   T_edge      duration of a double-integrator connection (ignored in 2D/3D).
 *   M           sub-steps per connection (checkpoints for collision and heuristic).
 *   x_init, x_goal   states (position, velocity); goal_radius defines X_goal as the
 *               position ball around x_goal. */
typedef struct {
  uint32_t n;
  uint32_t query_id;
  uint64_t seed;
  float r;
  float T_edge;
  int32_t M;
  float x_init[6];
  float x_goal[6];
  float goal_radius;
} mpap_roadmap_params;

/* One search query (Alg. 3).
 *   beta        perception-heuristic bound (plans with h > beta are cut, Eq. 2).
 *   lambda      group cost factor in (0, 1]; groups are {p open : cost <= i Lambda}
 *               with Lambda = round(lambda r_n 2^24) cost quanta.
 *   group_width_q  if > 0, Lambda in cost quanta directly (lambda is then ignored;
 *               needed for roadmaps given as plain graphs, which have no r_n).
 *   max_iters   wavefront cap (MPAP_ERR_ITER_LIMIT when reached), > 0.
 *   flags       bit 0 MPAP_QUERY_NO_GOAL_STOP: run until P_open is empty.
 *               bit 1 MPAP_QUERY_CHECK_INTERIOR: the perception constraint of
 *               Eq. 2 for all t: a candidate is cut when the heuristic exceeds
 *               beta at any sub-step of its last edge (max(Cmax, h + Smax) >
 *               beta), not only at its head (Alg. 3).
 *               bit 2 MPAP_QUERY_OWN_SHARE: the query draws only on its own
 *               share of the front pool and of the plan arena, never on the
 *               halves common to the batch, so whether it runs out of capacity
 *               does not depend on the other queries of the call.
 *   wait_us     limit of one grid-barrier wait of the device wavefront loop, in
 *               microseconds of GPU timer time (0: 20 s).  A batch uses the
 *               smallest non-zero value of its queries.  A wait that runs out
 *               ends the loop: unfinished queries report MPAP_ERR_TIMEOUT and
 *               the call returns it; the workspace stays usable. */
#define MPAP_QUERY_NO_GOAL_STOP 1u
#define MPAP_QUERY_CHECK_INTERIOR 2u
#define MPAP_QUERY_OWN_SHARE 4u
typedef struct {
  int64_t beta;
  int64_t group_width_q;
  float lambda;
  uint32_t max_iters;
  uint32_t flags;
  uint32_t wait_us;
} mpap_query;

/* Search result.  path is a caller-owned host array of path_cap entries; on
 * return path_len holds the number of nodes from x_init to the goal node (also
 * when path_cap is too small, in which case the status is MPAP_ERR_INVALID_ARG). */
typedef struct {
  int32_t status;
  int64_t cost;
  int64_t h;
  uint32_t path_len;
  uint32_t path_cap;
  uint32_t* path;
  uint32_t wavefronts;     /* executed iterations of the Explore loop */
  uint64_t expansions;     /* (p in group, edge out of p.head) pairs evaluated */
  uint64_t plans;          /* plans that entered a stored front */
} mpap_result;

/* Monte Carlo model (integer error walk; see mpap_certify).  sigma_fx and shift
 * are host arrays of K+1 int32 entries indexed by quality level. */
typedef struct {
  uint32_t rollouts;
  uint32_t call_id;
  uint64_t seed;
  int64_t delta_fx;
  const int32_t* sigma_fx;
  const int32_t* shift;
} mpap_mc_params;

typedef struct {
  uint32_t hits_loc;       /* rollouts whose localisation error reached delta (Eq. 1) */
  uint32_t hits_coll;      /* rollouts whose executed state hit X_obs or left the map */
  uint32_t hits_any;
  uint32_t rollouts;
} mpap_cert;

const char* mpap_status_string(int32_t status);
const char* mpap_last_error(void);

/* ---------------------------------------------------------------------------
 * Roadmap (Alg. 1 steps 1-2; Alg. 2 BuildGraph; Sec. 3 primitives SampleFree,
 * Cost, Near, Collision; Sec. 4.1 heuristic precomputed per edge).
 * Draws V = {x_init, x_goal} + SampleFree(n), connects every ordered pair with
 * Cost < r whose optimal connection is collision free, and stores per edge
 * {dst, cost_q, S, C} with the heuristic transfer h -> max(C, h + S).  The handle
 * owns all device memory.  Returns MPAP_ERR_SAMPLING if n free samples cannot be
 * found within 64 n + 4096 candidates, MPAP_ERR_CAPACITY if an edge field
 * overflows int32. */
int32_t mpap_build_roadmap(const mpap_scene* scene, const mpap_roadmap_params* params,
                           mpap_roadmap** out, void* stream);

/* Builds n roadmaps in one pass (every kernel covers all of them; three host
 * round trips in total).  For each i, rms[i] == NULL creates a new handle and a
 * non-null rms[i] is rebuilt in place, reusing its device buffers when they are
 * large enough (no allocation when sizes repeat).  Results are identical to n
 * calls of mpap_build_roadmap.  On error, handles created by this call are freed
 * and set to NULL; reused handles stay valid but hold an unspecified roadmap. */
int32_t mpap_build_roadmaps(uint32_t n, const mpap_scene* scenes, const mpap_roadmap_params* params,
                            mpap_roadmap** rms, void* stream);

/* The same graph construction over caller-given node states x (host, float[6][V],
 * SoA: p0, p1, p2, v0, v1, v2).  Node 0 is x_init and node 1 x_goal. */
int32_t mpap_build_roadmap_from_points(const mpap_scene* scene, uint32_t V, const float* x,
                                       float r, float T_edge, int32_t M, float goal_radius,
                                       mpap_roadmap** out, void* stream);

/* A roadmap given directly as a forward CSR graph (host arrays), for searches on
 * hand-made graphs.  row_ptr[V+1], dst/cost_q/S/C[E], is_goal[V]; cost_q >= 1.
 * Every edge is then a single step for the interior check (its peak is its end
 * value); mpap_roadmap_from_csr_peaks gives the peaks explicitly. */
int32_t mpap_roadmap_from_csr(uint32_t V, const uint32_t* row_ptr, const uint32_t* dst,
                              const int32_t* cost_q, const int32_t* S, const int32_t* C,
                              const uint8_t* is_goal, mpap_roadmap** out, void* stream);

/* mpap_roadmap_from_csr with the per-edge transfer peaks Smax/Cmax[E]: the
 * heuristic along edge e, entered with h, never exceeds max(Cmax, h + Smax)
 * (Smax >= S, Cmax >= C >= 0). */
int32_t mpap_roadmap_from_csr_peaks(uint32_t V, const uint32_t* row_ptr, const uint32_t* dst,
                                    const int32_t* cost_q, const int32_t* S, const int32_t* C,
                                    const int32_t* Smax, const int32_t* Cmax, const uint8_t* is_goal,
                                    mpap_roadmap** out, void* stream);

int32_t mpap_roadmap_info(const mpap_roadmap* rm, uint32_t* V, uint64_t* E);

/* Copies the roadmap to host arrays (any pointer may be NULL): x float[6][V],
 * is_goal[V], row_ptr[V+1], dst/cost_q/S/C[E] with every row sorted by
 * neighbour (on the device rows are kept in discovery order; no kernel depends
 * on it).  Synchronises the stream. */
int32_t mpap_roadmap_export(const mpap_roadmap* rm, float* x, uint8_t* is_goal, uint32_t* row_ptr,
                            uint32_t* dst, int32_t* cost_q, int32_t* S, int32_t* C, void* stream);

/* Per-edge transfer peaks (Smax, Cmax)[E] in the order of mpap_roadmap_export:
 * entering edge e with heuristic h, the heuristic after each of its M sub-steps
 * is at most max(Cmax, h + Smax), with equality at some sub-step (Sec. 4.1
 * heuristic; used by the interior check of Eq. 2). */
int32_t mpap_roadmap_export_peaks(const mpap_roadmap* rm, int32_t* Smax, int32_t* Cmax, void* stream);

/* Copies the node yaws of a roadmap in the camera-heading form (Sec. 4.1: a
 * single-integrator yaw state; drawn uniform in [-pi, pi) from Philox4x32-10
 * with counter (v, 2, query_id, 0) and key seed for sampled roadmaps, 0 for given
 * node states) to a host array of V floats; all zero for the grid form.
 * Synchronises the stream. */
int32_t mpap_roadmap_export_yaw(const mpap_roadmap* rm, float* yaw, void* stream);

/* Copies the reverse CSR the search reads (in-edges of every node, Alg. 3's
 * predecessor sets) to host arrays (any pointer may be NULL): rev_ptr[V+1];
 * src, cost_q, S, C, Smax, Cmax [E] with every row sorted by source.  Row u
 * holds one record per forward edge (v -> u) with that edge's fields, so it is
 * the transpose of mpap_roadmap_export.  Synchronises the stream. */
int32_t mpap_roadmap_export_reverse(const mpap_roadmap* rm, uint32_t* rev_ptr, uint32_t* src, int32_t* cost_q,
                                    int32_t* S, int32_t* C, int32_t* Smax, int32_t* Cmax, void* stream);

/* Online update of a built roadmap (the map changes, the nodes stay; Sec. 3 on
 * use within a mapping framework): nb_add boxes float[nb_add][3] are appended to
 * the roadmap's obstacles and, when grid is not NULL, its quality levels
 * uint8[G^Dp] are replaced.  An added box can only remove edges, so an edge is
 * tested against the added boxes only, and only when a conservative box around
 * its checkpoints (2D/3D: the segment's bounding box; 6D: the segment from p0 to
 * p0 + v0 T grown by sqrt(T^3 J / 3), J = cost - T, which bounds the connection's
 * deviation from it) meets one of them; its transfer and peaks are recomputed
 * only when that box meets a cell whose level the new grid changes.  The
 * forward and reverse CSR are then compacted.  The host inputs are staged in one
 * upload and the call synchronises the stream once, at its end; the box arrays
 * keep room for 64 more boxes than the scene had, so an update that adds no more
 * allocates nothing for them.  The roadmap afterwards is the one
 * mpap_build_roadmap_from_points
 * builds from the same nodes on the updated scene.  mem: MPAP_MEM_HOST or
 * MPAP_MEM_DEVICE for add_lo, add_hi and grid.  Synchronises the stream.
 * Returns MPAP_ERR_INVALID_ARG for a roadmap without geometry, more than 1024
 * boxes in all or null arrays; MPAP_ERR_CAPACITY when a new transfer does not
 * fit int32 (the roadmap is then left with those edges' values truncated). */
int32_t mpap_roadmap_update(mpap_roadmap* rm, int32_t nb_add, const float* add_lo, const float* add_hi,
                            const uint8_t* grid, int32_t mem, void* stream);

/* mpap_roadmap_update for n distinct roadmaps in one pass (one launch per
 * dimension for the edge tests, one scan, one compaction and one reverse build
 * for all of them): roadmap j gets nb_add[j] boxes add_lo[j], add_hi[j] and, when
 * grids is not NULL and grids[j] is not NULL, the levels grids[j].  Errors as for
 * mpap_roadmap_update, and MPAP_ERR_INVALID_ARG for a roadmap given twice. */
int32_t mpap_roadmap_update_batch(mpap_roadmap* const* rms, uint32_t n, const int32_t* nb_add,
                                  const float* const* add_lo, const float* const* add_hi,
                                  const uint8_t* const* grids, int32_t mem, void* stream);

/* Build statistics: Near tests (Cost < r evaluations) performed by the last
 * build of this roadmap, and the number of nodes in X_goal. */
int32_t mpap_roadmap_stats(const mpap_roadmap* rm, uint64_t* near_tests, uint32_t* n_goal);

void mpap_roadmap_free(mpap_roadmap* rm);

/* ---------------------------------------------------------------------------
 * Search workspace: device memory for the per-node Pareto fronts, the plan arena
 * and the wavefront work lists of up to `total_nodes` nodes summed over the
 * queries of one call.  Fronts live in one pool of total_nodes * front_cap
 * entries (24 bytes each; the product must not exceed 2^32 - 16): every node
 * draws two blocks from it (its live front and a merge target), of 16 entries
 * and up, replaced by blocks twice the needed size as its front grows, so single
 * fronts may be far larger than front_cap as long as the pool lasts.  Half of
 * the pool is shared out among the queries of a call in proportion to their
 * nodes; a query that fills its share draws on the other half, which all
 * queries of the call share (where a block lies changes no result).  Half of
 * the plan arena (max_plans records) is shared out the same way.
 * A query that runs out of pool, of plan arena or of group array (max_plans)
 * ends with MPAP_ERR_CAPACITY in its own result; the other queries of the batch
 * run on.  Candidates of one wavefront wait in 64 slots of 32 bytes per node
 * (2 KiB per node); a node's candidates beyond 64 go to two overflow areas of
 * max_plans records, shared out among the queries of a call like the pool.
 * Allocates with cudaMalloc; reused by every search call. */
int32_t mpap_workspace_create(uint64_t total_nodes, uint32_t front_cap, uint64_t max_plans,
                              mpap_workspace** out);
void mpap_workspace_free(mpap_workspace* ws);

/* Sizes reached by the last search call on `ws` (the paper has no counterpart:
 * this sizes workspaces): *max_front = the largest Pareto front any node held,
 * *pool_used = front-pool entries handed out (blocks of every size, summed over
 * the queries of the call and the pool's common half).  Either pointer may be
 * NULL.  Host only; MPAP_ERR_INVALID_ARG for a NULL workspace. */
int32_t mpap_workspace_stats(const mpap_workspace* ws, uint32_t* max_front, uint64_t* pool_used);

/* Alg. 3 Explore for one query on one roadmap.  The whole group loop is one
 * persistent kernel (cooperative launch, grid barriers between the expansion
 * and the merge of every wavefront); the host waits once.  RemoveDominated uses the weak Pareto order with
 * a total tie key (creation iteration, parent head, parent cost): an exact set
 * function, so fronts, cost, h and path are identical to a sequential execution
 * of Alg. 3.  Returns the result status (MPAP_OK or MPAP_NO_SOLUTION) or an
 * error. */
int32_t mpap_search(mpap_workspace* ws, mpap_roadmap* rm, const mpap_query* q, mpap_result* out,
                    void* stream);

/* nq independent queries in one lock-step wavefront loop (each query keeps its own
 * iteration count, group threshold and termination).  outs[i] receives the
 * result of qs[i] on rms[i]; the return value is MPAP_OK if every query ran to
 * completion (individual results may still be MPAP_NO_SOLUTION) or the first
 * error. */
int32_t mpap_search_batch(mpap_workspace* ws, mpap_roadmap* const* rms, const mpap_query* qs,
                          uint32_t nq, mpap_result* outs, void* stream);

/* Final Pareto fronts of query `index` of the last search on `ws` (for parity
 * checks): front_ptr[V+1] and (cost, h) pairs sorted by cost, up to cap entries;
 * *total receives the number of entries. */
int32_t mpap_search_fronts(mpap_workspace* ws, uint32_t index, uint32_t* front_ptr, int64_t* cost,
                           int64_t* h, uint64_t cap, uint64_t* total, void* stream);

/* ---------------------------------------------------------------------------
 * Monte Carlo certification (Alg. 1 step 4; Sec. 3 final phase; failure events
 * of Eq. 1 and of the robust motion planning problem).  For each rollout an
 * integer error e (units 2^-20) walks the plan's checkpoints: at quality level k,
 * e <- e - (e >> shift[k]) (skipped when shift[k] = 0), then
 * e <- e + (sigma_fx[k] xi) >> 16 with xi a sum of 12 uniform 16-bit draws minus
 * 6 * 2^16 (Philox4x32-10, counter (rollout, step, 0..4, call_id), key seed),
 * clamped to |e_i| <= 2^30.  Localisation fails when e.e >= delta_fx^2; the
 * executed state x_nom + e fails when it leaves the unit map or enters a closed
 * box.  path is a host array of node indices. */
int32_t mpap_certify(mpap_roadmap* rm, const uint32_t* path, uint32_t path_len,
                     const mpap_mc_params* mc, mpap_cert* out, void* stream);

/* n certifications in one launch: paths[i] (host) on rms[i] with mcs[i]. */
int32_t mpap_certify_batch(mpap_roadmap* const* rms, const uint32_t* const* paths,
                           const uint32_t* path_lens, const mpap_mc_params* mcs, uint32_t n,
                           mpap_cert* outs, void* stream);

/* Closed-loop VIO Monte Carlo model (Sec. 4.1: the nominal trajectory tracked by
 * an LQR controller, the state estimated by a Kalman filter that fuses an
 * inertial prediction with position fixes from the features in view).  The
 * paper gives no parameters; this is the library's reading.  Per position axis,
 * in 2^-20 units and per checkpoint step, the executed deviation (p, w) from the
 * nominal (w = velocity x step) and the estimation error (ep, ew): at checkpoint
 * s with quality level k,
 *   a  = -round((kp_q16 (p + ep) + kv_q16 (w + ew)) / 2^16)     LQR from the estimate
 *   p += w + (a >> 1);  w += a
 *   na = (q_a xi1) >> 16;  ep += ew + (na >> 1);  ew += na       inertial prediction
 *   if r_fx[k] > 0:  nu = (r_fx[k] xi2) >> 16;  t = nu - ep;
 *     ep += round(Lp_s t / 2^16);  ew += round(Lw_s t / 2^16)    position fix
 * all clamped to |x| <= 2^30, round(x / 2^16) = (x + 2^15) >> 16.  (Lp_s, Lw_s)
 * are the Kalman gains of step s from the covariance recursion in double (P_0 =
 * 0; prediction A P A^T + q_a^2 B B^T, A = [1 1; 0 1], B = (1/2, 1); update with
 * variance r_fx[k]^2 when r_fx[k] > 0) rounded to Q16.  xi1 and xi2 are sums of 12
 * uniform 16-bit draws minus 6 * 2^16: axis i takes the u16 halves (low first)
 * of Philox4x32-10 calls 3 i .. 3 i + 2 with counter (rollout, step, call,
 * call_id) and key seed, xi1 from the first six words and xi2 from the last six.
 * Localisation fails when ep.ep >= delta_fx^2 (Eq. 1); the executed position
 * nom + p fails when it leaves the unit map or enters a closed box.  r_fx is a
 * host array of K+1 entries (0: no fix at that level); kp_q16, kv_q16 are the
 * LQR gains per step in Q16 (a = -(kp p + kv w)). */
typedef struct {
  int32_t q_a;             /* inertial noise per step, 2^-20 units */
  int32_t kp_q16;
  int32_t kv_q16;
  const int32_t* r_fx;     /* [K+1] position-fix noise per quality level */
} mpap_vio_params;

/* The LQR gains of the VIO model for state cost diag(q_p, q_w) and control cost
 * r (> 0): per position axis x' = A x + B a with A = [1 1; 0 1], B = (1/2, 1)
 * over one checkpoint step, a = -(kp p + kv w) with (kp, kv) = (r + B^T P B)^-1
 * B^T P A, P the fixed point of the discrete Riccati recursion started at
 * diag(q_p, q_w) (double), returned in Q16.  Host only; MPAP_ERR_INVALID_ARG for
 * negative weights, r <= 0 or NULL outputs. */
int32_t mpap_vio_lqr_gains(double q_p, double q_w, double r, int32_t* kp_q16, int32_t* kv_q16);

/* n certifications under the VIO model in one launch: paths[i] (host) on rms[i]
 * with mcs[i] (rollouts, call_id, seed, delta_fx; its sigma_fx and shift are not
 * used and may be NULL) and vps[i].  Errors as for mpap_certify_batch, and
 * MPAP_ERR_INVALID_ARG for a null r_fx. */
int32_t mpap_certify_vio_batch(mpap_roadmap* const* rms, const uint32_t* const* paths,
                               const uint32_t* path_lens, const mpap_mc_params* mcs,
                               const mpap_vio_params* vps, uint32_t n, mpap_cert* outs, void* stream);

/* mpap_certify without any device allocation (the paper has no counterpart;
 * this serves deployment).  For callers that must not allocate device memory
 * while running -- a planner inside a robot's real-time control loop, where an
 * allocation can block or fragment a fixed memory budget, or a program whose
 * device memory is all held by another framework's allocator.  The scratch the
 * certification kernels need lives in one fixed device array inside the library
 * (about 1.1 MB, held on every GPU that loads the library until the process
 * exits); the caller passes the inputs (a built roadmap, the host plan and
 * tables) and the output struct as for mpap_certify, and gets identical counts.
 * Limits: path_len <= 4096 nodes, (path_len - 1) * M <= 65536 checkpoints,
 * K + 1 <= 256 levels, at most 512 boxes; larger inputs return
 * MPAP_ERR_INVALID_ARG with the reason in mpap_last_error().  Every call looks up
 * the array's device address on the current device (so it stays right after a
 * device reset); the first call on a device may load the library's device code
 * there, so make it before any stream capture on that device.  Every call on a device shares the one array and clears the
 * counters it needs, so calls that overlap on the GPU (other streams or threads)
 * race: serialise them.  Calls no cudaMalloc, cudaFree or allocating routine. */
int32_t mpap_certify_noalloc(const mpap_roadmap* rm, const uint32_t* path, uint32_t path_len,
                             const mpap_mc_params* mc, mpap_cert* out, void* stream);

/* ---------------------------------------------------------------------------
 * Launch-shape tuning (not in the paper; serves batched deployment).  The
 * library keeps a table of launch shapes keyed by (dimension, node-count bucket
 * floor(log2 V)); dim_kind 0 keys a batch that mixes dimensions, V the largest
 * roadmap of a batch.  mpap_build_roadmaps reads edge_warps for each dimension
 * group of its batch; mpap_search / mpap_search_batch read the wavefront
 * kernel's blocks per SM and the group size from which its expansion runs its
 * lanes over a node's group plans instead of its out-edges, and the size from
 * which a node's merge is spread over the whole grid.  Keys without an entry use
 * the defaults (8, 8, 8, 64, 2048).  The results of every call are
 * identical for every valid shape; only the time changes.  The table is
 * process-wide and guarded by a mutex.
 * ------------------------------------------------------------------------- */
typedef struct {
  uint32_t edge_warps;            /* warps per block of the edge kernel: 4 or 8 */
  uint32_t wave_blocks_per_sm;    /* blocks per SM of the persistent wavefront kernel:
                                     1 .. 64, capped at the number that fits */
  uint32_t plan_lanes_from;       /* group size from which the expansion puts its
                                     lanes on the group plans: 1 .. 64 */
  uint32_t front_cap;             /* advisory pool entries per node for mpap_workspace_create */
  uint32_t grid_merge_from;       /* front + candidates of one node from which its merge
                                     runs on every warp of the grid: 33 .. 2^30 */
} mpap_tuning;

/* The entry the library uses for (dim_kind, V): a stored one or the defaults. */
int32_t mpap_tuning_get(int32_t dim_kind, uint32_t V, mpap_tuning* out);
/* Stores t for the key of (dim_kind, V); MPAP_ERR_INVALID_ARG for an invalid shape. */
int32_t mpap_tuning_set(int32_t dim_kind, uint32_t V, const mpap_tuning* t);
int32_t mpap_tuning_clear(void);
/* Copies up to cap stored entries (keys as dim_kind and bucket) and sets *n to
 * the number stored (MPAP_ERR_INVALID_ARG if that exceeds cap). */
int32_t mpap_tuning_export(uint32_t cap, int32_t* dim_kind, uint32_t* bucket, mpap_tuning* t, uint32_t* n);

/* Grid search of the edge kernel's block size (4, 8 warps) on one batched build
 * of these n roadmaps: each candidate builds into rms (handles as for
 * mpap_build_roadmaps) `reps` times after one untimed build, timed with CUDA
 * events on `stream`.  The fastest is stored for every (dimension, bucket) group
 * of the batch; *best and *best_ms (per build) describe it. */
int32_t mpap_autotune_build(uint32_t n, const mpap_scene* scenes, const mpap_roadmap_params* params,
                            mpap_roadmap** rms, uint32_t reps, mpap_tuning* best, double* best_ms,
                            void* stream);

/* Grid search of the wavefront kernel's blocks per SM (1, 2, 4, 8; capped at
 * the number that fits) and of plan_lanes_from (4, 8, 16, 32) on one batched
 * search of these queries, `reps` timed searches per candidate after an
 * untimed one.  Stores the fastest for the batch key and
 * sets best->front_cap to twice the front-pool entries per node the search
 * used, rounded up to a power of two (at least 16).  Queries that run out of
 * the pool keep that status (it is part of the compared results).  Fails
 * with MPAP_ERR_CUDA (and stores nothing) if two shapes give different results. */
int32_t mpap_autotune_search(mpap_workspace* ws, mpap_roadmap* const* rms, const mpap_query* qs,
                             uint32_t nq, uint32_t reps, mpap_tuning* best, double* best_ms,
                             void* stream);

/* ---------------------------------------------------------------------------
 * Candidate plans and the certification surrogate.
 *
 * Alg. 3 ends by collecting P_candidates, every plan stored at a goal node, and
 * returning the cheapest; Alg. 1 then certifies that plan by Monte Carlo and, if
 * it fails, refines the bound and searches again.  The entry points below expose
 * the whole candidate set and a learned screen of it, so that a caller can try
 * the candidates in cost order but skip those a small network predicts will fail
 * certification, and spend Monte Carlo only on likely winners.  The network is
 * not in the paper (its only learned part is the error-rate heuristic of Sec.
 * 5.1, mpap_errnet_*); Monte Carlo stays the judge of every plan returned.
 * ------------------------------------------------------------------------- */

/* Candidates of query `index` of the last search on ws (Alg. 3 final lines), in
 * the solution order (cost, then h, then the tie key: creation wavefront, parent
 * head, parent cost; then head index), so candidate 0 is the plan mpap_search
 * returned.  Writes up to `cap` candidates to host arrays: cost[i], h[i] and the
 * node sequence path[path_ptr[i] .. path_ptr[i+1]) (path_ptr has cap+1 entries,
 * path has path_cap entries).  *n receives the number written and *total the
 * size of P_candidates.  MPAP_ERR_CAPACITY if the paths do not fit path_cap (the
 * counts are still set); MPAP_ERR_INVALID_ARG for a query that did not finish
 * with MPAP_OK. */
int32_t mpap_search_candidates(mpap_workspace* ws, uint32_t index, uint32_t cap, int64_t* cost,
                               int64_t* h, uint32_t* path_ptr, uint32_t* path, uint32_t path_cap,
                               uint32_t* n, uint32_t* total, void* stream);

/* mpap_search_candidates for queries 0 .. nq-1 of the last search on ws in one
 * launch (one block per query).  Host outputs in slices: query i writes up to cap
 * candidates to cost[i cap ..], h[i cap ..], offsets path_ptr[i (cap+1) ..] into
 * its path slice path[i path_cap ..], and n[i], total[i]; a query that did not
 * finish with MPAP_OK gets n[i] = total[i] = 0.  MPAP_ERR_CAPACITY if a query's
 * paths exceed path_cap. */
int32_t mpap_search_candidates_batch(mpap_workspace* ws, uint32_t nq, uint32_t cap, int64_t* cost,
                                     int64_t* h, uint32_t* path_ptr, uint32_t* path,
                                     uint32_t path_cap, uint32_t* n, uint32_t* total, void* stream);

/* Perception quality levels from mapped features: the visible-feature count of
 * the Sec. 4.1 heuristic at the centre c = ((2i + 1) / (2G), ...) of every cell of
 * a G^Dp grid (Dp = 2 for dim_kind 2, else 3), for each of Y = yaw_bins camera
 * headings.  A feature f (d = f - c) counts when
 *   |d|^2 <= range^2,
 *   hx dx + hy dy >= cos_half_fov sqrt(dx^2 + dy^2)   (horizontal field of view of
 *                                                      heading (hx, hy)), and
 *   the closed segment c -> f meets no closed box;
 * the level is min(count, K).  cos_half_fov <= -1 turns the field-of-view test
 * off, which with one heading gives a scene's all-direction quality grid.  Every
 * float operation is one IEEE operation in the order written.
 *   box_lo, box_hi   float[nb][3] (z ignored in 2D), nb in [0, 1024]
 *   features         float[n_features][3]
 *   headings         float[yaw_bins][2], unit vectors chosen by the caller
 *   levels           uint8[yaw_bins][G^Dp], x fastest (written)
 *   mem              MPAP_MEM_HOST (copies in and out, synchronises the stream) or
 *                    MPAP_MEM_DEVICE for all five arrays (asynchronous on stream).
 * Returns MPAP_ERR_INVALID_ARG for a bad dimension, grid size (G a power of two
 * in [1, 1024]), K outside [0, 255], null arrays, more than 2^22 features or
 * yaw_bins G^Dp above 2^31. */
int32_t mpap_feature_levels(int32_t dim_kind, int32_t nb, const float* box_lo, const float* box_hi,
                            uint32_t n_features, const float* features, int32_t grid_G, uint32_t yaw_bins,
                            const float* headings, float cos_half_fov, float range, int32_t K,
                            uint8_t* levels, int32_t mem, void* stream);

/* 48 trajectory features of each of n plans on one roadmap (input of the
 * surrogate).  Plan i is the host node sequence path[path_ptr[i] ..
 * path_ptr[i+1]) (at least 2 nodes).  Its Monte Carlo checkpoints (the M
 * sub-steps of every edge, as mpap_certify uses them, s = 0 .. steps-1) are split
 * into 16 bins, checkpoint s going to bin floor(16 s / steps).  For bin j:
 *   feat[j]      = max quality level in the bin / K
 *   feat[16 + j] = sum of quality levels in the bin / (64 K)
 *   feat[32 + j] = 4 min(0.25, clearance), the clearance of a checkpoint p being
 *                  min over boxes b of max_i max(lo_bi - p_i, p_i - hi_bi) and
 *                  over the walls of min_i min(p_i, 1 - p_i) (negative inside)
 * (an empty bin gives 0, 0, 1).  feat is a host array [n][48] of float. */
#define MPAP_FEATURES 48
int32_t mpap_plan_features(mpap_roadmap* rm, uint32_t n, const uint32_t* path_ptr,
                           const uint32_t* path, float* feat, void* stream);

/* mpap_plan_features for plans on several roadmaps in one launch: the plans of
 * rms[r] are plan_ptr[r] .. plan_ptr[r+1]-1 (plan_ptr has n_rm + 1 entries), plan
 * i is path[path_ptr[i] .. path_ptr[i+1]) and gets feat[48 (i - plan_ptr[0]) ..]. */
int32_t mpap_plan_features_batch(mpap_roadmap* const* rms, uint32_t n_rm, const uint32_t* plan_ptr,
                                 const uint32_t* path_ptr, const uint32_t* path, float* feat,
                                 void* stream);

/* The surrogate network: 48 -> 128 -> 128 -> 128 -> 2 with ReLU, logits of
 * (collision, localisation) failure; bfloat16 weights and activations in every
 * product, fp32 accumulation (tensor cores), fp32 master weights and biases,
 * Adam.  Packed parameters (fp32, MPAP_MLP_PARAMS): W1[128][48], b1[128],
 * W2[128][128], b2[128], W3[128][128], b3[128], W4[2][128], b4[2], W[o][i] being
 * the weight from input i to output o.  mpap_mlp_create initialises the weights
 * from Philox4x32-10 (uniform in +-1/sqrt(fan in)), biases zero, and sizes the
 * activations for batches of up to max_batch rows. */
#define MPAP_MLP_PARAMS 39554
typedef struct mpap_mlp mpap_mlp;
int32_t mpap_mlp_create(uint64_t seed, uint32_t max_batch, mpap_mlp** out);
void mpap_mlp_free(mpap_mlp* net);
int32_t mpap_mlp_get_params(mpap_mlp* net, float* params, void* stream);
/* Sets the parameters and clears the Adam state. */
int32_t mpap_mlp_set_params(mpap_mlp* net, const float* params, void* stream);

/* prob[n][2] = sigmoid(logits) of the features x[n][48].  x and prob are host
 * arrays, or device arrays when mem = MPAP_MEM_DEVICE.  n <= max_batch. */
int32_t mpap_mlp_forward(mpap_mlp* net, const float* x, uint32_t n, float* prob, int32_t mem,
                         void* stream);

/* One training step on the batch (x[n][48], soft labels y[n][2] in [0, 1]):
 * loss = mean over rows and both outputs of the binary cross-entropy of
 * sigmoid(logit) against y; gradients by back-propagation (the bfloat16
 * roundings of stored values pass gradients unchanged); if apply, one Adam step
 * (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr).  *loss (host, optional)
 * receives the loss before the step; grads (optional, MPAP_MLP_PARAMS floats,
 * host or device per mem) the packed gradient. */
int32_t mpap_mlp_train_step(mpap_mlp* net, const float* x, const float* y, uint32_t n, float lr,
                            int32_t apply, float* loss, float* grads, int32_t mem, void* stream);

/* ---------------------------------------------------------------------------
 * Learned error-rate heuristic (Sec. 5.1).  A feedforward network with two
 * hidden layers of eight ReLU units maps x = (v_x, v_y, v_z, w_x, w_y, w_z, n)
 * (linear and angular velocity, visible-feature count) to the mean and the
 * standard deviation of the Gaussian rate of the position-error magnitude:
 *   z = W3 relu(W2 relu(W1 x + b1) + b2) + b3,  mean = z0,
 *   std = softplus(z1) + 1e-3,
 * fitted by maximum likelihood: loss = mean over the batch of
 * log std + (r - mean)^2 / (2 std^2).  Packed parameters (fp32,
 * MPAP_ERRNET_PARAMS): W1[8][7], b1[8], W2[8][8], b2[8], W3[2][8], b3[2].
 * mpap_errnet_create draws weights uniform in +-1/sqrt(fan in) from seed, biases
 * zero.  All arithmetic is binary32 on the CUDA cores; batch gradients are
 * summed in a fixed order, so training is deterministic.
 * ------------------------------------------------------------------------- */
#define MPAP_ERRNET_PARAMS 154
#define MPAP_ERRNET_INPUTS 7
typedef struct mpap_errnet mpap_errnet;
int32_t mpap_errnet_create(uint64_t seed, uint32_t max_batch, mpap_errnet** out);
void mpap_errnet_free(mpap_errnet* net);
int32_t mpap_errnet_get_params(mpap_errnet* net, float* params, void* stream);
/* Sets the parameters and clears the Adam state. */
int32_t mpap_errnet_set_params(mpap_errnet* net, const float* params, void* stream);
/* out[n][2] = (mean, std) of the inputs x[n][7]; host arrays, or device arrays
 * with mem = MPAP_MEM_DEVICE.  n <= max_batch. */
int32_t mpap_errnet_forward(mpap_errnet* net, const float* x, uint32_t n, float* out, int32_t mem, void* stream);
/* One maximum-likelihood step on observed rates r[n]: *loss (optional) is the
 * loss before the step, grads (optional, MPAP_ERRNET_PARAMS floats) its
 * gradient; if apply, one Adam step (beta1 0.9, beta2 0.999, eps 1e-8,
 * bias-corrected) with learning rate lr.  1 <= n <= max_batch. */
int32_t mpap_errnet_train_step(mpap_errnet* net, const float* x, const float* r, uint32_t n, float lr, int32_t apply,
                               float* loss, float* grads, int32_t mem, void* stream);

/* The heuristic map: values (mean, std) map_val[n_map][2] known at mapped
 * states map_state[n_map][7] = (position 3, velocity 3, yaw) are interpolated
 * at query states q[n_q][7] by their k <= 16 nearest mapped states under
 *   d^2 = w[0] |dp|^2 + w[1] |dv|^2 + w[2] wrap(dyaw)^2,
 *   wrap(a) = a - 2 pi rint(a / 2 pi),
 * ties to the lower index, weighted by 1 / (d + 1e-6): out[n_q][2].  k larger
 * than n_map uses all mapped states.  mem: MPAP_MEM_HOST (copies in and out,
 * synchronises) or MPAP_MEM_DEVICE for all arrays but w (asynchronous). */
int32_t mpap_errmap_query(const float* map_state, const float* map_val, uint32_t n_map, const float* q, uint32_t n_q,
                          uint32_t k, const float* w, float* out, int32_t mem, void* stream);

/* The mapped mean rate at the centres ((2 i + 1) / (2 G), ...) of a G^Dp grid
 * (Dp = 2 for dim_kind 2, else 3; x fastest), for one velocity vel[3] and yaw,
 * as a quality level of the grid form of the heuristic, so that a roadmap built
 * on it accumulates the learned rate: the grid form gains dt (1 - k / n_f) per
 * sub-step, the learned one dt mean / mu_ref, so
 *   level = clamp(floor(n_f (1 - mean / mu_ref) + 1/2), 0, K)
 * (uint8 levels[G^Dp]).  Map arguments and mem as for mpap_errmap_query. */
int32_t mpap_errmap_levels(const float* map_state, const float* map_val, uint32_t n_map, uint32_t k, const float* w,
                           int32_t dim_kind, int32_t grid_G, const float* vel, float yaw, float mu_ref, int32_t n_f,
                           int32_t K, uint8_t* levels, int32_t mem, void* stream);

/* ---------------------------------------------------------------------------
 * Certification-driven choice of plans (Alg. 1 step 4; Sec. 3 on Monte Carlo
 * certification and the refinement of beta).
 *
 * Alg. 1 certifies the plan Explore returns for a bound beta and, from the
 * Monte Carlo outcome, loosens beta (more aggressive plans) or tightens it (more
 * conservative ones) and explores again until a robust plan is found.  The
 * paper leaves the update open; the rule of this library:
 *   - a plan passes when its any-failure count is at most max_hits;
 *   - with no failure seen yet, beta becomes 2 beta + 1 (at most 2^62) after a
 *     pass or after "no plan", and the query stops once a pass brings no
 *     cheaper plan than the previous pass;
 *   - with failures but no pass yet, beta becomes floor((b + f) / 2), b the
 *     largest bound known to give no plan (-1 if none), f the smallest failing
 *     bound;
 *   - with both, beta bisects between the largest passing and the smallest
 *     failing bound;
 *   - a query stops when no integer lies strictly between its bounds, after
 *     max_rounds explorations, or when a search ends with an error.
 * ------------------------------------------------------------------------- */
#define MPAP_REFINE_PASS 0
#define MPAP_REFINE_FAIL 1
#define MPAP_REFINE_NONE 2    /* the search found no plan (MPAP_NO_SOLUTION) */
#define MPAP_REFINE_ERROR 3   /* the search ended with an error (its status in hits) */

/* The bounds of one query's refinement; -1 marks an unknown bound (bounds are
 * non-negative).  Start from {-1, 0, -1, -1}. */
typedef struct {
  int64_t lo;        /* largest bound that passed */
  int64_t lo_cost;   /* cost of the plan found at lo */
  int64_t hi;        /* smallest bound that failed */
  int64_t none;      /* largest bound that gave no plan */
} mpap_refine_bounds;

/* Records the outcome (MPAP_REFINE_PASS, _FAIL or _NONE) of exploring at beta
 * (cost: the plan's cost, for a pass) and sets *next to the bound to explore
 * next, or -1 when the refinement stops.  Pure host code (no GPU needed).
 * MPAP_ERR_INVALID_ARG for a null pointer, a negative beta or another outcome. */
int32_t mpap_refine_advance(mpap_refine_bounds* b, int64_t beta, int32_t outcome, int64_t cost, int64_t* next);

/* One exploration of a refinement. */
typedef struct {
  int64_t beta;
  int64_t cost;      /* plan cost (pass, fail), -1 otherwise */
  int32_t outcome;   /* MPAP_REFINE_* */
  int32_t hits;      /* any-failure count (pass, fail), the search status (error), -1 (none) */
} mpap_refine_round;

/* Result of one query's refinement.  path and history are caller-owned host
 * arrays of path_cap and hist_cap entries (either may be NULL with cap 0). */
typedef struct {
  int32_t certified;        /* 1 if some bound passed */
  int32_t status;           /* MPAP_OK, or MPAP_ERR_INVALID_ARG if path_cap was too small */
  int64_t beta;             /* largest passing bound, -1 without a pass */
  int64_t cost, h;          /* the plan found at beta */
  uint32_t path_len, path_cap;
  uint32_t* path;
  mpap_cert cert;           /* its Monte Carlo certificate */
  uint32_t rounds;          /* explorations run */
  uint32_t hist_cap;
  mpap_refine_round* history;   /* the first min(rounds, hist_cap) explorations */
} mpap_refine_result;

/* Refines the bound of n queries in lock step: round t is one batched search
 * (mpap_search_batch) over the queries still refining, each with its current
 * bound, and one batched certification (mpap_certify_batch) of the plans found,
 * with call id t.  qs[i] gives query i's initial bound (beta) and its search
 * parameters; mcs[i] its Monte Carlo model (call_id ignored); max_hits[i] its
 * pass threshold.  outs[i] receives its result.  ws must hold the nodes of all
 * n roadmaps.  Returns MPAP_OK, or the first error that is not a search's own
 * (search errors end only their query, as MPAP_REFINE_ERROR in its history). */
int32_t mpap_refine_batch(mpap_workspace* ws, mpap_roadmap* const* rms, const mpap_query* qs,
                          const mpap_mc_params* mcs, const uint32_t* max_hits, uint32_t n,
                          uint32_t max_rounds, mpap_refine_result* outs, void* stream);

/* Screened certification of candidate plans (the paper has no counterpart: it
 * serves the learned surrogate).  Query i (rms[i]) has candidates c =
 * cand_ptr[i] .. cand_ptr[i+1]-1, usually P_candidates in solution order
 * (mpap_search_candidates_batch); candidate c is the node sequence
 * path[path_ptr[c] .. path_ptr[c+1]).  With use_net = 1 the network's
 * predicted any-failure probability 1 - (1 - p_coll)(1 - p_loc) (binary32,
 * from the 48 features feat[c][48], computed here when feat is NULL) orders
 * each query's candidates: those predicted at most tau first, then the others,
 * each group in index order; with use_net = 0 the order is the index order.
 * Then, in lock-step rounds (one batched certification per round), every
 * unresolved query certifies the next candidate of its order with call id
 * mcs[i].call_id + j (j its index within the query) until one has an
 * any-failure fraction hits_any / rollouts <= eps, or after max_calls (0: no
 * limit).  Outputs (host): chosen[i] (index within the query, -1 if none
 * passed), mc_calls[i], *rounds, and p_fail[c] (may be NULL).  net may be NULL
 * when use_net = 0.  Host arrays throughout. */
int32_t mpap_surrogate_screen(mpap_mlp* net, mpap_roadmap* const* rms, uint32_t nq, const uint32_t* cand_ptr,
                              const uint32_t* path_ptr, const uint32_t* path, const float* feat,
                              const mpap_mc_params* mcs, double eps, float tau, int32_t use_net,
                              uint32_t max_calls, int32_t* chosen, uint32_t* mc_calls, uint32_t* rounds,
                              float* p_fail, void* stream);

/* ---------------------------------------------------------------------------
 * Launch accounting and kernel timing (tracing).  The paper reports per-phase
 * computation times (Table 2); these entry points expose the same information
 * per kernel.  mpap_launch_count() counts every kernel this library has launched
 * since load or the last reset.  With mpap_profile_enable(1) every launch is
 * bracketed by CUDA events on its stream; mpap_profile_read() waits for them and
 * fills, for up to `cap` kernels, a 64-byte NUL-terminated name (names[64 i]),
 * the launch count and the total device milliseconds, and sets *n to the number
 * of distinct kernels (MPAP_ERR_INVALID_ARG if that exceeds cap).  Not for use
 * while a stream is being captured into a CUDA graph. */
int32_t mpap_profile_enable(int32_t on);
int32_t mpap_profile_reset(void);
uint64_t mpap_launch_count(void);
int32_t mpap_profile_read(uint32_t cap, char* names, uint64_t* launches, double* total_ms, uint32_t* n);

#ifdef __cplusplus
}
#endif

#endif /* MPAP_H_ */
