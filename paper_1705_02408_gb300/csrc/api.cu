// C ABI of libmpap (declared in include/mpap.h): argument validation and
// dispatch to the roadmap, search and certification implementations.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace mpap {
const char* last_error();
int32_t workspace_create(uint64_t total_nodes, uint32_t front_cap, uint64_t max_plans, uint32_t max_q,
                         mpap_workspace** out);
void workspace_free(mpap_workspace* ws);
int32_t search_batch_impl(mpap_workspace* ws, mpap_roadmap* const* rms, const mpap_query* qs, uint32_t nq,
                          mpap_result* outs, cudaStream_t st);
int32_t search_fronts_impl(mpap_workspace* ws, uint32_t index, uint32_t* front_ptr, int64_t* cost,
                           int64_t* h, uint64_t cap, uint64_t* total, cudaStream_t st);
int32_t roadmap_update_batch_impl(uint32_t n, mpap_roadmap* const* rms, const int32_t* nb_add,
                                  const float* const* add_lo, const float* const* add_hi,
                                  const uint8_t* const* grids, bool device, cudaStream_t st);
int32_t feature_levels_impl(int dp, int nb, const float* lo, const float* hi, uint32_t nf, const float* feat,
                            uint32_t G, uint32_t Y, const float* head, float cos_half, float range, int K,
                            uint8_t* out, bool device, cudaStream_t st);
int32_t certify_vio_batch_impl(mpap_roadmap* const* rms, const uint32_t* const* paths, const uint32_t* path_lens,
                               const mpap_mc_params* mcs, const mpap_vio_params* vps, uint32_t n, mpap_cert* outs,
                               cudaStream_t st);
int32_t certify_batch_impl(mpap_roadmap* const* rms, const uint32_t* const* paths, const uint32_t* path_lens,
                           const mpap_mc_params* mcs, uint32_t n, mpap_cert* outs, cudaStream_t st);
int32_t certify_noalloc_impl(const mpap_roadmap* rm, const uint32_t* path, uint32_t path_len,
                             const mpap_mc_params* mc, mpap_cert* out, cudaStream_t st);
int32_t search_candidates_impl(mpap_workspace* ws, uint32_t index, uint32_t cap, int64_t* cost, int64_t* h,
                               uint32_t* path_ptr, uint32_t* path, uint32_t path_cap, uint32_t* n_out,
                               uint32_t* total_out, cudaStream_t st);
int32_t plan_features_impl(mpap_roadmap* rm, uint32_t n, const uint32_t* path_ptr, const uint32_t* path, float* feat,
                           cudaStream_t st);
int32_t plan_features_batch_impl(mpap_roadmap* const* rms, uint32_t n_rm, const uint32_t* plan_ptr,
                                 const uint32_t* path_ptr, const uint32_t* path, float* feat, cudaStream_t st);
int32_t search_candidates_batch_impl(mpap_workspace* ws, uint32_t nq, uint32_t cap, int64_t* cost, int64_t* h,
                                     uint32_t* path_ptr, uint32_t* path, uint32_t path_cap, uint32_t* n_out,
                                     uint32_t* total_out, cudaStream_t st);
int32_t mlp_create(uint64_t seed, uint32_t max_batch, mpap_mlp** out);
void mlp_free(mpap_mlp* n);
int32_t mlp_get_params(mpap_mlp* n, float* params, cudaStream_t st);
int32_t mlp_set_params(mpap_mlp* n, const float* params, cudaStream_t st);
int32_t mlp_forward(mpap_mlp* nt, const float* x, uint32_t n, float* prob, int32_t mem, cudaStream_t st);
int32_t mlp_train_step(mpap_mlp* nt, const float* x, const float* y, uint32_t n, float lr, int32_t apply,
                       float* loss_out, float* grads_out, int32_t mem, cudaStream_t st);
int32_t tuning_set(int dim, uint32_t V, const mpap_tuning& t);
void tuning_clear();
int32_t tuning_export(uint32_t cap, int32_t* dims, uint32_t* buckets, mpap_tuning* t, uint32_t* n);
void batch_key(mpap_roadmap* const* rms, uint32_t nq, int& dim, uint32_t& V);
uint32_t workspace_last_max_front(const mpap_workspace* ws);
unsigned long long workspace_last_pool_used(const mpap_workspace* ws);
}  // namespace mpap

using mpap::set_error;

namespace {

cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

int32_t check_scene(const mpap_scene* sc) {
  if (!sc) {
    set_error("scene is null");
    return MPAP_ERR_INVALID_ARG;
  }
  if (sc->dim_kind != 2 && sc->dim_kind != 3 && sc->dim_kind != 6) {
    set_error("dim_kind must be 2, 3 or 6");
    return MPAP_ERR_INVALID_ARG;
  }
  if (sc->nb < 0 || (sc->nb > 0 && (!sc->box_lo || !sc->box_hi))) {
    set_error("bad obstacle arrays");
    return MPAP_ERR_INVALID_ARG;
  }
  if (sc->grid_G < 1 || sc->grid_G > 1024 || (sc->grid_G & (sc->grid_G - 1)) || !sc->grid_level) {
    set_error("grid_G must be a power of two in [1, 1024] with a level array");
    return MPAP_ERR_INVALID_ARG;
  }
  if (sc->n_f < 0 || sc->K < 0 || sc->K > 255) {
    set_error("bad n_f / K");
    return MPAP_ERR_INVALID_ARG;
  }
  if (sc->mem != MPAP_MEM_HOST && sc->mem != MPAP_MEM_DEVICE) {
    set_error("mem must be MPAP_MEM_HOST or MPAP_MEM_DEVICE");
    return MPAP_ERR_INVALID_ARG;
  }
  // 6D boxes are staged in shared memory by the edge kernel (48 KB default)
  if (sc->nb > 1024) {
    set_error("at most 1024 boxes");
    return MPAP_ERR_INVALID_ARG;
  }
  return MPAP_OK;
}

int32_t check_conn(float r, float T, int M, int dim) {
  if (!(r > 0.0f) || M < 1 || M > 4096 || (dim == 6 && !(T > 0.0f))) {
    set_error("need r > 0, 1 <= M <= 4096 and (6D) T > 0");
    return MPAP_ERR_INVALID_ARG;
  }
  return MPAP_OK;
}

}  // namespace

namespace {

int32_t batch_specs(uint32_t n, const mpap_scene* scenes, const mpap_roadmap_params* params,
                    std::vector<mpap::BuildSpec>& specs) {
  specs.resize(n);
  for (uint32_t i = 0; i < n; ++i) {
    int32_t rc = check_scene(&scenes[i]);
    if (!rc) rc = check_conn(params[i].r, params[i].T_edge, params[i].M, scenes[i].dim_kind);
    if (!rc && (params[i].n == 0 || params[i].n > 0x0FFFFFFFu)) {
      set_error("n must be in [1, 2^28)");
      rc = MPAP_ERR_INVALID_ARG;
    }
    if (rc) return rc;
    const mpap_roadmap_params& p = params[i];
    specs[i] = mpap::BuildSpec{&scenes[i], &p, nullptr, 0, p.r, p.T_edge, p.goal_radius, p.M};
  }
  return MPAP_OK;
}

// Device milliseconds per call of `reps` calls of f() after one untimed call.
template <typename F>
int32_t time_reps(cudaStream_t st, uint32_t reps, F f, double* ms) {
  int32_t rc = f();
  if (rc < 0) return rc;
  cudaEvent_t e0, e1;
  MPAP_CK(cudaEventCreate(&e0));
  MPAP_CK(cudaEventCreate(&e1));
  cudaEventRecord(e0, st);
  for (uint32_t r = 0; r < reps && rc >= 0; ++r) rc = f();
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float t = 0.0f;
  cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = (double)t / (double)(reps ? reps : 1);
  return rc < 0 ? rc : MPAP_OK;
}

}  // namespace

extern "C" {

const char* mpap_status_string(int32_t s) {
  switch (s) {
    case MPAP_OK: return "ok";
    case MPAP_NO_SOLUTION: return "no solution";
    case MPAP_ERR_INVALID_ARG: return "invalid argument";
    case MPAP_ERR_CAPACITY: return "capacity exceeded";
    case MPAP_ERR_TIMEOUT: return "device wait timed out";
    case MPAP_ERR_ITER_LIMIT: return "iteration limit";
    case MPAP_ERR_CUDA: return "CUDA error";
    case MPAP_ERR_SAMPLING: return "sampling failed";
    default: return "unknown status";
  }
}

const char* mpap_last_error(void) { return mpap::last_error(); }

int32_t mpap_build_roadmap(const mpap_scene* scene, const mpap_roadmap_params* p, mpap_roadmap** out,
                           void* stream) {
  int32_t rc = check_scene(scene);
  if (rc) return rc;
  if (!p || !out) {
    set_error("null params/out");
    return MPAP_ERR_INVALID_ARG;
  }
  if ((rc = check_conn(p->r, p->T_edge, p->M, scene->dim_kind))) return rc;
  if (p->n == 0 || p->n > 0x0FFFFFFFu) {
    set_error("n must be in [1, 2^28)");
    return MPAP_ERR_INVALID_ARG;
  }
  *out = nullptr;
  mpap::BuildSpec sp{scene, p, nullptr, 0, p->r, p->T_edge, p->goal_radius, p->M};
  return mpap::build_roadmaps_impl(1, &sp, out, S(stream));
}


int32_t mpap_build_roadmaps(uint32_t n, const mpap_scene* scenes, const mpap_roadmap_params* params,
                            mpap_roadmap** rms, void* stream) {
  if (n && (!scenes || !params || !rms)) {
    set_error("null argument");
    return MPAP_ERR_INVALID_ARG;
  }
  std::vector<mpap::BuildSpec> specs;
  int32_t rc = batch_specs(n, scenes, params, specs);
  if (rc) return rc;
  return mpap::build_roadmaps_impl(n, specs.data(), rms, S(stream));
}

int32_t mpap_build_roadmap_from_points(const mpap_scene* scene, uint32_t V, const float* x, float r, float T,
                                       int32_t M, float goal_radius, mpap_roadmap** out, void* stream) {
  int32_t rc = check_scene(scene);
  if (rc) return rc;
  if (!x || !out || V < 2) {
    set_error("need x, out and V >= 2");
    return MPAP_ERR_INVALID_ARG;
  }
  if ((rc = check_conn(r, T, M, scene->dim_kind))) return rc;
  *out = nullptr;
  mpap::BuildSpec sp{scene, nullptr, x, V, r, T, goal_radius, M};
  return mpap::build_roadmaps_impl(1, &sp, out, S(stream));
}

int32_t mpap_roadmap_from_csr(uint32_t V, const uint32_t* row_ptr, const uint32_t* dst, const int32_t* cost_q,
                              const int32_t* Sv, const int32_t* C, const uint8_t* is_goal, mpap_roadmap** out,
                              void* stream) {
  return mpap_roadmap_from_csr_peaks(V, row_ptr, dst, cost_q, Sv, C, nullptr, nullptr, is_goal, out, stream);
}

int32_t mpap_roadmap_from_csr_peaks(uint32_t V, const uint32_t* row_ptr, const uint32_t* dst,
                                    const int32_t* cost_q, const int32_t* Sv, const int32_t* C,
                                    const int32_t* Smax, const int32_t* Cmax, const uint8_t* is_goal,
                                    mpap_roadmap** out, void* stream) {
  if (!row_ptr || !is_goal || !out || V < 1) {
    set_error("need row_ptr, is_goal, out and V >= 1");
    return MPAP_ERR_INVALID_ARG;
  }
  const uint32_t E = row_ptr[V];
  if (E && (!dst || !cost_q || !Sv || !C)) {
    set_error("null edge arrays");
    return MPAP_ERR_INVALID_ARG;
  }
  if ((Smax == nullptr) != (Cmax == nullptr)) {
    set_error("give both Smax and Cmax or neither");
    return MPAP_ERR_INVALID_ARG;
  }
  for (uint32_t v = 0; v < V; ++v)
    if (row_ptr[v] > row_ptr[v + 1]) {
      set_error("row_ptr not monotone");
      return MPAP_ERR_INVALID_ARG;
    }
  for (uint32_t e = 0; e < E; ++e) {
    if (dst[e] >= V || cost_q[e] < 1 || C[e] < 0) {
      set_error("edge %u: dst out of range, cost_q < 1 or C < 0", e);
      return MPAP_ERR_INVALID_ARG;
    }
    if (Smax && (Smax[e] < Sv[e] || Cmax[e] < C[e])) {
      set_error("edge %u: need Smax >= S and Cmax >= C", e);
      return MPAP_ERR_INVALID_ARG;
    }
  }
  *out = nullptr;
  return mpap::roadmap_from_csr_impl(V, row_ptr, dst, cost_q, Sv, C, Smax, Cmax, is_goal, out, S(stream));
}

int32_t mpap_roadmap_export_yaw(const mpap_roadmap* rm, float* yaw, void* stream) {
  if (!rm || !yaw) {
    set_error("null argument");
    return MPAP_ERR_INVALID_ARG;
  }
  cudaStream_t st = S(stream);
  if (rm->n_head && rm->yaw && rm->V) {
    MPAP_CK(cudaMemcpyAsync(yaw, rm->yaw, sizeof(float) * (size_t)rm->V, cudaMemcpyDeviceToHost, st));
    MPAP_CK(cudaStreamSynchronize(st));
  } else {
    std::memset(yaw, 0, sizeof(float) * (size_t)rm->V);
  }
  return MPAP_OK;
}

int32_t mpap_roadmap_export_peaks(const mpap_roadmap* rm, int32_t* Smax, int32_t* Cmax, void* stream) {
  if (!rm) {
    set_error("null roadmap");
    return MPAP_ERR_INVALID_ARG;
  }
  cudaStream_t st = S(stream);
  const size_t E = (size_t)rm->E;
  std::vector<int4> ed(E ? E : 1);
  std::vector<int2> pk(E ? E : 1);
  std::vector<uint32_t> rp((size_t)rm->V + 1);
  if (E) {
    MPAP_CK(cudaMemcpyAsync(ed.data(), rm->fwd_edge, sizeof(int4) * E, cudaMemcpyDeviceToHost, st));
    MPAP_CK(cudaMemcpyAsync(pk.data(), rm->fwd_peak, sizeof(int2) * E, cudaMemcpyDeviceToHost, st));
  }
  MPAP_CK(cudaMemcpyAsync(rp.data(), rm->fwd_ptr, 4 * ((size_t)rm->V + 1), cudaMemcpyDeviceToHost, st));
  MPAP_CK(cudaStreamSynchronize(st));
  // the export's order: every row sorted by neighbour
  std::vector<uint32_t> idx(E ? E : 1);
  for (size_t e = 0; e < E; ++e) idx[e] = (uint32_t)e;
  for (uint32_t v = 0; v < rm->V; ++v)
    std::sort(idx.begin() + rp[v], idx.begin() + rp[v + 1],
              [&](uint32_t a, uint32_t b) { return ed[a].x < ed[b].x; });
  for (size_t e = 0; e < E; ++e) {
    if (Smax) Smax[e] = pk[idx[e]].x;
    if (Cmax) Cmax[e] = pk[idx[e]].y;
  }
  return MPAP_OK;
}

int32_t mpap_roadmap_export_reverse(const mpap_roadmap* rm, uint32_t* rev_ptr, uint32_t* src, int32_t* cost_q,
                                    int32_t* Sv, int32_t* C, int32_t* Smax, int32_t* Cmax, void* stream) {
  if (!rm) {
    set_error("null roadmap");
    return MPAP_ERR_INVALID_ARG;
  }
  cudaStream_t st = S(stream);
  const size_t E = (size_t)rm->E;
  std::vector<int4> ed(E ? E : 1);
  std::vector<int2> pk(E ? E : 1);
  std::vector<uint32_t> rp((size_t)rm->V + 1);
  if (E) {
    MPAP_CK(cudaMemcpyAsync(ed.data(), rm->rev_edge, sizeof(int4) * E, cudaMemcpyDeviceToHost, st));
    MPAP_CK(cudaMemcpyAsync(pk.data(), rm->rev_peak, sizeof(int2) * E, cudaMemcpyDeviceToHost, st));
  }
  MPAP_CK(cudaMemcpyAsync(rp.data(), rm->rev_ptr, 4 * ((size_t)rm->V + 1), cudaMemcpyDeviceToHost, st));
  MPAP_CK(cudaStreamSynchronize(st));
  // device rows are in arrival order; return them sorted by source
  std::vector<uint32_t> idx(E ? E : 1);
  for (size_t e = 0; e < E; ++e) idx[e] = (uint32_t)e;
  for (uint32_t v = 0; v < rm->V; ++v)
    std::sort(idx.begin() + rp[v], idx.begin() + rp[v + 1],
              [&](uint32_t a, uint32_t b) { return ed[a].x < ed[b].x; });
  if (rev_ptr) std::memcpy(rev_ptr, rp.data(), 4 * ((size_t)rm->V + 1));
  for (size_t e = 0; e < E; ++e) {
    const int4& r = ed[idx[e]];
    if (src) src[e] = (uint32_t)r.x;
    if (cost_q) cost_q[e] = r.y;
    if (Sv) Sv[e] = r.z;
    if (C) C[e] = r.w;
    if (Smax) Smax[e] = pk[idx[e]].x;
    if (Cmax) Cmax[e] = pk[idx[e]].y;
  }
  return MPAP_OK;
}

int32_t mpap_roadmap_update(mpap_roadmap* rm, int32_t nb_add, const float* add_lo, const float* add_hi,
                            const uint8_t* grid, int32_t mem, void* stream) {
  if (!rm || nb_add < 0 || (nb_add > 0 && (!add_lo || !add_hi))) {
    set_error("roadmap_update: null roadmap, negative box count or null box arrays");
    return MPAP_ERR_INVALID_ARG;
  }
  if (mem != MPAP_MEM_HOST && mem != MPAP_MEM_DEVICE) {
    set_error("roadmap_update: mem must be MPAP_MEM_HOST or MPAP_MEM_DEVICE");
    return MPAP_ERR_INVALID_ARG;
  }
  return mpap::roadmap_update_batch_impl(1, &rm, &nb_add, &add_lo, &add_hi, &grid, mem == MPAP_MEM_DEVICE,
                                         S(stream));
}

int32_t mpap_roadmap_update_batch(mpap_roadmap* const* rms, uint32_t n, const int32_t* nb_add,
                                  const float* const* add_lo, const float* const* add_hi,
                                  const uint8_t* const* grids, int32_t mem, void* stream) {
  if (n == 0) return MPAP_OK;
  if (!rms || !nb_add || !add_lo || !add_hi) {
    set_error("roadmap_update_batch: null array");
    return MPAP_ERR_INVALID_ARG;
  }
  for (uint32_t j = 0; j < n; ++j)
    if (!rms[j] || nb_add[j] < 0 || (nb_add[j] > 0 && (!add_lo[j] || !add_hi[j]))) {
      set_error("roadmap_update_batch: roadmap %u: null roadmap, negative box count or null box arrays", j);
      return MPAP_ERR_INVALID_ARG;
    }
  for (uint32_t j = 0; j < n; ++j)
    for (uint32_t k = j + 1; k < n; ++k)
      if (rms[j] == rms[k]) {
        set_error("roadmap_update_batch: roadmap %u appears twice", k);
        return MPAP_ERR_INVALID_ARG;
      }
  if (mem != MPAP_MEM_HOST && mem != MPAP_MEM_DEVICE) {
    set_error("roadmap_update_batch: mem must be MPAP_MEM_HOST or MPAP_MEM_DEVICE");
    return MPAP_ERR_INVALID_ARG;
  }
  return mpap::roadmap_update_batch_impl(n, rms, nb_add, add_lo, add_hi, grids, mem == MPAP_MEM_DEVICE, S(stream));
}

int32_t mpap_roadmap_info(const mpap_roadmap* rm, uint32_t* V, uint64_t* E) {
  if (!rm) {
    set_error("null roadmap");
    return MPAP_ERR_INVALID_ARG;
  }
  if (V) *V = rm->V;
  if (E) *E = rm->E;
  return MPAP_OK;
}

int32_t mpap_roadmap_export(const mpap_roadmap* rm, float* x, uint8_t* is_goal, uint32_t* row_ptr, uint32_t* dst,
                            int32_t* cost_q, int32_t* Sv, int32_t* C, void* stream) {
  if (!rm) {
    set_error("null roadmap");
    return MPAP_ERR_INVALID_ARG;
  }
  cudaStream_t st = S(stream);
  if (x) MPAP_CK(cudaMemcpyAsync(x, rm->x, sizeof(float) * 6 * (size_t)rm->V, cudaMemcpyDeviceToHost, st));
  if (is_goal) MPAP_CK(cudaMemcpyAsync(is_goal, rm->is_goal, rm->V, cudaMemcpyDeviceToHost, st));
  if (row_ptr)
    MPAP_CK(cudaMemcpyAsync(row_ptr, rm->fwd_ptr, 4 * ((size_t)rm->V + 1), cudaMemcpyDeviceToHost, st));
  if (dst || cost_q || Sv || C) {
    int4* tmp = new int4[rm->E ? rm->E : 1];
    if (rm->E && !mpap::cuda_ok(cudaMemcpyAsync(tmp, rm->fwd_edge, sizeof(int4) * rm->E, cudaMemcpyDeviceToHost, st),
                                "export edges")) {
      delete[] tmp;
      return MPAP_ERR_CUDA;
    }
    if (!mpap::cuda_ok(cudaStreamSynchronize(st), "sync")) {
      delete[] tmp;
      return MPAP_ERR_CUDA;
    }
    // device rows are in discovery order; return them sorted by neighbour
    std::vector<uint32_t> rp(rm->V + 1);
    if (!mpap::cuda_ok(cudaMemcpy(rp.data(), rm->fwd_ptr, 4 * ((size_t)rm->V + 1), cudaMemcpyDeviceToHost),
                       "export row pointers")) {
      delete[] tmp;
      return MPAP_ERR_CUDA;
    }
    for (uint32_t v = 0; v < rm->V; ++v)
      std::sort(tmp + rp[v], tmp + rp[v + 1], [](const int4& a, const int4& b) { return a.x < b.x; });
    for (uint64_t e = 0; e < rm->E; ++e) {
      if (dst) dst[e] = (uint32_t)tmp[e].x;
      if (cost_q) cost_q[e] = tmp[e].y;
      if (Sv) Sv[e] = tmp[e].z;
      if (C) C[e] = tmp[e].w;
    }
    delete[] tmp;
  }
  MPAP_CK(cudaStreamSynchronize(st));
  return MPAP_OK;
}

int32_t mpap_roadmap_stats(const mpap_roadmap* rm, uint64_t* near_tests, uint32_t* n_goal) {
  if (!rm) {
    set_error("null roadmap");
    return MPAP_ERR_INVALID_ARG;
  }
  if (near_tests) *near_tests = rm->near_tests;
  if (n_goal) *n_goal = rm->n_goal;
  return MPAP_OK;
}

void mpap_roadmap_free(mpap_roadmap* rm) { mpap::roadmap_free_impl(rm); }

int32_t mpap_workspace_create(uint64_t total_nodes, uint32_t front_cap, uint64_t max_plans,
                              mpap_workspace** out) {
  return mpap::workspace_create(total_nodes, front_cap, max_plans, 4096u, out);
}

void mpap_workspace_free(mpap_workspace* ws) { mpap::workspace_free(ws); }

int32_t mpap_workspace_stats(const mpap_workspace* ws, uint32_t* max_front, uint64_t* pool_used) {
  if (!ws) {
    set_error("mpap_workspace_stats: null workspace");
    return MPAP_ERR_INVALID_ARG;
  }
  if (max_front) *max_front = mpap::workspace_last_max_front(ws);
  if (pool_used) *pool_used = mpap::workspace_last_pool_used(ws);
  return MPAP_OK;
}

int32_t mpap_search(mpap_workspace* ws, mpap_roadmap* rm, const mpap_query* q, mpap_result* out, void* stream) {
  if (!ws || !rm || !q || !out) {
    set_error("null argument");
    return MPAP_ERR_INVALID_ARG;
  }
  int32_t rc = mpap::search_batch_impl(ws, &rm, q, 1, out, S(stream));
  if (rc < 0) return rc;
  return out->status;
}

int32_t mpap_search_batch(mpap_workspace* ws, mpap_roadmap* const* rms, const mpap_query* qs, uint32_t nq,
                          mpap_result* outs, void* stream) {
  if (!ws || (nq && (!rms || !qs || !outs))) {
    set_error("null argument");
    return MPAP_ERR_INVALID_ARG;
  }
  return mpap::search_batch_impl(ws, rms, qs, nq, outs, S(stream));
}

int32_t mpap_search_fronts(mpap_workspace* ws, uint32_t index, uint32_t* front_ptr, int64_t* cost, int64_t* h,
                           uint64_t cap, uint64_t* total, void* stream) {
  if (!ws) {
    set_error("null workspace");
    return MPAP_ERR_INVALID_ARG;
  }
  return mpap::search_fronts_impl(ws, index, front_ptr, cost, h, cap, total, S(stream));
}

int32_t mpap_certify(mpap_roadmap* rm, const uint32_t* path, uint32_t path_len, const mpap_mc_params* mc,
                     mpap_cert* out, void* stream) {
  if (!rm || !mc || !out || (path_len && !path)) {
    set_error("null argument");
    return MPAP_ERR_INVALID_ARG;
  }
  return mpap::certify_batch_impl(&rm, &path, &path_len, mc, 1, out, S(stream));
}

int32_t mpap_certify_noalloc(const mpap_roadmap* rm, const uint32_t* path, uint32_t path_len,
                             const mpap_mc_params* mc, mpap_cert* out, void* stream) {
  if (!rm || !mc || !out || (path_len && !path) || !mc->sigma_fx || !mc->shift) {
    set_error("null argument");
    return MPAP_ERR_INVALID_ARG;
  }
  return mpap::certify_noalloc_impl(rm, path, path_len, mc, out, S(stream));
}

int32_t mpap_certify_batch(mpap_roadmap* const* rms, const uint32_t* const* paths, const uint32_t* path_lens,
                           const mpap_mc_params* mcs, uint32_t n, mpap_cert* outs, void* stream) {
  if (n && (!rms || !paths || !path_lens || !mcs || !outs)) {
    set_error("null argument");
    return MPAP_ERR_INVALID_ARG;
  }
  return mpap::certify_batch_impl(rms, paths, path_lens, mcs, n, outs, S(stream));
}

int32_t mpap_vio_lqr_gains(double q_p, double q_w, double r, int32_t* kp_q16, int32_t* kv_q16) {
  if (!kp_q16 || !kv_q16 || !(q_p >= 0.0) || !(q_w >= 0.0) || !(r > 0.0)) {
    set_error("mpap_vio_lqr_gains: weights must be q_p, q_w >= 0 and r > 0, outputs non-null");
    return MPAP_ERR_INVALID_ARG;
  }
  // P <- Q + A^T P A - A^T P B (r + B^T P B)^-1 B^T P A, A = [1 1; 0 1], B = (1/2, 1)
  double p00 = q_p, p01 = 0.0, p11 = q_w;
  double k0 = 0.0, k1 = 0.0;
  for (int it = 0; it < 1000000; ++it) {
    // B^T P = (p00/2 + p01, p01/2 + p11); B^T P B; B^T P A
    const double bp0 = 0.5 * p00 + p01, bp1 = 0.5 * p01 + p11;
    const double bpb = 0.5 * bp0 + bp1;
    const double g0 = bp0, g1 = bp0 + bp1;            // B^T P A
    const double s = r + bpb;
    k0 = g0 / s;
    k1 = g1 / s;
    // A^T P A
    const double a00 = p00, a01 = p00 + p01, a11 = p00 + 2.0 * p01 + p11;
    const double n00 = q_p + a00 - g0 * k0;
    const double n01 = a01 - g0 * k1;
    const double n11 = q_w + a11 - g1 * k1;
    const double d = std::max(std::fabs(n00 - p00), std::max(std::fabs(n01 - p01), std::fabs(n11 - p11)));
    p00 = n00;
    p01 = n01;
    p11 = n11;
    if (d <= 1e-14 * std::max(1.0, std::max(std::fabs(p00), std::fabs(p11)))) break;
  }
  const double bp0 = 0.5 * p00 + p01, bp1 = 0.5 * p01 + p11;
  const double s = r + 0.5 * bp0 + bp1;
  *kp_q16 = (int32_t)llrint(bp0 / s * 65536.0);
  *kv_q16 = (int32_t)llrint((bp0 + bp1) / s * 65536.0);
  return MPAP_OK;
}

int32_t mpap_certify_vio_batch(mpap_roadmap* const* rms, const uint32_t* const* paths, const uint32_t* path_lens,
                               const mpap_mc_params* mcs, const mpap_vio_params* vps, uint32_t n, mpap_cert* outs,
                               void* stream) {
  if (n && (!rms || !paths || !path_lens || !mcs || !vps || !outs)) {
    set_error("null argument");
    return MPAP_ERR_INVALID_ARG;
  }
  return mpap::certify_vio_batch_impl(rms, paths, path_lens, mcs, vps, n, outs, S(stream));
}

int32_t mpap_search_candidates(mpap_workspace* ws, uint32_t index, uint32_t cap, int64_t* cost, int64_t* h,
                               uint32_t* path_ptr, uint32_t* path, uint32_t path_cap, uint32_t* n, uint32_t* total,
                               void* stream) {
  if (!ws || !n) {
    set_error("search_candidates: null workspace or count");
    return MPAP_ERR_INVALID_ARG;
  }
  if (cap > (1u << 16)) {
    set_error("search_candidates: cap must be at most 65536");
    return MPAP_ERR_INVALID_ARG;
  }
  return mpap::search_candidates_impl(ws, index, cap, cost, h, path_ptr, path, path_cap, n, total, S(stream));
}

int32_t mpap_plan_features(mpap_roadmap* rm, uint32_t n, const uint32_t* path_ptr, const uint32_t* path, float* feat,
                           void* stream) {
  return mpap::plan_features_impl(rm, n, path_ptr, path, feat, S(stream));
}

int32_t mpap_feature_levels(int32_t dim_kind, int32_t nb, const float* box_lo, const float* box_hi,
                            uint32_t n_features, const float* features, int32_t grid_G, uint32_t yaw_bins,
                            const float* headings, float cos_half_fov, float range, int32_t K,
                            uint8_t* levels, int32_t mem, void* stream) {
  if (dim_kind != 2 && dim_kind != 3 && dim_kind != 6) {
    set_error("feature_levels: dim_kind must be 2, 3 or 6");
    return MPAP_ERR_INVALID_ARG;
  }
  if (grid_G < 1 || grid_G > 1024 || (grid_G & (grid_G - 1)) || K < 0 || K > 255 || yaw_bins < 1 ||
      nb < 0 || nb > 1024 || n_features > (1u << 22) || !(range >= 0.0f) || std::isinf(range) ||
      std::isnan(cos_half_fov)) {
    set_error("feature_levels: need G a power of two in [1, 1024], K in [0, 255], yaw_bins >= 1, "
              "0 <= nb <= 1024, at most 2^22 features, a finite range >= 0");
    return MPAP_ERR_INVALID_ARG;
  }
  if (mem != MPAP_MEM_HOST && mem != MPAP_MEM_DEVICE) {
    set_error("feature_levels: mem must be MPAP_MEM_HOST or MPAP_MEM_DEVICE");
    return MPAP_ERR_INVALID_ARG;
  }
  if (!levels || !headings || (nb > 0 && (!box_lo || !box_hi)) || (n_features > 0 && !features)) {
    set_error("feature_levels: null array");
    return MPAP_ERR_INVALID_ARG;
  }
  const int dp = dim_kind == 2 ? 2 : 3;
  const unsigned long long cells = (unsigned long long)grid_G * grid_G * (dp == 3 ? grid_G : 1);
  if ((unsigned long long)yaw_bins * cells > (1ull << 31)) {
    set_error("feature_levels: yaw_bins x G^Dp above 2^31");
    return MPAP_ERR_INVALID_ARG;
  }
  return mpap::feature_levels_impl(dp, nb, box_lo, box_hi, n_features, features, (uint32_t)grid_G, yaw_bins,
                                   headings, cos_half_fov, range, K, levels, mem == MPAP_MEM_DEVICE, S(stream));
}

int32_t mpap_plan_features_batch(mpap_roadmap* const* rms, uint32_t n_rm, const uint32_t* plan_ptr,
                                 const uint32_t* path_ptr, const uint32_t* path, float* feat, void* stream) {
  return mpap::plan_features_batch_impl(rms, n_rm, plan_ptr, path_ptr, path, feat, S(stream));
}

int32_t mpap_search_candidates_batch(mpap_workspace* ws, uint32_t nq, uint32_t cap, int64_t* cost, int64_t* h,
                                     uint32_t* path_ptr, uint32_t* path, uint32_t path_cap, uint32_t* n,
                                     uint32_t* total, void* stream) {
  if (!ws || (nq && (!n || !cost || !h || !path_ptr || !path))) {
    set_error("search_candidates_batch: null argument");
    return MPAP_ERR_INVALID_ARG;
  }
  if (cap > (1u << 16)) {
    set_error("search_candidates_batch: cap must be at most 65536");
    return MPAP_ERR_INVALID_ARG;
  }
  return mpap::search_candidates_batch_impl(ws, nq, cap, cost, h, path_ptr, path, path_cap, n, total, S(stream));
}

int32_t mpap_mlp_create(uint64_t seed, uint32_t max_batch, mpap_mlp** out) {
  return mpap::mlp_create(seed, max_batch, out);
}

void mpap_mlp_free(mpap_mlp* net) { mpap::mlp_free(net); }

int32_t mpap_mlp_get_params(mpap_mlp* net, float* params, void* stream) {
  if (!net || !params) {
    set_error("mlp_get_params: null argument");
    return MPAP_ERR_INVALID_ARG;
  }
  return mpap::mlp_get_params(net, params, S(stream));
}

int32_t mpap_mlp_set_params(mpap_mlp* net, const float* params, void* stream) {
  if (!net || !params) {
    set_error("mlp_set_params: null argument");
    return MPAP_ERR_INVALID_ARG;
  }
  return mpap::mlp_set_params(net, params, S(stream));
}

int32_t mpap_mlp_forward(mpap_mlp* net, const float* x, uint32_t n, float* prob, int32_t mem, void* stream) {
  if (!net || (n && (!x || !prob)) || (mem != MPAP_MEM_HOST && mem != MPAP_MEM_DEVICE)) {
    set_error("mlp_forward: null argument or bad mem");
    return MPAP_ERR_INVALID_ARG;
  }
  return mpap::mlp_forward(net, x, n, prob, mem, S(stream));
}

int32_t mpap_mlp_train_step(mpap_mlp* net, const float* x, const float* y, uint32_t n, float lr, int32_t apply,
                            float* loss, float* grads, int32_t mem, void* stream) {
  if (!net || !x || !y || (mem != MPAP_MEM_HOST && mem != MPAP_MEM_DEVICE) || !(lr >= 0.0f)) {
    set_error("mlp_train_step: null argument, bad mem or negative lr");
    return MPAP_ERR_INVALID_ARG;
  }
  return mpap::mlp_train_step(net, x, y, n, lr, apply, loss, grads, mem, S(stream));
}

int32_t mpap_tuning_get(int32_t dim_kind, uint32_t V, mpap_tuning* out) {
  if (!out) {
    set_error("tuning_get: null output");
    return MPAP_ERR_INVALID_ARG;
  }
  *out = mpap::tuning_for(dim_kind, V);
  return MPAP_OK;
}

int32_t mpap_tuning_set(int32_t dim_kind, uint32_t V, const mpap_tuning* t) {
  if (!t) {
    set_error("tuning_set: null entry");
    return MPAP_ERR_INVALID_ARG;
  }
  return mpap::tuning_set(dim_kind, V, *t);
}

int32_t mpap_tuning_clear(void) {
  mpap::tuning_clear();
  return MPAP_OK;
}

int32_t mpap_tuning_export(uint32_t cap, int32_t* dim_kind, uint32_t* bucket, mpap_tuning* t, uint32_t* n) {
  if (!n) {
    set_error("tuning_export: null count");
    return MPAP_ERR_INVALID_ARG;
  }
  return mpap::tuning_export(cap, dim_kind, bucket, t, n);
}

int32_t mpap_autotune_build(uint32_t n, const mpap_scene* scenes, const mpap_roadmap_params* params,
                            mpap_roadmap** rms, uint32_t reps, mpap_tuning* best, double* best_ms, void* stream) {
  if (!n || !scenes || !params || !rms || !best || !best_ms || reps == 0) {
    set_error("autotune_build: null argument, empty batch or zero reps");
    return MPAP_ERR_INVALID_ARG;
  }
  std::vector<mpap::BuildSpec> specs;
  int32_t rc = batch_specs(n, scenes, params, specs);
  if (rc) return rc;
  // the (dimension, largest V) key of every dimension group of the batch
  std::vector<std::pair<int, uint32_t>> keys;
  for (int d : {2, 3, 6}) {
    uint32_t vmax = 0;
    for (uint32_t i = 0; i < n; ++i)
      if (scenes[i].dim_kind == d) vmax = std::max(vmax, params[i].n + 2u);
    if (vmax) keys.push_back({d, vmax});
  }
  const cudaStream_t st = S(stream);
  double best_t = 1e300;
  uint32_t best_w = 8;
  for (uint32_t warps : {4u, 8u}) {
    for (const auto& k : keys) {
      mpap_tuning t = mpap::tuning_for(k.first, k.second);
      t.edge_warps = warps;
      mpap::tuning_set(k.first, k.second, t);
    }
    double ms = 0.0;
    rc = time_reps(st, reps, [&] { return mpap::build_roadmaps_impl(n, specs.data(), rms, st); }, &ms);
    if (rc) return rc;
    if (ms < best_t) {
      best_t = ms;
      best_w = warps;
    }
  }
  for (const auto& k : keys) {
    mpap_tuning t = mpap::tuning_for(k.first, k.second);
    t.edge_warps = best_w;
    mpap::tuning_set(k.first, k.second, t);
  }
  *best = mpap::tuning_for(keys[0].first, keys[0].second);
  *best_ms = best_t;
  return MPAP_OK;
}

int32_t mpap_autotune_search(mpap_workspace* ws, mpap_roadmap* const* rms, const mpap_query* qs, uint32_t nq,
                             uint32_t reps, mpap_tuning* best, double* best_ms, void* stream) {
  if (!ws || !nq || !rms || !qs || !best || !best_ms || reps == 0) {
    set_error("autotune_search: null argument, empty batch or zero reps");
    return MPAP_ERR_INVALID_ARG;
  }
  int kdim = 0;
  uint32_t kV = 0;
  mpap::batch_key(rms, nq, kdim, kV);
  const mpap_tuning base = mpap::tuning_for(kdim, kV);
  const cudaStream_t st = S(stream);
  std::vector<std::vector<uint32_t>> paths(nq, std::vector<uint32_t>(4096));
  std::vector<mpap_result> outs(nq), ref;
  auto run = [&] {
    for (uint32_t i = 0; i < nq; ++i) {
      outs[i] = mpap_result{};
      outs[i].path = paths[i].data();
      outs[i].path_cap = 4096;
    }
    // a query out of its own pool share reports it in its status, which is
    // compared across shapes like every other result
    const int32_t rc = mpap::search_batch_impl(ws, rms, qs, nq, outs.data(), st);
    return rc == MPAP_ERR_CAPACITY ? MPAP_OK : rc;
  };
  double best_t = 1e300;
  mpap_tuning bt = base;
  unsigned long long pool_used = 0;
  uint64_t nodes = 0;
  for (uint32_t i = 0; i < nq; ++i) nodes += rms[i] ? rms[i]->V : 0u;
  const uint32_t blocks[] = {1, 2, 4, 8};
  const uint32_t lanes[] = {4, 8, 16, 32};
  for (uint32_t bps : blocks) {
    for (uint32_t lf : lanes) {
      mpap_tuning t = base;
      t.wave_blocks_per_sm = bps;
      t.plan_lanes_from = lf;
      mpap::tuning_set(kdim, kV, t);
      double ms = 0.0;
      const int32_t rc = time_reps(st, reps, run, &ms);
      if (rc < 0) {
        mpap::tuning_set(kdim, kV, base);
        return rc;
      }
      if (ref.empty()) {
        ref = outs;
      } else {
        for (uint32_t i = 0; i < nq; ++i)
          if (outs[i].status != ref[i].status || outs[i].cost != ref[i].cost || outs[i].h != ref[i].h ||
              outs[i].expansions != ref[i].expansions) {
            mpap::tuning_set(kdim, kV, base);
            set_error("autotune_search: query %u differs between launch shapes", i);
            return MPAP_ERR_CUDA;
          }
      }
      pool_used = std::max(pool_used, mpap::workspace_last_pool_used(ws));
      if (ms < best_t) {
        best_t = ms;
        bt = t;
      }
    }
  }
  uint32_t fc = 16;
  while ((uint64_t)fc * std::max<uint64_t>(nodes, 1) < 2 * pool_used) fc <<= 1;
  bt.front_cap = fc;
  mpap::tuning_set(kdim, kV, bt);
  *best = bt;
  *best_ms = best_t;
  return MPAP_OK;
}

}  // extern "C"
