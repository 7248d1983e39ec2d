// Host-side internals of libmpap: handle layouts and cross-file helpers.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/mpap.h"
#include "common.cuh"

struct mpap_roadmap {
  int dim = 2;
  uint32_t V = 0;
  uint64_t E = 0;
  int M = 16;
  int n_f = 12, K = 24, G = 1, nb = 0;
  float r = 0.0f, T = 0.25f, goal_radius = 0.0f;
  bool has_geometry = false;
  mpap::Geom geom{};           // device pointers below, constants filled
  // device arrays (owned; capacities in elements, reused by rebuilds)
  float* x = nullptr;          // [6][V]
  uint8_t* is_goal = nullptr;  // [V]
  uint32_t* goal_list = nullptr;
  uint32_t n_goal = 0;
  uint32_t* fwd_ptr = nullptr; // [V+1]
  int4* fwd_edge = nullptr;    // [E] {dst, cost_q, S, C}, rows in discovery order
  uint32_t* fwd_dst = nullptr; // [E] dst only (for marking out-neighbours)
  uint32_t* rev_ptr = nullptr; // [V+1]
  int4* rev_edge = nullptr;    // [E] {src, cost_q, S, C}
  int2* fwd_peak = nullptr;    // [E] {Smax, Cmax}: peak of the transfer over the edge
  int2* rev_peak = nullptr;    // [E] the same in reverse-CSR order
  float* box_lo = nullptr;     // [nb][3]
  float* box_hi = nullptr;
  uint8_t* grid = nullptr;
  int n_head = 0;              // camera-heading form: level tables per heading and node yaws
  uint8_t* head = nullptr;     // [n_head][G^Dp]
  float* yaw = nullptr;        // [V]
  size_t cap_head = 0, cap_yaw = 0;
  size_t cap_V = 0, cap_E = 0, cap_nb = 0, cap_cells = 0;
  uint64_t near_tests = 0;     // Cost < r tests evaluated by the last build
};

namespace mpap {

void set_error(const char* fmt, ...);
bool cuda_ok(cudaError_t e, const char* what);

#define MPAP_CK(call)                                   \
  do {                                                  \
    if (!::mpap::cuda_ok((call), #call)) return MPAP_ERR_CUDA; \
  } while (0)

// Fill the double-integrator constants and scalars of g from (T, M, ...).
void fill_geom_constants(Geom& g, int dim, int nb, int G, int n_f, int M, float r, float T);

// One roadmap to (re)build.  Exactly one of `params` (SampleFree) or `points`
// (caller-given node states, host, [6][V]) is set.
struct BuildSpec {
  const mpap_scene* scene;
  const mpap_roadmap_params* params;
  const float* points;
  uint32_t V_points;
  float r, T, goal_radius;
  int M;
};

// Builds every spec into rms[i] (a null rms[i] gets a new handle; an existing
// one is rebuilt in place, reusing its device buffers when large enough).
int32_t build_roadmaps_impl(uint32_t n, const BuildSpec* specs, mpap_roadmap** rms, cudaStream_t st);
// Smax/Cmax may be null: every edge is then one step (its peak is its end value).
int32_t roadmap_from_csr_impl(uint32_t V, const uint32_t* row_ptr, const uint32_t* dst,
                              const int32_t* cost_q, const int32_t* S, const int32_t* C,
                              const int32_t* Smax, const int32_t* Cmax,
                              const uint8_t* is_goal, mpap_roadmap** out, cudaStream_t st);
void roadmap_free_impl(mpap_roadmap* rm);

// Launch shapes from the tuning table (tune.cu), keyed by (dimension, node-count
// bucket floor(log2 V)); dimension 0 stands for a batch mixing dimensions.
// Entries absent from the table give the defaults.
mpap_tuning tuning_for(int dim, uint32_t V);
bool tuning_valid(const mpap_tuning& t);

// Stream-ordered scratch from the library's memory pool (kept mapped).
cudaError_t scratch_alloc(void** p, size_t bytes, cudaStream_t st);
void scratch_free(void* p, cudaStream_t st);

}  // namespace mpap
