// Certification-driven choice of plans (host side): the refinement of the
// perception bound of Alg. 1 step 4 (Sec. 3: Monte Carlo certification, then
// loosening or tightening beta and exploring again), and the screened
// certification of candidate plans that serves the learned surrogate.  Both
// sequence the library's batched kernels (search, certification, features,
// network); nothing here computes on the host beyond the bound rule and the
// candidate order.
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"

namespace mpap {

int32_t search_batch_impl(mpap_workspace* ws, mpap_roadmap* const* rms, const mpap_query* qs, uint32_t nq,
                          mpap_result* outs, cudaStream_t st);
int32_t certify_batch_impl(mpap_roadmap* const* rms, const uint32_t* const* paths, const uint32_t* path_lens,
                           const mpap_mc_params* mcs, uint32_t n, mpap_cert* outs, cudaStream_t st);
int32_t plan_features_batch_impl(mpap_roadmap* const* rms, uint32_t n_rm, const uint32_t* plan_ptr,
                                 const uint32_t* path_ptr, const uint32_t* path, float* feat, cudaStream_t st);
int32_t mlp_forward(mpap_mlp* nt, const float* x, uint32_t n, float* prob, int32_t mem, cudaStream_t st);
uint32_t mlp_max_batch(const mpap_mlp* nt);

namespace {

constexpr int64_t kBetaCap = (int64_t)1 << 62;

// floor(a / 2) for a possibly negative a (the bound rule halves -1 + f).
int64_t floor_half(__int128 a) { return (int64_t)(a >= 0 ? a / 2 : -((-a + 1) / 2)); }

}  // namespace

// The bound rule (see include/mpap.h): records the outcome at beta and
// returns the next bound, -1 to stop.
int64_t refine_next(mpap_refine_bounds& b, int64_t beta, int32_t outcome, int64_t cost) {
  bool cheaper = false;
  if (outcome == MPAP_REFINE_PASS) {
    cheaper = b.lo < 0 || cost < b.lo_cost;
    b.lo = beta;
    b.lo_cost = cost;
  } else if (outcome == MPAP_REFINE_FAIL) {
    b.hi = beta;
  } else {
    b.none = beta;
  }
  if (b.hi < 0) {
    // no failure seen: loosen while passes bring cheaper plans (or no plan exists)
    if (outcome == MPAP_REFINE_PASS && !cheaper) return -1;
    const int64_t nb = beta > (kBetaCap - 1) / 2 ? kBetaCap : 2 * beta + 1;   // min(2 beta + 1, 2^62)
    return nb > beta ? nb : -1;
  }
  if (b.lo < 0) {
    // failures only: tighten towards the largest bound known to give no plan
    const int64_t below = b.none < 0 ? -1 : b.none;
    const int64_t nb = floor_half((__int128)below + b.hi);
    return nb > below ? nb : -1;
  }
  const int64_t nb = floor_half((__int128)b.lo + b.hi);
  return nb > b.lo ? nb : -1;
}

}  // namespace mpap

extern "C" {

int32_t mpap_refine_advance(mpap_refine_bounds* b, int64_t beta, int32_t outcome, int64_t cost, int64_t* next) {
  if (!b || !next || beta < 0 ||
      (outcome != MPAP_REFINE_PASS && outcome != MPAP_REFINE_FAIL && outcome != MPAP_REFINE_NONE)) {
    mpap::set_error("refine_advance: null pointer, negative beta or an outcome other than pass, fail, none");
    return MPAP_ERR_INVALID_ARG;
  }
  *next = mpap::refine_next(*b, beta, outcome, cost);
  return MPAP_OK;
}

}  // extern "C"

namespace {

cudaStream_t S(void* s) { return static_cast<cudaStream_t>(s); }

}  // namespace

extern "C" {

int32_t mpap_refine_batch(mpap_workspace* ws, mpap_roadmap* const* rms, const mpap_query* qs,
                          const mpap_mc_params* mcs, const uint32_t* max_hits, uint32_t n,
                          uint32_t max_rounds, mpap_refine_result* outs, void* stream) {
  if (!ws || (n && (!rms || !qs || !mcs || !max_hits || !outs))) {
    mpap::set_error("refine_batch: null argument");
    return MPAP_ERR_INVALID_ARG;
  }
  const cudaStream_t st = S(stream);
  std::vector<mpap_refine_bounds> bounds(n, mpap_refine_bounds{-1, 0, -1, -1});
  std::vector<int64_t> beta(n);
  std::vector<uint32_t> active;
  for (uint32_t i = 0; i < n; ++i) {
    if (qs[i].beta < 0) {
      mpap::set_error("refine_batch: query %u has a negative initial bound", i);
      return MPAP_ERR_INVALID_ARG;
    }
    mpap_refine_result& o = outs[i];
    o.certified = 0;
    o.status = MPAP_OK;
    o.beta = -1;
    o.cost = o.h = -1;
    o.path_len = 0;
    o.cert = mpap_cert{0, 0, 0, 0};
    o.rounds = 0;
    beta[i] = qs[i].beta;
    active.push_back(i);
  }
  const uint32_t path_cap = 4096;
  std::vector<uint32_t> buf;
  std::vector<mpap_roadmap*> r_rm;
  std::vector<mpap_query> r_q;
  std::vector<mpap_result> r_out;
  auto record = [&](uint32_t i, int64_t b, int32_t outcome, int64_t cost, int32_t hits) {
    mpap_refine_result& o = outs[i];
    if (o.history && o.rounds < o.hist_cap) o.history[o.rounds] = mpap_refine_round{b, cost, outcome, hits};
    o.rounds += 1;
  };
  for (uint32_t t = 0; !active.empty() && t < max_rounds; ++t) {
    // one batched search over the queries still refining, each at its bound
    const uint32_t na = (uint32_t)active.size();
    buf.assign((size_t)na * path_cap, 0u);
    r_rm.resize(na);
    r_q.resize(na);
    r_out.assign(na, mpap_result{});
    for (uint32_t k = 0; k < na; ++k) {
      r_rm[k] = rms[active[k]];
      r_q[k] = qs[active[k]];
      r_q[k].beta = beta[active[k]];
      r_out[k].path = buf.data() + (size_t)k * path_cap;
      r_out[k].path_cap = path_cap;
    }
    const int32_t rc = mpap::search_batch_impl(ws, r_rm.data(), r_q.data(), na, r_out.data(), st);
    if (rc == MPAP_ERR_CUDA || rc == MPAP_ERR_INVALID_ARG) return rc;
    // one batched certification of the plans found, with call id t
    std::vector<uint32_t> found;
    std::vector<mpap_roadmap*> c_rm;
    std::vector<const uint32_t*> c_path;
    std::vector<uint32_t> c_len;
    std::vector<mpap_mc_params> c_mc;
    for (uint32_t k = 0; k < na; ++k) {
      if (r_out[k].status != MPAP_OK) continue;
      found.push_back(k);
      c_rm.push_back(r_rm[k]);
      c_path.push_back(r_out[k].path);
      c_len.push_back(r_out[k].path_len);
      mpap_mc_params m = mcs[active[k]];
      m.call_id = t;
      c_mc.push_back(m);
    }
    std::vector<mpap_cert> certs(found.size());
    if (!found.empty()) {
      const int32_t rc2 = mpap::certify_batch_impl(c_rm.data(), c_path.data(), c_len.data(), c_mc.data(),
                                                   (uint32_t)found.size(), certs.data(), st);
      if (rc2) return rc2;
    }
    std::vector<uint32_t> next;
    size_t f = 0;
    for (uint32_t k = 0; k < na; ++k) {
      const uint32_t i = active[k];
      const mpap_result& r = r_out[k];
      int32_t outcome;
      if (r.status == MPAP_OK) {
        const mpap_cert& c = certs[f++];
        outcome = c.hits_any <= max_hits[i] ? MPAP_REFINE_PASS : MPAP_REFINE_FAIL;
        if (outcome == MPAP_REFINE_PASS) {
          mpap_refine_result& o = outs[i];
          o.certified = 1;
          o.beta = beta[i];
          o.cost = r.cost;
          o.h = r.h;
          o.cert = c;
          o.path_len = r.path_len;
          if (o.path && o.path_cap >= r.path_len) {
            std::memcpy(o.path, r.path, 4 * (size_t)r.path_len);
            o.status = MPAP_OK;
          } else {
            o.status = MPAP_ERR_INVALID_ARG;
          }
        }
        record(i, beta[i], outcome, r.cost, (int32_t)c.hits_any);
      } else if (r.status == MPAP_NO_SOLUTION) {
        outcome = MPAP_REFINE_NONE;
        record(i, beta[i], outcome, -1, -1);
      } else {
        // a search error (capacity, iteration bound) ends this query's refinement
        record(i, beta[i], MPAP_REFINE_ERROR, -1, r.status);
        continue;
      }
      const int64_t nb = mpap::refine_next(bounds[i], beta[i], outcome, r.cost);
      if (nb >= 0) {
        beta[i] = nb;
        next.push_back(i);
      }
    }
    active.swap(next);
  }
  return MPAP_OK;
}

}  // extern "C"

extern "C" {

int32_t mpap_surrogate_screen(mpap_mlp* net, mpap_roadmap* const* rms, uint32_t nq, const uint32_t* cand_ptr,
                              const uint32_t* path_ptr, const uint32_t* path, const float* feat,
                              const mpap_mc_params* mcs, double eps, float tau, int32_t use_net,
                              uint32_t max_calls, int32_t* chosen, uint32_t* mc_calls, uint32_t* rounds,
                              float* p_fail, void* stream) {
  if (nq && (!rms || !cand_ptr || !path_ptr || !path || !mcs || !chosen || !mc_calls)) {
    mpap::set_error("surrogate_screen: null argument");
    return MPAP_ERR_INVALID_ARG;
  }
  if (use_net && !net) {
    mpap::set_error("surrogate_screen: use_net needs a network");
    return MPAP_ERR_INVALID_ARG;
  }
  const cudaStream_t st = S(stream);
  const uint32_t total = nq ? cand_ptr[nq] - cand_ptr[0] : 0u;
  for (uint32_t i = 0; i < nq; ++i) {
    if (cand_ptr[i + 1] < cand_ptr[i] || !rms[i]) {
      mpap::set_error("surrogate_screen: cand_ptr must not decrease and every roadmap must be set");
      return MPAP_ERR_INVALID_ARG;
    }
    chosen[i] = -1;
    mc_calls[i] = 0;
  }
  if (rounds) *rounds = 0;
  for (uint32_t c = cand_ptr[0]; c < cand_ptr[0] + total; ++c)
    if (path_ptr[c + 1] < path_ptr[c] + 2) {
      mpap::set_error("surrogate_screen: candidate %u has fewer than 2 nodes", c);
      return MPAP_ERR_INVALID_ARG;
    }
  // predicted any-failure probability of every candidate (one batched feature
  // launch when the caller gives none, forward passes of max_batch rows)
  std::vector<float> pf(total, 0.0f);
  if (use_net && total) {
    std::vector<float> fbuf;
    const float* X = feat;
    if (!X) {
      fbuf.resize((size_t)total * MPAP_FEATURES);
      const int32_t rc = mpap::plan_features_batch_impl(rms, nq, cand_ptr, path_ptr, path, fbuf.data(), st);
      if (rc) return rc;
      X = fbuf.data();
    }
    const uint32_t mb = mpap::mlp_max_batch(net);
    std::vector<float> prob((size_t)total * 2);
    for (uint32_t o = 0; o < total; o += mb) {
      const uint32_t k = std::min(mb, total - o);
      const int32_t rc = mpap::mlp_forward(net, X + (size_t)o * MPAP_FEATURES, k, prob.data() + (size_t)o * 2,
                                           MPAP_MEM_HOST, st);
      if (rc) return rc;
    }
    for (uint32_t c = 0; c < total; ++c) {
      const float q = (1.0f - prob[2 * c]) * (1.0f - prob[2 * c + 1]);
      pf[c] = 1.0f - q;
    }
  }
  if (p_fail)
    for (uint32_t c = 0; c < total; ++c) p_fail[c] = pf[c];
  // order per query: predicted passes first, then the rest, each in index order
  std::vector<std::vector<uint32_t>> order(nq);
  for (uint32_t i = 0; i < nq; ++i) {
    const uint32_t b = cand_ptr[i] - cand_ptr[0], e = cand_ptr[i + 1] - cand_ptr[0];
    for (uint32_t c = b; c < e; ++c)
      if (!use_net || pf[c] <= tau) order[i].push_back(c - b);
    if (use_net)
      for (uint32_t c = b; c < e; ++c)
        if (pf[c] > tau) order[i].push_back(c - b);
  }
  // lock-step rounds: one batched certification of every unresolved query's next candidate
  std::vector<uint32_t> live;
  for (uint32_t i = 0; i < nq; ++i)
    if (!order[i].empty()) live.push_back(i);
  uint32_t nr = 0;
  for (uint32_t t = 0; !live.empty(); ++t) {
    std::vector<uint32_t> batch;
    for (uint32_t i : live)
      if (t < order[i].size() && (max_calls == 0 || t < max_calls)) batch.push_back(i);
    if (batch.empty()) break;
    std::vector<mpap_roadmap*> c_rm;
    std::vector<const uint32_t*> c_path;
    std::vector<uint32_t> c_len;
    std::vector<mpap_mc_params> c_mc;
    for (uint32_t i : batch) {
      const uint32_t j = order[i][t];
      const uint32_t c = cand_ptr[i] + j;
      c_rm.push_back(rms[i]);
      c_path.push_back(path + path_ptr[c]);
      c_len.push_back(path_ptr[c + 1] - path_ptr[c]);
      mpap_mc_params m = mcs[i];
      m.call_id = mcs[i].call_id + j;
      c_mc.push_back(m);
    }
    std::vector<mpap_cert> certs(batch.size());
    const int32_t rc = mpap::certify_batch_impl(c_rm.data(), c_path.data(), c_len.data(), c_mc.data(),
                                                (uint32_t)batch.size(), certs.data(), st);
    if (rc) return rc;
    ++nr;
    std::vector<char> done(nq, 0);
    for (size_t k = 0; k < batch.size(); ++k) {
      const uint32_t i = batch[k];
      mc_calls[i] += 1;
      if ((double)certs[k].hits_any <= eps * (double)certs[k].rollouts) {
        chosen[i] = (int32_t)order[i][t];
        done[i] = 1;
      }
    }
    std::vector<uint32_t> still;
    for (uint32_t i : live)
      if (!done[i] && t + 1 < order[i].size()) still.push_back(i);
    live.swap(still);
  }
  if (rounds) *rounds = nr;
  return MPAP_OK;
}

}  // extern "C"
