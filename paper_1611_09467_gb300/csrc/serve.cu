// Continuous-batching serving loop for evaluation requests (host C++).
//
// Each lane's worker sizes its persistent grids to 1/nlanes of the GPU, so
// the kernels of concurrent requests run side by side.
// A request asks for ln|psi|, E_loc and/or Delta of a batch of configurations
// of one model (a context: lattice, D, Dc, tensors).  The server runs
// requests on `nlanes` lanes, each a CUDA stream with worker contexts (the
// model's buffers, private workspaces), so requests of different models and
// sizes overlap on the GPU.  A lane keeps one worker per model it
// has served (least recently used first), so switching models does not
// rebuild workspaces; idle workers are freed only when the budget requires.
// Requests wait in a queue until a lane is free and the HBM they need fits
// under the budget (footprint admission); a request that does not fit lets
// smaller queued ones pass.  Queued requests are admitted first come first
// served, or (peps_server_set_policy) by expected run time less the time
// they have waited: the expected run time is the request's configurations
// times its model's milliseconds per configuration, a running average over
// the model's finished launches.  Completion is
// observed through one event per lane; the latency of a request runs from
// submission to the poll that sees its event.  Results do not depend on the
// lane or on what else runs: every configuration is evaluated by the same
// kernels in the same order.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <deque>
#include <string>
#include <thread>
#include <vector>

#include "../../include/peps.h"
#include "kernels.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  long long id;
  peps_ctx* model;
  const uint64_t* S;
  int n;
  double* logabs;
  int8_t* sign;
  double* eloc;
  void* O;
  int32_t* status;
  Clock::time_point submitted;
  // chain requests: Metropolis sweeps on S (resident, updated in place) first
  uint64_t* S_mut = nullptr;
  int nsweeps = 0;
  uint64_t seed = 0, chain0 = 0, sweep0 = 0;
};

struct Worker {
  peps_ctx* model;
  peps_ctx* ctx;
  const uint64_t* last_S;   // configurations whose environments its cache holds
};

struct Lane {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  bool busy = false;
  std::vector<Request> reqs;   // the request, or the requests packed into one launch
  Clock::time_point launched;  // when its launch was issued
  int launched_n = 0;          // configurations in it
  // worker contexts of this lane, one per model, least recently used first
  std::vector<Worker> workers;
  peps_packer* packer = nullptr;
};

}  // namespace

struct peps_server {
  std::vector<Lane> lanes;
  std::deque<Request> queue;
  size_t budget = 0;
  double lane_gb = 0;
  long long next_id = 1;
  long long submitted = 0, completed = 0;
  std::vector<double> latency_ms;
  std::deque<std::pair<long long, double>> finished;   // retired, not yet reported by poll
  size_t peak_bytes = 0;
  int pack_max = 0, pack_width = 1;   // packing of small requests (peps_server_set_packing)
  int policy = 0;                     // 0 first come first served, 1 by expected run time less wait
  std::vector<std::pair<const peps_ctx*, double>> cost;   // per model: ms per configuration
};

namespace {

size_t in_use(const peps_server* s) {
  size_t b = 0;
  for (const Lane& l : s->lanes)
    for (const auto& w : l.workers) b += peps::ctx_workspace_bytes(w.ctx);
  return b;
}

int find_worker(const Lane& l, const peps_ctx* model) {
  for (size_t k = 0; k < l.workers.size(); ++k)
    if (l.workers[k].model == model) return (int)k;
  return -1;
}

// Bytes a lane would add to run request r (workspace growth, or a new worker).
size_t extra_bytes(const peps_server* s, const Lane& l, const Request& r) {
  const size_t need = peps::ctx_footprint(r.model, r.n, s->lane_gb, (int)s->lanes.size());
  const int k = find_worker(l, r.model);
  if (k >= 0) {
    const size_t have = peps::ctx_workspace_bytes(l.workers[k].ctx);
    return need > have ? need - have : 0;
  }
  return need;
}

// Frees least recently used workers of idle lanes (never `keep`) until
// `extra` more bytes fit under the budget; returns whether they do.  Freeing
// device memory synchronises the device, so this only runs when the budget
// requires it.
bool make_room(peps_server* s, size_t extra, const peps_ctx* keep) {
  while (in_use(s) + extra > s->budget) {
    Lane* victim_lane = nullptr;
    for (Lane& l : s->lanes) {
      if (l.busy) continue;
      for (const auto& w : l.workers)
        if (w.ctx != keep) {
          victim_lane = &l;
          break;
        }
      if (victim_lane) break;
    }
    if (!victim_lane) return false;
    for (auto it = victim_lane->workers.begin(); it != victim_lane->workers.end(); ++it)
      if (it->ctx != keep) {
        cudaStreamSynchronize(victim_lane->stream);
        peps_destroy(it->ctx);
        victim_lane->workers.erase(it);
        break;
      }
  }
  return true;
}

// The lane's worker of a model (created on first use; most recently used last).
peps_ctx* worker_for(peps_server* s, Lane& l, peps_ctx* model, Worker** wout) {
  int k = find_worker(l, model);
  if (k < 0) {
    peps_ctx* w = peps::ctx_clone(model, l.stream, s->lane_gb, (int)s->lanes.size());
    if (!w) return nullptr;
    peps_set_env_cache(w, 1);
    l.workers.push_back({model, w, nullptr});
    k = (int)l.workers.size() - 1;
  } else if (k != (int)l.workers.size() - 1) {
    const Worker w = l.workers[k];
    l.workers.erase(l.workers.begin() + k);
    l.workers.push_back(w);
    k = (int)l.workers.size() - 1;
  }
  *wout = &l.workers[k];
  return l.workers[k].ctx;
}

peps_status launch(peps_server* s, Lane& l, const Request& r) {
  Worker* wk = nullptr;
  peps_ctx* worker = worker_for(s, l, r.model, &wk);
  if (!worker) return PEPS_ENOMEM;
  if (r.nsweeps > 0) {
    const peps_status st = peps_mc_sweep(worker, r.S_mut, r.n, r.nsweeps, r.seed, r.chain0, r.sweep0, nullptr);
    if (st != PEPS_OK) return st;
  }
  const peps_status st = peps_evaluate(worker, r.S, r.n, r.logabs, r.sign, r.eloc, r.O, r.status);
  if (st != PEPS_OK) return st;
  wk->last_S = r.S;
  if (cudaEventRecord(l.done, l.stream) != cudaSuccess) return PEPS_ECUDA;
  l.busy = true;
  l.reqs.assign(1, r);
  l.launched = Clock::now();
  l.launched_n = r.n;
  s->peak_bytes = std::max(s->peak_bytes, in_use(s));
  return PEPS_OK;
}

// Several small requests of distinct models (one precision class) in one
// packed launch on the lane: their boundary sweeps share one kernel.
peps_status launch_packed(peps_server* s, Lane& l, const std::vector<Request>& rs) {
  if (!l.packer) {
    const peps_status st = peps_packer_create(l.stream, &l.packer);
    if (st != PEPS_OK) return st;
  }
  const int k = (int)rs.size();
  std::vector<peps_ctx*> ctxs(k);
  std::vector<const uint64_t*> S(k);
  std::vector<int> n(k);
  std::vector<double*> la(k), el(k);
  std::vector<int8_t*> sg(k);
  std::vector<void*> O(k);
  std::vector<int32_t*> st(k);
  for (int i = 0; i < k; ++i) {
    Worker* wk = nullptr;
    ctxs[i] = worker_for(s, l, rs[i].model, &wk);
    if (!ctxs[i]) return PEPS_ENOMEM;
    wk->last_S = nullptr;   // the packed launch bypasses the worker's cache
    S[i] = rs[i].S;
    n[i] = rs[i].n;
    la[i] = rs[i].logabs;
    sg[i] = rs[i].sign;
    el[i] = rs[i].eloc;
    O[i] = rs[i].O;
    st[i] = rs[i].status;
  }
  const peps_status r = peps_packer_evaluate(l.packer, k, ctxs.data(), S.data(), n.data(), la.data(), sg.data(),
                                             el.data(), O.data(), st.data());
  if (r != PEPS_OK) return r;
  if (cudaEventRecord(l.done, l.stream) != cudaSuccess) return PEPS_ECUDA;
  l.busy = true;
  l.reqs = rs;
  l.launched = Clock::now();
  l.launched_n = 0;
  for (const Request& r : rs) l.launched_n += r.n;
  s->peak_bytes = std::max(s->peak_bytes, in_use(s));
  return PEPS_OK;
}

// Expected run time of a request: its configurations times its model's
// running average of milliseconds per configuration (0 before the model's
// first finished launch, so a new model goes first).
double expected_ms(const peps_server* s, const Request& r) {
  for (const auto& c : s->cost)
    if (c.first == r.model) return c.second * r.n;
  return 0.0;
}

// Folds a finished launch into its models' averages: milliseconds from issue
// to the poll that saw it finish, per configuration of the launch.
void record_cost(peps_server* s, const Lane& l) {
  if (l.launched_n < 1) return;
  const double per = std::chrono::duration<double, std::milli>(Clock::now() - l.launched).count() / l.launched_n;
  for (const Request& r : l.reqs) {
    bool found = false;
    for (auto& c : s->cost)
      if (c.first == r.model) {
        c.second = 0.5 * c.second + 0.5 * per;
        found = true;
      }
    if (!found) s->cost.emplace_back(r.model, per);
  }
}

bool packable(const peps_server* s, const Request& r) {
  return s->pack_max > 0 && r.nsweeps == 0 && r.n <= s->pack_max;
}

// Retires finished lanes, then admits queued requests that fit.
peps_status step(peps_server* s) {
  for (Lane& l : s->lanes) {
    if (!l.busy) continue;
    const cudaError_t q = cudaEventQuery(l.done);
    if (q == cudaErrorNotReady) continue;
    if (q != cudaSuccess) return PEPS_ECUDA;
    l.busy = false;
    record_cost(s, l);
    for (const Request& r : l.reqs) {
      const double ms = std::chrono::duration<double, std::milli>(Clock::now() - r.submitted).count();
      s->completed += 1;
      s->latency_ms.push_back(ms);
      s->finished.emplace_back(r.id, ms);
    }
    l.reqs.clear();
  }
  for (;;) {
    bool any_free = false;
    for (const Lane& l : s->lanes) any_free = any_free || !l.busy;
    if (!any_free || s->queue.empty()) break;
    // candidates in admission order
    std::vector<size_t> order(s->queue.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    if (s->policy == 1) {
      const auto now = Clock::now();
      std::vector<double> key(order.size());
      for (size_t i = 0; i < order.size(); ++i)
        key[i] = expected_ms(s, s->queue[i]) -
                 std::chrono::duration<double, std::milli>(now - s->queue[i].submitted).count();
      std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return key[x] < key[y]; });
    }
    bool admitted = false;
    for (size_t oi : order) {
      auto it = s->queue.begin() + (std::ptrdiff_t)oi;
      Lane* free_lane = nullptr;
      // prefer a free lane whose worker of this model last held these
      // configurations (its environment cache), then one with a worker of the model
      auto score = [&](const Lane& l) {
        const int k = find_worker(l, it->model);
        if (k < 0) return 0;
        return l.workers[k].last_S == it->S ? 2 : 1;
      };
      for (Lane& l : s->lanes)
        if (!l.busy && (!free_lane || score(l) > score(*free_lane))) free_lane = &l;
      const size_t extra = extra_bytes(s, *free_lane, *it);
      const int k = find_worker(*free_lane, it->model);
      if (!make_room(s, extra, k >= 0 ? free_lane->workers[k].ctx : nullptr))
        continue;   // does not fit now: let a smaller queued request pass
      // co-admit other small queued requests of distinct models and the same
      // precision class into one packed launch (first come first served: only
      // requests behind this one)
      std::vector<std::deque<Request>::iterator> group;
      if (packable(s, *it)) {
        group.push_back(it);
        size_t grown = extra;
        for (auto jt = s->queue.begin(); jt != s->queue.end() && (int)group.size() < s->pack_width; ++jt) {
          if (jt == it || (s->policy == 0 && jt < it)) continue;
          if (!packable(s, *jt) || peps::ctx_is_fp64(jt->model) != peps::ctx_is_fp64(it->model)) continue;
          bool dup = false;
          for (auto& g : group) dup = dup || g->model == jt->model;
          if (dup) continue;
          const size_t e2 = extra_bytes(s, *free_lane, *jt);
          if (in_use(s) + grown + e2 > s->budget) continue;
          grown += e2;
          group.push_back(jt);
        }
      }
      peps_status st;
      if (group.size() > 1) {
        std::vector<Request> rs;
        for (auto& g : group) rs.push_back(*g);
        st = launch_packed(s, *free_lane, rs);
      } else {
        st = launch(s, *free_lane, *it);
        group.assign(1, it);
      }
      if (st != PEPS_OK) {
        // The request cannot run (its workspace does not fit in device memory,
        // or a launch failed).  It is retired as failed, with a negative
        // latency, so that the queue keeps moving; peps_last_error holds why.
        for (auto& g : group) s->finished.emplace_back(g->id, -1.0);
      }
      // remove the group from the queue (erasing inside a deque invalidates
      // its iterators, so the candidates are ordered again; every admission
      // occupies a lane, so this ends once the lanes are busy or nothing
      // more fits)
      std::vector<long long> ids;
      for (auto& g : group) ids.push_back(g->id);
      s->queue.erase(std::remove_if(s->queue.begin(), s->queue.end(),
                                    [&](const Request& q) {
                                      return std::find(ids.begin(), ids.end(), q.id) != ids.end();
                                    }),
                     s->queue.end());
      admitted = true;
      break;
    }
    if (!admitted) break;
  }
  return PEPS_OK;
}

double percentile(std::vector<double> v, double p) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double x = p / 100.0 * (double)(v.size() - 1);
  const size_t i = (size_t)std::floor(x);
  const size_t j = std::min(i + 1, v.size() - 1);
  return v[i] + (x - (double)i) * (v[j] - v[i]);
}

}  // namespace

extern "C" {

peps_status peps_server_create(int nlanes, double hbm_budget_gb, peps_server** out) {
  if (!out || nlanes < 1 || nlanes > 64 || !(hbm_budget_gb > 0)) {
    peps::set_last_error("need 1 <= nlanes <= 64, a positive budget and an output pointer");
    return PEPS_EINVAL;
  }
  peps_server* s = new peps_server();
  s->budget = (size_t)(hbm_budget_gb * 1e9);
  s->lane_gb = hbm_budget_gb / nlanes;
  s->lanes.resize(nlanes);
  for (Lane& l : s->lanes) {
    if (cudaStreamCreateWithFlags(&l.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&l.done, cudaEventDisableTiming) != cudaSuccess) {
      peps_server_destroy(s);
      peps::set_last_error("stream or event creation failed");
      return PEPS_ECUDA;
    }
  }
  *out = s;
  return PEPS_OK;
}

peps_status peps_server_destroy(peps_server* s) {
  if (!s) return PEPS_OK;
  for (Lane& l : s->lanes) {
    if (l.stream) cudaStreamSynchronize(l.stream);
    for (auto& w : l.workers) peps_destroy(w.ctx);
    l.workers.clear();
    if (l.packer) peps_packer_destroy(l.packer);
    if (l.done) cudaEventDestroy(l.done);
    if (l.stream) cudaStreamDestroy(l.stream);
  }
  delete s;
  return PEPS_OK;
}

peps_status peps_server_submit(peps_server* s, peps_ctx* model, const uint64_t* S_dev, int n, double* logabs_dev,
                               int8_t* sign_dev, double* eloc_dev, void* O_dev, int32_t* status_dev,
                               long long* id_out) {
  if (!s || !model || n < 1 || !S_dev) {
    peps::set_last_error("bad request");
    return PEPS_EINVAL;
  }
  Request r{s->next_id++, model, S_dev, n, logabs_dev, sign_dev, eloc_dev, O_dev, status_dev, Clock::now()};
  s->queue.push_back(r);
  s->submitted += 1;
  if (id_out) *id_out = r.id;
  return step(s);
}

peps_status peps_server_submit_chain(peps_server* s, peps_ctx* model, uint64_t* S_dev, int n, int nsweeps,
                                     uint64_t seed, uint64_t chain0, uint64_t sweep0, double* logabs_dev,
                                     int8_t* sign_dev, double* eloc_dev, void* O_dev, int32_t* status_dev,
                                     long long* id_out) {
  if (!s || !model || n < 1 || !S_dev || nsweeps < 0) {
    peps::set_last_error("bad chain request");
    return PEPS_EINVAL;
  }
  Request r{s->next_id++, model, S_dev, n, logabs_dev, sign_dev, eloc_dev, O_dev, status_dev, Clock::now()};
  r.S_mut = S_dev;
  r.nsweeps = nsweeps;
  r.seed = seed;
  r.chain0 = chain0;
  r.sweep0 = sweep0;
  s->queue.push_back(r);
  s->submitted += 1;
  if (id_out) *id_out = r.id;
  return step(s);
}

peps_status peps_server_set_packing(peps_server* s, int max_configs, int max_requests) {
  if (!s || max_configs < 0 || max_requests < 1 || max_requests > 64) {
    peps::set_last_error("need max_configs >= 0 and 1 <= max_requests <= 64");
    return PEPS_EINVAL;
  }
  s->pack_max = max_configs;
  s->pack_width = max_requests;
  return PEPS_OK;
}

peps_status peps_server_set_policy(peps_server* s, int policy) {
  if (!s || policy < 0 || policy > 1) {
    peps::set_last_error("policy is 0 (first come first served) or 1 (expected run time less wait)");
    return PEPS_EINVAL;
  }
  s->policy = policy;
  return PEPS_OK;
}

peps_status peps_server_poll(peps_server* s, int wait, long long* ids, double* latency_ms, int max, int* ndone) {
  if (!s || !ndone) {
    peps::set_last_error("bad argument");
    return PEPS_EINVAL;
  }
  *ndone = 0;
  for (;;) {
    const peps_status st = step(s);
    if (st != PEPS_OK) return st;
    while (!s->finished.empty() && *ndone < max) {
      if (ids) ids[*ndone] = s->finished.front().first;
      if (latency_ms) latency_ms[*ndone] = s->finished.front().second;
      s->finished.pop_front();
      *ndone += 1;
    }
    bool running = false;
    for (const Lane& l : s->lanes) running = running || l.busy;
    if (!wait || *ndone > 0 || (!running && s->queue.empty())) return PEPS_OK;
    if (!running && !s->queue.empty()) {
      peps::set_last_error("queued requests exceed the HBM budget even with every lane idle");
      return PEPS_ENOMEM;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

peps_status peps_server_stats(peps_server* s, double* stats) {
  if (!s || !stats) {
    peps::set_last_error("bad argument");
    return PEPS_EINVAL;
  }
  int running = 0;
  for (const Lane& l : s->lanes) running += l.busy ? 1 : 0;
  stats[0] = (double)s->submitted;
  stats[1] = (double)s->completed;
  stats[2] = (double)s->queue.size();
  stats[3] = (double)running;
  stats[4] = percentile(s->latency_ms, 50.0);
  stats[5] = percentile(s->latency_ms, 99.0);
  stats[6] = (double)in_use(s) / 1e9;
  stats[7] = (double)s->peak_bytes / 1e9;
  return PEPS_OK;
}

}  // extern "C"
