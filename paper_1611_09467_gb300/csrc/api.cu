// C ABI of libpeps.so: context, workspace, batching into chunks, launches.
#include <algorithm>
#include <functional>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/peps.h"
#include "device.cuh"
#include "kernels.h"

using namespace peps;

namespace {

thread_local std::string g_err;

peps_status fail(peps_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

peps_status cuda_fail(cudaError_t e, const char* where) {
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? PEPS_ENOMEM : PEPS_ECUDA;
}

}  // namespace

namespace peps {
void set_last_error(const char* msg) { g_err = msg ? msg : ""; }
}  // namespace peps

namespace {

#define PEPS_CUDA(call)                                  \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t b) {
    if (b <= bytes) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    cudaError_t e = cudaMalloc(&p, b);
    if (e == cudaSuccess) bytes = b;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
};

// Bond dimensions of the boundary MPS after each absorbed row, per sweep
// (0 = top-down, 1 = bottom-up), with K = min(Dc, rows, cols) at every cut.
void bond_dims(int Lx, int Ly, int D, int Dc, std::vector<int>& bd) {
  bd.assign((size_t)2 * Ly * (Lx + 1), 1);
  for (int dir = 0; dir < 2; ++dir) {
    std::vector<int> b(Lx + 1, 1);
    for (int j = 0; j < Ly; ++j) {
      const int r = dir == 0 ? j : Ly - 1 - j;
      const bool lr = (j % 2) == 0;
      std::vector<int> nb(Lx + 1, 1);
      auto outdim = [&](int rr) { return dir == 0 ? (rr == Ly - 1 ? 1 : D) : (rr == 0 ? 1 : D); };
      int k = 1;
      if (lr) {
        for (int c = 0; c < Lx; ++c) {
          const int o = outdim(r), rd = c == Lx - 1 ? 1 : D;
          const int m = k * o, n = b[c + 1] * rd;
          if (c < Lx - 1) {
            const int K = std::min(Dc, std::min(m, n));
            nb[c + 1] = K;
            k = K;
          }
        }
      } else {
        for (int c = Lx - 1; c >= 0; --c) {
          const int o = outdim(r), ld = c == 0 ? 1 : D;
          const int m = o * k, n = b[c] * ld;
          if (c > 0) {
            const int K = std::min(Dc, std::min(m, n));
            nb[c] = K;
            k = K;
          }
        }
      }
      std::copy(nb.begin(), nb.end(), bd.begin() + ((size_t)dir * Ly + j) * (Lx + 1));
      b = nb;
    }
  }
}

}  // namespace

struct peps_ctx {
  peps_params p;
  Geometry g;
  cudaStream_t stream = nullptr;
  int nsm = 0;
  int nslots = 0;
  size_t elem = 8;
  bool wm_smem = false;
  DevBuf A, A64, triv_mps, triv_t1, triv_t2, bd, tcB;   // the model: shared by clones
  peps_ctx* parent = nullptr;                        // set on clones (model buffers borrowed)
  DevBuf env, small, O, scratch, gsum, go;
  int chunk = 0;  // configurations per pass
  int res_boundary = 0, res_row = 0, res_pair = 0, res_mc = 0;  // resident CTAs per kernel
  bool pair_tc = false;  // two-row step on the tensor cores (PEPS_MIXED_TF32, D = 8, Dc = 16)
  // kernel variants (peps_autotune): row_generic 1 takes the generic single-row
  // kernel; pair_mode 0 the default two-row kernel (tensor cores where
  // pair_tc, else fused where one exists), 1 the fused SIMT kernel, 2 the generic one
  int row_generic = 0, pair_mode = 0;
  int boundary_ctas = 0;   // 0: the boundary kernel's resident CTA count, else this many (peps_autotune)
  DevBuf corr_sites, corr_x, corr_scratch;   // correlation functions (peps_correlations)
  // environment cache (peps_set_env_cache): the bits of the configurations
  // whose boundary sweeps are in env, and per configuration which sweeps are
  bool env_cache = false, cache_dirty = true;
  DevBuf Scache, cbits;
  unsigned long long tensor_gen = 0, env_gen = 0, cache_key = ~0ull;
  // CUDA-graph replay (peps_set_graphs): one instantiated graph per call signature
  bool graphs = false, capturing = false;
  struct GraphEntry {
    int op;
    const void* S;
    int n;
    const void* out[6];
    unsigned long long gen;
    cudaGraphExec_t exec;
  };
  std::vector<GraphEntry> gcache;
  unsigned long long ws_gen = 0;   // bumped whenever a workspace buffer moves
  long long graph_captures = 0, graph_replays = 0;
  double* pinned = nullptr;        // 4 doubles of page-locked host memory for graph read-backs
  // profiling: event pairs per kernel id
  bool prof = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev;
  double ms[8] = {0};
  long long launches[8] = {0};
};

namespace {
// Brackets one launch with events when profiling is on; counts launches always.
struct Prof {
  peps_ctx* c;
  int id;
  cudaEvent_t a = nullptr, b = nullptr;
  Prof(peps_ctx* c_, int id_) : c(c_), id(id_) {
    c->launches[id] += 1;
    if (c->prof && !c->capturing) {
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      cudaEventRecord(a, c->stream);
    }
  }
  ~Prof() {
    if (c->prof && !c->capturing) {
      cudaEventRecord(b, c->stream);
      c->ev.push_back({id, {a, b}});
    }
  }
};
}  // namespace

namespace {

// FP64 master copy of the site tensors: the context's A itself on the FP64
// path, a separate buffer otherwise.
double* master_tensors(peps_ctx* c) { return c->elem == 8 ? (double*)c->A.p : (double*)c->A64.p; }

// The working copies derived on the device from the FP64 master: the FP32
// tensors and, on the tensor-core path, the pre-arranged TF32 B tiles.
peps_status refresh_working_copies(peps_ctx* c) {
  ++c->tensor_gen;   // cached environments belong to the old tensors
  const size_t D4 = (size_t)c->g.D * c->g.D * c->g.D * c->g.D;
  const size_t nel = (size_t)c->g.N * 2 * D4;
  if (c->elem == 4) {
    PEPS_CUDA(c->A.ensure(nel * sizeof(float)));
    PEPS_CUDA(launch_to_f32((const double*)c->A64.p, (float*)c->A.p, nel, c->nsm, c->stream));
  }
  if (c->pair_tc) {
    PEPS_CUDA(c->tcB.ensure((size_t)2 * c->g.N * 2 * 2 * kTcTile * sizeof(float)));
    PEPS_CUDA(launch_tc_tiles(master_tensors(c), (float*)c->tcB.p, c->g.N, c->nsm, c->stream));
  }
  return PEPS_OK;
}

peps_status upload_tensors(peps_ctx* c, const double* A_host) {
  const size_t D4 = (size_t)c->g.D * c->g.D * c->g.D * c->g.D;
  const size_t bytes = (size_t)c->g.N * 2 * D4 * sizeof(double);
  DevBuf& m = c->elem == 8 ? c->A : c->A64;
  PEPS_CUDA(m.ensure(bytes));
  PEPS_CUDA(cudaMemcpyAsync(m.p, A_host, bytes, cudaMemcpyHostToDevice, c->stream));
  peps_status st = refresh_working_copies(c);
  if (st != PEPS_OK) return st;
  PEPS_CUDA(cudaStreamSynchronize(c->stream));
  return PEPS_OK;
}

template <typename R>
peps_status setup_trivial(peps_ctx* c) {
  const Geometry& g = c->g;
  const size_t envT = (size_t)g.Dc * g.D * g.Dc, envT2 = envT * g.D;
  std::vector<R> m((size_t)g.Lx * envT, R(0)), t1(envT, R(0)), t2(envT2, R(0));
  for (int col = 0; col < g.Lx; ++col) m[(size_t)col * envT] = R(1);
  t1[0] = R(1);
  t2[0] = R(1);
  PEPS_CUDA(c->triv_mps.ensure(m.size() * sizeof(R)));
  PEPS_CUDA(c->triv_t1.ensure(t1.size() * sizeof(R)));
  PEPS_CUDA(c->triv_t2.ensure(t2.size() * sizeof(R)));
  PEPS_CUDA(cudaMemcpy(c->triv_mps.p, m.data(), m.size() * sizeof(R), cudaMemcpyHostToDevice));
  PEPS_CUDA(cudaMemcpy(c->triv_t1.p, t1.data(), t1.size() * sizeof(R), cudaMemcpyHostToDevice));
  PEPS_CUDA(cudaMemcpy(c->triv_t2.p, t2.data(), t2.size() * sizeof(R), cudaMemcpyHostToDevice));
  std::vector<int> bd;
  bond_dims(g.Lx, g.Ly, g.D, g.Dc, bd);
  PEPS_CUDA(c->bd.ensure(bd.size() * sizeof(int)));
  PEPS_CUDA(cudaMemcpy(c->bd.p, bd.data(), bd.size() * sizeof(int), cudaMemcpyHostToDevice));
  return PEPS_OK;
}

// Layout of the per-chunk "small" buffer (doubles unless noted).
struct Small {
  double* logabs;
  double* eloc;
  double* eloc_h;
  double* eloc_v;
  double* w_row;
  double* lnU;
  int* flags;
  int* status;
  int8_t* sign;
  static size_t bytes(int chunk, int Ly) {
    return (size_t)chunk * (2 + 4 * (size_t)Ly) * 8 + (size_t)chunk * 2 * 4 + (size_t)chunk + 256;
  }
  void carve(void* base, int chunk, int Ly) {
    char* p = (char*)base;
    logabs = (double*)p; p += (size_t)chunk * 8;
    eloc = (double*)p; p += (size_t)chunk * 8;
    eloc_h = (double*)p; p += (size_t)chunk * Ly * 8;
    eloc_v = (double*)p; p += (size_t)chunk * Ly * 8;
    w_row = (double*)p; p += (size_t)chunk * Ly * 8;
    lnU = (double*)p; p += (size_t)chunk * Ly * 8;
    flags = (int*)p; p += (size_t)chunk * 4;
    status = (int*)p; p += (size_t)chunk * 4;
    sign = (int8_t*)p;
  }
};

size_t env_bytes_per_cfg(const peps_ctx* c) {
  const Geometry& g = c->g;
  return 2 * (size_t)g.Ly * g.Lx * g.Dc * g.D * g.Dc * c->elem;
}

size_t slot_elems(const peps_ctx* c) {
  const Geometry& g = c->g;
  size_t s = boundary_slot_elems(g, c->wm_smem);
  s = std::max(s, row_slot_elems(g));
  s = std::max(s, pair_slot_elems(g));
  s = std::max(s, mc_slot_elems(g, c->wm_smem));
  return (s + 31) / 32 * 32;
}

peps_status ensure_workspace(peps_ctx* c, int n, bool want_O) {
  const Geometry& g = c->g;
  const double budget = (c->p.workspace_gb > 0 ? c->p.workspace_gb : 24.0) * 1e9;
  const size_t D4 = (size_t)g.D * g.D * g.D * g.D;
  size_t per_cfg = env_bytes_per_cfg(c) + (want_O ? (size_t)g.N * D4 * c->elem : 0);
  int chunk = (int)std::max<double>(1.0, std::floor(budget / (double)per_cfg));
  chunk = std::min(chunk, std::max(n, 1));
  c->chunk = chunk;
  const void* before[4] = {c->env.p, c->small.p, c->O.p, c->scratch.p};
  PEPS_CUDA(c->env.ensure(env_bytes_per_cfg(c) * chunk));
  PEPS_CUDA(c->small.ensure(Small::bytes(chunk, g.Ly)));
  if (want_O) PEPS_CUDA(c->O.ensure((size_t)chunk * g.N * D4 * c->elem));
  PEPS_CUDA(c->scratch.ensure(slot_elems(c) * c->elem * c->nslots));
  const void* after[4] = {c->env.p, c->small.p, c->O.p, c->scratch.p};
  for (int i = 0; i < 4; ++i)
    if (before[i] != after[i]) ++c->ws_gen;   // captured graphs that read the old buffers are stale
  if (before[0] != after[0] || before[1] != after[1]) ++c->env_gen;   // cached environments are gone
  return PEPS_OK;
}

template <typename R>
KArgs<R> make_args(peps_ctx* c, const uint64_t* S, int n, const Small& sm) {
  KArgs<R> a;
  const Geometry& g = c->g;
  a.g = g;
  a.cache = nullptr;
  a.A = (const R*)c->A.p;
  a.triv_mps = (const R*)c->triv_mps.p;
  a.triv_t1 = (const R*)c->triv_t1.p;
  a.triv_t2 = (const R*)c->triv_t2.p;
  a.bd = (const int*)c->bd.p;
  a.S = S;
  a.n = n;
  const size_t half = (size_t)c->chunk * g.Ly * g.Lx * g.Dc * g.D * g.Dc;
  a.envU = (R*)c->env.p;
  a.envL = (R*)c->env.p + half;
  a.logabs = sm.logabs;
  a.sign = sm.sign;
  a.flags = sm.flags;
  a.eloc_h = sm.eloc_h;
  a.eloc_v = sm.eloc_v;
  a.w_row = sm.w_row;
  a.lnU = sm.lnU;
  a.O = nullptr;
  a.scratch = (R*)c->scratch.p;
  a.slot_elems = slot_elems(c);
  a.smem_wm = c->wm_smem ? 1 : 0;
  a.tcB = (const float*)c->tcB.p;
  return a;
}

// Single-row and two-row sandwich steps and the E(S)/status finalisation of
// one chunk whose environments are in place, on stream st.
template <typename R>
peps_status sandwich_chunk(peps_ctx* c, const KArgs<R>& a, const uint64_t* S, int n, bool need_env_l,
                           bool need_pairs, Small& sm, cudaStream_t st) {
  int grid;
  if (need_env_l) {
    grid = std::min(n * c->g.Ly, std::min(c->nslots, c->res_row));
    Prof pf(c, 1);
    PEPS_CUDA(launch_row<R>(a, std::max(grid, 1), st, c->row_generic));
  }
  if (need_pairs && c->g.Ly > 1) {
    grid = std::min(n * (c->g.Ly - 1), std::min(c->nslots, c->res_pair));
    Prof pf(c, 2);
    if constexpr (sizeof(R) == 4) {
      if (c->pair_tc && c->pair_mode == 0) {
        PEPS_CUDA(launch_pair_tc(a, std::max(grid, 1), st));
      } else {
        PEPS_CUDA(launch_pair<R>(a, std::max(grid, 1), st, c->pair_mode == 2));
      }
    } else {
      PEPS_CUDA(launch_pair<R>(a, std::max(grid, 1), st, c->pair_mode == 2));
    }
  } else {
    PEPS_CUDA(cudaMemsetAsync(sm.eloc_v, 0, (size_t)n * c->g.Ly * sizeof(double), st));
  }
  if (!need_env_l) PEPS_CUDA(cudaMemsetAsync(sm.eloc_h, 0, (size_t)n * c->g.Ly * sizeof(double), st));
  {
    Prof pf(c, 3);
    PEPS_CUDA(launch_finalize(c->g, S, n, sm.eloc_h, sm.eloc_v, sm.flags, sm.eloc, sm.status, need_env_l ? 1 : 0,
                              st));
  }
  return PEPS_OK;
}

// Environment cache for a call whose batch is one chunk: configurations whose
// bits equal the cached copy keep their boundary sweeps (k_cache_check clears
// the bits of the others).  The cache is reset when the tensors, the
// workspace or the chunk size changed, or after a call that wrote the
// environments without it.
template <typename R>
peps_status prepare_cache(peps_ctx* c, const uint64_t* S, int n, bool whole_batch, KArgs<R>& a) {
  if (!c->env_cache || !whole_batch) {
    c->cache_dirty = true;
    return PEPS_OK;
  }
  const Geometry& g = c->g;
  const void* p0[2] = {c->Scache.p, c->cbits.p};
  PEPS_CUDA(c->Scache.ensure((size_t)c->chunk * g.nwords * sizeof(uint64_t)));
  PEPS_CUDA(c->cbits.ensure((size_t)c->chunk * sizeof(unsigned)));
  const unsigned long long key = (c->tensor_gen * 1000003ull + c->env_gen) * 1000003ull + (unsigned long long)c->chunk;
  if (c->cache_dirty || key != c->cache_key || p0[0] != c->Scache.p || p0[1] != c->cbits.p) {
    PEPS_CUDA(cudaMemsetAsync(c->cbits.p, 0, (size_t)c->chunk * sizeof(unsigned), c->stream));
    c->cache_dirty = false;
    c->cache_key = key;
  }
  PEPS_CUDA(launch_cache_check(S, (uint64_t*)c->Scache.p, (unsigned*)c->cbits.p, n, g.nwords, c->stream));
  a.cache = (unsigned*)c->cbits.p;
  return PEPS_OK;
}

template <typename R>
peps_status evaluate_chunk(peps_ctx* c, const uint64_t* S, int n, bool need_env_l, bool need_pairs, R* O,
                           Small& sm, bool whole_batch = false) {
  KArgs<R> a = make_args<R>(c, S, n, sm);
  a.O = O;
  peps_status cst = prepare_cache<R>(c, S, n, whole_batch, a);
  if (cst != PEPS_OK) return cst;
  PEPS_CUDA(cudaMemsetAsync(sm.flags, 0, (size_t)n * sizeof(int), c->stream));
  const int dirs = need_env_l ? 2 : 1;
  // persistent kernels: never more CTAs than can be resident at once
  const int res = c->boundary_ctas > 0 ? std::min(c->boundary_ctas, c->res_boundary) : c->res_boundary;
  int grid = std::min(n * dirs, std::min(c->nslots, res));
  {
    Prof pf(c, 0);
    PEPS_CUDA(launch_boundary<R>(a, dirs, std::max(grid, 1), c->stream));
  }
  return sandwich_chunk<R>(c, a, S, n, need_env_l, need_pairs, sm, c->stream);
}

peps_status check_ctx(peps_ctx* c, const void* S, int n) {
  if (!c) return fail(PEPS_EINVAL, "null context");
  if (n < 0) return fail(PEPS_EINVAL, "negative batch size");
  if (n > 0 && !S) return fail(PEPS_EINVAL, "null configuration pointer");
  return PEPS_OK;
}

template <typename R>
peps_status evaluate_impl(peps_ctx* c, const uint64_t* S, int n, double* logabs, int8_t* sign, double* eloc, R* O,
                          int32_t* status) {
  if (n == 0) return PEPS_OK;
  const bool want_e = eloc != nullptr, want_O = O != nullptr;
  const bool need_l = want_e || want_O;
  peps_status st = ensure_workspace(c, n, false);
  if (st != PEPS_OK) return st;
  Small sm;
  sm.carve(c->small.p, c->chunk, c->g.Ly);
  const Geometry& g = c->g;
  const size_t D4 = (size_t)g.D * g.D * g.D * g.D;
  for (int c0 = 0; c0 < n; c0 += c->chunk) {
    const int m = std::min(c->chunk, n - c0);
    const uint64_t* Sc = S + (size_t)c0 * g.nwords;
    st = evaluate_chunk<R>(c, Sc, m, need_l, want_e, want_O ? O + (size_t)c0 * g.N * D4 : nullptr, sm, m == n);
    if (st != PEPS_OK) return st;
    if (logabs) PEPS_CUDA(cudaMemcpyAsync(logabs + c0, sm.logabs, m * 8, cudaMemcpyDeviceToDevice, c->stream));
    if (sign) PEPS_CUDA(cudaMemcpyAsync(sign + c0, sm.sign, m, cudaMemcpyDeviceToDevice, c->stream));
    if (eloc) PEPS_CUDA(cudaMemcpyAsync(eloc + c0, sm.eloc, m * 8, cudaMemcpyDeviceToDevice, c->stream));
    if (status) PEPS_CUDA(cudaMemcpyAsync(status + c0, sm.status, m * 4, cudaMemcpyDeviceToDevice, c->stream));
  }
  return PEPS_OK;
}

// Layout of the gradient sums (doubles), also the public layout of
// peps_gradient_sums: [0] sum E, [1] count, [2] sum E^2, [3] zero, then
// sum O [N][2][D^4], then sum E*O [N][2][D^4].
constexpr size_t kSumsHead = 4;

size_t grad_total(const peps_ctx* c) {
  const Geometry& g = c->g;
  return (size_t)g.N * 2 * g.D * g.D * g.D * g.D;
}

template <typename R>
peps_status gradient_sums_impl(peps_ctx* c, const uint64_t* S, int n, double* sums, bool accumulate,
                               double* logabs, int8_t* sign, double* eloc, int32_t* status) {
  const Geometry& g = c->g;
  const size_t D4 = (size_t)g.D * g.D * g.D * g.D;
  const size_t total = grad_total(c);
  peps_status st = ensure_workspace(c, n, true);
  if (st != PEPS_OK) return st;
  double* sumO = sums + kSumsHead;
  double* sumEO = sumO + total;
  if (!accumulate) PEPS_CUDA(cudaMemsetAsync(sums, 0, (kSumsHead + 2 * total) * sizeof(double), c->stream));
  Small sm;
  sm.carve(c->small.p, c->chunk, g.Ly);
  for (int c0 = 0; c0 < n; c0 += c->chunk) {
    const int m = std::min(c->chunk, n - c0);
    const uint64_t* Sc = S + (size_t)c0 * g.nwords;
    st = evaluate_chunk<R>(c, Sc, m, true, true, (R*)c->O.p, sm, m == n);
    if (st != PEPS_OK) return st;
    GradArgs ga;
    ga.N = g.N;
    ga.D4 = (int)D4;
    ga.nwords = g.nwords;
    ga.n = m;
    ga.S = Sc;
    ga.eloc = sm.eloc;
    ga.status = sm.status;
    ga.sumO = sumO;
    ga.sumEO = sumEO;
    {
      Prof pf(c, 4);
      PEPS_CUDA(launch_grad_accum<R>(ga, (const R*)c->O.p, c->stream));
    }
    {
      Prof pf(c, 5);
      PEPS_CUDA(launch_sum_eloc(sm.eloc, sm.status, m, sums, c->stream));
    }
    if (logabs) PEPS_CUDA(cudaMemcpyAsync(logabs + c0, sm.logabs, m * 8, cudaMemcpyDeviceToDevice, c->stream));
    if (sign) PEPS_CUDA(cudaMemcpyAsync(sign + c0, sm.sign, m, cudaMemcpyDeviceToDevice, c->stream));
    if (eloc) PEPS_CUDA(cudaMemcpyAsync(eloc + c0, sm.eloc, m * 8, cudaMemcpyDeviceToDevice, c->stream));
    if (status) PEPS_CUDA(cudaMemcpyAsync(status + c0, sm.status, m * 4, cudaMemcpyDeviceToDevice, c->stream));
  }
  return PEPS_OK;
}

peps_status gradient_finalize_impl(peps_ctx* c, const double* sums, double* e_site, double* e_var, double* grad,
                                   double* cov, int* n_used) {
  const size_t total = grad_total(c);
  if (grad || cov) {
    Prof pf(c, 6);
    PEPS_CUDA(launch_grad_finalize((int)total, 0, sums, sums + kSumsHead, sums + kSumsHead + total, grad, cov,
                                   c->stream));
  }
  double h[3] = {0, 0, 0};
  PEPS_CUDA(cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  PEPS_CUDA(cudaStreamSynchronize(c->stream));
  const double N = c->g.N;
  if (e_site) *e_site = h[1] > 0 ? h[0] / h[1] / N : NAN;
  if (e_var) *e_var = h[1] > 1 ? (h[2] - h[0] * h[0] / h[1]) / (h[1] - 1) / (N * N) : NAN;
  if (n_used) *n_used = (int)h[1];
  return PEPS_OK;
}

template <typename R>
peps_status gradient_impl(peps_ctx* c, const uint64_t* S, int n, double* e_site, double* grad, double* cov,
                          double* logabs, int8_t* sign, double* eloc, int32_t* status, int* n_used) {
  const size_t total = grad_total(c);
  PEPS_CUDA(c->gsum.ensure((kSumsHead + 2 * total) * sizeof(double)));
  peps_status st = gradient_sums_impl<R>(c, S, n, (double*)c->gsum.p, false, logabs, sign, eloc, status);
  if (st != PEPS_OK) return st;
  return gradient_finalize_impl(c, (const double*)c->gsum.p, e_site, nullptr, grad, cov, n_used);
}

template <typename R>
peps_status mc_impl(peps_ctx* c, uint64_t* S, int n, int nsweeps, uint64_t seed, uint64_t chain0, uint64_t sweep0,
                    int64_t* accepted) {
  if (n == 0 || nsweeps == 0) return PEPS_OK;
  peps_status st = ensure_workspace(c, 1, false);
  if (st != PEPS_OK) return st;
  Small sm;
  sm.carve(c->small.p, c->chunk, c->g.Ly);
  KArgs<R> a = make_args<R>(c, S, n, sm);
  const int grid = std::min(n, std::min(c->nslots, c->res_mc));
  Prof pf(c, 7);
  PEPS_CUDA(launch_mc<R>(a, S, nsweeps, seed, chain0, sweep0, (long long*)accepted, std::max(grid, 1), c->stream));
  return PEPS_OK;
}

// ------------------------------------------------------------ CUDA graphs
void drop_graphs(peps_ctx* c) {
  for (auto& e : c->gcache) cudaGraphExecDestroy(e.exec);
  c->gcache.clear();
}

// Runs `enqueue` (work enqueued on the context's stream only, no host
// synchronisation) through an instantiated CUDA graph: the first call with a
// signature (op, S, n, outputs) and the current workspace captures and
// instantiates it, later calls replay it.  Graphs are dropped when the
// workspace buffers move (ws_gen).
template <typename F>
peps_status run_graphed(peps_ctx* c, int op, const void* S, int n, const void* const out[6], F enqueue) {
  for (auto& e : c->gcache) {
    bool same = e.op == op && e.S == S && e.n == n && e.gen == c->ws_gen;
    for (int i = 0; same && i < 6; ++i) same = e.out[i] == out[i];
    if (same) {
      PEPS_CUDA(cudaGraphLaunch(e.exec, c->stream));
      ++c->graph_replays;
      return PEPS_OK;
    }
  }
  cudaGraph_t graph = nullptr;
  PEPS_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  c->capturing = true;
  peps_status st = enqueue();
  c->capturing = false;
  cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
  if (st != PEPS_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  if (c->gcache.size() >= 16) {
    cudaGraphExecDestroy(c->gcache.front().exec);
    c->gcache.erase(c->gcache.begin());
  }
  peps_ctx::GraphEntry ge;
  ge.op = op;
  ge.S = S;
  ge.n = n;
  for (int i = 0; i < 6; ++i) ge.out[i] = out[i];
  ge.gen = c->ws_gen;
  ge.exec = exec;
  c->gcache.push_back(ge);
  ++c->graph_captures;
  PEPS_CUDA(cudaGraphLaunch(exec, c->stream));
  return PEPS_OK;
}

peps_status ensure_pinned(peps_ctx* c) {
  if (!c->pinned) PEPS_CUDA(cudaMallocHost((void**)&c->pinned, 4 * sizeof(double)));
  return PEPS_OK;
}

template <typename R>
peps_status gradient_graphed(peps_ctx* c, const uint64_t* S, int n, double* e_site, double* grad, double* cov,
                             double* logabs, int8_t* sign, double* eloc, int32_t* status, int* n_used) {
  const size_t total = grad_total(c);
  const void* g0 = c->gsum.p;
  PEPS_CUDA(c->gsum.ensure((kSumsHead + 2 * total) * sizeof(double)));
  if (c->gsum.p != g0) ++c->ws_gen;
  peps_status st = ensure_workspace(c, n, true);
  if (st == PEPS_OK) st = ensure_pinned(c);
  if (st != PEPS_OK) return st;
  const void* out[6] = {grad, cov, logabs, sign, eloc, status};
  double* sums = (double*)c->gsum.p;
  st = run_graphed(c, 1, S, n, out, [&]() -> peps_status {
    peps_status s2 = gradient_sums_impl<R>(c, S, n, sums, false, logabs, sign, eloc, status);
    if (s2 != PEPS_OK) return s2;
    if (grad || cov) {
      Prof pf(c, 6);
      PEPS_CUDA(launch_grad_finalize((int)total, 0, sums, sums + kSumsHead, sums + kSumsHead + total, grad, cov,
                                     c->stream));
    }
    PEPS_CUDA(cudaMemcpyAsync(c->pinned, sums, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return PEPS_OK;
  });
  if (st != PEPS_OK) return st;
  PEPS_CUDA(cudaStreamSynchronize(c->stream));
  const double* h = c->pinned;
  if (e_site) *e_site = h[1] > 0 ? h[0] / h[1] / c->g.N : NAN;
  if (n_used) *n_used = (int)h[1];
  return PEPS_OK;
}

// ------------------------------------------------------------ kernel variants
// Resident CTA counts for the chosen single- and two-row kernels.
void apply_variants(peps_ctx* c) {
  const Geometry& g = c->g;
  if (c->elem == 8) {
    c->res_row = max_blocks_row<double>(g, c->row_generic);
    const int fused = max_blocks_pair_fused<double>(g);
    c->res_pair = (c->pair_mode == 2 || !fused) ? max_blocks_pair<double>(g) : fused;
  } else {
    c->res_row = max_blocks_row<float>(g, c->row_generic);
    const int fused = max_blocks_pair_fused<float>(g);
    if (c->pair_tc && c->pair_mode == 0) c->res_pair = max_blocks_pair_tc();
    else c->res_pair = (c->pair_mode == 2 || !fused) ? max_blocks_pair<float>(g) : fused;
  }
  c->nslots = std::max(std::max(c->res_boundary, c->res_row), std::max(c->res_pair, c->res_mc));
}

struct TuneKey {
  int Lx, Ly, D, Dc, prec, nsm;
  bool operator==(const TuneKey& o) const {
    return Lx == o.Lx && Ly == o.Ly && D == o.D && Dc == o.Dc && prec == o.prec && nsm == o.nsm;
  }
};
struct TuneVal {
  int row_generic, pair_mode, boundary_ctas;
  double workspace_gb;
};
std::vector<std::pair<TuneKey, TuneVal>> g_tuned;   // choices of peps_autotune in this process
std::mutex g_tune_mu;

TuneKey tune_key(const peps_ctx* c) { return {c->g.Lx, c->g.Ly, c->g.D, c->g.Dc, c->p.prec, c->nsm}; }

// ------------------------------------------------------------ packed launches
template <typename R>
peps_status packed_impl(peps_packer* pk, int nreq, peps_ctx* const* ctxs, const uint64_t* const* S, const int* n,
                        double* const* logabs, int8_t* const* sign, double* const* eloc, void* const* O,
                        int32_t* const* status);

}  // namespace

struct peps_packer {
  cudaStream_t stream = nullptr;
  DevBuf scratch, models, start;
  int nsm = 0;
};

namespace {

template <typename R>
peps_status packed_impl(peps_packer* pk, int nreq, peps_ctx* const* ctxs, const uint64_t* const* S, const int* n,
                        double* const* logabs, int8_t* const* sign, double* const* eloc, void* const* O,
                        int32_t* const* status) {
  bool any_env = false;
  for (int i = 0; i < nreq; ++i) any_env = any_env || (eloc && eloc[i]) || (O && O[i]);
  const int dirs = any_env ? 2 : 1;
  std::vector<KArgs<R>> args(nreq);
  std::vector<Small> sms(nreq);
  std::vector<int> start(nreq + 1, 0);
  size_t slot = 0, smem = 0;
  for (int i = 0; i < nreq; ++i) {
    peps_ctx* c = ctxs[i];
    peps_status st = ensure_workspace(c, n[i], false);
    if (st != PEPS_OK) return st;
    if (n[i] > c->chunk)
      return fail(PEPS_EINVAL, "a packed request must fit in one chunk of its context's workspace");
    sms[i].carve(c->small.p, c->chunk, c->g.Ly);
    args[i] = make_args<R>(c, S[i], n[i], sms[i]);
    c->cache_dirty = true;   // the packed launch writes this context's environments without the cache
    args[i].O = (O && O[i]) ? (R*)O[i] : nullptr;
    PEPS_CUDA(cudaMemsetAsync(sms[i].flags, 0, (size_t)n[i] * sizeof(int), pk->stream));
    start[i + 1] = start[i] + n[i] * dirs;
    slot = std::max(slot, boundary_slot_elems(c->g, c->wm_smem));
    smem = std::max(smem, dyn_smem_bytes(c->g, sizeof(R), true, c->wm_smem));
  }
  slot = (slot + 31) / 32 * 32;
  const int total = start[nreq];
  const int grid = std::max(1, std::min(total, max_blocks_boundary_packed<R>(smem)));
  PEPS_CUDA(pk->scratch.ensure(slot * sizeof(R) * grid));
  PEPS_CUDA(pk->models.ensure(sizeof(KArgs<R>) * nreq));
  PEPS_CUDA(pk->start.ensure(sizeof(int) * (nreq + 1)));
  // pageable sources: the copies have taken the data when the calls return
  PEPS_CUDA(cudaMemcpyAsync(pk->models.p, args.data(), sizeof(KArgs<R>) * nreq, cudaMemcpyHostToDevice, pk->stream));
  PEPS_CUDA(cudaMemcpyAsync(pk->start.p, start.data(), sizeof(int) * (nreq + 1), cudaMemcpyHostToDevice, pk->stream));
  PEPS_CUDA(launch_boundary_packed<R>((const KArgs<R>*)pk->models.p, (const int*)pk->start.p, nreq, dirs,
                                      (R*)pk->scratch.p, slot, smem, grid, pk->stream));
  for (int i = 0; i < nreq; ++i) {
    peps_ctx* c = ctxs[i];
    const bool want_e = eloc && eloc[i], want_O = O && O[i];
    peps_status st = sandwich_chunk<R>(c, args[i], S[i], n[i], want_e || want_O, want_e, sms[i], pk->stream);
    if (st != PEPS_OK) return st;
    const int m = n[i];
    if (logabs && logabs[i])
      PEPS_CUDA(cudaMemcpyAsync(logabs[i], sms[i].logabs, m * 8, cudaMemcpyDeviceToDevice, pk->stream));
    if (sign && sign[i]) PEPS_CUDA(cudaMemcpyAsync(sign[i], sms[i].sign, m, cudaMemcpyDeviceToDevice, pk->stream));
    if (want_e) PEPS_CUDA(cudaMemcpyAsync(eloc[i], sms[i].eloc, m * 8, cudaMemcpyDeviceToDevice, pk->stream));
    if (status && status[i])
      PEPS_CUDA(cudaMemcpyAsync(status[i], sms[i].status, m * 4, cudaMemcpyDeviceToDevice, pk->stream));
  }
  return PEPS_OK;
}

// ------------------------------------------------------------ correlations
template <typename R>
peps_status correlations_impl(peps_ctx* c, const uint64_t* S, int n, const int* sites, int nc, double* m2,
                              double* corr, int32_t* status) {
  const Geometry& g = c->g;
  peps_status st = ensure_workspace(c, n, false);
  if (st != PEPS_OK) return st;
  std::vector<int> tab((size_t)nc + g.N, -1);
  for (int p = 0; p < nc; ++p) {
    tab[p] = sites[p];
    tab[(size_t)nc + sites[p]] = p;
  }
  PEPS_CUDA(c->corr_sites.ensure(tab.size() * sizeof(int)));
  PEPS_CUDA(cudaMemcpyAsync(c->corr_sites.p, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  PEPS_CUDA(c->corr_x.ensure((size_t)c->chunk * sizeof(double)));
  const int res = max_blocks_corr<R>(g);
  const size_t slot = (corr_slot_elems(g, c->wm_smem) + 31) / 32 * 32;
  PEPS_CUDA(c->corr_scratch.ensure(slot * c->elem * res));
  if (corr) PEPS_CUDA(cudaMemsetAsync(corr, 0, (size_t)nc * nc * sizeof(double), c->stream));
  CorrArgs ca;
  ca.sites = (const int*)c->corr_sites.p;
  ca.pos = (const int*)c->corr_sites.p + nc;
  ca.nc = nc;
  ca.xsum = (double*)c->corr_x.p;
  ca.corr = corr;
  ca.slot_elems = slot;
  Small sm;
  sm.carve(c->small.p, c->chunk, g.Ly);
  for (int c0 = 0; c0 < n; c0 += c->chunk) {
    const int m = std::min(c->chunk, n - c0);
    const uint64_t* Sc = S + (size_t)c0 * g.nwords;
    st = evaluate_chunk<R>(c, Sc, m, true, false, nullptr, sm, m == n);
    if (st != PEPS_OK) return st;
    KArgs<R> a = make_args<R>(c, Sc, m, sm);
    a.scratch = (R*)c->corr_scratch.p;
    ca.status = sm.status;
    PEPS_CUDA(cudaMemsetAsync(ca.xsum, 0, (size_t)m * sizeof(double), c->stream));
    const int grid = std::max(1, std::min(m * nc, res));
    PEPS_CUDA(launch_corr<R>(a, ca, grid, c->stream));
    PEPS_CUDA(launch_corr_finalize(g, ca, Sc, m, sm.status, m2 ? m2 + c0 : nullptr, c->stream));
    if (status) PEPS_CUDA(cudaMemcpyAsync(status + c0, sm.status, m * 4, cudaMemcpyDeviceToDevice, c->stream));
  }
  return PEPS_OK;
}

}  // namespace

namespace peps {

// A worker context: same model (tensors, tables) as `c`, its own stream and
// workspace with the given budget.  The model's device buffers are borrowed.
peps_ctx* ctx_clone(peps_ctx* c, cudaStream_t stream, double workspace_gb, int share) {
  peps_ctx* k = new peps_ctx();
  k->p = c->p;
  k->p.workspace_gb = workspace_gb;
  k->g = c->g;
  k->stream = stream;
  k->nsm = c->nsm;
  k->nslots = c->nslots;
  k->elem = c->elem;
  k->wm_smem = c->wm_smem;
  // a worker that shares the GPU with `share` lanes sizes its persistent grids to its part
  auto part = [&](int r) { return std::max(std::min(r, c->nsm), r / std::max(share, 1)); };
  k->res_boundary = part(c->res_boundary);
  k->res_row = part(c->res_row);
  k->res_pair = part(c->res_pair);
  k->res_mc = part(c->res_mc);
  k->nslots = std::max(std::max(k->res_boundary, k->res_row), std::max(k->res_pair, k->res_mc));
  k->pair_tc = c->pair_tc;
  k->parent = c->parent ? c->parent : c;
  auto borrow = [](DevBuf& dst, const DevBuf& src) {
    dst.p = src.p;
    dst.bytes = src.bytes;
  };
  borrow(k->A, c->A);
  borrow(k->A64, c->A64);
  borrow(k->triv_mps, c->triv_mps);
  borrow(k->triv_t1, c->triv_t1);
  borrow(k->triv_t2, c->triv_t2);
  borrow(k->bd, c->bd);
  borrow(k->tcB, c->tcB);
  return k;
}

// Device bytes an evaluation of n configurations needs in a context's
// workspace (environments of one chunk, per-chunk outputs, scratch slots).
size_t ctx_footprint(peps_ctx* c, int n, double workspace_gb, int share) {
  const double budget = (workspace_gb > 0 ? workspace_gb : 24.0) * 1e9;
  const size_t per = env_bytes_per_cfg(c);
  size_t chunk = (size_t)std::max<double>(1.0, std::floor(budget / (double)per));
  chunk = std::min(chunk, (size_t)std::max(n, 1));
  const int part = std::max(std::min(c->nslots, c->nsm), c->nslots / std::max(share, 1));
  return per * chunk + Small::bytes((int)chunk, c->g.Ly) + slot_elems(c) * c->elem * part;
}

size_t ctx_workspace_bytes(peps_ctx* c) {
  return c->env.bytes + c->small.bytes + c->O.bytes + c->scratch.bytes + c->gsum.bytes;
}

cudaStream_t ctx_stream(peps_ctx* c) { return c->stream; }

bool ctx_is_fp64(const peps_ctx* c) { return c->elem == 8; }

}  // namespace peps

extern "C" {

const char* peps_status_str(peps_status s) {
  switch (s) {
    case PEPS_OK: return "PEPS_OK";
    case PEPS_EINVAL: return "PEPS_EINVAL";
    case PEPS_ENOMEM: return "PEPS_ENOMEM";
    case PEPS_ECUDA: return "PEPS_ECUDA";
    case PEPS_ETIMEOUT: return "PEPS_ETIMEOUT";
    case PEPS_ENUMERIC: return "PEPS_ENUMERIC";
  }
  return "PEPS_UNKNOWN";
}

const char* peps_last_error(void) { return g_err.c_str(); }

peps_status peps_create(const peps_params* p, const double* A_host, void* stream, peps_ctx** out) {
  g_err.clear();
  if (!p || !A_host || !out) return fail(PEPS_EINVAL, "null argument");
  if (p->Lx < 2 || p->Ly < 2 || p->Lx > kMaxL || p->Ly > kMaxL) return fail(PEPS_EINVAL, "Lx, Ly must be in [2, 64]");
  if ((long)p->Lx * p->Ly > 64L * kMaxWords) return fail(PEPS_EINVAL, "too many sites");
  if (p->d != 2) return fail(PEPS_EINVAL, "d must be 2");
  if (p->D < 1 || p->D > 16) return fail(PEPS_EINVAL, "D must be in [1, 16]");
  if (p->Dc < 1 || p->Dc > kMaxDc || p->Dc * p->D > kMaxDcD) return fail(PEPS_EINVAL, "need 1 <= Dc <= 32, Dc*D <= 256");
  if (p->prec != PEPS_FP64 && p->prec != PEPS_FP32 && p->prec != PEPS_MIXED_TF32)
    return fail(PEPS_EINVAL, "precision not available: use PEPS_FP64, PEPS_FP32 or PEPS_MIXED_TF32");
  if (!std::isfinite(p->J1) || !std::isfinite(p->J2)) return fail(PEPS_EINVAL, "non-finite coupling");
  // padded entries must be zero (open edges of dimension one, Eq. 1)
  const int D = p->D, Lx = p->Lx, Ly = p->Ly, N = Lx * Ly;
  const size_t D4 = (size_t)D * D * D * D;
  for (int i = 0; i < N; ++i) {
    const int r = i / Lx, col = i % Lx;
    const int dl = col == 0 ? 1 : D, dr = col == Lx - 1 ? 1 : D, du = r == 0 ? 1 : D, dd = r == Ly - 1 ? 1 : D;
    for (int s = 0; s < 2; ++s)
      for (size_t e = 0; e < D4; ++e) {
        const int l = (int)(e / (D * D * D)), rr = (int)(e / (D * D) % D), u = (int)(e / D % D), d = (int)(e % D);
        const double v = A_host[((size_t)i * 2 + s) * D4 + e];
        if (!std::isfinite(v)) return fail(PEPS_EINVAL, "non-finite tensor entry");
        if ((l >= dl || rr >= dr || u >= du || d >= dd) && v != 0.0)
          return fail(PEPS_EINVAL, "non-zero tensor entry past an open edge");
      }
  }
  peps_ctx* c = new peps_ctx();
  c->p = *p;
  c->g.Lx = Lx;
  c->g.Ly = Ly;
  c->g.D = D;
  c->g.Dc = p->Dc;
  c->g.N = N;
  c->g.nwords = (N + 63) / 64;
  c->g.J1 = p->J1;
  c->g.J2 = p->J2;
  c->g.fit = 0;
  c->stream = (cudaStream_t)stream;
  c->elem = p->prec == PEPS_FP64 ? 8 : 4;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "device query");
  }
  c->wm_smem = wm_fits_smem(c->g, c->elem);
  if (c->elem == 8) {
    c->res_boundary = max_blocks_boundary<double>(c->g);
    c->res_row = max_blocks_row<double>(c->g);
    c->res_pair = max_blocks_pair_fused<double>(c->g);
    if (!c->res_pair) c->res_pair = max_blocks_pair<double>(c->g);
    c->res_mc = max_blocks_mc<double>(c->g);
  } else {
    c->res_boundary = max_blocks_boundary<float>(c->g);
    c->res_row = max_blocks_row<float>(c->g);
    c->pair_tc = p->prec == PEPS_MIXED_TF32 && c->g.D == 8 && c->g.Dc == 16;
    c->res_pair = c->pair_tc ? max_blocks_pair_tc() : max_blocks_pair_fused<float>(c->g);
    if (!c->res_pair) c->res_pair = max_blocks_pair<float>(c->g);
    c->res_mc = max_blocks_mc<float>(c->g);
  }
  c->nslots = std::max(std::max(c->res_boundary, c->res_row), std::max(c->res_pair, c->res_mc));
  {
    // a choice peps_autotune made in this process for the same model shape
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (auto& kv : g_tuned)
      if (kv.first == tune_key(c)) {
        c->row_generic = kv.second.row_generic;
        c->pair_mode = kv.second.pair_mode;
        c->boundary_ctas = kv.second.boundary_ctas;
        if (c->p.workspace_gb <= 0) c->p.workspace_gb = kv.second.workspace_gb;
        apply_variants(c);
      }
  }
  peps_status st = upload_tensors(c, A_host);
  if (st == PEPS_OK) st = c->elem == 8 ? setup_trivial<double>(c) : setup_trivial<float>(c);
  if (st != PEPS_OK) {
    peps_destroy(c);
    return st;
  }
  *out = c;
  return PEPS_OK;
}

peps_status peps_destroy(peps_ctx* c) {
  if (!c) return PEPS_OK;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  for (auto& e : c->ev) {
    cudaEventDestroy(e.second.first);
    cudaEventDestroy(e.second.second);
  }
  drop_graphs(c);
  if (c->pinned) cudaFreeHost(c->pinned);
  DevBuf* work[] = {&c->env, &c->small, &c->O, &c->scratch, &c->gsum, &c->go, &c->corr_sites, &c->corr_x,
                    &c->corr_scratch, &c->Scache, &c->cbits};
  for (DevBuf* b : work) b->release();
  if (!c->parent) {
    DevBuf* model[] = {&c->tcB, &c->A, &c->A64, &c->triv_mps, &c->triv_t1, &c->triv_t2, &c->bd};
    for (DevBuf* b : model) b->release();
  }
  delete c;
  return PEPS_OK;
}

peps_status peps_set_tensors(peps_ctx* c, const double* A_host) {
  if (!c || !A_host) return fail(PEPS_EINVAL, "null argument");
  if (c->parent) return fail(PEPS_EINVAL, "a worker context shares its model's tensors");
  return upload_tensors(c, A_host);
}

peps_status peps_go_step(peps_ctx* c, const double* grad, double dt, uint64_t seed, uint64_t step, double* A_host) {
  if (!c || !grad) return fail(PEPS_EINVAL, "null argument");
  if (c->parent) return fail(PEPS_EINVAL, "a worker context shares its model's tensors");
  if (!std::isfinite(dt) || dt < 0.0) return fail(PEPS_EINVAL, "dt must be finite and non-negative");
  g_err.clear();
  const size_t D4 = (size_t)c->g.D * c->g.D * c->g.D * c->g.D;
  const size_t bytes = (size_t)c->g.N * 2 * D4 * sizeof(double);
  // a NaN or infinite derivative has no sign to step against: reject the step
  PEPS_CUDA(c->go.ensure(sizeof(int)));
  PEPS_CUDA(cudaMemsetAsync(c->go.p, 0, sizeof(int), c->stream));
  PEPS_CUDA(launch_go_check(grad, c->g, (int*)c->go.p, c->nsm, c->stream));
  int bad = 0;
  PEPS_CUDA(cudaMemcpyAsync(&bad, c->go.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  PEPS_CUDA(cudaStreamSynchronize(c->stream));
  if (bad) return fail(PEPS_EINVAL, "the derivative holds NaN or infinite entries; the tensors are unchanged");
  PEPS_CUDA(launch_go_step(master_tensors(c), grad, c->g, dt, seed, step, c->nsm, c->stream));
  peps_status st = refresh_working_copies(c);
  if (st != PEPS_OK) return st;
  if (A_host) PEPS_CUDA(cudaMemcpyAsync(A_host, master_tensors(c), bytes, cudaMemcpyDeviceToHost, c->stream));
  PEPS_CUDA(cudaStreamSynchronize(c->stream));
  return PEPS_OK;
}

peps_status peps_evaluate(peps_ctx* c, const uint64_t* S, int n, double* logabs, int8_t* sign, double* eloc, void* O,
                          int32_t* status) {
  peps_status st = check_ctx(c, S, n);
  if (st != PEPS_OK) return st;
  g_err.clear();
  if (c->graphs && n > 0) {
    peps_status st0 = ensure_workspace(c, n, false);
    if (st0 != PEPS_OK) return st0;
    const void* out[6] = {logabs, sign, eloc, O, status, nullptr};
    if (c->elem == 8)
      return run_graphed(c, 0, S, n, out,
                         [&]() { return evaluate_impl<double>(c, S, n, logabs, sign, eloc, (double*)O, status); });
    return run_graphed(c, 0, S, n, out,
                       [&]() { return evaluate_impl<float>(c, S, n, logabs, sign, eloc, (float*)O, status); });
  }
  if (c->elem == 8) return evaluate_impl<double>(c, S, n, logabs, sign, eloc, (double*)O, status);
  return evaluate_impl<float>(c, S, n, logabs, sign, eloc, (float*)O, status);
}

peps_status peps_amplitudes(peps_ctx* c, const uint64_t* S, int n, double* logabs, int8_t* sign, int32_t* status) {
  if (n > 0 && (!logabs || !sign)) return fail(PEPS_EINVAL, "null output");
  return peps_evaluate(c, S, n, logabs, sign, nullptr, nullptr, status);
}

peps_status peps_local_energy(peps_ctx* c, const uint64_t* S, int n, double* eloc, int32_t* status) {
  if (n > 0 && !eloc) return fail(PEPS_EINVAL, "null output");
  return peps_evaluate(c, S, n, nullptr, nullptr, eloc, nullptr, status);
}

peps_status peps_log_derivatives(peps_ctx* c, const uint64_t* S, int n, void* O) {
  if (n > 0 && !O) return fail(PEPS_EINVAL, "null output");
  return peps_evaluate(c, S, n, nullptr, nullptr, nullptr, O, nullptr);
}

peps_status peps_gradient(peps_ctx* c, const uint64_t* S, int n, double* e_site, double* grad, double* cov,
                          double* logabs, int8_t* sign, double* eloc, int32_t* status, int* n_used) {
  peps_status st = check_ctx(c, S, n);
  if (st != PEPS_OK) return st;
  if (n == 0) return fail(PEPS_EINVAL, "empty batch");
  g_err.clear();
  if (c->graphs) {
    if (c->elem == 8) return gradient_graphed<double>(c, S, n, e_site, grad, cov, logabs, sign, eloc, status, n_used);
    return gradient_graphed<float>(c, S, n, e_site, grad, cov, logabs, sign, eloc, status, n_used);
  }
  if (c->elem == 8) return gradient_impl<double>(c, S, n, e_site, grad, cov, logabs, sign, eloc, status, n_used);
  return gradient_impl<float>(c, S, n, e_site, grad, cov, logabs, sign, eloc, status, n_used);
}

peps_status peps_gradient_sums(peps_ctx* c, const uint64_t* S, int n, double* sums, int accumulate, double* logabs,
                               int8_t* sign, double* eloc, int32_t* status) {
  peps_status st = check_ctx(c, S, n);
  if (st != PEPS_OK) return st;
  if (!sums) return fail(PEPS_EINVAL, "null sums");
  g_err.clear();
  if (n == 0) {
    if (!accumulate)
      PEPS_CUDA(cudaMemsetAsync(sums, 0, (kSumsHead + 2 * grad_total(c)) * sizeof(double), c->stream));
    return PEPS_OK;
  }
  if (c->elem == 8) return gradient_sums_impl<double>(c, S, n, sums, accumulate != 0, logabs, sign, eloc, status);
  return gradient_sums_impl<float>(c, S, n, sums, accumulate != 0, logabs, sign, eloc, status);
}

peps_status peps_gradient_finalize(peps_ctx* c, const double* sums, double* e_site, double* e_var, double* grad,
                                   double* cov, int* n_used) {
  if (!c || !sums) return fail(PEPS_EINVAL, "null argument");
  g_err.clear();
  return gradient_finalize_impl(c, sums, e_site, e_var, grad, cov, n_used);
}

size_t peps_gradient_sums_len(const peps_ctx* c) { return c ? kSumsHead + 2 * grad_total(c) : 0; }

peps_status peps_mc_sweep(peps_ctx* c, uint64_t* S, int n, int nsweeps, uint64_t seed, uint64_t chain0,
                          uint64_t sweep0, int64_t* accepted) {
  peps_status st = check_ctx(c, S, n);
  if (st != PEPS_OK) return st;
  if (nsweeps < 0) return fail(PEPS_EINVAL, "negative sweep count");
  g_err.clear();
  if (c->elem == 8) return mc_impl<double>(c, S, n, nsweeps, seed, chain0, sweep0, accepted);
  return mc_impl<float>(c, S, n, nsweeps, seed, chain0, sweep0, accepted);
}

peps_status peps_correlations(peps_ctx* c, const uint64_t* S, int n, const int* sites_host, int nc, double* m2_dev,
                              double* corr_dev, int32_t* status_dev) {
  peps_status st = check_ctx(c, S, n);
  if (st != PEPS_OK) return st;
  if (nc < 1 || !sites_host) return fail(PEPS_EINVAL, "need at least one central site");
  std::vector<char> seen(c->g.N, 0);
  for (int p = 0; p < nc; ++p) {
    if (sites_host[p] < 0 || sites_host[p] >= c->g.N || seen[sites_host[p]])
      return fail(PEPS_EINVAL, "central sites must be distinct sites of the lattice");
    seen[sites_host[p]] = 1;
  }
  g_err.clear();
  if (n == 0) return PEPS_OK;
  if (c->elem == 8) return correlations_impl<double>(c, S, n, sites_host, nc, m2_dev, corr_dev, status_dev);
  return correlations_impl<float>(c, S, n, sites_host, nc, m2_dev, corr_dev, status_dev);
}

peps_status peps_set_truncation(peps_ctx* c, int fit_sweeps) {
  if (!c) return fail(PEPS_EINVAL, "null context");
  if (fit_sweeps < 0 || fit_sweeps > 64) return fail(PEPS_EINVAL, "need 0 <= fit_sweeps <= 64");
  if (c->parent) return fail(PEPS_EINVAL, "set the truncation on the model's context, not a serving worker");
  c->g.fit = fit_sweeps;
  c->cache_dirty = true;   // cached environments belong to the other truncation
  drop_graphs(c);          // the workspace slots change size
  return PEPS_OK;
}

peps_status peps_set_env_cache(peps_ctx* c, int on) {
  if (!c) return fail(PEPS_EINVAL, "null context");
  c->env_cache = on != 0;
  c->cache_dirty = true;
  return PEPS_OK;
}

peps_status peps_set_graphs(peps_ctx* c, int on) {
  if (!c) return fail(PEPS_EINVAL, "null context");
  if (on && !c->stream) return fail(PEPS_EINVAL, "graph capture needs a context created on a non-default stream");
  if (!on) drop_graphs(c);
  c->graphs = on != 0;
  return PEPS_OK;
}

peps_status peps_graph_stats(peps_ctx* c, long long* stats) {
  if (!c || !stats) return fail(PEPS_EINVAL, "null argument");
  stats[0] = (long long)c->gcache.size();
  stats[1] = c->graph_captures;
  stats[2] = c->graph_replays;
  return PEPS_OK;
}

peps_status peps_tuned_config(peps_ctx* c, int* vals, double* workspace_gb) {
  if (!c) return fail(PEPS_EINVAL, "null context");
  if (vals) {
    const bool fused = c->elem == 8 ? max_blocks_pair_fused<double>(c->g) > 0 : max_blocks_pair_fused<float>(c->g) > 0;
    vals[0] = c->pair_tc && c->pair_mode == 0 ? 0 : ((c->pair_mode == 2 || !fused) ? 2 : 1);
    vals[1] = c->row_generic;
    vals[2] = c->boundary_ctas > 0 ? std::min(c->boundary_ctas, c->res_boundary) : c->res_boundary;
    vals[3] = c->chunk;
  }
  if (workspace_gb) *workspace_gb = c->p.workspace_gb > 0 ? c->p.workspace_gb : 24.0;
  return PEPS_OK;
}

peps_status peps_autotune(peps_ctx* c, const uint64_t* S, int n, char* report, size_t report_len) {
  peps_status st = check_ctx(c, S, n);
  if (st != PEPS_OK) return st;
  if (n == 0) return fail(PEPS_EINVAL, "empty probe batch");
  if (c->parent) return fail(PEPS_EINVAL, "tune the model's context, not a serving worker");
  g_err.clear();
  drop_graphs(c);
  const bool graphs = c->graphs;
  c->graphs = false;
  std::string rep;
  cudaEvent_t e0, e1;
  PEPS_CUDA(cudaEventCreate(&e0));
  PEPS_CUDA(cudaEventCreate(&e1));
  // one untimed and one timed gradient pass over the probe batch
  auto trial = [&](double& ms) -> peps_status {
    for (int k = 0; k < 2; ++k) {
      PEPS_CUDA(cudaEventRecord(e0, c->stream));
      peps_status s2 = c->elem == 8
                           ? gradient_impl<double>(c, S, n, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                   nullptr, nullptr)
                           : gradient_impl<float>(c, S, n, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                  nullptr, nullptr);
      if (s2 != PEPS_OK) return s2;
      PEPS_CUDA(cudaEventRecord(e1, c->stream));
      PEPS_CUDA(cudaEventSynchronize(e1));
      float t = 0.f;
      PEPS_CUDA(cudaEventElapsedTime(&t, e0, e1));
      ms = t;
    }
    return PEPS_OK;
  };
  char buf[160];
  auto pick = [&](const char* what, std::vector<int> cands, std::function<void(int)> set,
                  std::function<const char*(int)> name) -> peps_status {
    double best = 1e300;
    int bi = cands[0];
    rep += what;
    rep += ":";
    for (int v : cands) {
      set(v);
      double ms = 0;
      peps_status s2 = trial(ms);
      if (s2 != PEPS_OK) return s2;
      snprintf(buf, sizeof(buf), " %s %.1f ms", name(v), ms);
      rep += buf;
      if (ms < best) {
        best = ms;
        bi = v;
      }
    }
    set(bi);
    snprintf(buf, sizeof(buf), " -> %s; ", name(bi));
    rep += buf;
    return PEPS_OK;
  };
  const bool fp64 = c->elem == 8;
  const bool fused_pair = fp64 ? max_blocks_pair_fused<double>(c->g) > 0 : max_blocks_pair_fused<float>(c->g) > 0;
  std::vector<int> pc;
  if (c->pair_tc) pc.push_back(0);
  if (fused_pair) pc.push_back(1);
  pc.push_back(2);
  static const char* pnames[] = {"tensor-core", "fused", "generic"};
  static const char* rnames[] = {"fused", "generic"};
  if (c->g.Ly > 1 && pc.size() > 1)
    st = pick("two-row kernel", pc, [&](int v) { c->pair_mode = v == 1 && !c->pair_tc ? 0 : v; apply_variants(c); },
              [&](int v) { return pnames[v]; });
  if (st == PEPS_OK)
    st = pick("single-row kernel", {0, 1}, [&](int v) { c->row_generic = v; apply_variants(c); },
              [&](int v) { return rnames[v]; });
  std::vector<std::string> bnames;
  if (st == PEPS_OK) {
    std::vector<int> bc = {c->res_boundary};
    if (c->res_boundary / 2 >= c->nsm) bc.push_back(c->res_boundary / 2);
    for (int v : bc) bnames.push_back(std::to_string(v) + " CTAs");
    std::vector<int> idx;
    for (size_t i = 0; i < bc.size(); ++i) idx.push_back((int)i);
    st = pick("boundary grid", idx, [&](int i) { c->boundary_ctas = bc[i]; },
              [&](int i) { return bnames[i].c_str(); });
  }
  if (st == PEPS_OK) {
    // a larger workspace budget means fewer chunks (fewer partial last waves)
    const double cur = c->p.workspace_gb > 0 ? c->p.workspace_gb : 24.0;
    size_t freeb = 0, totb = 0;
    cudaMemGetInfo(&freeb, &totb);
    const double cap = 0.6 * (double)(freeb + ctx_workspace_bytes(c)) / 1e9;
    std::vector<double> ws = {cur};
    for (double f : {2.0, 4.0})
      if (cur * f <= cap) ws.push_back(cur * f);
    const size_t per = env_bytes_per_cfg(c) + (size_t)c->g.N * c->g.D * c->g.D * c->g.D * c->g.D * c->elem;
    if ((double)n * per > cur * 1e9 && ws.size() > 1) {
      std::vector<std::string> wn;
      for (double w : ws) wn.push_back(std::to_string((int)w) + " GB");
      std::vector<int> idx;
      for (size_t i = 0; i < ws.size(); ++i) idx.push_back((int)i);
      st = pick("workspace", idx, [&](int i) { c->p.workspace_gb = ws[i]; },
                [&](int i) { return wn[i].c_str(); });
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->graphs = graphs;
  if (st != PEPS_OK) return st;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    TuneVal v{c->row_generic, c->pair_mode, c->boundary_ctas, c->p.workspace_gb};
    bool found = false;
    for (auto& kv : g_tuned)
      if (kv.first == tune_key(c)) {
        kv.second = v;
        found = true;
      }
    if (!found) g_tuned.push_back({tune_key(c), v});
  }
  if (report && report_len) {
    strncpy(report, rep.c_str(), report_len - 1);
    report[report_len - 1] = 0;
  }
  return PEPS_OK;
}

peps_status peps_packer_create(void* stream, peps_packer** out) {
  if (!out) return fail(PEPS_EINVAL, "null argument");
  peps_packer* pk = new peps_packer();
  pk->stream = (cudaStream_t)stream;
  *out = pk;
  return PEPS_OK;
}

peps_status peps_packer_destroy(peps_packer* pk) {
  if (!pk) return PEPS_OK;
  if (pk->stream) cudaStreamSynchronize(pk->stream);
  else cudaDeviceSynchronize();
  pk->scratch.release();
  pk->models.release();
  pk->start.release();
  delete pk;
  return PEPS_OK;
}

peps_status peps_packer_evaluate(peps_packer* pk, int nreq, peps_ctx* const* ctxs, const uint64_t* const* S,
                                 const int* n, double* const* logabs, int8_t* const* sign, double* const* eloc,
                                 void* const* O, int32_t* const* status) {
  if (!pk || nreq < 0 || (nreq > 0 && (!ctxs || !S || !n))) return fail(PEPS_EINVAL, "null argument");
  if (nreq == 0) return PEPS_OK;
  g_err.clear();
  const size_t elem = ctxs[0] ? ctxs[0]->elem : 0;
  for (int i = 0; i < nreq; ++i) {
    if (!ctxs[i]) return fail(PEPS_EINVAL, "null context");
    if (ctxs[i]->elem != elem) return fail(PEPS_EINVAL, "packed requests must share the precision class (FP64 or FP32)");
    if (n[i] <= 0 || !S[i]) return fail(PEPS_EINVAL, "every packed request needs configurations");
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return fail(PEPS_EINVAL, "a context may appear once per packed launch");
  }
  if (elem == 8) return packed_impl<double>(pk, nreq, ctxs, S, n, logabs, sign, eloc, O, status);
  return packed_impl<float>(pk, nreq, ctxs, S, n, logabs, sign, eloc, O, status);
}

peps_status peps_profile_enable(peps_ctx* c, int on) {
  if (!c) return fail(PEPS_EINVAL, "null context");
  c->prof = on != 0;
  return PEPS_OK;
}

peps_status peps_profile_read(peps_ctx* c, double* ms, long long* launches, int reset) {
  if (!c) return fail(PEPS_EINVAL, "null context");
  PEPS_CUDA(cudaStreamSynchronize(c->stream));
  for (auto& e : c->ev) {
    float t = 0.f;
    cudaEventElapsedTime(&t, e.second.first, e.second.second);
    c->ms[e.first] += t;
    cudaEventDestroy(e.second.first);
    cudaEventDestroy(e.second.second);
  }
  c->ev.clear();
  for (int i = 0; i < 8; ++i) {
    if (ms) ms[i] = c->ms[i];
    if (launches) launches[i] = c->launches[i];
    if (reset) {
      c->ms[i] = 0;
      c->launches[i] = 0;
    }
  }
  return PEPS_OK;
}

peps_status peps_synchronize(peps_ctx* c) {
  if (!c) return fail(PEPS_EINVAL, "null context");
  PEPS_CUDA(cudaStreamSynchronize(c->stream));
  return PEPS_OK;
}

// ----------------------------------------------------- host-side checks
static void host_gemm(const GemmDesc& g, const double* A, const double* B, double* C) {
  const int kn2 = g.ak.n2;
  for (int bt = 0; bt < g.nb; ++bt)
    for (int i = 0; i < g.M; ++i)
      for (int j = 0; j < g.N; ++j) {
        double s = 0;
        for (int k = 0; k < g.K; ++k) {
          const int k1 = k / kn2, k2 = k % kn2;
          const double a = A[(size_t)bt * g.sa + ixoff(g.am, i) + k1 * g.ak.s1 + k2 * g.ak.s2];
          const double b = B[(size_t)bt * g.sb + k1 * g.bk.s1 + k2 * g.bk.s2 + ixoff(g.bn, j)];
          s += a * b;
        }
        C[(size_t)bt * g.sc + ixoff(g.cm, i) + ixoff(g.cn, j)] = s;
      }
}

peps_status peps_debug_host_op(int op, int D, int Dc, const double* in0, const double* in1, const double* in2,
                               const double* in3, const double* in4, double* out) {
  if (op < 0 || op > 4 || D < 1 || Dc < 1 || !out) return fail(PEPS_EINVAL, "bad argument");
  const size_t tsz = (size_t)Dc * Dc * D * D * D;
  std::vector<double> t0(tsz, 0.0), t1(tsz, 0.0);
  const double* bufs[8] = {in0, in1, in2, in3, in4, t0.data(), t1.data(), out};
  for (int s = 0; s < op_nsteps(op); ++s) {
    const Step st = op_step_bufs(op, s);
    host_gemm(op_desc(op, st.s, D, Dc), bufs[st.a], bufs[st.b], const_cast<double*>(bufs[st.c]));
  }
  return PEPS_OK;
}

peps_status peps_debug_host_zip(int lr, int D, int Dc, const int* dims, const double* C, const double* M,
                                const double* T, double* X) {
  if (!dims || !C || !M || !T || !X) return fail(PEPS_EINVAL, "bad argument");
  ZipDims z{dims[0], dims[1], dims[2], dims[3], dims[4], dims[5], dims[6]};
  const int sl = dims[7], sr = dims[8], si = dims[9], so = dims[10];
  std::vector<double> Y((size_t)z.k * z.a * z.b * z.i * z.l * z.r * z.o + 16, 0.0);
  if (lr) {
    host_gemm(zip_lr_step(0, z, D, Dc, sl, sr, si, so), C, M, Y.data());
    host_gemm(zip_lr_step(1, z, D, Dc, sl, sr, si, so), Y.data(), T, X);
  } else {
    host_gemm(zip_rl_step(0, z, D, Dc, sl, sr, si, so), M, C, Y.data());
    host_gemm(zip_rl_step(1, z, D, Dc, sl, sr, si, so), Y.data(), T, X);
  }
  return PEPS_OK;
}

}  // extern "C"
