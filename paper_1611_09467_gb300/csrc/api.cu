// C ABI of libpeps.so: context, workspace, batching into chunks, launches.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
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
    if (c->prof) {
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      cudaEventRecord(a, c->stream);
    }
  }
  ~Prof() {
    if (c->prof) {
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
  int* flags;
  int* status;
  int8_t* sign;
  static size_t bytes(int chunk, int Ly) {
    return (size_t)chunk * (2 + 3 * (size_t)Ly) * 8 + (size_t)chunk * 2 * 4 + (size_t)chunk + 256;
  }
  void carve(void* base, int chunk, int Ly) {
    char* p = (char*)base;
    logabs = (double*)p; p += (size_t)chunk * 8;
    eloc = (double*)p; p += (size_t)chunk * 8;
    eloc_h = (double*)p; p += (size_t)chunk * Ly * 8;
    eloc_v = (double*)p; p += (size_t)chunk * Ly * 8;
    w_row = (double*)p; p += (size_t)chunk * Ly * 8;
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
  PEPS_CUDA(c->env.ensure(env_bytes_per_cfg(c) * chunk));
  PEPS_CUDA(c->small.ensure(Small::bytes(chunk, g.Ly)));
  if (want_O) PEPS_CUDA(c->O.ensure((size_t)chunk * g.N * D4 * c->elem));
  PEPS_CUDA(c->scratch.ensure(slot_elems(c) * c->elem * c->nslots));
  return PEPS_OK;
}

template <typename R>
KArgs<R> make_args(peps_ctx* c, const uint64_t* S, int n, const Small& sm) {
  KArgs<R> a;
  const Geometry& g = c->g;
  a.g = g;
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
  a.O = nullptr;
  a.scratch = (R*)c->scratch.p;
  a.slot_elems = slot_elems(c);
  a.smem_wm = c->wm_smem ? 1 : 0;
  a.tcB = (const float*)c->tcB.p;
  return a;
}

template <typename R>
peps_status evaluate_chunk(peps_ctx* c, const uint64_t* S, int n, bool need_env_l, bool need_pairs, R* O,
                           Small& sm) {
  KArgs<R> a = make_args<R>(c, S, n, sm);
  a.O = O;
  PEPS_CUDA(cudaMemsetAsync(sm.flags, 0, (size_t)n * sizeof(int), c->stream));
  const int dirs = need_env_l ? 2 : 1;
  // persistent kernels: never more CTAs than can be resident at once
  int grid = std::min(n * dirs, std::min(c->nslots, c->res_boundary));
  {
    Prof pf(c, 0);
    PEPS_CUDA(launch_boundary<R>(a, dirs, std::max(grid, 1), c->stream));
  }
  if (need_env_l) {
    grid = std::min(n * c->g.Ly, std::min(c->nslots, c->res_row));
    Prof pf(c, 1);
    PEPS_CUDA(launch_row<R>(a, std::max(grid, 1), c->stream));
  }
  if (need_pairs && c->g.Ly > 1) {
    grid = std::min(n * (c->g.Ly - 1), std::min(c->nslots, c->res_pair));
    Prof pf(c, 2);
    if constexpr (sizeof(R) == 4) {
      if (c->pair_tc) {
        PEPS_CUDA(launch_pair_tc(a, std::max(grid, 1), c->stream));
      } else {
        PEPS_CUDA(launch_pair<R>(a, std::max(grid, 1), c->stream));
      }
    } else {
      PEPS_CUDA(launch_pair<R>(a, std::max(grid, 1), c->stream));
    }
  } else {
    PEPS_CUDA(cudaMemsetAsync(sm.eloc_v, 0, (size_t)n * c->g.Ly * sizeof(double), c->stream));
  }
  if (!need_env_l) PEPS_CUDA(cudaMemsetAsync(sm.eloc_h, 0, (size_t)n * c->g.Ly * sizeof(double), c->stream));
  {
    Prof pf(c, 3);
    PEPS_CUDA(launch_finalize(c->g, S, n, sm.eloc_h, sm.eloc_v, sm.flags, sm.eloc, sm.status, need_env_l ? 1 : 0,
                              c->stream));
  }
  return PEPS_OK;
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
    st = evaluate_chunk<R>(c, Sc, m, need_l, want_e, want_O ? O + (size_t)c0 * g.N * D4 : nullptr, sm);
    if (st != PEPS_OK) return st;
    if (logabs) PEPS_CUDA(cudaMemcpyAsync(logabs + c0, sm.logabs, m * 8, cudaMemcpyDeviceToDevice, c->stream));
    if (sign) PEPS_CUDA(cudaMemcpyAsync(sign + c0, sm.sign, m, cudaMemcpyDeviceToDevice, c->stream));
    if (eloc) PEPS_CUDA(cudaMemcpyAsync(eloc + c0, sm.eloc, m * 8, cudaMemcpyDeviceToDevice, c->stream));
    if (status) PEPS_CUDA(cudaMemcpyAsync(status + c0, sm.status, m * 4, cudaMemcpyDeviceToDevice, c->stream));
  }
  return PEPS_OK;
}

template <typename R>
peps_status gradient_impl(peps_ctx* c, const uint64_t* S, int n, double* e_site, double* grad, double* cov,
                          double* logabs, int8_t* sign, double* eloc, int32_t* status, int* n_used) {
  const Geometry& g = c->g;
  const size_t D4 = (size_t)g.D * g.D * g.D * g.D;
  const size_t total = (size_t)g.N * 2 * D4;
  peps_status st = ensure_workspace(c, n, true);
  if (st != PEPS_OK) return st;
  PEPS_CUDA(c->gsum.ensure((2 * total + 2) * sizeof(double)));
  double* sumO = (double*)c->gsum.p;
  double* sumEO = sumO + total;
  double* sums = sumEO + total;
  PEPS_CUDA(cudaMemsetAsync(c->gsum.p, 0, (2 * total + 2) * sizeof(double), c->stream));
  Small sm;
  sm.carve(c->small.p, c->chunk, g.Ly);
  for (int c0 = 0; c0 < n; c0 += c->chunk) {
    const int m = std::min(c->chunk, n - c0);
    const uint64_t* Sc = S + (size_t)c0 * g.nwords;
    st = evaluate_chunk<R>(c, Sc, m, true, true, (R*)c->O.p, sm);
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
  {
    Prof pf(c, 6);
    PEPS_CUDA(launch_grad_finalize((int)total, 0, sums, sumO, sumEO, grad, cov, c->stream));
  }
  double h[2] = {0, 0};
  PEPS_CUDA(cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  PEPS_CUDA(cudaStreamSynchronize(c->stream));
  if (e_site) *e_site = h[1] > 0 ? h[0] / h[1] / g.N : NAN;
  if (n_used) *n_used = (int)h[1];
  return PEPS_OK;
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
  DevBuf* work[] = {&c->env, &c->small, &c->O, &c->scratch, &c->gsum, &c->go};
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
  if (c->elem == 8) return gradient_impl<double>(c, S, n, e_site, grad, cov, logabs, sign, eloc, status, n_used);
  return gradient_impl<float>(c, S, n, e_site, grad, cov, logabs, sign, eloc, status, n_used);
}

peps_status peps_mc_sweep(peps_ctx* c, uint64_t* S, int n, int nsweeps, uint64_t seed, uint64_t chain0,
                          uint64_t sweep0, int64_t* accepted) {
  peps_status st = check_ctx(c, S, n);
  if (st != PEPS_OK) return st;
  if (nsweeps < 0) return fail(PEPS_EINVAL, "negative sweep count");
  g_err.clear();
  if (c->elem == 8) return mc_impl<double>(c, S, n, nsweeps, seed, chain0, sweep0, accepted);
  return mc_impl<float>(c, S, n, nsweeps, seed, chain0, sweep0, accepted);
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
