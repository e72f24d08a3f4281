// Simple-update imaginary-time evolution (Sec. III, computational details):
// the initialiser the paper runs before its gradient optimisation.
//
// State: site tensors Gamma_i[s][l][r][u][d] (FP64, padded to D^4 per spin)
// and a weight vector lam_b of length D on every nearest-neighbour bond b
// (bond index: horizontal bonds row-major, then vertical bonds row-major).
// A two-site gate on bond (i, j) is applied by one CTA:
//   1. M_i = Gamma_i with the weights of its three other bonds and of the
//      bond itself absorbed, as a matrix [(outer legs), (s, x)]; M_j likewise
//      (without the bond's weight).  Column-major in the CTA's scratch slot.
//   2. Householder QR of each (m = D^3 rows, n = 2D columns): M = Q R (qr.cuh).
//   3. Theta[(a, s_i'), (s_j', b)] = sum G[s_i' s_j', s_i s_j] R_i[a, (s_i, x)] R_j[b, (s_j, x)].
//   4. One-sided Jacobi SVD of Theta (columns rotated until orthogonal):
//      the D largest singular values, normalised, are the new weight; the
//      matching left / right singular vectors are the new R_i', R_j'.
//   5. Gamma_i' = Q_i R_i' (reflectors applied in reverse) with the outer
//      weights divided out again (zero weights and entries past an open edge
//      give zero); Gamma_j' likewise.
// The gates of one group act on disjoint bonds, so a group is one launch
// with one CTA per bond.  Gate: exp(-dtau J S.S) = e^{-dtau J/4} (I - P_s) +
// e^{3 dtau J/4} P_s, P_s the singlet projector (S.S = 1/4 on the triplet,
// -3/4 on the singlet); a SWAP gate routes next-nearest pairs through their
// shared neighbour.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/peps.h"
#include "kernels.h"
#include "qr.cuh"

namespace peps {
namespace su {

constexpr int kT = 256;
constexpr int kW = kT / 32;

struct Geom {
  int Lx, Ly, D, nh;   // nh = Ly (Lx - 1) horizontal bonds
};

struct Upd {
  int i, j;            // i the left or upper site
  int kind;            // 0: exp(-dtau J1 S.S), 1: exp(-dtau J2 S.S), 2: SWAP
  int pad;
};

__device__ __forceinline__ int bond_of(const Geom& g, int site, int leg) {
  const int r = site / g.Lx, c = site % g.Lx;
  switch (leg) {
    case 0: return c > 0 ? r * (g.Lx - 1) + c - 1 : -1;
    case 1: return c < g.Lx - 1 ? r * (g.Lx - 1) + c : -1;
    case 2: return r > 0 ? g.nh + (r - 1) * g.Lx + c : -1;
    default: return r < g.Ly - 1 ? g.nh + r * g.Lx + c : -1;
  }
}

// Weight of index idx of a leg: the bond's weight, or on an open edge 1 for
// index 0 and 0 past the edge.
__device__ __forceinline__ double leg_w(const Geom& g, const double* lam, int site, int leg, int idx) {
  const int b = bond_of(g, site, leg);
  return b < 0 ? (idx == 0 ? 1.0 : 0.0) : lam[(size_t)b * g.D + idx];
}

__device__ __forceinline__ double inv_or_zero(double w) { return w != 0.0 ? 1.0 / w : 0.0; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum_d(double v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int k = 0; k < kW; ++k) t += red[k];
  return t;
}

// The gate's entry G[p][q], p = 2 s_i' + s_j', q = 2 s_i + s_j.
__device__ double gate_entry(int kind, double J1, double J2, double dtau, int p, int q) {
  if (kind == 2) {
    const int sw = ((q & 1) << 1) | (q >> 1);
    return p == sw ? 1.0 : 0.0;
  }
  const double J = kind == 0 ? J1 : J2;
  // singlet (|01> - |10>)/sqrt(2): components on indices 1 and 2
  const double ps = (p == 1 ? 1.0 : (p == 2 ? -1.0 : 0.0)) * (q == 1 ? 1.0 : (q == 2 ? -1.0 : 0.0)) * 0.5;
  const double id = p == q ? 1.0 : 0.0;
  return exp(-dtau * J * 0.25) * (id - ps) + exp(0.75 * dtau * J) * ps;
}

// One-sided Jacobi SVD of the row-major m2 x n2 matrix T (shared memory):
// columns are rotated pairwise (round-robin order, one warp per pair) until
// every pair is orthogonal to working precision; V (row-major n2 x n2)
// accumulates the rotations, so T_in = T_out V^T with T_out = U diag(sigma).
__device__ void jacobi_svd(double* T, int m2, int n2, double* V, int* s_rot) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int e = threadIdx.x; e < n2 * n2; e += blockDim.x) V[e] = (e / n2 == e % n2) ? 1.0 : 0.0;
  const int np = n2 + (n2 & 1);            // players, one dummy when n2 is odd
  const double tol = 1e-15 * (double)m2;
  for (int sweep = 0; sweep < 40; ++sweep) {
    if (threadIdx.x == 0) *s_rot = 0;
    __syncthreads();
    for (int round = 0; round < np - 1; ++round) {
      for (int k = warp; k < np / 2; k += kW) {
        int p, q;
        if (k == 0) {
          p = round;
          q = np - 1;
        } else {
          p = (round + k) % (np - 1);
          q = (round - k + np - 1) % (np - 1);
        }
        if (p >= n2 || q >= n2) continue;
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int r = lane; r < m2; r += 32) {
          const double a = T[r * n2 + p], b = T[r * n2 + q];
          al += a * a;
          be += b * b;
          ga += a * b;
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (ga != 0.0 && fabs(ga) > tol * sqrt(al * be)) {
          const double zeta = (be - al) / (2.0 * ga);
          const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
          for (int r = lane; r < m2; r += 32) {
            const double a = T[r * n2 + p], b = T[r * n2 + q];
            T[r * n2 + p] = c * a - s * b;
            T[r * n2 + q] = s * a + c * b;
          }
          for (int r = lane; r < n2; r += 32) {
            const double a = V[r * n2 + p], b = V[r * n2 + q];
            V[r * n2 + p] = c * a - s * b;
            V[r * n2 + q] = s * a + c * b;
          }
          if (lane == 0) *s_rot = 1;
        }
      }
      __syncthreads();
    }
    if (*s_rot == 0) break;
    __syncthreads();
  }
  __syncthreads();
}

struct Args {
  Geom g;
  double* Gam;             // [N][2][D^4]
  double* lam;             // [nbonds][D]
  const Upd* ups;          // this launch's updates, one per CTA
  double J1, J2, dtau;
  double* scratch;         // per CTA: 4 m n doubles (M_i, M_j, N_i, N_j)
  size_t slot;
};

// Shared memory: Theta and V (n2max^2 each, n2max = 4D), sigma, order, tau.
__host__ __device__ inline size_t smem_doubles(int D) {
  const size_t n2 = 4 * (size_t)D;
  return 2 * n2 * n2 + n2 + 2 * 2 * (size_t)D + 16;
}

__global__ void __launch_bounds__(kT) k_su_bond(Args a) {
  extern __shared__ __align__(16) double sm[];
  __shared__ double red[kW];
  __shared__ int s_rot, s_order[64];
  __shared__ double s_nrm;
  const Geom& g = a.g;
  const int D = g.D, n = 2 * D, m = D * D * D, D4 = D * D * D * D;
  const Upd up = a.ups[blockIdx.x];
  const int i = up.i, j = up.j;
  const bool hor = j == i + 1;
  const int li = hor ? 1 : 3, lj = hor ? 0 : 2;
  const int bond = bond_of(g, i, li);
  int oi[3], oj[3];
  for (int x = 0, t = 0; x < 4; ++x)
    if (x != li) oi[t++] = x;
  for (int x = 0, t = 0; x < 4; ++x)
    if (x != lj) oj[t++] = x;
  double* Mi = a.scratch + (size_t)blockIdx.x * a.slot;
  double* Mj = Mi + (size_t)m * n;
  double* Ni = Mj + (size_t)m * n;
  double* Nj = Ni + (size_t)m * n;
  const int n2max = 4 * D;
  double* Th = sm;
  double* V = Th + (size_t)n2max * n2max;
  double* sig = V + (size_t)n2max * n2max;
  double* tau_i = sig + n2max;
  double* tau_j = tau_i + n;
  // ---- 1. M_i, M_j with the weights absorbed
  for (int e = threadIdx.x; e < m * n; e += blockDim.x) {
    const int col = e / m, row = e % m;
    const int s = col / D, x = col % D;
    const int o[3] = {row / (D * D), row / D % D, row % D};
    int legs[4];
    legs[oi[0]] = o[0];
    legs[oi[1]] = o[1];
    legs[oi[2]] = o[2];
    legs[li] = x;
    double v = a.Gam[((size_t)i * 2 + s) * D4 + ((legs[0] * D + legs[1]) * D + legs[2]) * D + legs[3]];
    v *= leg_w(g, a.lam, i, oi[0], o[0]) * leg_w(g, a.lam, i, oi[1], o[1]) * leg_w(g, a.lam, i, oi[2], o[2]);
    v *= a.lam[(size_t)bond * D + x];
    Mi[e] = v;
    legs[oj[0]] = o[0];
    legs[oj[1]] = o[1];
    legs[oj[2]] = o[2];
    legs[lj] = x;
    double w = a.Gam[((size_t)j * 2 + s) * D4 + ((legs[0] * D + legs[1]) * D + legs[2]) * D + legs[3]];
    w *= leg_w(g, a.lam, j, oj[0], o[0]) * leg_w(g, a.lam, j, oj[1], o[1]) * leg_w(g, a.lam, j, oj[2], o[2]);
    Mj[e] = w;
  }
  __syncthreads();
  // ---- 2. QR of both
  qr::house_qr<double>(Mi, m, n, tau_i, red);
  qr::house_qr<double>(Mj, m, n, tau_j, red);
  const int ki = min(m, n), kj = min(m, n);
  const int m2 = 2 * ki, n2 = 2 * kj;
  // ---- 3. Theta[(a, s_i'), (s_j', b)]
  for (int e = threadIdx.x; e < m2 * n2; e += blockDim.x) {
    const int r = e / n2, c = e % n2;
    const int ai = r >> 1, sp = r & 1, sq = c / kj, bj = c % kj;
    double P[2][2];
    for (int si = 0; si < 2; ++si)
      for (int sj = 0; sj < 2; ++sj) {
        double t = 0.0;
        for (int x = 0; x < D; ++x) {
          const int ci = si * D + x, cj = sj * D + x;
          const double ri = ai <= ci ? Mi[(size_t)ci * m + ai] : 0.0;
          const double rj = bj <= cj ? Mj[(size_t)cj * m + bj] : 0.0;
          t += ri * rj;
        }
        P[si][sj] = t;
      }
    double v = 0.0;
    for (int q = 0; q < 4; ++q) v += gate_entry(up.kind, a.J1, a.J2, a.dtau, sp * 2 + sq, q) * P[q >> 1][q & 1];
    Th[e] = v;
  }
  __syncthreads();
  // ---- 4. SVD; the K largest singular values, in decreasing order
  jacobi_svd(Th, m2, n2, V, &s_rot);
  for (int c = threadIdx.x; c < n2; c += blockDim.x) {
    double t = 0.0;
    for (int r = 0; r < m2; ++r) t += Th[r * n2 + c] * Th[r * n2 + c];
    sig[c] = sqrt(t);
  }
  __syncthreads();
  const int K = min(D, min(m2, n2));
  if (threadIdx.x == 0) {
    bool used[64];
    for (int c = 0; c < n2; ++c) used[c] = false;
    double nrm2 = 0.0;
    for (int t = 0; t < K; ++t) {
      int best = -1;
      for (int c = 0; c < n2; ++c)
        if (!used[c] && (best < 0 || sig[c] > sig[best])) best = c;
      used[best] = true;
      s_order[t] = best;
      nrm2 += sig[best] * sig[best];
    }
    s_nrm = sqrt(nrm2);
  }
  __syncthreads();
  const double nrm = s_nrm;
  // ---- new weight
  for (int x = threadIdx.x; x < D; x += blockDim.x)
    a.lam[(size_t)bond * D + x] = x < K ? (nrm > 0.0 ? sig[s_order[x]] / nrm : sig[s_order[x]]) : 0.0;
  // ---- 5. N_i = [R_i'; 0], N_j = [R_j'; 0], then the reflectors
  for (int e = threadIdx.x; e < m * n; e += blockDim.x) {
    const int col = e / m, row = e % m;
    const int s = col / D, x = col % D;
    double vi = 0.0, vj = 0.0;
    if (x < K) {
      const int c = s_order[x];
      const double sg = sig[c];
      if (row < ki && sg > 0.0) vi = Th[(row * 2 + s) * n2 + c] / sg;
      if (row < kj) vj = V[(s * kj + row) * n2 + c];
    }
    Ni[e] = vi;
    Nj[e] = vj;
  }
  __syncthreads();
  qr::apply_q<double>(Mi, tau_i, Ni, m, n, n);
  qr::apply_q<double>(Mj, tau_j, Nj, m, n, n);
  // ---- back to Gamma with the outer weights divided out (the bond weight
  // was just written; no thread reads it below)
  for (int e = threadIdx.x; e < 2 * D4; e += blockDim.x) {
    const int s = e / D4, w = e % D4;
    const int legs[4] = {w / (D * D * D), w / (D * D) % D, w / D % D, w % D};
    {
      const int row = (legs[oi[0]] * D + legs[oi[1]]) * D + legs[oi[2]];
      const int col = s * D + legs[li];
      double v = Ni[(size_t)col * m + row];
      v *= inv_or_zero(leg_w(g, a.lam, i, oi[0], legs[oi[0]])) * inv_or_zero(leg_w(g, a.lam, i, oi[1], legs[oi[1]])) *
           inv_or_zero(leg_w(g, a.lam, i, oi[2], legs[oi[2]]));
      a.Gam[((size_t)i * 2) * D4 + e] = v;
    }
    {
      const int row = (legs[oj[0]] * D + legs[oj[1]]) * D + legs[oj[2]];
      const int col = s * D + legs[lj];
      double v = Nj[(size_t)col * m + row];
      v *= inv_or_zero(leg_w(g, a.lam, j, oj[0], legs[oj[0]])) * inv_or_zero(leg_w(g, a.lam, j, oj[1], legs[oj[1]])) *
           inv_or_zero(leg_w(g, a.lam, j, oj[2], legs[oj[2]]));
      a.Gam[((size_t)j * 2) * D4 + e] = v;
    }
  }
}

// A_i = Gamma_i times sqrt(lam) on each of its bonds, scaled to unit norm per
// site (one CTA per site).
__global__ void __launch_bounds__(kT) k_su_to_peps(Geom g, const double* Gam, const double* lam, double* A) {
  __shared__ double red[kW];
  const int i = blockIdx.x, D = g.D, D4 = D * D * D * D;
  const double* G = Gam + (size_t)i * 2 * D4;
  double* out = A + (size_t)i * 2 * D4;
  double s2 = 0.0;
  for (int e = threadIdx.x; e < 2 * D4; e += blockDim.x) {
    const int w = e % D4;
    const int legs[4] = {w / (D * D * D), w / (D * D) % D, w / D % D, w % D};
    double v = G[e];
    for (int leg = 0; leg < 4; ++leg) {
      const int b = bond_of(g, i, leg);
      if (b >= 0) v *= sqrt(lam[(size_t)b * D + legs[leg]]);
      else if (legs[leg] != 0) v = 0.0;
    }
    out[e] = v;
    s2 += v * v;
  }
  s2 = block_sum_d(s2, red);
  const double inv = s2 > 0.0 ? 1.0 / sqrt(s2) : 0.0;
  for (int e = threadIdx.x; e < 2 * D4; e += blockDim.x) out[e] *= inv;
}

// *out = max |a - b| / max |a| as two non-negative maxima (bit patterns of
// non-negative doubles order like their values).
__global__ void k_su_change(const double* a, const double* b, size_t n, unsigned long long* out) {
  double d = 0.0, m = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    d = fmax(d, fabs(a[e] - b[e]));
    m = fmax(m, fabs(a[e]));
  }
  atomicMax(&out[0], (unsigned long long)__double_as_longlong(d));
  atomicMax(&out[1], (unsigned long long)__double_as_longlong(m));
}

}  // namespace su
}  // namespace peps

using namespace peps;

struct peps_su {
  su::Geom g;
  double J1 = 1.0, J2 = 0.0;
  cudaStream_t stream = nullptr;
  int nsm = 0;
  std::vector<std::pair<int, int>> launches;   // (offset, count) into ups, in Trotter order
  su::Upd* ups = nullptr;
  double* scratch = nullptr;
  size_t slot = 0;
  int max_count = 0;
  double* A0 = nullptr;
  double* A1 = nullptr;
  unsigned long long* chg = nullptr;
};

namespace {

peps_status su_fail(peps_status s, const std::string& msg) {
  set_last_error(msg.c_str());
  return s;
}

#define SU_CUDA(call)                                                                          \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return su_fail(e_ == cudaErrorMemoryAllocation ? PEPS_ENOMEM : PEPS_ECUDA,               \
                     std::string(#call) + ": " + cudaGetErrorString(e_));                       \
  } while (0)

}  // namespace

extern "C" {

peps_status peps_su_create(const peps_params* p, void* stream, peps_su** out) {
  if (!p || !out) return su_fail(PEPS_EINVAL, "null argument");
  if (p->Lx < 2 || p->Ly < 2 || p->Lx > kMaxL || p->Ly > kMaxL || p->D < 1 || p->D > 16 || p->d != 2)
    return su_fail(PEPS_EINVAL, "need 2 <= Lx, Ly <= 64, 1 <= D <= 16, d = 2");
  if (!std::isfinite(p->J1) || !std::isfinite(p->J2)) return su_fail(PEPS_EINVAL, "non-finite coupling");
  peps_su* s = new peps_su();
  s->g = {p->Lx, p->Ly, p->D, p->Ly * (p->Lx - 1)};
  s->J1 = p->J1;
  s->J2 = p->J2;
  s->stream = (cudaStream_t)stream;
  const int Lx = p->Lx, Ly = p->Ly;
  std::vector<su::Upd> ups;
  auto group = [&](const std::vector<su::Upd>& v) {
    if (v.empty()) return;
    s->launches.push_back({(int)ups.size(), (int)v.size()});
    s->max_count = std::max(s->max_count, (int)v.size());
    ups.insert(ups.end(), v.begin(), v.end());
  };
  // nearest-neighbour groups: horizontal even / odd columns, vertical even / odd rows
  for (int par = 0; par < 2; ++par) {
    std::vector<su::Upd> v;
    for (int r = 0; r < Ly; ++r)
      for (int c = par; c < Lx - 1; c += 2) v.push_back({r * Lx + c, r * Lx + c + 1, 0, 0});
    group(v);
  }
  for (int par = 0; par < 2; ++par) {
    std::vector<su::Upd> v;
    for (int r = par; r < Ly - 1; r += 2)
      for (int c = 0; c < Lx; ++c) v.push_back({r * Lx + c, (r + 1) * Lx + c, 0, 0});
    group(v);
  }
  if (p->J2 != 0.0) {
    // next-nearest pairs through a shared neighbour: SWAP(i, j), gate(j, k),
    // SWAP(i, j), one group per (kind, column parity, row parity)
    for (int kind = 0; kind < 2; ++kind)
      for (int cp = 0; cp < 2; ++cp)
        for (int rp = 0; rp < 2; ++rp) {
          std::vector<su::Upd> sw, gt;
          for (int r = rp; r < Ly - 1; r += 2)
            for (int c = cp; c < Lx - 1; c += 2) {
              const int a = r * Lx + c;
              int i, j, k;
              if (kind == 0) {
                i = a;
                j = a + 1;
                k = a + 1 + Lx;
              } else {
                i = a + 1;
                j = a;
                k = a + Lx;
              }
              sw.push_back({std::min(i, j), std::max(i, j), 2, 0});
              gt.push_back({std::min(j, k), std::max(j, k), 1, 0});
            }
          group(sw);
          group(gt);
          group(sw);
        }
  }
  const int D = p->D, m = D * D * D, n = 2 * D;
  s->slot = (size_t)4 * m * n;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, dev);
  const size_t N = (size_t)Lx * Ly, D4 = (size_t)D * D * D * D;
  cudaError_t e = cudaMalloc((void**)&s->ups, sizeof(su::Upd) * ups.size());
  if (e == cudaSuccess) e = cudaMemcpy(s->ups, ups.data(), sizeof(su::Upd) * ups.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc((void**)&s->scratch, sizeof(double) * s->slot * s->max_count);
  if (e == cudaSuccess) e = cudaMalloc((void**)&s->A0, sizeof(double) * N * 2 * D4);
  if (e == cudaSuccess) e = cudaMalloc((void**)&s->A1, sizeof(double) * N * 2 * D4);
  if (e == cudaSuccess) e = cudaMalloc((void**)&s->chg, 2 * sizeof(unsigned long long));
  const size_t smem = su::smem_doubles(D) * sizeof(double);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(su::k_su_bond, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) {
    peps_su_destroy(s);
    return su_fail(e == cudaErrorMemoryAllocation ? PEPS_ENOMEM : PEPS_ECUDA,
                   std::string("simple-update set-up: ") + cudaGetErrorString(e));
  }
  *out = s;
  return PEPS_OK;
}

peps_status peps_su_destroy(peps_su* s) {
  if (!s) return PEPS_OK;
  if (s->stream) cudaStreamSynchronize(s->stream);
  else cudaDeviceSynchronize();
  cudaFree(s->ups);
  cudaFree(s->scratch);
  cudaFree(s->A0);
  cudaFree(s->A1);
  cudaFree(s->chg);
  delete s;
  return PEPS_OK;
}

peps_status peps_su_to_peps(peps_su* s, const double* Gam_dev, const double* lam_dev, double* A_dev) {
  if (!s || !Gam_dev || !lam_dev || !A_dev) return su_fail(PEPS_EINVAL, "null argument");
  su::k_su_to_peps<<<s->g.Lx * s->g.Ly, su::kT, 0, s->stream>>>(s->g, Gam_dev, lam_dev, A_dev);
  SU_CUDA(cudaGetLastError());
  return PEPS_OK;
}

peps_status peps_su_evolve(peps_su* s, double* Gam_dev, double* lam_dev, double dtau, int nsteps,
                           double* change_host) {
  if (!s || !Gam_dev || !lam_dev) return su_fail(PEPS_EINVAL, "null argument");
  if (!std::isfinite(dtau) || dtau < 0.0 || nsteps < 0) return su_fail(PEPS_EINVAL, "need dtau >= 0, nsteps >= 0");
  su::Args a;
  a.g = s->g;
  a.Gam = Gam_dev;
  a.lam = lam_dev;
  a.J1 = s->J1;
  a.J2 = s->J2;
  a.dtau = dtau;
  a.scratch = s->scratch;
  a.slot = s->slot;
  const size_t smem = su::smem_doubles(s->g.D) * sizeof(double);
  const size_t nA = (size_t)s->g.Lx * s->g.Ly * 2 * s->g.D * s->g.D * s->g.D * s->g.D;
  for (int step = 0; step < nsteps; ++step) {
    const bool last = step == nsteps - 1 && change_host;
    if (last) {
      su::k_su_to_peps<<<s->g.Lx * s->g.Ly, su::kT, 0, s->stream>>>(s->g, Gam_dev, lam_dev, s->A0);
      SU_CUDA(cudaGetLastError());
    }
    for (auto& l : s->launches) {
      a.ups = s->ups + l.first;
      su::k_su_bond<<<l.second, su::kT, smem, s->stream>>>(a);
      SU_CUDA(cudaGetLastError());
    }
    if (last) {
      su::k_su_to_peps<<<s->g.Lx * s->g.Ly, su::kT, 0, s->stream>>>(s->g, Gam_dev, lam_dev, s->A1);
      SU_CUDA(cudaGetLastError());
      SU_CUDA(cudaMemsetAsync(s->chg, 0, 2 * sizeof(unsigned long long), s->stream));
      su::k_su_change<<<s->nsm * 4, su::kT, 0, s->stream>>>(s->A1, s->A0, nA, s->chg);
      SU_CUDA(cudaGetLastError());
      unsigned long long h[2] = {0, 0};
      SU_CUDA(cudaMemcpyAsync(h, s->chg, sizeof(h), cudaMemcpyDeviceToHost, s->stream));
      SU_CUDA(cudaStreamSynchronize(s->stream));
      double d, m;
      std::memcpy(&d, &h[0], 8);
      std::memcpy(&m, &h[1], 8);
      *change_host = m > 0.0 ? d / m : 0.0;
    }
  }
  if (nsteps == 0 && change_host) *change_host = 0.0;
  return PEPS_OK;
}

}  // extern "C"
