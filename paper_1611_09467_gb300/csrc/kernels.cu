// CUDA kernels of the PEPS sampling path (sm_103a).
//
//   k_boundary : boundary-MPS sweeps (Fig. 1d): top-down U_r (gives ln|psi|,
//                sign) and bottom-up L_r, alternating zip-up with truncation
//                to Dc.  One CTA per (configuration, sweep direction).
//   k_row      : single-row sandwiches <U_{r-1}| row r |L_{r+1}>: W_r,
//                amplitude ratios of horizontal spin exchanges, Delta = B/W
//                (Sec. II).  One CTA per (configuration, row).  k_row_fused
//                is the same with every intermediate in shared memory, for
//                (D, Dc) = (2,4), (4,8), (6,12), (8,16).
//   k_pair     : two-row sandwiches <U_{r-1}| rows r,r+1 |L_{r+2}>: ratios
//                of vertical and diagonal exchanges.  One CTA per
//                (configuration, row pair).
//   k_finalize : E(S) = diagonal + sum of (J/2) ratios (Sec. II with the
//                Hamiltonian of Sec. IV), status.
//   k_grad_*   : sums of O and E*O over configurations for
//                dE/dA = 2<Delta E> - 2<Delta><E> (Sec. II).
//   k_mc       : Metropolis sweeps over nearest-neighbour spin exchanges.
//
// Kernels are persistent over work items (grid-stride), so the per-CTA
// scratch slots bound the workspace.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/peps.h"

#include "device.cuh"
#include "kernels.h"
#include "pair_fused.cuh"
#include "row_fused.cuh"
#include "pair_tc.cuh"

namespace peps {

__device__ __forceinline__ int spin_of(const uint64_t* sp, int i) { return (int)((sp[i >> 6] >> (i & 63)) & 1ull); }

template <typename R>
__device__ __forceinline__ const R* tptr(const KArgs<R>& a, int site, int s) {
  const size_t D4 = (size_t)a.g.D * a.g.D * a.g.D * a.g.D;
  return a.A + ((size_t)site * 2 + s) * D4;
}

struct TDims {
  int l, r, u, d;
};
__device__ __forceinline__ TDims tdims(const Geometry& g, int row, int col) {
  TDims t;
  t.l = col == 0 ? 1 : g.D;
  t.r = col == g.Lx - 1 ? 1 : g.D;
  t.u = row == 0 ? 1 : g.D;
  t.d = row == g.Ly - 1 ? 1 : g.D;
  return t;
}

// Kernels with large shared-memory footprints ask for the maximum carve-out so
// the occupancy the grids are sized for is the one the hardware grants.
template <typename F>
static cudaError_t prefer_shared(F* f, size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  return e;
}

// ---------------------------------------------------------------- layouts
size_t wm_smem_bytes(const Geometry& g, size_t elem) {
  const size_t P = (size_t)g.Dc * g.D;
  return P * (P + 1) * elem;
}

// Dynamic shared memory of a kernel: a region of reals followed by the GEMM
// offset tables.  For the kernels that truncate, the reals hold (truncation
// matrix if it fits) + the two singular-vector blocks during a truncation and
// the GEMM tiles otherwise; the two uses are never live together.
__host__ __device__ inline size_t trunc_smem_reals(const Geometry& g, bool wm_in_smem) {
  const size_t P = (size_t)g.Dc * g.D;
  return (wm_in_smem ? P * (P + 1) : 0) + 2 * P * (size_t)g.Dc;
}

__host__ __device__ inline size_t reals_region_bytes(const Geometry& g, size_t elem, bool truncates, bool wm_in_smem) {
  size_t r = (size_t)kGemmSmemReals;
  if (truncates) {
    const size_t t = trunc_smem_reals(g, wm_in_smem);
    r = r > t ? r : t;
  }
  return (r * elem + 15) / 16 * 16;
}

size_t dyn_smem_bytes(const Geometry& g, size_t elem, bool truncates, bool wm_in_smem) {
  return reals_region_bytes(g, elem, truncates, wm_in_smem) + (size_t)kGemmSmemInts * sizeof(int);
}

bool wm_fits_smem(const Geometry& g, size_t elem) {
  return dyn_smem_bytes(g, elem, true, true) <= 200 * 1024;
}

template <typename R>
__device__ __forceinline__ void smem_split(unsigned char* raw, const Geometry& g, bool truncates, bool wm_in_smem,
                                           R*& reals, int*& ints) {
  reals = reinterpret_cast<R*>(raw);
  ints = reinterpret_cast<int*>(raw + reals_region_bytes(g, sizeof(R), truncates, wm_in_smem));
}

static size_t zip_elems(const Geometry& g, bool wm_in_smem) {
  const size_t Dc = g.Dc, D = g.D, P = Dc * D;
  return 2 * Dc * Dc * D + Dc * Dc * D * D + P * P + trunc_ws_elems((int)P, g.Dc, !wm_in_smem);
}

size_t boundary_slot_elems(const Geometry& g, bool wm_in_smem) {
  const size_t envT = (size_t)g.Dc * g.D * g.Dc;
  return zip_elems(g, wm_in_smem) + (size_t)g.Lx * envT;
}

__host__ __device__ inline size_t tmp_elems(const Geometry& g) {
  const size_t Dc = g.Dc, D = g.D;
  return Dc * Dc * D * D * D;
}

size_t row_slot_elems(const Geometry& g) {
  const size_t envT = (size_t)g.Dc * g.D * g.Dc, D4 = (size_t)g.D * g.D * g.D * g.D;
  return (size_t)(g.Lx + 1) * envT + 4 * envT + D4 + 2 * tmp_elems(g);
}

size_t pair_slot_elems(const Geometry& g) {
  const size_t envT2 = (size_t)g.Dc * g.D * g.D * g.Dc;
  return (size_t)(g.Lx + 1) * envT2 + 4 * envT2 + 2 * tmp_elems(g);
}

size_t mc_slot_elems(const Geometry& g, bool wm_in_smem) {
  const size_t envT = (size_t)g.Dc * g.D * g.Dc;
  const size_t sand = row_slot_elems(g) > pair_slot_elems(g) ? row_slot_elems(g) : pair_slot_elems(g);
  return (size_t)g.Ly * g.Lx * envT + 2 * (size_t)g.Lx * envT + zip_elems(g, wm_in_smem) + sand;
}

// ------------------------------------------------------------ zip-up row
// Absorbs row `row` (spins `sp`) into the boundary MPS `Min` (padded
// [Lx][Dc][D][Dc], bond dims bdin), writing `Mout` (bond dims bdout).
// dir 0: the MPS faces the row's up legs (top-down sweep); dir 1: down legs.
// Returns ln of the norm divided out of the last tensor (Fig. 1d with the
// per-row normalisation that keeps the log scale).
template <typename R>
struct ZipBufs {
  R* C0;
  R* C1;
  R* Y;
  R* X;
  double* dred;   // >= kWarps doubles of shared memory
  R* gsm;         // GEMM shared scratch
  int* gism;
  TruncWork<R> tw;
};

template <typename R>
__device__ double absorb_row(const KArgs<R>& a, const R* Min, R* Mout, int row, int dir, bool lr, const int* bdin,
                        const uint64_t* sp, ZipBufs<R>& zb, R* red) {
  const Geometry& g = a.g;
  const int D = g.D, Dc = g.Dc, Lx = g.Lx;
  const int envT = Dc * D * Dc;
  const int D3 = D * D * D, DD = D * D;
  const int sl = D3, sr = DD;
  const int si = dir == 0 ? D : 1, so = dir == 0 ? 1 : D;
  for (int e = threadIdx.x; e < Lx * envT; e += blockDim.x) Mout[e] = R(0);
  R* Cc = zb.C0;
  R* Cn = zb.C1;
  if (threadIdx.x == 0) Cc[0] = R(1);
  __syncthreads();
  int kcur = 1;
  int last;
  if (lr) {
    for (int c = 0; c < Lx; ++c) {
      const TDims td = tdims(g, row, c);
      ZipDims z;
      z.k = kcur; z.a = bdin[c]; z.b = bdin[c + 1];
      z.i = dir == 0 ? td.u : td.d;
      z.l = td.l; z.r = td.r;
      z.o = dir == 0 ? td.d : td.u;
      const R* T = tptr(a, row * Lx + c, spin_of(sp, row * Lx + c));
      cta_gemm<R>(zip_lr_step(0, z, D, Dc, sl, sr, si, so), Cc, Min + (size_t)c * envT, zb.Y, false, zb.gsm, zb.gism);
      cta_gemm<R>(zip_lr_step(1, z, D, Dc, sl, sr, si, so), zb.Y, T, zb.X, false, zb.gsm, zb.gism);
      const int m = z.k * z.o, n = z.b * z.r;
      if (c < Lx - 1) {
        const int K = min(Dc, min(m, n));
        cta_topk_left<R>(zb.X, m, n, K, zb.tw, Mout + (size_t)c * envT, ix2(z.o, D * Dc, Dc), ix1(1), Cn,
                         ix1(n), ix1(1));
        R* t = Cc; Cc = Cn; Cn = t;
        kcur = K;
      } else {
        for (int e = threadIdx.x; e < m; e += blockDim.x) {
          const int k = e / z.o, o = e % z.o;
          Mout[(size_t)c * envT + k * D * Dc + o * Dc] = zb.X[e];
        }
        __syncthreads();
      }
    }
    last = Lx - 1;
  } else {
    for (int c = Lx - 1; c >= 0; --c) {
      const TDims td = tdims(g, row, c);
      ZipDims z;
      z.k = kcur; z.a = bdin[c]; z.b = bdin[c + 1];
      z.i = dir == 0 ? td.u : td.d;
      z.l = td.l; z.r = td.r;
      z.o = dir == 0 ? td.d : td.u;
      const R* T = tptr(a, row * Lx + c, spin_of(sp, row * Lx + c));
      cta_gemm<R>(zip_rl_step(0, z, D, Dc, sl, sr, si, so), Min + (size_t)c * envT, Cc, zb.Y, false, zb.gsm, zb.gism);
      cta_gemm<R>(zip_rl_step(1, z, D, Dc, sl, sr, si, so), zb.Y, T, zb.X, false, zb.gsm, zb.gism);
      const int m = z.o * z.k, n = z.a * z.l;
      if (c > 0) {
        const int K = min(Dc, min(m, n));
        cta_topk_left<R>(zb.X, m, n, K, zb.tw, Mout + (size_t)c * envT, ix2(z.k, Dc, 1), ix1(D * Dc), Cn,
                         ix1(1), ix1(K));
        R* t = Cc; Cc = Cn; Cn = t;
        kcur = K;
      } else {
        for (int e = threadIdx.x; e < m; e += blockDim.x) {
          const int o = e / z.k, k = e % z.k;
          Mout[o * Dc + k] = zb.X[e];
        }
        __syncthreads();
      }
    }
    last = 0;
  }
  // the norm is accumulated in FP64 in every precision: ln n enters ln|psi| directly
  double ss = 0.0;
  R* Ml = Mout + (size_t)last * envT;
  for (int e = threadIdx.x; e < envT; e += blockDim.x) ss += (double)Ml[e] * (double)Ml[e];
  ss = block_sum(ss, zb.dred);
  const double nrm = sqrt(ss);
  if (nrm > 0.0) {
    const R inv = (R)(1.0 / nrm);
    for (int e = threadIdx.x; e < envT; e += blockDim.x) Ml[e] *= inv;
  }
  __syncthreads();
  return nrm;
}

template <typename R>
__device__ void carve_zip(const Geometry& g, R*& p, ZipBufs<R>& zb, R* wm_smem, R* red, double* dred, R* wv,
                          R* gsm, int* gism) {
  zb.dred = dred;
  zb.gsm = gsm;
  zb.gism = gism;
  zb.tw.wv = wv;
  zb.tw.gsm = gsm;
  zb.tw.gism = gism;
  const size_t Dc = g.Dc, D = g.D, P = Dc * D;
  zb.C0 = p; p += Dc * Dc * D;
  zb.C1 = p; p += Dc * Dc * D;
  zb.Y = p; p += Dc * Dc * D * D;
  zb.X = p; p += P * P;
  TruncWork<R>& w = zb.tw;
  w.ldw = (int)P + 1;
  w.Wg = p; p += P * (P + 1);
  R* sh = gsm;   // shared reals region: [Wm][Ubs][Uks]
  if (wm_smem) {
    w.Wm = sh;
    sh += P * (P + 1);
  } else {
    w.Wm = p; p += P * (P + 1);
  }
  w.Ubs = sh; sh += P * Dc;
  w.Uks = sh;
  w.Qmax = (int)P;
  w.tau = p; p += 4 * P;
  w.t = p; p += 2 * P;
  w.t2 = p; p += 2 * P;
  w.lam = p; p += Dc;
  w.Z = p; p += Dc * 2 * P;
  w.lu = p; p += Dc * 6 * 2 * P;
  w.Ub = p; p += P * Dc;
  w.Uk = p; p += P * Dc;
  p += 64;
  w.red = red;
}

// ------------------------------------------------------------ k_boundary
template <typename R>
__global__ void __launch_bounds__(kThreads) k_boundary(KArgs<R> a, int dirs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ R red[64];
  __shared__ uint64_t sp[kMaxWords];
  __shared__ int ones[kMaxDcD + 1];
  const Geometry& g = a.g;
  const int Lx = g.Lx, Ly = g.Ly, Dc = g.Dc, D = g.D;
  const size_t envT = (size_t)Dc * D * Dc;
  R* p = a.scratch + (size_t)blockIdx.x * a.slot_elems;
  ZipBufs<R> zb;
  __shared__ double dred[kWarps];
  __shared__ R wv[kMaxDcD];
  R* gsm;
  int* gism;
  smem_split<R>(smem_raw, g, true, a.smem_wm != 0, gsm, gism);
  carve_zip<R>(g, p, zb, a.smem_wm ? gsm : nullptr, red, dred, wv, gsm, gism);
  R* lastbuf = p;
  for (int i = threadIdx.x; i <= Lx; i += blockDim.x) ones[i] = 1;
  for (int item = blockIdx.x; item < a.n * dirs; item += gridDim.x) {
    const int cfg = item / dirs, dir = item % dirs;
    __syncthreads();
    for (int i = threadIdx.x; i < g.nwords; i += blockDim.x) sp[i] = a.S[(size_t)cfg * g.nwords + i];
    __syncthreads();
    const R* Min = a.triv_mps;
    double ls = 0.0;
    bool zero = false;
    for (int j = 0; j < Ly; ++j) {
      const int r = dir == 0 ? j : Ly - 1 - j;
      if (dir == 1 && r == 0) break;
      R* Mout;
      if (dir == 0) Mout = r <= Ly - 2 ? a.envU + ((size_t)cfg * Ly + r) * Lx * envT : lastbuf;
      else Mout = a.envL + ((size_t)cfg * Ly + r) * Lx * envT;
      const int* bdin = j == 0 ? ones : a.bd + ((size_t)dir * Ly + (j - 1)) * (Lx + 1);
      const double nrm = absorb_row<R>(a, Min, Mout, r, dir, (j % 2) == 0, bdin, sp, zb, red);
      if (!(nrm > 0.0)) zero = true;
      else ls += log(nrm);
      Min = Mout;
    }
    if (dir == 0) {
      // All physical legs are one now: close the chain of matrices M_c[:, 0, :].
      __shared__ R vec[kMaxDc], nv[kMaxDc];
      if (threadIdx.x == 0) {
        const int* bdl = a.bd + ((size_t)0 * Ly + (Ly - 1)) * (Lx + 1);
        vec[0] = R(1);
        int na = 1;
        for (int c = 0; c < Lx; ++c) {
          const int nb = bdl[c + 1];
          const R* M = lastbuf + (size_t)c * envT;
          for (int b = 0; b < nb; ++b) {
            R s = R(0);
            for (int x = 0; x < na; ++x) s += vec[x] * M[(size_t)x * D * Dc + b];
            nv[b] = s;
          }
          for (int b = 0; b < nb; ++b) vec[b] = nv[b];
          na = nb;
        }
        const R v = vec[0];
        if (zero || v == R(0)) {
          a.logabs[cfg] = -INFINITY;
          a.sign[cfg] = 0;
          atomicOr(&a.flags[cfg], kFlagZeroW);
        } else {
          a.logabs[cfg] = ls + log(fabs((double)v));
          a.sign[cfg] = v > R(0) ? 1 : -1;
        }
      }
    } else if (zero && threadIdx.x == 0) {
      atomicOr(&a.flags[cfg], kFlagZeroW);
    }
  }
}

template <typename R>
__device__ R block_dot(const R* x, const R* y, int n, R* red) {
  R s = R(0);
  for (int e = threadIdx.x; e < n; e += blockDim.x) s += x[e] * y[e];
  return block_sum(s, red);
}

// ----------------------------------------------------------------- k_row
template <typename R>
__global__ void __launch_bounds__(kThreads) k_row(KArgs<R> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ R red[64];
  __shared__ uint64_t sp[kMaxWords];
  const Geometry& g = a.g;
  const int Lx = g.Lx, Ly = g.Ly, Dc = g.Dc, D = g.D;
  const int envT = Dc * D * Dc, D4 = D * D * D * D;
  R* gsm;
  int* gism;
  smem_split<R>(smem_raw, g, false, false, gsm, gism);
  R* p = a.scratch + (size_t)blockIdx.x * a.slot_elems;
  R* Gb = p; p += (size_t)(Lx + 1) * envT;
  R* F0 = p; p += envT;
  R* F1 = p; p += envT;
  R* X1 = p; p += envT;
  R* X2 = p; p += envT;
  R* Bb = p; p += D4;
  R* t0 = p; p += tmp_elems(g);
  R* t1 = p;
  __shared__ int eG[kMaxL + 1];   // G_c is stored scaled by 2^-eG[c]
  for (int item = blockIdx.x; item < a.n * Ly; item += gridDim.x) {
    const int cfg = item / Ly, r = item % Ly;
    __syncthreads();
    for (int i = threadIdx.x; i < g.nwords; i += blockDim.x) sp[i] = a.S[(size_t)cfg * g.nwords + i];
    for (int e = threadIdx.x; e < envT; e += blockDim.x) Gb[(size_t)Lx * envT + e] = a.triv_t1[e];
    if (threadIdx.x == 0) eG[Lx] = 0;
    __syncthreads();
    const R* Mu = r == 0 ? a.triv_mps : a.envU + ((size_t)cfg * Ly + (r - 1)) * Lx * envT;
    const R* Md = r == Ly - 1 ? a.triv_mps : a.envL + ((size_t)cfg * Ly + (r + 1)) * Lx * envT;
    int eacc = 0;
    for (int c = Lx - 1; c >= 0; --c) {
      const int site = r * Lx + c;
      run_op<R>(OP_COL1_RIGHT, D, Dc, Gb + (size_t)(c + 1) * envT, Mu + (size_t)c * envT,
                tptr(a, site, spin_of(sp, site)), Md + (size_t)c * envT, nullptr, Gb + (size_t)c * envT, t0, t1, gsm, gism);
      eacc += normalize_pow2(Gb + (size_t)c * envT, envT, red);
      if (threadIdx.x == 0) eG[c] = eacc;
    }
    const R W = Gb[0];
    const bool ok = W != R(0);
    double eh = 0.0;
    const R* F = a.triv_t1;
    int eF = 0;   // F is stored scaled by 2^-eF
    R* Fn = F0;
    for (int c = 0; c < Lx; ++c) {
      const int site = r * Lx + c;
      const int s = spin_of(sp, site);
      if (a.O != nullptr) {
        run_op<R>(OP_SITE_ENV, D, Dc, F, Mu + (size_t)c * envT, Md + (size_t)c * envT,
                  Gb + (size_t)(c + 1) * envT, nullptr, Bb, t0, t1, gsm, gism);
        R* Oo = a.O + ((size_t)cfg * g.N + site) * D4;
        const R inv = ok ? (R)ldexp(1.0 / (double)W, eF + eG[c + 1] - eG[0]) : R(0);
        for (int e = threadIdx.x; e < D4; e += blockDim.x) Oo[e] = Bb[e] * inv;
      }
      if (c < Lx - 1) {
        const int s2 = spin_of(sp, site + 1);
        if (s != s2) {
          run_op<R>(OP_COL1_LEFT, D, Dc, F, Mu + (size_t)c * envT, tptr(a, site, s2), Md + (size_t)c * envT,
                    nullptr, X1, t0, t1, gsm, gism);
          const int eX = normalize_pow2(X1, envT, red);
          run_op<R>(OP_COL1_LEFT, D, Dc, X1, Mu + (size_t)(c + 1) * envT, tptr(a, site + 1, s),
                    Md + (size_t)(c + 1) * envT, nullptr, X2, t0, t1, gsm, gism);
          const R wp = block_dot(X2, Gb + (size_t)(c + 2) * envT, envT, red);
          if (ok) eh += 0.5 * g.J1 * ldexp((double)wp / (double)W, eF + eX + eG[c + 2] - eG[0]);
        }
        run_op<R>(OP_COL1_LEFT, D, Dc, F, Mu + (size_t)c * envT, tptr(a, site, s), Md + (size_t)c * envT,
                  nullptr, Fn, t0, t1, gsm, gism);
        eF += normalize_pow2(Fn, envT, red);
        F = Fn;
        Fn = (Fn == F0) ? F1 : F0;
      }
    }
    if (threadIdx.x == 0) {
      a.eloc_h[(size_t)cfg * Ly + r] = eh;
      a.w_row[(size_t)cfg * Ly + r] = (double)W;
      if (!ok) atomicOr(&a.flags[cfg], kFlagZeroW);
    }
  }
}

// ------------------------------------------------------------- k_row_fused
// k_row with the fused shared-memory step and site environment
// (row_fused.cuh) for a fixed (D, Dc).  Transfers are stored [x'][x][y].
template <typename R, int D, int Dc>
__global__ void __launch_bounds__(kThreads) k_row_fused(KArgs<R> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ R red[64];
  __shared__ uint64_t sp[kMaxWords];
  R* sm = reinterpret_cast<R*>(smem_raw);
  const Geometry& g = a.g;
  const int Lx = g.Lx, Ly = g.Ly;
  constexpr int envT = Dc * D * Dc, D4 = D * D * D * D;
  R* p = a.scratch + (size_t)blockIdx.x * a.slot_elems;
  R* Gb = p; p += (size_t)(Lx + 1) * envT;
  R* F0 = p; p += envT;
  R* F1 = p; p += envT;
  R* X1 = p;
  __shared__ int eG[kMaxL + 1];   // G_c is stored scaled by 2^-eG[c]
  for (int item = blockIdx.x; item < a.n * Ly; item += gridDim.x) {
    const int cfg = item / Ly, r = item % Ly;
    __syncthreads();
    for (int i = threadIdx.x; i < g.nwords; i += blockDim.x) sp[i] = a.S[(size_t)cfg * g.nwords + i];
    for (int e = threadIdx.x; e < envT; e += blockDim.x) Gb[(size_t)Lx * envT + e] = a.triv_t1[e];
    if (threadIdx.x == 0) eG[Lx] = 0;
    __syncthreads();
    const R* Mu = r == 0 ? a.triv_mps : a.envU + ((size_t)cfg * Ly + (r - 1)) * Lx * envT;
    const R* Md = r == Ly - 1 ? a.triv_mps : a.envL + ((size_t)cfg * Ly + (r + 1)) * Lx * envT;
    int eacc = 0;
    for (int c = Lx - 1; c >= 0; --c) {
      const int site = r * Lx + c;
      int e = 0;
      row_step_fused<R, D, Dc>(true, Gb + (size_t)(c + 1) * envT, Gb + (size_t)c * envT, Mu + (size_t)c * envT,
                               tptr(a, site, spin_of(sp, site)), Md + (size_t)c * envT, nullptr, sm, red, &e);
      eacc += e;
      if (threadIdx.x == 0) eG[c] = eacc;
    }
    const R W = Gb[0];
    const bool ok = W != R(0);
    double eh = 0.0;
    const R* F = a.triv_t1;
    int eF = 0;   // F is stored scaled by 2^-eF
    R* Fn = F0;
    for (int c = 0; c < Lx; ++c) {
      const int site = r * Lx + c;
      const int s = spin_of(sp, site);
      const R* Muc = Mu + (size_t)c * envT;
      const R* Mdc = Md + (size_t)c * envT;
      if (a.O != nullptr)
        site_env_fused<R, D, Dc>(F, Muc, Mdc, Gb + (size_t)(c + 1) * envT,
                                 ok ? (R)ldexp(1.0 / (double)W, eF + eG[c + 1] - eG[0]) : R(0),
                                 a.O + ((size_t)cfg * g.N + site) * D4, sm);
      if (c < Lx - 1) {
        const int s2 = spin_of(sp, site + 1);
        if (s != s2) {
          int eX = 0;
          row_step_fused<R, D, Dc>(false, F, X1, Muc, tptr(a, site, s2), Mdc, nullptr, sm, red, &eX);
          const R wp = row_step_fused<R, D, Dc>(false, X1, nullptr, Mu + (size_t)(c + 1) * envT, tptr(a, site + 1, s),
                                                Md + (size_t)(c + 1) * envT, Gb + (size_t)(c + 2) * envT, sm, red);
          if (ok) eh += 0.5 * g.J1 * ldexp((double)wp / (double)W, eF + eX + eG[c + 2] - eG[0]);
        }
        int e1 = 0;
        row_step_fused<R, D, Dc>(false, F, Fn, Muc, tptr(a, site, s), Mdc, nullptr, sm, red, &e1);
        eF += e1;
        F = Fn;
        Fn = (Fn == F0) ? F1 : F0;
      }
    }
    if (threadIdx.x == 0) {
      a.eloc_h[(size_t)cfg * Ly + r] = eh;
      a.w_row[(size_t)cfg * Ly + r] = (double)W;
      if (!ok) atomicOr(&a.flags[cfg], kFlagZeroW);
    }
  }
}

// ---------------------------------------------------------------- k_pair
template <typename R>
__global__ void __launch_bounds__(kThreads) k_pair(KArgs<R> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ R red[64];
  __shared__ uint64_t sp[kMaxWords];
  const Geometry& g = a.g;
  const int Lx = g.Lx, Ly = g.Ly, Dc = g.Dc, D = g.D;
  const int envT = Dc * D * Dc, envT2 = Dc * D * D * Dc;
  R* gsm;
  int* gism;
  smem_split<R>(smem_raw, g, false, false, gsm, gism);
  R* p = a.scratch + (size_t)blockIdx.x * a.slot_elems;
  R* Hb = p; p += (size_t)(Lx + 1) * envT2;
  R* E0 = p; p += envT2;
  R* E1 = p; p += envT2;
  R* X1 = p; p += envT2;
  R* X2 = p; p += envT2;
  R* t0 = p; p += tmp_elems(g);
  R* t1 = p;
  const int npairs = Ly - 1;
  __shared__ int eH[kMaxL + 1];   // H_c is stored scaled by 2^-eH[c]
  for (int item = blockIdx.x; item < a.n * npairs; item += gridDim.x) {
    const int cfg = item / npairs, r = item % npairs;
    __syncthreads();
    for (int i = threadIdx.x; i < g.nwords; i += blockDim.x) sp[i] = a.S[(size_t)cfg * g.nwords + i];
    for (int e = threadIdx.x; e < envT2; e += blockDim.x) Hb[(size_t)Lx * envT2 + e] = a.triv_t2[e];
    if (threadIdx.x == 0) eH[Lx] = 0;
    __syncthreads();
    const R* Mu = r == 0 ? a.triv_mps : a.envU + ((size_t)cfg * Ly + (r - 1)) * Lx * envT;
    const R* Md = r + 2 > Ly - 1 ? a.triv_mps : a.envL + ((size_t)cfg * Ly + (r + 2)) * Lx * envT;
    int eacc = 0;
    for (int c = Lx - 1; c >= 0; --c) {
      const int s1 = r * Lx + c, s2 = (r + 1) * Lx + c;
      run_op<R>(OP_COL2_RIGHT, D, Dc, Hb + (size_t)(c + 1) * envT2, Mu + (size_t)c * envT,
                tptr(a, s1, spin_of(sp, s1)), tptr(a, s2, spin_of(sp, s2)), Md + (size_t)c * envT,
                Hb + (size_t)c * envT2, t0, t1, gsm, gism);
      eacc += normalize_pow2(Hb + (size_t)c * envT2, envT2, red);
      if (threadIdx.x == 0) eH[c] = eacc;
    }
    const R W = Hb[0];
    const bool ok = W != R(0);
    double ev = 0.0;
    const R* E = a.triv_t2;
    int eE = 0;   // E is stored scaled by 2^-eE
    R* En = E0;
    for (int c = 0; c < Lx; ++c) {
      const int i1 = r * Lx + c, i2 = (r + 1) * Lx + c;
      const int a1 = spin_of(sp, i1), a2 = spin_of(sp, i2);
      const R* Muc = Mu + (size_t)c * envT;
      const R* Mdc = Md + (size_t)c * envT;
      if (a1 != a2) {  // vertical pair (r,c)-(r+1,c)
        run_op<R>(OP_COL2_LEFT, D, Dc, E, Muc, tptr(a, i1, a2), tptr(a, i2, a1), Mdc, X1, t0, t1, gsm, gism);
        const R wp = block_dot(X1, Hb + (size_t)(c + 1) * envT2, envT2, red);
        if (ok) ev += 0.5 * g.J1 * ldexp((double)wp / (double)W, eE + eH[c + 1] - eH[0]);
      }
      if (c < Lx - 1 && g.J2 != 0.0) {
        const int j1 = i1 + 1, j2 = i2 + 1;
        const int b1 = spin_of(sp, j1), b2 = spin_of(sp, j2);
        const R* Mun = Mu + (size_t)(c + 1) * envT;
        const R* Mdn = Md + (size_t)(c + 1) * envT;
        if (a1 != b2) {  // diagonal (r,c)-(r+1,c+1)
          run_op<R>(OP_COL2_LEFT, D, Dc, E, Muc, tptr(a, i1, b2), tptr(a, i2, a2), Mdc, X1, t0, t1, gsm, gism);
          const int eX = normalize_pow2(X1, envT2, red);
          run_op<R>(OP_COL2_LEFT, D, Dc, X1, Mun, tptr(a, j1, b1), tptr(a, j2, a1), Mdn, X2, t0, t1, gsm, gism);
          const R wp = block_dot(X2, Hb + (size_t)(c + 2) * envT2, envT2, red);
          if (ok) ev += 0.5 * g.J2 * ldexp((double)wp / (double)W, eE + eX + eH[c + 2] - eH[0]);
        }
        if (b1 != a2) {  // anti-diagonal (r,c+1)-(r+1,c)
          run_op<R>(OP_COL2_LEFT, D, Dc, E, Muc, tptr(a, i1, a1), tptr(a, i2, b1), Mdc, X1, t0, t1, gsm, gism);
          const int eX = normalize_pow2(X1, envT2, red);
          run_op<R>(OP_COL2_LEFT, D, Dc, X1, Mun, tptr(a, j1, a2), tptr(a, j2, b2), Mdn, X2, t0, t1, gsm, gism);
          const R wp = block_dot(X2, Hb + (size_t)(c + 2) * envT2, envT2, red);
          if (ok) ev += 0.5 * g.J2 * ldexp((double)wp / (double)W, eE + eX + eH[c + 2] - eH[0]);
        }
      }
      if (c < Lx - 1) {
        run_op<R>(OP_COL2_LEFT, D, Dc, E, Muc, tptr(a, i1, a1), tptr(a, i2, a2), Mdc, En, t0, t1, gsm, gism);
        eE += normalize_pow2(En, envT2, red);
        E = En;
        En = (En == E0) ? E1 : E0;
      }
    }
    if (threadIdx.x == 0) {
      a.eloc_v[(size_t)cfg * Ly + r] = ev;
      if (!ok) atomicOr(&a.flags[cfg], kFlagZeroW);
    }
  }
}

// ------------------------------------------------------------ k_pair_fused
// k_pair with the fused shared-memory transfer step (pair_fused.cuh) for a
// fixed (D, Dc).  Transfers are stored [x'][x][y1][y2] (see pair_fused.cuh).
template <typename R, int D, int Dc>
__global__ void __launch_bounds__(kThreads) k_pair_fused(KArgs<R> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ R red[64];
  __shared__ uint64_t sp[kMaxWords];
  R* sm = reinterpret_cast<R*>(smem_raw);
  const Geometry& g = a.g;
  const int Lx = g.Lx, Ly = g.Ly;
  constexpr int envT = Dc * D * Dc, envT2 = Dc * D * D * Dc;
  R* p = a.scratch + (size_t)blockIdx.x * a.slot_elems;
  R* Hb = p; p += (size_t)(Lx + 1) * envT2;
  R* E0 = p; p += envT2;
  R* E1 = p; p += envT2;
  R* X1 = p;
  const int npairs = Ly - 1;
  __shared__ int eH[kMaxL + 1];   // H_c is stored scaled by 2^-eH[c]
  for (int item = blockIdx.x; item < a.n * npairs; item += gridDim.x) {
    const int cfg = item / npairs, r = item % npairs;
    __syncthreads();
    for (int i = threadIdx.x; i < g.nwords; i += blockDim.x) sp[i] = a.S[(size_t)cfg * g.nwords + i];
    for (int e = threadIdx.x; e < envT2; e += blockDim.x) Hb[(size_t)Lx * envT2 + e] = a.triv_t2[e];
    if (threadIdx.x == 0) eH[Lx] = 0;
    __syncthreads();
    const R* Mu = r == 0 ? a.triv_mps : a.envU + ((size_t)cfg * Ly + (r - 1)) * Lx * envT;
    const R* Md = r + 2 > Ly - 1 ? a.triv_mps : a.envL + ((size_t)cfg * Ly + (r + 2)) * Lx * envT;
    int eacc = 0;
    for (int c = Lx - 1; c >= 0; --c) {
      const int s1 = r * Lx + c, s2 = (r + 1) * Lx + c;
      int e = 0;
      pair_step_fused<R, D, Dc>(true, Hb + (size_t)(c + 1) * envT2, Hb + (size_t)c * envT2, Mu + (size_t)c * envT,
                                tptr(a, s1, spin_of(sp, s1)), tptr(a, s2, spin_of(sp, s2)), Md + (size_t)c * envT,
                                nullptr, sm, red, &e);
      eacc += e;
      if (threadIdx.x == 0) eH[c] = eacc;
    }
    const R W = Hb[0];
    const bool ok = W != R(0);
    double ev = 0.0;
    const R* E = a.triv_t2;
    int eE = 0;   // E is stored scaled by 2^-eE
    R* En = E0;
    for (int c = 0; c < Lx; ++c) {
      const int i1 = r * Lx + c, i2 = (r + 1) * Lx + c;
      const int a1 = spin_of(sp, i1), a2 = spin_of(sp, i2);
      const R* Muc = Mu + (size_t)c * envT;
      const R* Mdc = Md + (size_t)c * envT;
      if (a1 != a2) {  // vertical pair (r,c)-(r+1,c)
        const R wp = pair_step_fused<R, D, Dc>(false, E, nullptr, Muc, tptr(a, i1, a2), tptr(a, i2, a1), Mdc,
                                               Hb + (size_t)(c + 1) * envT2, sm, red);
        if (ok) ev += 0.5 * g.J1 * ldexp((double)wp / (double)W, eE + eH[c + 1] - eH[0]);
      }
      if (c < Lx - 1 && g.J2 != 0.0) {
        const int j1 = i1 + 1, j2 = i2 + 1;
        const int b1 = spin_of(sp, j1), b2 = spin_of(sp, j2);
        const R* Mun = Mu + (size_t)(c + 1) * envT;
        const R* Mdn = Md + (size_t)(c + 1) * envT;
        if (a1 != b2) {  // diagonal (r,c)-(r+1,c+1)
          int eX = 0;
          pair_step_fused<R, D, Dc>(false, E, X1, Muc, tptr(a, i1, b2), tptr(a, i2, a2), Mdc, nullptr, sm, red, &eX);
          const R wp = pair_step_fused<R, D, Dc>(false, X1, nullptr, Mun, tptr(a, j1, b1), tptr(a, j2, a1), Mdn,
                                                 Hb + (size_t)(c + 2) * envT2, sm, red);
          if (ok) ev += 0.5 * g.J2 * ldexp((double)wp / (double)W, eE + eX + eH[c + 2] - eH[0]);
        }
        if (b1 != a2) {  // anti-diagonal (r,c+1)-(r+1,c)
          int eX = 0;
          pair_step_fused<R, D, Dc>(false, E, X1, Muc, tptr(a, i1, a1), tptr(a, i2, b1), Mdc, nullptr, sm, red, &eX);
          const R wp = pair_step_fused<R, D, Dc>(false, X1, nullptr, Mun, tptr(a, j1, a2), tptr(a, j2, b2), Mdn,
                                                 Hb + (size_t)(c + 2) * envT2, sm, red);
          if (ok) ev += 0.5 * g.J2 * ldexp((double)wp / (double)W, eE + eX + eH[c + 2] - eH[0]);
        }
      }
      if (c < Lx - 1) {
        int e1 = 0;
        pair_step_fused<R, D, Dc>(false, E, En, Muc, tptr(a, i1, a1), tptr(a, i2, a2), Mdc, nullptr, sm, red, &e1);
        eE += e1;
        E = En;
        En = (En == E0) ? E1 : E0;
      }
    }
    if (threadIdx.x == 0) {
      a.eloc_v[(size_t)cfg * Ly + r] = ev;
      if (!ok) atomicOr(&a.flags[cfg], kFlagZeroW);
    }
  }
}

// ------------------------------------------------------------ k_pair_tc
// k_pair_fused with the tensor-core step (pair_tc.cuh), D = 8, Dc = 16, TF32
// inputs with FP32 accumulation.  Each CTA holds kTmemCols TMEM columns for
// its lifetime; a timed-out wait marks the configuration and ends the CTA
// after releasing TMEM.
__global__ void __launch_bounds__(kThreads, 2) k_pair_tc(KArgs<float> a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ float red[64];
  __shared__ uint64_t sp[kMaxWords];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ __align__(8) uint64_t tbar;
  __shared__ uint32_t tmem_holder;
  constexpr int D = 8, Dc = 16;
  float* sm = reinterpret_cast<float*>(smem_raw);
  const Geometry& g = a.g;
  const int Lx = g.Lx, Ly = g.Ly;
  constexpr int envT = Dc * D * Dc, envT2 = Dc * D * D * Dc;
  float* p = a.scratch + (size_t)blockIdx.x * a.slot_elems;
  float* Hb = p; p += (size_t)(Lx + 1) * envT2;
  float* E0 = p; p += envT2;
  float* E1 = p; p += envT2;
  float* X1 = p;
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(&tmem_holder)),
                 "r"(tc::kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc::smem_u32(&mbar)), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc::smem_u32(&tbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  PairTc st;
  st.tmem = tmem_holder;
  st.mbar = &mbar;
  st.tbar = &tbar;
  st.phase = 0;
  st.tphase = 0;
  st.ok = true;
  // B tiles of site i, spin s, direction dir (0 left, 1 right): TA at +0, TB at +kTcTile
  auto tile = [&](int dir, int i, int sp_) { return a.tcB + ((size_t)(dir * g.N + i) * 2 + sp_) * 2 * kTcTile; };
  const int npairs = Ly - 1;
  __shared__ int eH[kMaxL + 1];   // H_c is stored scaled by 2^-eH[c]
  for (int item = blockIdx.x; item < a.n * npairs && st.ok; item += gridDim.x) {
    const int cfg = item / npairs, r = item % npairs;
    __syncthreads();
    for (int i = threadIdx.x; i < g.nwords; i += blockDim.x) sp[i] = a.S[(size_t)cfg * g.nwords + i];
    for (int e = threadIdx.x; e < envT2; e += blockDim.x) Hb[(size_t)Lx * envT2 + e] = a.triv_t2[e];
    if (threadIdx.x == 0) eH[Lx] = 0;
    __syncthreads();
    const float* Mu = r == 0 ? a.triv_mps : a.envU + ((size_t)cfg * Ly + (r - 1)) * Lx * envT;
    const float* Md = r + 2 > Ly - 1 ? a.triv_mps : a.envL + ((size_t)cfg * Ly + (r + 2)) * Lx * envT;
    int eacc = 0;
    for (int c = Lx - 1; c >= 0; --c) {
      const int s1 = r * Lx + c, s2 = (r + 1) * Lx + c;
      int e = 0;
      pair_step_tc(st, true, Hb + (size_t)(c + 1) * envT2, Hb + (size_t)c * envT2, Mu + (size_t)c * envT,
                   tile(1, s1, spin_of(sp, s1)), tile(1, s2, spin_of(sp, s2)) + kTcTile, Md + (size_t)c * envT,
                   nullptr, sm, red, &e);
      eacc += e;
      if (threadIdx.x == 0) eH[c] = eacc;
    }
    __syncthreads();
    const float W = Hb[0];
    const bool ok = W != 0.f;
    double ev = 0.0;
    const float* E = a.triv_t2;
    int eE = 0;   // E is stored scaled by 2^-eE
    float* En = E0;
    for (int c = 0; c < Lx; ++c) {
      const int i1 = r * Lx + c, i2 = (r + 1) * Lx + c;
      const int a1 = spin_of(sp, i1), a2 = spin_of(sp, i2);
      const float* Muc = Mu + (size_t)c * envT;
      const float* Mdc = Md + (size_t)c * envT;
      if (a1 != a2) {
        const float wp = pair_step_tc(st, false, E, nullptr, Muc, tile(0, i1, a2), tile(0, i2, a1) + kTcTile, Mdc,
                                      Hb + (size_t)(c + 1) * envT2, sm, red);
        if (ok) ev += 0.5 * g.J1 * ldexp((double)wp / (double)W, eE + eH[c + 1] - eH[0]);
      }
      if (c < Lx - 1 && g.J2 != 0.0) {
        const int j1 = i1 + 1, j2 = i2 + 1;
        const int b1 = spin_of(sp, j1), b2 = spin_of(sp, j2);
        const float* Mun = Mu + (size_t)(c + 1) * envT;
        const float* Mdn = Md + (size_t)(c + 1) * envT;
        if (a1 != b2) {
          int eX = 0;
          pair_step_tc(st, false, E, X1, Muc, tile(0, i1, b2), tile(0, i2, a2) + kTcTile, Mdc, nullptr, sm, red,
                       &eX);
          __syncthreads();
          const float wp = pair_step_tc(st, false, X1, nullptr, Mun, tile(0, j1, b1), tile(0, j2, a1) + kTcTile, Mdn,
                                        Hb + (size_t)(c + 2) * envT2, sm, red);
          if (ok) ev += 0.5 * g.J2 * ldexp((double)wp / (double)W, eE + eX + eH[c + 2] - eH[0]);
        }
        if (b1 != a2) {
          int eX = 0;
          pair_step_tc(st, false, E, X1, Muc, tile(0, i1, a1), tile(0, i2, b1) + kTcTile, Mdc, nullptr, sm, red,
                       &eX);
          __syncthreads();
          const float wp = pair_step_tc(st, false, X1, nullptr, Mun, tile(0, j1, a2), tile(0, j2, b2) + kTcTile, Mdn,
                                        Hb + (size_t)(c + 2) * envT2, sm, red);
          if (ok) ev += 0.5 * g.J2 * ldexp((double)wp / (double)W, eE + eX + eH[c + 2] - eH[0]);
        }
      }
      if (c < Lx - 1) {
        int e1 = 0;
        pair_step_tc(st, false, E, En, Muc, tile(0, i1, a1), tile(0, i2, a2) + kTcTile, Mdc, nullptr, sm, red, &e1);
        __syncthreads();
        eE += e1;
        E = En;
        En = (En == E0) ? E1 : E0;
      }
    }
    if (threadIdx.x == 0) {
      a.eloc_v[(size_t)cfg * Ly + r] = ev;
      if (!ok) atomicOr(&a.flags[cfg], kFlagZeroW);
      if (!st.ok) atomicOr(&a.flags[cfg], kFlagTimeout);
    }
  }
  if (!st.ok && threadIdx.x == 0) {
    // configurations this CTA did not reach are marked too
    for (int item = blockIdx.x; item < a.n * npairs; item += gridDim.x) atomicOr(&a.flags[item / npairs], kFlagTimeout);
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_holder), "r"(tc::kTmemCols));
}

// ------------------------------------------------------------ k_finalize
// E(S) = sum over bonds of J (+1/4 parallel, -1/4 antiparallel) plus the
// exchange terms already summed per row / row pair.  Status: S^z != 0 ->
// invalid (1), zero amplitude -> numeric (5).
__global__ void k_finalize(Geometry g, const uint64_t* S, int n, const double* eloc_h, const double* eloc_v,
                           const int* flags, double* eloc, int* status, int have_eloc) {
  const int cfg = blockIdx.x * blockDim.x + threadIdx.x;
  if (cfg >= n) return;
  const uint64_t* sp = S + (size_t)cfg * g.nwords;
  int pc = 0;
  for (int w = 0; w < g.nwords; ++w) {
    uint64_t word = sp[w];
    if (w == g.nwords - 1 && (g.N & 63)) word &= (1ull << (g.N & 63)) - 1ull;
    pc += __popcll(word);
  }
  int st = 0;
  if ((g.N % 2 == 0) && pc != g.N / 2) st = 1;
  else if (flags[cfg] & kFlagTimeout) st = 4;
  else if (flags[cfg] & kFlagZeroW) st = 5;
  if (status) status[cfg] = st;
  if (!have_eloc || eloc == nullptr) return;
  double e = 0.0;
  const int Lx = g.Lx, Ly = g.Ly;
  for (int r = 0; r < Ly; ++r)
    for (int c = 0; c < Lx; ++c) {
      const int i = r * Lx + c, si = spin_of(sp, i);
      if (c + 1 < Lx) e += (si == spin_of(sp, i + 1) ? 0.25 : -0.25) * g.J1;
      if (r + 1 < Ly) e += (si == spin_of(sp, i + Lx) ? 0.25 : -0.25) * g.J1;
      if (r + 1 < Ly && c + 1 < Lx) e += (si == spin_of(sp, i + Lx + 1) ? 0.25 : -0.25) * g.J2;
      if (r + 1 < Ly && c + 1 < Lx) e += (spin_of(sp, i + 1) == spin_of(sp, i + Lx) ? 0.25 : -0.25) * g.J2;
    }
  for (int r = 0; r < Ly; ++r) e += eloc_h[(size_t)cfg * Ly + r];
  for (int r = 0; r + 1 < Ly; ++r) e += eloc_v[(size_t)cfg * Ly + r];
  eloc[cfg] = st == 0 ? e : NAN;
}

// ------------------------------------------------------- gradient sums
// sumO[i][s][p] += sum_cfg O_cfg[i][p] [s_i == s], sumEO likewise times E.
// Each thread owns elements (i, p) of both spin blocks, so no atomics.
template <typename R>
__global__ void k_grad_accum(GradArgs a, const R* __restrict__ O) {
  const size_t total = (size_t)a.N * a.D4;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / a.D4), p = (int)(e % a.D4);
    double o0 = 0, o1 = 0, eo0 = 0, eo1 = 0;
    for (int cfg = 0; cfg < a.n; ++cfg) {
      if (a.status[cfg] != 0) continue;
      const double o = (double)O[(size_t)cfg * total + e];
      const double E = a.eloc[cfg];
      if (spin_of(a.S + (size_t)cfg * a.nwords, i)) {
        o1 += o;
        eo1 += E * o;
      } else {
        o0 += o;
        eo0 += E * o;
      }
    }
    const size_t b0 = ((size_t)i * 2) * a.D4 + p, b1 = b0 + a.D4;
    a.sumO[b0] += o0;
    a.sumO[b1] += o1;
    a.sumEO[b0] += eo0;
    a.sumEO[b1] += eo1;
  }
}

// sums[0] += sum of E over configurations with status 0, sums[1] += their count.
__global__ void k_sum_eloc(const double* eloc, const int* status, int n, double* sums) {
  __shared__ double sh[2][kThreads];
  double s = 0, c = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    if (status[i] == 0) {
      s += eloc[i];
      c += 1;
    }
  sh[0][threadIdx.x] = s;
  sh[1][threadIdx.x] = c;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sums[0] += sh[0][0];
    sums[1] += sh[1][0];
  }
}

// grad = 2 (<E O> - <E><O>), cov = grad / 2.
__global__ void k_grad_finalize(int total, const double* sums, const double* sumO, const double* sumEO, double* grad,
                                double* cov) {
  const double n = sums[1];
  const double Ebar = n > 0 ? sums[0] / n : 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const double c = n > 0 ? sumEO[e] / n - Ebar * (sumO[e] / n) : 0.0;
    if (grad) grad[e] = 2.0 * c;
    if (cov) cov[e] = c;
  }
}

// ------------------------------------------------------------------- k_mc
// SplitMix64 output function (Steele, Lea & Flood 2014), used as a
// counter-based generator keyed by (seed, chain, sweep, bond).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double sampler_uniform(uint64_t seed, uint64_t chain, uint64_t sweep, uint64_t bond) {
  const uint64_t G = 0x9E3779B97F4A7C15ull;
  uint64_t h = seed;
  h = mix64(h + G * (1ull + chain));
  h = mix64(h + G * (1ull + sweep));
  h = mix64(h + G * (1ull + bond));
  return (double)(h >> 11) * 0x1.0p-53;
}

// ------------------------------------------------------------- k_go_step
// One gradient-optimisation update of the FP64 tensors (Sec. III):
// A <- A - p dt sign(dE/dA), p in [0, 1) per element, from the same SplitMix64
// construction keyed by (seed, step, element index).  Entries past an open
// edge, and entries whose derivative is zero, do not move.  (p dt) sign is
// exact once p dt is rounded; the _rn intrinsics keep the compiler from
// fusing, so the result is A - (p*dt)*sign evaluated in that order.
__global__ void k_go_step(double* A, const double* grad, Geometry geo, double dt, uint64_t seed, uint64_t step) {
  const uint64_t G = 0x9E3779B97F4A7C15ull;
  const size_t D = (size_t)geo.D, D4 = D * D * D * D, n = (size_t)geo.N * 2 * D4;
  const uint64_t hs = mix64(seed + G * (1ull + step));
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const double g = grad[e];
    if (!(g > 0.0) && !(g < 0.0)) continue;
    const int site = (int)(e / (2 * D4));
    const size_t w = e % D4;
    const size_t l = w / (D * D * D), r = w / (D * D) % D, u = w / D % D, d = w % D;
    const int row = site / geo.Lx, col = site % geo.Lx;
    if ((col == 0 && l) || (col == geo.Lx - 1 && r) || (row == 0 && u) || (row == geo.Ly - 1 && d)) continue;
    const uint64_t h = mix64(hs + G * (1ull + (uint64_t)e));
    const double p = (double)(h >> 11) * 0x1.0p-53;
    A[e] = __dsub_rn(A[e], __dmul_rn(__dmul_rn(p, dt), g > 0.0 ? 1.0 : -1.0));
  }
}

cudaError_t launch_go_step(double* A, const double* grad, const Geometry& geo, double dt, uint64_t seed,
                           uint64_t step, int nsm, cudaStream_t st) {
  const size_t n = (size_t)geo.N * 2 * geo.D * geo.D * geo.D * geo.D;
  const size_t blocks = (n + kThreads - 1) / kThreads;
  const int grid = (int)(blocks < (size_t)nsm * 8 ? blocks : (size_t)nsm * 8);
  if (grid < 1) return cudaSuccess;
  k_go_step<<<grid, kThreads, 0, st>>>(A, grad, geo, dt, seed, step);
  return cudaGetLastError();
}

// Metropolis sweeps (sampling with weight W^2, Sec. II) over nearest-neighbour
// exchanges: horizontal bonds row by row, then vertical bonds row pair by row
// pair.  Lower environments are rebuilt from the current S at the start of
// each pass; the upper environment grows from the updated rows; the row (or
// row-pair) transfers to the left are carried with the accepted spins.
template <typename R>
__global__ void __launch_bounds__(kThreads) k_mc(KArgs<R> a, uint64_t* S, int nsweeps, uint64_t seed, uint64_t chain0,
                                                 uint64_t sweep0, long long* accepted) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ R red[64];
  __shared__ uint64_t sp[kMaxWords];
  __shared__ int ones[kMaxDcD + 1];
  const Geometry& g = a.g;
  const int Lx = g.Lx, Ly = g.Ly, Dc = g.Dc, D = g.D;
  const size_t envT = (size_t)Dc * D * Dc, envT2 = envT * D;
  R* p = a.scratch + (size_t)blockIdx.x * a.slot_elems;
  R* envL = p; p += (size_t)Ly * Lx * envT;
  R* Ubuf[2];
  Ubuf[0] = p; p += (size_t)Lx * envT;
  Ubuf[1] = p; p += (size_t)Lx * envT;
  ZipBufs<R> zb;
  __shared__ double dred[kWarps];
  __shared__ R wv[kMaxDcD];
  R* gsm;
  int* gism;
  smem_split<R>(smem_raw, g, true, a.smem_wm != 0, gsm, gism);
  carve_zip<R>(g, p, zb, a.smem_wm ? gsm : nullptr, red, dred, wv, gsm, gism);
  R* Hb = p; p += (size_t)(Lx + 1) * envT2;
  R* Q[4];
  for (int q = 0; q < 4; ++q) { Q[q] = p; p += envT2; }
  R* t0 = p; p += tmp_elems(g);
  R* t1 = p;
  for (int i = threadIdx.x; i <= Lx; i += blockDim.x) ones[i] = 1;
  __shared__ int eH[kMaxL + 1];   // H_c is stored scaled by 2^-eH[c]
  const int nh = Ly * (Lx - 1);
  for (int chain = blockIdx.x; chain < a.n; chain += gridDim.x) {
    __syncthreads();
    for (int i = threadIdx.x; i < g.nwords; i += blockDim.x) sp[i] = S[(size_t)chain * g.nwords + i];
    __syncthreads();
    long long acc = 0;
    for (int k = 0; k < nsweeps; ++k) {
      const uint64_t sweep = sweep0 + (uint64_t)k;
      for (int pass = 0; pass < 2; ++pass) {
        // lower environments L_r, r = Ly-1 .. 1, from the current S
        const R* Min = a.triv_mps;
        for (int j = 0; j + 1 < Ly; ++j) {
          const int r = Ly - 1 - j;
          const int* bdin = j == 0 ? ones : a.bd + ((size_t)1 * Ly + (j - 1)) * (Lx + 1);
          R* Mout = envL + (size_t)r * Lx * envT;
          absorb_row<R>(a, Min, Mout, r, 1, (j % 2) == 0, bdin, sp, zb, red);
          Min = Mout;
        }
        const R* Mu = a.triv_mps;
        int ub = 0;
        const int rows = pass == 0 ? Ly : Ly - 1;
        for (int r = 0; r < rows; ++r) {
          const R* Md;
          if (pass == 0) Md = r == Ly - 1 ? a.triv_mps : envL + (size_t)(r + 1) * Lx * envT;
          else Md = r + 2 > Ly - 1 ? a.triv_mps : envL + (size_t)(r + 2) * Lx * envT;
          const size_t tsz = pass == 0 ? envT : envT2;
          const R* triv = pass == 0 ? a.triv_t1 : a.triv_t2;
          for (size_t e = threadIdx.x; e < tsz; e += blockDim.x) Hb[(size_t)Lx * tsz + e] = triv[e];
          if (threadIdx.x == 0) eH[Lx] = 0;
          __syncthreads();
          int eacc = 0;
          for (int c = Lx - 1; c >= 0; --c) {
            const int i1 = r * Lx + c;
            if (pass == 0)
              run_op<R>(OP_COL1_RIGHT, D, Dc, Hb + (size_t)(c + 1) * tsz, Mu + (size_t)c * envT,
                        tptr(a, i1, spin_of(sp, i1)), Md + (size_t)c * envT, nullptr, Hb + (size_t)c * tsz, t0, t1, gsm, gism);
            else
              run_op<R>(OP_COL2_RIGHT, D, Dc, Hb + (size_t)(c + 1) * tsz, Mu + (size_t)c * envT,
                        tptr(a, i1, spin_of(sp, i1)), tptr(a, i1 + Lx, spin_of(sp, i1 + Lx)),
                        Md + (size_t)c * envT, Hb + (size_t)c * tsz, t0, t1, gsm, gism);
            eacc += normalize_pow2(Hb + (size_t)c * tsz, (int)tsz, red);
            if (threadIdx.x == 0) eH[c] = eacc;
          }
          const R* E = triv;
          int e = 3;   // index in Q of the buffer E lives in (none yet)
          const int ncol = pass == 0 ? Lx - 1 : Lx;
          for (int c = 0; c < ncol; ++c) {
            const int i1 = r * Lx + c;
            const int i2 = pass == 0 ? i1 + 1 : i1 + Lx;
            const int s1 = spin_of(sp, i1), s2 = spin_of(sp, i2);
            R* X1 = Q[(e + 1) & 3];
            R* Xf = Q[(e + 2) & 3];
            R* X2 = Q[(e + 3) & 3];
            const R* Muc = Mu + (size_t)c * envT;
            const R* Mdc = Md + (size_t)c * envT;
            int chosen;
            if (s1 != s2) {
              R w, wp;
              if (pass == 0) {
                run_op<R>(OP_COL1_LEFT, D, Dc, E, Muc, tptr(a, i1, s1), Mdc, nullptr, X1, t0, t1, gsm, gism);
                run_op<R>(OP_COL1_LEFT, D, Dc, E, Muc, tptr(a, i1, s2), Mdc, nullptr, Xf, t0, t1, gsm, gism);
                run_op<R>(OP_COL1_LEFT, D, Dc, Xf, Mu + (size_t)(c + 1) * envT, tptr(a, i2, s1),
                          Md + (size_t)(c + 1) * envT, nullptr, X2, t0, t1, gsm, gism);
                w = block_dot(X1, Hb + (size_t)(c + 1) * tsz, (int)tsz, red);
                wp = block_dot(X2, Hb + (size_t)(c + 2) * tsz, (int)tsz, red);
              } else {
                run_op<R>(OP_COL2_LEFT, D, Dc, E, Muc, tptr(a, i1, s1), tptr(a, i2, s2), Mdc, X1, t0, t1, gsm, gism);
                run_op<R>(OP_COL2_LEFT, D, Dc, E, Muc, tptr(a, i1, s2), tptr(a, i2, s1), Mdc, Xf, t0, t1, gsm, gism);
                w = block_dot(X1, Hb + (size_t)(c + 1) * tsz, (int)tsz, red);
                wp = block_dot(Xf, Hb + (size_t)(c + 1) * tsz, (int)tsz, red);
              }
              const uint64_t bond = pass == 0 ? (uint64_t)(r * (Lx - 1) + c) : (uint64_t)(nh + r * Lx + c);
              const double u = sampler_uniform(seed, chain0 + (uint64_t)chain, sweep, bond);
              bool take;
              if (w == R(0)) {
                take = true;
              } else {
                // the E scale is common to w and wp; the H scales differ by a column in a horizontal exchange
                const double ratio =
                    pass == 0 ? ldexp((double)wp / (double)w, eH[c + 2] - eH[c + 1]) : (double)wp / (double)w;
                take = u < ratio * ratio;
              }
              if (take) {
                if (threadIdx.x == 0) {
                  sp[i1 >> 6] ^= 1ull << (i1 & 63);
                  sp[i2 >> 6] ^= 1ull << (i2 & 63);
                }
                ++acc;
                chosen = (e + 2) & 3;
              } else {
                chosen = (e + 1) & 3;
              }
              __syncthreads();
            } else {
              if (pass == 0)
                run_op<R>(OP_COL1_LEFT, D, Dc, E, Muc, tptr(a, i1, s1), Mdc, nullptr, X1, t0, t1, gsm, gism);
              else
                run_op<R>(OP_COL2_LEFT, D, Dc, E, Muc, tptr(a, i1, s1), tptr(a, i2, s2), Mdc, X1, t0, t1, gsm, gism);
              chosen = (e + 1) & 3;
            }
            e = chosen;
            E = Q[e];
            // E's own scale cancels in every ratio: renormalise without tracking
            normalize_pow2(Q[e], (int)tsz, red);
          }
          if (pass == 0 ? (r < Ly - 1) : true) {
            const int* bdin = r == 0 ? ones : a.bd + ((size_t)0 * Ly + (r - 1)) * (Lx + 1);
            absorb_row<R>(a, Mu, Ubuf[ub], r, 0, (r % 2) == 0, bdin, sp, zb, red);
            Mu = Ubuf[ub];
            ub ^= 1;
          }
        }
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < g.nwords; i += blockDim.x) S[(size_t)chain * g.nwords + i] = sp[i];
    if (threadIdx.x == 0 && accepted) accepted[chain] += acc;
  }
}

// --------------------------------------------------------------- launchers
template <typename R>
int max_blocks_boundary(const Geometry& g) {
  int dev = 0, nsm = 0, nb = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = dyn_smem_bytes(g, sizeof(R), true, wm_fits_smem(g, sizeof(R)));
  prefer_shared(k_boundary<R>, smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_boundary<R>, kThreads, smem);
  if (nb < 1) nb = 1;
  return nsm * nb;
}

template <typename R>
cudaError_t launch_boundary(const KArgs<R>& a, int dirs, int grid, cudaStream_t st) {
  const size_t smem = dyn_smem_bytes(a.g, sizeof(R), true, a.smem_wm != 0);
  cudaError_t e = prefer_shared(k_boundary<R>, smem);
  if (e != cudaSuccess) return e;
  k_boundary<R><<<grid, kThreads, smem, st>>>(a, dirs);
  return cudaGetLastError();
}

template <typename R>
int max_blocks_mc(const Geometry& g) {
  int dev = 0, nsm = 0, nb = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = dyn_smem_bytes(g, sizeof(R), true, wm_fits_smem(g, sizeof(R)));
  prefer_shared(k_mc<R>, smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_mc<R>, kThreads, smem);
  if (nb < 1) nb = 1;
  return nsm * nb;
}

template <typename R>
cudaError_t launch_mc(const KArgs<R>& a, uint64_t* S, int nsweeps, uint64_t seed, uint64_t chain0, uint64_t sweep0,
                      long long* accepted, int grid, cudaStream_t st) {
  const size_t smem = dyn_smem_bytes(a.g, sizeof(R), true, a.smem_wm != 0);
  cudaError_t e = prefer_shared(k_mc<R>, smem);
  if (e != cudaSuccess) return e;
  k_mc<R><<<grid, kThreads, smem, st>>>(a, S, nsweeps, seed, chain0, sweep0, accepted);
  return cudaGetLastError();
}

// (D, Dc) pairs with a fused single-row step and site environment.
template <typename R>
static int row_fused_id(const Geometry& g) {
  if (g.D == 2 && g.Dc == 4) return 1;
  if (g.D == 4 && g.Dc == 8) return 2;
  if (g.D == 6 && g.Dc == 12) return 3;
  if (g.D == 8 && g.Dc == 16) return 4;
  return 0;
}

template <typename R, int D, int Dc>
static int row_fused_blocks() {
  int dev = 0, nsm = 0, nb = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = (size_t)RowSmem<D, Dc>::total * sizeof(R);
  prefer_shared(k_row_fused<R, D, Dc>, smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_row_fused<R, D, Dc>, kThreads, smem);
  return nsm * (nb < 1 ? 1 : nb);
}

template <typename R, int D, int Dc>
static cudaError_t launch_row_fused(const KArgs<R>& a, int grid, cudaStream_t st) {
  const size_t smem = (size_t)RowSmem<D, Dc>::total * sizeof(R);
  cudaError_t e = prefer_shared(k_row_fused<R, D, Dc>, smem);
  if (e != cudaSuccess) return e;
  k_row_fused<R, D, Dc><<<grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename R>
int max_blocks_row(const Geometry& g) {
  switch (row_fused_id<R>(g)) {
    case 1: return row_fused_blocks<R, 2, 4>();
    case 2: return row_fused_blocks<R, 4, 8>();
    case 3: return row_fused_blocks<R, 6, 12>();
    case 4: return row_fused_blocks<R, 8, 16>();
  }
  int dev = 0, nsm = 0, nb = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = dyn_smem_bytes(g, sizeof(R), false, false);
  prefer_shared(k_row<R>, smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_row<R>, kThreads, smem);
  return nsm * (nb < 1 ? 1 : nb);
}

template <typename R>
int max_blocks_pair(const Geometry& g) {
  int dev = 0, nsm = 0, nb = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = dyn_smem_bytes(g, sizeof(R), false, false);
  prefer_shared(k_pair<R>, smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pair<R>, kThreads, smem);
  return nsm * (nb < 1 ? 1 : nb);
}

template <typename R>
cudaError_t launch_row(const KArgs<R>& a, int grid, cudaStream_t st) {
  switch (row_fused_id<R>(a.g)) {
    case 1: return launch_row_fused<R, 2, 4>(a, grid, st);
    case 2: return launch_row_fused<R, 4, 8>(a, grid, st);
    case 3: return launch_row_fused<R, 6, 12>(a, grid, st);
    case 4: return launch_row_fused<R, 8, 16>(a, grid, st);
  }
  const size_t smem = dyn_smem_bytes(a.g, sizeof(R), false, false);
  cudaError_t e = prefer_shared(k_row<R>, smem);
  if (e != cudaSuccess) return e;
  k_row<R><<<grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename R, int D, int Dc>
static cudaError_t launch_pair_fused(const KArgs<R>& a, int grid, cudaStream_t st) {
  const size_t smem = (size_t)PairSmem<D, Dc>::total * sizeof(R);
  cudaError_t e = prefer_shared(k_pair_fused<R, D, Dc>, smem);
  if (e != cudaSuccess) return e;
  k_pair_fused<R, D, Dc><<<grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename R, int D, int Dc>
static int fused_blocks() {
  int dev = 0, nsm = 0, nb = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = (size_t)PairSmem<D, Dc>::total * sizeof(R);
  prefer_shared(k_pair_fused<R, D, Dc>, smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pair_fused<R, D, Dc>, kThreads, smem);
  return nsm * (nb < 1 ? 1 : nb);
}

// (D, Dc) pairs with a fused two-row step; FP64 only where its shared memory fits.
template <typename R>
static int pair_fused_id(const Geometry& g) {
  if (g.D == 2 && g.Dc == 4) return 1;
  if (g.D == 4 && g.Dc == 8) return 2;
  if (sizeof(R) == 4 && g.D == 6 && g.Dc == 12) return 3;
  if (sizeof(R) == 4 && g.D == 8 && g.Dc == 16) return 4;
  return 0;
}

template <typename R>
int max_blocks_pair_fused(const Geometry& g) {
  switch (pair_fused_id<R>(g)) {
    case 1: return fused_blocks<R, 2, 4>();
    case 2: return fused_blocks<R, 4, 8>();
    case 3: return fused_blocks<R, sizeof(R) == 4 ? 6 : 2, sizeof(R) == 4 ? 12 : 4>();
    case 4: return fused_blocks<R, sizeof(R) == 4 ? 8 : 2, sizeof(R) == 4 ? 16 : 4>();
  }
  return 0;
}

int max_blocks_pair_tc() {
  int dev = 0, nsm = 0, nb = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = (size_t)PairTcSmem::total * sizeof(float) + 1024;
  prefer_shared(k_pair_tc, smem);
  cudaFuncSetAttribute(k_pair_tc, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pair_tc, kThreads, smem);
  // The occupancy query reports one resident CTA for this kernel, although
  // its registers and shared memory fit two (as ncu's occupancy section also
  // shows); take the residency from the kernel's own attributes as well.
  cudaFuncAttributes fa{};
  int smem_sm = 0, reserved = 0, regs_sm = 0;
  if (cudaFuncGetAttributes(&fa, k_pair_tc) == cudaSuccess &&
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) == cudaSuccess &&
      fa.numRegs > 0) {
    const size_t per_block = fa.sharedSizeBytes + smem + (size_t)reserved;
    const int by_smem = (int)((size_t)smem_sm / per_block);
    const int by_regs = regs_sm / (fa.numRegs * kThreads);
    nb = std::max(nb, std::min(by_smem, by_regs));
  }
  // each resident CTA holds kTmemCols of the SM's 512 TMEM columns
  nb = std::min(nb, 512 / tc::kTmemCols);
  return nsm * (nb < 1 ? 1 : nb);
}

cudaError_t launch_pair_tc(const KArgs<float>& a, int grid, cudaStream_t st) {
  const size_t smem = (size_t)PairTcSmem::total * sizeof(float) + 1024;
  cudaError_t e = prefer_shared(k_pair_tc, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_pair_tc, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  k_pair_tc<<<grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_pair(const KArgs<R>& a, int grid, cudaStream_t st) {
  switch (pair_fused_id<R>(a.g)) {
    case 1: return launch_pair_fused<R, 2, 4>(a, grid, st);
    case 2: return launch_pair_fused<R, 4, 8>(a, grid, st);
    case 3: return launch_pair_fused<R, sizeof(R) == 4 ? 6 : 2, sizeof(R) == 4 ? 12 : 4>(a, grid, st);
    case 4: return launch_pair_fused<R, sizeof(R) == 4 ? 8 : 2, sizeof(R) == 4 ? 16 : 4>(a, grid, st);
  }
  const size_t smem = dyn_smem_bytes(a.g, sizeof(R), false, false);
  cudaError_t e = prefer_shared(k_pair<R>, smem);
  if (e != cudaSuccess) return e;
  k_pair<R><<<grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_grad_accum(const GradArgs& a, const R* O, cudaStream_t st) {
  const size_t total = (size_t)a.N * a.D4;
  int grid = (int)((total + kThreads - 1) / kThreads);
  if (grid > 65535 * 8) grid = 65535 * 8;
  k_grad_accum<R><<<grid, kThreads, 0, st>>>(a, O);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const Geometry& g, const uint64_t* S, int n, const double* eloc_h, const double* eloc_v,
                            const int* flags, double* eloc, int* status, int have_eloc, cudaStream_t st) {
  k_finalize<<<(n + 127) / 128, 128, 0, st>>>(g, S, n, eloc_h, eloc_v, flags, eloc, status, have_eloc);
  return cudaGetLastError();
}

cudaError_t launch_sum_eloc(const double* eloc, const int* status, int n, double* sums, cudaStream_t st) {
  k_sum_eloc<<<1, kThreads, 0, st>>>(eloc, status, n, sums);
  return cudaGetLastError();
}

cudaError_t launch_grad_finalize(int total, int, const double* sums, const double* sumO, const double* sumEO,
                                 double* grad, double* cov, cudaStream_t st) {
  int grid = (total + kThreads - 1) / kThreads;
  if (grid > 65535) grid = 65535;
  k_grad_finalize<<<grid, kThreads, 0, st>>>(total, sums, sumO, sumEO, grad, cov);
  return cudaGetLastError();
}

#define PEPS_INST(R)                                                                                    \
  template int max_blocks_boundary<R>(const Geometry&);                                                 \
  template int max_blocks_mc<R>(const Geometry&);                                                       \
  template int max_blocks_row<R>(const Geometry&);                                                      \
  template int max_blocks_pair<R>(const Geometry&);                                                     \
  template int max_blocks_pair_fused<R>(const Geometry&);                                               \
  template cudaError_t launch_mc<R>(const KArgs<R>&, uint64_t*, int, uint64_t, uint64_t, uint64_t,      \
                                    long long*, int, cudaStream_t);                                      \
  template cudaError_t launch_boundary<R>(const KArgs<R>&, int, int, cudaStream_t);                     \
  template cudaError_t launch_row<R>(const KArgs<R>&, int, cudaStream_t);                               \
  template cudaError_t launch_pair<R>(const KArgs<R>&, int, cudaStream_t);                              \
  template cudaError_t launch_grad_accum<R>(const GradArgs&, const R*, cudaStream_t);
PEPS_INST(double)
PEPS_INST(float)

}  // namespace peps

// ===================================================================
// Allocation-free amplitudes.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// runtime's memory arena (a framework custom op, a plugin, a game or
// simulation engine) where a stray allocation would fragment or bypass the
// owner's allocator, or real-time code that must not allocate after start-up.
// peps_amplitudes_static serves them: it computes ln|psi| and sign with the
// top-down boundary-MPS sweep (the k_boundary sweep without the stored
// environments) and takes its per-CTA scratch from the file-scope array
// below instead of the context workspace.  The caller passes the site
// tensors, the configurations and the outputs, all in device memory.
// ===================================================================
namespace peps {

constexpr size_t kStaticScratchBytes = size_t(8) << 20;   // 8 MiB on every device that loads the library
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Bond dimensions of the boundary MPS after absorbing one row (top-down),
// the same rule K = min(Dc, rows, cols) the truncation applies.
__device__ void next_bonds(const int* bin, int* bout, int Lx, int D, int Dc, int outdim, bool lr) {
  for (int c = 0; c <= Lx; ++c) bout[c] = 1;
  int k = 1;
  if (lr) {
    for (int c = 0; c < Lx - 1; ++c) {
      const int K = min(Dc, min(k * outdim, bin[c + 1] * D));
      bout[c + 1] = K;
      k = K;
    }
  } else {
    for (int c = Lx - 1; c > 0; --c) {
      const int K = min(Dc, min(outdim * k, bin[c] * D));
      bout[c] = K;
      k = K;
    }
  }
}

__host__ __device__ inline size_t static_slot_elems(const Geometry& g, bool wm_in_smem) {
  const size_t envT = (size_t)g.Dc * g.D * g.Dc, Dc = g.Dc, D = g.D, P = Dc * D;
  const size_t zip = 2 * Dc * Dc * D + Dc * Dc * D * D + P * P + trunc_ws_elems((int)P, g.Dc, !wm_in_smem);
  return (zip + 2 * (size_t)g.Lx * envT + 63) / 64 * 64;
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_amplitudes_static(KArgs<R> a, R* scratch, size_t slot_elems) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ R red[64];
  __shared__ uint64_t sp[kMaxWords];
  __shared__ int bonds[2][kMaxDcD + 1];
  __shared__ double dred[kWarps];
  __shared__ R wv[kMaxDcD];
  __shared__ R vec[kMaxDc], nv[kMaxDc];
  const Geometry& g = a.g;
  const int Lx = g.Lx, Ly = g.Ly, Dc = g.Dc, D = g.D;
  const size_t envT = (size_t)Dc * D * Dc;
  R* gsm;
  int* gism;
  smem_split<R>(smem_raw, g, true, a.smem_wm != 0, gsm, gism);
  R* p = scratch + (size_t)blockIdx.x * slot_elems;
  ZipBufs<R> zb;
  carve_zip<R>(g, p, zb, a.smem_wm ? gsm : nullptr, red, dred, wv, gsm, gism);
  R* Mbuf[2];
  Mbuf[0] = p;
  Mbuf[1] = p + (size_t)Lx * envT;
  for (int cfg = blockIdx.x; cfg < a.n; cfg += gridDim.x) {
    __syncthreads();
    for (int i = threadIdx.x; i < g.nwords; i += blockDim.x) sp[i] = a.S[(size_t)cfg * g.nwords + i];
    // every buffer is written before it is read: the trivial MPS is rebuilt here
    for (size_t e = threadIdx.x; e < (size_t)Lx * envT; e += blockDim.x) Mbuf[0][e] = (e % envT) == 0 ? R(1) : R(0);
    for (int c = threadIdx.x; c <= Lx; c += blockDim.x) bonds[0][c] = 1;
    __syncthreads();
    double ls = 0.0;
    bool zero = false;
    int cur = 0;
    for (int r = 0; r < Ly; ++r) {
      const bool lr = (r % 2) == 0;
      const double nrm = absorb_row<R>(a, Mbuf[cur], Mbuf[cur ^ 1], r, 0, lr, bonds[cur], sp, zb, red);
      if (!(nrm > 0.0)) zero = true;
      else ls += log(nrm);
      if (threadIdx.x == 0) next_bonds(bonds[cur], bonds[cur ^ 1], Lx, D, Dc, r == Ly - 1 ? 1 : D, lr);
      __syncthreads();
      cur ^= 1;
    }
    if (threadIdx.x == 0) {
      const R* Ml = Mbuf[cur];
      vec[0] = R(1);
      int na = 1;
      for (int c = 0; c < Lx; ++c) {
        const int nb = bonds[cur][c + 1];
        const R* M = Ml + (size_t)c * envT;
        for (int b = 0; b < nb; ++b) {
          R s = R(0);
          for (int x = 0; x < na; ++x) s += vec[x] * M[(size_t)x * D * Dc + b];
          nv[b] = s;
        }
        for (int b = 0; b < nb; ++b) vec[b] = nv[b];
        na = nb;
      }
      int pc = 0;
      for (int w = 0; w < g.nwords; ++w) {
        uint64_t word = sp[w];
        if (w == g.nwords - 1 && (g.N & 63)) word &= (1ull << (g.N & 63)) - 1ull;
        pc += __popcll(word);
      }
      const R v = vec[0];
      int st = 0;
      if (zero || v == R(0)) {
        a.logabs[cfg] = -INFINITY;
        a.sign[cfg] = 0;
        st = 5;
      } else {
        a.logabs[cfg] = ls + log(fabs((double)v));
        a.sign[cfg] = v > R(0) ? 1 : -1;
      }
      if ((g.N % 2 == 0) && pc != g.N / 2) st = 1;
      if (a.flags) a.flags[cfg] = st;
    }
  }
}

// Device address of the static scratch, looked up once per device with that
// device current (the host-side symbol is only a stand-in, not an address).
static void* g_static_ptr[256];
static std::mutex g_static_mu;

static cudaError_t static_scratch_ptr(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return cudaSuccess;
}

template <typename R>
static peps_status amplitudes_static_impl(const peps_params* p, const void* A_dev, const uint64_t* S_dev, int n,
                                          double* logabs_dev, int8_t* sign_dev, int32_t* status_dev,
                                          cudaStream_t stream, char* err, size_t errlen) {
  Geometry g;
  g.Lx = p->Lx;
  g.Ly = p->Ly;
  g.D = p->D;
  g.Dc = p->Dc;
  g.N = p->Lx * p->Ly;
  g.nwords = (g.N + 63) / 64;
  g.J1 = p->J1;
  g.J2 = p->J2;
  const bool wm = wm_fits_smem(g, sizeof(R));
  const size_t slot = static_slot_elems(g, wm);
  const size_t slots = kStaticScratchBytes / (slot * sizeof(R));
  if (slots < 1) {
    snprintf(err, errlen,
             "lattice too large for the allocation-free path: one CTA needs %zu bytes of scratch, the static "
             "array holds %zu",
             slot * sizeof(R), kStaticScratchBytes);
    return PEPS_EINVAL;
  }
  void* base = nullptr;
  cudaError_t e = static_scratch_ptr(&base);
  if (e != cudaSuccess) {
    snprintf(err, errlen, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    return PEPS_ECUDA;
  }
  const size_t smem = dyn_smem_bytes(g, sizeof(R), true, wm);
  e = prefer_shared(k_amplitudes_static<R>, smem);
  int dev = 0, nsm = 0, nb = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_amplitudes_static<R>, kThreads, smem);
  if (e != cudaSuccess) {
    snprintf(err, errlen, "launch set-up: %s", cudaGetErrorString(e));
    return PEPS_ECUDA;
  }
  KArgs<R> a;
  memset(&a, 0, sizeof(a));
  a.g = g;
  a.A = (const R*)A_dev;
  a.S = S_dev;
  a.n = n;
  a.logabs = logabs_dev;
  a.sign = sign_dev;
  a.flags = status_dev;
  a.smem_wm = wm ? 1 : 0;
  long long grid = std::min<long long>((long long)n, (long long)slots);
  grid = std::min<long long>(grid, (long long)nsm * std::max(nb, 1));
  k_amplitudes_static<R><<<(int)grid, kThreads, smem, stream>>>(a, (R*)base, slot);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(err, errlen, "launch: %s", cudaGetErrorString(e));
    return PEPS_ECUDA;
  }
  return PEPS_OK;
}

}  // namespace peps

extern "C" peps_status peps_amplitudes_static(const peps_params* p, const void* A_dev, const uint64_t* S_dev,
                                              int n, double* logabs_dev, int8_t* sign_dev, int32_t* status_dev,
                                              void* cuda_stream) {
  char err[256] = {0};
  if (!p) {
    peps::set_last_error("null parameters");
    return PEPS_EINVAL;
  }
  if (p->Lx < 2 || p->Ly < 2 || p->Lx > 64 || p->Ly > 64 || (long)p->Lx * p->Ly > 64L * peps::kMaxWords ||
      p->d != 2 || p->D < 1 || p->D > 16 || p->Dc < 1 || p->Dc > peps::kMaxDc || p->Dc * p->D > peps::kMaxDcD) {
    peps::set_last_error("parameters out of range (see peps_params)");
    return PEPS_EINVAL;
  }
  if (p->prec != PEPS_FP64 && p->prec != PEPS_FP32) {
    peps::set_last_error("precision must be PEPS_FP64 or PEPS_FP32");
    return PEPS_EINVAL;
  }
  if (n < 0 || (n > 0 && (!A_dev || !S_dev || !logabs_dev || !sign_dev))) {
    peps::set_last_error("bad batch size or null pointer");
    return PEPS_EINVAL;
  }
  if (n == 0) return PEPS_OK;
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  const peps_status r =
      p->prec == PEPS_FP64
          ? peps::amplitudes_static_impl<double>(p, A_dev, S_dev, n, logabs_dev, sign_dev, status_dev, st, err,
                                                 sizeof(err))
          : peps::amplitudes_static_impl<float>(p, A_dev, S_dev, n, logabs_dev, sign_dev, status_dev, st, err,
                                                sizeof(err));
  if (r != PEPS_OK) peps::set_last_error(err);
  return r;
}
