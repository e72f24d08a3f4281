// Device helpers shared by the kernel translation units: spin and tensor
// access, shared-memory layouts, the zip-up row absorption (Fig. 1d) with its
// truncation, and the counter-based generator of the Metropolis and GO draws.
#pragma once

#include <algorithm>
#include <cstdio>
#include <cstring>

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


size_t dyn_smem_bytes(const Geometry& g, size_t elem, bool truncates, bool wm_in_smem);

template <typename R>
__device__ __forceinline__ void smem_split(unsigned char* raw, const Geometry& g, bool truncates, bool wm_in_smem,
                                           R*& reals, int*& ints) {
  reals = reinterpret_cast<R*>(raw);
  ints = reinterpret_cast<int*>(raw + reals_region_bytes(g, sizeof(R), truncates, wm_in_smem));
}


__host__ __device__ inline size_t tmp_elems(const Geometry& g) {
  const size_t Dc = g.Dc, D = g.D;
  return Dc * Dc * D * D * D;
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

template <typename R>
__device__ R block_dot(const R* x, const R* y, int n, R* red) {
  R s = R(0);
  for (int e = threadIdx.x; e < n; e += blockDim.x) s += x[e] * y[e];
  return block_sum(s, red);
}


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


}  // namespace peps
