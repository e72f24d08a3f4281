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
#include "qr.cuh"

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
// Buffers of the variational-fit truncation (present when g.fit > 0).
template <typename R>
struct FitBufs {
  R* F;      // [Lx + 1] left overlap transfers
  R* G;      // [Lx + 1] right overlap transfers
  R* Tt;     // [Lx][D^4] the row's tensors with u and d exchanged (bottom-up sweep)
  R* QM;     // QR work: the matrix, then its reflectors
  R* QN;     // QR work: Q
  R* qtau;
  R* t0;     // contraction temporaries
  R* t1;
};

// Element count of the fit buffers.
__host__ __device__ inline size_t fit_elems(const Geometry& g) {
  if (g.fit <= 0) return 0;
  const size_t Dc = g.Dc, D = g.D, envT = Dc * D * Dc, D4 = D * D * D * D;
  return 2 * (size_t)(g.Lx + 1) * envT + (size_t)g.Lx * D4 + 2 * Dc * Dc * D + Dc * D + 2 * tmp_elems(g) + 64;
}

template <typename R>
struct ZipBufs {
  R* C0;
  R* C1;
  R* Y;
  R* X;
  double* dred;   // >= kWarps doubles of shared memory
  R* gsm;         // GEMM shared scratch
  int* gism;
  int gsm_reals;  // its size in reals (free between truncations)
  TruncWork<R> tw;
  FitBufs<R> fb;
};

// Re-orthonormalises one candidate MPS tensor X (padded [Dc][D][Dc], true
// dims a x o x b) in place: by a QR of [(a, o), b] when `left` (a left
// isometry, the fit moving right) or an LQ of [a, (o, b)] (a right isometry,
// moving left), the triangular factor dropped.  Padded entries stay zero.
template <typename R>
__device__ void fit_orthonormalise(R* X, int a, int o, int b, int D, int Dc, bool left, FitBufs<R>& fb, R* red) {
  const int m = left ? a * o : o * b, n = left ? b : a;
  for (int e = threadIdx.x; e < m * n; e += blockDim.x) {
    const int col = e / m, row = e % m;
    const int ai = left ? row / o : col, di = left ? row % o : row / b, bi = left ? col : row % b;
    fb.QM[e] = X[(ai * D + di) * Dc + bi];
  }
  for (int e = threadIdx.x; e < m * n; e += blockDim.x) fb.QN[e] = (e % m == e / m) ? R(1) : R(0);
  __syncthreads();
  qr::house_qr<R>(fb.QM, m, n, fb.qtau, red);
  qr::apply_q<R>(fb.QM, fb.qtau, fb.QN, m, n, n);
  for (int e = threadIdx.x; e < Dc * D * Dc; e += blockDim.x) X[e] = R(0);
  __syncthreads();
  for (int e = threadIdx.x; e < m * n; e += blockDim.x) {
    const int col = e / m, row = e % m;
    const int ai = left ? row / o : col, di = left ? row % o : row / b, bi = left ? col : row % b;
    X[(ai * D + di) * Dc + bi] = fb.QN[e];
  }
  __syncthreads();
}

// Variational-fit sweeps (the boundary-MPS method by variational
// compression) on the zip-up result Mout of absorbing `row` into Min: g.fit
// sweeps of one-site ALS, each two passes from the zip-up's last column to
// the other end and back.  A pass computes the overlap transfers toward it
// once (the tensors there are isometries of the right kind), then per column
// sets the tensor to its environment in <P| Min T> (OP_FIT_SITE),
// re-orthonormalises it (except the pass's last column, the new centre) and
// extends the transfers.  Transfers are scaled by powers of two; the return
// value is the exponent the centre tensor is scaled by.  bdo: the tensors'
// bond dimensions.
template <typename R>
__device__ __noinline__ int fit_row(const KArgs<R>& a, const R* Min, R* Mout, int row, int dir, bool lr, const uint64_t* sp,
                       const int* bdo, ZipBufs<R>& zb, R* red) {
  const Geometry& g = a.g;
  const int D = g.D, Dc = g.Dc, Lx = g.Lx;
  const int envT = Dc * D * Dc, D4 = D * D * D * D;
  FitBufs<R>& fb = zb.fb;
  __shared__ int eF[kMaxL + 1], eG[kMaxL + 1];
  if (dir == 1) {
    // the lower sweep's MPS faces the row's d legs: exchange u and d
    for (int e = threadIdx.x; e < Lx * D4; e += blockDim.x) {
      const int c = e / D4, w = e % D4;
      const int l = w / (D * D * D), r = w / (D * D) % D, u = w / D % D, d = w % D;
      const int site = row * Lx + c;
      fb.Tt[e] = tptr(a, site, spin_of(sp, site))[((l * D + r) * D + d) * D + u];
    }
    __syncthreads();
  }
  auto Tc = [&](int c) -> const R* {
    const int site = row * Lx + c;
    return dir == 0 ? tptr(a, site, spin_of(sp, site)) : fb.Tt + (size_t)c * D4;
  };
  auto odim = [&](int c) {
    const TDims td = tdims(g, row, c);
    return dir == 0 ? td.d : td.u;
  };
  int ecentre = 0;
  for (int sw = 0; sw < g.fit; ++sw)
    for (int pass = 0; pass < 2; ++pass) {
      const bool moving_left = (pass == 0) == lr;
      if (moving_left) {
        for (int e = threadIdx.x; e < envT; e += blockDim.x) fb.F[e] = a.triv_t1[e];
        if (threadIdx.x == 0) eF[0] = 0;
        __syncthreads();
        for (int c = 0; c + 1 < Lx; ++c) {
          run_op<R>(OP_COL1_LEFT, D, Dc, fb.F + (size_t)c * envT, Min + (size_t)c * envT, Tc(c),
                    Mout + (size_t)c * envT, nullptr, fb.F + (size_t)(c + 1) * envT, fb.t0, fb.t1, zb.gsm, zb.gism);
          const int e = normalize_pow2(fb.F + (size_t)(c + 1) * envT, envT, red);
          if (threadIdx.x == 0) eF[c + 1] = eF[c] + e;
        }
        for (int e = threadIdx.x; e < envT; e += blockDim.x) fb.G[(size_t)Lx * envT + e] = a.triv_t1[e];
        if (threadIdx.x == 0) eG[Lx] = 0;
        __syncthreads();
        for (int c = Lx - 1; c >= 0; --c) {
          R* P = Mout + (size_t)c * envT;
          run_op<R>(OP_FIT_SITE, D, Dc, fb.F + (size_t)c * envT, Min + (size_t)c * envT, Tc(c),
                    fb.G + (size_t)(c + 1) * envT, nullptr, P, fb.t0, fb.t1, zb.gsm, zb.gism);
          if (c > 0) {
            fit_orthonormalise<R>(P, bdo[c], odim(c), bdo[c + 1], D, Dc, false, fb, red);
            run_op<R>(OP_COL1_RIGHT, D, Dc, fb.G + (size_t)(c + 1) * envT, Min + (size_t)c * envT, Tc(c), P,
                      nullptr, fb.G + (size_t)c * envT, fb.t0, fb.t1, zb.gsm, zb.gism);
            const int e = normalize_pow2(fb.G + (size_t)c * envT, envT, red);
            if (threadIdx.x == 0) eG[c] = eG[c + 1] + e;
            __syncthreads();
          } else {
            ecentre = eF[0] + eG[1];
          }
        }
      } else {
        for (int e = threadIdx.x; e < envT; e += blockDim.x) fb.G[(size_t)Lx * envT + e] = a.triv_t1[e];
        if (threadIdx.x == 0) eG[Lx] = 0;
        __syncthreads();
        for (int c = Lx - 1; c > 0; --c) {
          run_op<R>(OP_COL1_RIGHT, D, Dc, fb.G + (size_t)(c + 1) * envT, Min + (size_t)c * envT, Tc(c),
                    Mout + (size_t)c * envT, nullptr, fb.G + (size_t)c * envT, fb.t0, fb.t1, zb.gsm, zb.gism);
          const int e = normalize_pow2(fb.G + (size_t)c * envT, envT, red);
          if (threadIdx.x == 0) eG[c] = eG[c + 1] + e;
        }
        for (int e = threadIdx.x; e < envT; e += blockDim.x) fb.F[e] = a.triv_t1[e];
        if (threadIdx.x == 0) eF[0] = 0;
        __syncthreads();
        for (int c = 0; c < Lx; ++c) {
          R* P = Mout + (size_t)c * envT;
          run_op<R>(OP_FIT_SITE, D, Dc, fb.F + (size_t)c * envT, Min + (size_t)c * envT, Tc(c),
                    fb.G + (size_t)(c + 1) * envT, nullptr, P, fb.t0, fb.t1, zb.gsm, zb.gism);
          if (c < Lx - 1) {
            fit_orthonormalise<R>(P, bdo[c], odim(c), bdo[c + 1], D, Dc, true, fb, red);
            run_op<R>(OP_COL1_LEFT, D, Dc, fb.F + (size_t)c * envT, Min + (size_t)c * envT, Tc(c), P, nullptr,
                      fb.F + (size_t)(c + 1) * envT, fb.t0, fb.t1, zb.gsm, zb.gism);
            const int e = normalize_pow2(fb.F + (size_t)(c + 1) * envT, envT, red);
            if (threadIdx.x == 0) eF[c + 1] = eF[c] + e;
            __syncthreads();
          } else {
            ecentre = eF[c] + eG[c + 1];
          }
        }
      }
    }
  return ecentre;
}

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
  __shared__ int bdo[kMaxL + 1];   // bond dimensions of the new MPS (for the fit)
  if (threadIdx.x == 0) {
    Cc[0] = R(1);
    bdo[0] = bdo[Lx] = 1;
  }
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
      zip_gemm<R>(zip_lr_step(0, z, D, Dc, sl, sr, si, so), Cc, Min + (size_t)c * envT, zb.Y, zb.gsm, zb.gism,
                  zb.gsm_reals);
      zip_gemm<R>(zip_lr_step(1, z, D, Dc, sl, sr, si, so), zb.Y, T, zb.X, zb.gsm, zb.gism, zb.gsm_reals);
      const int m = z.k * z.o, n = z.b * z.r;
      if (c < Lx - 1) {
        const int K = min(Dc, min(m, n));
        cta_topk_left<R>(zb.X, m, n, K, zb.tw, Mout + (size_t)c * envT, ix2(z.o, D * Dc, Dc), ix1(1), Cn,
                         ix1(n), ix1(1));
        R* t = Cc; Cc = Cn; Cn = t;
        kcur = K;
        if (threadIdx.x == 0) bdo[c + 1] = K;
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
      zip_gemm<R>(zip_rl_step(0, z, D, Dc, sl, sr, si, so), Min + (size_t)c * envT, Cc, zb.Y, zb.gsm, zb.gism,
                  zb.gsm_reals);
      zip_gemm<R>(zip_rl_step(1, z, D, Dc, sl, sr, si, so), zb.Y, T, zb.X, zb.gsm, zb.gism, zb.gsm_reals);
      const int m = z.o * z.k, n = z.a * z.l;
      if (c > 0) {
        const int K = min(Dc, min(m, n));
        cta_topk_left<R>(zb.X, m, n, K, zb.tw, Mout + (size_t)c * envT, ix2(z.k, Dc, 1), ix1(D * Dc), Cn,
                         ix1(1), ix1(K));
        R* t = Cc; Cc = Cn; Cn = t;
        kcur = K;
        if (threadIdx.x == 0) bdo[c] = K;
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
  // variational-fit sweeps on the zip-up result; they end with the centre
  // at `last` again, scaled by 2^-efit
  int efit = 0;
  if (g.fit > 0) {
    __syncthreads();
    efit = fit_row<R>(a, Min, Mout, row, dir, lr, sp, bdo, zb, red);
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
  return efit != 0 ? ldexp(nrm, efit) : nrm;
}

template <typename R>
__device__ void carve_zip(const Geometry& g, R*& p, ZipBufs<R>& zb, R* wm_smem, R* red, double* dred, R* wv,
                          R* gsm, int* gism) {
  zb.dred = dred;
  zb.gsm = gsm;
  zb.gism = gism;
  zb.gsm_reals = (int)(reals_region_bytes(g, sizeof(R), true, wm_smem != nullptr) / sizeof(R));
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
  w.wm_shared = wm_smem != nullptr;
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
  FitBufs<R>& f = zb.fb;
  if (g.fit > 0) {
    const size_t envT = Dc * D * Dc, D4 = D * D * D * D;
    f.F = p; p += (size_t)(g.Lx + 1) * envT;
    f.G = p; p += (size_t)(g.Lx + 1) * envT;
    f.Tt = p; p += (size_t)g.Lx * D4;
    f.QM = p; p += Dc * Dc * D;
    f.QN = p; p += Dc * Dc * D;
    f.qtau = p; p += Dc * D;
    f.t0 = p; p += tmp_elems(g);
    f.t1 = p; p += tmp_elems(g);
    p += 64;
  } else {
    f.F = f.G = f.Tt = f.QM = f.QN = f.qtau = f.t0 = f.t1 = nullptr;
  }
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
