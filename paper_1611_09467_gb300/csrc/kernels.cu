// CUDA kernels of the PEPS sampling path (sm_103a): layouts, the boundary
// sweeps, E_loc and gradient reductions, the GO update and the
// allocation-free amplitudes.  The sandwich kernels are in row.cu and pair.cu,
// the Metropolis kernel in mc.cu.
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
#include <mutex>

#include "kernels_common.cuh"

namespace peps {

// ---------------------------------------------------------------- layouts
size_t wm_smem_bytes(const Geometry& g, size_t elem) {
  const size_t P = (size_t)g.Dc * g.D;
  return P * (P + 1) * elem;
}

// Dynamic shared memory of a kernel: a region of reals followed by the GEMM
// offset tables.  For the kernels that truncate, the reals hold (truncation
// matrix if it fits) + the two singular-vector blocks during a truncation and
size_t dyn_smem_bytes(const Geometry& g, size_t elem, bool truncates, bool wm_in_smem) {
  return reals_region_bytes(g, elem, truncates, wm_in_smem) + (size_t)kGemmSmemInts * sizeof(int);
}

bool wm_fits_smem(const Geometry& g, size_t elem) {
  return dyn_smem_bytes(g, elem, true, true) <= 200 * 1024;
}

static size_t zip_elems(const Geometry& g, bool wm_in_smem) {
  const size_t Dc = g.Dc, D = g.D, P = Dc * D;
  return 2 * Dc * Dc * D + Dc * Dc * D * D + P * P + trunc_ws_elems((int)P, g.Dc, !wm_in_smem) + 64 + fit_elems(g);
}

size_t boundary_slot_elems(const Geometry& g, bool wm_in_smem) {
  const size_t envT = (size_t)g.Dc * g.D * g.Dc;
  return zip_elems(g, wm_in_smem) + (size_t)g.Lx * envT;
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

// ------------------------------------------------------------ k_boundary
// One work item: the top-down (dir 0) or bottom-up (dir 1) boundary sweep of
// configuration cfg.  The upper environments U_r go to envU (the last row's
// MPS to `lastbuf`, then closed to psi), the lower ones L_r to envL.
template <typename R>
__device__ void boundary_item(const KArgs<R>& a, int cfg, int dir, R* lastbuf, ZipBufs<R>& zb, R* red,
                              uint64_t* sp, const int* ones) {
  const Geometry& g = a.g;
  const int Lx = g.Lx, Ly = g.Ly, Dc = g.Dc, D = g.D;
  const size_t envT = (size_t)Dc * D * Dc;
  if (a.cache) {
    // this sweep of this configuration is already in place (same bits, same
    // tensors, same workspace): its outputs were kept, only its flag is raised again
    const unsigned bits = a.cache[cfg];
    if (bits & (1u << dir)) {
      if ((bits & (4u << dir)) && threadIdx.x == 0) atomicOr(&a.flags[cfg], kFlagZeroW);
      return;
    }
  }
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
    if (dir == 0 && a.lnU && threadIdx.x == 0) a.lnU[(size_t)cfg * Ly + r] = nrm > 0.0 ? log(nrm) : -INFINITY;
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
  if (a.cache && threadIdx.x == 0) atomicOr(&a.cache[cfg], (1u << dir) | (zero ? (4u << dir) : 0u));
}

__global__ void k_cache_check(const uint64_t* S, uint64_t* Scache, unsigned* bits, int n, int nwords) {
  for (int cfg = blockIdx.x * blockDim.x + threadIdx.x; cfg < n; cfg += gridDim.x * blockDim.x) {
    bool same = true;
    for (int w = 0; w < nwords; ++w) same = same && S[(size_t)cfg * nwords + w] == Scache[(size_t)cfg * nwords + w];
    if (!same) {
      bits[cfg] = 0u;
      for (int w = 0; w < nwords; ++w) Scache[(size_t)cfg * nwords + w] = S[(size_t)cfg * nwords + w];
    }
  }
}

cudaError_t launch_cache_check(const uint64_t* S, uint64_t* Scache, unsigned* bits, int n, int nwords,
                               cudaStream_t st) {
  k_cache_check<<<(n + 127) / 128, 128, 0, st>>>(S, Scache, bits, n, nwords);
  return cudaGetLastError();
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_boundary(KArgs<R> a, int dirs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ R red[64];
  __shared__ uint64_t sp[kMaxWords];
  __shared__ int ones[kMaxDcD + 1];
  __shared__ double dred[kWarps];
  __shared__ R wv[kMaxDcD];
  const Geometry& g = a.g;
  R* p = a.scratch + (size_t)blockIdx.x * a.slot_elems;
  ZipBufs<R> zb;
  R* gsm;
  int* gism;
  smem_split<R>(smem_raw, g, true, a.smem_wm != 0, gsm, gism);
  carve_zip<R>(g, p, zb, a.smem_wm ? gsm : nullptr, red, dred, wv, gsm, gism);
  for (int i = threadIdx.x; i <= g.Lx; i += blockDim.x) ones[i] = 1;
  // items direction-major: consecutive items (one per CTA) share a direction,
  // so sweeps the environment cache skips do not leave half the CTAs idle
  for (int item = blockIdx.x; item < a.n * dirs; item += gridDim.x)
    boundary_item<R>(a, item % a.n, item / a.n, p, zb, red, sp, ones);
}

// The boundary sweeps of several models (lattices, D, Dc of one precision) in
// one persistent launch.  Work items are numbered model after model; start[m]
// is the first item of model m (start[nm] = total), each model contributing
// n * dirs items (direction-major within a model).  Every CTA has one scratch slot of slot_elems reals, sized
// for the largest model, and dynamic shared memory for the largest model; a
// CTA lays its slot and shared memory out again whenever its next item
// belongs to another model.  Per configuration the arithmetic is that of
// k_boundary, so results are bit-identical to separate launches.
template <typename R>
__global__ void __launch_bounds__(kThreads) k_boundary_packed(const KArgs<R>* __restrict__ models,
                                                              const int* __restrict__ start, int nm, int dirs,
                                                              R* scratch, size_t slot_elems) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ R red[64];
  __shared__ uint64_t sp[kMaxWords];
  __shared__ int ones[kMaxDcD + 1];
  __shared__ double dred[kWarps];
  __shared__ R wv[kMaxDcD];
  for (int i = threadIdx.x; i <= kMaxDcD; i += blockDim.x) ones[i] = 1;
  const int total = start[nm];
  int cur = -1;
  ZipBufs<R> zb;
  R* p = nullptr;
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    int m = cur < 0 ? 0 : cur;
    while (m + 1 < nm && start[m + 1] <= item) ++m;
    const KArgs<R>& a = models[m];
    if (m != cur) {
      __syncthreads();
      p = scratch + (size_t)blockIdx.x * slot_elems;
      R* gsm;
      int* gism;
      smem_split<R>(smem_raw, a.g, true, a.smem_wm != 0, gsm, gism);
      carve_zip<R>(a.g, p, zb, a.smem_wm ? gsm : nullptr, red, dred, wv, gsm, gism);
      cur = m;
    }
    const int local = item - start[m];
    boundary_item<R>(a, local % a.n, local / a.n, p, zb, red, sp, ones);
  }
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

// Over the configurations with status 0: sums[0] += sum of E, sums[1] += their
// count, sums[2] += sum of E^2.
__global__ void k_sum_eloc(const double* eloc, const int* status, int n, double* sums) {
  __shared__ double sh[3][kThreads];
  double s = 0, c = 0, q = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    if (status[i] == 0) {
      s += eloc[i];
      c += 1;
      q += eloc[i] * eloc[i];
    }
  sh[0][threadIdx.x] = s;
  sh[1][threadIdx.x] = c;
  sh[2][threadIdx.x] = q;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
      sh[2][threadIdx.x] += sh[2][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sums[0] += sh[0][0];
    sums[1] += sh[1][0];
    sums[2] += sh[2][0];
  }
}

// grad = 2 (<E O> - <E><O>), cov = grad / 2 (Sec. II), from the sums.
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

// Sets *bad when any derivative is NaN or infinite: the update of Sec. III
// moves an entry by the sign of its derivative, and such a derivative has none.
__global__ void k_go_check(const double* grad, size_t n, int* bad) {
  int b = 0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    if (!isfinite(grad[e])) b = 1;
  if (__syncthreads_or(b) && threadIdx.x == 0) atomicOr(bad, 1);
}

cudaError_t launch_go_check(const double* grad, const Geometry& geo, int* bad, int nsm, cudaStream_t st) {
  const size_t n = (size_t)geo.N * 2 * geo.D * geo.D * geo.D * geo.D;
  const size_t blocks = (n + kThreads - 1) / kThreads;
  const int grid = (int)(blocks < (size_t)nsm * 8 ? blocks : (size_t)nsm * 8);
  if (grid < 1) return cudaSuccess;
  k_go_check<<<grid, kThreads, 0, st>>>(grad, n, bad);
  return cudaGetLastError();
}

// The context's working copy of the tensors in FP32, from the FP64 ones.
__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, size_t n) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    b[e] = __double2float_rn(a[e]);
}

cudaError_t launch_to_f32(const double* a, float* b, size_t n, int nsm, cudaStream_t st) {
  const size_t blocks = (n + kThreads - 1) / kThreads;
  const int grid = (int)(blocks < (size_t)nsm * 8 ? blocks : (size_t)nsm * 8);
  if (grid < 1) return cudaSuccess;
  k_to_f32<<<grid, kThreads, 0, st>>>(a, b, n);
  return cudaGetLastError();
}

// Site tensors as the B tiles of the tensor-core two-row step (D = 8): per
// (direction, site, spin) TA[n = (yout, d)][k = (u, yin)] and
// TB[n = (yout, d)][k = (yin, u)] in the core-matrix layout, rounded to TF32
// (to nearest, ties away from zero), with (yin, yout) = (l, r) for direction 0
// and (r, l) for direction 1.  One thread per tile element.
__global__ void k_tc_tiles(const double* __restrict__ A, float* __restrict__ tiles, int N) {
  const size_t total = (size_t)2 * N * 2 * 2 * kTcTile;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int n = (int)(e % 4096) / 64, k = (int)(e % 64);
    const size_t tix = e / 4096;                  // ((dir * N + i) * 2 + sp) * 2 + which
    const int which = (int)(tix % 2), sp = (int)(tix / 2 % 2), i = (int)(tix / 4 % N), dir = (int)(tix / 4 / N);
    const int yout = n >> 3, d = n & 7;
    const int u = which == 0 ? (k >> 3) : (k & 7), yin = which == 0 ? (k & 7) : (k >> 3);
    const int l = dir == 0 ? yin : yout, r = dir == 0 ? yout : yin;
    const float v = __double2float_rn(A[((size_t)i * 2 + sp) * 4096 + l * 512 + r * 64 + u * 8 + d]);
    uint32_t t;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(v));
    const int dst = (n >> 3) * 16 * 32 + (k >> 2) * 32 + (n & 7) * 4 + (k & 3);
    tiles[tix * 4096 + dst] = __uint_as_float(t);
  }
}

cudaError_t launch_tc_tiles(const double* A, float* tiles, int N, int nsm, cudaStream_t st) {
  k_tc_tiles<<<nsm * 4, kThreads, 0, st>>>(A, tiles, N);
  return cudaGetLastError();
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

template <typename R>
int max_blocks_boundary_packed(size_t smem) {
  int dev = 0, nsm = 0, nb = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  prefer_shared(k_boundary_packed<R>, smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_boundary_packed<R>, kThreads, smem);
  return nsm * (nb < 1 ? 1 : nb);
}

template <typename R>
cudaError_t launch_boundary_packed(const KArgs<R>* models_dev, const int* start_dev, int nm, int dirs, R* scratch,
                                   size_t slot_elems, size_t smem, int grid, cudaStream_t st) {
  cudaError_t e = prefer_shared(k_boundary_packed<R>, smem);
  if (e != cudaSuccess) return e;
  k_boundary_packed<R><<<grid, kThreads, smem, st>>>(models_dev, start_dev, nm, dirs, scratch, slot_elems);
  return cudaGetLastError();
}

#define PEPS_INST(R)                                                                                    \
  template int max_blocks_boundary_packed<R>(size_t);                                                   \
  template cudaError_t launch_boundary_packed<R>(const KArgs<R>*, const int*, int, int, R*, size_t, size_t, \
                                                 int, cudaStream_t);                                    \
  template int max_blocks_boundary<R>(const Geometry&);                                                 \
  template cudaError_t launch_boundary<R>(const KArgs<R>&, int, int, cudaStream_t);                     \
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

// A slot is what k_boundary's slot holds (the zip-up buffers carve_zip takes,
// plus one boundary MPS) and one more boundary MPS: the sweep keeps the
// current and the next MPS, where k_boundary writes the next one to the
// environment array.
static size_t static_slot_elems(const Geometry& g, bool wm_in_smem) {
  const size_t envT = (size_t)g.Dc * g.D * g.Dc;
  return (boundary_slot_elems(g, wm_in_smem) + (size_t)g.Lx * envT + 63) / 64 * 64;
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

// Device address of the static scratch.  In host code the array's name is a
// stand-in, not a device address, so the address is looked up with
// cudaGetSymbolAddress, with the device current, the first time a context
// calls in.  The cache is keyed by the current CUDA context (not by the
// device ordinal): after cudaDeviceReset, or under another context on the same
// device, the module is loaded again at a new address, and the new context
// misses the cache and looks the address up again.
typedef int (*CtxGetCurrentFn)(void** ctx);

static CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (CtxGetCurrentFn)f;
  }
  return fn;
}

struct StaticPtr {
  void* ctx;
  void* ptr;
};
static StaticPtr g_static_ptr[64];
static int g_static_n = 0;
static std::mutex g_static_mu;

static cudaError_t static_scratch_ptr(void** out) {
  std::lock_guard<std::mutex> lock(g_static_mu);
  CtxGetCurrentFn get = ctx_get_current();
  void* ctx = nullptr;
  if (get && get(&ctx) == 0 && ctx) {
    for (int i = 0; i < g_static_n; ++i)
      if (g_static_ptr[i].ctx == ctx) {
        *out = g_static_ptr[i].ptr;
        return cudaSuccess;
      }
  }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);   // makes the device's context current if needed
  if (e != cudaSuccess) return e;
  ctx = nullptr;
  if (get && get(&ctx) == 0 && ctx) {
    int slot = -1;
    for (int i = 0; i < g_static_n; ++i)
      if (g_static_ptr[i].ctx == ctx) slot = i;
    if (slot < 0) slot = g_static_n < 64 ? g_static_n++ : 0;
    g_static_ptr[slot] = {ctx, p};
  }
  *out = p;
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
  g.fit = 0;
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

#ifdef PEPS_PHASE_TIMING
// Diagnostic build only: copies the truncation's phase counters (cycles
// summed over CTAs, see PEPS_PHASE) to out[16] and optionally clears them.
extern "C" int peps_phase_read(unsigned long long* out, int reset) {
  if (cudaDeviceSynchronize() != cudaSuccess) return 1;
  if (cudaMemcpyFromSymbol(out, ::peps_phase_cyc, 16 * sizeof(unsigned long long)) != cudaSuccess) return 1;
  if (reset) {
    const unsigned long long z[16] = {0};
    if (cudaMemcpyToSymbol(::peps_phase_cyc, z, sizeof(z)) != cudaSuccess) return 1;
  }
  return 0;
}
#endif
