// Two-row sandwich kernels <U_{r-1}| rows r,r+1 |L_{r+2}> (Sec. II): ratios
// of vertical and diagonal exchanges.  One CTA per (configuration, row pair):
// k_pair (generic), k_pair_fused (shared-memory slices, fixed D and Dc) and
// k_pair_tc (tcgen05 tensor cores, TF32, D = 8, Dc = 16).
#include "kernels_common.cuh"

namespace peps {

// ---------------------------------------------------------------- k_pair
template <typename R>
__global__ void __launch_bounds__(kThreads) k_pair(KArgs<R> a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
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
  extern __shared__ __align__(1024) unsigned char smem_raw[];
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
cudaError_t launch_pair(const KArgs<R>& a, int grid, cudaStream_t st, int generic) {
  switch (generic ? 0 : pair_fused_id<R>(a.g)) {
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

#define PEPS_INST(R)                                                                                    \
  template int max_blocks_pair<R>(const Geometry&);                                                     \
  template int max_blocks_pair_fused<R>(const Geometry&);                                               \
  template cudaError_t launch_pair<R>(const KArgs<R>&, int, cudaStream_t, int);
PEPS_INST(double)
PEPS_INST(float)

}  // namespace peps
