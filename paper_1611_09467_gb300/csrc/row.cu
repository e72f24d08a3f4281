// Single-row sandwich kernels <U_{r-1}| row r |L_{r+1}> (Sec. II): W_r, the
// amplitude ratios of horizontal spin exchanges and Delta = B/W.  One CTA per
// (configuration, row); k_row_fused keeps every intermediate in shared memory
// for (D, Dc) = (2,4), (4,8), (6,12), (8,16).
#include "kernels_common.cuh"

namespace peps {

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
      a.w_row[(size_t)cfg * Ly + r] = ldexp((double)W, eG[0]);
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
      a.w_row[(size_t)cfg * Ly + r] = ldexp((double)W, eG[0]);
      if (!ok) atomicOr(&a.flags[cfg], kFlagZeroW);
    }
  }
}

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
int max_blocks_row(const Geometry& g, int generic) {
  switch (generic ? 0 : row_fused_id<R>(g)) {
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
cudaError_t launch_row(const KArgs<R>& a, int grid, cudaStream_t st, int generic) {
  switch (generic ? 0 : row_fused_id<R>(a.g)) {
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

#define PEPS_INST(R)                                                                                    \
  template int max_blocks_row<R>(const Geometry&, int);                                                 \
  template cudaError_t launch_row<R>(const KArgs<R>&, int, cudaStream_t, int);
PEPS_INST(double)
PEPS_INST(float)

}  // namespace peps
