// Metropolis sweeps (sampling with weight W^2, Sec. II) over nearest-neighbour
// spin exchanges, one CTA per chain.
#include "kernels_common.cuh"

namespace peps {

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
#define PEPS_INST(R)                                                                                    \
  template int max_blocks_mc<R>(const Geometry&);                                                       \
  template cudaError_t launch_mc<R>(const KArgs<R>&, uint64_t*, int, uint64_t, uint64_t, uint64_t,      \
                                    long long*, int, cudaStream_t);
PEPS_INST(double)
PEPS_INST(float)

}  // namespace peps
