// Sampled spin-spin correlations and the staggered magnetisation (Sec. IV).
//
// For configurations drawn with weight W(S)^2 (Sec. II) the local value of
// S_i.S_j (i != j) is S^z_i S^z_j + [s_i != s_j] W(S^ij) / (2 W(S)), S^ij the
// configuration with s_i and s_j exchanged.  The paper's M^2 is the staggered
// sum (1/n^2) sum_{p,q} eps_p eps_q <S_p.S_q> over the n central sites.
//
// k_corr computes the exchange ratios of every antiparallel pair p < q of
// central sites, one CTA per (configuration, first site i = sites[p]):
// starting from the configuration's upper environment U_{r_i - 1}, it absorbs
// row r_i with s_i flipped and then the following rows (zip-up truncation to
// Dc, as k_boundary), and in every row r >= r_i meets the row and the lower
// environment L_{r+1} in a single-row sandwich; the site environment B_j of
// each later central site j, contracted with j's flipped tensor, is
// W(S^ij) up to the norms the sweeps divided out.  The ratio divides by the
// configuration's own single-row sandwich W_r (k_row) and carries the
// difference of the per-row log norms of the two sweeps above row r.
#include <algorithm>

#include "kernels_common.cuh"

namespace peps {

size_t corr_slot_elems(const Geometry& g, bool wm_in_smem) {
  const size_t envT = (size_t)g.Dc * g.D * g.Dc, D4 = (size_t)g.D * g.D * g.D * g.D;
  // zip-up buffers and one MPS (as k_boundary), a second MPS, the row's right
  // transfers, two left transfers, the site environment, two GEMM temporaries
  return boundary_slot_elems(g, wm_in_smem) + (size_t)g.Lx * envT + (size_t)(g.Lx + 1) * envT + 2 * envT + D4 +
         2 * tmp_elems(g) + 64;
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_corr(KArgs<R> a, CorrArgs c) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ R red[64];
  __shared__ uint64_t sp[kMaxWords];
  __shared__ int ones[kMaxDcD + 1];
  __shared__ double dred[kWarps];
  __shared__ R wv[kMaxDcD];
  __shared__ int eG[kMaxL + 1];   // G_col is stored scaled by 2^-eG[col]
  const Geometry& g = a.g;
  const int Lx = g.Lx, Ly = g.Ly, Dc = g.Dc, D = g.D;
  const size_t envT = (size_t)Dc * D * Dc;
  const int D4 = D * D * D * D;
  R* p = a.scratch + (size_t)blockIdx.x * c.slot_elems;
  ZipBufs<R> zb;
  R* gsm;
  int* gism;
  smem_split<R>(smem_raw, g, true, a.smem_wm != 0, gsm, gism);
  carve_zip<R>(g, p, zb, a.smem_wm ? gsm : nullptr, red, dred, wv, gsm, gism);
  R* Mbuf[2];
  Mbuf[0] = p; p += (size_t)Lx * envT;
  Mbuf[1] = p; p += (size_t)Lx * envT;
  R* Gb = p; p += (size_t)(Lx + 1) * envT;
  R* F0 = p; p += envT;
  R* F1 = p; p += envT;
  R* Bb = p; p += D4;
  R* t0 = p; p += tmp_elems(g);
  R* t1 = p;
  for (int k = threadIdx.x; k <= Lx; k += blockDim.x) ones[k] = 1;
  for (int item = blockIdx.x; item < a.n * c.nc; item += gridDim.x) {
    const int cfg = item / c.nc, pi = item % c.nc;
    const int i = c.sites[pi], ri = i / Lx;
    __syncthreads();
    for (int k = threadIdx.x; k < g.nwords; k += blockDim.x) sp[k] = a.S[(size_t)cfg * g.nwords + k];
    __syncthreads();
    if (c.status[cfg] != 0) continue;             // W(S) = 0 or S^z != 0: no ratios (uniform across the CTA)
    const int si = spin_of(sp, i);
    __syncthreads();
    if (threadIdx.x == 0) sp[i >> 6] ^= 1ull << (i & 63);   // S with s_i flipped
    const R* U0 = ri == 0 ? a.triv_mps : a.envU + ((size_t)cfg * Ly + (ri - 1)) * Lx * envT;
    for (size_t e = threadIdx.x; e < (size_t)Lx * envT; e += blockDim.x) Mbuf[0][e] = U0[e];
    __syncthreads();
    const double epsi = ((i / Lx + i % Lx) % 2 == 0) ? 1.0 : -1.0;
    double xs = 0.0, lsdiff = 0.0;
    int cur = 0;
    for (int r = ri; r < Ly; ++r) {
      const R* Mu = Mbuf[cur];
      const R* Md = r == Ly - 1 ? a.triv_mps : a.envL + ((size_t)cfg * Ly + (r + 1)) * Lx * envT;
      const double Wr = a.w_row[(size_t)cfg * Ly + r];
      // right transfers of the (modified) row
      for (int e = threadIdx.x; e < (int)envT; e += blockDim.x) Gb[(size_t)Lx * envT + e] = a.triv_t1[e];
      if (threadIdx.x == 0) eG[Lx] = 0;
      __syncthreads();
      int eacc = 0;
      for (int col = Lx - 1; col >= 0; --col) {
        const int site = r * Lx + col;
        run_op<R>(OP_COL1_RIGHT, D, Dc, Gb + (size_t)(col + 1) * envT, Mu + (size_t)col * envT,
                  tptr(a, site, spin_of(sp, site)), Md + (size_t)col * envT, nullptr, Gb + (size_t)col * envT, t0,
                  t1, gsm, gism);
        eacc += normalize_pow2(Gb + (size_t)col * envT, (int)envT, red);
        if (threadIdx.x == 0) eG[col] = eacc;
      }
      __syncthreads();
      const R* F = a.triv_t1;
      int eF = 0;
      R* Fn = F0;
      for (int col = 0; col < Lx; ++col) {
        const int j = r * Lx + col;
        const int sj = spin_of(sp, j);            // unchanged for j != i
        const int pj = c.pos[j];
        if (pj >= 0 && j > i && sj != si) {
          run_op<R>(OP_SITE_ENV, D, Dc, F, Mu + (size_t)col * envT, Md + (size_t)col * envT,
                    Gb + (size_t)(col + 1) * envT, nullptr, Bb, t0, t1, gsm, gism);
          const R w = block_dot(Bb, tptr(a, j, 1 - sj), D4, red);
          const double ratio = (Wr != 0.0 && lsdiff > -INFINITY)
                                   ? ldexp((double)w, eF + eG[col + 1]) / Wr * exp(lsdiff)
                                   : 0.0;
          const double epsj = ((j / Lx + j % Lx) % 2 == 0) ? 1.0 : -1.0;
          xs += epsi * epsj * ratio;
          if (c.corr && threadIdx.x == 0) {
            atomicAdd(&c.corr[(size_t)pi * c.nc + pj], 0.5 * ratio);
            atomicAdd(&c.corr[(size_t)pj * c.nc + pi], 0.5 * ratio);
          }
        }
        if (col < Lx - 1) {
          run_op<R>(OP_COL1_LEFT, D, Dc, F, Mu + (size_t)col * envT, tptr(a, j, sj), Md + (size_t)col * envT,
                    nullptr, Fn, t0, t1, gsm, gism);
          eF += normalize_pow2(Fn, (int)envT, red);
          F = Fn;
          Fn = (Fn == F0) ? F1 : F0;
        }
      }
      if (r < Ly - 1) {
        const int* bdin = r == 0 ? ones : a.bd + (size_t)(r - 1) * (Lx + 1);
        const double nrm = absorb_row<R>(a, Mbuf[cur], Mbuf[cur ^ 1], r, 0, (r % 2) == 0, bdin, sp, zb, red);
        lsdiff += (nrm > 0.0 ? log(nrm) : -INFINITY) - a.lnU[(size_t)cfg * Ly + r];
        cur ^= 1;
      }
    }
    if (threadIdx.x == 0 && xs != 0.0) atomicAdd(&c.xsum[cfg], xs);
  }
}

// M^2 per configuration: (1/n^2) [n/2 + (sum_p eps_p S^z_p)^2 + xsum] over the
// n central sites (the i = j terms give 3/4 each, the S^z S^z terms of i != j
// (sum eps S^z)^2 - n/4, the exchanges twice the p < q sum); NaN for a
// configuration with a non-zero status.
__global__ void k_corr_m2(Geometry g, CorrArgs c, const uint64_t* S, int n, const int* status, double* m2) {
  for (int cfg = blockIdx.x * blockDim.x + threadIdx.x; cfg < n; cfg += gridDim.x * blockDim.x) {
    if (status[cfg] != 0) {
      m2[cfg] = NAN;
      continue;
    }
    const uint64_t* sp = S + (size_t)cfg * g.nwords;
    double stag = 0.0;
    for (int p = 0; p < c.nc; ++p) {
      const int i = c.sites[p];
      const double sz = spin_of(sp, i) ? -0.5 : 0.5;
      stag += (((i / g.Lx + i % g.Lx) % 2 == 0) ? 1.0 : -1.0) * sz;
    }
    const double nc = (double)c.nc;
    m2[cfg] = (0.5 * nc + stag * stag + c.xsum[cfg]) / (nc * nc);
  }
}

// corr[p][q] += sum over configurations with status 0 of S^z_p S^z_q (p != q),
// 3/4 per configuration on the diagonal.
__global__ void k_corr_zz(Geometry g, CorrArgs c, const uint64_t* S, int n, const int* status) {
  const size_t total = (size_t)c.nc * c.nc;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / c.nc), q = (int)(e % c.nc);
    const int i = c.sites[p], j = c.sites[q];
    double s = 0.0;
    for (int cfg = 0; cfg < n; ++cfg) {
      if (status[cfg] != 0) continue;
      if (p == q) {
        s += 0.75;
        continue;
      }
      const uint64_t* sp = S + (size_t)cfg * g.nwords;
      s += (spin_of(sp, i) == spin_of(sp, j)) ? 0.25 : -0.25;
    }
    c.corr[e] += s;
  }
}

template <typename R>
int max_blocks_corr(const Geometry& g) {
  int dev = 0, nsm = 0, nb = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = dyn_smem_bytes(g, sizeof(R), true, wm_fits_smem(g, sizeof(R)));
  prefer_shared(k_corr<R>, smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_corr<R>, kThreads, smem);
  return nsm * (nb < 1 ? 1 : nb);
}

template <typename R>
cudaError_t launch_corr(const KArgs<R>& a, const CorrArgs& c, int grid, cudaStream_t st) {
  const size_t smem = dyn_smem_bytes(a.g, sizeof(R), true, a.smem_wm != 0);
  cudaError_t e = prefer_shared(k_corr<R>, smem);
  if (e != cudaSuccess) return e;
  k_corr<R><<<grid, kThreads, smem, st>>>(a, c);
  return cudaGetLastError();
}

cudaError_t launch_corr_finalize(const Geometry& g, const CorrArgs& c, const uint64_t* S, int n, const int* status,
                                 double* m2, cudaStream_t st) {
  if (m2) {
    k_corr_m2<<<(n + 127) / 128, 128, 0, st>>>(g, c, S, n, status, m2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (c.corr) {
    const size_t total = (size_t)c.nc * c.nc;
    k_corr_zz<<<(int)std::min<size_t>((total + 127) / 128, 65535), 128, 0, st>>>(g, c, S, n, status);
  }
  return cudaGetLastError();
}

#define PEPS_INST(R)                                                                                    \
  template int max_blocks_corr<R>(const Geometry&);                                                     \
  template cudaError_t launch_corr<R>(const KArgs<R>&, const CorrArgs&, int, cudaStream_t);
PEPS_INST(double)
PEPS_INST(float)

}  // namespace peps
