// Fused two-row transfer step (sandwich <U_{r-1}| rows r,r+1 |L_{r+2}>, one
// column) with every intermediate in shared memory.
//
// Direction-normalised form.  A transfer is stored [x'][x][y1][y2]: x' the
// bond of the lower environment L, x the bond of the upper environment U,
// y1 / y2 the horizontal bonds of rows r / r+1.  One step consumes the 'in'
// bonds of a column and produces its 'out' bonds:
//   left  (E_{c-1} -> E_c): in = (a, a', l1, l2), out = (b, b', r1, r2)
//   right (H_{c+1} -> H_c): in = (b, b', r1, r2), out = (a, a', l1, l2)
// so that <E_{c-1} | column c | H_{c+1}> is an elementwise product of E and H.
// The step is split over the in-bond x'_in of L (Dc slices); per slice
//   s1: P1[(y1i,u1)][(y2i,xo)]      = sum_{xi}        Ein[s][xi][y1i][y2i] Mu[xi][u1][xo]
//   s2: P2[(y2i,m)][(xo,y1o)]       = sum_{y1i,u1}    P1 T1[y1i][y1o][u1][m]
//   s3: P3[d2][(xo,y1o,y2o)]        = sum_{y2i,m}     P2 T2[y2i][y2o][m][d2]
//   s4: acc[(xo,y1o,y2o)][x'o]     += sum_{d2}        P3 Md[s][d2][x'o]
// with the accumulator in registers across slices.  This is the contraction
// of col2_left_step / col2_right_step, reordered; results agree to rounding.
#pragma once

#include "device.cuh"

namespace peps {

template <int D, int Dc>
struct PairSmem {
  static constexpr int DD = D * D;
  static constexpr int P1 = DD * D * Dc;     // also holds P3
  static constexpr int P2 = D * Dc * DD;
  static constexpr int T = DD * DD;
  static constexpr int MU = Dc * D * Dc;
  static constexpr int ES = Dc * DD;
  static constexpr int MD = D * Dc;
  static constexpr int total = P1 + P2 + 2 * T + MU + ES + MD;
  static constexpr int ROWS = Dc * DD;       // rows of the output (xo, y1o, y2o)
  static constexpr int RPT = (ROWS + kThreads - 1) / kThreads;   // rows per thread
};

// Four consecutive reals from a 16-byte aligned shared-memory address.
template <typename R>
__device__ __forceinline__ void load4(const R* p, R (&v)[4]) {
  if constexpr (sizeof(R) == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else {
    const double2 a = *reinterpret_cast<const double2*>(p);
    const double2 b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
}

// C[i][j] for a k-major pair A[K][M], B[K][N] in shared memory; the caller's
// functor places each output.  Every thread handles 4x4 micro-tiles.
template <typename R, int M, int N, int K, class Store>
__device__ __forceinline__ void smem_gemm_km(const R* __restrict__ A, const R* __restrict__ B, Store st) {
  constexpr int TMc = (M + 3) / 4, TNc = (N + 3) / 4;
  for (int t = threadIdx.x; t < TMc * TNc; t += kThreads) {
    const int i0 = (t / TNc) * 4, j0 = (t % TNc) * 4;
    R acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = R(0);
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
      R av[4], bv[4];
      if constexpr (M % 4 == 0 && N % 4 == 0) {
        // 16-byte groups (the callers' blocks start at multiples of 4 reals)
        load4(A + k * M + i0, av);
        load4(B + k * N + j0, bv);
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          av[q] = (M % 4 == 0 || i0 + q < M) ? A[k * M + i0 + q] : R(0);
          bv[q] = (N % 4 == 0 || j0 + q < N) ? B[k * N + j0 + q] : R(0);
        }
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b)
        if ((M % 4 == 0 || i0 + a < M) && (N % 4 == 0 || j0 + b < N)) st(i0 + a, j0 + b, acc[a][b]);
  }
}

// Two products C_h[i][j] = sum_k A_h[k][i] B_h[k][j] (h = 0, 1) of one shape
// (k-major, shared memory), both at once on TA x 4 micro-tiles: where one
// product has too few 4x4 tiles to occupy the CTA (M = D rows), the two
// together fill it with TA = 2; with a long reduction TA = 4 halves the
// shared-memory reads per multiply-add.  Each output is the same
// left-to-right chain of FMAs over k as in smem_gemm_km.  B rows (and A rows
// when TA = 4) are read as 16-byte groups: N (M), the offsets of the blocks
// and their rows must be multiples of 4 reals.  The functor gets (h, i, j,
// value).
template <typename R, int M, int N, int K, class Store, int TA = 2>
__device__ __forceinline__ void smem_gemm_km_x2(const R* __restrict__ A0, const R* __restrict__ A1,
                                                const R* __restrict__ B0, const R* __restrict__ B1, Store st) {
  static_assert(N % 4 == 0, "B rows are read as groups of four");
  static_assert(TA == 2 || (TA == 4 && M % 4 == 0), "A rows are read as groups of four");
  constexpr int TB = 4;
  constexpr int TMc = (M + TA - 1) / TA, TNc = N / TB, NT = TMc * TNc;
  for (int t = threadIdx.x; t < 2 * NT; t += kThreads) {
    const int h = t / NT, tt = t - h * NT;
    const R* A = h ? A1 : A0;
    const R* B = h ? B1 : B0;
    const int i0 = (tt / TNc) * TA, j0 = (tt % TNc) * TB;
    R acc[TA][TB];
#pragma unroll
    for (int a = 0; a < TA; ++a)
#pragma unroll
      for (int b = 0; b < TB; ++b) acc[a][b] = R(0);
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
      R av[TA], bv[TB];
      if constexpr (TA == 4) {
        load4(A + k * M + i0, av);
      } else {
#pragma unroll
        for (int q = 0; q < TA; ++q) av[q] = (M % TA == 0 || i0 + q < M) ? A[k * M + i0 + q] : R(0);
      }
      load4(B + k * N + j0, bv);
#pragma unroll
      for (int a = 0; a < TA; ++a)
#pragma unroll
        for (int b = 0; b < TB; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < TA; ++a)
#pragma unroll
      for (int b = 0; b < TB; ++b)
        if (M % TA == 0 || i0 + a < M) st(h, i0 + a, j0 + b, acc[a][b]);
  }
}

// One fused two-row transfer step.  right == false: left step (E_{c-1} -> E_c);
// right == true: right step (H_{c+1} -> H_c).  Mu, Md: padded [Dc][D][Dc]
// boundary-MPS tensors of column c; T1, T2: padded [l][r][u][d] site
// tensors of rows r, r+1 at the chosen spins.  If Hdot is null the result is
// written to Eout scaled by 2^-e (pow2_exponent of its largest entry) and e
// is stored in *e_out; otherwise <result, Hdot> is returned (all threads) and
// nothing is written.  Ends with a barrier.
template <typename R, int D, int Dc>
__device__ R pair_step_fused(bool right, const R* Ein, R* __restrict__ Eout, const R* __restrict__ Mu,
                             const R* __restrict__ T1, const R* __restrict__ T2, const R* __restrict__ Md,
                             const R* Hdot, R* sm, R* red, int* e_out = nullptr) {
  using S = PairSmem<D, Dc>;
  constexpr int DD = S::DD, D3 = DD * D;
  R* P1 = sm;
  R* P2 = P1 + S::P1;
  R* T1s = P2 + S::P2;
  R* T2s = T1s + S::T;
  R* Mus = T2s + S::T;
  R* Es = Mus + S::MU;
  R* Mds = Es + S::ES;
  R* P3 = P1;
  const int tid = threadIdx.x;
  __syncthreads();
  // direction-normalised copies: T?s[(yin,u)][(yout,d)], Mus[xin][(u,xout)]
  for (int e = tid; e < S::T; e += kThreads) {
    const int yin = e / D3, u = (e / DD) % D, yout = (e / D) % D, d = e % D;
    const int l = right ? yout : yin, r = right ? yin : yout;
    const int src = l * D3 + r * DD + u * D + d;
    T1s[e] = T1[src];
    T2s[e] = T2[src];
  }
  for (int e = tid; e < S::MU; e += kThreads) {
    const int xin = e / (D * Dc), u = (e / Dc) % D, xout = e % Dc;
    const int a = right ? xout : xin, b = right ? xin : xout;
    Mus[e] = Mu[a * D * Dc + u * Dc + b];
  }
  R acc[S::RPT][Dc];
#pragma unroll
  for (int q = 0; q < S::RPT; ++q)
#pragma unroll
    for (int x = 0; x < Dc; ++x) acc[q][x] = R(0);
  for (int s = 0; s < Dc; ++s) {
    // slice s of the input transfer ([x'][x][y1][y2] is slice-contiguous) and of Md
    for (int e = tid; e < S::ES; e += kThreads) Es[e] = Ein[s * S::ES + e];
    for (int e = tid; e < S::MD; e += kThreads) {
      const int d = e / Dc, xo = e % Dc;
      Mds[e] = right ? Md[xo * D * Dc + d * Dc + s] : Md[s * D * Dc + d * Dc + xo];
    }
    __syncthreads();
    // s1: rows (y1i, y2i), cols (u1, xo), k = xi
    smem_gemm_km<R, DD, D * Dc, Dc>(Es, Mus, [&](int i, int j, R v) {
      const int y1 = i / D, y2 = i % D, u1 = j / Dc, xo = j % Dc;
      P1[(y1 * D + u1) * (D * Dc) + y2 * Dc + xo] = v;
    });
    __syncthreads();
    // s2: rows (y2i, xo), cols (y1o, m), k = (y1i, u1)
    smem_gemm_km<R, D * Dc, DD, DD>(P1, T1s, [&](int i, int j, R v) {
      const int y2 = i / Dc, xo = i % Dc, y1o = j / D, m = j % D;
      P2[(y2 * D + m) * (Dc * D) + xo * D + y1o] = v;
    });
    __syncthreads();
    // s3: rows (xo, y1o), cols (y2o, d2), k = (y2i, m)
    smem_gemm_km<R, Dc * D, DD, DD>(P2, T2s, [&](int i, int j, R v) {
      const int y2o = j / D, d2 = j % D;
      P3[d2 * (Dc * DD) + i * D + y2o] = v;
    });
    __syncthreads();
    // s4: acc[(xo,y1o,y2o)][x'o] += sum_d2 P3[d2][row] Mds[d2][x'o]
#pragma unroll
    for (int d2 = 0; d2 < D; ++d2) {
#pragma unroll
      for (int q = 0; q < S::RPT; ++q) {
        const int row = q * kThreads + tid;
        if (S::ROWS % kThreads == 0 || row < S::ROWS) {
          const R p = P3[d2 * S::ROWS + row];
#pragma unroll
          for (int x = 0; x < Dc; ++x) acc[q][x] = fma(p, Mds[d2 * Dc + x], acc[q][x]);
        }
      }
    }
    __syncthreads();
  }
  R dot = R(0);
  if (Hdot == nullptr) {
    R mx = R(0);
#pragma unroll
    for (int q = 0; q < S::RPT; ++q) {
      const int row = q * kThreads + tid;
      if (S::ROWS % kThreads == 0 || row < S::ROWS)
#pragma unroll
        for (int x = 0; x < Dc; ++x) mx = fmax(mx, fabs(acc[q][x]));
    }
    const int e = pow2_exponent(block_max(mx, red));
    const R sc = pow2<R>(-e);
    if (e_out) *e_out = e;
#pragma unroll
    for (int q = 0; q < S::RPT; ++q) {
      const int row = q * kThreads + tid;
      if (S::ROWS % kThreads == 0 || row < S::ROWS)
#pragma unroll
        for (int x = 0; x < Dc; ++x) Eout[x * S::ROWS + row] = acc[q][x] * sc;
    }
    __syncthreads();
  } else {
#pragma unroll
    for (int q = 0; q < S::RPT; ++q) {
      const int row = q * kThreads + tid;
      if (S::ROWS % kThreads == 0 || row < S::ROWS)
#pragma unroll
        for (int x = 0; x < Dc; ++x) dot = fma(acc[q][x], Hdot[x * S::ROWS + row], dot);
    }
    dot = block_sum(dot, red);
  }
  return dot;
}

}  // namespace peps
