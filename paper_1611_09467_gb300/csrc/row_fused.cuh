// Fused single-row transfer step and site environment (sandwich
// <U_{r-1}| row r |L_{r+1}>, Fig. 1c) with every intermediate in shared
// memory.
//
// Direction-normalised form as in pair_fused.cuh.  A single-row transfer is
// stored [x'][x][y] (x' the bond of L, x the bond of U, y the horizontal
// bond), so <F_c, G_{c+1}> is an elementwise dot:
//   left  (F_{c-1} -> F_c): in = (a, a', l), out = (b, b', r)
//   right (G_{c+1} -> G_c): in = (b, b', r), out = (a, a', l)
// One step, sliced over the in-bond s of L:
//   s1: P[(yi,u)][xo]       = sum_xi    Fin[s][xi][yi] Mu[xi][u][xo]
//   s2: Q[d][(xo,yo)]       = sum_yi,u  P T[yi][yo][u][d]
//   s3: acc[x'o][(xo,yo)]  += sum_d     Q Md[s][d][x'o]
// The site environment (the B of Delta = B / W, Sec. II)
//   B[l,r,u,d] = sum F[a,l,a'] Mu[a,u,b] Md[a',d,b'] G[b,r,b']
// pairs F with Mu and Md with G first, sliced over a':
//   X[b][(l,u)]     = sum_a   F[s][a][l] Mu[a][u][b]
//   Y[b][(d,r)]     = sum_b'  Md[s][d][b'] G[b'][b][r]
//   acc[(l,u)][(d,r)] += sum_b X Y
// which needs half the multiply-adds of contracting the three boundary
// tensors into one block first.  Both are the contractions of
// col1_left_step / col1_right_step / site_env_step, reordered; results agree
// to rounding.
#pragma once

#include "pair_fused.cuh"

namespace peps {

template <int D, int Dc>
struct RowSmem {
  static constexpr int DD = D * D, D3 = DD * D, D4 = DD * DD;
  static constexpr int MU = Dc * D * Dc;   // Mu (step: [xi][(u,xo)]; site env: as stored)
  static constexpr int T = DD * DD;        // T as [(yi,u)][(yo,d)]
  static constexpr int FS = Dc * D;        // one slice of a transfer
  static constexpr int MD = D * Dc;        // one slice of Md
  static constexpr int P = DD * Dc;        // P[(yi,u)][xo]
  static constexpr int Q = D * Dc * D;     // Q[d][(xo,yo)]
  // slices are taken in pairs; the F and Md slices of consecutive pairs alternate
  static constexpr int step_total = MU + T + 4 * (FS + MD) + 2 * P + 2 * Q;
  static constexpr int env_total = MU + Dc * FS + 2 * (MD + FS) + 4 * Dc * DD;
  static constexpr int total = step_total > env_total ? step_total : env_total;
  static constexpr int OUT = Dc * D * Dc;  // outputs of a step
  static constexpr int OPT = (OUT + kThreads - 1) / kThreads;   // outputs per thread
  static constexpr int TM = (DD + 3) / 4;  // 4x4 tiles of the site-env accumulator per dimension
  static constexpr int TPT = (TM * TM + kThreads - 1) / kThreads;
  static_assert(D4 <= env_total, "site environment staging must fit the site-env buffers");
  static_assert(Dc % 2 == 0, "slices are processed in pairs");
};

// One fused single-row transfer step.  right == false: F_{c-1} -> F_c;
// right == true: G_{c+1} -> G_c.  Mu, Md: padded [Dc][D][Dc] boundary-MPS
// tensors of column c; T: padded [l][r][u][d] site tensor at the chosen spin.
// If Gdot is null the result is written to Fout scaled by 2^-e
// (pow2_exponent of its largest entry) and e is stored in *e_out; otherwise
// <result, Gdot> is returned (all threads) and nothing is written.  Ends with
// a barrier.
template <typename R, int D, int Dc>
__device__ R row_step_fused(bool right, const R* Fin, R* __restrict__ Fout, const R* __restrict__ Mu,
                            const R* __restrict__ T, const R* __restrict__ Md, const R* Gdot, R* sm,
                            R* red, int* e_out = nullptr) {
  using S = RowSmem<D, Dc>;
  constexpr int DD = S::DD, D3 = S::D3, XY = Dc * D;
  R* Mus = sm;
  R* Ts = Mus + S::MU;
  R* Fs0 = Ts + S::T;             // 4 F slices: pair parity x slice in pair
  R* Mds0 = Fs0 + 4 * S::FS;      // 4 Md slices
  R* Pb0 = Mds0 + 4 * S::MD;      // 2 P blocks (slice in pair)
  R* Qb0 = Pb0 + 2 * S::P;        // 2 Q blocks
  const int tid = threadIdx.x;
  __syncthreads();
  for (int e = tid; e < S::T; e += kThreads) {
    const int yin = e / D3, u = (e / DD) % D, yout = (e / D) % D, d = e % D;
    const int l = right ? yout : yin, r = right ? yin : yout;
    Ts[e] = T[l * D3 + r * DD + u * D + d];
  }
  for (int e = tid; e < S::MU; e += kThreads) {
    const int xin = e / (D * Dc), u = (e / Dc) % D, xout = e % Dc;
    const int a = right ? xout : xin, b = right ? xin : xout;
    Mus[e] = Mu[a * D * Dc + u * Dc + b];
  }
  // Outputs o = x'o * XY + (xo, yo).  When the CTA splits into whole groups
  // of XY threads, thread t owns row (xo, yo) = t % XY and the OPT
  // consecutive x'o from (t / XY) * OPT, so the Q entry of a row is loaded
  // once per d and the Md entries as 16-byte groups; otherwise t owns
  // o = q * kThreads + t.
  constexpr bool grouped = kThreads % XY == 0 && Dc % (kThreads / XY) == 0 && S::OPT == Dc / (kThreads / XY);
  const int grow = tid % XY, gx = (tid / XY) * S::OPT;
  auto out_index = [&](int q) { return grouped ? (gx + q) * XY + grow : q * kThreads + tid; };
  R acc[S::OPT];
#pragma unroll
  for (int q = 0; q < S::OPT; ++q) acc[q] = R(0);
  // three barriers per pair of slices: the slice buffers of consecutive pairs
  // alternate, so loading pair p+1 cannot overwrite what s3 of pair p reads
  for (int s0 = 0; s0 < Dc; s0 += 2) {
    const int par = (s0 >> 1) & 1;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int s = s0 + h;
      R* Fs = Fs0 + (2 * par + h) * S::FS;
      R* Mds = Mds0 + (2 * par + h) * S::MD;
      for (int e = tid; e < S::FS; e += kThreads) Fs[e] = Fin[s * XY + e];   // [xi][yi]
      for (int e = tid; e < S::MD; e += kThreads) {
        const int d = e / Dc, xo = e % Dc;
        Mds[e] = right ? Md[xo * D * Dc + d * Dc + s] : Md[s * D * Dc + d * Dc + xo];
      }
    }
    __syncthreads();
    // the two slices of the pair together: each product alone has too few
    // 4x4 tiles to occupy the CTA
    smem_gemm_km_x2<R, D, D * Dc, Dc>(Fs0 + (2 * par) * S::FS, Fs0 + (2 * par + 1) * S::FS, Mus, Mus,
                                      [&](int h, int i, int j, R v) {
                                        const int u = j / Dc, xo = j % Dc;      // i = yi, j = (u, xo)
                                        Pb0[h * S::P + (i * D + u) * Dc + xo] = v;
                                      });
    __syncthreads();
    auto store_q = [&](int h, int i, int j, R v) {
      const int yo = j / D, d = j % D;          // i = xo, j = (yo, d)
      Qb0[h * S::Q + d * XY + i * D + yo] = v;
    };
    // K = D^2 is long enough for 4x4 tiles when the rows split into fours
    smem_gemm_km_x2<R, Dc, DD, DD, decltype(store_q), Dc % 4 == 0 ? 4 : 2>(Pb0, Pb0 + S::P, Ts, Ts, store_q);
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const R* Qb = Qb0 + h * S::Q;
      const R* Mds = Mds0 + (2 * par + h) * S::MD;
      if constexpr (grouped) {
        // per output the same chain of FMAs over d as below
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const R qv = Qb[d * XY + grow];
          R md[S::OPT];
          if constexpr (sizeof(R) == 4 && S::OPT % 4 == 0) {
#pragma unroll
            for (int q = 0; q < S::OPT; q += 4) {
              const float4 m4 = *reinterpret_cast<const float4*>(Mds + d * Dc + gx + q);
              md[q] = m4.x; md[q + 1] = m4.y; md[q + 2] = m4.z; md[q + 3] = m4.w;
            }
          } else {
#pragma unroll
            for (int q = 0; q < S::OPT; ++q) md[q] = Mds[d * Dc + gx + q];
          }
#pragma unroll
          for (int q = 0; q < S::OPT; ++q) acc[q] = fma(qv, md[q], acc[q]);
        }
      } else {
#pragma unroll
        for (int q = 0; q < S::OPT; ++q) {
          const int o = q * kThreads + tid;
          if (S::OUT % kThreads == 0 || o < S::OUT) {
            const int row = o % XY, xo2 = o / XY;
            R v = acc[q];
#pragma unroll
            for (int d = 0; d < D; ++d) v = fma(Qb[d * XY + row], Mds[d * Dc + xo2], v);
            acc[q] = v;
          }
        }
      }
    }
  }
  R dot = R(0);
  if (Gdot == nullptr) {
    R mx = R(0);
#pragma unroll
    for (int q = 0; q < S::OPT; ++q)
      if (grouped || S::OUT % kThreads == 0 || q * kThreads + tid < S::OUT) mx = fmax(mx, fabs(acc[q]));
    const int e = pow2_exponent(block_max(mx, red));
    const R sc = pow2<R>(-e);
    if (e_out) *e_out = e;
#pragma unroll
    for (int q = 0; q < S::OPT; ++q) {
      const int o = out_index(q);
      if (grouped || S::OUT % kThreads == 0 || o < S::OUT) Fout[o] = acc[q] * sc;
    }
    __syncthreads();
  } else {
#pragma unroll
    for (int q = 0; q < S::OPT; ++q) {
      const int o = out_index(q);
      if (grouped || S::OUT % kThreads == 0 || o < S::OUT) dot = fma(acc[q], Gdot[o], dot);
    }
    dot = block_sum(dot, red);
  }
  return dot;
}

// Site environment of column c, scaled: Bout[l][r][u][d] = scale * B, from
// F_{c-1} ([a'][a][l]), Mu, Md (padded [Dc][D][Dc]) and G_{c+1} ([b'][b][r]).
// Ends with a barrier.
template <typename R, int D, int Dc>
__device__ void site_env_fused(const R* F, const R* __restrict__ Mu, const R* __restrict__ Md,
                               const R* G, R scale, R* __restrict__ Bout, R* sm) {
  using S = RowSmem<D, Dc>;
  constexpr int DD = S::DD, D3 = S::D3, XY = Dc * D, TM = S::TM;
  R* Mus = sm;                 // Mu as stored: [a][(u,b)]
  R* Gs = Mus + S::MU;         // G: [b'][(b,r)]
  R* Mdk0 = Gs + Dc * XY;      // two slices of Md: [b'][d]
  R* Fs0 = Mdk0 + 2 * S::MD;   // two slices of F: [a][l]
  R* Xs0 = Fs0 + 2 * S::FS;    // two [b][(l,u)]
  R* Ys0 = Xs0 + 2 * Dc * DD;  // two [b][(d,r)]
  const int tid = threadIdx.x;
  __syncthreads();
  for (int e = tid; e < S::MU; e += kThreads) Mus[e] = Mu[e];
  for (int e = tid; e < Dc * XY; e += kThreads) Gs[e] = G[e];
  R acc[S::TPT][4][4];
#pragma unroll
  for (int t = 0; t < S::TPT; ++t)
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[t][i][j] = R(0);
  // three barriers per pair of slices of a'
  for (int s0 = 0; s0 < Dc; s0 += 2) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int s = s0 + h;
      R* Mdk = Mdk0 + h * S::MD;
      R* Fs = Fs0 + h * S::FS;
      for (int e = tid; e < S::MD; e += kThreads) {
        const int bp = e / D, d = e % D;
        Mdk[e] = Md[s * D * Dc + d * Dc + bp];
      }
      for (int e = tid; e < S::FS; e += kThreads) Fs[e] = F[s * XY + e];
    }
    __syncthreads();
    // X: rows l, cols (u, b), k = a;  Y: rows d, cols (b, r), k = b'
    smem_gemm_km_x2<R, D, D * Dc, Dc>(Fs0, Fs0 + S::FS, Mus, Mus, [&](int h, int i, int j, R v) {
      Xs0[h * Dc * DD + (j % Dc) * DD + i * D + j / Dc] = v;
    });
    smem_gemm_km_x2<R, D, Dc * D, Dc>(Mdk0, Mdk0 + S::MD, Gs, Gs, [&](int h, int i, int j, R v) {
      Ys0[h * Dc * DD + (j / D) * DD + i * D + j % D] = v;
    });
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const R* Xs = Xs0 + h * Dc * DD;
      const R* Ys = Ys0 + h * Dc * DD;
#pragma unroll
      for (int t = 0; t < S::TPT; ++t) {
        const int tile = t * kThreads + tid;
        if ((TM * TM) % kThreads == 0 || tile < TM * TM) {
          const int i0 = (tile / TM) * 4, j0 = (tile % TM) * 4;
#pragma unroll 4
          for (int b = 0; b < Dc; ++b) {
            R xv[4], yv[4];
            if constexpr (DD % 4 == 0) {
              load4(Xs + b * DD + i0, xv);
              load4(Ys + b * DD + j0, yv);
            } else {
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                xv[q] = (DD % 4 == 0 || i0 + q < DD) ? Xs[b * DD + i0 + q] : R(0);
                yv[q] = (DD % 4 == 0 || j0 + q < DD) ? Ys[b * DD + j0 + q] : R(0);
              }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
              for (int j = 0; j < 4; ++j) acc[t][i][j] = fma(xv[i], yv[j], acc[t][i][j]);
          }
        }
      }
    }
    __syncthreads();
  }
  // stage [l][r][u][d] in shared memory, then write coalesced
  R* Bs = sm;
#pragma unroll
  for (int t = 0; t < S::TPT; ++t) {
    const int tile = t * kThreads + tid;
    if ((TM * TM) % kThreads == 0 || tile < TM * TM) {
      const int i0 = (tile / TM) * 4, j0 = (tile % TM) * 4;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int lu = i0 + i, dr = j0 + j;
          if ((DD % 4 == 0 || (lu < DD && dr < DD))) {
            const int l = lu / D, u = lu % D, d = dr / D, r = dr % D;
            Bs[l * D3 + r * DD + u * D + d] = acc[t][i][j] * scale;
          }
        }
    }
  }
  __syncthreads();
  for (int e = tid; e < S::D4; e += kThreads) Bout[e] = Bs[e];
  __syncthreads();
}

}  // namespace peps
