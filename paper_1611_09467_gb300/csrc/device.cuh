// Device building blocks: CTA-wide strided GEMM, reductions, contraction
// programs, and the truncation of the boundary MPS (dominant left singular
// subspace of a small dense matrix).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "contract.cuh"

// Phase markers inside the truncation.  Empty in the library; the
// diagnostic build (-DPEPS_PHASE_TIMING, phase_timing.py) makes thread 0 of
// each CTA add the clock64 cycles since the previous marker to counter k
// (k = 0: the cycles since the last truncation ended, to counter 7).  Each
// marker is a barrier there, so that build is only for the breakdown.
#ifdef PEPS_PHASE_TIMING
static __device__ unsigned long long peps_phase_cyc[16];
__device__ __forceinline__ void peps_phase_mark(int k) {
  __shared__ long long peps_phase_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    const long long t = clock64();
    const long long d = t - peps_phase_last;
    if (d > 0 && d < (1ll << 34)) atomicAdd(&peps_phase_cyc[k == 0 ? 7 : k], (unsigned long long)d);
    peps_phase_last = t;
  }
  __syncthreads();
}
#define PEPS_PHASE(k) peps_phase_mark(k)
#else
#define PEPS_PHASE(k)
#endif

namespace peps {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

template <typename R> struct Eps;
template <> struct Eps<double> {
  static constexpr double eps = 2.220446049250313e-16;
  static constexpr double tiny = 2.2250738585072014e-308;
  static constexpr int bits = 53;
};
template <> struct Eps<float> {
  static constexpr float eps = 1.1920929e-07f;
  static constexpr float tiny = 1.17549435e-38f;
  static constexpr int bits = 24;
};

__device__ __forceinline__ double dsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float dsqrt(float x) { return sqrtf(x); }

// One step of a compensated dot product in FP32 (Ogita, Rump and Oishi,
// "Accurate sum and dot product", SIAM J. Sci. Comput. 26 (2005), Dot2):
// the product's rounding error comes exactly from an FMA (TwoProduct), the
// sum's from Knuth's TwoSum, and both go into c.  s + c then carries the dot
// product as if accumulated in twice the working precision.  The explicit
// _rn intrinsics keep the compiler from contracting or reassociating them.
__device__ __forceinline__ void dot2_step(float a, float b, float& s, float& c) {
  const float p = __fmul_rn(a, b);
  const float pe = __fmaf_rn(a, b, -p);
  const float t = __fadd_rn(s, p);
  const float z = __fsub_rn(t, s);
  const float se = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
  s = t;
  c = __fadd_rn(c, __fadd_rn(pe, se));
}

template <typename R>
__device__ __forceinline__ R warp_sum(R v, int width = 32) {
  for (int o = width / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, width);
  return v;
}
template <typename R>
__device__ __forceinline__ R warp_max(R v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum; `red` is shared scratch of >= kWarps elements.  All threads
// get the result.  Contains two barriers.
template <typename R>
__device__ R block_sum(R v, R* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  R s = 0;
  for (int i = 0; i < kWarps; ++i) s += red[i];
  __syncthreads();
  return s;
}

// Block-wide maximum; same contract as block_sum.
template <typename R>
__device__ R block_max(R v, R* red) {
  v = warp_max(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  R s = red[0];
  for (int i = 1; i < kWarps; ++i) s = fmax(s, red[i]);
  __syncthreads();
  return s;
}

// Power-of-two renormalisation of the transfer vectors of the sandwiches.
// A sandwich value between unit-norm environments can fall far below the
// FP32 range (it is psi divided by the norms of all other rows), so every
// stored transfer is scaled by an exact power of two and its exponent is
// carried beside it; ratios and Delta add the exponents back in FP64.
// pow2_exponent(m) = floor(log2 m) read from the bits of m, clamped so that
// 2^-e is a normal number; 0 for m = 0 or m not finite.
__device__ __forceinline__ int pow2_exponent(float m) {
  const int ef = (int)((__float_as_uint(m) >> 23) & 0xffu);
  if (!(m > 0.f) || ef == 0xff) return 0;
  const int e = ef - 127;
  return e < -126 ? -126 : (e > 126 ? 126 : e);
}
__device__ __forceinline__ int pow2_exponent(double m) {
  const int ef = (int)((__double_as_longlong(m) >> 52) & 0x7ffll);
  if (!(m > 0.0) || ef == 0x7ff) return 0;
  const int e = ef - 1023;
  return e < -1022 ? -1022 : (e > 1022 ? 1022 : e);
}
// 2^e for e in the clamped range of pow2_exponent
template <typename R>
__device__ __forceinline__ R pow2(int e);
template <>
__device__ __forceinline__ float pow2<float>(int e) { return __uint_as_float((unsigned)(e + 127) << 23); }
template <>
__device__ __forceinline__ double pow2<double>(int e) {
  return __longlong_as_double((long long)(e + 1023) << 52);
}

// Scales x[0..n) in place by 2^-e, e = pow2_exponent(max |x|), and returns e.
// x must be complete (written before a barrier); ends with a barrier.
template <typename R>
__device__ int normalize_pow2(R* x, int n, R* red) {
  R m = R(0);
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(x[i]));
  m = block_max(m, red);
  const int e = pow2_exponent(m);
  if (e != 0) {
    const R sc = pow2<R>(-e);
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] *= sc;
  }
  __syncthreads();
  return e;
}

// ------------------------------------------------------------- CTA GEMM
// Shared-memory tiled GEMM over the index maps of a descriptor (see
// contract.cuh).  Per output tile (TM x TN) the K range is walked in chunks
// of 16: the A and B chunks are gathered from global memory through the
// offset tables into shared memory, then every thread accumulates an
// MT x NT micro-tile in registers.  The CTA tile shape follows N (the
// contraction steps have N in {16, 32, 64, 128, 256+}).  Shared memory:
// kGemmSmemReals reals + kGemmSmemInts ints supplied by the caller.
// A and B are often written earlier by the same kernel (carries, blocks,
// singular vectors), so they are not declared __restrict__: that would let
// the compiler read them through the non-coherent read-only path, which is
// only valid for data that no thread writes while the kernel runs.  The same
// holds for the transfer inputs of the fused steps.
constexpr int kGemmTK = 16;
constexpr int kMaxK = 1024;
constexpr int kGemmSmemReals = kGemmTK * (512 + 16);
constexpr int kGemmSmemInts = 2 * kMaxK + 2 * 512 + 2 * 256;

template <typename R, int TM, int TN, int MT, int NT>
__device__ __noinline__ void gemm_tiles(const GemmDesc& g, const R* A, const R* B,
                                        R* __restrict__ C, bool accumulate, R* sm, int* ism) {
  constexpr int TK = kGemmTK;
  constexpr int GX = TN / NT, GY = TM / MT;
  static_assert(GX * GY == kThreads, "thread grid must cover the CTA");
  R* As = sm;                  // [TK][TM]
  R* Bs = sm + TK * TM;        // [TK][TN]
  int* ktA = ism;              // [K]
  int* ktB = ism + kMaxK;      // [K]
  int* rA = ism + 2 * kMaxK;   // [TM]
  int* rC = rA + TM;           // [TM]
  int* cB = rC + TM;           // [TN]
  int* cC = cB + TN;           // [TN]
  const int tid = threadIdx.x;
  const int tx = tid % GX, ty = tid / GX;
  __syncthreads();
  for (int k = tid; k < g.K; k += blockDim.x) {
    const int k1 = k / g.ak.n2, k2 = k - k1 * g.ak.n2;
    ktA[k] = k1 * g.ak.s1 + k2 * g.ak.s2;
    ktB[k] = k1 * g.bk.s1 + k2 * g.bk.s2;
  }
  const int tiles_m = (g.M + TM - 1) / TM, tiles_n = (g.N + TN - 1) / TN;
  for (int bt = 0; bt < g.nb; ++bt) {
    const R* Ab = A + (size_t)bt * g.sa;
    const R* Bb = B + (size_t)bt * g.sb;
    R* Cb = C + (size_t)bt * g.sc;
    for (int tmi = 0; tmi < tiles_m; ++tmi)
      for (int tni = 0; tni < tiles_n; ++tni) {
        const int i0 = tmi * TM, j0 = tni * TN;
        __syncthreads();
        for (int e = tid; e < TM; e += blockDim.x) {
          const int i = min(i0 + e, g.M - 1);
          rA[e] = ixoff(g.am, i);
          rC[e] = ixoff(g.cm, i);
        }
        for (int e = tid; e < TN; e += blockDim.x) {
          const int j = min(j0 + e, g.N - 1);
          cB[e] = ixoff(g.bn, j);
          cC[e] = ixoff(g.cn, j);
        }
        R acc[MT][NT];
#pragma unroll
        for (int m = 0; m < MT; ++m)
#pragma unroll
          for (int n = 0; n < NT; ++n) acc[m][n] = R(0);
        for (int k0 = 0; k0 < g.K; k0 += TK) {
          __syncthreads();
          for (int e = tid; e < TM * TK; e += kThreads) {
            const int i = e % TM, kk = e / TM, k = k0 + kk;
            As[kk * TM + i] = k < g.K ? Ab[rA[i] + ktA[k]] : R(0);
          }
          for (int e = tid; e < TN * TK; e += kThreads) {
            const int j = e % TN, kk = e / TN, k = k0 + kk;
            Bs[kk * TN + j] = k < g.K ? Bb[ktB[k] + cB[j]] : R(0);
          }
          __syncthreads();
#pragma unroll
          for (int kk = 0; kk < TK; ++kk) {
            R a[MT], b[NT];
#pragma unroll
            for (int m = 0; m < MT; ++m) a[m] = As[kk * TM + ty * MT + m];
#pragma unroll
            for (int n = 0; n < NT; ++n) b[n] = Bs[kk * TN + tx * NT + n];
#pragma unroll
            for (int m = 0; m < MT; ++m)
#pragma unroll
              for (int n = 0; n < NT; ++n) acc[m][n] = fma(a[m], b[n], acc[m][n]);
          }
        }
#pragma unroll
        for (int m = 0; m < MT; ++m) {
          const int i = ty * MT + m;
          if (i0 + i >= g.M) break;
#pragma unroll
          for (int n = 0; n < NT; ++n) {
            const int j = tx * NT + n;
            if (j0 + j >= g.N) break;
            R* p = Cb + rC[i] + cC[j];
            *p = accumulate ? *p + acc[m][n] : acc[m][n];
          }
        }
      }
  }
  __syncthreads();
}

// C (+)= A B for a descriptor; the whole CTA takes part and the call ends
// with a barrier.  `sm`/`ism` point to the GEMM's shared-memory scratch.
template <typename R>
__device__ void cta_gemm(const GemmDesc& g, const R* A, const R* B, R* __restrict__ C,
                         bool accumulate, R* sm, int* ism) {
  if (g.N >= 256 && g.M <= 32) gemm_tiles<R, 16, 256, 4, 4>(g, A, B, C, accumulate, sm, ism);
  else if (g.N >= 128) gemm_tiles<R, 64, 128, 4, 8>(g, A, B, C, accumulate, sm, ism);
  else if (g.N >= 64 && g.M >= 128) gemm_tiles<R, 128, 64, 8, 4>(g, A, B, C, accumulate, sm, ism);
  else if (g.N >= 48) gemm_tiles<R, 64, 64, 4, 4>(g, A, B, C, accumulate, sm, ism);
  else if (g.N >= 24) gemm_tiles<R, 256, 32, 8, 4>(g, A, B, C, accumulate, sm, ism);
  else gemm_tiles<R, 512, 16, 8, 4>(g, A, B, C, accumulate, sm, ism);
}

// C = A B for a descriptor with K <= KM, the whole reduction staged at once:
// per tile of TM rows every load is issued before the first store to shared
// memory, so one load latency is exposed per tile rather than one per 16-wide
// K chunk, and a tile costs two barriers.  FP32 tiles are multiplied with
// packed FP32x2 multiply-adds.  Each output is the same left-to-right chain
// of fused multiply-adds over k as in gemm_tiles, so the results are
// identical.  `sm` holds K * (TM + TN) reals; `ism` the offset tables.
template <typename R, int TM, int TN, int MT, int NT, int KM>
__device__ __noinline__ void gemm_wk(const GemmDesc& g, const R* A, const R* B, R* __restrict__ C, R* sm,
                                     int* ism) {
  constexpr int GX = TN / NT, GY = TM / MT;
  static_assert(GX * GY == kThreads, "thread grid must cover the CTA");
  static_assert(MT % 4 == 0 && NT % 4 == 0, "tiles are read as 16-byte groups");
  constexpr int LA = TM * KM / kThreads, LB = TN * KM / kThreads;
  const int K = g.K;
  R* As = sm;            // [K][TM]
  R* Bs = sm + K * TM;   // [K][TN]
  int* ktA = ism;
  int* ktB = ism + KM;
  int* rA = ism + 2 * KM;
  int* rC = rA + TM;
  int* cB = rC + TM;
  int* cC = cB + TN;
  const int tid = threadIdx.x;
  const int tx = tid % GX, ty = tid / GX;
  __syncthreads();
  for (int k = tid; k < K; k += kThreads) {
    const int k1 = k / g.ak.n2, k2 = k - k1 * g.ak.n2;
    ktA[k] = k1 * g.ak.s1 + k2 * g.ak.s2;
    ktB[k] = k1 * g.bk.s1 + k2 * g.bk.s2;
  }
  const int tiles_m = (g.M + TM - 1) / TM, tiles_n = (g.N + TN - 1) / TN;
  for (int bt = 0; bt < g.nb; ++bt) {
    const R* Ab = A + (size_t)bt * g.sa;
    const R* Bb = B + (size_t)bt * g.sb;
    R* Cb = C + (size_t)bt * g.sc;
    for (int tni = 0; tni < tiles_n; ++tni)
      for (int tmi = 0; tmi < tiles_m; ++tmi) {
        const int i0 = tmi * TM, j0 = tni * TN;
        __syncthreads();
        for (int e = tid; e < TM; e += kThreads) {
          const int i = min(i0 + e, g.M - 1);
          rA[e] = ixoff(g.am, i);
          rC[e] = ixoff(g.cm, i);
        }
        for (int e = tid; e < TN; e += kThreads) {
          const int j = min(j0 + e, g.N - 1);
          cB[e] = ixoff(g.bn, j);
          cC[e] = ixoff(g.cn, j);
        }
        __syncthreads();
        R va[LA], vb[LB];
#pragma unroll
        for (int q = 0; q < LA; ++q) {
          const int e = tid + q * kThreads, kk = e / TM, i = e % TM;
          va[q] = kk < K ? Ab[rA[i] + ktA[kk]] : R(0);
        }
#pragma unroll
        for (int q = 0; q < LB; ++q) {
          const int e = tid + q * kThreads, kk = e / TN, j = e % TN;
          vb[q] = kk < K ? Bb[ktB[kk] + cB[j]] : R(0);
        }
#pragma unroll
        for (int q = 0; q < LA; ++q) {
          const int e = tid + q * kThreads;
          if (e / TM < K) As[e] = va[q];
        }
#pragma unroll
        for (int q = 0; q < LB; ++q) {
          const int e = tid + q * kThreads;
          if (e / TN < K) Bs[e] = vb[q];
        }
        __syncthreads();
        R acc[MT][NT];
        if constexpr (sizeof(R) == 4) {
          float2 acc2[MT][NT / 2];
#pragma unroll
          for (int m = 0; m < MT; ++m)
#pragma unroll
            for (int n = 0; n < NT / 2; ++n) acc2[m][n] = make_float2(0.f, 0.f);
#pragma unroll 4
          for (int kk = 0; kk < K; ++kk) {
            float a[MT], b[NT];
#pragma unroll
            for (int m = 0; m < MT; m += 4) {
              const float4 t = *reinterpret_cast<const float4*>(As + kk * TM + ty * MT + m);
              a[m] = t.x; a[m + 1] = t.y; a[m + 2] = t.z; a[m + 3] = t.w;
            }
#pragma unroll
            for (int n = 0; n < NT; n += 4) {
              const float4 t = *reinterpret_cast<const float4*>(Bs + kk * TN + tx * NT + n);
              b[n] = t.x; b[n + 1] = t.y; b[n + 2] = t.z; b[n + 3] = t.w;
            }
#pragma unroll
            for (int m = 0; m < MT; ++m)
#pragma unroll
              for (int n = 0; n < NT / 2; ++n)
                acc2[m][n] = __ffma2_rn(make_float2(a[m], a[m]), make_float2(b[2 * n], b[2 * n + 1]), acc2[m][n]);
          }
#pragma unroll
          for (int m = 0; m < MT; ++m)
#pragma unroll
            for (int n = 0; n < NT / 2; ++n) {
              acc[m][2 * n] = acc2[m][n].x;
              acc[m][2 * n + 1] = acc2[m][n].y;
            }
        } else {
#pragma unroll
          for (int m = 0; m < MT; ++m)
#pragma unroll
            for (int n = 0; n < NT; ++n) acc[m][n] = R(0);
          for (int kk = 0; kk < K; ++kk) {
            R a[MT], b[NT];
#pragma unroll
            for (int m = 0; m < MT; ++m) a[m] = As[kk * TM + ty * MT + m];
#pragma unroll
            for (int n = 0; n < NT; ++n) b[n] = Bs[kk * TN + tx * NT + n];
#pragma unroll
            for (int m = 0; m < MT; ++m)
#pragma unroll
              for (int n = 0; n < NT; ++n) acc[m][n] = fma(a[m], b[n], acc[m][n]);
          }
        }
        int cc[NT];
#pragma unroll
        for (int n = 0; n < NT; ++n) cc[n] = cC[tx * NT + n];
#pragma unroll
        for (int m = 0; m < MT; ++m) {
          const int i = ty * MT + m;
          if (i0 + i >= g.M) break;
          const int rc = rC[i];
#pragma unroll
          for (int n = 0; n < NT; ++n) {
            if (j0 + tx * NT + n >= g.N) break;
            Cb[rc + cc[n]] = acc[m][n];
          }
        }
      }
  }
  __syncthreads();
}

// Reals of shared scratch gemm_wk needs for a descriptor, or 0 when the
// descriptor is outside its shapes (cta_gemm takes those).
PEPS_HD int zip_gemm_reals(const GemmDesc& g) {
  if (g.N > 64 && g.N <= 128 && g.K <= 16) return g.K * (64 + 128);
  if (g.N <= 64 && g.K <= 64) return g.K * (128 + 64);
  return 0;
}

// C = A B for the zip-up contractions: gemm_wk when the descriptor fits it
// and `sm_reals` reals of shared scratch, else cta_gemm.  Same results either
// way.
template <typename R>
__device__ __noinline__ void zip_gemm(const GemmDesc& g, const R* A, const R* B, R* __restrict__ C, R* sm, int* ism,
                         int sm_reals) {
  const int need = zip_gemm_reals(g);
  if (need > 0 && need <= sm_reals) {
    if (g.N > 64) gemm_wk<R, 64, 128, 4, 8, 16>(g, A, B, C, sm, ism);
    else gemm_wk<R, 128, 64, 8, 4, 64>(g, A, B, C, sm, ism);
  } else {
    cta_gemm<R>(g, A, B, C, false, sm, ism);
  }
}

// ------------------------------------------------- contraction programs
enum OpId { OP_COL1_LEFT = 0, OP_COL1_RIGHT = 1, OP_SITE_ENV = 2, OP_COL2_LEFT = 3, OP_COL2_RIGHT = 4, OP_FIT_SITE = 5 };
enum BufId { IN0 = 0, IN1, IN2, IN3, IN4, TMP0, TMP1, OUT };
struct Step {
  int s, a, b, c;
};

PEPS_HD int op_nsteps(int op) { return (op == OP_COL2_LEFT || op == OP_COL2_RIGHT) ? 4 : 3; }

// Which buffers each step reads and writes.  Inputs per op:
//   COL1_LEFT : IN0 = F_{c-1}, IN1 = Mu, IN2 = T, IN3 = Md        -> F_c
//   COL1_RIGHT: IN0 = G_{c+1}, IN1 = Mu, IN2 = T, IN3 = Md        -> G_c
//   SITE_ENV  : IN0 = F_{c-1}, IN1 = Mu, IN2 = Md, IN3 = G_{c+1}  -> B_c
//   COL2_LEFT : IN0 = E_{c-1}, IN1 = Mu, IN2 = T1, IN3 = T2, IN4 = Md -> E_c
//   COL2_RIGHT: IN0 = H_{c+1}, IN1 = Mu, IN2 = T1, IN3 = T2, IN4 = Md -> H_c
//   FIT_SITE  : IN0 = F_{c-1}, IN1 = Mu, IN2 = T, IN3 = G_{c+1}   -> P_c
PEPS_HD Step op_step_bufs(int op, int s) {
  switch (op) {
    case OP_FIT_SITE:
    case OP_COL1_LEFT:
      return s == 0 ? Step{0, IN0, IN1, TMP0} : s == 1 ? Step{1, TMP0, IN2, TMP1} : Step{2, TMP1, IN3, OUT};
    case OP_COL1_RIGHT:
      return s == 0 ? Step{0, IN1, IN0, TMP0} : s == 1 ? Step{1, TMP0, IN2, TMP1} : Step{2, TMP1, IN3, OUT};
    case OP_SITE_ENV:
      return s == 0 ? Step{0, IN2, IN3, TMP0} : s == 1 ? Step{1, IN1, TMP0, TMP1} : Step{2, IN0, TMP1, OUT};
    case OP_COL2_LEFT:
      return s == 0 ? Step{0, IN0, IN1, TMP0}
           : s == 1 ? Step{1, TMP0, IN2, TMP1}
           : s == 2 ? Step{2, TMP1, IN3, TMP0}
                    : Step{3, TMP0, IN4, OUT};
    default:
      return s == 0 ? Step{0, IN1, IN0, TMP0}
           : s == 1 ? Step{1, TMP0, IN2, TMP1}
           : s == 2 ? Step{2, TMP1, IN3, TMP0}
                    : Step{3, TMP0, IN4, OUT};
  }
}

PEPS_HD GemmDesc op_desc(int op, int s, int D, int Dc) {
  switch (op) {
    case OP_COL1_LEFT: return col1_left_step(s, D, Dc);
    case OP_COL1_RIGHT: return col1_right_step(s, D, Dc);
    case OP_SITE_ENV: return site_env_step(s, D, Dc);
    case OP_FIT_SITE: return fit_site_step(s, D, Dc);
    case OP_COL2_LEFT: return col2_left_step(s, D, Dc);
    default: return col2_right_step(s, D, Dc);
  }
}

// Runs one contraction program with the whole CTA; ends with a barrier.
template <typename R>
__device__ void run_op(int op, int D, int Dc, const R* in0, const R* in1, const R* in2, const R* in3,
                       const R* in4, R* out, R* t0, R* t1, R* sm, int* ism) {
  const int ns = op_nsteps(op);
  for (int s = 0; s < ns; ++s) {
    const Step st = op_step_bufs(op, s);
    const GemmDesc g = op_desc(op, st.s, D, Dc);
    const R* bufs[8] = {in0, in1, in2, in3, in4, t0, t1, out};
    cta_gemm<R>(g, bufs[st.a], bufs[st.b], const_cast<R*>(bufs[st.c]), false, sm, ism);
  }
}

// ------------------------------------------------------------ truncation
// Dominant-K left singular subspace of a dense m x n matrix X (row-major),
// used for the boundary-MPS cut-off (Fig. 1d, Dc).  Route: Householder
// bidiagonalisation (Golub & Kahan 1965), the K largest singular values by
// Sturm-count bisection on the Golub-Kahan tridiagonal form
// [[0, B], [B^T, 0]] (perfect-shuffle ordering), singular vectors by inverse
// iteration on that form, classical Gram-Schmidt with re-orthogonalisation,
// and back-transformation by the stored reflectors.  Only the subspace
// matters downstream (the kept projector is unique when sigma_K > sigma_K+1),
// so any orthonormal basis of it is a valid result.
template <typename R>
struct TruncWork {
  R* Wm;      // P x ldw
  int ldw;
  R* Wg;      // P x ldw in global memory: the reflectors of the register-tiled path
  R* tau;     // 4 * Qmax: tau left, tau right, scale left, scale right
  R* t;       // 2 * Qmax off-diagonal of the Golub-Kahan form
  R* t2;      // squares of t
  R* lam;     // Kmax
  R* Z;       // Kmax x 2Qmax
  R* lu;      // Kmax x 6 x 2Qmax: inverse-iteration workspace when it is not in shared memory
  R* Ub;      // Qmax x Kmax (unused when Ubs is set)
  R* Uk;      // Pmax x Kmax compact copy of the result in global memory
  R* Ubs;     // Qmax x Kmax in shared memory (after the truncation matrix)
  R* Uks;     // Pmax x Kmax in shared memory
  R* red;     // >= 64 (shared)
  R* wv;      // >= 256 (shared): reflector products
  R* gsm;     // GEMM shared scratch (may alias Wm: used only after the reflectors are dead)
  int* gism;
  int Qmax;
  int wm_shared;   // Wm is in shared memory
};

// Element counts of the truncation workspace for P, Q <= pq and K <= kmax.
PEPS_HD size_t trunc_ws_elems(int pq, int kmax, bool with_wm) {
  size_t e = 0;
  if (with_wm) e += (size_t)pq * (pq + 1);
  e += (size_t)pq * (pq + 1);             // Wg
  e += 4 * (size_t)pq + 2 * (size_t)pq * 2;   // tau + scale factors (4 pq), t, t2
  e += kmax;                              // lam
  e += (size_t)kmax * 2 * pq;             // Z
  e += (size_t)kmax * 6 * 2 * pq;         // lu
  e += (size_t)pq * kmax * 2;             // Ub, Uk
  return e + 64;
}

// Householder vector for x = (alpha, rest): returns tau, scale for rest, beta.
template <typename R>
__device__ __forceinline__ void householder(R alpha, R ss, R& tau, R& scale, R& beta) {
  if (ss <= R(0)) {
    tau = R(0);
    scale = R(0);
    beta = alpha;
  } else {
    const R nrm = dsqrt(alpha * alpha + ss);
    beta = alpha >= R(0) ? -nrm : nrm;
    tau = (beta - alpha) / beta;
    scale = R(1) / (alpha - beta);
  }
}

// The same for FP32 with the hardware-approximate division (2 ulp): the
// register-tiled bidiagonalisation forms these scalars on its critical path.
__device__ __forceinline__ void householder_fast(float alpha, float ss, float& tau, float& scale, float& beta) {
  if (ss <= 0.f) {
    tau = 0.f;
    scale = 0.f;
    beta = alpha;
  } else {
    const float nrm = sqrtf(alpha * alpha + ss);
    beta = alpha >= 0.f ? -nrm : nrm;
    tau = __fdividef(beta - alpha, beta);
    scale = __fdividef(1.f, alpha - beta);
  }
}

// Division inside the Sturm counts and the inverse-iteration factorisation:
// IEEE in FP64, the hardware approximation (2 ulp) in FP32, where it sits on
// a long dependent chain.
__device__ __forceinline__ double sturm_div(double a, double b) { return a / b; }
__device__ __forceinline__ float sturm_div(float a, float b) { return __fdividef(a, b); }

// Number of eigenvalues below x of the zero-diagonal symmetric tridiagonal
// with squared off-diagonals t2 (pivots of the LDL^T factorisation of T - x).
template <typename R>
__device__ int sturm_count(const R* t2, int n2, R x, R pivmin) {
  int cnt = 0;
  R q = -x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < R(0)) ++cnt;
  for (int i = 1; i < n2; ++i) {
    q = -x - sturm_div(t2[i - 1], q);
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < R(0)) ++cnt;
  }
  return cnt;
}

// Inverse iteration for one eigenvalue of the n2 x n2 zero-diagonal
// symmetric tridiagonal with off-diagonal t: Gaussian elimination with
// partial pivoting on (T - lam I), two solves from a fixed pseudo-random
// start vector.  Sequential, one thread per eigenvalue.  Five passes over
// the vector: factorisation fused with the first forward elimination, back
// substitution, the second forward elimination (which also applies the
// scaling of the first iterate), back substitution, and the output pass.
// Each iterate is scaled only by its largest entry (the solve can amplify by
// 1/pivtiny); the caller normalises the vectors.  The recurrences carry their
// running values in registers; memory only receives the factors and reads
// back values that do not depend on the running recurrence, so loads can be
// issued ahead.  Workspace: four real arrays (reciprocal pivots, first
// super-diagonal of U, multipliers of L, right-hand side) and one byte per
// row for the interchanges, each interleaved across the K threads (element i
// of thread k at i * K + k) so lock-step accesses of a warp are contiguous.
// The second super-diagonal of U is t[i+1] where rows i, i+1 were
// interchanged and zero otherwise, so it is not stored.
template <typename R>
__device__ void inverse_iteration(const R* t, int n2, R lam, R pivtiny, R* wsR, unsigned char* wsP, int K, int k,
                                  R* z, int zs, unsigned seed) {
  const size_t st = (size_t)n2 * K;
  R* rdd = wsR + k;      // reciprocal pivots of U
  R* du = rdd + st;      // first super-diagonal of U
  R* mult = du + st;     // multipliers of L
  R* b = mult + st;      // right-hand side / solution
  unsigned char* piv = wsP + k;   // 1 where rows i, i+1 were interchanged
#define IX(i) ((size_t)(i) * K)
  unsigned h = seed * 2654435761u + 12345u;
  auto start = [&]() {
    h ^= h << 13; h ^= h >> 17; h ^= h << 5;
    return R((int)(h & 0xffffu) - 32768) / R(32768) + R(0.001);
  };
  // ---- factorisation, carrying dd[i], du[i] (current row) and dd[i+1],
  // du[i+1], with the forward elimination of the start vector (carrying b[i])
  R cur_d = -lam, cur_u = n2 > 1 ? t[0] : R(0);
  R bi = start();
  for (int i = 0; i < n2 - 1; ++i) {
    const R sub = t[i];
    R next_d = -lam;
    R next_u = i + 1 < n2 - 1 ? t[i + 1] : R(0);
    const R bn = start();
    R d_i, u_i, l;
    if (fabs(cur_d) >= fabs(sub)) {
      d_i = cur_d == R(0) ? pivtiny : cur_d;
      l = sturm_div(sub, d_i);
      u_i = cur_u;
      next_d -= l * cur_u;
      piv[IX(i)] = 0;
      b[IX(i)] = bi;
      bi = bn - l * bi;
    } else {
      l = sturm_div(cur_d, sub);
      d_i = sub;
      u_i = next_d;
      next_d = cur_u - l * next_d;
      next_u = -l * next_u;
      piv[IX(i)] = 1;
      b[IX(i)] = bn;
      bi = bi - l * bn;
    }
    if (fabs(d_i) < pivtiny) d_i = d_i < R(0) ? -pivtiny : pivtiny;
    rdd[IX(i)] = sturm_div(R(1), d_i);
    du[IX(i)] = u_i;
    mult[IX(i)] = l;
    cur_d = next_d;
    cur_u = next_u;
  }
  if (fabs(cur_d) < pivtiny) cur_d = cur_d < R(0) ? -pivtiny : pivtiny;
  rdd[IX(n2 - 1)] = sturm_div(R(1), cur_d);
  du[IX(n2 - 1)] = R(0);
  piv[IX(n2 - 1)] = 0;
  b[IX(n2 - 1)] = bi;
  R sc = R(1);   // scale of the current iterate still to be applied
  for (int it = 0; it < 2; ++it) {
    if (it == 1) {
      // ---- forward: row interchanges and L^-1 on the scaled iterate
      R bf = b[IX(0)] * sc;
#pragma unroll 4
      for (int i = 0; i < n2 - 1; ++i) {
        const R bn = b[IX(i + 1)] * sc;
        const R l = mult[IX(i)];
        if (piv[IX(i)] == 0) {
          b[IX(i)] = bf;
          bf = bn - l * bf;
        } else {
          b[IX(i)] = bn;
          bf = bf - l * bn;
        }
      }
      b[IX(n2 - 1)] = bf;
    }
    // ---- backward: U^-1, carrying y[i+1], y[i+2]; track max |y|
    R y1 = R(0), y2 = R(0), mx = R(0);
#pragma unroll 4
    for (int i = n2 - 1; i >= 0; --i) {
      const R du2 = (piv[IX(i)] != 0 && i + 1 < n2 - 1) ? t[i + 1] : R(0);
      const R y = (b[IX(i)] - du[IX(i)] * y1 - du2 * y2) * rdd[IX(i)];
      b[IX(i)] = y;
      mx = fmax(mx, fabs(y));
      y2 = y1;
      y1 = y;
    }
    sc = mx > R(0) ? R(1) / mx : R(1);
  }
  for (int i = 0; i < n2; ++i) z[(size_t)i * zs] = b[IX(i)] * sc;
#undef IX
}

// v[k] for a run-time k
__device__ __forceinline__ float sel8(const float (&v)[8], int k) {
  float x = v[0];
#pragma unroll
  for (int q = 1; q < 8; ++q) x = k == q ? v[q] : x;
  return x;
}
// Column c of a pair-packed 8 x 8 tile.  c is uniform across the CTA, so a
// branch on it costs no divergence and each case is eight register moves
// (selecting by comparisons would cost about seven instructions per entry).
__device__ __forceinline__ void col_of(const float2 (&a)[8][4], int c, float (&out)[8]) {
#define PEPS_COL_CASE(C)                                                      \
  case C:                                                                     \
    _Pragma("unroll") for (int r = 0; r < 8; ++r) out[r] = ((C) & 1) ? a[r][(C) >> 1].y : a[r][(C) >> 1].x; \
    break;
  switch (c) {
    PEPS_COL_CASE(0) PEPS_COL_CASE(1) PEPS_COL_CASE(2) PEPS_COL_CASE(3)
    PEPS_COL_CASE(4) PEPS_COL_CASE(5) PEPS_COL_CASE(6) default: PEPS_COL_CASE(7)
  }
#undef PEPS_COL_CASE
}
// Row r of a pair-packed 8 x 8 tile; r is uniform across the CTA.
__device__ __forceinline__ void row_of(const float2 (&a)[8][4], int r, float (&out)[8]) {
#define PEPS_ROW_CASE(R)                                                      \
  case R:                                                                     \
    _Pragma("unroll") for (int k = 0; k < 4; ++k) {                           \
      out[2 * k] = a[R][k].x;                                                 \
      out[2 * k + 1] = a[R][k].y;                                             \
    }                                                                         \
    break;
  switch (r) {
    PEPS_ROW_CASE(0) PEPS_ROW_CASE(1) PEPS_ROW_CASE(2) PEPS_ROW_CASE(3)
    PEPS_ROW_CASE(4) PEPS_ROW_CASE(5) PEPS_ROW_CASE(6) default: PEPS_ROW_CASE(7)
  }
#undef PEPS_ROW_CASE
}
// Householder bidiagonalisation of an FP32 matrix of at most 128 x 128 held
// in registers: thread (ti, tj) owns the 8 x 8 tile of rows 8 ti.., columns
// 8 tj.., with ti = lane % 16 and tj = 2 warp + lane / 16, so the 16 tiles of a
// tile column sit in one half-warp (column sums are shuffle reductions) and
// the tiles of a tile row in one lane position of every half-warp.  A tile is
// kept as column pairs and updated with packed FP32x2 multiply-adds; the
// active row and column are picked out of the tile by selects (a register
// array cannot be indexed at run time).  Not inlined: its own register
// allocation holds the 64-element tile without spilling.  The
// arithmetic is that of the shared-memory version below (same reflectors,
// same stored factors); only the order of the partial sums differs.  One
// column costs four barriers: broadcast of the left reflector, the row norm
// of the right reflector, and two for the cross-warp sums of W u (per-warp
// shares, then row totals).  Column sums within a half-warp are a
// reduce-scatter followed by an all-gather, the same additions as a
// butterfly in fewer shuffles.  Warps whose two tile columns lie left of the
// active column skip the products.  On return W
// (P x Q, leading dimension ld) holds the unscaled reflectors; t and tau4
// (tau left, tau right, scale left, scale right, qm apart) are set as by the
// shared-memory version.
static __device__ __noinline__ void bidiag_tiles_f32(const float* X, int n, bool tall, int P, int Q, float* W, int ld,
                                                 float* t, float* tau4, int qm) {
  __shared__ __align__(16) float zp[kWarps * 128];   // per-warp partial sums of W u
  __shared__ __align__(16) float vL[128];            // left reflector, by row
  __shared__ __align__(16) float zt[128];            // row totals of W u
  __shared__ float sc[2];                            // tau_left, alpha_right
  __shared__ __align__(16) float rnp[16];            // row-norm partials, by tile column
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, ti = lane & 15;
  const int tj = warp * 2 + (lane >> 4);
  const int r0 = ti * 8, c0 = tj * 8;
  const unsigned hmask = (lane & 16) ? 0xffff0000u : 0x0000ffffu;
  float2 a[8][4];   // a[r][q] = columns (2q, 2q+1) of row r of the tile
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = r0 + r, c = c0 + 2 * q;
      float x0 = 0.f, x1 = 0.f;
      if (i < P) {
        if (c < Q) x0 = tall ? X[i * n + c] : X[c * n + i];
        if (c + 1 < Q) x1 = tall ? X[i * n + c + 1] : X[(c + 1) * n + i];
      }
      a[r][q] = make_float2(x0, x1);
    }
  for (int jb = 0; jb < Q; jb += 8) {
    const int tb = jb >> 3;   // tile row / column of j
#pragma unroll 1
    for (int jj = 0; jj < 8; ++jj) {
      const int j = jb + jj;
      if (j < Q) {
        // ---- left reflector on column j (rows j..P-1), formed by the owning half-warp
        if (tj == tb) {
          float col[8];
          col_of(a, jj, col);
          float ss = 0.f;
#pragma unroll
          for (int r = 0; r < 8; ++r)
            if (r0 + r > j) ss = fmaf(col[r], col[r], ss);
#pragma unroll
          for (int o = 8; o >= 1; o >>= 1) ss += __shfl_xor_sync(hmask, ss, o);
          const float alpha = __shfl_sync(hmask, sel8(col, jj), (lane & 16) | tb);
          float tau, scale, beta;
          householder_fast(alpha, ss, tau, scale, beta);
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            const int i = r0 + r;
            vL[i] = i == j ? 1.f : (i > j ? scale * col[r] : 0.f);
          }
          if (ti == 0) {
            sc[0] = tau;
            t[2 * j] = beta;
            tau4[j] = tau;
            tau4[2 * qm + j] = scale;
          }
        }
        __syncthreads();
        if (warp * 16 + 15 > j) {   // some column of this warp lies right of j
          const float tau = sc[0];
          float v[8];
          const float4 v0 = *reinterpret_cast<const float4*>(vL + r0);
          const float4 v1 = *reinterpret_cast<const float4*>(vL + r0 + 4);
          v[0] = v0.x; v[1] = v0.y; v[2] = v0.z; v[3] = v0.w;
          v[4] = v1.x; v[5] = v1.y; v[6] = v1.z; v[7] = v1.w;
          float2 wc[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float2 s = make_float2(0.f, 0.f);
#pragma unroll
            for (int r = 0; r < 8; ++r) s = __ffma2_rn(make_float2(v[r], v[r]), a[r][q], s);
            wc[q] = s;
          }
          {
            // reduce-scatter over the half-warp (lane bits 3, 2, 1 pick the
            // column), then all-gather
            float w8[8];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              w8[2 * q] = wc[q].x;
              w8[2 * q + 1] = wc[q].y;
            }
            const bool b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
            float k4[4], k2[2];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const float snd = b3 ? w8[i] : w8[i + 4], kp = b3 ? w8[i + 4] : w8[i];
              k4[i] = kp + __shfl_xor_sync(0xffffffffu, snd, 8);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i) {
              const float snd = b2 ? k4[i] : k4[i + 2], kp = b2 ? k4[i + 2] : k4[i];
              k2[i] = kp + __shfl_xor_sync(0xffffffffu, snd, 4);
            }
            float k1;
            {
              const float snd = b1 ? k2[0] : k2[1], kp = b1 ? k2[1] : k2[0];
              k1 = kp + __shfl_xor_sync(0xffffffffu, snd, 2);
            }
            k1 += __shfl_xor_sync(0xffffffffu, k1, 1);
            const int hb = lane & 16;
#pragma unroll
            for (int c = 0; c < 8; ++c)
              w8[c] = __shfl_sync(0xffffffffu, k1, hb | ((c >> 2) << 3) | (((c >> 1) & 1) << 2) | ((c & 1) << 1));
#pragma unroll
            for (int q = 0; q < 4; ++q) wc[q] = make_float2(w8[2 * q], w8[2 * q + 1]);
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            wc[q].x = (c0 + 2 * q > j) ? -tau * wc[q].x : 0.f;
            wc[q].y = (c0 + 2 * q + 1 > j) ? -tau * wc[q].y : 0.f;
          }
#pragma unroll
          for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) a[r][q] = __ffma2_rn(make_float2(v[r], v[r]), wc[q], a[r][q]);
        }
        if (j < Q - 1) {
          // ---- right reflector on row j (columns j+1..Q-1)
          const int ja = (jj + 1) & 7;       // local column of j+1
          const int ta = (j + 1) >> 3;       // its tile column
          // warp-uniform: some column of this warp lies right of j.  A warp
          // whose columns all lie left of j has a zero share of the row norm
          // and of W u, and nothing to update, so it skips both.
          const bool act = warp * 16 + 15 > j;
          float row[8];
          if (act) row_of(a, jj, row);
          if (ti == tb) {
            float ss = 0.f;
            if (act) {
#pragma unroll
              for (int c = 0; c < 8; ++c)
                if (c0 + c > j + 1) ss = fmaf(row[c], row[c], ss);
              if (tj == ta) sc[1] = sel8(row, ja);
            }
            rnp[tj] = ss;
          }
          __syncthreads();
          float ssr = 0.f;
#pragma unroll
          for (int q = 0; q < 16; q += 4) {
            const float4 p4 = *reinterpret_cast<const float4*>(rnp + q);
            ssr += p4.x;
            ssr += p4.y;
            ssr += p4.z;
            ssr += p4.w;
          }
          float tr, sr, br;
          householder_fast(sc[1], ssr, tr, sr, br);
          if (tid == 0) {
            t[2 * j + 1] = br;
            tau4[qm + j] = tr;
            tau4[3 * qm + j] = sr;
          }
          float2 u[4];
          float z[8];
          if (act) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const float2 x = make_float2(__shfl_sync(0xffffffffu, row[2 * q], (lane & 16) | tb),
                                           __shfl_sync(0xffffffffu, row[2 * q + 1], (lane & 16) | tb));
              const int c = c0 + 2 * q;
              u[q].x = c == j + 1 ? 1.f : (c > j + 1 ? sr * x.x : 0.f);
              u[q].y = c + 1 == j + 1 ? 1.f : (c + 1 > j + 1 ? sr * x.y : 0.f);
            }
#pragma unroll
            for (int r = 0; r < 8; ++r) {
              float2 s = make_float2(0.f, 0.f);
#pragma unroll
              for (int q = 0; q < 4; ++q) s = __ffma2_rn(a[r][q], u[q], s);
              z[r] = s.x + s.y;
            }
#pragma unroll
            for (int r = 0; r < 8; ++r) z[r] += __shfl_xor_sync(0xffffffffu, z[r], 16);
            if (lane < 16) {
              *reinterpret_cast<float4*>(zp + warp * 128 + r0) = make_float4(z[0], z[1], z[2], z[3]);
              *reinterpret_cast<float4*>(zp + warp * 128 + r0 + 4) = make_float4(z[4], z[5], z[6], z[7]);
            }
          }
          __syncthreads();
          // Row totals of W u, one thread per row, the warps' shares added in
          // warp order; a warp whose columns all lie left of j has a zero
          // share and did not write it.  Every thread then reads the totals
          // of its eight rows (one more barrier instead of each of the 16
          // threads of a row adding all eight shares again).
          if (tid < 128) {
            float zs = 0.f;
#pragma unroll
            for (int q = 0; q < kWarps; ++q)
              if (q * 16 + 15 > j) zs += zp[q * 128 + tid];
            zt[tid] = zs;
          }
          __syncthreads();
          if (act) {
            const float4 p0 = *reinterpret_cast<const float4*>(zt + r0);
            const float4 p1 = *reinterpret_cast<const float4*>(zt + r0 + 4);
            z[0] = p0.x; z[1] = p0.y; z[2] = p0.z; z[3] = p0.w;
            z[4] = p1.x; z[5] = p1.y; z[6] = p1.z; z[7] = p1.w;
#pragma unroll
            for (int r = 0; r < 8; ++r) {
              const float zr = (r0 + r > j) ? -tr * z[r] : 0.f;
#pragma unroll
              for (int q = 0; q < 4; ++q) a[r][q] = __ffma2_rn(make_float2(zr, zr), u[q], a[r][q]);
            }
          }
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = r0 + r, c = c0 + 2 * q;
      if (i < P && c < Q) W[i * ld + c] = a[r][q].x;
      if (i < P && c + 1 < Q) W[i * ld + c + 1] = a[r][q].y;
    }
  __syncthreads();
}

// Writes U_K (m x K) through (uo_r, uo_c) and C' = U_K^T X (K x n) through
// (co_r, co_c).  X is not modified.  K <= min(m, n), K <= 32.
template <typename R>
__device__ void cta_topk_left(const R* X, int m, int n, int K, TruncWork<R>& w, R* Uout, Ix uo_r,
                              Ix uo_c, R* Cout, Ix co_r, Ix co_c) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (K == m) {
    // Nothing is cut: any orthonormal basis of R^m works; take the identity.
    for (int e = tid; e < m * m; e += blockDim.x) {
      const int i = e / m, k = e % m;
      Uout[ixoff(uo_r, i) + ixoff(uo_c, k)] = i == k ? R(1) : R(0);
    }
    for (int e = tid; e < m * n; e += blockDim.x) {
      const int k = e / n, j = e % n;
      Cout[ixoff(co_r, k) + ixoff(co_c, j)] = X[e];
    }
    __syncthreads();
    return;
  }
  PEPS_PHASE(0);
  const bool tall = m >= n;
  const int P = tall ? m : n, Q = tall ? n : m;
  const int ld = w.ldw;
  R* W = w.Wm;
  R* tauL = w.tau;
  R* tauR = w.tau + w.Qmax;
  R* red = w.red;
  bool tiled = false;
  if constexpr (sizeof(R) == 4) {
    if (P > 32 && P <= 128) {   // below 33 rows the shared-memory version is as fast
      // the reflectors go to global memory: shared memory then holds the
      // inverse-iteration workspace
      W = w.Wg;
      bidiag_tiles_f32(X, n, tall, P, Q, W, ld, w.t, w.tau, w.Qmax);
      tiled = true;
    }
  }
  if (!tiled) {
    for (int e = tid; e < m * n; e += blockDim.x) {
      const int i = e / n, j = e % n;
      if (tall) W[i * ld + j] = X[e];
      else W[j * ld + i] = X[e];
    }
    __syncthreads();
    // ---------------- bidiagonalisation: W = Q_L B Q_R^T, B upper bidiagonal
    // Reflectors are kept unscaled in W with their scale factors in sL / sR
    // (v = scale * stored, implicit 1 on the diagonal / super-diagonal).  The
    // norm each Householder vector needs is accumulated while the previous
    // rank-1 update writes those entries, and every thread forms the scalars
    // itself, so one column costs four barriers.
    R* wv = w.wv;
    R* sL = w.tau + 2 * w.Qmax;        // left scale factors (t2 is filled later)
    R* sR = sL + w.Qmax;
    R* part = red + 40;                // per-warp partial norms (8)
    {
      R ss = R(0);
      for (int i = 1 + tid; i < P; i += blockDim.x) ss += W[i * ld] * W[i * ld];
      ss = block_sum(ss, red + 16);
      if (tid < kWarps) part[tid] = tid == 0 ? ss : R(0);
      __syncthreads();
    }
    for (int j = 0; j < Q; ++j) {
      // -- left reflector on column j (rows j..P-1); its norm is in part[]
      R colnorm = R(0);
      for (int q = 0; q < kWarps; ++q) colnorm += part[q];
      R tau, scale, beta;
      householder(W[j * ld + j], colnorm, tau, scale, beta);
      if (tid == 0) {
        w.t[2 * j] = beta;
        tauL[j] = tau;
        sL[j] = scale;
      }
      const int ncol = Q - j - 1;
      R rownorm = R(0);                // squared norm of row j beyond j+1 after the left update
      if (tau != R(0) && ncol > 0) {
        // wv[c] = tau * (W[j][c] + scale * sum_{i>j} W[i][j] W[i][c])
        int tpc = kThreads / ncol;
        tpc = tpc >= 32 ? 32 : tpc >= 16 ? 16 : tpc >= 8 ? 8 : tpc >= 4 ? 4 : tpc >= 2 ? 2 : 1;
        const int cpr = kThreads / tpc;
        for (int cb = 0; cb < ncol; cb += cpr) {
          const int cl = cb + tid / tpc, gl = tid % tpc;
          const bool act = cl < ncol;
          const int c = j + 1 + (act ? cl : 0);
          R s0 = R(0), s1 = R(0), s2 = R(0), s3 = R(0);
          int i = j + 1 + gl;
          for (; i + 3 * tpc < P; i += 4 * tpc) {
            s0 += W[i * ld + j] * W[i * ld + c];
            s1 += W[(i + tpc) * ld + j] * W[(i + tpc) * ld + c];
            s2 += W[(i + 2 * tpc) * ld + j] * W[(i + 2 * tpc) * ld + c];
            s3 += W[(i + 3 * tpc) * ld + j] * W[(i + 3 * tpc) * ld + c];
          }
          for (; i < P; i += tpc) s0 += W[i * ld + j] * W[i * ld + c];
          const R sacc = warp_sum((s0 + s1) + (s2 + s3), tpc);
          if (act && gl == 0) wv[c] = tau * (W[j * ld + c] + scale * sacc);
        }
        __syncthreads();
        // W[i][c] -= wv[c] v_i for i >= j, c > j; warp 0 takes row j and its norm
        for (int i = j + warp; i < P; i += kWarps) {
          const R v = i == j ? R(1) : scale * W[i * ld + j];
          R rn = R(0);
          for (int c = j + 1 + lane; c < Q; c += 32) {
            const R x = W[i * ld + c] - wv[c] * v;
            W[i * ld + c] = x;
            if (c >= j + 2) rn += x * x;
          }
          if (i == j) {
            rn = warp_sum(rn);
            if (lane == 0) red[5] = rn;
          }
        }
        __syncthreads();
        rownorm = red[5];
      } else if (ncol > 0) {
        if (warp == 0) {
          R rn = R(0);
          for (int c = j + 2 + lane; c < Q; c += 32) rn += W[j * ld + c] * W[j * ld + c];
          rn = warp_sum(rn);
          if (lane == 0) red[5] = rn;
        }
        __syncthreads();
        rownorm = red[5];
      }
      if (j < Q - 1) {
        // -- right reflector on row j (columns j+1..Q-1)
        R tr, sr, br;
        householder(W[j * ld + j + 1], rownorm, tr, sr, br);
        if (tid == 0) {
          w.t[2 * j + 1] = br;
          tauR[j] = tr;
          sR[j] = sr;
        }
        const int nrow = P - j - 1;
        if (tr != R(0)) {
          // wv[i] = tr * (W[i][j+1] + sr * sum_{c>j+1} W[i][c] W[j][c])
          int tpc = kThreads / nrow;
          tpc = tpc >= 32 ? 32 : tpc >= 16 ? 16 : tpc >= 8 ? 8 : tpc >= 4 ? 4 : tpc >= 2 ? 2 : 1;
          const int rpr = kThreads / tpc;
          for (int rb = 0; rb < nrow; rb += rpr) {
            const int rl = rb + tid / tpc, gl = tid % tpc;
            const bool act = rl < nrow;
            const int i = j + 1 + (act ? rl : 0);
            R s0 = R(0), s1 = R(0), s2 = R(0), s3 = R(0);
            int c = j + 2 + gl;
            for (; c + 3 * tpc < Q; c += 4 * tpc) {
              s0 += W[i * ld + c] * W[j * ld + c];
              s1 += W[i * ld + c + tpc] * W[j * ld + c + tpc];
              s2 += W[i * ld + c + 2 * tpc] * W[j * ld + c + 2 * tpc];
              s3 += W[i * ld + c + 3 * tpc] * W[j * ld + c + 3 * tpc];
            }
            for (; c < Q; c += tpc) s0 += W[i * ld + c] * W[j * ld + c];
            const R sacc = warp_sum((s0 + s1) + (s2 + s3), tpc);
            if (act && gl == 0) wv[i] = tr * (W[i * ld + j + 1] + sr * sacc);
          }
          __syncthreads();
          // W[i][c] -= wv[i] v'_c for i > j, c > j; lane 0 of each warp sums column j+1 below row j+1
          R vl[8];
  #pragma unroll
          for (int t = 0; t < 8; ++t) {
            const int c = j + 1 + lane + 32 * t;
            vl[t] = c == j + 1 ? R(1) : (c < Q ? sr * W[j * ld + c] : R(0));
          }
          R cn = R(0);
          for (int i = j + 1 + warp; i < P; i += kWarps) {
            const R wi = wv[i];
  #pragma unroll
            for (int t = 0; t < 8; ++t) {
              const int c = j + 1 + lane + 32 * t;
              if (c < Q) {
                const R x = W[i * ld + c] - wi * vl[t];
                W[i * ld + c] = x;
                if (t == 0 && lane == 0 && i > j + 1) cn += x * x;
              }
            }
          }
          if (lane == 0) part[warp] = cn;
          __syncthreads();
        } else {
          // no right update: column j+1's norm below row j+1 as it stands
          R cn = R(0);
          for (int i = j + 2 + tid; i < P; i += blockDim.x) cn += W[i * ld + j + 1] * W[i * ld + j + 1];
          cn = block_sum(cn, red + 16);
          if (tid < kWarps) part[tid] = tid == 0 ? cn : R(0);
          __syncthreads();
        }
      }
    }
    // the last column's diagonal entry (w.t[2Q-2], written by thread 0) is
    // read by another warp in the bisection set-up below
    __syncthreads();
  }   // !tiled
  PEPS_PHASE(1);
  // ---------------- Sturm bisection for the K largest singular values
  const int n2 = 2 * Q;
  R tmax = R(0);
  for (int i = tid; i < n2 - 1; i += blockDim.x) {
    const R v = w.t[i];
    w.t2[i] = v * v;
    tmax = fmax(tmax, fabs(v));
  }
  tmax = warp_max(tmax);
  if (lane == 0) red[8 + warp] = tmax;
  __syncthreads();
  tmax = R(0);
  for (int i = 0; i < kWarps; ++i) tmax = fmax(tmax, red[8 + i]);
  __syncthreads();
  const R bound = R(2) * tmax * (R(1) + R(4) * Eps<R>::eps) + Eps<R>::tiny;
  const R pivmin = Eps<R>::tiny * R(1024) * fmax(R(1), tmax * tmax);
  {
    const int G = K <= 16 ? 16 : 8;
    const int gid = tid / G, gl = tid % G;
    const int gbase = (lane / G) * G;
    const double lg = log((double)(G + 1));
    // (G+1)^nit >= 2^(bits+2): the final interval is below a quarter ulp of the bound
    const int nit = (int)((Eps<R>::bits + 2) * 0.6931471805599453 / lg) + 1;
    const int idx = n2 - 1 - gid;  // ascending index of the (gid+1)-th largest eigenvalue
    R lo = R(0), hi = bound;
    for (int it = 0; it < nit; ++it) {
      const R step = (hi - lo) / R(G + 1);
      bool pred = true;
      if (gid < K) {
        const R x = lo + step * R(gl + 1);
        pred = sturm_count(w.t2, n2, x, pivmin) <= idx;
      }
      const unsigned bal = __ballot_sync(0xffffffffu, pred);
      const unsigned bits = (bal >> gbase) & ((G == 32) ? 0xffffffffu : ((1u << G) - 1u));
      const int gstar = __popc(bits) - 1;
      const R nlo = gstar >= 0 ? lo + step * R(gstar + 1) : lo;
      const R nhi = gstar + 1 < G ? lo + step * R(gstar + 2) : hi;
      lo = nlo;
      hi = nhi;
    }
    if (gid < K && gl == 0) w.lam[gid] = R(0.5) * (lo + hi);
  }
  __syncthreads();
  PEPS_PHASE(2);
  // ---------------- inverse iteration, one thread per vector
  const R pivtiny = Eps<R>::eps * fmax(tmax, Eps<R>::tiny * R(1e10));
  {
    // in shared memory (the matrix buffer, free on the register-tiled path,
    // and the Ub buffer for the interchange bytes) when it fits
    const bool in_smem = tiled && (size_t)4 * n2 * K <= (size_t)w.Qmax * w.ldw;
    R* wsR = in_smem ? w.Wm : w.lu;
    unsigned char* wsP = in_smem ? reinterpret_cast<unsigned char*>(w.Ubs)
                                 : reinterpret_cast<unsigned char*>(w.lu + (size_t)4 * n2 * K);
    if (tid < K) inverse_iteration(w.t, n2, w.lam[tid], pivtiny, wsR, wsP, K, tid, w.Z + tid, K, (unsigned)(tid + 1));
  }
  __syncthreads();
  PEPS_PHASE(3);
  // extract u-parts (odd positions) for a tall matrix, v-parts (even) for a wide one
  R* Ub = w.Ubs;
  for (int e = tid; e < Q * K; e += blockDim.x) {
    const int i = e / K, k = e % K;
    Ub[e] = w.Z[(size_t)(2 * i + (tall ? 1 : 0)) * K + k];
  }
  __syncthreads();
  // ---------------- orthonormal basis of the kept vectors: CholeskyQR2
  // (G = Ub^T Ub = R^T R, Ub <- Ub R^-1, twice; Fukaya et al. 2014).  Each
  // pass costs three barriers.  If a direction of Ub is below 1e-3 of its
  // norm (a cluster or a zero singular value), Gram-Schmidt with replacement
  // of degenerate directions (below) takes over from the current Ub.
  bool need_cgs = false;
  {
    __shared__ int cq_bad;
    R* G = w.Uks;   // K x K, free until the back-transformation
    for (int pass = 0; pass < 2 && !need_cgs; ++pass) {
      for (int e = tid; e < K * K; e += blockDim.x) {
        const int a = e / K, b = e % K;
        if (b < a) continue;
        R sacc = R(0);
        for (int i = 0; i < Q; ++i) sacc += Ub[i * K + a] * Ub[i * K + b];
        G[e] = sacc;
      }
      __syncthreads();
      if (warp == 0) {
        // right-looking Cholesky of the upper triangle in place; lane l owns column l
        const R d0 = lane < K ? G[lane * K + lane] : R(0);
        int bad = 0;
        for (int j = 0; j < K && !bad; ++j) {
          const R d = G[j * K + j];
          const R dj0 = __shfl_sync(0xffffffffu, d0, j);
          if (!(d > R(1e-6) * dj0) || !(dj0 > R(0))) {
            bad = 1;
            break;
          }
          const R r = dsqrt(d);
          __syncwarp();
          if (lane > j && lane < K) G[j * K + lane] /= r;
          __syncwarp();
          if (lane == j) G[j * K + j] = r;
          if (lane > j && lane < K) {
            const R gjl = G[j * K + lane];
            for (int mm = j + 1; mm <= lane; ++mm) G[mm * K + lane] -= G[j * K + mm] * gjl;
          }
          __syncwarp();
        }
        if (lane == 0) cq_bad = bad;
      }
      __syncthreads();
      if (cq_bad) {
        need_cgs = true;
        break;
      }
      // Ub <- Ub R^-1, one thread per row (forward substitution in place)
      for (int i = tid; i < Q; i += blockDim.x) {
        for (int l = 0; l < K; ++l) {
          R x = Ub[i * K + l];
          for (int k = 0; k < l; ++k) x -= Ub[i * K + k] * G[k * K + l];
          Ub[i * K + l] = x / G[l * K + l];
        }
      }
      __syncthreads();
    }
  }
  // ---------------- Gram-Schmidt with re-orthogonalisation (CGS2), fallback
  for (int j = 0; j < K && need_cgs; ++j) {
    for (int attempt = 0; attempt <= Q; ++attempt) {
      R s = R(0);
      for (int i = tid; i < Q; i += blockDim.x) s += Ub[i * K + j] * Ub[i * K + j];
      R nrm0 = dsqrt(block_sum(s, red + 16));
      if (nrm0 > R(0)) {
        for (int i = tid; i < Q; i += blockDim.x) Ub[i * K + j] /= nrm0;
        __syncthreads();
      }
      for (int pass = 0; pass < 2; ++pass) {
        for (int p = warp; p < j; p += kWarps) {
          R d = R(0);
          for (int i = lane; i < Q; i += 32) d += Ub[i * K + p] * Ub[i * K + j];
          d = warp_sum(d);
          if (lane == 0) red[32 + p] = d;
        }
        __syncthreads();
        for (int i = tid; i < Q; i += blockDim.x) {
          R v = Ub[i * K + j];
          for (int p = 0; p < j; ++p) v -= red[32 + p] * Ub[i * K + p];
          Ub[i * K + j] = v;
        }
        __syncthreads();
      }
      s = R(0);
      for (int i = tid; i < Q; i += blockDim.x) s += Ub[i * K + j] * Ub[i * K + j];
      const R nrm = dsqrt(block_sum(s, red + 16));
      if (nrm0 > R(0) && nrm > R(1e-3)) {
        for (int i = tid; i < Q; i += blockDim.x) Ub[i * K + j] /= nrm;
        __syncthreads();
        break;
      }
      // degenerate direction (zero singular value or lost vector): try a unit vector
      const int q = (j + attempt) % Q;
      for (int i = tid; i < Q; i += blockDim.x) Ub[i * K + j] = i == q ? R(1) : R(0);
      __syncthreads();
    }
  }
  PEPS_PHASE(4);
  // ---------------- back-transformation by the stored reflectors, in blocks
  // U = H_0 H_1 ... H_{nref-1} [Ub; 0].  A block of nb consecutive reflectors
  // is applied at once as U -= V (T (V^T U)), with V = [v_j0 .. v_j0+nb-1] and
  // T the upper triangular factor of the compact WY form (Schreiber & Van
  // Loan 1989), built by the forward recurrence T_kk = tau_k,
  // T_{0:k,k} = -tau_k T_{0:k,0:k} (V_{:,0:k}^T v_k).  Reflector j has its
  // implicit 1 at row j (tall block) or j+1 (wide block) and scale * stored
  // entries below it.  V is written out per block into the Ub buffer, which
  // is free once Ub has been copied to Uk (nb <= K keeps it in bounds).
  R* Uk = w.Uks;
  const int rowsU = tall ? P : Q;
  for (int e = tid; e < rowsU * K; e += blockDim.x) {
    const int i = e / K, k = e % K;
    Uk[e] = i < Q ? Ub[i * K + k] : R(0);
  }
  __syncthreads();
  {
    constexpr int NBMAX = 8, KMAX = 32;   // reflectors per block; K <= 32
    __shared__ R bt_g[NBMAX][NBMAX], bt_t[NBMAX][NBMAX], bt_w1[NBMAX][KMAX + NBMAX], bt_w2[NBMAX][KMAX];
    const R* taus = tall ? tauL : tauR;
    const R* scs = tall ? w.tau + 2 * w.Qmax : w.tau + 3 * w.Qmax;
    if constexpr (sizeof(R) == 4) {
      // Register-tiled path: the reflectors, their factors and scales move
      // from global memory to shared memory once (the truncation matrix
      // buffer is free after the inverse iteration), all loads of a round in
      // flight together, instead of one exposed load latency per block below.
      __shared__ float bt_tau[128], bt_scs[128];
      if (tiled && w.wm_shared && Q <= 128) {
        R* Ws = w.Wm;
        const int tot = P * ld;
        for (int e0 = 0; e0 < tot; e0 += 8 * kThreads) {
          R v[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * kThreads + tid;
            v[u] = e < tot ? W[e] : R(0);
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * kThreads + tid;
            if (e < tot) Ws[e] = v[u];
          }
        }
        for (int e = tid; e < Q; e += kThreads) {
          bt_tau[e] = taus[e];
          bt_scs[e] = scs[e];
        }
        W = Ws;
        taus = bt_tau;
        scs = bt_scs;
        __syncthreads();
      }
    }
    const int nref = tall ? Q : Q - 1;
    bool applied = false;
    if constexpr (sizeof(R) == 4) {
      if (tiled && w.wm_shared && Q <= 128 && rowsU <= 128 && K <= 2 * kWarps) {
        // Reflectors in shared memory, at most 128 rows and 16 columns: one
        // column of U per half-warp (lane l holds rows l, l + 16, ...), the
        // reflectors applied one at a time, last first.  Each is a dot
        // product over the half-warp (shuffles) and an axpy; columns are
        // independent, so there is no barrier.
        const int c = warp * 2 + (lane >> 4), l = lane & 15;
        float u[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int i = l + 16 * r;
          u[r] = (c < K && i < rowsU) ? Uk[i * K + c] : 0.f;
        }
        for (int j = nref - 1; j >= 0; --j) {
          const int pv = tall ? j : j + 1;
          const float tj = taus[j], sj = scs[j];
          float v[8], d = 0.f;
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            const int i = l + 16 * r;
            const float wv = (i > pv && i < rowsU) ? (tall ? W[i * ld + j] : W[j * ld + i]) : 0.f;
            v[r] = i == pv ? 1.f : sj * wv;
            d = fmaf(v[r], u[r], d);
          }
#pragma unroll
          for (int o = 8; o >= 1; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
          const float cf = -tj * d;
#pragma unroll
          for (int r = 0; r < 8; ++r) u[r] = fmaf(cf, v[r], u[r]);
        }
        if (c < K) {
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            const int i = l + 16 * r;
            if (i < rowsU) Uk[i * K + c] = u[r];
          }
        }
        __syncthreads();
        applied = true;
      }
    }
    const int NB = K < NBMAX ? K : NBMAX;
    R* Vs = Ub;   // [rowsU][nb]
    for (int j0 = (nref > 0 && !applied) ? ((nref - 1) / NB) * NB : -1; j0 >= 0; j0 -= NB) {
      const int nb = min(NB, nref - j0);
      const int p0 = tall ? j0 : j0 + 1;
      for (int e = tid; e < (rowsU - p0) * nb; e += blockDim.x) {
        const int i = p0 + e / nb, aa = e % nb, j = j0 + aa, pv = tall ? j : j + 1;
        Vs[i * nb + aa] = i < pv ? R(0) : (i == pv ? R(1) : scs[j] * (tall ? W[i * ld + j] : W[j * ld + i]));
      }
      __syncthreads();
      // [W1 | G] = V^T [U | V] (nb x (K + nb)); two threads per dot product
      const int ncol = K + nb, nd = nb * ncol;
      for (int d0 = 0; d0 < nd; d0 += kThreads / 2) {
        const int d = d0 + (tid >> 1), part = tid & 1;
        R sacc = R(0);
        if (d < nd) {
          const int aa = d / ncol, c = d % ncol;
          const int pa = p0 + aa;   // first non-zero row of v_aa
          if (c < K) {
            for (int i = pa + part; i < rowsU; i += 2) sacc += Vs[i * nb + aa] * Uk[i * K + c];
          } else {
            for (int i = pa + part; i < rowsU; i += 2) sacc += Vs[i * nb + aa] * Vs[i * nb + (c - K)];
          }
        }
        sacc += __shfl_xor_sync(0xffffffffu, sacc, 1);
        if (part == 0 && d < nd) {
          const int aa = d / ncol, c = d % ncol;
          if (c < K) bt_w1[aa][c] = sacc;
          else bt_g[aa][c - K] = sacc;
        }
      }
      __syncthreads();
      // T, one thread per row: T[i][i] = tau_i, T[i][k] = -tau_k sum_{m=i}^{k-1} T[i][m] G[m][k]
      if (tid < nb) {
        const int i = tid;
        for (int k = 0; k < nb; ++k) bt_t[i][k] = R(0);
        bt_t[i][i] = taus[j0 + i];
        for (int k = i + 1; k < nb; ++k) {
          R acc = R(0);
          for (int m = i; m < k; ++m) acc += bt_t[i][m] * bt_g[m][k];
          bt_t[i][k] = -taus[j0 + k] * acc;
        }
      }
      __syncthreads();
      // W2 = T W1
      for (int e = tid; e < nb * K; e += blockDim.x) {
        const int aa = e / K, cc = e % K;
        R acc = R(0);
        for (int bb = aa; bb < nb; ++bb) acc += bt_t[aa][bb] * bt_w1[bb][cc];
        bt_w2[aa][cc] = acc;
      }
      __syncthreads();
      // U -= V W2 on rows p0.. (V is zero above its first pivot)
      for (int e = tid; e < (rowsU - p0) * K; e += blockDim.x) {
        const int i = p0 + e / K, cc = e % K;
        R acc = R(0);
        for (int aa = 0; aa < nb; ++aa) acc += Vs[i * nb + aa] * bt_w2[aa][cc];
        Uk[i * K + cc] -= acc;
      }
      __syncthreads();
    }
  }
  PEPS_PHASE(5);
  // ---------------- outputs, after one Newton-Schulz step towards the
  // nearest orthonormal basis (Higham, Functions of Matrices, Sec. 8.3):
  // U <- U (3/2 I - 1/2 U^T U).  In FP32 the reflectors leave U^T U - I at
  // ~1e-6, and each cut then applies a slightly wrong projector; the step
  // squares that defect.  The K x K factor goes into the free Ub buffer.
  //
  // FP32: U^T U and the carry U^T X are compensated dot products.  The kept
  // vectors are localised, so a plain FP32 sum drops most of their small
  // terms against the running sum, and always with the same sign: over the
  // 240 cuts of a 16x16 sweep that biased ln|psi| by ~3e-5, ten times the
  // error of an FP32 LAPACK SVD sweep.  The step is applied as
  // U + U (-1/2 (U^T U - I)), so its small correction is not rounded
  // against 1.
  if constexpr (sizeof(R) == 4) {
    float* Mns = reinterpret_cast<float*>(Ub);
    const float* Uf = reinterpret_cast<const float*>(Uk);
    for (int e = tid; e < K * K; e += blockDim.x) {
      const int a = e / K, b = e % K;
      float s = 0.f, c = 0.f;
      for (int i = 0; i < m; ++i) dot2_step(Uf[i * K + a], Uf[i * K + b], s, c);
      // s is within a factor 2 of 1 on the diagonal, so s - 1 is exact
      Mns[e] = -0.5f * (a == b ? __fadd_rn(__fsub_rn(s, 1.f), c) : __fadd_rn(s, c));
    }
    __syncthreads();
    // Up to kNsPer entries per thread, the new U replaces the old one in
    // shared memory once every thread has read the old one; larger U go to
    // the global copy.
    constexpr int kNsPer = 8;
    const bool u_shared = m * K <= kNsPer * kThreads;
    float* Us = reinterpret_cast<float*>(Uk);
    if (u_shared) {
      float nv[kNsPer];
#pragma unroll
      for (int q = 0; q < kNsPer; ++q) {
        const int e = tid + q * kThreads;
        if (e < m * K) {
          const int i = e / K, k = e % K;
          float corr = 0.f;
          for (int a = 0; a < K; ++a) corr = fmaf(Uf[i * K + a], Mns[a * K + k], corr);
          nv[q] = Uf[i * K + k] + corr;
          Uout[ixoff(uo_r, i) + ixoff(uo_c, k)] = nv[q];
        }
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < kNsPer; ++q) {
        const int e = tid + q * kThreads;
        if (e < m * K) Us[e] = nv[q];
      }
    } else {
      for (int e = tid; e < m * K; e += blockDim.x) {
        const int i = e / K, k = e % K;
        float corr = 0.f;
        for (int a = 0; a < K; ++a) corr = fmaf(Uf[i * K + a], Mns[a * K + k], corr);
        const float v = Uf[i * K + k] + corr;
        Uout[ixoff(uo_r, i) + ixoff(uo_c, k)] = v;
        w.Uk[e] = v;
      }
    }
    __syncthreads();
    // C' = U_K^T X, X row-major m x n.  One work item is a column j and a
    // chunk of 8 rows of C'; its X column is read once (coalesced over j),
    // eight rows at a time so that eight loads are in flight together.
    constexpr int CH = 8, XB = 8;
    const float* Uo = u_shared ? Us : reinterpret_cast<const float*>(w.Uk);
    const float* Xf = reinterpret_cast<const float*>(X);
    const int nchunk = (K + CH - 1) / CH;
    for (int item = tid; item < n * nchunk; item += blockDim.x) {
      const int j = item % n, a0 = (item / n) * CH;
      float s[CH], c[CH];
#pragma unroll
      for (int q = 0; q < CH; ++q) s[q] = c[q] = 0.f;
      for (int ib = 0; ib < m; ib += XB) {
        float xb[XB];
#pragma unroll
        for (int u = 0; u < XB; ++u) xb[u] = ib + u < m ? Xf[(ib + u) * n + j] : 0.f;
#pragma unroll
        for (int u = 0; u < XB; ++u) {
          const int i = ib + u;
          if (i < m) {
#pragma unroll
            for (int q = 0; q < CH; ++q)
              if (a0 + q < K) dot2_step(Uo[i * K + a0 + q], xb[u], s[q], c[q]);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < CH; ++q)
        if (a0 + q < K) Cout[ixoff(co_r, a0 + q) + ixoff(co_c, j)] = __fadd_rn(s[q], c[q]);
    }
    __syncthreads();
  } else {
    R* Mns = Ub;
    for (int e = tid; e < K * K; e += blockDim.x) {
      const int a = e / K, b = e % K;
      R sacc = R(0);
      for (int i = 0; i < m; ++i) sacc += Uk[i * K + a] * Uk[i * K + b];
      Mns[e] = (a == b ? R(1.5) : R(0)) - R(0.5) * sacc;
    }
    __syncthreads();
    for (int e = tid; e < m * K; e += blockDim.x) {
      const int i = e / K, k = e % K;
      R v = R(0);
      for (int a = 0; a < K; ++a) v += Uk[i * K + a] * Mns[a * K + k];
      Uout[ixoff(uo_r, i) + ixoff(uo_c, k)] = v;
      w.Uk[e] = v;
    }
    __syncthreads();
    // C' = U_K^T X
    GemmDesc g = gemm(K, n, m, ix1(1), kx(m, 0, K), kx(m, 0, n), ix1(1), co_r, co_c);
    cta_gemm<R>(g, w.Uk, X, Cout, false, w.gsm, w.gism);
  }
  PEPS_PHASE(6);
}

}  // namespace peps
