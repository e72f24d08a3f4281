// Two-row transfer step on the 5th-generation tensor cores (tcgen05, TF32
// inputs, FP32 accumulation in tensor memory) for D = 8, Dc = 16.
//
// Same contraction and slice order as pair_fused.cuh (slices over the in-bond
// s of the lower environment), written as four MMAs per slice, D = A B^T with
// both operands K-major in shared memory:
//   s1: D1[(u1,xo)][(y1i,y2i)]  = sum_xi        Mu[(u1,xo)][xi]        Ein[s][(y1i,y2i)][xi]    M128 N64 K16
//   s2: D2[(y2i,xo)][(y1o,m)]   = sum_(y1i,u1)  P1[(y2i,xo)][(y1i,u1)] T1[(y1o,m)][(y1i,u1)]    M128 N64 K64
//   s3: D3[(xo,y1o)][(y2o,d2)]  = sum_(y2i,m)   P2[(xo,y1o)][(y2i,m)]  T2[(y2o,d2)][(y2i,m)]    M128 N64 K64
//   s4: D4[(xo,y1o,y2o)][x'o]  += sum_d2        P3[row][d2]           Md[s][x'o][d2]           8 x (M128 N16 K8)
// D1..D3 share 64 TMEM columns (each is read out before the next MMA), D4
// (1024 x 16 FP32) stays in TMEM across all slices.  Between MMAs the
// accumulator is read with tcgen05.ld, rounded to TF32 and stored in the next
// operand's layout.
//
// Shared-memory operand layout (no swizzle): core matrices of 8 rows x 16
// bytes; element (row, k) of an R x K tile at
//   (row / 8) * sbo + (k / 4) * 32 + (row % 8) * 4 + (k % 4)   floats,
// i.e. leading (K-direction) byte offset 128 and stride (8-row) byte offset
// 4 sbo.  The B operands and the A operands of s1 and s2 are dense
// (sbo = K * 8).  The A operands of s3 and s4 are written by lanes that hold
// the same row of different 8-row groups; their 8-row groups are padded by 16
// bytes (sbo = K * 8 + 4) so that eight such 16-byte stores fall in distinct
// banks.
#pragma once

#include <cstdint>

#include "device.cuh"
#include "kernels.h"

namespace peps {

namespace tc {

constexpr int kTmemCols = 256;           // per CTA: 64 (D1..D3) + 128 (D4), rounded to a power of two
constexpr uint32_t kColP = 0, kColE = 64;
constexpr long kWaitLimit = 1l << 26;    // bounded mbarrier waits

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ int kmaj(int row, int k, int K) {
  return (row >> 3) * (K >> 2) * 32 + (k >> 2) * 32 + (row & 7) * 4 + (k & 3);
}
// The same with an explicit 8-row stride of `sbo` floats.
__device__ __forceinline__ int kmaj_sbo(int row, int k, int sbo) {
  return (row >> 3) * sbo + (k >> 2) * 32 + (row & 7) * 4 + (k & 3);
}

// Shared-memory matrix descriptor; sbo_bytes = 0 means the dense K * 32.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, int K, uint32_t sbo_bytes = 0) {
  const uint32_t lbo = 128, sbo = sbo_bytes ? sbo_bytes : (uint32_t)K * 32;
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// One MMA chain D[M x N] (+)= A[M x K] B[N x K]^T, K in steps of 8; single
// thread.  a_sbo: A's 8-row stride in bytes (0: dense).
__device__ __forceinline__ void mma_chain(uint32_t tmem_d, const float* A, const float* B, int M, int N, int K,
                                          bool accumulate, uint32_t a_sbo = 0) {
  const uint32_t idesc = idesc_tf32(M, N);
  const uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
  for (int ks = 0; ks < K / 8; ++ks) {
    const uint64_t ad = sdesc(a0 + ks * 256, K, a_sbo), bd = sdesc(b0 + ks * 256, K);
    const uint32_t acc = (accumulate || ks > 0) ? 1u : 0u;
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
  }
}

__device__ __forceinline__ void commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar)));
}

// Bounded wait for the given phase parity; returns false on timeout.
__device__ __forceinline__ bool wait_phase(uint64_t* mbar, uint32_t parity) {
  const uint32_t a = smem_u32(mbar);
  for (long it = 0; it < kWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(a), "r"(parity));
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;"); }

}  // namespace tc

struct PairTcSmem {
  // 8-row strides (floats) of the padded A operands of s3 (K = 64) and s4 (K = 8)
  static constexpr int sbo3 = 64 * 8 + 4, sbo4 = 8 * 8 + 4, tile4 = 16 * sbo4;
  static constexpr int A1 = 128 * 16, B1 = 64 * 16, AB = 8 * tile4, B2 = 64 * 64, B3 = 64 * 64, B4 = 16 * 8;
  static constexpr int total = A1 + B1 + AB + B2 + B3 + B4;   // floats
};

// Site tensors pre-arranged as B operands (TF32-rounded, core-matrix layout):
// for direction dir (0 left, 1 right), site i and spin s, two 64 x 64 tiles
//   TA[n = (yout, d)][k = (u, yin)]   (B of s2: contraction order (u1, y1i))
//   TB[n = (yout, d)][k = (yin, u)]   (B of s3: contraction order (y2i, m))
// with (yin, yout) = (l, r) for dir 0 and (r, l) for dir 1; offset of a
// tile: ((dir * N + i) * 2 + s) * 2 * 4096 (+ 4096 for TB).

// State shared by the steps of one CTA.
struct PairTc {
  uint32_t tmem;      // base TMEM address (lane 0, first column)
  uint64_t* mbar;     // completion barrier of the MMA chains
  uint64_t* tbar;     // completion barrier of the bulk copies
  uint32_t phase;     // parity of the next MMA completion
  uint32_t tphase;    // parity of the next copy completion
  bool ok;            // false after a timed-out wait
};

// Waits (all threads) for the chain issued by thread 0.  Uniform.
__device__ __forceinline__ bool tc_issue_wait(PairTc& st) {
  if (threadIdx.x == 0) tc::commit(st.mbar);
  const bool done = tc::wait_phase(st.mbar, st.phase & 1u);
  st.phase += 1;
  tc::tc_fence_after();
  const bool all = __syncthreads_and(done ? 1 : 0) != 0;
  if (!all) st.ok = false;
  return all;
}

__device__ __forceinline__ void ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int q = 0; q < 32; ++q) v[q] = tc::to_tf32(__uint_as_float(r[q]));
}

__device__ __forceinline__ void st4(float* p, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}

// One two-row transfer step, D = 8, Dc = 16, TF32 tensor cores.  Arguments
// as pair_step_fused, plus the pre-arranged B tiles of T1 (TA) and T2 (TB).
// Returns <result, Hdot> when Hdot is given; otherwise writes the result
// scaled by 2^-e to Eout and stores e in *e_out, as pair_step_fused.
static __device__ float pair_step_tc(PairTc& st, bool right, const float* Ein, float* __restrict__ Eout,
                              const float* __restrict__ Mu, const float* __restrict__ TA1,
                              const float* __restrict__ TB2, const float* __restrict__ Md,
                              const float* Hdot, float* sm, float* red, int* e_out = nullptr) {
  constexpr int D = 8, Dc = 16;
  using S = PairTcSmem;
  float* A1 = sm;
  float* B1 = A1 + S::A1;
  float* AB = B1 + S::B1;
  float* B2 = AB + S::AB;
  float* B3 = B2 + S::B2;
  float* B4 = B3 + S::B3;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  const int half = warp >> 2;   // warps 0-3 and 4-7 split the TMEM columns
  const int row = (warp & 3) * 32 + lane;
  if (!st.ok) return 0.f;
  __syncthreads();
  // ---- B2, B3: two 16 KB bulk copies (TMA engine) of the pre-arranged tiles
  if (tid == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(st.tbar)),
                 "r"(2 * kTcTile * 4));
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     tc::smem_u32(B2)),
                 "l"(TA1), "r"(kTcTile * 4), "r"(tc::smem_u32(st.tbar))
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     tc::smem_u32(B3)),
                 "l"(TB2), "r"(kTcTile * 4), "r"(tc::smem_u32(st.tbar))
                 : "memory");
  }
  // ---- A1 = Mu as [m = (u1, xo)][k = xi]; two 16-byte groups of xi per thread
  {
    const int m = tid >> 1, xq = (tid & 1) * 8;
    const int u1 = m / Dc, xo = m % Dc;
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int xi = xq + j;
      const int a = right ? xo : xi, b = right ? xi : xo;
      v[j] = tc::to_tf32(Mu[a * D * Dc + u1 * Dc + b]);
    }
    st4(A1 + tc::kmaj(m, xq, 16), v[0], v[1], v[2], v[3]);
    st4(A1 + tc::kmaj(m, xq + 4, 16), v[4], v[5], v[6], v[7]);
  }
  {
    const bool got = tc::wait_phase(st.tbar, st.tphase & 1u);
    st.tphase += 1;
    if (__syncthreads_and(got ? 1 : 0) == 0) {
      st.ok = false;
      return 0.f;
    }
  }
  // Slice s+1 of Ein and Md is loaded into registers as soon as slice s is
  // staged, so the loads complete under slice s's four MMA stages.
  // this thread's B1 entries (consecutive lanes take consecutive rows, so the
  // 16-byte stores of a warp fall in distinct banks) and B4 entries (tid < 32)
  const int bn = tid & 63, bxq = (tid >> 6) * 4;
  const int mxo = tid & 15, mdq = (tid >> 4) * 4;
  auto load_slice = [&](int s, float (&e)[4], float (&md)[4]) {
    const float* src = Ein + s * (Dc * 64) + bn;
#pragma unroll
    for (int j = 0; j < 4; ++j) e[j] = src[(bxq + j) * 64];
    if (tid < 32) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int d = mdq + j;
        md[j] = right ? Md[mxo * D * Dc + d * Dc + s] : Md[s * D * Dc + d * Dc + mxo];
      }
    }
  };
  float pe[4], pm[4] = {0.f, 0.f, 0.f, 0.f};
  load_slice(0, pe, pm);
  for (int s = 0; s < Dc; ++s) {
    // ---- B1 = Ein slice as [n = (y1i, y2i)][k = xi]; B4 = Md slice as [x'o][d2]
    st4(B1 + tc::kmaj(bn, bxq, 16), tc::to_tf32(pe[0]), tc::to_tf32(pe[1]), tc::to_tf32(pe[2]),
        tc::to_tf32(pe[3]));
    if (tid < 32)
      st4(B4 + tc::kmaj(mxo, mdq, 8), tc::to_tf32(pm[0]), tc::to_tf32(pm[1]), tc::to_tf32(pm[2]),
          tc::to_tf32(pm[3]));
    if (s + 1 < Dc) load_slice(s + 1, pe, pm);
    tc::fence_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    // ---- s1: D1[(u1,xo)][(y1i,y2i)]
    if (tid == 0) tc::mma_chain(st.tmem + tc::kColP, A1, B1, 128, 64, 16, false);
    if (!tc_issue_wait(st)) return 0.f;
    {
      // A2[m = (y2i, xo)][k = (u1, y1i)]: this thread holds y1i = 4*half .. +3 for every y2i
      float v[32];
      ld32(st.tmem + lane_base + tc::kColP + half * 32, v);
      const int u1 = row >> 4, xo = row & 15;
#pragma unroll
      for (int y2 = 0; y2 < 8; ++y2)
        st4(AB + tc::kmaj(y2 * Dc + xo, u1 * D + half * 4, 64), v[y2], v[8 + y2], v[16 + y2], v[24 + y2]);
    }
    tc::fence_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    // ---- s2: D2[(y2i,xo)][(y1o,m)]
    if (tid == 0) tc::mma_chain(st.tmem + tc::kColP, AB, B2, 128, 64, 64, false);
    if (!tc_issue_wait(st)) return 0.f;
    {
      // A3[m = (xo, y1o)][k = (y2i, m)]: this thread holds y1o = 4*half .. +3, all m
      float v[32];
      ld32(st.tmem + lane_base + tc::kColP + half * 32, v);
      const int y2 = row >> 4, xo = row & 15;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int y1o = half * 4 + j;
        st4(AB + tc::kmaj_sbo(xo * D + y1o, y2 * D, S::sbo3), v[j * 8 + 0], v[j * 8 + 1], v[j * 8 + 2],
            v[j * 8 + 3]);
        st4(AB + tc::kmaj_sbo(xo * D + y1o, y2 * D + 4, S::sbo3), v[j * 8 + 4], v[j * 8 + 5], v[j * 8 + 6],
            v[j * 8 + 7]);
      }
    }
    tc::fence_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    // ---- s3: D3[(xo,y1o)][(y2o,d2)]
    if (tid == 0) tc::mma_chain(st.tmem + tc::kColP, AB, B3, 128, 64, 64, false, S::sbo3 * 4);
    if (!tc_issue_wait(st)) return 0.f;
    {
      // A4 (8 tiles of 128 rows): row (xo, y1o, y2o), k = d2; this thread holds y2o = 4*half .. +3
      float v[32];
      ld32(st.tmem + lane_base + tc::kColP + half * 32, v);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int m = row * D + half * 4 + j;
        float* tile = AB + (m >> 7) * S::tile4;
        st4(tile + tc::kmaj_sbo(m & 127, 0, S::sbo4), v[j * 8 + 0], v[j * 8 + 1], v[j * 8 + 2], v[j * 8 + 3]);
        st4(tile + tc::kmaj_sbo(m & 127, 4, S::sbo4), v[j * 8 + 4], v[j * 8 + 5], v[j * 8 + 6], v[j * 8 + 7]);
      }
    }
    tc::fence_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    // ---- s4: eight M=128 tiles accumulate into D4 across the slices
    if (tid == 0)
      for (int t = 0; t < 8; ++t)
        tc::mma_chain(st.tmem + tc::kColE + t * 16, AB + t * S::tile4, B4, 128, 16, 8, s > 0, S::sbo4 * 4);
    if (!tc_issue_wait(st)) return 0.f;
  }
  // ---- result: tile t rows t*128 + row, 16 columns x'o
  float dot = 0.f;
  if (Hdot == nullptr) {
    float mx = 0.f;
    for (int t = half; t < 8; t += 2) {
      float v[16];
      tc::ld16(st.tmem + lane_base + tc::kColE + t * 16, v);
#pragma unroll
      for (int x = 0; x < Dc; ++x) mx = fmaxf(mx, fabsf(v[x]));
    }
    tc::tc_fence_before();
    const int e = pow2_exponent(block_max(mx, red));
    tc::tc_fence_after();
    const float sc = pow2<float>(-e);
    if (e_out) *e_out = e;
    for (int t = half; t < 8; t += 2) {
      float v[16];
      tc::ld16(st.tmem + lane_base + tc::kColE + t * 16, v);
      const int m = t * 128 + row;
#pragma unroll
      for (int x = 0; x < Dc; ++x) Eout[x * 1024 + m] = v[x] * sc;
    }
  } else {
    for (int t = half; t < 8; t += 2) {
      float v[16];
      tc::ld16(st.tmem + lane_base + tc::kColE + t * 16, v);
      const int m = t * 128 + row;
#pragma unroll
      for (int x = 0; x < Dc; ++x) dot = fmaf(v[x], Hdot[x * 1024 + m], dot);
    }
  }
  tc::tc_fence_before();
  if (Hdot != nullptr) dot = block_sum(dot, red);
  __syncthreads();
  tc::tc_fence_after();
  return dot;
}

}  // namespace peps
