// Throughput probes for the roofline denominators of the kernels here: FP32
// and FP64 fused multiply-add on the SIMT pipes, and TF32 tcgen05.mma on the
// tensor cores.  Each runs long independent chains on every SM and is timed
// with CUDA events; the results are the pipes' sustained rates on this GPU,
// not a model of them.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/peps.h"
#include "pair_tc.cuh"

namespace peps {
namespace probe {

constexpr int kT = 256;

// 8 independent FMA chains per thread, `iters` rounds; the result is stored
// only if it is NaN (never, for these inputs), so the chains are not removed.
template <typename T>
__global__ void __launch_bounds__(kT) k_fma(int iters, T a, T b, T* sink) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = x[k] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s != s) sink[threadIdx.x] = s;
}

// One CTA per SM (its shared-memory request leaves room for one): thread 0
// issues `iters` chains of tcgen05.mma kind::tf32, M = 128, N = n (<= 256),
// K = 8 per instruction (4 per chain), from shared-memory operands into one
// TMEM accumulator, then commits them to an mbarrier and waits (bounded) for
// their completion.  Operand values are irrelevant.
__global__ void __launch_bounds__(128) k_tf32_mma(int iters, int n, int* timeout_flag) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_holder;
  float* A = reinterpret_cast<float*>(smem_raw);        // 128 x 32 (K-major core matrices)
  float* B = A + 128 * 32;                              // 256 x 32
  for (int e = threadIdx.x; e < (128 + 256) * 32; e += blockDim.x) A[e] = 0.0f;
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(&tmem_holder)),
                 "r"(256));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc::smem_u32(&mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  tc::fence_async_smem();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tmem_holder;
  bool ok = true;
  if (threadIdx.x == 0) {
    for (int it = 0; it < iters; ++it) tc::mma_chain(tmem, A, B, 128, n, 32, it > 0);
    tc::commit(&mbar);
    ok = tc::wait_phase(&mbar, 0);
    if (!ok) atomicOr(timeout_flag, 1);
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
}

}  // namespace probe
}  // namespace peps

namespace {

template <typename T>
double time_fma(int nsm, double* tflops) {
  using namespace peps::probe;
  T* sink = nullptr;
  if (cudaMalloc(&sink, kT * sizeof(T)) != cudaSuccess) return -1;
  const int grid = nsm * 8, iters = sizeof(T) == 4 ? 1 << 14 : 1 << 12;
  k_fma<T><<<grid, kT>>>(64, (T)0.999, (T)1e-4, sink);   // warm-up
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a);
  k_fma<T><<<grid, kT>>>(iters, (T)0.999, (T)1e-4, sink);
  cudaEventRecord(b);
  cudaEventSynchronize(b);
  float ms = 0;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(sink);
  const double flops = 2.0 * 8 * (double)iters * grid * kT;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return ms;
}


// Times `iters` chains of M128 x N x K32 TF32 MMAs on every SM (one CTA per SM).
peps_status time_tf32_mma(int nsm, int n, double* tflops) {
  using namespace peps::probe;
  int* flag = nullptr;
  if (cudaMalloc(&flag, sizeof(int)) != cudaSuccess) return PEPS_ENOMEM;
  cudaMemset(flag, 0, sizeof(int));
  const size_t smem = 120 * 1024;   // > half of an SM's shared memory: one CTA per SM
  cudaFuncSetAttribute(k_tf32_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int iters = 4096;
  k_tf32_mma<<<nsm, 128, smem>>>(16, n, flag);   // warm-up
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a);
  k_tf32_mma<<<nsm, 128, smem>>>(iters, n, flag);
  cudaEventRecord(b);
  cudaEventSynchronize(b);
  float ms = 0;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  int h = 0;
  cudaMemcpy(&h, flag, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(flag);
  if (cudaGetLastError() != cudaSuccess) return PEPS_ECUDA;
  if (h) return PEPS_ETIMEOUT;
  *tflops = 2.0 * 128 * n * 32 * (double)iters * nsm / (ms * 1e-3) / 1e12;
  return PEPS_OK;
}

}  // namespace

extern "C" {

/* Measured peaks: out[0] FP32 FMA TFLOP/s (SIMT), out[1] FP64 FMA TFLOP/s
 * (SIMT), out[2] TF32 tcgen05.mma TFLOP/s (dense, FP32 accumulation).
 * Synchronises the device.  PEPS_ETIMEOUT if the tensor-core probe's bounded
 * wait gave up. */
peps_status peps_measure_peaks(double* out) {
  if (!out) return PEPS_EINVAL;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PEPS_ECUDA;
  if (time_fma<float>(nsm, &out[0]) < 0 || time_fma<double>(nsm, &out[1]) < 0) return PEPS_ECUDA;
  return time_tf32_mma(nsm, 256, &out[2]);
}

peps_status peps_measure_tf32_mma_shape(int n, double* tflops) {
  if (!tflops || !(n == 16 || n == 32 || n == 64 || n == 128 || n == 256)) return PEPS_EINVAL;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PEPS_ECUDA;
  return time_tf32_mma(nsm, n, tflops);
}

}  // extern "C"
