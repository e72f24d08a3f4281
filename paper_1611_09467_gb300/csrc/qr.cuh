// Householder QR of small column-major matrices by one CTA (LAPACK's
// convention: beta = -sign(alpha) |x|, tau = (beta - alpha) / beta, the
// reflector v = [1; x / (alpha - beta)] stored below the diagonal), and the
// application of Q = H_0 H_1 ... H_{k-1} to another matrix.  Used by the
// variational-fit truncation (re-orthonormalising MPS tensors) and the
// simple update (isolating a bond).
#pragma once

namespace peps {
namespace qr {

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the CTA; `red` holds >= 32 reals of shared memory.  Uniform result.
template <typename R>
__device__ R block_sum(R v, R* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  R t = R(0);
  for (int k = 0; k < nw; ++k) t += red[k];
  return t;
}

// In place on the column-major m x n matrix M: R in the upper triangle of the
// first min(m, n) rows, the reflectors below it, tau[k] their factors.
template <typename R>
__device__ void house_qr(R* M, int m, int n, R* tau, R* red) {
  const int k_end = min(m, n);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  __shared__ R s_scale;
  for (int k = 0; k < k_end; ++k) {
    R* x = M + (size_t)k * m;
    R s2 = R(0);
    for (int r = k + 1 + threadIdx.x; r < m; r += blockDim.x) s2 += x[r] * x[r];
    s2 = block_sum<R>(s2, red);
    if (threadIdx.x == 0) {
      const R alpha = x[k];
      if (s2 == R(0)) {
        tau[k] = R(0);
        s_scale = R(0);
      } else {
        const R nrm = sqrt(alpha * alpha + s2);
        const R beta = alpha <= R(0) ? nrm : -nrm;
        tau[k] = (beta - alpha) / beta;
        s_scale = R(1) / (alpha - beta);
        x[k] = beta;
      }
    }
    __syncthreads();
    const R sc = s_scale;
    if (sc != R(0))
      for (int r = k + 1 + threadIdx.x; r < m; r += blockDim.x) x[r] *= sc;
    __syncthreads();
    const R t = tau[k];
    if (t != R(0)) {
      for (int c = k + 1 + warp; c < n; c += nw) {
        R* y = M + (size_t)c * m;
        R w = R(0);
        for (int r = k + 1 + lane; r < m; r += 32) w += x[r] * y[r];
        w = warp_sum(w) + y[k];
        w *= t;
        if (lane == 0) y[k] -= w;
        __syncwarp();
        for (int r = k + 1 + lane; r < m; r += 32) y[r] -= w * x[r];
      }
    }
    __syncthreads();
  }
}

// N <- H_0 H_1 ... H_{k-1} N, k = min(m, n_qr) reflectors of house_qr(M, m,
// n_qr), N column-major m x ncols.
template <typename R>
__device__ void apply_q(const R* M, const R* tau, R* N, int m, int n_qr, int ncols) {
  const int k_end = min(m, n_qr);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  for (int k = k_end - 1; k >= 0; --k) {
    const R t = tau[k];
    if (t != R(0)) {
      const R* v = M + (size_t)k * m;
      for (int c = warp; c < ncols; c += nw) {
        R* y = N + (size_t)c * m;
        R w = R(0);
        for (int r = k + 1 + lane; r < m; r += 32) w += v[r] * y[r];
        w = warp_sum(w) + y[k];
        w *= t;
        if (lane == 0) y[k] -= w;
        __syncwarp();
        for (int r = k + 1 + lane; r < m; r += 32) y[r] -= w * v[r];
      }
    }
    __syncthreads();
  }
}

}  // namespace qr
}  // namespace peps
