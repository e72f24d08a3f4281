// Kernel arguments and launchers shared by the device code and the C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace peps {

constexpr int kMaxWords = 64;        // up to 4096 sites
constexpr int kMaxL = 64;            // Lx, Ly <= 64
constexpr int kMaxDc = 32;           // K <= 32 in the truncation
constexpr int kMaxDcD = 256;         // Dc * D <= 256

// Floats per pre-arranged B tile of the tensor-core two-row step.
constexpr int kTcTile = 4096;

// Per-configuration status bits written by the kernels.
constexpr int kFlagZeroW = 1;        // some W (psi, a row or a row pair) is exactly zero
constexpr int kFlagTimeout = 2;      // a bounded device wait gave up

struct Geometry {
  int Lx, Ly, D, Dc, N, nwords;
  double J1, J2;
  int fit;               // variational-fit sweeps after each zip-up (0: the zip-up truncation alone)
};

template <typename R>
struct KArgs {
  Geometry g;
  const R* A;             // [N][2][D^4] padded site tensors
  const R* triv_mps;      // [Lx][Dc*D*Dc] trivial boundary MPS (value 1)
  const R* triv_t1;       // [Dc*D*Dc] trivial single-row transfer
  const R* triv_t2;       // [Dc*D*D*Dc] trivial two-row transfer
  const int* bd;          // [2][Ly][Lx+1] bond dimensions after absorbing j rows (per sweep)
  const uint64_t* S;      // [n][nwords]
  int n;
  R* envU;                // [n][Ly][Lx][Dc*D*Dc] upper environments U_r
  R* envL;                // [n][Ly][Lx][Dc*D*Dc] lower environments L_r
  double* logabs;         // [n]
  int8_t* sign;           // [n]
  int* flags;             // [n]
  double* eloc_h;         // [n][Ly]
  double* eloc_v;         // [n][Ly]
  double* w_row;          // [n][Ly] single-row sandwich values W_r between the unit-norm environments
  double* lnU;            // [n][Ly] ln of the norm divided out after absorbing row r (top-down sweep), or null
  unsigned* cache;        // [n] environment cache bits (bit dir: sweep dir in place; bit 2 + dir: it met W = 0), or null
  R* O;                   // [n][N][D^4] or null
  const float* tcB;       // tensor-core path: site tensors pre-arranged as B tiles (pair_tc.cuh)
  R* scratch;             // per-CTA slots
  size_t slot_elems;
  int smem_wm;            // 1 if the truncation matrix lives in dynamic shared memory
};

struct GradArgs {
  int N, D4, nwords, n;
  const uint64_t* S;
  const double* eloc;
  const int* status;
  double* sumO;           // [N][2][D4]
  double* sumEO;          // [N][2][D4]
};

// Slot sizes (elements) of each kernel's per-CTA scratch.
size_t boundary_slot_elems(const Geometry& g, bool wm_in_smem);
size_t row_slot_elems(const Geometry& g);
size_t pair_slot_elems(const Geometry& g);
size_t mc_slot_elems(const Geometry& g, bool wm_in_smem);
size_t wm_smem_bytes(const Geometry& g, size_t elem);
bool wm_fits_smem(const Geometry& g, size_t elem);

template <typename R> cudaError_t launch_boundary(const KArgs<R>& a, int dirs, int grid, cudaStream_t st);
// generic != 0 takes the generic kernel even where a fused one exists for (D, Dc).
template <typename R> cudaError_t launch_row(const KArgs<R>& a, int grid, cudaStream_t st, int generic = 0);
template <typename R> cudaError_t launch_pair(const KArgs<R>& a, int grid, cudaStream_t st, int generic = 0);
template <typename R> cudaError_t launch_mc(const KArgs<R>& a, uint64_t* S, int nsweeps, uint64_t seed,
                                            uint64_t chain0, uint64_t sweep0, long long* accepted,
                                            int grid, cudaStream_t st);
template <typename R> int max_blocks_boundary(const Geometry& g);
// Boundary sweeps of several models in one launch (k_boundary_packed): models_dev
// [nm] kernel arguments in device memory, start_dev [nm + 1] first work item of
// each model (n * dirs items per model), one scratch slot of slot_elems reals
// per CTA, smem bytes of dynamic shared memory (the largest model's).
template <typename R> int max_blocks_boundary_packed(size_t smem);
template <typename R> cudaError_t launch_boundary_packed(const KArgs<R>* models_dev, const int* start_dev, int nm,
                                                         int dirs, R* scratch, size_t slot_elems, size_t smem,
                                                         int grid, cudaStream_t st);
size_t dyn_smem_bytes(const Geometry& g, size_t elem, bool truncates, bool wm_in_smem);
template <typename R> int max_blocks_mc(const Geometry& g);
template <typename R> int max_blocks_row(const Geometry& g, int generic = 0);
template <typename R> int max_blocks_pair(const Geometry& g);
template <typename R> int max_blocks_pair_fused(const Geometry& g);   // 0: no fused step for (D, Dc)
template <typename R> cudaError_t launch_grad_accum(const GradArgs& a, const R* O, cudaStream_t st);

// Sampled spin-spin exchange ratios for the correlation functions (Sec. IV).
struct CorrArgs {
  const int* sites;       // [nc] sites of the central region
  const int* pos;         // [N] index of a site in `sites`, or -1
  const int* status;      // [n] per-configuration status (k_finalize); non-zero ones are skipped
  int nc;
  double* xsum;           // [n] sum over antiparallel pairs p < q of eps_p eps_q W(S^pq)/W(S)
  double* corr;           // [nc][nc] += (1/2) W(S^pq)/W(S) at (p, q) and (q, p), or null
  size_t slot_elems;      // per-CTA scratch
};
size_t corr_slot_elems(const Geometry& g, bool wm_in_smem);
template <typename R> int max_blocks_corr(const Geometry& g);
template <typename R> cudaError_t launch_corr(const KArgs<R>& a, const CorrArgs& c, int grid, cudaStream_t st);
// M^2 per configuration and the S^z S^z part of the correlation sums.
cudaError_t launch_corr_finalize(const Geometry& g, const CorrArgs& c, const uint64_t* S, int n, const int* status,
                                 double* m2, cudaStream_t st);

// Tensor-core two-row step (TF32, D = 8, Dc = 16).
int max_blocks_pair_tc();
cudaError_t launch_pair_tc(const KArgs<float>& a, int grid, cudaStream_t st);

cudaError_t launch_finalize(const Geometry& g, const uint64_t* S, int n, const double* eloc_h,
                            const double* eloc_v, const int* flags, double* eloc, int* status,
                            int have_eloc, cudaStream_t st);
cudaError_t launch_grad_finalize(int total, int n_ok_dev_unused, const double* sums, const double* sumO,
                                 const double* sumEO, double* grad, double* cov, cudaStream_t st);
// One gradient-optimisation update (Sec. III) of the FP64 tensors A [N][2][D^4] in place.
cudaError_t launch_go_step(double* A, const double* grad, const Geometry& geo, double dt, uint64_t seed,
                           uint64_t step, int nsm, cudaStream_t st);
// Environment cache: for each configuration whose bits S differ from the
// cached copy, clear its cache bits and store the new bits.
cudaError_t launch_cache_check(const uint64_t* S, uint64_t* Scache, unsigned* bits, int n, int nwords,
                               cudaStream_t st);
// *bad |= 1 when a derivative of [N][2][D^4] is NaN or infinite.
cudaError_t launch_go_check(const double* grad, const Geometry& geo, int* bad, int nsm, cudaStream_t st);
// FP64 -> FP32 copy of n tensor entries.
cudaError_t launch_to_f32(const double* a, float* b, size_t n, int nsm, cudaStream_t st);
// Tensor-core B tiles (D = 8) of the FP64 site tensors [N][2][8^4].
cudaError_t launch_tc_tiles(const double* A, float* tiles, int N, int nsm, cudaStream_t st);
// Records the calling thread's error message (returned by peps_last_error).
void set_last_error(const char* msg);

}  // namespace peps

struct peps_ctx;

namespace peps {

// Worker contexts for the serving loop (api.cu).
peps_ctx* ctx_clone(peps_ctx* c, cudaStream_t stream, double workspace_gb, int share);
size_t ctx_footprint(peps_ctx* c, int n, double workspace_gb, int share);
size_t ctx_workspace_bytes(peps_ctx* c);
cudaStream_t ctx_stream(peps_ctx* c);
bool ctx_is_fp64(const peps_ctx* c);

cudaError_t launch_sum_eloc(const double* eloc, const int* status, int n, double* sums, cudaStream_t st);

}  // namespace peps
