/*
 * peps.h -- C ABI of the GB300 PEPS sampling path (libpeps.so).
 *
 * The library evaluates, for a fixed finite open-boundary PEPS (Eq. 1 of
 * Liu, Dong, Han, Guo, He, "Gradient optimization of finite projected
 * entangled pair states", arXiv:1611.09467) and a batch of spin
 * configurations S, the quantities of the Monte Carlo scheme of Sec. II:
 *   - W(S) = psi(S), the single-layer network at fixed S (Fig. 1c),
 *     contracted row by row with a boundary MPS of bond dimension Dc (Fig. 1d);
 *   - E(S) = sum_S' W(S')/W(S) <S'|H|S> for the J1-J2 Heisenberg model of
 *     Sec. IV (spin 1/2, S = sigma/2, open boundaries);
 *   - Delta(S) = B(S)/W(S) = d ln psi / dA (Sec. II, B the environment of a site);
 *   - the MC estimates of the energy and of dE/dA = 2<Delta E> - 2<Delta><E>;
 *   - Metropolis sweeps that sample S with weight W^2.
 *
 * Conventions
 *   - Lattice Ly rows x Lx columns, site i = row * Lx + col.  Spin s in {0,1},
 *     s = 0 is S^z = +1/2.  A configuration is ceil(N/64) uint64 words,
 *     bit i of word i/64 is s_i.
 *   - Site tensors A[N][d=2][D][D][D][D] in the index order (l, r, u, d) of
 *     Eq. 1, padded to D on open edges: entries past the true edge dimension
 *     (one) must be zero.
 *   - All array arguments named *_dev are device pointers owned by the caller
 *     (the library never frees them); *_host are host pointers.  Work is
 *     enqueued on the context's stream; calls return after enqueueing except
 *     where noted.  Return values report argument, allocation and launch
 *     errors only; per-configuration problems go to status_dev.
 *   - Per-configuration status: 0 ok, PEPS_EINVAL (popcount != N/2),
 *     PEPS_ENUMERIC (some W is exactly zero: ln|psi| = -inf, sign 0, E and
 *     Delta undefined, excluded from the averages).
 *   - A context is not thread-safe; use one context per stream.
 *   - Readings of points the paper leaves open: zip-up truncation with SVD
 *     cut to the Dc largest singular values, rows absorbed with alternating
 *     direction; ratios and Delta use the environments of S and the W of the
 *     same single-row (horizontal pairs, Delta) or two-row (vertical and
 *     diagonal pairs) sandwich; next-nearest pairs are both diagonals of
 *     each plaquette.
 */
#ifndef PEPS_H
#define PEPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct peps_ctx peps_ctx;

typedef enum {
  PEPS_OK = 0,
  PEPS_EINVAL = 1,    /* invalid argument or configuration */
  PEPS_ENOMEM = 2,    /* device allocation failed */
  PEPS_ECUDA = 3,     /* CUDA runtime or launch error */
  PEPS_ETIMEOUT = 4,  /* a bounded device wait gave up */
  PEPS_ENUMERIC = 5   /* zero amplitude */
} peps_status;

typedef enum {
  PEPS_FP64 = 0,        /* contractions and truncation in FP64 */
  PEPS_FP32 = 1,        /* contractions and truncation in FP32; log scales and reductions FP64 */
  PEPS_MIXED_TF32 = 2,  /* PEPS_FP32 with the two-row sandwich transfers on the tensor cores
                           (tcgen05, TF32 inputs, FP32 accumulation) where D = 8, Dc = 16 */
  PEPS_MIXED_BF16 = 3   /* reserved: tensor-core absorptions */
} peps_precision;

typedef struct {
  int Lx, Ly;          /* columns, rows; 2 <= Lx, Ly <= 64, N = Lx * Ly <= 4096 */
  int d;               /* local dimension, must be 2 */
  int D;               /* virtual bond dimension, 1 <= D <= 16 */
  int Dc;              /* boundary-MPS cut-off, 1 <= Dc <= 32, Dc * D <= 256 */
  double J1, J2;       /* nearest / next-nearest couplings (Sec. IV) */
  int prec;            /* peps_precision */
  double workspace_gb; /* device workspace budget for environments; 0 -> 24 GB */
} peps_params;

/* Creates a context: validates the parameters, copies A_host
 * ([N][2][D^4] FP64, padded as above) to the device in the context's
 * precision.  cuda_stream is a cudaStream_t (NULL = legacy default stream).
 * Fig. 1c / Eq. 1. */
peps_status peps_create(const peps_params* params, const double* A_host, void* cuda_stream, peps_ctx** out);

/* Frees the context and its device memory. */
peps_status peps_destroy(peps_ctx* ctx);

/* Replaces the site tensors (same shapes).  Eq. 1. */
peps_status peps_set_tensors(peps_ctx* ctx, const double* A_host);

/* One gradient-optimisation update of the site tensors (Sec. III):
 *   A(n+1) = A(n) - p * dt * sign(dE/dA),  p uniform in [0, 1) per element.
 * p is drawn on the device: SplitMix64's output function keyed by (seed,
 * step, element index e of [N][2][D^4]), h = mix(seed + G (1 + step)), then
 * h = mix(h + G (1 + e)), G = 0x9E3779B97F4A7C15, p = (h >> 11) * 2^-53.
 *   grad_dev  [N][2][D^4] FP64 device array, dE/dA (e.g. peps_gradient's grad).
 *   dt        step length (finite, >= 0).
 *   A_host    optional [N][2][D^4] FP64 host array, caller-owned: receives the
 *             updated tensors; NULL skips the copy.
 * The update runs in place on the context's FP64 copy of the tensors, on the
 * device; the FP32 and tensor-core copies are then rebuilt from it on the
 * device, so the context evaluates the updated tensors (as after
 * peps_set_tensors with them).  Entries past an open edge and entries with
 * zero derivative do not move.  Synchronises the context's stream.  Errors:
 * PEPS_EINVAL (null context or gradient, bad dt, a NaN or infinite entry in
 * grad_dev -- the tensors are then left unchanged -- or a serving worker
 * context), PEPS_ENOMEM / PEPS_ECUDA. */
peps_status peps_go_step(peps_ctx* ctx, const double* grad_dev, double dt, uint64_t seed, uint64_t step,
                         double* A_host);

/* ln|psi(S)| and sign psi(S) from the top-down boundary-MPS sweep (Fig. 1d).
 * S_dev [n][ceil(N/64)]; logabs_dev [n] FP64; sign_dev [n] int8 (+1, -1, 0);
 * status_dev [n] int32 or NULL. */
peps_status peps_amplitudes(peps_ctx* ctx, const uint64_t* S_dev, int n, double* logabs_dev, int8_t* sign_dev,
                            int32_t* status_dev);

/* E(S) per configuration (Sec. II local energy, Sec. IV Hamiltonian).
 * eloc_dev [n] FP64; status_dev [n] or NULL. */
peps_status peps_local_energy(peps_ctx* ctx, const uint64_t* S_dev, int n, double* eloc_dev, int32_t* status_dev);

/* Delta(S) = B/W (Sec. II) for the spin block selected by each s_i:
 * O_dev [n][N][D^4] in the context's precision (double for PEPS_FP64,
 * float otherwise), index order (l, r, u, d), zero at padded entries. */
peps_status peps_log_derivatives(peps_ctx* ctx, const uint64_t* S_dev, int n, void* O_dev);

/* All per-configuration outputs in one pass; any output may be NULL (work
 * not needed for the requested outputs is skipped). */
peps_status peps_evaluate(peps_ctx* ctx, const uint64_t* S_dev, int n, double* logabs_dev, int8_t* sign_dev,
                          double* eloc_dev, void* O_dev, int32_t* status_dev);

/* MC estimates over the n given configurations (plain sample means; the
 * configurations are taken as samples of W^2, Sec. II):
 *   energy per site <E>/N -> *energy_per_site_host (this call synchronises
 *   the stream), grad_dev [N][2][D^4] FP64 = 2(<Delta E> - <Delta><E>),
 *   cov_dev (optional) = grad / 2.  Optional per-configuration outputs
 *   logabs_dev, sign_dev, eloc_dev, status_dev may be NULL.  Configurations
 *   with a non-zero status are left out of the means.
 *   *n_used_host (optional) receives the number of configurations used. */
peps_status peps_gradient(peps_ctx* ctx, const uint64_t* S_dev, int n, double* energy_per_site_host, double* grad_dev,
                          double* cov_dev, double* logabs_dev, int8_t* sign_dev, double* eloc_dev,
                          int32_t* status_dev, int* n_used_host);

/* The sums behind peps_gradient's estimates, for reductions across batches
 * or ranks: the estimator of Sec. II is built from sums over configurations,
 * so the sums of disjoint batches add (one allreduce across GPUs) before
 * peps_gradient_finalize forms the means.  sums_dev is a device array of
 * peps_gradient_sums_len(ctx) = 4 + 2 N 2 D^4 doubles:
 *   [0] sum of E(S), [1] number of configurations used, [2] sum of E(S)^2,
 *   [3] zero, then sum of Delta [N][2][D^4] (zero in the block a
 *   configuration's spin does not select), then sum of E(S) Delta [N][2][D^4],
 * over the configurations with status 0.  accumulate = 0 overwrites the
 * sums, 1 adds to them.  Per-configuration outputs as in peps_gradient. */
peps_status peps_gradient_sums(peps_ctx* ctx, const uint64_t* S_dev, int n, double* sums_dev, int accumulate,
                               double* logabs_dev, int8_t* sign_dev, double* eloc_dev, int32_t* status_dev);
size_t peps_gradient_sums_len(const peps_ctx* ctx);

/* Energy and gradient from sums laid out as above (e.g. after adding the
 * sums of every rank): energy per site <E>/N, the sample variance of E/N
 * (var(E)/N^2, NaN below two configurations), grad_dev = 2(<Delta E> -
 * <Delta><E>), cov_dev = grad/2 (Sec. II).  Every output may be NULL.
 * Synchronises the context's stream. */
peps_status peps_gradient_finalize(peps_ctx* ctx, const double* sums_dev, double* energy_per_site_host,
                                   double* energy_var_host, double* grad_dev, double* cov_dev, int* n_used_host);

/* nsweeps Metropolis sweeps per configuration (chain), in place on S_dev.
 * A sweep visits the nearest-neighbour bonds in the order: horizontal
 * row-major, then vertical row-major; an antiparallel pair is exchanged with
 * probability min(1, (W(S')/W(S))^2) (sampling with weight W^2, Sec. II),
 * with W(S')/W(S) computed from the environments of the current S as in
 * peps_local_energy.  The uniform draw for (chain, sweep, bond) is
 * u = (h >> 11) * 2^-53 with h = SplitMix64 keyed by (seed, chain0 + index,
 * sweep0 + k, bond index); accepted_dev [n] int64 (optional) is incremented
 * by the number of accepted exchanges. */
peps_status peps_mc_sweep(peps_ctx* ctx, uint64_t* S_dev, int n, int nsweeps, uint64_t seed, uint64_t chain0,
                          uint64_t sweep0, int64_t* accepted_dev);

/* Sampled spin-spin correlations and the staggered magnetisation (Sec. IV).
 * For configurations drawn with weight W^2 the local value of S_i.S_j
 * (i != j) is S^z_i S^z_j + [s_i != s_j] W(S^ij) / (2 W(S)), S^ij with s_i and
 * s_j exchanged; the paper's M^2 is (1/n^2) sum_{p,q} eps_p eps_q <S_p.S_q>
 * over n central sites, eps = (-1)^(row + col) (k = (pi, pi)).  Reading of
 * the ratio for a pair i < j in rows r_i <= r_j: the configuration's upper
 * environment U_{r_i - 1} absorbs row r_i with s_i flipped and the rows
 * below it (zip-up truncation to Dc, Fig. 1d); in row r_j it meets the row
 * with s_j flipped and the lower environment L_{r_j + 1} in a single-row
 * sandwich, divided by the configuration's own single-row sandwich of row
 * r_j, with the difference of the per-row norms the two sweeps divided out.
 * Exact when nothing is truncated.  Cost per configuration: one partial
 * boundary sweep per central site.
 *   sites_host [nc]: distinct central sites (host); m2_dev [n] (optional):
 *   the local M^2 of each configuration (NaN where status != 0);
 *   corr_dev [nc][nc] (optional): the sums over the configurations with
 *   status 0 of the local S_p.S_q (3/4 on the diagonal; divide by their
 *   number for the estimates); status_dev [n] (optional) as peps_evaluate. */
peps_status peps_correlations(peps_ctx* ctx, const uint64_t* S_dev, int n, const int* sites_host, int nc,
                              double* m2_dev, double* corr_dev, int32_t* status_dev);

/* Truncation mode of the boundary MPS (Sec. II, Fig. 1d).  fit_sweeps = 0
 * (the default): zip-up with SVD truncation to Dc at every column.
 * fit_sweeps > 0: the variational-fit truncation, the boundary-MPS method by
 * variational compression: after the zip-up, fit_sweeps one-site ALS sweeps
 * (each from the zip-up's last column to the other end and back) maximise the
 * overlap of the new boundary MPS with the uncut row applied to the old one,
 * at the zip-up's bond dimensions; every column is set to its environment in
 * that overlap and re-orthonormalised by a QR or LQ (Householder), the
 * centre ends where the zip-up left it.  Applies to every boundary sweep of
 * the context (evaluations, gradient, Metropolis, correlations).  Results
 * differ from the zip-up's (a different truncation) and equal exact
 * contraction when nothing is cut.  fit_sweeps <= 64. */
peps_status peps_set_truncation(peps_ctx* ctx, int fit_sweeps);

/* Environment cache.  With on != 0 a context keeps, next to the boundary
 * environments in its workspace, a copy of the configurations they belong
 * to.  A later peps_evaluate, peps_gradient or peps_correlations call whose
 * batch fits in one chunk compares each configuration with the cached one on
 * the device, and where the bits are unchanged (same slot, same tensors,
 * same workspace) skips that configuration's boundary sweeps, keeping its
 * ln|psi|, sign and environments; a changed configuration (a new request, a
 * Metropolis move) is swept again.  So amplitudes, then E_loc, then Delta of
 * one batch sweep the boundary once, and so does an evaluation after a
 * Metropolis sweep for the chains that did not move.  Results are
 * bit-identical to calls without the cache.  The cache is reset by
 * peps_set_tensors, peps_go_step, a batch larger than one chunk, or a packed
 * launch that used the context. */
peps_status peps_set_env_cache(peps_ctx* ctx, int on);

/* ---- batching: graphs, tuning, packed launches ----
 * CUDA-graph replay.  With on != 0, peps_evaluate and peps_gradient capture
 * the device work of a call (every chunk's kernel launches, memsets and
 * copies, and the read-back of the energy into page-locked memory) into a
 * CUDA graph on the first call with a given signature (S_dev, n and the
 * output pointers), instantiate it, and replay it on later calls with the
 * same signature: the launch sequence is issued once per call instead of
 * kernel by kernel.  Up to 16 signatures are kept; all are dropped when the
 * context's workspace buffers move (a larger batch) and when graphs are
 * turned off.  Results are bit-identical to calls without graphs.  Needs a
 * context created on a non-default stream (PEPS_EINVAL otherwise).  While
 * capturing, per-kernel profiling events are not recorded. */
peps_status peps_set_graphs(peps_ctx* ctx, int on);
/* stats[3]: graphs cached, captures and replays since the context was created. */
peps_status peps_graph_stats(peps_ctx* ctx, long long* stats);

/* Autotuner.  Times full gradient passes (one untimed, one timed, CUDA
 * events on the context's stream) over the probe batch S_dev [n] for each
 * candidate, one setting after another, and keeps the fastest:
 *   - the two-row kernel: tensor cores (PEPS_MIXED_TF32, D = 8, Dc = 16),
 *     the fused shared-memory kernel (where one exists for (D, Dc)), or the
 *     generic one;
 *   - the single-row kernel: fused (where one exists) or generic;
 *   - the persistent grid of the boundary sweeps: the resident CTA count or
 *     half of it;
 *   - the workspace budget (configurations per chunk): the current one, x2,
 *     x4 (within 60% of device memory), tried only when the probe batch
 *     spans more than one chunk.
 * The variants compute the same quantities; FP32 results may differ in the
 * last bits between variants.  The choice is kept in the context and in a
 * process-wide table: contexts created later for the same (Lx, Ly, D, Dc,
 * precision, SM count) start with it.  report (optional, report_len bytes)
 * receives every trial's time and the choice.  Synchronises the stream. */
peps_status peps_autotune(peps_ctx* ctx, const uint64_t* S_dev, int n, char* report, size_t report_len);

/* The context's kernel settings: vals[0] two-row kernel (0 tensor cores,
 * 1 fused, 2 generic), vals[1] single-row kernel (0 fused, 1 generic),
 * vals[2] boundary-sweep CTAs, vals[3] configurations per chunk of the last
 * call; *workspace_gb the workspace budget. */
peps_status peps_tuned_config(peps_ctx* ctx, int* vals /* [4] */, double* workspace_gb);

/* Packed launches.  A packer evaluates requests of several models (contexts
 * of different lattices, D and Dc, all PEPS_FP64 or all of the FP32 family)
 * with the boundary sweeps of all requests in ONE persistent kernel launch:
 * work items are (request, configuration, sweep direction) numbered request
 * after request, each CTA finds its request by the item's index and lays its
 * scratch slot and shared memory out for that model.  The sandwich and
 * finalisation steps then run per request.  Everything runs on the packer's
 * stream (cudaStream_t, NULL = legacy default) using each context's
 * workspace, so the contexts must have no work in flight on their own
 * streams.  Per request i: S[i] [n[i]][ceil(N_i/64)], outputs as in
 * peps_evaluate (each array of pointers, or any of its entries, may be
 * NULL); a request must fit in one chunk of its context's workspace
 * (PEPS_EINVAL otherwise) and a context may appear once per call.  Results
 * are bit-identical to peps_evaluate on each context alone. */
typedef struct peps_packer peps_packer;
peps_status peps_packer_create(void* cuda_stream, peps_packer** out);
peps_status peps_packer_destroy(peps_packer* packer);
peps_status peps_packer_evaluate(peps_packer* packer, int nreq, peps_ctx* const* ctxs, const uint64_t* const* S_dev,
                                 const int* n, double* const* logabs_dev, int8_t* const* sign_dev,
                                 double* const* eloc_dev, void* const* O_dev, int32_t* const* status_dev);

/* Per-kernel timing of this context's launches: when enabled, CUDA events
 * are recorded on the context's stream around every kernel the library
 * launches.  peps_profile_read synchronises the stream and returns, per
 * kernel id (0 boundary sweeps, 1 single-row sandwiches, 2 two-row
 * sandwiches, 3 E_loc/status finalisation, 4 gradient sums, 5 energy sum,
 * 6 gradient finalisation, 7 Metropolis sweeps), the summed milliseconds
 * and the number of launches since the last reset; reset clears them. */
peps_status peps_profile_enable(peps_ctx* ctx, int on);
peps_status peps_profile_read(peps_ctx* ctx, double* ms /* [8] */, long long* launches /* [8] */, int reset);

/* Allocation-free amplitudes.  The paper has no counterpart to this call: it
 * exists for callers that cannot call cudaMalloc, such as code running inside
 * another runtime's memory arena (framework custom ops, plugins, engines) or
 * real-time code that must not allocate after start-up.  It computes what
 * peps_amplitudes computes (ln|psi| and sign from the top-down boundary-MPS
 * sweep) without a context and without allocating: the per-CTA scratch is a
 * file-scope static device array of 8 MiB that every GPU loading the
 * library holds until exit (a 16x16 D=8 Dc=16 FP32 slot takes 0.54 MB, so
 * 15 CTAs run at once; FP64 with Dc*D = 256 on 64 columns does not fit).
 *   params     lattice, D, Dc, prec (PEPS_FP64 or PEPS_FP32); J1, J2 unused.
 *   A_dev      device [N][2][D^4] site tensors in the precision of prec
 *              (double or float), padded as for peps_create.
 *   S_dev      device [n][ceil(N/64)] configurations.
 *   logabs_dev, sign_dev: device [n] outputs; status_dev: device [n] or NULL.
 *   cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * Lattices whose per-CTA scratch exceeds the static array are rejected with
 * PEPS_EINVAL and a message naming the sizes.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  Every
 * call shares the one array and leaves its contents behind (the kernel
 * writes everything before reading it), so calls that overlap on the GPU,
 * on any stream, race: serialise them. */
peps_status peps_amplitudes_static(const peps_params* params, const void* A_dev, const uint64_t* S_dev, int n,
                                   double* logabs_dev, int8_t* sign_dev, int32_t* status_dev, void* cuda_stream);

/* ---- simple-update initialiser (Sec. III, computational details) ----
 * Imaginary-time evolution exp(-dtau H) of the J1-J2 Heisenberg model by
 * first-order Trotter steps of two-site gates, each applied with the simple
 * update: the weights of the bonds around the pair are absorbed, a QR of each
 * site tensor isolates the bond (O(D^5)), the gate acts on the reduced
 * tensors, an SVD cuts the bond back to D and its D largest singular values
 * (normalised to unit 2-norm) become the bond's new weight.  A step applies
 * the horizontal bonds at even then odd columns, the vertical bonds at even
 * then odd rows, and with J2 != 0 each next-nearest pair (i, k) as
 * SWAP(i, j), gate(j, k), SWAP(i, j) through their shared neighbour j.  Each
 * group of bonds without a shared site is one launch, one CTA per bond, in
 * FP64.  The paper runs dtau = 0.01 until the relative change of the tensors
 * falls below 1e-6, then dtau = 0.001.
 *   State, caller-owned device arrays (FP64):
 *     Gam_dev [N][2][D^4]: Gamma_i[s][l][r][u][d], padded like A, zero past open edges;
 *     lam_dev [nbonds][D]: bond weights, bonds numbered horizontal (row-major)
 *                          then vertical (row-major), nbonds = Ly(Lx-1) + (Ly-1)Lx.
 *   peps_su_create: params' Lx, Ly, D, J1, J2 (Dc, prec unused); the handle owns
 *     the bond tables and per-CTA scratch (4 D^3 2D doubles per bond of a group).
 *   peps_su_evolve: nsteps Trotter steps with time step dtau (>= 0), in place;
 *     change_host (optional) receives max|A' - A| / max|A| over the last step,
 *     A the PEPS of peps_su_to_peps (synchronises the stream when given).
 *   peps_su_to_peps: A_dev [N][2][D^4] = Gamma_i times sqrt(lam) on each of its
 *     bonds, scaled to unit Frobenius norm per site (the tensors of Eq. 1 that
 *     peps_create takes).
 * Work is enqueued on the handle's stream; errors: PEPS_EINVAL (arguments),
 * PEPS_ENOMEM / PEPS_ECUDA. */
typedef struct peps_su peps_su;
peps_status peps_su_create(const peps_params* params, void* cuda_stream, peps_su** out);
peps_status peps_su_destroy(peps_su* su);
peps_status peps_su_evolve(peps_su* su, double* Gam_dev, double* lam_dev, double dtau, int nsteps, double* change_host);
peps_status peps_su_to_peps(peps_su* su, const double* Gam_dev, const double* lam_dev, double* A_dev);

/* ---- serving: continuous batching of evaluation requests ----
 * A server owns `nlanes` lanes (CUDA streams).  Each request asks for the
 * outputs of peps_evaluate for n configurations of one model (a context
 * created with peps_create); requests of different models, lattices and
 * sizes run concurrently on different lanes, each lane with its own worker
 * context (the model's tensors are shared, the workspace is private; each
 * lane's workspace budget is hbm_budget_gb / nlanes).  A queued request is
 * admitted when a lane is free and the HBM it needs fits under
 * hbm_budget_gb; smaller requests may pass one that does not fit yet.
 * Results are the same as peps_evaluate alone.  Inputs must be ready on the
 * device when submitted; outputs are valid once the request id is returned
 * by peps_server_poll.  The model contexts must outlive the server's use of
 * them.  Not thread-safe. */
typedef struct peps_server peps_server;
peps_status peps_server_create(int nlanes, double hbm_budget_gb, peps_server** out);
peps_status peps_server_destroy(peps_server* server);
peps_status peps_server_submit(peps_server* server, peps_ctx* model, const uint64_t* S_dev, int n,
                               double* logabs_dev, int8_t* sign_dev, double* eloc_dev, void* O_dev,
                               int32_t* status_dev, long long* id_out);
/* A chain request: the Markov chains' configurations S_dev (device, owned
 * by the caller, kept there between requests) first take nsweeps Metropolis
 * sweeps in place (peps_mc_sweep's keyed draws: seed, chain0, sweep0), then
 * are evaluated as by peps_server_submit.  Lane workers keep their boundary
 * environments (peps_set_env_cache) and a chain's request prefers the lane
 * that served the same S_dev last, so chains that did not move are not swept
 * again. */
peps_status peps_server_submit_chain(peps_server* server, peps_ctx* model, uint64_t* S_dev, int n, int nsweeps,
                                     uint64_t seed, uint64_t chain0, uint64_t sweep0, double* logabs_dev,
                                     int8_t* sign_dev, double* eloc_dev, void* O_dev, int32_t* status_dev,
                                     long long* id_out);
/* Packing: a free lane that admits a request of at most max_configs
 * configurations also takes up to max_requests - 1 further queued ones of
 * other models (same precision class, each within max_configs, all within
 * the HBM budget) and runs them as one packed launch (peps_packer_evaluate):
 * their boundary sweeps share one kernel.  max_configs = 0 (the default)
 * turns packing off.  Results equal the requests run alone. */
peps_status peps_server_set_packing(peps_server* server, int max_configs, int max_requests);
/* Admission order of queued requests.  0 (the default): first come first
 * served.  1: smallest expected run time less time waited first, where the
 * expected run time is the request's configurations times its model's
 * running average of milliseconds per configuration over finished launches
 * (0 before the model's first), so short requests pass long ones until the
 * long ones have waited about as long as they will run.  Results do not
 * depend on the order.  PEPS_EINVAL for another value. */
peps_status peps_server_set_policy(peps_server* server, int policy);
/* Retires finished requests and admits queued ones.  wait != 0 blocks until
 * at least one request finishes (or nothing is left).  Up to max finished ids
 * and their latencies (ms, submission to completion) are written; *ndone is
 * their number.  A request that could not be launched (its workspace does not
 * fit in device memory, or a launch failed) is returned with latency -1 and
 * its outputs are not valid; peps_last_error says why. */
peps_status peps_server_poll(peps_server* server, int wait, long long* ids, double* latency_ms, int max, int* ndone);
/* stats[8]: submitted, completed, queued, running, p50 and p99 latency (ms),
 * HBM in use and peak HBM (GB) of the lanes' workspaces. */
peps_status peps_server_stats(peps_server* server, double* stats);

/* Measured throughput of the pipes the kernels run on, for roofline
 * denominators: out[0] FP32 fused multiply-add on the SIMT pipe, out[1] FP64
 * likewise, out[2] dense TF32 tcgen05.mma (FP32 accumulation), in TFLOP/s.
 * Long independent chains on every SM, timed with CUDA events; synchronises
 * the device.  PEPS_ETIMEOUT if the tensor-core probe's bounded wait gave up.
 * The paper has no counterpart. */
peps_status peps_measure_peaks(double* out /* [3] */);
/* Measured rate of dense TF32 tcgen05.mma instructions of one shape, M = 128,
 * N = n (16, 32, 64, 128 or 256), K = 8, both operands in shared memory,
 * chained into one TMEM accumulator on every SM: *tflops in TFLOP/s.  The
 * tensor-core kernels issue N = 64 and N = 16 instructions, whose rate can be
 * below the N = 256 figure of peps_measure_peaks.  Synchronises the device;
 * PEPS_EINVAL for another n, PEPS_ETIMEOUT if the bounded wait gave up. */
peps_status peps_measure_tf32_mma_shape(int n, double* tflops);

/* Waits for the context's stream. */
peps_status peps_synchronize(peps_ctx* ctx);

/* Human-readable name of a status code. */
const char* peps_status_str(peps_status s);

/* Last error message of the calling thread (empty if none). */
const char* peps_last_error(void);

/* Host-only check of the contraction programs, no GPU involved: runs the
 * same index descriptors the kernels use on host FP64 buffers.
 *   op 0 single-row left transfer   in: F, Mu, T, Md        out: F'
 *   op 1 single-row right transfer  in: G, Mu, T, Md        out: G'
 *   op 2 site environment B         in: F, Mu, Md, G        out: B
 *   op 3 two-row left transfer      in: E, Mu, T1, T2, Md   out: E'
 *   op 4 two-row right transfer     in: H, Mu, T1, T2, Md   out: H'
 * Tensors are padded as documented in contract.cuh. */
peps_status peps_debug_host_op(int op, int D, int Dc, const double* in0, const double* in1, const double* in2,
                               const double* in3, const double* in4, double* out);

/* Host-only check of one zip-up column (Fig. 1d): dims = {k, a, b, i, l, r, o,
 * sl, sr, si, so}; lr = 1 left-to-right (carry C [k][a][l], output X
 * [(k,o)][(b,r)]), lr = 0 right-to-left (carry C [b][r][k], output X
 * [(o,k)][(a,l)]).  M padded [Dc][D][Dc], T padded D^4 read with strides. */
peps_status peps_debug_host_zip(int lr, int D, int Dc, const int* dims, const double* C, const double* M,
                                const double* T, double* X);

#ifdef __cplusplus
}
#endif

#endif /* PEPS_H */
