"""Seeded synthetic inputs shared by the CUDA path, its tests and the FP64 oracle.

This module holds no arithmetic of the PEPS method itself: it only draws
random numbers and packs them into the layouts both sides read.

* Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
  pseudorandom number generators", OOPSLA 2014), used as a counter-based
  generator: every draw is the SplitMix64 output function applied to a key
  built from (seed, counters...).  Draws are therefore independent of the
  order in which they are made and fully vectorisable.
* Gaussian entries use the Box-Muller transform on two keyed uniforms.
* Site tensors follow Eq. 1: A_i(l, r, u, d, s) with virtual bonds of
  dimension D and open edges of dimension one.  They are stored padded to
  D^4 per (site, spin) in the order [site][s][l][r][u][d]; entries whose
  index exceeds the true edge dimension are zero.
* Spin configurations S are bit-packed: bit i of word i // 64 is s_i,
  site i = row * Lx + col, s = 0 meaning S^z = +1/2.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Per-workload seeds: base + workload number (1..5).
SEED_BASE = 1611094670


def splitmix64_mix(z):
    """SplitMix64 output function (finaliser) on uint64 arrays."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def keyed_u64(seed, *counters):
    """One SplitMix64 draw per broadcast element of the counters.

    h = mix(seed + GOLDEN * (1 + c0)), then h = mix(h + GOLDEN * (1 + c_k)) for
    every further counter.  Counters broadcast like numpy arrays.
    """
    h = np.asarray(np.uint64(seed))
    with np.errstate(over="ignore"):
        for c in counters:
            c = np.asarray(c).astype(np.uint64)
            h = splitmix64_mix(h + GOLDEN * (np.uint64(1) + c))
    return h


def keyed_uniform(seed, *counters):
    """Uniform double in [0, 1): top 53 bits of a keyed draw times 2^-53."""
    return (keyed_u64(seed, *counters) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def keyed_normal(seed, *counters):
    """Standard normal by Box-Muller from two keyed uniforms (extra counter 0 / 1)."""
    u1 = 1.0 - keyed_uniform(seed, *counters, 0)  # in (0, 1]
    u2 = keyed_uniform(seed, *counters, 1)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def true_dims(Ly: int, Lx: int, D: int) -> np.ndarray:
    """[N, 4] true bond dimensions (l, r, u, d) per site: D inside, 1 on open edges."""
    dims = np.full((Ly * Lx, 4), D, dtype=np.int64)
    for r in range(Ly):
        for c in range(Lx):
            i = r * Lx + c
            if c == 0:
                dims[i, 0] = 1
            if c == Lx - 1:
                dims[i, 1] = 1
            if r == 0:
                dims[i, 2] = 1
            if r == Ly - 1:
                dims[i, 3] = 1
    return dims


def edge_mask(Ly: int, Lx: int, D: int) -> np.ndarray:
    """[N, 1, D, D, D, D] boolean mask of the entries inside the true dimensions."""
    dims = true_dims(Ly, Lx, D)
    idx = np.arange(D)
    m = ((idx[None, :, None, None, None] < dims[:, 0, None, None, None, None])
         & (idx[None, None, :, None, None] < dims[:, 1, None, None, None, None])
         & (idx[None, None, None, :, None] < dims[:, 2, None, None, None, None])
         & (idx[None, None, None, None, :] < dims[:, 3, None, None, None, None]))
    return m[:, None]


def make_tensors(Ly: int, Lx: int, D: int, seed: int, d: int = 2,
                 bias_zero_index: bool = False) -> np.ndarray:
    """Padded site tensors A[N][d][D][D][D][D] (float64).

    Entries are i.i.d. N(0, 1), keyed by (site, s, flat index) so the draw does
    not depend on D's padding order.  With ``bias_zero_index`` 1.0 is added to
    A_i[s=0][0][0][0][0] (the all-zero-index element).  Each site is then
    scaled to unit Frobenius norm over both spin components and its true
    dimensions; padded entries are zero.
    """
    N = Ly * Lx
    site = np.arange(N)[:, None, None]
    s = np.arange(d)[None, :, None]
    flat = np.arange(D ** 4)[None, None, :]
    A = keyed_normal(seed, 0, site, s, flat).reshape(N, d, D, D, D, D)
    if bias_zero_index:
        A[:, 0, 0, 0, 0, 0] += 1.0
    A = A * edge_mask(Ly, Lx, D)
    norms = np.sqrt((A.reshape(N, -1) ** 2).sum(axis=1))
    return A / norms[:, None, None, None, None, None]


def near_product_tensors(Ly: int, Lx: int, D: int, seed: int, d: int = 2, eta: float = 1.0) -> np.ndarray:
    """Padded site tensors [N][d][D][D][D][D] (float64) near a product state.

    A_i[s] = phi_i(s) on the all-zero bond index plus i.i.d. N(0, 1) noise
    scaled so that its expected Frobenius norm is ``eta`` times that of the
    product part; phi_i = (cos t_i, sin t_i) with t_i keyed uniform in
    [pi/8, 3pi/8].  Each site is then scaled to unit Frobenius norm over its
    true dimensions.  Such tensors have decaying bond spectra, as optimised
    ground-state PEPS do, so truncation to Dc is well conditioned; i.i.d.
    tensors at D = 8, Dc = 16 are not (FP32-sized perturbations move the FP64
    ln|psi| by O(1)).  Entries are keyed by (site, s, flat index).
    """
    N = Ly * Lx
    site = np.arange(N)[:, None, None]
    s = np.arange(d)[None, :, None]
    flat = np.arange(D ** 4)[None, None, :]
    eps = eta / np.sqrt(d * D ** 4)
    A = eps * keyed_normal(seed, 0, site, s, flat).reshape(N, d, D, D, D, D)
    t = np.pi / 8 + np.pi / 4 * keyed_uniform(seed, 2, np.arange(N))
    A[:, 0, 0, 0, 0, 0] += np.cos(t)
    A[:, 1, 0, 0, 0, 0] += np.sin(t)
    A = A * edge_mask(Ly, Lx, D)
    norms = np.sqrt((A.reshape(N, -1) ** 2).sum(axis=1))
    return A / norms[:, None, None, None, None, None]


def n_words(N: int) -> int:
    return (N + 63) // 64


def pack_spins(spins: np.ndarray) -> np.ndarray:
    """[n, N] array of 0/1 -> [n, ceil(N/64)] uint64 bit-packed configurations."""
    spins = np.asarray(spins, dtype=np.uint64)
    n, N = spins.shape
    out = np.zeros((n, n_words(N)), dtype=np.uint64)
    for i in range(N):
        out[:, i // 64] |= spins[:, i] << np.uint64(i % 64)
    return out


def unpack_spins(packed: np.ndarray, N: int) -> np.ndarray:
    """[n, ceil(N/64)] uint64 -> [n, N] uint8 spins."""
    packed = np.asarray(packed, dtype=np.uint64)
    out = np.zeros((packed.shape[0], N), dtype=np.uint8)
    for i in range(N):
        out[:, i] = (packed[:, i // 64] >> np.uint64(i % 64)) & np.uint64(1)
    return out


def random_sz0(n: int, N: int, seed: int, first: int = 0) -> np.ndarray:
    """n uniformly random S^z = 0 configurations as [n, N] uint8 spins.

    Each configuration draws one keyed uniform per site; the N/2 sites with
    the smallest draws carry s = 1.  This is a uniformly random permutation
    of N/2 ones and N/2 zeros.  ``first`` offsets the configuration counter,
    so chunks of a large batch are reproducible on their own.
    """
    if N % 2:
        raise ValueError("S^z = 0 needs an even number of sites")
    cfg = np.arange(first, first + n)[:, None]
    site = np.arange(N)[None, :]
    keys = keyed_u64(seed, 1, cfg, site)
    order = np.argsort(keys, axis=1, kind="stable")
    spins = np.zeros((n, N), dtype=np.uint8)
    np.put_along_axis(spins, order[:, : N // 2], 1, axis=1)
    return spins


# ---------------------------------------------------------------- workloads
# The synthetic workloads, shaped like the paper's lattices (square lattices
# up to 16x16, D up to 10, Dc = 2D, J1 = 1, J2/J1 in {0, 0.5}).  All draw
# their configurations uniformly in the S^z = 0 sector; Metropolis draws
# (peps_mc_sweep) would change which configurations are evaluated, not the
# work per configuration.
WORKLOADS = {
    "4x4_D2_Dc4": dict(L=4, D=2, Dc=4, J2=0.5, n=64, bias=False, cfg=1,
                       sampling="uniform"),
    "8x8_D4_Dc8": dict(L=8, D=4, Dc=8, J2=0.5, n=4096, bias=True, cfg=2,
                       sampling="uniform"),
    "10x10_D6_Dc12": dict(L=10, D=6, Dc=12, J2=0.5, n=8192, bias=False, cfg=3,
                          sampling="uniform"),
    "16x16_D8_Dc16": dict(L=16, D=8, Dc=16, J2=0.5, n=16384, bias=False, cfg=4,
                          sampling="uniform"),
    "16x16_D10_Dc20": dict(L=16, D=10, Dc=20, J2=0.5, n=16384, bias=False, cfg=4,
                           sampling="uniform"),
    # the same shapes with near-product tensors: for accuracy checks at full size
    "16x16_D8_Dc16_np": dict(L=16, D=8, Dc=16, J2=0.5, n=16384, bias=False, cfg=5,
                             sampling="uniform", tensors="near_product"),
    "16x16_D10_Dc20_np": dict(L=16, D=10, Dc=20, J2=0.5, n=16384, bias=False, cfg=6,
                              sampling="uniform", tensors="near_product"),
}


def workload_inputs(name: str, n: int | None = None, first: int = 0):
    """(A, spins) for a named workload; ``n`` overrides the batch size."""
    w = WORKLOADS[name]
    seed = SEED_BASE + w["cfg"]
    if w.get("tensors") == "near_product":
        A = near_product_tensors(w["L"], w["L"], w["D"], seed)
    else:
        A = make_tensors(w["L"], w["L"], w["D"], seed, bias_zero_index=w["bias"])
    spins = random_sz0(w["n"] if n is None else n, w["L"] * w["L"], seed, first)
    return A, spins
