"""Seeded synthetic inputs for the dense-banded SaP solver.

This module is shared by the CPU oracle tests, the GPU tests and the benchmark.
It holds *no* arithmetic of the method (no factorisation, no spikes, no
matrix-vector product, no Krylov step): it only draws matrices and vectors.
The right-hand side b = A x_true is formed by whichever side consumes the
inputs (the oracle's SpMV in the tests, the library's SpMV in the benchmark).

Random numbers come from one counter-based generator, value = f(seed, stream,
index): the SplitMix64 output function (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) applied to a 64-bit counter built
from the three integers.  The top 53 bits give a double in [0, 1), mapped to
U(-1, 1).  Streams: 0 for the band, 1 for x_true, 2 for the adjoint seed
vector (g-bar / loss weights w).

Band storage is the "tall and thin" layout of Section 3.1 (matrix storage):
an N x (2K+1) array stored column-major, with the diagonal in column K, so
that a_ij sits at band[(K + i - j) * N + j] (0-based).  Entries whose row
index i falls outside [0, N) are padding and are set to 0 here.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "uniform", "dense_banded", "dense_banded_spd", "x_true", "adjoint_seed", "convection_diffusion",
    "batch_specs", "CONFIG_SEED_BASE", "config_seed", "BandedSystem",
]

CONFIG_SEED_BASE = 1509079190

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def config_seed(c: int) -> int:
    """Seed of workload configuration c (1-based)."""
    return CONFIG_SEED_BASE + int(c)


def _splitmix64(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def _counter(seed: int, stream: int, index: np.ndarray) -> np.ndarray:
    """64-bit counter: golden-ratio-spaced key of (seed, stream) plus index."""
    with np.errstate(over="ignore"):
        key = _splitmix64(np.array([(seed & 0xFFFFFFFF) | ((stream & 0xFFFF) << 32)],
                                   dtype=np.uint64))[0]
        return key + index.astype(np.uint64) * _GOLDEN


def uniform(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n draws of U(-1, 1) (53-bit mantissas) at counters offset..offset+n-1."""
    idx = np.arange(offset, offset + n, dtype=np.uint64)
    bits = _splitmix64(_counter(seed, stream, idx)) >> np.uint64(11)
    u01 = bits.astype(np.float64) * (1.0 / 9007199254740992.0)  # 2^-53
    return 2.0 * u01 - 1.0


@dataclass
class BandedSystem:
    """A banded system in band storage plus its exact solution."""
    band: np.ndarray      # float64, shape ((2K+1) * N,), band[(K+i-j)*N + j] = a_ij
    N: int
    K: int
    x_true: np.ndarray    # float64, shape (N,)
    name: str = ""


def _valid_mask(N: int, K: int) -> np.ndarray:
    """mask[c, j] is True where row i = j + c - K lies in [0, N)."""
    c = np.arange(2 * K + 1)[:, None]
    j = np.arange(N)[None, :]
    i = j + c - K
    return (i >= 0) & (i < N)


def dense_banded(N: int, K: int, d: float, seed: int) -> np.ndarray:
    """Random dense band: off-diagonal in-band a_ij ~ U(-1, 1) and
    a_ii = d * sum_{j != i} |a_ij| (degree of diagonal dominance d, Eq. (2.6)
    of Section 2.1).  Returns the band as a flat float64 array of (2K+1)*N."""
    if K < 1 or N < 1:
        raise ValueError("need N >= 1 and K >= 1")
    W = 2 * K + 1
    band = uniform(seed, 0, W * N).reshape(W, N)
    band[~_valid_mask(N, K)] = 0.0
    band[K, :] = 0.0
    # row abs-sums: entry band[c, j] belongs to row i = j + c - K
    rowsum = np.zeros(N)
    for c in range(W):
        if c == K:
            continue
        lo = max(0, K - c)
        hi = min(N, N + K - c)
        rowsum[lo + c - K: hi + c - K] += np.abs(band[c, lo:hi])
    band[K, :] = d * rowsum
    return band.reshape(-1)


def dense_banded_spd(N: int, K: int, d: float, seed: int) -> np.ndarray:
    """Random symmetric dense band: the strictly lower in-band entries
    a_ij (i > j) ~ U(-1, 1), mirrored a_ji = a_ij, and a_ii = d * sum_{j != i}
    |a_ij|.  With d > 1 the matrix is strictly diagonally dominant with a
    positive diagonal, hence symmetric positive definite (Gershgorin), the case
    in which the outer iteration is a conjugate gradient method (Section 3).
    Returns the band as a flat float64 array of (2K+1)*N."""
    if K < 1 or N < 1:
        raise ValueError("need N >= 1 and K >= 1")
    W = 2 * K + 1
    band = uniform(seed, 0, W * N).reshape(W, N)
    band[~_valid_mask(N, K)] = 0.0
    band[: K + 1, :] = 0.0
    # a_ij with i > j sits at band[c, j], c = K + i - j > K; its mirror a_ji at
    # band[2K - c, i], i = j + c - K
    for c in range(K + 1, W):
        lo, hi = 0, N - (c - K)
        band[W - 1 - c, lo + c - K: hi + c - K] = band[c, lo:hi]
    rowsum = np.zeros(N)
    for c in range(W):
        if c == K:
            continue
        lo = max(0, K - c)
        hi = min(N, N + K - c)
        rowsum[lo + c - K: hi + c - K] += np.abs(band[c, lo:hi])
    band[K, :] = d * rowsum
    return band.reshape(-1)


def x_true(N: int, seed: int) -> np.ndarray:
    """Exact solution x_true ~ U(-1, 1) (stream 1)."""
    return uniform(seed, 1, N)


def adjoint_seed(N: int, seed: int) -> np.ndarray:
    """Adjoint right-hand side g-bar / loss weights w ~ U(-1, 1) (stream 2)."""
    return uniform(seed, 2, N)


def convection_diffusion(nx: int = 400, ny: int = 250, peclet: float = 10.0,
                         seed: int = CONFIG_SEED_BASE + 4,
                         angle_deg: float = 30.0) -> tuple[np.ndarray, int, int]:
    """Nonsymmetric 2-D convection-diffusion operator, 5-point stencil, first-order
    upwind convection, on an nx x ny grid of unit cells.  Unknowns are ordered
    lexicographically with the ny-index fastest, so K = ny.

    Recipe: per-cell diffusivity kappa_c ~ U(0.5, 2) (stream 0); face
    diffusivity = harmonic mean of the two cells (the cell's own value on a
    boundary face); constant velocity v = Pe * (cos a, sin a) with
    Pe = |v| h / kappa_ref, h = kappa_ref = 1; homogeneous Dirichlet data
    (off-grid neighbours dropped).  Diagonal = sum of face diffusivities plus
    outflow fluxes, giving a weakly diagonally dominant M-matrix.
    Returns (band, N, K)."""
    N = nx * ny
    K = ny
    W = 2 * K + 1
    u = uniform(seed, 0, N)
    kap = 0.5 + 1.5 * (u + 1.0) * 0.5
    kap = kap.reshape(nx, ny)
    vx = peclet * math.cos(math.radians(angle_deg))
    vy = peclet * math.sin(math.radians(angle_deg))
    band = np.zeros((W, N))
    diag = np.zeros((nx, ny))
    idx = np.arange(N).reshape(nx, ny)

    def harm(a, b):
        return 2.0 * a * b / (a + b)

    # faces: (dx, dy, normal velocity)
    for dx, dy, vn in ((1, 0, vx), (-1, 0, -vx), (0, 1, vy), (0, -1, -vy)):
        xs = np.arange(nx)[:, None] + dx
        ys = np.arange(ny)[None, :] + dy
        inside = (xs >= 0) & (xs < nx) & (ys >= 0) & (ys < ny)
        inside = np.broadcast_to(inside, (nx, ny))
        xs_c = np.clip(np.broadcast_to(xs, (nx, ny)), 0, nx - 1)
        ys_c = np.clip(np.broadcast_to(ys, (nx, ny)), 0, ny - 1)
        knb = kap[xs_c, ys_c]
        kf = np.where(inside, harm(kap, knb), kap)
        diag += kf + max(vn, 0.0)
        off = -kf + min(vn, 0.0)        # inflow adds -|v.n| to the neighbour column
        rows = idx[inside]
        cols = idx[xs_c, ys_c][inside]
        c = K + rows - cols
        band[c, cols] = off[inside]
    band[K, :] = diag.reshape(-1)
    return band.reshape(-1), N, K


def batch_specs(n_systems: int = 64, seed: int = CONFIG_SEED_BASE + 5,
                n_lo: int = 10000, n_hi: int = 100000, k_lo: int = 8, k_hi: int = 64):
    """Sizes (N_s, K_s) and seeds of a batch of banded systems with
    N ~ U{n_lo..n_hi} and K ~ U{k_lo..k_hi}; system s uses seed base+1000+s."""
    uN = uniform(seed, 3, n_systems)
    uK = uniform(seed, 4, n_systems)
    Ns = n_lo + np.floor((uN + 1.0) * 0.5 * (n_hi - n_lo + 1)).astype(np.int64)
    Ks = k_lo + np.floor((uK + 1.0) * 0.5 * (k_hi - k_lo + 1)).astype(np.int64)
    Ns = np.minimum(Ns, n_hi)
    Ks = np.minimum(Ks, k_hi)
    seeds = [seed + 1000 + s for s in range(n_systems)]
    return [(int(n), int(k), int(sd)) for n, k, sd in zip(Ns, Ks, seeds)]


@dataclass
class SparseSystem:
    """A sparse system in CSR form (rows sorted by column) and the hidden
    structure it was made from: row i of the matrix is row rowsrc[i] of a
    banded matrix M0 (half-bandwidth K0, diagonally dominant, sparse within
    the band), renumbered by the symmetric permutation sym (M0 index k is
    index sym[k] here)."""
    n: int
    rowptr: np.ndarray    # int64, n + 1
    col: np.ndarray       # int32, nnz
    val: np.ndarray       # float64, nnz
    K0: int
    rowsrc: np.ndarray    # int64, n: M0 row of row i (before the renumbering)
    sym: np.ndarray       # int64, n


def _perm_from(seed: int, stream: int, n: int) -> np.ndarray:
    """A permutation of 0..n-1 from n counter-based draws (argsort of U(-1,1))."""
    return np.argsort(uniform(seed, stream, n), kind="stable").astype(np.int64)


def sparse_scrambled(n: int, K0: int, fill: float, d: float, seed: int) -> SparseSystem:
    """Synthetic sparse matrix of the kind the sparse front end (Sec. 2.2) is
    for: M0 banded with half-bandwidth K0, each in-band off-diagonal present
    with probability `fill` (value U(-1, 1)), its diagonal d times the row's
    off-diagonal abs-sum plus 0.01 (every row has a nonzero diagonal; for
    d < 1 off-diagonal entries can outweigh it, for d >= 1 it is the row's
    largest entry);
    then its rows shuffled (the heavy entries leave the diagonal, for the
    matching to restore) and all indices renumbered by a random symmetric
    permutation (the band hidden, for the bandwidth reduction to recover):
    A[r, sym[k]] = M0[rowsrc[r], k]."""
    W = 2 * K0 + 1
    keep = uniform(seed, 10, W * n).reshape(W, n)
    vals = uniform(seed, 11, W * n).reshape(W, n)
    rows, cols, vs = [], [], []
    absum = np.zeros(n)
    for c in range(W):
        off = c - K0                       # column j = i + off
        if off == 0:
            continue
        i = np.arange(max(0, -off), min(n, n - off))
        m = keep[c, i] * 0.5 + 0.5 < fill
        i = i[m]
        rows.append(i)
        cols.append(i + off)
        vs.append(vals[c, i])
        np.add.at(absum, i, np.abs(vals[c, i]))
    rows.append(np.arange(n))
    cols.append(np.arange(n))
    sgn = np.where(uniform(seed, 12, n) < 0, -1.0, 1.0)
    vs.append(sgn * (d * absum + 0.01))
    r0 = np.concatenate(rows)
    c0 = np.concatenate(cols)
    v0 = np.concatenate(vs)
    rowshuf = _perm_from(seed, 13, n)      # row i of the shuffled matrix is M0 row rowshuf[i]
    pos = np.empty(n, dtype=np.int64)
    pos[rowshuf] = np.arange(n)            # M0 row k lands at shuffled row pos[k]
    sym = _perm_from(seed, 14, n)          # index k -> sym[k]
    ri = sym[pos[r0]]
    ci = sym[c0]
    order = np.lexsort((ci, ri))
    ri, ci, vv = ri[order], ci[order], v0[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, ri + 1, 1)
    rowptr = np.cumsum(rowptr)
    rowsrc = np.empty(n, dtype=np.int64)
    rowsrc[sym] = rowshuf                  # final row sym[i] holds M0 row rowshuf[i]
    return SparseSystem(n, rowptr, ci.astype(np.int32), vv, K0, rowsrc, sym)


@dataclass
class BlockScrambled:
    """A banded matrix (half-bandwidth K) whose diagonal blocks [off[i],
    off[i+1]) are narrow bands in hidden numberings: block entry (a, b) is
    nonzero iff |hid[a] - hid[b]| <= k0[i] (hid: local index -> hidden one,
    a permutation inside windows of `window` indices), with the full K x K
    coupling corners between neighbouring blocks."""
    band: np.ndarray      # float64, (2K+1) N
    N: int
    K: int
    off: np.ndarray       # int64, P + 1 (given)
    k0: np.ndarray        # int64, P: hidden half-bandwidth of each block
    hid: np.ndarray       # int64, N: hidden local index of each local index
    window: int


def block_scrambled(N: int, K: int, off, d: float, seed: int, k0_lo: float = 0.4) -> BlockScrambled:
    """Synthetic input of the third-stage reordering (Sec. 2.2): after the
    DB-CM reorderings the band (half-bandwidth K) is sparse inside, and each
    diagonal block reordered on its own has a bandwidth of its own.  Values
    as in dense_banded (same seed and stream 0; diagonal d times the row's
    off-diagonal abs-sum, couplings included); the pattern of block i is a
    dense band of half-bandwidth k0_i <= w (k0_i = round(w u), u ~ U(k0_lo, 1),
    stream 15) seen through a random permutation inside consecutive windows of
    w = (K + 1) // 2 indices (stream 16): two indices within k0_i of each other
    in the hidden numbering are at most 2w - 1 <= K apart, so every entry lies
    in the band.  `off` is the block partition (P + 1 offsets)."""
    off = np.asarray(off, dtype=np.int64)
    P = len(off) - 1
    w = (K + 1) // 2
    if w < 1:
        raise ValueError("need K >= 1")
    W = 2 * K + 1
    band = uniform(seed, 0, W * N).reshape(W, N)
    band[~_valid_mask(N, K)] = 0.0
    band[K, :] = 0.0
    u = uniform(seed, 15, P) * 0.5 + 0.5
    k0 = np.maximum(1, np.rint(w * (k0_lo + (1.0 - k0_lo) * u))).astype(np.int64)
    k0 = np.minimum(k0, w)
    draws = uniform(seed, 16, N)
    hid = np.empty(N, dtype=np.int64)
    blk = np.empty(N, dtype=np.int64)
    for i in range(P):
        s, e = int(off[i]), int(off[i + 1])
        blk[s:e] = i
        for a0 in range(s, e, w):
            a1 = min(e, a0 + w)
            hid[a0:a1] = (a0 - s) + np.argsort(draws[a0:a1], kind="stable")
    j = np.arange(N)
    for c in range(W):
        if c == K:
            continue
        i = j + c - K
        ok = (i >= 0) & (i < N)
        ii, jj = i[ok], j[ok]
        same = blk[ii] == blk[jj]
        far = np.abs(hid[ii] - hid[jj]) > k0[blk[jj]]
        row = band[c]
        row[jj[same & far]] = 0.0
    rowsum = np.zeros(N)
    for c in range(W):
        if c == K:
            continue
        lo = max(0, K - c)
        hi = min(N, N + K - c)
        rowsum[lo + c - K: hi + c - K] += np.abs(band[c, lo:hi])
    band[K, :] = d * rowsum
    return BlockScrambled(band.reshape(-1), N, K, off, k0, hid, w)
