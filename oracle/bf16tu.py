"""Oracle of the BF16 trailing-update block LU (precision SAP_FP32_BF16TU).

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the tests may use it;
the library never imports it and it shares no code with the CUDA path.

What it computes: the block LU of Sec. 3.1 (Doolittle, no pivoting, boosted
pivots as in Sec. 2.2), organised in panels of ``nb`` columns as a blocked
right-looking elimination: for each panel the panel columns are eliminated
exactly (FP64), then U12 = L11^{-1} A12, then the trailing matrix is updated by
A22 -= L21 U12 with both operands rounded to bfloat16 (round to nearest, ties
to even) and the products summed in FP64.  With the rounding replaced by the
identity this is exactly the plain block LU, which the pins check.  The
factors are returned in the oracle's dense-band layout (n, 2K+1), element
(r, c) at [r, c - r + K].
"""
from __future__ import annotations

import numpy as np


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Nearest bfloat16 value (8 significant bits), ties to the even significand.

    From the definition: x is first rounded to binary32; of the two binary32
    values with zero low 16 bits that bracket it (truncation toward zero and
    the next one away from zero) the nearer is taken, the one with an even
    bit 16 on a tie.  Finite inputs only."""
    x32 = np.asarray(x, dtype=np.float32)
    u = x32.view(np.uint32).astype(np.uint64)
    low = u & np.uint64(0xFFFF)
    down = u - low                                  # |value| truncated
    up = down + np.uint64(0x10000)                  # next magnitude
    half = np.uint64(0x8000)
    even_down = ((down >> np.uint64(16)) & np.uint64(1)) == 0
    take_up = (low > half) | ((low == half) & ~even_down)
    r = np.where(take_up, up, down).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def dense_block(band: np.ndarray, N: int, K: int, s: int, n: int) -> np.ndarray:
    """Rows/columns [s, s+n) of the banded A as a dense n x n array (band layout
    band[(K + i - j) N + j] = a_ij)."""
    b = np.asarray(band, dtype=np.float64).reshape(2 * K + 1, N)
    A = np.zeros((n, n))
    for r in range(n):
        for c in range(max(0, r - K), min(n, r + K + 1)):
            A[r, c] = b[K + r - c, s + c]
    return A


def block_lu_panels(A: np.ndarray, K: int, tau: float, nb: int = 16, rnd=bf16_round):
    """Blocked LU of the n x n block A (band half-width K), returns the dense
    packed factors (unit L below the diagonal, U on and above) and the number
    of boosted pivots."""
    A = np.array(A, dtype=np.float64)
    n = A.shape[0]
    boosted = 0
    for k0 in range(0, n, nb):
        k1 = min(n, k0 + nb)
        hi = min(n, k1 + K)                  # rows/columns the panel can reach
        # the panel columns k0 .. k1-1, exactly, over rows k0 .. hi-1
        for k in range(k0, k1):
            p = A[k, k]
            if abs(p) < tau:
                p = tau if p >= 0 else -tau
                boosted += 1
            A[k, k] = p
            A[k + 1:hi, k] /= p
            A[k + 1:hi, k + 1:k1] -= np.outer(A[k + 1:hi, k], A[k, k + 1:k1])
        if k1 >= n:
            break
        # U12 = L11^{-1} A12 (unit lower L11), columns k1 .. hi-1
        for k in range(k0, k1):
            A[k + 1:k1, k1:hi] -= np.outer(A[k + 1:k1, k], A[k, k1:hi])
        # trailing update with rounded operands
        A[k1:hi, k1:hi] -= rnd(A[k1:hi, k0:k1]) @ rnd(A[k0:k1, k1:hi])
    return A, boosted


def to_dense_band(F: np.ndarray, K: int) -> np.ndarray:
    n = F.shape[0]
    out = np.zeros((n, 2 * K + 1))
    for r in range(n):
        for c in range(max(0, r - K), min(n, r + K + 1)):
            out[r, c - r + K] = F[r, c]
    return out


def block_factors(band: np.ndarray, N: int, K: int, s: int, n: int, tau: float, rnd=bf16_round, nb: int = 16):
    """Factors of the block [s, s+n) in the dense-band layout, and the boosts."""
    F, boosted = block_lu_panels(dense_block(band, N, K, s, n), K, tau, nb, rnd)
    return to_dense_band(F, K), boosted
