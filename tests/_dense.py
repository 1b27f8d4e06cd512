"""Dense helpers for tests (band <-> dense conversion, written from the
storage definition a_ij = band[(K + i - j) * N + j])."""
import numpy as np


def band_to_dense(band, N, K):
    A = np.zeros((N, N))
    b = np.asarray(band).reshape(2 * K + 1, N)
    for c in range(2 * K + 1):
        j = np.arange(N)
        i = j + c - K
        m = (i >= 0) & (i < N)
        A[i[m], j[m]] = b[c, m]
    return A


def dense_to_band(A, K):
    N = A.shape[0]
    band = np.zeros((2 * K + 1, N))
    for c in range(2 * K + 1):
        j = np.arange(N)
        i = j + c - K
        m = (i >= 0) & (i < N)
        band[c, m] = A[i[m], j[m]]
    return band.reshape(-1)


def block_factor_to_dense(f, K):
    """Oracle dense-band row-major block storage f[r, c - r + K] -> dense (n x n)."""
    n = f.shape[0]
    M = np.zeros((n, n))
    for r in range(n):
        for d in range(-K, K + 1):
            c = r + d
            if 0 <= c < n:
                M[r, c] = f[r, d + K]
    return M
