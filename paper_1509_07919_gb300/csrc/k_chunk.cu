// Chunk matrices of the blocked triangular sweeps (factor phase).
//
// The preconditioner apply (Eq. (2.3)) solves banded triangular systems with
// the block factors.  Its sweeps process 32-row chunks in sweep order; with
// positions p numbered in sweep order (rows ascending for the forward
// sweeps L and U^T, descending for the backward sweeps U and L^T) every
// sweep is a lower-triangular recurrence in p.  Writing y_c, z_c for the 32
// positions of chunk c, A_c for the chunk's 32 x 32 lower-triangular
// diagonal block and B_{c,k} for its coupling to chunk c - k (nonzero for
// k = 1 .. ng, ng = ceil(K / 32)),
//     z_c = A_c^{-1} y_c - sum_k (A_c^{-1} B_{c,k}) z_{c-k}.
// This kernel forms, per chunk and sweep kind, MINV_c = A_c^{-1} and
// G_{c,k} = A_c^{-1} B_{c,k} from the stored LU factors, so that a sweep
// streams one contiguous block of 32 x 32 matrices per chunk and its
// dependent chain is the single product G_{c,1} z_{c-1}.  Same linear
// operator as substitution, different rounding order.
#include <cuda_runtime.h>
#include <cstdint>
#include "sap_internal.cuh"

namespace sap {

namespace {

constexpr int CH = 32;

// Entry of the sweep matrix in position coordinates: row position pr, column
// position pc (pc <= pr), for sweep kind MODE, or 0 outside the band or the
// block.  F[c * ld + q] = entry (r, q), c = K + r - q (unit-lower L below,
// U on and above the diagonal).
template <int MODE, typename T>
__device__ __forceinline__ T sweep_entry(const T* F, int K, int n, int ld, int pr, int pc) {
  const bool fwd = (MODE == 0 || MODE == 2);          // LF, UTF
  const int r = fwd ? pr : ld - 1 - pr;
  const int q = fwd ? pc : ld - 1 - pc;
  if (r >= n || q >= n || r < 0 || q < 0) return (pr == pc) ? T(1) : T(0);   // padding rows: identity
  int fr, fq;               // factor entry (fr, fq)
  bool unit;
  if (MODE == 0) { fr = r; fq = q; unit = true; }       // L(r, q), q <= r
  else if (MODE == 1) { fr = r; fq = q; unit = false; } // U(r, q), q >= r
  else if (MODE == 2) { fr = q; fq = r; unit = false; } // U^T(r, q) = U(q, r)
  else { fr = q; fq = r; unit = true; }                 // L^T(r, q) = L(q, r)
  if (pr == pc && unit) return T(1);
  const int c = K + fr - fq;
  if (c < 0 || c > 2 * K) return T(0);
  return F[(int64_t)c * ld + fq];
}

template <typename T, int MODE>
__global__ void __launch_bounds__(128)
k_chunk_mats(const T* __restrict__ Fall, int K, Dev d, const int64_t* __restrict__ cbase, T* __restrict__ out) {
  __shared__ T A[CH][CH + 1];
  __shared__ T X[CH][CH + 1];     // MINV, column j computed by thread j
  __shared__ T Bc[CH][CH + 1];
  const int ng = (K + CH - 1) / CH;
  const int b = blockIdx.y;
  const int ld = (int)d.ld[b];
  const int nch = ld / CH;
  const int c = blockIdx.x;
  if (c >= nch) return;
  const int n = (int)(d.off[b + 1] - d.off[b]);
  const T* F = Fall + d.fbase[b];
  const int tid = threadIdx.x;
  const int p0 = c * CH;
  for (int e = tid; e < CH * CH; e += blockDim.x) {
    const int t = e / CH, j = e % CH;
    // in-chunk lower-triangular block
    A[t][j] = (j <= t) ? sweep_entry<MODE>(F, K, n, ld, p0 + t, p0 + j) : T(0);
    X[t][j] = T(0);
  }
  __syncthreads();
  // MINV = A^{-1} (lower triangular): thread j solves A x = e_j by substitution
  if (tid < CH) {
    const int j = tid;
    X[j][j] = T(1) / A[j][j];
    for (int r = j + 1; r < CH; ++r) {
      T acc = T(0);
      for (int q = j; q < r; ++q) acc += A[r][q] * X[q][j];
      X[r][j] = -acc / A[r][r];
    }
  }
  __syncthreads();
  // stored column-major (element (t, j) at j * 32 + t): the sweep's lane t
  // reads its row as 32 conflict-free shared-memory loads
  T* M = out + cbase[b] + (int64_t)c * (1 + ng) * CH * CH;
  for (int e = tid; e < CH * CH; e += blockDim.x) {
    const int j = e / CH, t = e % CH;
    M[e] = X[t][j];
  }
  for (int k = 1; k <= ng; ++k) {
    __syncthreads();
    for (int e = tid; e < CH * CH; e += blockDim.x) {
      const int t = e / CH, j = e % CH;
      const int dist = k * CH + t - j;    // position distance to column j of chunk c - k
      Bc[t][j] = (c >= k && dist <= K) ? sweep_entry<MODE>(F, K, n, ld, p0 + t, p0 - k * CH + j) : T(0);
    }
    __syncthreads();
    T* G = M + (int64_t)k * CH * CH;
    for (int e = tid; e < CH * CH; e += blockDim.x) {
      const int j = e / CH, t = e % CH;
      T acc = T(0);
      for (int q = 0; q <= t; ++q) acc += X[t][q] * Bc[q][j];
      G[e] = acc;
    }
  }
}

}  // namespace

template <typename T>
cudaError_t launch_chunk_mats(const T* F, int K, int P, Dev d, const int64_t* cbase, int max_nch, int mode, T* out,
                              cudaStream_t s) {
  dim3 grid(max_nch, P);
  count_launches(1);
  switch (mode) {
    case 0: k_chunk_mats<T, 0><<<grid, 128, 0, s>>>(F, K, d, cbase, out); break;
    case 1: k_chunk_mats<T, 1><<<grid, 128, 0, s>>>(F, K, d, cbase, out); break;
    case 2: k_chunk_mats<T, 2><<<grid, 128, 0, s>>>(F, K, d, cbase, out); break;
    default: k_chunk_mats<T, 3><<<grid, 128, 0, s>>>(F, K, d, cbase, out); break;
  }
  return cudaGetLastError();
}

template cudaError_t launch_chunk_mats<float>(const float*, int, int, Dev, const int64_t*, int, int, float*,
                                              cudaStream_t);
template cudaError_t launch_chunk_mats<double>(const double*, int, int, Dev, const int64_t*, int, int, double*,
                                               cudaStream_t);

}  // namespace sap
