// SaP-C factor phase per interface i (between blocks i and i+1):
//   coupling blocks B_i, C_{i+1} read from the band (Sec. 2.1, Fig. 2.1);
//   spike tips from the bottom LU / top UL K x K blocks (Sec. 2.1,
//   computational savings; Eq. (2.2)):
//     V^(b)_i     = U_bb^{-1} L_bb^{-1} B_i
//     W^(t)_{i+1} = L'_tt^{-1} U'_tt^{-1} C_{i+1}
//   reduced matrix Rbar_i = I - W^(t)_{i+1} V^(b)_i (Eq. (2.5a)) in FP64,
//   factored by partial pivoting and inverted, so that each preconditioner
//   application solves Eq. (2.5b) by one FP64 matrix-vector product.
// For the SaP preconditioner of A^T (adjoint) the same kernel uses the
// stored factors transposed: A_i^T = U_i^T L_i^T, A_{i+1}^T = L'^T U'^T,
// couplings B'_i = C_{i+1}^T, C'_{i+1} = B_i^T:
//     V'^(b)_i     = L_bb^{-T} U_bb^{-T} C_{i+1}^T
//     W'^(t)_{i+1} = U'_tt^{-T} L'_tt^{-T} B_i^T
// One CTA per interface; K x K working matrices in shared memory, or (wide
// bands, GM) in a per-interface global scratch that stays L2-resident.
#include <cuda_runtime.h>
#include <cstdint>
#include "sap_internal.cuh"

namespace sap {

namespace {

constexpr int NT = 256;

// Solve op(M) x = x in place for the column `col` of X (K x K row-major in
// shared memory), M in shared memory (row-major K x K).  lower: the
// triangle of M used; unit: implicit unit diagonal; trans: use M^T.
template <typename T>
__device__ void tri_col(const T* M, int K, bool lower, bool unit, bool trans, T* X, int col) {
  // effective matrix E = trans ? M^T : M; E is lower iff (lower != trans)
  const bool elower = (lower != trans);
  auto E = [&](int r, int q) -> T { return trans ? M[q * K + r] : M[r * K + q]; };
  if (elower) {
    for (int r = 0; r < K; ++r) {
      T a0 = X[r * K + col], a1 = T(0), a2 = T(0), a3 = T(0);
      int q = 0;
      for (; q + 3 < r; q += 4) {
        a0 -= E(r, q) * X[q * K + col];
        a1 -= E(r, q + 1) * X[(q + 1) * K + col];
        a2 -= E(r, q + 2) * X[(q + 2) * K + col];
        a3 -= E(r, q + 3) * X[(q + 3) * K + col];
      }
      for (; q < r; ++q) a0 -= E(r, q) * X[q * K + col];
      T v = (a0 + a1) + (a2 + a3);
      X[r * K + col] = unit ? v : v / E(r, r);
    }
  } else {
    for (int r = K - 1; r >= 0; --r) {
      T a0 = X[r * K + col], a1 = T(0), a2 = T(0), a3 = T(0);
      int q = r + 1;
      for (; q + 3 < K; q += 4) {
        a0 -= E(r, q) * X[q * K + col];
        a1 -= E(r, q + 1) * X[(q + 1) * K + col];
        a2 -= E(r, q + 2) * X[(q + 2) * K + col];
        a3 -= E(r, q + 3) * X[(q + 3) * K + col];
      }
      for (; q < K; ++q) a0 -= E(r, q) * X[q * K + col];
      T v = (a0 + a1) + (a2 + a3);
      X[r * K + col] = unit ? v : v / E(r, r);
    }
  }
}

// Bytes of one interface's working matrices: R (FP64), factor tile and
// right-hand sides (T), the latter two reused as one FP64 K x K workspace for
// the inverse (2 sizeof(T) >= 8).
__host__ __device__ inline size_t spike_ws_bytes(int K, int tsize) {
  return (size_t)K * K * (sizeof(double) + 2 * (size_t)tsize);
}
__host__ __device__ inline size_t spike_ws_stride(int K, int tsize) { return (spike_ws_bytes(K, tsize) + 255) & ~(size_t)255; }

template <typename T, bool GM>
__global__ void __launch_bounds__(NT)
k_spikes(const double* __restrict__ band, int64_t N, int K, Dev d, const T* __restrict__ F,
         const T* __restrict__ ULt, bool adjoint, T* __restrict__ Vout, T* __restrict__ Wout,
         double* __restrict__ Rinv, double* __restrict__ R0, int* __restrict__ pivout, int* singular,
         unsigned char* __restrict__ gws) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int KK = K * K;
  unsigned char* ws = GM ? gws + (size_t)blockIdx.x * spike_ws_stride(K, sizeof(T)) : smem_raw;
  double* R = reinterpret_cast<double*>(ws);                   // K x K FP64
  T* Mx = reinterpret_cast<T*>(R + KK);                        // K x K factor tile
  T* X = Mx + KK;                                              // K x K right-hand sides / tips
  int* pivs = reinterpret_cast<int*>(smem_raw + (GM ? 0 : spike_ws_bytes(K, sizeof(T))));   // K pivots
  __shared__ double red_v[NT / 32];
  __shared__ int red_i[NT / 32];

  const int i = blockIdx.x;
  const int tid = threadIdx.x;
  const int64_t s = d.off[i + 1];              // first row of block i+1
  const int64_t n0 = d.off[i + 1] - d.off[i];  // rows of block i
  const int64_t ld = d.ld[i];
  const T* Fi = F + d.fbase[i];
  const T* ULi = ULt + (int64_t)i * KK;        // top tiles of block i+1
  T* Vi = Vout + (int64_t)i * KK;
  T* Wi = Wout + (int64_t)i * KK;

  // ---- V tip: M = [L_bb | U_bb] packed (bottom K x K of block i's LU) ----
  for (int e = tid; e < KK; e += NT) {
    int r = e / K, q = e % K;
    int64_t gr = n0 - K + r, gq = n0 - K + q;
    Mx[e] = Fi[(int64_t)(K + gr - gq) * ld + gq];
    // RHS: forward B_i(r,q) = a(s-K+r, s+q) (q <= r); adjoint C_{i+1}^T(r,q) = C(q,r) = a(s+q, s-K+r)
    double v = 0.0;
    if (!adjoint) { if (q <= r) v = band[(int64_t)(r - q) * N + s + q]; }
    else { if (r >= q) v = band[(int64_t)(2 * K + q - r) * N + s - K + r]; }
    X[e] = (T)v;
  }
  __syncthreads();
  for (int col = tid; col < K; col += NT) {
    if (!adjoint) {
      tri_col(Mx, K, true, true, false, X, col);    // L_bb (unit lower)
      tri_col(Mx, K, false, false, false, X, col);  // U_bb
    } else {
      tri_col(Mx, K, false, false, true, X, col);   // U_bb^T (lower)
      tri_col(Mx, K, true, true, true, X, col);     // L_bb^T (unit upper)
    }
  }
  __syncthreads();
  for (int e = tid; e < KK; e += NT) Vi[e] = X[e];
  __syncthreads();

  // ---- W tip: M = [U'_tt | L'_tt] packed top tiles of block i+1's UL ----
  for (int e = tid; e < KK; e += NT) {
    int r = e / K, q = e % K;
    Mx[e] = ULi[e];
    // RHS: forward C_{i+1}(r,q) = a(s+r, s-K+q) (q >= r); adjoint B_i^T(r,q) = B(q,r) = a(s-K+q, s+r)
    double v = 0.0;
    if (!adjoint) { if (q >= r) v = band[(int64_t)(2 * K + r - q) * N + s - K + q]; }
    else { if (r <= q) v = band[(int64_t)(q - r) * N + s + r]; }
    X[e] = (T)v;
  }
  __syncthreads();
  for (int col = tid; col < K; col += NT) {
    if (!adjoint) {
      tri_col(Mx, K, false, true, false, X, col);   // U'_tt (unit upper)
      tri_col(Mx, K, true, false, false, X, col);   // L'_tt (lower)
    } else {
      tri_col(Mx, K, true, false, true, X, col);    // L'_tt^T (upper)
      tri_col(Mx, K, false, true, true, X, col);    // U'_tt^T (unit lower)
    }
  }
  __syncthreads();
  for (int e = tid; e < KK; e += NT) Wi[e] = X[e];
  // ---- Rbar = I - W V in FP64 (V re-read from global, W in X) ----
  __syncthreads();
  for (int e = tid; e < KK; e += NT) Mx[e] = Vi[e];
  __syncthreads();
  for (int e = tid; e < KK; e += NT) {
    int r = e / K, c = e % K;
    double a0 = (r == c) ? 1.0 : 0.0, a1 = 0.0;
    int q = 0;
    for (; q + 1 < K; q += 2) {
      a0 -= (double)X[r * K + q] * (double)Mx[q * K + c];
      a1 -= (double)X[r * K + q + 1] * (double)Mx[(q + 1) * K + c];
    }
    for (; q < K; ++q) a0 -= (double)X[r * K + q] * (double)Mx[q * K + c];
    R[e] = a0 + a1;
    R0[(int64_t)i * KK + e] = a0 + a1;
  }
  __syncthreads();
  // ---- GEPP of Rbar (ties to the lowest row) ----
  for (int k = 0; k < K; ++k) {
    double best = -1.0;
    int bi = k;
    for (int r = k + tid; r < K; r += NT) {
      double v = fabs(R[r * K + k]);
      if (v > best) { best = v; bi = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      double ov = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if ((tid & 31) == 0) { red_v[tid >> 5] = best; red_i[tid >> 5] = bi; }
    __syncthreads();
    if (tid == 0) {
      double bv = red_v[0]; int bx = red_i[0];
      for (int w = 1; w < NT / 32; ++w)
        if (red_v[w] > bv || (red_v[w] == bv && red_i[w] < bx)) { bv = red_v[w]; bx = red_i[w]; }
      pivs[k] = bx;
      if (bv == 0.0) atomicExch(singular, 1);
    }
    __syncthreads();
    const int p = pivs[k];
    if (p != k)
      for (int c = tid; c < K; c += NT) { double t = R[k * K + c]; R[k * K + c] = R[p * K + c]; R[p * K + c] = t; }
    __syncthreads();
    const double pv = R[k * K + k];
    for (int r = k + 1 + tid; r < K; r += NT) R[r * K + k] = (pv != 0.0) ? R[r * K + k] / pv : 0.0;
    __syncthreads();
    const int m = K - k - 1;
    for (int e = tid; e < m * m; e += NT) {
      int r = k + 1 + e / m, c = k + 1 + e % m;
      R[r * K + c] -= R[r * K + k] * R[k * K + c];
    }
    __syncthreads();
  }
  // ---- inverse Rinv = U^{-1} L^{-1} P (P R = L U), column by column ----
  double* Xd = reinterpret_cast<double*>(Mx);   // reuse Mx + X as a K x K FP64 workspace
  for (int e = tid; e < KK; e += NT) Xd[e] = 0.0;
  __syncthreads();
  for (int col = tid; col < K; col += NT) {
    // right-hand side P e_col: apply the recorded swaps to e_col
    int pos = col;
    for (int k = 0; k < K; ++k) {
      if (pivs[k] == pos) pos = k;
      else if (k == pos) pos = pivs[k];
    }
    Xd[pos * K + col] = 1.0;
    tri_col(R, K, true, true, false, Xd, col);
    tri_col(R, K, false, false, false, Xd, col);
  }
  __syncthreads();
  for (int e = tid; e < KK; e += NT) Rinv[(int64_t)i * KK + e] = Xd[e];
  for (int k = tid; k < K; k += NT) pivout[(int64_t)i * K + k] = pivs[k];
}

}  // namespace

size_t spike_scratch_bytes(int K, int P, bool fp64) {
  const int ts = fp64 ? 8 : 4;
  if (P < 2 || spike_ws_bytes(K, ts) + (size_t)K * sizeof(int) <= kSmemPerBlock) return 0;
  return (size_t)(P - 1) * spike_ws_stride(K, ts);
}

template <typename T>
cudaError_t launch_spikes(const double* band, int64_t N, int K, int P, Dev d, const T* F, const T* ULt,
                          bool adjoint, T* V, T* Wt, double* Rinv, double* R0, int* piv, int* singular,
                          void* gscratch, cudaStream_t s) {
  if (P < 2) return cudaSuccess;
  const bool gm = spike_scratch_bytes(K, P, sizeof(T) == 8) > 0;
  if (gm && !gscratch) return cudaErrorInvalidValue;
  const size_t smem = (gm ? 0 : spike_ws_bytes(K, sizeof(T))) + (size_t)K * sizeof(int);
  auto kern = gm ? k_spikes<T, true> : k_spikes<T, false>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  count_launches(1);
  kern<<<P - 1, NT, smem, s>>>(band, N, K, d, F, ULt, adjoint, V, Wt, Rinv, R0, piv, singular,
                               static_cast<unsigned char*>(gscratch));
  return cudaGetLastError();
}

template cudaError_t launch_spikes<float>(const double*, int64_t, int, int, Dev, const float*, const float*, bool,
                                          float*, float*, double*, double*, int*, int*, void*, cudaStream_t);
template cudaError_t launch_spikes<double>(const double*, int64_t, int, int, Dev, const double*, const double*,
                                           bool, double*, double*, double*, double*, int*, int*, void*,
                                           cudaStream_t);

}  // namespace sap
