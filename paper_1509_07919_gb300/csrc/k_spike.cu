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

// Solve op(M) x = x in place for the column `col` of X (K rows, row pitch
// ldx), M row-major K x K.  lower: the triangle of M used; unit: implicit
// unit diagonal; trans: use M^T.
template <typename T>
__device__ void tri_col(const T* M, int K, bool lower, bool unit, bool trans, T* X, int col, int ldx) {
  // effective matrix E = trans ? M^T : M; E is lower iff (lower != trans)
  const bool elower = (lower != trans);
  auto E = [&](int r, int q) -> T { return trans ? M[q * K + r] : M[r * K + q]; };
  if (elower) {
    for (int r = 0; r < K; ++r) {
      T a0 = X[r * ldx + col], a1 = T(0), a2 = T(0), a3 = T(0);
      int q = 0;
      for (; q + 3 < r; q += 4) {
        a0 -= E(r, q) * X[q * ldx + col];
        a1 -= E(r, q + 1) * X[(q + 1) * ldx + col];
        a2 -= E(r, q + 2) * X[(q + 2) * ldx + col];
        a3 -= E(r, q + 3) * X[(q + 3) * ldx + col];
      }
      for (; q < r; ++q) a0 -= E(r, q) * X[q * ldx + col];
      T v = (a0 + a1) + (a2 + a3);
      X[r * ldx + col] = unit ? v : v / E(r, r);
    }
  } else {
    for (int r = K - 1; r >= 0; --r) {
      T a0 = X[r * ldx + col], a1 = T(0), a2 = T(0), a3 = T(0);
      int q = r + 1;
      for (; q + 3 < K; q += 4) {
        a0 -= E(r, q) * X[q * ldx + col];
        a1 -= E(r, q + 1) * X[(q + 1) * ldx + col];
        a2 -= E(r, q + 2) * X[(q + 2) * ldx + col];
        a3 -= E(r, q + 3) * X[(q + 3) * ldx + col];
      }
      for (; q < K; ++q) a0 -= E(r, q) * X[q * ldx + col];
      T v = (a0 + a1) + (a2 + a3);
      X[r * ldx + col] = unit ? v : v / E(r, r);
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

// GEPP of the K x K FP64 matrix R in place (P R = L U, unit L below the
// diagonal), ties to the lowest row index; pivs[k] = row swapped with k.  The
// whole CTA (NTH threads) takes part.
template <int NTH>
__device__ void rbar_gepp(double* R, int K, int* pivs, int* singular, double* red_v, int* red_i) {
  const int tid = threadIdx.x;
  for (int k = 0; k < K; ++k) {
    double best = -1.0;
    int bi = k;
    for (int r = k + tid; r < K; r += NTH) {
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
      for (int w = 1; w < NTH / 32; ++w)
        if (red_v[w] > bv || (red_v[w] == bv && red_i[w] < bx)) { bv = red_v[w]; bx = red_i[w]; }
      pivs[k] = bx;
      if (bv == 0.0) atomicExch(singular, 1);
    }
    __syncthreads();
    const int p = pivs[k];
    if (p != k)
      for (int c = tid; c < K; c += NTH) { double t = R[k * K + c]; R[k * K + c] = R[p * K + c]; R[p * K + c] = t; }
    __syncthreads();
    const double pv = R[k * K + k];
    for (int r = k + 1 + tid; r < K; r += NTH) R[r * K + k] = (pv != 0.0) ? R[r * K + k] / pv : 0.0;
    __syncthreads();
    const int m = K - k - 1;
    for (int e = tid; e < m * m; e += NTH) {
      int r = k + 1 + e / m, c = k + 1 + e % m;
      R[r * K + c] -= R[r * K + k] * R[k * K + c];
    }
    __syncthreads();
  }
}

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

  if (GM) {     // wide bands: the dense bottom LU tile only; the solves run in k_tip_cols
    for (int e = tid; e < KK; e += NT) {
      const int r = e / K, q = e % K;
      const int64_t gr = n0 - K + r, gq = n0 - K + q;
      Mx[e] = Fi[(int64_t)(K + gr - gq) * ld + gq];
    }
    return;
  }
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
      tri_col(Mx, K, true, true, false, X, col, K);    // L_bb (unit lower)
      tri_col(Mx, K, false, false, false, X, col, K);  // U_bb
    } else {
      tri_col(Mx, K, false, false, true, X, col, K);   // U_bb^T (lower)
      tri_col(Mx, K, true, true, true, X, col, K);     // L_bb^T (unit upper)
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
      tri_col(Mx, K, false, true, false, X, col, K);   // U'_tt (unit upper)
      tri_col(Mx, K, true, false, false, X, col, K);   // L'_tt (lower)
    } else {
      tri_col(Mx, K, true, false, true, X, col, K);    // L'_tt^T (upper)
      tri_col(Mx, K, false, true, true, X, col, K);    // U'_tt^T (unit lower)
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
  rbar_gepp<NT>(R, K, pivs, singular, red_v, red_i);
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
    tri_col(R, K, true, true, false, Xd, col, K);
    tri_col(R, K, false, false, false, Xd, col, K);
  }
  __syncthreads();
  for (int e = tid; e < KK; e += NT) Rinv[(int64_t)i * KK + e] = Xd[e];
  for (int k = tid; k < K; k += NT) pivout[(int64_t)i * K + k] = pivs[k];
}

// ---- wide bands: tips, Rbar, GEPP and inverse spread over more CTAs ----

// Spike tips, 32 columns per CTA (one per thread, K x 32 right-hand sides in
// shared memory), the factor tiles read row-wise from global memory:
// blockIdx.z = 0 the V tip (dense bottom LU tile, copied by k_spikes),
// 1 the W tip (top UL tiles); grid (ceil(K / 32), P - 1, 2).
template <typename T>
__global__ void __launch_bounds__(32)
k_tip_cols(const double* __restrict__ band, int64_t N, int K, Dev d, const T* __restrict__ ULt, bool adjoint,
           T* __restrict__ Vout, T* __restrict__ Wout, const unsigned char* __restrict__ gws) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Xs = reinterpret_cast<T*>(smem_raw);    // K x 32
  const int i = blockIdx.y;
  const int lane = threadIdx.x;
  const int col = blockIdx.x * 32 + lane;
  const int64_t s = d.off[i + 1];
  const int64_t KK = (int64_t)K * K;
  const bool vtip = blockIdx.z == 0;
  const T* M = vtip ? reinterpret_cast<const T*>(gws + (size_t)i * spike_ws_stride(K, sizeof(T)) +
                                                 (size_t)K * K * sizeof(double))
                    : ULt + i * KK;
  if (col < K) {
    for (int r = 0; r < K; ++r) {
      const int q = col;
      double v = 0.0;
      if (vtip) {   // forward B_i(r,q) = a(s-K+r, s+q) (q <= r); adjoint C_{i+1}^T(r,q) = a(s+q, s-K+r)
        if (!adjoint) { if (q <= r) v = band[(int64_t)(r - q) * N + s + q]; }
        else { if (r >= q) v = band[(int64_t)(2 * K + q - r) * N + s - K + r]; }
      } else {      // forward C_{i+1}(r,q) = a(s+r, s-K+q) (q >= r); adjoint B_i^T(r,q) = a(s-K+q, s+r)
        if (!adjoint) { if (q >= r) v = band[(int64_t)(2 * K + r - q) * N + s - K + q]; }
        else { if (r <= q) v = band[(int64_t)(q - r) * N + s + r]; }
      }
      Xs[r * 32 + lane] = (T)v;
    }
    if (vtip) {
      if (!adjoint) {
        tri_col(M, K, true, true, false, Xs, lane, 32);    // L_bb (unit lower)
        tri_col(M, K, false, false, false, Xs, lane, 32);  // U_bb
      } else {
        tri_col(M, K, false, false, true, Xs, lane, 32);   // U_bb^T (lower)
        tri_col(M, K, true, true, true, Xs, lane, 32);     // L_bb^T (unit upper)
      }
    } else {
      if (!adjoint) {
        tri_col(M, K, false, true, false, Xs, lane, 32);   // U'_tt (unit upper)
        tri_col(M, K, true, false, false, Xs, lane, 32);   // L'_tt (lower)
      } else {
        tri_col(M, K, true, false, true, Xs, lane, 32);    // L'_tt^T (upper)
        tri_col(M, K, false, true, true, Xs, lane, 32);    // U'_tt^T (unit lower)
      }
    }
    T* out = (vtip ? Vout : Wout) + i * KK;
    for (int r = 0; r < K; ++r) out[(int64_t)r * K + col] = Xs[r * 32 + lane];
  }
}

// Rbar_i = I - W^(t)_{i+1} V^(b)_i in FP64 (R0, and a copy in the interface's
// workspace for the GEPP), 64 x 64 output tiles, 16-deep panels of W and V
// staged in shared memory; grid (tiles, tiles, P - 1).
constexpr int RT = 64, RQ = 16;
template <typename T>
__global__ void __launch_bounds__(256)
k_rbar_form(const T* __restrict__ V, const T* __restrict__ Wt, int K, double* __restrict__ R0,
            unsigned char* __restrict__ gws) {
  __shared__ double As[RQ][RT + 1];   // W(r0 + x, q0 + q) at As[q][x]
  __shared__ double Bs[RQ][RT + 1];   // V(q0 + q, c0 + y) at Bs[q][y]
  const int i = blockIdx.z;
  const int64_t KK = (int64_t)K * K;
  const T* Wi = Wt + i * KK;
  const T* Vi = V + i * KK;
  const int r0 = blockIdx.y * RT, c0 = blockIdx.x * RT;
  const int tid = threadIdx.x, tr = tid / 16, tc = tid % 16;
  double acc[4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) acc[x][y] = 0.0;
  for (int q0 = 0; q0 < K; q0 += RQ) {
    for (int e = tid; e < RT * RQ; e += 256) {
      const int x = e / RQ, q = e % RQ;          // W rows, consecutive q per thread group
      const int r = r0 + x, qq = q0 + q;
      As[q][x] = (r < K && qq < K) ? (double)Wi[(int64_t)r * K + qq] : 0.0;
      const int q2 = e / RT, y = e % RT;         // V rows q, consecutive columns
      const int qv = q0 + q2, c = c0 + y;
      Bs[q2][y] = (qv < K && c < K) ? (double)Vi[(int64_t)qv * K + c] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < RQ; ++q) {
      double a[4], b[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) a[x] = As[q][tr + 16 * x];
#pragma unroll
      for (int y = 0; y < 4; ++y) b[y] = Bs[q][tc + 16 * y];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] += a[x] * b[y];
    }
    __syncthreads();
  }
  double* Rw = reinterpret_cast<double*>(gws + (size_t)i * spike_ws_stride(K, sizeof(T)));
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int r = r0 + tr + 16 * x;
    if (r >= K) continue;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int c = c0 + tc + 16 * y;
      if (c >= K) continue;
      const double v = (r == c ? 1.0 : 0.0) - acc[x][y];
      R0[i * KK + (int64_t)r * K + c] = v;
      Rw[(int64_t)r * K + c] = v;
    }
  }
}

// GEPP of every Rbar_i in its workspace (one CTA of 1024 threads per
// interface: the L2-resident rank-1 updates want many loads in flight).
// Blocked GEPP of the reduced matrices Rbar_i (K x K FP64, row-major in the
// global workspace, wide bands): right-looking, kGeppNB-column panels, two
// launches per panel.  k_gepp_panel (one CTA per interface) takes the
// panel's pivots (column maxima, ties to the lowest row), swaps whole rows,
// forms the multipliers and updates the panel, then the panel's rows of U
// to its right (unit lower solve with L11); k_gepp_update subtracts L21 U12
// from the trailing matrix in 64 x 64 tiles over all interfaces.  Every entry
// receives the same fused multiply-adds in the same order as in the
// unblocked elimination (a row's deferred updates move with it in a swap),
// so the factors and pivots are those of the one-column-at-a-time GEPP.
constexpr int kGeppNB = 16;
constexpr int kPanelThreads = 512;
template <typename T>
__global__ void __launch_bounds__(kPanelThreads)
k_gepp_panel(int K, int k0, unsigned char* __restrict__ gws, int* __restrict__ pivout, int* singular) {
  __shared__ double red_v[kPanelThreads / 32];
  __shared__ int red_i[kPanelThreads / 32];
  __shared__ int psh;
  const int i = blockIdx.x;
  const int tid = threadIdx.x;
  double* R = reinterpret_cast<double*>(gws + (size_t)i * spike_ws_stride(K, sizeof(T)));
  const int kend = min(K, k0 + kGeppNB);
  for (int c = k0; c < kend; ++c) {
    double best = -1.0;
    int bi = c;
    for (int r = c + tid; r < K; r += kPanelThreads) {
      const double v = fabs(R[(int64_t)r * K + c]);
      if (v > best) { best = v; bi = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if ((tid & 31) == 0) { red_v[tid >> 5] = best; red_i[tid >> 5] = bi; }
    __syncthreads();
    if (tid == 0) {
      double bv = red_v[0];
      int bx = red_i[0];
      for (int w = 1; w < kPanelThreads / 32; ++w)
        if (red_v[w] > bv || (red_v[w] == bv && red_i[w] < bx)) { bv = red_v[w]; bx = red_i[w]; }
      pivout[(int64_t)i * K + c] = bx;
      psh = bx;
      if (bv == 0.0) atomicExch(singular, 1);
    }
    __syncthreads();
    const int p = psh;
    if (p != c)
      for (int j = tid; j < K; j += kPanelThreads) {
        const double t = R[(int64_t)c * K + j];
        R[(int64_t)c * K + j] = R[(int64_t)p * K + j];
        R[(int64_t)p * K + j] = t;
      }
    __syncthreads();
    const double pv = R[(int64_t)c * K + c];
    for (int r = c + 1 + tid; r < K; r += kPanelThreads)
      R[(int64_t)r * K + c] = (pv != 0.0) ? R[(int64_t)r * K + c] / pv : 0.0;
    __syncthreads();
    // the panel's columns right of c (lane group of 16 threads per row)
    const int cc = c + 1 + (tid & (kGeppNB - 1));
    if (cc < kend)
      for (int r = c + 1 + tid / kGeppNB; r < K; r += kPanelThreads / kGeppNB)
        R[(int64_t)r * K + cc] -= R[(int64_t)r * K + c] * R[(int64_t)c * K + cc];
    __syncthreads();
  }
  // U12: the panel's rows right of the panel, unit lower solve with L11 (the
  // rank-1 steps of the panel's columns in order)
  for (int j = kend + tid; j < K; j += kPanelThreads)
    for (int r = k0 + 1; r < kend; ++r) {
      double acc = R[(int64_t)r * K + j];
      for (int q = k0; q < r; ++q) acc -= R[(int64_t)r * K + q] * R[(int64_t)q * K + j];
      R[(int64_t)r * K + j] = acc;
    }
}

// Trailing update of a panel: R[r][j] -= sum_q L21[r][q] U12[q][j] over the
// panel's columns q in order, rows and columns from k0 + kGeppNB, 64 x 64
// tiles (256 threads, 4 x 4 entries each, columns interleaved by 16).  Grid
// (tiles, tiles, P - 1).
template <typename T>
__global__ void __launch_bounds__(256)
k_gepp_update(int K, int k0, unsigned char* __restrict__ gws) {
  __shared__ double Ls[64][kGeppNB + 1];
  __shared__ double Us[kGeppNB][64];
  const int i = blockIdx.z;
  double* R = reinterpret_cast<double*>(gws + (size_t)i * spike_ws_stride(K, sizeof(T)));
  const int m0 = k0 + kGeppNB;
  const int rt = m0 + (int)blockIdx.y * 64, ct = m0 + (int)blockIdx.x * 64;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int e = tid; e < 64 * kGeppNB; e += 256) {
    const int rr = e / kGeppNB, q = e % kGeppNB;
    Ls[rr][q] = rt + rr < K ? R[(int64_t)(rt + rr) * K + k0 + q] : 0.0;
  }
  for (int e = tid; e < kGeppNB * 64; e += 256) {
    const int q = e / 64, cc = e % 64;
    Us[q][cc] = ct + cc < K ? R[(int64_t)(k0 + q) * K + ct + cc] : 0.0;
  }
  __syncthreads();
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int row = rt + ty + 16 * a;
    if (row >= K) break;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int col = ct + tx + 16 * b;
      if (col >= K) continue;
      double acc = R[(int64_t)row * K + col];
#pragma unroll
      for (int q = 0; q < kGeppNB; ++q) acc -= Ls[ty + 16 * a][q] * Us[q][tx + 16 * b];
      R[(int64_t)row * K + col] = acc;
    }
  }
}

// Rbar_i^{-1} = U^{-1} L^{-1} P from the GEPP factors, 32 columns per CTA
// (K x 32 right-hand sides in shared memory, lane = column); the eight warps
// split every row's dot product (q = w mod 8, two accumulators each: FP64
// multiply-add latency is long on GB300) and warp 0 finishes the row.
// Grid (ceil(K / 32), P - 1).
constexpr int kInvWarps = 8;
template <typename T>
__global__ void __launch_bounds__(32 * kInvWarps)
k_rbar_inv(int K, const unsigned char* __restrict__ gws, const int* __restrict__ pivin, double* __restrict__ Rinv) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* Xs = reinterpret_cast<double*>(smem_raw);                  // K x 32
  double* part = Xs + (size_t)K * 32;                                 // kInvWarps x 32
  int* pv = reinterpret_cast<int*>(part + kInvWarps * 32);            // K pivots
  const int i = blockIdx.y;
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  const int col = blockIdx.x * 32 + lane;
  const double* R = reinterpret_cast<const double*>(gws + (size_t)i * spike_ws_stride(K, sizeof(T)));
  for (int k = threadIdx.x; k < K; k += 32 * kInvWarps) pv[k] = pivin[(int64_t)i * K + k];
  for (int e = threadIdx.x; e < K * 32; e += 32 * kInvWarps) Xs[e] = 0.0;
  __syncthreads();
  if (wq == 0 && col < K) {
    int pos = col;        // P e_col: the recorded swaps applied to e_col
    for (int k = 0; k < K; ++k) {
      if (pv[k] == pos) pos = k;
      else if (k == pos) pos = pv[k];
    }
    Xs[pos * 32 + lane] = 1.0;
  }
  __syncthreads();
  // forward: unit lower L (below the diagonal of R)
  for (int r = 1; r < K; ++r) {
    const double* row = R + (int64_t)r * K;
    double a0 = 0.0, a1 = 0.0;
    int q = wq;
    for (; q + kInvWarps < r; q += 2 * kInvWarps) {
      a0 += row[q] * Xs[q * 32 + lane];
      a1 += row[q + kInvWarps] * Xs[(q + kInvWarps) * 32 + lane];
    }
    if (q < r) a0 += row[q] * Xs[q * 32 + lane];
    part[wq * 32 + lane] = a0 + a1;
    __syncthreads();
    if (wq == 0) {
      double sum = 0.0;
#pragma unroll
      for (int w = 0; w < kInvWarps; ++w) sum += part[w * 32 + lane];
      Xs[r * 32 + lane] -= sum;
    }
    __syncthreads();
  }
  // backward: U (on and above the diagonal)
  for (int r = K - 1; r >= 0; --r) {
    const double* row = R + (int64_t)r * K;
    double a0 = 0.0, a1 = 0.0;
    int q = r + 1 + wq;
    for (; q + kInvWarps < K; q += 2 * kInvWarps) {
      a0 += row[q] * Xs[q * 32 + lane];
      a1 += row[q + kInvWarps] * Xs[(q + kInvWarps) * 32 + lane];
    }
    if (q < K) a0 += row[q] * Xs[q * 32 + lane];
    part[wq * 32 + lane] = a0 + a1;
    __syncthreads();
    if (wq == 0) {
      double sum = 0.0;
#pragma unroll
      for (int w = 0; w < kInvWarps; ++w) sum += part[w * 32 + lane];
      Xs[r * 32 + lane] = (Xs[r * 32 + lane] - sum) / row[r];
    }
    __syncthreads();
  }
  if (col < K) {
    double* out = Rinv + (int64_t)i * K * K;
    for (int r = wq; r < K; r += kInvWarps) out[(int64_t)r * K + col] = Xs[r * 32 + lane];
  }
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
                          void* gscratch, cudaStream_t s, cudaEvent_t ev_rd) {
  if (P < 2) return ev_rd ? cudaEventRecord(ev_rd, s) : cudaSuccess;
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
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (!gm) return ev_rd ? cudaEventRecord(ev_rd, s) : cudaSuccess;   // Rbar_i formed inside k_spikes
  unsigned char* gws = static_cast<unsigned char*>(gscratch);
  const size_t tsm = (size_t)K * 32 * sizeof(T);
  if (tsm > 48 * 1024) {
    e = cudaFuncSetAttribute(k_tip_cols<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm);
    if (e != cudaSuccess) return e;
  }
  count_launches(1);
  k_tip_cols<T><<<dim3((K + 31) / 32, P - 1, 2), 32, tsm, s>>>(band, N, K, d, ULt, adjoint, V, Wt, gws);
  if (ev_rd && (e = cudaEventRecord(ev_rd, s)) != cudaSuccess) return e;
  const int tiles = (K + RT - 1) / RT;
  count_launches(2);
  k_rbar_form<T><<<dim3(tiles, tiles, P - 1), 256, 0, s>>>(V, Wt, K, R0, gws);
  for (int k0 = 0; k0 < K; k0 += kGeppNB) {
    count_launches(1);
    k_gepp_panel<T><<<P - 1, kPanelThreads, 0, s>>>(K, k0, gws, piv, singular);
    const int m = K - k0 - kGeppNB;
    if (m > 0) {
      const int t = (m + 63) / 64;
      count_launches(1);
      k_gepp_update<T><<<dim3(t, t, P - 1), 256, 0, s>>>(K, k0, gws);
    }
  }
  const size_t ism = (size_t)(K + kInvWarps) * 32 * sizeof(double) + (size_t)K * sizeof(int);
  if (ism > 48 * 1024) {
    e = cudaFuncSetAttribute(k_rbar_inv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ism);
    if (e != cudaSuccess) return e;
  }
  k_rbar_inv<T><<<dim3((K + 31) / 32, P - 1), 32 * kInvWarps, ism, s>>>(K, gws, piv, Rinv);
  return cudaGetLastError();
}

size_t reduced_ws_bytes(int K, int nI, bool fp64) { return (size_t)nI * spike_ws_stride(K, fp64 ? 8 : 4); }

template <typename T>
cudaError_t launch_reduced(const T* V, const T* Wt, int K, int nI, double* Rinv, double* R0, int* piv, int* singular,
                           void* gscratch, cudaStream_t s) {
  if (nI < 1) return cudaSuccess;
  if (!gscratch) return cudaErrorInvalidValue;
  unsigned char* gws = static_cast<unsigned char*>(gscratch);
  const int tiles = (K + RT - 1) / RT;
  count_launches(2);
  k_rbar_form<T><<<dim3(tiles, tiles, nI), 256, 0, s>>>(V, Wt, K, R0, gws);
  for (int k0 = 0; k0 < K; k0 += kGeppNB) {
    count_launches(1);
    k_gepp_panel<T><<<nI, kPanelThreads, 0, s>>>(K, k0, gws, piv, singular);
    const int m = K - k0 - kGeppNB;
    if (m > 0) {
      const int t = (m + 63) / 64;
      count_launches(1);
      k_gepp_update<T><<<dim3(t, t, nI), 256, 0, s>>>(K, k0, gws);
    }
  }
  const size_t ism = (size_t)(K + kInvWarps) * 32 * sizeof(double) + (size_t)K * sizeof(int);
  if (ism > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_rbar_inv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ism);
    if (e != cudaSuccess) return e;
  }
  k_rbar_inv<T><<<dim3((K + 31) / 32, nI), 32 * kInvWarps, ism, s>>>(K, gws, piv, Rinv);
  return cudaGetLastError();
}

template cudaError_t launch_reduced<float>(const float*, const float*, int, int, double*, double*, int*, int*, void*,
                                           cudaStream_t);
template cudaError_t launch_reduced<double>(const double*, const double*, int, int, double*, double*, int*, int*,
                                            void*, cudaStream_t);

template cudaError_t launch_spikes<float>(const double*, int64_t, int, int, Dev, const float*, const float*, bool,
                                          float*, float*, double*, double*, int*, int*, void*, cudaStream_t,
                                          cudaEvent_t);
template cudaError_t launch_spikes<double>(const double*, int64_t, int, int, Dev, const double*, const double*,
                                           bool, double*, double*, double*, double*, int*, int*, void*,
                                           cudaStream_t, cudaEvent_t);

}  // namespace sap
