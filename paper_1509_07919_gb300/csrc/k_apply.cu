// Preconditioner apply z = M^{-1} r (Sec. 2.1): the block-diagonal solve
// D g = r (Eq. (2.3)) as two banded triangular sweeps per block, and for
// SaP-C the truncated reduced systems (Eq. (2.5)) and the purification
// solves that follow them.
//
// Sweep kernel: one CTA (4 warps) per block, both sweeps in one launch.  A
// sweep is a linear recurrence over positions p = 0..n-1,
//     z_p = ( y_p - sum_{d=1..K} coef(p, d) z_{p-d} ) / diag(p),
// processed in chunks of 32 positions:
//   - warp 0 (the solver) runs the dependent chain of a chunk: lane t holds
//     row t; for j = 0..31 it broadcasts z_j with one shuffle and every
//     lane applies the in-chunk coefficient and, at the same time, the
//     coefficient that couples row t of the *next* chunk to z_j;
//   - warps 1..3 (helpers) prepare the next chunk meanwhile: they load the
//     right-hand side and the coefficients (pre-scaled by 1/diag, so the
//     chain has no division) into shared memory, and sum the "older"
//     contributions (d > 32 + t) from a shared-memory ring of past z.
// The four sweep kinds (L forward, U backward, U^T forward, L^T backward)
// differ only in how (p, d) maps to the factor storage
//   F[c * ld + q] = entry (r, q) of block i, c = K + r - q.
#include <cuda_runtime.h>
#include <cstdint>
#include "sap_internal.cuh"

namespace sap {

namespace {

constexpr int NW = 4;               // warps per sweep CTA
constexpr int CHK = 32;             // chunk length

enum Mode { LF = 0, UB = 1, UTF = 2, LTB = 3 };

template <int MODE>
__device__ __forceinline__ int64_t row_of(int64_t p, int64_t n) {
  return (MODE == LF || MODE == UTF) ? p : n - 1 - p;
}
// address of coef(p, d) (row r = row_of(p)), valid for 1 <= d <= K, d <= p
template <int MODE>
__device__ __forceinline__ int64_t coef_idx(int64_t r, int d, int K, int64_t ld) {
  if (MODE == LF) return (int64_t)(K + d) * ld + r - d;   // l(r, r-d)
  if (MODE == UB) return (int64_t)(K - d) * ld + r + d;   // u(r, r+d)
  if (MODE == UTF) return (int64_t)(K - d) * ld + r;      // u(r-d, r)
  return (int64_t)(K + d) * ld + r;                       // l(r+d, r)
}
template <int MODE> __device__ __forceinline__ constexpr bool unit_diag() { return MODE == LF || MODE == LTB; }

template <typename T> __device__ __forceinline__ T to_t(double v) { return (T)v; }

struct SweepIO {
  // input: y(r) = in[r] - corrections (top rows: ctop[r], bottom rows: cbot[r-(n-K)])
  const double* in_d;      // FP64 input (first sweep)
  const void* in_t;        // T input (second sweep), or nullptr
  const double* ctop;      // K corrections for rows 0..K-1, or nullptr
  const double* cbot;      // K corrections for rows n-K..n-1, or nullptr
  double* out_d;           // FP64 output or nullptr
  void* out_t;             // T output or nullptr
};

template <typename T>
struct SweepSmem {
  T coef1[2][CHK][CHK];   // [buf][j][t]: in-chunk coefficient of row t on z_j
  T coef2[2][CHK][CHK];   // [buf][j][t]: row t of the next chunk on z_j of this chunk
  T yhat[2][CHK];
  T older[2][NW - 1][CHK];
};

template <typename T, int MODE>
__device__ __forceinline__ T load_y(const SweepIO& io, int64_t r, int64_t n, int K) {
  if (io.in_t) return reinterpret_cast<const T*>(io.in_t)[r];
  double v = io.in_d[r];
  if (io.ctop && r < K) v -= io.ctop[r];
  if (io.cbot && r >= n - K) v -= io.cbot[r - (n - K)];
  return to_t<T>(v);
}

// Helpers (warps 1..NW-1): prepare chunk c (yhat, coef1, older) and coef2 of chunk c+1.
template <typename T, int MODE>
__device__ __forceinline__ void stage_chunk(SweepSmem<T>& sm, const T* __restrict__ F, int64_t ld, int K,
                                            int64_t n, int64_t c, const SweepIO& io, const T* ring,
                                            int ringmask) {
  const int ht = threadIdx.x - 32;           // 0 .. 32*(NW-1)-1
  const int nh = 32 * (NW - 1);
  const int lane = threadIdx.x & 31;
  const int hw = (threadIdx.x >> 5) - 1;     // helper warp index
  const int buf = c & 1;
  const int64_t p0 = c * CHK;
  // yhat and the in-chunk coefficients of chunk c, coef2 of chunk c+1
  for (int e = ht; e < CHK * CHK * 2 + CHK; e += nh) {
    if (e < CHK) {
      int64_t p = p0 + e;
      T v = T(0);
      if (p < n) {
        int64_t r = row_of<MODE>(p, n);
        v = load_y<T, MODE>(io, r, n, K);
        if (!unit_diag<MODE>()) v = v / F[(int64_t)K * ld + r];
      }
      sm.yhat[buf][e] = v;
      continue;
    }
    int f = e - CHK;
    int part = f / (CHK * CHK);               // 0 = coef1(c), 1 = coef2(c+1)
    int g = f % (CHK * CHK);
    int d = g / CHK + 1;                      // distance 1..32 (coef1) or d-offset (coef2)
    int t = g % CHK;                          // row lane (coalesced along the diagonal)
    if (part == 0) {
      // coef1[j][t], j = t - d, needs 1 <= d <= min(t, K)
      if (d <= t) {
        int64_t p = p0 + t;
        T v = T(0);
        if (d <= K && p < n) {
          int64_t r = row_of<MODE>(p, n);
          v = F[coef_idx<MODE>(r, d, K, ld)];
          if (!unit_diag<MODE>()) v = v / F[(int64_t)K * ld + r];
        }
        sm.coef1[buf][t - d][t] = v;
      }
    } else {
      // coef2 of chunk c+1: row t of chunk c+1 on z_j of chunk c, distance dd = 32 + t - j
      // here enumerate j = d - 1 (0..31)
      int j = d - 1;
      int dd = CHK + t - j;
      int64_t p = p0 + CHK + t;
      T v = T(0);
      if (dd <= K && p < n) {
        int64_t r = row_of<MODE>(p, n);
        v = F[coef_idx<MODE>(r, dd, K, ld)];
        if (!unit_diag<MODE>()) v = v / F[(int64_t)K * ld + r];
      }
      sm.coef2[buf][j][t] = v;
    }
  }
  // zero the upper part of coef1 (j >= t) once per buffer use
  for (int e = ht; e < CHK * CHK; e += nh) {
    int j = e / CHK, t = e % CHK;
    if (j >= t) sm.coef1[buf][j][t] = T(0);
  }
  // older contributions of chunk c: d in [33 + t, K], z positions < 32 (c-1)
  {
    const int t = lane;
    const int64_t p = p0 + t;
    T acc = T(0);
    if (p < n && K > CHK + t) {
      int64_t r = row_of<MODE>(p, n);
      T dinv = T(1);
      if (!unit_diag<MODE>()) dinv = T(1) / F[(int64_t)K * ld + r];
      for (int d = CHK + 1 + t + hw; d <= K; d += NW - 1) {
        if (d > p) break;
        acc += F[coef_idx<MODE>(r, d, K, ld)] * ring[(p - d) & ringmask];
      }
      acc *= dinv;
    }
    sm.older[buf][hw][t] = acc;
  }
}

template <typename T, int MODE>
__device__ void sweep(SweepSmem<T>& sm, T* ring, int ringmask, const T* __restrict__ F, int64_t ld, int K,
                      int64_t n, const SweepIO& io) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int64_t nchunks = (n + CHK - 1) / CHK;
  if (warp > 0) stage_chunk<T, MODE>(sm, F, ld, K, n, 0, io, ring, ringmask);
  __syncthreads();
  T recent = T(0);  // warp 0: contribution of the previous chunk to this chunk's row `lane`
  for (int64_t c = 0; c < nchunks; ++c) {
    const int buf = c & 1;
    if (warp == 0) {
      T s = sm.yhat[buf][lane] - recent;
#pragma unroll
      for (int w = 0; w < NW - 1; ++w) s -= sm.older[buf][w][lane];
      T nxt = T(0);
#pragma unroll
      for (int j = 0; j < CHK; ++j) {
        T zj = __shfl_sync(0xffffffffu, s, j);
        s -= sm.coef1[buf][j][lane] * zj;
        nxt += sm.coef2[buf][j][lane] * zj;
      }
      recent = nxt;
      const int64_t p = c * CHK + lane;
      ring[p & ringmask] = s;
      if (p < n) {
        int64_t r = row_of<MODE>(p, n);
        if (io.out_d) io.out_d[r] = (double)s;
        else reinterpret_cast<T*>(io.out_t)[r] = s;
      }
    } else if (c + 1 < nchunks) {
      stage_chunk<T, MODE>(sm, F, ld, K, n, c + 1, io, ring, ringmask);
    }
    __syncthreads();
  }
}

template <typename T, bool TRANS>
__global__ void __launch_bounds__(NW * 32)
k_block_solve(const T* __restrict__ Fall, int K, Dev d, const double* __restrict__ r_in,
              double* __restrict__ z_out, T* __restrict__ tmp, const double* __restrict__ ctop_all,
              const double* __restrict__ cbot_all, int P, int ringsize) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SweepSmem<T>& sm = *reinterpret_cast<SweepSmem<T>*>(smem_raw);
  T* ring = reinterpret_cast<T*>(smem_raw + sizeof(SweepSmem<T>));
  const int b = blockIdx.x;
  const int64_t s = d.off[b];
  const int64_t n = d.off[b + 1] - s;
  const int64_t ld = d.ld[b];
  const T* F = Fall + d.fbase[b];
  SweepIO io1{r_in + s, nullptr, nullptr, nullptr, nullptr, tmp + s};
  if (ctop_all && b > 0) io1.ctop = ctop_all + (int64_t)(b - 1) * K;
  if (cbot_all && b + 1 < P) io1.cbot = cbot_all + (int64_t)b * K;
  if (!TRANS) sweep<T, LF>(sm, ring, ringsize - 1, F, ld, K, n, io1);
  else sweep<T, UTF>(sm, ring, ringsize - 1, F, ld, K, n, io1);
  SweepIO io2{nullptr, tmp + s, nullptr, nullptr, z_out + s, nullptr};
  if (!TRANS) sweep<T, UB>(sm, ring, ringsize - 1, F, ld, K, n, io2);
  else sweep<T, LTB>(sm, ring, ringsize - 1, F, ld, K, n, io2);
}

// ---- SaP-C reduced systems (Eq. (2.5)) and purification right-hand sides ----
// One CTA per interface i, FP64 arithmetic (tips upcast from T):
//   rhs = g^(t)_{i+1} - W^(t)_{i+1} g^(b)_i,  xt = Rbar_i^{-1} rhs,
//   xb = g^(b)_i - V^(b)_i xt,
//   cbot_i = B_i xt       (subtracted from the bottom K rows of block i)
//   ctop_i = C_{i+1} xb   (subtracted from the top K rows of block i+1)
// For the adjoint SaP (A^T): B'_i = C_{i+1}^T, C'_{i+1} = B_i^T.
// Rbar_i^{-1} is formed once in the factor phase from its GEPP factors.
template <typename M>
__device__ __forceinline__ double rowdot(const M* __restrict__ a, const double* x, int K) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int q = 0;
  for (; q + 3 < K; q += 4) {
    s0 += (double)a[q] * x[q];
    s1 += (double)a[q + 1] * x[q + 1];
    s2 += (double)a[q + 2] * x[q + 2];
    s3 += (double)a[q + 3] * x[q + 3];
  }
  for (; q < K; ++q) s0 += (double)a[q] * x[q];
  return (s0 + s1) + (s2 + s3);
}

template <typename T, bool TRANS>
__global__ void k_reduced(const double* __restrict__ band, int64_t N, int K, Dev d,
                          const T* __restrict__ V, const T* __restrict__ Wt, const double* __restrict__ Rinv,
                          const double* __restrict__ g, double* __restrict__ ctop, double* __restrict__ cbot) {
  extern __shared__ __align__(16) double sh[];
  double* gb = sh;           // K
  double* gt = gb + K;       // K
  double* xt = gt + K;       // K
  double* xb = xt + K;       // K
  double* rhs = xb + K;      // K
  const int i = blockIdx.x;
  const int64_t s = d.off[i + 1];
  const int64_t KK = (int64_t)K * K;
  const T* Vi = V + i * KK;
  const T* Wi = Wt + i * KK;
  const double* Ri = Rinv + i * KK;
  for (int t = threadIdx.x; t < K; t += blockDim.x) {
    gb[t] = g[s - K + t];
    gt[t] = g[s + t];
  }
  __syncthreads();
  for (int r = threadIdx.x; r < K; r += blockDim.x) rhs[r] = gt[r] - rowdot(Wi + r * K, gb, K);
  __syncthreads();
  for (int r = threadIdx.x; r < K; r += blockDim.x) xt[r] = rowdot(Ri + r * K, rhs, K);
  __syncthreads();
  for (int r = threadIdx.x; r < K; r += blockDim.x) xb[r] = gb[r] - rowdot(Vi + r * K, xt, K);
  __syncthreads();
  // corrections.  B_i(r, c) = a(s-K+r, s+c) = band[(r-c) N + s+c], c <= r
  //               C_{i+1}(r, c) = a(s+r, s-K+c) = band[(2K+r-c) N + s-K+c], c >= r
  for (int r = threadIdx.x; r < K; r += blockDim.x) {
    double accb = 0.0, accc = 0.0;
    if (!TRANS) {
      for (int c = 0; c <= r; ++c) accb += band[(int64_t)(r - c) * N + s + c] * xt[c];
      for (int c = r; c < K; ++c) accc += band[(int64_t)(2 * K + r - c) * N + s - K + c] * xb[c];
    } else {
      // B'_i = C_{i+1}^T: B'(r, c) = C(c, r), nonzero for c <= r
      for (int c = 0; c <= r; ++c) accb += band[(int64_t)(2 * K + c - r) * N + s - K + r] * xt[c];
      // C'_{i+1} = B_i^T: C'(r, c) = B(c, r), nonzero for c >= r
      for (int c = r; c < K; ++c) accc += band[(int64_t)(c - r) * N + s + r] * xb[c];
    }
    cbot[(int64_t)i * K + r] = accb;
    ctop[(int64_t)i * K + r] = accc;
  }
}

template <typename T>
size_t sweep_smem(int K, int* ringsize) {
  int ring = 64;
  while (ring < K + 2 * CHK + 32) ring <<= 1;
  *ringsize = ring;
  return sizeof(SweepSmem<T>) + ring * sizeof(T);
}

template <typename T, bool TRANS>
cudaError_t launch_block_solve(const T* F, int K, int P, Dev d, const double* r, double* z, T* tmp,
                               const double* ctop, const double* cbot, cudaStream_t s) {
  int ring;
  size_t smem = sweep_smem<T>(K, &ring);
  auto kern = k_block_solve<T, TRANS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  count_launches(1);
  kern<<<P, NW * 32, smem, s>>>(F, K, d, r, z, tmp, ctop, cbot, P, ring);
  return cudaGetLastError();
}

}  // namespace

// scratch layout (doubles): [0, N) g ; then T tmp (N); then ctop, cbot ((P-1) K each)
template <typename T>
cudaError_t launch_apply(const double* band, int64_t N, int K, int P, Dev d, const Factors<T>& f,
                         int variant, bool transpose, const double* r, double* z, double* scratch,
                         cudaStream_t s) {
  double* g = scratch;
  T* tmp = reinterpret_cast<T*>(scratch + N);
  double* ctop = scratch + 2 * N;
  double* cbot = ctop + (int64_t)(P > 1 ? P - 1 : 1) * K;
  cudaError_t e;
  if (variant == SAP_D || P == 1) {
    return transpose ? launch_block_solve<T, true>(f.F, K, P, d, r, z, tmp, nullptr, nullptr, s)
                     : launch_block_solve<T, false>(f.F, K, P, d, r, z, tmp, nullptr, nullptr, s);
  }
  e = transpose ? launch_block_solve<T, true>(f.F, K, P, d, r, g, tmp, nullptr, nullptr, s)
                : launch_block_solve<T, false>(f.F, K, P, d, r, g, tmp, nullptr, nullptr, s);
  if (e != cudaSuccess) return e;
  size_t sm = 5 * (size_t)K * sizeof(double);
  count_launches(1);
  if (!transpose)
    k_reduced<T, false><<<P - 1, 128, sm, s>>>(band, N, K, d, f.V, f.Wt, f.R, g, ctop, cbot);
  else
    k_reduced<T, true><<<P - 1, 128, sm, s>>>(band, N, K, d, f.Va, f.Wa, f.Ra, g, ctop, cbot);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return transpose ? launch_block_solve<T, true>(f.F, K, P, d, r, z, tmp, ctop, cbot, s)
                   : launch_block_solve<T, false>(f.F, K, P, d, r, z, tmp, ctop, cbot, s);
}

template cudaError_t launch_apply<float>(const double*, int64_t, int, int, Dev, const Factors<float>&, int, bool,
                                         const double*, double*, double*, cudaStream_t);
template cudaError_t launch_apply<double>(const double*, int64_t, int, int, Dev, const Factors<double>&, int,
                                          bool, const double*, double*, double*, cudaStream_t);

}  // namespace sap
