// Banded LU / UL factorisation of the diagonal blocks A_i without pivoting,
// with pivot boosting (Sec. 2.2, Sec. 3.1 "LU/UL factorizations").
//
// One CTA factors one block.  The active (K+1) x (K+1) window of the
// right-looking elimination lives in registers: a 16 x 16 thread grid, each
// thread owning R x R fixed *physical* window slots (rows ty + 16 y,
// columns tx + 16 x).  Window rows and columns are addressed modulo
// M = K + 1, so sliding the window by one step only replaces the physical
// row and column of the pivot; no data moves.  Per step k:
//   1. read the pivot row/column (published in shared memory by their
//      owners at the end of step k-1), boost the pivot, 1/p;
//   2. rank-1 update of every owned slot outside the pivot row/column;
//   3. write L(:,k) and U(k,:) (LU) or the last K rows/columns (UL) out;
//   4. reload the pivot's physical row/column with the entering band row
//      k+K+1 / column k+K+1 (pristine entries of A, prefetched into a
//      shared-memory ring by cp.async one chunk of steps ahead);
//   5. publish the next pivot row/column; one __syncthreads.
// The UL factorisation is the same elimination run on the reversed block
// J A_i J: if J A_i J = L~ U~ (unit L~) then A_i = (J L~ J)(J U~ J) = U' L'
// with unit upper U'.  Only the last K rows/columns of L~, U~ are kept,
// flipped back into the top K x K tiles of U' and L'.
#include <cuda_runtime.h>
#include <cstdint>
#include "sap_internal.cuh"

namespace sap {

namespace {

constexpr int TDIM = 16;           // thread grid is TDIM x TDIM
constexpr int NTHREADS = TDIM * TDIM;
constexpr int CH = 16;             // steps per prefetch chunk
constexpr int NSTAGE = 2 * CH;     // ring of two chunks

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Entries of the block in local coordinates (r, q), reversed when REV.
// Returns a pointer into the band, or nullptr for a structural zero.
template <bool REV>
__device__ __forceinline__ const double* elem_ptr(const double* band, int64_t N, int K, int64_t s,
                                                  int64_t n, int64_t r, int64_t q) {
  if (r < 0 || q < 0 || r >= n || q >= n) return nullptr;
  int64_t gi = REV ? s + n - 1 - r : s + r;
  int64_t gj = REV ? s + n - 1 - q : s + q;
  int64_t c = (int64_t)K + gi - gj;
  if (c < 0 || c > 2 * (int64_t)K) return nullptr;
  return band + c * N + gj;
}

// Prefetch the entering row / column of steps [k0, k0 + CH) into ring slots.
// For step k the entering row is r = k + M with columns q = k+1+m (m < M),
// the entering column is q = k + M with rows r = k+1+m (m < M-1).
template <bool REV>
__device__ __forceinline__ void prefetch_chunk(double* stage, int Mp, const double* band, int64_t N,
                                               int K, int64_t s, int64_t n, int64_t k0) {
  const int M = K + 1;
  const int total = CH * (2 * M);
  for (int e = threadIdx.x; e < total; e += NTHREADS) {
    int kk = e % CH;
    int t = e / CH;           // 0..2M-1
    int which = t / M;        // 0 = row, 1 = column
    int m = t % M;
    int64_t k = k0 + kk;
    double* dst = stage + ((size_t)((k % NSTAGE) * 2 + which) * Mp + m);
    const double* src = nullptr;
    if (which == 0) src = elem_ptr<REV>(band, N, K, s, n, k + M, k + 1 + m);
    else if (m < M - 1) src = elem_ptr<REV>(band, N, K, s, n, k + 1 + m, k + M);
    if (src) cp_async8(dst, src);
    else *dst = 0.0;
  }
  cp_async_commit();
}

template <typename T, int R, bool REV>
__global__ void __launch_bounds__(NTHREADS)
k_band_lu(const double* __restrict__ band, int64_t N, int K, Dev d, int block0,
          const double* __restrict__ absmax, double eps, T* __restrict__ out,
          unsigned long long* __restrict__ n_boosted) {
  extern __shared__ __align__(16) double stage[];   // [NSTAGE][2][Mp]
  __shared__ T colbuf[2][TDIM * R];
  __shared__ T rowbuf[2][TDIM * R];

  const int b = block0 + blockIdx.x;
  const int64_t s = d.off[b];
  const int64_t n = d.off[b + 1] - s;
  const int M = K + 1;
  const int Mp = (M + 1) & ~1;
  const int tx = threadIdx.x % TDIM, ty = threadIdx.x / TDIM;
  const T tau = (T)(eps * absmax[0]);
  unsigned long long nb = 0;

  // output addressing
  const int64_t ld = REV ? 0 : d.ld[b];
  T* F = REV ? out + (int64_t)(b - 1) * K * K : out + d.fbase[b];

  // initial window: rows/cols 0..K, physical == logical
  T a[R][R];
#pragma unroll
  for (int y = 0; y < R; ++y)
#pragma unroll
    for (int x = 0; x < R; ++x) {
      int pr = ty + TDIM * y, pc = tx + TDIM * x;
      const double* p = (pr < M && pc < M) ? elem_ptr<REV>(band, N, K, s, n, pr, pc) : nullptr;
      a[y][x] = p ? (T)(*p) : T(0);
      if (pr < M && pc == 0) colbuf[0][pr] = a[y][x];
      if (pc < M && pr == 0) rowbuf[0][pc] = a[y][x];
    }
  prefetch_chunk<REV>(stage, Mp, band, N, K, s, n, 0);
  cp_async_wait_all();
  __syncthreads();

  int pk = 0;  // physical index of the pivot row/column (k mod M)
  for (int64_t k = 0; k < n; ++k) {
    if (k % CH == 0 && k + CH < n) prefetch_chunk<REV>(stage, Mp, band, N, K, s, n, k + CH);
    const T* cb = colbuf[k & 1];
    const T* rb = rowbuf[k & 1];
    T p = rb[pk];
    if ((p < T(0) ? -p : p) < tau) {
      p = p >= T(0) ? tau : -tau;
      ++nb;
    }
    const T rinv = T(1) / p;
    const int pk1 = (pk + 1 == M) ? 0 : pk + 1;

    T l[R], u[R];
#pragma unroll
    for (int y = 0; y < R; ++y) {
      int pr = ty + TDIM * y;
      l[y] = (pr < M && pr != pk) ? cb[pr] * rinv : T(0);
    }
#pragma unroll
    for (int x = 0; x < R; ++x) {
      int pc = tx + TDIM * x;
      u[x] = (pc < M && pc != pk) ? rb[pc] : T(0);
    }
#pragma unroll
    for (int y = 0; y < R; ++y)
#pragma unroll
      for (int x = 0; x < R; ++x) a[y][x] -= l[y] * u[x];

    // ---- outputs of step k ----
    if (!REV) {
      if (tx == 0) {
#pragma unroll
        for (int y = 0; y < R; ++y) {
          int pr = ty + TDIM * y;
          if (pr < M && pr != pk) {
            int off = pr - pk; if (off < 0) off += M;      // logical row = k + off
            if (k + off < n) F[(int64_t)(K + off) * ld + k] = l[y];
          }
        }
      }
      if (ty == 0) {
#pragma unroll
        for (int x = 0; x < R; ++x) {
          int pc = tx + TDIM * x;
          if (pc < M) {
            int off = pc - pk; if (off < 0) off += M;      // logical col = k + off
            if (k + off < n) F[(int64_t)(K - off) * ld + k + off] = (off == 0) ? p : rb[pc];
          }
        }
      }
    } else if (k >= n - K) {
      // keep the last K rows/cols of L~ and U~ of J A J, flipped:
      // U'(n-1-i, n-1-k) = L~(i, k), L'(n-1-k, n-1-j) = U~(k, j)
      if (tx == 0) {
#pragma unroll
        for (int y = 0; y < R; ++y) {
          int pr = ty + TDIM * y;
          if (pr < M && pr != pk) {
            int off = pr - pk; if (off < 0) off += M;
            int64_t i = k + off;
            if (i < n) F[(n - 1 - i) * K + (n - 1 - k)] = l[y];
          }
        }
      }
      if (ty == 0) {
#pragma unroll
        for (int x = 0; x < R; ++x) {
          int pc = tx + TDIM * x;
          if (pc < M) {
            int off = pc - pk; if (off < 0) off += M;
            int64_t j = k + off;
            if (j < n) F[(n - 1 - k) * K + (n - 1 - j)] = (off == 0) ? p : rb[pc];
          }
        }
      }
    }

    // ---- chunk boundary: the next chunk must have landed ----
    const double* st = stage + (size_t)((k % NSTAGE) * 2) * Mp;
    // ---- reload the pivot's physical row / column with entering data ----
#pragma unroll
    for (int y = 0; y < R; ++y) {
      int pr = ty + TDIM * y;
      if (pr >= M) continue;
#pragma unroll
      for (int x = 0; x < R; ++x) {
        int pc = tx + TDIM * x;
        if (pc >= M) continue;
        if (pr == pk) {          // entering row k+M, column logical k+1+m
          int m = pc - pk1; if (m < 0) m += M;
          a[y][x] = (T)st[m];
        } else if (pc == pk) {   // entering column k+M, row logical k+1+m
          int m = pr - pk1; if (m < 0) m += M;
          a[y][x] = (T)st[Mp + m];
        }
      }
    }
    // ---- publish pivot row / column of step k+1 ----
    T* ncb = colbuf[(k + 1) & 1];
    T* nrb = rowbuf[(k + 1) & 1];
#pragma unroll
    for (int y = 0; y < R; ++y)
#pragma unroll
      for (int x = 0; x < R; ++x) {
        int pr = ty + TDIM * y, pc = tx + TDIM * x;
        if (pr < M && pc == pk1) ncb[pr] = a[y][x];
        if (pc < M && pr == pk1) nrb[pc] = a[y][x];
      }
    if ((k + 1) % CH == 0) cp_async_wait_all();
    __syncthreads();
    pk = pk1;
  }
  if (threadIdx.x == 0 && nb) atomicAdd(n_boosted, nb);
}

template <typename T, bool REV>
cudaError_t launch_lu_impl(const double* band, int64_t N, int K, int nblocks, int block0, Dev d,
                           const double* absmax, double eps, T* out, unsigned long long* nb,
                           cudaStream_t s) {
  if (nblocks <= 0) return cudaSuccess;
  const int M = K + 1;
  const int Mp = (M + 1) & ~1;
  size_t smem = (size_t)NSTAGE * 2 * Mp * sizeof(double);
  int R = (M <= 16) ? 1 : (M <= 32) ? 2 : (M <= 64) ? 4 : 8;
  cudaError_t e = cudaSuccess;
#define SAP_LAUNCH_LU(RR)                                                                           \
  do {                                                                                              \
    auto kern = k_band_lu<T, RR, REV>;                                                             \
    if (smem > 48 * 1024) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    if (e != cudaSuccess) return e;                                                                 \
    count_launches(1);                                                                             \
    kern<<<nblocks, NTHREADS, smem, s>>>(band, N, K, d, block0, absmax, eps, out, nb);             \
  } while (0)
  switch (R) {
    case 1: SAP_LAUNCH_LU(1); break;
    case 2: SAP_LAUNCH_LU(2); break;
    case 4: SAP_LAUNCH_LU(4); break;
    default: SAP_LAUNCH_LU(8); break;
  }
#undef SAP_LAUNCH_LU
  return cudaGetLastError();
}

// ---- max |a_ij| over the in-band entries (boost threshold scale) ----
__global__ void k_absmax(const double* __restrict__ band, int64_t N, int K, double* out) {
  const int64_t total = (int64_t)(2 * K + 1) * N;
  double m = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t c = e / N, j = e - c * N;
    int64_t i = j + c - K;
    if (i >= 0 && i < N) m = fmax(m, fabs(band[e]));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0)
    atomicMax(reinterpret_cast<unsigned long long*>(out), (unsigned long long)__double_as_longlong(m));
}

}  // namespace

cudaError_t launch_absmax(const double* band, int64_t N, int K, double* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  count_launches(1);
  k_absmax<<<152 * 4, 256, 0, s>>>(band, N, K, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_factor_lu(const double* band, int64_t N, int K, int P, Dev d, const double* absmax,
                             double eps, T* F, unsigned long long* nb, cudaStream_t s) {
  return launch_lu_impl<T, false>(band, N, K, P, 0, d, absmax, eps, F, nb, s);
}

template <typename T>
cudaError_t launch_factor_ul(const double* band, int64_t N, int K, int P, Dev d, const double* absmax,
                             double eps, T* ULt, unsigned long long* nb, cudaStream_t s) {
  // UL tiles are only needed for blocks 1..P-1 (the W^(t) tips)
  return launch_lu_impl<T, true>(band, N, K, P - 1, 1, d, absmax, eps, ULt, nb, s);
}

template cudaError_t launch_factor_lu<float>(const double*, int64_t, int, int, Dev, const double*, double,
                                             float*, unsigned long long*, cudaStream_t);
template cudaError_t launch_factor_lu<double>(const double*, int64_t, int, int, Dev, const double*, double,
                                              double*, unsigned long long*, cudaStream_t);
template cudaError_t launch_factor_ul<float>(const double*, int64_t, int, int, Dev, const double*, double,
                                             float*, unsigned long long*, cudaStream_t);
template cudaError_t launch_factor_ul<double>(const double*, int64_t, int, int, Dev, const double*, double,
                                              double*, unsigned long long*, cudaStream_t);

}  // namespace sap
