// SaP with a bandwidth of its own per block (Sec. 2.2, third-stage
// reordering).  Every block A_i of the partition is renumbered on its own,
// Ahat_i = Pi_i A_i Pi_i^T (half-bandwidth K_i), and factored as a banded
// matrix of its own; the coupling blocks B_i, C_{i+1} keep their places in the
// global numbering, so in a block's new numbering the rows they touch are
// spread over the block and SaP-C needs the entire spikes (Sec. 3.1, use of
// registers and shared memory):
//   Vhat_i     = Ahat_i^{-1}     Pi_i     [0; B_i]       (n_i x K)
//   What_{i+1} = Ahat_{i+1}^{-1} Pi_{i+1} [C_{i+1}; 0]   (n_{i+1} x K)
// whose rows at the interface (old bottom K rows of block i, old top K rows
// of block i+1) are the tips V^(b)_i, W^(t)_{i+1} of Eq. (2.5a).
// Kernels: per-block bandwidth, the reordered blocks gathered from the band,
// the permutations of vectors, the entire spikes (forward and backward banded
// sweeps over L-row groups, the group's values in registers, Sec. 3.1), and
// the two steps of the apply after the block solves: the truncated reduced
// solve (Eq. (2.5b,c)) and z_i = g_i - Vhat_i x^(t)_{i+1} - What_i x^(b)_{i-1}
// (= A_i^{-1}(r_i - [C_i x^(b)_{i-1}; 0] - [0; B_i x^(t)_{i+1}]) by linearity).
#include <cuda_runtime.h>
#include <algorithm>
#include <cstdint>
#include "sap_internal.cuh"

namespace sap {

namespace {

constexpr int kGridStride = 152 * 8;   // CTAs of the grid-stride kernels

__device__ __forceinline__ int block_of(const BlockMap& m, int64_t g) {
  const int64_t big = m.pr * (m.q + 1);
  return g < big ? (int)(g / (m.q + 1)) : (int)(m.pr + (g - big) / m.q);
}

// Half-bandwidth of every reordered block: max |perm(i) - perm(j)| over the
// nonzero band entries (i, j) with both indices in one block (one atomic per
// warp and block).
__global__ void __launch_bounds__(256) k_block_bw(const double* __restrict__ band, BlockMap m, int* __restrict__ Kout) {
  const int64_t total = (int64_t)(2 * m.K + 1) * m.N;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < total; base += stride) {
    const int64_t e = base + threadIdx.x;
    int b = -1, d = 0;
    if (e < total) {
      const int c = (int)(e / m.N);
      const int64_t j = e - (int64_t)c * m.N;
      const int64_t i = j + c - m.K;
      if (c != m.K && i >= 0 && i < m.N && band[e] != 0.0) {
        const int bi = block_of(m, i), bj = block_of(m, j);
        if (bi == bj) {
          b = bi;
          d = abs(m.perm[i] - m.perm[j]);
        }
      }
    }
    const unsigned grp = __match_any_sync(0xffffffffu, b);
    const int mx = __reduce_max_sync(grp, d);
    if (b >= 0 && (int)(threadIdx.x & 31) == __ffs(grp) - 1) atomicMax(Kout + b, mx);
  }
}

// The reordered blocks in the band storage of sap.h, each of its own
// half-bandwidth: entry (a, c) of block b (local indices) goes to
// hb[hbase_b + (K_b + perm(a) - perm(c)) n_b + perm(c)].  The caller zeroes
// hb first; an entry beyond K_b (a pattern that changed since the bandwidths
// were taken) sets *err.
__global__ void __launch_bounds__(256) k_block_gather(const double* __restrict__ band, BlockMap m, double* __restrict__ hb,
                                                      int* __restrict__ err) {
  const int64_t total = (int64_t)(2 * m.K + 1) * m.N;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
    const int c = (int)(e / m.N);
    const int64_t j = e - (int64_t)c * m.N;
    const int64_t i = j + c - m.K;
    if (i < 0 || i >= m.N) continue;
    const double v = band[e];
    if (v == 0.0) continue;
    const int bi = block_of(m, i);
    if (bi != block_of(m, j)) continue;
    const int64_t n = m.off[bi + 1] - m.off[bi];
    const int Kb = m.Kb[bi];
    const int pa = m.perm[i], pc = m.perm[j];
    const int dd = pa - pc;
    if (dd > Kb || dd < -Kb) {
      atomicExch(err, 1);
      continue;
    }
    hb[m.hbase[bi] + (int64_t)(Kb + dd) * n + pc] = v;
  }
}

// to_new: y[off_b + perm(g)] = x[g]; else y[g] = x[off_b + perm(g)].
__global__ void __launch_bounds__(256) k_block_perm(BlockMap m, const double* __restrict__ x, double* __restrict__ y,
                                                    int to_new, Gate gt) {
  if (gate_skip(gt)) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < m.N; g += stride) {
    const int64_t p = m.off[block_of(m, g)] + m.perm[g];
    if (to_new) y[p] = x[g];
    else y[g] = x[p];
  }
}

__device__ __forceinline__ void cp_async_elem(void* dst, const void* src, bool valid, int bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int sz = valid ? bytes : 0;          // 0: the destination is zero-filled
  if (bytes == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(sz));
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(sz));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

constexpr int kSpkRows = 16;   // L: rows per group of the spike sweeps (Sec. 3.1: at most 20)

// Shared-memory row stride of the history ring: CPB columns plus a pad that
// puts the TPC threads of a column (consecutive lanes, consecutive ring rows)
// and the columns of a warp on distinct banks.
template <typename T, int CPB, int TPC>
__host__ __device__ constexpr int ring_stride() {
  return CPB + (sizeof(T) == 4 ? 32 / TPC : 16 / TPC);
}

// Entire spikes of interface i (blockIdx.z): side 0 (blockIdx.y) Vhat_i of
// block i, side 1 What_{i+1} of block i+1; CPB right-hand-side columns per
// CTA (blockIdx.x), TPC threads per column.  Forward sweep L y = Pi rhs over
// groups of L = kSpkRows rows from the first row with a nonzero right-hand
// side: the group's L values of the column are accumulated in registers
// (each thread a strided share of the K_b rows of history from the ring in
// shared memory, summed over the column's threads by shuffles), then the
// group's own unit-lower triangle in registers; backward sweep U x = y over
// groups from the last row the same way, dividing by the diagonal.  The
// factor coefficients a group needs (K_b x L, plus the diagonal) are staged
// in shared memory by cp.async, the next group's while the current one is
// computed (double buffer).  Then the tip rows are copied out.
template <typename T, int CPB, int TPC>
__global__ void __launch_bounds__(CPB * TPC)
k_full_spikes(const double* __restrict__ band, BlockMap m, int R, int CWmax, const void* const* __restrict__ Fp,
              const int64_t* __restrict__ ldp, T* __restrict__ spk, const int64_t* __restrict__ sbase,
              T* __restrict__ Vtip, T* __restrict__ Wtip) {
  constexpr int NT = CPB * TPC;
  constexpr int LR = kSpkRows;
  constexpr int RS = ring_stride<T, CPB, TPC>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ring = reinterpret_cast<T*>(smem_raw);              // R x RS: values of the last rows, by row mod R
  T* Cb = ring + (size_t)R * RS;                          // 2 x (LR x CWmax) group coefficients
  T* Db = Cb + 2 * LR * CWmax;                            // 2 x LR diagonal entries (backward)
  __shared__ int rmin_s;
  const int i = blockIdx.z, side = blockIdx.y;
  const int b = i + side;
  const int64_t s0 = m.off[b];
  const int n = (int)(m.off[b + 1] - s0);
  const int Kb = m.Kb[b];
  const int K = m.K;
  const int64_t N = m.N;
  const int CW = Kb + LR;
  const T* F = static_cast<const T*>(Fp[b]);
  const int64_t ld = ldp[b];
  const int64_t sif = m.off[i + 1];
  const int tid = threadIdx.x, cl = tid / TPC, part = tid % TPC;
  const int col = blockIdx.x * CPB + cl;
  const bool colok = col < K;
  T* out = spk + sbase[2 * i + side];

  for (int e = tid; e < R * RS; e += NT) ring[e] = T(0);
  for (int e = tid; e < 2 * LR * CWmax; e += NT) Cb[e] = T(0);
  if (tid == 0) rmin_s = n;
  __syncthreads();
  {
    int loc = n;
    for (int r = tid; r < K; r += NT) loc = min(loc, m.perm[s0 + (side == 0 ? n - K + r : r)]);
    atomicMin(&rmin_s, loc);
  }
  __syncthreads();
  const int rstart = rmin_s / LR * LR;

  // right-hand side of new row r in this thread's column: [0; B_i] or [C_{i+1}; 0]
  auto rhs = [&](int r) -> T {
    const int a = m.pinv[s0 + r];
    double v = 0.0;
    if (side == 0) {
      const int rr = a - (n - K);                       // B_i(rr, col) = a(sif - K + rr, sif + col)
      if (rr >= 0 && col <= rr) v = band[(int64_t)(rr - col) * N + sif + col];
    } else if (a < K && col >= a) {                     // C_{i+1}(a, col) = a(sif + a, sif - K + col)
      v = band[(int64_t)(2 * K + a - col) * N + sif - K + col];
    }
    return (T)v;
  };
  // coefficients of the forward group at r0: C[l][Kb + l - d] = L(r0 + l, r0 + l - d), d = 1..Kb
  auto stage_fwd = [&](int r0, T* C) {
    for (int e = tid; e < Kb * LR; e += NT) {
      const int d = 1 + e / LR, l = e % LR;
      const int r = r0 + l, q = r - d;
      const bool ok = r < n && q >= 0;
      cp_async_elem(C + l * CW + (Kb + l - d), ok ? (const void*)(F + (int64_t)(Kb + d) * ld + q) : (const void*)F, ok,
                    (int)sizeof(T));
    }
    cp_async_commit();
  };
  // backward group at reverse index u0 (rows r = n - 1 - u0 - l): C[l][Kb + l - e] = U(r, r + e), D[l] = U(r, r)
  auto stage_bwd = [&](int u0, T* C, T* D) {
    for (int e = tid; e < Kb * LR; e += NT) {
      const int dd = 1 + e / LR, l = e % LR;
      const int r = n - 1 - (u0 + l), q = r + dd;
      const bool ok = r >= 0 && q < n;
      cp_async_elem(C + l * CW + (Kb + l - dd), ok ? (const void*)(F + (int64_t)(Kb - dd) * ld + q) : (const void*)F,
                    ok, (int)sizeof(T));
    }
    for (int l = tid; l < LR; l += NT) {
      const int r = n - 1 - (u0 + l);
      const bool ok = r >= 0;
      cp_async_elem(D + l, ok ? (const void*)(F + (int64_t)Kb * ld + r) : (const void*)F, ok, (int)sizeof(T));
    }
    cp_async_commit();
  };

  // ---- forward: L y = Pi rhs ----
  int buf = 0;
  if (rstart < n) stage_fwd(rstart, Cb);
  for (int r0 = rstart; r0 < n; r0 += LR) {
    cp_async_wait_all();
    __syncthreads();                                     // this group's coefficients; the ring's last rows
    const T* C = Cb + buf * LR * CWmax;
    if (r0 + LR < n) stage_fwd(r0 + LR, Cb + (buf ^ 1) * LR * CWmax);
    T acc[LR];
#pragma unroll
    for (int l = 0; l < LR; ++l) acc[l] = (part == 0 && colok && r0 + l < n) ? rhs(r0 + l) : T(0);
    for (int t = part; t < Kb; t += TPC) {
      const T y = ring[((r0 - Kb + t) & (R - 1)) * RS + cl];
#pragma unroll
      for (int l = 0; l < LR; ++l) acc[l] -= C[l * CW + t] * y;
    }
#pragma unroll
    for (int l = 0; l < LR; ++l)
#pragma unroll
      for (int o = TPC / 2; o > 0; o >>= 1) acc[l] += __shfl_xor_sync(0xffffffffu, acc[l], o);
#pragma unroll
    for (int l = 1; l < LR; ++l)
#pragma unroll
      for (int k = 0; k < l; ++k) acc[l] -= C[l * CW + Kb + k] * acc[k];
#pragma unroll
    for (int l = 0; l < LR; ++l)
      if (l % TPC == part && r0 + l < n) {
        ring[((r0 + l) & (R - 1)) * RS + cl] = acc[l];
        if (colok) out[(int64_t)(r0 + l) * K + col] = acc[l];
      }
    buf ^= 1;
  }
  cp_async_wait_all();
  __syncthreads();
  for (int e = tid; e < R * RS; e += NT) ring[e] = T(0);
  __syncthreads();

  // ---- backward: U x = y (reverse index u = n - 1 - r) ----
  buf = 0;
  stage_bwd(0, Cb, Db);
  for (int u0 = 0; u0 < n; u0 += LR) {
    cp_async_wait_all();
    __syncthreads();
    const T* C = Cb + buf * LR * CWmax;
    const T* D = Db + buf * LR;
    if (u0 + LR < n) stage_bwd(u0 + LR, Cb + (buf ^ 1) * LR * CWmax, Db + (buf ^ 1) * LR);
    T acc[LR];
#pragma unroll
    for (int l = 0; l < LR; ++l) {
      const int r = n - 1 - (u0 + l);
      acc[l] = (part == 0 && colok && r >= rstart) ? out[(int64_t)r * K + col] : T(0);
    }
    for (int t = part; t < Kb; t += TPC) {
      const T x = ring[((u0 - Kb + t) & (R - 1)) * RS + cl];
#pragma unroll
      for (int l = 0; l < LR; ++l) acc[l] -= C[l * CW + t] * x;
    }
#pragma unroll
    for (int l = 0; l < LR; ++l)
#pragma unroll
      for (int o = TPC / 2; o > 0; o >>= 1) acc[l] += __shfl_xor_sync(0xffffffffu, acc[l], o);
#pragma unroll
    for (int l = 0; l < LR; ++l) {
#pragma unroll
      for (int k = 0; k < l; ++k) acc[l] -= C[l * CW + Kb + k] * acc[k];
      acc[l] = acc[l] / D[l];
    }
#pragma unroll
    for (int l = 0; l < LR; ++l) {
      const int r = n - 1 - (u0 + l);
      if (l % TPC == part && r >= 0) {
        ring[((u0 + l) & (R - 1)) * RS + cl] = acc[l];
        if (colok) out[(int64_t)r * K + col] = acc[l];
      }
    }
    buf ^= 1;
  }
  cp_async_wait_all();
  __syncthreads();
  // tips: the spike rows of the old interface rows
  T* tip = (side == 0 ? Vtip : Wtip) + (int64_t)i * K * K;
  for (int e = tid; e < K * CPB; e += NT) {
    const int rr = e / CPB, c2 = blockIdx.x * CPB + e % CPB;
    if (c2 < K) {
      const int a = side == 0 ? n - K + rr : rr;
      tip[(int64_t)rr * K + c2] = out[(int64_t)m.perm[s0 + a] * K + c2];
    }
  }
}

// Truncated reduced solve of every interface (Eq. (2.5b,c)) on g = D^{-1} r
// held in the blocks' new numbering: g^(b)_i, g^(t)_{i+1} gathered through the
// permutations, x^(t)_{i+1} = Rbar_i^{-1} (g^(t)_{i+1} - W^(t)_{i+1} g^(b)_i),
// x^(b)_i = g^(b)_i - V^(b)_i x^(t)_{i+1}.  One CTA per interface, a warp per
// row of each K x K product.
template <typename T>
__global__ void __launch_bounds__(256)
k_block_reduced(BlockMap m, const double* __restrict__ gh, const T* __restrict__ V, const T* __restrict__ Wt,
                const double* __restrict__ Rinv, double* __restrict__ xt, double* __restrict__ xb, Gate gt) {
  if (gate_skip(gt)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int K = m.K;
  double* gb = reinterpret_cast<double*>(smem_raw);
  double* gtv = gb + K;
  double* rhs = gtv + K;
  const int i = blockIdx.x;
  const int64_t s0 = m.off[i], s1 = m.off[i + 1];
  const int n0 = (int)(s1 - s0);
  const int64_t KK = (int64_t)K * K;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int r = threadIdx.x; r < K; r += blockDim.x) {
    gb[r] = gh[s0 + m.perm[s0 + n0 - K + r]];
    gtv[r] = gh[s1 + m.perm[s1 + r]];
  }
  __syncthreads();
  auto rowdot = [&](const T* Mr, const double* v) {
    double a = 0.0;
    for (int k = lane; k < K; k += 32) a += (double)Mr[k] * v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    return a;
  };
  for (int r = w; r < K; r += 8) {
    const double a = rowdot(Wt + i * KK + (int64_t)r * K, gb);
    if (lane == 0) rhs[r] = gtv[r] - a;
  }
  __syncthreads();
  for (int r = w; r < K; r += 8) {
    const double* Rr = Rinv + i * KK + (int64_t)r * K;
    double a = 0.0;
    for (int k = lane; k < K; k += 32) a += Rr[k] * rhs[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) {
      gtv[r] = a;                                        // x^(t)_{i+1}
      xt[(int64_t)i * K + r] = a;
    }
  }
  __syncthreads();
  for (int r = w; r < K; r += 8) {
    const double a = rowdot(V + i * KK + (int64_t)r * K, gtv);
    if (lane == 0) xb[(int64_t)i * K + r] = gb[r] - a;
  }
}

// z[off_b + pinv(r)] = g[off_b + r] - Vhat_b[r] . x^(t)_{b+1} - What_b[r] . x^(b)_{b-1}
// for every new row r of every block b: a warp per row.
template <typename T>
__global__ void __launch_bounds__(256)
k_block_correct(BlockMap m, const double* __restrict__ gh, const T* __restrict__ spk, const int64_t* __restrict__ sbase,
                const double* __restrict__ xt, const double* __restrict__ xb, double* __restrict__ z, Gate gt) {
  if (gate_skip(gt)) return;
  const int K = m.K;
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t G = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); G < m.N; G += nw) {
    const int b = block_of(m, G);
    const int64_t s = m.off[b];
    const int64_t r = G - s;
    double a = 0.0;
    if (b < m.P - 1) {
      const T* v = spk + sbase[2 * b] + r * K;
      const double* x = xt + (int64_t)b * K;
      for (int k = lane; k < K; k += 32) a += (double)v[k] * x[k];
    }
    if (b > 0) {
      const T* v = spk + sbase[2 * (b - 1) + 1] + r * K;
      const double* x = xb + (int64_t)(b - 1) * K;
      for (int k = lane; k < K; k += 32) a += (double)v[k] * x[k];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) z[s + m.pinv[G]] = gh[G] - a;
  }
}

int pow2_at_least(int x) {
  int r = 1;
  while (r < x) r <<= 1;
  return r;
}

template <typename T, int CPB, int TPC>
size_t spikes_smem(int R, int CWmax) {
  return ((size_t)R * ring_stride<T, CPB, TPC>() + 2 * (size_t)kSpkRows * CWmax + 2 * kSpkRows) * sizeof(T);
}

}  // namespace

cudaError_t launch_block_bw(const double* band, const BlockMap& m, int* Kout, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(Kout, 0, (size_t)m.P * sizeof(int), s);
  if (e != cudaSuccess) return e;
  count_launches(1);
  k_block_bw<<<kGridStride, 256, 0, s>>>(band, m, Kout);
  return cudaGetLastError();
}

cudaError_t launch_block_gather(const double* band, const BlockMap& m, double* hb, int64_t hb_elems, int* err,
                                cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(hb, 0, (size_t)hb_elems * sizeof(double), s);
  if (e != cudaSuccess) return e;
  count_launches(1);
  k_block_gather<<<kGridStride, 256, 0, s>>>(band, m, hb, err);
  return cudaGetLastError();
}

cudaError_t launch_block_perm(const BlockMap& m, const double* x, double* y, bool to_new, cudaStream_t s, Gate gt) {
  count_launches(1);
  const int grid = (int)std::min<int64_t>(kGridStride, (m.N + 255) / 256);
  k_block_perm<<<grid, 256, 0, s>>>(m, x, y, to_new ? 1 : 0, gt);
  return cudaGetLastError();
}

size_t full_spikes_smem(int Kbmax, bool fp64) {
  const int R = pow2_at_least(Kbmax + kSpkRows), CW = Kbmax + kSpkRows;
  if (fp64) {
    const size_t a = spikes_smem<double, 64, 4>(R, CW);
    return a <= kSmemPerBlock ? a : spikes_smem<double, 32, 8>(R, CW);
  }
  const size_t a = spikes_smem<float, 64, 4>(R, CW);
  return a <= kSmemPerBlock ? a : spikes_smem<float, 32, 8>(R, CW);
}

template <typename T>
cudaError_t launch_full_spikes(const double* band, const BlockMap& m, int Kbmax, const void* const* Fp,
                               const int64_t* ldp, T* spk, const int64_t* sbase, T* Vtip, T* Wtip, cudaStream_t s) {
  if (m.P < 2) return cudaSuccess;
  const int R = pow2_at_least(Kbmax + kSpkRows), CW = Kbmax + kSpkRows;
  const size_t wide = spikes_smem<T, 64, 4>(R, CW);
  cudaError_t e;
  count_launches(1);
  if (wide <= kSmemPerBlock) {
    e = cudaFuncSetAttribute(k_full_spikes<T, 64, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wide);
    if (e != cudaSuccess) return e;
    k_full_spikes<T, 64, 4><<<dim3((m.K + 63) / 64, 2, m.P - 1), 256, wide, s>>>(band, m, R, CW, Fp, ldp, spk, sbase,
                                                                                 Vtip, Wtip);
  } else {
    const size_t narrow = spikes_smem<T, 32, 8>(R, CW);
    if (narrow > kSmemPerBlock) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(k_full_spikes<T, 32, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)narrow);
    if (e != cudaSuccess) return e;
    k_full_spikes<T, 32, 8><<<dim3((m.K + 31) / 32, 2, m.P - 1), 256, narrow, s>>>(band, m, R, CW, Fp, ldp, spk,
                                                                                   sbase, Vtip, Wtip);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_block_reduced(const BlockMap& m, const double* gh, const T* V, const T* Wt, const double* Rinv,
                                 double* xt, double* xb, cudaStream_t s, Gate gt) {
  if (m.P < 2) return cudaSuccess;
  const size_t smem = 3 * (size_t)m.K * sizeof(double);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_block_reduced<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  count_launches(1);
  k_block_reduced<T><<<m.P - 1, 256, smem, s>>>(m, gh, V, Wt, Rinv, xt, xb, gt);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_block_correct(const BlockMap& m, const double* gh, const T* spk, const int64_t* sbase,
                                 const double* xt, const double* xb, double* z, cudaStream_t s, Gate gt) {
  count_launches(1);
  const int grid = (int)std::min<int64_t>(kGridStride * 2, (m.N + 7) / 8);
  k_block_correct<T><<<grid, 256, 0, s>>>(m, gh, spk, sbase, xt, xb, z, gt);
  return cudaGetLastError();
}

template cudaError_t launch_full_spikes<float>(const double*, const BlockMap&, int, const void* const*, const int64_t*,
                                               float*, const int64_t*, float*, float*, cudaStream_t);
template cudaError_t launch_full_spikes<double>(const double*, const BlockMap&, int, const void* const*,
                                                const int64_t*, double*, const int64_t*, double*, double*,
                                                cudaStream_t);
template cudaError_t launch_block_reduced<float>(const BlockMap&, const double*, const float*, const float*,
                                                 const double*, double*, double*, cudaStream_t, Gate);
template cudaError_t launch_block_reduced<double>(const BlockMap&, const double*, const double*, const double*,
                                                  const double*, double*, double*, cudaStream_t, Gate);
template cudaError_t launch_block_correct<float>(const BlockMap&, const double*, const float*, const int64_t*,
                                                 const double*, const double*, double*, cudaStream_t, Gate);
template cudaError_t launch_block_correct<double>(const BlockMap&, const double*, const double*, const int64_t*,
                                                  const double*, const double*, double*, cudaStream_t, Gate);

}  // namespace sap
