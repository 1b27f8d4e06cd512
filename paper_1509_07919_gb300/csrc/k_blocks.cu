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
// the permutations of vectors, the entire spikes (forward and backward sweeps
// of every block in 32-row chunk steps with its chunk matrices, a 32 x 32
// sub-block of the spike per step, Sec. 3.1), and the two steps of the apply
// after the block solves: the truncated reduced
// solve (Eq. (2.5b,c)) and z_i = g_i - Vhat_i x^(t)_{i+1} - What_i x^(b)_{i-1}
// (= A_i^{-1}(r_i - [C_i x^(b)_{i-1}; 0] - [0; B_i x^(t)_{i+1}]) by linearity).
#include <cuda_runtime.h>
#include <algorithm>
#include <cstdint>
#include <type_traits>
#include "sap_internal.cuh"

namespace sap {

namespace {

constexpr int kGridStride = 152 * 8;   // CTAs of the grid-stride kernels

// block of row g (N < 2^31: 32-bit arithmetic)
__device__ __forceinline__ int block_of(const BlockMap& m, int64_t g64) {
  const unsigned g = (unsigned)g64, q = (unsigned)m.q, pr = (unsigned)m.pr;
  const unsigned big = pr * (q + 1);
  return g < big ? (int)(g / (q + 1)) : (int)(pr + (g - big) / q);
}

// Half-bandwidth of every reordered block: max |perm(i) - perm(j)| over the
// nonzero band entries (i, j) with both indices in one block (one atomic per
// warp and block).
// Grid (x, 2K + 1): blockIdx.y is the diagonal c, x strides over the columns j.
__global__ void __launch_bounds__(256) k_block_bw(const double* __restrict__ band, BlockMap m, int* __restrict__ Kout) {
  const int c = blockIdx.y;
  const double* col = band + (int64_t)c * m.N;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < m.N; base += stride) {
    const int64_t j = base + threadIdx.x;
    int b = -1, d = 0;
    if (j < m.N) {
      const int64_t i = j + c - m.K;
      if (c != m.K && i >= 0 && i < m.N && col[j] != 0.0) {
        const int bj = block_of(m, j);
        if (i >= m.off[bj] && i < m.off[bj + 1]) {
          b = bj;
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
  const int c = blockIdx.y;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m.N; j += stride) {
    const int64_t i = j + c - m.K;
    if (i < 0 || i >= m.N) continue;
    const double v = band[(int64_t)c * m.N + j];
    if (v == 0.0) continue;
    const int bi = block_of(m, j);
    if (i < m.off[bi] || i >= m.off[bi + 1]) continue;
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

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src));
}

constexpr int kChunk = 32;     // rows per chunk of the blocks' sweep matrices

// Entire spikes of interface i (blockIdx.z): side 0 (blockIdx.y) Vhat_i of
// block i, side 1 What_{i+1} of block i+1; CPB right-hand-side columns per
// CTA (blockIdx.x); output rows of KS elements (K columns, zero padding).
// The block's sweeps are blocked in 32-row chunks with the matrices its
// factorisation formed for the preconditioner apply (positions p in sweep
// order, MINV_c and G_{c,k}, k = 1..ng, column-major, contiguous per chunk):
//     Z_c = MINV_c Y_c - sum_k G_{c,k} Z_{c-k}
// for a 32 x CPB tile of the spike at once (Sec. 3.1: a sub-block of the
// spike per step instead of one column, the block's coefficients in shared
// memory).  Forward (L) from the chunk of the first nonzero right-hand-side
// row, then backward (U) over all chunks.  Each step's matrices (and the
// old row numbers of its rows, or its y values in the backward sweep) are
// staged by cp.async while the previous step computes; the last ng tiles stay
// in shared memory.  Thread (warp w, lane t) computes row t of the tile for
// columns w CPW .. w CPW + CPW - 1.  Then the tip rows are copied out.
template <typename T, int CPB>
__global__ void __launch_bounds__(256)
k_full_spikes(const double* __restrict__ band, BlockMap m, int KS, int ngmax, const void* const* __restrict__ Mfp,
              const void* const* __restrict__ Mbp, const int* __restrict__ ngp, const int64_t* __restrict__ ldp,
              T* __restrict__ spk, const int64_t* __restrict__ sbase, T* __restrict__ Vtip, T* __restrict__ Wtip,
              int adj) {
  constexpr int NT = 256, CH = kChunk, CPW = CPB / 8;
  constexpr int MM = CH * CH;
  static_assert(CPW * sizeof(T) % 16 == 0, "a thread's columns are read as 16-byte vectors");
  // row stride of the tiles: CPB plus 16 bytes, so that the 16-byte row writes
  // of 8 consecutive lanes (rows) fall on distinct banks
  constexpr int RSZ = CPB + 16 / (int)sizeof(T);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int SL = ngmax + 1;                               // ring slots (chunk c at c mod SL)
  T* Mbuf = reinterpret_cast<T*>(smem_raw);               // 2 x (1 + ngmax) x 32 x 32
  T* ring = Mbuf + 2 * (size_t)SL * MM;                   // SL x 32 x RSZ
  T* Rb = ring + (size_t)SL * CH * RSZ;                   // 2 x 32 x RSZ right-hand sides
  int* Pb = reinterpret_cast<int*>(Rb + 2 * CH * RSZ);    // 2 x 32 old row numbers
  __shared__ int rmin_s;
  const int i = blockIdx.z, side = blockIdx.y;
  const int b = i + side;
  const int64_t s0 = m.off[b];
  const int n = (int)(m.off[b + 1] - s0);
  const int K = m.K;
  const int64_t N = m.N;
  const int ng = ngp[b];
  const int ld = (int)ldp[b];
  const int nch = ld / CH;
  const int64_t msz = (int64_t)(1 + ng) * MM;             // elements of one chunk's matrices
  const T* Mf = static_cast<const T*>(Mfp[b]);
  const T* Mb = static_cast<const T*>(Mbp[b]);
  const int64_t sif = m.off[i + 1];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int c0 = blockIdx.x * CPB;
  T* out = spk + sbase[2 * i + side];

  for (int e = tid; e < SL * CH * RSZ; e += NT) ring[e] = T(0);
  if (tid == 0) rmin_s = n;
  __syncthreads();
  {
    int loc = n;
    for (int r = tid; r < K; r += NT) loc = min(loc, m.perm[s0 + (side == 0 ? n - K + r : r)]);
    atomicMin(&rmin_s, loc);
  }
  __syncthreads();
  const int rstart = rmin_s;
  const int cstart = rstart / CH;

  // right-hand side at old local row a, column col: [0; B_i] or [C_{i+1}; 0]; for the
  // preconditioner of A^T (adj) [0; C_{i+1}^T] or [B_i^T; 0]
  auto rhs = [&](int a, int col) -> T {
    double v = 0.0;
    if (!adj) {
      if (side == 0) {
        const int rr = a - (n - K);                     // B_i(rr, col) = a(sif - K + rr, sif + col)
        if (rr >= 0 && col <= rr) v = band[(int64_t)(rr - col) * N + sif + col];
      } else if (a < K && col >= a) {                   // C_{i+1}(a, col) = a(sif + a, sif - K + col)
        v = band[(int64_t)(2 * K + a - col) * N + sif - K + col];
      }
    } else {
      if (side == 0) {
        const int rr = a - (n - K);                     // C_{i+1}^T(rr, col) = a(sif + col, sif - K + rr)
        if (rr >= 0 && rr >= col) v = band[(int64_t)(2 * K + col - rr) * N + sif - K + rr];
      } else if (a < K && a <= col) {                   // B_i^T(a, col) = a(sif - K + col, sif + a)
        v = band[(int64_t)(col - a) * N + sif + a];
      }
    }
    return (T)v;
  };
  auto stage_mats = [&](const T* Msrc, int c, T* dst) {
    const char* src = reinterpret_cast<const char*>(Msrc + (int64_t)c * msz);
    const int nv = (int)(msz * sizeof(T) / 16);
    for (int e = tid; e < nv; e += NT) cp_async16(reinterpret_cast<char*>(dst) + 16 * e, src + 16 * e);
  };
  // forward step c: its matrices and the old row numbers of rows 32 c .. 32 c + 31
  auto stage_fwd = [&](int c, int bf) {
    stage_mats(Mf, c, Mbuf + (size_t)bf * SL * MM);
    if (tid < CH) {
      const int r = c * CH + tid;
      const bool ok = r < n;
      cp_async_elem(Pb + bf * CH + tid, ok ? (const void*)(m.pinv + s0 + r) : (const void*)m.pinv, ok, 4);
    }
    cp_async_commit();
  };
  // backward step c: its matrices and y at rows r = ld - 1 - p (0 where there is none)
  auto stage_bwd = [&](int c, int bf) {
    stage_mats(Mb, c, Mbuf + (size_t)bf * SL * MM);
    T* Y = Rb + bf * CH * RSZ;
    for (int e = tid; e < CH * CPB; e += NT) {
      const int t = e / CPB, cc = e % CPB;
      const int r = ld - 1 - (c * CH + t);
      const bool ok = r < n && r >= rstart && c0 + cc < K;
      cp_async_elem(Y + t * RSZ + cc, ok ? (const void*)(out + (int64_t)r * KS + c0 + cc) : (const void*)out, ok,
                    (int)sizeof(T));
    }
    cp_async_commit();
  };
  // Z_c (row lane, columns w CPW ..) = MINV_c Y_c - sum_k G_{c,k} Z_{c-k}; the
  // tile rows are read as 16-byte broadcasts (CPW T per thread)
  using Vec = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  constexpr int VPT = CPW * sizeof(T) / 16;
  auto mac = [&](const T* Mx, const T* Yt, T* acc, T sgn) {
#pragma unroll 8
    for (int j = 0; j < CH; ++j) {
      const T mv = sgn * Mx[j * CH + lane];
      const Vec* yr = reinterpret_cast<const Vec*>(Yt + j * RSZ + w * CPW);
#pragma unroll
      for (int v = 0; v < VPT; ++v) {
        const Vec y4 = yr[v];
        const T* e = reinterpret_cast<const T*>(&y4);
#pragma unroll
        for (int u = 0; u < (int)(16 / sizeof(T)); ++u) acc[v * (16 / sizeof(T)) + u] += mv * e[u];
      }
    }
  };
  auto step = [&](int c, int cfirst, const T* M, const T* Y, bool with_rhs, T* acc) {
#pragma unroll
    for (int q = 0; q < CPW; ++q) acc[q] = T(0);
    if (with_rhs) mac(M, Y, acc, T(1));
    const int kmax = min(ng, c - cfirst);
    for (int k = 1; k <= kmax; ++k) mac(M + k * MM, ring + (size_t)((c - k) % SL) * CH * RSZ, acc, T(-1));
  };

  // ---- forward: L y = Pi rhs ----
  int bf = 0;
  stage_fwd(cstart, 0);
  for (int c = cstart; c < nch; ++c) {
    cp_async_wait_all();
    __syncthreads();                                     // step c's staged data; the ring's last tiles
    if (c + 1 < nch) stage_fwd(c + 1, bf ^ 1);
    T* Y = Rb + bf * CH * RSZ;
    int any = 0;
    for (int e = tid; e < CH * CPB; e += NT) {
      const int t = e / CPB, cc = e % CPB;
      const int r = c * CH + t;
      const T v = (r < n && c0 + cc < K) ? rhs(Pb[bf * CH + t], c0 + cc) : T(0);
      Y[t * RSZ + cc] = v;
      any |= v != T(0);
    }
    const bool nz = __syncthreads_or(any) != 0;          // most steps have no right-hand-side row
    T acc[CPW];
    step(c, cstart, Mbuf + (size_t)bf * SL * MM, Y, nz, acc);
    T* Zc = ring + (size_t)(c % SL) * CH * RSZ;
    const int r = c * CH + lane;
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      Vec x;
      T* xe = reinterpret_cast<T*>(&x);
#pragma unroll
      for (int u = 0; u < (int)(16 / sizeof(T)); ++u) xe[u] = acc[v * (16 / sizeof(T)) + u];
      reinterpret_cast<Vec*>(Zc + lane * RSZ + w * CPW)[v] = x;
    }
#pragma unroll
    for (int q = 0; q < CPW; ++q) {
      const int col = c0 + w * CPW + q;
      if (r < n && col < K) out[(int64_t)r * KS + col] = acc[q];
    }
    bf ^= 1;
  }
  cp_async_wait_all();
  __syncthreads();
  for (int e = tid; e < SL * CH * RSZ; e += NT) ring[e] = T(0);
  __syncthreads();

  // ---- backward: U x = y (positions from the last row) ----
  bf = 0;
  stage_bwd(0, 0);
  for (int c = 0; c < nch; ++c) {
    cp_async_wait_all();
    __syncthreads();
    if (c + 1 < nch) stage_bwd(c + 1, bf ^ 1);
    T acc[CPW];
    step(c, 0, Mbuf + (size_t)bf * SL * MM, Rb + bf * CH * RSZ, true, acc);
    T* Zc = ring + (size_t)(c % SL) * CH * RSZ;
    const int r = ld - 1 - (c * CH + lane);
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      Vec x;
      T* xe = reinterpret_cast<T*>(&x);
#pragma unroll
      for (int u = 0; u < (int)(16 / sizeof(T)); ++u) xe[u] = acc[v * (16 / sizeof(T)) + u];
      reinterpret_cast<Vec*>(Zc + lane * RSZ + w * CPW)[v] = x;
    }
#pragma unroll
    for (int q = 0; q < CPW; ++q) {
      const int col = c0 + w * CPW + q;
      if (r < n && col < K) out[(int64_t)r * KS + col] = acc[q];
    }
    bf ^= 1;
  }
  cp_async_wait_all();
  __syncthreads();
  // tips: the spike rows of the old interface rows
  T* tip = (side == 0 ? Vtip : Wtip) + (int64_t)i * K * K;
  for (int e = tid; e < K * CPB; e += NT) {
    const int rr = e / CPB, c2 = c0 + e % CPB;
    if (c2 < K) {
      const int a = side == 0 ? n - K + rr : rr;
      tip[(int64_t)rr * K + c2] = out[(int64_t)m.perm[s0 + a] * KS + c2];
    }
  }
}

// Truncated reduced solve of every interface (Eq. (2.5b,c)) on g = D^{-1} r
// held in the blocks' new numbering: g^(b)_i, g^(t)_{i+1} gathered through the
// permutations, x^(t)_{i+1} = Rbar_i^{-1} (g^(t)_{i+1} - W^(t)_{i+1} g^(b)_i),
// x^(b)_i = g^(b)_i - V^(b)_i x^(t)_{i+1}.  One CTA of 32 warps per interface,
// a warp per row of each K x K product.
constexpr int kRedWarps = 32;
template <typename T>
__global__ void __launch_bounds__(32 * kRedWarps)
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
  for (int r = w; r < K; r += kRedWarps) {
    const double a = rowdot(Wt + i * KK + (int64_t)r * K, gb);
    if (lane == 0) rhs[r] = gtv[r] - a;
  }
  __syncthreads();
  for (int r = w; r < K; r += kRedWarps) {
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
  for (int r = w; r < K; r += kRedWarps) {
    const double a = rowdot(V + i * KK + (int64_t)r * K, gtv);
    if (lane == 0) xb[(int64_t)i * K + r] = gb[r] - a;
  }
}

// z[off_b + pinv(r)] = g[off_b + r] - Vhat_b[r] . x^(t)_{b+1} - What_b[r] . x^(b)_{b-1}
// for every new row r of every block b: CTA (row chunk, block b), the two
// x vectors in shared memory (zero padded to KS), a warp per row, 16-byte
// loads of the spike rows (KS elements, 16-byte aligned).  The products are
// formed in the factor precision (the spikes' own; with FP32 factors the FP64
// pipe, a small fraction of the FP32 rate on this part, would bound them), the
// subtraction from g in FP64.
constexpr int kCorrRows = 128;
template <typename T>
__global__ void __launch_bounds__(256)
k_block_correct(BlockMap m, const double* __restrict__ gh, const T* __restrict__ spk, const int64_t* __restrict__ sbase,
                int KS, const double* __restrict__ xt, const double* __restrict__ xb, double* __restrict__ z, Gate gt) {
  if (gate_skip(gt)) return;
  constexpr int VW = 16 / sizeof(T);
  using Vec = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* xs = reinterpret_cast<T*>(smem_raw);                // 2 x KS
  const int K = m.K, b = blockIdx.y;
  const int64_t s = m.off[b];
  const int n = (int)(m.off[b + 1] - s);
  const int r0 = blockIdx.x * kCorrRows;
  if (r0 >= n) return;
  const bool hasV = b < m.P - 1, hasW = b > 0;
  for (int k = threadIdx.x; k < KS; k += blockDim.x) {
    xs[k] = (T)(hasV && k < K ? xt[(int64_t)b * K + k] : 0.0);
    xs[KS + k] = (T)(hasW && k < K ? xb[(int64_t)(b - 1) * K + k] : 0.0);
  }
  __syncthreads();
  const T* V = hasV ? spk + sbase[2 * b] : nullptr;
  const T* W = hasW ? spk + sbase[2 * (b - 1) + 1] : nullptr;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nv = KS / VW;
  const int r1 = min(n, r0 + kCorrRows);
  for (int r = r0 + w; r < r1; r += 8) {
    T a = T(0);
    for (int v = lane; v < nv; v += 32) {
      const Vec x0 = reinterpret_cast<const Vec*>(xs)[v];
      const Vec x1 = reinterpret_cast<const Vec*>(xs + KS)[v];
      const T* p0 = reinterpret_cast<const T*>(&x0);
      const T* p1 = reinterpret_cast<const T*>(&x1);
      if (hasV) {
        const Vec q = reinterpret_cast<const Vec*>(V + (int64_t)r * KS)[v];
        const T* e = reinterpret_cast<const T*>(&q);
#pragma unroll
        for (int u = 0; u < VW; ++u) a += e[u] * p0[u];
      }
      if (hasW) {
        const Vec q = reinterpret_cast<const Vec*>(W + (int64_t)r * KS)[v];
        const T* e = reinterpret_cast<const T*>(&q);
#pragma unroll
        for (int u = 0; u < VW; ++u) a += e[u] * p1[u];
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) z[s + m.pinv[s + r]] = gh[s + r] - (double)a;
  }
}

// x-extent of the (columns x diagonals) grids: about kGridStride CTAs in all
int spread_x(const BlockMap& m) {
  const int64_t want = std::max<int64_t>(1, kGridStride / (2 * m.K + 1));
  return (int)std::min<int64_t>(want, (m.N + 255) / 256);
}


template <typename T, int CPB>
size_t spikes_smem(int ngmax) {
  const size_t SL = (size_t)ngmax + 1, RSZ = CPB + 16 / sizeof(T);
  return (2 * SL * kChunk * kChunk + SL * kChunk * RSZ + 2 * (size_t)kChunk * RSZ) * sizeof(T) +
         2 * kChunk * sizeof(int);
}

}  // namespace

cudaError_t launch_block_bw(const double* band, const BlockMap& m, int* Kout, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(Kout, 0, (size_t)m.P * sizeof(int), s);
  if (e != cudaSuccess) return e;
  count_launches(1);
  k_block_bw<<<dim3(spread_x(m), 2 * m.K + 1), 256, 0, s>>>(band, m, Kout);
  return cudaGetLastError();
}

cudaError_t launch_block_gather(const double* band, const BlockMap& m, double* hb, int64_t hb_elems, int* err,
                                cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(hb, 0, (size_t)hb_elems * sizeof(double), s);
  if (e != cudaSuccess) return e;
  count_launches(1);
  k_block_gather<<<dim3(spread_x(m), 2 * m.K + 1), 256, 0, s>>>(band, m, hb, err);
  return cudaGetLastError();
}

cudaError_t launch_block_perm(const BlockMap& m, const double* x, double* y, bool to_new, cudaStream_t s, Gate gt) {
  count_launches(1);
  const int grid = (int)std::min<int64_t>(kGridStride, (m.N + 255) / 256);
  k_block_perm<<<grid, 256, 0, s>>>(m, x, y, to_new ? 1 : 0, gt);
  return cudaGetLastError();
}

int spike_row_stride(int K, bool fp64) {
  const int vw = fp64 ? 2 : 4;
  return (K + vw - 1) / vw * vw;
}

// columns per CTA of the spike kernel: 32 (measured on GB300 at N = 200000,
// P = 50: FP32 K = 100 1.25 ms against 1.50 ms with 64 columns, twice the CTAs
// on the latency-bound chunk chains; K = 400 6.28 against 6.36 ms), or 16 for
// FP64 blocks whose 32-column tiles exceed shared memory (at least 16 bytes of
// columns per thread)
template <typename T>
int spike_cols(int ngmax) {
  if (spikes_smem<T, 32>(ngmax) <= kSmemPerBlock) return 32;
  return sizeof(T) == 8 && spikes_smem<T, 16>(ngmax) <= kSmemPerBlock ? 16 : 0;
}

size_t full_spikes_smem(int ngmax, bool fp64) {
  if (fp64) {
    const int c = spike_cols<double>(ngmax);
    return c == 32 ? spikes_smem<double, 32>(ngmax) : spikes_smem<double, 16>(ngmax);
  }
  return spike_cols<float>(ngmax) == 32 ? spikes_smem<float, 32>(ngmax) : kSmemPerBlock + 1;
}

template <typename T, int CPB>
cudaError_t launch_spikes_cols(const double* band, const BlockMap& m, int ngmax, const void* const* Mfp,
                               const void* const* Mbp, const int* ngp, const int64_t* ldp, T* spk,
                               const int64_t* sbase, T* Vtip, T* Wtip, bool adjoint, cudaStream_t s) {
  const size_t smem = spikes_smem<T, CPB>(ngmax);
  cudaError_t e = cudaFuncSetAttribute(k_full_spikes<T, CPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  count_launches(1);
  k_full_spikes<T, CPB><<<dim3((m.K + CPB - 1) / CPB, 2, m.P - 1), 256, smem, s>>>(
      band, m, spike_row_stride(m.K, sizeof(T) == 8), ngmax, Mfp, Mbp, ngp, ldp, spk, sbase, Vtip, Wtip,
      adjoint ? 1 : 0);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_full_spikes(const double* band, const BlockMap& m, int ngmax, const void* const* Mfp,
                               const void* const* Mbp, const int* ngp, const int64_t* ldp, T* spk,
                               const int64_t* sbase, T* Vtip, T* Wtip, bool adjoint, cudaStream_t s) {
  if (m.P < 2) return cudaSuccess;
  const int c = spike_cols<T>(ngmax);
  if (c == 32)
    return launch_spikes_cols<T, 32>(band, m, ngmax, Mfp, Mbp, ngp, ldp, spk, sbase, Vtip, Wtip, adjoint, s);
  if constexpr (sizeof(T) == 8) {
    if (c == 16)
      return launch_spikes_cols<T, 16>(band, m, ngmax, Mfp, Mbp, ngp, ldp, spk, sbase, Vtip, Wtip, adjoint, s);
  }
  return cudaErrorInvalidValue;
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
  k_block_reduced<T><<<m.P - 1, 32 * kRedWarps, smem, s>>>(m, gh, V, Wt, Rinv, xt, xb, gt);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_block_correct(const BlockMap& m, int max_rows, const double* gh, const T* spk,
                                 const int64_t* sbase, const double* xt, const double* xb, double* z, cudaStream_t s,
                                 Gate gt) {
  const int KS = spike_row_stride(m.K, sizeof(T) == 8);
  const size_t smem = 2 * (size_t)KS * sizeof(T);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_block_correct<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  count_launches(1);
  k_block_correct<T><<<dim3((max_rows + kCorrRows - 1) / kCorrRows, m.P), 256, smem, s>>>(m, gh, spk, sbase, KS, xt, xb,
                                                                                        z, gt);
  return cudaGetLastError();
}

template cudaError_t launch_full_spikes<float>(const double*, const BlockMap&, int, const void* const*,
                                               const void* const*, const int*, const int64_t*, float*, const int64_t*,
                                               float*, float*, bool, cudaStream_t);
template cudaError_t launch_full_spikes<double>(const double*, const BlockMap&, int, const void* const*,
                                                const void* const*, const int*, const int64_t*, double*,
                                                const int64_t*, double*, double*, bool, cudaStream_t);
template cudaError_t launch_block_reduced<float>(const BlockMap&, const double*, const float*, const float*,
                                                 const double*, double*, double*, cudaStream_t, Gate);
template cudaError_t launch_block_reduced<double>(const BlockMap&, const double*, const double*, const double*,
                                                  const double*, double*, double*, cudaStream_t, Gate);
template cudaError_t launch_block_correct<float>(const BlockMap&, int, const double*, const float*, const int64_t*,
                                                 const double*, const double*, double*, cudaStream_t, Gate);
template cudaError_t launch_block_correct<double>(const BlockMap&, int, const double*, const double*, const int64_t*,
                                                  const double*, const double*, double*, cudaStream_t, Gate);

}  // namespace sap
