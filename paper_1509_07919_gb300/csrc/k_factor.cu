// Banded LU / UL factorisation of the diagonal blocks A_i without pivoting,
// with pivot boosting (Sec. 2.2, Sec. 3.1 "LU/UL factorizations").
//
// One CTA (8 warps; 16 with the window in global memory) factors one block
// with a blocked right-looking elimination over panels of NB = 16 columns.
// The active window, rows and columns [k0, k0 + K + NB) of the block, lives
// in shared memory (or, for bands too wide for it, in an L2-resident global
// scratch), addressed modulo M2 = K + NB rounded up in both directions, so
// that sliding it by a panel only replaces NB physical rows and columns.  Per
// panel:
//   A1. warp 0 factors the 16 x 16 diagonal block in registers (pivot row by
//       shuffles, boosted pivot, multipliers); meanwhile the other warps
//       cp.async the entering band rows/columns of the next window into a
//       staging buffer;
//   A2/B. L21 = A21 U11^{-1} (one thread per row) and U12 = L11^{-1} A12 (one
//       thread per column), on the two halves of the CTA;
//   C. trailing update A22 -= L21 U12 (K x K, 4 x 4 register tiles, 8 x 4 for
//      FP32 in the global window, or on the tensor cores, see below);
//   D. the finished panel rows of U and columns of L go to global memory and
//      the staged entering rows/columns replace the retired ones.
// Four barriers per 16 columns.  Entries outside the band (and outside the
// block) are kept as exact zeros, so no band masks are needed inside the
// arithmetic.
// The UL factorisation is the same elimination run on the reversed block
// J A_i J: if J A_i J = L~ U~ (unit L~) then A_i = (J L~ J)(J U~ J) = U' L'
// with unit upper U'.  Only the last K rows/columns of L~, U~ are kept,
// flipped back into the top K x K tiles of U' and L'.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include "sap_internal.cuh"
#include "tc_sm103.cuh"

namespace sap {

namespace {

constexpr int NB = 16;             // panel width
// 512 threads for the global-memory window (its L2-resident read-modify-write
// of the trailing matrix wants more loads in flight), 256 otherwise
__host__ __device__ constexpr int lu_threads(bool gw, bool tc) { return gw && !tc ? 512 : 256; }

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
template <typename X> __device__ __forceinline__ void cp_async_t(X* smem, const X* gmem) {
  if (sizeof(X) == 4) cp_async4(smem, gmem); else cp_async8(smem, gmem);
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Entries of the block in local coordinates (r, q), reversed when REV.
// Returns a pointer into the band, or nullptr for a structural zero.
template <bool REV, typename BT>
__device__ __forceinline__ const BT* elem_ptr(const BT* band, int64_t N, int K, int64_t s,
                                              int n, int r, int q) {
  if (r < 0 || q < 0 || r >= n || q >= n) return nullptr;
  int64_t gi = REV ? s + n - 1 - r : s + r;
  int64_t gj = REV ? s + n - 1 - q : s + q;
  int64_t c = (int64_t)K + gi - gj;
  if (c < 0 || c > 2 * (int64_t)K) return nullptr;
  return band + c * N + gj;
}


// Window geometry: M2 = K + NB rounded up to a multiple of NB, row pitch
// LDW = M2 + 4 (16-byte aligned rows; 128-bit row reads are conflict-free).
// The base (physical index of logical offset 0) is a multiple of NB, so a
// panel's NB columns, and any 4-aligned group of offsets, never wrap.
struct Win {
  int M2, LDW, base;
  __device__ __forceinline__ int ph(int off) const { int x = base + off; return x >= M2 ? x - M2 : x; }
};
__host__ __device__ inline int win_m2(int K) { return (K + NB + NB - 1) / NB * NB; }


// 4 consecutive T from a 16-byte (float) / 32-byte-capable (double) aligned address
template <typename T>
__device__ __forceinline__ void ld4(const T* p, T (&v)[4]) {
  if (sizeof(T) == 4) {
    float4 x = *reinterpret_cast<const float4*>(p);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  } else {
    double2 x = *reinterpret_cast<const double2*>(p);
    double2 y = *reinterpret_cast<const double2*>(p + 2);
    v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
  }
}
template <typename T>
__device__ __forceinline__ void st4(T* p, const T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
  }
}
// the same for global memory, cached in L2 only (entries touched once per
// panel, which would otherwise push the panel operands out of L1)
template <typename T>
__device__ __forceinline__ void ld4_cg(const T* p, T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 x = __ldcg(reinterpret_cast<const float4*>(p));
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  } else {
    const double2 x = __ldcg(reinterpret_cast<const double2*>(p));
    const double2 y = __ldcg(reinterpret_cast<const double2*>(p + 2));
    v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
  }
}
template <typename T>
__device__ __forceinline__ void st4_cg(T* p, const T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    __stcg(reinterpret_cast<float4*>(p), make_float4(v[0], v[1], v[2], v[3]));
  } else {
    __stcg(reinterpret_cast<double2*>(p), make_double2(v[0], v[1]));
    __stcg(reinterpret_cast<double2*>(p + 2), make_double2(v[2], v[3]));
  }
}

// Reciprocal of a pivot.  FP32: the hardware approximation refined by one
// Newton-Raphson step for 1/p (x1 = x0 + x0 (1 - p x0)); FP64: division.
template <typename T> __device__ __forceinline__ T pivot_rcp(T p) { return T(1) / p; }
template <> __device__ __forceinline__ float pivot_rcp<float>(float p) {
  float x;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(x) : "f"(p));
  return fmaf(x, fmaf(-p, x, 1.0f), x);
}
// Boosted pivot (Sec. 2.2): |p| < tau becomes sign(p) tau (sign(0) = +1);
// past the block's last row (padding) the pivot is 1, its rows being zero.
template <typename T>
__device__ __forceinline__ T boost_pivot(T p, bool inside, T tau, unsigned long long& nb) {
  if (!inside) return T(1);
  if ((p < T(0) ? -p : p) < tau) {
    ++nb;
    return p >= T(0) ? tau : -tau;
  }
  return p;
}

// A1: LU (unit lower L, boosted pivots) of the 16 x 16 diagonal block at
// physical rows / columns pb .. pb + 15 of a window with row pitch LDW, whose
// first row is block row pk0; one warp, lane r holding row r: per column the
// pivot row is broadcast by shuffles and every lower row eliminates it.  The
// pivots' reciprocals go to RV.
template <typename T>
__device__ __forceinline__ void diag_lu16(T* W, int LDW, int pb, int pk0, int n, T tau, T* RV,
                                          unsigned long long& nb) {
  const int lane = threadIdx.x & 31;
  T pv[NB];
  if (lane < NB) {
    const T* row = &W[(pb + lane) * LDW + pb];
#pragma unroll
    for (int c4 = 0; c4 < NB / 4; ++c4) {
      T v[4];
      ld4(row + 4 * c4, v);
#pragma unroll
      for (int x = 0; x < 4; ++x) pv[4 * c4 + x] = v[x];
    }
  } else {
#pragma unroll
    for (int c = 0; c < NB; ++c) pv[c] = T(0);
  }
  T myrinv = T(0);
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    T u[NB];
#pragma unroll
    for (int c = j; c < NB; ++c) u[c] = __shfl_sync(0xffffffffu, pv[c], j);
    const T p = boost_pivot(u[j], pk0 + j < n, tau, nb);
    const T rinv = pivot_rcp(p);
    if (lane > j) {
      const T l = pv[j] * rinv;
      pv[j] = l;
#pragma unroll
      for (int c = j + 1; c < NB; ++c) pv[c] = fma(-l, u[c], pv[c]);
    } else if (lane == j) {
      pv[j] = p;
      myrinv = rinv;
    }
  }
  if (lane < NB) {
    T* row = &W[(pb + lane) * LDW + pb];
#pragma unroll
    for (int c4 = 0; c4 < NB / 4; ++c4) st4(row + 4 * c4, {pv[4 * c4], pv[4 * c4 + 1], pv[4 * c4 + 2], pv[4 * c4 + 3]});
    RV[lane] = myrinv;
  }
}

// Tensor-core trailing update (TC): per panel the rank-16 product L21 U12 is
// formed by tcgen05 MMAs, BF16 operands (RN) and FP32 accumulation, in
// 128 x 128 pieces of TMEM (four at a time), and subtracted from the FP32
// window; pivots, the panel and U12 stay FP32.  Operand rows r (trailing rows
// of L21, trailing columns of U12) in the no-swizzle K-major layout: element
// (r, q) at (r / 8) 128 + (q / 8) 64 + (r % 8) 8 + q % 8 BF16 elements.
constexpr int kTcPiece = 128;
struct TcCtx {
  __nv_bfloat16* A = nullptr;   // Kp x 16 (L21)
  __nv_bfloat16* B = nullptr;   // Kp x 16 (U12 transposed)
  uint64_t* bar = nullptr;      // MMA completion
  uint32_t taddr = 0;           // TMEM base
  unsigned ph = 0;              // next phase parity of bar
  bool failed = false;          // a bounded wait of this thread gave up
  int* err = nullptr;
  int spin = kDefaultSpin;      // polls of a bounded wait (err[1])
};
__host__ __device__ inline int tc_rows(int K) { return ((K + 15) / 16 * 16 + kTcPiece - 1) / kTcPiece * kTcPiece; }
__host__ __device__ inline uint32_t tc_cols(int K) {
  const int nmt = tc_rows(K) / kTcPiece;
  return nmt * nmt >= 4 ? 512u : (uint32_t)(nmt * nmt * kTcPiece);   // 1 piece: 128, more: 4 pieces
}
__host__ __device__ inline size_t tc_bytes(int K) { return (size_t)tc_rows(K) * 16 * 2 * 2 + 16; }

// Operand buffers, barrier and TMEM of the CTA (whole CTA; warp 0 allocates).
__device__ void tc_setup(unsigned char* base, int K, TcCtx& t, int* err) {
  const int Kp = tc_rows(K);
  t.A = reinterpret_cast<__nv_bfloat16*>(base);
  t.B = t.A + Kp * 16;
  t.bar = reinterpret_cast<uint64_t*>(t.B + Kp * 16);
  uint32_t* slot = reinterpret_cast<uint32_t*>(t.bar + 1);
  t.err = err;
  t.spin = spin_limit_of(err);
  for (int e = threadIdx.x; e < Kp * 16; e += blockDim.x) {
    t.A[e] = __float2bfloat16_rn(0.f);
    t.B[e] = __float2bfloat16_rn(0.f);
  }
  if (threadIdx.x == 0) {
    tc::mbar_init(t.bar, 1);
    tc::mbar_fence_init();
  }
  if (threadIdx.x < 32) {
    tc::tmem_alloc(slot, tc_cols(K));
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  t.taddr = *slot;
}
__device__ void tc_teardown(TcCtx& t, int K) {
  // a thread whose wait gave up waits once more (bounded) for the MMAs in flight
  if (t.failed) {
    bool again = false;
    tc::mbar_wait_bounded(t.bar, t.ph ^ 1u, kDefaultSpin, nullptr, again);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc::fence_after_sync();
    tc::tmem_dealloc(t.taddr, tc_cols(K));
  }
}

// Factor one block (rows s .. s+n-1 of the band) with the whole CTA; F: the
// block's factor storage (LU) or flipped top tiles (REV, ld unused).
// GW: the window in global memory at wglob (M2 x LDW, L2-resident) instead
// of shared memory; wide bands whose (K+16)^2 window does not fit in
// shared memory use the global form, the staging buffers stay in shared memory.
template <typename T, bool REV, bool GW, bool TC, int NTH>
__device__ void band_lu_block(unsigned char* smem_raw, const T* __restrict__ band, int64_t N, int K, int64_t s,
                              int n, int64_t ld, T* __restrict__ F, const T tau,
                              unsigned long long* __restrict__ n_boosted, T* wglob, TcCtx& tcx) {
  static_assert(!TC || sizeof(T) == 4, "the tensor-core trailing update is an FP32-factor mode");
  static_assert(!TC || NTH == 256, "the tensor-core readback splits TMEM columns over two warpgroups");
  const int M2 = win_m2(K);
  const int LDW = M2 + 4;
  const int KA = K + NB;          // active rows/cols of the window in a panel step
  const int ME = M2 - NB;         // rows of the next window that are already resident
  T* W = GW ? wglob : reinterpret_cast<T*>(smem_raw);
  const size_t woff = GW ? 0 : ((size_t)M2 * LDW * sizeof(T) + 15) & ~(size_t)15;
  T* ER = reinterpret_cast<T*>(smem_raw + woff);   // NB x M2 entering rows
  T* EC = ER + NB * M2;                              // ME x NB entering columns
  T* RV = EC + ME * NB;                              // NB reciprocals of the panel's pivots
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned long long nb = 0;

  Win w{M2, LDW, 0};
  // initial window: logical rows/cols [0, M2), physical == logical
  for (int e = tid; e < M2 * M2; e += NTH) {
    int r = e / M2, q = e % M2;
    const T* p = elem_ptr<REV>(band, N, K, s, n, r, q);
    W[r * LDW + q] = p ? *p : T(0);
  }
  __syncthreads();

  // Prefetch of the rows and columns that enter the window when it slides
  // after the panel at k0 (warps 1..): cp.async into ER / EC.  The band is
  // stored by diagonals, so a matrix row or column is strided by N in memory;
  // the entries are enumerated as (jj, e), e fastest, with offset jo = jj + e
  // (mod M2, resp. ME): for one jj and consecutive e the diagonal is the same
  // and the band addresses are consecutive (16 entries, 64 bytes per half
  // warp) instead of one sector per entry.
  auto prefetch = [&](int k0) {
    const int ht = tid - 32, nh = NTH - 32;
    // entering rows i = k0 + M2 + e (columns of the next window, offsets jo from k0 + NB)
    for (int y = ht; y < NB * M2; y += nh) {
      const int e = y % NB, jj = y / NB;
      int jo = jj + e;
      if (jo >= M2) jo -= M2;
      T* dst = &ER[e * M2 + jo];
      const T* src = elem_ptr<REV>(band, N, K, s, n, k0 + M2 + e, k0 + NB + jo);
      if (src) cp_async_t(dst, src);
      else *dst = T(0);
    }
    // entering columns j = k0 + M2 + e for resident rows i = k0 + NB + ro (ro < ME)
    for (int y = ht; y < ME * NB; y += nh) {
      const int e = y % NB, jj = y / NB;
      int ro = jj + e;
      if (ro >= ME) ro -= ME;
      T* dst = &EC[ro * NB + e];
      const T* src = elem_ptr<REV>(band, N, K, s, n, k0 + NB + ro, k0 + M2 + e);
      if (src) cp_async_t(dst, src);
      else *dst = T(0);
    }
    cp_async_commit();
  };
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int base = w.base;     // physical column of the panel start (multiple of NB)
    // ---- A1 (warp 0) || prefetch (warps 1..) ----
    if (warp == 0) diag_lu16<T>(W, LDW, base, k0, n, tau, RV, nb);
    else prefetch(k0);
    __syncthreads();

    // ---- A2: L21 = A21 U11^{-1} (rows NB..KA-1, threads 0..127) ||
    //      B:  U12 = L11^{-1} A12 (columns NB..KA-1, threads 128..255) ----
    if (tid < NTH / 2) {
      for (int ro = NB + tid; ro < KA; ro += NTH / 2) {
        T* row = &W[w.ph(ro) * LDW + base];
        T x[NB];
#pragma unroll
        for (int c4 = 0; c4 < NB / 4; ++c4) {
          T v[4];
          ld4(row + 4 * c4, v);
#pragma unroll
          for (int y = 0; y < 4; ++y) x[4 * c4 + y] = v[y];
        }
#pragma unroll
        for (int j = 0; j < NB; ++j) {
          T acc = x[j];
#pragma unroll
          for (int q = 0; q < j; ++q) acc -= x[q] * W[(base + q) * LDW + base + j];
          x[j] = acc * RV[j];
        }
#pragma unroll
        for (int c4 = 0; c4 < NB / 4; ++c4) st4(row + 4 * c4, {x[4 * c4], x[4 * c4 + 1], x[4 * c4 + 2], x[4 * c4 + 3]});
      }
    } else {
      for (int c = NB + tid - NTH / 2; c < KA; c += NTH / 2) {
        const int pc = w.ph(c);
        T x[NB];
#pragma unroll
        for (int r = 0; r < NB; ++r) x[r] = W[(base + r) * LDW + pc];
#pragma unroll
        for (int r = 1; r < NB; ++r) {
          T acc = x[r];
#pragma unroll
          for (int q = 0; q < r; ++q) acc -= W[(base + r) * LDW + base + q] * x[q];
          x[r] = acc;
        }
#pragma unroll
        for (int r = 1; r < NB; ++r) W[(base + r) * LDW + pc] = x[r];
      }
    }
    __syncthreads();

    // ---- D1: write the finished panel (U rows k0.., L columns k0..) ----
    // Four entries per thread are read before any is stored, so that the
    // window reads overlap (each entry is written once, to its own place).
    auto write_panel = [&](int t0, int nthr) {
      constexpr int U = 4;
      const int tot = NB * (2 * K + 1);
      for (int e0 = t0; e0 < tot; e0 += U * nthr) {
        T v[U];
        int64_t dst[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int e = e0 + u * nthr;
          dst[u] = -1;
          if (e >= tot) continue;
          const int dg = e / NB, t = e % NB;    // diagonal index c = K + i - j, position in panel
          int i, j;
          if (dg <= K) { i = k0 + t; j = i + (K - dg); }     // U(i, j), j - i = K - dg
          else { j = k0 + t; i = j + (dg - K); }             // L(i, j), i - j = dg - K
          if (i >= n || j >= n) continue;
          if (!REV) {
            dst[u] = (int64_t)dg * ld + j;
          } else {
            // keep the last K rows/cols of L~ and U~ of J A J, flipped:
            // U'(n-1-i, n-1-k) = L~(i, k), L'(n-1-k, n-1-j) = U~(k, j)
            const int kk = (dg <= K) ? i : j;
            if (kk < n - K) continue;
            dst[u] = (int64_t)(n - 1 - i) * K + (n - 1 - j);
          }
          v[u] = W[w.ph(i - k0) * LDW + w.ph(j - k0)];
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (dst[u] >= 0) F[dst[u]] = v[u];
      }
    };
    // ---- C: A22 -= L21 U12 over window rows/cols [NB, NB + K) ----
    if constexpr (TC) {
      const int Kr = (K + 15) / 16 * 16;        // trailing rows / cols touched (16-aligned groups)
      for (int e = tid; e < Kr * NB; e += NTH) {
        const int r = e / NB, q = e % NB;
        const T a = r < K ? W[w.ph(NB + r) * LDW + base + q] : T(0);     // L21(r, q)
        const T b = r < K ? W[(base + q) * LDW + w.ph(NB + r)] : T(0);    // U12(q, r)
        const int off = (r >> 3) * 128 + (q >> 3) * 64 + (r & 7) * 8 + (q & 7);
        tcx.A[off] = __float2bfloat16_rn((float)a);
        tcx.B[off] = __float2bfloat16_rn((float)b);
      }
      tc::fence_async_smem();
      __syncthreads();
      const int nmt = (Kr + kTcPiece - 1) / kTcPiece;
      const int npieces = nmt * nmt;
      constexpr uint32_t idesc = tc::idesc_bf16_f32(kTcPiece, kTcPiece);
      const int qd = warp & 3, hw = warp >> 2;
      for (int g0 = 0; g0 < npieces; g0 += 4) {
        const int gn = npieces - g0 < 4 ? npieces - g0 : 4;
        if (tid == 0) {
          tc::fence_after_sync();
          for (int p = 0; p < gn; ++p) {
            const int mt = (g0 + p) / nmt, nc = (g0 + p) % nmt;
            tc::mma_bf16(tcx.taddr + (uint32_t)(kTcPiece * p), tc::smem_desc(tcx.A + mt * kTcPiece * 16, 128, 256),
                         tc::smem_desc(tcx.B + nc * kTcPiece * 16, 128, 256), idesc, 0u);
          }
          tc::mma_commit(tcx.bar);
        }
        if (g0 == 0) write_panel(tid, NTH);   // overlaps the MMAs (it reads only the panel's rows / columns)
        tc::mbar_wait_bounded(tcx.bar, tcx.ph, tcx.spin, tcx.err, tcx.failed);
        tcx.ph ^= 1u;
        tc::fence_after_sync();
        for (int p = 0; p < gn; ++p) {
          const int mt = (g0 + p) / nmt, nc = (g0 + p) % nmt;
          const int r = mt * kTcPiece + qd * 32 + lane;      // trailing row of this lane
          for (int j = hw; j < kTcPiece / 16; j += 2) {
            const int c0 = nc * kTcPiece + j * 16;          // first of 16 trailing columns
            if (c0 >= Kr) break;                            // warp-uniform
            float v[16];
            tc::ld_32x32b_x16(tcx.taddr + ((uint32_t)(qd * 32) << 16) + (uint32_t)(kTcPiece * p + j * 16), v);
            if (r < Kr) {
              T* row = &W[w.ph(NB + r) * LDW + w.ph(NB + c0)];   // 16-aligned offsets never wrap
#pragma unroll
              for (int y4 = 0; y4 < 4; ++y4) {
                float4 x = *reinterpret_cast<float4*>(row + 4 * y4);
                x.x -= v[4 * y4]; x.y -= v[4 * y4 + 1]; x.z -= v[4 * y4 + 2]; x.w -= v[4 * y4 + 3];
                *reinterpret_cast<float4*>(row + 4 * y4) = x;
              }
            }
          }
        }
        tc::fence_before_sync();
        __syncthreads();     // TMEM read before the next group's MMAs overwrite it
      }
    } else
    {
      // TR x 4 tiles of trailing entries per thread (rows / columns in
      // 4-aligned groups up to 4 nt >= K).  In the global window FP32 takes
      // 8-row tiles: the L1 wavefronts per update (operand rows of L21 are
      // warp-broadcast, U12 columns and the trailing entries per lane) are
      // what bounds it, and a taller tile reuses each U12 load twice.
      constexpr int TR = (GW && sizeof(T) == 4) ? 8 : 4;
      const int nt = (K + 3) / 4, rl = 4 * nt, nr = (rl + TR - 1) / TR;
      for (int t = tid; t < nr * nt; t += NTH) {
        const int ti = t / nt, tj = t % nt;
        const int r0 = w.ph(NB + TR * ti), c0 = w.ph(NB + 4 * tj);   // TR- and 4-groups never wrap
        // the tile's trailing entries are loaded first, so that their L2
        // latency hides behind the products (rows past 4 nt, read in the last
        // 8-row tile, lie inside the window and are not written back)
        T v[TR][4], acc[TR][4];
        if constexpr (GW) {
#pragma unroll
          for (int x = 0; x < TR; ++x) ld4_cg(&W[(r0 + x) * LDW + c0], v[x]);
        }
#pragma unroll
        for (int x = 0; x < TR; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] = T(0);
#pragma unroll
        for (int q4 = 0; q4 < NB / 4; ++q4) {
          T bq[4][4];
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) ld4(&W[(base + 4 * q4 + qq) * LDW + c0], bq[qq]);
#pragma unroll
          for (int x = 0; x < TR; ++x) {
            T a[4];
            ld4(&W[(r0 + x) * LDW + base + 4 * q4], a);
#pragma unroll
            for (int qq = 0; qq < 4; ++qq)
#pragma unroll
              for (int y = 0; y < 4; ++y) acc[x][y] += a[qq] * bq[qq][y];
          }
        }
#pragma unroll
        for (int x = 0; x < TR; ++x) {
          if (TR * ti + x >= rl) break;     // rows past 4 nt: only in the last 8-row tile
          T* row = &W[(r0 + x) * LDW + c0];
          if constexpr (!GW) ld4(row, v[x]);
#pragma unroll
          for (int y = 0; y < 4; ++y) v[x][y] -= acc[x][y];
          if constexpr (GW) st4_cg(row, v[x]); else st4(row, v[x]);
        }
      }
    }
    if constexpr (!TC) write_panel(tid, NTH);
    if (warp > 0) cp_async_wait_all();
    __syncthreads();
    // ---- D2: slide the window by NB: entering rows/cols replace the panel's ----
    {
      Win w2{M2, LDW, w.ph(NB)};        // next window: logical offset 0 = k0 + NB
      for (int e = warp; e < NB; e += NTH / 32) {
        T* row = &W[w2.ph(ME + e) * LDW];                      // row k0+M2+e = next offset ME+e
        for (int jo = lane; jo < M2; jo += 32) row[w2.ph(jo)] = ER[e * M2 + jo];
      }
      for (int y = tid; y < ME * NB; y += NTH) {
        const int ro = y / NB, e = y % NB;
        W[w2.ph(ro) * LDW + w2.ph(ME + e)] = EC[y];           // column k0+M2+e, row k0+NB+ro
      }
      w = w2;
    }
    __syncthreads();
  }
  if (warp == 0 && lane == 0 && nb) atomicAdd(n_boosted, nb);
}

// ---------------------------------------------------------------------------
// TMA-staged block LU (window in shared memory; FP32 without the tensor-core
// update, and FP64): the elimination of band_lu_block (the same A1, A2/B and
// C arithmetic per entry, so the same factors bit for bit), with the band
// staged and the panel steps scheduled differently.
//  * The band enters through the tensor memory accelerator.  Per 16-column
//    group G of the block, one 2-D box of the band array covers the group's
//    columns (its start rounded down to 16 bytes) and the K diagonals of the
//    local lower triangle ("kept" ring, R = D + M2/16 slots: the entering
//    rows of later panels read them), and, for the D groups ahead of the
//    window, one box of the other K + 1 diagonals ("head" ring, D + 1 slots).
//    One thread issues each group D panels ahead; an mbarrier per slot counts
//    the bytes.  No per-element loads of the band remain in the loop.
//  * The window has two spare panels of physical rows and columns (M3 =
//    M2 + 32, addressed modulo M3).  While warp 0 factors a panel's diagonal
//    block (A1), the other warps write out the previous panel and scatter the
//    next window's entering rows and columns from the boxes into the slots
//    of the panel retired two steps earlier (every position of those rows
//    and columns within the next window: band values, exact zeros outside
//    the band and the block).
//  * The trailing update takes 4 x 4 register tiles in warp blocks of 4 x 8
//    tiles, so that the operand rows and columns of a warp's loads broadcast.
// Three barriers per 16 columns.
struct TmaLuGeom {
  int M2, M3, LDW, BW, R, RH, D;
  size_t kept_bytes, head_bytes, off_kept, off_head, off_rv, off_bar, smem;
};
__host__ __device__ inline size_t r128(size_t x) { return (x + 127) & ~(size_t)127; }
__host__ __device__ inline TmaLuGeom tma_lu_geom(int K, int tsz, int D) {
  TmaLuGeom g;
  g.M2 = win_m2(K);
  g.M3 = g.M2 + 2 * NB;
  g.LDW = g.M3 + 4;
  g.BW = tsz == 4 ? 20 : 18;            // 16 columns + the alignment slack, a multiple of 16 bytes
  g.D = D;
  g.R = D + g.M2 / NB;
  g.RH = D + 1;
  g.kept_bytes = r128((size_t)g.BW * K * tsz);
  g.head_bytes = r128((size_t)g.BW * (K + 1) * tsz);
  size_t off = r128((size_t)g.M3 * g.LDW * tsz);
  g.off_kept = off;
  off += (size_t)g.R * g.kept_bytes;
  g.off_head = off;
  off += (size_t)g.RH * g.head_bytes;
  g.off_rv = off;
  off += r128((size_t)NB * tsz);
  g.off_bar = off;
  off += (size_t)(g.R + g.RH) * sizeof(uint64_t);
  off += 16;                                  // the failure flag
  g.smem = off;
  return g;
}

template <typename T, bool REV>
__global__ void __launch_bounds__(256)
k_band_lu_tma(const __grid_constant__ CUtensorMap tm_kept, const __grid_constant__ CUtensorMap tm_head,
              const T* __restrict__ band, int64_t N, int K, Dev d, int block0,
              const double* __restrict__ absmax, double eps, T* __restrict__ out,
              unsigned long long* __restrict__ n_boosted, int* __restrict__ err, int D) {
  constexpr int NTH = 256;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const TmaLuGeom g = tma_lu_geom(K, (int)sizeof(T), D);
  const int b = block0 + blockIdx.x;
  const int64_t s = d.off[b];
  const int n = (int)(d.off[b + 1] - s);
  const int64_t ld = REV ? 0 : d.ld[b];
  T* __restrict__ F = REV ? out + (int64_t)(b - 1) * K * K : out + d.fbase[b];
  const T tau = (T)(eps * absmax[0]);
  const int M2 = g.M2, M3 = g.M3, LDW = g.LDW, BW = g.BW, R = g.R, RH = g.RH;
  const int KA = K + NB;
  const int G0 = M2 / NB;                    // groups of the initial window
  const int ngroups = (n + NB - 1) / NB;     // groups with columns inside the block
  T* W = reinterpret_cast<T*>(smem_raw);
  unsigned char* kept = smem_raw + g.off_kept;
  unsigned char* head = smem_raw + g.off_head;
  T* RV = reinterpret_cast<T*>(smem_raw + g.off_rv);
  uint64_t* kbar = reinterpret_cast<uint64_t*>(smem_raw + g.off_bar);
  uint64_t* hbar = kbar + R;
  int& sfail = *reinterpret_cast<int*>(hbar + RH);   // a bounded wait gave up: no more copies, no more waits
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int spin = spin_limit_of(err);
  constexpr int kAlign = 16 / (int)sizeof(T);   // elements per 16 bytes
  bool failed = false;
  unsigned long long nb = 0;

  // first band column of the box of local column group G (rounded down to 16 bytes; may be negative)
  auto box_x = [&](int G) -> int {
    const int64_t xs = REV ? s + n - (int64_t)NB * G - NB : s + (int64_t)NB * G;
    return (int)(xs - (((xs % kAlign) + kAlign) % kAlign));
  };
  // ring slots: group G's kept box is slot G mod R, its head box (G >= G0)
  // slot (G - G0) mod RH; the indices are stepped, not divided (integer
  // division by a runtime value is a long dependent chain)
  auto kept_slot = [&](int ks) { return reinterpret_cast<T*>(kept + (size_t)ks * g.kept_bytes); };
  auto head_slot = [&](int hs) { return reinterpret_cast<T*>(head + (size_t)hs * g.head_bytes); };
  // the issuing thread (tid 32): group gnext and onwards are not issued yet;
  // gks / ghs: gnext's kept slot and (from G0 on) head slot
  int gnext = 0, gks = 0, ghs = 0;
  auto issue_next = [&]() {
    const int G = gnext++;
    const int ks = gks;
    if (++gks == R) gks = 0;
    int hs = -1;
    if (G >= G0) {
      hs = ghs;
      if (++ghs == RH) ghs = 0;
    }
    if (G >= ngroups) return;
    const int x = box_x(G);
    tc::mbar_expect_tx(&kbar[ks], (unsigned)(BW * K * sizeof(T)));
    tc::tma_load_2d(kept_slot(ks), &tm_kept, x, REV ? 0 : K + 1, &kbar[ks]);
    if (hs >= 0) {
      tc::mbar_expect_tx(&hbar[hs], (unsigned)(BW * (K + 1) * sizeof(T)));
      tc::tma_load_2d(head_slot(hs), &tm_head, x, REV ? K : 0, &hbar[hs]);
    }
  };
  // bounded waits by non-blocking polls (the boxes are issued several panels
  // ahead) on a slot's barrier for the phase of the given parity
  auto wait_box = [&](uint64_t* bar, unsigned parity) {
    if (*(volatile int*)&sfail) return;
    tc::mbar_poll_bounded(bar, parity, spin, err, failed);
    if (failed) sfail = 1;
  };
  // Column of local column q in its group's box: the box starts at the group's
  // first band column rounded down to 16 bytes, i.e. cadj columns early.
  const int cadj = (int)((REV ? s + n : s) & (kAlign - 1));
  auto box_col = [&](int q) { return REV ? NB - 1 - (q & (NB - 1)) + cadj : (q & (NB - 1)) + cadj; };
  // box row of an entry with local offset dl = r - q below (kept, dl >= 1) or on / above (head) the diagonal
  auto kept_row = [&](int dl) { return REV ? K - dl : dl - 1; };
  auto head_row = [&](int dl) { return REV ? -dl : K + dl; };

  // ---- prologue: barriers, the first groups in flight, the initial window from global memory ----
  if (tid == 0) {
    for (int i = 0; i < R + RH; ++i) tc::mbar_init(&kbar[i], 1);
    tc::mbar_fence_init();
    sfail = 0;
  }
  __syncthreads();
  if (tid == 32)
    while (gnext < G0 + g.D) issue_next();      // kept boxes of groups 0 .., head boxes from G0 on
  for (int e = tid; e < M2 * M2; e += NTH) {    // logical rows / columns [0, M2), physical == logical
    const int r = e / M2, q = e % M2;
    const T* p = elem_ptr<REV>(band, N, K, s, n, r, q);
    W[r * LDW + q] = p ? *p : T(0);
  }
  if (tid == 32) {
    for (int G = 0; G < G0 && G < ngroups; ++G) wait_box(&kbar[G], 0u);   // slot G, first phase
    if (G0 < ngroups) {                       // the group entering in the first panel
      wait_box(&kbar[G0], 0u);
      wait_box(&hbar[0], 0u);
    }
  }
  __syncthreads();
  if (warp == 0) diag_lu16<T>(W, LDW, 0, 0, n, tau, RV, nb);      // A1 of the first panel
  __syncthreads();

  // Write-out of the finished panel at block row kp (U rows, L columns in the
  // factor layout), entries e = 16 dg + t enumerated by nw workers (nw a
  // multiple of 16, so a worker keeps t and steps dg by nw / 16).  LU: U(kp + t,
  // kp + t + K - dg) for dg <= K and L(kp + t + dg - K, kp + t) for dg > K go to
  // F[dg ld + j]; window and factor addresses advance by constants along a
  // worker's entries.  UL keeps only the flipped last K rows / columns.
  auto write_panel = [&](int kp, int sp, int wid, int nw) {   // sp: slot of block index kp
    const int t = wid & (NB - 1);
    const int step = nw >> 4;
    if (REV) {
      if (kp + NB <= n - K) return;          // no entry of the last K rows / columns
      for (int dg = wid >> 4; dg <= 2 * K; dg += step) {
        int oi, oj;
        if (dg <= K) { oi = t; oj = t + K - dg; }
        else { oj = t; oi = t + dg - K; }
        const int i = kp + oi, j = kp + oj;
        if (i >= n || j >= n || (dg <= K ? i : j) < n - K) continue;
        int pi = sp + oi, pj = sp + oj;
        if (pi >= M3) pi -= M3;
        if (pj >= M3) pj -= M3;
        F[(int64_t)(n - 1 - i) * K + (n - 1 - j)] = W[pi * LDW + pj];
      }
      return;
    }
    const int i0 = kp + t;                   // U row / L column of this worker
    if (i0 >= n) return;
    const int ulast = (n - 1 - i0) < K ? (n - 1 - i0) : K;   // U: j = i0 + K - dg <= n - 1
    // U part, dg <= K: window (sp + t, sp + t + K - dg), factor dg (ld - 1) + i0 + K
    {
      int dg = wid >> 4;
      int pi = sp + t;
      if (pi >= M3) pi -= M3;
      const T* wrow = W + pi * LDW;
      int pj = sp + t + K - dg;
      if (pj >= M3) pj -= M3;
      int64_t dst = (int64_t)dg * (ld - 1) + i0 + K;
      const int64_t dstep = (int64_t)step * (ld - 1);
      for (; dg <= K; dg += 4 * step) {       // four entries read before any is stored
        T v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          v[u] = wrow[pj];
          pj -= step;
          if (pj < 0) pj += M3;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int d = dg + u * step;
          if (d <= K && K - d <= ulast) F[dst] = v[u];
          dst += dstep;
        }
      }
      dg = wid >> 4;                         // this worker's first L entry
      while (dg <= K) dg += step;
      // L part, dg > K: window (sp + t + dg - K, sp + t), factor dg ld + i0
      int pl = sp + t + dg - K;               // dg - K < K + 16
      if (pl >= M3) pl -= M3;
      const int pc = pi;
      int64_t dl = (int64_t)dg * ld + i0;
      const int64_t lstep = (int64_t)step * ld;
      for (; dg <= 2 * K; dg += 4 * step) {
        T v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          v[u] = W[pl * LDW + pc];
          pl += step;
          if (pl >= M3) pl -= M3;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int d = dg + u * step;
          if (d <= 2 * K && i0 + d - K < n) F[dl] = v[u];
          dl += lstep;
        }
      }
    }
  };
  // The rows and columns that enter the window after the panel at k0 (block
  // indices ge .. ge + 15, ge = k0 + M2), over the next window's range, into
  // their slots (those of the panel retired two steps earlier); values from
  // the boxes inside the band and the block, exact zeros elsewhere (every
  // position of a reused slot is rewritten: its old entry may have been in
  // the band).  nw workers, a multiple of 16: a worker keeps e and steps t.
  // sge / s16: slots of block indices ge and k0 + 16; ksn / hsn: kept and head
  // slots of group ge / 16; g1: kept slot of group k0 / 16 + 1
  auto fill = [&](int k0, int sge, int s16, int ksn, int hsn, int g1, int wid, int nw) {
    const int ge = k0 + M2;
    const int e = wid & (NB - 1);
    const int step = nw >> 4;
    const int t0 = wid >> 4;
    // entering column q = ge + e, rows r = k0 + 16 + t (t < M2): dl = r - q runs
    // from 16 + t0 - M2 - e up by step; head box rows K + dl (dl <= 0), kept box
    // rows dl - 1 (REV: -dl and K - dl); window rows advance by step
    {
      const T* kb = kept_slot(ksn) + box_col(e);
      const T* hb = head_slot(hsn) + box_col(e);
      const int q = ge + e;
      T* wcol = W + sge + e;
      int pr = s16 + t0;
      if (pr >= M3) pr -= M3;
      const int dl0 = NB + t0 - M2 - e;
      const int rmax = n - 1 - k0 - NB;      // t <= rmax: row inside the block
      for (int t = t0, dl = dl0; t < M2; t += step, dl += step) {
        T v = T(0);
        if (q < n && t <= rmax && dl <= K && dl >= -K)
          v = dl >= 1 ? kb[(REV ? K - dl : dl - 1) * BW] : hb[(REV ? -dl : K + dl) * BW];
        wcol[pr * LDW] = v;
        pr += step;
        if (pr >= M3) pr -= M3;
      }
    }
    // entering row r = ge + e, columns q = k0 + 16 + t (t < M2 - 16): dl = r - q
    // runs down from M2 - 16 + e - t0; kept boxes of the groups k0 / 16 + 1 + t / 16
    {
      const bool rin = ge + e < n;
      T* wrow = W + (sge + e) * LDW;
      int pc = s16 + t0;
      if (pc >= M3) pc -= M3;
      const int qmax = n - 1 - k0 - NB;      // t <= qmax: column inside the block
      for (int t = t0, dl = M2 - NB + e - t0; t < M2 - NB; t += step, dl -= step) {
        T v = T(0);
        if (rin && t <= qmax && dl <= K) {
          int ks = g1 + (t >> 4);
          if (ks >= R) ks -= R;
          v = reinterpret_cast<const T*>(kept + (size_t)ks * g.kept_bytes)[(REV ? K - dl : dl - 1) * BW + box_col(t)];
        }
        wrow[pc] = v;
        pc += step;
        if (pc >= M3) pc -= M3;
      }
    }
  };
  // one 4 x 4 tile (ti, tj) of C: A22 -= L21 U12 over window offsets 16 + 4 ti .., 16 + 4 tj ..
  auto update_tile = [&](int base, int ti, int tj) {
    int r0 = base + NB + 4 * ti, c0 = base + NB + 4 * tj;   // 4-groups never wrap
    if (r0 >= M3) r0 -= M3;
    if (c0 >= M3) c0 -= M3;
    T acc[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[x][y] = T(0);
#pragma unroll
    for (int q4 = 0; q4 < NB / 4; ++q4) {
      T bq[4][4];
#pragma unroll
      for (int qq = 0; qq < 4; ++qq) ld4(&W[(base + 4 * q4 + qq) * LDW + c0], bq[qq]);
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        T a[4];
        ld4(&W[(r0 + x) * LDW + base + 4 * q4], a);
#pragma unroll
        for (int qq = 0; qq < 4; ++qq)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] += a[qq] * bq[qq][y];
      }
    }
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      T* row = &W[(r0 + x) * LDW + c0];
      T v[4];
      ld4(row, v);
#pragma unroll
      for (int y = 0; y < 4; ++y) v[y] -= acc[x][y];
      st4(row, v);
    }
  };
  const int nt = (K + 3) / 4;                // trailing tiles per side
  const int dt = nt < 4 ? nt : 4;            // tiles of the next diagonal block per side
  const int nrest = nt * nt - dt * dt;       // the other tiles
  // the write-out's workers in the solve phase: the warps none of whose threads
  // has a solve row / column (in each half of the CTA, warps (w & 3) with
  // 32 (w & 3) >= K), else every thread after its solves
  const int wfree = 4 - (K + 31) / 32 > 0 ? 4 - (K + 31) / 32 : 0;   // free warps per half
  const int nwo = wfree > 0 ? 2 * 32 * wfree : NTH;
  const int wl = warp & 3;
  const int wwo = wfree > 0 ? (wl >= 4 - wfree ? ((warp >> 2) * wfree + wl - (4 - wfree)) * 32 + lane : -1) : tid;

  // Phase B's workers besides warp 0: warp 4, which shares warp 0's scheduler,
  // stays free of C tiles so that A1's dependency chain (the critical path)
  // does not compete for that scheduler's pipes; it waits for the next boxes.
  constexpr bool kFreeWarp4 = true;
  constexpr int NWB = kFreeWarp4 ? NTH - 64 : NTH - 32;
  const int wbid = warp == 0 || (kFreeWarp4 && warp == 4) ? -1
                   : (kFreeWarp4 && warp > 4 ? tid - 64 : tid - 32);
  // this thread's tiles of the rest of C (the same every panel), packed ti << 16 | tj
  constexpr int kMaxTiles = 6;               // enough for K <= 127 over 192 threads
  int mytile[kMaxTiles];
  {
    const int wc = wbid;
#pragma unroll
    for (int k = 0; k < kMaxTiles; ++k) {
      const int u = wc + k * NWB;
      mytile[k] = -1;
      if (wc < 0 || u >= nrest) continue;
      int ti, tj;
      if (u < dt * (nt - dt)) { ti = u / (nt - dt); tj = dt + u % (nt - dt); }
      else { const int v = u - dt * (nt - dt); ti = dt + v / nt; tj = v % nt; }
      mytile[k] = (ti << 16) | tj;
    }
  }
  const int dti = lane < dt * dt ? lane / dt : 0, dtj = lane < dt * dt ? lane % dt : 0;
  // per-panel state, stepped by 16 block indices a panel: slots of k0, k0 - 16,
  // k0 + 16 and k0 + M2; the kept / head slots and parities of group (k0 + M2) / 16;
  // the kept slot of group k0 / 16 + 1
  int base = 0, pbase = M3 - NB, s16 = NB, sge = M2;
  int ksn = G0, kpar = 0, hsn = 0, hpar = 0, g1 = 1;
  auto step16 = [&](int& x) { x += NB; if (x >= M3) x -= M3; };
  int k0 = 0;
  for (; k0 < n; k0 += NB) {
    auto ph = [&](int off) { const int x = base + off; return x >= M3 ? x - M3 : x; };
    // ---- phase A: L21 = A21 U11^{-1} (threads 0..127) || U12 = L11^{-1} A12 (128..255)
    //      || the previous panel's write-out (the other threads) ----
    if (tid < NTH / 2) {
      for (int ro = NB + tid; ro < KA; ro += NTH / 2) {
        T* row = &W[ph(ro) * LDW + base];
        T x[NB];
#pragma unroll
        for (int c4 = 0; c4 < NB / 4; ++c4) {
          T v[4];
          ld4(row + 4 * c4, v);
#pragma unroll
          for (int y = 0; y < 4; ++y) x[4 * c4 + y] = v[y];
        }
#pragma unroll
        for (int j = 0; j < NB; ++j) {
          T acc = x[j];
#pragma unroll
          for (int q = 0; q < j; ++q) acc -= x[q] * W[(base + q) * LDW + base + j];
          x[j] = acc * RV[j];
        }
#pragma unroll
        for (int c4 = 0; c4 < NB / 4; ++c4) st4(row + 4 * c4, {x[4 * c4], x[4 * c4 + 1], x[4 * c4 + 2], x[4 * c4 + 3]});
      }
    } else {
      for (int c = NB + tid - NTH / 2; c < KA; c += NTH / 2) {
        const int pc = ph(c);
        T x[NB];
#pragma unroll
        for (int r = 0; r < NB; ++r) x[r] = W[(base + r) * LDW + pc];
#pragma unroll
        for (int r = 1; r < NB; ++r) {
          T acc = x[r];
#pragma unroll
          for (int q = 0; q < r; ++q) acc -= W[(base + r) * LDW + base + q] * x[q];
          x[r] = acc;
        }
#pragma unroll
        for (int r = 1; r < NB; ++r) W[(base + r) * LDW + pc] = x[r];
      }
    }
    if (k0 > 0 && wwo >= 0) write_panel(k0 - NB, pbase, wwo, nwo);
    __syncthreads();

    // ---- phase B: warp 0 updates the next panel's diagonal block and factors it
    //      (A1 one panel ahead) || the rest of C, the next group's copies and the
    //      next window's entering rows / columns (warps 1-3, 5-7; warp 4, which
    //      shares warp 0's scheduler, stays idle) ----
    if (warp == 0) {
      if (lane < dt * dt) update_tile(base, dti, dtj);
      __syncwarp();
      if (k0 + NB < n) diag_lu16<T>(W, LDW, ph(NB), k0 + NB, n, tau, RV, nb);
    } else if (kFreeWarp4 && warp == 4) {
      // warp 4 (idle here, beside warp 0 on its scheduler): the boxes of the
      // group whose columns enter in the next panel's phase B
      if (lane == 0 && k0 / NB + G0 + 1 < ngroups) {
        int ks = ksn + 1, kq = kpar, hs = hsn + 1, hq = hpar;
        if (ks == R) { ks = 0; kq ^= 1; }
        if (hs == RH) { hs = 0; hq ^= 1; }
        wait_box(&kbar[ks], (unsigned)kq);
        wait_box(&hbar[hs], (unsigned)hq);
      }
    } else {
#pragma unroll
      for (int k = 0; k < kMaxTiles; ++k)
        if (mytile[k] >= 0) update_tile(base, mytile[k] >> 16, mytile[k] & 0xffff);
      if (tid == 32 && !*(volatile int*)&sfail) issue_next();   // group k0 / 16 + G0 + D (the slot's
                                                                // last readers are behind the barriers)
      if (!kFreeWarp4 && tid == NTH / 2 && k0 / NB + G0 + 1 < ngroups) {   // the next group's boxes
        int ks = ksn + 1, kq = kpar, hs = hsn + 1, hq = hpar;
        if (ks == R) { ks = 0; kq ^= 1; }
        if (hs == RH) { hs = 0; hq ^= 1; }
        wait_box(&kbar[ks], (unsigned)kq);
        wait_box(&hbar[hs], (unsigned)hq);
      }
      fill(k0, sge, s16, ksn, hsn, g1, wbid, NWB);
    }
    __syncthreads();
    pbase = base;
    step16(base);
    step16(s16);
    step16(sge);
    if (++ksn == R) { ksn = 0; kpar ^= 1; }
    if (++hsn == RH) { hsn = 0; hpar ^= 1; }
    if (++g1 == R) g1 = 0;
  }
  // the last panel's write-out; then no copy may be left in flight
  if (k0 > 0) write_panel(k0 - NB, pbase, tid, NTH);
  if (tid == 32) {
    for (int G = gnext - R > 0 ? gnext - R : 0; G < gnext; ++G) {
      if (G >= ngroups) break;
      bool gave_up = false;
      tc::mbar_wait_bounded(&kbar[G % R], (unsigned)((G / R) & 1), kDefaultSpin, nullptr, gave_up);
    }
    for (int G = gnext - RH > G0 ? gnext - RH : G0; G < gnext; ++G) {
      if (G >= ngroups) break;
      bool gave_up = false;
      tc::mbar_wait_bounded(&hbar[(G - G0) % RH], (unsigned)(((G - G0) / RH) & 1), kDefaultSpin, nullptr,
                            gave_up);
    }
  }
  if (warp == 0 && lane == 0 && nb) atomicAdd(n_boosted, nb);
}

// shared memory of the factor kernel: window (unless global) + staging
// (+ the tensor-core operands, barrier and TMEM slot)
__host__ __device__ inline size_t lu_smem_hd(int K, bool fp64, bool global_window, bool tc) {
  const int M2 = win_m2(K);
  const size_t ts = fp64 ? sizeof(double) : sizeof(float);
  size_t b = ((size_t)NB * M2 + (size_t)(M2 - NB) * NB + NB) * ts;
  if (!global_window) b += ((size_t)M2 * (M2 + 4) * ts + 15) & ~(size_t)15;
  if (tc) b = ((b + 127) & ~(size_t)127) + tc_bytes(K);
  return b;
}
__host__ __device__ inline size_t lu_tc_offset(int K, bool global_window) {
  return (lu_smem_hd(K, false, global_window, false) + 127) & ~(size_t)127;
}

template <typename T, bool REV, bool GW, bool TC>
__global__ void __launch_bounds__(lu_threads(GW, TC))
k_band_lu(const T* __restrict__ band, int64_t N, int K, Dev d, int block0,
          const double* __restrict__ absmax, double eps, T* __restrict__ out,
          unsigned long long* __restrict__ n_boosted, T* __restrict__ wscratch, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int b = block0 + blockIdx.x;
  const int64_t s = d.off[b];
  const int n = (int)(d.off[b + 1] - s);
  const int64_t ld = REV ? 0 : d.ld[b];
  T* F = REV ? out + (int64_t)(b - 1) * K * K : out + d.fbase[b];
  const int M2 = win_m2(K);
  T* wg = GW ? wscratch + (int64_t)blockIdx.x * M2 * (M2 + 4) : nullptr;
  TcCtx tcx;
  if constexpr (TC) tc_setup(smem_raw + lu_tc_offset(K, GW), K, tcx, err);
  band_lu_block<T, REV, GW, TC, lu_threads(GW, TC)>(smem_raw, band, N, K, s, n, ld, F, (T)(eps * absmax[0]),
                                                   n_boosted, wg, tcx);
  if constexpr (TC) tc_teardown(tcx, K);
}

// Persistent LU over a work list of blocks of many systems (LuItem, longest
// first): each CTA takes the next item from an atomic counter until the list
// is exhausted, so one launch factors every block of a batch.
template <typename T, bool GW, bool TC>
__global__ void __launch_bounds__(lu_threads(GW, TC))
k_band_lu_items(const LuItem* __restrict__ items, int nitems, unsigned* __restrict__ counter,
                T* __restrict__ wscratch, int64_t wstride, int Kmax, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int cur;
  TcCtx tcx;
  if constexpr (TC) tc_setup(smem_raw + lu_tc_offset(Kmax, GW), Kmax, tcx, err);
  for (;;) {
    if (threadIdx.x == 0) cur = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int it = cur;
    __syncthreads();          // every thread has read cur before it changes
    if (it >= nitems) break;
    const LuItem I = items[it];
    band_lu_block<T, false, GW, TC, lu_threads(GW, TC)>(smem_raw, reinterpret_cast<const T*>(I.band), I.N, I.K, I.s, I.n, I.ld,
                                    reinterpret_cast<T*>(I.F), (T)(I.eps * I.absmax[0]), I.nb,
                                    GW ? wscratch + (int64_t)blockIdx.x * wstride : nullptr, tcx);
    __syncthreads();
  }
  if constexpr (TC) tc_teardown(tcx, Kmax);
}

template <typename T, bool REV, bool GW>
auto lu_kernel(bool tc) {
  if constexpr (sizeof(T) == 4) return tc ? k_band_lu<T, REV, GW, true> : k_band_lu<T, REV, GW, false>;
  else return k_band_lu<T, REV, GW, false>;
}

// cuTensorMapEncodeTiled from the driver (through the runtime's entry-point
// query, so that the library needs no link to libcuda)
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p) {
      cudaGetLastError();
      return nullptr;
    }
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// Tensor map of the band array as a 2-D tensor: N columns (innermost) by 2K + 1
// diagonals, boxes of bw columns by `rows` diagonals.  False where TMA cannot
// address it (the base or the row pitch not 16-byte aligned).
bool band_tensor_map(CUtensorMap* m, const void* band, int64_t N, int K, int tsz, int bw, int rows) {
  EncodeTiledFn f = encode_tiled();
  if (!f || (reinterpret_cast<uintptr_t>(band) & 15u) || ((N * tsz) & 15) || rows < 1 || rows > 256) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)(2 * K + 1)};
  const cuuint64_t strides[1] = {(cuuint64_t)N * (cuuint64_t)tsz};
  const cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)rows};
  const cuuint32_t es[2] = {1, 1};
  return f(m, tsz == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<void*>(band),
           dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The band staging of the shared-window LU: TMA boxes (default) or, with the
// environment variable SAP_LU_STAGING=cp_async, the per-element cp.async
// staging of band_lu_block (both give the same factors; the switch exists to
// compare them).
bool lu_tma_wanted() {
  const char* v = std::getenv("SAP_LU_STAGING");
  return !(v && std::strcmp(v, "cp_async") == 0);
}

// Launch k_band_lu_tma when it applies (shared-memory window with the ring of
// boxes, TMA-addressable band); cudaErrorNotSupported otherwise.
template <typename T, bool REV>
cudaError_t launch_lu_tma(const T* band, int64_t N, int K, int nblocks, int block0, Dev d, const double* absmax,
                          double eps, T* out, unsigned long long* nb, int* err, cudaStream_t s) {
  if (!lu_tma_wanted() || K + 1 > 256) return cudaErrorNotSupported;
  // prefetch depth: the deepest ring (up to 8 groups ahead) that fits
  int D = 8;
  TmaLuGeom g = tma_lu_geom(K, (int)sizeof(T), D);
  while (D > 1 && g.smem + 1024 > kSmemPerBlock) g = tma_lu_geom(K, (int)sizeof(T), --D);
  if (g.smem + 1024 > kSmemPerBlock) return cudaErrorNotSupported;
  CUtensorMap tk, th;
  if (!band_tensor_map(&tk, band, N, K, (int)sizeof(T), g.BW, K) ||
      !band_tensor_map(&th, band, N, K, (int)sizeof(T), g.BW, K + 1))
    return cudaErrorNotSupported;
  auto kern = k_band_lu_tma<T, REV>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
  if (e != cudaSuccess) return e;
  // its ring and spare panels take more shared memory than the per-element
  // staging: where that costs a wave of CTAs (many blocks, wide bands) the
  // per-element staging runs instead
  {
    int dev = 0, sms = 0, occ_t = 0, occ_c = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return cudaErrorNotSupported;
    const size_t smem_c = lu_smem_used(K, sizeof(T) == 8, false, false);
    auto classic = lu_kernel<T, REV, false>(false);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_t, kern, 256, g.smem) != cudaSuccess ||
        cudaFuncSetAttribute(classic, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_c, classic, lu_threads(false, false), smem_c) !=
            cudaSuccess) {
      cudaGetLastError();
      return cudaErrorNotSupported;
    }
    const int waves_t = occ_t > 0 ? (nblocks + sms * occ_t - 1) / (sms * occ_t) : 1 << 30;
    const int waves_c = occ_c > 0 ? (nblocks + sms * occ_c - 1) / (sms * occ_c) : 1 << 30;
    if (waves_t > waves_c) return cudaErrorNotSupported;
  }
  count_launches(1);
  kern<<<nblocks, 256, g.smem, s>>>(tk, th, band, N, K, d, block0, absmax, eps, out, nb, err, D);
  return cudaGetLastError();
}

template <typename T, bool REV>
cudaError_t launch_lu_impl(const T* band, int64_t N, int K, int nblocks, int block0, Dev d,
                           const double* absmax, double eps, T* out, unsigned long long* nb,
                           T* wscratch, bool tc, int* err, cudaStream_t s) {
  if (nblocks <= 0) return cudaSuccess;
  tc = tc && sizeof(T) == 4;
  const bool gw = lu_window_global(K, sizeof(T) == 8, tc);
  if (gw && !wscratch) return cudaErrorInvalidValue;
  if (!tc && !gw) {
    const cudaError_t et = launch_lu_tma<T, REV>(band, N, K, nblocks, block0, d, absmax, eps, out, nb, err, s);
    if (et != cudaErrorNotSupported) return et;
  }
  const size_t smem = lu_smem_used(K, sizeof(T) == 8, gw, tc);
  auto kern = gw ? lu_kernel<T, REV, true>(tc) : lu_kernel<T, REV, false>(tc);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  count_launches(1);
  kern<<<nblocks, lu_threads(gw, tc), smem, s>>>(band, N, K, d, block0, absmax, eps, out, nb, wscratch, err);
  return cudaGetLastError();
}

}  // namespace

size_t lu_smem_used(int K, bool fp64, bool global_window, bool tc) { return lu_smem_hd(K, fp64, global_window, tc); }
bool lu_window_global(int K, bool fp64, bool tc) { return lu_smem_used(K, fp64, false, tc) > kSmemPerBlock; }
size_t lu_window_elems(int K) {
  const int M2 = win_m2(K);
  return (size_t)M2 * (M2 + 4);
}

size_t lu_smem_bytes(int K, bool fp64, bool tc) { return lu_smem_used(K, fp64, lu_window_global(K, fp64, tc), tc); }

namespace {

// ---- max |a_ij| over the in-band entries (boost threshold scale) ----
// Grid (gx, 2K+1): blockIdx.y is the band row c (entries a(j + c - K, j)),
// whose valid columns are j in [max(0, K - c), min(N, N + K - c)).
__device__ __forceinline__ void absmax_commit(double m, double* out) {
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0)
    atomicMax(reinterpret_cast<unsigned long long*>(out), (unsigned long long)__double_as_longlong(m));
}

__global__ void k_absmax(const double* __restrict__ band, int64_t N, int K, double* out) {
  const int c = blockIdx.y;
  const int64_t lo = K - c > 0 ? K - c : 0;
  const int64_t hi = N + K - c < N ? N + K - c : N;
  const double* row = band + (int64_t)c * N;
  double m = 0.0;
  for (int64_t j = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < hi; j += (int64_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs(row[j]));
  absmax_commit(m, out);
}

// max |a_ij| over the in-band entries and an FP32 copy of the band (RN),
// padding slots written as 0: the FP32 factorisation then loads FP32.
__global__ void k_absmax_cast(const double* __restrict__ band, int64_t N, int K, double* out,
                              float* __restrict__ bandf) {
  const int c = blockIdx.y;
  const int64_t lo = K - c > 0 ? K - c : 0;
  const int64_t hi = N + K - c < N ? N + K - c : N;
  const double* row = band + (int64_t)c * N;
  float* rowf = bandf + (int64_t)c * N;
  double m = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
    float v = 0.f;
    if (j >= lo && j < hi) {
      const double a = row[j];
      m = fmax(m, fabs(a));
      v = (float)a;
    }
    rowf[j] = v;
  }
  absmax_commit(m, out);
}

}  // namespace

static dim3 absmax_grid(int K) {
  const int rows = 2 * K + 1;
  const int gx = std::max(1, 152 * 8 / rows);
  return dim3(gx, rows);
}

cudaError_t launch_absmax_cast(const double* band, int64_t N, int K, double* out, float* bandf, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  count_launches(1);
  k_absmax_cast<<<absmax_grid(K), 256, 0, s>>>(band, N, K, out, bandf);
  return cudaGetLastError();
}

cudaError_t launch_absmax(const double* band, int64_t N, int K, double* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  count_launches(1);
  k_absmax<<<absmax_grid(K), 256, 0, s>>>(band, N, K, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_factor_lu(const T* band, int64_t N, int K, int P, Dev d, const double* absmax,
                             double eps, T* F, unsigned long long* nb, T* wscratch, bool tc, int* err,
                             cudaStream_t s) {
  return launch_lu_impl<T, false>(band, N, K, P, 0, d, absmax, eps, F, nb, wscratch, tc, err, s);
}

template <typename T>
cudaError_t launch_factor_ul(const T* band, int64_t N, int K, int P, Dev d, const double* absmax,
                             double eps, T* ULt, unsigned long long* nb, T* wscratch, bool tc, int* err,
                             cudaStream_t s) {
  // UL tiles are only needed for blocks 1..P-1 (the W^(t) tips)
  return launch_lu_impl<T, true>(band, N, K, P - 1, 1, d, absmax, eps, ULt, nb, wscratch, tc, err, s);
}

int lu_items_grid(int nitems, int Kmax, bool fp64, bool tc) {
  tc = tc && !fp64;
  const size_t smem = lu_smem_bytes(Kmax, fp64, tc);
  const bool gw = lu_window_global(Kmax, fp64, tc);
  int per_sm = 0;
  auto occ = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, lu_threads(gw, tc), smem);
  };
  if (fp64) gw ? occ(k_band_lu_items<double, true, false>) : occ(k_band_lu_items<double, false, false>);
  else if (tc) gw ? occ(k_band_lu_items<float, true, true>) : occ(k_band_lu_items<float, false, true>);
  else gw ? occ(k_band_lu_items<float, true, false>) : occ(k_band_lu_items<float, false, false>);
  // resident CTAs hold their TMEM for the whole launch: no more per SM than fit in its 512 columns
  if (tc) per_sm = std::min(per_sm, (int)(512u / tc_cols(Kmax)));
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max(1, std::min(nitems, std::max(1, per_sm) * sms));
}

template <typename T>
cudaError_t launch_factor_lu_items(const LuItem* items, int nitems, int Kmax, unsigned* counter, T* wscratch,
                                   bool tc, int* err, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  const bool fp64 = sizeof(T) == 8;
  tc = tc && !fp64;
  const bool gw = lu_window_global(Kmax, fp64, tc);
  if (gw && !wscratch) return cudaErrorInvalidValue;
  const size_t smem = lu_smem_bytes(Kmax, fp64, tc);
  void (*kern)(const LuItem*, int, unsigned*, T*, int64_t, int, int*);
  if constexpr (sizeof(T) == 4) {
    if (tc) kern = gw ? k_band_lu_items<T, true, true> : k_band_lu_items<T, false, true>;
    else kern = gw ? k_band_lu_items<T, true, false> : k_band_lu_items<T, false, false>;
  } else {
    kern = gw ? k_band_lu_items<T, true, false> : k_band_lu_items<T, false, false>;
  }
  const int grid = lu_items_grid(nitems, Kmax, fp64, tc);   // also sets the shared-memory attribute
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  count_launches(1);
  kern<<<grid, lu_threads(gw, tc), smem, s>>>(items, nitems, counter, wscratch, (int64_t)lu_window_elems(Kmax),
                                              Kmax, err);
  return cudaGetLastError();
}

template cudaError_t launch_factor_lu_items<float>(const LuItem*, int, int, unsigned*, float*, bool, int*,
                                                   cudaStream_t);
template cudaError_t launch_factor_lu_items<double>(const LuItem*, int, int, unsigned*, double*, bool, int*,
                                                    cudaStream_t);

template cudaError_t launch_factor_lu<float>(const float*, int64_t, int, int, Dev, const double*, double,
                                             float*, unsigned long long*, float*, bool, int*, cudaStream_t);
template cudaError_t launch_factor_lu<double>(const double*, int64_t, int, int, Dev, const double*, double,
                                              double*, unsigned long long*, double*, bool, int*, cudaStream_t);
template cudaError_t launch_factor_ul<float>(const float*, int64_t, int, int, Dev, const double*, double,
                                             float*, unsigned long long*, float*, bool, int*, cudaStream_t);
template cudaError_t launch_factor_ul<double>(const double*, int64_t, int, int, Dev, const double*, double,
                                              double*, unsigned long long*, double*, bool, int*, cudaStream_t);

}  // namespace sap
