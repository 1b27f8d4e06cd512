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
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <algorithm>
#include <cstdint>
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

template <typename T> __device__ __forceinline__ T rcp(T p) { return T(1) / p; }
template <> __device__ __forceinline__ float rcp<float>(float p) { return __frcp_rn(p); }

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

  // A1: LU of the NB x NB diagonal block at physical rows / columns pb ..
  // pb + NB - 1 of the panel that starts at block row pk0 (warp 0): pivot row
  // by shuffles, boosted pivot, multipliers; the reciprocals of the pivots go
  // to RV.
  auto factor_diag = [&](int pb, int pk0) {
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
      T p = u[j];
      if (pk0 + j < n) {
        if ((p < T(0) ? -p : p) < tau) {
          p = p >= T(0) ? tau : -tau;
          ++nb;
        }
      } else {
        p = T(1);   // padding past the block: rows there are all zero
      }
      const T rinv = rcp(p);
      if (lane > j) {
        const T l = pv[j] * rinv;
        pv[j] = l;
#pragma unroll
        for (int c = j + 1; c < NB; ++c) pv[c] -= l * u[c];
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
  };
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
    if (warp == 0) factor_diag(base, k0);
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

template <typename T, bool REV>
cudaError_t launch_lu_impl(const T* band, int64_t N, int K, int nblocks, int block0, Dev d,
                           const double* absmax, double eps, T* out, unsigned long long* nb,
                           T* wscratch, bool tc, int* err, cudaStream_t s) {
  if (nblocks <= 0) return cudaSuccess;
  tc = tc && sizeof(T) == 4;
  const bool gw = lu_window_global(K, sizeof(T) == 8, tc);
  if (gw && !wscratch) return cudaErrorInvalidValue;
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
