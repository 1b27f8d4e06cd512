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

constexpr int LDS = CH + 1;      // padded shared-memory row

// S[t][j] = sweep entry (p0 + t, p0 - k * 32 + j) where its position
// distance k * 32 + t - j lies in [0, K], else 0 (identity padding comes
// from sweep_entry).  The NWARPS warps walk the 63 diagonals t - j = const
// with lane = j, so each load of the band-stored factor reads consecutive
// addresses; all loads of a thread are issued before its stores.
template <int MODE, int NWARPS, typename T>
__device__ __forceinline__ void load_tile(T* S, const T* F, int K, int n, int ld, int p0, int k, int c) {
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  constexpr int ROWS = (2 * CH - 1 + NWARPS - 1) / NWARPS;
  T v[ROWS];
#pragma unroll
  for (int i = 0; i < ROWS; ++i) {
    const int delta = warp + i * NWARPS - (CH - 1);   // t - j
    const int t = lane + delta;
    const int dist = k * CH + delta;
    v[i] = (delta < CH && t >= 0 && t < CH && c >= k && dist >= 0 && dist <= K)
               ? sweep_entry<MODE>(F, K, n, ld, p0 + t, p0 - k * CH + lane)
               : T(0);
  }
#pragma unroll
  for (int i = 0; i < ROWS; ++i) {
    const int delta = warp + i * NWARPS - (CH - 1);
    const int t = lane + delta;
    if (delta < CH && t >= 0 && t < CH) S[t * LDS + lane] = v[i];
  }
}

// One CTA per chunk: the 32 (1 + NG) columns of [MINV_c | G_{c,1} .. G_{c,NG}]
// are the solutions of A_c x = e_j and A_c x = (column j of B_{c,k}), all
// solved at once by forward substitution, TPC threads per column (thread
// `part` keeps x_r for r = part mod TPC in registers; the partial dot
// products of a row are combined by shuffles).  Same matrices as forming
// A_c^{-1} and multiplying, different rounding order.
template <int NG>
struct ChunkCfg {
  static constexpr int NCOL = CH * (1 + NG);
  static constexpr int TPC = NG == 1 ? 8 : (NG <= 3 ? 4 : (NG <= 7 ? 2 : 1));
  static constexpr int NTH = NCOL * TPC;      // 512, 384, 512, 320, 384, 448, 512
};

template <typename T>
size_t chunk_smem_bytes(int K) {
  const int ng = (K + CH - 1) / CH;
  return (size_t)(1 + ng) * CH * LDS * sizeof(T) + CH * sizeof(T);
}

template <typename T, int MODE, int NG>
__global__ void __launch_bounds__(ChunkCfg<NG>::NTH)
k_chunk_mats(const T* __restrict__ Fall, int K, Dev d, const int64_t* __restrict__ cbase, T* __restrict__ out) {
  using C = ChunkCfg<NG>;
  constexpr int TPC = C::TPC, NW = C::NTH / 32, XR = CH / TPC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* A = reinterpret_cast<T*>(smem_raw);        // in-chunk block, then B_1 .. B_NG
  T* Bs = A + CH * LDS;
  T* Rd = Bs + NG * CH * LDS;
  const int b = blockIdx.y;
  const int ld = (int)d.ld[b];
  const int nch = ld / CH;
  const int c = blockIdx.x;
  if (c >= nch) return;
  const int n = (int)(d.off[b + 1] - d.off[b]);
  const T* F = Fall + d.fbase[b];
  const int tid = threadIdx.x;
  const int p0 = c * CH;
  load_tile<MODE, NW>(A, F, K, n, ld, p0, 0, c);
#pragma unroll
  for (int k = 1; k <= NG; ++k) load_tile<MODE, NW>(Bs + (k - 1) * CH * LDS, F, K, n, ld, p0, k, c);
  __syncthreads();
  if (tid < CH) Rd[tid] = T(1) / A[tid * LDS + tid];
  __syncthreads();
  const int col = tid / TPC, part = tid % TPC;
  const T* Bcol = col >= CH ? Bs + ((col - CH) / CH) * CH * LDS + (col % CH) : nullptr;
  T xr[XR];
#pragma unroll
  for (int r = 0; r < CH; ++r) {
    T acc = T(0);
#pragma unroll
    for (int m = 0; m <= r / TPC; ++m) {
      const int q = m * TPC + part;
      if (q < r) acc += A[r * LDS + q] * xr[m];
    }
#pragma unroll
    for (int o = TPC / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    const T rhs = Bcol ? Bcol[r * LDS] : (r == col ? T(1) : T(0));
    const T x = (rhs - acc) * Rd[r];
    if (r % TPC == part) xr[r / TPC] = x;
  }
  // stored column-major (element (t, j) at j * 32 + t): the sweep's lane t
  // reads its row as 32 conflict-free shared-memory loads.  The columns are
  // staged in the tile area (row stride 33) and the chunk's contiguous block
  // written out by consecutive threads.
  __syncthreads();                  // the tiles are read no more
  T* St = A;
#pragma unroll
  for (int m = 0; m < XR; ++m) St[col * LDS + m * TPC + part] = xr[m];
  __syncthreads();
  T* M = out + cbase[b] + (int64_t)c * (1 + NG) * CH * CH;
  for (int e = tid; e < C::NCOL * CH; e += C::NTH) M[e] = St[(e / CH) * LDS + e % CH];
}

// The same solves for wide bands (ng > 7 couplings, ng known at run time):
// one thread per column (32 (1 + ng) threads), the tiles loaded by the first
// eight warps.  Same rounding order as k_chunk_mats with TPC = 1.
constexpr int kWideMaxNg = 17;
constexpr int kWideMaxThreads = CH * (1 + kWideMaxNg);

template <typename T, int MODE>
__global__ void __launch_bounds__(kWideMaxThreads)
k_chunk_mats_wide(const T* __restrict__ Fall, int K, int ng, Dev d, const int64_t* __restrict__ cbase,
                  T* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* A = reinterpret_cast<T*>(smem_raw);        // in-chunk block, then B_1 .. B_ng
  T* Bs = A + CH * LDS;
  T* Rd = Bs + ng * CH * LDS;
  const int b = blockIdx.y;
  const int ld = (int)d.ld[b];
  const int nch = ld / CH;
  const int c = blockIdx.x;
  if (c >= nch) return;
  const int n = (int)(d.off[b + 1] - d.off[b]);
  const T* F = Fall + d.fbase[b];
  const int tid = threadIdx.x;
  const int p0 = c * CH;
  if (tid < 8 * 32) {
    load_tile<MODE, 8>(A, F, K, n, ld, p0, 0, c);
    for (int k = 1; k <= ng; ++k) load_tile<MODE, 8>(Bs + (k - 1) * CH * LDS, F, K, n, ld, p0, k, c);
  }
  __syncthreads();
  if (tid < CH) Rd[tid] = T(1) / A[tid * LDS + tid];
  __syncthreads();
  const int col = tid;
  const T* Bcol = col >= CH ? Bs + ((col - CH) / CH) * CH * LDS + (col % CH) : nullptr;
  T xr[CH];
#pragma unroll
  for (int r = 0; r < CH; ++r) {
    T acc = T(0);
#pragma unroll
    for (int q = 0; q < r; ++q) acc += A[r * LDS + q] * xr[q];
    const T rhs = Bcol ? Bcol[r * LDS] : (r == col ? T(1) : T(0));
    xr[r] = (rhs - acc) * Rd[r];
  }
  __syncthreads();                  // staged like k_chunk_mats, then written out contiguously
  T* St = A;
#pragma unroll
  for (int m = 0; m < CH; ++m) St[col * LDS + m] = xr[m];
  __syncthreads();
  T* M = out + cbase[b] + (int64_t)c * (1 + ng) * CH * CH;
  const int ncol = CH * (1 + ng);
  for (int e = tid; e < ncol * CH; e += ncol) M[e] = St[(e / CH) * LDS + e % CH];
}

template <typename T, int MODE, int NG>
void launch_mode(dim3 grid, size_t smem, const T* F, int K, Dev d, const int64_t* cbase, T* out, cudaStream_t s) {
  auto kern = k_chunk_mats<T, MODE, NG>;
  if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  kern<<<grid, ChunkCfg<NG>::NTH, smem, s>>>(F, K, d, cbase, out);
}

template <typename T, int MODE>
void launch_mode_ng(int ng, dim3 grid, size_t smem, const T* F, int K, Dev d, const int64_t* cbase, T* out,
                    cudaStream_t s) {
  switch (ng) {
    case 1: launch_mode<T, MODE, 1>(grid, smem, F, K, d, cbase, out, s); break;
    case 2: launch_mode<T, MODE, 2>(grid, smem, F, K, d, cbase, out, s); break;
    case 3: launch_mode<T, MODE, 3>(grid, smem, F, K, d, cbase, out, s); break;
    case 4: launch_mode<T, MODE, 4>(grid, smem, F, K, d, cbase, out, s); break;
    case 5: launch_mode<T, MODE, 5>(grid, smem, F, K, d, cbase, out, s); break;
    case 6: launch_mode<T, MODE, 6>(grid, smem, F, K, d, cbase, out, s); break;
    case 7: launch_mode<T, MODE, 7>(grid, smem, F, K, d, cbase, out, s); break;
    default: {
      auto kern = k_chunk_mats_wide<T, MODE>;
      if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      kern<<<grid, CH * (1 + ng), smem, s>>>(F, K, ng, d, cbase, out);
    } break;
  }
}

}  // namespace

size_t chunk_mats_smem_bytes(int K, bool fp64) {
  if ((K + CH - 1) / CH > kWideMaxNg) return ~(size_t)0;     // more couplings than one CTA has columns for
  return fp64 ? chunk_smem_bytes<double>(K) : chunk_smem_bytes<float>(K);
}

template <typename T>
cudaError_t launch_chunk_mats(const T* F, int K, int P, Dev d, const int64_t* cbase, int max_nch, int mode, T* out,
                              cudaStream_t s) {
  dim3 grid(max_nch, P);
  const size_t smem = chunk_smem_bytes<T>(K);
  const int ng = (K + CH - 1) / CH;
  if (ng > kWideMaxNg) return cudaErrorInvalidValue;
  count_launches(1);
  switch (mode) {
    case 0: launch_mode_ng<T, 0>(ng, grid, smem, F, K, d, cbase, out, s); break;
    case 1: launch_mode_ng<T, 1>(ng, grid, smem, F, K, d, cbase, out, s); break;
    case 2: launch_mode_ng<T, 2>(ng, grid, smem, F, K, d, cbase, out, s); break;
    default: launch_mode_ng<T, 3>(ng, grid, smem, F, K, d, cbase, out, s); break;
  }
  return cudaGetLastError();
}

namespace {

// ---- transfer matrices of the segmented sweeps ----
//
// A sweep of one block can be cut at chunk boundaries into S segments that
// run concurrently.  Segment s (chunks [c0, c1)) sees the rest of the sweep
// only through its history h: the z values of the ng chunks before c0.  Run
// with zero history it yields zhat; by linearity its true values are
// z = zhat + X h, with
//     X_c = - sum_{k=1..ng} G_{c,k} X_{c-k},   c = c0 .. c1-1,
// started from X_{c0-ng+i} = the identity rows of history chunk i.  Only the
// last KH = hist_width(K) history positions couple into the segment (the
// columns of X for the others stay exactly zero), so this kernel stores, per
// block and segment s >= 1, the KH columns of X for those positions
// (column-major over the segment's positions, cpsmax 32 rows per segment) for
// the correction z += X h of the apply, and the transfer matrix T_s (those
// columns on the segment's last KH positions, KH x KH, row-major), which
// carries the history from segment to segment:
//     tail_s = zhat_tail_s + T_s tail_{s-1}.
// One CTA per block and segment s >= 1; thread (q, rg) computes column q of
// rows rg R .. rg R + R - 1 of every X_c (broadcast 16-byte reads of G,
// conflict-free reads of X; X rows padded by one element so that the
// column-major store reads them conflict-free too).
template <typename T, int NG>
struct SegTrans {
  static constexpr int NGW = CH * NG;
  static constexpr int XLD = NGW + 1;                      // padded X row
  static constexpr int RG = (NG == 3) ? 2 : 256 / NGW;   // row groups
  static constexpr int R = CH / RG;                        // rows per thread
  static constexpr int NTH = NGW * RG;
  static constexpr size_t xbytes = (size_t)(NG + 1) * CH * XLD * sizeof(T);
  static constexpr size_t gbytes = (size_t)NG * CH * CH * sizeof(T);
  // G double-buffered (the next chunk's couplings in flight) when it fits
  static constexpr bool DB = xbytes + 2 * gbytes <= 227 * 1024;
  static constexpr size_t smem = xbytes + (DB ? 2 : 1) * gbytes;
};

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; };
template <> struct Vec16<double> { using type = double2; };

template <typename T, int NG>
__global__ void __launch_bounds__(256)
k_seg_trans(const T* __restrict__ Mall, const int64_t* __restrict__ cbase, Dev d, int S, int cpsmax, int kh,
            T* __restrict__ Tout, T* __restrict__ Xout) {
  using C = SegTrans<T, NG>;
  constexpr int NGW = C::NGW, XLD = C::XLD, R = C::R, NTH = C::NTH;
  constexpr int E = 16 / (int)sizeof(T);
  using V = typename Vec16<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Gbuf = reinterpret_cast<T*>(smem_raw);       // G_{c,1..NG}, column-major as stored (x2 if DB)
  T* X = Gbuf + (C::DB ? 2 : 1) * NG * CH * CH;   // (NG + 1) ring slots x 32 x XLD
  const int b = blockIdx.y, s = blockIdx.x + 1;
  const int nch = (int)(d.ld[b] / CH);
  const int cps = seg_chunks(nch, S);
  const int c0 = s * cps, c1 = min(nch, c0 + cps);
  if (c0 >= c1) return;
  const int tid = threadIdx.x;
  auto slot = [](int c) { return ((c % (NG + 1)) + (NG + 1)) % (NG + 1); };
  for (int e = tid; e < (NG + 1) * CH * XLD; e += NTH) X[e] = T(0);
  __syncthreads();
  for (int e = tid; e < NG * CH; e += NTH)        // history chunk i = e / 32, row t = e % 32, column e
    X[slot(c0 - NG + e / CH) * CH * XLD + (e % CH) * XLD + e] = T(1);
  const int q = tid % NGW, rg = tid / NGW;
  const T* Mb = Mall + cbase[b];
  const int64_t xm = (int64_t)cpsmax * CH;        // rows of one segment's X
  const int KH = kh;                              // stored history width
  const int hoff = NGW - KH;                      // first stored history column
  T* Xb = Xout + ((int64_t)b * (S - 1) + (s - 1)) * xm * KH;
  // cp.async of chunk cc's couplings into buffer `buf`
  auto stage = [&](int cc, int buf) {
    const char* src = reinterpret_cast<const char*>(Mb + (int64_t)cc * (1 + NG) * CH * CH + CH * CH);
    const unsigned dst = (unsigned)__cvta_generic_to_shared(Gbuf + buf * NG * CH * CH);
    for (int o = tid * 16; o < (int)C::gbytes; o += NTH * 16)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst + o), "l"(src + o) : "memory");
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  if (C::DB) stage(c0, 0);
  for (int c = c0; c < c1; ++c) {
    const int cur = C::DB ? (c - c0) & 1 : 0;
    __syncthreads();    // readers of the previous G buffer and X_c are done
    if (C::DB) {
      if (c + 1 < c1) stage(c + 1, cur ^ 1);
      else asm volatile("cp.async.commit_group;\n" ::: "memory");
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");      // chunk c landed
    } else {
      stage(c, 0);
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    __syncthreads();
    const T* Gs = Gbuf + cur * NG * CH * CH;
    T acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = T(0);
    for (int k = 1; k <= NG; ++k) {
      const T* Xk = X + slot(c - k) * CH * XLD + q;
      const T* Gk = Gs + (k - 1) * CH * CH + rg * R;
#pragma unroll 4
      for (int j = 0; j < CH; ++j) {
        const T x = Xk[j * XLD];
        const V* g = reinterpret_cast<const V*>(Gk + j * CH);
#pragma unroll
        for (int v = 0; v < R / E; ++v) {
          const V gv = g[v];
          const T* pg = reinterpret_cast<const T*>(&gv);
#pragma unroll
          for (int e = 0; e < E; ++e) acc[v * E + e] -= pg[e] * x;
        }
      }
    }
    T* Xc = X + slot(c) * CH * XLD;
#pragma unroll
    for (int r = 0; r < R; ++r) Xc[(rg * R + r) * XLD + q] = acc[r];
    __syncthreads();
    // X_c to global (its KH stored columns), column-major over the segment's
    // positions (coalesced)
    const int64_t pr = (int64_t)(c - c0) * CH;
    for (int e = tid; e < CH * KH; e += NTH) {
      const int t = e % CH, qq = e / CH;
      Xb[(int64_t)qq * xm + pr + t] = Xc[t * XLD + hoff + qq];
    }
  }
  __syncthreads();
  T* To = Tout + ((int64_t)b * S + s) * KH * KH;
  for (int e = tid; e < KH * KH; e += NTH) {
    const int row = hoff + e / KH, col = hoff + e % KH;   // row = 32 i + t: chunk c1 - NG + i, position t
    To[e] = X[slot(c1 - NG + row / CH) * CH * XLD + (row % CH) * XLD + col];
  }
}

// The same X and T for more than 4 couplings per chunk (ng known at run
// time), where the 32 ng history columns of X no longer fit one CTA's shared
// memory: the KH stored history columns split into tiles of 32, one CTA per
// (tile, segment s >= 1, block); the ng + 1 most recent 32 x 32 tiles of X in
// a ring (row stride padded by 16 bytes: the 16-byte row writes of a warp fall
// on distinct banks), the couplings G_{c,1..ng} of each chunk staged by
// cp.async while the previous chunk is computed.  Thread (warp w, lane t)
// forms row t of the tile for columns 4 w .. 4 w + 3:
//     X_c = - sum_k G_{c,k} X_{c-k},   X = the identity on the history positions.
constexpr int kWideTile = 32;
template <typename T>
__host__ __device__ inline size_t seg_trans_wide_smem(int ng) {
  const size_t rs = kWideTile + 16 / sizeof(T);
  return (2 * (size_t)ng * CH * CH + (size_t)(ng + 1) * CH * rs) * sizeof(T);
}

template <typename T>
__global__ void __launch_bounds__(256)
k_seg_trans_wide(const T* __restrict__ Mall, const int64_t* __restrict__ cbase, Dev d, int S, int cpsmax, int kh,
                 int ng, T* __restrict__ Tout, T* __restrict__ Xout) {
  constexpr int NT = 256, CPB = kWideTile, CPW = CPB / 8;
  constexpr int RS = CPB + 16 / (int)sizeof(T);
  constexpr int MM = CH * CH;
  using V = typename Vec16<T>::type;
  constexpr int E = 16 / (int)sizeof(T);
  static_assert(CPW % E == 0, "a thread's columns are whole 16-byte vectors");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Gbuf = reinterpret_cast<T*>(smem_raw);              // 2 x ng x 32 x 32
  T* ring = Gbuf + 2 * (size_t)ng * MM;                   // (ng + 1) x 32 x RS
  const int b = blockIdx.z, s = blockIdx.y + 1;
  const int q0 = blockIdx.x * CPB;                        // first stored history column of the tile
  const int nch = (int)(d.ld[b] / CH);
  const int cps = seg_chunks(nch, S);
  const int c0 = s * cps, c1 = min(nch, c0 + cps);
  if (c0 >= c1) return;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int SL = ng + 1;
  auto slot = [&](int c) { return ((c % SL) + SL) % SL; };
  for (int e = tid; e < SL * CH * RS; e += NT) ring[e] = T(0);
  __syncthreads();
  // history: stored column qq is position c0 32 - kh + qq, where X = 1
  for (int e = tid; e < CPB; e += NT) {
    const int qq = q0 + e;
    if (qq < kh) {
      const int pos = c0 * CH - kh + qq;
      ring[slot(pos / CH) * CH * RS + (pos % CH) * RS + e] = T(1);
    }
  }
  const T* Mb = Mall + cbase[b];
  const int64_t xm = (int64_t)cpsmax * CH;
  T* Xb = Xout + ((int64_t)b * (S - 1) + (s - 1)) * xm * kh;
  auto stage = [&](int cc, int buf) {
    const char* src = reinterpret_cast<const char*>(Mb + (int64_t)cc * (1 + ng) * MM + MM);
    const unsigned dst = (unsigned)__cvta_generic_to_shared(Gbuf + (size_t)buf * ng * MM);
    const int nbytes = ng * MM * (int)sizeof(T);
    for (int o = tid * 16; o < nbytes; o += NT * 16)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst + o), "l"(src + o) : "memory");
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  stage(c0, 0);
  for (int c = c0; c < c1; ++c) {
    const int cur = (c - c0) & 1;
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();                                     // chunk c's couplings; the ring's last tiles
    if (c + 1 < c1) stage(c + 1, cur ^ 1);
    const T* Gs = Gbuf + (size_t)cur * ng * MM;
    T acc[CPW];
#pragma unroll
    for (int u = 0; u < CPW; ++u) acc[u] = T(0);
    for (int k = 1; k <= ng; ++k) {
      const T* G = Gs + (size_t)(k - 1) * MM;
      const T* Z = ring + (size_t)slot(c - k) * CH * RS + w * CPW;
#pragma unroll 8
      for (int j = 0; j < CH; ++j) {
        const T gv = G[j * CH + lane];
#pragma unroll
        for (int v = 0; v < CPW / E; ++v) {
          const V z4 = reinterpret_cast<const V*>(Z + j * RS)[v];
          const T* pz = reinterpret_cast<const T*>(&z4);
#pragma unroll
          for (int e = 0; e < E; ++e) acc[v * E + e] -= gv * pz[e];
        }
      }
    }
    T* Zc = ring + (size_t)slot(c) * CH * RS + lane * RS + w * CPW;
#pragma unroll
    for (int v = 0; v < CPW / E; ++v) {
      V x;
      T* xe = reinterpret_cast<T*>(&x);
#pragma unroll
      for (int e = 0; e < E; ++e) xe[e] = acc[v * E + e];
      reinterpret_cast<V*>(Zc)[v] = x;
    }
    // X_c to global, column-major over the segment's positions (lane = position: coalesced)
    const int64_t pr = (int64_t)(c - c0) * CH + lane;
#pragma unroll
    for (int u = 0; u < CPW; ++u) {
      const int qq = q0 + w * CPW + u;
      if (qq < kh) Xb[(int64_t)qq * xm + pr] = acc[u];
    }
  }
  __syncthreads();
  // T_s: row a of the stored columns on the segment's last kh positions
  T* To = Tout + ((int64_t)b * S + s) * kh * kh;
  for (int e = tid; e < kh * CPB; e += NT) {
    const int a = e / CPB, u = e % CPB;
    const int qq = q0 + u;
    if (qq < kh) {
      const int pos = c1 * CH - kh + a;
      To[(int64_t)a * kh + qq] = ring[slot(pos / CH) * CH * RS + (pos % CH) * RS + u];
    }
  }
}

template <typename T, int NG>
cudaError_t seg_trans_ng(const T* M, const int64_t* cbase, int P, int S, int cpsmax, int kh, Dev d, T* tout,
                         T* xout, cudaStream_t s) {
  using C = SegTrans<T, NG>;
  auto kern = k_seg_trans<T, NG>;
  if (C::smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<dim3(S - 1, P), C::NTH, C::smem, s>>>(M, cbase, d, S, cpsmax, kh, tout, xout);
  return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t launch_seg_trans(const T* M, const int64_t* cbase, int K, int P, int S, int cpsmax, Dev d, T* tout,
                             T* xout, cudaStream_t s) {
  if (S < 2) return cudaSuccess;
  count_launches(1);
  const int ng = (K + CH - 1) / CH;
  switch (ng) {
    case 1: return seg_trans_ng<T, 1>(M, cbase, P, S, cpsmax, hist_width(K), d, tout, xout, s);
    case 2: return seg_trans_ng<T, 2>(M, cbase, P, S, cpsmax, hist_width(K), d, tout, xout, s);
    case 3: return seg_trans_ng<T, 3>(M, cbase, P, S, cpsmax, hist_width(K), d, tout, xout, s);
    case 4: return seg_trans_ng<T, 4>(M, cbase, P, S, cpsmax, hist_width(K), d, tout, xout, s);
    default: {
      const size_t smem = seg_trans_wide_smem<T>(ng);
      if (smem > kSmemPerBlock) return cudaErrorInvalidValue;
      cudaError_t e = cudaFuncSetAttribute(k_seg_trans_wide<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
      if (e != cudaSuccess) return e;
      const int kh = hist_width(K);
      k_seg_trans_wide<T><<<dim3((kh + kWideTile - 1) / kWideTile, S - 1, P), 256, smem, s>>>(
          M, cbase, d, S, cpsmax, kh, ng, tout, xout);
      return cudaGetLastError();
    }
  }
}

template cudaError_t launch_seg_trans<float>(const float*, const int64_t*, int, int, int, int, Dev, float*, float*,
                                             cudaStream_t);
template cudaError_t launch_seg_trans<double>(const double*, const int64_t*, int, int, int, int, Dev, double*,
                                              double*, cudaStream_t);

template cudaError_t launch_chunk_mats<float>(const float*, int, int, Dev, const int64_t*, int, int, float*,
                                              cudaStream_t);
template cudaError_t launch_chunk_mats<double>(const double*, int, int, Dev, const int64_t*, int, int, double*,
                                               cudaStream_t);

}  // namespace sap
