// Preconditioner apply z = M^{-1} r (Sec. 2.1): the block-diagonal solve
// D g = r (Eq. (2.3)) as two banded triangular sweeps per block, and for
// SaP-C the truncated reduced systems (Eq. (2.5)) and the purification
// solves that follow them.
//
// Sweep kernel: one CTA (4 warps) per block, both sweeps in one launch.  A
// sweep is a linear recurrence over positions p (rows in sweep order),
//     z_p = ( y_p - sum_{d=1..K} coef(p, d) z_{p-d} ) / diag(p),
// processed in chunks of 32 positions:
//   - warp 0 (the solver) runs the dependent chain of a chunk: lane t holds
//     row t; for j = 0..31 it broadcasts z_j with one shuffle and every
//     lane applies its in-chunk coefficient and, in the same step, the
//     coefficient that couples row t of the *next* chunk to z_j.  The
//     coefficients are pre-scaled by 1/diag off the chain, so one step of
//     the chain is one shuffle and one FMA;
//   - warps 1..7 (helpers) stream the factor columns of later chunks into a
//     shared-memory ring with cp.async (PF chunks ahead) and sum the
//     "older" contributions (d > 32 + t) of the next chunk from that ring
//     and a ring of past z.
// The four sweep kinds (L forward, U backward, U^T forward, L^T backward)
// differ only in which diagonals are staged and where a row's coefficients
// sit: factor storage is F[c * ld + q] = entry (r, q), c = K + r - q.
// Positions run over [0, ld) (ld = n rounded up to 32); a backward sweep
// maps row r to p = ld - 1 - r.  Positions without a row are padding and
// produce z = 0.
#include <cuda_runtime.h>
#include <cstdint>
#include "sap_internal.cuh"

namespace sap {

namespace {

constexpr int NW = 8;               // warps per sweep CTA: 1 solver + 7 helpers
constexpr int CHK = 32;             // chunk length

enum Mode { LF = 0, UB = 1, UTF = 2, LTB = 3 };

template <int MODE> __device__ __forceinline__ constexpr bool fwd_mode() { return MODE == LF || MODE == UTF; }
template <int MODE> __device__ __forceinline__ constexpr bool unit_diag() { return MODE == LF || MODE == LTB; }
// row-oriented: coef(p, d) sits in column position p - d; column-oriented: in p
template <int MODE> __device__ __forceinline__ constexpr bool row_oriented() { return MODE == LF || MODE == UB; }
// diagonal c of the factor for distance d
template <int MODE> __device__ __forceinline__ int diag_of(int K, int d) {
  return (MODE == LF || MODE == LTB) ? K + d : K - d;
}

__device__ __forceinline__ void cpa4(void* smem, const void* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cpa8(void* smem, const void* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
template <typename X> __device__ __forceinline__ X rcp_t(X v) { return X(1) / v; }
template <> __device__ __forceinline__ float rcp_t<float>(float v) { return __frcp_rn(v); }
template <typename X> __device__ __forceinline__ void cpa(X* smem, const X* gmem) {
  if (sizeof(X) == 4) cpa4(smem, gmem); else cpa8(smem, gmem);
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N_> __device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N_) : "memory"); }

struct SweepGeom {
  int K;
  int n, ld;     // rows of the block, positions (n rounded up to 32)
  int RQ;        // ring length in column positions (multiple of 32)
  int ZR;        // z history ring length (power of 2 >= K + 96)
  int DR;        // ring rows: distances d = 0 .. DR-1 (DR >= 64; rows > K are zero)
  int DRP;       // slot pitch of the ring (even, >= DR): R[slot * DRP + d]
};

template <typename T, typename YT>
struct SweepSh {
  T* R;          // RQ x DRP ring of factor columns: R[slot * DRP + d], d = distance
  YT* Y;         // (PF+1) x 32 ring of right-hand sides
  T* Z;          // ZR ring of computed z (indexed by position mod ZR, ZR a power of 2)
  T* C1;         // [2][32][32]: in-chunk coefficients, pre-scaled by 1/diag, [j][t]
  T* C2;         // [2][32][32]: next-chunk row t on z_j of this chunk, pre-scaled
  T* YH;         // [2][32]: right-hand side pre-scaled by 1/diag
  T* older;      // [2][NOLD][32]: contributions of z older than the previous chunk
  double* corr;  // 2K corrections (top K rows, bottom K rows)
};

constexpr int NOLD = 3;   // helper warps that sum the older contributions

template <int MODE>
__device__ __forceinline__ int row_of(int p, int ld) { return fwd_mode<MODE>() ? p : ld - 1 - p; }
// Ring slot of column position pos (the factor column q = row_of(pos) mod RQ).
template <int MODE>
__device__ __forceinline__ int slot_of(int pos, const SweepGeom& g) { return row_of<MODE>(pos, g.ld) % g.RQ; }
// Slot of pos - d given sl = slot_of(pos), 0 <= d < RQ.
template <int MODE>
__device__ __forceinline__ int slot_back(int sl, int d, int RQ) {
  if (fwd_mode<MODE>()) { int x = sl - d; return x < 0 ? x + RQ : x; }
  int x = sl + d; return x >= RQ ? x - RQ : x;
}
// Slot of p0 + j for a chunk start p0 (multiple of 32) with sb = slot_of(p0): never wraps.
template <int MODE>
__device__ __forceinline__ int slot_in_chunk(int sb, int j) { return fwd_mode<MODE>() ? sb + j : sb - j; }

// Helpers: issue the cp.async copies of chunk cc (factor columns and y).
// Ring rows d = 1..K (and d = 0, the diagonal, for non-unit sweeps) are
// streamed; rows K+1..DR-1 stay zero for the whole kernel.
template <typename T, typename YT, int MODE, int PF>
__device__ __forceinline__ void prefetch(const SweepSh<T, YT>& sh, const SweepGeom& g, const T* __restrict__ F,
                                         const YT* __restrict__ yin, int cc) {
  const int p0 = cc * CHK;
  if (p0 < g.ld) {
    const int d0 = unit_diag<MODE>() ? 1 : 0;
    const int sb = slot_of<MODE>(p0, g);
    const int q0 = row_of<MODE>(p0, g.ld);
    const int sgn = fwd_mode<MODE>() ? 1 : -1;
    // helper warp hw copies distances d = d0 + hw, d0 + hw + (NW-1), ... for
    // column t = lane: 32 consecutive factor columns of one diagonal per warp
    const int lane = threadIdx.x & 31, hw = (threadIdx.x >> 5) - 1;
    const int dstep = NW - 1;
    // the factor diagonal of distance d is K + d (L sweeps) or K - d (U sweeps)
    const int64_t sstride = (int64_t)((MODE == LF || MODE == LTB) ? 1 : -1) * dstep * g.ld;
    int d = d0 + hw;
    const T* src = F + (int64_t)diag_of<MODE>(g.K, d) * g.ld + (q0 + sgn * lane);
    T* dst = &sh.R[(sb + sgn * lane) * g.DRP + d];
    for (; d <= g.K; d += dstep, src += sstride, dst += dstep) cpa(dst, src);
    if (hw == 0) {
      const int r = q0 + sgn * lane;
      YT* ydst = &sh.Y[(cc % (PF + 1)) * CHK + lane];
      if (r < g.n) cpa(ydst, &yin[r]);
      else *ydst = YT(0);
    }
  }
  cpa_commit();
}

// Helpers: build the pre-scaled tiles of chunk cb (needs ring chunks cb, cb+1)
// and, in warps 1..NOLD, its older contributions (needs z of chunks <= cb-2).
template <typename T, typename YT, int MODE, int PF, int DRPC>
__device__ __forceinline__ void build_tiles(const SweepSh<T, YT>& sh, const SweepGeom& g, int cb,
                                            bool has_top, bool has_bot) {
  const int lane = threadIdx.x & 31, hw = (threadIdx.x >> 5) - 1;
  const int K = g.K, RQ = g.RQ;
  const int DRP = DRPC ? DRPC : g.DRP;
  const int buf = cb & 1;
  const int p0 = cb * CHK;
  if (p0 >= g.ld) return;
  const int p = p0 + lane;                  // this lane's row in chunk cb
  const int p2 = p + CHK;                   // and in chunk cb + 1
  const bool valid = row_of<MODE>(p, g.ld) < g.n;
  const bool valid2 = p2 < g.ld && row_of<MODE>(p2, g.ld) < g.n;
  const int sb = slot_of<MODE>(p0, g);
  const int sp = slot_in_chunk<MODE>(sb, lane);
  const int sb2 = p0 + CHK < g.ld ? slot_of<MODE>(p0 + CHK, g) : sb;
  const int sp2 = slot_in_chunk<MODE>(sb2, lane);
  T dinv = T(1), dinv2 = T(1);
  if (!unit_diag<MODE>()) {
    dinv = valid ? rcp_t(sh.R[sp * DRP]) : T(0);
    dinv2 = valid2 ? rcp_t(sh.R[sp2 * DRP]) : T(0);
  }
  T* C1 = sh.C1 + buf * CHK * CHK;
  T* C2 = sh.C2 + buf * CHK * CHK;
  for (int j = hw; j < CHK; j += NW - 1) {
    const int d1 = lane - j, d2 = CHK + lane - j;
    const int sl1 = row_oriented<MODE>() ? slot_in_chunk<MODE>(sb, j) : sp;
    const int sl2 = row_oriented<MODE>() ? slot_in_chunk<MODE>(sb, j) : sp2;
    C1[j * CHK + lane] = (d1 >= 1) ? sh.R[sl1 * DRP + d1] * dinv : T(0);   // rows > K are zero
    C2[j * CHK + lane] = sh.R[sl2 * DRP + d2] * dinv2;
  }
  if (hw == 0) {
    const int r = row_of<MODE>(p, g.ld);
    T yv = T(0);
    if (valid) {
      yv = (T)sh.Y[(cb % (PF + 1)) * CHK + lane];
      if (has_top && r < K) yv -= (T)sh.corr[r];
      if (has_bot && r >= g.n - K) yv -= (T)sh.corr[K + (r - (g.n - K))];
    }
    sh.YH[buf * CHK + lane] = yv * dinv;
  }
  if (hw < NOLD) {
    // older contributions of row p: d in [33 + lane, K], z positions <= 32 cb - 33
    T acc = T(0);
    if (valid && K > CHK + lane) {
      const int zp = p & (g.ZR - 1);
      for (int d = CHK + 1 + lane + hw; d <= K && d <= p; d += NOLD) {
        const int sl = row_oriented<MODE>() ? slot_back<MODE>(sp, d, RQ) : sp;
        acc += sh.R[sl * DRP + d] * sh.Z[(zp - d) & (g.ZR - 1)];
      }
      acc *= dinv;
    }
    sh.older[(buf * NOLD + hw) * CHK + lane] = acc;
  }
}

template <typename T, typename YT, int MODE, int PF, int DRPC>
__device__ void sweep(const SweepSh<T, YT>& sh, const SweepGeom& g, const T* __restrict__ F,
                      const YT* __restrict__ yin, bool has_top, bool has_bot, double* __restrict__ out_d,
                      T* __restrict__ out_t) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nch = g.ld / CHK;
  // prologue: chunks 0..PF-1 in flight; tiles of chunk 0 need ring chunks 0, 1
  if (warp > 0) {
    for (int cc = 0; cc < PF; ++cc) prefetch<T, YT, MODE, PF>(sh, g, F, yin, cc);
    cpa_wait<PF - 2>();
  }
  __syncthreads();
  if (warp > 0) {
    build_tiles<T, YT, MODE, PF, DRPC>(sh, g, 0, has_top, has_bot);
    cpa_wait<PF - 3>();     // chunk 2 landed: tiles of chunk 1 can be built in iteration 0
  }
  __syncthreads();
  T recent = T(0);   // warp 0: prev-chunk contribution to this chunk's row (pre-scaled)
  for (int c = 0; c < nch; ++c) {
    const int buf = c & 1;
    if (warp == 0) {
      const T* C1 = sh.C1 + buf * CHK * CHK + lane;
      const T* C2 = sh.C2 + buf * CHK * CHK + lane;
      T s = sh.YH[buf * CHK + lane] - recent;
#pragma unroll
      for (int w = 0; w < NOLD; ++w) s -= sh.older[(buf * NOLD + w) * CHK + lane];
      T nxt = T(0);
#pragma unroll
      for (int j = 0; j < CHK; ++j) {
        const T c1 = C1[j * CHK];
        const T c2 = C2[j * CHK];
        const T zj = __shfl_sync(0xffffffffu, s, j);
        s -= c1 * zj;
        nxt += c2 * zj;
      }
      recent = nxt;
      const int p = c * CHK + lane;
      sh.Z[p & (g.ZR - 1)] = s;
      const int r = row_of<MODE>(p, g.ld);
      if (r < g.n) {
        if (out_d) out_d[r] = (double)s;
        else out_t[r] = s;
      }
    } else {
      prefetch<T, YT, MODE, PF>(sh, g, F, yin, c + PF);
      build_tiles<T, YT, MODE, PF, DRPC>(sh, g, c + 1, has_top, has_bot);
      cpa_wait<PF - 3>();   // chunk c + 3 landed (tiles of chunk c + 2 need chunks c + 2, c + 3)
    }
    __syncthreads();
  }
  if (warp > 0) cpa_wait<0>();
  __syncthreads();
}

template <typename T> __host__ __device__ constexpr int pf_of() { return sizeof(T) == 4 ? 5 : 4; }

__host__ __device__ inline int ring_rows(int K) { return (K > 2 * CHK - 1 ? K : 2 * CHK - 1) + 1; }
// even slot pitch: all four sweep kinds read the ring without bank conflicts
__host__ __device__ inline int ring_pitch(int K) { return (ring_rows(K) + 2) & ~1; }
constexpr int kSmallDRP = 66;   // ring_pitch(K) for K <= 63
__host__ __device__ inline int z_ring(int K) { int z = 64; while (z < K + 3 * CHK) z <<= 1; return z; }

template <typename T>
size_t sweep_smem(int K, int* RQ_out) {
  constexpr int PF = pf_of<T>();
  int RQ = ((K + CHK * (PF + 1)) + CHK - 1) / CHK * CHK;
  *RQ_out = RQ;
  size_t b = (size_t)ring_pitch(K) * RQ * sizeof(T);
  b = (b + 15) & ~(size_t)15;
  b += (size_t)(PF + 1) * CHK * sizeof(double);   // Y ring (largest input type)
  b += (size_t)z_ring(K) * sizeof(T);             // Z ring
  b = (b + 15) & ~(size_t)15;
  b += (size_t)2 * 2 * CHK * CHK * sizeof(T);     // C1, C2
  b += (size_t)2 * CHK * sizeof(T);               // YH
  b += (size_t)2 * NOLD * CHK * sizeof(T);        // older
  b = (b + 15) & ~(size_t)15;
  b += (size_t)2 * K * sizeof(double);            // corrections
  return b;
}

template <typename T, typename YT, int PF>
__device__ __forceinline__ SweepSh<T, YT> carve(unsigned char* base, const SweepGeom& g) {
  SweepSh<T, YT> sh;
  size_t off = 0;
  sh.R = reinterpret_cast<T*>(base);
  off = (size_t)g.DRP * g.RQ * sizeof(T);
  off = (off + 15) & ~(size_t)15;
  sh.Y = reinterpret_cast<YT*>(base + off);
  off += (size_t)(PF + 1) * CHK * sizeof(double);
  sh.Z = reinterpret_cast<T*>(base + off);
  off += (size_t)g.ZR * sizeof(T);
  off = (off + 15) & ~(size_t)15;
  sh.C1 = reinterpret_cast<T*>(base + off);
  off += (size_t)2 * CHK * CHK * sizeof(T);
  sh.C2 = reinterpret_cast<T*>(base + off);
  off += (size_t)2 * CHK * CHK * sizeof(T);
  sh.YH = reinterpret_cast<T*>(base + off);
  off += (size_t)2 * CHK * sizeof(T);
  sh.older = reinterpret_cast<T*>(base + off);
  off += (size_t)2 * NOLD * CHK * sizeof(T);
  off = (off + 15) & ~(size_t)15;
  sh.corr = reinterpret_cast<double*>(base + off);
  return sh;
}

template <typename T, bool TRANS, int DRPC>
__global__ void __launch_bounds__(NW * 32)
k_block_solve(const T* __restrict__ Fall, int K, Dev d, const double* __restrict__ r_in,
              double* __restrict__ z_out, T* __restrict__ tmp, const double* __restrict__ ctop_all,
              const double* __restrict__ cbot_all, int P, int RQ) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int PF = pf_of<T>();
  const int b = blockIdx.x;
  const int64_t s = d.off[b];
  SweepGeom g;
  g.K = K;
  g.n = (int)(d.off[b + 1] - s);
  g.ld = (int)d.ld[b];
  g.RQ = RQ;
  g.DR = ring_rows(K);
  g.DRP = ring_pitch(K);
  g.ZR = z_ring(K);
  const T* F = Fall + d.fbase[b];
  const bool has_top = ctop_all && b > 0;
  const bool has_bot = cbot_all && b + 1 < P;
  {
    SweepSh<T, double> sh = carve<T, double, PF>(smem_raw, g);
    // ring distances beyond K are read as zero coefficients and never streamed
    const int nz = g.DRP - K - 1;
    for (int e = threadIdx.x; e < RQ * nz; e += blockDim.x) sh.R[(e / nz) * g.DRP + K + 1 + e % nz] = T(0);
    for (int t = threadIdx.x; t < K; t += blockDim.x) {
      sh.corr[t] = has_top ? ctop_all[(int64_t)(b - 1) * K + t] : 0.0;
      sh.corr[K + t] = has_bot ? cbot_all[(int64_t)b * K + t] : 0.0;
    }
    __syncthreads();
    if (!TRANS) sweep<T, double, LF, PF, DRPC>(sh, g, F, r_in + s, has_top, has_bot, nullptr, tmp + s);
    else sweep<T, double, UTF, PF, DRPC>(sh, g, F, r_in + s, has_top, has_bot, nullptr, tmp + s);
  }
  {
    SweepSh<T, T> sh = carve<T, T, PF>(smem_raw, g);
    if (!TRANS) sweep<T, T, UB, PF, DRPC>(sh, g, F, tmp + s, false, false, z_out + s, nullptr);
    else sweep<T, T, LTB, PF, DRPC>(sh, g, F, tmp + s, false, false, z_out + s, nullptr);
  }
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

template <typename T, bool TRANS>
cudaError_t launch_block_solve(const T* F, int K, int P, Dev d, const double* r, double* z, T* tmp,
                               const double* ctop, const double* cbot, cudaStream_t s) {
  int RQ;
  size_t smem = sweep_smem<T>(K, &RQ);
  auto kern = (ring_pitch(K) == kSmallDRP) ? k_block_solve<T, TRANS, kSmallDRP> : k_block_solve<T, TRANS, 0>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  count_launches(1);
  kern<<<P, NW * 32, smem, s>>>(F, K, d, r, z, tmp, ctop, cbot, P, RQ);
  return cudaGetLastError();
}

}  // namespace

size_t sweep_smem_bytes(int K, bool fp64) {
  int RQ;
  return fp64 ? sweep_smem<double>(K, &RQ) : sweep_smem<float>(K, &RQ);
}

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
