// Preconditioner apply z = M^{-1} r (Sec. 2.1): the block-diagonal solve
// D g = r (Eq. (2.3)) as two banded triangular sweeps per block, and for
// SaP-C the truncated reduced systems (Eq. (2.5)) and the purification
// solves that follow them.
//
// Sweep kernels: per block and segment one CTA of 2 + NPW warps (NPW = 1
// prepare warp for ceil(K/32) <= 3 couplings, 2 up to 7, 4 above).  A sweep
// is a lower-triangular recurrence over positions p (rows in sweep order),
// processed in chunks of 32 positions with the chunk matrices of k_chunk.cu
// (MINV_c and the couplings G_{c,k}, k = 1..ng, ng = ceil(K/32)):
//     z_c = w_c - G_{c,1} z_{c-1},
//     w_c = MINV_c (y_c - corrections) - sum_{k>=2} G_{c,k} z_{c-k}.
//   - warp 0 runs the dependent chain: one 32 x 32 product per chunk, with
//     z_{c-1} broadcast from its own registers by shuffles;
//   - warps 1 .. NPW form w_{c+1} one chunk ahead (warp 1 also streams the
//     right-hand side with cp.async), each a share of the G_k products;
//   - the last warp streams each chunk's matrices (one contiguous block) into
//     a shared-memory ring (4 or, for the widest bands, 2 chunks ahead) with a
//     bulk (TMA) copy and waits on the slot's mbarrier; the other warps see
//     the data through the CTA barrier.
// Positions run over [0, ld) (ld = n rounded up to 32); a backward sweep
// maps row r to p = ld - 1 - r.  Positions without a row produce 0.
// With S > 1 segments per block the chunks of a sweep are cut into S ranges
// swept concurrently in two passes (see k_sweep and the transfer matrices of
// k_chunk.cu), so that P blocks occupy S P CTAs.
#include <cuda_runtime.h>
#include <cstdint>
#include "sap_internal.cuh"

namespace sap {

namespace {

constexpr int NWS = 3;              // warps per sweep CTA
constexpr int CHK = 32;             // chunk length
constexpr int PF = 4;               // chunks prefetched ahead (2 where a 4-deep ring does not fit)

enum Mode { LF = 0, UB = 1, UTF = 2, LTB = 3 };

template <int MODE> __device__ __forceinline__ constexpr bool fwd_mode() { return MODE == LF || MODE == UTF; }

__device__ __forceinline__ void cpa4(void* smem, const void* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cpa8(void* smem, const void* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
template <typename X> __device__ __forceinline__ void cpa(X* smem, const X* gmem) {
  if (sizeof(X) == 4) cpa4(smem, gmem); else cpa8(smem, gmem);
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N_> __device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N_) : "memory"); }

// ---- mbarrier-tracked bulk (TMA) copies global -> shared ----
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
// Non-blocking test of a barrier phase (one poll of a bounded wait).
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
// Bounded wait for a barrier phase: after `limit` polls the thread records a
// timeout in err[0], stops waiting for good and lets the kernel run to its
// end.  Returns true if the phase completed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int limit, int* err, bool& failed) {
  if (failed) return false;
  for (int i = 0; i < limit; ++i)
    if (mbar_test_wait(bar, parity)) return true;
  failed = true;
  if (err) atomicExch(err, 1);
  return false;
}

// Column-major 32 x 32 matrix row `lane` against a broadcast vector: all
// loads issued before the multiply-adds.
template <typename T>
__device__ __forceinline__ T coldot32(const T* __restrict__ Mcm, const T* __restrict__ v, int lane) {
  T m[CHK], x[CHK];
#pragma unroll
  for (int j = 0; j < CHK; ++j) m[j] = Mcm[j * CHK + lane];
#pragma unroll
  for (int j = 0; j < CHK; ++j) x[j] = v[j];
  T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
#pragma unroll
  for (int j = 0; j < CHK; j += 4) {
    a0 += m[j] * x[j];
    a1 += m[j + 1] * x[j + 1];
    a2 += m[j + 2] * x[j + 2];
    a3 += m[j + 3] * x[j + 3];
  }
  return (a0 + a1) + (a2 + a3);
}

// 16-byte vector of T.
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; };
template <> struct Vec16<double> { using type = double2; };

struct SweepGeom {
  int K, n, ld, ng;
};

template <typename T, typename YT>
struct SweepSh {
  T* M;          // (PF+1) x (1+ng) x 32 x 32 ring of chunk matrices, column-major
  YT* Y;         // (PF+1) x 32 ring of right-hand sides
  T* zh;         // (ng+1) x 32: z of the most recent chunks (chunk mod (ng+1))
  T* W;          // [2][NPW][32]: partial sums of w of the next chunk, one per prepare warp
  T* yb;         // 32: y - corrections of the chunk being prepared
  double* corr;  // 2K corrections (top K rows, bottom K rows)
  uint64_t* bar; // PF+1 mbarriers: chunk matrices of a ring slot landed
};

template <int MODE>
__device__ __forceinline__ int row_of(int p, int ld) { return fwd_mode<MODE>() ? p : ld - 1 - p; }

// Copy warp: bulk-copy local chunk lc's matrices into ring slot lc % (PFD+1).
// Chunks past the segment (lc >= nc) only arrive on the barrier, so that every
// slot completes one phase per chunk index.  Lane 0 keeps the slots with a
// copy in flight (inflight) and the parity of the phase each completes (ifpar,
// the slot's bit of ph at issue); after a wait gave up (failed) no copy is
// issued any more, so that the in-flight ones can be drained.
template <int PFD, typename T, typename YT>
__device__ __forceinline__ void prefetch_mats(const SweepSh<T, YT>& sh, const SweepGeom& g, const T* __restrict__ Mg,
                                              int lc, int nc, bool failed, unsigned ph, unsigned& inflight,
                                              unsigned& ifpar) {
  if ((threadIdx.x & 31) != 0 || failed) return;
  const int slot = lc % (PFD + 1);
  const int mat = (1 + g.ng) * CHK * CHK;
  if (lc < nc) {
    const unsigned bytes = (unsigned)(mat * sizeof(T));
    mbar_expect_tx(&sh.bar[slot], bytes);
    bulk_g2s(sh.M + slot * mat, Mg + (int64_t)lc * mat, bytes, &sh.bar[slot]);
    inflight |= 1u << slot;
    ifpar = (ifpar & ~(1u << slot)) | (ph & (1u << slot));
  } else {
    mbar_arrive(&sh.bar[slot]);
  }
}

// After a wait of this thread gave up: wait (bounded by kDefaultSpin polls
// each) for the copies still in flight, so that none lands in shared memory
// after the sweep has moved on or the CTA has exited.
template <int PFD>
__device__ __forceinline__ void drain_copies(uint64_t* bar, unsigned inflight, unsigned ifpar) {
  for (int sl = 0; sl <= PFD; ++sl)
    if (inflight & (1u << sl)) {
      bool gave_up = false;
      mbar_wait(&bar[sl], (ifpar >> sl) & 1u, kDefaultSpin, nullptr, gave_up);
    }
}

// Warp 1: cp.async of local chunk lc's right-hand side (one commit group per
// chunk); p0: first position of the segment.
template <int PFD, typename T, typename YT, int MODE>
__device__ __forceinline__ void prefetch_y(const SweepSh<T, YT>& sh, const SweepGeom& g, const YT* __restrict__ yin,
                                           int lc, int nc, int p0) {
  const int lane = threadIdx.x & 31;
  if (lc < nc) {
    const int r = row_of<MODE>(p0 + lc * CHK + lane, g.ld);
    YT* ydst = &sh.Y[(lc % (PFD + 1)) * CHK + lane];
    if (r < g.n) cpa(ydst, &yin[r]);
    else *ydst = YT(0);
  }
  cpa_commit();
}

// One sweep over the nc chunks of a segment starting at chunk c0 of a block
// (Mg: the block's chunk matrices), with zero history.  Local chunk
// lc = c - c0; z history slot of local chunk lc (lc >= -ng) is
// (lc + ng + 1) % (ng + 1), the ng chunks before the segment occupying slots
// 1..ng (zero).  out receives z of the segment's rows; tail (if not null) the
// z of its last hist_width(K) positions, oldest first.
template <typename T, typename YT, typename OT, int MODE, int PFD = PF, int NPW = 1>
__device__ void sweep(const SweepSh<T, YT>& sh, const SweepGeom& g, const T* __restrict__ Mg,
                      const YT* __restrict__ yin, bool has_top, bool has_bot, OT* __restrict__ out, int c0, int nc,
                      T* __restrict__ tail, unsigned& ph, bool& failed, int* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int K = g.K, ng = g.ng;
  const int mat = (1 + ng) * CHK * CHK;
  const int p0 = c0 * CHK;
  const T* Ms = Mg + (int64_t)c0 * mat;
  // warp roles: 0 the chain, 1 .. NPW the preparation of the next chunk's w
  // (warp 1 also fetches y), NPW + 1 the bulk copies of the chunk matrices.
  // ph: per-slot parity of the next barrier phase (lane 0 of the copy warp),
  // carried from sweep to sweep of one CTA
  constexpr int WCOPY = NPW + 1;
  const bool prep = NPW == 1 ? warp == 1 : (warp >= 1 && warp <= NPW);
  // copy warp, lane 0: copies in flight and their phase parities (see prefetch_mats)
  unsigned inflight = 0u, ifpar = 0u;
  const int spin = (warp == WCOPY && lane == 0) ? spin_limit_of(err) : 0;
  auto wait_chunk = [&](int lc) {     // copy warp: lane 0 polls
    const int sl = lc % (PFD + 1);
    if (lane == 0 && mbar_wait(&sh.bar[sl], (ph >> sl) & 1u, spin, err, failed)) inflight &= ~(1u << sl);
    ph ^= 1u << sl;
    __syncwarp();
  };
  auto issue = [&](int lc) { prefetch_mats<PFD>(sh, g, Ms, lc, nc, failed, ph, inflight, ifpar); };
  auto zslot = [&](int lc) { return (lc + ng + 1) % (ng + 1); };
  // w_lb = MINV (y - corrections) - sum_{k>=2} G_k z_{lb-k}: prepare warp j
  // (0-based) forms the MINV term (j = 0) and the G_k terms with k = j + 2 mod
  // NPW; warp 0 adds the NPW partial sums in order
  auto prepare = [&](int lb) {
    const int slot = lb % (PFD + 1);
    const T* Mc = sh.M + slot * mat;
    if constexpr (NPW == 1) {
      const int r = row_of<MODE>(p0 + lb * CHK + lane, g.ld);
      T yv = T(0);
      if (r < g.n) {
        yv = (T)sh.Y[slot * CHK + lane];
        if (has_top && r < K) yv -= (T)sh.corr[r];
        if (has_bot && r >= g.n - K) yv -= (T)sh.corr[K + (r - (g.n - K))];
      }
      sh.yb[lane] = yv;
      __syncwarp();
      T w = coldot32(Mc, sh.yb, lane);
      for (int k = 2; k <= ng; ++k) w -= coldot32(Mc + k * CHK * CHK, sh.zh + zslot(lb - k) * CHK, lane);
      sh.W[(lb & 1) * CHK + lane] = w;
      __syncwarp();
    } else {
      const int j = warp - 1;
      T w = T(0);
      if (j == 0) {
        const int r = row_of<MODE>(p0 + lb * CHK + lane, g.ld);
        T yv = T(0);
        if (r < g.n) {
          yv = (T)sh.Y[slot * CHK + lane];
          if (has_top && r < K) yv -= (T)sh.corr[r];
          if (has_bot && r >= g.n - K) yv -= (T)sh.corr[K + (r - (g.n - K))];
        }
        sh.yb[lane] = yv;
        __syncwarp();
        w = coldot32(Mc, sh.yb, lane);
      }
      for (int k = 2 + j; k <= ng; k += NPW) w -= coldot32(Mc + k * CHK * CHK, sh.zh + zslot(lb - k) * CHK, lane);
      sh.W[((lb & 1) * NPW + j) * CHK + lane] = w;
      __syncwarp();
    }
  };
  // z history: zero
  for (int t = threadIdx.x; t < (ng + 1) * CHK; t += blockDim.x) sh.zh[t] = T(0);
  __syncthreads();
  // prologue: matrices of local chunks 0..PFD-1 in flight, 0 and 1 landed, w_0 formed
  if (warp == WCOPY) {
    for (int lc = 0; lc < PFD; ++lc) issue(lc);
    wait_chunk(0);
    wait_chunk(1);
  } else if (warp == 1) {
    for (int lc = 0; lc < PFD; ++lc) prefetch_y<PFD, T, YT, MODE>(sh, g, yin, lc, nc, p0);
    cpa_wait<PFD - 1>();
    __syncwarp();
  }
  __syncthreads();
  if (prep) prepare(0);
  __syncthreads();
  // warp 0: z of the previous chunk, lane t holds position t
  T zprev = T(0);
  for (int lc = 0; lc < nc; ++lc) {
    if (warp == 0) {
      const T* G1 = sh.M + (lc % (PFD + 1)) * mat + CHK * CHK;
      T m[CHK];
#pragma unroll
      for (int j = 0; j < CHK; ++j) m[j] = G1[j * CHK + lane];
      const T* Wl = sh.W + (lc & 1) * NPW * CHK + lane;
      T a0 = Wl[0], a1 = T(0), a2 = T(0), a3 = T(0);
      if constexpr (NPW > 1) {
#pragma unroll
        for (int j = 1; j < NPW; ++j) a0 += Wl[j * CHK];
      }
#pragma unroll
      for (int j = 0; j < CHK; j += 4) {
        a0 -= m[j] * __shfl_sync(0xffffffffu, zprev, j);
        a1 -= m[j + 1] * __shfl_sync(0xffffffffu, zprev, j + 1);
        a2 -= m[j + 2] * __shfl_sync(0xffffffffu, zprev, j + 2);
        a3 -= m[j + 3] * __shfl_sync(0xffffffffu, zprev, j + 3);
      }
      const T z = (a0 + a1) + (a2 + a3);
      zprev = z;
      sh.zh[zslot(lc) * CHK + lane] = z;
      const int r = row_of<MODE>(p0 + lc * CHK + lane, g.ld);
      if (out && r < g.n) out[r] = (OT)z;
    } else if (warp == 1) {
      prefetch_y<PFD, T, YT, MODE>(sh, g, yin, lc + PFD, nc, p0);
      if (lc + 1 < nc) {
        cpa_wait<PFD - 1>();     // y of chunk lc + 1 landed
        __syncwarp();
        prepare(lc + 1);
      }
    } else if (NPW > 1 && prep) {
      if (lc + 1 < nc) prepare(lc + 1);
    } else {
      issue(lc + PFD);
      wait_chunk(lc + 2);       // read by the prepare warps in iteration lc + 1, by warp 0 in lc + 2
    }
    __syncthreads();
  }
  // copy warp: consume the phases of the remaining prefetched chunks
  if (warp == WCOPY) {
    for (int lc = nc + 2; lc < nc + PFD; ++lc) wait_chunk(lc);
    if (lane == 0 && failed) drain_copies<PFD>(sh.bar, inflight, ifpar);
  }
  if (warp == 1) cpa_wait<0>();
  if (tail && warp == 0) {     // the last KH positions of the segment's last ng chunks
    const int off = ng * CHK - hist_width(K);
    for (int i = 0; i < ng; ++i) {
      const int j = i * CHK + lane - off;
      if (j >= 0) tail[j] = sh.zh[zslot(nc - ng + i) * CHK + lane];
    }
  }
  __syncthreads();
}

__host__ __device__ inline int n_couplings(int K) { return (K + CHK - 1) / CHK; }

template <typename T, int PFD = PF, int NPW = 1>
size_t sweep_smem(int K) {
  const int ng = n_couplings(K);
  size_t b = (size_t)(PFD + 1) * (1 + ng) * CHK * CHK * sizeof(T);   // chunk matrices
  b += (size_t)(PFD + 1) * CHK * sizeof(double);                      // Y ring (largest input type)
  b += (size_t)(ng + 1) * CHK * sizeof(T);                           // z history
  b += (size_t)(2 * NPW + 1) * CHK * sizeof(T);                      // W partials, yb
  b = (b + 15) & ~(size_t)15;
  b += (size_t)2 * K * sizeof(double);                               // corrections
  b = (b + 15) & ~(size_t)15;
  b += (size_t)(PFD + 1) * sizeof(uint64_t);                          // mbarriers
  return b;
}

template <typename T, typename YT, int PFD = PF, int NPW = 1>
__device__ __forceinline__ SweepSh<T, YT> carve(unsigned char* base, const SweepGeom& g) {
  SweepSh<T, YT> sh;
  size_t off = 0;
  sh.M = reinterpret_cast<T*>(base);
  off = (size_t)(PFD + 1) * (1 + g.ng) * CHK * CHK * sizeof(T);
  sh.Y = reinterpret_cast<YT*>(base + off);
  off += (size_t)(PFD + 1) * CHK * sizeof(double);
  sh.zh = reinterpret_cast<T*>(base + off);
  off += (size_t)(g.ng + 1) * CHK * sizeof(T);
  sh.W = reinterpret_cast<T*>(base + off);
  off += 2 * NPW * CHK * sizeof(T);
  sh.yb = reinterpret_cast<T*>(base + off);
  off += CHK * sizeof(T);
  off = (off + 15) & ~(size_t)15;
  sh.corr = reinterpret_cast<double*>(base + off);
  off += (size_t)2 * g.K * sizeof(double);
  off = (off + 15) & ~(size_t)15;
  sh.bar = reinterpret_cast<uint64_t*>(base + off);
  return sh;
}

// One sweep kind over every block, split into S segments of ceil(nch / S)
// chunks (Dev partition; grid (S, P)), all with zero history: segment 0 is
// exact; every segment writes its rows (zhat) and, but the last, the z of its
// last ng chunks (its zero-history tail).  k_seg_chain turns the tails into
// true histories, k_seg_correct then adds X h.
// ctop/cbot: SaP-C corrections of the right-hand side (forward sweeps of the
// second block solve only).
// PFD chunks of matrices in flight, NPW warps preparing the next chunk's w
// (1 up to 4 couplings per chunk; 2 or 4 for the wider bands, as in k_block_solve).
template <typename T, typename YT, typename OT, int MODE, int PFD = PF, int NPW = 1>
__global__ void __launch_bounds__((NPW + 2) * 32)
k_sweep(const T* __restrict__ Mall, const int64_t* __restrict__ cbase, int K, Dev d, const YT* __restrict__ yin,
        OT* __restrict__ out, T* __restrict__ tails, const double* __restrict__ ctop_all,
        const double* __restrict__ cbot_all, int P, int S, int* __restrict__ err, Gate gt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (gate_skip(gt)) return;
  const int b = blockIdx.y;
  const int seg = (int)blockIdx.x;
  const int64_t s = d.off[b];
  SweepGeom g;
  g.K = K;
  g.n = (int)(d.off[b + 1] - s);
  g.ld = (int)d.ld[b];
  g.ng = n_couplings(K);
  const int nch = g.ld / CHK;
  const int cps = seg_chunks(nch, S);
  const int c0 = seg * cps, c1 = min(nch, c0 + cps);
  if (c0 >= c1) return;
  const int KH = hist_width(K);
  const bool has_top = ctop_all && b > 0;
  const bool has_bot = cbot_all && b + 1 < P;
  bool failed = false;   // a barrier wait of this thread timed out
  SweepSh<T, YT> sh = carve<T, YT, PFD, NPW>(smem_raw, g);
  if (threadIdx.x == 0) {
    for (int q = 0; q <= PF; ++q) mbar_init(&sh.bar[q], 1);
    mbar_fence_init();
  }
  for (int t = threadIdx.x; t < K; t += blockDim.x) {
    sh.corr[t] = has_top ? ctop_all[(int64_t)(b - 1) * K + t] : 0.0;
    sh.corr[K + t] = has_bot ? cbot_all[(int64_t)b * K + t] : 0.0;
  }
  T* tail = (tails && seg + 1 < S) ? tails + ((int64_t)b * S + seg) * KH : nullptr;
  unsigned ph = 0;
  sweep<T, YT, OT, MODE, PFD, NPW>(sh, g, Mall + cbase[b], yin + s, has_top, has_bot, out + s, c0, c1 - c0, tail, ph,
                         failed, err);
}

constexpr int kCorrThreads = 256;

// Segment histories (grid P, kCorrThreads threads): the zero-history tails
// written by k_sweep are turned in place into the true tails by the transfer
// recurrence
//     tail_j = zhat_tail_j + T_j tail_{j-1},  j = 1 .. S-2  (tail_0 exact),
// so that segment s >= 1 finds its history in tail_{s-1}.  The T_j are
// staged into shared memory by cp.async in rounds of up to RB matrices (one
// memory latency per round); within a step TPR threads share a row (rotated
// column order: conflict-free) and combine by shuffles.
template <typename T>
__host__ __device__ inline int chain_ring(int K, int S) {   // matrices per staging round
  const int kh = hist_width(K);
  const size_t one = (size_t)kh * kh * sizeof(T);
  int rb = (int)((200 * 1024) / one);
  rb = rb > 8 ? 8 : rb;
  rb = rb > S - 2 ? S - 2 : rb;
  return rb < 1 ? 1 : rb;
}
template <typename T>
size_t chain_smem(int K, int S) {
  const int kh = hist_width(K);
  return (size_t)chain_ring<T>(K, S) * kh * kh * sizeof(T) + (size_t)(S + 1) * kh * sizeof(T);
}

// GT: the transfer matrices are read from global memory (L2) instead of
// being staged, for histories whose KH x KH matrix exceeds shared memory.
template <typename T, bool GT>
__global__ void __launch_bounds__(kCorrThreads)
k_seg_chain(const T* __restrict__ Tall, T* __restrict__ tails, int K, Dev d, int S, Gate gt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (gate_skip(gt)) return;
  const int b = blockIdx.x;
  const int NGW = hist_width(K);                   // history width
  const int nch = (int)(d.ld[b] / CHK);
  const int cps = seg_chunks(nch, S);
  const int nseg = (nch + cps - 1) / cps;          // nonempty segments of this block
  const int RB = GT ? S : chain_ring<T>(K, S);
  T* Ts = reinterpret_cast<T*>(smem_raw);         // RB x NGW x NGW (staged T_j; none for GT)
  T* zt = GT ? Ts : Ts + (size_t)RB * NGW * NGW;  // S x NGW tails (in place: zero-history -> true)
  T* tb = tails + (int64_t)b * S * NGW;
  // threads per row: the largest power of two <= 8 dividing NGW with NGW TPR <= 256
  int TPR = 1;
  while (TPR < 8 && NGW % (2 * TPR) == 0 && NGW * 2 * TPR <= kCorrThreads) TPR *= 2;
  const int part = threadIdx.x % TPR;
  const int RPP = kCorrThreads / TPR;              // rows per pass (NGW may exceed it)
  const int jend = nseg - 1;                       // tails 1 .. nseg-2 are needed
  auto stage = [&](void* dsts, const void* srcg, int nbytes) {
    const char* src = reinterpret_cast<const char*>(srcg);
    const unsigned dst = (unsigned)__cvta_generic_to_shared(dsts);
    for (int o = threadIdx.x * 16; o < nbytes; o += blockDim.x * 16)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst + o), "l"(src + o) : "memory");
  };
  if (jend < 2) return;                            // tail_0 is exact: nothing to carry
  // all tails of the block and the first round of T_j in one memory latency
  stage(zt, tb, jend * NGW * (int)sizeof(T));
  for (int j0 = 1; j0 < jend; j0 += RB) {
    const int nr = min(RB, jend - j0);
    if (j0 > 1) __syncthreads();    // previous round's readers of Ts are done
    if (!GT) stage(Ts, Tall + ((int64_t)b * S + j0) * NGW * NGW, nr * NGW * NGW * (int)sizeof(T));
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    for (int u = 0; u < nr; ++u) {
      const int j = j0 + u;
      const T* Tj = GT ? Tall + ((int64_t)b * S + j) * NGW * NGW : Ts + (size_t)u * NGW * NGW;
      const T* hp = zt + (size_t)(j - 1) * NGW;    // true tail_{j-1}
      for (int i0 = 0; i0 < NGW; i0 += RPP) {
        const int i = i0 + (int)threadIdx.x / TPR;
        T acc = T(0);
        if (i < NGW) {
          const T* row = Tj + (size_t)i * NGW;
          int q = (part + TPR * i) % NGW;
          for (int m = 0; m < NGW / TPR; ++m) {
            acc += row[q] * hp[q];
            q += TPR;
            if (q >= NGW) q -= NGW;
          }
        }
        for (int o = TPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (i < NGW && part == 0) {
          const T t = zt[(size_t)j * NGW + i] + acc;
          zt[(size_t)j * NGW + i] = t;
          tb[(int64_t)j * NGW + i] = t;
        }
      }
      __syncthreads();
    }
  }
}

// History correction z_p += sum_q X[q][p] h_q of segments s >= 1, h = the
// true tail_{s-1}; grid (row tiles of kCorrThreads positions, S - 1, P), one
// position per thread, X column-major (coalesced).  CHAIN: the tails are
// still the zero-history ones of k_sweep and each CTA first runs the transfer
// recurrence tail_j = zhat_tail_j + T_j tail_{j-1} up to j = s-1 itself
// (T_1 .. T_{s-1} and the tails staged by cp.async in one round, TPR threads
// per row as in k_seg_chain), which saves the separate chain launch for short
// chains; otherwise k_seg_chain has already made the tails true.
template <typename T>
__host__ __device__ inline size_t fused_chain_smem(int K, int S) {
  const int kh = hist_width(K);
  return ((size_t)(S > 2 ? S - 2 : 0) * kh * kh + (size_t)(S - 1) * kh) * sizeof(T);
}
constexpr size_t kFusedChainMaxSmem = 96 * 1024;

template <typename T, typename OT, int MODE, bool CHAIN>
__global__ void __launch_bounds__(kCorrThreads)
k_seg_correct(const T* __restrict__ Xall, const T* __restrict__ tails, const T* __restrict__ Tall, int K, Dev d,
              int S, int cpsmax, OT* __restrict__ out, Gate gt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (gate_skip(gt)) return;
  const int b = blockIdx.z;
  const int seg = (int)blockIdx.y + 1;
  const int NGW = hist_width(K);                   // history width
  const int ld = (int)d.ld[b];
  const int64_t s = d.off[b];
  const int n = (int)(d.off[b + 1] - s);
  const int nch = ld / CHK;
  const int cps = seg_chunks(nch, S);
  const int c0 = seg * cps, c1 = min(nch, c0 + cps);
  const int p = blockIdx.x * kCorrThreads + threadIdx.x;
  if (c0 >= c1 || (int)blockIdx.x * kCorrThreads >= (c1 - c0) * CHK) return;
  const T* h = nullptr;
  if (CHAIN && seg >= 2) {
    T* Ts = reinterpret_cast<T*>(smem_raw);                   // T_1 .. T_{seg-1}
    T* zt = Ts + (size_t)(seg - 1) * NGW * NGW;               // tails 0 .. seg-1
    auto stage = [&](void* dsts, const void* srcg, int nbytes) {
      const char* src = reinterpret_cast<const char*>(srcg);
      const unsigned dst = (unsigned)__cvta_generic_to_shared(dsts);
      for (int o = threadIdx.x * 16; o < nbytes; o += blockDim.x * 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst + o), "l"(src + o) : "memory");
    };
    stage(zt, tails + (int64_t)b * S * NGW, seg * NGW * (int)sizeof(T));
    stage(Ts, Tall + ((int64_t)b * S + 1) * NGW * NGW, (seg - 1) * NGW * NGW * (int)sizeof(T));
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    int TPR = 1;
    while (TPR < 8 && NGW % (2 * TPR) == 0 && NGW * 2 * TPR <= kCorrThreads) TPR *= 2;
    const int part = threadIdx.x % TPR;
    const int RPP = kCorrThreads / TPR;            // rows per pass
    for (int j = 1; j < seg; ++j) {
      const T* Tj = Ts + (size_t)(j - 1) * NGW * NGW;
      const T* hp = zt + (size_t)(j - 1) * NGW;
      for (int i0 = 0; i0 < NGW; i0 += RPP) {
        const int i = i0 + (int)threadIdx.x / TPR;
        T acc = T(0);
        if (i < NGW) {
          const T* row = Tj + (size_t)i * NGW;
          int q = (part + TPR * i) % NGW;
          for (int m = 0; m < NGW / TPR; ++m) {
            acc += row[q] * hp[q];
            q += TPR;
            if (q >= NGW) q -= NGW;
          }
        }
        for (int o = TPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (i < NGW && part == 0) zt[(size_t)j * NGW + i] += acc;
      }
      __syncthreads();
    }
    h = zt + (size_t)(seg - 1) * NGW;
  } else {
    T* hd = reinterpret_cast<T*>(smem_raw);       // the true tail_{s-1} (NGW values)
    for (int t = threadIdx.x; t < NGW; t += blockDim.x) hd[t] = tails[((int64_t)b * S + seg - 1) * NGW + t];
    __syncthreads();
    h = hd;
  }
  if (p >= (c1 - c0) * CHK) return;
  const int r = row_of<MODE>(c0 * CHK + p, ld);
  if (r >= n) return;
  const int64_t xm = (int64_t)cpsmax * CHK;
  const T* Xp = Xall + ((int64_t)b * (S - 1) + (seg - 1)) * xm * NGW + p;
  T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
#pragma unroll 2
  for (int q = 0; q < NGW; q += 4) {
    a0 += Xp[(int64_t)q * xm] * h[q];
    a1 += Xp[(int64_t)(q + 1) * xm] * h[q + 1];
    a2 += Xp[(int64_t)(q + 2) * xm] * h[q + 2];
    a3 += Xp[(int64_t)(q + 3) * xm] * h[q + 3];
  }
  OT* ob = out + s;
  ob[r] = (OT)((T)ob[r] + ((a0 + a1) + (a2 + a3)));
}

// Unsegmented block solve (S = 1): one CTA per block runs the forward and
// then the backward sweep of its block.  Measured faster than two launches of
// k_sweep with S = 1 (125 us against about 150 us per apply on the
// N = 200000, K = 50, P = 50 FP32 system).
template <typename T, bool TRANS, int PFD, int NPW>
__global__ void __launch_bounds__(32 * (NPW + 2))
k_block_solve(const T* __restrict__ M1all, const T* __restrict__ M2all, const int64_t* __restrict__ cbase, int K,
              Dev d, const double* __restrict__ r_in, double* __restrict__ z_out, T* __restrict__ tmp,
              const double* __restrict__ ctop_all, const double* __restrict__ cbot_all, int P,
              int* __restrict__ err, Gate gt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (gate_skip(gt)) return;
  const int b = blockIdx.x;
  const int64_t s = d.off[b];
  SweepGeom g;
  g.K = K;
  g.n = (int)(d.off[b + 1] - s);
  g.ld = (int)d.ld[b];
  g.ng = n_couplings(K);
  const int nch = g.ld / CHK;
  const bool has_top = ctop_all && b > 0;
  const bool has_bot = cbot_all && b + 1 < P;
  unsigned ph = 0;
  bool failed = false;
  {
    SweepSh<T, double> sh = carve<T, double, PFD, NPW>(smem_raw, g);
    if (threadIdx.x == 0) {
      for (int q = 0; q <= PFD; ++q) mbar_init(&sh.bar[q], 1);
      mbar_fence_init();
    }
    for (int t = threadIdx.x; t < K; t += blockDim.x) {
      sh.corr[t] = has_top ? ctop_all[(int64_t)(b - 1) * K + t] : 0.0;
      sh.corr[K + t] = has_bot ? cbot_all[(int64_t)b * K + t] : 0.0;
    }
    if (!TRANS)
      sweep<T, double, T, LF, PFD, NPW>(sh, g, M1all + cbase[b], r_in + s, has_top, has_bot, tmp + s, 0, nch, nullptr, ph,
                              failed, err);
    else
      sweep<T, double, T, UTF, PFD, NPW>(sh, g, M1all + cbase[b], r_in + s, has_top, has_bot, tmp + s, 0, nch, nullptr, ph,
                               failed, err);
  }
  {
    SweepSh<T, T> sh = carve<T, T, PFD, NPW>(smem_raw, g);
    if (!TRANS)
      sweep<T, T, double, UB, PFD, NPW>(sh, g, M2all + cbase[b], tmp + s, false, false, z_out + s, 0, nch, nullptr, ph,
                              failed, err);
    else
      sweep<T, T, double, LTB, PFD, NPW>(sh, g, M2all + cbase[b], tmp + s, false, false, z_out + s, 0, nch, nullptr, ph,
                               failed, err);
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
                          const double* __restrict__ g, double* __restrict__ ctop, double* __restrict__ cbot,
                          Gate gate) {
  extern __shared__ __align__(16) double sh[];
  if (gate_skip(gate)) return;
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

// The same reduced solves for wide bands, one kernel per dependent step so
// that each step spreads over (ceil(K / 32), P - 1) CTAs of 8 warps:
//   k_red_mv   y = base - A x (or A x) for the 32 rows of its CTA, a warp per
//              row reading A's row coalesced, x staged in shared memory;
//   k_red_cpl  cbot, ctop from the band, lanes over rows and warps over band
//              diagonals (consecutive rows of a diagonal are contiguous).
// Same arithmetic as k_reduced, different summation order.
constexpr int kRedRows = 32;
enum RedStep { RED_RHS = 0, RED_XT = 1, RED_XB = 2 };

template <typename M, int STEP>
__global__ void __launch_bounds__(256)
k_red_mv(const M* __restrict__ A, int K, Dev d, const double* __restrict__ g, const double* __restrict__ xin,
         double* __restrict__ y, Gate gate) {
  extern __shared__ __align__(16) double xs[];     // K
  if (gate_skip(gate)) return;
  const int i = blockIdx.y;
  const int64_t s = d.off[i + 1];
  const int64_t KK = (int64_t)K * K;
  const M* Ai = A + i * KK;
  // x: g^(b)_i (RHS step) or the previous step's vector of this interface
  for (int t = threadIdx.x; t < K; t += blockDim.x) xs[t] = STEP == RED_RHS ? g[s - K + t] : xin[(int64_t)i * K + t];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int rr = warp; rr < kRedRows; rr += 8) {
    const int r = blockIdx.x * kRedRows + rr;
    if (r >= K) break;
    const M* row = Ai + (int64_t)r * K;
    double a0 = 0.0, a1 = 0.0;
    int q = lane;
    for (; q + 32 < K; q += 64) {
      a0 += (double)row[q] * xs[q];
      a1 += (double)row[q + 32] * xs[q + 32];
    }
    if (q < K) a0 += (double)row[q] * xs[q];
    double acc = a0 + a1;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      double v;
      if (STEP == RED_RHS) v = g[s + r] - acc;                       // g^(t)_{i+1} - W g^(b)_i
      else if (STEP == RED_XT) v = acc;                             // Rbar^{-1} rhs
      else v = g[s - K + r] - acc;                                  // g^(b)_i - V xt
      y[(int64_t)i * K + r] = v;
    }
  }
}

template <bool TRANS>
__global__ void __launch_bounds__(256)
k_red_cpl(const double* __restrict__ band, int64_t N, int K, Dev d, const double* __restrict__ xt,
          const double* __restrict__ xb, double* __restrict__ ctop, double* __restrict__ cbot, Gate gate) {
  __shared__ double pb[8][kRedRows], pc[8][kRedRows];
  if (gate_skip(gate)) return;
  const int i = blockIdx.y;
  const int64_t s = d.off[i + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = blockIdx.x * kRedRows + lane;
  const double* xti = xt + (int64_t)i * K;
  const double* xbi = xb + (int64_t)i * K;
  double accb = 0.0, accc = 0.0;
  if (r < K) {
    // B (or B' = C^T): entries (r, r - dd), dd = 0 .. r; C (or C' = B^T): entries (r, r + e), e = 0 .. K-1-r
    for (int dd = warp; dd <= r; dd += 8) {
      const double a = TRANS ? band[(int64_t)(2 * K - dd) * N + s - K + r] : band[(int64_t)dd * N + s + r - dd];
      accb += a * xti[r - dd];
    }
    for (int e = warp; e < K - r; e += 8) {
      const double a = TRANS ? band[(int64_t)e * N + s + r] : band[(int64_t)(2 * K - e) * N + s - K + r + e];
      accc += a * xbi[r + e];
    }
  }
  pb[warp][lane] = accb;
  pc[warp][lane] = accc;
  __syncthreads();
  if (warp == 0 && r < K) {
    double b = 0.0, c = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      b += pb[w][lane];
      c += pc[w][lane];
    }
    cbot[(int64_t)i * K + r] = b;
    ctop[(int64_t)i * K + r] = c;
  }
}

// K from which the reduced solves run as the four step kernels above
constexpr int kRedStagedK = 96;

template <typename T, typename YT, typename OT, int MODE>
cudaError_t launch_sweep(const T* M, const T* Tm, const T* Xm, const Factors<T>& f, int K, int P, Dev d,
                         const YT* yin, OT* out, const double* ctop, const double* cbot, cudaStream_t s, Gate gt) {
  // up to 4 couplings per chunk one preparation warp and 4 chunks in flight;
  // wider bands 2 (<= 7 couplings) or 4 preparation warps, 4 chunks in flight
  // where the ring fits, else 2
  const int ng = n_couplings(K);
  size_t smem;
  int threads;
  void (*kern)(const T*, const int64_t*, int, Dev, const YT*, OT*, T*, const double*, const double*, int, int, int*,
               Gate);
  if (ng <= 4) {
    smem = sweep_smem<T>(K);
    kern = k_sweep<T, YT, OT, MODE>;
    threads = NWS * 32;
  } else if (ng <= 7) {
    const bool deep = sweep_smem<T, PF, 2>(K) <= kSmemPerBlock;
    smem = deep ? sweep_smem<T, PF, 2>(K) : sweep_smem<T, 2, 2>(K);
    kern = deep ? k_sweep<T, YT, OT, MODE, PF, 2> : k_sweep<T, YT, OT, MODE, 2, 2>;
    threads = 4 * 32;
  } else {
    const bool deep = sweep_smem<T, PF, 4>(K) <= kSmemPerBlock;
    smem = deep ? sweep_smem<T, PF, 4>(K) : sweep_smem<T, 2, 4>(K);
    kern = deep ? k_sweep<T, YT, OT, MODE, PF, 4> : k_sweep<T, YT, OT, MODE, 2, 4>;
    threads = 6 * 32;
  }
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int S = f.S;
  count_launches(1);
  kern<<<dim3(S, P), threads, smem, s>>>(M, f.cbase, K, d, yin, out, f.tails, ctop, cbot, P, S, f.err, gt);
  e = cudaGetLastError();
  if (e != cudaSuccess || S == 1) return e;
  const int tiles = (f.cpsmax * CHK + kCorrThreads - 1) / kCorrThreads;
  const size_t fsm = fused_chain_smem<T>(K, S);
  if (S > 2 && fsm <= kFusedChainMaxSmem) {     // short chains: run inside the correction
    auto corr = k_seg_correct<T, OT, MODE, true>;
    if (fsm > 48 * 1024) {
      e = cudaFuncSetAttribute(corr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm);
      if (e != cudaSuccess) return e;
    }
    count_launches(1);
    corr<<<dim3(tiles, S - 1, P), kCorrThreads, fsm, s>>>(Xm, f.tails, Tm, K, d, S, f.cpsmax, out, gt);
    return cudaGetLastError();
  }
  if (S > 2) {
    size_t csmem = chain_smem<T>(K, S);
    auto chain = k_seg_chain<T, false>;
    if (csmem > kSmemPerBlock) {        // one transfer matrix exceeds shared memory: read them from L2
      csmem = (size_t)(S + 1) * hist_width(K) * sizeof(T);
      chain = k_seg_chain<T, true>;
    }
    if (csmem > 48 * 1024) {
      e = cudaFuncSetAttribute(chain, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csmem);
      if (e != cudaSuccess) return e;
    }
    count_launches(1);
    chain<<<P, kCorrThreads, csmem, s>>>(Tm, f.tails, K, d, S, gt);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  count_launches(1);
  k_seg_correct<T, OT, MODE, false><<<dim3(tiles, S - 1, P), kCorrThreads, (size_t)hist_width(K) * sizeof(T), s>>>(
      Xm, f.tails, Tm, K, d, S, f.cpsmax, out, gt);
  return cudaGetLastError();
}

// Block-diagonal solve D g = r: forward then backward sweep of every block
// (L then U; for the transposed operator U^T then L^T).
template <typename T, bool TRANS>
cudaError_t launch_block_solve(const Factors<T>& f, int K, int P, Dev d, const double* r, double* z, T* tmp,
                               const double* ctop, const double* cbot, cudaStream_t s, Gate gt) {
  cudaError_t e;
  if (f.S == 1) {
    // four chunks in flight where the ring fits, two for the widest bands;
    // the next chunk's couplings split over 1, 2 or 4 prepare warps
    const int ng = n_couplings(K);
    const int npw = ng <= 3 ? 1 : (ng <= 7 ? 2 : 4);
    const bool deep = (npw == 1 ? sweep_smem<T, PF, 1>(K) : npw == 2 ? sweep_smem<T, PF, 2>(K)
                                                                     : sweep_smem<T, PF, 4>(K)) <= kSmemPerBlock;
    size_t smem;
    void (*kern)(const T*, const T*, const int64_t*, int, Dev, const double*, double*, T*, const double*,
                 const double*, int, int*, Gate);
    if (npw == 1) {
      smem = sweep_smem<T, PF, 1>(K);
      kern = k_block_solve<T, TRANS, PF, 1>;
    } else if (npw == 2) {
      smem = deep ? sweep_smem<T, PF, 2>(K) : sweep_smem<T, 2, 2>(K);
      kern = deep ? k_block_solve<T, TRANS, PF, 2> : k_block_solve<T, TRANS, 2, 2>;
    } else {
      smem = deep ? sweep_smem<T, PF, 4>(K) : sweep_smem<T, 2, 4>(K);
      kern = deep ? k_block_solve<T, TRANS, PF, 4> : k_block_solve<T, TRANS, 2, 4>;
    }
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    count_launches(1);
    kern<<<P, 32 * (npw + 2), smem, s>>>(TRANS ? f.Mutf : f.Mlf, TRANS ? f.Mltb : f.Mub, f.cbase, K, d, r, z, tmp,
                                         ctop, cbot, P, f.err, gt);
    return cudaGetLastError();
  }
  if (!TRANS) {
    e = launch_sweep<T, double, T, LF>(f.Mlf, f.Tlf, f.Xlf, f, K, P, d, r, tmp, ctop, cbot, s, gt);
    if (e != cudaSuccess) return e;
    return launch_sweep<T, T, double, UB>(f.Mub, f.Tub, f.Xub, f, K, P, d, tmp, z, nullptr, nullptr, s, gt);
  }
  e = launch_sweep<T, double, T, UTF>(f.Mutf, f.Tutf, f.Xutf, f, K, P, d, r, tmp, ctop, cbot, s, gt);
  if (e != cudaSuccess) return e;
  return launch_sweep<T, T, double, LTB>(f.Mltb, f.Tltb, f.Xltb, f, K, P, d, tmp, z, nullptr, nullptr, s, gt);
}

}  // namespace

// the unsegmented sweep's smallest ring (two chunks ahead, four prepare warps): the limit on K
size_t sweep_smem_bytes(int K, bool fp64) { return fp64 ? sweep_smem<double, 2, 4>(K) : sweep_smem<float, 2, 4>(K); }
bool seg_sweeps_fit(int K, bool fp64) {
  const int ng = n_couplings(K);
  if (ng <= 4) return (fp64 ? sweep_smem<double>(K) : sweep_smem<float>(K)) <= kSmemPerBlock;
  // the shallow ring of the launched shape, and the wide transfer kernel's tiles
  const size_t ts = fp64 ? 8 : 4;
  const size_t sw = ng <= 7 ? (fp64 ? sweep_smem<double, 2, 2>(K) : sweep_smem<float, 2, 2>(K))
                            : (fp64 ? sweep_smem<double, 2, 4>(K) : sweep_smem<float, 2, 4>(K));
  const size_t tr = (2 * (size_t)ng * CHK * CHK + (size_t)(ng + 1) * CHK * (32 + 16 / ts)) * ts;
  return sw <= kSmemPerBlock && tr <= kSmemPerBlock;
}
int chunk_couplings(int K) { return n_couplings(K); }

// scratch layout (doubles): [0, N) g ; then T tmp (N); then ctop, cbot ((P-1) K each);
// then (wide bands, SaP-C) rhs, xt, xb of the reduced solves ((P-1) K each)
template <typename T>
cudaError_t launch_apply(const double* band, int64_t N, int K, int P, Dev d, const Factors<T>& f,
                         int variant, bool transpose, const double* r, double* z, double* scratch,
                         cudaStream_t s, Gate gt) {
  double* g = scratch;
  T* tmp = reinterpret_cast<T*>(scratch + N);
  double* ctop = scratch + 2 * N;
  double* cbot = ctop + (int64_t)(P > 1 ? P - 1 : 1) * K;
  cudaError_t e;
  if (variant == SAP_D || P == 1) {
    return transpose ? launch_block_solve<T, true>(f, K, P, d, r, z, tmp, nullptr, nullptr, s, gt)
                     : launch_block_solve<T, false>(f, K, P, d, r, z, tmp, nullptr, nullptr, s, gt);
  }
  e = transpose ? launch_block_solve<T, true>(f, K, P, d, r, g, tmp, nullptr, nullptr, s, gt)
                : launch_block_solve<T, false>(f, K, P, d, r, g, tmp, nullptr, nullptr, s, gt);
  if (e != cudaSuccess) return e;
  if (K < kRedStagedK) {
    size_t sm = 5 * (size_t)K * sizeof(double);
    count_launches(1);
    if (!transpose)
      k_reduced<T, false><<<P - 1, 128, sm, s>>>(band, N, K, d, f.V, f.Wt, f.R, g, ctop, cbot, gt);
    else
      k_reduced<T, true><<<P - 1, 128, sm, s>>>(band, N, K, d, f.Va, f.Wa, f.Ra, g, ctop, cbot, gt);
  } else {
    double* rhs = cbot + (int64_t)(P - 1) * K;     // three (P - 1) K vectors after cbot
    double* xt = rhs + (int64_t)(P - 1) * K;
    double* xb = xt + (int64_t)(P - 1) * K;
    const dim3 grid((K + kRedRows - 1) / kRedRows, P - 1);
    const size_t sm = (size_t)K * sizeof(double);
    count_launches(4);
    k_red_mv<T, RED_RHS><<<grid, 256, sm, s>>>(transpose ? f.Wa : f.Wt, K, d, g, nullptr, rhs, gt);
    k_red_mv<double, RED_XT><<<grid, 256, sm, s>>>(transpose ? f.Ra : f.R, K, d, g, rhs, xt, gt);
    k_red_mv<T, RED_XB><<<grid, 256, sm, s>>>(transpose ? f.Va : f.V, K, d, g, xt, xb, gt);
    if (!transpose) k_red_cpl<false><<<grid, 256, 0, s>>>(band, N, K, d, xt, xb, ctop, cbot, gt);
    else k_red_cpl<true><<<grid, 256, 0, s>>>(band, N, K, d, xt, xb, ctop, cbot, gt);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return transpose ? launch_block_solve<T, true>(f, K, P, d, r, z, tmp, ctop, cbot, s, gt)
                   : launch_block_solve<T, false>(f, K, P, d, r, z, tmp, ctop, cbot, s, gt);
}

template cudaError_t launch_apply<float>(const double*, int64_t, int, int, Dev, const Factors<float>&, int, bool,
                                         const double*, double*, double*, cudaStream_t, Gate);
template cudaError_t launch_apply<double>(const double*, int64_t, int, int, Dev, const Factors<double>&, int,
                                          bool, const double*, double*, double*, cudaStream_t, Gate);

}  // namespace sap
