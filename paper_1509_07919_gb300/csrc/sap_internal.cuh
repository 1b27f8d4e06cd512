// Internal declarations shared by the libsap translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <vector>
#include "../../include/sap.h"

namespace sap {

// Upper bound of the half-bandwidth searched by sap_max_K; the limit in force
// is the largest K whose sweep ring (two chunks ahead at least) and factor
// staging fit in shared memory (512 for FP32, 256 for FP64 factors).
constexpr int kMaxK = 600;
constexpr size_t kSmemPerBlock = 232448;   // opt-in shared memory per CTA on sm_103

// Dynamic shared memory of the sweep and factor kernels for half-bandwidth K.
size_t sweep_smem_bytes(int K, bool fp64);
// Coupling matrices per chunk of the blocked sweeps: ceil(K / 32).
int chunk_couplings(int K);
// The segmented sweeps' kernel (its ring of chunk matrices) fits in shared
// memory for half-bandwidth K (FP32 up to K = 512, FP64 up to K = 256).
bool seg_sweeps_fit(int K, bool fp64);
// tc: the tensor-core (BF16 operand, FP32 accumulate) trailing update of the
// FP32 factorisation, used from K = kTcMinK on (precision SAP_FP32_BF16TU).
constexpr int kTcMinK = 64;
size_t lu_smem_bytes(int K, bool fp64, bool tc = false);
// Factor window: in shared memory when it fits, else in a global scratch of
// lu_window_elems(K) elements per CTA (L2-resident); lu_smem_used gives the
// shared memory of either form.
size_t lu_smem_used(int K, bool fp64, bool global_window, bool tc = false);
bool lu_window_global(int K, bool fp64, bool tc = false);
size_t lu_window_elems(int K);
// CTAs of the persistent work-list LU for nitems items of half-bandwidth <= Kmax.
int lu_items_grid(int nitems, int Kmax, bool fp64, bool tc = false);
// Shared memory of the chunk-matrix kernel.
size_t chunk_mats_smem_bytes(int K, bool fp64);

// Factor storage of one block (per block i, local rows/cols 0..n_i-1):
// "diagonal-major" like the input band, indexed by the column:
//   F_i[c * ld_i + q] = factor entry (r, q) with c = K + r - q,
// c > K: unit-lower L, c <= K: U (diagonal at c = K).
struct Layout {
  int64_t N = 0;
  int K = 0, P = 0, W = 0;
  std::vector<int64_t> off;    // P+1 row offsets
  std::vector<int64_t> fbase;  // element offset of block i in the factor array
  std::vector<int64_t> ld;     // leading dimension of block i
  int64_t f_elems = 0;
  int64_t c_elems = 0;   // chunk-matrix elements per sweep kind (all blocks)
  int max_nch = 0;       // most 32-row chunks in one block
  int S = 1;             // sweep segments per block
};

struct Dev {  // device copies of the partition, passed to kernels
  const int64_t* off;
  const int64_t* fbase;
  const int64_t* ld;
};

template <typename T>
struct Factors {
  T* F = nullptr;        // LU factors of all blocks
  T* ULt = nullptr;      // per block i >= 1: top K x K of [U'|L'] (row-major, U' strictly upper, L' on/below)
  T* V = nullptr;        // per interface: V^(b)_i (K x K row-major)
  T* Wt = nullptr;       // per interface: W^(t)_{i+1}
  double* R = nullptr;   // per interface: Rbar_i^{-1} (from its GEPP factors), FP64
  int* piv = nullptr;    // per interface: pivots of Rbar_i
  double* R0 = nullptr;  // per interface: Rbar_i before factoring (kept for inspection)
  // adjoint SaP (built on demand)
  T* Va = nullptr; T* Wa = nullptr; double* Ra = nullptr; int* piva = nullptr; double* Ra0 = nullptr;
  // chunk matrices of the blocked sweeps (MINV, G per 32-row chunk, sweep order):
  // L forward, U backward (built with the factors), U^T forward, L^T backward
  // (built on the first transposed apply).  cbase[i]: offset of block i.
  T* Mlf = nullptr; T* Mub = nullptr; T* Mutf = nullptr; T* Mltb = nullptr;
  const int64_t* cbase = nullptr;
  // segmented sweeps (S segments per block): per block and segment s >= 1 the
  // KH x KH transfer matrix of each sweep kind (KH = hist_width(K), row-major,
  // segment 0 unused) and its history response X, and the per-apply tails
  // (last KH values of each segment) of the zero-history pass
  int S = 1;
  T* Tlf = nullptr; T* Tub = nullptr; T* Tutf = nullptr; T* Tltb = nullptr;
  T* Xlf = nullptr; T* Xub = nullptr; T* Xutf = nullptr; T* Xltb = nullptr;   // history responses
  int cpsmax = 0;        // chunks of the longest segment
  T* tails = nullptr;    // P x S x KH
  int* err = nullptr;    // int[2]: [0] set to nonzero by a device-side wait that timed out, [1] its poll limit
};

// Device-side control of the Krylov iteration.  A launch carrying a Gate
// does nothing when the solve has finished (flags[F_DONE]); the true-residual
// launches of an exit test run only when the test asked for them
// (flags[F_CHECK]) and the residual replacement only when the true residual
// failed (flags[F_REPLACE]).  Kernels read the flags at entry and return
// uniformly per CTA, so a gated-off launch costs only its launch.
enum FlagSlot { F_DONE = 0, F_CHECK, F_REPLACE, F_STATUS, F_RESTARTS, F_ROUNDS, F_COUNT };
// G_KEEP: active and no restart flagged (the CG step's own p update).
enum GateMode { G_ALWAYS = 0, G_ACTIVE = 1, G_CHECK = 2, G_REPLACE = 3, G_KEEP = 4 };
struct Gate {
  const int* flags = nullptr;
  int mode = G_ALWAYS;
};
__device__ __forceinline__ bool gate_skip(const Gate& g) {
  if (!g.flags || g.mode == G_ALWAYS) return false;
  if (g.flags[F_DONE]) return true;
  if (g.mode == G_CHECK) return g.flags[F_CHECK] == 0;
  if (g.mode == G_REPLACE) return g.flags[F_REPLACE] == 0;
  if (g.mode == G_KEEP) return g.flags[F_REPLACE] != 0;
  return false;
}

// Bounded device waits.  The error word of a handle is int[2]: err[0] is set
// to nonzero by a wait that gave up, err[1] holds the number of polls a wait
// makes before it gives up (sap_options_t.spin_limit; 0 selects kDefaultSpin).
constexpr int kDefaultSpin = 1 << 24;
__host__ __device__ inline int spin_limit_value(int64_t opt) {
  return opt <= 0 ? kDefaultSpin : (opt > 0x7fffffff ? 0x7fffffff : (int)opt);
}
__device__ __forceinline__ int spin_limit_of(const int* err) {
  if (!err) return kDefaultSpin;
  const int v = *(volatile const int*)(err + 1);
  return v > 0 ? v : kDefaultSpin;
}

// Host-side count of kernel launches issued by the library (for reporting).
void count_launches(int n);
// one bounded wait on a barrier nothing completes (sets *err after `limit` polls)
cudaError_t launch_wait_selftest(int limit, int* err, cudaStream_t s);
long long launches_so_far();

// ---- launchers (each returns cudaGetLastError()) ----
cudaError_t launch_spmv(const double* band, int64_t N, int K, const double* x, double* y,
                        bool transpose, cudaStream_t s, Gate gt = Gate());
// A sparse operator in the reordered numbering of the sparse front end
// (include/sap_sparse.h): entry (i, j) of the CSR matrix at (rownew[i],
// colnew[j]) with value (r_i a_ij) s_j (r, s null: 1).  Borrowed pointers.
struct CsrOp {
  int64_t n = 0, nnz = 0;
  const int64_t* rowptr = nullptr;
  const int32_t* col = nullptr;
  const double* val = nullptr;
  const int32_t* rownew = nullptr;
  const int32_t* colnew = nullptr;
  const double* r = nullptr;
  const double* s = nullptr;
};
// y = A' x for the reordered operator A' of a CsrOp (one warp per stored row).
cudaError_t launch_spmv_pcsr(const CsrOp& A, const double* x, double* y, cudaStream_t s, Gate gt = Gate());
cudaError_t launch_absmax(const double* band, int64_t N, int K, double* out, cudaStream_t s);
cudaError_t launch_grad_band(const double* lam, const double* x, int64_t N, int K, double* g,
                             cudaStream_t s);

// FP32 path: absmax plus an FP32 copy of the band (the factor kernels load it)
cudaError_t launch_absmax_cast(const double* band, int64_t N, int K, double* out, float* bandf, cudaStream_t s);
// One block of a batched LU work list (band, factor storage and boost
// threshold of its own system).
struct LuItem {
  const void* band;          // the system's band in the factor precision
  void* F;                   // the block's factor storage
  const double* absmax;      // the system's max |a_ij|
  unsigned long long* nb;    // the system's boosted-pivot counter
  int64_t N, s, ld;          // system order, first row of the block, factor leading dimension
  double eps;                // relative boost threshold
  int K, n;                  // half-bandwidth, block rows
};
template <typename T>
cudaError_t launch_factor_lu_items(const LuItem* items, int nitems, int Kmax, unsigned* counter, T* wscratch,
                                   bool tc, int* err, cudaStream_t s);

template <typename T>
cudaError_t launch_factor_lu(const T* band, int64_t N, int K, int P, Dev d, const double* absmax,
                             double eps, T* F, unsigned long long* n_boosted, T* wscratch, bool tc, int* err,
                             cudaStream_t s);
template <typename T>
cudaError_t launch_factor_ul(const T* band, int64_t N, int K, int P, Dev d, const double* absmax,
                             double eps, T* ULt, unsigned long long* n_boosted, T* wscratch, bool tc, int* err,
                             cudaStream_t s);
template <typename T>
cudaError_t launch_spikes(const double* band, int64_t N, int K, int P, Dev d, const T* F, const T* ULt,
                          bool adjoint, T* V, T* Wt, double* Rinv, double* R0, int* piv, int* singular,
                          void* gscratch, cudaStream_t s, cudaEvent_t ev_rd = nullptr);
// ev_rd (optional) is recorded between the spike tips and the reduced systems
// (Rbar_i, its GEPP and inverse); where one kernel per interface does both
// (K x K matrices in shared memory) it is recorded after that kernel.
// Global scratch of the spike kernel (0 when its K x K matrices fit in shared
// memory): one workspace per interface, shared by the forward and adjoint tips.
size_t spike_scratch_bytes(int K, int P, bool fp64);
template <typename T>
cudaError_t launch_chunk_mats(const T* F, int K, int P, Dev d, const int64_t* cbase, int max_nch, int mode, T* out,
                              cudaStream_t s);
// Transfer matrices (tout: P x S x KH^2) and history responses X (xout:
// P x (S-1) x KH x cpsmax 32, column-major per segment), KH = hist_width(K), of
// segments 1..S-1 of every block, from the chunk matrices M of one sweep kind.
template <typename T>
cudaError_t launch_seg_trans(const T* M, const int64_t* cbase, int K, int P, int S, int cpsmax, Dev d, T* tout,
                             T* xout, cudaStream_t s);
// Width of a segment's history in the segmented sweeps: only the last K
// positions before a segment couple into it, rounded up to a multiple of 4
// (16-byte rows for FP32) and at most 32 ceil(K/32).
__host__ __device__ inline int hist_width(int K) { return (K + 3) / 4 * 4; }
// Chunks of 32 rows per segment of a block with nch chunks: ceil(nch / S).
__host__ __device__ inline int seg_chunks(int nch, int S) { return (nch + S - 1) / S; }
template <typename T>
cudaError_t launch_apply(const double* band, int64_t N, int K, int P, Dev d, const Factors<T>& f,
                         int variant, bool transpose, const double* r, double* z, double* scratch,
                         cudaStream_t s, Gate gt = Gate());

// Rbar_i = I - W^(t)_{i+1} V^(b)_i from given tips (nI interfaces), its GEPP
// and inverse (the wide-band kernels of launch_spikes) in a workspace of
// reduced_ws_bytes(K, nI, fp64) bytes.
size_t reduced_ws_bytes(int K, int nI, bool fp64);
template <typename T>
cudaError_t launch_reduced(const T* V, const T* Wt, int K, int nI, double* Rinv, double* R0, int* piv, int* singular,
                           void* gws, cudaStream_t s);

// ---- SaP with a bandwidth of its own per block (third-stage reordering) ----
// Partition and block permutations on the device.  perm[g] is the new local
// index of global row/column g inside its block (Ahat_b = Pi_b A_b Pi_b^T),
// pinv[off_b + r] the old local index of new local row r.
struct BlockMap {
  int64_t N = 0;
  int K = 0, P = 0;
  int64_t q = 0, pr = 0;            // blocks 0..pr-1 have q + 1 rows, the others q
  const int64_t* off = nullptr;     // P + 1
  const int32_t* perm = nullptr;    // N
  const int32_t* pinv = nullptr;    // N
  const int32_t* Kb = nullptr;      // P: half-bandwidth of each reordered block
  const int64_t* hbase = nullptr;   // P: offset of block b's band in the reordered-band buffer
};
// Kout[b] = max |perm(i) - perm(j)| over the nonzero entries of block b (P ints).
cudaError_t launch_block_bw(const double* band, const BlockMap& m, int* Kout, cudaStream_t s);
// The reordered blocks (band storage, half-bandwidth Kb[b], n_b columns) into
// the zeroed buffer hb (hb_elems doubles); *err set on an entry beyond Kb[b].
cudaError_t launch_block_gather(const double* band, const BlockMap& m, double* hb, int64_t hb_elems, int* err,
                                cudaStream_t s);
// to_new: y = Pi x (y[off_b + perm(g)] = x[g]); else y = Pi^T x.
cudaError_t launch_block_perm(const BlockMap& m, const double* x, double* y, bool to_new, cudaStream_t s,
                              Gate gt = Gate());
// Dynamic shared memory of the entire-spike kernel for blocks of up to ngmax
// chunk couplings (chunk_couplings(K_b)).
size_t full_spikes_smem(int ngmax, bool fp64);
// Row stride of the stored entire spikes: K rounded up to 16 bytes (the
// padding stays zero).
int spike_row_stride(int K, bool fp64);
// Entire spikes of every interface i into spk (row-major n x KS at
// sbase[2 i] for Vhat_i, sbase[2 i + 1] for What_{i+1}) by the sweeps of
// each block b with its chunk matrices (Mfp[b]: forward L, Mbp[b]: backward
// U, ngp[b] couplings per chunk, leading dimension ldp[b]), and their tips
// V^(b)_i, W^(t)_{i+1} (K x K row-major per interface).  adjoint: the spikes of
// the preconditioner of A^T (Mfp / Mbp then the blocks' U^T forward and L^T
// backward matrices; couplings B'_i = C_{i+1}^T, C'_{i+1} = B_i^T).
template <typename T>
cudaError_t launch_full_spikes(const double* band, const BlockMap& m, int ngmax, const void* const* Mfp,
                               const void* const* Mbp, const int* ngp, const int64_t* ldp, T* spk,
                               const int64_t* sbase, T* Vtip, T* Wtip, bool adjoint, cudaStream_t s);
// x^(t), x^(b) of every interface from g = D^{-1} r (new numbering), Eq. (2.5b,c).
template <typename T>
cudaError_t launch_block_reduced(const BlockMap& m, const double* gh, const T* V, const T* Wt, const double* Rinv,
                                 double* xt, double* xb, cudaStream_t s, Gate gt = Gate());
// z = Pi^T (g - Vhat x^(t) - What x^(b)) block by block (max_rows: the largest block).
template <typename T>
cudaError_t launch_block_correct(const BlockMap& m, int max_rows, const double* gh, const T* spk,
                                 const int64_t* sbase, const double* xt, const double* xb, double* z, cudaStream_t s,
                                 Gate gt = Gate());

// Krylov vector kernels (FP64)
struct Krylov;  // defined in sap_api.cu

}  // namespace sap
