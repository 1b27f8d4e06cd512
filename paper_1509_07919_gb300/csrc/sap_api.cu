// C ABI of libsap (include/sap.h): handle management, the factor pipeline
// and the outer BiCGStab(2) loop (Sec. 2.1.1) around the device kernels.
#include <cuda_runtime.h>
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <atomic>
#include <memory>
#include <new>
#include <vector>
#include "sap_internal.cuh"
#include "sap_sparse.h"
#include "sap_blocks.h"
#include "krylov.cuh"

using namespace sap;

namespace sap {
static std::atomic<long long> g_launches{0};
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace sap

namespace {

#define CK(x)                                    \
  do {                                           \
    cudaError_t e_ = (x);                        \
    if (e_ != cudaSuccess) return SAP_ERR_CUDA;  \
  } while (0)

struct DevMem {
  std::vector<void*> ptrs;
  template <typename T>
  sap_status_t alloc(T** p, size_t n) {
    void* q = nullptr;
    if (n == 0) n = 1;
    if (cudaMalloc(&q, n * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      return SAP_ERR_OOM;
    }
    ptrs.push_back(q);
    *p = static_cast<T*>(q);
    return SAP_OK;
  }
  ~DevMem() {
    for (void* p : ptrs) cudaFree(p);
  }
};

#define TRY(x)                           \
  do {                                   \
    sap_status_t s_ = (x);               \
    if (s_ != SAP_OK) return s_;         \
  } while (0)

// Precision-independent part of the solver.
struct SolverBase {
  virtual ~SolverBase() = default;
  virtual sap_status_t alloc() = 0;
  virtual sap_status_t factor(cudaStream_t s) = 0;
  virtual sap_status_t factor_pre(cudaStream_t s) = 0;       // before the block LU
  virtual sap_status_t factor_post(cudaStream_t s) = 0;      // after the block LU
  virtual void lu_items(std::vector<LuItem>& out) const = 0;  // this system's blocks as LU work items
  virtual sap_status_t build_adjoint(cudaStream_t s) = 0;
  // the same launched on s without waiting; adjoint_singular() reads its outcome later
  virtual sap_status_t build_adjoint_async(cudaStream_t s) = 0;
  virtual sap_status_t adjoint_singular() = 0;
  virtual sap_status_t apply(const double* r, double* z, bool transpose, cudaStream_t s, Gate gt = Gate()) = 0;
  // build what a transposed apply needs (adjoint tips, transposed sweep matrices); synchronises
  virtual sap_status_t prepare_transposed(cudaStream_t s) = 0;
  virtual sap_status_t block_lu(int i, double* host, cudaStream_t s) = 0;
  virtual sap_status_t interface(int i, int which, bool adjoint, double* host, cudaStream_t s) = 0;
  // SAP_ERR_TIMEOUT (and reset) if a device-side wait gave up since the last call
  virtual sap_status_t take_device_error(cudaStream_t s) = 0;
  virtual sap_status_t take_factor_error() = 0;
  virtual bool tc_used() const = 0;
  virtual int* err_flag() = 0;
  // a transposed preconditioner can be built (not for per-block reorderings)
  virtual bool has_transposed() const { return true; }
  // the blocks' own half-bandwidths (handles of sap_factor_blocks), else null
  virtual const std::vector<int>* block_bandwidths() const { return nullptr; }
};

}  // namespace

struct sap_handle {
  Layout L;
  sap_options_t opt{};
  const double* band = nullptr;
  // Krylov operator other than the band (sap_set_operator_csr): the sparse
  // matrix whose dropped band the preconditioner was built from
  sap::CsrOp csr{};
  DevMem mem;
  Dev d{};
  const int64_t* dcbase = nullptr;   // per block offset of the chunk matrices
  double* absmax = nullptr;
  unsigned long long* n_boosted = nullptr;
  int* singular = nullptr;
  int* singular_a = nullptr;   // the same for the adjoint's reduced matrices (built apart, maybe concurrently)
  // Krylov workspace
  double* vec = nullptr;      // 11 N doubles: r0 r1 r2 u0 u1 u2 rt tmp t, b and x of the iteration
  // one outer BiCGStab(2) iteration captured as a CUDA graph, per direction
  // (0 forward, 1 adjoint) and Krylov workspace (+2: the second one);
  // captured on first use, replayed per iteration
  cudaGraphExec_t gexec[4] = {nullptr, nullptr, nullptr, nullptr};
  // the whole iteration loop as one graph: a WHILE node whose body is one
  // round (the iteration and the round counter that sets its condition)
  cudaGraphExec_t wexec[4] = {nullptr, nullptr, nullptr, nullptr};
  bool wfailed[4] = {false, false, false, false};
  long long wlaunches[4] = {0, 0, 0, 0};   // kernels in one round of it
  cudaStream_t ks = nullptr;          // internal stream of the iteration (capturable)
  // background stream of the transposed sweep matrices (see Solver::factor_post)
  cudaStream_t ts = nullptr;
  cudaEvent_t ev_ts = nullptr, ev_td = nullptr;
  // the backward-sweep (U) chunk and transfer matrices are built on fs,
  // concurrently with the forward (L) ones on the factor stream
  cudaStream_t fs = nullptr;
  cudaEvent_t ev_fs0 = nullptr, ev_fs1 = nullptr;
  // SaP-C: the UL factorisation runs on its own stream, concurrently with the LU
  cudaStream_t us = nullptr;
  cudaEvent_t ev_us0 = nullptr, ev_us1 = nullptr;
  cudaEvent_t evu[2] = {nullptr, nullptr};      // T_UL bracket (on us)
  bool ts_pending = false;
  cudaEvent_t evf = nullptr, evj = nullptr;   // fork from / join to the caller's stream
  long long glaunches[4] = {0, 0, 0, 0};   // kernels in each graph
  bool gfailed[4] = {false, false, false, false};  // capture unavailable: launch directly
  // second Krylov workspace (vectors, scalars, flags, readbacks, stream, events)
  // for an adjoint solve that runs concurrently with the forward one
  // (sap_solve_pair); allocated on first use
  struct Ws2 {
    double* vec = nullptr;
    KrylovDev kd{};
    int* flags = nullptr;
    double* host_s = nullptr;
    int* host_f = nullptr;
    cudaStream_t ks = nullptr;
    cudaEvent_t evf = nullptr, evj = nullptr, ev0 = nullptr, ev1 = nullptr;
  } w2;
  KrylovDev kd{};
  double* host_s = nullptr;   // pinned scalar readback
  int* flags = nullptr;       // F_COUNT device control flags of the Krylov iteration
  int* host_f = nullptr;      // pinned flag readback
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaEvent_t evp[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t ev_rd = nullptr;   // SaP-C: between the spike tips and the reduced systems
  cudaEvent_t ev_lu[2] = {nullptr, nullptr};   // around the block LU kernel
  float t_factor_ms = 0.f, t_lu_ms = 0.f, t_ul_ms = 0.f, t_spk_ms = 0.f, t_rdcd_ms = 0.f, t_prep_ms = 0.f;
  double* band_owned = nullptr;  // the band, when the handle was made from host memory (sap_factor_host)
  double* host_stage = nullptr;  // 2 N doubles for sap_solve_host, allocated on first use
  double* host_stage4 = nullptr; // 4 N doubles for sap_solve_pair_host, allocated on first use
  std::unique_ptr<SolverBase> impl;
  ~sap_handle() {
    for (cudaGraphExec_t g : gexec)
      if (g) cudaGraphExecDestroy(g);
    for (cudaGraphExec_t g : wexec)
      if (g) cudaGraphExecDestroy(g);
    if (ks) cudaStreamDestroy(ks);
    if (ts) cudaStreamDestroy(ts);
    if (ev_ts) cudaEventDestroy(ev_ts);
    if (ev_td) cudaEventDestroy(ev_td);
    if (us) cudaStreamDestroy(us);
    if (fs) cudaStreamDestroy(fs);
    if (ev_fs0) cudaEventDestroy(ev_fs0);
    if (ev_fs1) cudaEventDestroy(ev_fs1);
    if (ev_us0) cudaEventDestroy(ev_us0);
    if (ev_us1) cudaEventDestroy(ev_us1);
    for (cudaEvent_t e : evu)
      if (e) cudaEventDestroy(e);
    if (evf) cudaEventDestroy(evf);
    if (evj) cudaEventDestroy(evj);
    if (host_s) cudaFreeHost(host_s);
    if (host_f) cudaFreeHost(host_f);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (w2.host_s) cudaFreeHost(w2.host_s);
    if (w2.host_f) cudaFreeHost(w2.host_f);
    if (w2.ks) cudaStreamDestroy(w2.ks);
    for (cudaEvent_t e : {w2.evf, w2.evj, w2.ev0, w2.ev1})
      if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : evp)
      if (e) cudaEventDestroy(e);
    if (ev_rd) cudaEventDestroy(ev_rd);
    for (cudaEvent_t e : ev_lu)
      if (e) cudaEventDestroy(e);
  }
};

namespace {

// B_i (which 0) or C_{i+1} (which 1) of interface i read from the band, or
// (adjoint) their roles for A^T: B'_i = C_{i+1}^T, C'_{i+1} = B_i^T.
sap_status_t read_coupling(sap_handle* h, int i, int which, bool adjoint, double* host, cudaStream_t s) {
  const int K = h->L.K;
  const int64_t KK = (int64_t)K * K;
  std::vector<double> tmp((size_t)KK, 0.0);
  const int64_t N = h->L.N, sr = h->L.off[i + 1];
  for (int r = 0; r < K; ++r)
    for (int c = 0; c < K; ++c) {
      // forward: B(r,c) = a(s-K+r, s+c); C(r,c) = a(s+r, s-K+c)
      int64_t gi, gj;
      bool isB = (which == 0) != adjoint;
      int rr = adjoint ? c : r, cc = adjoint ? r : c;
      if (isB) { gi = sr - K + rr; gj = sr + cc; } else { gi = sr + rr; gj = sr - K + cc; }
      int64_t cidx = K + gi - gj;
      double v = 0.0;
      if (cidx >= 0 && cidx <= 2 * K)
        CK(cudaMemcpyAsync(&v, h->band + cidx * N + gj, sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      tmp[(size_t)(r * K + c)] = v;
    }
  std::memcpy(host, tmp.data(), (size_t)KK * sizeof(double));
  return SAP_OK;
}

template <typename T>
struct Solver : SolverBase {
  sap_handle* h;
  Factors<T> f;
  double* scratch = nullptr;   // apply scratch: g (N), T tmp (N), ctop/cbot
  double* scratch_t = nullptr; // the same for transposed applies (an adjoint solve may run concurrently)
  T* tails_t = nullptr;        // segment tails of the transposed sweeps
  float* bandf = nullptr;      // FP32 copy of the band (FP32 factorisation only)
  T* wlu = nullptr;            // factor windows in global memory (bands too wide for shared memory)
  T* wul = nullptr;            // the same for the UL factorisation (it runs concurrently with the LU)
  void* wspk = nullptr;        // spike-kernel workspaces in global memory (same)
  void* wspk_a = nullptr;      // the adjoint's (its tips may be built concurrently with the forward ones)
  bool adjoint_ready = false;
  bool adjoint_unchecked = false;  // adjoint tips launched without the singular check
  bool transposed_ready = false;
  explicit Solver(sap_handle* hh) : h(hh) {}

  // elements of one sweep kind's transfer matrices: P x S x KH^2
  size_t trans_elems() const {
    const size_t kh = (size_t)hist_width(h->L.K);
    return (size_t)h->L.P * h->L.S * kh * kh;
  }
  // elements of one sweep kind's history responses: P x (S - 1) x KH x cpsmax 32
  size_t xresp_elems() const {
    const size_t kh = (size_t)hist_width(h->L.K);
    return (size_t)h->L.P * (h->L.S - 1) * kh * (size_t)seg_chunks(h->L.max_nch, h->L.S) * 32;
  }

  sap_status_t alloc() override {
    const Layout& L = h->L;
    const int K = L.K, P = L.P;
    const int64_t KK = (int64_t)K * K;
    const int nI = P > 1 ? P - 1 : 1;
    TRY(h->mem.alloc(&f.F, (size_t)L.f_elems));
    // the padding columns [n_i, ld_i) of every block are read by the sweeps and must be 0
    CK(cudaMemset(f.F, 0, (size_t)L.f_elems * sizeof(T)));
    TRY(h->mem.alloc(&scratch, (size_t)(2 * L.N + 5 * nI * K + 8)));
    if (sizeof(T) == 4) TRY(h->mem.alloc(&bandf, (size_t)L.N * L.W));
    if (lu_window_global(K, sizeof(T) == 8, tc())) {
      TRY(h->mem.alloc(&wlu, (size_t)P * lu_window_elems(K)));
      if (h->opt.variant == SAP_C && P > 1) TRY(h->mem.alloc(&wul, (size_t)(P - 1) * lu_window_elems(K)));
    }
    TRY(h->mem.alloc(&f.err, 2));
    {
      const int e2[2] = {0, spin_limit_value(h->opt.spin_limit)};   // flag, polls per bounded wait
      CK(cudaMemcpy(f.err, e2, sizeof(e2), cudaMemcpyHostToDevice));
    }
    TRY(h->mem.alloc(&f.Mlf, (size_t)L.c_elems));
    TRY(h->mem.alloc(&f.Mub, (size_t)L.c_elems));
    f.cbase = h->dcbase;
    f.S = L.S;
    if (L.S > 1) {
      TRY(h->mem.alloc(&f.Tlf, trans_elems()));
      TRY(h->mem.alloc(&f.Tub, trans_elems()));
      TRY(h->mem.alloc(&f.Xlf, xresp_elems()));
      TRY(h->mem.alloc(&f.Xub, xresp_elems()));
      f.cpsmax = seg_chunks(L.max_nch, L.S);
      TRY(h->mem.alloc(&f.tails, (size_t)P * L.S * hist_width(K)));
    }
    if (h->opt.variant == SAP_C && P > 1) {
      TRY(h->mem.alloc(&f.ULt, (size_t)(nI * KK)));
      TRY(h->mem.alloc(&f.V, (size_t)(nI * KK)));
      TRY(h->mem.alloc(&f.Wt, (size_t)(nI * KK)));
      TRY(h->mem.alloc(&f.R, (size_t)(nI * KK)));
      TRY(h->mem.alloc(&f.R0, (size_t)(nI * KK)));
      TRY(h->mem.alloc(&f.piv, (size_t)(nI * K)));
      const size_t sb = spike_scratch_bytes(K, P, sizeof(T) == 8);
      if (sb) {
        unsigned char* q = nullptr;
        TRY(h->mem.alloc(&q, sb));
        wspk = q;
      }
    }
    return SAP_OK;
  }

  // Factor phases, bracketed by events: T_LU (absmax + LU + sweep matrices,
  // evp[0..1]), T_UL (SaP-C, evu[0..1] on the side stream us, concurrent with
  // the LU), T_SPK (B/C, tips, Rbar, its GEPP and inverse, evp[2..3]).
  // factor_pre and factor_post surround the block LU, so that a batch can run
  // one LU launch over all its systems in between.
  sap_status_t factor_pre(cudaStream_t s) override {
    const Layout& L = h->L;
    // the background build of the previous factorisation reads F: wait for it
    if (h->ts_pending) CK(cudaStreamWaitEvent(s, h->ev_td, 0));
    h->ts_pending = false;
    CK(cudaMemsetAsync(h->singular_a, 0, sizeof(int), s));
    adjoint_ready = false;
    adjoint_unchecked = false;
    transposed_ready = false;
    CK(cudaEventRecord(h->evp[0], s));
    if (sizeof(T) == 4) CK(launch_absmax_cast(h->band, L.N, L.K, h->absmax, bandf, s));
    else CK(launch_absmax(h->band, L.N, L.K, h->absmax, s));
    if (h->opt.variant == SAP_C && L.P > 1) {
      // UL of blocks 1..P-1 on the side stream, overlapping the LU; factor_post joins it
      if (!h->us) {
        CK(cudaStreamCreateWithFlags(&h->us, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&h->ev_us0, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&h->ev_us1, cudaEventDisableTiming));
        CK(cudaEventCreate(&h->evu[0]));
        CK(cudaEventCreate(&h->evu[1]));
      }
      CK(cudaEventRecord(h->ev_us0, s));
      CK(cudaStreamWaitEvent(h->us, h->ev_us0, 0));
      CK(cudaEventRecord(h->evu[0], h->us));
      CK(launch_factor_ul<T>(band_in_T(), L.N, L.K, L.P, h->d, h->absmax, h->opt.boost_eps, f.ULt, h->n_boosted,
                             wul, tc(), f.err, h->us));
      CK(cudaEventRecord(h->evu[1], h->us));
      CK(cudaEventRecord(h->ev_us1, h->us));
    }
    return SAP_OK;
  }
  void lu_items(std::vector<LuItem>& out) const override {
    const Layout& L = h->L;
    for (int i = 0; i < L.P; ++i) {
      LuItem it{};
      it.band = band_in_T();
      it.F = f.F + L.fbase[i];
      it.absmax = h->absmax;
      it.nb = h->n_boosted;
      it.N = L.N;
      it.s = L.off[i];
      it.ld = L.ld[i];
      it.eps = h->opt.boost_eps;
      it.K = L.K;
      it.n = (int)(L.off[i + 1] - L.off[i]);
      out.push_back(it);
    }
  }
  sap_status_t factor_post(cudaStream_t s) override {
    const Layout& L = h->L;
    const int K = L.K, P = L.P;
    // a handle that has run a transposed apply gets its transposed sweep
    // matrices rebuilt in the background from the new factors, overlapping the
    // forward ones and whatever follows on s (typically the forward solve);
    // transposed applies wait for them
    // (SaP-C: also the adjoint's tips and reduced matrices, once the UL is done)
    const bool bg_adj = h->opt.variant == SAP_C && P > 1 && f.Va != nullptr;
    if (f.Mutf || bg_adj) {
      if (!h->ts) {
        CK(cudaStreamCreateWithFlags(&h->ts, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&h->ev_ts, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&h->ev_td, cudaEventDisableTiming));
      }
      CK(cudaEventRecord(h->ev_ts, s));
      CK(cudaStreamWaitEvent(h->ts, h->ev_ts, 0));
      if (f.Mutf) TRY(build_transposed(h->ts));
      if (bg_adj) {
        CK(cudaStreamWaitEvent(h->ts, h->ev_us1, 0));   // the UL started by factor_pre
        TRY(launch_adjoint_tips(h->ts));
        adjoint_ready = true;
        adjoint_unchecked = true;
      }
      CK(cudaEventRecord(h->ev_td, h->ts));
      h->ts_pending = true;
    }
    // forward-sweep matrices on s, backward-sweep ones on fs, joined before s goes on
    if (!h->fs) {
      CK(cudaStreamCreateWithFlags(&h->fs, cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&h->ev_fs0, cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&h->ev_fs1, cudaEventDisableTiming));
    }
    CK(cudaEventRecord(h->ev_fs0, s));
    CK(cudaStreamWaitEvent(h->fs, h->ev_fs0, 0));
    CK(launch_chunk_mats<T>(f.F, K, P, h->d, f.cbase, L.max_nch, 1, f.Mub, h->fs));
    CK(launch_seg_trans<T>(f.Mub, f.cbase, K, P, L.S, f.cpsmax, h->d, f.Tub, f.Xub, h->fs));
    CK(cudaEventRecord(h->ev_fs1, h->fs));
    CK(launch_chunk_mats<T>(f.F, K, P, h->d, f.cbase, L.max_nch, 0, f.Mlf, s));
    CK(launch_seg_trans<T>(f.Mlf, f.cbase, K, P, L.S, f.cpsmax, h->d, f.Tlf, f.Xlf, s));
    CK(cudaStreamWaitEvent(s, h->ev_fs1, 0));
    CK(cudaEventRecord(h->evp[1], s));
    if (h->opt.variant == SAP_C && P > 1) {
      CK(cudaStreamWaitEvent(s, h->ev_us1, 0));      // the UL started by factor_pre
      CK(cudaEventRecord(h->evp[2], s));
      CK(launch_spikes<T>(h->band, L.N, K, P, h->d, f.F, f.ULt, false, f.V, f.Wt, f.R, f.R0, f.piv,
                          h->singular, wspk, s, h->ev_rd));
    } else {
      CK(cudaEventRecord(h->evp[2], s));
      CK(cudaEventRecord(h->ev_rd, s));
    }
    CK(cudaEventRecord(h->evp[3], s));
    return SAP_OK;
  }
  sap_status_t factor(cudaStream_t s) override {
    const Layout& L = h->L;
    TRY(factor_pre(s));
    CK(cudaEventRecord(h->ev_lu[0], s));
    CK(launch_factor_lu<T>(band_in_T(), L.N, L.K, L.P, h->d, h->absmax, h->opt.boost_eps, f.F, h->n_boosted,
                           wlu, tc(), f.err, s));
    CK(cudaEventRecord(h->ev_lu[1], s));
    return factor_post(s);
  }

  sap_status_t build_adjoint_async(cudaStream_t s) override {
    if (adjoint_ready || h->opt.variant != SAP_C || h->L.P < 2) return SAP_OK;
    TRY(launch_adjoint_tips(s));
    adjoint_ready = true;       // ordered before the adjoint iteration on s
    adjoint_unchecked = true;
    return SAP_OK;
  }
  sap_status_t adjoint_singular() override {
    if (!adjoint_unchecked) return SAP_OK;
    adjoint_unchecked = false;
    if (h->ts_pending) CK(cudaEventSynchronize(h->ev_td));   // tips built in the background
    int sing = 0;
    CK(cudaMemcpy(&sing, h->singular_a, sizeof(int), cudaMemcpyDeviceToHost));
    if (!sing) return SAP_OK;
    CK(cudaMemset(h->singular_a, 0, sizeof(int)));
    adjoint_ready = false;
    return SAP_ERR_SINGULAR;
  }
  sap_status_t launch_adjoint_tips(cudaStream_t s) {
    const int K = h->L.K, nI = h->L.P - 1;
    const int64_t KK = (int64_t)K * K;
    if (!f.Va) {
      TRY(h->mem.alloc(&f.Va, (size_t)(nI * KK)));
      TRY(h->mem.alloc(&f.Wa, (size_t)(nI * KK)));
      TRY(h->mem.alloc(&f.Ra, (size_t)(nI * KK)));
      TRY(h->mem.alloc(&f.Ra0, (size_t)(nI * KK)));
      TRY(h->mem.alloc(&f.piva, (size_t)(nI * K)));
    }
    const size_t sb = spike_scratch_bytes(K, h->L.P, sizeof(T) == 8);
    if (sb && !wspk_a) {
      unsigned char* q = nullptr;
      TRY(h->mem.alloc(&q, sb));
      wspk_a = q;
    }
    CK(launch_spikes<T>(h->band, h->L.N, K, h->L.P, h->d, f.F, f.ULt, true, f.Va, f.Wa, f.Ra, f.Ra0, f.piva,
                        h->singular_a, wspk_a, s));
    return SAP_OK;
  }
  sap_status_t build_adjoint(cudaStream_t s) override {
    if (adjoint_ready && !adjoint_unchecked) return SAP_OK;
    if (adjoint_ready) return adjoint_singular();     // built in the background: its outcome
    if (h->opt.variant != SAP_C || h->L.P < 2) return SAP_OK;
    TRY(launch_adjoint_tips(s));
    int sing = 0;
    CK(cudaMemcpyAsync(&sing, h->singular_a, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (sing) {
      CK(cudaMemset(h->singular_a, 0, sizeof(int)));
      return SAP_ERR_SINGULAR;
    }
    adjoint_ready = true;
    return SAP_OK;
  }

  // the tensor-core trailing update of the FP32 factorisation (SAP_FP32_BF16TU, K >= kTcMinK)
  // (only where the window stays in shared memory with the operand buffers: measured slower otherwise)
  bool tc() const {
    return sizeof(T) == 4 && h->opt.precision == SAP_FP32_BF16TU && h->L.K >= kTcMinK &&
           !lu_window_global(h->L.K, false, true);
  }
  bool tc_used() const override { return tc(); }
  // a bounded wait of the factor kernels gave up (their error flag, then reset)
  sap_status_t take_factor_error() override {
    int e = 0;
    CK(cudaMemcpy(&e, f.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (!e) return SAP_OK;
    CK(cudaMemset(f.err, 0, sizeof(int)));
    return SAP_ERR_TIMEOUT;
  }
  int* err_flag() override { return f.err; }

  // the band in the factor precision: the borrowed FP64 band, or its FP32 copy
  const T* band_in_T() const {
    if (sizeof(T) == 8) return reinterpret_cast<const T*>(h->band);
    return reinterpret_cast<const T*>(bandf);
  }

  // chunk matrices of the transposed sweeps (U^T forward, L^T backward)
  sap_status_t build_transposed(cudaStream_t s) {
    if (transposed_ready) return SAP_OK;
    const Layout& L = h->L;
    if (!f.Mutf) {
      TRY(h->mem.alloc(&f.Mutf, (size_t)L.c_elems));
      TRY(h->mem.alloc(&f.Mltb, (size_t)L.c_elems));
      const int nI = L.P > 1 ? L.P - 1 : 1;
      TRY(h->mem.alloc(&scratch_t, (size_t)(2 * L.N + 5 * nI * L.K + 8)));
      if (L.S > 1) TRY(h->mem.alloc(&tails_t, (size_t)L.P * L.S * hist_width(L.K)));
      if (L.S > 1) {
        TRY(h->mem.alloc(&f.Tutf, trans_elems()));
        TRY(h->mem.alloc(&f.Tltb, trans_elems()));
        TRY(h->mem.alloc(&f.Xutf, xresp_elems()));
        TRY(h->mem.alloc(&f.Xltb, xresp_elems()));
      }
    }
    CK(launch_chunk_mats<T>(f.F, L.K, L.P, h->d, f.cbase, L.max_nch, 2, f.Mutf, s));
    CK(launch_chunk_mats<T>(f.F, L.K, L.P, h->d, f.cbase, L.max_nch, 3, f.Mltb, s));
    CK(launch_seg_trans<T>(f.Mutf, f.cbase, L.K, L.P, L.S, f.cpsmax, h->d, f.Tutf, f.Xutf, s));
    CK(launch_seg_trans<T>(f.Mltb, f.cbase, L.K, L.P, L.S, f.cpsmax, h->d, f.Tltb, f.Xltb, s));
    transposed_ready = true;
    return SAP_OK;
  }

  sap_status_t prepare_transposed(cudaStream_t s) override {
    if (h->ts_pending) CK(cudaStreamWaitEvent(s, h->ev_td, 0));   // built in the background after the LU
    TRY(build_adjoint(s));
    return build_transposed(s);
  }

  sap_status_t apply(const double* r, double* z, bool transpose, cudaStream_t s, Gate gt) override {
    if (!transpose) {
      CK(launch_apply<T>(h->band, h->L.N, h->L.K, h->L.P, h->d, f, h->opt.variant, false, r, z, scratch, s, gt));
      return SAP_OK;
    }
    // inside a stream capture (a Krylov run's captured iteration) the run's
    // begin() has prepared the transposed data on the caller's stream: no wait
    // on the background build's event may enter the graph
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs == cudaStreamCaptureStatusNone)
      TRY(prepare_transposed(s));
    Factors<T> ft = f;              // transposed applies own their scratch and segment tails
    ft.tails = tails_t;
    CK(launch_apply<T>(h->band, h->L.N, h->L.K, h->L.P, h->d, ft, h->opt.variant, true, r, z, scratch_t, s, gt));
    return SAP_OK;
  }

  sap_status_t take_device_error(cudaStream_t s) override {
    int e = 0;
    CK(cudaMemcpyAsync(&e, f.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (!e) return SAP_OK;
    CK(cudaMemsetAsync(f.err, 0, sizeof(int), s));
    return SAP_ERR_TIMEOUT;
  }

  sap_status_t block_lu(int i, double* host, cudaStream_t s) override {
    const Layout& L = h->L;
    const int64_t n = L.off[i + 1] - L.off[i], ld = L.ld[i];
    const int W = L.W, K = L.K;
    std::vector<T> buf((size_t)(W * ld));
    CK(cudaMemcpyAsync(buf.data(), f.F + L.fbase[i], buf.size() * sizeof(T), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    // device layout F[c ld + q] = (r, q), c = K + r - q  ->  host f[r W + (q - r + K)]
    for (int64_t r = 0; r < n; ++r)
      for (int dq = -K; dq <= K; ++dq) {
        int64_t q = r + dq;
        double v = 0.0;
        if (q >= 0 && q < n) v = (double)buf[(size_t)((K + r - q) * ld + q)];
        host[r * W + (dq + K)] = v;
      }
    return SAP_OK;
  }

  sap_status_t interface(int i, int which, bool adjoint, double* host, cudaStream_t s) override {
    const int K = h->L.K;
    const int64_t KK = (int64_t)K * K;
    if (h->opt.variant != SAP_C || h->L.P < 2 || i < 0 || i >= h->L.P - 1 || which < 0 || which > 4)
      return SAP_ERR_INVALID_ARG;
    if (adjoint) TRY(build_adjoint(s));
    if (which <= 1) return read_coupling(h, i, which, adjoint, host, s);
    if (which == 4) {
      const double* src = (adjoint ? f.Ra0 : f.R0) + i * KK;
      CK(cudaMemcpyAsync(host, src, (size_t)KK * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      return SAP_OK;
    }
    const T* src = (which == 2 ? (adjoint ? f.Va : f.V) : (adjoint ? f.Wa : f.Wt)) + i * KK;
    std::vector<T> buf((size_t)KK);
    CK(cudaMemcpyAsync(buf.data(), src, (size_t)KK * sizeof(T), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int64_t e = 0; e < KK; ++e) host[e] = (double)buf[(size_t)e];
    return SAP_OK;
  }
};

constexpr int kSMs = 152;               // SMs of a GB300
constexpr int kMaxAutoSegments = 64;

sap_status_t check_options(const sap_options_t* o, int64_t N, int K) {
  if (!o) return SAP_ERR_INVALID_ARG;
  if (N < 2 || K < 1 || K >= N) return SAP_ERR_INVALID_ARG;
  if (o->P < 1 || o->P > N) return SAP_ERR_INVALID_ARG;
  if (o->variant != SAP_D && o->variant != SAP_C) return SAP_ERR_INVALID_ARG;
  if (o->precision != SAP_FP64 && o->precision != SAP_FP32 && o->precision != SAP_FP32_BF16TU)
    return SAP_ERR_INVALID_ARG;
  if (o->segments < 0) return SAP_ERR_INVALID_ARG;
  if (o->krylov != SAP_KRYLOV_BICGSTAB2 && o->krylov != SAP_KRYLOV_CG) return SAP_ERR_INVALID_ARG;
  return SAP_OK;
}

// The handle's internal stream and its fork/join events, created on first use.
sap_status_t ensure_stream(sap_handle* h) {
  if (h->ks) return SAP_OK;
  CK(cudaStreamCreateWithFlags(&h->ks, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&h->evf, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&h->evj, cudaEventDisableTiming));
  return SAP_OK;
}

// The second Krylov workspace, created on first use.
sap_status_t ensure_ws2(sap_handle* h) {
  auto& w = h->w2;
  if (w.ks) return SAP_OK;
  const int64_t N = h->L.N;
  TRY(h->mem.alloc(&w.vec, (size_t)(11 * N)));
  TRY(h->mem.alloc(&w.kd.S, S_COUNT));
  TRY(h->mem.alloc(&w.kd.part, kKrylovBlocks * 4));
  TRY(h->mem.alloc(&w.kd.ticket, 1));
  TRY(h->mem.alloc(&w.flags, F_COUNT));
  CK(cudaMemset(w.kd.ticket, 0, sizeof(unsigned)));
  CK(cudaMemset(w.vec, 0, 11 * N * sizeof(double)));
  if (cudaMallocHost(&w.host_s, S_COUNT * sizeof(double)) != cudaSuccess) return SAP_ERR_OOM;
  if (cudaMallocHost(&w.host_f, F_COUNT * sizeof(int)) != cudaSuccess) return SAP_ERR_OOM;
  CK(cudaEventCreateWithFlags(&w.evf, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&w.evj, cudaEventDisableTiming));
  CK(cudaEventCreate(&w.ev0));
  CK(cudaEventCreate(&w.ev1));
  CK(cudaStreamCreateWithFlags(&w.ks, cudaStreamNonBlocking));
  return SAP_OK;
}

// One Krylov solve (BiCGStab(2), or preconditioned CG when the handle's
// krylov option asks for it), split at its host synchronisation points so
// that a batch of solves can share them: begin() (setup, scalar readback),
// then rounds (one outer BiCGStab(2) iteration, or kCgSteps CG steps, each;
// flag readback), then finish().  Between
// two steps the caller synchronises the handle's stream.  All work runs on
// the handle's internal stream (stream capture needs a non-legacy stream),
// ordered after the caller's stream at begin() and before it at the end of
// finish().
constexpr int kCgSteps = 4;   // CG steps per captured round

struct KrylovRun {
  sap_handle* h = nullptr;
  bool tr = false;
  bool cg = false;       // preconditioned CG instead of BiCGStab(2)
  cudaStream_t user = nullptr, s = nullptr;
  const double* b_user = nullptr;
  double* x_user = nullptr;
  int64_t N = 0;
  double *r[3], *u[3], *rt, *tmp, *t, *b, *x;
  KrylovDev kd, ka, kc;
  // the workspace of this run: the handle's own (ws 0) or its second one (ws 1)
  double* vec = nullptr;
  int* flags = nullptr;
  double* hs = nullptr;
  int* hf = nullptr;
  cudaEvent_t evf = nullptr, evj = nullptr, ev0 = nullptr, ev1 = nullptr;
  Gate gA, gC, gR;
  KrylovDev kr, kk;      // gated on the restart flag / on its absence (CG)
  double tol = 0.0, bn = 0.0;
  sap_info_t inf{};
  sap_status_t status = SAP_ERR_NOT_CONVERGED;
  bool done = false;     // converged or broken down (or b = 0)
  int it = 0;            // outer iterations launched
  int gi = 0;

  // the iteration's operator: the band, or the sparse operator set on the handle
  cudaError_t spmv(const double* xin, double* yout, Gate g = Gate()) {
    if (h->csr.rowptr) return launch_spmv_pcsr(h->csr, xin, yout, s, g);
    return launch_spmv(h->band, N, h->L.K, xin, yout, tr, s, g);
  }

  sap_status_t init(sap_handle* hh, const double* bu, double* xu, bool transposed, cudaStream_t us, int ws = 0) {
    h = hh; tr = transposed; user = us; b_user = bu; x_user = xu;
    if (tr && h->csr.rowptr) return SAP_ERR_NOT_IMPLEMENTED;    // no transposed sparse operator
    if (tr && !h->impl->has_transposed()) return SAP_ERR_NOT_IMPLEMENTED;
    cg = h->opt.krylov == SAP_KRYLOV_CG;
    TRY(ensure_stream(h));
    N = h->L.N;
    if (ws == 0) {
      s = h->ks; vec = h->vec; kd = h->kd; flags = h->flags; hs = h->host_s; hf = h->host_f;
      evf = h->evf; evj = h->evj; ev0 = h->ev0; ev1 = h->ev1;
    } else {
      TRY(ensure_ws2(h));
      s = h->w2.ks; vec = h->w2.vec; kd = h->w2.kd; flags = h->w2.flags; hs = h->w2.host_s; hf = h->w2.host_f;
      evf = h->w2.evf; evj = h->w2.evj; ev0 = h->w2.ev0; ev1 = h->w2.ev1;
    }
    for (int k = 0; k < 3; ++k) {
      r[k] = vec + k * N;
      u[k] = vec + (3 + k) * N;
    }
    rt = vec + 6 * N;
    tmp = vec + 7 * N;
    t = vec + 8 * N;
    // the iteration works on handle-owned copies of b and x, so that its
    // captured graph does not depend on the caller's pointers
    b = vec + 9 * N;
    x = vec + 10 * N;
    kd.flags = flags;
    ka = kd;
    ka.gmode = G_ACTIVE;
    kc = kd;
    kc.gmode = G_CHECK;
    kr = kd;
    kr.gmode = G_REPLACE;
    kk = kd;
    kk.gmode = G_KEEP;
    gA.flags = gC.flags = gR.flags = flags;
    gA.mode = G_ACTIVE;
    gC.mode = G_CHECK;
    gR.mode = G_REPLACE;
    tol = h->opt.tol;
    inf.iters = 0;
    inf.relres = 1.0;
    gi = (tr ? 1 : 0) + 2 * ws;
    return SAP_OK;
  }

  // setup launches and the readback of ||b||^2, ||M^{-1} b||^2
  sap_status_t begin() {
    if (tr) TRY(h->impl->prepare_transposed(user));
    CK(cudaEventRecord(evf, user));
    CK(cudaStreamWaitEvent(s, evf, 0));
    CK(cudaEventRecord(ev0, s));
    CK(cudaMemcpyAsync(b, b_user, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(x, 0, N * sizeof(double), s));
    CK(cudaMemsetAsync(flags, 0, F_COUNT * sizeof(int), s));
    CK(kr_init(kd, s));
    CK(kr_norm2(b, N, kd, S_BN2, s));
    if (cg) {
      // r = b - A x0 = b, z = M^{-1} r, p = z, (r, z)  (vectors: r = r0, z = r1, p = u0, q = u1)
      CK(cudaMemcpyAsync(r[0], b, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
      TRY(h->impl->apply(r[0], r[1], tr, s));
      CK(kr_cg_start(r[0], r[1], u[0], N, kd, s));
      CK(cudaMemcpyAsync(hs, kd.S + S_RN2, 5 * sizeof(double), cudaMemcpyDeviceToHost, s));
      return SAP_OK;
    }
    TRY(h->impl->apply(b, r[0], tr, s));
    CK(kr_norm2(r[0], N, kd, S_BTN2, s));
    CK(cudaMemcpyAsync(rt, r[0], N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(u[0], 0, N * sizeof(double), s));
    CK(cudaMemcpyAsync(hs, kd.S + S_RN2, 5 * sizeof(double), cudaMemcpyDeviceToHost, s));
    return SAP_OK;
  }
  // after the stream synchronised: b = 0 finishes at once
  void after_begin() {
    bn = std::sqrt(hs[S_BN2 - S_RN2]);
    if (bn == 0.0) {
      inf.relres = 0.0;
      status = SAP_OK;
      done = true;
    }
  }

  // exit test; after the MR update (qoff = 1) a failed confirmation restarts
  // the method from x: r^0 = M^{-1}(b - A x), r~0 = r^0, u^0 = 0, scalars reset
  sap_status_t exit_test(double qoff) {
    CK(kr_exit_check(kd, tol, qoff, s));
    CK(spmv(x, tmp, gC));
    CK(kr_residual(b, tmp, t, N, kc, S_TN2, s));
    CK(kr_exit_decide(kd, tol, qoff, s));
    if (qoff != 1.0) return SAP_OK;
    TRY(h->impl->apply(t, r[0], tr, s, gR));
    KrylovDev kr = kd;
    kr.gmode = G_REPLACE;
    CK(kr_restart(r[0], rt, u[0], N, kr, s));
    return SAP_OK;
  }
  // one CG step (Saad, Alg. 9.1) with its exit test and, gated, the restart
  sap_status_t cg_step() {
    double *rr = r[0], *z = r[1], *p = u[0], *q = u[1];
    CK(spmv(p, q, gA));                                             // q = A p
    CK(kr_cg_alpha(p, q, N, ka, s));
    CK(kr_cg_xr(x, rr, p, q, N, ka, s));
    CK(kr_cg_check(kd, tol, s));
    CK(spmv(x, tmp, gC));                                           // true residual, if flagged
    CK(kr_residual(b, tmp, t, N, kc, S_TN2, s));
    CK(kr_cg_decide(kd, tol, h->opt.max_iters, s));
    CK(kr_copy(t, rr, N, kr, s));                                   // restart: r = b - A x
    TRY(h->impl->apply(rr, z, tr, s, gA));                          // z = M^{-1} r
    CK(kr_cg_start(rr, z, p, N, kr, s));                            // restart: p = z
    CK(kr_cg_beta(rr, z, N, kk, s));
    CK(kr_cg_p(z, p, N, kk, s));
    return SAP_OK;
  }
  sap_status_t iteration() {
    if (cg) {
      for (int k = 0; k < kCgSteps; ++k) TRY(cg_step());
      return SAP_OK;
    }
    for (int j = 0; j < 2; ++j) {
      CK(kr_bicg_rho(r[j], rt, N, ka, j, s));
      CK(kr_bicg_u(u[0], u[1], r[0], r[1], N, ka, j, s));
      CK(spmv(u[j], tmp, gA));
      TRY(h->impl->apply(tmp, u[j + 1], tr, s, gA));
      CK(kr_bicg_gamma(u[j + 1], rt, N, ka, s));
      CK(kr_bicg_r(r[0], r[1], u[0], u[1], u[2], x, N, ka, j, s));
      TRY(exit_test(j == 0 ? 0.25 : 0.75));
      CK(spmv(r[j], tmp, gA));
      TRY(h->impl->apply(tmp, r[j + 1], tr, s, gA));
    }
    CK(kr_mr(x, r[0], r[1], r[2], u[0], u[1], u[2], N, ka, s));
    return exit_test(1.0);
  }
  // capture the iteration once per handle and direction; on any capture
  // failure the iteration is launched directly instead
  void capture() {
    if (h->gexec[gi] || h->gfailed[gi]) return;
    const long long l0 = launches_so_far();
    cudaGraph_t graph = nullptr;
    bool ok = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    const sap_status_t cst = ok ? iteration() : SAP_ERR_CUDA;
    if (ok) ok = cudaStreamEndCapture(s, &graph) == cudaSuccess && cst == SAP_OK;
    if (ok) ok = cudaGraphInstantiate(&h->gexec[gi], graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
      if (h->gexec[gi]) cudaGraphExecDestroy(h->gexec[gi]);
      h->gexec[gi] = nullptr;
      h->gfailed[gi] = true;
      cudaGetLastError();
    }
    h->glaunches[gi] = launches_so_far() - l0;
    count_launches(-(int)h->glaunches[gi]);     // captured, not run
  }
  // CG: the device finishes the solve at the iteration cap (a round may end early)
  int step() const { return cg ? kCgSteps : 1; }
  int cap() const { return h->opt.max_iters + (cg ? kCgSteps : 0); }
  bool active() const { return !done && it < cap(); }
  // The whole loop as one graph launch: a conditional WHILE node whose body is
  // one round, ended by kr_while_next, which counts the rounds in
  // flags[F_ROUNDS] and keeps the node going while the solve is not done and
  // the count is below the cap; built once per handle and direction.  Returns
  // false where conditional graphs are unavailable (the host loop then runs).
  bool device_loop = false;
  void build_while() {
    const long long l0 = launches_so_far();
    cudaGraph_t parent = nullptr, round_g = nullptr;
    cudaGraphConditionalHandle hnd = 0;
    cudaGraphNode_t node = nullptr, child = nullptr;
    bool ok = cudaGraphCreate(&parent, 0) == cudaSuccess;
    ok = ok && cudaGraphConditionalHandleCreate(&hnd, parent, 1, cudaGraphCondAssignDefault) == cudaSuccess;
    // one round captured on its own first; a conditional body takes it only
    // if it holds kernel, memset, memcpy, empty and child-graph nodes alone
    if (ok) {
      ok = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      sap_status_t cst = ok ? iteration() : SAP_ERR_CUDA;
      if (ok && cst == SAP_OK && kr_while_next(hnd, flags, step(), cap(), s) != cudaSuccess) cst = SAP_ERR_CUDA;
      if (ok) ok = cudaStreamEndCapture(s, &round_g) == cudaSuccess && cst == SAP_OK && round_g;
    }
    if (ok) {
      size_t nn = 0;
      ok = cudaGraphGetNodes(round_g, nullptr, &nn) == cudaSuccess;
      std::vector<cudaGraphNode_t> nodes(nn);
      if (ok && nn) ok = cudaGraphGetNodes(round_g, nodes.data(), &nn) == cudaSuccess;
      for (size_t q = 0; ok && q < nn; ++q) {
        cudaGraphNodeType ty;
        ok = cudaGraphNodeGetType(nodes[q], &ty) == cudaSuccess &&
             (ty == cudaGraphNodeTypeKernel || ty == cudaGraphNodeTypeMemset || ty == cudaGraphNodeTypeMemcpy ||
              ty == cudaGraphNodeTypeEmpty || ty == cudaGraphNodeTypeGraph);
      }
    }
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = hnd;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    ok = ok && cudaGraphAddNode(&node, parent, nullptr, nullptr, 0, &p) == cudaSuccess;
    ok = ok && cudaGraphAddChildGraphNode(&child, p.conditional.phGraph_out[0], nullptr, 0, round_g) == cudaSuccess;
    ok = ok && cudaGraphInstantiate(&h->wexec[gi], parent, 0) == cudaSuccess;
    if (round_g) cudaGraphDestroy(round_g);
    if (parent) cudaGraphDestroy(parent);
    if (!ok) {
      if (h->wexec[gi]) cudaGraphExecDestroy(h->wexec[gi]);
      h->wexec[gi] = nullptr;
      h->wfailed[gi] = true;
      cudaGetLastError();
    }
    h->wlaunches[gi] = launches_so_far() - l0;
    count_launches(-(int)h->wlaunches[gi]);     // captured, not run
  }
  bool launch_device_loop() {
    if (!h->wexec[gi] && !h->wfailed[gi]) build_while();
    if (!h->wexec[gi]) return false;
    if (cudaGraphLaunch(h->wexec[gi], s) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    device_loop = true;
    return true;
  }
  // one outer iteration and the readback of the control flags
  sap_status_t round() {
    capture();
    if (h->gexec[gi]) {
      CK(cudaGraphLaunch(h->gexec[gi], s));
      count_launches((int)h->glaunches[gi]);
    } else {
      TRY(iteration());
    }
    it += cg ? kCgSteps : 1;
    CK(cudaMemcpyAsync(hf, flags, F_COUNT * sizeof(int), cudaMemcpyDeviceToHost, s));
    return SAP_OK;
  }
  void after_round() { done = hf[F_DONE] != 0; }

  // results; synchronises the handle's stream and joins the caller's
  sap_status_t finish(sap_info_t* info) {
    if (bn != 0.0) {
      CK(cudaMemcpyAsync(hs, kd.S, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(hf, flags, F_COUNT * sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      inf.n_restarts = hf[F_RESTARTS];
      if (device_loop) count_launches((int)((hf[F_ROUNDS] / step()) * h->wlaunches[gi]));
      if (hf[F_DONE]) {
        status = (sap_status_t)hf[F_STATUS];
        inf.iters = hs[S_QUART];
        inf.relres = hs[S_RELRES];
      } else {
        status = SAP_ERR_NOT_CONVERGED;
        inf.iters = h->opt.max_iters;
      }
      if (status != SAP_OK) {
        CK(spmv(x, tmp));
        CK(kr_residual(b, tmp, t, N, kd, S_TN2, s));
        CK(cudaMemcpyAsync(hs, kd.S + S_RN2, 5 * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        inf.relres = std::sqrt(hs[S_TN2 - S_RN2]) / bn;
      }
    }
    CK(cudaMemcpyAsync(x_user, x, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaEventRecord(ev1, s));
    CK(cudaEventSynchronize(ev1));
    if (h->impl->take_device_error(s) != SAP_OK) status = SAP_ERR_TIMEOUT;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    inf.n_matvec = (int64_t)std::llround((cg ? 1.0 : 4.0) * inf.iters);
    inf.t_solve_ms = ms;
    inf.t_kry_ms = ms;
    inf.t_factor_ms = h->t_factor_ms;
    inf.t_lu_ms = h->t_lu_ms;
    inf.t_prep_ms = h->t_prep_ms;
    inf.t_ul_ms = h->t_ul_ms;
    inf.t_bc_ms = 0.f;            // B_i, C_{i+1} are read in place by the tip kernels
    inf.t_spk_ms = h->t_spk_ms;
    inf.t_rdcd_ms = h->t_rdcd_ms;
    inf.P = h->L.P;
    inf.segments = h->L.S;
    inf.graphed = (h->gexec[gi] != nullptr || device_loop) ? 1 : 0;
    inf.tc_update = h->impl->tc_used() ? 1 : 0;
    unsigned long long nb = 0;
    CK(cudaMemcpy(&nb, h->n_boosted, sizeof(nb), cudaMemcpyDeviceToHost));
    inf.n_boosted = (int64_t)nb;
    CK(cudaEventRecord(evj, s));
    CK(cudaStreamWaitEvent(user, evj, 0));
    if (info) *info = inf;
    return status;
  }
};

// BiCGStab(2) (Sleijpen & Fokkema 1993, l = 2) on M^{-1} A x = M^{-1} b, or
// on the transposed system.  The iteration runs device-driven: every launch
// carries a Gate on the solve's control flags, the exit tests after the first
// and third matvec and after the MR step are device kernels (a true-residual
// check is flagged when ||r^0|| <= tol ||M^{-1} b||; if the true residual
// then fails, the residual replacement r^0 = M^{-1}(b - A x) is flagged), and
// the host reads the flags once per outer iteration, which runs as one
// captured CUDA graph.  Launches after the accepted exit do nothing.
sap_status_t krylov(sap_handle* h, const double* b_user, double* x_user, bool tr, sap_info_t* info,
                    cudaStream_t s) {
  KrylovRun k;
  TRY(k.init(h, b_user, x_user, tr, s));
  TRY(k.begin());
  CK(cudaStreamSynchronize(k.s));
  k.after_begin();
  if (k.active() && k.launch_device_loop()) return k.finish(info);
  while (k.active()) {
    TRY(k.round());
    CK(cudaStreamSynchronize(k.s));
    k.after_round();
  }
  return k.finish(info);
}

// Factorisation in two steps (a batch launches all systems before waiting):
// launch_factor queues the factor phases on s, finish_factor waits for them,
// reads the phase times and the singular flag.
sap_status_t launch_factor(sap_handle* h, cudaStream_t s) {
  CK(cudaMemsetAsync(h->n_boosted, 0, sizeof(unsigned long long), s));
  CK(cudaMemsetAsync(h->singular, 0, sizeof(int), s));
  return h->impl->factor(s);
}

sap_status_t finish_factor(sap_handle* h) {
  CK(cudaEventSynchronize(h->evp[3]));
  CK(cudaGetLastError());
  float t_lu_phase = 0.f;
  cudaEventElapsedTime(&t_lu_phase, h->evp[0], h->evp[1]);
  cudaEventElapsedTime(&h->t_lu_ms, h->ev_lu[0], h->ev_lu[1]);
  h->t_prep_ms = std::max(0.f, t_lu_phase - h->t_lu_ms);
  h->t_ul_ms = 0.f;
  if (h->opt.variant == SAP_C && h->L.P > 1) cudaEventElapsedTime(&h->t_ul_ms, h->evu[0], h->evu[1]);
  cudaEventElapsedTime(&h->t_spk_ms, h->evp[2], h->ev_rd);
  cudaEventElapsedTime(&h->t_rdcd_ms, h->ev_rd, h->evp[3]);
  cudaEventElapsedTime(&h->t_factor_ms, h->evp[0], h->evp[3]);
  int sing = 0;
  CK(cudaMemcpy(&sing, h->singular, sizeof(int), cudaMemcpyDeviceToHost));
  if (sing) return SAP_ERR_SINGULAR;
  return h->impl->take_factor_error();
}

sap_status_t run_factor(sap_handle* h, cudaStream_t s) {
  TRY(launch_factor(h, s));
  return finish_factor(h);
}

// The solver of a handle whose blocks are reordered on their own (defined below).
SolverBase* new_blocks_solver(sap_handle* h, const int32_t* perm_dev, cudaStream_t s);

// A handle with its layout and device memory, not yet factored.  With
// blockperm (sap_factor_blocks) its solver factors every block after its own
// permutation, at its own half-bandwidth (K may then exceed sap_max_K).
sap_status_t create_handle(const double* band_dev, int64_t N, int32_t K, const sap_options_t* opt_in,
                           cudaStream_t s, std::unique_ptr<sap_handle>& out, const int32_t* blockperm = nullptr) {
  if (!band_dev) return SAP_ERR_INVALID_ARG;
  TRY(check_options(opt_in, N, K));
  sap_options_t opt = *opt_in;
  if (opt.max_iters <= 0) opt.max_iters = 500;
  if (!(opt.tol > 0.0)) opt.tol = 1e-10;
  if (!(opt.boost_eps > 0.0)) opt.boost_eps = opt.precision == SAP_FP64 ? 0x1p-53 : 0x1p-24;
  if (!blockperm && K > sap_max_K(opt.precision)) return SAP_ERR_NOT_IMPLEMENTED;
  out.reset(new (std::nothrow) sap_handle());
  if (!out) return SAP_ERR_OOM;
  sap_handle* h = out.get();
  h->opt = opt;
  h->band = band_dev;
  Layout& L = h->L;
  L.N = N; L.K = K; L.P = opt.P; L.W = 2 * K + 1;
  L.off.resize(L.P + 1);
  {
    int64_t q = N / L.P, pr = N - (int64_t)L.P * q;
    L.off[0] = 0;
    for (int i = 0; i < L.P; ++i) L.off[i + 1] = L.off[i] + q + (i < pr ? 1 : 0);
  }
  L.fbase.resize(L.P);
  L.ld.resize(L.P);
  int64_t acc = 0;
  for (int i = 0; i < L.P; ++i) {
    int64_t n = L.off[i + 1] - L.off[i];
    if (n < 1) return SAP_ERR_INVALID_ARG;
    if (opt.variant == SAP_C && L.P > 1 && n < 2 * (int64_t)K) return SAP_ERR_INVALID_ARG;
    L.ld[i] = (n + 31) / 32 * 32;
    L.fbase[i] = acc;
    acc += L.ld[i] * L.W;
  }
  L.f_elems = acc;
  std::vector<int64_t> cb(L.P);
  int64_t cacc = 0;
  L.max_nch = 0;
  for (int i = 0; i < L.P; ++i) {
    cb[i] = cacc;
    const int nch = (int)(L.ld[i] / 32);
    cacc += (int64_t)nch * (1 + chunk_couplings(K)) * 32 * 32;
    if (nch > L.max_nch) L.max_nch = nch;
  }
  L.c_elems = cacc;
  {
    // sweep segments.  Automatic count (measured on GB300): FP32 factors:
    // up to two CTAs per SM over all blocks, segments of at least 16 chunks,
    // used only if that gives at least 4 segments per block.  FP64 factors:
    // the transfer matrices cost more to form (FP64 arithmetic is slow on
    // this part): one CTA per SM, segments of at least 32 chunks, at least 6
    // per block.  Never more than kMaxAutoSegments.  Any count is lowered to
    // keep max(ng, 2) chunks of 32 rows in every full segment; segmentation
    // needs the segmented sweep's ring of chunk matrices in shared memory
    // (FP32 up to K = 512, FP64 up to K = 256).
    // The automatic count stays at one segment above 4 couplings per chunk:
    // there the serial chain of KH x KH transfer matrices (254 KB each at
    // K = 250) and the correction's stream of X outweigh the shorter chunk
    // chains (measured: the 400 x 250 convection-diffusion refactor + pair
    // solve, K = 250, P = 32, 59.6 ms unsegmented, 78.2 / 127.2 / 163.3 ms
    // with 3 / 6 / 9 segments).
    int min_nch = L.max_nch;
    for (int i = 0; i < L.P; ++i) min_nch = std::min(min_nch, (int)(L.ld[i] / 32));
    const int ngc = chunk_couplings(K);
    int S = opt.segments;
    if (S == 0) {
      const bool f32 = opt.precision != SAP_FP64;
      S = std::min((f32 ? 2 : 1) * kSMs / L.P, min_nch / (f32 ? 16 : 32));
      S = S < (f32 ? 4 : 6) ? 1 : std::min(S, kMaxAutoSegments);
      if (ngc > 4) S = 1;
    }
    S = std::min(S, std::max(1, min_nch / std::max(ngc, 2)));
    if (!seg_sweeps_fit(K, opt.precision == SAP_FP64)) S = 1;
    L.S = std::max(1, S);
  }
  int64_t *doff, *dfb, *dld, *dcb;
  TRY(h->mem.alloc(&doff, L.P + 1));
  TRY(h->mem.alloc(&dfb, L.P));
  TRY(h->mem.alloc(&dld, L.P));
  CK(cudaMemcpyAsync(doff, L.off.data(), (L.P + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(dfb, L.fbase.data(), L.P * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(dld, L.ld.data(), L.P * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  TRY(h->mem.alloc(&dcb, L.P));
  CK(cudaMemcpyAsync(dcb, cb.data(), L.P * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  h->dcbase = dcb;
  h->d = Dev{doff, dfb, dld};
  TRY(h->mem.alloc(&h->absmax, 1));
  TRY(h->mem.alloc(&h->n_boosted, 1));
  TRY(h->mem.alloc(&h->singular, 1));
  TRY(h->mem.alloc(&h->singular_a, 1));
  CK(cudaMemsetAsync(h->singular_a, 0, sizeof(int), s));
  TRY(h->mem.alloc(&h->vec, (size_t)(11 * N)));
  TRY(h->mem.alloc(&h->kd.S, S_COUNT));
  TRY(h->mem.alloc(&h->kd.part, kKrylovBlocks * 4));
  TRY(h->mem.alloc(&h->kd.ticket, 1));
  TRY(h->mem.alloc(&h->flags, F_COUNT));
  CK(cudaMemsetAsync(h->n_boosted, 0, sizeof(unsigned long long), s));
  CK(cudaMemsetAsync(h->singular, 0, sizeof(int), s));
  CK(cudaMemsetAsync(h->kd.ticket, 0, sizeof(unsigned), s));
  CK(cudaMemsetAsync(h->vec, 0, 11 * N * sizeof(double), s));
  if (cudaMallocHost(&h->host_s, S_COUNT * sizeof(double)) != cudaSuccess) return SAP_ERR_OOM;
  if (cudaMallocHost(&h->host_f, F_COUNT * sizeof(int)) != cudaSuccess) return SAP_ERR_OOM;
  CK(cudaEventCreate(&h->ev0));
  CK(cudaEventCreate(&h->ev1));
  for (auto& e : h->evp) CK(cudaEventCreate(&e));
  CK(cudaEventCreate(&h->ev_rd));
  CK(cudaEventCreate(&h->ev_lu[0]));
  CK(cudaEventCreate(&h->ev_lu[1]));
  if (blockperm) h->impl.reset(new_blocks_solver(h, blockperm, s));
  else if (opt.precision == SAP_FP64) h->impl.reset(new Solver<double>(h));
  else h->impl.reset(new Solver<float>(h));
  if (!h->impl) return SAP_ERR_OOM;
  TRY(h->impl->alloc());
  return SAP_OK;
}

}  // namespace

struct sap_batch {
  std::vector<sap_handle*> hs;
  LuItem* items = nullptr;       // device work list of all blocks, longest first
  unsigned* counter = nullptr;   // work-list position of the persistent LU
  void* wlu = nullptr;           // per-CTA factor windows when Kmax's window exceeds shared memory
  int nitems = 0, Kmax = 1;
  bool fp64 = false;
  bool tc = false;               // tensor-core trailing updates (SAP_FP32_BF16TU, Kmax >= kTcMinK)
  cudaEvent_t ev = nullptr;
  ~sap_batch() {
    for (sap_handle* h : hs) delete h;
    if (items) cudaFree(items);
    if (counter) cudaFree(counter);
    if (wlu) cudaFree(wlu);
    if (ev) cudaEventDestroy(ev);
  }
};

namespace {

// Partition count of system i of a batch (opt.P == 0): about two blocks per
// SM over the whole batch, in proportion to N_i; SaP-C keeps N_i / P >= 2 K_i.
int batch_partitions(int64_t N, int K, int64_t total_rows, int variant) {
  const double share = (double)N / (double)total_rows;
  int64_t P = (int64_t)std::llround(2.0 * 152.0 * share);
  if (P < 1) P = 1;
  const int64_t pmax = variant == SAP_C ? std::max<int64_t>(1, N / (2 * (int64_t)K)) : std::max<int64_t>(1, N / 64);
  return (int)std::min(P, pmax);
}

// The batch's LU work list: every block of every system, longest first (LPT
// order on the elimination cost n K^2), copied to the device once.
sap_status_t build_work_list(sap_batch* B) {
  std::vector<LuItem> items;
  for (sap_handle* h : B->hs) {
    h->impl->lu_items(items);
    B->Kmax = std::max(B->Kmax, h->L.K);
  }
  B->tc = !B->fp64 && B->hs[0]->opt.precision == SAP_FP32_BF16TU && B->Kmax >= kTcMinK &&
          !lu_window_global(B->Kmax, false, true);
  std::stable_sort(items.begin(), items.end(), [](const LuItem& a, const LuItem& b) {
    return (double)a.n * a.K * a.K > (double)b.n * b.K * b.K;
  });
  B->nitems = (int)items.size();
  if (cudaMalloc(&B->items, items.size() * sizeof(LuItem)) != cudaSuccess ||
      cudaMalloc(&B->counter, sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    return SAP_ERR_OOM;
  }
  CK(cudaMemcpy(B->items, items.data(), items.size() * sizeof(LuItem), cudaMemcpyHostToDevice));
  if (lu_window_global(B->Kmax, B->fp64, B->tc)) {
    const size_t bytes = (size_t)lu_items_grid(B->nitems, B->Kmax, B->fp64, B->tc) * lu_window_elems(B->Kmax) *
                         (B->fp64 ? sizeof(double) : sizeof(float));
    if (cudaMalloc(&B->wlu, bytes) != cudaSuccess) {
      cudaGetLastError();
      return SAP_ERR_OOM;
    }
  }
  CK(cudaEventCreateWithFlags(&B->ev, cudaEventDisableTiming));
  return SAP_OK;
}

// Factor a batch: each system's threshold pass (and FP32 cast) on its own
// internal stream, then ONE persistent LU launch over the work list of all
// blocks, then each system's sweep matrices (and SaP-C tips) on its stream
// again; wait for all; s is ordered after them.
sap_status_t factor_batch(sap_batch* B, cudaStream_t s) {
  CK(cudaEventRecord(B->ev, s));
  for (sap_handle* h : B->hs) {
    TRY(ensure_stream(h));
    CK(cudaStreamWaitEvent(h->ks, B->ev, 0));
    CK(cudaMemsetAsync(h->n_boosted, 0, sizeof(unsigned long long), h->ks));
    CK(cudaMemsetAsync(h->singular, 0, sizeof(int), h->ks));
    TRY(h->impl->factor_pre(h->ks));
    CK(cudaEventRecord(h->evj, h->ks));
    CK(cudaStreamWaitEvent(s, h->evj, 0));
  }
  // the work list's error flag: the first system's (every system's factor phase reads its own)
  int* err = B->hs[0]->impl->err_flag();
  for (sap_handle* h : B->hs) CK(cudaEventRecord(h->ev_lu[0], s));
  CK(B->fp64 ? launch_factor_lu_items<double>(B->items, B->nitems, B->Kmax, B->counter,
                                              static_cast<double*>(B->wlu), false, err, s)
             : launch_factor_lu_items<float>(B->items, B->nitems, B->Kmax, B->counter,
                                             static_cast<float*>(B->wlu), B->tc, err, s));
  for (sap_handle* h : B->hs) CK(cudaEventRecord(h->ev_lu[1], s));
  CK(cudaEventRecord(B->ev, s));
  for (sap_handle* h : B->hs) {
    CK(cudaStreamWaitEvent(h->ks, B->ev, 0));
    TRY(h->impl->factor_post(h->ks));
  }
  sap_status_t st = SAP_OK;
  for (sap_handle* h : B->hs) {
    const sap_status_t e = finish_factor(h);
    if (st == SAP_OK) st = e;
    CK(cudaEventRecord(h->evj, h->ks));
    CK(cudaStreamWaitEvent(s, h->evj, 0));
  }
  return st;
}

// Solves in lockstep rounds of one outer iteration each: every unfinished
// run replays its iteration on its own stream, then the host waits for all.
sap_status_t run_lockstep(std::vector<KrylovRun>& k) {
  const size_t n = k.size();
  for (size_t i = 0; i < n; ++i) TRY(k[i].begin());
  for (size_t i = 0; i < n; ++i) {
    CK(cudaStreamSynchronize(k[i].s));
    k[i].after_begin();
  }
  // every run whose loop can go on the device: one launch each, no rounds
  for (size_t i = 0; i < n; ++i)
    if (k[i].active() && k[i].launch_device_loop()) k[i].done = true;
  std::vector<char> ran(n);
  for (;;) {
    bool any = false;
    for (size_t i = 0; i < n; ++i) {
      ran[i] = k[i].active();
      if (ran[i]) {
        TRY(k[i].round());
        any = true;
      }
    }
    if (!any) break;
    for (size_t i = 0; i < n; ++i)
      if (ran[i]) {
        CK(cudaStreamSynchronize(k[i].s));
        k[i].after_round();
      }
  }
  return SAP_OK;
}

// All systems' solves (forward or adjoint) in lockstep rounds.
sap_status_t solve_batch(sap_batch* B, const double* const* b, double* const* x, bool tr, sap_info_t* infos,
                         int32_t* statuses, cudaStream_t s) {
  const size_t n = B->hs.size();
  std::vector<KrylovRun> k(n);
  for (size_t i = 0; i < n; ++i) {
    if (!b[i] || !x[i] || b[i] == x[i]) return SAP_ERR_INVALID_ARG;
    TRY(k[i].init(B->hs[i], b[i], x[i], tr, s));
  }
  TRY(run_lockstep(k));
  sap_status_t st = SAP_OK;
  for (size_t i = 0; i < n; ++i) {
    const sap_status_t e = k[i].finish(infos ? &infos[i] : nullptr);
    if (statuses) statuses[i] = e;
    if (st == SAP_OK) st = e;
  }
  return st;
}

// Every system's forward and adjoint solve together: 2n runs in lockstep,
// the adjoint ones on each handle's second workspace.
sap_status_t solve_pair_batch(sap_batch* B, const double* const* b, double* const* x, const double* const* g,
                              double* const* lam, sap_info_t* ix, sap_info_t* il, int32_t* statuses,
                              cudaStream_t s) {
  const size_t n = B->hs.size();
  std::vector<KrylovRun> k(2 * n);
  for (size_t i = 0; i < n; ++i) {
    if (!b[i] || !x[i] || !g[i] || !lam[i] || b[i] == x[i] || g[i] == lam[i] || x[i] == lam[i])
      return SAP_ERR_INVALID_ARG;
    TRY(k[i].init(B->hs[i], b[i], x[i], false, s, 0));
    TRY(k[n + i].init(B->hs[i], g[i], lam[i], true, s, 1));
    // SaP-C: each system's adjoint tips on its adjoint stream, overlapping the forward iterations
    CK(cudaEventRecord(B->hs[i]->w2.evj, s));
    CK(cudaStreamWaitEvent(k[n + i].s, B->hs[i]->w2.evj, 0));
    TRY(B->hs[i]->impl->build_adjoint_async(k[n + i].s));
  }
  TRY(run_lockstep(k));
  sap_status_t st = SAP_OK;
  for (size_t i = 0; i < 2 * n; ++i) {
    sap_info_t* inf = i < n ? (ix ? &ix[i] : nullptr) : (il ? &il[i - n] : nullptr);
    sap_status_t e = k[i].finish(inf);
    if (i >= n) {
      const sap_status_t sg = B->hs[i - n]->impl->adjoint_singular();
      if (sg != SAP_OK) e = sg;
    }
    if (statuses) statuses[i] = e;
    if (st == SAP_OK) st = e;
  }
  return st;
}

// ---- SaP with a bandwidth of its own per block (third-stage reordering) ----
// Every block b of the partition is reordered by its permutation into
// Ahat_b (half-bandwidth K_b), held as a one-block SaP-D handle of its own
// (factors, chunk and transfer matrices of the sweeps at K_b).  Factor: the
// reordered bands gathered from the band, each block's threshold pass on its
// own stream, ONE persistent LU launch over all blocks (LPT work list, boost
// threshold from the whole band), each block's sweep matrices on its stream;
// SaP-C then the entire spikes, their tips and the reduced matrices.  Apply:
// Pi r, the blocks' sweeps on their streams (fork and join by events, so the
// Krylov iteration's capture takes them in), then Pi^T g (SaP-D) or the
// reduced solve and the spike correction (SaP-C).
template <typename T>
struct Blocks : SolverBase {
  sap_handle* h;
  const int32_t* perm_src;
  cudaStream_t cs;                     // creation stream
  std::vector<std::unique_ptr<sap_handle>> sub;
  std::vector<int> Kb;
  std::vector<int64_t> hbase;
  BlockMap m{};
  int32_t *perm = nullptr, *pinv = nullptr, *dKb = nullptr;
  int64_t* dhbase = nullptr;
  double* hb = nullptr;
  int64_t hb_elems = 0;
  LuItem* items = nullptr;
  unsigned* counter = nullptr;
  T* wlu = nullptr;
  int nitems = 0, Kbmax = 1;
  bool tcu = false;
  const void** dMf = nullptr;          // per block: chunk matrices of its forward (L) and backward (U) sweeps
  const void** dMb = nullptr;
  int* dng = nullptr;                  // per block: couplings per chunk
  int ngmax = 1;
  int64_t* dldp = nullptr;
  T* spk = nullptr;
  int64_t* dsbase = nullptr;
  Factors<T> f;                        // V, Wt, R, R0, piv of the interfaces; err
  unsigned char* gws = nullptr;
  double *rh = nullptr, *gh = nullptr, *xt = nullptr, *xb = nullptr;
  int* gerr = nullptr;                 // an entry beyond its block's K_b at the gather
  cudaEvent_t evfork = nullptr;
  int64_t spk_elems = 0;
  // the preconditioner of A^T, built on the first transposed use after a factorisation:
  // its own spikes, tips and reduced matrices (f.Va, f.Wa, f.Ra, f.piva), apply scratch,
  // and per block a stream of its own for the transposed sweeps (an adjoint solve may run
  // concurrently with the forward one)
  bool adjoint_ready = false;
  bool amats_set = false;
  const void** dMfa = nullptr;         // per block: chunk matrices of its U^T forward and L^T backward sweeps
  const void** dMba = nullptr;
  T* spk_a = nullptr;
  unsigned char* gws_a = nullptr;
  double *rh_t = nullptr, *gh_t = nullptr, *xt_t = nullptr, *xb_t = nullptr;
  cudaEvent_t evfork_t = nullptr;
  std::vector<cudaStream_t> tst;
  std::vector<cudaEvent_t> tev;
  // the factorisation's launches (some 250 over the blocks' streams) captured
  // once as a graph and replayed by later factorisations, on an internal stream
  // joined to the caller's by events
  int nfactor = 0;
  cudaGraphExec_t fexec = nullptr;
  bool fgraph_failed = false;
  long long flaunches = 0;
  cudaStream_t fks = nullptr;
  cudaEvent_t evin = nullptr, evout = nullptr;
  Blocks(sap_handle* hh, const int32_t* p, cudaStream_t s) : h(hh), perm_src(p), cs(s) {}
  ~Blocks() override {
    if (fexec) cudaGraphExecDestroy(fexec);
    if (fks) cudaStreamDestroy(fks);
    if (evin) cudaEventDestroy(evin);
    if (evout) cudaEventDestroy(evout);
    if (evfork) cudaEventDestroy(evfork);
    if (evfork_t) cudaEventDestroy(evfork_t);
    for (cudaStream_t x : tst)
      if (x) cudaStreamDestroy(x);
    for (cudaEvent_t e : tev)
      if (e) cudaEventDestroy(e);
  }
  bool coupled() const { return h->opt.variant == SAP_C && h->L.P > 1; }

  sap_status_t alloc() override {
    const Layout& L = h->L;
    const int P = L.P, K = L.K;
    const int64_t N = L.N;
    if (!perm_src || P < 1 || N >= (int64_t(1) << 31)) return SAP_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(cs));
    // the permutations: checked per block, inverted on the host
    std::vector<int32_t> hp((size_t)N), hpi((size_t)N);
    CK(cudaMemcpy(hp.data(), perm_src, (size_t)N * sizeof(int32_t), cudaMemcpyDeviceToHost));
    for (int b = 0; b < P; ++b) {
      const int64_t s0 = L.off[b], n = L.off[b + 1] - s0;
      std::vector<char> seen((size_t)n, 0);
      for (int64_t a = 0; a < n; ++a) {
        const int32_t v = hp[(size_t)(s0 + a)];
        if (v < 0 || v >= n || seen[(size_t)v]) return SAP_ERR_INVALID_ARG;
        seen[(size_t)v] = 1;
        hpi[(size_t)(s0 + v)] = (int32_t)a;
      }
    }
    TRY(h->mem.alloc(&perm, (size_t)N));
    TRY(h->mem.alloc(&pinv, (size_t)N));
    TRY(h->mem.alloc(&dKb, (size_t)P));
    TRY(h->mem.alloc(&dhbase, (size_t)P));
    TRY(h->mem.alloc(&gerr, 1));
    CK(cudaMemcpy(perm, hp.data(), (size_t)N * sizeof(int32_t), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(pinv, hpi.data(), (size_t)N * sizeof(int32_t), cudaMemcpyHostToDevice));
    m.N = N;
    m.K = K;
    m.P = P;
    m.q = N / P;
    m.pr = N - (int64_t)P * m.q;
    m.off = h->d.off;
    m.perm = perm;
    m.pinv = pinv;
    m.Kb = dKb;
    m.hbase = dhbase;
    // the blocks' half-bandwidths
    CK(launch_block_bw(h->band, m, dKb, cs));
    Kb.assign((size_t)P, 0);
    CK(cudaMemcpyAsync(Kb.data(), dKb, (size_t)P * sizeof(int), cudaMemcpyDeviceToHost, cs));
    CK(cudaStreamSynchronize(cs));
    hbase.assign((size_t)P, 0);
    int64_t acc = 0;
    for (int b = 0; b < P; ++b) {
      const int64_t n = L.off[b + 1] - L.off[b];
      Kb[(size_t)b] = std::max(1, Kb[(size_t)b]);
      if (Kb[(size_t)b] >= n) return SAP_ERR_INVALID_ARG;
      if (Kb[(size_t)b] > sap_max_K(h->opt.precision)) return SAP_ERR_NOT_IMPLEMENTED;
      Kbmax = std::max(Kbmax, Kb[(size_t)b]);
      hbase[(size_t)b] = acc;
      acc += n * (2 * (int64_t)Kb[(size_t)b] + 1);
    }
    hb_elems = acc;
    CK(cudaMemcpy(dKb, Kb.data(), (size_t)P * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(dhbase, hbase.data(), (size_t)P * sizeof(int64_t), cudaMemcpyHostToDevice));
    TRY(h->mem.alloc(&hb, (size_t)hb_elems));
    CK(cudaMemset(hb, 0, (size_t)hb_elems * sizeof(double)));
    // the blocks as one-block SaP-D handles on their reordered bands
    sub.resize((size_t)P);
    std::vector<LuItem> it;
    for (int b = 0; b < P; ++b) {
      sap_options_t ob = h->opt;
      ob.P = 1;
      ob.variant = SAP_D;
      TRY(create_handle(hb + hbase[(size_t)b], L.off[b + 1] - L.off[b], Kb[(size_t)b], &ob, cs, sub[(size_t)b]));
      TRY(ensure_stream(sub[(size_t)b].get()));
      sub[(size_t)b]->impl->lu_items(it);
    }
    for (LuItem& x : it) {            // one boost threshold (the whole band's) and one counter
      x.absmax = h->absmax;
      x.nb = h->n_boosted;
    }
    std::stable_sort(it.begin(), it.end(), [](const LuItem& a, const LuItem& c) {
      return (double)a.n * a.K * a.K > (double)c.n * c.K * c.K;
    });
    nitems = (int)it.size();
    TRY(h->mem.alloc(&items, it.size()));
    TRY(h->mem.alloc(&counter, 1));
    CK(cudaMemcpy(items, it.data(), it.size() * sizeof(LuItem), cudaMemcpyHostToDevice));
    const bool fp64 = sizeof(T) == 8;
    tcu = !fp64 && h->opt.precision == SAP_FP32_BF16TU && Kbmax >= kTcMinK && !lu_window_global(Kbmax, false, true);
    if (lu_window_global(Kbmax, fp64, tcu))
      TRY(h->mem.alloc(&wlu, (size_t)lu_items_grid(nitems, Kbmax, fp64, tcu) * lu_window_elems(Kbmax)));
    TRY(h->mem.alloc(&f.err, 2));
    {
      const int e2[2] = {0, spin_limit_value(h->opt.spin_limit)};
      CK(cudaMemcpy(f.err, e2, sizeof(e2), cudaMemcpyHostToDevice));
    }
    TRY(h->mem.alloc(&rh, (size_t)N));
    TRY(h->mem.alloc(&gh, (size_t)N));
    CK(cudaEventCreateWithFlags(&evfork, cudaEventDisableTiming));
    if (!h->evu[0]) {
      CK(cudaEventCreate(&h->evu[0]));
      CK(cudaEventCreate(&h->evu[1]));
    }
    if (coupled()) {
      const int nI = P - 1;
      const int64_t KK = (int64_t)K * K;
      std::vector<const void*> mf((size_t)P), mb((size_t)P);
      std::vector<int> ngv((size_t)P);
      std::vector<int64_t> ldv((size_t)P), sb((size_t)(2 * nI));
      for (int b = 0; b < P; ++b) {
        auto* sv = dynamic_cast<Solver<T>*>(sub[(size_t)b]->impl.get());
        if (!sv) return SAP_ERR_CUDA;
        mf[(size_t)b] = sv->f.Mlf;
        mb[(size_t)b] = sv->f.Mub;
        ngv[(size_t)b] = chunk_couplings(Kb[(size_t)b]);
        ngmax = std::max(ngmax, ngv[(size_t)b]);
        ldv[(size_t)b] = sub[(size_t)b]->L.ld[0];
      }
      if (full_spikes_smem(ngmax, fp64) > kSmemPerBlock) return SAP_ERR_NOT_IMPLEMENTED;
      const int KS = spike_row_stride(K, fp64);
      int64_t so = 0;
      for (int i = 0; i < nI; ++i) {
        sb[(size_t)(2 * i)] = so;
        so += (L.off[i + 1] - L.off[i]) * KS;
        sb[(size_t)(2 * i + 1)] = so;
        so += (L.off[i + 2] - L.off[i + 1]) * KS;
      }
      TRY(h->mem.alloc(&dMf, (size_t)P));
      TRY(h->mem.alloc(&dMb, (size_t)P));
      TRY(h->mem.alloc(&dng, (size_t)P));
      TRY(h->mem.alloc(&dldp, (size_t)P));
      TRY(h->mem.alloc(&dsbase, sb.size()));
      spk_elems = so;
      TRY(h->mem.alloc(&spk, (size_t)so));
      CK(cudaMemset(spk, 0, (size_t)so * sizeof(T)));     // the row padding is read (times 0) by the correction
      CK(cudaMemcpy(dMf, mf.data(), mf.size() * sizeof(void*), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(dMb, mb.data(), mb.size() * sizeof(void*), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(dng, ngv.data(), ngv.size() * sizeof(int), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(dldp, ldv.data(), ldv.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(dsbase, sb.data(), sb.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
      TRY(h->mem.alloc(&f.V, (size_t)(nI * KK)));
      TRY(h->mem.alloc(&f.Wt, (size_t)(nI * KK)));
      TRY(h->mem.alloc(&f.R, (size_t)(nI * KK)));
      TRY(h->mem.alloc(&f.R0, (size_t)(nI * KK)));
      TRY(h->mem.alloc(&f.piv, (size_t)(nI * K)));
      TRY(h->mem.alloc(&gws, reduced_ws_bytes(K, nI, fp64)));
      TRY(h->mem.alloc(&xt, (size_t)(nI * K)));
      TRY(h->mem.alloc(&xb, (size_t)(nI * K)));
    }
    return SAP_OK;
  }

  // a block has transposed sweep data: its factorisation then rebuilds them in
  // the background, a branch the factorisation's graph cannot hold
  bool blocks_transposed() const {
    for (const auto& q : sub) {
      auto* sv = dynamic_cast<Solver<T>*>(q->impl.get());
      if (!sv || sv->f.Mutf) return true;
    }
    return false;
  }
  void capture_factor() {
    const long long l0 = launches_so_far();
    cudaGraph_t g = nullptr;
    bool ok = true;
    if (!fks) {
      ok = cudaStreamCreateWithFlags(&fks, cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&evin, cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&evout, cudaEventDisableTiming) == cudaSuccess;
    }
    ok = ok && cudaStreamBeginCapture(fks, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    const sap_status_t st = ok ? factor_seq(fks) : SAP_ERR_CUDA;
    if (ok) ok = cudaStreamEndCapture(fks, &g) == cudaSuccess && st == SAP_OK && g;
    if (ok) ok = cudaGraphInstantiate(&fexec, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) {
      if (fexec) cudaGraphExecDestroy(fexec);
      fexec = nullptr;
      fgraph_failed = true;
      cudaGetLastError();
    }
    flaunches = launches_so_far() - l0;
    count_launches(-(int)flaunches);     // captured, not run
  }
  sap_status_t factor(cudaStream_t s) override {
    adjoint_ready = false;               // rebuilt on the next transposed use
    // from the second factorisation on (the first creates the blocks' streams
    // and events) one graph launch, unless a block has transposed data
    if (++nfactor >= 2 && !fgraph_failed && !blocks_transposed()) {
      if (!fexec) capture_factor();
      if (fexec) {
        CK(cudaEventRecord(evin, s));
        CK(cudaStreamWaitEvent(fks, evin, 0));
        CK(cudaGraphLaunch(fexec, fks));
        count_launches((int)flaunches);
        CK(cudaEventRecord(evout, fks));
        CK(cudaStreamWaitEvent(s, evout, 0));
        return SAP_OK;
      }
    }
    return factor_seq(s);
  }
  // the handle's phase events: inside a capture a record node of their own
  // (a plain record there only marks a fork or join), so that a replay sets them
  static cudaError_t rec(cudaEvent_t e, cudaStream_t s) {
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cst) == cudaSuccess && cst == cudaStreamCaptureStatusActive)
      return cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    return cudaEventRecord(e, s);
  }
  sap_status_t factor_seq(cudaStream_t s) {
    const Layout& L = h->L;
    CK(rec(h->evp[0], s));
    CK(launch_absmax(h->band, L.N, L.K, h->absmax, s));
    CK(cudaMemsetAsync(gerr, 0, sizeof(int), s));
    CK(launch_block_gather(h->band, m, hb, hb_elems, gerr, s));
    CK(cudaEventRecord(evfork, s));
    for (auto& q : sub) {
      CK(cudaStreamWaitEvent(q->ks, evfork, 0));
      TRY(q->impl->factor_pre(q->ks));
      CK(cudaEventRecord(q->evj, q->ks));
      CK(cudaStreamWaitEvent(s, q->evj, 0));
    }
    CK(rec(h->ev_lu[0], s));
    CK(launch_factor_lu_items<T>(items, nitems, Kbmax, counter, wlu, tcu, f.err, s));
    CK(rec(h->ev_lu[1], s));
    CK(cudaEventRecord(evfork, s));
    for (auto& q : sub) {
      CK(cudaStreamWaitEvent(q->ks, evfork, 0));
      TRY(q->impl->factor_post(q->ks));
      CK(cudaEventRecord(q->evj, q->ks));
      CK(cudaStreamWaitEvent(s, q->evj, 0));
    }
    CK(rec(h->evp[1], s));
    CK(rec(h->evu[0], s));    // no UL factorisation: an empty T_UL bracket
    CK(rec(h->evu[1], s));
    CK(rec(h->evp[2], s));
    if (coupled()) {
      CK(launch_full_spikes<T>(h->band, m, ngmax, dMf, dMb, dng, dldp, spk, dsbase, f.V, f.Wt, false, s));
      CK(rec(h->ev_rd, s));
      CK(launch_reduced<T>(f.V, f.Wt, L.K, L.P - 1, f.R, f.R0, f.piv, h->singular, gws, s));
    } else {
      CK(rec(h->ev_rd, s));
    }
    CK(rec(h->evp[3], s));
    return SAP_OK;
  }
  sap_status_t factor_pre(cudaStream_t) override { return SAP_ERR_NOT_IMPLEMENTED; }
  sap_status_t factor_post(cudaStream_t) override { return SAP_ERR_NOT_IMPLEMENTED; }
  void lu_items(std::vector<LuItem>&) const override {}
  // the preconditioner of A^T: the blocks' transposed sweep matrices (their own
  // prepare_transposed), then the entire spikes of A^T and its reduced matrices; synchronises s
  sap_status_t build_adjoint(cudaStream_t s) override {
    if (adjoint_ready) return SAP_OK;
    const Layout& L = h->L;
    const int P = L.P, K = L.K;
    if (!rh_t) {
      TRY(h->mem.alloc(&rh_t, (size_t)L.N));
      TRY(h->mem.alloc(&gh_t, (size_t)L.N));
      CK(cudaEventCreateWithFlags(&evfork_t, cudaEventDisableTiming));
      tst.assign((size_t)P, nullptr);
      tev.assign((size_t)P, nullptr);
      for (int b = 0; b < P; ++b) {
        CK(cudaStreamCreateWithFlags(&tst[(size_t)b], cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&tev[(size_t)b], cudaEventDisableTiming));
      }
    }
    if (coupled()) {
      const int nI = P - 1;
      const int64_t KK = (int64_t)K * K;
      if (!spk_a) {
        TRY(h->mem.alloc(&spk_a, (size_t)spk_elems));
        CK(cudaMemset(spk_a, 0, (size_t)spk_elems * sizeof(T)));
        TRY(h->mem.alloc(&f.Va, (size_t)(nI * KK)));
        TRY(h->mem.alloc(&f.Wa, (size_t)(nI * KK)));
        TRY(h->mem.alloc(&f.Ra, (size_t)(nI * KK)));
        TRY(h->mem.alloc(&f.Ra0, (size_t)(nI * KK)));
        TRY(h->mem.alloc(&f.piva, (size_t)(nI * K)));
        TRY(h->mem.alloc(&gws_a, reduced_ws_bytes(K, nI, sizeof(T) == 8)));
        TRY(h->mem.alloc(&xt_t, (size_t)(nI * K)));
        TRY(h->mem.alloc(&xb_t, (size_t)(nI * K)));
        TRY(h->mem.alloc(&dMfa, (size_t)P));
        TRY(h->mem.alloc(&dMba, (size_t)P));
      }
      if (!amats_set) {          // allocated by the blocks' first transposed preparation, then fixed
        std::vector<const void*> mf((size_t)P), mb((size_t)P);
        for (int b = 0; b < P; ++b) {
          auto* sv = dynamic_cast<Solver<T>*>(sub[(size_t)b]->impl.get());
          if (!sv || !sv->f.Mutf || !sv->f.Mltb) return SAP_ERR_CUDA;
          mf[(size_t)b] = sv->f.Mutf;
          mb[(size_t)b] = sv->f.Mltb;
        }
        CK(cudaMemcpy(dMfa, mf.data(), mf.size() * sizeof(void*), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(dMba, mb.data(), mb.size() * sizeof(void*), cudaMemcpyHostToDevice));
        amats_set = true;
      }
      CK(cudaMemsetAsync(h->singular_a, 0, sizeof(int), s));
      CK(launch_full_spikes<T>(h->band, m, ngmax, dMfa, dMba, dng, dldp, spk_a, dsbase, f.Va, f.Wa, true, s));
      CK(launch_reduced<T>(f.Va, f.Wa, K, nI, f.Ra, f.Ra0, f.piva, h->singular_a, gws_a, s));
      int sing = 0;
      CK(cudaMemcpyAsync(&sing, h->singular_a, sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (sing) return SAP_ERR_SINGULAR;
    }
    adjoint_ready = true;
    return SAP_OK;
  }
  sap_status_t prepare_transposed(cudaStream_t s) override {
    for (auto& q : sub) TRY(q->impl->prepare_transposed(s));
    return build_adjoint(s);
  }
  sap_status_t build_adjoint_async(cudaStream_t s) override { return prepare_transposed(s); }
  sap_status_t adjoint_singular() override { return SAP_OK; }
  const std::vector<int>* block_bandwidths() const override { return &Kb; }

  sap_status_t apply_transposed(const double* r, double* z, cudaStream_t s, Gate gt) {
    const Layout& L = h->L;
    // inside a Krylov run's capture begin() has prepared A^T's preconditioner on the caller's stream
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cst) != cudaSuccess || cst == cudaStreamCaptureStatusNone)
      TRY(prepare_transposed(s));
    if (!adjoint_ready) return SAP_ERR_NOT_IMPLEMENTED;
    CK(launch_block_perm(m, r, rh_t, true, s, gt));
    CK(cudaEventRecord(evfork_t, s));
    for (int b = 0; b < L.P; ++b) {
      CK(cudaStreamWaitEvent(tst[(size_t)b], evfork_t, 0));
      TRY(sub[(size_t)b]->impl->apply(rh_t + L.off[b], gh_t + L.off[b], true, tst[(size_t)b], gt));
      CK(cudaEventRecord(tev[(size_t)b], tst[(size_t)b]));
      CK(cudaStreamWaitEvent(s, tev[(size_t)b], 0));
    }
    if (!coupled()) {
      CK(launch_block_perm(m, gh_t, z, false, s, gt));
      return SAP_OK;
    }
    CK(launch_block_reduced<T>(m, gh_t, f.Va, f.Wa, f.Ra, xt_t, xb_t, s, gt));
    CK(launch_block_correct<T>(m, (int)(L.off[1] - L.off[0]), gh_t, spk_a, dsbase, xt_t, xb_t, z, s, gt));
    return SAP_OK;
  }
  sap_status_t apply(const double* r, double* z, bool transpose, cudaStream_t s, Gate gt) override {
    if (transpose) return apply_transposed(r, z, s, gt);
    const Layout& L = h->L;
    CK(launch_block_perm(m, r, rh, true, s, gt));
    CK(cudaEventRecord(evfork, s));
    for (int b = 0; b < L.P; ++b) {
      sap_handle* q = sub[(size_t)b].get();
      CK(cudaStreamWaitEvent(q->ks, evfork, 0));
      TRY(q->impl->apply(rh + L.off[b], gh + L.off[b], false, q->ks, gt));
      CK(cudaEventRecord(q->evj, q->ks));
      CK(cudaStreamWaitEvent(s, q->evj, 0));
    }
    if (!coupled()) {
      CK(launch_block_perm(m, gh, z, false, s, gt));
      return SAP_OK;
    }
    CK(launch_block_reduced<T>(m, gh, f.V, f.Wt, f.R, xt, xb, s, gt));
    CK(launch_block_correct<T>(m, (int)(L.off[1] - L.off[0]), gh, spk, dsbase, xt, xb, z, s, gt));
    return SAP_OK;
  }

  sap_status_t take_device_error(cudaStream_t s) override {
    sap_status_t st = SAP_OK;
    for (auto& q : sub) {
      const sap_status_t e = q->impl->take_device_error(s);
      if (st == SAP_OK) st = e;
    }
    int e = 0;
    CK(cudaMemcpyAsync(&e, f.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (e) {
      CK(cudaMemsetAsync(f.err, 0, sizeof(int), s));
      st = SAP_ERR_TIMEOUT;
    }
    return st;
  }
  sap_status_t take_factor_error() override {
    int g = 0, e = 0;
    CK(cudaMemcpy(&g, gerr, sizeof(int), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&e, f.err, sizeof(int), cudaMemcpyDeviceToHost));
    sap_status_t st = SAP_OK;
    for (auto& q : sub) {
      const sap_status_t x = q->impl->take_factor_error();
      if (st == SAP_OK) st = x;
    }
    if (e) {
      CK(cudaMemset(f.err, 0, sizeof(int)));
      st = SAP_ERR_TIMEOUT;
    }
    if (g) return SAP_ERR_INVALID_ARG;
    return st;
  }
  bool tc_used() const override { return tcu; }
  int* err_flag() override { return f.err; }
  sap_status_t block_lu(int, double*, cudaStream_t) override { return SAP_ERR_NOT_IMPLEMENTED; }
  sap_status_t interface(int i, int which, bool adjoint, double* host, cudaStream_t s) override {
    const int K = h->L.K;
    const int64_t KK = (int64_t)K * K;
    if (!coupled() || i < 0 || i >= h->L.P - 1 || which < 0 || which > 4) return SAP_ERR_INVALID_ARG;
    if (adjoint) TRY(prepare_transposed(s));
    if (which <= 1) return read_coupling(h, i, which, adjoint, host, s);
    if (which == 4) {
      CK(cudaMemcpyAsync(host, (adjoint ? f.Ra0 : f.R0) + i * KK, (size_t)KK * sizeof(double),
                         cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      return SAP_OK;
    }
    std::vector<T> buf((size_t)KK);
    CK(cudaMemcpyAsync(buf.data(), (which == 2 ? (adjoint ? f.Va : f.V) : (adjoint ? f.Wa : f.Wt)) + i * KK,
                       (size_t)KK * sizeof(T), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int64_t e = 0; e < KK; ++e) host[e] = (double)buf[(size_t)e];
    return SAP_OK;
  }
};

SolverBase* new_blocks_solver(sap_handle* h, const int32_t* perm_dev, cudaStream_t s) {
  if (h->opt.precision == SAP_FP64) return new (std::nothrow) Blocks<double>(h, perm_dev, s);
  return new (std::nothrow) Blocks<float>(h, perm_dev, s);
}

}  // namespace

extern "C" {

void sap_default_options(sap_options_t* o) {
  if (!o) return;
  o->P = 1;
  o->variant = SAP_D;
  o->precision = SAP_FP64;
  o->max_iters = 500;
  o->tol = 1e-10;
  o->boost_eps = 0.0;
  o->spin_limit = 0;
  o->segments = 0;
  o->krylov = SAP_KRYLOV_BICGSTAB2;
}

int64_t sap_kernel_launches(void) { return (int64_t)sap::g_launches.load(); }

int32_t sap_max_K(int32_t precision) {
  const bool fp64 = precision == SAP_FP64;
  int K = kMaxK;
  const bool tc = precision == SAP_FP32_BF16TU;
  while (K > 1 && (sweep_smem_bytes(K, fp64) > kSmemPerBlock || lu_smem_bytes(K, fp64, tc) > kSmemPerBlock ||
                   chunk_mats_smem_bytes(K, fp64) > kSmemPerBlock))
    --K;
  return K;
}

sap_status_t sap_factor(const double* band_dev, int64_t N, int32_t K, const sap_options_t* opt_in,
                        cudaStream_t s, sap_handle_t* out) {
  if (!out) return SAP_ERR_INVALID_ARG;
  *out = nullptr;
  if (!opt_in) return SAP_ERR_INVALID_ARG;
  sap_options_t opt = *opt_in;
  if (opt.P == 0) {
    // P = 0: the partition count (and, with segments = 0, the segment count)
    // measured fastest by the autotuner over its default candidates
    if (!band_dev || N < 2 || K < 1 || K >= N) return SAP_ERR_INVALID_ARG;
    int32_t bp = 0, bs = 0;
    const int32_t seg_user = opt.segments;
    TRY(sap_autotune(band_dev, N, K, &opt, nullptr, 0, seg_user > 0 ? &seg_user : nullptr, seg_user > 0 ? 1 : 0,
                     nullptr, s, &bp, &bs, nullptr, nullptr));
    opt.P = bp;
    opt.segments = bs;
  }
  std::unique_ptr<sap_handle> h;
  TRY(create_handle(band_dev, N, K, &opt, s, h));
  TRY(run_factor(h.get(), s));
  *out = h.release();
  return SAP_OK;
}

sap_status_t sap_factor_blocks(const double* band_dev, int64_t N, int32_t K, const int32_t* perm_dev,
                               const sap_options_t* opt, cudaStream_t s, sap_handle_t* out) {
  if (!out) return SAP_ERR_INVALID_ARG;
  *out = nullptr;
  if (!opt || !perm_dev || opt->P < 1) return SAP_ERR_INVALID_ARG;
  std::unique_ptr<sap_handle> h;
  TRY(create_handle(band_dev, N, K, opt, s, h, perm_dev));
  TRY(run_factor(h.get(), s));
  *out = h.release();
  return SAP_OK;
}

sap_status_t sap_get_block_bandwidths(sap_handle_t h, int32_t* Ki) {
  if (!h || !Ki) return SAP_ERR_INVALID_ARG;
  const std::vector<int>* k = h->impl->block_bandwidths();
  if (!k) return SAP_ERR_INVALID_ARG;
  for (size_t b = 0; b < k->size(); ++b) Ki[b] = (*k)[b];
  return SAP_OK;
}

sap_status_t sap_refactor(sap_handle_t h, cudaStream_t s) {
  if (!h) return SAP_ERR_INVALID_ARG;
  return run_factor(h, s);
}

sap_status_t sap_solve(sap_handle_t h, const double* b, double* x, sap_info_t* info, cudaStream_t s) {
  if (!h || !b || !x || b == x) return SAP_ERR_INVALID_ARG;
  return krylov(h, b, x, false, info, s);
}

sap_status_t sap_solve_adjoint(sap_handle_t h, const double* g, double* lam, sap_info_t* info, cudaStream_t s) {
  if (!h || !g || !lam || g == lam) return SAP_ERR_INVALID_ARG;
  TRY(h->impl->build_adjoint(s));
  return krylov(h, g, lam, true, info, s);
}

sap_status_t sap_solve_pair(sap_handle_t h, const double* b, double* x, const double* g, double* lam,
                            sap_info_t* info_x, sap_info_t* info_lam, cudaStream_t s) {
  if (!h || !b || !x || !g || !lam || b == x || g == lam || x == lam) return SAP_ERR_INVALID_ARG;
  // forward on the handle's workspace, adjoint on the second one: two streams,
  // lockstep rounds, one host synchronisation per round for both
  KrylovRun k[2];
  TRY(k[0].init(h, b, x, false, s, 0));
  TRY(k[1].init(h, g, lam, true, s, 1));
  // SaP-C: the adjoint's tips and reduced matrices are built on the adjoint's
  // stream while the forward iteration starts
  CK(cudaEventRecord(h->w2.evj, s));
  CK(cudaStreamWaitEvent(k[1].s, h->w2.evj, 0));
  TRY(h->impl->build_adjoint_async(k[1].s));
  TRY(k[0].begin());
  TRY(k[1].begin());
  for (auto& r : k) {
    CK(cudaStreamSynchronize(r.s));
    r.after_begin();
  }
  for (auto& r : k)
    if (r.active() && r.launch_device_loop()) r.done = true;     // finished by the device, read in finish()
  for (;;) {
    bool ran[2] = {k[0].active(), k[1].active()};
    if (!ran[0] && !ran[1]) break;
    for (int i = 0; i < 2; ++i)
      if (ran[i]) TRY(k[i].round());
    for (int i = 0; i < 2; ++i)
      if (ran[i]) {
        CK(cudaStreamSynchronize(k[i].s));
        k[i].after_round();
      }
  }
  const sap_status_t sx = k[0].finish(info_x);
  sap_status_t sl = k[1].finish(info_lam);
  const sap_status_t sg = h->impl->adjoint_singular();
  if (sg != SAP_OK) sl = sg;
  return sx != SAP_OK ? sx : sl;
}

sap_status_t sap_solve_host(sap_handle_t h, const double* b_host, double* x_host, sap_info_t* info,
                            cudaStream_t s) {
  if (!h || !b_host || !x_host) return SAP_ERR_INVALID_ARG;
  const int64_t N = h->L.N;
  if (!h->host_stage) TRY(h->mem.alloc(&h->host_stage, (size_t)(2 * N)));
  double* xb = h->host_stage;
  CK(cudaMemcpyAsync(xb, b_host, N * sizeof(double), cudaMemcpyHostToDevice, s));
  sap_status_t st = krylov(h, xb, xb + N, false, info, s);
  CK(cudaMemcpyAsync(x_host, xb + N, N * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return st;
}

sap_status_t sap_factor_host(const double* band_host, int64_t N, int32_t K, const sap_options_t* opt,
                             cudaStream_t s, sap_handle_t* out) {
  if (!out) return SAP_ERR_INVALID_ARG;
  *out = nullptr;
  if (!band_host || !opt || N < 2 || K < 1 || K >= N) return SAP_ERR_INVALID_ARG;
  const size_t bytes = (size_t)(2 * (int64_t)K + 1) * (size_t)N * sizeof(double);
  double* d = nullptr;
  if (cudaMalloc(&d, bytes) != cudaSuccess) {
    cudaGetLastError();
    return SAP_ERR_OOM;
  }
  std::unique_ptr<double, cudaError_t (*)(void*)> guard(d, cudaFree);
  CK(cudaMemcpyAsync(d, band_host, bytes, cudaMemcpyHostToDevice, s));
  sap_handle_t h = nullptr;
  TRY(sap_factor(d, N, K, opt, s, &h));
  h->mem.ptrs.push_back(guard.release());     // freed with the handle
  h->band_owned = d;
  *out = h;
  return SAP_OK;
}

sap_status_t sap_refactor_host(sap_handle_t h, const double* band_host, cudaStream_t s) {
  if (!h || !band_host || !h->band_owned) return SAP_ERR_INVALID_ARG;
  const size_t bytes = (size_t)h->L.W * (size_t)h->L.N * sizeof(double);
  CK(cudaMemcpyAsync(h->band_owned, band_host, bytes, cudaMemcpyHostToDevice, s));
  return run_factor(h, s);
}

sap_status_t sap_solve_pair_host(sap_handle_t h, const double* b_host, const double* g_host, double* x_host,
                                 double* lam_host, sap_info_t* info_x, sap_info_t* info_lam, cudaStream_t s) {
  if (!h || !b_host || !g_host || !x_host || !lam_host || x_host == lam_host) return SAP_ERR_INVALID_ARG;
  const int64_t N = h->L.N;
  if (!h->host_stage4) TRY(h->mem.alloc(&h->host_stage4, (size_t)(4 * N)));
  double *db = h->host_stage4, *dg = db + N, *dx = dg + N, *dl = dx + N;
  CK(cudaMemcpyAsync(db, b_host, N * sizeof(double), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(dg, g_host, N * sizeof(double), cudaMemcpyHostToDevice, s));
  const sap_status_t st = sap_solve_pair(h, db, dx, dg, dl, info_x, info_lam, s);
  CK(cudaMemcpyAsync(x_host, dx, N * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(lam_host, dl, N * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return st;
}

sap_status_t sap_grad_band(sap_handle_t h, const double* lam, const double* x, double* g, cudaStream_t s) {
  if (!h || !lam || !x || !g) return SAP_ERR_INVALID_ARG;
  CK(launch_grad_band(lam, x, h->L.N, h->L.K, g, s));
  return SAP_OK;
}

sap_status_t sap_apply_preconditioner(sap_handle_t h, const double* r, double* z, int32_t transpose,
                                      cudaStream_t s) {
  if (!h || !r || !z || r == z) return SAP_ERR_INVALID_ARG;
  return h->impl->apply(r, z, transpose != 0, s);
}

sap_status_t sap_spmv(const double* band, int64_t N, int32_t K, const double* x, double* y, int32_t transpose,
                      cudaStream_t s) {
  if (!band || !x || !y || x == y || N < 1 || K < 0 || K >= N) return SAP_ERR_INVALID_ARG;
  CK(launch_spmv(band, N, K, x, y, transpose != 0, s));
  return SAP_OK;
}

sap_status_t sap_selftest_wait_timeout(int32_t spin_limit, cudaStream_t s) {
  if (spin_limit < 1) return SAP_ERR_INVALID_ARG;
  int* err = nullptr;
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return SAP_ERR_OOM;
  }
  int e = 0;
  sap_status_t st = SAP_OK;
  if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess ||
      launch_wait_selftest(spin_limit, err, s) != cudaSuccess ||
      cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    st = SAP_ERR_CUDA;
  cudaFree(err);
  if (st != SAP_OK) return st;
  return e ? SAP_ERR_TIMEOUT : SAP_OK;
}

int32_t sap_num_partitions(sap_handle_t h) { return h ? h->L.P : -1; }

sap_status_t sap_set_operator_csr(sap_handle_t h, int64_t n, int64_t nnz, const int64_t* rowptr_dev,
                                  const int32_t* col_dev, const double* val_dev, const int32_t* rownew_dev,
                                  const int32_t* colnew_dev, const double* rscale_dev, const double* cscale_dev) {
  if (!h) return SAP_ERR_INVALID_ARG;
  if (rowptr_dev && (n != h->L.N || nnz < 0 || !col_dev || !val_dev || (rscale_dev == nullptr) != (cscale_dev == nullptr)))
    return SAP_ERR_INVALID_ARG;
  // the captured iterations embed the previous operator's launches
  CK(cudaDeviceSynchronize());
  for (int g = 0; g < 4; ++g) {
    if (h->gexec[g]) cudaGraphExecDestroy(h->gexec[g]);
    if (h->wexec[g]) cudaGraphExecDestroy(h->wexec[g]);
    h->gexec[g] = h->wexec[g] = nullptr;
    h->gfailed[g] = h->wfailed[g] = false;
    h->glaunches[g] = h->wlaunches[g] = 0;
  }
  h->csr = sap::CsrOp{};
  if (rowptr_dev) {
    h->csr.n = n;
    h->csr.nnz = nnz;
    h->csr.rowptr = rowptr_dev;
    h->csr.col = col_dev;
    h->csr.val = val_dev;
    h->csr.rownew = rownew_dev;
    h->csr.colnew = colnew_dev;
    h->csr.r = rscale_dev;
    h->csr.s = cscale_dev;
  }
  return SAP_OK;
}

sap_status_t sap_get_partition(sap_handle_t h, int64_t* off) {
  if (!h || !off) return SAP_ERR_INVALID_ARG;
  std::memcpy(off, h->L.off.data(), (h->L.P + 1) * sizeof(int64_t));
  return SAP_OK;
}

sap_status_t sap_get_block_lu(sap_handle_t h, int32_t i, double* f, cudaStream_t s) {
  if (!h || !f || i < 0 || i >= h->L.P) return SAP_ERR_INVALID_ARG;
  return h->impl->block_lu(i, f, s);
}

sap_status_t sap_get_interface(sap_handle_t h, int32_t i, int32_t which, int32_t adjoint, double* m,
                               cudaStream_t s) {
  if (!h || !m) return SAP_ERR_INVALID_ARG;
  return h->impl->interface(i, which, adjoint != 0, m, s);
}

int64_t sap_n_boosted(sap_handle_t h) {
  if (!h) return -1;
  unsigned long long nb = 0;
  if (cudaMemcpy(&nb, h->n_boosted, sizeof(nb), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
  return (int64_t)nb;
}

sap_status_t sap_destroy(sap_handle_t h) {
  if (!h) return SAP_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  delete h;
  return SAP_OK;
}

const char* sap_status_string(sap_status_t s) {
  switch (s) {
    case SAP_OK: return "ok";
    case SAP_ERR_INVALID_ARG: return "invalid argument";
    case SAP_ERR_OOM: return "out of device memory";
    case SAP_ERR_NOT_CONVERGED: return "not converged";
    case SAP_ERR_BREAKDOWN: return "BiCGStab(2) breakdown";
    case SAP_ERR_TIMEOUT: return "device wait timed out";
    case SAP_ERR_CUDA: return "CUDA error";
    case SAP_ERR_NOT_IMPLEMENTED: return "not implemented for these sizes";
    case SAP_ERR_SINGULAR: return "singular reduced matrix";
  }
  return "unknown status";
}

sap_status_t sap_autotune(const double* band, int64_t N, int32_t K, const sap_options_t* opt_in,
                          const int32_t* P_cands, int32_t nP, const int32_t* seg_cands, int32_t nS,
                          const double* b_dev, cudaStream_t s, int32_t* best_P, int32_t* best_segments,
                          float* ms_out, int32_t* n_out) {
  if (!band || !opt_in || !best_P || !best_segments || N < 2 || K < 1 || K >= N) return SAP_ERR_INVALID_ARG;
  if (nP < 0 || nS < 0 || (nP > 0 && !P_cands) || (nS > 0 && !seg_cands)) return SAP_ERR_INVALID_ARG;
  const int64_t pmax = opt_in->variant == SAP_C ? std::max<int64_t>(1, N / (2 * (int64_t)K))
                                                : std::max<int64_t>(1, N / 64);
  std::vector<int32_t> Ps;
  if (nP > 0) {
    for (int32_t i = 0; i < nP && Ps.size() < 16; ++i)
      if (P_cands[i] >= 1 && P_cands[i] <= N) Ps.push_back(P_cands[i]);
  } else {
    for (int64_t rows : {16000, 8000, 4000, 2000, 1000}) {
      int64_t P = std::max<int64_t>(1, std::min<int64_t>(pmax, (N + rows / 2) / rows));
      if (std::find(Ps.begin(), Ps.end(), (int32_t)P) == Ps.end()) Ps.push_back((int32_t)P);
    }
    // one and two blocks per SM: whole waves of the one-CTA-per-block LU and sweeps
    for (int64_t P : {(int64_t)kSMs, 2 * (int64_t)kSMs})
      if (P <= pmax && std::find(Ps.begin(), Ps.end(), (int32_t)P) == Ps.end()) Ps.push_back((int32_t)P);
  }
  if (Ps.empty()) return SAP_ERR_INVALID_ARG;
  std::vector<int32_t> Ss;
  if (nS > 0) Ss.assign(seg_cands, seg_cands + nS);
  else Ss.push_back(0);
  if (n_out) *n_out = (int32_t)Ps.size();
  // right-hand side and solution buffers
  double* buf = nullptr;
  if (cudaMalloc(&buf, 3 * (size_t)N * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return SAP_ERR_OOM;
  }
  std::unique_ptr<double, cudaError_t (*)(void*)> guard(buf, cudaFree);
  double* ones = buf;
  double* bb = buf + N;
  double* xx = buf + 2 * N;
  if (!b_dev) {
    std::vector<double> h1((size_t)N, 1.0);
    CK(cudaMemcpyAsync(ones, h1.data(), (size_t)N * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(launch_spmv(band, N, K, ones, bb, false, s));
    CK(cudaStreamSynchronize(s));
    b_dev = bb;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = -1.f;
  sap_status_t last = SAP_ERR_INVALID_ARG;
  for (size_t i = 0; i < Ps.size(); ++i)
    for (size_t j = 0; j < Ss.size(); ++j) {
      sap_options_t o = *opt_in;
      o.P = Ps[i];
      o.segments = Ss[j];
      float ms = -1.f;
      sap_handle_t h = nullptr;
      sap_status_t st = sap_factor(band, N, K, &o, s, &h);
      if (st == SAP_OK) st = sap_solve(h, b_dev, xx, nullptr, s);       // warm-up, captures the graph
      for (int rep = 0; rep < 2 && st == SAP_OK; ++rep) {
        cudaEventRecord(e0, s);
        st = sap_refactor(h, s);
        if (st == SAP_OK) st = sap_solve(h, b_dev, xx, nullptr, s);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (st == SAP_OK && (ms < 0.f || t < ms)) ms = t;
      }
      if (h) sap_destroy(h);
      if (st != SAP_OK) {
        last = st;
        ms = -1.f;
      }
      if (ms_out) ms_out[i * Ss.size() + j] = ms;
      if (ms >= 0.f && (best < 0.f || ms < best)) {
        best = ms;
        *best_P = Ps[i];
        *best_segments = Ss[j];
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best >= 0.f ? SAP_OK : last;
}

sap_status_t sap_factor_batched(int32_t n, const double* const* bands, const int64_t* N, const int32_t* K,
                                const sap_options_t* opt, cudaStream_t s, sap_batch_t* out) {
  if (!out) return SAP_ERR_INVALID_ARG;
  *out = nullptr;
  if (n < 1 || !bands || !N || !K || !opt) return SAP_ERR_INVALID_ARG;
  int64_t total = 0;
  for (int32_t i = 0; i < n; ++i) {
    if (!bands[i] || N[i] < 2 || K[i] < 1 || K[i] >= N[i]) return SAP_ERR_INVALID_ARG;
    total += N[i];
  }
  std::unique_ptr<sap_batch> B(new (std::nothrow) sap_batch());
  if (!B) return SAP_ERR_OOM;
  for (int32_t i = 0; i < n; ++i) {
    sap_options_t o = *opt;
    if (o.P == 0) o.P = batch_partitions(N[i], K[i], total, o.variant);
    if (o.segments == 0) o.segments = 1;
    std::unique_ptr<sap_handle> h;
    TRY(create_handle(bands[i], N[i], K[i], &o, s, h));
    B->hs.push_back(h.release());
  }
  B->fp64 = opt->precision == SAP_FP64;
  TRY(build_work_list(B.get()));
  TRY(factor_batch(B.get(), s));
  *out = B.release();
  return SAP_OK;
}

sap_status_t sap_refactor_batched(sap_batch_t b, cudaStream_t s) {
  if (!b) return SAP_ERR_INVALID_ARG;
  return factor_batch(b, s);
}

sap_status_t sap_solve_batched(sap_batch_t b, const double* const* bv, double* const* xv, sap_info_t* infos,
                               int32_t* statuses, cudaStream_t s) {
  if (!b || !bv || !xv) return SAP_ERR_INVALID_ARG;
  return solve_batch(b, bv, xv, false, infos, statuses, s);
}

sap_status_t sap_solve_adjoint_batched(sap_batch_t b, const double* const* gv, double* const* lv,
                                       sap_info_t* infos, int32_t* statuses, cudaStream_t s) {
  if (!b || !gv || !lv) return SAP_ERR_INVALID_ARG;
  return solve_batch(b, gv, lv, true, infos, statuses, s);
}

sap_status_t sap_solve_pair_batched(sap_batch_t b, const double* const* bv, double* const* xv,
                                    const double* const* gv, double* const* lv, sap_info_t* infos_x,
                                    sap_info_t* infos_lambda, int32_t* statuses, cudaStream_t s) {
  if (!b || !bv || !xv || !gv || !lv) return SAP_ERR_INVALID_ARG;
  return solve_pair_batch(b, bv, xv, gv, lv, infos_x, infos_lambda, statuses, s);
}

sap_status_t sap_grad_band_batched(sap_batch_t b, const double* const* lam, const double* const* x,
                                   double* const* g, cudaStream_t s) {
  if (!b || !lam || !x || !g) return SAP_ERR_INVALID_ARG;
  for (size_t i = 0; i < b->hs.size(); ++i) TRY(sap_grad_band(b->hs[i], lam[i], x[i], g[i], s));
  return SAP_OK;
}

int32_t sap_batch_size(sap_batch_t b) { return b ? (int32_t)b->hs.size() : 0; }

int32_t sap_batch_partitions(sap_batch_t b, int32_t i) {
  if (!b || i < 0 || i >= (int32_t)b->hs.size()) return -1;
  return b->hs[i]->L.P;
}

sap_status_t sap_batch_destroy(sap_batch_t b) {
  if (!b) return SAP_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  delete b;
  return SAP_OK;
}

}  // extern "C"
