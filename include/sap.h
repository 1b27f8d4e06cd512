/*
 * sap.h — C ABI of libsap, a GB300-native (sm_103a) dense-banded
 * split-and-parallelize (SaP) solver: banded LU/UL block factorisation
 * without pivoting (boosted pivots), SaP-D / SaP-C preconditioning and an
 * outer BiCGStab(2), in FP64 or with an FP32 preconditioner (FP64 Krylov).
 *
 * Method: Li, Serban, Negrut, "Analysis of a splitting approach for the
 * parallel solution of linear systems on GPU cards", Sections 2.1-2.2
 * (method), 3.1 (storage, partition, LU/UL, mixed precision).
 *
 * Conventions shared by every entry point
 *   Band storage (Sec. 3.1 "Matrix storage"): the N x N matrix A with
 *     half-bandwidth K is an N x (2K+1) array in column-major order with the
 *     diagonal in column K, i.e. a_ij = band[(K + i - j) * N + j], 0-based,
 *     float64.  Slots whose row index i = j + c - K lies outside [0, N) are
 *     padding: never read, written as 0 where the library writes a band.
 *   Pointers named *_dev are device pointers on the current CUDA device;
 *     pointers named *_host are host pointers.  Vectors are float64, length N.
 *   Streams: every call is ordered on the given stream (0 = legacy default).
 *     Calls that return solver status synchronise that stream before they
 *     return; the others are asynchronous.
 *   Errors: no call throws or aborts; each returns a sap_status_t.  On an
 *     error the output buffers hold unspecified values and the handle stays
 *     usable unless the status is SAP_ERR_CUDA.
 *   Threading: a handle must not be used from two host threads at once.
 */
#ifndef SAP_H
#define SAP_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#if defined(__GNUC__)
#define SAP_API __attribute__((visibility("default")))
#else
#define SAP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sap_handle *sap_handle_t;

typedef enum {
    SAP_OK = 0,
    SAP_ERR_INVALID_ARG = 1,   /* bad size or option, see each call */
    SAP_ERR_OOM = 2,           /* device allocation failed */
    SAP_ERR_NOT_CONVERGED = 3, /* iteration cap reached; x holds the last iterate */
    SAP_ERR_BREAKDOWN = 4,     /* BiCGStab(2) scalar rho, gamma, sigma or omega became 0 */
    SAP_ERR_TIMEOUT = 5,       /* a device-side wait hit its spin limit */
    SAP_ERR_CUDA = 6,          /* a CUDA runtime call failed */
    SAP_ERR_NOT_IMPLEMENTED = 7,
    SAP_ERR_SINGULAR = 8       /* an exactly singular reduced matrix Rbar_i */
} sap_status_t;

typedef enum { SAP_D = 0, SAP_C = 1 } sap_variant_t;          /* Sec. 2.1.1 */
/* Sec. 3.1 mixed precision.  SAP_FP32_BF16TU (a GB300 addition): FP32 factors
 * whose block LU/UL trailing updates (the rank-16 products of each 16-column
 * panel) run on the tensor cores with BF16 operands (RN) and FP32
 * accumulation, for K >= 64 as long as the factor window stays in shared
 * memory with the operand buffers (K <= 192); elsewhere it equals SAP_FP32
 * (sap_info_t.tc_update reports which ran).  Pivots, panels, tips, sweeps and
 * everything FP64 as with SAP_FP32.  The factors carry BF16-level error and
 * the FP64 BiCGStab(2) makes up for it, with more iterations where the
 * preconditioner is sensitive to it. */
typedef enum { SAP_FP64 = 0, SAP_FP32 = 1, SAP_FP32_BF16TU = 2 } sap_precision_t;

/* Outer Krylov iteration (Sec. 3): BiCGStab(2) with left preconditioning, or,
 * for a symmetric positive definite A, the preconditioned conjugate gradient
 * method (Saad 2003, Alg. 9.1) with the SaP factorisation as M.  CG counts
 * whole iterations (one SpMV and one preconditioner application each; iters
 * in sap_info_t is then an integer), exits on ||b - A x|| <= tol ||b|| by its
 * recursive residual confirmed by the true one, and restarts from the
 * current x when the confirmation fails.  SaP-D's M is SPD for SPD A;
 * SaP-C's truncated-spike M need not be symmetric.  Both run device-driven
 * (every launch gated on device flags; a round, one BiCGStab(2) iteration or
 * four CG steps, is one captured CUDA graph): the whole loop is one launch of
 * a graph whose conditional WHILE node repeats the round until the device
 * flags the exit or the iteration cap, with one host readback at the end;
 * where such a graph cannot be built, the round's graph is replayed with one
 * host readback per round.  sap_solve_pair and the batch calls run either. */
typedef enum { SAP_KRYLOV_BICGSTAB2 = 0, SAP_KRYLOV_CG = 1 } sap_krylov_t;

typedef struct {
    int32_t P;            /* number of diagonal blocks, 1 <= P <= N (Sec. 3.1); 0 makes
                             sap_factor run sap_autotune over its default candidates
                             first and use the fastest P (and, if segments is 0, the
                             fastest segment count); sap_num_partitions tells which */
    int32_t variant;      /* sap_variant_t */
    int32_t precision;    /* sap_precision_t: precision of factors, tips and sweeps;
                             the Krylov vectors, SpMV, dot products, the true
                             residual and the reduced systems Rbar_i are FP64 */
    int32_t max_iters;    /* Krylov iteration cap (default 500 if <= 0) */
    double tol;           /* target ||b - A x||_2 / ||b||_2 (default 1e-10 if <= 0) */
    double boost_eps;     /* relative pivot-boost threshold (Sec. 2.2): a pivot with
                             |p| < boost_eps * max|a_ij| becomes sign(p) times that
                             value; <= 0 selects the unit roundoff of `precision` */
    int64_t spin_limit;   /* polls a bounded device-side wait makes before it gives
                             up (0 = default, 2^24; values above 2^31 - 1 are
                             clamped).  A wait that gives up stops the kernel's
                             further copies, drains those in flight, lets the kernel
                             finish with unspecified values, and the call returns
                             SAP_ERR_TIMEOUT.  A poll is one non-blocking mbarrier
                             test in the sweeps and one mbarrier try_wait (which may
                             suspend the thread for a hardware-defined time) in the
                             tensor-core factorisation.  No counterpart in the paper. */
    int32_t segments;     /* sweep segments per block (0 = automatic, 1 = none): the
                             two banded triangular sweeps of every block are split
                             into this many consecutive row ranges that run on
                             separate CTAs, in two passes (zero history, then the
                             true history carried over by the precomputed transfer
                             matrices of the ranges); the same operator as one
                             sequential sweep up to rounding.  The paper sweeps each
                             block with one thread block; this is a GB300 addition
                             to fill the SMs when P is small.  Values that leave a
                             range shorter than ceil(K/32) chunks of 32 rows are
                             lowered automatically; segmentation needs K <= 512
                             with FP32 factors, K <= 256 with FP64 (1 above);
                             the automatic count uses it for K <= 128 only. */
    int32_t krylov;       /* sap_krylov_t: the outer iteration */
} sap_options_t;

typedef struct {
    double iters;         /* BiCGStab(2) iterations in quarters (Sec. 4.1.1); CG: whole */
    double relres;        /* final true ||b - A x||_2 / ||b||_2 (FP64) */
    int64_t n_boosted;    /* boosted pivots in all LU and UL factorisations */
    int64_t n_matvec;     /* preconditioned matvecs M^{-1} A v of the iteration: 4 per
                             outer iteration, 1 or 3 in one that exits early (= 4 iters).
                             Not counted: the first apply M^{-1} b, the SpMV of each
                             true-residual check, and the SpMV + apply of a restart */
    int64_t n_restarts;   /* restarts from the current x after a true-residual check that
                             failed behind the MR update (one SpMV + one apply each) */
    float t_factor_ms;    /* device time of the last factorisation (all phases) */
    float t_solve_ms;     /* device time of the Krylov phase of the last solve */
    float t_lu_ms;        /* T_LU (Sec. 4.3.2 breakdown): the block LU kernel */
    float t_ul_ms;        /* SaP-C: block UL (top tiles only) */
    float t_spk_ms;       /* SaP-C T_SPK: spike tips V^(b)_i, W^(t)_{i+1}; where the K x K
                             matrices fit in shared memory one kernel per interface also
                             forms Rbar_i, its GEPP and inverse, and they count here */
    int32_t segments;     /* sweep segments per block in use (sap_options_t.segments) */
    int32_t graphed;      /* 1 if the iterations ran from captured CUDA graphs (the device loop or per-round replays) */
    int32_t tc_update;    /* 1 if the block LU/UL trailing updates ran on the tensor cores */
    int32_t P;            /* partition count in use (the autotuner's choice when P = 0) */
    float t_bc_ms;        /* SaP-C T_BC (Sec. 4.3.2 breakdown): 0, B_i and C_{i+1} are read in
                             place from the band by the tip and reduced-solve kernels */
    float t_rdcd_ms;      /* SaP-C T_LUrdcd: forming Rbar_i, its GEPP and explicit inverse
                             (0 where fused into the tip kernel, see t_spk_ms) */
    float t_kry_ms;       /* T_Kry: device time of the Krylov phase (= t_solve_ms) */
    float t_prep_ms;      /* the rest of the LU phase (GB300 additions): the boost-threshold
                             pass with the FP32 cast of the band, and the sweeps' per-chunk
                             inverse / coupling and segment transfer matrices */
    int32_t reserved1;    /* 0 */
} sap_info_t;

/* Defaults as documented above. */
SAP_API void sap_default_options(sap_options_t *opt);

/* Factor the SaP preconditioner of A (Sec. 2.1, 3.1): partition into P
 * blocks, LU of every block A_i; for SaP-C also the UL of every block, the
 * coupling blocks B_i, C_{i+1}, the spike tips V^(b)_i, W^(t)_{i+1}
 * (Eq. (2.2) via the bottom LU / top UL blocks) and the reduced matrices
 * Rbar_i = I - W^(t)_{i+1} V^(b)_i factored by partial pivoting (Eq. (2.5a)).
 *   band_dev: device band of A (borrowed: it must stay allocated and
 *             unchanged until sap_destroy, the SpMV reads it).
 *   N >= 2, 1 <= K < N.  SaP-C needs every block to have >= 2K rows.
 *   *out receives a new handle owning all other device memory.
 * Errors: INVALID_ARG (sizes, options, N_i < 2K for SaP-C), NOT_IMPLEMENTED
 * (K above sap_max_K), OOM, SINGULAR, TIMEOUT (a bounded device wait of the
 * tensor-core factorisation gave up), CUDA.  Synchronises `stream`; with
 * P = 0 it first factors and solves once per autotuner candidate. */
SAP_API sap_status_t sap_factor(const double *band_dev, int64_t N, int32_t K,
                        const sap_options_t *opt, cudaStream_t stream,
                        sap_handle_t *out);

/* Recompute the factorisation in place after the values of the borrowed
 * band changed (same N, K, options; no allocation).  The adjoint reduced
 * matrices are rebuilt on the next adjoint call.  Synchronises `stream`. */
SAP_API sap_status_t sap_refactor(sap_handle_t h, cudaStream_t stream);

/* Solve A x = b by left-preconditioned BiCGStab(2) (Sec. 2.1.1) from
 * x0 = 0 to the handle's tolerance.  b_dev, x_dev: device, length N, must
 * not alias.  info may be NULL.  Synchronises `stream`. */
SAP_API sap_status_t sap_solve(sap_handle_t h, const double *b_dev, double *x_dev,
                       sap_info_t *info, cudaStream_t stream);

/* The forward solve A x = b and the adjoint solve A^T lambda = gbar
 * together (a GB300 addition, for a gbar that does not depend on x, e.g. the
 * gradient of a linear functional w^T x): the two BiCGStab(2) iterations run
 * concurrently on two internal streams with separate Krylov workspaces (the
 * second allocated on the first call) and separate apply scratch, in lockstep
 * rounds with one host synchronisation per round for both.  Each result is
 * what sap_solve / sap_solve_adjoint return for it.  No two of b, x, gbar,
 * lambda may alias (b and gbar may be the same array).  Returns the first
 * non-OK status (forward first).  Synchronises `stream`. */
SAP_API sap_status_t sap_solve_pair(sap_handle_t h, const double *b_dev, double *x_dev, const double *gbar_dev,
                                    double *lambda_dev, sap_info_t *info_x, sap_info_t *info_lambda,
                                    cudaStream_t stream);

/* Solve A^T lambda = gbar with the same machinery on A^T: SpMV with A^T and
 * SaP on A^T built from the stored factors transposed (A_i^T = U_i^T L_i^T;
 * couplings B'_i = C_{i+1}^T, C'_{i+1} = B_i^T; its own reduced matrices,
 * built on the first call).  Synchronises `stream`. */
SAP_API sap_status_t sap_solve_adjoint(sap_handle_t h, const double *gbar_dev, double *lambda_dev,
                               sap_info_t *info, cudaStream_t stream);

/* grad_band = -lambda x^T restricted to the band (the gradient of a scalar
 * loss l(x), x = A^{-1} b, with respect to the band entries, given
 * lambda = A^{-T} dl/dx); padding slots are written as 0.  grad_band_dev has
 * (2K+1) N float64.  Asynchronous. */
SAP_API sap_status_t sap_grad_band(sap_handle_t h, const double *lambda_dev, const double *x_dev,
                           double *grad_band_dev, cudaStream_t stream);

/* One preconditioner application z = M^{-1} r (transpose = 0) or the SaP
 * preconditioner of A^T (transpose = 1): SaP-D Eq. (2.3), SaP-C Eq. (2.5)
 * plus purification (Sec. 2.1).  Asynchronous. */
SAP_API sap_status_t sap_apply_preconditioner(sap_handle_t h, const double *r_dev, double *z_dev,
                                      int32_t transpose, cudaStream_t stream);

/* y = A x (transpose = 0) or y = A^T x (transpose = 1) on the band, FP64.
 * Stateless; x and y must not alias.  Asynchronous. */
SAP_API sap_status_t sap_spmv(const double *band_dev, int64_t N, int32_t K, const double *x_dev,
                      double *y_dev, int32_t transpose, cudaStream_t stream);

/* Solve with host buffers: copies b_host to the device, runs sap_solve and
 * copies x back into x_host (host <-> device copies included). */
SAP_API sap_status_t sap_solve_host(sap_handle_t h, const double *b_host, double *x_host,
                            sap_info_t *info, cudaStream_t stream);

/* Host-buffer forms of sap_factor, sap_refactor and sap_solve_pair (a GB300
 * addition for callers whose data lives in host memory; page-locked buffers
 * copy fastest).  sap_factor_host copies band_host ((2K+1) N float64, the
 * layout above) into device memory that the handle owns and factors it;
 * sap_refactor_host copies new band values into that memory and refactors
 * (INVALID_ARG for a handle made by sap_factor, whose band is borrowed);
 * sap_solve_pair_host copies b_host and g_host in, runs sap_solve_pair and
 * copies x and lambda back (device staging of 4 N doubles allocated on the
 * first call).  Each synchronises `stream`; errors as the device forms. */
SAP_API sap_status_t sap_factor_host(const double *band_host, int64_t N, int32_t K,
                                     const sap_options_t *opt, cudaStream_t stream, sap_handle_t *out);
SAP_API sap_status_t sap_refactor_host(sap_handle_t h, const double *band_host, cudaStream_t stream);
SAP_API sap_status_t sap_solve_pair_host(sap_handle_t h, const double *b_host, const double *g_host,
                                         double *x_host, double *lam_host, sap_info_t *info_x,
                                         sap_info_t *info_lambda, cudaStream_t stream);

/* Inspection of the factorisation, for tests.  Copies into host buffers.
 *   sap_get_partition: off_host[P+1] block offsets.
 *   sap_get_block_lu:  LU of block i as a dense-band row-major n_i x (2K+1)
 *     float64 array f[r*(2K+1) + (c - r + K)] (unit L below, U on/above).
 *   sap_get_interface: K x K row-major float64 matrix of interface i
 *     (0 <= i < P-1): which 0 = B_i, 1 = C_{i+1}, 2 = V^(b)_i,
 *     3 = W^(t)_{i+1}, 4 = Rbar_i before factoring; adjoint = 1 gives the
 *     matrices of the SaP preconditioner of A^T (built on demand).
 * Synchronise `stream`. */
SAP_API sap_status_t sap_get_partition(sap_handle_t h, int64_t *off_host);
SAP_API sap_status_t sap_get_block_lu(sap_handle_t h, int32_t i, double *f_host, cudaStream_t stream);
SAP_API sap_status_t sap_get_interface(sap_handle_t h, int32_t i, int32_t which, int32_t adjoint,
                               double *m_host, cudaStream_t stream);

/* Partition count P of the handle (the autotuner's choice when the options
 * asked for P = 0), or -1 for a NULL handle. */
SAP_API int32_t sap_num_partitions(sap_handle_t h);

/* Number of boosted pivots so far (LU and UL). */
SAP_API int64_t sap_n_boosted(sap_handle_t h);

/* Release the handle and its device memory (synchronises the device). */
SAP_API sap_status_t sap_destroy(sap_handle_t h);

/* Static description of a status code. */
SAP_API const char *sap_status_string(sap_status_t s);

/* Direct banded solve A x = b that allocates no device memory.  There is no
 * counterpart in the paper: it exists for callers that cannot call
 * cudaMalloc (cudaMalloc may synchronise the device, which latency-critical
 * loops cannot afford, and some host programs own all device memory and
 * forbid new driver allocations).  It runs the kernels of sap_factor with
 * P = 1, SaP-D, followed by sap_apply_preconditioner: one banded LU without
 * pivoting (pivots boosted at the unit roundoff of `precision` times
 * max|a_ij|) and the forward and backward sweeps, so x = A^{-1} b up to the
 * factorisation's rounding; no Krylov iteration.
 *   All intermediates live in one file-scope device array of 32 MiB that
 *   every GPU loading the library holds until the process exits.  With
 *   n = N rounded up to 32, s = sizeof(factor) (8 for SAP_FP64, 4 for
 *   SAP_FP32) and r(x) = x rounded up to a multiple of 256, the call needs
 *     256 + r(n (2K+1) s)                     factors
 *         + 2 r(n 32 (1 + ceil(K/32)) s)      chunk matrices of the two sweeps
 *         + r((2N + 2K + 8) 8)                sweep scratch
 *         + r(N (2K+1) 4)                     FP32 only: the FP32 copy of the band
 *         + r(M (M + 4) s)                    K > 208 (FP32) or K > 128 (FP64) only:
 *                                             the factor window, M = K + 16 rounded up to 16
 *   bytes and returns SAP_ERR_INVALID_ARG beyond 2^25.  Examples: K = 25 fits
 *   up to N = 23,168 in FP64 and N = 35,840 in FP32.
 *   The caller provides band_dev, b_dev and x_dev (device, float64) and,
 *   optionally, timeout_dev: a device int32 that receives, in stream order,
 *   1 if one of the call's bounded device waits gave up (x then holds
 *   unspecified values) and 0 otherwise; read it once the stream has
 *   completed.  With timeout_dev = NULL a timeout goes unreported.
 *   The first call on a device also looks up the array's device address
 *   (a host-side runtime query, made once per device).
 *   Every call uses the same array and overwrites the previous call's
 *   contents, so calls that overlap on the GPU (other streams or threads)
 *   race; order them on one stream.  Asynchronous on `stream`.
 * Errors: INVALID_ARG (sizes, null or aliased pointers, too large for the
 * array), NOT_IMPLEMENTED (K above sap_max_K), CUDA. */
SAP_API sap_status_t sap_band_solve_noalloc(const double *band_dev, int64_t N, int32_t K,
                                           const double *b_dev, double *x_dev, int32_t precision,
                                           int32_t *timeout_dev, cudaStream_t stream);

/* ---- Autotuner ----
 * Not in the paper (a GB300 addition): picks the partition count P and the
 * sweep segment count for one matrix by measurement.  Every candidate
 * (P_cands[i], seg_cands[j]) is factored and solved (refactor + solve timed
 * with CUDA events on `stream`, best of two) and the fastest is returned.
 *   opt: the other options (variant, precision, tol, ...); opt->P and
 *        opt->segments are ignored.
 *   P_cands, nP: candidate partition counts; nP == 0 uses N / {16000, 8000,
 *        4000, 2000, 1000} rounded, clipped to [1, N/64] (SaP-D) or
 *        [1, N/(2K)] (SaP-C), then 152 and 304 (one and two blocks per SM
 *        of a GB300) where within that bound, duplicates removed.
 *   seg_cands, nS: candidate segment counts; nS == 0 uses {0} (automatic).
 *   b_dev: right-hand side for the timing (N doubles on the device), or NULL
 *        for b = A * ones.
 *   ms_out (optional, nP' x nS entries in candidate order, nP' = the number of
 *        P candidates actually used, at most 16): measured ms, -1 for a
 *        candidate that failed; n_out (optional) receives nP'.
 * Errors: INVALID_ARG, or the status of the last candidate when all fail.
 * Synchronises; allocates and frees one handle per candidate. */
SAP_API sap_status_t sap_autotune(const double *band_dev, int64_t N, int32_t K, const sap_options_t *opt,
                                  const int32_t *P_cands, int32_t nP, const int32_t *seg_cands, int32_t nS,
                                  const double *b_dev, cudaStream_t stream, int32_t *best_P,
                                  int32_t *best_segments, float *ms_out, int32_t *n_out);

/* ---- Batches of independent banded systems ----
 * Not in the paper (a GB300 addition): n systems of their own N_i and K_i,
 * each with its own SaP preconditioner, factored and solved together.  Every
 * system runs on its own internal stream, so their kernels overlap on the
 * GPU; a batched solve launches every unfinished system's device-driven
 * Krylov loop (see sap_krylov_t; where it cannot run, one outer iteration per
 * round, a replay of the system's captured graph) and synchronises the host
 * once per round for the whole batch.
 *   opt applies to every system; opt->P == 0 picks P_i per system so that
 *   the batch has about two blocks per SM in total, P_i in proportion to N_i
 *   (at least 1; SaP-C keeps N_i / P_i >= 2 K_i); opt->segments == 0 means
 *   unsegmented sweeps (the batch already fills the SMs).
 *   bands_dev[i]: device band of system i (borrowed, as for sap_factor).
 * Errors: as sap_factor, for the first system that fails (nothing is
 * returned then). */
typedef struct sap_batch *sap_batch_t;
SAP_API sap_status_t sap_factor_batched(int32_t n, const double *const *bands_dev, const int64_t *N,
                                        const int32_t *K, const sap_options_t *opt, cudaStream_t stream,
                                        sap_batch_t *out);
/* Refactor every system after its band values changed (no allocation). */
SAP_API sap_status_t sap_refactor_batched(sap_batch_t b, cudaStream_t stream);
/* Solve A_i x_i = b_i (or A_i^T lambda_i = g_i) for all i.  infos and
 * statuses (per system, optional) receive each solve's report and status;
 * the return value is SAP_OK or the first failing status.  Synchronises. */
SAP_API sap_status_t sap_solve_batched(sap_batch_t b, const double *const *b_dev, double *const *x_dev,
                                       sap_info_t *infos, int32_t *statuses, cudaStream_t stream);
SAP_API sap_status_t sap_solve_adjoint_batched(sap_batch_t b, const double *const *g_dev,
                                               double *const *lambda_dev, sap_info_t *infos,
                                               int32_t *statuses, cudaStream_t stream);
/* Every system's forward and adjoint solve together (as sap_solve_pair, all
 * 2n iterations in the same lockstep rounds).  statuses (optional) has 2n
 * entries: the forward solves, then the adjoint ones.  Synchronises. */
SAP_API sap_status_t sap_solve_pair_batched(sap_batch_t b, const double *const *b_dev, double *const *x_dev,
                                            const double *const *g_dev, double *const *lambda_dev,
                                            sap_info_t *infos_x, sap_info_t *infos_lambda, int32_t *statuses,
                                            cudaStream_t stream);
/* grad_band_i = -lambda_i x_i^T restricted to the band of system i. */
SAP_API sap_status_t sap_grad_band_batched(sap_batch_t b, const double *const *lambda_dev,
                                           const double *const *x_dev, double *const *grad_band_dev,
                                           cudaStream_t stream);
/* Number of systems, and the partition count chosen for system i (-1 if out of range). */
SAP_API int32_t sap_batch_size(sap_batch_t b);
SAP_API int32_t sap_batch_partitions(sap_batch_t b, int32_t i);
SAP_API sap_status_t sap_batch_destroy(sap_batch_t b);

/* Failure-detection self-test (not in the paper; the device-side waits of
 * this library are bounded): launches one CTA whose thread waits, with the
 * same bounded mbarrier wait the sweep and factor kernels use, on a barrier
 * that nothing completes, polling `spin_limit` times.  Returns
 * SAP_ERR_TIMEOUT when the wait gave up and reported it (the expected
 * outcome; the CUDA context stays usable), SAP_OK if the wait completed (a
 * defect), INVALID_ARG for spin_limit < 1, OOM, CUDA.  Synchronises
 * `stream`; allocates and frees one device int. */
SAP_API sap_status_t sap_selftest_wait_timeout(int32_t spin_limit, cudaStream_t stream);

/* Number of CUDA kernels this library has launched in this process so far
 * (host-side counter, all handles and threads). */
SAP_API int64_t sap_kernel_launches(void);

/* Largest half-bandwidth K this build factors, per precision (both variants):
 * 512 with FP32 factors, 256 with FP64 factors.  The limit is the sweep's
 * shared-memory ring of per-chunk matrices; factor windows and spike
 * workspaces that exceed shared memory move to global memory. */
SAP_API int32_t sap_max_K(int32_t precision);

#ifdef __cplusplus
}
#endif
#endif /* SAP_H */
