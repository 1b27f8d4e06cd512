/*
 * Plain FP64 CPU oracle of the dense-banded split-and-parallelize (SaP) solver
 * (Li, Serban, Negrut, "Analysis of a splitting approach for the parallel
 * solution of linear systems on GPU cards").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA path is checked against.  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may load it; the product
 * path never does.  It shares no code, header or helper with the CUDA path.
 *
 * Everything is double precision, written as plain loops in the order the
 * paper states each step, and single threaded as built for the tests.  The
 * loops over the independent diagonal blocks carry OpenMP pragmas: a second
 * build with -fopenmp (the CPU baseline's multi-core leg) runs the blocks in
 * parallel with every block's arithmetic unchanged, so its results are bit
 * for bit those of the single-threaded build; the vector reductions of the
 * Krylov loops stay sequential.  Where the paper is silent the reading used
 * is stated next to the code.
 *
 * Conventions
 *   - Band storage (Section 3.1, "Matrix storage"): an N x (2K+1) array in
 *     column-major order with the diagonal in column K, i.e.
 *     a_ij = band[(K + i - j) * N + j], 0-based.
 *   - Partition (Section 3.1, "Number of partitions and partition size"):
 *     the first P_r blocks have floor(N/P)+1 rows, the rest floor(N/P), with
 *     N = P floor(N/P) + P_r.
 *   - Block factors are kept in a private dense-band row-major array:
 *     element (r, c) of a block (local indices, |r - c| <= K) is
 *     f[r * W + (c - r + K)], W = 2K+1.  LU: unit lower L strictly below the
 *     diagonal, U on and above it.  UL: unit upper U' strictly above the
 *     diagonal, L' on and below it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_INVALID_ARG 1
#define ORC_ERR_OOM 2
#define ORC_ERR_NOT_CONVERGED 3
#define ORC_ERR_BREAKDOWN 4
#define ORC_ERR_SINGULAR 8

/* ------------------------------------------------------------------ */
/* band access                                                          */
/* ------------------------------------------------------------------ */

/* a_ij of the band, 0 outside the band or the matrix (Section 3.1). */
static double band_get(const double *band, int64_t N, int K, int64_t i, int64_t j)
{
    if (i < 0 || j < 0 || i >= N || j >= N) return 0.0;
    int64_t c = (int64_t)K + i - j;
    if (c < 0 || c > 2 * (int64_t)K) return 0.0;
    return band[c * N + j];
}

/* ------------------------------------------------------------------ */
/* partition (Section 3.1)                                              */
/* ------------------------------------------------------------------ */

void orc_partition(int64_t N, int32_t P, int64_t *offsets)
{
    int64_t q = N / P, pr = N - (int64_t)P * q;
    offsets[0] = 0;
    for (int32_t i = 0; i < P; ++i)
        offsets[i + 1] = offsets[i] + q + (i < pr ? 1 : 0);
}

/* ------------------------------------------------------------------ */
/* matrix-vector products on the band                                   */
/* ------------------------------------------------------------------ */

/* y = A x (transpose = 0) or y = A^T x (transpose = 1). */
void orc_spmv(const double *band, int64_t N, int K, const double *x, double *y, int transpose)
{
    for (int64_t i = 0; i < N; ++i) {
        double s = 0.0;
        int64_t lo = i - K < 0 ? 0 : i - K, hi = i + K >= N ? N - 1 : i + K;
        for (int64_t j = lo; j <= hi; ++j)
            s += (transpose ? band_get(band, N, K, j, i) : band_get(band, N, K, i, j)) * x[j];
        y[i] = s;
    }
}

/* ------------------------------------------------------------------ */
/* block LU / UL without pivoting, with pivot boosting (Section 2.2)    */
/* ------------------------------------------------------------------ */

#define F(f, W, K, r, c) ((f)[(int64_t)(r) * (W) + ((c) - (r) + (K))])

/* Pivot boosting: a pivot with |p| < tau is replaced by sign(p) * tau,
 * sign(0) = +1 (reading of the boosting rule of Section 2.2). */
static double boost(double p, double tau, int64_t *nb)
{
    if (fabs(p) < tau) {
        ++*nb;
        return p >= 0.0 ? tau : -tau;
    }
    return p;
}

/* Copy block [s, s+n) of the band into private dense-band storage f. */
static void load_block(const double *band, int64_t N, int K, int64_t s, int64_t n, double *f)
{
    int W = 2 * K + 1;
    for (int64_t r = 0; r < n; ++r)
        for (int d = -K; d <= K; ++d) {
            int64_t c = r + d;
            f[r * W + (d + K)] = (c >= 0 && c < n) ? band_get(band, N, K, s + r, s + c) : 0.0;
        }
}

/* Right-looking Doolittle LU restricted to the band: A_i = L_i U_i with unit
 * lower L.  Returns the number of boosted pivots. */
int64_t orc_block_lu(double *f, int64_t n, int K, double tau)
{
    int W = 2 * K + 1;
    int64_t nb = 0;
    for (int64_t k = 0; k < n; ++k) {
        double p = boost(F(f, W, K, k, k), tau, &nb);
        F(f, W, K, k, k) = p;
        int64_t last = k + K < n - 1 ? k + K : n - 1;
        for (int64_t i = k + 1; i <= last; ++i)
            F(f, W, K, i, k) /= p;
        for (int64_t i = k + 1; i <= last; ++i) {
            double lik = F(f, W, K, i, k);
            for (int64_t j = k + 1; j <= last; ++j)
                F(f, W, K, i, j) -= lik * F(f, W, K, k, j);
        }
    }
    return nb;
}

/* UL factorisation A_i = U'_i L'_i with unit upper U' (Section 2.1, the
 * "additional UL factorization"): the same elimination run from the last
 * row/column upwards. */
int64_t orc_block_ul(double *f, int64_t n, int K, double tau)
{
    int W = 2 * K + 1;
    int64_t nb = 0;
    for (int64_t k = n - 1; k >= 0; --k) {
        double p = boost(F(f, W, K, k, k), tau, &nb);
        F(f, W, K, k, k) = p;
        int64_t first = k - K > 0 ? k - K : 0;
        for (int64_t i = first; i < k; ++i)
            F(f, W, K, i, k) /= p;
        for (int64_t i = first; i < k; ++i) {
            double uik = F(f, W, K, i, k);
            for (int64_t j = first; j < k; ++j)
                F(f, W, K, i, j) -= uik * F(f, W, K, k, j);
        }
    }
    return nb;
}

/* ------------------------------------------------------------------ */
/* small dense helpers (K x K, row-major)                               */
/* ------------------------------------------------------------------ */

/* LU with partial pivoting, ties to the lowest row index.  piv[k] = row
 * swapped with k.  Returns 0 or ORC_ERR_SINGULAR on an exact zero pivot. */
int orc_dense_getrf(double *a, int n, int32_t *piv)
{
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(a[k * n + k]);
        for (int i = k + 1; i < n; ++i)
            if (fabs(a[i * n + k]) > best) { best = fabs(a[i * n + k]); p = i; }
        piv[k] = p;
        if (best == 0.0) return ORC_ERR_SINGULAR;
        if (p != k)
            for (int j = 0; j < n; ++j) { double t = a[k * n + j]; a[k * n + j] = a[p * n + j]; a[p * n + j] = t; }
        for (int i = k + 1; i < n; ++i) {
            a[i * n + k] /= a[k * n + k];
            double l = a[i * n + k];
            for (int j = k + 1; j < n; ++j) a[i * n + j] -= l * a[k * n + j];
        }
    }
    return 0;
}

/* Solve with the output of orc_dense_getrf, one right-hand side in place. */
void orc_dense_getrs(const double *a, int n, const int32_t *piv, double *x)
{
    for (int k = 0; k < n; ++k)
        if (piv[k] != k) { double t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < i; ++j) x[i] -= a[i * n + j] * x[j];
    for (int i = n - 1; i >= 0; --i) {
        for (int j = i + 1; j < n; ++j) x[i] -= a[i * n + j] * x[j];
        x[i] /= a[i * n + i];
    }
}

/* ------------------------------------------------------------------ */
/* the SaP preconditioner object                                        */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t N;
    int K, P, variant;        /* variant 0 = SaP-D, 1 = SaP-C */
    double tau;
    int64_t *off;             /* P+1 block offsets */
    double **lu;              /* per block: LU in dense-band storage */
    double **ul;              /* per block (SaP-C): UL in dense-band storage */
    /* per interface i = 0..P-2 (between blocks i and i+1), K x K row-major */
    double **B, **C;          /* B_i (block i -> i+1), C_{i+1} (block i+1 -> i) */
    double **V, **Wt;         /* V^(b)_i, W^(t)_{i+1} */
    double **R;               /* Rbar_i, LU-factored in place after orc_factor */
    double **R0;              /* Rbar_i before factoring (kept for tests) */
    int32_t **piv;
    int64_t n_boosted;
} orc_sap;

static void *xcalloc(size_t n, size_t s) { return calloc(n ? n : 1, s ? s : 1); }

void orc_free(orc_sap *h)
{
    if (!h) return;
    for (int i = 0; i < h->P; ++i) {
        if (h->lu) free(h->lu[i]);
        if (h->ul) free(h->ul[i]);
    }
    for (int i = 0; i + 1 < h->P; ++i) {
        if (h->B) free(h->B[i]);
        if (h->C) free(h->C[i]);
        if (h->V) free(h->V[i]);
        if (h->Wt) free(h->Wt[i]);
        if (h->R) free(h->R[i]);
        if (h->R0) free(h->R0[i]);
        if (h->piv) free(h->piv[i]);
    }
    free(h->lu); free(h->ul); free(h->B); free(h->C); free(h->V); free(h->Wt);
    free(h->R); free(h->R0); free(h->piv); free(h->off);
    free(h);
}

/* Spike tips of interface i (Section 2.1, computational savings paragraph):
 *   V^(b)_i     = U_bb^{-1} L_bb^{-1} B_i      (bottom K x K blocks of L_i, U_i)
 *   W^(t)_{i+1} = L'_tt^{-1} U'_tt^{-1} C_{i+1} (top K x K blocks of U'_{i+1}, L'_{i+1})
 * which are the bottom K rows of V_i and the top K rows of W_{i+1} in
 * Eq. (2.2). */
static void spike_tips(const orc_sap *h, int i)
{
    int K = h->K, W = 2 * K + 1;
    const double *lu = h->lu[i];
    int64_t n = h->off[i + 1] - h->off[i];
    int64_t b0 = n - K;                         /* first row of the bottom block */
    const double *ul = h->ul[i + 1];
    double *V = h->V[i], *Wt = h->Wt[i];
    for (int col = 0; col < K; ++col) {
        /* V: forward with unit L_bb, then backward with U_bb */
        double y[K > 0 ? K : 1];
        for (int r = 0; r < K; ++r) {
            double s = h->B[i][r * K + col];
            for (int q = 0; q < r; ++q)
                if (r - q <= K) s -= F(lu, W, K, b0 + r, b0 + q) * y[q];
            y[r] = s;
        }
        for (int r = K - 1; r >= 0; --r) {
            double s = y[r];
            for (int q = r + 1; q < K; ++q) s -= F(lu, W, K, b0 + r, b0 + q) * y[q];
            y[r] = s / F(lu, W, K, b0 + r, b0 + r);
        }
        for (int r = 0; r < K; ++r) V[r * K + col] = y[r];
        /* W: backward with unit U'_tt, then forward with L'_tt */
        for (int r = K - 1; r >= 0; --r) {
            double s = h->C[i][r * K + col];
            for (int q = r + 1; q < K; ++q) s -= F(ul, W, K, r, q) * y[q];
            y[r] = s;
        }
        for (int r = 0; r < K; ++r) {
            double s = y[r];
            for (int q = 0; q < r; ++q) s -= F(ul, W, K, r, q) * y[q];
            y[r] = s / F(ul, W, K, r, r);
        }
        for (int r = 0; r < K; ++r) Wt[r * K + col] = y[r];
    }
}

/* Factor the SaP preconditioner of the band: partition, LU of every block
 * (Section 3.1), and for SaP-C the UL of every block, the coupling blocks
 * B_i and C_{i+1}, the spike tips and Rbar_i = I - W^(t)_{i+1} V^(b)_i
 * factored by partial pivoting (Eq. (2.5a)).
 * tau is the absolute boosting threshold. */
int orc_factor(const double *band, int64_t N, int K, int P, int variant, double tau, orc_sap **out)
{
    *out = NULL;
    if (N < 1 || K < 1 || K >= N || P < 1 || P > N) return ORC_ERR_INVALID_ARG;
    orc_sap *h = (orc_sap *)xcalloc(1, sizeof(orc_sap));
    if (!h) return ORC_ERR_OOM;
    h->N = N; h->K = K; h->P = P; h->variant = variant; h->tau = tau;
    h->off = (int64_t *)xcalloc(P + 1, sizeof(int64_t));
    orc_partition(N, P, h->off);
    for (int i = 0; i < P; ++i) {
        int64_t n = h->off[i + 1] - h->off[i];
        if (n < 1 || (variant == 1 && P > 1 && n < 2 * (int64_t)K)) { orc_free(h); return ORC_ERR_INVALID_ARG; }
    }
    int W = 2 * K + 1;
    int64_t nbst = 0;
    h->lu = (double **)xcalloc(P, sizeof(double *));
    /* the blocks are independent (Section 2.1); built with -fopenmp the loops
     * over blocks below run in parallel, each block's arithmetic unchanged */
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : nbst)
    for (int i = 0; i < P; ++i) {
        int64_t n = h->off[i + 1] - h->off[i];
        h->lu[i] = (double *)xcalloc((size_t)(n * W), sizeof(double));
        load_block(band, N, K, h->off[i], n, h->lu[i]);
        nbst += orc_block_lu(h->lu[i], n, K, tau);
    }
    h->n_boosted += nbst;
    if (variant == 1 && P > 1) {
        h->ul = (double **)xcalloc(P, sizeof(double *));
        nbst = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : nbst)
        for (int i = 0; i < P; ++i) {
            int64_t n = h->off[i + 1] - h->off[i];
            h->ul[i] = (double *)xcalloc((size_t)(n * W), sizeof(double));
            load_block(band, N, K, h->off[i], n, h->ul[i]);
            nbst += orc_block_ul(h->ul[i], n, K, tau);
        }
        h->n_boosted += nbst;
        h->B = (double **)xcalloc(P - 1, sizeof(double *));
        h->C = (double **)xcalloc(P - 1, sizeof(double *));
        h->V = (double **)xcalloc(P - 1, sizeof(double *));
        h->Wt = (double **)xcalloc(P - 1, sizeof(double *));
        h->R = (double **)xcalloc(P - 1, sizeof(double *));
        h->R0 = (double **)xcalloc(P - 1, sizeof(double *));
        h->piv = (int32_t **)xcalloc(P - 1, sizeof(int32_t *));
        int singular = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : singular)
        for (int i = 0; i < P - 1; ++i) {
            int64_t s = h->off[i + 1];
            h->B[i] = (double *)xcalloc((size_t)K * K, sizeof(double));
            h->C[i] = (double *)xcalloc((size_t)K * K, sizeof(double));
            h->V[i] = (double *)xcalloc((size_t)K * K, sizeof(double));
            h->Wt[i] = (double *)xcalloc((size_t)K * K, sizeof(double));
            h->R[i] = (double *)xcalloc((size_t)K * K, sizeof(double));
            h->R0[i] = (double *)xcalloc((size_t)K * K, sizeof(double));
            h->piv[i] = (int32_t *)xcalloc((size_t)K, sizeof(int32_t));
            for (int r = 0; r < K; ++r)
                for (int c = 0; c < K; ++c) {
                    h->B[i][r * K + c] = band_get(band, N, K, s - K + r, s + c);
                    h->C[i][r * K + c] = band_get(band, N, K, s + r, s - K + c);
                }
            spike_tips(h, i);
            for (int r = 0; r < K; ++r)
                for (int c = 0; c < K; ++c) {
                    double acc = (r == c) ? 1.0 : 0.0;
                    for (int q = 0; q < K; ++q) acc -= h->Wt[i][r * K + q] * h->V[i][q * K + c];
                    h->R[i][r * K + c] = acc;
                    h->R0[i][r * K + c] = acc;
                }
            if (orc_dense_getrf(h->R[i], K, h->piv[i])) singular = 1;   /* exact singularity */
        }
        if (singular) { orc_free(h); return ORC_ERR_SINGULAR; }
    }
    *out = h;
    return ORC_OK;
}

/* Solve A_i y = y in place with the block LU (forward with unit L, then
 * backward with U). */
static void block_solve(const double *lu, int64_t n, int K, double *y)
{
    int W = 2 * K + 1;
    for (int64_t r = 0; r < n; ++r) {
        double s = y[r];
        int64_t q0 = r - K > 0 ? r - K : 0;
        for (int64_t q = q0; q < r; ++q) s -= F(lu, W, K, r, q) * y[q];
        y[r] = s;
    }
    for (int64_t r = n - 1; r >= 0; --r) {
        double s = y[r];
        int64_t q1 = r + K < n - 1 ? r + K : n - 1;
        for (int64_t q = r + 1; q <= q1; ++q) s -= F(lu, W, K, r, q) * y[q];
        y[r] = s / F(lu, W, K, r, r);
    }
}

/* Truncated reduced system of interface i, Eq. (2.5):
 *   Rbar_i xt = gt - W^(t)_{i+1} gb,   xb = gb - V^(b)_i xt,
 * with gb = g^(b)_i (bottom K entries of block i) and gt = g^(t)_{i+1}
 * (top K entries of block i+1). */
void orc_reduced_solve(const orc_sap *h, int i, const double *gb, const double *gt,
                       double *xb, double *xt)
{
    int K = h->K;
    for (int rr = 0; rr < K; ++rr) {
        double acc = gt[rr];
        for (int q = 0; q < K; ++q) acc -= h->Wt[i][rr * K + q] * gb[q];
        xt[rr] = acc;
    }
    orc_dense_getrs(h->R[i], K, h->piv[i], xt);
    for (int rr = 0; rr < K; ++rr) {
        double acc = gb[rr];
        for (int q = 0; q < K; ++q) acc -= h->V[i][rr * K + q] * xt[q];
        xb[rr] = acc;
    }
}

/* Preconditioner apply z = M^{-1} r.
 *   SaP-D (Section 2.1.1): z = D^{-1} r, D = diag(A_1..A_P)       (Eq. (2.3))
 *   SaP-C: g = D^{-1} r; for every interface the truncated reduced system
 *   of Eq. (2.5): rhs = g^(t)_{i+1} - W^(t)_{i+1} g^(b)_i, solve
 *   Rbar_i xt = rhs, xb = g^(b)_i - V^(b)_i xt; then the purification
 *   solves A_i z_i = r_i - [C_i xb_{i-1}; 0; 0] - [0; 0; B_i xt_{i+1}]. */
void orc_apply(const orc_sap *h, const double *r, double *z)
{
    int64_t N = h->N;
    int K = h->K, P = h->P;
    memcpy(z, r, (size_t)N * sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < P; ++i)
        block_solve(h->lu[i], h->off[i + 1] - h->off[i], K, z + h->off[i]);
    if (h->variant != 1 || P == 1) return;
    double *xt = (double *)xcalloc((size_t)(P - 1) * K, sizeof(double));
    double *xb = (double *)xcalloc((size_t)(P - 1) * K, sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < P - 1; ++i) {
        int64_t s = h->off[i + 1];
        orc_reduced_solve(h, i, z + s - K, z + s, xb + (int64_t)i * K, xt + (int64_t)i * K);
    }
    /* purification: fresh right-hand sides, then the block solves again */
    memcpy(z, r, (size_t)N * sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < P; ++i) {
        int64_t s = h->off[i], n = h->off[i + 1] - s;
        double *zi = z + s;
        if (i > 0) {            /* - C_i xb_{i-1} on the top K rows */
            const double *Cm = h->C[i - 1], *b = xb + (int64_t)(i - 1) * K;
            for (int rr = 0; rr < K; ++rr)
                for (int q = 0; q < K; ++q) zi[rr] -= Cm[rr * K + q] * b[q];
        }
        if (i + 1 < P) {        /* - B_i xt_{i+1} on the bottom K rows */
            const double *Bm = h->B[i], *t = xt + (int64_t)i * K;
            for (int rr = 0; rr < K; ++rr)
                for (int q = 0; q < K; ++q) zi[n - K + rr] -= Bm[rr * K + q] * t[q];
        }
        block_solve(h->lu[i], n, K, zi);
    }
    free(xt); free(xb);
}

/* ------------------------------------------------------------------ */
/* BiCGStab(l), l = 2, left preconditioned                              */
/* ------------------------------------------------------------------ */
/* Sleijpen & Fokkema, "BiCGstab(l) for linear equations involving
 * unsymmetric matrices with complex spectrum", ETNA 1 (1993), Algorithm 3.1,
 * applied to A~ = M^{-1} A and b~ = M^{-1} b with x0 = 0 (Section 4.3.3) and
 * shadow residual r~0 = r^0.  The paper uses l = 2 and left preconditioning
 * (Section 2.1.1).  Exit tests sit after each BiCG residual update (matvec 1
 * and 3 of the iteration) and after the minimal-residual update (matvec 4);
 * the iteration count is matvecs / 4, i.e. quarters (Section 4.1.1).
 * Convergence: ||r^0||_2 <= tol ||b~||_2, confirmed by the true residual
 * ||b - A x||_2 <= tol ||b||_2 in FP64.  A failed confirmation after matvec 1
 * or 3 lets the iteration go on unchanged; one after the minimal-residual
 * update restarts the method from the current x: r^0 = M^{-1}(b - A x),
 * r~0 = r^0, u^0 = 0, rho0 = alpha = omega as at the start (the recurrences
 * of the old cycle no longer describe the replaced residual). */

typedef struct {
    double iters;      /* in quarters */
    double relres;     /* true ||b - A x|| / ||b|| */
    int64_t n_matvec;
    int64_t n_restarts;
} orc_info;

static double dot(const double *a, const double *b, int64_t n)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* y = M^{-1} (A v) */
static void op(const orc_sap *h, const double *band, const double *v, double *y, double *tmp)
{
    orc_spmv(band, h->N, h->K, v, tmp, 0);
    orc_apply(h, tmp, y);
}

/* trace (optional, may be NULL): for each exit test, 4 doubles:
 * matvec count, ||r^0||, ||M^{-1}(b - A x)||, true relres. */
int orc_bicgstab2(const orc_sap *h, const double *band, const double *b, double *x,
                  double tol, int max_iters, orc_info *info, double *trace, int trace_cap)
{
    int64_t N = h->N;
    double *buf = (double *)xcalloc((size_t)N * 9, sizeof(double));
    if (!buf) return ORC_ERR_OOM;
    double *r[3] = {buf, buf + N, buf + 2 * N};
    double *u[3] = {buf + 3 * N, buf + 4 * N, buf + 5 * N};
    double *rt = buf + 6 * N, *tmp = buf + 7 * N, *tmp2 = buf + 8 * N;
    int status = ORC_ERR_NOT_CONVERGED;
    int ntrace = 0;
    memset(x, 0, (size_t)N * sizeof(double));
    info->iters = 0; info->relres = 1.0; info->n_matvec = 0; info->n_restarts = 0;
    double bnorm = sqrt(dot(b, b, N));
    if (bnorm == 0.0) { info->relres = 0.0; free(buf); return ORC_OK; }
    orc_apply(h, b, r[0]);                       /* r^0 = b~ - A~ x0 = M^{-1} b */
    double btnorm = sqrt(dot(r[0], r[0], N));
    memcpy(rt, r[0], (size_t)N * sizeof(double));
    double rho0 = 1.0, alpha = 0.0, omega = 1.0;
    int64_t nmv = 0;

    for (int it = 0; it < max_iters; ++it) {
        rho0 = -omega * rho0;
        for (int j = 0; j < 2; ++j) {                  /* BiCG part */
            double rho1 = dot(r[j], rt, N);
            if (rho0 == 0.0) { status = ORC_ERR_BREAKDOWN; goto done; }
            double beta = alpha * rho1 / rho0;
            rho0 = rho1;
            for (int i = 0; i <= j; ++i)
                for (int64_t k = 0; k < N; ++k) u[i][k] = r[i][k] - beta * u[i][k];
            op(h, band, u[j], u[j + 1], tmp); ++nmv;
            double gamma = dot(u[j + 1], rt, N);
            if (gamma == 0.0) { status = ORC_ERR_BREAKDOWN; goto done; }
            alpha = rho0 / gamma;
            for (int i = 0; i <= j; ++i)
                for (int64_t k = 0; k < N; ++k) r[i][k] -= alpha * u[i + 1][k];
            for (int64_t k = 0; k < N; ++k) x[k] += alpha * u[0][k];
            /* exit test after matvec 1 (j = 0) and 3 (j = 1) */
            {
                double rn = sqrt(dot(r[0], r[0], N));
                int pass = rn <= tol * btnorm;
                double rel = -1.0, pn = -1.0;
                if (pass || trace) {
                    orc_spmv(band, N, h->K, x, tmp, 0);
                    for (int64_t k = 0; k < N; ++k) tmp[k] = b[k] - tmp[k];
                    rel = sqrt(dot(tmp, tmp, N)) / bnorm;
                    if (trace) { orc_apply(h, tmp, tmp2); pn = sqrt(dot(tmp2, tmp2, N)); }
                }
                if (trace && ntrace < trace_cap) {
                    double *t = trace + 4 * ntrace++;
                    t[0] = (double)(4 * it + (j == 0 ? 1 : 3)); t[1] = rn; t[2] = pn; t[3] = rel;
                }
                if (pass && rel <= tol) {
                    info->iters = it + (j == 0 ? 0.25 : 0.75); info->relres = rel;
                    status = ORC_OK; goto done;
                }
            }
            op(h, band, r[j], r[j + 1], tmp); ++nmv;
        }
        /* MR part (modified Gram-Schmidt on r^1, r^2) */
        double sigma1 = dot(r[1], r[1], N);
        if (sigma1 == 0.0) { status = ORC_ERR_BREAKDOWN; goto done; }
        double gp1 = dot(r[0], r[1], N) / sigma1;
        double tau12 = dot(r[2], r[1], N) / sigma1;
        for (int64_t k = 0; k < N; ++k) r[2][k] -= tau12 * r[1][k];
        double sigma2 = dot(r[2], r[2], N);
        if (sigma2 == 0.0) { status = ORC_ERR_BREAKDOWN; goto done; }
        double gp2 = dot(r[0], r[2], N) / sigma2;
        double gamma2 = gp2;
        omega = gamma2;
        double gamma1 = gp1 - tau12 * gamma2;
        double gpp1 = gamma2;
        for (int64_t k = 0; k < N; ++k) {
            x[k] += gamma1 * r[0][k] + gpp1 * r[1][k];
            r[0][k] -= gp2 * r[2][k] + gp1 * r[1][k];
            u[0][k] -= gamma2 * u[2][k] + gamma1 * u[1][k];
        }
        {   /* exit test after matvec 4 */
            double rn = sqrt(dot(r[0], r[0], N));
            int pass = rn <= tol * btnorm;
            double rel = -1.0, pn = -1.0;
            if (pass || trace) {
                orc_spmv(band, N, h->K, x, tmp, 0);
                for (int64_t k = 0; k < N; ++k) tmp[k] = b[k] - tmp[k];
                rel = sqrt(dot(tmp, tmp, N)) / bnorm;
                if (trace) { orc_apply(h, tmp, tmp2); pn = sqrt(dot(tmp2, tmp2, N)); }
            }
            if (trace && ntrace < trace_cap) {
                double *t = trace + 4 * ntrace++;
                t[0] = (double)(4 * it + 4); t[1] = rn; t[2] = pn; t[3] = rel;
            }
            if (pass) {
                if (rel <= tol) {
                    info->iters = it + 1.0; info->relres = rel;
                    status = ORC_OK; goto done;
                }
                /* restart from the current x */
                orc_apply(h, tmp, r[0]);
                memcpy(rt, r[0], (size_t)N * sizeof(double));
                memset(u[0], 0, (size_t)N * sizeof(double));
                rho0 = 1.0; alpha = 0.0; omega = 1.0;
                ++info->n_restarts;
            }
        }
        if (omega == 0.0) { status = ORC_ERR_BREAKDOWN; goto done; }
        info->iters = it + 1.0;
    }
done:
    info->n_matvec = nmv;
    if (status != ORC_OK) {
        orc_spmv(band, N, h->K, x, tmp, 0);
        for (int64_t k = 0; k < N; ++k) tmp[k] = b[k] - tmp[k];
        info->relres = sqrt(dot(tmp, tmp, N)) / bnorm;
    }
    free(buf);
    return status;
}

/* ------------------------------------------------------------------ */
/* conjugate gradient (symmetric positive definite A)                   */
/* ------------------------------------------------------------------ */

/* Section 3: when A is symmetric positive definite the outer iteration is a
 * conjugate gradient method instead of BiCGStab(2), preconditioned by the
 * SaP factorisation (Section 4.1 lists both methods).  The iteration is the
 * preconditioned CG of Saad, "Iterative methods for sparse linear systems",
 * 2nd ed., Algorithm 9.1, from x_0 = 0:
 *   r_0 = b,  z_0 = M^{-1} r_0,  p_0 = z_0;  per iteration j:
 *   alpha_j = (r_j, z_j) / (A p_j, p_j)
 *   x_{j+1} = x_j + alpha_j p_j,   r_{j+1} = r_j - alpha_j A p_j
 *   z_{j+1} = M^{-1} r_{j+1}
 *   beta_j  = (r_{j+1}, z_{j+1}) / (r_j, z_j),   p_{j+1} = z_{j+1} + beta_j p_j
 * One matrix-vector product and one preconditioner application per
 * iteration; the count is in whole iterations.  Readings (the paper gives
 * none for CG): the exit test is the unpreconditioned recursive residual,
 * ||r_{j+1}||_2 <= tol ||b||_2, confirmed by the true residual
 * ||b - A x||_2 <= tol ||b||_2; a failed confirmation restarts the method
 * from the current x with the true residual (r = b - A x, z = M^{-1} r,
 * p = z), as the BiCGStab(2) restart does.  SaP-D's M (the block diagonal of
 * an SPD A) is SPD; SaP-C's truncated-spike M need not be symmetric, and CG
 * then runs with it as it stands.
 *
 * trace (optional, may be NULL): per iteration 4 doubles: iteration number
 * j + 1, ||r_{j+1}||_2, (r_j, z_j), true relative residual (-1 when the
 * recursive test did not pass). */
int orc_pcg(const orc_sap *h, const double *band, const double *b, double *x,
            double tol, int max_iters, orc_info *info, double *trace, int trace_cap)
{
    int64_t N = h->N;
    double *buf = (double *)xcalloc((size_t)N * 4, sizeof(double));
    if (!buf) return ORC_ERR_OOM;
    double *r = buf, *z = buf + N, *p = buf + 2 * N, *q = buf + 3 * N;
    int status = ORC_ERR_NOT_CONVERGED;
    int ntrace = 0;
    memset(x, 0, (size_t)N * sizeof(double));
    info->iters = 0; info->relres = 1.0; info->n_matvec = 0; info->n_restarts = 0;
    double bnorm = sqrt(dot(b, b, N));
    if (bnorm == 0.0) { info->relres = 0.0; free(buf); return ORC_OK; }
    memcpy(r, b, (size_t)N * sizeof(double));      /* r_0 = b - A x_0, x_0 = 0 */
    orc_apply(h, r, z);
    memcpy(p, z, (size_t)N * sizeof(double));
    double rz = dot(r, z, N);
    int64_t nmv = 0;

    for (int it = 0; it < max_iters; ++it) {
        orc_spmv(band, N, h->K, p, q, 0); ++nmv;     /* q = A p_j */
        double pq = dot(p, q, N);
        if (pq == 0.0) { status = ORC_ERR_BREAKDOWN; goto done; }
        double alpha = rz / pq;
        for (int64_t k = 0; k < N; ++k) {
            x[k] += alpha * p[k];
            r[k] -= alpha * q[k];
        }
        info->iters = it + 1.0;
        double rn = sqrt(dot(r, r, N));
        double rel = -1.0;
        int restarted = 0;
        if (rn <= tol * bnorm) {
            orc_spmv(band, N, h->K, x, q, 0);
            for (int64_t k = 0; k < N; ++k) q[k] = b[k] - q[k];
            rel = sqrt(dot(q, q, N)) / bnorm;
            if (rel <= tol) {
                if (trace && ntrace < trace_cap) {
                    double *t = trace + 4 * ntrace++;
                    t[0] = it + 1.0; t[1] = rn; t[2] = rz; t[3] = rel;
                }
                info->relres = rel;
                status = ORC_OK; goto done;
            }
            memcpy(r, q, (size_t)N * sizeof(double));   /* restart from the current x */
            ++info->n_restarts;
            restarted = 1;
        }
        if (trace && ntrace < trace_cap) {
            double *t = trace + 4 * ntrace++;
            t[0] = it + 1.0; t[1] = rn; t[2] = rz; t[3] = rel;
        }
        orc_apply(h, r, z);                          /* z_{j+1} = M^{-1} r_{j+1} */
        double rz1 = dot(r, z, N);
        if (restarted) {
            memcpy(p, z, (size_t)N * sizeof(double));
        } else {
            if (rz == 0.0) { status = ORC_ERR_BREAKDOWN; goto done; }
            double beta = rz1 / rz;
            for (int64_t k = 0; k < N; ++k) p[k] = z[k] + beta * p[k];
        }
        rz = rz1;
    }
done:
    info->n_matvec = nmv;
    if (status != ORC_OK) {
        orc_spmv(band, N, h->K, x, q, 0);
        for (int64_t k = 0; k < N; ++k) q[k] = b[k] - q[k];
        info->relres = sqrt(dot(q, q, N)) / bnorm;
    }
    free(buf);
    return status;
}

/* ------------------------------------------------------------------ */
/* adjoint                                                              */
/* ------------------------------------------------------------------ */

/* Band of A^T: (A^T)_ij = a_ji, stored with the same convention. */
void orc_transpose_band(const double *band, int64_t N, int K, double *bandT)
{
    for (int64_t c = 0; c <= 2 * (int64_t)K; ++c)
        for (int64_t j = 0; j < N; ++j) {
            int64_t i = j + c - K;   /* (A^T)_ij lives at bandT[c*N + j] */
            bandT[c * N + j] = band_get(band, N, K, j, i);
        }
}

/* Gradient of a scalar loss l(x) with x = A^{-1} b, given lambda = A^{-T} dl/dx:
 * dl/db = lambda and dl/da_ij = -lambda_i x_j for (i, j) in the band, 0 on
 * the padding of the band storage. */
void orc_grad_band(int64_t N, int K, const double *lambda, const double *x, double *grad)
{
    for (int64_t c = 0; c <= 2 * (int64_t)K; ++c)
        for (int64_t j = 0; j < N; ++j) {
            int64_t i = j + c - K;
            grad[c * N + j] = (i >= 0 && i < N) ? -lambda[i] * x[j] : 0.0;
        }
}

/* ------------------------------------------------------------------ */
/* accessors for tests                                                  */
/* ------------------------------------------------------------------ */

int64_t orc_n_boosted(const orc_sap *h) { return h->n_boosted; }
void orc_offsets(const orc_sap *h, int64_t *off) { memcpy(off, h->off, (size_t)(h->P + 1) * sizeof(int64_t)); }

/* Factors of block i in dense-band row-major storage (n_i x W). which: 0 = LU, 1 = UL. */
int orc_get_block(const orc_sap *h, int i, int which, double *out)
{
    if (i < 0 || i >= h->P) return ORC_ERR_INVALID_ARG;
    double *src = which == 0 ? h->lu[i] : (h->ul ? h->ul[i] : NULL);
    if (!src) return ORC_ERR_INVALID_ARG;
    int64_t n = h->off[i + 1] - h->off[i];
    memcpy(out, src, (size_t)(n * (2 * h->K + 1)) * sizeof(double));
    return ORC_OK;
}

/* K x K matrices of interface i: which 0 = B_i, 1 = C_{i+1}, 2 = V^(b)_i,
 * 3 = W^(t)_{i+1}, 4 = Rbar_i (unfactored). */
int orc_get_interface(const orc_sap *h, int i, int which, double *out)
{
    if (h->variant != 1 || i < 0 || i + 1 >= h->P) return ORC_ERR_INVALID_ARG;
    double **m[5] = {h->B, h->C, h->V, h->Wt, h->R0};
    if (which < 0 || which > 4) return ORC_ERR_INVALID_ARG;
    memcpy(out, m[which][i], (size_t)h->K * h->K * sizeof(double));
    return ORC_OK;
}

/* Boosting threshold tau = eps * max |a_ij| over the in-band entries of A. */
double orc_band_absmax(const double *band, int64_t N, int K)
{
    double m = 0.0;
    for (int64_t c = 0; c <= 2 * (int64_t)K; ++c)
        for (int64_t j = 0; j < N; ++j) {
            int64_t i = j + c - K;
            if (i >= 0 && i < N && fabs(band[c * N + j]) > m) m = fabs(band[c * N + j]);
        }
    return m;
}
