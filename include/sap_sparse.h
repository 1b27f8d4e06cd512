/* Sparse front end of SaP (Sec. 2.2; implementation notes Sec. 3.2, 3.3):
 * the reorderings that turn a sparse A_s into a diagonally heavy matrix of
 * small half-bandwidth K, its assembly into the dense band storage of sap.h,
 * and the permutation of right-hand sides and solutions between the two.
 *
 * Matrices are CSR on the device: rowptr (int64, n + 1 entries, rowptr[0] =
 * 0), col (int32, nnz, column indices of each row in ascending order, no
 * duplicates), val (float64, nnz).  A permutation is given as "new index of
 * old index": p[old] = new, int32 on the device.  The reordered matrix has
 * entry (i, j) of A_s at (rownew[i], colnew[j]), scaled to
 * (rscale[i] * a_ij) * cscale[j] when scale factors are used.
 *
 * As in the paper (Sec. 3.2, 3.3), the sequential graph searches (the
 * matching's initial match and augmenting paths, the Cuthill-McKee level
 * structure and ordering) run on the host inside these calls; the parallel
 * stages (weights, scale factors, bandwidth, band assembly, permutations) run
 * as CUDA kernels.  Calls that run host stages synchronise `stream`; the
 * others are asynchronous on it.  The caller owns every array. */
#ifndef SAP_SPARSE_H
#define SAP_SPARSE_H

#include "sap.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Diagonal boosting (Sec. 2.2, Eq. (DBrelated); stages S1-S4 of Sec. 3.2):
 * the row permutation sigma that maximises prod_i |a_{i sigma(i)}|, i.e. the
 * minimum perfect matching of the bipartite row-column graph with weights
 * c_ij = log a_i - log |a_ij| (a_i = max_j |a_ij|; no edge for a_ij = 0).
 * S1 (weights) on the GPU; S2 (initial partial match from u_i = min_j c_ij,
 * v_j = min_i (c_ij - u_i)) and S3 (Dijkstra shortest augmenting paths on
 * the reduced costs) on the host; S4 (scale factors) on the GPU.
 *   rownew_dev (out, n): rownew[i] = sigma(i), the column matched to row i,
 *     i.e. the new position of row i (its matched entry lands on the diagonal).
 *   rscale_dev, cscale_dev (out, n, optional, both or neither): the scaling
 *     of Sec. 3.2 S4 to an I-matrix, r_i = exp(u_i) / a_i, s_j = exp(v_j) from
 *     the matching's dual potentials: |r_i a_ij s_j| <= 1, = 1 on the matching.
 *   logprod (out, host, optional): sum_i log |a_{i sigma(i)}|.
 * Errors: INVALID_ARG (sizes, null pointers, a row without entries),
 * SINGULAR (no perfect matching: structurally singular A_s), OOM, CUDA.
 * Synchronises `stream`. */
SAP_API sap_status_t sap_db_reorder(int64_t n, int64_t nnz, const int64_t *rowptr_dev, const int32_t *col_dev,
                                    const double *val_dev, int32_t *rownew_dev, double *rscale_dev,
                                    double *cscale_dev, double *logprod, cudaStream_t stream);

/* Cuthill-McKee bandwidth reduction (Sec. 2.2; Sec. 3.3) of the pattern of
 * B + B^T, where B is A_s with row i moved to rownew[i] (rownew_dev NULL: the
 * identity), so that the diagonal B received from the matching stays on the
 * diagonal.  Per connected component: a breadth-first search in which the
 * unvisited neighbours of each node are taken in non-descending degree (ties
 * to the lower index), from the best of up to 5 start nodes: first the
 * component's node of lowest degree, then each time the untried node of
 * lowest degree in the last BFS level, kept while the BFS tree gets taller
 * and its widest level narrower (Sec. 3.3).
 *   perm_dev (out, n): perm[old] = new (applied to rows and columns of B).
 *   K_out (out, host, optional): the half-bandwidth of the result, max over
 *     the entries (i, j) of A_s of |perm[rownew[i]] - perm[j]|.
 * Errors: INVALID_ARG, OOM, CUDA.  Synchronises `stream`. */
SAP_API sap_status_t sap_cm_reorder(int64_t n, int64_t nnz, const int64_t *rowptr_dev, const int32_t *col_dev,
                                    const int32_t *rownew_dev, int32_t *perm_dev, int32_t *K_out,
                                    cudaStream_t stream);

/* out[i] = outer[inner[i]] (n entries): e.g. the final row positions
 * perm[rownew[i]] of the two reorderings.  Errors: INVALID_ARG, CUDA.
 * Asynchronous. */
SAP_API sap_status_t sap_perm_compose(int64_t n, const int32_t *outer_dev, const int32_t *inner_dev,
                                      int32_t *out_dev, cudaStream_t stream);

/* Half-bandwidth of the reordered matrix: max |rownew[i] - colnew[j]| over
 * the stored entries (rownew_dev / colnew_dev NULL: identity).  K_out: host.
 * Errors: INVALID_ARG, CUDA.  Synchronises `stream`. */
SAP_API sap_status_t sap_sparse_bandwidth(int64_t n, int64_t nnz, const int64_t *rowptr_dev,
                                          const int32_t *col_dev, const int32_t *rownew_dev,
                                          const int32_t *colnew_dev, int32_t *K_out, cudaStream_t stream);

/* Dense band of the reordered (and scaled) matrix in the storage of sap.h,
 * band[(K + I - J) * n + J] = entry (I, J), every other band entry 0: the
 * matrix "regarded as dense banded" of Sec. 2.2, ready for sap_factor.
 *   band_dev (out, (2K + 1) n doubles); rscale_dev / cscale_dev NULL: 1.
 *   drop: nonzero drops the entries outside the band (the element drop-off of
 *     Sec. 2.2: the band is then the preconditioner's approximation A-hat of
 *     the reordered matrix, see sap_set_operator_csr); 0 makes such an entry
 *     an error.
 * Errors: INVALID_ARG (also, with drop = 0, when an entry falls outside the
 * band K, checked by the kernel and reported after the stream completes),
 * CUDA.  Synchronises `stream`. */
SAP_API sap_status_t sap_sparse_to_band(int64_t n, int64_t nnz, const int64_t *rowptr_dev, const int32_t *col_dev,
                                        const double *val_dev, const int32_t *rownew_dev,
                                        const int32_t *colnew_dev, const double *rscale_dev,
                                        const double *cscale_dev, int32_t K, int32_t drop, double *band_dev,
                                        cudaStream_t stream);

/* Element drop-off (Sec. 2.2, Sec. 3.4's T_Drop): the half-bandwidth K' <= K
 * of the band kept after dropping the entries farthest from the diagonal,
 * the smallest K' whose dropped entries (|I - J| > K') weigh at most `frac`
 * of all, the weight of an entry being |(r_i a_ij) s_j| (rscale_dev /
 * cscale_dev NULL: |a_ij|); K is the reordered matrix's half-bandwidth.
 * frac = 0 keeps every entry (K' = K unless the outermost diagonals are
 * empty); a large frac keeps the diagonal only (K' = 0: diagonal
 * preconditioning).  Weights per distance from the diagonal are summed on the
 * GPU.  Kdrop_out: host.  Errors: INVALID_ARG, OOM, CUDA.  Synchronises
 * `stream`. */
SAP_API sap_status_t sap_sparse_drop_bandwidth(int64_t n, int64_t nnz, const int64_t *rowptr_dev,
                                               const int32_t *col_dev, const double *val_dev,
                                               const int32_t *rownew_dev, const int32_t *colnew_dev,
                                               const double *rscale_dev, const double *cscale_dev, int32_t K,
                                               double frac, int32_t *Kdrop_out, cudaStream_t stream);

/* Krylov operator of a handle other than its band (Sec. 2.2: the outer
 * iteration runs on the reordered sparse matrix, the preconditioner is SaP of
 * its dropped band): after this call sap_solve iterates on A' x = b', A' the
 * reordered and scaled sparse matrix (entry (i, j) of the CSR matrix at
 * (rownew[i], colnew[j]) with value (r_i a_ij) s_j; rownew_dev / colnew_dev
 * NULL: identity; rscale_dev / cscale_dev NULL: 1), n equal to the handle's
 * N; the handle's band stays the preconditioner's.  The arrays are borrowed
 * (kept alive by the caller while the handle uses them).  rowptr_dev NULL
 * restores the band as the operator.  Transposed solves (sap_solve_adjoint,
 * sap_solve_pair, sap_grad_band) on a handle with a sparse operator return
 * NOT_IMPLEMENTED.  Errors: INVALID_ARG, CUDA.  Synchronises the device (the
 * handle's captured iterations are discarded). */
SAP_API sap_status_t sap_set_operator_csr(sap_handle_t h, int64_t n, int64_t nnz, const int64_t *rowptr_dev,
                                          const int32_t *col_dev, const double *val_dev,
                                          const int32_t *rownew_dev, const int32_t *colnew_dev,
                                          const double *rscale_dev, const double *cscale_dev);

/* Right-hand side of the reordered system: out[rownew[i]] = r_i b_i
 * (rscale_dev NULL: r = 1).  Errors: INVALID_ARG, CUDA.  Asynchronous. */
SAP_API sap_status_t sap_sparse_permute_rhs(int64_t n, const double *b_dev, const int32_t *rownew_dev,
                                            const double *rscale_dev, double *out_dev, cudaStream_t stream);

/* Solution of A_s x = b from that of the reordered system: x_j = s_j y[colnew[j]]
 * (cscale_dev NULL: s = 1).  Errors: INVALID_ARG, CUDA.  Asynchronous. */
SAP_API sap_status_t sap_sparse_unpermute_solution(int64_t n, const double *y_dev, const int32_t *colnew_dev,
                                                   const double *cscale_dev, double *x_dev, cudaStream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* SAP_SPARSE_H */
