/* SaP with a bandwidth of its own per block: the third-stage reordering of
 * Sec. 2.2 ("Third-stage reordering") and the entire-spike computation of
 * Sec. 3.1 ("Use of registers and shared memory").
 *
 * After the DB-CM reorderings the band of A (half-bandwidth K, the storage of
 * sap.h) is often sparse inside.  Split into the blocks A_i of the partition
 * (the same partition as sap_factor's for N and P), each block is renumbered
 * on its own by a symmetric permutation Pi_i, Ahat_i = Pi_i A_i Pi_i^T, whose
 * half-bandwidth K_i can be well below K; the blocks are factored at their own
 * K_i (memory N_i (2 K_i + 1), work about 2 N_i K_i^2 each).  The coupling
 * blocks B_i, C_{i+1} keep their places, so in a block's new numbering the
 * rows they touch are spread over the block: SaP-C then computes the entire
 * spikes A_i^{-1}[0; B_i], A_{i+1}^{-1}[C_{i+1}; 0] (N_i x K each, kept on
 * the device) by multi-right-hand-side sweeps with the factors of Ahat_i and
 * takes the tips V^(b)_i, W^(t)_{i+1} out of them; no UL factorisation is
 * used.  The preconditioner is the SaP-D / SaP-C one of Eq. (2.3)-(2.5) on A:
 * in exact arithmetic it does not depend on the blocks' numbering.
 *
 * A permutation is given as "new index of old index", local to each block:
 * perm[off_i + a] = new local index of local row/column a of block i (int32,
 * a permutation of 0..N_i-1 in every block), on the device. */
#ifndef SAP_BLOCKS_H
#define SAP_BLOCKS_H

#include "sap.h"

#ifdef __cplusplus
extern "C" {
#endif

/* The third-stage reordering (Sec. 2.2): Cuthill-McKee of the pattern of
 * A_i + A_i^T (the nonzero band entries with row and column in block i) for
 * every block of the partition of N into P blocks, on its own; per connected
 * component the multi-start rule of sap_cm_reorder (sap_sparse.h).
 *   perm_dev (out, N int32, device): the block permutations as above.
 *   Ki_host (out, P int32, host, optional): half-bandwidth of each Ahat_i,
 *     max |perm(a) - perm(b)| over its nonzeros (0 for a diagonal block).
 * The graph searches run on the host (as in the paper, Sec. 3.3), the blocks
 * spread over up to 16 threads (independent, as the paper runs this stage in
 * parallel for every A_i): the band is copied to the host once ((2K + 1) N
 * doubles).
 * Errors: INVALID_ARG (sizes, null pointers, P < 1 or N < P), OOM, CUDA.
 * Synchronises `stream`. */
SAP_API sap_status_t sap_block_cm_reorder(const double *band_dev, int64_t N, int32_t K, int32_t P,
                                          int32_t *perm_dev, int32_t *Ki_host, cudaStream_t stream);

/* Factor the SaP preconditioner of A with every block reordered by its
 * permutation (band_dev, N, K as for sap_factor; perm_dev as above, read
 * during this call only).  opt->P >= 1 is required (no autotuning); the
 * variant, precision, tolerance, iteration cap, boosting (threshold tau from
 * max |a_ij| over the whole band, couplings included) and spin limit are as
 * for sap_factor; opt->segments applies to every block's sweeps.  K_i =
 * max(1, bandwidth of Ahat_i); every K_i must be at most sap_max_K(precision)
 * and below N_i, while K itself may exceed sap_max_K.  SaP-C needs N_i >= 2 K.
 * The returned handle works with sap_solve, sap_solve_host, sap_solve_adjoint,
 * sap_solve_pair, sap_grad_band, sap_apply_preconditioner (either direction),
 * sap_refactor (same pattern: an entry of the new values outside its block's
 * K_i is INVALID_ARG), sap_set_operator_csr (forward solves only, as for
 * sap_factor handles), sap_num_partitions and sap_destroy.  The
 * preconditioner of A^T (same partition and permutations: the blocks of A^T
 * renumbered are Ahat_i^T, factored by the stored factors transposed;
 * couplings B'_i = C_{i+1}^T, C'_{i+1} = B_i^T; its own entire spikes, tips
 * and reduced matrices) is built on the first transposed use after each
 * factorisation.  sap_get_block_lu returns NOT_IMPLEMENTED.  sap_get_interface
 * gives B, C, V, W and Rbar (which = 0..4), of A or (adjoint) of A^T, as for
 * sap_factor.
 * Device memory: the reordered bands (FP64, sum N_i (2 K_i + 1)), the factors
 * and sweep matrices of every block at its own K_i, for SaP-C the entire
 * spikes (2 N K elements of the factor precision) and the reduced matrices,
 * the same again for A^T once a transposed operation has run.
 * Errors: INVALID_ARG (sizes, a perm that is not a permutation per block,
 * P < 1), NOT_IMPLEMENTED (a K_i above sap_max_K), SINGULAR (a reduced
 * matrix), TIMEOUT, OOM, CUDA.  Synchronises `stream`. */
SAP_API sap_status_t sap_factor_blocks(const double *band_dev, int64_t N, int32_t K, const int32_t *perm_dev,
                                       const sap_options_t *opt, cudaStream_t stream, sap_handle_t *out);

/* Half-bandwidths K_i of the reordered blocks of a handle made by
 * sap_factor_blocks (Ki_host: P int32, host).  INVALID_ARG for any other
 * handle. */
SAP_API sap_status_t sap_get_block_bandwidths(sap_handle_t h, int32_t *Ki_host);

#ifdef __cplusplus
}
#endif

#endif /* SAP_BLOCKS_H */
