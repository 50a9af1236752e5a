/*
 * sselinv.h -- selected inversion on the compression pattern and the contour-integral
 * inverse square root (libsformat.so; Sec. 4.2 "Sparse selected inversion", Eq. (blockInv),
 * and Sec. 4.4 "Matrix functions", Eq. (ContInt)).
 *
 * For a symmetric matrix A stored on a symmetric pattern S (block-CSR of sformat.h, every
 * non-empty diagonal block present) and a shift sigma with A + sigma I positive definite:
 *
 *   factor   A + sigma I = L D L^T, L block unit lower triangular, D block diagonal, with the
 *            clusters as supernodes (dense blocks), eliminated in a minimum-degree order of
 *            the block graph of S; the pattern of L is S's lower part plus the fill of that
 *            order (elimination game).
 *   invert   Z = (A + sigma I)^{-1} on the pattern of L by the recurrences that follow from
 *            Eq. (blockInv) applied supernode by supernode (Takahashi-type):
 *              Z(i,k) = - sum_{j in struct(k)} Z(i,j) L(j,k)          (i in struct(k))
 *              Z(k,k) = D(k,k)^{-1} - sum_{j in struct(k)} Z(j,k)^T L(j,k)
 *            struct(k) = the positions below k in column k of L.  The pattern of L contains
 *            S, so P_S(Z) is the exact inverse on S up to rounding.
 *
 * Both run in FP64 on the device, one elimination-tree level after another (the blocks of
 * one level are independent): the factor from the leaves up, the inversion from the root
 * down.  Value buffers are DEVICE pointers on S (s_pattern_nnz doubles) owned by the caller;
 * the plan owns the factor (three buffers of the size of L: L D, L with D^{-1} in its
 * diagonal blocks, Z) and the term lists of both sweeps, built once by the symbolic analysis
 * (8 bytes per block product: 5.8 GB at N = 65536 in 2D with q = 3).  A plan serves one
 * stream at a time: its factor and scratch buffers are shared by all its calls.  Blocks are
 * at most 64 wide (S_ERR_ARG otherwise); the symbolic analysis keeps one bit per pair of
 * non-empty clusters on the host, so at most 32768 non-empty clusters.
 */
#ifndef SSELINV_H
#define SSELINV_H

#include <stdint.h>

#include "sformat.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct s_selinv_t* s_selinv;

/* Host only (no device work): the elimination order and the size of the factor for a
 * symmetric block pattern given as host CSR arrays (n_clusters rows, rowptr n_clusters+1,
 * colidx sorted per row) and the cluster sizes bsize (clusters of size 0 are left out and
 * placed last).  Minimum degree on the block graph, ties to the smaller cluster id;
 * perm[p] = cluster eliminated p-th (n_clusters entries).  *l_blocks = blocks of L
 * including the diagonal (non-empty clusters only), *levels = height of the elimination
 * tree.  S_ERR_PATTERN when the pattern is not symmetric. */
s_status s_selinv_order(int32_t n_clusters, const int64_t* rowptr, const int32_t* colidx, const int32_t* bsize,
                        int32_t* perm, int64_t* l_blocks, int32_t* levels);

/* Symbolic analysis of pattern S and device allocation of the factor (synchronous, current
 * device).  S must be symmetric with every non-empty diagonal block (S_ERR_PATTERN);
 * S_ERR_NOMEM when the host analysis or the device buffers do not fit. */
s_status s_selinv_create(s_pattern S, s_selinv* out);
s_status s_selinv_destroy(s_selinv p);

/* Sizes of the factor: blocks and entries of L (lower part with the diagonal), levels of
 * the elimination tree, and the FP64 operations of one factorization and of one inversion
 * (multiply-add = 2). */
s_status s_selinv_stats(s_selinv p, int64_t* l_blocks, int64_t* l_entries, int32_t* levels, double* flops_factor,
                        double* flops_invert);

/* A + sigma I = L D L^T for the values A (device, on S; only the blocks of S's lower part in
 * the elimination order are read, A must be symmetric).  Enqueued on `stream`.  A pivot
 * block that is not positive definite (a non-positive or non-finite Gauss-Jordan pivot) is
 * recorded and reported by s_selinv_status. */
s_status s_selinv_factor(s_selinv p, const double* A, double sigma, void* stream);

/* Z = (A + sigma I)^{-1} on the pattern of L from the last s_selinv_factor, then
 * out = alpha P_S(Z) + beta out (device, on S; beta = 0 ignores out's contents).  Enqueued
 * on `stream`. */
s_status s_selinv_invert(s_selinv p, double alpha, double beta, double* out, void* stream);

/* Synchronises `stream`; S_ERR_NOT_SPD if a factorization since the last call met a pivot
 * block that was not positive definite (the record is then cleared), else S_OK. */
s_status s_selinv_status(s_selinv p, void* stream);

/* Eq. (ContInt): out = P_S(A^{-1/2}) ~ sum_k weight_k P_S((A + w_k^2 I)^{-1}) with the
 * n-node rule of s_contour_nodes for the spectral interval [c_lo, c_hi]: n factorizations and
 * inversions on `stream`, then a status check as s_selinv_status (synchronous). */
s_status s_selinv_invsqrt(s_selinv p, const double* A, double c_lo, double c_hi, int32_t n, double* out,
                          void* stream);

/* Host only: shifts w_k^2 and weights of the n-node rule of Eq. (ContInt) for 0 < c_lo <= c_hi:
 * m = 1 - c_lo/c_hi, t_k = K(m) (k - 1/2)/n, w_k = sqrt(c_lo) sn(t_k|m)/cn(t_k|m), weight_k =
 * 2 K(m) sqrt(c_lo) dn(t_k|m) / (pi n cn(t_k|m)^2), where K(m) is the complete elliptic integral
 * of the first kind (the constant of the substitution w = sqrt(c_lo) sn/cn, which maps
 * [0, K(m)] onto [0, inf)).  K(m) by the arithmetic-geometric mean, sn/cn/dn by the descending
 * arithmetic-geometric mean scheme of Abramowitz and Stegun 16.4. */
s_status s_contour_nodes(double c_lo, double c_hi, int32_t n, double* shifts, double* weights);

#ifdef __cplusplus
}
#endif
#endif /* SSELINV_H */
