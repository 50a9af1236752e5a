/*
 * sbuild.h -- input preparation for the S-format library (libsformat.so): cluster tree,
 * samplet two-scale transforms, compression pattern and compressed kernel matrix values.
 * Not part of the hot path; it produces the inputs that s_pattern_create and the value
 * buffers of sformat.h consume.
 *
 *   cluster tree      Def. cluster-tree (Sec. 3.2): balanced binary tree, a cluster with
 *                     more than `leaf` points is split along the longest edge of its
 *                     bounding box, points ordered by that coordinate (ties: original
 *                     index), first son = first floor(|nu|/2) points; clusters numbered
 *                     breadth first.
 *   samplets          refinement relation and Eq. (QR) (Sec. 3.2): per cluster the
 *                     Householder QR of the moment matrix of the sons' scaling functions
 *                     (monomials of total degree <= q in the cluster's box coordinates
 *                     (x - centre) / (half longest edge)); min(m_q, n_in) scaling
 *                     functions, the rest samplets; the root keeps its scaling functions
 *                     as coordinates ahead of its samplets.
 *   pattern           eta-admissibility Eq. (cutoff) over all cluster pairs of T x T, with
 *                     bounding-box diameters and distances (bounding-box lemma).
 *   values            K^eta = P_S(T K T^T) (Thm. (S-compression)) for the Matern kernel
 *                     (Sec. 2, half-integer closed form) times `kscale`, plus `nugget` on
 *                     the diagonal; then the a-posteriori threshold of Sec. 5: a block is
 *                     kept iff it is a diagonal block or an entry has |a| >= tau (decided
 *                     on the pair, so the kept pattern is symmetric), entries below tau
 *                     in kept blocks are set to zero.  Computed exactly on the device in
 *                     float arithmetic (O(N^2) kernel evaluations) and stored as double.
 *
 * All arrays returned by the query functions are owned by the builder and live until
 * s_build_destroy.  Errors return a non-zero s_status with a message in s_last_error().
 */
#ifndef SBUILD_H
#define SBUILD_H

#include <stdint.h>

#include "sformat.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct s_build_t* s_build;

/* Tree, two-scale transforms and the eta pattern from n points (row-major n x d host
 * doubles, d in 1..3).  q >= 0 polynomial degree, leaf >= 1, eta > 0 (INFINITY: full
 * pattern).  Host only; uses all host cores. */
s_status s_build_create(int64_t n, int32_t d, const double* points, int32_t leaf, int32_t q, double eta,
                        s_build* out);
s_status s_build_destroy(s_build b);

/* Sizes: clusters, a-priori blocks and entries of the eta pattern. */
s_status s_build_sizes(s_build b, int32_t* n_clusters, int64_t* n_blocks, int64_t* nnz);
/* Borrowed host arrays: block_offset (n_clusters+1), level (n_clusters), rowptr
 * (n_clusters+1), colidx (n_blocks) of the a-priori pattern; perm (n): original index of
 * each point in tree order. */
s_status s_build_arrays(s_build b, const int64_t** block_offset, const int32_t** level, const int64_t** rowptr,
                        const int32_t** colidx, const int64_t** perm);
/* Dense transform for small n (n <= 8192): T row-major n x n into host `T`, rows in
 * samplet order, columns in original point order. */
s_status s_build_dense_transform(s_build b, double* T);

/* Samplet coordinates of a vector: out = T v for host v in original point order (the fast
 * transform with the tree's two-scale matrices; host, O(n m_q)). */
s_status s_build_transform(s_build b, const double* v, double* out);

/* Values on the device.  nu in {0.5, 1.5, 2.5}, ell > 0.  On success *pattern is a new
 * pattern of the kept blocks (the caller destroys it) and the builder holds its
 * s_pattern_nnz(*pattern) values in device memory until s_build_take_values (or the next
 * s_build_values / s_build_destroy).  Uses the current device; synchronous. */
s_status s_build_values(s_build b, double nu, double ell, double kscale, double nugget, double tau,
                        s_pattern* pattern);
/* d/dell of the compressed values on a given pattern `on` (a sub-pattern of this builder's
 * eta pattern, e.g. the kept pattern of s_build_values): P_on(T dK/dell T^T) times kscale,
 * no nugget, no threshold, written to the caller's device buffer `out`
 * (s_pattern_nnz(on) doubles).  Same device algorithm as s_build_values. */
s_status s_build_values_dell(s_build b, double nu, double ell, double kscale, s_pattern on, double* out);
/* y = (kscale K + nugget I) v for host vectors v, y of length n in original point order, with
 * every entry of the uncompressed kernel matrix K evaluated on the device (float evaluations,
 * double row sums; O(n^2), about a second at n = 2^20).  With the samplet transform
 * (s_build_transform) and the compressed values it estimates the compression error
 * ||T K T^T w - K^eta w|| / ||T K T^T w|| for w = T v without forming T K T^T (Thm.
 * (S-compression) bounds that error).  Synchronous. */
s_status s_build_kernel_matvec(s_build b, double nu, double ell, double kscale, double nugget, const double* v,
                               double* y);
/* Copies the held values into the caller's device buffer `dst` (s_pattern_nnz doubles)
 * on `stream`, waits for the copy, and releases the builder's copy. */
s_status s_build_take_values(s_build b, double* dst, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SBUILD_H */
