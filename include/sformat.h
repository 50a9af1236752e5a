/*
 * sformat.h -- C ABI of the GB300 samplet S-format algebra library (libsformat.so).
 *
 * The library computes with samplet-compressed kernel matrices in the S-format of
 * Harbrecht, Multerer, Schenk, Schwab, "Multiresolution kernel matrix algebra"
 * (arXiv 2211.11681): matrices in samplet coordinates, stored only on a block pattern S of
 * cluster pairs (nu, nu') of one cluster tree (Sec. 3.3, Thm. (S-compression), Eq. (cutoff)).
 *
 * Storage ("block-CSR"): the matrix dimension N is split into n_clusters consecutive row
 * ranges, cluster nu owning rows block_offset[nu] .. block_offset[nu+1]-1 (its samplets;
 * the root cluster also owns the root scaling functions).  The pattern lists, for every
 * block row nu, the block columns colidx[rowptr[nu] .. rowptr[nu+1]-1] in strictly
 * increasing order.  Block k = (nu, colidx[k]) holds bsize(nu) x bsize(colidx[k]) entries,
 * row-major; the blocks are packed one after the other in pattern order, so the value
 * buffer of a matrix on pattern S holds s_pattern_nnz(S) entries and block k starts at
 * entry s_pattern_block_offsets(S)[k].
 *
 * Value buffers are DEVICE pointers owned by the caller; the library never frees them.
 * Their element type is double for S_FP64 and S_FP64_DF (and for s_add/s_funm with
 * S_FP64), float for S_FP32 and S_BF16X3.  Handles are owned by the library: destroy
 * them explicitly.  Every call returns an s_status; on error nothing is freed and output
 * buffers are unspecified.  Calls that take a stream enqueue asynchronously on it (a
 * cudaStream_t passed as void*, NULL = legacy default stream); a device fault surfaces as
 * S_ERR_CUDA at the next call that synchronises.  s_last_error() returns a
 * thread-local message for the last failing call of the calling thread.
 *
 * All operands of one call must come from the same cluster tree: patterns carry a hash
 * of (block_offset, level), and mismatches return S_ERR_MISMATCH.
 */
#ifndef SFORMAT_H
#define SFORMAT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct s_pattern_t* s_pattern;
typedef struct s_plan_t* s_plan;

typedef enum {
  S_OK = 0,
  S_ERR_ARG = -1,           /* bad argument (null pointer, size, enum)               */
  S_ERR_PATTERN = -2,       /* malformed pattern arrays                               */
  S_ERR_MISMATCH = -3,      /* operands from different trees / incompatible patterns  */
  S_ERR_NOMEM = -4,         /* device or host allocation failed                       */
  S_ERR_CUDA = -5,          /* a CUDA call failed; see s_last_error()                 */
  S_ERR_NOT_CONVERGED = -6, /* Newton-Schulz iteration diverged (see s_funm)          */
  S_ERR_TIMEOUT = -7,       /* a bounded device-side wait ran out                     */
  S_ERR_NOT_SPD = -8        /* a factorization met a pivot block that is not positive
                               definite (sselinv.h)                                    */
} s_status;

/* Arithmetic of a product.
 *   S_FP64     double in, double out, double multiply-add.
 *   S_FP64_DF  double in, double out; each operand split into a pair of floats
 *              (hi + lo) and the products formed in float-pair arithmetic with float
 *              error-free transformations; about 2^-44 relative per operation.
 *   S_FP32     float in, float out, float multiply-add; the partial sum of each few lambda
 *              blocks is folded into the running sum by an error-free two-sum (compensated
 *              summation over lambda).  The default kernel reads both operands K-major: A as
 *              stored and B through a padded copy of its transposed blocks that the plan keeps
 *              (s_pattern_nnz(S_B) floats, rounded up per block to multiples of 4 in each
 *              dimension), unless s_plan_set_symmetric_a was set and the product is called
 *              with B = A on one pattern whose block sizes are multiples of 4.
 *   S_BF16X3   float in, float out; each operand split into three bfloat16 parts,
 *              the six leading cross products on the tensor cores, float accumulate.
 *   S_TF32X3   float in, float out; each operand split as hi + lo, both rounded to TF32
 *              (10 fraction bits), the three products hi*hi + hi*lo + lo*hi on the tcgen05
 *              tensor cores, each lambda slice (at most 24 wide) accumulated in fp32 in
 *              tensor memory and the slices summed in fp32 registers by error-free two-sums
 *              (compensated).  Blocks may be at most 96 wide.  Inputs must be finite. */
typedef enum { S_FP64 = 0, S_FP32 = 1, S_BF16X3 = 2, S_FP64_DF = 3, S_TF32X3 = 4 } s_prec;

typedef enum { S_SQRT = 0, S_EXP = 1, S_EXP_NEG = 2 } s_fn;

/* ---- patterns ------------------------------------------------------------------------ */

/* Create a pattern from host arrays (copied; the caller keeps ownership).
 *   n_clusters   number of clusters (block rows), >= 1.
 *   block_offset n_clusters+1 row offsets, block_offset[0] = 0, non-decreasing; a cluster
 *                may own zero rows, in which case its block row and column must be empty.
 *   level        n_clusters cluster levels (root = 0), used only for the tree hash.
 *   rowptr       n_clusters+1 block-row pointers, rowptr[0] = 0, non-decreasing.
 *   colidx       rowptr[n_clusters] block columns, strictly increasing within a row, in
 *                [0, n_clusters).
 * Validates every array (S_ERR_PATTERN on a violation) and uploads it to the current
 * device.  The pattern of Eq. (cutoff) is one instance; any block pattern is accepted. */
s_status s_pattern_create(int32_t n_clusters, const int64_t* block_offset, const int32_t* level,
                          const int64_t* rowptr, const int32_t* colidx, s_pattern* out);
s_status s_pattern_destroy(s_pattern p);
/* Number of stored entries (length of a value buffer), or -1 for a NULL pattern. */
int64_t s_pattern_nnz(s_pattern p);
/* Number of blocks, or -1. */
int64_t s_pattern_nblocks(s_pattern p);
/* Copies the nblocks+1 entry offsets of the blocks into host memory `out`. */
s_status s_pattern_block_offsets(s_pattern p, int64_t* out);
/* Borrowed host copies of the pattern's arrays (valid until s_pattern_destroy):
 * n_clusters, block_offset (n_clusters+1), rowptr (n_clusters+1), colidx (nblocks). */
s_status s_pattern_host_arrays(s_pattern p, int32_t* n_clusters, const int64_t** block_offset,
                               const int64_t** rowptr, const int32_t** colidx);

/* Batching: one pattern that holds `count` independent matrices side by side (block
 * diagonal in the union of their clusters, each part from its own tree).  The value buffer
 * of the result is the concatenation of the parts' value buffers in order, so one masked
 * product on the result computes all the parts' products in one launch.  The parts may be
 * destroyed afterwards. */
s_status s_pattern_concat(int32_t count, const s_pattern* parts, s_pattern* out);

/* ---- masked product, Eq. (product) of Thm. (product), Sec. 4.1 ---------------------- */

/* Symbolic phase of C = P_{S_C}(A B): checks that the three patterns share one tree,
 * builds the intersection work list of S_C x (S_A, S_B) on the device and counts the
 * block triples (nu, lambda, nu') and useful flops sum 2 n_nu n_lambda n_nu'.  The plan
 * keeps references to the patterns, which must outlive it. */
s_status s_plan_create(s_pattern A, s_pattern B, s_pattern C, s_prec prec, s_plan* out);
s_status s_plan_destroy(s_plan plan);
/* Exact triple count and useful flop count of the plan's product. */
s_status s_plan_stats(s_plan plan, int64_t* triples, double* flops);
/* Autotuner of S_FP64, S_FP32 and S_FP64_DF plans: times the kernel variants of the plan's
 * arithmetic (output tile edge, the micro-tile of one lane, for float also the lambda extent
 * of a stage) on the given operands and keeps the fastest for this plan's forward product.
 * (S_FP64 plans have tile edges 20 and 10; a plan whose output blocks have a
 * root-mean-square edge of at most 12 starts with 10, the others with 20.)
 * Each variant runs one timed warm-up launch; one more than twice as slow as the best so far
 * stops there, the others are timed over three more launches.  Float tile and row-panel
 * shapes narrower than the root-mean-square block edge of S_C are skipped.  C is
 * overwritten.  *chosen (optional) receives the variant index.  S_BF16X3 and S_TF32X3
 * plans have one shape (no-op).  Synchronises the stream. */
s_status s_plan_autotune(s_plan plan, const void* A, const void* B, void* C, void* stream, int* chosen);
/* Selects kernel variant `variant` (0 .. s_plan_num_variants_of(plan)-1) for the plan's
 * forward product by hand (S_FP64, S_FP32 and S_FP64_DF plans). */
s_status s_plan_set_variant(s_plan plan, int variant);
/* Number of float variants; number of variants of a plan's arithmetic (1 when fixed). */
int s_plan_num_variants(void);
int s_plan_num_variants_of(s_plan plan);
/* Declares that A's values are symmetric (A(nu, lambda) = A(lambda, nu)^T, as for a kernel
 * matrix in samplet coordinates).  The forward product then reads A(nu, lambda) through the
 * stored block (lambda, nu), which the float kernel stages with contiguous 16-byte copies.
 * Checks that A's pattern is symmetric (S_ERR_PATTERN otherwise); the values are the
 * caller's promise.  symmetric = 0 restores the default.  For an S_TF32X3 plan the flag
 * needs B's pattern to be A's and the product to be called with B = A (the same buffer);
 * the kernel then reads B(lambda, nu') through the stored block (nu', lambda) and both
 * operands from one set of split planes.  For an S_FP32 plan whose B pattern is A's, the
 * K-major kernel then reads B(lambda, nu') through the stored (nu', lambda) when called with
 * B = A (no transposed copy; the plan releases it), and falls back to the other kernel shape
 * of its tile list when called with another B. */
s_status s_plan_set_symmetric_a(s_plan plan, int symmetric);
/* Shape of a variant of the plan's arithmetic (variant < 0: the current one): output tile edge, the
 * micro-tile of one lane, and the largest lambda extent staged at once (consecutive small
 * lambda blocks are packed into one stage up to this extent).  Float variants 0 (the default)
 * and 1 are the K-major kernel: each lambda block staged by one bulk copy, the micro-tile a
 * quarter of each tile's padded edge (reported as 0 x 0), lambda staged in pieces of at most
 * 20; variant 1 addresses full 20-wide pieces with a compile-time row pitch.  For an S_TF32X3 plan: 32 rows
 * of a panel, 128 MMA rows (member columns), 32 MMA columns, lambda extent 24 per stage.
 * Any output may be NULL. */
s_status s_plan_variant(s_plan plan, int variant, int* tile, int* micro_rows, int* micro_cols, int* stage_k);

/* C = P_{S_C}(A B): for every block (nu, nu') of S_C,
 *   C(nu, nu') = sum over lambda with (nu,lambda) in S_A and (lambda,nu') in S_B of
 *                A(nu,lambda) B(lambda,nu');
 * no entry outside S_C is formed.  A, B, C are device value buffers on S_A, S_B, S_C in
 * the plan's element type; C must not alias A or B.  Deterministic: each output entry is
 * summed in a fixed order, so the same inputs give the same bits.  S_TF32X3
 * waits on its own tensor-core work and the K-major S_FP32 kernel on its own bulk copies,
 * each with a limit of about one second; if that ever runs out, the outputs are unspecified
 * (NaN where written after the time-out) and the plan records the time-out: the plan's next
 * s_mul_masked, s_graph_launch or s_plan_status returns S_ERR_TIMEOUT (launching nothing)
 * and clears the record. */
s_status s_mul_masked(s_plan plan, const void* A, const void* B, void* C, void* stream);

/* Synchronises `stream`, then reports the plan's device-side record: S_ERR_TIMEOUT (and the
 * record cleared) if a bounded wait of an earlier product or adjoint of this plan ran out,
 * else S_OK.  The kernels that wait on the device are the S_TF32X3 kernel (its tensor-core
 * work) and the K-major S_FP32 kernel (its bulk copies); the others never set the record. */
s_status s_plan_status(s_plan plan, void* stream);
/* Diagnostics: *word receives the host address of the plan's forward time-out word (pinned
 * host memory mapped into the device, 0 = no time-out).  A kernel stores 1 there when its
 * wait runs out; writing 1 from the host plants a time-out record, which is how the status
 * path is tested without making a device wait run out.  The word belongs to the plan (valid
 * until s_plan_destroy). */
s_status s_plan_timeout_word(s_plan plan, unsigned int** word);

/* Adjoint of s_mul_masked (reverse mode):  dA = P_{S_A}(dC B^T),  dB = P_{S_B}(A^T dC).
 * Either output may be NULL to skip it.  Same element type as the plan. */
s_status s_mul_masked_adjoint(s_plan plan, const void* dC, const void* A, const void* B, void* dA, void* dB,
                              void* stream);

/* CUDA graph of one s_mul_masked call on fixed buffers: captured on a private stream and
 * instantiated once; s_graph_launch replays it on any stream.  The plan and the buffers
 * must outlive the graph. */
typedef struct s_graph_t* s_graph;
s_status s_graph_capture_mul(s_plan plan, const void* A, const void* B, void* C, s_graph* out);
s_status s_graph_launch(s_graph g, void* stream);
s_status s_graph_destroy(s_graph g);

/* ---- addition, Sec. 4.1 ---------------------------------------------------------------- */

/* C = alpha A + beta B + gamma I on one pattern (B may be NULL when beta = 0; gamma != 0
 * needs every non-empty diagonal block in the pattern, else S_ERR_PATTERN).  prec selects
 * double (S_FP64) or float (S_FP32) buffers.  C may alias A or B. */
s_status s_add(s_pattern p, s_prec prec, double alpha, const void* A, double beta, const void* B, double gamma,
               void* C, void* stream);

/* Block-sparse times dense: Y = A X for `nvec` vectors, X and Y stored one vector after the
 * other (N x nvec, column-major, N = the pattern's dimension), double device buffers; Y must
 * not alias X.  With X an N x 10 matrix of uniform random entries this evaluates the error
 * estimator e_F(M) = ||M X||_F / ||X||_F of the multiplication benchmark (Sec. 5.1) for
 * M = A B - P_S(A B) as A (B X) - C X without forming M.  Asynchronous on the stream. */
s_status s_spmm(s_pattern p, const double* A, const double* X, int nvec, double* Y, void* stream);

/* ---- norm estimate and matrix functions ---------------------------------------------- */

/* Largest eigenvalue of a symmetric A (double buffer) by `iters` power steps with
 * Rayleigh quotients (Sec. 5.3), start vector all ones; the result is written to host
 * *lambda (the call synchronises the stream). */
s_status s_norm_est(s_pattern p, const double* A, int iters, double* lambda, void* stream);

/* Same estimate as s_norm_est, for callers that cannot allocate device memory during the
 * call (for example an application whose device memory is owned entirely by its own pool
 * allocator, or a latency-critical caller that must avoid cudaMalloc's device-wide
 * synchronisation).  The paper has no counterpart: this is a deployment variant.
 * It allocates nothing: its work vectors live in a static device array inside the library
 * sized for matrix dimensions up to 1048576 (2 x 2^20 doubles + 2, about 16 MiB), which every
 * GPU that loads the library holds until the process exits.  Larger patterns return
 * S_ERR_ARG.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before any stream
 * capture.  All calls share the one array, which keeps the contents of the last call (the
 * call clears what must start at zero): calls whose work overlaps on the GPU, on any
 * streams, race and give undefined results.  The pattern and A stay caller-owned; the call
 * synchronises the stream and writes the estimate to host *lambda. */
s_status s_norm_est_noalloc(s_pattern p, const double* A, int iters, double* lambda, void* stream);

typedef struct {
  int steps;          /* Newton-Schulz steps (S_SQRT); 0 = 25                              */
  int taylor_degree;  /* Taylor degree (S_EXP, S_EXP_NEG); 0 = 8                            */
  s_prec prec;        /* arithmetic of the products: S_FP64, S_FP64_DF, S_FP32, or a split
                         tensor-core form S_TF32X3 / S_BF16X3 (float iterates as for S_FP32) */
  double scale;       /* S_SQRT: c with Y_0 = A/c (0 = 1.01 * norm estimate);
                         S_EXP*: lambda used for the squaring count (0 = norm estimate)     */
  int squarings;      /* S_EXP*: -1 = from lambda, else forced count                        */
  double* residual;   /* optional host out: S_SQRT residual ||P_S(X X) - A||_F / ||A||_F    */
  void* checkpoints;  /* optional device buffer of 2*steps*nnz iterates: (Y_k, Z_k) per step,
                         doubles for S_FP64 and S_FP64_DF, floats for S_FP32                */
  int refine;         /* S_SQRT: residual-correction steps in double after the iteration:
                         R = A/c - P_S(Y Y), Y <- Y + P_S(Z R)/2 (Newton's method for
                         Y^2 = A/c with Z standing in for Y^{-1}); 0 = none               */
} s_funm_opts;

/* F = f(A) on A's pattern, every product masked to that pattern (the pattern must hold
 * its diagonal blocks).  A and F are double device buffers.
 *   S_SQRT     A^{1/2} by coupled Newton-Schulz: Y_0 = A/c, Z_0 = I,
 *              T_k = (3I - P_S(Z_k Y_k))/2, Y_{k+1} = P_S(Y_k T_k), Z_{k+1} = P_S(T_k Z_k),
 *              F = sqrt(c) Y_steps.  S_ERR_NOT_CONVERGED when ||T_k - I||_F is not finite, or
 *              grew by more than 1.5x on two consecutive steps while above 1e-3 of ||T_0 - I||_F.
 *   S_EXP, S_EXP_NEG   exp(+-A) by the power series of Sec. 4.4 truncated at the Taylor
 *              degree, Horner's rule on X = +-A/2^s, then s masked squarings,
 *              s = max(0, ceil(log2(lambda/0.5))).  With prec S_FP32 (or a split tensor-core
 *              form) the Horner products run in that arithmetic and the squarings in double.
 * With prec S_FP32, S_SQRT autotunes the float product kernel's shape on A first
 * (s_plan_autotune).  With prec S_FP64_DF the iterates are double and the products run in
 * double-float arithmetic.
 * Synchronises the stream once (norm estimate) unless opts->scale is given. */
s_status s_funm(s_pattern p, s_fn fn, const double* A, double* F, const s_funm_opts* opts, void* stream);

/* Reverse mode of S_SQRT (coupled Newton-Schulz, same recurrences as s_funm) with the
 * scaling c frozen: given dF = dL/dF on A's pattern and the per-step checkpoints
 * (Y_k, Z_k), k = 0..steps-1, that s_funm wrote into opts->checkpoints (2*steps*nnz
 * doubles), writes dA = dL/dA on A's pattern.  Each step replays P = P_S(Z_k Y_k) and
 * T_k = (3I - P)/2 and applies the adjoints of Y' = P_S(Y T), Z' = P_S(T Z) and
 * P = P_S(Z Y), each a pair of masked products (see s_mul_masked_adjoint).  Double
 * buffers; prec S_FP64.  Allocates its work buffers; synchronises the stream. */
s_status s_funm_sqrt_backward(s_pattern p, int steps, double c, const double* checkpoints, const double* dF,
                              double* dA, void* stream);

/* The same reverse mode for the iteration run in another arithmetic: prec S_FP64 is
 * s_funm_sqrt_backward; prec S_FP32 differentiates the float iteration of s_funm with prec
 * S_FP32 (its residual corrections, a small change of the result, are not differentiated):
 * `checkpoints` holds 2*steps*nnz floats written by that s_funm call, every adjoint product
 * is a compensated-float masked product (S_FP32 plans) and the adjoint iterates are float;
 * dF and dA are double.  About half the memory and a fraction of the time of the double
 * form, at float accuracy (relative error of dA near 1e-6).  Allocates its work buffers;
 * synchronises the stream. */
s_status s_funm_sqrt_backward_prec(s_pattern p, s_prec prec, int steps, double c, const void* checkpoints,
                                   const double* dF, double* dA, void* stream);

/* Loss of the differentiation checks: *out (host) = z^T X z = sum over the blocks (nu, nu') of
 * the pattern of z_nu^T X(nu, nu') z_nu', with z a device vector of the pattern's dimension in
 * samplet coordinates (fixed-order reduction; synchronises the stream). */
s_status s_quad_form(s_pattern p, const double* X, const double* z, double* out, void* stream);
/* Its gradient: dX(nu, nu') = z_nu z_nu'^T on every block of the pattern. */
s_status s_quad_form_grad(s_pattern p, const double* z, double* dX, void* stream);

/* ---- diagnostics ------------------------------------------------------------------------ */
/* Measured multiply-add rate of this device in flop/s (2 per fused multiply-add), for the
 * roofline denominators of the float (S_FP32) and double (S_FP64) product kernels:
 * independent FMA chains on every lane of a grid of 8 CTAs of 256 threads per SM, the second of
 * two launches timed with CUDA events on `stream`.  Synchronises the stream. */
s_status s_peak_fma(s_prec prec, double* flops_per_s, void* stream);
const char* s_last_error(void);
/* Library version string. */
const char* s_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SFORMAT_H */
