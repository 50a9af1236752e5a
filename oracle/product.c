/*
 * Plain C, FP64 oracle for the S-format masked product and block-sparse matrix-vector
 * product.  TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the CPU
 * baseline of the benchmark load it; the product library never does.
 *
 * Masked product, Eq. (product) of Thm. (product), Sec. 4.1: for every block (nu, nu') of
 * the output pattern S_C,
 *     C(nu, nu') = sum_{lambda : (nu,lambda) in S_A, (lambda,nu') in S_B} A(nu,lambda) B(lambda,nu'),
 * each term a plain i-k-j block product in double precision, lambda in increasing order.
 * Entries outside S_C are never formed ("exact on the given compression pattern",
 * Sec. 4.1).  No BLAS, no blocking, no reordering beyond the definition.
 *
 * Block-CSR layout (the oracle's own): cluster nu owns bsize[nu] rows; block k of row nu
 * is (nu, col[k]) for rowptr[nu] <= k < rowptr[nu+1], columns sorted; its entries are
 * row-major at val[voff[k] ...].  All index arrays are int64.
 */
#include <stdint.h>
#include <string.h>

static int64_t find_block(const int64_t* rowptr, const int64_t* col, int64_t row, int64_t c) {
  int64_t lo = rowptr[row], hi = rowptr[row + 1];
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (col[mid] < c) lo = mid + 1;
    else hi = mid;
  }
  return (lo < rowptr[row + 1] && col[lo] == c) ? lo : -1;
}

/* One output block k of C. */
static void one_block(int64_t k, const int64_t* bsize,
                      const int64_t* a_rowptr, const int64_t* a_col, const int64_t* a_voff, const double* a_val,
                      const int64_t* b_rowptr, const int64_t* b_col, const int64_t* b_voff, const double* b_val,
                      const int64_t* c_brow, const int64_t* c_col, const int64_t* c_voff, double* c_val) {
  int64_t i = c_brow[k], j = c_col[k];
  int64_t ni = bsize[i], nj = bsize[j];
  double* C = c_val + c_voff[k];
  memset(C, 0, sizeof(double) * (size_t)(ni * nj));
  for (int64_t ka = a_rowptr[i]; ka < a_rowptr[i + 1]; ++ka) {
    int64_t lam = a_col[ka];
    int64_t kb = find_block(b_rowptr, b_col, lam, j);
    if (kb < 0) continue;
    int64_t nl = bsize[lam];
    const double* A = a_val + a_voff[ka];
    const double* B = b_val + b_voff[kb];
    for (int64_t r = 0; r < ni; ++r)
      for (int64_t t = 0; t < nl; ++t) {
        double a = A[r * nl + t];
        for (int64_t c = 0; c < nj; ++c) C[r * nj + c] += a * B[t * nj + c];
      }
  }
}

/* C = P_{S_C}(A B).  If subset != NULL only the listed C blocks are computed. */
int oracle_mul_masked(const int64_t* bsize,
                      const int64_t* a_rowptr, const int64_t* a_col, const int64_t* a_voff, const double* a_val,
                      const int64_t* b_rowptr, const int64_t* b_col, const int64_t* b_voff, const double* b_val,
                      int64_t c_nblocks, const int64_t* c_brow, const int64_t* c_col, const int64_t* c_voff,
                      double* c_val, const int64_t* subset, int64_t nsubset, int nthreads) {
  int64_t n = subset ? nsubset : c_nblocks;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
  for (int64_t s = 0; s < n; ++s) {
    int64_t k = subset ? subset[s] : s;
    one_block(k, bsize, a_rowptr, a_col, a_voff, a_val, b_rowptr, b_col, b_voff, b_val, c_brow, c_col, c_voff,
              c_val);
  }
  return 0;
}

/* Number of block triples (nu, lambda, nu') the product visits and its useful flop count
   sum 2 n_nu n_lambda n_nu' (over the listed C blocks if subset != NULL). */
int oracle_mul_count(const int64_t* bsize, const int64_t* a_rowptr, const int64_t* a_col,
                     const int64_t* b_rowptr, const int64_t* b_col, int64_t c_nblocks, const int64_t* c_brow,
                     const int64_t* c_col, const int64_t* subset, int64_t nsubset, int64_t* triples, double* flops) {
  int64_t t = 0;
  double f = 0.0;
  int64_t n = subset ? nsubset : c_nblocks;
  for (int64_t s = 0; s < n; ++s) {
    int64_t k = subset ? subset[s] : s;
    int64_t i = c_brow[k], j = c_col[k];
    for (int64_t ka = a_rowptr[i]; ka < a_rowptr[i + 1]; ++ka) {
      int64_t lam = a_col[ka];
      if (find_block(b_rowptr, b_col, lam, j) < 0) continue;
      ++t;
      f += 2.0 * (double)bsize[i] * (double)bsize[lam] * (double)bsize[j];
    }
  }
  *triples = t;
  *flops = f;
  return 0;
}

/* y = A x, block by block, for the norm estimate. */
int oracle_spmv(int64_t nclusters, const int64_t* bsize, const int64_t* boff, const int64_t* rowptr,
                const int64_t* col, const int64_t* voff, const double* val, const double* x, double* y) {
  for (int64_t i = 0; i < nclusters; ++i) {
    int64_t ni = bsize[i];
    for (int64_t r = 0; r < ni; ++r) y[boff[i] + r] = 0.0;
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      int64_t j = col[k], nj = bsize[j];
      const double* A = val + voff[k];
      for (int64_t r = 0; r < ni; ++r) {
        double s = 0.0;
        for (int64_t c = 0; c < nj; ++c) s += A[r * nj + c] * x[boff[j] + c];
        y[boff[i] + r] += s;
      }
    }
  }
  return 0;
}
