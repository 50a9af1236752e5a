// Streaming kernels on S-format value buffers: C = alpha A + beta B + gamma I (addition on
// a common pattern, Sec. 4.1), block-sparse matrix-vector product and reductions used by
// the norm estimate and the drivers.  All HBM-bound.
#include <algorithm>

#include "common.cuh"

namespace sf {

template <typename T>
__global__ void axpby_kernel(int64_t n, T alpha, const T* __restrict__ A, T beta, const T* __restrict__ B,
                             T* __restrict__ C) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
    T v = alpha * A[i];
    if (B) v = fma(beta, B[i], v);
    C[i] = v;
  }
}

template <typename T>
__global__ void add_diag_kernel(int32_t nc, const int32_t* diag, const int32_t* bsize, const int64_t* voff, T gamma,
                                T* C) {
  const int32_t nu = blockIdx.x;
  if (nu >= nc) return;
  const int k = diag[nu];
  if (k < 0) return;
  const int n = bsize[nu];
  for (int r = threadIdx.x; r < n; r += blockDim.x) C[voff[k] + (int64_t)r * n + r] += gamma;
}

static int grid_for(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 8));
}

s_status run_add(const s_pattern_t* p, s_prec prec, double alpha, const void* A, double beta, const void* B,
                 double gamma, void* C, cudaStream_t st) {
  const int64_t n = p->d.nnz;
  if (gamma != 0.0 && !p->has_all_diag) return set_error(S_ERR_PATTERN, "s_add: gamma*I needs every diagonal block");
  if (prec == S_FP64) {
    if (n) axpby_kernel<double><<<grid_for(n), 256, 0, st>>>(n, alpha, (const double*)A, beta, (const double*)B, (double*)C);
    if (gamma != 0.0)
      add_diag_kernel<double><<<p->d.nc, 64, 0, st>>>(p->d.nc, p->d.diag, p->d.bsize, p->d.voff, gamma, (double*)C);
  } else if (prec == S_FP32) {
    if (n)
      axpby_kernel<float><<<grid_for(n), 256, 0, st>>>(n, (float)alpha, (const float*)A, (float)beta, (const float*)B,
                                                       (float*)C);
    if (gamma != 0.0)
      add_diag_kernel<float><<<p->d.nc, 64, 0, st>>>(p->d.nc, p->d.diag, p->d.bsize, p->d.voff, (float)gamma, (float*)C);
  } else {
    return set_error(S_ERR_ARG, "s_add: prec must be S_FP64 or S_FP32");
  }
  SF_CUDA(cudaGetLastError());
  return S_OK;
}

// y = A x.  One CTA per block row; each warp accumulates a private partial row sum over a
// strided subset of the row's blocks; the partials are added in warp order.
constexpr int kSpmvWarps = 4;
__global__ void spmv_kernel(int32_t nc, const int32_t* bsize, const int64_t* boff, const int64_t* rowptr,
                            const int32_t* colidx, const int64_t* voff, const double* __restrict__ A,
                            const double* __restrict__ x, double* __restrict__ y, int maxb) {
  extern __shared__ double part[];  // kSpmvWarps * maxb
  const int nu = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int ni = bsize[nu];
  for (int r = threadIdx.x; r < kSpmvWarps * maxb; r += blockDim.x) part[r] = 0.0;
  __syncthreads();
  for (int64_t k = rowptr[nu] + w; k < rowptr[nu + 1]; k += kSpmvWarps) {
    const int j = colidx[k], nj = bsize[j];
    const double* blk = A + voff[k];
    const double* xj = x + boff[j];
    for (int r = lane; r < ni; r += 32) {
      double s = 0.0;
      for (int c = 0; c < nj; ++c) s = fma(blk[(int64_t)r * nj + c], xj[c], s);
      part[w * maxb + r] += s;
    }
  }
  __syncthreads();
  for (int r = threadIdx.x; r < ni; r += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < kSpmvWarps; ++q) s += part[q * maxb + r];
    y[boff[nu] + r] = s;
  }
}

s_status run_spmv_f64(const s_pattern_t* p, const double* A, const double* x, double* y, cudaStream_t st) {
  const int maxb = std::max(1, p->d.max_bsize);
  spmv_kernel<<<p->d.nc, kSpmvWarps * 32, sizeof(double) * kSpmvWarps * maxb, st>>>(
      p->d.nc, p->d.bsize, p->d.boff, p->d.rowptr, p->d.colidx, p->d.voff, A, x, y, maxb);
  SF_CUDA(cudaGetLastError());
  return S_OK;
}

}  // namespace sf

using namespace sf;

extern "C" s_status s_spmm(s_pattern p, const double* A, const double* X, int nvec, double* Y, void* stream) {
  if (!p || !A || !X || !Y || nvec < 0) return set_error(S_ERR_ARG, "s_spmm: bad argument");
  if (X == Y) return set_error(S_ERR_ARG, "s_spmm: Y aliases X");
  const int64_t n = p->d.n;
  for (int j = 0; j < nvec && n > 0; ++j) {
    s_status st = run_spmv_f64(p, A, X + (int64_t)j * n, Y + (int64_t)j * n, (cudaStream_t)stream);
    if (st) return st;
  }
  return S_OK;
}

extern "C" s_status s_add(s_pattern p, s_prec prec, double alpha, const void* A, double beta, const void* B,
                          double gamma, void* C, void* stream) {
  if (!p || !A || !C || (beta != 0.0 && !B)) return set_error(S_ERR_ARG, "s_add: NULL argument");
  return run_add(p, prec, alpha, A, beta, beta != 0.0 ? B : nullptr, gamma, C, (cudaStream_t)stream);
}
