// Largest-eigenvalue estimate that allocates no device memory.
//
// s_norm_est() takes its work vectors from cudaMalloc on every call.  Some callers cannot
// allow that: an application whose device memory is handed out entirely by its own pool
// allocator, or a latency-sensitive caller that must not pay cudaMalloc's implicit
// device-wide synchronisation.  s_norm_est_noalloc() computes the same power iteration
// with Rayleigh quotients (Sec. 5.3) using a scratch array of fixed size that lives in
// this file as a static __device__ variable: two vectors of up to kNoallocMaxN doubles plus
// two reduction slots (16 MiB + 16 B).  Every GPU that loads the library keeps that array
// until the process exits.
#include <mutex>
#include <string>

#include "common.cuh"

namespace sf {

constexpr int64_t kNoallocMaxN = int64_t(1) << 20;  // largest matrix dimension accepted

// [x (kNoallocMaxN) | y (kNoallocMaxN) | x.y | y.y]
static __device__ __align__(256) double g_noalloc_scratch[2 * kNoallocMaxN + 2];

namespace {

__global__ void na_fill(int64_t n, double v, double* x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = v;
}

// out = a.b, one CTA, fixed summation order
__global__ void na_dot(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double* out) {
  __shared__ double red[1024];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s = fma(a[i], b[i], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// x = y / sqrt(*yy); x unchanged when y = 0
__global__ void na_normalize(int64_t n, const double* y, const double* yy, double* x) {
  const double s = *yy;
  if (s <= 0.0) return;
  const double inv = 1.0 / sqrt(s);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = y[i] * inv;
}

std::mutex g_noalloc_mu;
double* g_noalloc_ptr[256] = {};  // device address of g_noalloc_scratch, per device ordinal

// Device address of the scratch array on the current device.  In host code the symbol
// g_noalloc_scratch is only a host-side stand-in; the address comes from
// cudaGetSymbolAddress, looked up once per device with that device current.
s_status noalloc_scratch(double** out) {
  int dev = 0;
  SF_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return set_error(S_ERR_ARG, "s_norm_est_noalloc: device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_ptr[dev] = (double*)p;
  }
  *out = g_noalloc_ptr[dev];
  return S_OK;
}

}  // namespace
}  // namespace sf

using namespace sf;

extern "C" s_status s_norm_est_noalloc(s_pattern p, const double* A, int iters, double* lambda, void* stream) {
  if (!p || !A || !lambda || iters < 1) return set_error(S_ERR_ARG, "s_norm_est_noalloc: bad argument");
  const int64_t n = p->d.n;
  if (n > kNoallocMaxN)
    return set_error(S_ERR_ARG, "s_norm_est_noalloc: matrix dimension " + std::to_string(n) +
                                    " exceeds the static scratch limit of 1048576");
  double* s = nullptr;
  s_status st = noalloc_scratch(&s);
  if (st) return st;
  cudaStream_t cs = (cudaStream_t)stream;
  double* x = s;
  double* y = s + kNoallocMaxN;
  double* sc = s + 2 * kNoallocMaxN;  // sc[0] = x.y, sc[1] = y.y; cleared on every call
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096));
  na_fill<<<grid, 256, 0, cs>>>(n, 1.0 / std::sqrt((double)n), x);
  SF_CUDA(cudaMemsetAsync(sc, 0, 2 * sizeof(double), cs));
  for (int it = 0; it < iters; ++it) {
    if ((st = run_spmv_f64(p, A, x, y, cs))) return st;
    na_dot<<<1, 1024, 0, cs>>>(n, x, y, sc);
    na_dot<<<1, 1024, 0, cs>>>(n, y, y, sc + 1);
    na_normalize<<<grid, 256, 0, cs>>>(n, y, sc + 1, x);
  }
  SF_CUDA(cudaGetLastError());
  double h[2] = {0.0, 0.0};
  SF_CUDA(cudaMemcpyAsync(h, sc, sizeof(h), cudaMemcpyDeviceToHost, cs));
  SF_CUDA(cudaStreamSynchronize(cs));
  *lambda = h[0];
  return S_OK;
}
