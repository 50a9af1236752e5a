// Arithmetic-rate probe for the roofline denominators of the product kernels: independent
// fused multiply-add chains on every lane of a grid that fills the device, timed with CUDA
// events.  Diagnostic only (not part of the S-format algebra).
#include <algorithm>

#include "common.cuh"

namespace sf {
namespace {

constexpr int kPeakChains = 8;  // independent chains per thread (covers the FMA latency)

template <typename T>
__global__ void __launch_bounds__(256) peak_fma_kernel(int iters, T a, T b, T* out) {
  T c[kPeakChains];
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) c[k] = (T)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) c[k] = c[k] * a + b;  // one fused multiply-add
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) s += c[k];
  if (s == (T)-1.2345) out[blockIdx.x] = s;  // keeps the chains live; never true for these inputs
}

}  // namespace
}  // namespace sf

using namespace sf;

extern "C" s_status s_peak_fma(s_prec prec, double* flops_per_s, void* stream) {
  if (!flops_per_s || (prec != S_FP32 && prec != S_FP64)) return set_error(S_ERR_ARG, "s_peak_fma: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  const int blocks = sm_count() * 8, threads = 256;
  const int iters = prec == S_FP32 ? 1 << 16 : 1 << 13;
  void* out = nullptr;
  SF_CUDA(cudaMalloc(&out, sizeof(double) * blocks));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms = 0.0f;
  cudaError_t e = cudaSuccess;
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first launch warms up
    cudaEventRecord(e0, st);
    if (prec == S_FP32)
      peak_fma_kernel<float><<<blocks, threads, 0, st>>>(iters, 0.999999f, 1e-7f, (float*)out);
    else
      peak_fma_kernel<double><<<blocks, threads, 0, st>>>(iters, 0.999999, 1e-7, (double*)out);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return cuda_error(e, "s_peak_fma");
  *flops_per_s = 2.0 * (double)blocks * threads * kPeakChains * iters / (ms * 1e-3);
  return S_OK;
}
