// Norm estimate (power iteration with Rayleigh quotients, as Sec. 5.3 estimates
// ||K^eta||_2) and the two matrix-function drivers built on the masked product:
// coupled Newton-Schulz for A^{1/2} and the truncated power series of exp (Sec. 4.4) by
// Horner's rule with scaling and squaring.  Every iterate lives on A's pattern.
#include <cmath>
#include <vector>

#include "common.cuh"

namespace sf {

// out[0] = sum_i a_i b_i  (single CTA tree reduction in a fixed order: deterministic)
__global__ void dot_kernel(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double* out) {
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

__global__ void fill_kernel(int64_t n, double v, double* x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) x[i] = v;
}

// x = y / sqrt(yy[0])  (yy = y.y on the device); leaves x unchanged when y = 0
__global__ void normalize_kernel(int64_t n, const double* y, const double* yy, double* x) {
  const double s = *yy;
  if (s <= 0.0) return;
  const double inv = 1.0 / sqrt(s);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = y[i] * inv;
}

// out[0] = ||T - I||_F^2 = sum T_ij^2 - 2 trace(T) + n on a pattern holding every diagonal
// block (single CTA, fixed order)
template <typename T>
__global__ void dist_to_identity_kernel(int64_t nnz, const T* __restrict__ v, int32_t nc, const int32_t* diag,
                                        const int32_t* bsize, const int64_t* voff, double n, double* out) {
  __shared__ double red[1024];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < nnz; i += blockDim.x) s += (double)v[i] * (double)v[i];
  for (int32_t nu = threadIdx.x; nu < nc; nu += blockDim.x) {
    const int k = diag[nu];
    if (k < 0) continue;
    const int b = bsize[nu];
    for (int r = 0; r < b; ++r) s -= 2.0 * (double)v[voff[k] + (int64_t)r * b + r];
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0] + n;
}

template <typename S, typename D>
__global__ void convert_kernel(int64_t n, const S* a, D* b, double scale) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (D)((double)a[i] * scale);
}

static int grid_of(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096)); }

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { cudaFree(p); }
};

// Declared after the buffers a call uses: its destructor runs first and waits for the
// queued kernels, so no buffer is freed under a running kernel.
struct SyncOnExit {
  cudaStream_t s;
  ~SyncOnExit() { cudaStreamSynchronize(s); }
};

s_status norm_estimate(const s_pattern_t* p, const double* A, int iters, double* lambda, cudaStream_t st) {
  const int64_t n = p->d.n;
  DevBuf bx, by, bs;
  SF_CUDA(cudaMalloc(&bx.p, sizeof(double) * n));
  SF_CUDA(cudaMalloc(&by.p, sizeof(double) * n));
  SF_CUDA(cudaMalloc(&bs.p, sizeof(double) * 2));
  SyncOnExit sync{st};
  double* x = (double*)bx.p;
  double* y = (double*)by.p;
  double* sc = (double*)bs.p;  // sc[0] = x.y (Rayleigh quotient), sc[1] = y.y
  fill_kernel<<<grid_of(n), 256, 0, st>>>(n, 1.0 / std::sqrt((double)n), x);
  SF_CUDA(cudaMemsetAsync(sc, 0, sizeof(double) * 2, st));
  for (int it = 0; it < iters; ++it) {
    s_status s = run_spmv_f64(p, A, x, y, st);
    if (s) return s;
    dot_kernel<<<1, 1024, 0, st>>>(n, x, y, sc);
    dot_kernel<<<1, 1024, 0, st>>>(n, y, y, sc + 1);
    normalize_kernel<<<grid_of(n), 256, 0, st>>>(n, y, sc + 1, x);
  }
  SF_CUDA(cudaGetLastError());
  double h[2];
  SF_CUDA(cudaMemcpyAsync(h, sc, sizeof(h), cudaMemcpyDeviceToHost, st));
  SF_CUDA(cudaStreamSynchronize(st));
  *lambda = h[0];
  return S_OK;
}

}  // namespace sf

using namespace sf;

extern "C" s_status s_norm_est(s_pattern p, const double* A, int iters, double* lambda, void* stream) {
  if (!p || !A || !lambda || iters < 1) return set_error(S_ERR_ARG, "s_norm_est: bad argument");
  return norm_estimate(p, A, iters, lambda, (cudaStream_t)stream);
}

extern "C" s_status s_funm(s_pattern p, s_fn fn, const double* A, double* F, const s_funm_opts* opts, void* stream) {
  if (!p || !A || !F) return set_error(S_ERR_ARG, "s_funm: NULL argument");
  if (!p->has_all_diag) return set_error(S_ERR_PATTERN, "s_funm: the pattern must hold every diagonal block");
  cudaStream_t st = (cudaStream_t)stream;
  s_funm_opts o = {};
  if (opts) o = *opts;
  const s_prec prec = o.prec;
  if (prec != S_FP64 && prec != S_FP32) return set_error(S_ERR_ARG, "s_funm: prec must be S_FP64 or S_FP32");
  const size_t w = prec == S_FP64 ? sizeof(double) : sizeof(float);
  const int64_t nnz = p->d.nnz;
  s_plan plan = nullptr;
  s_status s = s_plan_create(p, p, p, prec, &plan);
  if (s) return s;
  struct PlanGuard {
    s_plan q;
    ~PlanGuard() { s_plan_destroy(q); }
  } pg{plan};
  const int64_t g = grid_of(nnz);
  if (fn == S_SQRT) {
    const int steps = o.steps > 0 ? o.steps : 25;
    double c = o.scale;
    if (c <= 0.0) {
      double lam = 0.0;
      if ((s = norm_estimate(p, A, 50, &lam, st))) return s;
      c = 1.01 * lam;
    }
    if (!(c > 0.0)) return set_error(S_ERR_ARG, "s_funm: non-positive scaling (is A positive definite?)");
    DevBuf bY, bZ, bT, bP, bA, bN;
    SF_CUDA(cudaMalloc(&bY.p, w * nnz + 16));
    SF_CUDA(cudaMalloc(&bZ.p, w * nnz + 16));
    SF_CUDA(cudaMalloc(&bT.p, w * nnz + 16));
    SF_CUDA(cudaMalloc(&bP.p, w * nnz + 16));
    SF_CUDA(cudaMalloc(&bN.p, sizeof(double) * (steps + 1)));
    SyncOnExit sync{st};
    void *Y = bY.p, *Z = bZ.p, *T = bT.p, *P = bP.p;
    const void* Ain = A;
    if (prec == S_FP32) {
      SF_CUDA(cudaMalloc(&bA.p, w * nnz + 16));
      convert_kernel<double, float><<<g, 256, 0, st>>>(nnz, A, (float*)bA.p, 1.0);
      Ain = bA.p;
    }
    // Y_0 = A / c, Z_0 = I
    if ((s = run_add(p, prec, 1.0 / c, Ain, 0.0, nullptr, 0.0, Y, st))) return s;
    SF_CUDA(cudaMemsetAsync(Z, 0, w * nnz, st));
    if ((s = run_add(p, prec, 1.0, Z, 0.0, nullptr, 1.0, Z, st))) return s;
    for (int k = 0; k < steps; ++k) {
      if (o.checkpoints && prec == S_FP64) {
        double* ck = (double*)o.checkpoints + (int64_t)2 * k * nnz;
        SF_CUDA(cudaMemcpyAsync(ck, Y, w * nnz, cudaMemcpyDeviceToDevice, st));
        SF_CUDA(cudaMemcpyAsync(ck + nnz, Z, w * nnz, cudaMemcpyDeviceToDevice, st));
      }
      if ((s = run_mul(plan->fwd, prec, Z, Y, P, st))) return s;                 // P = P_S(Z Y)
      if ((s = run_add(p, prec, -0.5, P, 0.0, nullptr, 1.5, T, st))) return s;   // T = (3I - P)/2
      if (prec == S_FP64)
        dist_to_identity_kernel<double><<<1, 1024, 0, st>>>(nnz, (const double*)T, p->d.nc, p->d.diag, p->d.bsize,
                                                            p->d.voff, (double)p->d.n, (double*)bN.p + k);
      else
        dist_to_identity_kernel<float><<<1, 1024, 0, st>>>(nnz, (const float*)T, p->d.nc, p->d.diag, p->d.bsize,
                                                           p->d.voff, (double)p->d.n, (double*)bN.p + k);
      if ((s = run_mul(plan->fwd, prec, Y, T, P, st))) return s;                 // Y' = P_S(Y T)
      std::swap(Y, P);
      if ((s = run_mul(plan->fwd, prec, T, Z, P, st))) return s;                 // Z' = P_S(T Z)
      std::swap(Z, P);
    }
    const double sc = std::sqrt(c);
    if (prec == S_FP64) {
      if ((s = run_add(p, prec, sc, Y, 0.0, nullptr, 0.0, F, st))) return s;
    } else {
      convert_kernel<float, double><<<g, 256, 0, st>>>(nnz, (const float*)Y, F, sc);
      SF_CUDA(cudaGetLastError());
    }
    // divergence: ||T_k - I||_F grew by more than 1.5x on two consecutive steps
    {
      std::vector<double> dk(steps);
      SF_CUDA(cudaMemcpyAsync(dk.data(), bN.p, sizeof(double) * steps, cudaMemcpyDeviceToHost, st));
      SF_CUDA(cudaStreamSynchronize(st));
      for (int k = 2; k < steps; ++k)
        if (dk[k] > 2.25 * dk[k - 1] && dk[k - 1] > 2.25 * dk[k - 2])   // squared norms: 1.5^2
          return set_error(S_ERR_NOT_CONVERGED, "s_funm: Newton-Schulz iteration diverged at step " + std::to_string(k));
    }
    if (o.residual) {
      // ||P_S(F F) - A||_F / ||A||_F in double
      s_plan p64 = nullptr;
      if ((s = s_plan_create(p, p, p, S_FP64, &p64))) return s;
      PlanGuard pg2{p64};
      DevBuf bR, bd;
      SF_CUDA(cudaMalloc(&bR.p, sizeof(double) * nnz + 16));
      SF_CUDA(cudaMalloc(&bd.p, sizeof(double) * 2));
      SyncOnExit sync2{st};
      if ((s = run_mul(p64->fwd, S_FP64, F, F, bR.p, st))) return s;
      if ((s = run_add(p, S_FP64, 1.0, bR.p, -1.0, A, 0.0, bR.p, st))) return s;
      dot_kernel<<<1, 1024, 0, st>>>(nnz, (const double*)bR.p, (const double*)bR.p, (double*)bd.p);
      dot_kernel<<<1, 1024, 0, st>>>(nnz, A, A, (double*)bd.p + 1);
      double h[2];
      SF_CUDA(cudaMemcpyAsync(h, bd.p, sizeof(h), cudaMemcpyDeviceToHost, st));
      SF_CUDA(cudaStreamSynchronize(st));
      *o.residual = std::sqrt(h[0]) / std::sqrt(h[1]);
    }
    return S_OK;
  }
  if (fn == S_EXP || fn == S_EXP_NEG) {
    const int m = o.taylor_degree > 0 ? o.taylor_degree : 8;
    int sq = o.squarings;
    if (sq < 0 || !opts) {
      double lam = o.scale;
      if (lam <= 0.0 && (s = norm_estimate(p, A, 50, &lam, st))) return s;
      lam = std::fabs(lam);
      sq = lam <= 0.5 ? 0 : std::max(0, (int)std::ceil(std::log2(lam / 0.5)));
    }
    const double sign = fn == S_EXP ? 1.0 : -1.0;
    DevBuf bX, bE, bW;
    SF_CUDA(cudaMalloc(&bX.p, w * nnz + 16));
    SF_CUDA(cudaMalloc(&bE.p, w * nnz + 16));
    SF_CUDA(cudaMalloc(&bW.p, w * nnz + 16));
    SyncOnExit sync{st};
    void *X = bX.p, *E = bE.p, *W = bW.p;
    const double xs = sign / std::ldexp(1.0, sq);
    if (prec == S_FP64) {
      if ((s = run_add(p, prec, xs, A, 0.0, nullptr, 0.0, X, st))) return s;
    } else {
      convert_kernel<double, float><<<g, 256, 0, st>>>(nnz, A, (float*)X, xs);
    }
    if ((s = run_add(p, prec, 1.0 / m, X, 0.0, nullptr, 1.0, E, st))) return s;   // E = I + X/m
    for (int k = m - 1; k >= 1; --k) {
      if ((s = run_mul(plan->fwd, prec, X, E, W, st))) return s;                   // W = P_S(X E)
      if ((s = run_add(p, prec, 1.0 / k, W, 0.0, nullptr, 1.0, E, st))) return s; // E = I + W/k
    }
    for (int r = 0; r < sq; ++r) {
      if ((s = run_mul(plan->fwd, prec, E, E, W, st))) return s;                   // E = P_S(E E)
      std::swap(E, W);
    }
    if (prec == S_FP64) {
      SF_CUDA(cudaMemcpyAsync(F, E, w * nnz, cudaMemcpyDeviceToDevice, st));
    } else {
      convert_kernel<float, double><<<g, 256, 0, st>>>(nnz, (const float*)E, F, 1.0);
      SF_CUDA(cudaGetLastError());
    }
    SF_CUDA(cudaStreamSynchronize(st));
    return S_OK;
  }
  return set_error(S_ERR_ARG, "s_funm: unknown function");
}
