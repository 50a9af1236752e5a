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

// part[k] = z_nu^T X(nu, nu') z_nu' for block k = (nu, nu')
__global__ void quad_part_kernel(int64_t nb, const int32_t* brow, const int32_t* bcol, const int32_t* bsize,
                                 const int64_t* boff, const int64_t* voff, const double* X, const double* z,
                                 double* part) {
  const int lane = threadIdx.x & 31;
  const int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (k >= nb) return;
  const int i = brow[k], j = bcol[k];
  const int ni = bsize[i], nj = bsize[j];
  const double* x = X + voff[k];
  const double* zi = z + boff[i];
  const double* zj = z + boff[j];
  double s = 0.0;
  for (int e = lane; e < ni * nj; e += 32) {
    const int r = e / nj, c = e - r * nj;
    s = fma(zi[r] * x[e], zj[c], s);
  }
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) part[k] = s;
}

// dX(nu, nu') = z_nu z_nu'^T on every block of the pattern
__global__ void quad_grad_kernel(int64_t nb, const int32_t* brow, const int32_t* bcol, const int32_t* bsize,
                                 const int64_t* boff, const int64_t* voff, const double* z, double* dX) {
  const int lane = threadIdx.x & 31;
  const int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (k >= nb) return;
  const int i = brow[k], j = bcol[k];
  const int ni = bsize[i], nj = bsize[j];
  for (int e = lane; e < ni * nj; e += 32) {
    const int r = e / nj, c = e - r * nj;
    dX[voff[k] + e] = z[boff[i] + r] * z[boff[j] + c];
  }
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
  if (prec != S_FP64 && prec != S_FP32 && prec != S_FP64_DF && prec != S_TF32X3 && prec != S_BF16X3)
    return set_error(S_ERR_ARG, "s_funm: prec must be S_FP64, S_FP64_DF, S_FP32, S_TF32X3 or S_BF16X3");
  // iterates are double for S_FP64 and S_FP64_DF (products in double-float), float for S_FP32
  // and for the split tensor-core forms (S_TF32X3, S_BF16X3: float in, float out)
  const s_prec aprec = (prec == S_FP64 || prec == S_FP64_DF) ? S_FP64 : S_FP32;
  const size_t w = aprec == S_FP64 ? sizeof(double) : sizeof(float);
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
    if (aprec == S_FP32) {
      SF_CUDA(cudaMalloc(&bA.p, w * nnz + 16));
      convert_kernel<double, float><<<g, 256, 0, st>>>(nnz, A, (float*)bA.p, 1.0);
      Ain = bA.p;
      if (prec == S_FP32 && (s = s_plan_autotune(plan, Ain, Ain, P, st, nullptr))) return s;  // kernel shape
    }
    if (prec == S_FP64_DF) {
      if ((s = s_plan_autotune(plan, A, A, P, st, nullptr))) return s;  // kernel shape
    }
    // Y_0 = A / c, Z_0 = I
    if ((s = run_add(p, aprec, 1.0 / c, Ain, 0.0, nullptr, 0.0, Y, st))) return s;
    SF_CUDA(cudaMemsetAsync(Z, 0, w * nnz, st));
    if ((s = run_add(p, aprec, 1.0, Z, 0.0, nullptr, 1.0, Z, st))) return s;
    const int refine = std::max(0, o.refine);
    for (int k = 0; k < steps; ++k) {
      if (o.checkpoints) {  // (Y_k, Z_k) in the iterates' element type
        char* ck = (char*)o.checkpoints + (int64_t)2 * k * nnz * (int64_t)w;
        SF_CUDA(cudaMemcpyAsync(ck, Y, w * nnz, cudaMemcpyDeviceToDevice, st));
        SF_CUDA(cudaMemcpyAsync(ck + (int64_t)nnz * w, Z, w * nnz, cudaMemcpyDeviceToDevice, st));
      }
      if ((s = run_mul(plan->fwd, prec, Z, Y, P, st))) return s;                 // P = P_S(Z Y)
      if ((s = run_add(p, aprec, -0.5, P, 0.0, nullptr, 1.5, T, st))) return s;   // T = (3I - P)/2
      if (aprec == S_FP64)
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
    if (refine == 0) {
      if (aprec == S_FP64) {
        if ((s = run_add(p, aprec, sc, Y, 0.0, nullptr, 0.0, F, st))) return s;
      } else {
        convert_kernel<float, double><<<g, 256, 0, st>>>(nnz, (const float*)Y, F, sc);
        SF_CUDA(cudaGetLastError());
      }
    } else {
      // residual correction in double (Newton's method for Y^2 = A/c with the inverse of Y
      // replaced by the coupled iterate Z):  R = A/c - P_S(Y Y),  Y <- Y + P_S(Z R)/2
      s_plan p64 = nullptr;
      if ((s = s_plan_create(p, p, p, S_FP64, &p64))) return s;
      PlanGuard pg64{p64};
      DevBuf dY, dZ, dR, dW;
      const size_t b8 = sizeof(double) * nnz + 16;
      SF_CUDA(cudaMalloc(&dY.p, b8));
      SF_CUDA(cudaMalloc(&dZ.p, b8));
      SF_CUDA(cudaMalloc(&dR.p, b8));
      SF_CUDA(cudaMalloc(&dW.p, b8));
      SyncOnExit sync64{st};
      double *Y8 = (double*)dY.p, *Z8 = (double*)dZ.p, *R8 = (double*)dR.p, *W8 = (double*)dW.p;
      if (aprec == S_FP64) {
        SF_CUDA(cudaMemcpyAsync(Y8, Y, b8 - 16, cudaMemcpyDeviceToDevice, st));
        SF_CUDA(cudaMemcpyAsync(Z8, Z, b8 - 16, cudaMemcpyDeviceToDevice, st));
      } else {
        convert_kernel<float, double><<<g, 256, 0, st>>>(nnz, (const float*)Y, Y8, 1.0);
        convert_kernel<float, double><<<g, 256, 0, st>>>(nnz, (const float*)Z, Z8, 1.0);
      }
      for (int r = 0; r < refine; ++r) {
        if ((s = run_mul(p64->fwd, S_FP64, Y8, Y8, W8, st))) return s;                 // W = P_S(Y Y)
        if ((s = run_add(p, S_FP64, 1.0 / c, A, -1.0, W8, 0.0, R8, st))) return s;     // R = A/c - W
        if ((s = run_mul(p64->fwd, S_FP64, Z8, R8, W8, st))) return s;                 // W = P_S(Z R)
        if ((s = run_add(p, S_FP64, 1.0, Y8, 0.5, W8, 0.0, Y8, st))) return s;         // Y += W/2
      }
      if ((s = run_add(p, S_FP64, sc, Y8, 0.0, nullptr, 0.0, F, st))) return s;
      SF_CUDA(cudaStreamSynchronize(st));
    }
    // divergence: ||T_k - I||_F grew by more than 1.5x on two consecutive steps while still above
    // 1e-3 of its starting value (below that the iteration has converged and the distance only
    // fluctuates at the level of the masking and rounding errors)
    {
      std::vector<double> dk(steps);
      SF_CUDA(cudaMemcpyAsync(dk.data(), bN.p, sizeof(double) * steps, cudaMemcpyDeviceToHost, st));
      SF_CUDA(cudaStreamSynchronize(st));
      for (int k = 0; k < steps; ++k) {
        const bool grew = k >= 2 && dk[k] > 2.25 * dk[k - 1] && dk[k - 1] > 2.25 * dk[k - 2] &&  // squared: 1.5^2
                          dk[k] > 1e-6 * dk[0];
        if (!std::isfinite(dk[k]) || grew)
          return set_error(S_ERR_NOT_CONVERGED, "s_funm: Newton-Schulz iteration diverged at step " + std::to_string(k));
      }
    }
    if ((s = s_plan_status(plan, st))) return s;
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
    if (aprec == S_FP64) {
      if ((s = run_add(p, aprec, xs, A, 0.0, nullptr, 0.0, X, st))) return s;
    } else {
      convert_kernel<double, float><<<g, 256, 0, st>>>(nnz, A, (float*)X, xs);
    }
    if ((s = run_add(p, aprec, 1.0 / m, X, 0.0, nullptr, 1.0, E, st))) return s;   // E = I + X/m
    for (int k = m - 1; k >= 1; --k) {
      if ((s = run_mul(plan->fwd, prec, X, E, W, st))) return s;                   // W = P_S(X E)
      if ((s = run_add(p, aprec, 1.0 / k, W, 0.0, nullptr, 1.0, E, st))) return s; // E = I + W/k
    }
    if (aprec == S_FP64) {
      for (int r = 0; r < sq; ++r) {
        if ((s = run_mul(plan->fwd, prec, E, E, W, st))) return s;                 // E = P_S(E E)
        std::swap(E, W);
      }
      SF_CUDA(cudaMemcpyAsync(F, E, w * nnz, cudaMemcpyDeviceToDevice, st));
    } else {
      // float Horner, double squarings: E (float) -> F, then F = P_S(F F) s times
      convert_kernel<float, double><<<g, 256, 0, st>>>(nnz, (const float*)E, F, 1.0);
      SF_CUDA(cudaGetLastError());
      if (sq > 0) {
        s_plan p64 = nullptr;
        if ((s = s_plan_create(p, p, p, S_FP64, &p64))) return s;
        PlanGuard pg64{p64};
        DevBuf dW;
        SF_CUDA(cudaMalloc(&dW.p, sizeof(double) * nnz + 16));
        SyncOnExit sync64{st};
        double* a = F;
        double* bq = (double*)dW.p;
        for (int r = 0; r < sq; ++r) {
          if ((s = run_mul(p64->fwd, S_FP64, a, a, bq, st))) return s;
          std::swap(a, bq);
        }
        if (a != F) SF_CUDA(cudaMemcpyAsync(F, a, sizeof(double) * nnz, cudaMemcpyDeviceToDevice, st));
        SF_CUDA(cudaStreamSynchronize(st));
      }
    }
    SF_CUDA(cudaStreamSynchronize(st));
    return S_OK;
  }
  return set_error(S_ERR_ARG, "s_funm: unknown function");
}

// Reverse mode of the coupled Newton-Schulz iteration of s_funm(S_SQRT) with c frozen, in
// double (prec S_FP64: double checkpoints, double adjoint products) or in float (prec S_FP32:
// float checkpoints, compensated-float adjoint products, float adjoint iterates; dF and dA
// stay double).
static s_status sqrt_backward(s_pattern p, s_prec prec, int steps, double c, const void* ck, const double* dF,
                              double* dA, cudaStream_t st) {
  const int64_t nnz = p->d.nnz;
  const size_t w = prec == S_FP32 ? sizeof(float) : sizeof(double);
  s_plan plan = nullptr;
  s_status s = s_plan_create(p, p, p, prec, &plan);
  if (s) return s;
  struct PlanGuard {
    s_plan q;
    ~PlanGuard() { s_plan_destroy(q); }
  } pg{plan};
  const size_t bytes = w * nnz + 16;
  DevBuf b[10];
  for (auto& x : b) SF_CUDA(cudaMalloc(&x.p, bytes));
  SyncOnExit sync{st};
  void *dY = b[0].p, *dZ = b[1].p, *P = b[2].p, *T = b[3].p, *dYa = b[4].p, *dT1 = b[5].p, *dT2 = b[6].p;
  void *dZa = b[7].p, *dZb = b[8].p, *dYb = b[9].p;
  const int64_t g = grid_of(nnz);
  // X = sqrt(c) Y_steps:  dY_steps = sqrt(c) dF,  dZ_steps = 0
  if (prec == S_FP32) {
    convert_kernel<double, float><<<g, 256, 0, st>>>(nnz, dF, (float*)dY, std::sqrt(c));
    SF_CUDA(cudaGetLastError());
  } else if ((s = run_add(p, S_FP64, std::sqrt(c), dF, 0.0, nullptr, 0.0, dY, st))) {
    return s;
  }
  SF_CUDA(cudaMemsetAsync(dZ, 0, w * nnz, st));
  for (int k = steps - 1; k >= 0; --k) {
    const void* Y = (const char*)ck + (int64_t)2 * k * nnz * (int64_t)w;
    const void* Z = (const char*)Y + (int64_t)nnz * w;
    if ((s = run_mul(plan->fwd, prec, Z, Y, P, st))) return s;                  // P = P_S(Z Y)
    if ((s = run_add(p, prec, -0.5, P, 0.0, nullptr, 1.5, T, st))) return s;    // T = (3I - P)/2
    // Y' = P_S(Y T): dY_a = P_S(dY' T^T), dT_1 = P_S(Y^T dY')
    if ((s = s_mul_masked_adjoint(plan, dY, Y, T, dYa, dT1, st))) return s;
    // Z' = P_S(T Z): dT_2 = P_S(dZ' Z^T), dZ_a = P_S(T^T dZ')
    if ((s = s_mul_masked_adjoint(plan, dZ, T, Z, dT2, dZa, st))) return s;
    // T = (3I - P)/2: dP = -(dT_1 + dT_2)/2, kept in dT1
    if ((s = run_add(p, prec, -0.5, dT1, -0.5, dT2, 0.0, dT1, st))) return s;
    // P = P_S(Z Y): dZ_b = P_S(dP Y^T), dY_b = P_S(Z^T dP)
    if ((s = s_mul_masked_adjoint(plan, dT1, Z, Y, dZb, dYb, st))) return s;
    if ((s = run_add(p, prec, 1.0, dYa, 1.0, dYb, 0.0, dY, st))) return s;
    if ((s = run_add(p, prec, 1.0, dZa, 1.0, dZb, 0.0, dZ, st))) return s;
  }
  // Y_0 = A / c
  if (prec == S_FP32) {
    convert_kernel<float, double><<<g, 256, 0, st>>>(nnz, (const float*)dY, dA, 1.0 / c);
    SF_CUDA(cudaGetLastError());
  } else if ((s = run_add(p, S_FP64, 1.0 / c, dY, 0.0, nullptr, 0.0, dA, st))) {
    return s;
  }
  SF_CUDA(cudaStreamSynchronize(st));
  return s_plan_status(plan, st);
}

extern "C" s_status s_funm_sqrt_backward(s_pattern p, int steps, double c, const double* ck, const double* dF,
                                         double* dA, void* stream) {
  if (!p || !ck || !dF || !dA || steps < 1 || !(c > 0.0)) return set_error(S_ERR_ARG, "s_funm_sqrt_backward: bad argument");
  if (!p->has_all_diag) return set_error(S_ERR_PATTERN, "s_funm_sqrt_backward: the pattern must hold every diagonal block");
  return sqrt_backward(p, S_FP64, steps, c, ck, dF, dA, (cudaStream_t)stream);
}

extern "C" s_status s_funm_sqrt_backward_prec(s_pattern p, s_prec prec, int steps, double c, const void* ck,
                                              const double* dF, double* dA, void* stream) {
  if (!p || !ck || !dF || !dA || steps < 1 || !(c > 0.0))
    return set_error(S_ERR_ARG, "s_funm_sqrt_backward_prec: bad argument");
  if (prec != S_FP64 && prec != S_FP32) return set_error(S_ERR_ARG, "s_funm_sqrt_backward_prec: prec must be S_FP64 or S_FP32");
  if (!p->has_all_diag)
    return set_error(S_ERR_PATTERN, "s_funm_sqrt_backward_prec: the pattern must hold every diagonal block");
  return sqrt_backward(p, prec, steps, c, ck, dF, dA, (cudaStream_t)stream);
}

extern "C" s_status s_quad_form(s_pattern p, const double* X, const double* z, double* out, void* stream) {
  if (!p || !X || !z || !out) return set_error(S_ERR_ARG, "s_quad_form: NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t nb = p->d.nblocks;
  DevBuf part, tot;
  SF_CUDA(cudaMalloc(&part.p, sizeof(double) * (nb + 1)));
  SF_CUDA(cudaMalloc(&tot.p, sizeof(double)));
  SyncOnExit sync{st};
  SF_CUDA(cudaMemsetAsync(tot.p, 0, sizeof(double), st));
  if (nb) {
    quad_part_kernel<<<(unsigned)((nb * 32 + 255) / 256), 256, 0, st>>>(nb, p->d.brow, p->d.colidx, p->d.bsize,
                                                                      p->d.boff, p->d.voff, X, z, (double*)part.p);
    // fixed-order sum of the block parts: dot with a vector of ones
    DevBuf ones;
    SF_CUDA(cudaMalloc(&ones.p, sizeof(double) * nb));
    fill_kernel<<<grid_of(nb), 256, 0, st>>>(nb, 1.0, (double*)ones.p);
    dot_kernel<<<1, 1024, 0, st>>>(nb, (const double*)part.p, (const double*)ones.p, (double*)tot.p);
    SF_CUDA(cudaGetLastError());
    SF_CUDA(cudaMemcpyAsync(out, tot.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    SF_CUDA(cudaStreamSynchronize(st));
  } else {
    *out = 0.0;
  }
  return S_OK;
}

extern "C" s_status s_quad_form_grad(s_pattern p, const double* z, double* dX, void* stream) {
  if (!p || !z || (!dX && p->d.nnz > 0)) return set_error(S_ERR_ARG, "s_quad_form_grad: NULL argument");
  const int64_t nb = p->d.nblocks;
  if (nb)
    quad_grad_kernel<<<(unsigned)((nb * 32 + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        nb, p->d.brow, p->d.colidx, p->d.bsize, p->d.boff, p->d.voff, z, dX);
  SF_CUDA(cudaGetLastError());
  return S_OK;
}
