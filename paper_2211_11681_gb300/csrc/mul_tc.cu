// Masked product C = P_{S_C}(op(X) op(Y)) (Eq. (product)) on the 5th-generation tensor
// cores, in split-TF32 arithmetic (S_TF32X3).
//
// Work unit: a panel = one row slice (up to 32 rows r0 ..) of block row nu of S_C together
// with up to 8 column slices ("members", up to 32 columns each, 128 columns in all) of the
// blocks (nu, nu'_j) of that row.  For every lambda of row nu of op(X) that meets at least one
// member, one stage computes
//     D[m][n] += sum_t Y_j(lambda)[c][t] * X(nu, lambda)[r0 + n][t],   m = moff_j + c,
// a short M=128 x N=16|32 x K=8.. tcgen05.mma chain into a tensor-memory accumulator of its
// own: the 128 member columns are the MMA rows and the panel's rows of nu the MMA columns, so
// the X(nu, lambda) slice is staged once for all members.  Members without block (lambda, nu'_j)
// get zero rows.  Each operand is split as x ~ hi + lo with hi = x rounded to TF32 (10
// fraction bits) and lo = x - hi rounded to TF32; both are stored as fp32 words whose low 13
// bits are zero, which is exactly what the tensor core reads of them.  The three products
// hi*hi + hi*lo + lo*hi are exact in the MMA; the dropped lo*lo and the rounding of lo are each
// below 2^-22 |x y|, with random signs.  The tensor core's fp32 accumulation drops low bits
// with a bias, so each stage starts a fresh accumulator (at most 9 MMAs deep) and the stage
// sums are added over lambda in registers by error-free two-sums (compensated summation);
// independent accumulators also let the MMAs of consecutive stages overlap.
//
// Staging: operands are K-major in the tensor core's no-swizzle canonical layout (8-row x
// 16-byte core matrices; K-adjacent core matrices 128 bytes apart, 8-row groups kTcSBO bytes
// apart), filled with 16-byte cp.async copies from blocks stored row-major along lambda's
// index t.  A pre-pass writes the split planes, per-block transposed where an operand's
// stored orientation runs the other way.  kTcS stage buffers rotate; copies run kTcD stages
// ahead of the MMAs, and an mbarrier per buffer (signalled by tcgen05.commit) tells when the
// tensor core has finished the stage: its shared-memory buffer is free and its accumulator
// (kTcN tensor-memory columns per buffer) can be read.  The stage entries of a panel come
// into shared memory kTcE at a time, so no stage waits on a global load of its own entry.
//
// The stage list of every panel (which lambda, which members, source offsets) is built once
// per plan on the device (symbolic phase).
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace sf {
namespace {

constexpr int kTcThreads = 256;
constexpr int kTcS = 6;                                    // stage buffers
constexpr int kTcD = 4;                                    // copy lookahead in stages (< kTcS)
constexpr int kTcE = 64;                                   // stage entries loaded at once
constexpr uint32_t kTcSBO = kTcKC * 32;                    // bytes between 8-row groups
constexpr uint32_t kTcAPlane = kTcM / 8 * kTcSBO;          // one plane of the member operand
constexpr uint32_t kTcBPlane = kTcN / 8 * kTcSBO;          // one plane of the X operand
constexpr uint32_t kTcBuf = 2 * kTcAPlane + 2 * kTcBPlane;  // hi, lo of both
constexpr size_t kTcSmem = (size_t)kTcS * kTcBuf;
constexpr int kTcCols = 256;                               // tensor-memory columns (>= kTcS * kTcN)
static_assert(kTcS * kTcN <= kTcCols, "tensor memory");
static_assert(kTcKC % 8 == 0 && kTcSmem <= 200 * 1024 && kTcD < kTcS, "stage buffers");
static_assert(sizeof(TcEntry) % 16 == 0, "entries move as 16-byte words");

int tc_num_sms() { return sm_count(); }

__device__ __forceinline__ uint32_t tc_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ int tc_lower_bound(const int32_t* a, int lo, int hi, int32_t v) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(a + mid) < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// ---- pre-pass: split planes, and per-block transposes ----------------------------------
// v rounded to the nearest value with 10 fraction bits (ties away from zero), by adding half
// of the dropped bits' unit to the magnitude field and clearing them
__device__ __forceinline__ float tf32_rn(float v) {
  return __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xFFFFE000u);
}

__global__ void tf32_split_kernel(int64_t n, const float* __restrict__ x, float* __restrict__ hi,
                                  float* __restrict__ lo) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = x[i], h = tf32_rn(v);
    hi[i] = h;
    lo[i] = tf32_rn(v - h);
  }
}

// block b (rows x cols, row-major) -> split parts of its transpose (cols x rows), written in
// the block's own value range
__global__ void tf32_transpose_kernel(int64_t nb, const int32_t* __restrict__ bsize, const int32_t* __restrict__ brow,
                                      const int32_t* __restrict__ colidx, const int64_t* __restrict__ voff,
                                      const float* __restrict__ x, float* __restrict__ hi, float* __restrict__ lo) {
  const int lane = threadIdx.x & 31;
  for (int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; b < nb;
       b += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int rows = bsize[brow[b]], cols = bsize[colidx[b]];
    const int64_t base = voff[b];
    for (int e = lane; e < rows * cols; e += 32) {
      const int r = e / cols, c = e - r * cols;
      const float v = x[base + e], h = tf32_rn(v);
      const int64_t o = base + (int64_t)c * rows + r;
      hi[o] = h;
      lo[o] = tf32_rn(v - h);
    }
  }
}

// ---- symbolic phase: stage list of every panel -----------------------------------------
struct TcSide {
  const int64_t* ptr;
  const int32_t* idx;
  const int32_t* blk;
  const int64_t* voff;
};

struct TcListArgs {
  TcSide x, y;
  const int32_t* bsize;
  const int32_t* c_brow;
  const int32_t* c_col;
  const Tile* tiles;
  const int2* pidx;
  int64_t npanels;
};

// One warp per panel.  FILL = false: count[t] = number of stages of panel t.  FILL = true:
// write them at out[pstart[t] ..].  A lambda meeting at least one member gives
// ceil(n_lambda / kTcKC) stages (slices of its index range).
template <bool FILL>
__global__ void tc_list_kernel(TcListArgs a, int64_t* __restrict__ count, const int64_t* __restrict__ pstart,
                               TcEntry* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; t < a.npanels; t += nw) {
    const int2 pi = a.pidx[t];
    const Tile* tl = a.tiles + pi.x;
    const int cnt = pi.y;
    const int nu = a.c_brow[tl[0].blk];
    const int r0 = tl[0].r0;
    int py0[kTcP], py1[kTcP], c0v[kTcP];
#pragma unroll
    for (int j = 0; j < kTcP; ++j) {
      py0[j] = py1[j] = c0v[j] = 0;
      if (j < cnt) {
        const int nup = a.c_col[tl[j].blk];
        py0[j] = (int)a.y.ptr[nup];
        py1[j] = (int)a.y.ptr[nup + 1];
        c0v[j] = tl[j].c0;
      }
    }
    int64_t pos = FILL ? pstart[t] : 0;
    const int px1 = (int)a.x.ptr[nu + 1];
    for (int px = (int)a.x.ptr[nu]; px < px1; px += 32) {
      const int i = px + lane;
      const int32_t lam = i < px1 ? __ldg(a.x.idx + i) : INT32_MAX;
      int by[kTcP];
      bool any = false;
#pragma unroll
      for (int j = 0; j < kTcP; ++j) {
        by[j] = -1;
        if (j < cnt) {
          const int p = tc_lower_bound(a.y.idx, py0[j], py1[j], lam);
          const bool hit = i < px1 && p < py1[j] && __ldg(a.y.idx + p) == lam;
          if (hit) by[j] = a.y.blk ? __ldg(a.y.blk + p) : p;
          any |= hit;
          py0[j] = __shfl_sync(0xffffffffu, p, 31);
        }
      }
      const int nl = any ? a.bsize[lam] : 0;
      const int nsl = (nl + kTcKC - 1) / kTcKC;
      int incl = nsl;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      const int total = __shfl_sync(0xffffffffu, incl, 31);
      if (FILL && any) {
        const int bx = a.x.blk ? __ldg(a.x.blk + i) : i;
        const int64_t xb = a.x.voff[bx] + (int64_t)r0 * nl;
        int64_t yb[kTcP];
#pragma unroll
        for (int j = 0; j < kTcP; ++j) yb[j] = by[j] >= 0 ? a.y.voff[by[j]] + (int64_t)c0v[j] * nl : -1;
        int64_t o = pos + incl - nsl;
        for (int s = 0; s < nsl; ++s, ++o) {
          const int t0 = s * kTcKC;
          TcEntry e;
          e.x = xb + t0;
#pragma unroll
          for (int j = 0; j < kTcP; ++j) e.y[j] = yb[j] >= 0 ? yb[j] + t0 : -1;
          e.nl = nl;
          e.wd = min(kTcKC, nl - t0);
          out[o] = e;
        }
      }
      pos += total;
    }
    if (!FILL && lane == 0) count[t] = pos;
  }
}

// ---- the product kernel ------------------------------------------------------------------
struct TcArgs {
  const int32_t* bsize;
  const int32_t* c_brow;
  const int32_t* c_col;
  const int64_t* c_voff;
  const Tile* tiles;
  const int2* pidx;
  int64_t npanels;
  const int64_t* pstart;
  const TcEntry* ent;
  const float* xh;
  const float* xl;
  const float* yh;
  const float* yl;
  float* C;
  unsigned int* counter;
  unsigned int* err;
};

__device__ __forceinline__ uint64_t tc_desc(uint32_t addr) {
  // no-swizzle K-major: start >> 4 | LBO (K-adjacent core matrices) >> 4 << 16 |
  // SBO (8-row groups) >> 4 << 32 | descriptor version 1 << 46
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(kTcSBO >> 4) << 32) |
         ((uint64_t)1 << 46);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_cp16(void* dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(tc_smem(dst)), "l"(src));
}
__device__ __forceinline__ void tc_cp4(void* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(tc_smem(dst)), "l"(src));
}

// Wait for phase `parity` of an mbarrier, for at most about one second of SM clocks; on
// time-out record it (CTA flag and global error word) and stop waiting from then on.
__device__ __forceinline__ void tc_wait(uint64_t* bar, uint32_t parity, volatile int* abort, unsigned int* err) {
  if (*abort) return;
  const uint32_t addr = tc_smem(bar);
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return;
    if (clock64() - t0 > (1ll << 31)) {
      *abort = 1;
      *(volatile unsigned int*)err = 1u;  // host-mapped word: a plain store, then a system fence
      __threadfence_system();
      return;
    }
    if (*abort) return;
  }
}

__global__ void __launch_bounds__(kTcThreads, 1) mul_tf32x3_kernel(TcArgs a) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  __shared__ __align__(8) uint64_t mbar[kTcS];
  __shared__ uint32_t tmem_base;
  __shared__ int32_t rowtab[kTcM];  // member << 8 | column of each MMA row
  __shared__ int64_t mC[kTcP];      // C offset of each member's tile origin
  __shared__ int32_t mnj[kTcP];     // row pitch of each member's C block
  __shared__ int32_t swd[kTcS];     // lambda extent staged in each buffer
  __shared__ __align__(16) TcEntry sent[2][kTcE];  // stage entries, two chunks
  __shared__ int s_panel_ok, s_th, s_mused;
  __shared__ int64_t s_e0, s_ne;
  __shared__ volatile int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // every buffer starts at zero: K-padding columns of the member planes are never written
  // again and must hold finite values (their X-side partners are zero)
  for (int i = tid; i < (int)(kTcSmem / 16); i += kTcThreads)
    reinterpret_cast<float4*>(tsm)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  if (tid == 0) {
    for (int b = 0; b < kTcS; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(tc_smem(&mbar[b])));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    s_abort = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(tc_smem(&tmem_base)),
                 "n"(kTcCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t sbase = tc_smem(tsm);
  int64_t g = 0;   // stages this CTA has issued
  int64_t gd = 0;  // stages whose accumulators have been added
  const int q = warp & 3, h = warp >> 2;  // this warp's TMEM lanes 32q .. and columns 16h ..
  float acc[16], cmp[16];  // stage sums, compensated: acc + cmp (error-free two-sums)

  for (;;) {
    if (tid == 0) {
      const unsigned int t = atomicAdd(a.counter, 1u);
      s_panel_ok = t < a.npanels;
      if (t < a.npanels) {
        const int2 pi = a.pidx[t];
        const Tile* tl = a.tiles + pi.x;
        const int nu = a.c_brow[tl[0].blk];
        const int r0 = tl[0].r0;
        s_th = min(kTcN, a.bsize[nu] - r0);
        int m = 0;
        for (int j = 0; j < pi.y; ++j) {
          const Tile tj = tl[j];
          const int nj = a.bsize[a.c_col[tj.blk]];
          const int w = min(kTcN, nj - tj.c0);
          mC[j] = a.c_voff[tj.blk] + (int64_t)r0 * nj + tj.c0;
          mnj[j] = nj;
          for (int c = 0; c < w; ++c) rowtab[m + c] = (j << 8) | c;
          m += w;
        }
        s_mused = m;
        s_e0 = a.pstart[t];
        s_ne = a.pstart[t + 1] - a.pstart[t];
      }
    }
    __syncthreads();
    if (!s_panel_ok) break;
    const int th = s_th, mused = s_mused;
    const int64_t e0 = s_e0, ne = s_ne;
#pragma unroll
    for (int u = 0; u < 16; ++u) acc[u] = cmp[u] = 0.0f;
    // stage k has finished: add its accumulator (rows 32q + lane, columns 16h ..) to acc, the
    // rounding error of every addition kept in cmp
    auto drain = [&](int64_t k) {
      const int b = (int)(k % kTcS);
      tc_wait(&mbar[b], (uint32_t)((k / kTcS) & 1), &s_abort, a.err);
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      if (16 * h < th) {
        uint32_t v[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
            "[%16];\n"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * kTcN + 16 * h)));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const float x = __uint_as_float(v[u]);
          const float sm = acc[u] + x;
          const float bp = sm - acc[u];
          cmp[u] += (acc[u] - (sm - bp)) + (x - bp);
          acc[u] = sm;
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    };
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)((th <= 16 ? 16 : 32) >> 3) << 17) |
                           ((uint32_t)(kTcM >> 4) << 24);

    for (int64_t m = 0; m < ne + kTcD - 1; ++m) {
      if (m < ne) {
        // ---- stage m: copies into buffer (g + m) % kTcS -------------------------------
        const int64_t gm = g + m;
        const int b = (int)(gm % kTcS);
        while (gd <= gm - kTcS) drain(gd++);  // frees buffer b and its accumulator
        if (m % kTcE == 0) {
          // entries m .. m + kTcE - 1 of this panel -> chunk (m / kTcE) & 1, which the
          // threads last read at stages m - 2 kTcE .. m - kTcE - 1 (or in an earlier panel)
          const int cnt = (int)min((int64_t)kTcE, ne - m);
          const uint4* src = reinterpret_cast<const uint4*>(a.ent + e0 + m);
          uint4* dst = reinterpret_cast<uint4*>(sent[(m / kTcE) & 1]);
          constexpr int kW = (int)(sizeof(TcEntry) / 16);
          for (int i = tid; i < cnt * kW; i += kTcThreads) dst[i] = __ldg(src + i);
          __syncthreads();
        }
        const TcEntry* en = &sent[(m / kTcE) & 1][m % kTcE];
        const int nl = en->nl, wd = en->wd;
        const int64_t xo = en->x;
        if (tid == 0) swd[b] = wd;
        unsigned char* buf = tsm + (size_t)b * kTcBuf;
        const int nkc = (wd + 3) >> 2;         // 16-byte chunks holding data
        const int nkp = ((wd + 7) >> 3) << 1;  // chunks the MMAs read
        const bool nl4 = (nl & 3) == 0;
        // member columns -> rows of the A planes
        const float rk = 1.0f / (float)nkc;
        for (int e = tid; e < mused * nkc; e += kTcThreads) {
          const int r = __float2int_rz(((float)e + 0.5f) * rk), kc = e - r * nkc;
          const int rt = rowtab[r];
          const int64_t ys = en->y[rt >> 8];
          const uint32_t off = (uint32_t)(r >> 3) * kTcSBO + kc * 128 + (r & 7) * 16;
          float* dh = reinterpret_cast<float*>(buf + off);
          float* dl = reinterpret_cast<float*>(buf + kTcAPlane + off);
          if (ys < 0) {
            *reinterpret_cast<float4*>(dh) = make_float4(0.f, 0.f, 0.f, 0.f);
            *reinterpret_cast<float4*>(dl) = make_float4(0.f, 0.f, 0.f, 0.f);
            continue;
          }
          const int64_t src = ys + (int64_t)(rt & 255) * nl + 4 * kc;
          if (nl4 && (ys & 3) == 0 && 4 * kc + 4 <= wd) {
            tc_cp16(dh, a.yh + src);
            tc_cp16(dl, a.yl + src);
          } else {
            for (int u = 0; u < 4; ++u)
              if (4 * kc + u < wd) {
                tc_cp4(dh + u, a.yh + src + u);
                tc_cp4(dl + u, a.yl + src + u);
              }
          }
        }
        // rows r0 .. r0 + th of X(nu, lambda) -> rows of the B planes, zero K padding
        const float rp = 1.0f / (float)nkp;
        for (int e = tid; e < th * nkp; e += kTcThreads) {
          const int r = __float2int_rz(((float)e + 0.5f) * rp), kc = e - r * nkp;
          const uint32_t off = 2 * kTcAPlane + (uint32_t)(r >> 3) * kTcSBO + kc * 128 + (r & 7) * 16;
          float* dh = reinterpret_cast<float*>(buf + off);
          float* dl = reinterpret_cast<float*>(buf + kTcBPlane + off);
          if (4 * kc >= wd) {
            *reinterpret_cast<float4*>(dh) = make_float4(0.f, 0.f, 0.f, 0.f);
            *reinterpret_cast<float4*>(dl) = make_float4(0.f, 0.f, 0.f, 0.f);
            continue;
          }
          const int64_t src = xo + (int64_t)r * nl + 4 * kc;
          if (nl4 && (xo & 3) == 0 && 4 * kc + 4 <= wd) {
            tc_cp16(dh, a.xh + src);
            tc_cp16(dl, a.xl + src);
          } else {
            for (int u = 0; u < 4; ++u) {
              if (4 * kc + u < wd) {
                tc_cp4(dh + u, a.xh + src + u);
                tc_cp4(dl + u, a.xl + src + u);
              } else {
                dh[u] = 0.0f;
                dl[u] = 0.0f;
              }
            }
          }
        }
      }
      asm volatile("cp.async.commit_group;\n" ::);
      if (m >= kTcD - 1) {
        // ---- stage m - kTcD + 1: its copies are complete; one thread issues the MMAs -----
        const int64_t e = m - (kTcD - 1);
        asm volatile("cp.async.wait_group %0;\n" ::"n"(kTcD - 1));
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0) {
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
          const int b = (int)((g + e) % kTcS);
          const int kst = (swd[b] + 7) >> 3;
          const uint32_t ah = sbase + (uint32_t)b * kTcBuf, al = ah + kTcAPlane;
          const uint32_t bh = ah + 2 * kTcAPlane, bl = bh + kTcBPlane;
          const uint32_t td = tmem + (uint32_t)(b * kTcN);  // this stage's accumulator
          for (int s = 0; s < kst; ++s) {
            const uint32_t o = (uint32_t)s * 256;  // K = 8 tf32 = two 16-byte core matrices
            tc_mma(td, tc_desc(al + o), tc_desc(bh + o), idesc, s > 0 ? 1u : 0u);
            tc_mma(td, tc_desc(ah + o), tc_desc(bl + o), idesc, 1u);
            tc_mma(td, tc_desc(ah + o), tc_desc(bh + o), idesc, 1u);
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              tc_smem(&mbar[b])));
        }
      }
    }
    g += ne;
    // ---- epilogue: remaining stage sums, then acc -> C -----------------------------------
    while (gd < g) drain(gd++);
    if (16 * h < th) {
      const int mrow = 32 * q + lane;
      if (mrow < mused) {
        const int rt = rowtab[mrow];
        const int j = rt >> 8;
        float* cp = a.C + mC[j] + (rt & 255);
        const int64_t nj = mnj[j];
        const bool bad = s_abort != 0;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int n = 16 * h + u;
          if (n < th) cp[n * nj] = bad ? __int_as_float(0x7fc00000) : acc[u] + cmp[u];
        }
      }
    }
    __syncthreads();
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(kTcCols));
}

static s_status tc_split(const s_pattern_t* p, bool transpose, const float* x, float* hi, float* lo, cudaStream_t st) {
  const int64_t n = p->d.nnz, nb = p->d.nblocks;
  if (n == 0) return S_OK;
  if (transpose) {
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((nb * 32 + 255) / 256, (int64_t)tc_num_sms() * 16));
    tf32_transpose_kernel<<<grid, 256, 0, st>>>(nb, p->d.bsize, p->d.brow, p->d.colidx, p->d.voff, x, hi, lo);
  } else {
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)tc_num_sms() * 16));
    tf32_split_kernel<<<grid, 256, 0, st>>>(n, x, hi, lo);
  }
  SF_CUDA(cudaGetLastError());
  return S_OK;
}

}  // namespace

void tc_free(MulDesc* d) {
  cudaFree(d->ptiles);
  cudaFree(d->pidx);
  cudaFree(d->tc_pstart);
  cudaFree(d->tc_ent);
  cudaFree(d->tc_xl);
  cudaFree(d->tc_xh);
  cudaFree(d->tc_yl);
  cudaFree(d->tc_yh);
  d->ptiles = nullptr;
  d->pidx = nullptr;
  d->tc_pstart = nullptr;
  d->tc_ent = nullptr;
  d->tc_xl = d->tc_xh = d->tc_yl = d->tc_yh = nullptr;
  d->npanels = 0;
  d->tc_nentries = 0;
}

// Panels of S_C and their stage lists; scratch planes for the split operands.
s_status tc_prepare(MulDesc* d) {
  const s_pattern_t* C = d->pc;
  tc_free(d);
  if (d->pc->d.max_bsize > kTcMaxB || d->px->d.max_bsize > kTcMaxB || d->py->d.max_bsize > kTcMaxB)
    return set_error(S_ERR_ARG, "S_TF32X3: blocks wider than 96 are not supported");
  std::vector<Tile> tl;
  std::vector<int2> idx;
  for (int32_t nu = 0; nu < C->d.nc; ++nu) {
    const int ni = C->bsize[nu];
    for (int r0 = 0; r0 < ni; r0 += kTcN) {
      int rows = 0, cnt = 0;
      bool open = false;
      for (int64_t k = C->rowptr[nu]; k < C->rowptr[nu + 1]; ++k) {
        const int nj = C->bsize[C->colidx[k]];
        for (int c0 = 0; c0 < nj; c0 += kTcN) {
          const int w = std::min(kTcN, nj - c0);
          if (!open || cnt == kTcP || rows + w > kTcM) {
            idx.push_back(make_int2((int)tl.size(), 0));
            rows = cnt = 0;
            open = true;
          }
          tl.push_back(Tile{(int32_t)k, (int16_t)r0, (int16_t)c0});
          idx.back().y++;
          rows += w;
          ++cnt;
        }
      }
    }
  }
  const int64_t np = (int64_t)idx.size();
  int64_t* cnt_d = nullptr;
  cudaError_t e = cudaMalloc(&d->ptiles, sizeof(Tile) * std::max<size_t>(tl.size(), 1));
  if (e == cudaSuccess) e = cudaMalloc(&d->pidx, sizeof(int2) * std::max<int64_t>(np, 1));
  if (e == cudaSuccess) e = cudaMalloc(&d->tc_pstart, sizeof(int64_t) * (np + 1));
  if (e == cudaSuccess) e = cudaMalloc(&cnt_d, sizeof(int64_t) * std::max<int64_t>(np, 1));
  if (e == cudaSuccess && !tl.empty())
    e = cudaMemcpy(d->ptiles, tl.data(), sizeof(Tile) * tl.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && np) e = cudaMemcpy(d->pidx, idx.data(), sizeof(int2) * np, cudaMemcpyHostToDevice);
  d->npanels = np;
  d->panel_edge = kTcN;
  d->panel_size = kTcP;
  TcListArgs la;
  la.x = TcSide{d->x.ptr, d->x.idx, d->x.blk, d->x.voff};
  la.y = TcSide{d->y.ptr, d->y.idx, d->y.blk, d->y.voff};
  la.bsize = C->d.bsize;
  la.c_brow = C->d.brow;
  la.c_col = C->d.colidx;
  la.tiles = d->ptiles;
  la.pidx = d->pidx;
  la.npanels = np;
  std::vector<int64_t> ps(np + 1, 0);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((np * 32 + 255) / 256, (int64_t)tc_num_sms() * 32));
  if (e == cudaSuccess && np) {
    tc_list_kernel<false><<<grid, 256>>>(la, cnt_d, nullptr, nullptr);
    e = cudaGetLastError();
    std::vector<int64_t> cn(np, 0);
    if (e == cudaSuccess) e = cudaMemcpy(cn.data(), cnt_d, sizeof(int64_t) * np, cudaMemcpyDeviceToHost);
    for (int64_t t = 0; t < np; ++t) ps[t + 1] = ps[t] + cn[t];
  }
  if (e == cudaSuccess) e = cudaMemcpy(d->tc_pstart, ps.data(), sizeof(int64_t) * (np + 1), cudaMemcpyHostToDevice);
  d->tc_nentries = ps[np];
  if (e == cudaSuccess) e = cudaMalloc(&d->tc_ent, sizeof(TcEntry) * std::max<int64_t>(d->tc_nentries, 1));
  if (e == cudaSuccess && np) {
    tc_list_kernel<true><<<grid, 256>>>(la, nullptr, d->tc_pstart, d->tc_ent);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  cudaFree(cnt_d);
  // split planes (hi, lo) of both operands, in the orientation the kernel stages; a symmetric
  // plan (B = A) reads both operands from A's planes
  const int64_t nx = std::max<int64_t>(d->px->d.nnz, 1), ny = std::max<int64_t>(d->py->d.nnz, 1);
  const bool own_y = !(d->tc_sym && d->px == d->py);
  if (e == cudaSuccess) e = cudaMalloc(&d->tc_xh, sizeof(float) * nx);
  if (e == cudaSuccess) e = cudaMalloc(&d->tc_xl, sizeof(float) * nx);
  if (e == cudaSuccess && own_y) e = cudaMalloc(&d->tc_yh, sizeof(float) * ny);
  if (e == cudaSuccess && own_y) e = cudaMalloc(&d->tc_yl, sizeof(float) * ny);
  if (e != cudaSuccess) return cuda_error(e, "S_TF32X3 plan");
  return S_OK;
}

s_status launch_tc(const MulDesc& d, const void* X, const void* Y, void* C, cudaStream_t st) {
  if (!d.tc_pstart || !d.tc_xh || !d.tc_xl) return set_error(S_ERR_ARG, "internal: S_TF32X3 plan not prepared");
  s_status s0 = take_timeout(d);
  if (s0) return s0;
  if (d.tc_sym && X != Y)
    return set_error(S_ERR_ARG, "s_mul_masked: a symmetric S_TF32X3 plan must be called with B = A");
  s_status s;
  // X planes: rows of op(X)(nu, lambda) along lambda's index, i.e. the stored blocks unless
  // op(X) is a transpose
  if ((s = tc_split(d.px, d.x.trans, (const float*)X, d.tc_xh, d.tc_xl, st))) return s;
  // Y planes: columns of op(Y)(lambda, nu') along lambda's index, i.e. the stored blocks when
  // op(Y) is a transpose; the same planes as X's when both are one buffer in one orientation
  const float* yh = d.tc_xh;
  const float* yl = d.tc_xl;
  if (!(X == Y && d.px == d.py && d.x.trans == !d.y.trans)) {
    if (!d.tc_yh || !d.tc_yl) return set_error(S_ERR_ARG, "internal: S_TF32X3 plan has no planes for B");
    if ((s = tc_split(d.py, !d.y.trans, (const float*)Y, d.tc_yh, d.tc_yl, st))) return s;
    yh = d.tc_yh;
    yl = d.tc_yl;
  }
  if (d.npanels == 0) return S_OK;
  SF_CUDA(cudaMemsetAsync(d.counter, 0, sizeof(unsigned int), st));
  TcArgs a;
  a.bsize = d.pc->d.bsize;
  a.c_brow = d.pc->d.brow;
  a.c_col = d.pc->d.colidx;
  a.c_voff = d.pc->d.voff;
  a.tiles = d.ptiles;
  a.pidx = d.pidx;
  a.npanels = d.npanels;
  a.pstart = d.tc_pstart;
  a.ent = d.tc_ent;
  a.xh = d.tc_xh;
  a.xl = d.tc_xl;
  a.yh = yh;
  a.yl = yl;
  a.C = (float*)C;
  a.counter = d.counter;
  a.err = d.err;
  SF_CUDA(cudaFuncSetAttribute(mul_tf32x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem));
  const int grid = (int)std::min<int64_t>(d.npanels, (int64_t)tc_num_sms());
  mul_tf32x3_kernel<<<grid, kTcThreads, kTcSmem, st>>>(a);
  SF_CUDA(cudaGetLastError());
  return S_OK;
}

}  // namespace sf
