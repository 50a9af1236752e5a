// Masked block-sparse product C = P_{S_C}(op(X) op(Y)), Eq. (product) of Thm. (product),
// Sec. 4.1, and its symbolic phase.
//
// Work decomposition: every block (nu, nu') of S_C is cut into output tiles of at most
// kTile x kTile entries; one warp owns one tile for the whole lambda-sum, so each output
// entry is accumulated by one thread in increasing lambda order (deterministic, no
// atomics).  The lambda set of a tile is the intersection of the sorted block-index lists
// row(op(X), nu) and col(op(Y), nu'); a warp intersects them 32 entries of the X list at a
// time by binary search in the Y list.  Warps take tiles from a device counter
// (persistent grid sized to the SM count); tiles follow the block order of S_C.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <new>

#include "common.cuh"

namespace sf {

struct DevSide {
  const int64_t* ptr;
  const int32_t* idx;
  const int32_t* blk;
  const int64_t* voff;
};

struct MulArgs {
  DevSide x, y;
  const int32_t* bsize;
  const int32_t* c_brow;
  const int32_t* c_col;
  const int64_t* c_voff;
  const Tile* tiles;
  int64_t ntiles;
  unsigned int* counter;
};

static DevSide dev_side(const Side& s) { return DevSide{s.ptr, s.idx, s.blk, s.voff}; }

__device__ __forceinline__ int lower_bound_dev(const int32_t* a, int lo, int hi, int32_t v) {
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (__ldg(a + mid) < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// ---- symbolic: per C block, matched lambda count and useful flops ----------------------
__global__ void count_kernel(DevSide x, DevSide y, const int32_t* bsize, const int32_t* c_brow, const int32_t* c_col,
                             int64_t nblocks, unsigned long long* triples, double* block_flops) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t k = warp; k < nblocks; k += nwarps) {
    const int nu = c_brow[k], nup = c_col[k];
    const int px0 = (int)x.ptr[nu], px1 = (int)x.ptr[nu + 1];
    int py0 = (int)y.ptr[nup];
    const int py1 = (int)y.ptr[nup + 1];
    double fl = 0.0;
    unsigned int cnt = 0;
    for (int base = px0; base < px1 && py0 < py1; base += 32) {
      const int i = base + lane;
      const int32_t lam = i < px1 ? __ldg(x.idx + i) : INT32_MAX;
      const int pos = lower_bound_dev(y.idx, py0, py1, lam);
      const bool hit = i < px1 && pos < py1 && __ldg(y.idx + pos) == lam;
      if (hit) {
        cnt++;
        fl += 2.0 * bsize[lam];
      }
      const int last = __shfl_sync(0xffffffffu, pos, 31);
      py0 = last;
    }
    for (int o = 16; o; o >>= 1) {
      cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
      fl += __shfl_xor_sync(0xffffffffu, fl, o);
    }
    if (lane == 0) {
      block_flops[k] = fl * bsize[nu] * bsize[nup];
      atomicAdd(triples, (unsigned long long)cnt);
    }
  }
}

// tiles per block
__global__ void tile_count_kernel(const int32_t* bsize, const int32_t* c_brow, const int32_t* c_col, int64_t nblocks,
                                  int edge, int32_t* ntile) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= nblocks) return;
  int ni = bsize[c_brow[k]], nj = bsize[c_col[k]];
  ntile[k] = ((ni + edge - 1) / edge) * ((nj + edge - 1) / edge);
}

__global__ void tile_fill_kernel(const int64_t* first, const int32_t* bsize, const int32_t* c_brow,
                                 const int32_t* c_col, int64_t nblocks, int edge, Tile* tiles) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= nblocks) return;
  int ni = bsize[c_brow[k]], nj = bsize[c_col[k]];
  int64_t t = first[k];
  for (int r0 = 0; r0 < ni; r0 += edge)
    for (int c0 = 0; c0 < nj; c0 += edge) tiles[t++] = Tile{(int32_t)k, (int16_t)r0, (int16_t)c0};
}

// ---- numeric kernels ----------------------------------------------------------------------
constexpr int kWarps = 8;
template <typename T>
constexpr bool kCompensated = sizeof(T) == 4;
// Double product: tile edge TT (20, or 10 for patterns of blocks at most about 10 wide),
// every lane holding (TT^2 + 31) / 32 entries of the tile.
template <typename T, int TT, bool TX, bool TY>
__global__ void __launch_bounds__(kWarps * 32) mul_kernel(MulArgs a, const T* __restrict__ X,
                                                          const T* __restrict__ Y, T* __restrict__ C) {
  constexpr int kTile = TT;
  constexpr int kPer = (TT * TT + 31) / 32;  // accumulators per lane
  __shared__ T sX[kWarps][kTile * kTile];
  __shared__ T sY[kWarps][kTile * kTile];
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  T* xs = sX[w];
  T* ys = sY[w];
  for (;;) {
    unsigned int t = 0;
    if (lane == 0) t = atomicAdd(a.counter, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= a.ntiles) break;
    const Tile tile = a.tiles[t];
    const int k = tile.blk;
    const int nu = a.c_brow[k], nup = a.c_col[k];
    const int ni = a.bsize[nu], nj = a.bsize[nup];
    const int th = min(kTile, ni - tile.r0), tw = min(kTile, nj - tile.c0);
    const int nout = th * tw;
    T acc[kPer], comp[kPer];
#pragma unroll
    for (int m = 0; m < kPer; ++m) acc[m] = comp[m] = T(0);
    const int px0 = (int)a.x.ptr[nu], px1 = (int)a.x.ptr[nu + 1];
    int py0 = (int)a.y.ptr[nup];
    const int py1 = (int)a.y.ptr[nup + 1];
    for (int base = px0; base < px1 && py0 < py1; base += 32) {
      const int i = base + lane;
      const int32_t lam = i < px1 ? __ldg(a.x.idx + i) : INT32_MAX;
      const int pos = lower_bound_dev(a.y.idx, py0, py1, lam);
      const bool hit = i < px1 && pos < py1 && __ldg(a.y.idx + pos) == lam;
      unsigned int mask = __ballot_sync(0xffffffffu, hit);
      const int kx = hit ? (a.x.blk ? __ldg(a.x.blk + i) : i) : 0;
      const int ky = hit ? (a.y.blk ? __ldg(a.y.blk + pos) : pos) : 0;
      py0 = __shfl_sync(0xffffffffu, pos, 31);
      while (mask) {
        const int l = __ffs(mask) - 1;
        mask &= mask - 1;
        const int lm = __shfl_sync(0xffffffffu, lam, l);
        const int bx = __shfl_sync(0xffffffffu, kx, l);
        const int by = __shfl_sync(0xffffffffu, ky, l);
        const int nl = a.bsize[lm];
        const T* xb = X + a.x.voff[bx];
        const T* yb = Y + a.y.voff[by];
        for (int t0 = 0; t0 < nl; t0 += kTile) {
          const int tk = min(kTile, nl - t0);
          // op(X)(r0+r, t0+t) -> xs[r*tk+t];  op(Y)(t0+t, c0+c) -> ys[t*tw+c]
          for (int e = lane; e < th * tk; e += 32) {
            const int r = e / tk, tt = e - r * tk;
            const int gr = tile.r0 + r, gt = t0 + tt;
            xs[e] = TX ? xb[(int64_t)gt * ni + gr] : xb[(int64_t)gr * nl + gt];
          }
          for (int e = lane; e < tk * tw; e += 32) {
            const int tt = e / tw, c = e - tt * tw;
            const int gt = t0 + tt, gc = tile.c0 + c;
            ys[e] = TY ? yb[(int64_t)gc * nl + gt] : yb[(int64_t)gt * nj + gc];
          }
          __syncwarp();
#pragma unroll
          for (int m = 0; m < kPer; ++m) {
            const int e = lane + 32 * m;
            if (e < nout) {
              const int r = e / tw, c = e - r * tw;
              const T* xr = xs + r * tk;
              const T* yc = ys + c;
              if (kCompensated<T>) {
                // float: partial over this lambda block, then an error-free two-sum into
                // (acc, comp); the long lambda-sums would otherwise lose ~1e-6 (Sec. 4.1
                // sums over all lambda levels)
                T s = T(0);
                for (int tt = 0; tt < tk; ++tt) s = fma(xr[tt], yc[tt * tw], s);
                const T hi = acc[m] + s;
                const T bp = hi - acc[m];
                comp[m] += (acc[m] - (hi - bp)) + (s - bp);
                acc[m] = hi;
              } else {
                T s = acc[m];
                for (int tt = 0; tt < tk; ++tt) s = fma(xr[tt], yc[tt * tw], s);
                acc[m] = s;
              }
            }
          }
          __syncwarp();
        }
      }
    }
    T* cb = C + a.c_voff[k];
#pragma unroll
    for (int m = 0; m < kPer; ++m) {
      const int e = lane + 32 * m;
      if (e < nout) {
        const int r = e / tw, c = e - r * tw;
        cb[(int64_t)(tile.r0 + r) * nj + tile.c0 + c] = kCompensated<T> ? acc[m] + comp[m] : acc[m];
      }
    }
  }
}

// Float product: one warp per output tile as above, with register micro-tiles and
// double-buffered asynchronous staging.  Template parameters: tile edge TT and the
// micro-tile MR x MC of a lane; lane (mr, mc) of the first (TT/MR)(TT/MC) lanes owns rows
// MR*mr .. MR*mr+MR-1 and columns MC*mc .. MC*mc+MC-1 of the tile.  The warp first lists
// the matching lambda blocks of a batch, then streams them slice by slice (a slice = TT
// values of lambda): while one slice is multiplied out of shared memory, the copies of the
// next are in flight (cp.async; 4-byte copies scatter op(X) transposed into sA[t][r],
// op(Y) lands in sB[t][c], 16-byte copies where rows are contiguous and aligned).  Each t
// step loads MR values of sA and MC values of sB and does MR*MC FMAs.  Products are summed
// in a float partial that is folded into the accumulator with an error-free two-sum every
// kFold lambda blocks (compensated summation over lambda).
constexpr int kF32Warps = 4;
constexpr int kStages = 64;      // matching lambda blocks listed per batch
constexpr int kFold = 4;         // lambda blocks per two-sum

struct Stage {
  int32_t bx, by;   // X and Y block ids
  int16_t nl, t0;   // lambda block size, first t of this slice
};

__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src));
}
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// M consecutive floats from shared memory (aligned to M floats when M is 2 or 4)
template <int M>
__device__ __forceinline__ void lds(const float* p, float* out) {
  if constexpr (M == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    out[0] = v.x, out[1] = v.y, out[2] = v.z, out[3] = v.w;
  } else if constexpr (M == 2) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    out[0] = v.x, out[1] = v.y;
  } else {
#pragma unroll
    for (int q = 0; q < M; ++q) out[q] = p[q];
  }
}

// Copies lambda slice [t0, t0 + wd) of op(X) rows r0.. (th of them) and op(Y) columns
// c0.. (tw of them) into rows k0 .. k0 + wd - 1 of the stage buffers: xs[k][r], ys[k][c].
template <int TT, bool TX, bool TY>
__device__ __forceinline__ void stage_copy(const Stage& sg, int t0, int wd, int k0, const float* __restrict__ X,
                                           const float* __restrict__ Y, const int64_t* xvoff, const int64_t* yvoff,
                                           int ni, int nj, int r0, int c0, int th, int tw, int lane, float* xs,
                                           float* ys) {
  const int nl = sg.nl;
  const float* xb = X + xvoff[sg.bx];
  const float* yb = Y + yvoff[sg.by];
  xs += k0 * TT;
  ys += k0 * TT;
  const bool xvec = TT % 4 == 0 && TX && r0 == 0 && th == ni && (ni & 3) == 0 &&
                    ((reinterpret_cast<uintptr_t>(xb) & 15) == 0);
  if (xvec) {
    // op(X) = X^T: row t of the stored block (lambda, nu) is column t of op(X), i.e. one
    // contiguous run of xs[t][.]
    const float rni = 1.0f / (float)ni;
    for (int q = lane; q < (wd * ni) >> 2; q += 32) {
      const int e = q << 2;
      const int tt = __float2int_rz(((float)e + 0.5f) * rni), r = e - tt * ni;
      cp_async16(xs + tt * TT + r, xb + (int64_t)(t0 + tt) * ni + r);
    }
  } else {
    const float rwd = 1.0f / (float)wd;
    for (int e = lane; e < th * wd; e += 32) {
      const int r = __float2int_rz(((float)e + 0.5f) * rwd), tt = e - r * wd;
      const int gr = r0 + r, gt = t0 + tt;
      cp_async4(xs + tt * TT + r, TX ? xb + (int64_t)gt * ni + gr : xb + (int64_t)gr * nl + gt);
    }
  }
  // 16-byte copies need 16-byte aligned shared rows: TT a multiple of 4
  const bool vec = TT % 4 == 0 && !TY && c0 == 0 && tw == nj && (nj & 3) == 0 &&
                   ((reinterpret_cast<uintptr_t>(yb) & 15) == 0);
  if (vec) {
    const float rnj = 1.0f / (float)nj;
    for (int q = lane; q < (wd * nj) >> 2; q += 32) {
      const int e = q << 2;
      const int tt = __float2int_rz(((float)e + 0.5f) * rnj), c = e - tt * nj;
      cp_async16(ys + tt * TT + c, yb + (int64_t)(t0 + tt) * nj + c);
    }
  } else {
    const float rtw = 1.0f / (float)tw;
    for (int e = lane; e < wd * tw; e += 32) {
      const int tt = __float2int_rz(((float)e + 0.5f) * rtw), c = e - tt * tw;
      const int gt = t0 + tt, gc = c0 + c;
      cp_async4(ys + tt * TT + c, TY ? yb + (int64_t)gc * nl + gt : yb + (int64_t)gt * nj + gc);
    }
  }
}

// A pack: the lambda work of one stage, either whole consecutive lambda blocks [m0, m1)
// whose widths add up to at most KM, or one KM-wide slice [t0, t0 + K) of a block wider
// than KM.  All lanes compute the same packs.
struct Pack {
  int m0, m1, t0, K, done;  // done: lambda blocks completed by this pack
};

template <int KM>
__device__ __forceinline__ Pack next_pack(const Stage* st, int nm, int m, int t0) {
  Pack pk;
  pk.m0 = m;
  pk.t0 = t0;
  const int nl = st[m].nl;
  if (nl > KM) {
    pk.K = min(KM, nl - t0);
    pk.m1 = m + 1;
    pk.done = (t0 + pk.K >= nl) ? 1 : 0;
    return pk;
  }
  int k = 0, m1 = m;
  while (m1 < nm && st[m1].nl <= KM && k + st[m1].nl <= KM) {
    k += st[m1].nl;
    ++m1;
  }
  pk.m1 = m1;
  pk.K = k;
  pk.done = m1 - m;
  return pk;
}

template <int TT, int KM, bool TX, bool TY>
__device__ __forceinline__ void pack_copy(const Pack& pk, const Stage* st, const float* __restrict__ X,
                                          const float* __restrict__ Y, const int64_t* xvoff, const int64_t* yvoff,
                                          int ni, int nj, int r0, int c0, int th, int tw, int lane, float* xs,
                                          float* ys) {
  if (st[pk.m0].nl > KM) {
    stage_copy<TT, TX, TY>(st[pk.m0], pk.t0, pk.K, 0, X, Y, xvoff, yvoff, ni, nj, r0, c0, th, tw, lane, xs, ys);
    return;
  }
  int k0 = 0;
  for (int j = pk.m0; j < pk.m1; ++j) {
    const int nl = st[j].nl;
    stage_copy<TT, TX, TY>(st[j], 0, nl, k0, X, Y, xvoff, yvoff, ni, nj, r0, c0, th, tw, lane, xs, ys);
    k0 += nl;
  }
}

template <int TT, int MR, int MC, int KM, bool TX, bool TY>
__global__ void __launch_bounds__(kF32Warps * 32, 4) mul_f32_kernel(MulArgs a, const float* __restrict__ X,
                                                                    const float* __restrict__ Y,
                                                                    float* __restrict__ C) {
  constexpr int GR = TT / MR, GC = TT / MC, NA = GR * GC, NQ = MR * MC;
  static_assert(TT % MR == 0 && TT % MC == 0 && NA <= 32 && TT % 2 == 0 && (MR != 4 || TT % 4 == 0) &&
                    (MC != 4 || TT % 4 == 0) && KM >= TT,
                "bad micro-tile");
  extern __shared__ __align__(16) float fsm[];   // [warp][buf][A | B][KM * TT]
  __shared__ Stage sStage[kF32Warps][kStages];  // the batch's matching lambda blocks
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  float* wbase = fsm + (size_t)w * 4 * KM * TT;
  Stage* st = sStage[w];
  const bool active = lane < NA;
  const int mr = active ? lane / GC : 0, mc = active ? lane % GC : 0;
  const int rl = MR * mr, cl = MC * mc;
  for (;;) {
    unsigned int t = 0;
    if (lane == 0) t = atomicAdd(a.counter, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= a.ntiles) break;
    const Tile tile = a.tiles[t];
    const int k = tile.blk;
    const int nu = a.c_brow[k], nup = a.c_col[k];
    const int ni = a.bsize[nu], nj = a.bsize[nup];
    const int th = min(TT, ni - tile.r0), tw = min(TT, nj - tile.c0);
    float acc[NQ], comp[NQ], p[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = comp[q] = p[q] = 0.0f;
    int folded = 0;  // lambda blocks summed into p since the last two-sum
    const int px1 = (int)a.x.ptr[nu + 1];
    int px = (int)a.x.ptr[nu];
    int py0 = (int)a.y.ptr[nup];
    const int py1 = (int)a.y.ptr[nup + 1];
    while (px < px1 && py0 < py1) {
      // ---- list up to kStages matching lambda blocks ------------------------------------
      int nm = 0;
      while (px < px1 && py0 < py1 && nm <= kStages - 32) {
        const int i = px + lane;
        const int32_t lam = i < px1 ? __ldg(a.x.idx + i) : INT32_MAX;
        const int pos = lower_bound_dev(a.y.idx, py0, py1, lam);
        const bool hit = i < px1 && pos < py1 && __ldg(a.y.idx + pos) == lam;
        const unsigned int mask = __ballot_sync(0xffffffffu, hit);
        if (hit) {
          const int kx = a.x.blk ? __ldg(a.x.blk + i) : i;
          const int ky = a.y.blk ? __ldg(a.y.blk + pos) : pos;
          const int o = nm + __popc(mask & ((1u << lane) - 1u));
          st[o] = Stage{kx, ky, (int16_t)a.bsize[lam], 0};
        }
        nm += __popc(mask);
        py0 = __shfl_sync(0xffffffffu, pos, 31);
        px += 32;
      }
      __syncwarp();
      if (nm == 0) continue;
      // ---- stream the packs: the copies of the next pack overlap the FMAs of the current
      Pack cur = next_pack<KM>(st, nm, 0, 0);
      pack_copy<TT, KM, TX, TY>(cur, st, X, Y, a.x.voff, a.y.voff, ni, nj, tile.r0, tile.c0, th, tw, lane, wbase,
                                wbase + KM * TT);
      cp_commit();
      int buf = 0;
      for (;;) {
        const int nm_next = cur.done ? cur.m1 : cur.m0;
        const int nt_next = cur.done ? 0 : cur.t0 + cur.K;
        const bool more = nm_next < nm;
        Pack nxt;
        if (more) {
          nxt = next_pack<KM>(st, nm, nm_next, nt_next);
          float* nb = wbase + (buf ^ 1) * 2 * KM * TT;
          pack_copy<TT, KM, TX, TY>(nxt, st, X, Y, a.x.voff, a.y.voff, ni, nj, tile.r0, tile.c0, th, tw, lane, nb,
                                    nb + KM * TT);
          cp_commit();
          cp_wait<1>();
        } else {
          cp_wait<0>();
        }
        __syncwarp();
        if (active) {
          const float* xs = wbase + buf * 2 * KM * TT;
          const float* ys = xs + KM * TT;
          auto step = [&](int tt) {
            float ar[MR], br[MC];
            lds<MR>(xs + tt * TT + rl, ar);
            lds<MC>(ys + tt * TT + cl, br);
#pragma unroll
            for (int ii = 0; ii < MR; ++ii)
#pragma unroll
              for (int jj = 0; jj < MC; ++jj) p[ii * MC + jj] = fmaf(ar[ii], br[jj], p[ii * MC + jj]);
          };
          if (cur.K == KM) {
#pragma unroll
            for (int tt = 0; tt < KM; ++tt) step(tt);
          } else {
#pragma unroll 4
            for (int tt = 0; tt < cur.K; ++tt) step(tt);
          }
        }
        __syncwarp();
        folded += cur.done;
        if (folded >= kFold) {
          folded = 0;
#pragma unroll
          for (int qq = 0; qq < NQ; ++qq) {
            const float hi = acc[qq] + p[qq];
            const float bp = hi - acc[qq];
            comp[qq] += (acc[qq] - (hi - bp)) + (p[qq] - bp);
            acc[qq] = hi;
            p[qq] = 0.0f;
          }
        }
        if (!more) break;
        cur = nxt;
        buf ^= 1;
      }
    }
    if (active) {
      float* cb = C + a.c_voff[k];
#pragma unroll
      for (int ii = 0; ii < MR; ++ii)
#pragma unroll
        for (int jj = 0; jj < MC; ++jj) {
          const int qq = ii * MC + jj;
          const float hi = acc[qq] + p[qq];
          const float bp = hi - acc[qq];
          const float err = (acc[qq] - (hi - bp)) + (p[qq] - bp);
          const int r = rl + ii, c = cl + jj;
          if (r < th && c < tw) cb[(int64_t)(tile.r0 + r) * nj + tile.c0 + c] = hi + (comp[qq] + err);
        }
    }
  }
}

// Double-float product (S_FP64_DF): double operands arrive pre-split into float pairs
// (hi, lo) with hi + lo = a to 2^-48; each term a*b is formed as the exact float product
// hi*hi (fmaf recovers its rounding error) plus the cross terms hi*lo + lo*hi, and added
// to the lambda block's float-pair partial with an error-free two-sum (~12 float
// instructions per multiply-add).  At the end of each lambda block the partial is added to
// the running float-pair total by a full pair addition with renormalisation, so the
// rounding of the low words grows with the number of lambda blocks, not of terms.  Same
// tiling, listing and cp.async streaming as the float kernel; tiles of 20 with 4x4
// micro-tiles; shared memory is dynamic (float2).
__global__ void split_kernel(int64_t n, const double* __restrict__ a, float2* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = a[i];
    const float hi = __double2float_rn(v);
    out[i] = make_float2(hi, __double2float_rn(v - (double)hi));
  }
}

__device__ __forceinline__ void cp_async8(float2* dst, const float2* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src));
}

template <int TT, bool TX, bool TY>
__device__ __forceinline__ void stage_copy_df(const Stage& sg, const float2* __restrict__ X,
                                              const float2* __restrict__ Y, const int64_t* xvoff,
                                              const int64_t* yvoff, int ni, int nj, int r0, int c0, int th, int tw,
                                              int lane, float2* xs, float2* ys) {
  const int nl = sg.nl, t0 = sg.t0;
  const int tk = min(TT, nl - t0);
  const float2* xb = X + xvoff[sg.bx];
  const float2* yb = Y + yvoff[sg.by];
  const float rtk = 1.0f / (float)tk, rtw = 1.0f / (float)tw;
  for (int e = lane; e < th * tk; e += 32) {
    const int r = __float2int_rz(((float)e + 0.5f) * rtk), tt = e - r * tk;
    const int gr = r0 + r, gt = t0 + tt;
    cp_async8(xs + tt * TT + r, TX ? xb + (int64_t)gt * ni + gr : xb + (int64_t)gr * nl + gt);
  }
  for (int e = lane; e < tk * tw; e += 32) {
    const int tt = __float2int_rz(((float)e + 0.5f) * rtw), c = e - tt * tw;
    const int gt = t0 + tt, gc = c0 + c;
    cp_async8(ys + tt * TT + c, TY ? yb + (int64_t)gc * nl + gt : yb + (int64_t)gt * nj + gc);
  }
}

constexpr int kDfWarps = 4;
struct DfVariant {
  int tt, mr, mc;
};
constexpr DfVariant kDfVariants[] = {{20, 4, 4}, {10, 2, 2}};
constexpr int kNumDfVariants = 2;
static size_t df_smem(int v) {  // [warp][buf][A|B][TT*TT] float2
  return sizeof(float2) * kDfWarps * 2 * 2 * kDfVariants[v].tt * kDfVariants[v].tt;
}

template <int TT, int MR, int MC, bool TX, bool TY>
__global__ void __launch_bounds__(kDfWarps * 32, 3) mul_df_kernel(MulArgs a, const float2* __restrict__ X,
                                                                  const float2* __restrict__ Y,
                                                                  double* __restrict__ C) {
  constexpr int GC = TT / MC, NA = (TT / MR) * GC, NQ = MR * MC;
  static_assert(TT % MR == 0 && TT % MC == 0 && NA <= 32, "bad micro-tile");
  extern __shared__ __align__(16) float2 dsm[];
  __shared__ Stage sStage[kDfWarps][kStages];
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  float2* base = dsm + (size_t)w * 4 * TT * TT;  // [buf0: A, B][buf1: A, B]
  Stage* st = sStage[w];
  const bool active = lane < NA;
  const int mr = active ? lane / GC : 0, mc = active ? lane % GC : 0;
  const int rl = MR * mr, cl = MC * mc;
  for (;;) {
    unsigned int t = 0;
    if (lane == 0) t = atomicAdd(a.counter, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= a.ntiles) break;
    const Tile tile = a.tiles[t];
    const int k = tile.blk;
    const int nu = a.c_brow[k], nup = a.c_col[k];
    const int ni = a.bsize[nu], nj = a.bsize[nup];
    const int th = min(TT, ni - tile.r0), tw = min(TT, nj - tile.c0);
    float sh[NQ], sl[NQ], ph[NQ], pl[NQ];  // running total and lambda-block partial
#pragma unroll
    for (int q = 0; q < NQ; ++q) sh[q] = sl[q] = ph[q] = pl[q] = 0.0f;
    const int px1 = (int)a.x.ptr[nu + 1];
    int px = (int)a.x.ptr[nu];
    int py0 = (int)a.y.ptr[nup];
    const int py1 = (int)a.y.ptr[nup + 1];
    while (px < px1 && py0 < py1) {
      int nm = 0;
      while (px < px1 && py0 < py1 && nm <= kStages - 32) {
        const int i = px + lane;
        const int32_t lam = i < px1 ? __ldg(a.x.idx + i) : INT32_MAX;
        const int pos = lower_bound_dev(a.y.idx, py0, py1, lam);
        const bool hit = i < px1 && pos < py1 && __ldg(a.y.idx + pos) == lam;
        const unsigned int mask = __ballot_sync(0xffffffffu, hit);
        if (hit) {
          const int kx = a.x.blk ? __ldg(a.x.blk + i) : i;
          const int ky = a.y.blk ? __ldg(a.y.blk + pos) : pos;
          st[nm + __popc(mask & ((1u << lane) - 1u))] = Stage{kx, ky, (int16_t)a.bsize[lam], 0};
        }
        nm += __popc(mask);
        py0 = __shfl_sync(0xffffffffu, pos, 31);
        px += 32;
      }
      __syncwarp();
      if (nm == 0) continue;
      int m = 0, q = 0, buf = 0;
      stage_copy_df<TT, TX, TY>(st[0], X, Y, a.x.voff, a.y.voff, ni, nj, tile.r0, tile.c0, th, tw, lane, base,
                                base + TT * TT);
      cp_commit();
      for (;;) {
        const Stage cur = st[m];
        const int t0 = q * TT;
        const bool last_slice = t0 + TT >= (int)cur.nl;
        const int nm2 = last_slice ? m + 1 : m, nq2 = last_slice ? 0 : q + 1;
        const bool more = nm2 < nm;
        if (more) {
          Stage sg = st[nm2];
          sg.t0 = (int16_t)(nq2 * TT);
          float2* nb = base + (buf ^ 1) * 2 * TT * TT;
          stage_copy_df<TT, TX, TY>(sg, X, Y, a.x.voff, a.y.voff, ni, nj, tile.r0, tile.c0, th, tw, lane, nb,
                                    nb + TT * TT);
          cp_commit();
          cp_wait<1>();
        } else {
          cp_wait<0>();
        }
        __syncwarp();
        const int tk = min(TT, (int)cur.nl - t0);
        if (active) {
          const float2* xs = base + buf * 2 * TT * TT;
          const float2* ys = xs + TT * TT;
          for (int tt = 0; tt < tk; ++tt) {
            float2 av[MR], bv[MC];
#pragma unroll
            for (int u = 0; u < MR; ++u) av[u] = xs[tt * TT + rl + u];
#pragma unroll
            for (int u = 0; u < MC; ++u) bv[u] = ys[tt * TT + cl + u];
#pragma unroll
            for (int ii = 0; ii < MR; ++ii)
#pragma unroll
              for (int jj = 0; jj < MC; ++jj) {
                const int qq = ii * MC + jj;
                const float p = av[ii].x * bv[jj].x;
                float e = fmaf(av[ii].x, bv[jj].x, -p);
                e = fmaf(av[ii].x, bv[jj].y, e);
                e = fmaf(av[ii].y, bv[jj].x, e);
                const float hi = ph[qq] + p;
                const float bp = hi - ph[qq];
                pl[qq] += ((ph[qq] - (hi - bp)) + (p - bp)) + e;
                ph[qq] = hi;
              }
          }
        }
        __syncwarp();
        if (last_slice) {
          // (sh, sl) += (ph, pl): two-sum of the high words, low words added, renormalised
#pragma unroll
          for (int qq = 0; qq < NQ; ++qq) {
            const float s1 = sh[qq] + ph[qq];
            const float bp = s1 - sh[qq];
            const float e1 = ((sh[qq] - (s1 - bp)) + (ph[qq] - bp)) + (sl[qq] + pl[qq]);
            const float s2 = s1 + e1;
            sl[qq] = e1 - (s2 - s1);
            sh[qq] = s2;
            ph[qq] = pl[qq] = 0.0f;
          }
        }
        if (!more) break;
        m = nm2;
        q = nq2;
        buf ^= 1;
      }
    }
    if (active) {
      double* cb = C + a.c_voff[k];
#pragma unroll
      for (int ii = 0; ii < MR; ++ii)
#pragma unroll
        for (int jj = 0; jj < MC; ++jj) {
          const int r = rl + ii, c = cl + jj;
          if (r < th && c < tw)
            cb[(int64_t)(tile.r0 + r) * nj + tile.c0 + c] = (double)sh[ii * MC + jj] + (double)sl[ii * MC + jj];
        }
    }
  }
}

// Split-bfloat16 tensor-core product (S_BF16X3): float operands pre-split into three
// bfloat16 planes, a = a0 + a1 + a2 to 2^-24 relative; the six leading cross products
// a_i b_j (i + j <= 2, smallest first) run on the tensor cores as m16n8k8 bf16 MMAs with
// float accumulation, per lambda block, and the lambda sum is compensated as in the float
// kernel.  Output tiles of 20 x 20 padded to 32 x 24 (two m16, three n8), lambda slices of 20
// padded to 24 (three k8).  Staging: 4- or 8-byte cp.async copies of the planes into
// double-buffered shared tiles, op(X) as [k][m] (80-byte rows) or [m][k] (48-byte rows),
// op(Y) as [k][n] (80-byte rows), all read by ldmatrix (.trans where k is the row).
__global__ void split3_kernel(int64_t n, const float* __restrict__ a, __nv_bfloat16* __restrict__ p0,
                              __nv_bfloat16* __restrict__ p1, __nv_bfloat16* __restrict__ p2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = a[i];
    const __nv_bfloat16 h0 = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(h0);
    const __nv_bfloat16 h1 = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(h1);
    p0[i] = h0;
    p1[i] = h1;
    p2[i] = __float2bfloat16_rn(r2);
  }
}

constexpr int kTcWarps = 4;
constexpr int kTcK = 24;        // padded lambda slice (three k8)
constexpr int kTcLdKM = 40;     // [k][m] and [k][n] row length in bf16 (80 bytes)
constexpr int kTcLdMK = 24;     // [m][k] row length in bf16 (48 bytes)
constexpr int kTcPlane = 32 * kTcLdKM;  // bf16 per operand plane per buffer (covers both layouts)
// per warp: [buf 2][operand 2][plane 3][kTcPlane]
constexpr size_t kTcSmem = sizeof(__nv_bfloat16) * kTcWarps * 2 * 2 * 3 * kTcPlane;

__device__ __forceinline__ void cp_async_b(void* dst, const void* src, int bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if (bytes == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src));
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src));
}

struct Planes {
  const __nv_bfloat16* p[3];
};

// Copy one lambda slice of op(X) and op(Y) (three planes each) into the stage buffer.
template <bool TX, bool TY>
__device__ __forceinline__ void tc_stage_copy(const Stage& sg, const Planes& X, const Planes& Y, const int64_t* xvoff,
                                              const int64_t* yvoff, int ni, int nj, int r0, int c0, int th, int tw,
                                              int lane, __nv_bfloat16* xs, __nv_bfloat16* ys) {
  const int nl = sg.nl, t0 = sg.t0;
  const int tk = min(kTile, nl - t0);
  const int64_t xo = xvoff[sg.bx], yo = yvoff[sg.by];
  // op(X): TX -> stored (lambda, nu) rows t: [k][m] layout, a run of th along m per k
  //        !TX -> stored (nu, lambda) rows r: [m][k] layout, a run of tk along k per m
  const int xrun = TX ? th : tk, xrows = TX ? tk : th;
  // bf16 per copy: 4 (8 bytes) when row length, run start and run length are multiples of
  // 4, else 2 (4 bytes; all block sizes and tile offsets are even, block offsets are
  // multiples of 4 entries since they are sums of products of even sizes)
  const int xch = (((TX ? (ni | r0 | th) : (nl | t0 | tk)) & 3) == 0) ? 4 : 2;
  const int xper = xrun / xch;
  const float rxp = 1.0f / (float)xper;
  for (int e = lane; e < xrows * xper; e += 32) {
    const int row = __float2int_rz(((float)e + 0.5f) * rxp), q = e - row * xper;
    const int64_t src = TX ? xo + (int64_t)(t0 + row) * ni + r0 + q * xch : xo + (int64_t)(r0 + row) * nl + t0 + q * xch;
    __nv_bfloat16* dst = xs + (TX ? row * kTcLdKM : row * kTcLdMK) + q * xch;
#pragma unroll
    for (int pl = 0; pl < 3; ++pl) cp_async_b(dst + pl * kTcPlane, X.p[pl] + src, xch * 2);
  }
  // op(Y): !TY -> stored (lambda, nu') rows t: [k][n], a run of tw along n per k
  const int ych = ((nj | c0 | tw) & 3) == 0 ? 4 : 2;
  const int yper = tw / ych;
  if (!TY) {
    const float ryp = 1.0f / (float)yper;
    for (int e = lane; e < tk * yper; e += 32) {
      const int row = __float2int_rz(((float)e + 0.5f) * ryp), q = e - row * yper;
      const int64_t src = yo + (int64_t)(t0 + row) * nj + c0 + q * ych;
#pragma unroll
      for (int pl = 0; pl < 3; ++pl)
        cp_async_b(ys + pl * kTcPlane + row * kTcLdKM + q * ych, Y.p[pl] + src, ych * 2);
    }
  } else {
    // TY: stored (nu', lambda): element (t, c) at c * nl + t; scalar copies
    const float rtw = 1.0f / (float)tw;
    for (int e = lane; e < tk * tw; e += 32) {
      const int row = __float2int_rz(((float)e + 0.5f) * rtw), c = e - row * tw;
#pragma unroll
      for (int pl = 0; pl < 3; ++pl)
        ys[pl * kTcPlane + row * kTcLdKM + c] = Y.p[pl][yo + (int64_t)(c0 + c) * nl + t0 + row];
    }
  }
}

__device__ __forceinline__ void ldsm_x2(unsigned& r0, unsigned& r1, const void* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(a));
}
__device__ __forceinline__ void ldsm_x2_t(unsigned& r0, unsigned& r1, const void* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(a));
}
__device__ __forceinline__ void ldsm_x1_t(unsigned& r0, const void* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x1.trans.shared.b16 {%0}, [%1];\n" : "=r"(r0) : "r"(a));
}
__device__ __forceinline__ void mma_bf16_k8(float* c, unsigned a0, unsigned a1, unsigned b0) {
  asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
               : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
               : "r"(a0), "r"(a1), "r"(b0));
}

template <bool TX, bool TY>
__global__ void __launch_bounds__(kTcWarps * 32, 2) mul_bf16x3_kernel(MulArgs a, Planes X, Planes Y,
                                                                      float* __restrict__ C) {
  extern __shared__ __align__(16) __nv_bfloat16 tsm[];
  __shared__ Stage sStage[kTcWarps][kStages];
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  __nv_bfloat16* base = tsm + (size_t)w * 2 * 2 * 3 * kTcPlane;  // [buf][X|Y][plane][kTcPlane]
  Stage* st = sStage[w];
  // zero the warp's buffers once: padding rows/columns stay zero
  for (int e = lane; e < 2 * 2 * 3 * kTcPlane / 2; e += 32) reinterpret_cast<unsigned*>(base)[e] = 0u;
  __syncwarp();
  const int g = lane >> 2, tq = lane & 3;
  // ldmatrix row addresses: lanes 0-7 give rows of matrix 0, 8-15 of matrix 1
  const int lr = lane & 7, lm = (lane >> 3) & 1;
  for (;;) {
    unsigned int t = 0;
    if (lane == 0) t = atomicAdd(a.counter, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= a.ntiles) break;
    const Tile tile = a.tiles[t];
    const int k = tile.blk;
    const int nu = a.c_brow[k], nup = a.c_col[k];
    const int ni = a.bsize[nu], nj = a.bsize[nup];
    const int th = min(kTile, ni - tile.r0), tw = min(kTile, nj - tile.c0);
    float pc[2][3][4], acc[2][3][4], comp[2][3][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) pc[i][j][q] = acc[i][j][q] = comp[i][j][q] = 0.0f;
    int folded = 0;
    int tk_b0 = kTile, tk_b1 = kTile;  // width of the slice last copied into each buffer
    const int px1 = (int)a.x.ptr[nu + 1];
    int px = (int)a.x.ptr[nu];
    int py0 = (int)a.y.ptr[nup];
    const int py1 = (int)a.y.ptr[nup + 1];
    while (px < px1 && py0 < py1) {
      int nm = 0;
      while (px < px1 && py0 < py1 && nm <= kStages - 32) {
        const int i = px + lane;
        const int32_t lam = i < px1 ? __ldg(a.x.idx + i) : INT32_MAX;
        const int pos = lower_bound_dev(a.y.idx, py0, py1, lam);
        const bool hit = i < px1 && pos < py1 && __ldg(a.y.idx + pos) == lam;
        const unsigned int mask = __ballot_sync(0xffffffffu, hit);
        if (hit) {
          const int kx = a.x.blk ? __ldg(a.x.blk + i) : i;
          const int ky = a.y.blk ? __ldg(a.y.blk + pos) : pos;
          st[nm + __popc(mask & ((1u << lane) - 1u))] = Stage{kx, ky, (int16_t)a.bsize[lam], 0};
        }
        nm += __popc(mask);
        py0 = __shfl_sync(0xffffffffu, pos, 31);
        px += 32;
      }
      __syncwarp();
      if (nm == 0) continue;
      int m = 0, q = 0, buf = 0;
      // slices narrower than an earlier one in the same buffer leave stale k rows/columns:
      // zero them before copying (K padding must be zero in both operands)
      auto prep = [&](int b, int tk) {
        if (tk < (b ? tk_b1 : tk_b0)) {
          __nv_bfloat16* xb = base + (b * 2 + 0) * 3 * kTcPlane;
          __nv_bfloat16* yb = base + (b * 2 + 1) * 3 * kTcPlane;
          const __nv_bfloat16 z = __float2bfloat16_rn(0.0f);
          for (int kk = tk; kk < kTile; ++kk)      // lane = m (or n) index
#pragma unroll
            for (int pl = 0; pl < 3; ++pl) {
              if (TX) xb[pl * kTcPlane + kk * kTcLdKM + lane] = z;
              else if (lane < kTcLdMK) xb[pl * kTcPlane + lane * kTcLdMK + kk] = z;
              yb[pl * kTcPlane + kk * kTcLdKM + lane] = z;
            }
        }
        if (b) tk_b1 = tk;
        else tk_b0 = tk;
      };
      {
        const int tk0 = min(kTile, (int)st[0].nl);
        prep(0, tk0);
        __syncwarp();
        tc_stage_copy<TX, TY>(st[0], X, Y, a.x.voff, a.y.voff, ni, nj, tile.r0, tile.c0, th, tw, lane,
                              base, base + 3 * kTcPlane);
        cp_commit();
      }
      for (;;) {
        const Stage cur = st[m];
        const int t0 = q * kTile;
        const bool last_slice = t0 + kTile >= (int)cur.nl;
        const int nm2 = last_slice ? m + 1 : m, nq2 = last_slice ? 0 : q + 1;
        const bool more = nm2 < nm;
        if (more) {
          Stage sg = st[nm2];
          sg.t0 = (int16_t)(nq2 * kTile);
          prep(buf ^ 1, min(kTile, (int)sg.nl - (int)sg.t0));
          __syncwarp();
          __nv_bfloat16* nb = base + (buf ^ 1) * 2 * 3 * kTcPlane;
          tc_stage_copy<TX, TY>(sg, X, Y, a.x.voff, a.y.voff, ni, nj, tile.r0, tile.c0, th, tw, lane, nb,
                                nb + 3 * kTcPlane);
          cp_commit();
          cp_wait<1>();
        } else {
          cp_wait<0>();
        }
        __syncwarp();
        {
          const __nv_bfloat16* xs = base + buf * 2 * 3 * kTcPlane;
          const __nv_bfloat16* ys = xs + 3 * kTcPlane;
#pragma unroll
          for (int kk = 0; kk < 3; ++kk) {
            // fragments of the three planes for this k8 step
            unsigned af[3][2][2], bfr[3][3];
#pragma unroll
            for (int pl = 0; pl < 3; ++pl) {
#pragma unroll
              for (int mi = 0; mi < 2; ++mi) {
                if (TX) {
                  // [k][m]: matrix 0 = m 0-7, matrix 1 = m 8-15 of this m16, rows k
                  const __nv_bfloat16* pa = xs + pl * kTcPlane + (kk * 8 + lr) * kTcLdKM + mi * 16 + lm * 8;
                  ldsm_x2_t(af[pl][mi][0], af[pl][mi][1], pa);
                } else {
                  const __nv_bfloat16* pa = xs + pl * kTcPlane + (mi * 16 + lm * 8 + lr) * kTcLdMK + kk * 8;
                  ldsm_x2(af[pl][mi][0], af[pl][mi][1], pa);
                }
              }
#pragma unroll
              for (int nj8 = 0; nj8 < 3; ++nj8) {
                const __nv_bfloat16* pb = ys + pl * kTcPlane + (kk * 8 + lr) * kTcLdKM + nj8 * 8;
                ldsm_x1_t(bfr[pl][nj8], pb);
              }
            }
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
              for (int nj8 = 0; nj8 < 3; ++nj8) {
                float* c = pc[mi][nj8];
                mma_bf16_k8(c, af[2][mi][0], af[2][mi][1], bfr[0][nj8]);
                mma_bf16_k8(c, af[1][mi][0], af[1][mi][1], bfr[1][nj8]);
                mma_bf16_k8(c, af[0][mi][0], af[0][mi][1], bfr[2][nj8]);
                mma_bf16_k8(c, af[1][mi][0], af[1][mi][1], bfr[0][nj8]);
                mma_bf16_k8(c, af[0][mi][0], af[0][mi][1], bfr[1][nj8]);
                mma_bf16_k8(c, af[0][mi][0], af[0][mi][1], bfr[0][nj8]);
              }
          }
        }
        __syncwarp();
        if (last_slice && ++folded == kFold) {
          folded = 0;
#pragma unroll
          for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
              for (int qq = 0; qq < 4; ++qq) {
                const float hi = acc[i][j][qq] + pc[i][j][qq];
                const float bp = hi - acc[i][j][qq];
                comp[i][j][qq] += (acc[i][j][qq] - (hi - bp)) + (pc[i][j][qq] - bp);
                acc[i][j][qq] = hi;
                pc[i][j][qq] = 0.0f;
              }
        }
        if (!more) break;
        m = nm2;
        q = nq2;
        buf ^= 1;
      }
    }
    float* cb = C + a.c_voff[k];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
          const int r = i * 16 + g + (qq >= 2 ? 8 : 0), c = j * 8 + 2 * tq + (qq & 1);
          const float hi = acc[i][j][qq] + pc[i][j][qq];
          const float bp = hi - acc[i][j][qq];
          const float err = (acc[i][j][qq] - (hi - bp)) + (pc[i][j][qq] - bp);
          if (r < th && c < tw) cb[(int64_t)(tile.r0 + r) * nj + tile.c0 + c] = hi + (comp[i][j][qq] + err);
        }
  }
}

// Row-panel float product for small blocks.  One warp owns up to P consecutive output
// tiles of one block row: the same rows r0 .. r0 + th of block row nu, in different column
// blocks nu'_j.  For every lambda of row nu the slice of op(X)(nu, lambda) is staged once
// and reused by each member j whose block (lambda, nu'_j) exists in op(Y); absent members
// skip both the copy and the FMAs.  Lane (mr, mc) owns the same MR x MC micro-position in
// every member tile.  The lambda listing (ballot plus one binary search per member),
// cp.async double buffering and the compensated lambda sums follow the tile kernel.
constexpr int kPMax = 4;
struct PStage {
  int32_t bx;
  int16_t nl, pad;
  int32_t by[kPMax];  // -1: block (lambda, nu'_j) absent
};

struct PanelArgs {
  const Tile* ptiles;
  const int2* pidx;  // (first tile, tile count) of each panel
  int64_t npanels;
};

// Slice [t0, t0 + wd) of op(X)(nu, lambda), rows r0 .. r0 + th, into xs[k][r] (k-major).
template <int TT, bool TX>
__device__ __forceinline__ void panel_copy_x(const float* xb, int t0, int wd, int ni, int nl, int r0, int th,
                                             int lane, float* xs) {
  const bool xvec = TT % 4 == 0 && TX && r0 == 0 && th == ni && (ni & 3) == 0 &&
                    ((reinterpret_cast<uintptr_t>(xb) & 15) == 0);
  if (xvec) {
    const float rni = 1.0f / (float)ni;
    for (int q = lane; q < (wd * ni) >> 2; q += 32) {
      const int e = q << 2;
      const int tt = __float2int_rz(((float)e + 0.5f) * rni), r = e - tt * ni;
      cp_async16(xs + tt * TT + r, xb + (int64_t)(t0 + tt) * ni + r);
    }
  } else {
    const float rwd = 1.0f / (float)wd;
    for (int e = lane; e < th * wd; e += 32) {
      const int r = __float2int_rz(((float)e + 0.5f) * rwd), tt = e - r * wd;
      const int gr = r0 + r, gt = t0 + tt;
      cp_async4(xs + tt * TT + r, TX ? xb + (int64_t)gt * ni + gr : xb + (int64_t)gr * nl + gt);
    }
  }
}

// Slice [t0, t0 + wd) of op(Y)(lambda, nu'), columns c0 .. c0 + tw, into ys[k][c].
template <int TT, bool TY>
__device__ __forceinline__ void panel_copy_y(const float* yb, int t0, int wd, int nj, int nl, int c0, int tw,
                                             int lane, float* ys) {
  const bool vec = TT % 4 == 0 && !TY && c0 == 0 && tw == nj && (nj & 3) == 0 &&
                   ((reinterpret_cast<uintptr_t>(yb) & 15) == 0);
  if (vec) {
    const float rnj = 1.0f / (float)nj;
    for (int q = lane; q < (wd * nj) >> 2; q += 32) {
      const int e = q << 2;
      const int tt = __float2int_rz(((float)e + 0.5f) * rnj), c = e - tt * nj;
      cp_async16(ys + tt * TT + c, yb + (int64_t)(t0 + tt) * nj + c);
    }
  } else {
    const float rtw = 1.0f / (float)tw;
    for (int e = lane; e < wd * tw; e += 32) {
      const int tt = __float2int_rz(((float)e + 0.5f) * rtw), c = e - tt * tw;
      const int gt = t0 + tt, gc = c0 + c;
      cp_async4(ys + tt * TT + c, TY ? yb + (int64_t)gc * nl + gt : yb + (int64_t)gt * nj + gc);
    }
  }
}

template <int TT, int MR, int MC, int P, bool TX, bool TY>
__global__ void __launch_bounds__(kF32Warps * 32, 4) mul_f32_panel_kernel(MulArgs a, PanelArgs pa,
                                                                          const float* __restrict__ X,
                                                                          const float* __restrict__ Y,
                                                                          float* __restrict__ C) {
  constexpr int GR = TT / MR, GC = TT / MC, NA = GR * GC, NQ = MR * MC, BUF = (1 + P) * TT * TT;
  static_assert(TT % MR == 0 && TT % MC == 0 && NA <= 32 && TT % 2 == 0 && P >= 1 && P <= kPMax &&
                    (MR != 4 || TT % 4 == 0) && (MC != 4 || TT % 4 == 0),
                "bad panel shape");
  extern __shared__ __align__(16) float psm[];  // [warp][buf][X | Y_0 .. Y_{P-1}][TT * TT]
  __shared__ PStage sSt[kF32Warps][kStages];
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  float* wbase = psm + (size_t)w * 2 * BUF;
  PStage* st = sSt[w];
  const bool active = lane < NA;
  const int mr = active ? lane / GC : 0, mc = active ? lane % GC : 0;
  const int rl = MR * mr, cl = MC * mc;
  for (;;) {
    unsigned int t = 0;
    if (lane == 0) t = atomicAdd(a.counter, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= pa.npanels) break;
    const int2 pi = pa.pidx[t];
    const Tile* tl = pa.ptiles + pi.x;
    const int cnt = pi.y;
    const int nu = a.c_brow[tl[0].blk];
    const int ni = a.bsize[nu];
    const int r0 = tl[0].r0;
    const int th = min(TT, ni - r0);
    int kj[P], njv[P], c0v[P], twv[P], py0[P], py1[P];
#pragma unroll
    for (int j = 0; j < P; ++j) {
      kj[j] = -1, njv[j] = 0, c0v[j] = 0, twv[j] = 0, py0[j] = 0, py1[j] = 0;
      if (j < cnt) {
        const Tile tj = tl[j];
        const int nup = a.c_col[tj.blk];
        kj[j] = tj.blk;
        njv[j] = a.bsize[nup];
        c0v[j] = tj.c0;
        twv[j] = min(TT, njv[j] - c0v[j]);
        py0[j] = (int)a.y.ptr[nup];
        py1[j] = (int)a.y.ptr[nup + 1];
      }
    }
    float acc[P][NQ], comp[P][NQ], p[P][NQ];
#pragma unroll
    for (int j = 0; j < P; ++j)
#pragma unroll
      for (int q = 0; q < NQ; ++q) acc[j][q] = comp[j][q] = p[j][q] = 0.0f;
    int folded = 0;  // lambda blocks summed into p since the last two-sum
    const int px1 = (int)a.x.ptr[nu + 1];
    int px = (int)a.x.ptr[nu];
    while (px < px1) {
      // ---- list up to kStages lambdas that meet at least one member ---------------------
      int nm = 0;
      while (px < px1 && nm <= kStages - 32) {
        const int i = px + lane;
        const int32_t lam = i < px1 ? __ldg(a.x.idx + i) : INT32_MAX;
        PStage ps;
        bool any = false;
#pragma unroll
        for (int j = 0; j < kPMax; ++j) ps.by[j] = -1;
#pragma unroll
        for (int j = 0; j < P; ++j) {
          if (j < cnt) {
            const int pos = lower_bound_dev(a.y.idx, py0[j], py1[j], lam);
            const bool hit = i < px1 && pos < py1[j] && __ldg(a.y.idx + pos) == lam;
            if (hit) ps.by[j] = a.y.blk ? __ldg(a.y.blk + pos) : pos;
            any |= hit;
            py0[j] = __shfl_sync(0xffffffffu, pos, 31);
          }
        }
        const unsigned int mask = __ballot_sync(0xffffffffu, any);
        if (any) {
          ps.bx = a.x.blk ? __ldg(a.x.blk + i) : i;
          ps.nl = (int16_t)a.bsize[lam];
          ps.pad = 0;
          st[nm + __popc(mask & ((1u << lane) - 1u))] = ps;
        }
        nm += __popc(mask);
        px += 32;
      }
      __syncwarp();
      if (nm == 0) continue;
      // ---- stream TT-wide slices of the listed lambdas; the next slice's copies overlap
      // ---- the current slice's FMAs
      auto issue = [&](int m, int t0, float* b) {
        const PStage& sg = st[m];
        const int wd = min(TT, (int)sg.nl - t0);
        panel_copy_x<TT, TX>(X + a.x.voff[sg.bx], t0, wd, ni, sg.nl, r0, th, lane, b);
#pragma unroll
        for (int j = 0; j < P; ++j)
          if (sg.by[j] >= 0)
            panel_copy_y<TT, TY>(Y + a.y.voff[sg.by[j]], t0, wd, njv[j], sg.nl, c0v[j], twv[j], lane,
                                 b + (1 + j) * TT * TT);
        cp_commit();
      };
      int m = 0, t0 = 0, buf = 0;
      issue(0, 0, wbase);
      for (;;) {
        const PStage cur = st[m];
        const bool last_slice = t0 + TT >= (int)cur.nl;
        const int m2 = last_slice ? m + 1 : m, t2 = last_slice ? 0 : t0 + TT;
        const bool more = m2 < nm;
        if (more) {
          issue(m2, t2, wbase + (buf ^ 1) * BUF);
          cp_wait<1>();
        } else {
          cp_wait<0>();
        }
        __syncwarp();
        const int tk = min(TT, (int)cur.nl - t0);
        if (active) {
          const float* xs = wbase + buf * BUF;
          for (int tt = 0; tt < tk; ++tt) {
            float ar[MR];
            lds<MR>(xs + tt * TT + rl, ar);
#pragma unroll
            for (int j = 0; j < P; ++j) {
              if (cur.by[j] >= 0) {
                float br[MC];
                lds<MC>(xs + (1 + j) * TT * TT + tt * TT + cl, br);
#pragma unroll
                for (int ii = 0; ii < MR; ++ii)
#pragma unroll
                  for (int jj = 0; jj < MC; ++jj) p[j][ii * MC + jj] = fmaf(ar[ii], br[jj], p[j][ii * MC + jj]);
              }
            }
          }
        }
        __syncwarp();
        if (last_slice && ++folded == kFold) {
          folded = 0;
#pragma unroll
          for (int j = 0; j < P; ++j)
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
              const float hi = acc[j][q] + p[j][q];
              const float bp = hi - acc[j][q];
              comp[j][q] += (acc[j][q] - (hi - bp)) + (p[j][q] - bp);
              acc[j][q] = hi;
              p[j][q] = 0.0f;
            }
        }
        if (!more) break;
        m = m2;
        t0 = t2;
        buf ^= 1;
      }
    }
    if (active) {
#pragma unroll
      for (int j = 0; j < P; ++j) {
        if (j < cnt) {
          float* cb = C + a.c_voff[kj[j]];
#pragma unroll
          for (int ii = 0; ii < MR; ++ii)
#pragma unroll
            for (int jj = 0; jj < MC; ++jj) {
              const int q = ii * MC + jj;
              const float hi = acc[j][q] + p[j][q];
              const float bp = hi - acc[j][q];
              const float err = (acc[j][q] - (hi - bp)) + (p[j][q] - bp);
              const int r = rl + ii, c = cl + jj;
              if (r < th && c < twv[j]) cb[(int64_t)(r0 + r) * njv[j] + c0v[j] + c] = hi + (comp[j][q] + err);
            }
        }
      }
    }
  }
}

// Panel list of S_C for tile edge `edge` and at most `P` tiles per panel: for every block
// row nu and row offset r0, the column tiles of the row's blocks in column order, cut into
// runs of P.
static s_status build_panels(MulDesc* d, int edge, int P) {
  const s_pattern_t* C = d->pc;
  cudaFree(d->ptiles);
  cudaFree(d->pidx);
  d->ptiles = nullptr;
  d->pidx = nullptr;
  d->npanels = 0;
  std::vector<Tile> tl;
  std::vector<int2> idx;
  for (int32_t nu = 0; nu < C->d.nc; ++nu) {
    const int ni = C->bsize[nu];
    for (int r0 = 0; r0 < ni; r0 += edge) {
      int run = 0;
      for (int64_t k = C->rowptr[nu]; k < C->rowptr[nu + 1]; ++k) {
        const int nj = C->bsize[C->colidx[k]];
        for (int c0 = 0; c0 < nj; c0 += edge) {
          if (run == 0) idx.push_back(make_int2((int)tl.size(), 0));
          tl.push_back(Tile{(int32_t)k, (int16_t)r0, (int16_t)c0});
          idx.back().y++;
          if (++run == P) run = 0;
        }
      }
    }
  }
  cudaError_t e = cudaMalloc(&d->ptiles, sizeof(Tile) * std::max<size_t>(tl.size(), 1));
  if (e == cudaSuccess) e = cudaMalloc(&d->pidx, sizeof(int2) * std::max<size_t>(idx.size(), 1));
  if (e == cudaSuccess && !tl.empty())
    e = cudaMemcpy(d->ptiles, tl.data(), sizeof(Tile) * tl.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !idx.empty())
    e = cudaMemcpy(d->pidx, idx.data(), sizeof(int2) * idx.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_error(e, "build_panels");
  d->npanels = (int64_t)idx.size();
  d->panel_edge = edge;
  d->panel_size = P;
  return S_OK;
}

// The float kernel variants the autotuner chooses from: tile edge and lane micro-tile.
struct F32Variant {
  int tt, mr, mc, km;  // tile edge, lane micro-tile, largest lambda extent of one stage
  int panel;           // 0: one tile per warp; P > 0: row panels of up to P tiles per warp
  int nt;              // K-major kernel with bulk-copy staging (mul_nt.cu), micro-tile per tile:
                       // 1 = runtime row pitch, 2 = compile-time pitch for full 20-wide pieces
};
constexpr F32Variant kF32Variants[] = {{20, 0, 0, 20, 0, 1},  {20, 0, 0, 20, 0, 2},  {20, 4, 4, 20, 0, 0},
                                       {20, 4, 4, 40, 0, 0},  {16, 4, 2, 32, 0, 0},  {12, 3, 2, 36, 0, 0},
                                       {10, 2, 2, 40, 0, 0},  {8, 2, 1, 32, 0, 0},   {12, 3, 2, 12, 3, 0},
                                       {10, 2, 2, 10, 4, 0},  {8, 2, 1, 8, 4, 0}};
constexpr int kNumF32Variants = 11;
constexpr int kF32Fallback = 2;  // tile kernel of the K-major variants' tile list, for unaligned buffers

static int num_sms() { return sm_count(); }

// Tile edges of the double product's variants; plans of narrow blocks start with the 10-wide one.
constexpr int kF64Edges[] = {20, 10};
constexpr int kNumF64Variants = 2;
static int f64_default_variant(const s_pattern_t* C) {
  const double rms = std::sqrt((double)C->d.nnz / (double)std::max<int64_t>(C->d.nblocks, 1));
  return rms <= 12.0 ? 1 : 0;
}

static Side side_of(const s_pattern_t* p, bool row_side, bool trans) {
  // row_side: the list indexed by the output row (X side); otherwise by the output column.
  const DevPattern& d = p->d;
  bool use_csr = row_side ? !trans : trans;
  if (use_csr) return Side{d.rowptr, d.colidx, nullptr, d.voff, trans};
  return Side{d.colptr, d.rowidx, d.cscblk, d.voff, trans};
}

// Tile list of S_C for tile edge `edge`, in block order: breadth-first block rows are
// spatially coherent, so warps that run at the same time share lambda blocks in L2, and
// the coarse (heavy) rows come first.
s_status build_tiles(MulDesc* d, int edge) {
  const s_pattern_t* C = d->pc;
  const int64_t nb = C->d.nblocks;
  cudaFree(d->tiles);
  d->tiles = nullptr;
  d->ntiles = 0;
  d->edge = edge;
  if (nb == 0) {
    SF_CUDA(cudaMalloc(&d->tiles, sizeof(Tile)));
    return S_OK;
  }
  int32_t* ntile = nullptr;
  int64_t* first = nullptr;
  cudaError_t e = cudaMalloc(&ntile, sizeof(int32_t) * nb);
  if (e == cudaSuccess) e = cudaMalloc(&first, sizeof(int64_t) * (nb + 1));
  if (e == cudaSuccess) {
    const int g = (int)((nb + 255) / 256);
    tile_count_kernel<<<g, 256>>>(C->d.bsize, C->d.brow, C->d.colidx, nb, edge, ntile);
    e = cudaGetLastError();
    std::vector<int32_t> nt(nb);
    std::vector<int64_t> fst(nb + 1, 0);
    if (e == cudaSuccess) e = cudaMemcpy(nt.data(), ntile, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) {
      for (int64_t k = 0; k < nb; ++k) fst[k + 1] = fst[k] + nt[k];
      d->ntiles = fst[nb];
      e = cudaMemcpy(first, fst.data(), sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMalloc(&d->tiles, sizeof(Tile) * std::max<int64_t>(d->ntiles, 1));
    if (e == cudaSuccess) {
      tile_fill_kernel<<<g, 256>>>(first, C->d.bsize, C->d.brow, C->d.colidx, nb, edge, d->tiles);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  cudaFree(ntile);
  cudaFree(first);
  if (e != cudaSuccess) return cuda_error(e, "build_tiles");
  return S_OK;
}

s_status build_desc(const s_pattern_t* X, bool tx, const s_pattern_t* Y, bool ty, const s_pattern_t* C, s_prec prec,
                    MulDesc* out) {
  (void)prec;
  MulDesc d;
  d.x = side_of(X, true, tx);
  d.y = side_of(Y, false, ty);
  d.pc = C;
  d.px = X;
  d.py = Y;
  const int64_t nb = C->d.nblocks;
  unsigned long long* dtrip = nullptr;
  double* bflops = nullptr;
  s_status st = S_OK;
  cudaError_t e = cudaMalloc(&dtrip, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(dtrip, 0, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&bflops, sizeof(double) * std::max<int64_t>(nb, 1));
  if (e == cudaSuccess) e = cudaMalloc(&d.counter, sizeof(unsigned int));
  if (e == cudaSuccess && nb > 0) {
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((nb * 32 + threads - 1) / threads, (int64_t)num_sms() * 16);
    count_kernel<<<blocks, threads>>>(dev_side(d.x), dev_side(d.y), C->d.bsize, C->d.brow, C->d.colidx, nb, dtrip,
                                      bflops);
    e = cudaGetLastError();
    unsigned long long tr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&tr, dtrip, sizeof(tr), cudaMemcpyDeviceToHost);
    std::vector<double> bf(nb);
    if (e == cudaSuccess) e = cudaMemcpy(bf.data(), bflops, sizeof(double) * nb, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) {
      d.triples = (int64_t)tr;
      double f = 0.0;
      for (double v : bf) f += v;
      d.flops = f;
    }
  }
  cudaFree(dtrip);
  cudaFree(bflops);
  if (e == cudaSuccess) {
    // the time-out word lives in pinned host memory mapped into the device: a kernel's store
    // reaches the host without a copy, and the next call on the plan reads it without a sync
    e = cudaHostAlloc((void**)&d.err_host, sizeof(unsigned int), cudaHostAllocMapped);
    if (e == cudaSuccess) {
      *(volatile unsigned int*)d.err_host = 0u;
      e = cudaHostGetDevicePointer((void**)&d.err, d.err_host, 0);
    }
  }
  if (e != cudaSuccess) st = cuda_error(e, "s_plan_create(symbolic)");
  if (!st && prec == S_FP64) {
    d.variant = f64_default_variant(C);
    st = build_tiles(&d, kF64Edges[d.variant]);
  } else if (!st) {
    st = build_tiles(&d, kF32Variants[0].tt);
  }
  if (!st && prec == S_BF16X3) {
    // three bfloat16 planes per operand; every block size must be even (4-byte copies)
    for (const s_pattern_t* q : {X, Y, C})
      for (int32_t b : q->bsize)
        if (b & 1) st = set_error(S_ERR_ARG, "S_BF16X3 needs even block sizes");
    if (!st) {
      e = cudaMalloc(&d.bf_x, sizeof(__nv_bfloat16) * 3 * std::max<int64_t>(X->d.nnz, 1));
      if (e == cudaSuccess) e = cudaMalloc(&d.bf_y, sizeof(__nv_bfloat16) * 3 * std::max<int64_t>(Y->d.nnz, 1));
      if (e != cudaSuccess) st = cuda_error(e, "cudaMalloc(split-bfloat16 scratch)");
    }
  }
  if (!st && prec == S_TF32X3) st = tc_prepare(&d);
  if (!st && prec == S_FP32) st = nt_configure(&d, tx, ty, false);
  if (!st && prec == S_FP64_DF) {
    // split operands (float pairs), reused by every call of this plan
    e = cudaMalloc(&d.df_x, sizeof(float2) * std::max<int64_t>(X->d.nnz, 1));
    if (e == cudaSuccess) e = cudaMalloc(&d.df_y, sizeof(float2) * std::max<int64_t>(Y->d.nnz, 1));
    if (e != cudaSuccess) st = cuda_error(e, "cudaMalloc(double-float scratch)");
  }
  if (st) {
    free_desc(&d);
    return st;
  }
  *out = d;
  return S_OK;
}

void free_desc(MulDesc* d) {
  tc_free(d);
  nt_free_side(&d->ntx);
  nt_free_side(&d->nty);
  if (d->err_host) cudaFreeHost(d->err_host);
  d->err_host = nullptr;
  d->err = nullptr;
  cudaFree(d->ptiles);
  cudaFree(d->pidx);
  d->ptiles = nullptr;
  d->pidx = nullptr;
  d->npanels = 0;
  cudaFree(d->tiles);
  cudaFree(d->counter);
  cudaFree(d->df_x);
  cudaFree(d->df_y);
  d->df_x = d->df_y = nullptr;
  cudaFree(d->bf_x);
  cudaFree(d->bf_y);
  d->bf_x = d->bf_y = nullptr;
  d->tiles = nullptr;
  d->counter = nullptr;
  d->ntiles = 0;
}

using F32Kernel = void (*)(MulArgs, const float*, const float*, float*);

template <int V>
static F32Kernel f32_kernel(bool tx, bool ty) {
  static_assert(kF32Variants[V].nt == 0 && kF32Variants[V].panel == 0, "tile variant expected");
  constexpr int TT = kF32Variants[V].tt, MR = kF32Variants[V].mr, MC = kF32Variants[V].mc, KM = kF32Variants[V].km;
  return tx ? (ty ? mul_f32_kernel<TT, MR, MC, KM, true, true> : mul_f32_kernel<TT, MR, MC, KM, true, false>)
            : (ty ? mul_f32_kernel<TT, MR, MC, KM, false, true> : mul_f32_kernel<TT, MR, MC, KM, false, false>);
}

using F32PanelKernel = void (*)(MulArgs, PanelArgs, const float*, const float*, float*);
template <int V>
static F32PanelKernel f32_panel_kernel(bool tx, bool ty) {
  constexpr int TT = kF32Variants[V].tt, MR = kF32Variants[V].mr, MC = kF32Variants[V].mc,
                P = kF32Variants[V].panel;
  return tx ? (ty ? mul_f32_panel_kernel<TT, MR, MC, P, true, true> : mul_f32_panel_kernel<TT, MR, MC, P, true, false>)
            : (ty ? mul_f32_panel_kernel<TT, MR, MC, P, false, true>
                  : mul_f32_panel_kernel<TT, MR, MC, P, false, false>);
}

static F32Kernel f32_kernel_of(int v, bool tx, bool ty) {
  switch (v) {
    case 3: return f32_kernel<3>(tx, ty);
    case 4: return f32_kernel<4>(tx, ty);
    case 5: return f32_kernel<5>(tx, ty);
    case 6: return f32_kernel<6>(tx, ty);
    case 7: return f32_kernel<7>(tx, ty);
    default: return f32_kernel<2>(tx, ty);
  }
}

static size_t f32_smem(int v) {
  const F32Variant& f = kF32Variants[v];
  if (f.panel) return sizeof(float) * kF32Warps * 2 * (1 + f.panel) * f.tt * f.tt;
  return sizeof(float) * kF32Warps * 4 * f.km * f.tt;
}

static s_status launch_f32_panel(const MulDesc& d, const void* X, const void* Y, void* C, cudaStream_t st) {
  const F32Variant& f = kF32Variants[d.variant];
  if (d.panel_edge != f.tt || d.panel_size != f.panel || !d.pidx)
    return set_error(S_ERR_ARG, "internal: panel list does not match variant");
  if (d.npanels == 0) return S_OK;
  MulArgs a;
  a.x = dev_side(d.x);
  a.y = dev_side(d.y);
  a.bsize = d.pc->d.bsize;
  a.c_brow = d.pc->d.brow;
  a.c_col = d.pc->d.colidx;
  a.c_voff = d.pc->d.voff;
  a.tiles = d.tiles;
  a.ntiles = d.ntiles;
  a.counter = d.counter;
  SF_CUDA(cudaMemsetAsync(d.counter, 0, sizeof(unsigned int), st));
  F32PanelKernel kern = d.variant == 8   ? f32_panel_kernel<8>(d.x.trans, d.y.trans)
                        : d.variant == 9 ? f32_panel_kernel<9>(d.x.trans, d.y.trans)
                                         : f32_panel_kernel<10>(d.x.trans, d.y.trans);
  const size_t smem = f32_smem(d.variant);
  SF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  SF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kF32Warps * 32, smem));
  if (per_sm < 1) per_sm = 1;
  const int64_t want = (d.npanels + kF32Warps - 1) / kF32Warps;
  const int grid = (int)std::min<int64_t>(want, (int64_t)num_sms() * per_sm);
  kern<<<grid, kF32Warps * 32, smem, st>>>(a, PanelArgs{d.ptiles, d.pidx, d.npanels}, (const float*)X,
                                           (const float*)Y, (float*)C);
  SF_CUDA(cudaGetLastError());
  return S_OK;
}

template <typename T>
static s_status launch_typed(const MulDesc& d, const void* X, const void* Y, void* C, cudaStream_t st) {
  MulArgs a;
  a.x = dev_side(d.x);
  a.y = dev_side(d.y);
  a.bsize = d.pc->d.bsize;
  a.c_brow = d.pc->d.brow;
  a.c_col = d.pc->d.colidx;
  a.c_voff = d.pc->d.voff;
  a.tiles = d.tiles;
  a.ntiles = d.ntiles;
  a.counter = d.counter;
  if (d.ntiles == 0) return S_OK;
  SF_CUDA(cudaMemsetAsync(d.counter, 0, sizeof(unsigned int), st));
  int per_sm = 0;
  using K = void (*)(MulArgs, const T*, const T*, T*);
  K kern;
  int warps;
  size_t dsmem = 0;
  if constexpr (sizeof(T) == 4) {
    if (kF32Variants[d.variant].panel) return launch_f32_panel(d, X, Y, C, st);
    if (d.edge != kF32Variants[d.variant].tt) return set_error(S_ERR_ARG, "internal: tile list does not match variant");
    int v = d.variant;
    if (kF32Variants[v].nt) {
      if (nt_usable(d, X, Y)) return launch_nt(d, X, Y, C, st, kF32Variants[v].nt == 2);
      v = kF32Fallback;  // same tile list (edge 20); reads any alignment
    }
    kern = f32_kernel_of(v, d.x.trans, d.y.trans);
    warps = kF32Warps;
    dsmem = f32_smem(v);
    SF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsmem));
  } else {
    const int tt = kF64Edges[d.variant < kNumF64Variants ? d.variant : 0];
    if (d.edge != tt) return set_error(S_ERR_ARG, "internal: tile list does not match the double variant");
    if (tt == 10)
      kern = d.x.trans ? (d.y.trans ? mul_kernel<T, 10, true, true> : mul_kernel<T, 10, true, false>)
                       : (d.y.trans ? mul_kernel<T, 10, false, true> : mul_kernel<T, 10, false, false>);
    else
      kern = d.x.trans ? (d.y.trans ? mul_kernel<T, 20, true, true> : mul_kernel<T, 20, true, false>)
                       : (d.y.trans ? mul_kernel<T, 20, false, true> : mul_kernel<T, 20, false, false>);
    warps = kWarps;
  }
  SF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, dsmem));
  if (per_sm < 1) per_sm = 1;
  int64_t want = (d.ntiles + warps - 1) / warps;
  int grid = (int)std::min<int64_t>(want, (int64_t)num_sms() * per_sm);
  kern<<<grid, warps * 32, dsmem, st>>>(a, (const T*)X, (const T*)Y, (T*)C);
  SF_CUDA(cudaGetLastError());
  return S_OK;
}

static s_status launch_df(const MulDesc& d, const void* X, const void* Y, void* C, cudaStream_t st) {
  if (d.ntiles == 0) return S_OK;
  if (!d.df_x || !d.df_y) return set_error(S_ERR_ARG, "internal: double-float scratch missing");
  const int64_t nx = d.px->d.nnz, ny = d.py->d.nnz;
  const int gx = (int)std::max<int64_t>(1, std::min<int64_t>((nx + 255) / 256, (int64_t)num_sms() * 16));
  const int gy = (int)std::max<int64_t>(1, std::min<int64_t>((ny + 255) / 256, (int64_t)num_sms() * 16));
  if (nx) split_kernel<<<gx, 256, 0, st>>>(nx, (const double*)X, d.df_x);
  const float2* ysplit = d.df_x;
  if (Y != X || d.px != d.py) {
    if (ny) split_kernel<<<gy, 256, 0, st>>>(ny, (const double*)Y, d.df_y);
    ysplit = d.df_y;
  }
  MulArgs a;
  a.x = dev_side(d.x);
  a.y = dev_side(d.y);
  a.bsize = d.pc->d.bsize;
  a.c_brow = d.pc->d.brow;
  a.c_col = d.pc->d.colidx;
  a.c_voff = d.pc->d.voff;
  a.tiles = d.tiles;
  a.ntiles = d.ntiles;
  a.counter = d.counter;
  SF_CUDA(cudaMemsetAsync(d.counter, 0, sizeof(unsigned int), st));
  using K = void (*)(MulArgs, const float2*, const float2*, double*);
  const int v = d.variant < kNumDfVariants ? d.variant : 0;
  if (d.edge != kDfVariants[v].tt) return set_error(S_ERR_ARG, "internal: tile list does not match variant");
  K kern;
  if (v == 1)
    kern = d.x.trans ? (d.y.trans ? mul_df_kernel<10, 2, 2, true, true> : mul_df_kernel<10, 2, 2, true, false>)
                     : (d.y.trans ? mul_df_kernel<10, 2, 2, false, true> : mul_df_kernel<10, 2, 2, false, false>);
  else
    kern = d.x.trans ? (d.y.trans ? mul_df_kernel<20, 4, 4, true, true> : mul_df_kernel<20, 4, 4, true, false>)
                     : (d.y.trans ? mul_df_kernel<20, 4, 4, false, true> : mul_df_kernel<20, 4, 4, false, false>);
  const size_t smem = df_smem(v);
  SF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  SF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kDfWarps * 32, smem));
  if (per_sm < 1) per_sm = 1;
  const int64_t want = (d.ntiles + kDfWarps - 1) / kDfWarps;
  const int grid = (int)std::min<int64_t>(want, (int64_t)num_sms() * per_sm);
  kern<<<grid, kDfWarps * 32, smem, st>>>(a, d.df_x, ysplit, (double*)C);
  SF_CUDA(cudaGetLastError());
  return S_OK;
}

static s_status launch_bf16x3(const MulDesc& d, const void* X, const void* Y, void* C, cudaStream_t st) {
  if (d.ntiles == 0) return S_OK;
  if (d.edge != kTile) return set_error(S_ERR_ARG, "internal: split-bfloat16 kernel needs 20-wide tiles");
  if (!d.bf_x || !d.bf_y) return set_error(S_ERR_ARG, "internal: split-bfloat16 scratch missing");
  const int64_t nx = d.px->d.nnz, ny = d.py->d.nnz;
  const int gx = (int)std::max<int64_t>(1, std::min<int64_t>((nx + 255) / 256, (int64_t)num_sms() * 16));
  const int gy = (int)std::max<int64_t>(1, std::min<int64_t>((ny + 255) / 256, (int64_t)num_sms() * 16));
  if (nx) split3_kernel<<<gx, 256, 0, st>>>(nx, (const float*)X, d.bf_x, d.bf_x + nx, d.bf_x + 2 * nx);
  Planes px{{d.bf_x, d.bf_x + nx, d.bf_x + 2 * nx}};
  Planes py = px;
  if (Y != X || d.px != d.py) {
    if (ny) split3_kernel<<<gy, 256, 0, st>>>(ny, (const float*)Y, d.bf_y, d.bf_y + ny, d.bf_y + 2 * ny);
    py = Planes{{d.bf_y, d.bf_y + ny, d.bf_y + 2 * ny}};
  }
  MulArgs a;
  a.x = dev_side(d.x);
  a.y = dev_side(d.y);
  a.bsize = d.pc->d.bsize;
  a.c_brow = d.pc->d.brow;
  a.c_col = d.pc->d.colidx;
  a.c_voff = d.pc->d.voff;
  a.tiles = d.tiles;
  a.ntiles = d.ntiles;
  a.counter = d.counter;
  SF_CUDA(cudaMemsetAsync(d.counter, 0, sizeof(unsigned int), st));
  using K = void (*)(MulArgs, Planes, Planes, float*);
  K kern = d.x.trans ? (d.y.trans ? mul_bf16x3_kernel<true, true> : mul_bf16x3_kernel<true, false>)
                     : (d.y.trans ? mul_bf16x3_kernel<false, true> : mul_bf16x3_kernel<false, false>);
  SF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem));
  int per_sm = 0;
  SF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTcWarps * 32, kTcSmem));
  if (per_sm < 1) per_sm = 1;
  const int64_t want = (d.ntiles + kTcWarps - 1) / kTcWarps;
  const int grid = (int)std::min<int64_t>(want, (int64_t)num_sms() * per_sm);
  kern<<<grid, kTcWarps * 32, kTcSmem, st>>>(a, px, py, (float*)C);
  SF_CUDA(cudaGetLastError());
  return S_OK;
}

s_status take_timeout(const MulDesc& d) {
  volatile unsigned int* w = d.err_host;
  if (!w || *w == 0u) return S_OK;
  *w = 0u;
  return set_error(S_ERR_TIMEOUT,
                   "an earlier product of this plan gave up waiting on its own device-side copies or tensor-core "
                   "work; its outputs are unspecified (NaN where written after the time-out)");
}

s_status run_mul(const MulDesc& d, s_prec prec, const void* X, const void* Y, void* C, cudaStream_t st) {
  switch (prec) {
    case S_FP64:
      return launch_typed<double>(d, X, Y, C, st);
    case S_FP32:
      return launch_typed<float>(d, X, Y, C, st);
    case S_FP64_DF:
      return launch_df(d, X, Y, C, st);
    case S_BF16X3:
      return launch_bf16x3(d, X, Y, C, st);
    case S_TF32X3:
      return launch_tc(d, X, Y, C, st);
    default:
      return set_error(S_ERR_ARG, "precision not supported by this product path");
  }
}

static s_status check_same_tree(const s_pattern_t* a, const s_pattern_t* b) {
  if (a->tree_hash != b->tree_hash || a->d.nc != b->d.nc)
    return set_error(S_ERR_MISMATCH, "operands come from different cluster trees");
  return S_OK;
}

}  // namespace sf

using namespace sf;

extern "C" s_status s_plan_create(s_pattern A, s_pattern B, s_pattern C, s_prec prec, s_plan* out) {
  if (!out) return set_error(S_ERR_ARG, "s_plan_create: out is NULL");
  *out = nullptr;
  if (!A || !B || !C) return set_error(S_ERR_ARG, "s_plan_create: NULL pattern");
  if (prec != S_FP64 && prec != S_FP32 && prec != S_FP64_DF && prec != S_BF16X3 && prec != S_TF32X3)
    return set_error(S_ERR_ARG, "s_plan_create: unsupported precision");
  s_status st;
  if ((st = check_same_tree(A, B)) || (st = check_same_tree(A, C))) return st;
  s_plan_t* p = new (std::nothrow) s_plan_t();
  if (!p) return set_error(S_ERR_NOMEM, "host allocation");
  p->prec = prec;
  p->a = A;
  p->b = B;
  p->c = C;
  if ((st = build_desc(A, false, B, false, C, prec, &p->fwd))) {
    delete p;
    return st;
  }
  *out = p;
  return S_OK;
}

extern "C" s_status s_plan_destroy(s_plan p) {
  if (!p) return S_OK;
  free_desc(&p->fwd);
  if (p->adj_built) {
    free_desc(&p->adjA);
    free_desc(&p->adjB);
  }
  delete p;
  return S_OK;
}

extern "C" s_status s_plan_status(s_plan p, void* stream) {
  if (!p) return set_error(S_ERR_ARG, "s_plan_status: NULL plan");
  SF_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  s_status st = take_timeout(p->fwd);
  if (p->adj_built) {
    const s_status sa = take_timeout(p->adjA), sb = take_timeout(p->adjB);
    if (!st) st = sa ? sa : sb;
  }
  return st;
}

extern "C" s_status s_plan_timeout_word(s_plan p, unsigned int** word) {
  if (!p || !word) return set_error(S_ERR_ARG, "s_plan_timeout_word: NULL argument");
  *word = p->fwd.err_host;
  return S_OK;
}

extern "C" s_status s_plan_stats(s_plan p, int64_t* triples, double* flops) {
  if (!p) return set_error(S_ERR_ARG, "s_plan_stats: NULL plan");
  if (triples) *triples = p->fwd.triples;
  if (flops) *flops = p->fwd.flops;
  return S_OK;
}

extern "C" s_status s_mul_masked(s_plan p, const void* A, const void* B, void* C, void* stream) {
  if (!p || !A || !B || !C) return set_error(S_ERR_ARG, "s_mul_masked: NULL argument");
  if (C == A || C == B) return set_error(S_ERR_ARG, "s_mul_masked: C aliases an input");
  return run_mul(p->fwd, p->prec, A, B, C, (cudaStream_t)stream);
}

extern "C" s_status s_mul_masked_adjoint(s_plan p, const void* dC, const void* A, const void* B, void* dA, void* dB,
                                         void* stream) {
  if (!p || !dC) return set_error(S_ERR_ARG, "s_mul_masked_adjoint: NULL argument");
  if (!p->adj_built) {
    s_status st;
    // dA = P_{S_A}(dC B^T): X = dC on S_C (as is), Y = B transposed, output S_A
    if ((st = build_desc(p->c, false, p->b, true, p->a, p->prec, &p->adjA))) return st;
    // dB = P_{S_B}(A^T dC): X = A transposed, Y = dC as is, output S_B
    if ((st = build_desc(p->a, true, p->c, false, p->b, p->prec, &p->adjB))) {
      free_desc(&p->adjA);
      return st;
    }
    p->adj_built = true;
  }
  s_status st = S_OK;
  if (dA) {
    if (!B) return set_error(S_ERR_ARG, "s_mul_masked_adjoint: dA needs B");
    if ((st = run_mul(p->adjA, p->prec, dC, B, dA, (cudaStream_t)stream))) return st;
  }
  if (dB) {
    if (!A) return set_error(S_ERR_ARG, "s_mul_masked_adjoint: dB needs A");
    if ((st = run_mul(p->adjB, p->prec, A, dC, dB, (cudaStream_t)stream))) return st;
  }
  return S_OK;
}

extern "C" s_status s_plan_autotune(s_plan p, const void* A, const void* B, void* C, void* stream, int* chosen) {
  if (!p || !A || !B || !C) return set_error(S_ERR_ARG, "s_plan_autotune: NULL argument");
  if (p->prec != S_FP32 && p->prec != S_FP64_DF && p->prec != S_FP64) {
    if (chosen) *chosen = 0;
    return S_OK;  // one kernel shape for the split tensor-core paths
  }
  const bool df = p->prec == S_FP64_DF, f64 = p->prec == S_FP64;
  const int nvar = df ? kNumDfVariants : (f64 ? kNumF64Variants : kNumF32Variants);
  auto edge_of = [&](int v) { return df ? kDfVariants[v].tt : (f64 ? kF64Edges[v] : kF32Variants[v].tt); };
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  SF_CUDA(cudaEventCreate(&e0));
  SF_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int bestv = 0;
  s_status s = S_OK;
  // Row panels pay off only when most blocks of S_C are at most one tile wide: skip them
  // when the root-mean-square block edge of S_C exceeds the panel's tile edge.
  const s_pattern_t* pc = p->fwd.pc;
  const double rms_edge = std::sqrt((double)pc->d.nnz / (double)std::max<int64_t>(pc->d.nblocks, 1));
  for (int v = 0; v < nvar && !s; ++v) {
    const bool fl = !df && !f64;
    const bool panel = fl && kF32Variants[v].panel;
    if (panel && rms_edge > kF32Variants[v].tt) continue;
    // tile shapes narrower than 20 only where the blocks are no wider than their tiles
    if (fl && !panel && !kF32Variants[v].nt && kF32Variants[v].tt < 20 && rms_edge > kF32Variants[v].tt) continue;
    if (f64 && kF64Edges[v] < 20 && rms_edge > 12.0) continue;
    if ((s = build_tiles(&p->fwd, edge_of(v)))) break;
    if (panel && (s = build_panels(&p->fwd, kF32Variants[v].tt, kF32Variants[v].panel))) break;
    p->fwd.variant = v;
    // warm-up launch, timed: a shape more than twice as slow as the best so far is not timed again
    cudaEventRecord(e0, st);
    if ((s = run_mul(p->fwd, p->prec, A, B, C, st))) break;
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      s = cuda_error(e, "s_plan_autotune");
      break;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms > 2.0f * best / 3.0f) {
      p->tune_ms[v] = ms;
      continue;
    }
    cudaEventRecord(e0, st);
    for (int r = 0; r < 3 && !s; ++r) s = run_mul(p->fwd, p->prec, A, B, C, st);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      s = cuda_error(e, "s_plan_autotune");
      break;
    }
    cudaEventElapsedTime(&ms, e0, e1);
    p->tune_ms[v] = ms / 3.0f;
    if (ms < best) {
      best = ms;
      bestv = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s) return s;
  if ((s = build_tiles(&p->fwd, edge_of(bestv)))) return s;
  if (!df && !f64 && kF32Variants[bestv].panel &&
      (s = build_panels(&p->fwd, kF32Variants[bestv].tt, kF32Variants[bestv].panel)))
    return s;
  p->fwd.variant = bestv;
  if (chosen) *chosen = bestv;
  return S_OK;
}

extern "C" s_status s_plan_variant(s_plan p, int variant, int* tile, int* micro_rows, int* micro_cols,
                                   int* stage_k) {
  if (!p) return set_error(S_ERR_ARG, "s_plan_variant: NULL plan");
  if (variant < 0) variant = p->fwd.variant;
  if (p->prec == S_FP64_DF) {
    if (variant >= kNumDfVariants) return set_error(S_ERR_ARG, "s_plan_variant: no such variant");
    if (tile) *tile = kDfVariants[variant].tt;
    if (micro_rows) *micro_rows = kDfVariants[variant].mr;
    if (micro_cols) *micro_cols = kDfVariants[variant].mc;
    if (stage_k) *stage_k = kDfVariants[variant].tt;
    return S_OK;
  }
  if (p->prec == S_FP64) {
    if (variant >= kNumF64Variants) return set_error(S_ERR_ARG, "s_plan_variant: no such variant");
    if (tile) *tile = kF64Edges[variant];
    if (micro_rows) *micro_rows = 1;
    if (micro_cols) *micro_cols = 1;
    if (stage_k) *stage_k = kF64Edges[variant];
    return S_OK;
  }
  if (p->prec == S_TF32X3) {
    if (tile) *tile = kTcN;
    if (micro_rows) *micro_rows = kTcM;
    if (micro_cols) *micro_cols = kTcN;
    if (stage_k) *stage_k = kTcKC;
    return S_OK;
  }
  if (variant >= kNumF32Variants) return set_error(S_ERR_ARG, "s_plan_variant: no such variant");
  if (tile) *tile = kF32Variants[variant].tt;  // K-major variant: micro-tile 0 x 0 = per tile
  if (micro_rows) *micro_rows = kF32Variants[variant].mr;
  if (micro_cols) *micro_cols = kF32Variants[variant].mc;
  if (stage_k) *stage_k = kF32Variants[variant].km;
  return S_OK;
}

extern "C" s_status s_plan_set_variant(s_plan p, int variant) {
  if (!p) return set_error(S_ERR_ARG, "s_plan_set_variant: NULL plan");
  if (p->prec != S_FP32 && p->prec != S_FP64_DF && p->prec != S_FP64)
    return set_error(S_ERR_ARG, "s_plan_set_variant: only double, float and double-float plans have variants");
  const bool df = p->prec == S_FP64_DF, f64 = p->prec == S_FP64;
  if (variant < 0 || variant >= (df ? kNumDfVariants : (f64 ? kNumF64Variants : kNumF32Variants)))
    return set_error(S_ERR_ARG, "s_plan_set_variant: no such variant");
  s_status s = build_tiles(&p->fwd, df ? kDfVariants[variant].tt
                                       : (f64 ? kF64Edges[variant] : kF32Variants[variant].tt));
  if (!s && !df && !f64 && kF32Variants[variant].panel)
    s = build_panels(&p->fwd, kF32Variants[variant].tt, kF32Variants[variant].panel);
  if (s) return s;
  p->fwd.variant = variant;
  return S_OK;
}

extern "C" int s_plan_num_variants(void) { return kNumF32Variants; }
extern "C" int s_plan_num_variants_of(s_plan p) {
  if (!p) return 0;
  return p->prec == S_FP32     ? kNumF32Variants
         : p->prec == S_FP64_DF ? kNumDfVariants
         : p->prec == S_FP64    ? kNumF64Variants
                                : 1;
}

extern "C" s_status s_plan_set_symmetric_a(s_plan p, int symmetric) {
  if (!p) return set_error(S_ERR_ARG, "s_plan_set_symmetric_a: NULL plan");
  const s_pattern_t* A = p->a;
  if (symmetric) {
    // the pattern must be symmetric: CSR and CSC index lists coincide
    if (A->rowptr.size() < 2) return S_OK;
    std::vector<int64_t> cnt(A->d.nc + 1, 0);
    for (int32_t c : A->colidx) cnt[c + 1]++;
    for (int32_t i = 0; i < A->d.nc; ++i)
      if (cnt[i + 1] != A->rowptr[i + 1] - A->rowptr[i])
        return set_error(S_ERR_PATTERN, "s_plan_set_symmetric_a: the pattern of A is not symmetric");
    for (int32_t i = 0; i < A->d.nc; ++i)
      for (int64_t k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k) {
        const int32_t j = A->colidx[k];
        auto b = A->colidx.begin() + A->rowptr[j], e = A->colidx.begin() + A->rowptr[j + 1];
        if (!std::binary_search(b, e, i))
          return set_error(S_ERR_PATTERN, "s_plan_set_symmetric_a: the pattern of A is not symmetric");
      }
  }
  if (p->prec == S_TF32X3) {
    // the tensor-core kernel wants op(B)(lambda, nu') column by column along lambda's index:
    // with B = A symmetric that is the stored block (nu', lambda), read through B's rows
    if (symmetric && p->b != p->a)
      return set_error(S_ERR_ARG, "s_plan_set_symmetric_a: an S_TF32X3 plan needs B's pattern to be A's");
    p->fwd.y = side_of(p->b, false, symmetric != 0);
    p->fwd.tc_sym = symmetric != 0;
    return tc_prepare(&p->fwd);
  }
  // read A(nu, lambda) as the transpose of the stored block (lambda, nu): same values when A
  // is symmetric, and column-contiguous staging for the float kernel
  p->fwd.x = side_of(A, true, symmetric != 0);
  // the K-major float kernel reads A as stored and, for B = A, B(lambda, nu') through A's rows
  if (p->prec == S_FP32) return nt_configure(&p->fwd, false, false, symmetric != 0 && p->b == p->a);
  return S_OK;
}
