// Float masked product C = P_{S_C}(op(X) op(Y)) (Eq. (product), Sec. 4.1) with both operands
// staged K-major: every lambda block reaches shared memory as one contiguous bulk copy.
//
// Operand layout ("K-major"): for the X side the slice op(X)(nu, lambda) is held as
// [row of nu][t], for the Y side op(Y)(lambda, nu') as [column of nu'][t], t running over
// lambda's samplets, both padded with zeros to multiples of 4 in each dimension.  Where a
// value buffer already stores its blocks that way (op(X) = X, op(Y) = Y^T, or op(Y) = B with
// B = A declared symmetric, all block sizes multiples of 4) the kernel reads it directly;
// otherwise a pre-pass writes a padded, per-block transposed copy into plan-owned scratch.
// Either way the rows r0 .. r0+th of a slice are one contiguous run of memory, so one
// cp.async.bulk copy, issued by one lane and tracked by an mbarrier, stages it.
//
// Work decomposition: one warp owns one output tile (at most 20 x 20 entries of one block of
// S_C) for the whole lambda sum.  The tile, padded to 4 MR x 4 MC, is cut into a 4 x 4 grid
// of MR x MC micro-tiles; each half-warp (16 lanes) holds the whole grid, and the two halves
// take alternate lambda blocks of the tile's intersection list (split-K), so all 32 lanes
// work whatever the block widths.  A lane's step over 4 values of t is MR + MC 16-byte
// shared loads and 4 MR MC fused multiply-adds.  Each lambda block's partial sum is kept in
// a float register per entry and folded into the running sum with an error-free two-sum
// every kNtFold blocks, the rounding error carried in the partial; at the end the two
// halves' sums are combined the same way.  The summation order is fixed (deterministic).
//
// Pipeline per warp: two stage buffers, each holding one lambda chunk (at most kNtKC values of
// t) per half-warp; the copies of the next stage are in flight while the current one is
// multiplied.  Waits on the mbarriers are bounded (about one second of SM clocks); on time-out
// the plan's time-out word is set and the warp stops.
#include <algorithm>
#include <cstring>

#include "common.cuh"

namespace sf {
namespace {

constexpr int kNtWarps = 4;
constexpr int kNtKC = 20;                        // lambda values per staged chunk
constexpr int kNtEnt = 32;                       // matching lambda blocks listed at once
constexpr int kNtRegion = 20 * kNtKC;            // floats of one operand slice (<= 20 rows)
constexpr int kNtHalf = 2 * kNtRegion + 16;      // X | Y of one half-warp, + 64-byte bank shift
constexpr int kNtBuf = 2 * kNtHalf;              // one stage buffer: both halves
constexpr int kNtFold = 4;                       // lambda blocks per two-sum fold
constexpr size_t kNtSmem = sizeof(float) * kNtWarps * 2 * kNtBuf;

struct NtEntry {
  int64_t xo, yo;  // float offsets of the X and Y slices (rows r0.. / columns c0..)
  int32_t nlp;     // padded lambda extent (row pitch of both slices)
  int32_t pad;
};

struct NtArgs {
  const int64_t* xptr;  // op(X) row lists: lambda ids xidx, block ids xblk (nullptr: position)
  const int32_t* xidx;
  const int32_t* xblk;
  const int64_t* xoff;  // float offset of each block in X's K-major buffer
  const float* X;
  const int64_t* yptr;  // op(Y) column lists
  const int32_t* yidx;
  const int32_t* yblk;
  const int64_t* yoff;
  const float* Y;
  const int32_t* bsize;
  const int32_t* c_brow;
  const int32_t* c_col;
  const int64_t* c_voff;
  const Tile* tiles;
  int64_t ntiles;
  unsigned int* counter;
  unsigned int* err;
  float* C;
};

__device__ __forceinline__ uint32_t nt_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ int nt_lower_bound(const int32_t* a, int lo, int hi, int32_t v) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(a + mid) < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ void nt_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(nt_smem(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void nt_bulk(float* dst, const float* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          nt_smem(dst)),
      "l"(src), "r"(bytes), "r"(nt_smem(bar))
      : "memory");
}

// Wait for phase `parity` of an mbarrier for at most about one second of SM clocks; returns
// false on time-out.
__device__ __forceinline__ bool nt_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t addr = nt_smem(bar);
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > (1ll << 31)) return false;
  }
}

// One staged piece of a lambda block: slice starts in the K-major X and Y buffers, the
// block's padded extent (global row pitch), this piece's t0 and extent, and whether it ends
// the block (last = -1: no piece).  All lanes hold the same values.
struct NtChunk {
  int64_t xo, yo;
  int nlp, t0, kc, last;
};

// Producer of a tile's pieces in increasing lambda order: lists matching lambda blocks
// kNtEnt at a time (ballot over 32 entries of op(X)'s row list, binary search in op(Y)'s
// column list) into the warp's entry table, then cuts each block into pieces of at most
// kNtKC values of t.
struct NtLister {
  const NtArgs* a;
  NtEntry* ent;
  int px, px1, py0, py1;
  int r0, c0;
  int nm, e, t0;

  __device__ __forceinline__ void refill(int lane) {
    __syncwarp();
    nm = 0;
    e = 0;
    while (nm == 0 && px < px1 && py0 < py1) {
      while (px < px1 && py0 < py1 && nm <= kNtEnt - 32) {
        const int i = px + lane;
        const int32_t lam = i < px1 ? __ldg(a->xidx + i) : INT32_MAX;
        const int pos = nt_lower_bound(a->yidx, py0, py1, lam);
        const bool hit = i < px1 && pos < py1 && __ldg(a->yidx + pos) == lam;
        const unsigned int mask = __ballot_sync(0xffffffffu, hit);
        if (hit) {
          const int kx = a->xblk ? __ldg(a->xblk + i) : i;
          const int ky = a->yblk ? __ldg(a->yblk + pos) : pos;
          const int nlp = (__ldg(a->bsize + lam) + 3) & ~3;
          NtEntry en;
          en.xo = __ldg(a->xoff + kx) + (int64_t)r0 * nlp;
          en.yo = __ldg(a->yoff + ky) + (int64_t)c0 * nlp;
          en.nlp = nlp;
          en.pad = 0;
          ent[nm + __popc(mask & ((1u << lane) - 1u))] = en;
        }
        nm += __popc(mask);
        py0 = __shfl_sync(0xffffffffu, pos, 31);
        px += 32;
      }
    }
    __syncwarp();
  }

  __device__ __forceinline__ NtChunk next(int lane) {
    NtChunk c;
    if (e >= nm) refill(lane);
    if (e >= nm) {
      c.xo = c.yo = 0;
      c.nlp = c.t0 = c.kc = 0;
      c.last = -1;
      return c;
    }
    const NtEntry en = ent[e];
    c.xo = en.xo;
    c.yo = en.yo;
    c.nlp = en.nlp;
    c.t0 = t0;
    if (t0 == 0 && en.nlp <= kNtKC) {  // the common case: the whole block in one piece
      c.kc = en.nlp;
      c.last = 1;
      ++e;
      return c;
    }
    c.kc = min(kNtKC, en.nlp - t0);
    c.last = t0 + c.kc >= en.nlp ? 1 : 0;
    if (c.last) {
      ++e;
      t0 = 0;
    } else {
      t0 += c.kc;
    }
    return c;
  }
};

// Issue the copies of one stage (piece c0 for half-warp 0, c1 for half-warp 1) into `buf`,
// completing on `bar`.  A whole lambda block moves as one copy per operand (its rows r0.. /
// columns c0.. are contiguous); a piece of a wider block as one copy per row.
template <int TH, int TW>
__device__ __forceinline__ void nt_issue(const NtArgs& a, const NtChunk& c0, const NtChunk& c1, float* buf,
                                         uint64_t* bar, int lane) {
  const bool v0 = c0.last >= 0, v1 = c1.last >= 0;
  if ((!v0 || c0.kc == c0.nlp) && (!v1 || c1.kc == c1.nlp)) {
    // whole blocks: lane 2h + o copies operand o (X, Y) of half-warp h's piece
    if (lane == 0) nt_expect(bar, (uint32_t)((TH + TW) * 4 * ((v0 ? c0.kc : 0) + (v1 ? c1.kc : 0))));
    __syncwarp();
    if (lane < 4) {
      const int h = lane >> 1, o = lane & 1;
      const NtChunk& c = h ? c1 : c0;
      if (h ? v1 : v0) {
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        nt_bulk(buf + h * kNtHalf + o * kNtRegion, o ? a.Y + c.yo : a.X + c.xo, (uint32_t)((o ? TW : TH) * c.nlp * 4),
                bar);
      }
    }
    return;
  }
  const uint32_t bytes = (uint32_t)((TH + TW) * 4 * ((v0 ? c0.kc : 0) + (v1 ? c1.kc : 0)));
  const int n0 = v0 ? (c0.kc == c0.nlp ? 2 : TH + TW) : 0;
  const int n1 = v1 ? (c1.kc == c1.nlp ? 2 : TH + TW) : 0;
  // (the caller's __syncwarp ends every read of buf before this point)
  if (lane == 0) nt_expect(bar, bytes);
  __syncwarp();
  if (lane < n0 + n1) asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  for (int j = lane; j < n0 + n1; j += 32) {
    const int h = j < n0 ? 0 : 1;
    const int q = h ? j - n0 : j;
    const NtChunk& c = h ? c1 : c0;
    const int nq = h ? n1 : n0;
    float* dst = buf + h * kNtHalf;
    if (nq == 2) {
      if (q == 0) nt_bulk(dst, a.X + c.xo, (uint32_t)(TH * c.nlp * 4), bar);
      else nt_bulk(dst + kNtRegion, a.Y + c.yo, (uint32_t)(TW * c.nlp * 4), bar);
    } else if (q < TH) {
      nt_bulk(dst + q * c.kc, a.X + c.xo + (int64_t)q * c.nlp + c.t0, (uint32_t)(c.kc * 4), bar);
    } else {
      const int r = q - TH;
      nt_bulk(dst + kNtRegion + r * c.kc, a.Y + c.yo + (int64_t)r * c.nlp + c.t0, (uint32_t)(c.kc * 4), bar);
    }
  }
}

template <int MR, int MC, int KC>
__device__ __forceinline__ void nt_fma_fixed(const float* xs, const float* ys, float* p) {
#pragma unroll 1
  for (int t = 0; t < KC; t += 4) {
    float4 xv[MR];
#pragma unroll
    for (int i = 0; i < MR; ++i) xv[i] = *reinterpret_cast<const float4*>(xs + i * KC + t);
#pragma unroll
    for (int j = 0; j < MC; ++j) {
      const float4 yv = *reinterpret_cast<const float4*>(ys + j * KC + t);
#pragma unroll
      for (int i = 0; i < MR; ++i) {
        float s = p[i * MC + j];
        s = fmaf(xv[i].x, yv.x, s);
        s = fmaf(xv[i].y, yv.y, s);
        s = fmaf(xv[i].z, yv.z, s);
        s = fmaf(xv[i].w, yv.w, s);
        p[i * MC + j] = s;
      }
    }
  }
}

// The FMAs of one staged piece: MR rows of the X slice and MC rows of the Y slice (row pitch
// kc), 4 values of t per step.  With CONST the full 20-wide piece, the common case, runs with
// a compile-time row pitch (one address per step, constant offsets for the rows).
template <int MR, int MC, bool CONST>
__device__ __forceinline__ void nt_fma_chunk(const float* xs, const float* ys, int kc, float* p) {
  if (CONST && kc == kNtKC) {
    nt_fma_fixed<MR, MC, kNtKC>(xs, ys, p);
    return;
  }
  for (int t = 0; t < kc; t += 4) {
    float4 xv[MR];
#pragma unroll
    for (int i = 0; i < MR; ++i) xv[i] = *reinterpret_cast<const float4*>(xs + i * kc + t);
#pragma unroll
    for (int j = 0; j < MC; ++j) {
      const float4 yv = *reinterpret_cast<const float4*>(ys + j * kc + t);
#pragma unroll
      for (int i = 0; i < MR; ++i) {
        float s = p[i * MC + j];
        s = fmaf(xv[i].x, yv.x, s);
        s = fmaf(xv[i].y, yv.y, s);
        s = fmaf(xv[i].z, yv.z, s);
        s = fmaf(xv[i].w, yv.w, s);
        p[i * MC + j] = s;
      }
    }
  }
}

// acc + p as an error-free two-sum: acc <- rounded sum, p <- its rounding error
__device__ __forceinline__ void nt_fold(float& acc, float& p) {
  const float s = acc + p;
  const float bp = s - acc;
  const float e = (acc - (s - bp)) + (p - bp);
  acc = s;
  p = e;
}

// One output tile whose padded extent is 4MR x 4MC.  Returns false on a time-out.
template <int MR, int MC, bool CONST>
__device__ bool nt_tile(const NtArgs& a, const Tile& tile, int k, int nu, int nup, int ni, int nj, float* wbase,
                        uint64_t* bars, NtEntry* ent, uint32_t& phase, int lane) {
  constexpr int TH = 4 * MR, TW = 4 * MC, NQ = MR * MC;
  const int half = lane >> 4, hl = lane & 15;
  const int mr = hl >> 2, mc = hl & 3;
  const int th = min(20, ni - tile.r0), tw = min(20, nj - tile.c0);
  float acc[NQ], p[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = p[q] = 0.0f;
  int folded = 0;
  bool ok = true;
  NtLister L;
  L.a = &a;
  L.ent = ent;
  L.px = (int)a.xptr[nu];
  L.px1 = (int)a.xptr[nu + 1];
  L.py0 = (int)a.yptr[nup];
  L.py1 = (int)a.yptr[nup + 1];
  L.r0 = tile.r0;
  L.c0 = tile.c0;
  L.nm = L.e = L.t0 = 0;
  int buf = 0;
  {
    const NtChunk c0 = L.next(lane);
    const NtChunk c1 = L.next(lane);
    int kc = half ? c1.kc : c0.kc;
    int last = half ? c1.last : c0.last;
    if (c0.last >= 0) nt_issue<TH, TW>(a, c0, c1, wbase, bars, lane);
    while (c0.last >= 0) {
      const NtChunk n0 = L.next(lane);
      const NtChunk n1 = L.next(lane);
      const bool more = n0.last >= 0;
      if (more) nt_issue<TH, TW>(a, n0, n1, wbase + (buf ^ 1) * kNtBuf, bars + (buf ^ 1), lane);
      const bool got = nt_wait(bars + buf, (phase >> buf) & 1u);
      phase ^= 1u << buf;
      if (!__all_sync(0xffffffffu, got)) {
        ok = false;
        if (more) {  // let the copies already issued land before the warp leaves
          nt_wait(bars + (buf ^ 1), (phase >> (buf ^ 1)) & 1u);
          phase ^= 1u << (buf ^ 1);
        }
        break;
      }
      if (last >= 0) {
        const float* hb = wbase + buf * kNtBuf + half * kNtHalf;
        nt_fma_chunk<MR, MC, CONST>(hb + mr * MR * kc, hb + kNtRegion + mc * MC * kc, kc, p);
        if (last && ++folded == kNtFold) {
          folded = 0;
#pragma unroll
          for (int q = 0; q < NQ; ++q) nt_fold(acc[q], p[q]);
        }
      }
      __syncwarp();
      if (!more) break;
      kc = half ? n1.kc : n0.kc;
      last = half ? n1.last : n0.last;
      buf ^= 1;
    }
  }
  // ---- combine the halves and write the tile -------------------------------------------
  float* cb = a.C + a.c_voff[k];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const float oa = __shfl_xor_sync(0xffffffffu, acc[q], 16);
    const float op = __shfl_xor_sync(0xffffffffu, p[q], 16);
    float s = acc[q];
    float e = oa;
    nt_fold(s, e);  // s = acc0 + acc1, e = its rounding error
    const int i = q / MC, j = q - i * MC;
    const int r = mr * MR + i, c = mc * MC + j;
    if (half == 0 && r < th && c < tw)
      cb[(int64_t)(tile.r0 + r) * nj + tile.c0 + c] = ok ? s + (e + (p[q] + op)) : __int_as_float(0x7fc00000);
  }
  return ok;
}

template <bool CONST>
__global__ void __launch_bounds__(kNtWarps * 32, 4) mul_f32_nt_kernel(NtArgs a) {
  extern __shared__ __align__(128) float nsm[];  // [warp][buffer][kNtBuf]
  __shared__ __align__(8) uint64_t bars[kNtWarps][2];
  __shared__ __align__(16) NtEntry sent[kNtWarps][kNtEnt];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float* wbase = nsm + (size_t)w * 2 * kNtBuf;  // the warp's two stage buffers
  if (lane == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(nt_smem(&bars[w][0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(nt_smem(&bars[w][1])));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncwarp();
  uint32_t phase = 0;
  for (;;) {
    unsigned int t = 0;
    if (lane == 0) t = atomicAdd(a.counter, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= a.ntiles) break;
    const Tile tile = a.tiles[t];
    const int k = tile.blk;
    const int nu = a.c_brow[k], nup = a.c_col[k];
    const int ni = a.bsize[nu], nj = a.bsize[nup];
    const int mr = (min(20, ni - tile.r0) + 3) >> 2, mc = (min(20, nj - tile.c0) + 3) >> 2;  // 1..5 each
    bool ok = true;
    float* wb = wbase;
    uint64_t* bw = bars[w];
    NtEntry* en = sent[w];
#define SF_NT_CASE(R, Cc) \
  case (R - 1) * 5 + (Cc - 1): ok = nt_tile<R, Cc, CONST>(a, tile, k, nu, nup, ni, nj, wb, bw, en, phase, lane); break;
    switch ((mr - 1) * 5 + (mc - 1)) {
      SF_NT_CASE(1, 1) SF_NT_CASE(1, 2) SF_NT_CASE(1, 3) SF_NT_CASE(1, 4) SF_NT_CASE(1, 5)
      SF_NT_CASE(2, 1) SF_NT_CASE(2, 2) SF_NT_CASE(2, 3) SF_NT_CASE(2, 4) SF_NT_CASE(2, 5)
      SF_NT_CASE(3, 1) SF_NT_CASE(3, 2) SF_NT_CASE(3, 3) SF_NT_CASE(3, 4) SF_NT_CASE(3, 5)
      SF_NT_CASE(4, 1) SF_NT_CASE(4, 2) SF_NT_CASE(4, 3) SF_NT_CASE(4, 4) SF_NT_CASE(4, 5)
      SF_NT_CASE(5, 1) SF_NT_CASE(5, 2) SF_NT_CASE(5, 3) SF_NT_CASE(5, 4) SF_NT_CASE(5, 5)
      default: break;
    }
#undef SF_NT_CASE
    if (!ok) {
      if (lane == 0) {
        *(volatile unsigned int*)a.err = 1u;  // host-mapped word: plain store, then a system fence
        __threadfence_system();
      }
      break;
    }
  }
}

// Padded K-major copy of a pattern's blocks: block b (rows x cols, row-major in `src` at
// voff[b]) is written at poff[b] as rows_p x cols_p (trans = false) or cols_p x rows_p (its
// transpose, trans = true), sizes rounded up to multiples of 4 and the padding zero.
__global__ void nt_prepare_kernel(int64_t nb, const int32_t* __restrict__ bsize, const int32_t* __restrict__ brow,
                                  const int32_t* __restrict__ bcol, const int64_t* __restrict__ voff,
                                  const int64_t* __restrict__ poff, int trans, const float* __restrict__ src,
                                  float* __restrict__ dst) {
  const int lane = threadIdx.x & 31;
  for (int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; b < nb;
       b += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int rows = bsize[brow[b]], cols = bsize[bcol[b]];
    const int orows = trans ? cols : rows, ocols = trans ? rows : cols;  // output orientation
    const int orp = (orows + 3) & ~3, ocp = (ocols + 3) & ~3;
    const float* s = src + voff[b];
    float* d = dst + poff[b];
    for (int e = lane; e < orp * ocp; e += 32) {
      const int i = e / ocp, j = e - i * ocp;
      float v = 0.0f;
      if (i < orows && j < ocols) v = trans ? s[(int64_t)j * cols + i] : s[(int64_t)i * cols + j];
      d[e] = v;
    }
  }
}

}  // namespace

// ---- host side --------------------------------------------------------------------------

static bool all_multiple_of_4(const s_pattern_t* p) {
  for (int32_t b : p->bsize)
    if (b & 3) return false;
  return true;
}

// Float offsets of the padded blocks of pattern p (nblocks entries) on the device.
static s_status padded_offsets(const s_pattern_t* p, int64_t** out, int64_t* total) {
  const int64_t nb = p->d.nblocks;
  std::vector<int64_t> off(std::max<int64_t>(nb, 1), 0);
  int64_t s = 0;
  for (int64_t b = 0; b < nb; ++b) {
    off[b] = s;
    const int64_t r = (p->bsize[p->brow[b]] + 3) & ~3, c = (p->bsize[p->colidx[b]] + 3) & ~3;
    s += r * c;
  }
  *total = s;
  SF_CUDA(cudaMalloc(out, sizeof(int64_t) * off.size()));
  SF_CUDA(cudaMemcpy(*out, off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice));
  return S_OK;
}

void nt_free_side(NtSideDesc* s) {
  cudaFree(s->poff);
  cudaFree(s->scratch);
  *s = NtSideDesc();
}

// Configure one side of the K-major product: `pat` is the stored operand's pattern, `list` the
// row (X) or column (Y) lists of op(.), `trans` whether the K-major slice is the transpose of
// the stored block.  Direct when no transpose is needed and every block size is a multiple
// of 4; otherwise padded offsets and a scratch buffer for the prepared copy.
static s_status nt_side(const s_pattern_t* pat, const Side& list, bool trans, NtSideDesc* s) {
  nt_free_side(s);
  s->ptr = list.ptr;
  s->idx = list.idx;
  s->blk = list.blk;
  s->pat = pat;
  s->trans = trans;
  s->prep = trans || !all_multiple_of_4(pat);
  if (!s->prep) {
    s->off = pat->d.voff;
    return S_OK;
  }
  s_status st = padded_offsets(pat, &s->poff, &s->len);
  if (st) return st;
  s->off = s->poff;
  SF_CUDA(cudaMalloc(&s->scratch, sizeof(float) * std::max<int64_t>(s->len, 1)));
  return S_OK;
}

// K-major sides of a float descriptor (forward or adjoint) for C = op(X) op(Y), op(X) = X^T
// when x_trans and op(Y) = Y^T when y_trans.  X side: op(X) rows; the stored
// block of a row-list entry is (nu, lambda) when op(X) = X (CSR row) and (lambda, nu) when
// op(X) = X^T (CSC column).  Y side: op(Y) columns; with op(Y) = Y^T the stored block of a
// CSR-row entry (nu', lambda) is already [column][t]; with op(Y) = Y the CSC-column entry
// (lambda, nu') is transposed, unless `y_sym` (Y = X declared symmetric and called with one
// buffer) lets the kernel read Y(nu', lambda) through Y's own CSR rows.
s_status nt_configure(MulDesc* d, bool x_trans, bool y_trans, bool y_sym) {
  const DevPattern& px = d->px->d;
  const DevPattern& py = d->py->d;
  Side xl = x_trans ? Side{px.colptr, px.rowidx, px.cscblk, px.voff, true}
                    : Side{px.rowptr, px.colidx, nullptr, px.voff, false};
  s_status st = nt_side(d->px, xl, x_trans, &d->ntx);
  if (st) return st;
  Side yl;
  bool ytrans;
  if (y_trans || y_sym) {
    yl = Side{py.rowptr, py.colidx, nullptr, py.voff, false};
    ytrans = false;
  } else {
    yl = Side{py.colptr, py.rowidx, py.cscblk, py.voff, true};
    ytrans = true;
  }
  if (y_sym && !x_trans && d->ntx.prep) {
    // B = A read through A's rows: the same padded blocks as the X side, one copy for both
    nt_free_side(&d->nty);
    d->nty.ptr = yl.ptr;
    d->nty.idx = yl.idx;
    d->nty.blk = yl.blk;
    d->nty.pat = d->py;
    d->nty.off = d->ntx.off;
    d->nty.from_x = true;
  } else if ((st = nt_side(d->py, yl, ytrans, &d->nty))) {
    return st;
  }
  d->nt_ysym = y_sym;
  return S_OK;
}

static s_status nt_prepare(const NtSideDesc& s, const float* src, cudaStream_t st) {
  const DevPattern& p = s.pat->d;
  if (p.nblocks == 0) return S_OK;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((p.nblocks * 32 + 255) / 256, (int64_t)sm_count() * 16));
  nt_prepare_kernel<<<grid, 256, 0, st>>>(p.nblocks, p.bsize, p.brow, p.colidx, p.voff, s.poff, s.trans ? 1 : 0, src,
                                          s.scratch);
  SF_CUDA(cudaGetLastError());
  return S_OK;
}

bool nt_usable(const MulDesc& d, const void* X, const void* Y) {
  if (!d.ntx.off || !d.nty.off) return false;
  // bulk copies read 16-byte aligned sources
  if (!d.ntx.prep && (reinterpret_cast<uintptr_t>(X) & 15)) return false;
  if (!d.nty.prep && !d.nty.from_x && (reinterpret_cast<uintptr_t>(Y) & 15)) return false;
  // a symmetric Y side reads B through A's rows: only valid for B = A
  if (d.nt_ysym && X != Y) return false;
  return true;
}

s_status launch_nt(const MulDesc& d, const void* X, const void* Y, void* C, cudaStream_t st, bool const_pitch) {
  if (d.ntiles == 0) return S_OK;
  s_status s = take_timeout(d);
  if (s) return s;
  const float* xb = (const float*)X;
  const float* yb = (const float*)Y;
  if (d.ntx.prep) {
    if ((s = nt_prepare(d.ntx, (const float*)X, st))) return s;
    xb = d.ntx.scratch;
  }
  if (d.nty.from_x) {
    yb = xb;
  } else if (d.nty.prep) {
    if ((s = nt_prepare(d.nty, (const float*)Y, st))) return s;
    yb = d.nty.scratch;
  }
  NtArgs a;
  a.xptr = d.ntx.ptr;
  a.xidx = d.ntx.idx;
  a.xblk = d.ntx.blk;
  a.xoff = d.ntx.off;
  a.X = xb;
  a.yptr = d.nty.ptr;
  a.yidx = d.nty.idx;
  a.yblk = d.nty.blk;
  a.yoff = d.nty.off;
  a.Y = yb;
  a.bsize = d.pc->d.bsize;
  a.c_brow = d.pc->d.brow;
  a.c_col = d.pc->d.colidx;
  a.c_voff = d.pc->d.voff;
  a.tiles = d.tiles;
  a.ntiles = d.ntiles;
  a.counter = d.counter;
  a.err = d.err;
  a.C = (float*)C;
  SF_CUDA(cudaMemsetAsync(d.counter, 0, sizeof(unsigned int), st));
  void (*kern)(NtArgs) = const_pitch ? mul_f32_nt_kernel<true> : mul_f32_nt_kernel<false>;
  SF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kNtSmem));
  int per_sm = 0;
  SF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kNtWarps * 32, kNtSmem));
  if (per_sm < 1) per_sm = 1;
  const int64_t want = (d.ntiles + kNtWarps - 1) / kNtWarps;
  const int grid = (int)std::min<int64_t>(want, (int64_t)sm_count() * per_sm);
  kern<<<grid, kNtWarps * 32, kNtSmem, st>>>(a);
  SF_CUDA(cudaGetLastError());
  return S_OK;
}

}  // namespace sf
