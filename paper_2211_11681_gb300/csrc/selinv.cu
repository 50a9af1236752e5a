// Selected inversion on the compression pattern (Sec. 4.2 "Sparse selected inversion",
// Eq. (blockInv)) and the contour-integral inverse square root (Sec. 4.4, Eq. (ContInt)),
// in FP64.
//
// Supernodes are the clusters: every non-empty cluster is one block column of the factor,
// its samplets a dense block.  The host picks a minimum-degree elimination order of the
// block graph of S, plays the elimination game to get the pattern of L (position space,
// i >= k), and lists the blocks of every level of the elimination tree.  Blocks whose
// columns sit on one level are independent, so each level is one launch per step:
//
//   factor, levels from the leaves up (A + sigma I = L D L^T, W = L D kept beside L):
//     update  W(i,k) = A(i,k) + sigma [i = k] - sum_{j < k} W(i,j) L(k,j)^T over the j in
//             both row i and row k of L;
//     pivot   D(k,k) = W(k,k) inverted by Gauss-Jordan in shared memory (positive definite:
//             no pivoting; a pivot that is not positive is recorded), then
//             L(i,k) = W(i,k) D(k,k)^{-1} for the blocks of column k (a CTA per supernode
//             and slice of its column), D^{-1} stored in L's diagonal block;
//   inversion, levels from the root down (Takahashi-type recurrences from Eq. (blockInv)):
//     off     Z(i,k) = - sum_{j in struct(k)} Z(i,j) L(j,k), Z(i,j) read from block
//             (max, min) of Z, transposed when i < j;
//     diag    Z(k,k) = D(k,k)^{-1} - sum_{j in struct(k)} Z(j,k)^T L(j,k) (a CTA per
//             supernode, its warps splitting the sum);
//   scatter   out = alpha P_S(Z) + beta out, blocks of S read from Z or its transpose.
//
// The terms of every sum are fixed by the pattern of L, so the plan lists them once (the
// symbolic phase of both sweeps): per block of L the pairs (W(i,j), L(k,j)) of the update and
// (Z(i,j), L(j,k)) of the inversion.  The update and off-diagonal steps give one warp an
// output block (512-entry tiles of it, 16 entries per lane) and a contiguous part of its
// term list: near the root the elimination tree is a chain whose levels hold few, long sums,
// so the host splits each list into `split` parts (split-K) to keep every SM sub-partition
// busy.  With split > 1 the parts land in a scratch buffer and the next launch of the level
// (pivot, diag) adds them in a fixed order, so results do not depend on scheduling.  The
// operand blocks of each term are staged in shared memory 16 columns at a time (row pitch 17
// doubles: rows fall in different banks) by cp.async into one of two buffers per warp, the
// next unit's copies in flight while the current unit is multiplied.
//
// Every entry a launch reads was written by an earlier launch (descendants sit on lower
// levels, ancestors on higher ones) or by its own CTA before a barrier, so the kernels need
// no synchronisation beyond stream order and no waits.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "sselinv.h"

namespace sf {
namespace {

constexpr int kSiMaxB = 64;               // widest block
constexpr int kSiEnt = 16;                // output entries per lane
constexpr int kSiTileEnt = 32 * kSiEnt;   // entries of one work item
constexpr int kSiWarps = 4;               // warps per CTA of the block kernels
constexpr int kSiThreads = 128;           // threads of the pivot and diagonal kernels
constexpr int kSiSlice = 8;               // column blocks per pivot CTA
constexpr int kSiU = 16;                  // columns of t staged per slice
constexpr int kSiUp = kSiU + 1;           // row pitch of a staged slice (doubles)
constexpr int kSiMaxSplit = 64;           // parts of one split sum
constexpr int kSiPartTerms = 4;           // fewest terms of one part
constexpr int kSiMaxClusters = 32768;     // non-empty clusters of the host bitset analysis

struct SiItem {
  int32_t blk;  // CSC block of L
  int32_t col;  // its column position
  int32_t e0;   // first entry of the tile
};

struct SiDev {
  const int32_t* bs;      // block size per position
  const int64_t* colptr;  // CSC of L: column k holds blocks colptr[k] .. colptr[k+1]-1,
  const int32_t* colrow;  //   the diagonal first, then the rows of struct(k) ascending
  const int64_t* loff;    // entry offset of each CSC block (rows x cols, row-major)
  const int64_t* lpo;     // entry offset of each CSC block among the blocks of its level
  const int32_t* colcol;  // column position of each CSC block
  const int64_t* uptr;    // factor terms of CSC block q: uptr[q] .. uptr[q+1]-1, pairs of
  const int32_t* uw;      //   CSC blocks W(i,j), L(k,j)
  const int32_t* ul;
  const int64_t* optr;    // inversion terms of CSC block q = (i,k), i > k: for every j in
  const int32_t* oz;      //   struct(k) the block of Z(i,j) (~index: stored as Z(j,i)) and
  const int32_t* ol;      //   the block L(j,k)
  const int64_t* aoff;    // per CSC block: entry offset of the S block with its rows and
                          // columns (-1: not in S)
  double* W;              // L D (D in the diagonal blocks)
  double* L;              // L (D^{-1} in the diagonal blocks)
  double* Z;              // the inverse on the pattern of L
  double* P;              // partial sums of split launches: [part][entries of the level]
  unsigned int* flag;     // mapped host word: 1 = a pivot block was not positive definite
  int maxb;               // widest block of the plan
};

// Entry coordinates of a lane's kSiEnt entries of a rows x cols tile starting at e0.
__device__ __forceinline__ void si_entries(int e0, int ne, int cols, int lane, int* rr, int* cc) {
#pragma unroll
  for (int m = 0; m < kSiEnt; ++m) {
    const int e = e0 + lane + 32 * m;
    rr[m] = e < ne ? e / cols : -1;
    cc[m] = e < ne ? e - rr[m] * cols : 0;
  }
}

// acc[m] += sign * sum_t a[rr[m]][t] b[cc[m]][t] over t < uw (staged slices).
__device__ __forceinline__ void si_dot(const double* a, const double* b, int uw, const int* rr, const int* cc,
                                       double sign, double* acc) {
#pragma unroll
  for (int m = 0; m < kSiEnt; ++m) {
    if (rr[m] < 0) continue;
    const double* ar = a + rr[m] * kSiUp;
    const double* br = b + cc[m] * kSiUp;
    double t0 = 0.0, t1 = 0.0;
    int t = 0;
    for (; t + 4 <= uw; t += 4) {
      t0 = fma(ar[t], br[t], t0);
      t1 = fma(ar[t + 1], br[t + 1], t1);
      t0 = fma(ar[t + 2], br[t + 2], t0);
      t1 = fma(ar[t + 3], br[t + 3], t1);
    }
    for (; t < uw; ++t) t0 = fma(ar[t], br[t], t0);
    acc[m] = fma(sign, t0 + t1, acc[m]);
  }
}

// Stage rows x uw values into dst[r * kSiUp + t] (zero padded to uw4 columns):
// value(r, t) = src[r * rs + t * ts] (rs, ts: the source's row and column strides).  Plain
// (coherent) loads: the diagonal kernel reads blocks its own CTA wrote before a barrier.
__device__ __forceinline__ void si_stage(double* dst, const double* src, int rows, int uw, int uw4, int rs, int ts,
                                         int lane) {
  if (ts == 1) {
    for (int idx = lane; idx < rows * uw4; idx += 32) {
      const int r = idx / uw4, t = idx - r * uw4;
      dst[r * kSiUp + t] = t < uw ? src[(int64_t)r * rs + t] : 0.0;
    }
  } else {
    for (int idx = lane; idx < rows * uw4; idx += 32) {  // rows fastest: coalesced when rs = 1
      const int t = idx / rows, r = idx - t * rows;
      dst[r * kSiUp + t] = t < uw ? src[(int64_t)t * ts + (int64_t)r * rs] : 0.0;
    }
  }
}

// Asynchronous 8-byte copy global -> shared (cp.async, zero fill when !valid; src must still
// point into the buffer), and its group commit / wait.
__device__ __forceinline__ void si_cp8(double* dst, const double* src, bool valid) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 8 : 0) : "memory");
}
__device__ __forceinline__ void si_cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void si_cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void si_cp_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// si_stage with cp.async: the copies complete at the lane's next wait on their group.
__device__ __forceinline__ void si_stage_async(double* dst, const double* src, int rows, int uw, int uw4, int rs,
                                               int ts, int lane) {
  if (ts == 1) {
    for (int idx = lane; idx < rows * uw4; idx += 32) {
      const int r = idx / uw4, t = idx - r * uw4;
      si_cp8(dst + r * kSiUp + t, t < uw ? src + (int64_t)r * rs + t : src, t < uw);
    }
  } else {
    for (int idx = lane; idx < rows * uw4; idx += 32) {
      const int t = idx / rows, r = idx - t * rows;
      si_cp8(dst + r * kSiUp + t, t < uw ? src + (int64_t)t * ts + (int64_t)r * rs : src, t < uw);
    }
  }
}

// factor update: W(i,k) = A(i,k) + sigma [i = k] - sum_j W(i,j) L(k,j)^T over the block's term
// list; warp gw serves item gw / split and the part gw % split of the list.  The term list
// is walked in units of one term and 16 columns of t; the next unit's blocks are copied into
// the warp's second stage buffer (cp.async) while the current unit is multiplied.
__global__ void __launch_bounds__(kSiWarps * 32) si_update_kernel(SiDev s, const SiItem* __restrict__ items,
                                                                   int64_t nitems, int split, int64_t E,
                                                                   const double* __restrict__ A, double sigma) {
  extern __shared__ double sh[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (gw >= nitems * split) return;
  const int64_t itn = gw / split;
  const int part = (int)(gw - itn * split);
  const SiItem it = items[itn];
  const int i = s.colrow[it.blk], k = it.col;
  const int bi = s.bs[i], bk = s.bs[k];
  const int ne = bi * bk;
  const size_t half = (size_t)2 * s.maxb * kSiUp;       // one stage buffer: operand a | operand b
  double* buf = sh + (size_t)w * 2 * half;
  int rr[kSiEnt], cc[kSiEnt];
  si_entries(it.e0, ne, bk, lane, rr, cc);
  double acc[kSiEnt];
  const int64_t ao = s.aoff[it.blk];
#pragma unroll
  for (int m = 0; m < kSiEnt; ++m) {
    double v = 0.0;
    if (part == 0 && rr[m] >= 0) {
      if (ao >= 0) v = A[ao + it.e0 + lane + 32 * m];
      if (i == k && rr[m] == cc[m]) v += sigma;
    }
    acc[m] = v;
  }
  const int64_t t0 = s.uptr[it.blk], nt = s.uptr[it.blk + 1] - t0;
  int64_t t = t0 + nt * part / split;
  const int64_t te = t0 + nt * (part + 1) / split;
  auto issue = [&](int64_t tt, int u0, double* dst) {
    const int bw = s.uw[tt], bl = s.ul[tt];
    const int bj = s.bs[s.colcol[bw]];
    const int uw = min(kSiU, bj - u0), uw4 = (uw + 3) & ~3;
    si_stage_async(dst, s.W + s.loff[bw] + u0, bi, uw, uw4, bj, 1, lane);             // W(i,j)
    si_stage_async(dst + s.maxb * kSiUp, s.L + s.loff[bl] + u0, bk, uw, uw4, bj, 1, lane);  // L(k,j)
  };
  int u0 = 0, cur = 0;
  if (t < te) issue(t, 0, buf);
  si_cp_commit();
  while (t < te) {
    const int bj = s.bs[s.colcol[s.uw[t]]];
    const int uwc = min(kSiU, bj - u0);
    int64_t tn = t;
    int un = u0 + kSiU;
    if (un >= bj) {
      tn = t + 1;
      un = 0;
    }
    if (tn < te) issue(tn, un, buf + (cur ^ 1) * half);
    si_cp_commit();
    si_cp_wait1();
    __syncwarp();
    const double* cb = buf + cur * half;
    si_dot(cb, cb + s.maxb * kSiUp, uwc, rr, cc, -1.0, acc);
    __syncwarp();
    t = tn;
    u0 = un;
    cur ^= 1;
  }
  si_cp_wait0();
  double* out = split > 1 ? s.P + (int64_t)part * E + s.lpo[it.blk] : s.W + s.loff[it.blk];
#pragma unroll
  for (int m = 0; m < kSiEnt; ++m)
    if (rr[m] >= 0) out[it.e0 + lane + 32 * m] = acc[m];
}

// Gauss-Jordan inverse of the bk x bk block M (row-major, shared) without pivoting; returns
// false (in every thread) if a pivot was not a positive finite number.
__device__ bool si_gauss_jordan(double* M, int bk, double* prow, double* pcol) {
  bool ok = true;
  for (int p = 0; p < bk; ++p) {
    const double piv = M[p * bk + p];
    if (!(piv > 0.0) || !isfinite(piv)) ok = false;
    const double inv = 1.0 / piv;
    for (int t = threadIdx.x; t < bk; t += blockDim.x) {
      prow[t] = t == p ? inv : M[p * bk + t] * inv;
      pcol[t] = M[t * bk + p];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < bk * bk; idx += blockDim.x) {
      const int r = idx / bk, c = idx - r * bk;
      if (r == p) M[idx] = prow[c];
      else M[idx] = (c == p ? 0.0 : M[idx]) - pcol[r] * prow[c];
    }
    __syncthreads();
  }
  return ok;
}

// Entry `idx` of CSC block q after the update of its level: W itself, or the sum of the
// `split` parts in part order.
__device__ __forceinline__ double si_assembled(const SiDev& s, const double* base, int64_t q, int idx, int split,
                                               int64_t E) {
  if (split <= 1) return base[s.loff[q] + idx];
  const double* p = s.P + s.lpo[q] + idx;
  double v = p[0];
  for (int t = 1; t < split; ++t) v += p[(int64_t)t * E];
  return v;
}

// pivot: D(k,k)^{-1} and L(i,k) = W(i,k) D(k,k)^{-1}; CTA (x, y) serves supernode sn[x] and
// the column blocks y*kSiSlice+1 .. of it; slice 0 stores D^{-1}.  With split > 1 the blocks
// are first assembled from the update's parts (and W(i,k) stored).
__global__ void __launch_bounds__(kSiThreads) si_pivot_kernel(SiDev s, const int32_t* __restrict__ sn, int split,
                                                              int64_t E) {
  extern __shared__ double smem[];
  __shared__ double prow[kSiMaxB], pcol[kSiMaxB];
  const int k = sn[blockIdx.x];
  const int bk = s.bs[k];
  const int64_t c0 = s.colptr[k], c1 = s.colptr[k + 1];
  const int64_t q0 = c0 + 1 + (int64_t)blockIdx.y * kSiSlice;
  if (blockIdx.y > 0 && q0 >= c1) return;
  double* M = smem;
  double* Wb = smem + (size_t)s.maxb * s.maxb;
  for (int idx = threadIdx.x; idx < bk * bk; idx += blockDim.x) M[idx] = si_assembled(s, s.W, c0, idx, split, E);
  __syncthreads();
  const bool ok = si_gauss_jordan(M, bk, prow, pcol);
  if (blockIdx.y == 0) {
    if (!ok && threadIdx.x == 0) {
      *(volatile unsigned int*)s.flag = 1u;
      __threadfence_system();
    }
    double* Dinv = s.L + s.loff[c0];
    for (int idx = threadIdx.x; idx < bk * bk; idx += blockDim.x) Dinv[idx] = M[idx];
  }
  const int64_t q1 = min(c1, q0 + kSiSlice);
  for (int64_t q = q0; q < q1; ++q) {
    const int bi = s.bs[s.colrow[q]];
    double* Wq = s.W + s.loff[q];
    for (int idx = threadIdx.x; idx < bi * bk; idx += blockDim.x) {
      const double v = si_assembled(s, s.W, q, idx, split, E);
      Wb[idx] = v;
      if (split > 1) Wq[idx] = v;
    }
    __syncthreads();
    double* Lq = s.L + s.loff[q];
    for (int idx = threadIdx.x; idx < bi * bk; idx += blockDim.x) {
      const int r = idx / bk, c = idx - r * bk;
      const double* wr = Wb + r * bk;
      double t = 0.0;
      for (int u = 0; u < bk; ++u) t = fma(wr[u], M[u * bk + c], t);
      Lq[idx] = t;
    }
    __syncthreads();
  }
}

// inversion, off-diagonal blocks: Z(i,k) = - sum_{j in struct(k)} Z(i,j) L(j,k) over the block's
// term list; warp gw serves item gw / split and the part gw % split of the list, staged and
// prefetched as in the update.
__global__ void __launch_bounds__(kSiWarps * 32) si_offdiag_kernel(SiDev s, const SiItem* __restrict__ items,
                                                                    int64_t nitems, int split, int64_t E) {
  extern __shared__ double sh[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (gw >= nitems * split) return;
  const int64_t itn = gw / split;
  const int part = (int)(gw - itn * split);
  const SiItem it = items[itn];
  const int i = s.colrow[it.blk], k = it.col;
  const int bi = s.bs[i], bk = s.bs[k];
  const int ne = bi * bk;
  const size_t half = (size_t)2 * s.maxb * kSiUp;
  double* buf = sh + (size_t)w * 2 * half;
  int rr[kSiEnt], cc[kSiEnt];
  si_entries(it.e0, ne, bk, lane, rr, cc);
  double acc[kSiEnt];
#pragma unroll
  for (int m = 0; m < kSiEnt; ++m) acc[m] = 0.0;
  const int64_t t0 = s.optr[it.blk], nt = s.optr[it.blk + 1] - t0;
  int64_t t = t0 + nt * part / split;
  const int64_t te = t0 + nt * (part + 1) / split;
  auto issue = [&](int64_t tt, int u0, double* dst) {
    const int zb = s.oz[tt], qq = s.ol[tt];
    const int bj = s.bs[s.colrow[qq]];
    const int uw = min(kSiU, bj - u0), uw4 = (uw + 3) & ~3;
    if (zb < 0)  // Z(i,j) = Z(j,i)^T, block bj x bi
      si_stage_async(dst, s.Z + s.loff[~zb] + (int64_t)u0 * bi, bi, uw, uw4, 1, bi, lane);
    else
      si_stage_async(dst, s.Z + s.loff[zb] + u0, bi, uw, uw4, bj, 1, lane);
    si_stage_async(dst + s.maxb * kSiUp, s.L + s.loff[qq] + (int64_t)u0 * bk, bk, uw, uw4, 1, bk, lane);  // L(j,k)
  };
  int u0 = 0, cur = 0;
  if (t < te) issue(t, 0, buf);
  si_cp_commit();
  while (t < te) {
    const int bj = s.bs[s.colrow[s.ol[t]]];
    const int uwc = min(kSiU, bj - u0);
    int64_t tn = t;
    int un = u0 + kSiU;
    if (un >= bj) {
      tn = t + 1;
      un = 0;
    }
    if (tn < te) issue(tn, un, buf + (cur ^ 1) * half);
    si_cp_commit();
    si_cp_wait1();
    __syncwarp();
    const double* cb = buf + cur * half;
    si_dot(cb, cb + s.maxb * kSiUp, uwc, rr, cc, -1.0, acc);
    __syncwarp();
    t = tn;
    u0 = un;
    cur ^= 1;
  }
  si_cp_wait0();
  double* out = split > 1 ? s.P + (int64_t)part * E + s.lpo[it.blk] : s.Z + s.loff[it.blk];
#pragma unroll
  for (int m = 0; m < kSiEnt; ++m)
    if (rr[m] >= 0) out[it.e0 + lane + 32 * m] = acc[m];
}

// inversion, diagonal blocks: Z(k,k) = D^{-1} - sum_{j in struct(k)} Z(j,k)^T L(j,k).  CTA
// (x, y) serves supernode sn[x] and the column blocks y*kSiSlice+1 .. of it: with split > 1
// it first assembles those Z(j,k) from the off-diagonal parts, then its warps split the
// slice's terms and add them in warp order.  With one slice the CTA writes Z(k,k); with
// several, each slice stores its sum in Q and the last slice to finish (counted per
// supernode in `cnt`, which it resets) adds the slices in slice order and writes Z(k,k).
__global__ void __launch_bounds__(kSiWarps * 32) si_diag_kernel(SiDev s, const int32_t* __restrict__ sn, int split,
                                                                int64_t E, int slices, unsigned int* cnt,
                                                                double* Q) {
  extern __shared__ double sh[];
  __shared__ int last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int k = sn[blockIdx.x];
  const int bk = s.bs[k];
  const int64_t c0 = s.colptr[k], c1 = s.colptr[k + 1];
  const int64_t qs = c0 + 1 + (int64_t)blockIdx.y * kSiSlice, qe = min(c1, qs + kSiSlice);
  if (split > 1 && qe > qs) {
    const int64_t z0 = s.loff[qs], len = s.loff[qe] - z0;
    const double* p = s.P + s.lpo[qs];
    for (int64_t idx = threadIdx.x; idx < len; idx += blockDim.x) {
      double v = p[idx];
      for (int t = 1; t < split; ++t) v += p[(int64_t)t * E + idx];
      s.Z[z0 + idx] = v;
    }
    __syncthreads();
  }
  double* sa = sh + (size_t)w * 2 * s.maxb * kSiUp;
  double* sb = sa + (size_t)s.maxb * kSiUp;
  double* red = sh + (size_t)kSiWarps * 2 * s.maxb * kSiUp;  // [warp][kSiTileEnt]
  const double* Dinv = s.L + s.loff[c0];
  double* Zkk = s.Z + s.loff[c0];
  const int ne = bk * bk;
  const int64_t qst = (int64_t)s.maxb * s.maxb;                             // slice stride in Q
  double* mine = Q + ((int64_t)blockIdx.x * slices + blockIdx.y) * qst;      // this slice's sum
  for (int e0 = 0; e0 < ne; e0 += kSiTileEnt) {
    int rr[kSiEnt], cc[kSiEnt];
    si_entries(e0, ne, bk, lane, rr, cc);
    double acc[kSiEnt];
#pragma unroll
    for (int m = 0; m < kSiEnt; ++m) acc[m] = 0.0;
    for (int64_t q = qs + w; q < qe; q += kSiWarps) {
      const int bj = s.bs[s.colrow[q]];
      const double* Zq = s.Z + s.loff[q];  // bj x bk
      const double* Lq = s.L + s.loff[q];
      for (int u0 = 0; u0 < bj; u0 += kSiU) {
        const int uw = min(kSiU, bj - u0), uw4 = (uw + 3) & ~3;
        __syncwarp();
        si_stage(sa, Zq + (int64_t)u0 * bk, bk, uw, uw4, 1, bk, lane);
        si_stage(sb, Lq + (int64_t)u0 * bk, bk, uw, uw4, 1, bk, lane);
        __syncwarp();
        si_dot(sa, sb, uw, rr, cc, 1.0, acc);
      }
    }
#pragma unroll
    for (int m = 0; m < kSiEnt; ++m) red[w * kSiTileEnt + lane + 32 * m] = acc[m];
    __syncthreads();
    for (int idx = threadIdx.x; idx < kSiTileEnt && e0 + idx < ne; idx += blockDim.x) {
      double v = red[idx];
      for (int t = 1; t < kSiWarps; ++t) v += red[t * kSiTileEnt + idx];
      if (slices == 1) Zkk[e0 + idx] = Dinv[e0 + idx] - v;
      else mine[e0 + idx] = v;
    }
    __syncthreads();
  }
  if (slices == 1) return;
  // the last slice of this supernode adds all slices in order
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(cnt + k, 1u) == (unsigned int)(slices - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  const double* all = Q + (int64_t)blockIdx.x * slices * qst;
  for (int idx = threadIdx.x; idx < ne; idx += blockDim.x) {
    double v = 0.0;
    for (int t = 0; t < slices; ++t) v += ((volatile const double*)all)[(int64_t)t * qst + idx];
    Zkk[idx] = Dinv[idx] - v;
  }
  if (threadIdx.x == 0) cnt[k] = 0u;
}

// out = alpha P_S(Z) + beta out: one warp per block of S
__global__ void si_scatter_kernel(int64_t nblocks, const int32_t* __restrict__ sbsize,
                                  const int32_t* __restrict__ sbrow, const int32_t* __restrict__ scol,
                                  const int64_t* __restrict__ svoff, const int32_t* __restrict__ s2l,
                                  const int8_t* __restrict__ s2t, const int64_t* __restrict__ loff,
                                  const double* __restrict__ Z, double alpha, double beta, double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  for (int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; b < nblocks;
       b += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int br = sbsize[sbrow[b]], bc = sbsize[scol[b]];
    const int lb = s2l[b];
    if (lb < 0) continue;  // an empty block
    const bool tr = s2t[b] != 0;
    const double* zb = Z + loff[lb];
    double* o = out + svoff[b];
    for (int e = lane; e < br * bc; e += 32) {
      const int r = e / bc, c = e - r * bc;
      const double z = tr ? zb[(int64_t)c * br + r] : zb[e];
      o[e] = beta == 0.0 ? alpha * z : alpha * z + beta * o[e];
    }
  }
}

// ---- host: symbolic analysis ------------------------------------------------------------

struct Symbolic {
  int32_t m = 0;                         // non-empty clusters
  std::vector<int32_t> perm;             // position -> cluster (non-empty first)
  std::vector<int32_t> pos;              // cluster -> position (-1: empty cluster)
  std::vector<std::vector<int32_t>> st;  // struct(p): positions below p in column p, ascending
};

// Symmetric, sorted, in-range pattern check; returns S_ERR_PATTERN on a violation.
s_status check_symmetric(int32_t nc, const int64_t* rowptr, const int32_t* colidx) {
  for (int32_t r = 0; r < nc; ++r) {
    for (int64_t q = rowptr[r]; q < rowptr[r + 1]; ++q) {
      const int32_t c = colidx[q];
      if (c < 0 || c >= nc || (q > rowptr[r] && colidx[q - 1] >= c))
        return set_error(S_ERR_PATTERN, "selected inversion: pattern rows must be sorted and in range");
      const int32_t* b = colidx + rowptr[c];
      const int32_t* e = colidx + rowptr[c + 1];
      const int32_t* f = std::lower_bound(b, e, r);
      if (f == e || *f != r) return set_error(S_ERR_PATTERN, "selected inversion: the pattern is not symmetric");
    }
  }
  return S_OK;
}

// Minimum degree on the block graph (exact degrees, bitset rows), ties to the smaller id.
s_status symbolic(int32_t nc, const int64_t* rowptr, const int32_t* colidx, const int32_t* bsize, Symbolic* out) {
  s_status st = check_symmetric(nc, rowptr, colidx);
  if (st) return st;
  std::vector<int32_t> vid(nc, -1), cl;
  for (int32_t c = 0; c < nc; ++c)
    if (bsize[c] > 0) {
      vid[c] = (int32_t)cl.size();
      cl.push_back(c);
    }
  const int32_t m = (int32_t)cl.size();
  if (m > kSiMaxClusters) return set_error(S_ERR_ARG, "selected inversion: more than 32768 non-empty clusters");
  const int64_t W = (m + 63) / 64;
  std::vector<uint64_t> adj((size_t)m * W, 0ull), alive((size_t)W, 0ull);
  for (int32_t v = 0; v < m; ++v) alive[v >> 6] |= 1ull << (v & 63);
  for (int32_t v = 0; v < m; ++v) {
    const int32_t r = cl[v];
    for (int64_t q = rowptr[r]; q < rowptr[r + 1]; ++q) {
      const int32_t u = vid[colidx[q]];
      if (u >= 0 && u != v) adj[(size_t)v * W + (u >> 6)] |= 1ull << (u & 63);
    }
  }
  std::vector<int32_t> deg(m);
  for (int32_t v = 0; v < m; ++v) {
    int d = 0;
    for (int64_t w = 0; w < W; ++w) d += __builtin_popcountll(adj[(size_t)v * W + w]);
    deg[v] = d;
  }
  std::vector<uint8_t> done(m, 0);
  std::vector<int32_t> order;
  order.reserve(m);
  std::vector<std::vector<int32_t>> nbv(m);
  std::vector<int32_t> nb;
  for (int32_t step = 0; step < m; ++step) {
    int32_t v = -1;
    for (int32_t u = 0; u < m; ++u)
      if (!done[u] && (v < 0 || deg[u] < deg[v])) v = u;
    done[v] = 1;
    alive[v >> 6] &= ~(1ull << (v & 63));
    order.push_back(v);
    uint64_t* av = &adj[(size_t)v * W];
    nb.clear();
    for (int64_t w = 0; w < W; ++w) {
      uint64_t x = av[w] & alive[w];
      av[w] = x;
      while (x) {
        const int b = __builtin_ctzll(x);
        x &= x - 1;
        nb.push_back((int32_t)(w * 64 + b));
      }
    }
    nbv[v] = nb;
    for (int32_t u : nb) {
      uint64_t* au = &adj[(size_t)u * W];
      int d = 0;
      for (int64_t w = 0; w < W; ++w) {
        const uint64_t x = (au[w] | av[w]) & alive[w];
        au[w] = x;
        d += __builtin_popcountll(x);
      }
      au[u >> 6] &= ~(1ull << (u & 63));
      deg[u] = d - 1;  // the union held u itself (u is a neighbour of v)
    }
  }
  out->m = m;
  out->perm.assign(nc, 0);
  out->pos.assign(nc, -1);
  std::vector<int32_t> vpos(m);
  for (int32_t p = 0; p < m; ++p) {
    vpos[order[p]] = p;
    out->perm[p] = cl[order[p]];
    out->pos[cl[order[p]]] = p;
  }
  int32_t p = m;
  for (int32_t c = 0; c < nc; ++c)
    if (bsize[c] <= 0) out->perm[p++] = c;
  out->st.assign(m, {});
  for (int32_t q = 0; q < m; ++q) {
    const int32_t v = order[q];
    std::vector<int32_t>& s = out->st[q];
    s.reserve(nbv[v].size());
    for (int32_t u : nbv[v]) s.push_back(vpos[u]);
    std::sort(s.begin(), s.end());
  }
  return S_OK;
}

std::vector<int32_t> etree_levels(const Symbolic& sy, int32_t* height) {
  std::vector<int32_t> lvl(sy.m, 0);
  int32_t h = 0;
  for (int32_t p = 0; p < sy.m; ++p) {
    if (!sy.st[p].empty()) {
      const int32_t par = sy.st[p][0];
      lvl[par] = std::max(lvl[par], lvl[p] + 1);
    }
    h = std::max(h, lvl[p] + 1);
  }
  *height = sy.m ? h : 0;
  return lvl;
}

template <typename T>
s_status upload(T** dst, const std::vector<T>& v) {
  const cudaError_t e = cudaMalloc((void**)dst, sizeof(T) * std::max<size_t>(v.size(), 1));
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    *dst = nullptr;
    return set_error(S_ERR_NOMEM, "selected inversion: no device memory for the plan's lists");
  }
  SF_CUDA(e);
  if (!v.empty()) SF_CUDA(cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
  return S_OK;
}

// ---- host: elliptic functions for Eq. (ContInt) ------------------------------------------

// K(m) = pi / (2 AGM(1, sqrt(1 - m))), 0 <= m < 1.
double ellip_k(double m) {
  double a = 1.0, b = std::sqrt(1.0 - m);
  for (int it = 0; it < 64 && std::fabs(a - b) > 1e-16 * a; ++it) {
    const double an = 0.5 * (a + b);
    b = std::sqrt(a * b);
    a = an;
  }
  return M_PI / (a + b);
}

// sn, cn, dn(u|m) by the descending arithmetic-geometric mean (Abramowitz and Stegun 16.4):
// a_0 = 1, b_0 = sqrt(1-m), c_0 = sqrt(m); a_n, b_n the AGM steps, c_n = (a_{n-1} - b_{n-1})/2
// until c_N is negligible; phi_N = 2^N a_N u and phi_{n-1} = (phi_n + asin(c_n sin(phi_n)/a_n))/2;
// sn = sin phi_0, cn = cos phi_0, dn = cos phi_0 / cos(phi_1 - phi_0).
void ellip_j(double u, double m, double* sn, double* cn, double* dn) {
  if (m <= 0.0) {
    *sn = std::sin(u);
    *cn = std::cos(u);
    *dn = 1.0;
    return;
  }
  double a[40], c[40];
  a[0] = 1.0;
  double b = std::sqrt(1.0 - m);
  c[0] = std::sqrt(m);
  int n = 0;
  while (n < 38 && std::fabs(c[n]) > 1e-16) {
    a[n + 1] = 0.5 * (a[n] + b);
    c[n + 1] = 0.5 * (a[n] - b);
    b = std::sqrt(a[n] * b);
    ++n;
  }
  double phi = std::ldexp(a[n] * u, n);
  double prev = phi;
  for (int j = n; j >= 1; --j) {
    prev = phi;
    phi = 0.5 * (phi + std::asin(c[j] * std::sin(phi) / a[j]));
  }
  *sn = std::sin(phi);
  *cn = std::cos(phi);
  *dn = n >= 1 ? *cn / std::cos(prev - phi) : 1.0;
}

}  // namespace
}  // namespace sf

using namespace sf;

struct s_selinv_t {
  const s_pattern_t* S = nullptr;
  int32_t m = 0, height = 0, maxb = 0;
  int64_t nl = 0, nent = 0, nterms = 0;
  double flops_factor = 0.0, flops_invert = 0.0;
  // level lists (host offsets into the device arrays)
  std::vector<int64_t> upd_ptr, off_ptr, sn_ptr;
  std::vector<int32_t> lvl_slices;  // pivot CTAs per supernode on each level
  std::vector<int64_t> lvl_ent;     // entries of the blocks of each level's columns
  std::vector<int32_t> upd_split, off_split;  // parts of the update and off-diagonal sums
  unsigned int* cnt = nullptr;      // per supernode: slices of the diagonal kernel finished
  double* Q = nullptr;              // slice sums of the diagonal kernel
  // device
  int32_t* bs = nullptr;
  int64_t* colptr = nullptr;
  int32_t* colrow = nullptr;
  int64_t* loff = nullptr;
  int32_t* colcol = nullptr;
  int64_t* uptr = nullptr;
  int32_t* uw = nullptr;
  int32_t* ul = nullptr;
  int64_t* optr = nullptr;
  int32_t* oz = nullptr;
  int32_t* ol = nullptr;
  int64_t* aoff = nullptr;
  int64_t* lpo = nullptr;
  double* P = nullptr;
  SiItem* upd = nullptr;
  SiItem* off = nullptr;
  int32_t* sn = nullptr;
  int32_t* s2l = nullptr;
  int8_t* s2t = nullptr;
  double* W = nullptr;
  double* L = nullptr;
  double* Z = nullptr;
  unsigned int* flag = nullptr;
  unsigned int* flag_host = nullptr;
};

static void selinv_free(s_selinv_t* p) {
  cudaFree(p->bs);
  cudaFree(p->colptr);
  cudaFree(p->colrow);
  cudaFree(p->loff);
  cudaFree(p->colcol);
  cudaFree(p->uptr);
  cudaFree(p->uw);
  cudaFree(p->ul);
  cudaFree(p->optr);
  cudaFree(p->oz);
  cudaFree(p->ol);
  cudaFree(p->aoff);
  cudaFree(p->lpo);
  cudaFree(p->P);
  cudaFree(p->cnt);
  cudaFree(p->Q);
  cudaFree(p->upd);
  cudaFree(p->off);
  cudaFree(p->sn);
  cudaFree(p->s2l);
  cudaFree(p->s2t);
  cudaFree(p->W);
  cudaFree(p->L);
  cudaFree(p->Z);
  if (p->flag_host) cudaFreeHost(p->flag_host);
}

static SiDev dev_of(const s_selinv_t* p) {
  SiDev s;
  s.bs = p->bs;
  s.colptr = p->colptr;
  s.colrow = p->colrow;
  s.loff = p->loff;
  s.colcol = p->colcol;
  s.uptr = p->uptr;
  s.uw = p->uw;
  s.ul = p->ul;
  s.optr = p->optr;
  s.oz = p->oz;
  s.ol = p->ol;
  s.aoff = p->aoff;
  s.lpo = p->lpo;
  s.W = p->W;
  s.L = p->L;
  s.Z = p->Z;
  s.P = p->P;
  s.flag = p->flag;
  s.maxb = p->maxb;
  return s;
}

static s_status selinv_build(s_selinv_t* p) {
  const s_pattern_t* S = p->S;
  const int32_t nc = (int32_t)S->bsize.size();
  Symbolic sy;
  s_status st = symbolic(nc, S->rowptr.data(), S->colidx.data(), S->bsize.data(), &sy);
  if (st) return st;
  const int32_t m = sy.m;
  p->m = m;
  std::vector<int32_t> lvl = etree_levels(sy, &p->height);
  std::vector<int32_t> bs(std::max(m, 1), 0);
  for (int32_t q = 0; q < m; ++q) {
    bs[q] = S->bsize[sy.perm[q]];
    if (bs[q] > kSiMaxB) return set_error(S_ERR_ARG, "selected inversion: blocks wider than 64");
    p->maxb = std::max(p->maxb, bs[q]);
  }
  // CSC of L
  std::vector<int64_t> colptr(m + 1, 0), loff;
  std::vector<int32_t> colrow;
  for (int32_t k = 0; k < m; ++k) colptr[k + 1] = colptr[k] + 1 + (int64_t)sy.st[k].size();
  const int64_t nl = colptr[m];
  if (nl >= INT32_MAX) return set_error(S_ERR_ARG, "selected inversion: factor has more than 2^31 blocks");
  colrow.reserve(nl);
  loff.reserve(nl + 1);
  int64_t e = 0;
  double ff = 0.0, fi = 0.0;
  for (int32_t k = 0; k < m; ++k) {
    colrow.push_back(k);
    loff.push_back(e);
    e += (int64_t)bs[k] * bs[k];
    double T = 0.0, T2 = 0.0;
    for (int32_t i : sy.st[k]) {
      colrow.push_back(i);
      loff.push_back(e);
      e += (int64_t)bs[i] * bs[k];
      T += bs[i];
      T2 += (double)bs[i] * bs[i];
    }
    const double b = bs[k];
    // update pairs (i >= i') of struct(k) and the pivot; inversion: struct(k) x struct(k)
    ff += b * (T * T + T2) + 2.0 * b * b * b + 2.0 * b * b * T;
    fi += 2.0 * b * T * T + 2.0 * b * b * T;
  }
  loff.push_back(e);
  p->nl = nl;
  p->nent = e;
  p->flops_factor = ff;
  p->flops_invert = fi;
  // CSR of L: row i holds its columns ascending (the diagonal last)
  std::vector<int64_t> rowptr(m + 1, 0);
  for (int64_t q = 0; q < nl; ++q) ++rowptr[colrow[q] + 1];
  for (int32_t i = 0; i < m; ++i) rowptr[i + 1] += rowptr[i];
  std::vector<int32_t> rowcol(nl), rowblk(nl);
  {
    std::vector<int64_t> fill(rowptr.begin(), rowptr.end() - 1);
    for (int32_t k = 0; k < m; ++k)
      for (int64_t q = colptr[k]; q < colptr[k + 1]; ++q) {
        const int32_t i = colrow[q];
        rowcol[fill[i]] = k;
        rowblk[fill[i]] = (int32_t)q;
        ++fill[i];
      }
  }
  // S blocks of each L block, and L blocks of each S block
  std::vector<int64_t> aoff(nl, -1);
  const int64_t snb = (int64_t)S->colidx.size();
  std::vector<int32_t> s2l(std::max<int64_t>(snb, 1), -1);
  std::vector<int8_t> s2t(std::max<int64_t>(snb, 1), 0);
  for (int32_t r = 0; r < nc; ++r) {
    for (int64_t b = S->rowptr[r]; b < S->rowptr[r + 1]; ++b) {
      const int32_t c = S->colidx[b];
      const int32_t pr = sy.pos[r], pc = sy.pos[c];
      if (pr < 0 || pc < 0) continue;
      const int32_t hi = std::max(pr, pc), lo = std::min(pr, pc);
      const int32_t* f = std::lower_bound(colrow.data() + colptr[lo], colrow.data() + colptr[lo + 1], hi);
      if (f == colrow.data() + colptr[lo + 1] || *f != hi)
        return set_error(S_ERR_PATTERN, "selected inversion: internal error, S not inside the factor");
      const int64_t q = f - colrow.data();
      s2l[b] = (int32_t)q;
      s2t[b] = pr < pc ? 1 : 0;
      if (pr >= pc) aoff[q] = S->voff[b];
    }
  }
  for (int32_t k = 0; k < m; ++k)
    if (aoff[colptr[k]] < 0) return set_error(S_ERR_PATTERN, "selected inversion: pattern lacks a diagonal block");
  // Term lists of both sweeps (fixed by the pattern of L), per CSC block q = (i,k):
  //   factor:    the j < k in both row i and row k of L, as CSC blocks W(i,j), L(k,j);
  //   inversion: (i > k) for every j in struct(k), the block holding Z(i,j) (~index when it is
  //              stored as Z(j,i)) and the block L(j,k).
  std::vector<int64_t> uptr(nl + 1, 0), optr(nl + 1, 0);
  std::vector<int32_t> uw, ul, oz, ol, colcol(nl);
  for (int32_t k = 0; k < m; ++k) {
    const int64_t rk0 = rowptr[k], rk1 = rowptr[k + 1] - 1;  // row k below its diagonal
    for (int64_t q = colptr[k]; q < colptr[k + 1]; ++q) {
      const int32_t i = colrow[q];
      colcol[q] = k;
      for (int64_t a = rowptr[i], ae = rowptr[i + 1], b = rk0; a < ae && b < rk1 && rowcol[a] < k;) {
        if (rowcol[a] < rowcol[b]) {
          ++a;
        } else if (rowcol[b] < rowcol[a]) {
          ++b;
        } else {
          uw.push_back(rowblk[a]);
          ul.push_back(rowblk[b]);
          ++a;
          ++b;
        }
      }
      uptr[q + 1] = (int64_t)uw.size();
      if (q > colptr[k]) {
        int64_t ra = rowptr[i], ca = colptr[i] + 1;
        const int64_t re = rowptr[i + 1], ce = colptr[i + 1];
        for (int64_t qq = colptr[k] + 1; qq < colptr[k + 1]; ++qq) {
          const int32_t j = colrow[qq];
          int32_t zb;
          if (j < i) {
            while (ra < re && rowcol[ra] < j) ++ra;
            if (ra == re || rowcol[ra] != j) return set_error(S_ERR_PATTERN, "selected inversion: internal error");
            zb = rowblk[ra];
          } else if (j == i) {
            zb = (int32_t)colptr[i];
          } else {
            while (ca < ce && colrow[ca] < j) ++ca;
            if (ca == ce || colrow[ca] != j) return set_error(S_ERR_PATTERN, "selected inversion: internal error");
            zb = ~(int32_t)ca;
          }
          oz.push_back(zb);
          ol.push_back((int32_t)qq);
        }
      }
      optr[q + 1] = (int64_t)oz.size();
    }
  }
  p->nterms = (int64_t)uw.size() + (int64_t)oz.size();
  // level lists, level-local entry offsets, and the split of each level's long sums
  const int32_t H = p->height;
  std::vector<std::vector<int32_t>> bylvl(H);
  for (int32_t k = 0; k < m; ++k) bylvl[lvl[k]].push_back(k);
  std::vector<SiItem> upd, off;
  std::vector<int32_t> sn;
  std::vector<int64_t> lpo(nl, 0);
  p->upd_ptr.assign(1, 0);
  p->off_ptr.assign(1, 0);
  p->sn_ptr.assign(1, 0);
  p->lvl_slices.assign(H, 1);
  p->lvl_ent.assign(H, 0);
  p->upd_split.assign(H, 1);
  p->off_split.assign(H, 1);
  const int64_t target = 16LL * kSiWarps * sm_count();  // sixteen warps per SM sub-partition
  int64_t scratch = 0, qneed = 0;
  for (int32_t l = 0; l < H; ++l) {
    int64_t longest = 0, ent = 0, maxu = 0, maxo = 0;
    const int64_t u0 = (int64_t)upd.size(), o0 = (int64_t)off.size();
    for (int32_t k : bylvl[l]) {
      sn.push_back(k);
      longest = std::max<int64_t>(longest, colptr[k + 1] - colptr[k] - 1);
      for (int64_t q = colptr[k]; q < colptr[k + 1]; ++q) {
        maxu = std::max<int64_t>(maxu, uptr[q + 1] - uptr[q]);
        maxo = std::max<int64_t>(maxo, optr[q + 1] - optr[q]);
        const int ne = bs[colrow[q]] * bs[k];
        lpo[q] = ent;
        ent += ne;
        for (int e0 = 0; e0 < ne; e0 += kSiTileEnt) {
          upd.push_back(SiItem{(int32_t)q, k, e0});
          if (q > colptr[k]) off.push_back(SiItem{(int32_t)q, k, e0});
        }
      }
    }
    const int64_t nu = (int64_t)upd.size() - u0, no = (int64_t)off.size() - o0;
    auto choose = [&](int64_t items, int64_t terms) {  // parts of at least kSiPartTerms terms
      int64_t sp = items > 0 ? (target + items - 1) / items : 1;
      sp = std::min<int64_t>(sp, std::min<int64_t>(kSiMaxSplit, (terms + kSiPartTerms - 1) / kSiPartTerms));
      while (sp > 1 && sp * ent > (int64_t)1 << 27) --sp;  // scratch at most 1 GiB
      return (int32_t)std::max<int64_t>(1, sp);
    };
    p->upd_split[l] = choose(nu, maxu);
    p->off_split[l] = choose(no, maxo);
    const int32_t sp = std::max(p->upd_split[l], p->off_split[l]);
    if (sp > 1) scratch = std::max<int64_t>(scratch, (int64_t)sp * ent);
    p->lvl_ent[l] = ent;
    p->lvl_slices[l] = (int32_t)std::max<int64_t>(1, (longest + kSiSlice - 1) / kSiSlice);
    if (p->lvl_slices[l] > 1)
      qneed = std::max<int64_t>(qneed, (int64_t)bylvl[l].size() * p->lvl_slices[l] * p->maxb * p->maxb);
    p->upd_ptr.push_back((int64_t)upd.size());
    p->off_ptr.push_back((int64_t)off.size());
    p->sn_ptr.push_back((int64_t)sn.size());
  }
  if ((st = upload(&p->bs, bs)) || (st = upload(&p->colptr, colptr)) || (st = upload(&p->colrow, colrow)) ||
      (st = upload(&p->loff, loff)) || (st = upload(&p->colcol, colcol)) || (st = upload(&p->uptr, uptr)) ||
      (st = upload(&p->uw, uw)) || (st = upload(&p->ul, ul)) || (st = upload(&p->optr, optr)) ||
      (st = upload(&p->oz, oz)) || (st = upload(&p->ol, ol)) || (st = upload(&p->aoff, aoff)) ||
      (st = upload(&p->lpo, lpo)) ||
      (st = upload(&p->upd, upd)) ||
      (st = upload(&p->off, off)) || (st = upload(&p->sn, sn)) || (st = upload(&p->s2l, s2l)) ||
      (st = upload(&p->s2t, s2t)))
    return st;
  const size_t vb = sizeof(double) * (size_t)std::max<int64_t>(e, 1);
  cudaError_t ce = cudaMalloc(&p->W, vb);
  if (ce == cudaSuccess) ce = cudaMalloc(&p->L, vb);
  if (ce == cudaSuccess) ce = cudaMalloc(&p->Z, vb);
  if (ce == cudaSuccess && scratch > 0) ce = cudaMalloc(&p->P, sizeof(double) * (size_t)scratch);
  if (ce == cudaSuccess && qneed > 0) ce = cudaMalloc(&p->Q, sizeof(double) * (size_t)qneed);
  if (ce == cudaSuccess) ce = cudaMalloc(&p->cnt, sizeof(unsigned int) * (size_t)std::max(m, 1));
  if (ce == cudaSuccess) ce = cudaMemset(p->cnt, 0, sizeof(unsigned int) * (size_t)std::max(m, 1));
  if (ce == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return set_error(S_ERR_NOMEM, "selected inversion: no device memory for the factor");
  }
  SF_CUDA(ce);
  SF_CUDA(cudaHostAlloc((void**)&p->flag_host, sizeof(unsigned int), cudaHostAllocMapped));
  *(volatile unsigned int*)p->flag_host = 0u;
  SF_CUDA(cudaHostGetDevicePointer((void**)&p->flag, p->flag_host, 0));
  return S_OK;
}

extern "C" {

s_status s_selinv_order(int32_t n_clusters, const int64_t* rowptr, const int32_t* colidx, const int32_t* bsize,
                        int32_t* perm, int64_t* l_blocks, int32_t* levels) {
  if (n_clusters < 1 || !rowptr || !colidx || !bsize || !perm)
    return set_error(S_ERR_ARG, "s_selinv_order: null argument or no clusters");
  if (rowptr[0] != 0) return set_error(S_ERR_PATTERN, "s_selinv_order: rowptr[0] != 0");
  for (int32_t r = 0; r < n_clusters; ++r)
    if (rowptr[r + 1] < rowptr[r]) return set_error(S_ERR_PATTERN, "s_selinv_order: rowptr decreases");
  Symbolic sy;
  s_status st;
  try {
    st = symbolic(n_clusters, rowptr, colidx, bsize, &sy);
  } catch (const std::bad_alloc&) {
    st = set_error(S_ERR_NOMEM, "s_selinv_order: host memory exhausted");
  }
  if (st) return st;
  std::memcpy(perm, sy.perm.data(), sizeof(int32_t) * n_clusters);
  int64_t nl = sy.m;
  for (const auto& s : sy.st) nl += (int64_t)s.size();
  if (l_blocks) *l_blocks = nl;
  int32_t h = 0;
  etree_levels(sy, &h);
  if (levels) *levels = h;
  return S_OK;
}

s_status s_selinv_create(s_pattern S, s_selinv* out) {
  if (!S || !out) return set_error(S_ERR_ARG, "s_selinv_create: null argument");
  s_selinv_t* p = new s_selinv_t();
  p->S = S;
  s_status st;
  try {
    st = selinv_build(p);
  } catch (const std::bad_alloc&) {
    st = set_error(S_ERR_NOMEM, "selected inversion: host memory exhausted in the symbolic analysis");
  }
  if (st) {
    selinv_free(p);
    delete p;
    return st;
  }
  *out = p;
  return S_OK;
}

s_status s_selinv_destroy(s_selinv p) {
  if (!p) return S_OK;
  selinv_free(p);
  delete p;
  return S_OK;
}

s_status s_selinv_stats(s_selinv p, int64_t* l_blocks, int64_t* l_entries, int32_t* levels, double* flops_factor,
                        double* flops_invert) {
  if (!p) return set_error(S_ERR_ARG, "s_selinv_stats: null plan");
  if (l_blocks) *l_blocks = p->nl;
  if (l_entries) *l_entries = p->nent;
  if (levels) *levels = p->height;
  if (flops_factor) *flops_factor = p->flops_factor;
  if (flops_invert) *flops_invert = p->flops_invert;
  return S_OK;
}

// Dynamic shared memory of the block kernels (per-warp staging of two operand slices, and
// the diagonal kernel's warp sums) and of the pivot kernel (D^{-1} and one W block).
static size_t stage_bytes(const s_selinv_t* p) {  // two stage buffers per warp
  return sizeof(double) * (size_t)kSiWarps * 4 * p->maxb * kSiUp;
}
static size_t diag_bytes(const s_selinv_t* p) {  // one stage buffer per warp and the warp sums
  return sizeof(double) * ((size_t)kSiWarps * 2 * p->maxb * kSiUp + (size_t)kSiWarps * kSiTileEnt);
}
static size_t pivot_bytes(const s_selinv_t* p) { return sizeof(double) * 2 * (size_t)p->maxb * p->maxb; }

static s_status set_smem(const void* fn, size_t bytes) {
  if (bytes > 48 * 1024) SF_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return S_OK;
}

s_status s_selinv_factor(s_selinv p, const double* A, double sigma, void* stream) {
  if (!p || (!A && p->S->d.nnz > 0)) return set_error(S_ERR_ARG, "s_selinv_factor: null argument");
  if (p->m == 0) return S_OK;
  cudaStream_t cs = (cudaStream_t)stream;
  const SiDev s = dev_of(p);
  s_status st;
  if ((st = set_smem((const void*)si_update_kernel, stage_bytes(p))) ||
      (st = set_smem((const void*)si_pivot_kernel, pivot_bytes(p))))
    return st;
  for (int32_t l = 0; l < p->height; ++l) {
    const int64_t n = p->upd_ptr[l + 1] - p->upd_ptr[l];
    const int split = p->upd_split[l];
    if (n > 0) {
      const int64_t grid = (n * split + kSiWarps - 1) / kSiWarps;
      si_update_kernel<<<(unsigned)grid, kSiWarps * 32, stage_bytes(p), cs>>>(s, p->upd + p->upd_ptr[l], n, split,
                                                                              p->lvl_ent[l], A, sigma);
    }
    const int64_t ns = p->sn_ptr[l + 1] - p->sn_ptr[l];
    if (ns > 0) {
      dim3 g((unsigned)ns, (unsigned)p->lvl_slices[l]);
      si_pivot_kernel<<<g, kSiThreads, pivot_bytes(p), cs>>>(s, p->sn + p->sn_ptr[l], n > 0 ? split : 1,
                                                             p->lvl_ent[l]);
    }
  }
  SF_CUDA(cudaGetLastError());
  return S_OK;
}

s_status s_selinv_invert(s_selinv p, double alpha, double beta, double* out, void* stream) {
  if (!p || (!out && p->S->d.nnz > 0)) return set_error(S_ERR_ARG, "s_selinv_invert: null argument");
  cudaStream_t cs = (cudaStream_t)stream;
  if (p->m > 0) {
    const SiDev s = dev_of(p);
    s_status st;
    if ((st = set_smem((const void*)si_offdiag_kernel, stage_bytes(p))) ||
        (st = set_smem((const void*)si_diag_kernel, diag_bytes(p))))
      return st;
    SF_CUDA(cudaMemsetAsync(p->cnt, 0, sizeof(unsigned int) * (size_t)p->m, cs));
    for (int32_t l = p->height - 1; l >= 0; --l) {
      const int64_t n = p->off_ptr[l + 1] - p->off_ptr[l];
      const int split = n > 0 ? p->off_split[l] : 1;
      if (n > 0) {
        const int64_t grid = (n * split + kSiWarps - 1) / kSiWarps;
        si_offdiag_kernel<<<(unsigned)grid, kSiWarps * 32, stage_bytes(p), cs>>>(s, p->off + p->off_ptr[l], n,
                                                                                 split, p->lvl_ent[l]);
      }
      const int64_t ns = p->sn_ptr[l + 1] - p->sn_ptr[l];
      if (ns > 0) {
        dim3 g((unsigned)ns, (unsigned)p->lvl_slices[l]);
        si_diag_kernel<<<g, kSiWarps * 32, diag_bytes(p), cs>>>(s, p->sn + p->sn_ptr[l], split, p->lvl_ent[l],
                                                                p->lvl_slices[l], p->cnt, p->Q);
      }
    }
  }
  const DevPattern& d = p->S->d;
  if (d.nblocks > 0) {
    const int64_t grid = std::min<int64_t>((d.nblocks * 32 + 255) / 256, (int64_t)sm_count() * 8);
    si_scatter_kernel<<<(unsigned)std::max<int64_t>(grid, 1), 256, 0, cs>>>(
        d.nblocks, d.bsize, d.brow, d.colidx, d.voff, p->s2l, p->s2t, p->loff, p->Z, alpha, beta, out);
  }
  SF_CUDA(cudaGetLastError());
  return S_OK;
}

s_status s_selinv_status(s_selinv p, void* stream) {
  if (!p) return set_error(S_ERR_ARG, "s_selinv_status: null plan");
  SF_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  volatile unsigned int* w = p->flag_host;
  if (w && *w) {
    *w = 0u;
    return set_error(S_ERR_NOT_SPD, "selected inversion: a pivot block was not positive definite");
  }
  return S_OK;
}

s_status s_contour_nodes(double c_lo, double c_hi, int32_t n, double* shifts, double* weights) {
  if (!(c_lo > 0.0) || !(c_hi >= c_lo) || !std::isfinite(c_hi) || n < 1 || !shifts || !weights)
    return set_error(S_ERR_ARG, "s_contour_nodes: need 0 < c_lo <= c_hi and n >= 1");
  const double m = 1.0 - c_lo / c_hi;
  const double K = ellip_k(m);
  const double sc = std::sqrt(c_lo);
  for (int32_t k = 0; k < n; ++k) {
    const double t = K * (k + 0.5) / n;
    double sn, cn, dn;
    ellip_j(t, m, &sn, &cn, &dn);
    const double w = sc * sn / cn;
    shifts[k] = w * w;
    weights[k] = 2.0 * K * sc / (M_PI * n) * dn / (cn * cn);
  }
  return S_OK;
}

s_status s_selinv_invsqrt(s_selinv p, const double* A, double c_lo, double c_hi, int32_t n, double* out,
                          void* stream) {
  if (!p || n < 1 || n > 1024) return set_error(S_ERR_ARG, "s_selinv_invsqrt: null plan or n outside 1..1024");
  std::vector<double> w2(n), wt(n);
  s_status st = s_contour_nodes(c_lo, c_hi, n, w2.data(), wt.data());
  if (st) return st;
  for (int32_t k = 0; k < n; ++k) {
    if ((st = s_selinv_factor(p, A, w2[k], stream))) return st;
    if ((st = s_selinv_invert(p, wt[k], k ? 1.0 : 0.0, out, stream))) return st;
  }
  return s_selinv_status(p, stream);
}

}  // extern "C"
