// Input preparation on the device: K^eta = P_S(T K T^T) (Thm. (S-compression)) for a
// Matern kernel (Sec. 2), exactly (all N^2 kernel evaluations) in float arithmetic, with
// the a-posteriori threshold of Sec. 5.  Not on the hot path.
//
// Columns are processed in chunks: a chunk is a maximal cluster g with at most kChunk
// points.  For a chunk, U = K(all points, points of g) (N x |g|, tree order) is evaluated
// and transformed in place by the two-scale matrices Q of Eq. (QR): first along the
// columns inside g's subtree, then along all rows, level by level (the "slots" of a
// cluster are the rows/columns its transform reads and writes).  Afterwards U holds
// T K T_g^T: every block (a, b) of the pattern with b in g's subtree and a <= b is copied
// to an upper-triangle staging buffer together with its largest |entry|.  g's scaling
// columns are kept for the clusters above the chunks, which are then transformed and
// extracted the same way from the sons' scaling columns.  Finally the kept pattern is
// decided per unordered block pair and the values are assembled in double.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "build_internal.h"
#include "common.cuh"

namespace sf {

constexpr int kChunk = 1024;   // columns per chunk
constexpr int kRowTile = 8;    // rows per CTA of the evaluation kernel
constexpr int kColTile = 128;  // columns per CTA of the row transform
constexpr int kMaxIn = 64;     // largest n_in handled by the transform kernels

struct Geo {
  const float* x;          // N x 3 points in tree order
  const float* Q;          // all Q matrices, float, row-major nin x nin at qoff[c]
  const int64_t* qoff;
  const int32_t* slots;    // tree-order positions, slot_off[c] .. + nin(c)
  const int64_t* slot_off;
  const int32_t* nin;
  const int32_t* ns;
};

__device__ __forceinline__ float matern(float r, int p, float inv_ell, float scale) {
  // half-integer closed form, Sec. 2: nu = p + 1/2; p >= 3 encodes d/dell of nu = (p-3) + 1/2
  if (p >= 3) {
    // kappa = f(t), t = sqrt(2 nu) r / ell, dkappa/dell = -f'(t) t / ell
    const int q = p - 3;
    const float a = q == 0 ? 1.0f : (q == 1 ? 1.7320508075688772f : 2.23606797749979f);
    const float t = a * r * inv_ell;
    const float e = __expf(-t);
    float g;  // -f'(t) * t
    if (q == 0) g = t * e;
    else if (q == 1) g = t * t * e;
    else g = t * t * (1.0f + t) * (1.0f / 3.0f) * e;
    return scale * g * inv_ell;
  }
  if (p == 0) return scale * __expf(-r * inv_ell);
  if (p == 1) {
    const float t = 1.7320508075688772f * r * inv_ell;
    return scale * (1.0f + t) * __expf(-t);
  }
  const float t = 2.23606797749979f * r * inv_ell;
  return scale * (1.0f + t + t * t * (1.0f / 3.0f)) * __expf(-t);
}

// K(rows i0.., chunk columns) into shared memory, then the column transforms of every
// cluster of the chunk's subtree (bottom-up), then the tile to U (row-major N x w).
__global__ void eval_colfwt_kernel(Geo g, int64_t n, int64_t q0, int w, const int32_t* sub, const int32_t* sub_lvl_off,
                                   int nlev, int p, float inv_ell, float scale, int maxm, float* U) {
  extern __shared__ float tile[];  // kRowTile x w, then per warp Q (maxm^2) and slots (maxm)
  const int64_t i0 = (int64_t)blockIdx.x * kRowTile;
  const int rows = (int)min((int64_t)kRowTile, n - i0);
  for (int e = threadIdx.x; e < kRowTile * w; e += blockDim.x) {
    const int r = e / w, j = e - r * w;
    float v = 0.0f;
    if (r < rows) {
      const float* xi = g.x + (i0 + r) * 3;
      const float* xj = g.x + (q0 + j) * 3;
      const float dx = xi[0] - xj[0], dy = xi[1] - xj[1], dz = xi[2] - xj[2];
      v = matern(sqrtf(dx * dx + dy * dy + dz * dz), p, inv_ell, scale);
    }
    tile[e] = v;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  // per warp: the cluster's Q (m x m) and slots, staged once and applied to every row
  float* qs = tile + kRowTile * w + warp * (maxm * maxm + maxm);
  int* ss = reinterpret_cast<int*>(qs + maxm * maxm);
  for (int L = 0; L < nlev; ++L) {  // sub is ordered deepest level first
    const int c0 = sub_lvl_off[L], c1 = sub_lvl_off[L + 1];
    for (int ci = c0 + warp; ci < c1; ci += nwarp) {
      const int c = sub[ci];
      const int m = g.nin[c];
      const int32_t* sl = g.slots + g.slot_off[c];
      const float* Q = g.Q + g.qoff[c];
      for (int e = lane; e < m * m; e += 32) qs[e] = Q[e];
      for (int e = lane; e < m; e += 32) ss[e] = sl[e] - (int)q0;
      __syncwarp();
      for (int r = 0; r < rows; ++r) {
        float* row = tile + r * w;
        float o0 = 0.0f, o1 = 0.0f;
        for (int ii = 0; ii < m; ++ii) {
          const float in = row[ss[ii]];
          if (lane < m) o0 = fmaf(in, qs[ii * m + lane], o0);
          if (lane + 32 < m) o1 = fmaf(in, qs[ii * m + lane + 32], o1);
        }
        __syncwarp();
        if (lane < m) row[ss[lane]] = o0;
        if (lane + 32 < m) row[ss[lane + 32]] = o1;
        __syncwarp();
      }
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < rows * w; e += blockDim.x) U[(i0 + e / w) * w + e % w] = tile[e];
}

// In-place row transform of one level: rows slots(c) of U (ld w) <- Q_c^T rows.
__global__ void rowfwt_kernel(Geo g, const int32_t* lvl, int w, float* U) {
  __shared__ float in[kMaxIn][kColTile];
  __shared__ float Qs[kMaxIn * kMaxIn];
  const int c = lvl[blockIdx.x];
  const int j0 = blockIdx.y * kColTile;
  const int cols = min(kColTile, w - j0);
  const int m = g.nin[c];
  const int32_t* sl = g.slots + g.slot_off[c];
  const float* Q = g.Q + g.qoff[c];
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) Qs[e] = Q[e];
  for (int e = threadIdx.x; e < m * kColTile; e += blockDim.x) {
    const int ii = e / kColTile, j = e - ii * kColTile;
    in[ii][j] = j < cols ? U[(int64_t)sl[ii] * w + j0 + j] : 0.0f;
  }
  __syncthreads();
  const int j = threadIdx.x % kColTile;
  for (int jj = threadIdx.x / kColTile; jj < m; jj += blockDim.x / kColTile) {
    float s = 0.0f;
    for (int ii = 0; ii < m; ++ii) s = fmaf(Qs[ii * m + jj], in[ii][j], s);
    if (j < cols) U[(int64_t)sl[jj] * w + j0 + j] = s;
  }
}

// In-place column transform of an N x m matrix G (row-major): G[r,:] <- G[r,:] Q.
__global__ void colfwt_rows_kernel(int64_t n, int m, const float* Q, float* G) {
  __shared__ float Qs[kMaxIn * kMaxIn];
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) Qs[e] = Q[e];
  __syncthreads();
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n) return;
  float in[kMaxIn];
  for (int ii = 0; ii < m; ++ii) in[ii] = G[r * m + ii];
  for (int jj = 0; jj < m; ++jj) {
    float s = 0.0f;
    for (int ii = 0; ii < m; ++ii) s = fmaf(in[ii], Qs[ii * m + jj], s);
    G[r * m + jj] = s;
  }
}

// Extraction: entry e = block (a, b): staging[off + i*nb + j] = Src[rowslot[boff[a]+i], col[j]]
// with col[j] = colmap[cm_off[e] + j] - q0; bmax[k] = max |entry|.  One warp per entry.
struct Ext {
  const int32_t* a;
  const int32_t* b;
  const int64_t* off;   // staging offset
  const int32_t* k;     // upper-triangle block id (for bmax)
  const int32_t* cm;    // column map base index of each entry into colmap
};

__global__ void extract_kernel(Ext ex, int64_t nent, const int32_t* bsize, const int64_t* boff,
                               const int32_t* rowslot, const int32_t* colmap, int64_t q0, const float* Src,
                               int64_t ld, float* staging, float* bmax) {
  const int lane = threadIdx.x & 31;
  const int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (e >= nent) return;
  const int a = ex.a[e], b = ex.b[e];
  const int na = bsize[a], nb = bsize[b];
  const int32_t* cm = colmap + ex.cm[e];
  float* dst = staging + ex.off[e];
  float mx = 0.0f;
  for (int t = lane; t < na * nb; t += 32) {
    const int i = t / nb, j = t - i * nb;
    const float v = Src[(int64_t)rowslot[boff[a] + i] * ld + (cm[j] - q0)];
    dst[t] = v;
    mx = fmaxf(mx, fabsf(v));
  }
  for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) bmax[ex.k[e]] = mx;
}

// U[:, cols] -> S (N x m, row-major)
__global__ void gather_cols_kernel(int64_t n, int m, const int32_t* cols, int64_t q0, const float* U, int w,
                                   float* S) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * m) return;
  const int64_t r = t / m;
  const int j = (int)(t - r * m);
  S[t] = U[r * w + (cols[j] - q0)];
}

// concatenate two N x m0 / N x m1 row-major blocks into G (N x (m0+m1))
__global__ void concat_kernel(int64_t n, int m0, const float* A, int m1, const float* B, float* G) {
  const int m = m0 + m1;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * m) return;
  const int64_t r = t / m;
  const int j = (int)(t - r * m);
  G[t] = j < m0 ? A[r * m0 + j] : B[r * m1 + (j - m0)];
}

// Final values: block (a, b) of the kept pattern from the staged block of the pair, the
// nugget on the diagonal, entries below tau set to zero.
__global__ void assemble_kernel(int64_t nblk, const int32_t* brow, const int32_t* bcol, const int64_t* voff,
                                const int64_t* src_off, const int32_t* bsize, const float* staging, double nugget,
                                double tau, double* out) {
  const int lane = threadIdx.x & 31;
  const int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (k >= nblk) return;
  const int a = brow[k], b = bcol[k];
  const int na = bsize[a], nb = bsize[b];
  const float* s = staging + src_off[k];
  double* o = out + voff[k];
  for (int t = lane; t < na * nb; t += 32) {
    const int i = t / nb, j = t - i * nb;
    double v = a <= b ? (double)s[t] : (double)s[j * na + i];  // staged block is (min, max)
    if (a == b && i == j) v += nugget;
    o[t] = fabs(v) < tau ? 0.0 : v;
  }
}

template <typename T>
static s_status dmalloc(T** p, size_t count) {
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * std::max<size_t>(count, 1));
  if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(build values)");
  return S_OK;
}

template <typename T>
static s_status upload(T** p, const std::vector<T>& v) {
  s_status st = dmalloc(p, v.size());
  if (st) return st;
  if (!v.empty()) SF_CUDA(cudaMemcpy(*p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
  return S_OK;
}

struct Frees {
  std::vector<void*> ptrs;
  void add(void* p) { ptrs.push_back(p); }
  ~Frees() {
    for (void* p : ptrs) cudaFree(p);
  }
};

}  // namespace sf

using namespace sf;

s_build_t::~s_build_t() { cudaFree(dvals); }

// Values of the kernel (deriv = false) or of its ell-derivative (deriv = true).  Without a
// given pattern the kept pattern is decided by tau and returned in *pattern with the values
// held by the builder; with a given pattern (a sub-pattern of the eta pattern) the values on
// it are written to `out` (no threshold, no nugget).
static s_status values_impl(s_build b, double nu, double ell, double kscale, double nugget, double tau, bool deriv,
                            const s_pattern_t* given, double* out, s_pattern* pattern) {
  int p;
  if (std::fabs(nu - 0.5) < 1e-12) p = 0;
  else if (std::fabs(nu - 1.5) < 1e-12) p = 1;
  else if (std::fabs(nu - 2.5) < 1e-12) p = 2;
  else return set_error(S_ERR_ARG, "s_build_values: nu must be 0.5, 1.5 or 2.5");
  if (!(ell > 0.0)) return set_error(S_ERR_ARG, "s_build_values: ell must be positive");
  if (deriv) p += 3;
  const int64_t n = b->n;
  const int nc = (int)b->cl.size();
  for (const auto& c : b->cl)
    if (c.nin > kMaxIn) return set_error(S_ERR_ARG, "s_build_values: a cluster has more than 64 inputs");
  Frees fr;
  s_status st;
  // ---- geometry and transforms on the device ----------------------------------------
  std::vector<float> xf((size_t)n * 3, 0.0f);
  for (int64_t i = 0; i < n; ++i)
    for (int a = 0; a < b->d; ++a) xf[i * 3 + a] = (float)b->points[b->perm[i] * b->d + a];
  std::vector<int64_t> qoff(nc + 1, 0);
  for (int c = 0; c < nc; ++c) qoff[c + 1] = qoff[c] + (int64_t)b->cl[c].nin * b->cl[c].nin;
  std::vector<float> qf(qoff[nc]);
  std::vector<int32_t> nin(nc), ns(nc);
  for (int c = 0; c < nc; ++c) {
    for (size_t t = 0; t < b->cl[c].Q.size(); ++t) qf[qoff[c] + t] = (float)b->cl[c].Q[t];
    nin[c] = b->cl[c].nin;
    ns[c] = b->cl[c].ns;
  }
  Geo g{};
  float *dx, *dq;
  int64_t *dqoff, *dslot_off, *dboff;
  int32_t *dslots, *dnin, *dns, *drowslot, *dbsize;
  if ((st = upload(&dx, xf)) || (st = upload(&dq, qf)) || (st = upload(&dqoff, qoff)) ||
      (st = upload(&dslots, b->slots)) || (st = upload(&dslot_off, b->slot_off)) || (st = upload(&dnin, nin)) ||
      (st = upload(&dns, ns)) || (st = upload(&drowslot, b->rowslot)) || (st = upload(&dboff, b->block_offset)) ||
      (st = upload(&dbsize, b->bsize)))
    return st;
  for (void* q : {(void*)dx, (void*)dq, (void*)dqoff, (void*)dslots, (void*)dslot_off, (void*)dnin, (void*)dns,
                  (void*)drowslot, (void*)dboff, (void*)dbsize})
    fr.add(q);
  g.x = dx;
  g.Q = dq;
  g.qoff = dqoff;
  g.slots = dslots;
  g.slot_off = dslot_off;
  g.nin = dnin;
  g.ns = dns;
  // ---- upper-triangle block list (a <= b) and its staging offsets ---------------------
  const std::vector<int64_t>& rp = b->rowptr;
  const std::vector<int32_t>& ci = b->colidx;
  const int64_t nb_all = (int64_t)ci.size();
  std::vector<int32_t> ut_id(nb_all, -1);  // CSR block -> upper-triangle id (a <= b only)
  std::vector<int64_t> ut_off;
  int64_t nut = 0, stage_total = 0;
  for (int a = 0; a < nc; ++a)
    for (int64_t k = rp[a]; k < rp[a + 1]; ++k)
      if (ci[k] >= a) {
        ut_id[k] = (int32_t)nut++;
        ut_off.push_back(stage_total);
        stage_total += (int64_t)b->bsize[a] * b->bsize[ci[k]];
      }
  // column map of a cluster: its coordinate slots (root: scaling then samplets)
  std::vector<int64_t> cm_base(nc);
  std::vector<int32_t> colmap;
  for (int c = 0; c < nc; ++c) {
    cm_base[c] = (int64_t)colmap.size();
    const int32_t* sl = b->slots.data() + b->slot_off[c];
    const int base = c == 0 ? 0 : b->cl[c].ns;
    for (int j = 0; j < b->bsize[c]; ++j) colmap.push_back(sl[base + j]);
  }
  // per column cluster b: entries (a, b) with a <= b, a in row(b) (the pattern is symmetric)
  auto entries_of = [&](int bb, std::vector<int32_t>& ea, std::vector<int32_t>& eb, std::vector<int64_t>& eo,
                        std::vector<int32_t>& ek, std::vector<int32_t>& ecm, int64_t cm_shift) {
    for (int64_t k = rp[bb]; k < rp[bb + 1]; ++k) {
      const int a = ci[k];
      if (a > bb) break;
      // block (a, bb) sits in row a
      const int32_t* beg = ci.data() + rp[a];
      const int32_t* end = ci.data() + rp[a + 1];
      const int32_t* pos = std::lower_bound(beg, end, bb);
      if (pos == end || *pos != bb) continue;  // pattern not symmetric here: skip
      const int64_t kab = rp[a] + (pos - beg);
      ea.push_back(a);
      eb.push_back(bb);
      eo.push_back(ut_off[ut_id[kab]]);
      ek.push_back(ut_id[kab]);
      ecm.push_back((int32_t)(cm_base[bb] + cm_shift));
    }
  };
  float *dstage, *dbmax;
  int32_t* dcolmap;
  if ((st = dmalloc(&dstage, stage_total)) || (st = dmalloc(&dbmax, nut)) || (st = upload(&dcolmap, colmap))) return st;
  fr.add(dstage);
  fr.add(dbmax);
  fr.add(dcolmap);
  SF_CUDA(cudaMemset(dbmax, 0, sizeof(float) * std::max<int64_t>(nut, 1)));
  // ---- chunks: maximal clusters with at most kChunk points ------------------------------
  std::vector<int32_t> chunks, upper;  // chunk roots in left-to-right order; clusters above
  {
    std::vector<int32_t> st2{0};
    while (!st2.empty()) {
      int c = st2.back();
      st2.pop_back();
      if (b->cl[c].hi - b->cl[c].lo <= kChunk || b->cl[c].son[0] < 0) {
        chunks.push_back(c);
      } else {
        upper.push_back(c);
        st2.push_back(b->cl[c].son[1]);
        st2.push_back(b->cl[c].son[0]);
      }
    }
  }
  int wmax = 0;
  for (int c : chunks) wmax = std::max<int>(wmax, (int)(b->cl[c].hi - b->cl[c].lo));
  float* dU;
  if ((st = dmalloc(&dU, (size_t)n * wmax))) return st;
  fr.add(dU);
  // levels of the row tree, deepest first
  std::vector<std::vector<int32_t>> bylev(b->depth + 1);
  for (int c = 0; c < nc; ++c) bylev[b->cl[c].level].push_back(c);
  std::vector<int32_t> lvl_flat, lvl_off{0};
  for (int L = b->depth; L >= 0; --L) {
    lvl_flat.insert(lvl_flat.end(), bylev[L].begin(), bylev[L].end());
    lvl_off.push_back((int32_t)lvl_flat.size());
  }
  int32_t* dlvl;
  if ((st = upload(&dlvl, lvl_flat))) return st;
  fr.add(dlvl);
  int maxm = 1;
  for (const auto& c : b->cl) maxm = std::max(maxm, c.nin);
  const size_t smem = sizeof(float) * ((size_t)kRowTile * wmax + 8 * (size_t)(maxm * maxm + maxm));
  SF_CUDA(cudaFuncSetAttribute(eval_colfwt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // scaling columns of finished clusters, waiting for their sibling: (cluster, N x ns buffer)
  std::vector<std::pair<int32_t, float*>> stack;
  auto run_extract = [&](std::vector<int32_t>& ea, std::vector<int32_t>& eb, std::vector<int64_t>& eo,
                         std::vector<int32_t>& ek, std::vector<int32_t>& ecm, int64_t q0, const float* src,
                         int64_t ld) -> s_status {
    if (ea.empty()) return S_OK;
    int32_t *da, *db, *dk, *dcm;
    int64_t* dof;
    s_status s2;
    if ((s2 = upload(&da, ea)) || (s2 = upload(&db, eb)) || (s2 = upload(&dof, eo)) || (s2 = upload(&dk, ek)) ||
        (s2 = upload(&dcm, ecm)))
      return s2;
    Ext ex{da, db, dof, dk, dcm};
    const int64_t ne = (int64_t)ea.size();
    extract_kernel<<<(unsigned)((ne * 32 + 255) / 256), 256>>>(ex, ne, dbsize, dboff, drowslot, dcolmap, q0, src, ld,
                                                             dstage, dbmax);
    cudaError_t e = cudaGetLastError();
    cudaDeviceSynchronize();
    cudaFree(da);
    cudaFree(db);
    cudaFree(dof);
    cudaFree(dk);
    cudaFree(dcm);
    if (e != cudaSuccess) return cuda_error(e, "extract_kernel");
    return S_OK;
  };
  std::vector<int32_t> ea, eb, ek, ecm;
  std::vector<int64_t> eo;
  for (int gch : chunks) {
    const BCluster& G = b->cl[gch];
    const int64_t q0 = G.lo;
    const int w = (int)(G.hi - G.lo);
    // subtree of the chunk, deepest level first
    std::vector<std::vector<int32_t>> sl(b->depth + 1);
    std::vector<int32_t> st3{gch};
    std::vector<int32_t> members;
    while (!st3.empty()) {
      int c = st3.back();
      st3.pop_back();
      members.push_back(c);
      sl[b->cl[c].level].push_back(c);
      if (b->cl[c].son[0] >= 0) {
        st3.push_back(b->cl[c].son[0]);
        st3.push_back(b->cl[c].son[1]);
      }
    }
    std::vector<int32_t> sub, sub_off{0};
    for (int L = b->depth; L >= G.level; --L) {
      sub.insert(sub.end(), sl[L].begin(), sl[L].end());
      sub_off.push_back((int32_t)sub.size());
    }
    int32_t *dsub, *dsuboff;
    if ((st = upload(&dsub, sub)) || (st = upload(&dsuboff, sub_off))) return st;
    eval_colfwt_kernel<<<(unsigned)((n + kRowTile - 1) / kRowTile), 256, smem>>>(
        g, n, q0, w, dsub, dsuboff, (int)sub_off.size() - 1, p, (float)(1.0 / ell), (float)kscale, maxm, dU);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      cudaFree(dsub);
      cudaFree(dsuboff);
      return cuda_error(e, "eval_colfwt_kernel");
    }
    for (int L = 0; L < (int)lvl_off.size() - 1; ++L) {
      const int cnt = lvl_off[L + 1] - lvl_off[L];
      if (!cnt) continue;
      dim3 grid(cnt, (w + kColTile - 1) / kColTile);
      rowfwt_kernel<<<grid, 256>>>(g, dlvl + lvl_off[L], w, dU);
    }
    SF_CUDA(cudaGetLastError());
    ea.clear(); eb.clear(); eo.clear(); ek.clear(); ecm.clear();
    for (int c : members)
      if (b->bsize[c] > 0) entries_of(c, ea, eb, eo, ek, ecm, 0);
    st = run_extract(ea, eb, eo, ek, ecm, q0, dU, w);
    cudaFree(dsub);
    cudaFree(dsuboff);
    if (st) return st;
    if (gch == 0) break;  // the whole tree was one chunk
    // keep g's scaling columns
    float* S;
    if ((st = dmalloc(&S, (size_t)n * std::max(1, G.ns)))) return st;
    int32_t* dcols;
    std::vector<int32_t> cols(b->slots.begin() + b->slot_off[gch], b->slots.begin() + b->slot_off[gch] + G.ns);
    if ((st = upload(&dcols, cols))) {
      cudaFree(S);
      return st;
    }
    gather_cols_kernel<<<(unsigned)((n * G.ns + 255) / 256), 256>>>(n, G.ns, dcols, q0, dU, w, S);
    cudaDeviceSynchronize();
    cudaFree(dcols);
    stack.push_back({gch, S});
    // combine finished siblings upwards
    while (stack.size() >= 2) {
      auto s1 = stack[stack.size() - 1], s0 = stack[stack.size() - 2];
      const int par = b->cl[s0.first].parent;
      if (par < 0 || par != b->cl[s1.first].parent || b->cl[par].son[0] != s0.first) break;
      stack.pop_back();
      stack.pop_back();
      const BCluster& P = b->cl[par];
      const int m = P.nin;
      float* Gm;
      if ((st = dmalloc(&Gm, (size_t)n * m))) return st;
      concat_kernel<<<(unsigned)((n * m + 255) / 256), 256>>>(n, b->cl[s0.first].ns, s0.second,
                                                              b->cl[s1.first].ns, s1.second, Gm);
      colfwt_rows_kernel<<<(unsigned)((n + 127) / 128), 128>>>(n, m, dq + qoff[par], Gm);
      cudaFree(s0.second);
      cudaFree(s1.second);
      SF_CUDA(cudaGetLastError());
      // extraction reads G's columns: the column of coordinate j of par is j (+ns for
      // non-root), expressed through the column map as slot -> G column by a shifted map
      ea.clear(); eb.clear(); eo.clear(); ek.clear(); ecm.clear();
      if (b->bsize[par] > 0) entries_of(par, ea, eb, eo, ek, ecm, 0);
      // G's column of slot sl[t] is t: build a private map for par
      std::vector<int32_t> pm(b->bsize[par]);
      const int base = par == 0 ? 0 : P.ns;
      for (int j = 0; j < b->bsize[par]; ++j) pm[j] = base + j;
      int32_t* dpm = nullptr;
      if (!ea.empty()) {
        if ((st = upload(&dpm, pm))) return st;
        // run extraction with the private map: point every entry's cm at dpm via q0 = 0
        int32_t *da, *db, *dk, *dcm;
        int64_t* dof;
        std::vector<int32_t> zero(ea.size(), 0);
        if ((st = upload(&da, ea)) || (st = upload(&db, eb)) || (st = upload(&dof, eo)) || (st = upload(&dk, ek)) ||
            (st = upload(&dcm, zero)))
          return st;
        Ext ex{da, db, dof, dk, dcm};
        const int64_t ne = (int64_t)ea.size();
        extract_kernel<<<(unsigned)((ne * 32 + 255) / 256), 256>>>(ex, ne, dbsize, dboff, drowslot, dpm, 0, Gm, m,
                                                                 dstage, dbmax);
        cudaError_t e2 = cudaGetLastError();
        cudaDeviceSynchronize();
        cudaFree(da);
        cudaFree(db);
        cudaFree(dof);
        cudaFree(dk);
        cudaFree(dcm);
        cudaFree(dpm);
        if (e2 != cudaSuccess) return cuda_error(e2, "extract_kernel(upper)");
      }
      if (par == 0) {
        cudaFree(Gm);
        break;
      }
      // scaling columns of par = first ns columns of G
      float* S2;
      if ((st = dmalloc(&S2, (size_t)n * std::max(1, P.ns)))) return st;
      std::vector<int32_t> first(P.ns);
      for (int j = 0; j < P.ns; ++j) first[j] = j;
      int32_t* dfirst;
      if ((st = upload(&dfirst, first))) return st;
      gather_cols_kernel<<<(unsigned)((n * P.ns + 255) / 256), 256>>>(n, P.ns, dfirst, 0, Gm, m, S2);
      cudaDeviceSynchronize();
      cudaFree(dfirst);
      cudaFree(Gm);
      stack.push_back({par, S2});
    }
  }
  for (auto& s : stack) cudaFree(s.second);
  SF_CUDA(cudaDeviceSynchronize());
  // ---- kept pattern (decided per unordered pair), or the given one ----------------------
  std::vector<float> bmax(nut);
  SF_CUDA(cudaMemcpy(bmax.data(), dbmax, sizeof(float) * nut, cudaMemcpyDeviceToHost));
  auto pair_source = [&](int a, int c) -> int64_t {  // upper-triangle id of {a, c}, or -1
    const int lo = std::min(a, c), hi = std::max(a, c);
    const int32_t* beg = ci.data() + rp[lo];
    const int32_t* end = ci.data() + rp[lo + 1];
    const int32_t* pos = std::lower_bound(beg, end, hi);
    if (pos == end || *pos != hi) return -1;
    return ut_id[rp[lo] + (pos - beg)];
  };
  std::vector<int64_t> krp(nc + 1, 0);
  std::vector<int32_t> kci;
  std::vector<int64_t> ksrc;
  if (given) {
    if (given->d.nc != nc) return set_error(S_ERR_MISMATCH, "s_build_values_dell: pattern from another tree");
    for (int a = 0; a < nc; ++a) {
      for (int64_t k = given->rowptr[a]; k < given->rowptr[a + 1]; ++k) {
        const int c = given->colidx[k];
        const int64_t u = pair_source(a, c);
        if (u < 0) return set_error(S_ERR_PATTERN, "s_build_values_dell: block outside the eta pattern");
        kci.push_back(c);
        ksrc.push_back(ut_off[u]);
      }
      krp[a + 1] = (int64_t)kci.size();
    }
  } else {
    for (int a = 0; a < nc; ++a) {
      for (int64_t k = rp[a]; k < rp[a + 1]; ++k) {
        const int c = ci[k];
        const int64_t u = pair_source(a, c);
        if (u < 0) continue;
        if (a == c || (double)bmax[u] >= tau) {
          kci.push_back(c);
          ksrc.push_back(ut_off[u]);
        }
      }
      krp[a + 1] = (int64_t)kci.size();
    }
  }
  s_pattern pat = nullptr;
  const s_pattern_t* tgt = given;
  if (!given) {
    if ((st = s_pattern_create(nc, b->block_offset.data(), b->level.data(), krp.data(), kci.data(), &pat))) return st;
    tgt = pat;
  }
  const int64_t nnz = tgt->d.nnz;
  double* vals = out;
  if (!given) {
    cudaError_t e = cudaMalloc(&vals, sizeof(double) * std::max<int64_t>(nnz, 1));
    if (e != cudaSuccess) {
      s_pattern_destroy(pat);
      return cuda_error(e, "cudaMalloc(values)");
    }
  }
  int64_t* dsrc;
  if ((st = upload(&dsrc, ksrc))) {
    if (!given) {
      s_pattern_destroy(pat);
      cudaFree(vals);
    }
    return st;
  }
  fr.add(dsrc);
  const int64_t nk = (int64_t)kci.size();
  if (nk)
    assemble_kernel<<<(unsigned)((nk * 32 + 255) / 256), 256>>>(nk, tgt->d.brow, tgt->d.colidx, tgt->d.voff, dsrc,
                                                              dbsize, dstage, given ? 0.0 : nugget,
                                                              given ? 0.0 : tau, vals);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    if (!given) {
      s_pattern_destroy(pat);
      cudaFree(vals);
    }
    return cuda_error(e, "assemble_kernel");
  }
  if (!given) {
    *pattern = pat;
    b->dvals = vals;
    b->nvals = nnz;
  }
  return S_OK;
}

extern "C" s_status s_build_values(s_build b, double nu, double ell, double kscale, double nugget, double tau,
                                   s_pattern* pattern) {
  if (!b || !pattern) return set_error(S_ERR_ARG, "s_build_values: NULL argument");
  *pattern = nullptr;
  cudaFree(b->dvals);
  b->dvals = nullptr;
  b->nvals = 0;
  return values_impl(b, nu, ell, kscale, nugget, tau, false, nullptr, nullptr, pattern);
}

// y = (kscale K + nugget I) v with every kernel entry evaluated (no compression): one thread
// per row, columns streamed through shared memory 1024 at a time; each tile's terms summed in
// float, the tiles in double.
constexpr int kMvTile = 1024;
__global__ void __launch_bounds__(256) kmatvec_kernel(const float* __restrict__ x, int64_t n, int p, float inv_ell,
                                                      float scale, const float* __restrict__ v, double* __restrict__ y) {
  __shared__ float sx[kMvTile][3];
  __shared__ float sv[kMvTile];
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool row = i < n;
  const float xi0 = row ? x[i * 3] : 0.f, xi1 = row ? x[i * 3 + 1] : 0.f, xi2 = row ? x[i * 3 + 2] : 0.f;
  double acc = 0.0;
  for (int64_t j0 = 0; j0 < n; j0 += kMvTile) {
    const int cnt = (int)(n - j0 < kMvTile ? n - j0 : (int64_t)kMvTile);
    __syncthreads();
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      sx[t][0] = x[(j0 + t) * 3];
      sx[t][1] = x[(j0 + t) * 3 + 1];
      sx[t][2] = x[(j0 + t) * 3 + 2];
      sv[t] = v[j0 + t];
    }
    __syncthreads();
    float part = 0.f;
    for (int t = 0; t < cnt; ++t) {
      const float d0 = xi0 - sx[t][0], d1 = xi1 - sx[t][1], d2 = xi2 - sx[t][2];
      const float r = sqrtf(fmaf(d0, d0, fmaf(d1, d1, d2 * d2)));
      part = fmaf(matern(r, p, inv_ell, scale), sv[t], part);
    }
    acc += (double)part;
  }
  if (row) y[i] = acc;
}

extern "C" s_status s_build_kernel_matvec(s_build b, double nu, double ell, double kscale, double nugget,
                                          const double* v, double* y) {
  if (!b || !v || !y) return set_error(S_ERR_ARG, "s_build_kernel_matvec: NULL argument");
  int p;
  if (std::fabs(nu - 0.5) < 1e-12) p = 0;
  else if (std::fabs(nu - 1.5) < 1e-12) p = 1;
  else if (std::fabs(nu - 2.5) < 1e-12) p = 2;
  else return set_error(S_ERR_ARG, "s_build_kernel_matvec: nu must be 0.5, 1.5 or 2.5");
  if (!(ell > 0.0)) return set_error(S_ERR_ARG, "s_build_kernel_matvec: ell must be positive");
  const int64_t n = b->n;
  std::vector<float> xf((size_t)n * 3, 0.0f), vf(n);
  for (int64_t i = 0; i < n; ++i) {
    for (int a = 0; a < b->d; ++a) xf[i * 3 + a] = (float)b->points[i * b->d + a];
    vf[i] = (float)v[i];
  }
  Frees fr;
  s_status st;
  float *dx, *dv;
  double* dy;
  if ((st = upload(&dx, xf)) || (st = upload(&dv, vf)) || (st = dmalloc(&dy, (size_t)n))) return st;
  fr.add(dx);
  fr.add(dv);
  fr.add(dy);
  kmatvec_kernel<<<(unsigned)((n + 255) / 256), 256>>>(dx, n, p, (float)(1.0 / ell), (float)kscale, dv, dy);
  SF_CUDA(cudaGetLastError());
  SF_CUDA(cudaMemcpy(y, dy, sizeof(double) * n, cudaMemcpyDeviceToHost));
  for (int64_t i = 0; i < n; ++i) y[i] += nugget * v[i];
  return S_OK;
}

extern "C" s_status s_build_values_dell(s_build b, double nu, double ell, double kscale, s_pattern on, double* out) {
  if (!b || !on || (!out && on->d.nnz > 0)) return set_error(S_ERR_ARG, "s_build_values_dell: NULL argument");
  return values_impl(b, nu, ell, kscale, 0.0, 0.0, true, on, out, nullptr);
}

extern "C" s_status s_build_take_values(s_build b, double* dst, void* stream) {
  if (!b || (!dst && b->nvals > 0)) return set_error(S_ERR_ARG, "s_build_take_values: NULL argument");
  if (!b->dvals) return set_error(S_ERR_ARG, "s_build_take_values: no values (call s_build_values first)");
  if (b->nvals) SF_CUDA(cudaMemcpyAsync(dst, b->dvals, sizeof(double) * b->nvals, cudaMemcpyDeviceToDevice,
                                        (cudaStream_t)stream));
  SF_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  cudaFree(b->dvals);
  b->dvals = nullptr;
  b->nvals = 0;
  return S_OK;
}
