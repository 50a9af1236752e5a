// Block patterns: validation, host/device copies, block-CSC index, tree hash.
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include "common.cuh"

namespace sf {

static thread_local std::string g_err;

s_status set_error(s_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

s_status cuda_error(cudaError_t e, const char* what) {
  return set_error(e == cudaErrorMemoryAllocation ? S_ERR_NOMEM : S_ERR_CUDA,
                   std::string(what) + ": " + cudaGetErrorString(e));
}

// SM count of the current device, queried once per device ordinal (grids are sized from it,
// so a plan made on one device must not inherit another device's count).
int sm_count() {
  static std::mutex mu;
  static int cache[256] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return 1;
  std::lock_guard<std::mutex> lk(mu);
  if (cache[dev] <= 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    cache[dev] = n;
  }
  return cache[dev];
}

template <typename T>
static s_status upload(T** dst, const T* src, size_t n) {
  if (n == 0) n = 1;  // keep a valid pointer for empty arrays
  cudaError_t e = cudaMalloc((void**)dst, n * sizeof(T));
  if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(pattern)");
  if (src) {
    e = cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemcpy(pattern)");
  }
  return S_OK;
}

static void free_dev(DevPattern& d) {
  cudaFree(d.bsize);
  cudaFree(d.boff);
  cudaFree(d.rowptr);
  cudaFree(d.colidx);
  cudaFree(d.brow);
  cudaFree(d.voff);
  cudaFree(d.colptr);
  cudaFree(d.rowidx);
  cudaFree(d.cscblk);
  cudaFree(d.diag);
  d = DevPattern();
}

static uint64_t fnv(uint64_t h, const void* p, size_t bytes) {
  const unsigned char* c = (const unsigned char*)p;
  for (size_t i = 0; i < bytes; ++i) {
    h ^= c[i];
    h *= 1099511628211ull;
  }
  return h;
}

}  // namespace sf

using namespace sf;

extern "C" const char* s_last_error(void) { return g_err.c_str(); }
extern "C" const char* s_version(void) { return "sformat-gb300 0.1 (sm_103a)"; }

extern "C" s_status s_pattern_create(int32_t nc, const int64_t* block_offset, const int32_t* level,
                                     const int64_t* rowptr, const int32_t* colidx, s_pattern* out) {
  if (!out) return set_error(S_ERR_ARG, "s_pattern_create: out is NULL");
  *out = nullptr;
  if (nc < 1 || !block_offset || !level || !rowptr || (!colidx && rowptr[nc] > 0))
    return set_error(S_ERR_ARG, "s_pattern_create: bad argument");
  if (block_offset[0] != 0 || rowptr[0] != 0) return set_error(S_ERR_PATTERN, "offsets must start at 0");
  int32_t maxb = 0;
  for (int32_t i = 0; i < nc; ++i) {
    int64_t b = block_offset[i + 1] - block_offset[i];
    if (b < 0 || b > 32767) return set_error(S_ERR_PATTERN, "block_offset not non-decreasing or block > 32767");
    if (rowptr[i + 1] < rowptr[i]) return set_error(S_ERR_PATTERN, "rowptr not non-decreasing");
    if (level[i] < 0) return set_error(S_ERR_PATTERN, "negative level");
    if (b > maxb) maxb = (int32_t)b;
  }
  int64_t nb = rowptr[nc];
  if (nb > INT32_MAX) return set_error(S_ERR_PATTERN, "more than 2^31-1 blocks");
  s_pattern_t* p = new (std::nothrow) s_pattern_t();
  if (!p) return set_error(S_ERR_NOMEM, "host allocation");
  p->bsize.resize(nc);
  p->level.assign(level, level + nc);
  p->boff.assign(block_offset, block_offset + nc + 1);
  p->rowptr.assign(rowptr, rowptr + nc + 1);
  p->colidx.assign(colidx, colidx + nb);
  p->brow.resize(nb);
  p->voff.resize(nb + 1);
  p->diag.assign(nc, -1);
  for (int32_t i = 0; i < nc; ++i) p->bsize[i] = (int32_t)(block_offset[i + 1] - block_offset[i]);
  int64_t off = 0;
  for (int32_t i = 0; i < nc; ++i) {
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      int32_t j = colidx[k];
      if (j < 0 || j >= nc || (k > rowptr[i] && colidx[k - 1] >= j)) {
        delete p;
        return set_error(S_ERR_PATTERN, "colidx out of range or not strictly increasing in row " + std::to_string(i));
      }
      if (p->bsize[i] == 0 || p->bsize[j] == 0) {
        delete p;
        return set_error(S_ERR_PATTERN, "block touches a cluster with zero rows");
      }
      if (j == i) p->diag[i] = (int32_t)k;
      p->brow[k] = i;
      p->voff[k] = off;
      off += (int64_t)p->bsize[i] * p->bsize[j];
    }
    if (p->bsize[i] > 0 && p->diag[i] < 0) p->has_all_diag = false;
  }
  p->voff[nb] = off;
  uint64_t h = 1469598103934665603ull;
  h = fnv(h, block_offset, sizeof(int64_t) * (nc + 1));
  h = fnv(h, level, sizeof(int32_t) * nc);
  p->tree_hash = h;
  // block-CSC: for column j the rows i with (i,j) in S, increasing, and the CSR block ids
  std::vector<int64_t> colptr(nc + 1, 0);
  for (int64_t k = 0; k < nb; ++k) colptr[colidx[k] + 1]++;
  for (int32_t j = 0; j < nc; ++j) colptr[j + 1] += colptr[j];
  std::vector<int64_t> fill(colptr.begin(), colptr.end() - 1);
  std::vector<int32_t> rowidx(nb), cscblk(nb);
  for (int32_t i = 0; i < nc; ++i)
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      int64_t pos = fill[colidx[k]]++;
      rowidx[pos] = i;
      cscblk[pos] = (int32_t)k;
    }
  DevPattern& d = p->d;
  d.nc = nc;
  d.n = block_offset[nc];
  d.nblocks = nb;
  d.nnz = off;
  d.max_bsize = maxb;
  s_status st;
  if ((st = upload(&d.bsize, p->bsize.data(), nc)) || (st = upload(&d.boff, block_offset, nc + 1)) ||
      (st = upload(&d.rowptr, rowptr, nc + 1)) || (st = upload(&d.colidx, colidx, nb)) ||
      (st = upload(&d.brow, p->brow.data(), nb)) || (st = upload(&d.voff, p->voff.data(), nb + 1)) ||
      (st = upload(&d.colptr, colptr.data(), nc + 1)) || (st = upload(&d.rowidx, rowidx.data(), nb)) ||
      (st = upload(&d.cscblk, cscblk.data(), nb)) || (st = upload(&d.diag, p->diag.data(), nc))) {
    free_dev(d);
    delete p;
    return st;
  }
  *out = p;
  return S_OK;
}

extern "C" s_status s_pattern_destroy(s_pattern p) {
  if (!p) return S_OK;
  free_dev(p->d);
  delete p;
  return S_OK;
}

extern "C" int64_t s_pattern_nnz(s_pattern p) { return p ? p->d.nnz : -1; }
extern "C" int64_t s_pattern_nblocks(s_pattern p) { return p ? p->d.nblocks : -1; }

extern "C" s_status s_pattern_block_offsets(s_pattern p, int64_t* out) {
  if (!p || !out) return set_error(S_ERR_ARG, "s_pattern_block_offsets: NULL argument");
  std::memcpy(out, p->voff.data(), sizeof(int64_t) * p->voff.size());
  return S_OK;
}

extern "C" s_status s_pattern_host_arrays(s_pattern p, int32_t* n_clusters, const int64_t** block_offset,
                                          const int64_t** rowptr, const int32_t** colidx) {
  if (!p) return set_error(S_ERR_ARG, "s_pattern_host_arrays: NULL pattern");
  if (n_clusters) *n_clusters = p->d.nc;
  if (block_offset) *block_offset = p->boff.data();
  if (rowptr) *rowptr = p->rowptr.data();
  if (colidx) *colidx = p->colidx.data();
  return S_OK;
}

extern "C" s_status s_pattern_concat(int32_t count, const s_pattern* parts, s_pattern* out) {
  if (!out) return set_error(S_ERR_ARG, "s_pattern_concat: out is NULL");
  *out = nullptr;
  if (count < 1 || !parts) return set_error(S_ERR_ARG, "s_pattern_concat: no parts");
  std::vector<int64_t> bo{0}, rp{0};
  std::vector<int32_t> lv, ci;
  int64_t nc_total = 0;
  for (int32_t q = 0; q < count; ++q) {
    const s_pattern_t* p = parts[q];
    if (!p) return set_error(S_ERR_ARG, "s_pattern_concat: NULL part");
    if (nc_total + p->d.nc > INT32_MAX) return set_error(S_ERR_ARG, "s_pattern_concat: too many clusters");
    const int64_t row0 = bo.back(), blk0 = rp.back();
    for (int32_t i = 0; i < p->d.nc; ++i) {
      bo.push_back(row0 + p->boff[i + 1]);
      rp.push_back(blk0 + p->rowptr[i + 1]);
      lv.push_back(p->level[i]);
    }
    for (int32_t c : p->colidx) ci.push_back((int32_t)(c + nc_total));
    nc_total += p->d.nc;
  }
  return s_pattern_create((int32_t)nc_total, bo.data(), lv.data(), rp.data(), ci.data(), out);
}
