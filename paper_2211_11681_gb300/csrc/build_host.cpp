// Input preparation on the host: cluster tree, samplet two-scale transforms (own
// Householder QR), in-place transform slots and the eta pattern.  See include/sbuild.h for
// the conventions (they match the paper's construction, Sec. 3.2-3.3).
#include <omp.h>

#include <algorithm>
#include <string>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "build_internal.h"

namespace sf {

// graded monomial exponents, first exponent largest first within a degree
static std::vector<std::array<int, 3>> exponents(int d, int q) {
  std::vector<std::array<int, 3>> out;
  for (int g = 0; g <= q; ++g) {
    std::vector<std::array<int, 3>> deg;
    for (int a = 0; a <= g; ++a)
      for (int b = 0; b <= (d >= 2 ? g : 0); ++b)
        for (int c = 0; c <= (d >= 3 ? g : 0); ++c)
          if (a + b + c == g) deg.push_back({a, b, c});
    std::sort(deg.begin(), deg.end(), [](const std::array<int, 3>& x, const std::array<int, 3>& y) { return x > y; });
    out.insert(out.end(), deg.begin(), deg.end());
  }
  return out;
}

// Full Householder QR of the n x m row-major matrix R (overwritten); Q (n x n row-major)
// with A = Q R.  Reflector u = x - beta e1, beta = -sign(x0)|x|, none when x[1:] = 0.
static void householder(int n, int m, std::vector<double>& R, std::vector<double>& Q) {
  Q.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
  std::vector<double> u(n), tmp(std::max(n, m));
  for (int k = 0; k < std::min(n, m); ++k) {
    int len = n - k;
    if (len <= 1) continue;
    bool rest = false;
    for (int i = 1; i < len; ++i)
      if (R[(size_t)(k + i) * m + k] != 0.0) rest = true;
    if (!rest) continue;
    double nx = 0.0;
    for (int i = 0; i < len; ++i) nx += R[(size_t)(k + i) * m + k] * R[(size_t)(k + i) * m + k];
    nx = std::sqrt(nx);
    double x0 = R[(size_t)k * m + k];
    double beta = x0 >= 0.0 ? -nx : nx;
    for (int i = 0; i < len; ++i) u[i] = R[(size_t)(k + i) * m + k];
    u[0] -= beta;
    double nu = 0.0;
    for (int i = 0; i < len; ++i) nu += u[i] * u[i];
    nu = std::sqrt(nu);
    for (int i = 0; i < len; ++i) u[i] /= nu;
    // R[k:, :] -= 2 u (u^T R[k:, :])
    for (int j = 0; j < m; ++j) {
      double s = 0.0;
      for (int i = 0; i < len; ++i) s += u[i] * R[(size_t)(k + i) * m + j];
      tmp[j] = s;
    }
    for (int i = 0; i < len; ++i)
      for (int j = 0; j < m; ++j) R[(size_t)(k + i) * m + j] -= 2.0 * u[i] * tmp[j];
    // Q[:, k:] -= 2 (Q[:, k:] u) u^T
    for (int r = 0; r < n; ++r) {
      double s = 0.0;
      for (int i = 0; i < len; ++i) s += Q[(size_t)r * n + k + i] * u[i];
      for (int i = 0; i < len; ++i) Q[(size_t)r * n + k + i] -= 2.0 * s * u[i];
    }
  }
}

static double diam_of(const BCluster& c, int d) {
  double s = 0.0;
  for (int a = 0; a < d; ++a) s += (c.bmax[a] - c.bmin[a]) * (c.bmax[a] - c.bmin[a]);
  return std::sqrt(s);
}

static double dist_of(const BCluster& x, const BCluster& y, int d) {
  double s = 0.0;
  for (int a = 0; a < d; ++a) {
    double g = std::max(0.0, std::max(x.bmin[a] - y.bmax[a], y.bmin[a] - x.bmax[a]));
    s += g * g;
  }
  return std::sqrt(s);
}

s_status build_tree_basis(s_build_t* b) {
  const int64_t n = b->n;
  const int d = b->d;
  const double* x = b->points.data();
  b->perm.resize(n);
  std::iota(b->perm.begin(), b->perm.end(), 0);
  // breadth-first construction
  b->cl.clear();
  b->cl.push_back(BCluster{});
  b->cl[0].lo = 0;
  b->cl[0].hi = n;
  b->cl[0].level = 0;
  b->cl[0].parent = -1;
  for (size_t head = 0; head < b->cl.size(); ++head) {
    BCluster& c = b->cl[head];
    for (int a = 0; a < 3; ++a) {
      c.bmin[a] = 0.0;
      c.bmax[a] = 0.0;
    }
    for (int a = 0; a < d; ++a) {
      double lo = INFINITY, hi = -INFINITY;
      for (int64_t i = c.lo; i < c.hi; ++i) {
        double v = x[b->perm[i] * d + a];
        lo = std::min(lo, v);
        hi = std::max(hi, v);
      }
      c.bmin[a] = lo;
      c.bmax[a] = hi;
    }
    int64_t cnt = c.hi - c.lo;
    if (cnt > b->leaf) {
      int dim = 0;
      double best = -1.0;
      for (int a = 0; a < d; ++a)
        if (c.bmax[a] - c.bmin[a] > best) {
          best = c.bmax[a] - c.bmin[a];
          dim = a;
        }
      std::sort(b->perm.begin() + c.lo, b->perm.begin() + c.hi, [&](int64_t p, int64_t q) {
        double vp = x[p * d + dim], vq = x[q * d + dim];
        return vp < vq || (vp == vq && p < q);
      });
      int64_t mid = c.lo + cnt / 2;
      int64_t lo = c.lo, hi = c.hi;
      int lev = c.level;
      int32_t id = (int32_t)head;
      BCluster s0{}, s1{};
      s0.lo = lo;
      s0.hi = mid;
      s1.lo = mid;
      s1.hi = hi;
      s0.level = s1.level = lev + 1;
      s0.parent = s1.parent = id;
      b->cl[head].son[0] = (int32_t)b->cl.size();
      b->cl[head].son[1] = (int32_t)b->cl.size() + 1;
      b->cl.push_back(s0);  // may reallocate: do not use c afterwards
      b->cl.push_back(s1);
    } else {
      c.son[0] = c.son[1] = -1;
    }
  }
  const int nc = (int)b->cl.size();
  int maxlev = 0;
  for (auto& c : b->cl) maxlev = std::max(maxlev, c.level);
  b->depth = maxlev;
  // two-scale transforms bottom-up, level by level
  auto ex = exponents(d, b->q);
  const int mq = (int)ex.size();
  b->mq = mq;
  std::vector<std::vector<double>> phi(nc);  // |c| x ns(c) weights in point order
  std::vector<std::vector<int32_t>> bylevel(maxlev + 1);
  for (int i = 0; i < nc; ++i) bylevel[b->cl[i].level].push_back(i);
  for (int lev = maxlev; lev >= 0; --lev) {
    const auto& ids = bylevel[lev];
#pragma omp parallel for schedule(dynamic, 4)
    for (size_t t = 0; t < ids.size(); ++t) {
      BCluster& c = b->cl[ids[t]];
      const int64_t m = c.hi - c.lo;
      double centre[3] = {0, 0, 0}, half = 0.0;
      for (int a = 0; a < d; ++a) {
        centre[a] = 0.5 * (c.bmin[a] + c.bmax[a]);
        half = std::max(half, 0.5 * (c.bmax[a] - c.bmin[a]));
      }
      if (half <= 0.0) half = 1.0;
      // local monomials P (m x mq)
      std::vector<double> P((size_t)m * mq);
      for (int64_t i = 0; i < m; ++i) {
        const double* xp = x + b->perm[c.lo + i] * d;
        double y[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a) y[a] = (xp[a] - centre[a]) / half;
        for (int k = 0; k < mq; ++k) {
          double v = 1.0;
          for (int a = 0; a < d; ++a)
            for (int e = 0; e < ex[k][a]; ++e) v *= y[a];
          P[(size_t)i * mq + k] = v;
        }
      }
      int nin;
      std::vector<double> Mt;  // nin x mq
      if (c.son[0] < 0) {
        nin = (int)m;
        Mt = P;
      } else {
        const BCluster& s0 = b->cl[c.son[0]];
        const BCluster& s1 = b->cl[c.son[1]];
        nin = s0.ns + s1.ns;
        Mt.assign((size_t)nin * mq, 0.0);
        int64_t off = 0;
        int row = 0;
        for (int si = 0; si < 2; ++si) {
          const BCluster& s = si ? s1 : s0;
          const std::vector<double>& ph = phi[si ? c.son[1] : c.son[0]];
          int64_t ms = s.hi - s.lo;
          for (int j = 0; j < s.ns; ++j) {
            for (int k = 0; k < mq; ++k) {
              double acc = 0.0;
              for (int64_t i = 0; i < ms; ++i) acc += ph[(size_t)i * s.ns + j] * P[(size_t)(off + i) * mq + k];
              Mt[(size_t)(row + j) * mq + k] = acc;
            }
          }
          row += s.ns;
          off += ms;
        }
      }
      std::vector<double> Q;
      householder(nin, mq, Mt, Q);
      c.nin = nin;
      c.ns = std::min(mq, nin);
      c.nsamp = nin - c.ns;
      c.Q = Q;
      // scaling weights Phi = Psi Q[:, :ns]
      std::vector<double>& ph = phi[ids[t]];
      ph.assign((size_t)m * c.ns, 0.0);
      if (c.son[0] < 0) {
        for (int64_t i = 0; i < m; ++i)
          for (int j = 0; j < c.ns; ++j) ph[(size_t)i * c.ns + j] = Q[(size_t)i * nin + j];
      } else {
        int64_t off = 0;
        int row = 0;
        for (int si = 0; si < 2; ++si) {
          const BCluster& s = b->cl[c.son[si]];
          const std::vector<double>& ps = phi[c.son[si]];
          int64_t ms = s.hi - s.lo;
          for (int64_t i = 0; i < ms; ++i)
            for (int j = 0; j < c.ns; ++j) {
              double acc = 0.0;
              for (int k = 0; k < s.ns; ++k) acc += ps[(size_t)i * s.ns + k] * Q[(size_t)(row + k) * nin + j];
              ph[(size_t)(off + i) * c.ns + j] = acc;
            }
          row += s.ns;
          off += ms;
        }
      }
    }
    if (lev + 1 <= maxlev)
      for (int id : bylevel[lev + 1]) std::vector<double>().swap(phi[id]);
  }
  // block sizes and offsets (breadth-first), in-place transform slots
  b->bsize.assign(nc, 0);
  b->block_offset.assign(nc + 1, 0);
  b->level.assign(nc, 0);
  for (int i = 0; i < nc; ++i) {
    const BCluster& c = b->cl[i];
    b->bsize[i] = c.nsamp + (i == 0 ? c.ns : 0);
    b->block_offset[i + 1] = b->block_offset[i] + b->bsize[i];
    b->level[i] = c.level;
  }
  if (b->block_offset[nc] != n) return set_error(S_ERR_ARG, "internal: samplet count differs from n");
  b->slot_off.assign(nc + 1, 0);
  for (int i = 0; i < nc; ++i) b->slot_off[i + 1] = b->slot_off[i] + b->cl[i].nin;
  b->slots.assign(b->slot_off[nc], 0);
  for (int lev = maxlev; lev >= 0; --lev)
    for (int id : bylevel[lev]) {
      const BCluster& c = b->cl[id];
      int32_t* sl = b->slots.data() + b->slot_off[id];
      if (c.son[0] < 0) {
        for (int64_t i = 0; i < c.hi - c.lo; ++i) sl[i] = (int32_t)(c.lo + i);
      } else {
        int pos = 0;
        for (int si = 0; si < 2; ++si) {
          const BCluster& s = b->cl[c.son[si]];
          const int32_t* ss = b->slots.data() + b->slot_off[c.son[si]];
          for (int j = 0; j < s.ns; ++j) sl[pos++] = ss[j];
        }
      }
    }
  // rowslot: position (in tree point order) holding samplet row g after the transform
  b->rowslot.assign(n, 0);
  for (int i = 0; i < nc; ++i) {
    const BCluster& c = b->cl[i];
    const int32_t* sl = b->slots.data() + b->slot_off[i];
    int64_t g = b->block_offset[i];
    if (i == 0)
      for (int j = 0; j < c.ns; ++j) b->rowslot[g++] = sl[j];
    for (int j = 0; j < c.nsamp; ++j) b->rowslot[g++] = sl[c.ns + j];
  }
  return S_OK;
}

s_status build_pattern(s_build_t* b, double eta) {
  const int nc = (int)b->cl.size();
  const int d = b->d;
  std::vector<double> diam(nc);
  for (int i = 0; i < nc; ++i) diam[i] = diam_of(b->cl[i], d);
  std::vector<std::vector<int32_t>> rows(nc);
  const bool all = std::isinf(eta);
#pragma omp parallel
  {
    std::vector<int32_t> stack;
#pragma omp for schedule(dynamic, 16)
    for (int a = 0; a < nc; ++a) {
      if (b->bsize[a] == 0) continue;
      std::vector<int32_t>& row = rows[a];
      stack.clear();
      stack.push_back(0);
      while (!stack.empty()) {
        int c = stack.back();
        stack.pop_back();
        bool keep = all || a == c ||
                    dist_of(b->cl[a], b->cl[c], d) < eta * std::max(diam[a], diam[c]);
        if (!keep) continue;  // admissible: so are all pairs below it
        if (b->bsize[c] > 0) row.push_back(c);
        if (b->cl[c].son[0] >= 0) {
          stack.push_back(b->cl[c].son[1]);
          stack.push_back(b->cl[c].son[0]);
        }
      }
      std::sort(row.begin(), row.end());
    }
  }
  b->rowptr.assign(nc + 1, 0);
  for (int a = 0; a < nc; ++a) b->rowptr[a + 1] = b->rowptr[a] + (int64_t)rows[a].size();
  b->colidx.resize(b->rowptr[nc]);
  b->nnz_apriori = 0;
  for (int a = 0; a < nc; ++a) {
    std::copy(rows[a].begin(), rows[a].end(), b->colidx.begin() + b->rowptr[a]);
    for (int32_t c : rows[a]) b->nnz_apriori += (int64_t)b->bsize[a] * b->bsize[c];
  }
  return S_OK;
}

}  // namespace sf

using namespace sf;

extern "C" s_status s_build_create(int64_t n, int32_t d, const double* points, int32_t leaf, int32_t q, double eta,
                                   s_build* out) {
  if (!out) return set_error(S_ERR_ARG, "s_build_create: out is NULL");
  *out = nullptr;
  if (n < 1 || d < 1 || d > 3 || !points || leaf < 1 || q < 0 || !(eta > 0.0) || n > INT32_MAX)
    return set_error(S_ERR_ARG, "s_build_create: bad argument");
  for (int64_t i = 0; i < n * d; ++i)
    if (!std::isfinite(points[i])) return set_error(S_ERR_ARG, "s_build_create: non-finite coordinate");
  s_build_t* b = new (std::nothrow) s_build_t();
  if (!b) return set_error(S_ERR_NOMEM, "host allocation");
  b->n = n;
  b->d = d;
  b->leaf = leaf;
  b->q = q;
  b->points.assign(points, points + n * d);
  s_status st;
  if ((st = build_tree_basis(b)) || (st = build_pattern(b, eta))) {
    delete b;
    return st;
  }
  *out = b;
  return S_OK;
}

extern "C" s_status s_build_destroy(s_build b) {
  delete b;
  return S_OK;
}

extern "C" s_status s_build_sizes(s_build b, int32_t* n_clusters, int64_t* n_blocks, int64_t* nnz) {
  if (!b) return set_error(S_ERR_ARG, "s_build_sizes: NULL builder");
  if (n_clusters) *n_clusters = (int32_t)b->cl.size();
  if (n_blocks) *n_blocks = (int64_t)b->colidx.size();
  if (nnz) *nnz = b->nnz_apriori;
  return S_OK;
}

extern "C" s_status s_build_arrays(s_build b, const int64_t** block_offset, const int32_t** level,
                                   const int64_t** rowptr, const int32_t** colidx, const int64_t** perm) {
  if (!b) return set_error(S_ERR_ARG, "s_build_arrays: NULL builder");
  if (block_offset) *block_offset = b->block_offset.data();
  if (level) *level = b->level.data();
  if (rowptr) *rowptr = b->rowptr.data();
  if (colidx) *colidx = b->colidx.data();
  if (perm) *perm = b->perm.data();
  return S_OK;
}

extern "C" s_status s_build_dense_transform(s_build b, double* T) {
  if (!b || !T) return set_error(S_ERR_ARG, "s_build_dense_transform: NULL argument");
  const int64_t n = b->n;
  if (n > 8192) return set_error(S_ERR_ARG, "s_build_dense_transform: n > 8192");
  // apply the in-place transform to the identity: column j = e_{perm^-1}... build W (n x n,
  // rows = tree-order point positions, cols = original points), then run the level-wise
  // in-place row transform and read rows through rowslot.
  std::vector<double> W((size_t)n * n, 0.0);
  for (int64_t i = 0; i < n; ++i) W[(size_t)i * n + b->perm[i]] = 1.0;
  const int nc = (int)b->cl.size();
  std::vector<std::vector<int32_t>> bylevel(b->depth + 1);
  for (int i = 0; i < nc; ++i) bylevel[b->cl[i].level].push_back(i);
  std::vector<double> buf;
  for (int lev = b->depth; lev >= 0; --lev)
    for (int id : bylevel[lev]) {
      const BCluster& c = b->cl[id];
      const int32_t* sl = b->slots.data() + b->slot_off[id];
      const int m = c.nin;
      buf.assign((size_t)m * n, 0.0);
      for (int j = 0; j < m; ++j)      // out row j = sum_i Q[i][j] in row i
        for (int i = 0; i < m; ++i) {
          double qv = c.Q[(size_t)i * m + j];
          if (qv == 0.0) continue;
          const double* src = &W[(size_t)sl[i] * n];
          double* dst = &buf[(size_t)j * n];
          for (int64_t k = 0; k < n; ++k) dst[k] += qv * src[k];
        }
      for (int j = 0; j < m; ++j) std::memcpy(&W[(size_t)sl[j] * n], &buf[(size_t)j * n], sizeof(double) * n);
    }
  for (int64_t g = 0; g < n; ++g) std::memcpy(T + (size_t)g * n, &W[(size_t)b->rowslot[g] * n], sizeof(double) * n);
  return S_OK;
}

extern "C" s_status s_build_transform(s_build b, const double* v, double* out) {
  if (!b || !v || !out) return set_error(S_ERR_ARG, "s_build_transform: NULL argument");
  const int64_t n = b->n;
  // tree order, then the in-place two-scale transform level by level (bottom-up)
  std::vector<double> w(n);
  for (int64_t i = 0; i < n; ++i) w[i] = v[b->perm[i]];
  const int nc = (int)b->cl.size();
  std::vector<std::vector<int32_t>> bylevel(b->depth + 1);
  for (int i = 0; i < nc; ++i) bylevel[b->cl[i].level].push_back(i);
  std::vector<double> in, o;
  for (int lev = b->depth; lev >= 0; --lev)
    for (int id : bylevel[lev]) {
      const BCluster& c = b->cl[id];
      const int32_t* sl = b->slots.data() + b->slot_off[id];
      const int m = c.nin;
      in.assign(m, 0.0);
      o.assign(m, 0.0);
      for (int i = 0; i < m; ++i) in[i] = w[sl[i]];
      for (int j = 0; j < m; ++j) {
        double acc = 0.0;
        for (int i = 0; i < m; ++i) acc += c.Q[(size_t)i * m + j] * in[i];
        o[j] = acc;
      }
      for (int j = 0; j < m; ++j) w[sl[j]] = o[j];
    }
  for (int64_t g = 0; g < n; ++g) out[g] = w[b->rowslot[g]];
  return S_OK;
}
