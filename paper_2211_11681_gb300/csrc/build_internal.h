// Internal state of the input builder (include/sbuild.h).
#pragma once
#include <array>
#include <string>
#include <cstdint>
#include <vector>

#include "sbuild.h"
#include "sformat.h"

namespace sf {

s_status set_error(s_status st, const std::string& msg);

struct BCluster {
  int64_t lo = 0, hi = 0;  // point range in tree order
  int32_t level = 0, parent = -1;
  int32_t son[2] = {-1, -1};
  double bmin[3] = {0, 0, 0}, bmax[3] = {0, 0, 0};
  int nin = 0, ns = 0, nsamp = 0;
  std::vector<double> Q;   // nin x nin row-major two-scale matrix of Eq. (QR)
};

}  // namespace sf

struct s_build_t {
  int64_t n = 0;
  int d = 0, leaf = 0, q = 0, mq = 0, depth = 0;
  std::vector<double> points;       // n x d, original order
  std::vector<int64_t> perm;        // tree order -> original index
  std::vector<sf::BCluster> cl;     // breadth first
  std::vector<int32_t> bsize, level;
  std::vector<int64_t> block_offset;
  std::vector<int64_t> slot_off;    // nc+1
  std::vector<int32_t> slots;       // in-place transform slots of each cluster (nin each)
  std::vector<int32_t> rowslot;     // samplet row -> slot after the transform
  std::vector<int64_t> rowptr;      // a-priori eta pattern
  std::vector<int32_t> colidx;
  int64_t nnz_apriori = 0;
  double* dvals = nullptr;          // device values of the last s_build_values call
  int64_t nvals = 0;
  ~s_build_t();
};
