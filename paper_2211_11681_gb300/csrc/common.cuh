// Internal definitions shared by the translation units of libsformat.so.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "sformat.h"

namespace sf {

// Thread-local error message; set_error returns the status for `return set_error(...)`.
s_status set_error(s_status st, const std::string& msg);
s_status cuda_error(cudaError_t e, const char* what);
// SM count of the current device (cached per device ordinal).
int sm_count();

#define SF_CUDA(call)                                     \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return sf::cuda_error(e_, #call); \
  } while (0)

// Device copy of a block pattern (Sec. 3.3: cluster pairs of one tree), with the
// block-CSR rows and the transposed (block-CSC) index, both sorted.
struct DevPattern {
  int32_t nc = 0;
  int64_t n = 0;        // matrix dimension
  int64_t nblocks = 0;
  int64_t nnz = 0;
  int32_t max_bsize = 0;
  // device arrays
  int32_t* bsize = nullptr;   // nc
  int64_t* boff = nullptr;    // nc+1 row offsets
  int64_t* rowptr = nullptr;  // nc+1
  int32_t* colidx = nullptr;  // nblocks
  int32_t* brow = nullptr;    // nblocks: block row of each block
  int64_t* voff = nullptr;    // nblocks+1 entry offsets
  int64_t* colptr = nullptr;  // nc+1 (CSC)
  int32_t* rowidx = nullptr;  // nblocks: block rows of column, sorted
  int32_t* cscblk = nullptr;  // nblocks: CSR block index of each CSC entry
  int32_t* diag = nullptr;    // nc: block index of (nu,nu) or -1
};

}  // namespace sf

struct s_pattern_t {
  sf::DevPattern d;
  // host copies
  std::vector<int32_t> bsize, level, colidx, brow, diag;
  std::vector<int64_t> boff, rowptr, voff;
  uint64_t tree_hash = 0;
  bool has_all_diag = true;
};

namespace sf {

// One side of a masked product: op(X) with op = identity or transpose.  The index list
// of row nu of op(X) is idx[ptr[nu] .. ptr[nu+1]) with X block ids blk[...].
struct Side {
  const int64_t* ptr;
  const int32_t* idx;
  const int32_t* blk;  // nullptr: blk = position (CSR of X itself)
  const int64_t* voff;
  bool trans;
};

// Work item of the product kernels: one output tile of one block of C.
struct Tile {
  int32_t blk;  // C block id
  int16_t r0;   // first row of the tile inside the block
  int16_t c0;   // first column
};

// S_TF32X3 product (mul_tc.cu): MMA rows (member columns) and columns (own rows) of a panel,
// members per panel, lambda extent of one stage, widest block supported.
constexpr int kTcM = 128;
constexpr int kTcN = 32;
constexpr int kTcP = 8;
constexpr int kTcKC = 24;
constexpr int kTcMaxB = 96;

// One stage of an S_TF32X3 panel: source offsets (in the split value planes) of the X slice
// and of each member's Y slice (-1: member has no block for this lambda), lambda's block
// size (row pitch of the slices) and the staged extent.
struct TcEntry {
  int64_t x;
  int64_t y[kTcP];
  int32_t nl, wd;
};

// One operand side of the K-major float product (mul_nt.cu): the op(X) row lists or op(Y)
// column lists, and where the kernel finds each block's K-major slice data: directly in the
// caller's buffer (offsets = the pattern's voff) or in a padded, per-block transposed copy
// written by a pre-pass into `scratch` (offsets poff).
struct NtSideDesc {
  const int64_t* ptr = nullptr;
  const int32_t* idx = nullptr;
  const int32_t* blk = nullptr;
  const int64_t* off = nullptr;   // nullptr: side not configured
  const s_pattern_t* pat = nullptr;
  bool prep = false;              // true: the kernel reads `scratch`
  bool trans = false;             // prepared copy holds the stored blocks transposed
  bool from_x = false;            // Y side: reads the X side's prepared copy (B = A, symmetric)
  int64_t* poff = nullptr;
  float* scratch = nullptr;
  int64_t len = 0;
};

struct MulDesc {
  Side x, y;                 // C = op(X) op(Y) on S_C
  const s_pattern_t* pc;
  const s_pattern_t* px;
  const s_pattern_t* py;
  Tile* tiles = nullptr;     // device tile list, block order
  int64_t ntiles = 0;
  int edge = 20;             // tile edge of the list
  int variant = 0;           // float kernel variant (autotuned)
  Tile* ptiles = nullptr;    // row-panel variants: tiles ordered by (row, r0, column)
  int2* pidx = nullptr;      // per panel: first tile in ptiles, tile count
  int64_t npanels = 0;
  int panel_edge = 0, panel_size = 0;
  int64_t* tc_pstart = nullptr;  // S_TF32X3: first stage of each panel (npanels + 1)
  TcEntry* tc_ent = nullptr;     // S_TF32X3: stages of all panels
  int64_t tc_nentries = 0;
  float* tc_xh = nullptr;        // S_TF32X3 split planes (hi, lo) of both operands
  float* tc_xl = nullptr;
  float* tc_yh = nullptr;
  float* tc_yl = nullptr;
  unsigned int* err = nullptr;       // time-out word, device view: set to 1 when a bounded wait
  unsigned int* err_host = nullptr;  // of a kernel ran out; pinned host memory mapped into the
                                     // device, so the host reads it without a sync
  bool tc_sym = false;             // symmetric plan: B = A, Y read through its stored transpose
  NtSideDesc ntx, nty;             // K-major float product sides (S_FP32)
  bool nt_ysym = false;            // Y side read through X's rows (B = A, symmetric)
  float2* df_x = nullptr;    // S_FP64_DF: split operands (hi, lo)
  float2* df_y = nullptr;
  struct __nv_bfloat16* bf_x = nullptr;  // S_BF16X3: three bfloat16 planes per operand
  struct __nv_bfloat16* bf_y = nullptr;
  unsigned int* counter = nullptr;  // device work counter
  int64_t triples = 0;
  double flops = 0.0;
};

s_status build_desc(const s_pattern_t* X, bool tx, const s_pattern_t* Y, bool ty, const s_pattern_t* C, s_prec prec,
                    MulDesc* d);
void free_desc(MulDesc* d);
s_status tc_prepare(MulDesc* d);
void tc_free(MulDesc* d);
s_status launch_tc(const MulDesc& d, const void* X, const void* Y, void* C, cudaStream_t st);
// S_ERR_TIMEOUT (and the record cleared) if the descriptor's time-out word is set, else S_OK.
s_status take_timeout(const MulDesc& d);
// K-major float product (mul_nt.cu): configure the sides of a float descriptor, whether a call
// with these buffers can use it, the launch, and the release of its scratch.
s_status nt_configure(MulDesc* d, bool x_trans, bool y_trans, bool y_sym);
bool nt_usable(const MulDesc& d, const void* X, const void* Y);
s_status launch_nt(const MulDesc& d, const void* X, const void* Y, void* C, cudaStream_t st, bool const_pitch);
void nt_free_side(NtSideDesc* s);
s_status run_mul(const MulDesc& d, s_prec prec, const void* X, const void* Y, void* C, cudaStream_t st);

// Element-wise kernels (add.cu)
s_status run_add(const s_pattern_t* p, s_prec prec, double alpha, const void* A, double beta, const void* B,
                 double gamma, void* C, cudaStream_t st);
s_status run_spmv_f64(const s_pattern_t* p, const double* A, const double* x, double* y, cudaStream_t st);

constexpr int kTile = 20;  // output tile edge of the product kernels

}  // namespace sf

struct s_plan_t {
  s_prec prec;
  const s_pattern_t* a;
  const s_pattern_t* b;
  const s_pattern_t* c;
  sf::MulDesc fwd;
  sf::MulDesc adjA;  // dA = P_{S_A}(dC B^T), built on first use
  sf::MulDesc adjB;  // dB = P_{S_B}(A^T dC)
  bool adj_built = false;
  float tune_ms[16] = {0};
};
