// Internal declarations shared by the host builder and the CUDA translation unit.
#pragma once

#include <cstdarg>
#include <cstdint>
#include <vector>

#include "../../include/gbgreen.h"

namespace gb {

// Thread-local last-error message; returns `st` so callers can `return fail(...)`.
gb_status fail(gb_status st, const char* fmt, ...);
void clear_error();

struct HostBSR {
  int64_t n = 0, nb = 0, nnz = 0, nnzb = 0;
  int32_t max_row = 0;
  std::vector<int32_t> blk_ptr, blk_col;
  std::vector<double> blk_h, blk_s, minv;  // 16 doubles per block, row-major
  std::vector<int64_t> row_ptr;
  std::vector<int32_t> col_idx;
  std::vector<double> h_val, s_val;
  double lam_min = 0.0, lam_max = 0.0;  // spectrum bounds of M^-1 S (block Jacobi M)
  // Block-bidiagonal form of the banded Cholesky factor S = L L^T on 64-row
  // blocks (see block_factor), FP64, when S's half-bandwidth bf_bw is at most
  // 63 (0: not available).  bf holds four [bf_nblk][64][64] arrays, each
  // stored k-major (entry (r, k) of the block's matrix at k * 64 + r):
  // D_i^-1, D_i^-T, E_i = D_i^-1 C_i and F_i = D_i^-T C_{i+1}^T.
  int32_t bf_bw = 0;
  int64_t bf_nblk = 0;
  std::vector<double> bf;
};

gb_status validate_csr(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* h,
                       const double* s);
gb_status build_host_bsr(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* h,
                         const double* s, HostBSR* out);
void preconditioned_s_bounds(HostBSR* hb);
void block_factor(HostBSR* hb);

// The FP32 factor rearranged for the tensor-core passes of the exact inner
// solve (block_chol.cuh): per 64-row block two tiles of kMmaTilePairs
// fragments (FWD: D^-1 then E; BWD: D^-T then F), each fragment the 32 x 4
// values one warp loads for an m16n8k8 TF32 A operand.  Returns
// 2 * nblk * kMmaTileFloats floats (empty without a factor).
constexpr int kMmaTilePairs = 52;                     // 20 triangular + up to 32 band fragments
constexpr int kMmaTileFloats = kMmaTilePairs * 128;  // 26,624 bytes
std::vector<float> mma_tiles(const HostBSR& hb);

}  // namespace gb
