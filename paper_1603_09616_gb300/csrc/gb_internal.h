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
  // Banded Cholesky S = L L^T on the padded size 4 nb (rows >= n are identity),
  // FP32, when S's half-bandwidth chol_bw is at most 63 (0: not available):
  // chol_up[i*64 + t] = L(i+1+t, i), chol_row[i*64 + t] = L(i, i-1-t), zero
  // outside the band; chol_invd[i] = 1 / L(i, i).
  int32_t chol_bw = 0;
  std::vector<float> chol_up, chol_row, chol_invd;
};

gb_status validate_csr(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* h,
                       const double* s);
gb_status build_host_bsr(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* h,
                         const double* s, HostBSR* out);
void preconditioned_s_bounds(HostBSR* hb);
void band_cholesky(HostBSR* hb);

}  // namespace gb
