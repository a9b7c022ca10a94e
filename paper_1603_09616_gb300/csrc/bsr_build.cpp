// Host side of gb_build_bsr: CSR validation and regrouping into 4x4 blocks.
//
// The operators H and S of (z S - H) x = b (Introduction) arrive as one CSR
// pattern.  The GPU kernels work on 4x4 blocks over the orbital index: a block
// row covers orbitals 4I..4I+3, a stored block (I, J) holds every pattern entry
// with row in block row I and column in block column J (missing entries and
// rows past n are zero).  Carbon atoms (4 orbitals, ordered consecutively and
// 4-aligned by the generators) fill whole blocks; 1-orbital hydrogens pack
// four to a block.  The builder also inverts S's diagonal blocks (Cholesky) for
// the block-Jacobi preconditioner of the inner CG.
#include "gb_internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace gb {

static bool chol4_inverse(const double* a, double* inv) {
  // a: 4x4 symmetric; returns false unless positive definite.
  double l[16] = {0};
  for (int i = 0; i < 4; ++i) {
    for (int j = 0; j <= i; ++j) {
      double s = a[i * 4 + j];
      for (int k = 0; k < j; ++k) s -= l[i * 4 + k] * l[j * 4 + k];
      if (i == j) {
        if (!(s > 0.0) || !std::isfinite(s)) return false;
        l[i * 4 + i] = std::sqrt(s);
      } else {
        l[i * 4 + j] = s / l[j * 4 + j];
      }
    }
  }
  // inverse of L (lower triangular)
  double li[16] = {0};
  for (int i = 0; i < 4; ++i) {
    li[i * 4 + i] = 1.0 / l[i * 4 + i];
    for (int j = 0; j < i; ++j) {
      double s = 0.0;
      for (int k = j; k < i; ++k) s += l[i * 4 + k] * li[k * 4 + j];
      li[i * 4 + j] = -s / l[i * 4 + i];
    }
  }
  // A^-1 = L^-T L^-1
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = 0.0;
      for (int k = std::max(i, j); k < 4; ++k) s += li[k * 4 + i] * li[k * 4 + j];
      inv[i * 4 + j] = s;
    }
  return true;
}

gb_status validate_csr(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* h,
                       const double* s) {
  if (n <= 0 || n >= (int64_t(1) << 31)) return fail(GB_EINVAL, "n must be in [1, 2^31)");
  if (!row_ptr || !col_idx || !h || !s) return fail(GB_EINVAL, "NULL CSR array");
  if (row_ptr[0] != 0) return fail(GB_EINVAL, "row_ptr[0] must be 0");
  for (int64_t i = 0; i < n; ++i)
    if (row_ptr[i + 1] < row_ptr[i]) return fail(GB_EINVAL, "row_ptr must be non-decreasing");
  const int64_t nnz = row_ptr[n];
  if (nnz >= (int64_t(1) << 31)) return fail(GB_EINVAL, "nnz must be < 2^31");
  for (int64_t i = 0; i < n; ++i) {
    bool diag = false;
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
      const int32_t c = col_idx[e];
      if (c < 0 || c >= n) return fail(GB_EINVAL, "column index out of range in row %lld", (long long)i);
      if (e > row_ptr[i] && col_idx[e - 1] >= c)
        return fail(GB_EINVAL, "columns not strictly increasing in row %lld", (long long)i);
      if (c == i) diag = true;
      if (!std::isfinite(h[e]) || !std::isfinite(s[e])) return fail(GB_EINVAL, "non-finite value in row %lld", (long long)i);
    }
    if (!diag) return fail(GB_EINVAL, "diagonal entry missing in row %lld", (long long)i);
  }
  // symmetry of pattern and values
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
      const int32_t j = col_idx[e];
      if (j <= i) continue;
      const int32_t* lo = col_idx + row_ptr[j];
      const int32_t* hi = col_idx + row_ptr[j + 1];
      const int32_t* f = std::lower_bound(lo, hi, (int32_t)i);
      if (f == hi || *f != i) return fail(GB_EINVAL, "pattern not symmetric at (%lld, %d)", (long long)i, j);
      const int64_t t = f - col_idx;
      if (h[t] != h[e] || s[t] != s[e]) return fail(GB_EINVAL, "H or S not symmetric at (%lld, %d)", (long long)i, j);
    }
  }
  return GB_OK;
}

gb_status build_host_bsr(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* h,
                         const double* s, HostBSR* out) {
  gb_status st = validate_csr(n, row_ptr, col_idx, h, s);
  if (st != GB_OK) return st;
  const int64_t nb = (n + 3) / 4;
  out->n = n;
  out->nb = nb;
  out->nnz = row_ptr[n];
  out->blk_ptr.assign(nb + 1, 0);
  out->blk_col.clear();
  std::vector<int32_t> cols;
  int32_t max_row = 0;
  for (int64_t i = 0; i < n; ++i) max_row = std::max<int32_t>(max_row, (int32_t)(row_ptr[i + 1] - row_ptr[i]));
  out->max_row = max_row;
  for (int64_t I = 0; I < nb; ++I) {
    cols.clear();
    for (int64_t i = 4 * I; i < std::min<int64_t>(4 * I + 4, n); ++i)
      for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) cols.push_back(col_idx[e] / 4);
    std::sort(cols.begin(), cols.end());
    cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
    out->blk_col.insert(out->blk_col.end(), cols.begin(), cols.end());
    out->blk_ptr[I + 1] = (int32_t)out->blk_col.size();
  }
  const int64_t nnzb = (int64_t)out->blk_col.size();
  out->nnzb = nnzb;
  out->blk_h.assign(nnzb * 16, 0.0);
  out->blk_s.assign(nnzb * 16, 0.0);
  for (int64_t I = 0; I < nb; ++I) {
    const int32_t b0 = out->blk_ptr[I], b1 = out->blk_ptr[I + 1];
    for (int64_t i = 4 * I; i < std::min<int64_t>(4 * I + 4, n); ++i) {
      for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        const int32_t J = col_idx[e] / 4;
        const int32_t* f = std::lower_bound(out->blk_col.data() + b0, out->blk_col.data() + b1, J);
        const int64_t b = f - out->blk_col.data();
        const int r = (int)(i - 4 * I), c = col_idx[e] % 4;
        out->blk_h[b * 16 + r * 4 + c] = h[e];
        out->blk_s[b * 16 + r * 4 + c] = s[e];
      }
    }
  }
  // block-Jacobi inverses of S's diagonal blocks (padding rows get a unit diagonal)
  out->minv.assign(nb * 16, 0.0);
  for (int64_t I = 0; I < nb; ++I) {
    const int32_t b0 = out->blk_ptr[I], b1 = out->blk_ptr[I + 1];
    const int32_t* f = std::lower_bound(out->blk_col.data() + b0, out->blk_col.data() + b1, (int32_t)I);
    double a[16];
    std::memcpy(a, out->blk_s.data() + (f - out->blk_col.data()) * 16, sizeof a);
    for (int r = 0; r < 4; ++r)
      if (4 * I + r >= n) a[r * 4 + r] = 1.0;
    if (!chol4_inverse(a, out->minv.data() + I * 16))
      return fail(GB_ENOTSPD, "diagonal 4x4 block %lld of S is not positive definite", (long long)I);
  }
  out->row_ptr.assign(row_ptr, row_ptr + n + 1);
  out->col_idx.assign(col_idx, col_idx + row_ptr[n]);
  out->h_val.assign(h, h + row_ptr[n]);
  out->s_val.assign(s, s + row_ptr[n]);
  return GB_OK;
}

// Extreme eigenvalues of M^-1 S (M = block diagonal of S) by Lanczos on the
// symmetric similar operator T = L^-1 S L^-T (M = L L^T per 4x4 block), then
// bisection on the Sturm count of the tridiagonal matrix.  These bounds set
// the Chebyshev inner iteration of the mixed path.
void preconditioned_s_bounds(HostBSR* hb) {
  const int64_t nb = hb->nb, n4 = 4 * nb;
  // Cholesky factors of the diagonal blocks: minv = L^-T L^-1, so recover L^-1
  // from the diagonal blocks directly.
  std::vector<double> linv(nb * 16, 0.0);
  for (int64_t I = 0; I < nb; ++I) {
    const int32_t b0 = hb->blk_ptr[I], b1 = hb->blk_ptr[I + 1];
    const int32_t* f = std::lower_bound(hb->blk_col.data() + b0, hb->blk_col.data() + b1, (int32_t)I);
    double a[16], l[16] = {0};
    std::memcpy(a, hb->blk_s.data() + (f - hb->blk_col.data()) * 16, sizeof a);
    for (int r = 0; r < 4; ++r)
      if (4 * I + r >= hb->n) a[r * 4 + r] = 1.0;
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j <= i; ++j) {
        double v = a[i * 4 + j];
        for (int k = 0; k < j; ++k) v -= l[i * 4 + k] * l[j * 4 + k];
        l[i * 4 + j] = (i == j) ? std::sqrt(v) : v / l[j * 4 + j];
      }
    double* li = linv.data() + I * 16;
    for (int i = 0; i < 4; ++i) {
      li[i * 4 + i] = 1.0 / l[i * 4 + i];
      for (int j = 0; j < i; ++j) {
        double v = 0.0;
        for (int k = j; k < i; ++k) v += l[i * 4 + k] * li[k * 4 + j];
        li[i * 4 + j] = -v / l[i * 4 + i];
      }
    }
  }
  auto apply_T = [&](const std::vector<double>& v, std::vector<double>& out, std::vector<double>& tmp) {
    // tmp = L^-T v, out = S tmp, out = L^-1 out (per block)
    for (int64_t I = 0; I < nb; ++I)
      for (int r = 0; r < 4; ++r) {
        double acc = 0.0;
        for (int t = 0; t < 4; ++t) acc += linv[I * 16 + t * 4 + r] * v[4 * I + t];
        tmp[4 * I + r] = acc;
      }
    for (int64_t I = 0; I < nb; ++I) {
      double acc[4] = {0, 0, 0, 0};
      for (int32_t b = hb->blk_ptr[I]; b < hb->blk_ptr[I + 1]; ++b) {
        const int32_t J = hb->blk_col[b];
        const double* blk = hb->blk_s.data() + (size_t)b * 16;
        for (int r = 0; r < 4; ++r)
          for (int t = 0; t < 4; ++t) acc[r] += blk[r * 4 + t] * tmp[4 * J + t];
      }
      for (int r = 0; r < 4; ++r) {
        double v2 = 0.0;
        for (int t = 0; t <= r; ++t) v2 += linv[I * 16 + r * 4 + t] * acc[t];
        out[4 * I + r] = (4 * I + r < hb->n) ? v2 : 0.0;
      }
    }
  };
  const int steps = (int)std::min<int64_t>(60, std::max<int64_t>(2, hb->n));
  std::vector<double> v(n4, 0.0), vp(n4, 0.0), w(n4), tmp(n4);
  uint64_t st = 0x9E3779B97F4A7C15ull;  // deterministic start vector
  double nrm = 0.0;
  for (int64_t i = 0; i < hb->n; ++i) {
    st ^= st << 13; st ^= st >> 7; st ^= st << 17;
    v[i] = (double)(st >> 11) / 9007199254740992.0 - 0.5;
    nrm += v[i] * v[i];
  }
  nrm = std::sqrt(nrm);
  for (auto& x : v) x /= nrm;
  std::vector<double> alpha, beta;
  double bprev = 0.0;
  for (int j = 0; j < steps; ++j) {
    apply_T(v, w, tmp);
    for (int64_t i = 0; i < n4; ++i) w[i] -= bprev * vp[i];
    double al = 0.0;
    for (int64_t i = 0; i < n4; ++i) al += w[i] * v[i];
    for (int64_t i = 0; i < n4; ++i) w[i] -= al * v[i];
    double bn = 0.0;
    for (int64_t i = 0; i < n4; ++i) bn += w[i] * w[i];
    bn = std::sqrt(bn);
    alpha.push_back(al);
    if (bn < 1e-12 || j == steps - 1) break;
    beta.push_back(bn);
    for (int64_t i = 0; i < n4; ++i) {
      vp[i] = v[i];
      v[i] = w[i] / bn;
    }
    bprev = bn;
  }
  const int m = (int)alpha.size();
  auto count_below = [&](double x) {  // Sturm count of eigenvalues < x
    int c = 0;
    double q = alpha[0] - x;
    if (q < 0) ++c;
    for (int i = 1; i < m; ++i) {
      const double qq = (q == 0.0) ? 1e-300 : q;
      q = alpha[i] - x - beta[i - 1] * beta[i - 1] / qq;
      if (q < 0) ++c;
    }
    return c;
  };
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? std::fabs(beta[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(beta[i]) : 0.0);
    lo = std::min(lo, alpha[i] - r);
    hi = std::max(hi, alpha[i] + r);
  }
  auto bisect = [&](int k) {  // k-th smallest eigenvalue of the tridiagonal matrix
    double a = lo, b = hi;
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (a + b);
      if (count_below(mid) > k) b = mid;
      else a = mid;
    }
    return 0.5 * (a + b);
  };
  hb->lam_min = bisect(0);
  hb->lam_max = bisect(m - 1);
}

// Block-bidiagonal form of the banded Cholesky factor of S, for an exact S^-1
// (triangular solves instead of an iteration).  S's entries come from the 4x4
// blocks; rows past n (block padding) and past 4 nb (64-row padding) are
// identity.  The band factor S = L L^T is taken column by column in FP64; with
// half-bandwidth bw <= 63, L cut into 64-row blocks is block lower bidiagonal:
// diagonal blocks D_i (lower triangular) and sub-diagonal blocks C_i whose
// nonzeros sit in their last bw columns.  The solve then reads
//   L y = r  :  y_i = D_i^-1 r_i - E_i y_{i-1},      E_i = D_i^-1 C_i,
//   L^T x = y:  x_i = D_i^-T y_i - F_i x_{i+1},      F_i = D_i^-T C_{i+1}^T,
// where every D_i^-1 r_i is independent of the others and only the E / F
// products form the sequential chain.  Skipped (bf_bw = 0) when the
// half-bandwidth exceeds 63 or a pivot is not positive.
void block_factor(HostBSR* hb) {
  hb->bf_bw = 0;
  hb->bf_nblk = 0;
  hb->bf.clear();
  const int64_t n4 = 4 * hb->nb, n = hb->n;
  int64_t bw = 0;
  for (int64_t I = 0; I < hb->nb; ++I)
    for (int32_t b = hb->blk_ptr[I]; b < hb->blk_ptr[I + 1]; ++b) {
      const int64_t J = hb->blk_col[b];
      for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
          const int64_t i = 4 * I + r, j = 4 * J + c;
          if (i < n && j < n && j <= i && hb->blk_s[(size_t)b * 16 + r * 4 + c] != 0.0) bw = std::max(bw, i - j);
        }
    }
  if (bw > 63) return;
  const int64_t w = bw + 1;  // stored band entries per row, diagonal last
  std::vector<double> L((size_t)(n4 * w), 0.0);
  auto at = [&](int64_t i, int64_t j) -> double& { return L[(size_t)(i * w + (j - i + bw))]; };
  for (int64_t I = 0; I < hb->nb; ++I)
    for (int32_t b = hb->blk_ptr[I]; b < hb->blk_ptr[I + 1]; ++b) {
      const int64_t J = hb->blk_col[b];
      for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
          const int64_t i = 4 * I + r, j = 4 * J + c;
          if (i < n && j < n && j <= i && i - j <= bw) at(i, j) = hb->blk_s[(size_t)b * 16 + r * 4 + c];
        }
    }
  for (int64_t i = n; i < n4; ++i) at(i, i) = 1.0;
  for (int64_t i = 0; i < n4; ++i) {
    const int64_t j0 = std::max<int64_t>(0, i - bw);
    for (int64_t j = j0; j <= i; ++j) {
      double sum = at(i, j);
      for (int64_t k = std::max(j0, j - bw); k < j; ++k) sum -= at(i, k) * at(j, k);
      if (j < i) {
        at(i, j) = sum / at(j, j);
      } else {
        if (!(sum > 0.0)) return;
        at(i, i) = std::sqrt(sum);
      }
    }
  }
  // L(i, j) on the 64-row padded size (identity past 4 nb)
  auto Lget = [&](int64_t i, int64_t j) -> double {
    if (i >= n4 || j >= n4) return i == j ? 1.0 : 0.0;
    if (j > i || i - j > bw) return 0.0;
    return at(i, j);
  };
  const int64_t nblk = (n4 + 63) / 64;
  const size_t T = 4096, part = (size_t)nblk * T;
  hb->bf.assign(4 * part, 0.0);
  double* df = hb->bf.data();
  double* db = df + part;
  double* ef = db + part;
  double* fb = ef + part;
  std::vector<double> D(T), Di(T), C(T);
  for (int64_t blk = 0; blk < nblk; ++blk) {
    const int64_t base = 64 * blk;
    for (int r = 0; r < 64; ++r)
      for (int c = 0; c < 64; ++c) D[r * 64 + c] = c <= r ? Lget(base + r, base + c) : 0.0;
    // Di = D^-1 by forward substitution on each unit column
    std::fill(Di.begin(), Di.end(), 0.0);
    for (int c = 0; c < 64; ++c)
      for (int r = c; r < 64; ++r) {
        double s = (r == c) ? 1.0 : 0.0;
        for (int k = c; k < r; ++k) s -= D[r * 64 + k] * Di[k * 64 + c];
        Di[r * 64 + c] = s / D[r * 64 + r];
      }
    // k-major storage: M[k * 64 + r] = (matrix)[r][k]
    for (int k = 0; k < 64; ++k)
      for (int r = 0; r < 64; ++r) {
        df[blk * T + k * 64 + r] = Di[r * 64 + k];
        db[blk * T + k * 64 + r] = Di[k * 64 + r];
      }
    if (blk > 0) {  // E = Di C_blk, C_blk = L(block blk, block blk-1)
      for (int r = 0; r < 64; ++r)
        for (int c = 0; c < 64; ++c) C[r * 64 + c] = Lget(base + r, base - 64 + c);
      for (int r = 0; r < 64; ++r)
        for (int k = 0; k < 64; ++k) {
          double s = 0.0;
          for (int q = 0; q <= r; ++q) s += Di[r * 64 + q] * C[q * 64 + k];
          ef[blk * T + k * 64 + r] = s;
        }
    }
    if (blk + 1 < nblk) {  // F = Di^T C_{blk+1}^T, C_{blk+1} = L(block blk+1, block blk)
      for (int r = 0; r < 64; ++r)
        for (int c = 0; c < 64; ++c) C[r * 64 + c] = Lget(base + 64 + r, base + c);
      for (int r = 0; r < 64; ++r)
        for (int k = 0; k < 64; ++k) {
          double s = 0.0;
          for (int q = r; q < 64; ++q) s += Di[q * 64 + r] * C[k * 64 + q];
          fb[blk * T + k * 64 + r] = s;
        }
    }
  }
  hb->bf_bw = (int32_t)bw;
  hb->bf_nblk = nblk;
}

// Fragment order of an m16n8k8 TF32 A operand (PTX mma): lane l = 4 g + t
// holds a0 = A(g, t), a1 = A(g + 8, t), a2 = A(g, t + 4), a3 = A(g + 8, t + 4)
// of the 16 x 8 tile (rows 16 mi.., columns 8 ks..).  A fragment is stored as
// 128 consecutive floats, lane l's four values at 4 l .. 4 l + 3.
static void put_fragment(const double* M, int mi, int ks, float* dst) {  // M k-major: (r, k) at k * 64 + r
  for (int l = 0; l < 32; ++l) {
    const int g = l >> 2, t = l & 3;
    for (int sl = 0; sl < 4; ++sl) {
      const int r = 16 * mi + g + 8 * (sl & 1), k = 8 * ks + t + 4 * (sl >> 1);
      dst[l * 4 + sl] = (float)M[(size_t)k * 64 + r];
    }
  }
}

// Per block: the FWD tile holds the D^-1 fragments a lower-triangular product
// needs (k-step ks, row tile mi >= ks / 2; 20 of them, by ks then mi), then
// the E fragments of k-steps (64 - bw) / 8 .. 7 (by ks then mi); the BWD tile
// holds the D^-T fragments with mi <= ks / 2 (20), then the F fragments of
// k-steps 0 .. ceil(bw / 8) - 1.
std::vector<float> mma_tiles(const HostBSR& hb) {
  std::vector<float> out;
  if (hb.bf_bw <= 0 || hb.bf.empty()) return out;
  const int64_t nblk = hb.bf_nblk;
  const size_t part = (size_t)nblk * 4096;
  const double* df = hb.bf.data();
  const double* db = df + part;
  const double* ef = db + part;
  const double* fb = ef + part;
  const int bw = hb.bf_bw, ksE0 = (64 - bw) / 8, nF = (bw + 7) / 8;
  out.assign((size_t)2 * nblk * kMmaTileFloats, 0.f);
  for (int64_t blk = 0; blk < nblk; ++blk) {
    float* fwd = out.data() + (size_t)(2 * blk) * kMmaTileFloats;
    float* bwd = fwd + kMmaTileFloats;
    int p = 0;
    for (int ks = 0; ks < 8; ++ks)
      for (int mi = ks / 2; mi < 4; ++mi) put_fragment(df + (size_t)blk * 4096, mi, ks, fwd + 128 * p++);
    for (int ks = ksE0; ks < 8; ++ks)
      for (int mi = 0; mi < 4; ++mi) put_fragment(ef + (size_t)blk * 4096, mi, ks, fwd + 128 * p++);
    p = 0;
    for (int ks = 0; ks < 8; ++ks)
      for (int mi = 0; mi <= ks / 2; ++mi) put_fragment(db + (size_t)blk * 4096, mi, ks, bwd + 128 * p++);
    for (int ks = 0; ks < nF; ++ks)
      for (int mi = 0; mi < 4; ++mi) put_fragment(fb + (size_t)blk * 4096, mi, ks, bwd + 128 * p++);
  }
  return out;
}

}  // namespace gb
