// C ABI of the GB300 shifted Green's-function library (declared in gbgreen.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "gb_internal.h"
#include "panel.cuh"

namespace gb {

static thread_local char g_err[512];

gb_status fail(gb_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return st;
}
void clear_error() { g_err[0] = 0; }

static gb_status cuda_fail(cudaError_t e, const char* what) {
  return fail(GB_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define GB_CUDA(call)                                 \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Caller-owned device buffers are read and written with vector accesses of
// their element size (complex doubles as 16-byte double2): a pointer off that
// boundary is an error, found here instead of as a misaligned access.
static bool misaligned(const void* p, size_t bytes) { return p && (reinterpret_cast<uintptr_t>(p) % bytes) != 0; }
static gb_status check_outputs(const gb_outputs* o) {
  if (misaligned(o->ldos, 8) || misaligned(o->rho, 8) || misaligned(o->edm, 8) || misaligned(o->q, 8) ||
      misaligned(o->e_loc, 8) || misaligned(o->resid, 8) || misaligned(o->iters, 4) ||
      misaligned(o->inner_iters, 4) || misaligned(o->col_status, 4) || misaligned(o->g_proj, 16))
    return fail(GB_EINVAL, "an output is not aligned to its element (g_proj: 16 bytes)");
  return GB_OK;
}

}  // namespace gb

struct gb_matrix {
  int device = 0;
  int64_t n = 0, nb = 0, nnz = 0, nnzb = 0;
  int32_t max_row = 0;
  std::vector<int64_t> h_row_ptr;  // host copy of the pattern's row pointers
  void* base = nullptr;
  gbk::DevMat dm{};
};

namespace gb {
const gbk::DevMat* devmat_of(const gb_matrix* m) { return &m->dm; }
}  // namespace gb

using namespace gb;

// ------------------------------------------------------------ standalone SpMM
namespace {

// Single-column panels (FP32): one warp per block row, lane l takes the
// stored blocks b0 + l, b0 + l + 32, ... with ALL W columns, so the warp reads
// consecutive 64-byte blocks (one coalesced stream of the matrix) and each x
// gather is one contiguous run of 4 rows x W columns; a xor-shuffle reduction
// then sums the 4 x W complex partials.
template <int WC>
__device__ __forceinline__ void spmm_row_lanes_f(const gbk::DevMat& m, const float* __restrict__ A,
                                                 const float2* __restrict__ x, float2* __restrict__ y, int lane,
                                                 int I) {
  float2 acc[4][WC];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < WC; ++c) acc[r][c] = make_float2(0.f, 0.f);
  const int b1 = m.blk_ptr[I + 1];
  for (int b = m.blk_ptr[I] + lane; b < b1; b += 32) {
    const int J = __ldg(m.blk_col + b);
    const float4* ab = reinterpret_cast<const float4*>(A + (size_t)b * 16);
    float4 a[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) a[r] = __ldg(ab + r);
    float2 xv[4][WC];
    const float2* xr = x + (size_t)(4 * J) * WC;
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
      for (int c = 0; c < WC; ++c) xv[t][c] = xr[t * WC + c];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < WC; ++c) {
        acc[r][c].x = fmaf(a[r].x, xv[0][c].x, acc[r][c].x);
        acc[r][c].y = fmaf(a[r].x, xv[0][c].y, acc[r][c].y);
        acc[r][c].x = fmaf(a[r].y, xv[1][c].x, acc[r][c].x);
        acc[r][c].y = fmaf(a[r].y, xv[1][c].y, acc[r][c].y);
        acc[r][c].x = fmaf(a[r].z, xv[2][c].x, acc[r][c].x);
        acc[r][c].y = fmaf(a[r].z, xv[2][c].y, acc[r][c].y);
        acc[r][c].x = fmaf(a[r].w, xv[3][c].x, acc[r][c].x);
        acc[r][c].y = fmaf(a[r].w, xv[3][c].y, acc[r][c].y);
      }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < WC; ++c) {
        acc[r][c].x += __shfl_xor_sync(0xffffffffu, acc[r][c].x, off);
        acc[r][c].y += __shfl_xor_sync(0xffffffffu, acc[r][c].y, off);
      }
  const int nrow = min(4, m.n - 4 * I);
  // lane r * WC + c stores (row r, column c)
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < WC; ++c)
      if (lane == r * WC + c && r < nrow) y[(size_t)(4 * I + r) * WC + c] = acc[r][c];
}

// Narrow FP32 panels (W = 1, 2, 4): one warp per block row, lane l owns row
// r = l % 4 of the stored blocks b0 + l / 4, b0 + l / 4 + 8, ...  The lanes of
// a warp read 8 whole consecutive blocks per step (512 contiguous bytes: each
// 32-byte sector requested once), the 4 lanes of a block share its x gather
// (same addresses, one request), and every lane accumulates a single row, so
// the reduction is three xor-shuffle levels over the 8 block slots.  Requires
// x 16-byte aligned (float4 loads of the 4 x W gathered entries).
// acc[c] += (row of a block) . x[4 rows, column c]; the complex x entry
// (row t, column c) is float2 number t * WC + c of the gathered float4s.
template <int WC>
__device__ __forceinline__ void quad_fma(const float4& a, const float4 (&xv)[2 * WC], float2 (&acc)[WC]) {
#pragma unroll
  for (int c = 0; c < WC; ++c) {
    float xr[4], xi[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int f = t * WC + c;
      const float4 q = xv[f >> 1];
      xr[t] = (f & 1) ? q.z : q.x;
      xi[t] = (f & 1) ? q.w : q.y;
    }
    acc[c].x = fmaf(a.x, xr[0], fmaf(a.y, xr[1], fmaf(a.z, xr[2], fmaf(a.w, xr[3], acc[c].x))));
    acc[c].y = fmaf(a.x, xi[0], fmaf(a.y, xi[1], fmaf(a.z, xi[2], fmaf(a.w, xi[3], acc[c].y))));
  }
}

// The kernel is bound by loads in flight: the block columns are fetched a
// step ahead, W = 1 keeps two 8-block steps in flight per lane and W = 2 one,
// at 40 registers (48 warps per SM) without spills.
template <int WC>
__global__ void __launch_bounds__(256, 6)
    spmm_quad_kernel(const gbk::DevMat m, const float* __restrict__ A, const float2* __restrict__ x,
                     float2* __restrict__ y) {
  const long long I = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  if (I >= m.nb) return;  // uniform per warp
  const int lane = threadIdx.x & 31, r = lane & 3, s = lane >> 2;
  constexpr int U = WC == 1 ? 2 : 1;  // steps of 8 blocks in flight per lane
  constexpr int NQ = 2 * WC;  // float4 per gathered 4 x WC complex x block
  float2 acc[WC];
#pragma unroll
  for (int c = 0; c < WC; ++c) acc[c] = make_float2(0.f, 0.f);
  const int b1 = m.blk_ptr[I + 1];
  const float4* __restrict__ A4 = reinterpret_cast<const float4*>(A);
  const float4* __restrict__ X4 = reinterpret_cast<const float4*>(x);
  int b = m.blk_ptr[I] + s;
  // block columns one step ahead: the x gathers of a step then wait for one
  // memory round trip, not two (column index, then x)
  int Jn[U];
#pragma unroll
  for (int u = 0; u < U; ++u) Jn[u] = b + 8 * u < b1 ? __ldcs(m.blk_col + b + 8 * u) : 0;
  for (; b + 8 * (U - 1) < b1; b += 8 * U) {
    int J[U];
    float4 a[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      J[u] = Jn[u];
      const int bn = b + 8 * U + 8 * u;
      Jn[u] = bn < b1 ? __ldcs(m.blk_col + bn) : 0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) a[u] = __ldcs(A4 + (size_t)(b + 8 * u) * 4 + r);
    float4 xv[U][NQ];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int q = 0; q < NQ; ++q) xv[u][q] = __ldg(X4 + (size_t)J[u] * NQ + q);
#pragma unroll
    for (int u = 0; u < U; ++u) quad_fma<WC>(a[u], xv[u], acc);
  }
  for (; b < b1; b += 8) {
    const int J = Jn[0];  // the loop above leaves the next step's columns in Jn
    const float4 a = __ldcs(A4 + (size_t)b * 4 + r);
#pragma unroll
    for (int u = 0; u + 1 < U; ++u) Jn[u] = Jn[u + 1];
    float4 xv[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) xv[q] = __ldg(X4 + (size_t)J * NQ + q);
    quad_fma<WC>(a, xv, acc);
  }
#pragma unroll
  for (int off = 4; off < 32; off <<= 1)
#pragma unroll
    for (int c = 0; c < WC; ++c) {
      acc[c].x += __shfl_xor_sync(0xffffffffu, acc[c].x, off);
      acc[c].y += __shfl_xor_sync(0xffffffffu, acc[c].y, off);
    }
  if (s == 0 && 4 * I + r < m.n) {
#pragma unroll
    for (int c = 0; c < WC; ++c) y[(size_t)(4 * I + r) * WC + c] = acc[c];
  }
}

// FP64 narrow panels (W = 1, 2), same quad layout as the FP32 kernel above:
// lane l accumulates row l mod 4 of the blocks b0 + floor(l / 4) + 8k, so a
// warp step reads 8 whole consecutive blocks (1 KB of values) and the 4 lanes
// of a block share its x gather.  The product is bound by the FP64 FMA pipe
// (GB300 runs FP64 at 1/64 of its FP32 rate), so the layout's job is to keep
// enough loads in flight that the pipe never waits: two 8-block steps per lane.
template <int WC>
__global__ void __launch_bounds__(256, 4)
    spmm_quad_d_kernel(const gbk::DevMat m, const double* __restrict__ A, const double2* __restrict__ x,
                       double2* __restrict__ y) {
  const long long I = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  if (I >= m.nb) return;  // uniform per warp
  const int lane = threadIdx.x & 31, r = lane & 3, s = lane >> 2;
  constexpr int U = 2;
  constexpr int NX = 4 * WC;  // double2 per gathered 4 x WC complex x block
  double2 acc[WC];
#pragma unroll
  for (int c = 0; c < WC; ++c) acc[c] = make_double2(0.0, 0.0);
  const int b1 = m.blk_ptr[I + 1];
  const double2* __restrict__ A2 = reinterpret_cast<const double2*>(A);
  auto step = [&](const double2 (&a)[2], const double2 (&xv)[NX]) {
    const double ar[4] = {a[0].x, a[0].y, a[1].x, a[1].y};
#pragma unroll
    for (int c = 0; c < WC; ++c)
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        acc[c].x = fma(ar[t], xv[t * WC + c].x, acc[c].x);
        acc[c].y = fma(ar[t], xv[t * WC + c].y, acc[c].y);
      }
  };
  int b = m.blk_ptr[I] + s;
  for (; b + 8 * (U - 1) < b1; b += 8 * U) {
    int J[U];
    double2 a[U][2], xv[U][NX];
#pragma unroll
    for (int u = 0; u < U; ++u) J[u] = __ldcs(m.blk_col + b + 8 * u);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      a[u][0] = __ldcs(A2 + (size_t)(b + 8 * u) * 8 + 2 * r);
      a[u][1] = __ldcs(A2 + (size_t)(b + 8 * u) * 8 + 2 * r + 1);
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int q = 0; q < NX; ++q) xv[u][q] = __ldg(x + (size_t)J[u] * NX + q);
#pragma unroll
    for (int u = 0; u < U; ++u) step(a[u], xv[u]);
  }
  for (; b < b1; b += 8) {
    const int J = __ldcs(m.blk_col + b);
    const double2 a[2] = {__ldcs(A2 + (size_t)b * 8 + 2 * r), __ldcs(A2 + (size_t)b * 8 + 2 * r + 1)};
    double2 xv[NX];
#pragma unroll
    for (int q = 0; q < NX; ++q) xv[q] = __ldg(x + (size_t)J * NX + q);
    step(a, xv);
  }
#pragma unroll
  for (int off = 4; off < 32; off <<= 1)
#pragma unroll
    for (int c = 0; c < WC; ++c) {
      acc[c].x += __shfl_xor_sync(0xffffffffu, acc[c].x, off);
      acc[c].y += __shfl_xor_sync(0xffffffffu, acc[c].y, off);
    }
  if (s == 0 && 4 * I + r < m.n) {
#pragma unroll
    for (int c = 0; c < WC; ++c) y[(size_t)(4 * I + r) * WC + c] = acc[c];
  }
}

// Wide panels (FP32: W = 4..64 in powers of two; FP64: W = 4..32): one warp
// per block row, split into G = 32 / CL groups of CL lanes; group g takes the
// blocks b0 + g + G k, and lane c of a group owns columns [c * PC, (c+1) * PC)
// of the panel (PC = 2 complex columns per lane in FP32, read and written as
// one float4; 1 in FP64).  A block's values are read by every lane of its
// group at one address (a broadcast), its x rows by the group as contiguous
// runs, and each value feeds PC complex columns from registers.  The groups
// then add up through xor shuffles.  Requires x and y 16-byte aligned.
// The kernel waits on loads (ncu at W = 8: long-scoreboard stalls dominate),
// so it keeps one step in flight per lane at <= 64 registers, which lets 32
// warps share an SM (two steps at 106 registers left 11 warps active).
template <int CL>
__global__ void __launch_bounds__(256, 4)
    spmm_wide_kernel(const gbk::DevMat m, const float* __restrict__ A, const float4* __restrict__ x,
                     float4* __restrict__ y) {
  constexpr int G = 32 / CL;
  const long long I = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  if (I >= m.nb) return;
  const int lane = threadIdx.x & 31, g = lane / CL, c = lane - g * CL;
  float4 acc[4];  // row r: (re, im) of columns 2c and 2c + 1
#pragma unroll
  for (int r = 0; r < 4; ++r) acc[r] = make_float4(0.f, 0.f, 0.f, 0.f);
  const float4* __restrict__ A4 = reinterpret_cast<const float4*>(A);
  auto step = [&](const float4 (&a)[4], const float4 (&xv)[4]) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const float ar[4] = {a[r].x, a[r].y, a[r].z, a[r].w};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        acc[r].x = fmaf(ar[t], xv[t].x, acc[r].x);
        acc[r].y = fmaf(ar[t], xv[t].y, acc[r].y);
        acc[r].z = fmaf(ar[t], xv[t].z, acc[r].z);
        acc[r].w = fmaf(ar[t], xv[t].w, acc[r].w);
      }
    }
  };
  const int b1 = m.blk_ptr[I + 1];
  int b = m.blk_ptr[I] + g;
  constexpr int U = 1;
  int Jn[U];  // block columns one step ahead (one round trip per step)
#pragma unroll
  for (int u = 0; u < U; ++u) Jn[u] = b + G * u < b1 ? __ldcs(m.blk_col + b + G * u) : 0;
  for (; b + G * (U - 1) < b1; b += G * U) {
    int J[U];
    float4 a[U][4], xv[U][4];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      J[u] = Jn[u];
      const int bn = b + G * U + G * u;
      Jn[u] = bn < b1 ? __ldcs(m.blk_col + bn) : 0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int r = 0; r < 4; ++r) a[u][r] = __ldcs(A4 + (size_t)(b + G * u) * 4 + r);
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int t = 0; t < 4; ++t) xv[u][t] = __ldg(x + (size_t)(4 * J[u] + t) * CL + c);
#pragma unroll
    for (int u = 0; u < U; ++u) step(a[u], xv[u]);
  }
  for (; b < b1; b += G) {
    const int J = Jn[0];
#pragma unroll
    for (int u = 0; u + 1 < U; ++u) Jn[u] = Jn[u + 1];
    float4 a[4], xv[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) a[r] = __ldcs(A4 + (size_t)b * 4 + r);
#pragma unroll
    for (int t = 0; t < 4; ++t) xv[t] = __ldg(x + (size_t)(4 * J + t) * CL + c);
    step(a, xv);
  }
#pragma unroll
  for (int off = CL; off < 32; off <<= 1)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      acc[r].x += __shfl_xor_sync(0xffffffffu, acc[r].x, off);
      acc[r].y += __shfl_xor_sync(0xffffffffu, acc[r].y, off);
      acc[r].z += __shfl_xor_sync(0xffffffffu, acc[r].z, off);
      acc[r].w += __shfl_xor_sync(0xffffffffu, acc[r].w, off);
    }
  if (g == 0) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (4 * I + r < m.n) y[(size_t)(4 * I + r) * CL + c] = acc[r];
  }
}

template <int CL>
__global__ void __launch_bounds__(256, 3)
    spmm_wide_d_kernel(const gbk::DevMat m, const double* __restrict__ A, const double2* __restrict__ x,
                       double2* __restrict__ y) {
  constexpr int G = 32 / CL;
  const long long I = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  if (I >= m.nb) return;
  const int lane = threadIdx.x & 31, g = lane / CL, c = lane - g * CL;
  double2 acc[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) acc[r] = make_double2(0.0, 0.0);
  const double2* __restrict__ A2 = reinterpret_cast<const double2*>(A);
  const int b1 = m.blk_ptr[I + 1];
  for (int b = m.blk_ptr[I] + g; b < b1; b += G) {
    const int J = __ldcs(m.blk_col + b);
    double2 a[8], xv[4];
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = __ldcs(A2 + (size_t)b * 8 + q);
#pragma unroll
    for (int t = 0; t < 4; ++t) xv[t] = __ldg(x + (size_t)(4 * J + t) * CL + c);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const double ar[4] = {a[2 * r].x, a[2 * r].y, a[2 * r + 1].x, a[2 * r + 1].y};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        acc[r].x = fma(ar[t], xv[t].x, acc[r].x);
        acc[r].y = fma(ar[t], xv[t].y, acc[r].y);
      }
    }
  }
#pragma unroll
  for (int off = CL; off < 32; off <<= 1)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      acc[r].x += __shfl_xor_sync(0xffffffffu, acc[r].x, off);
      acc[r].y += __shfl_xor_sync(0xffffffffu, acc[r].y, off);
    }
  if (g == 0) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (4 * I + r < m.n) y[(size_t)(4 * I + r) * CL + c] = acc[r];
  }
}

template <bool F64>
__global__ void spmm_kernel(const gbk::DevMat m, int which, int W, const void* __restrict__ xv,
                            void* __restrict__ yv) {
  const int lane = threadIdx.x & 31;
  if constexpr (!F64) {
    if (W == 1) {  // x not 16-byte aligned (else spmm_quad_kernel): lane per block
      const long long warp0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
      const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
      const float* A = which ? m.sb_hi : m.hb_hi;
      const float2* x = static_cast<const float2*>(xv);
      float2* y = static_cast<float2*>(yv);
      for (long long I = warp0; I < m.nb; I += nwarps) spmm_row_lanes_f<1>(m, A, x, y, lane, (int)I);
      return;
    }
  }
  if (W <= 8) {
    // narrow panels: one warp per block row, lanes split the stored blocks
    const long long warp0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    int Wp = 1;
    while (Wp < W) Wp <<= 1;
    const int c = lane % Wp;
    const bool active = c < W;
    for (long long I = warp0; I < m.nb; I += nwarps) {
      const int nrow = min(4, m.n - 4 * (int)I);
      if constexpr (F64) {
        double2 acc[4];
        gbk::wbsr_row_d(m, which ? m.sb : m.hb, static_cast<const double2*>(xv), W, Wp, lane, (int)I, active, acc);
        double2* y = static_cast<double2*>(yv);
        if (lane < Wp && active)
          for (int r = 0; r < nrow; ++r) y[(size_t)(4 * I + r) * W + c] = acc[r];
      } else {
        float2 acc[4];
        gbk::wbsr_row_f(m, which ? m.sb_hi : m.hb_hi, static_cast<const float2*>(xv), W, Wp, lane, (int)I, active,
                        acc);
        float2* y = static_cast<float2*>(yv);
        if (lane < Wp && active)
          for (int r = 0; r < nrow; ++r) y[(size_t)(4 * I + r) * W + c] = acc[r];
      }
    }
    return;
  }
  // wide panels: one thread per (block row, column), consecutive threads take consecutive columns
  const long long items = (long long)m.nb * W;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < items;
       it += (long long)gridDim.x * blockDim.x) {
    const int I = (int)(it / W), c = (int)(it - (long long)I * W);
    const int nrow = min(4, m.n - 4 * I);
    if constexpr (F64) {
      double2 acc[4];
      gbk::bsr_row_d(m, which ? m.sb : m.hb, static_cast<const double2*>(xv), W, c, I, acc);
      double2* y = static_cast<double2*>(yv);
      for (int r = 0; r < nrow; ++r) y[(size_t)(4 * I + r) * W + c] = acc[r];
    } else {
      float2 acc[4];
      gbk::bsr_row_f(m, which ? m.sb_hi : m.hb_hi, static_cast<const float2*>(xv), W, c, I, acc);
      float2* y = static_cast<float2*>(yv);
      for (int r = 0; r < nrow; ++r) y[(size_t)(4 * I + r) * W + c] = acc[r];
    }
  }
}

}  // namespace

// The standalone SpMM reads rows 4J..4J+3 of x for every stored block column
// J; when n % 4 != 0 the last block column reaches past row n-1 (its matrix
// entries are zero there), so gb_spmm reads from a zero-padded copy of x.

extern "C" {

int32_t gb_abi_version(void) { return GB_ABI_VERSION; }

const char* gb_last_error(void) { return gb::g_err; }

gb_status gb_bsr_to_host(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* h_val,
                         const double* s_val, int64_t* nb, int64_t* nnzb, int32_t* blk_ptr, int32_t* blk_col,
                         double* blk_h, double* blk_s) {
  clear_error();
  if (!nb || !nnzb) return fail(GB_EINVAL, "nb and nnzb must not be NULL");
  HostBSR hb;
  gb_status st = build_host_bsr(n, row_ptr, col_idx, h_val, s_val, &hb);
  if (st != GB_OK) return st;
  *nb = hb.nb;
  *nnzb = hb.nnzb;
  if (blk_ptr) std::memcpy(blk_ptr, hb.blk_ptr.data(), sizeof(int32_t) * hb.blk_ptr.size());
  if (blk_col) std::memcpy(blk_col, hb.blk_col.data(), sizeof(int32_t) * hb.blk_col.size());
  if (blk_h) std::memcpy(blk_h, hb.blk_h.data(), sizeof(double) * hb.blk_h.size());
  if (blk_s) std::memcpy(blk_s, hb.blk_s.data(), sizeof(double) * hb.blk_s.size());
  return GB_OK;
}

gb_status gb_block_factor_to_host(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* h_val,
                                  const double* s_val, int32_t* bw, int64_t* nblk, double* factor) {
  clear_error();
  if (!bw || !nblk) return fail(GB_EINVAL, "bw and nblk must not be NULL");
  HostBSR hb;
  gb_status st = build_host_bsr(n, row_ptr, col_idx, h_val, s_val, &hb);
  if (st != GB_OK) return st;
  block_factor(&hb);
  *bw = hb.bf_bw;
  *nblk = hb.bf_nblk;
  if (factor && !hb.bf.empty()) std::memcpy(factor, hb.bf.data(), sizeof(double) * hb.bf.size());
  return GB_OK;
}

gb_status gb_build_bsr(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* h_val,
                       const double* s_val, void* stream, gb_matrix** out) {
  clear_error();
  if (!out) return fail(GB_EINVAL, "out must not be NULL");
  *out = nullptr;
  HostBSR hb;
  gb_status st = build_host_bsr(n, row_ptr, col_idx, h_val, s_val, &hb);
  if (st != GB_OK) return st;
  preconditioned_s_bounds(&hb);
  block_factor(&hb);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0;
  GB_CUDA(cudaGetDevice(&dev));

  const size_t nnzb = hb.nnzb, nbl = hb.nb, nnz = hb.nnz;
  // one allocation, 256-byte aligned pieces
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  const size_t o_bp = take(sizeof(int) * (nbl + 1)), o_bc = take(sizeof(int) * nnzb);
  const size_t o_hb = take(sizeof(double) * nnzb * 16), o_sb = take(sizeof(double) * nnzb * 16);
  const size_t o_hh = take(sizeof(float) * nnzb * 16), o_hl = take(sizeof(float) * nnzb * 16);
  const size_t o_sh = take(sizeof(float) * nnzb * 16), o_sl = take(sizeof(float) * nnzb * 16);
  const size_t o_mi = take(sizeof(double) * nbl * 16), o_m32 = take(sizeof(float) * nbl * 16);
  const size_t o_rp = take(sizeof(int) * (n + 1)), o_ci = take(sizeof(int) * nnz);
  const size_t o_hv = take(sizeof(double) * nnz), o_sv = take(sizeof(double) * nnz);
  const size_t nbf = hb.bf.size();  // 4 x nblk x 4096 factor entries (0: no factor)
  const std::vector<float> mt = mma_tiles(hb);
  static_assert(kMmaTileFloats == gbk::kMmaTileFloatsDev, "tile size of host and device");
  const size_t o_bf64 = take(sizeof(double) * nbf), o_bfm = take(sizeof(float) * mt.size());
  const size_t total = off;

  std::vector<char> host(total, 0);
  auto put = [&](size_t o, const void* src, size_t bytes) { std::memcpy(host.data() + o, src, bytes); };
  put(o_bp, hb.blk_ptr.data(), sizeof(int) * (nbl + 1));
  put(o_bc, hb.blk_col.data(), sizeof(int) * nnzb);
  put(o_hb, hb.blk_h.data(), sizeof(double) * nnzb * 16);
  put(o_sb, hb.blk_s.data(), sizeof(double) * nnzb * 16);
  {
    float* hh = reinterpret_cast<float*>(host.data() + o_hh);
    float* hl = reinterpret_cast<float*>(host.data() + o_hl);
    float* sh = reinterpret_cast<float*>(host.data() + o_sh);
    float* sl = reinterpret_cast<float*>(host.data() + o_sl);
    for (size_t i = 0; i < nnzb * 16; ++i) {
      const float a = (float)hb.blk_h[i];
      hh[i] = a;
      hl[i] = (float)(hb.blk_h[i] - (double)a);
      const float b = (float)hb.blk_s[i];
      sh[i] = b;
      sl[i] = (float)(hb.blk_s[i] - (double)b);
    }
    float* m32 = reinterpret_cast<float*>(host.data() + o_m32);
    for (size_t i = 0; i < nbl * 16; ++i) m32[i] = (float)hb.minv[i];
  }
  put(o_mi, hb.minv.data(), sizeof(double) * nbl * 16);
  {
    int* rp = reinterpret_cast<int*>(host.data() + o_rp);
    for (int64_t i = 0; i <= n; ++i) rp[i] = (int)hb.row_ptr[i];
  }
  put(o_ci, hb.col_idx.data(), sizeof(int) * nnz);
  put(o_hv, hb.h_val.data(), sizeof(double) * nnz);
  put(o_sv, hb.s_val.data(), sizeof(double) * nnz);
  if (nbf) {
    put(o_bf64, hb.bf.data(), sizeof(double) * nbf);
    put(o_bfm, mt.data(), sizeof(float) * mt.size());
  }

  gb_matrix* m = new gb_matrix();
  m->device = dev;
  m->n = n;
  m->nb = hb.nb;
  m->nnz = hb.nnz;
  m->nnzb = hb.nnzb;
  m->max_row = hb.max_row;
  m->h_row_ptr = hb.row_ptr;
  cudaError_t e = cudaMalloc(&m->base, total);
  if (e != cudaSuccess) {
    delete m;
    return fail(GB_ENOMEM, "cudaMalloc(%zu bytes) for the matrix failed: %s", total, cudaGetErrorString(e));
  }
  e = cudaMemcpyAsync(m->base, host.data(), total, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaFree(m->base);
    delete m;
    return cuda_fail(e, "matrix upload");
  }
  char* b = static_cast<char*>(m->base);
  gbk::DevMat& d = m->dm;
  d.n = (int)n;
  d.nb = (int)hb.nb;
  d.blk_ptr = reinterpret_cast<const int*>(b + o_bp);
  d.blk_col = reinterpret_cast<const int*>(b + o_bc);
  d.hb = reinterpret_cast<const double*>(b + o_hb);
  d.sb = reinterpret_cast<const double*>(b + o_sb);
  d.hb_hi = reinterpret_cast<const float*>(b + o_hh);
  d.hb_lo = reinterpret_cast<const float*>(b + o_hl);
  d.sb_hi = reinterpret_cast<const float*>(b + o_sh);
  d.sb_lo = reinterpret_cast<const float*>(b + o_sl);
  d.minv = reinterpret_cast<const double*>(b + o_mi);
  d.minv32 = reinterpret_cast<const float*>(b + o_m32);
  d.row_ptr = reinterpret_cast<const int*>(b + o_rp);
  d.col_idx = reinterpret_cast<const int*>(b + o_ci);
  d.h_val = reinterpret_cast<const double*>(b + o_hv);
  d.s_val = reinterpret_cast<const double*>(b + o_sv);
  d.s_lam_min = hb.lam_min;
  d.s_lam_max = hb.lam_max;
  d.bf_bw = nbf ? hb.bf_bw : 0;
  d.bf_nblk = nbf ? (int)hb.bf_nblk : 0;
  d.bf64 = nbf ? reinterpret_cast<const double*>(b + o_bf64) : nullptr;
  d.bfm = nbf ? reinterpret_cast<const float*>(b + o_bfm) : nullptr;
  *out = m;
  return GB_OK;
}

gb_status gb_matrix_get_info(const gb_matrix* m, gb_matrix_info* info) {
  clear_error();
  if (!m || !info) return fail(GB_EINVAL, "NULL argument");
  info->n = m->n;
  info->nnz = m->nnz;
  info->nb = m->nb;
  info->nnzb = m->nnzb;
  info->max_row = m->max_row;
  info->block = 4;
  info->device = m->device;
  info->factor_bw = m->dm.bf_bw;
  info->s_lam_min = m->dm.s_lam_min;
  info->s_lam_max = m->dm.s_lam_max;
  info->factor_nblk = m->dm.bf_nblk;
  return GB_OK;
}

void gb_free(gb_matrix* m) {
  if (!m) return;
  if (m->base) {
    cudaDeviceSynchronize();
    cudaFree(m->base);
  }
  delete m;
}

gb_status gb_spmm(const gb_matrix* m, int32_t which, gb_precision prec, int32_t w, const void* x, void* y,
                  void* stream) {
  clear_error();
  if (!m || !x || !y) return fail(GB_EINVAL, "NULL argument");
  if (which != 0 && which != 1) return fail(GB_EINVAL, "which must be 0 (H) or 1 (S)");
  if (w < 1 || w > 64) return fail(GB_EINVAL, "w must be in [1, 64]");
  if (prec != GB_FP64 && prec != GB_MIXED) return fail(GB_EINVAL, "bad precision");
  if (misaligned(x, prec == GB_FP64 ? 16 : 8) || misaligned(y, prec == GB_FP64 ? 16 : 8))
    return fail(GB_EINVAL, "x and y must be aligned to their complex element (16 bytes FP64, 8 FP32)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t esz = prec == GB_FP64 ? 16 : 8;
  const int64_t n4 = 4 * m->nb;
  const void* xin = x;
  void* pad = nullptr;
  if (n4 != m->n) {  // last block column reads rows up to 4*nb - 1: pad x with zero rows
    GB_CUDA(cudaMallocAsync(&pad, esz * n4 * w, s));
    cudaError_t pe = cudaMemsetAsync(pad, 0, esz * n4 * w, s);
    if (pe == cudaSuccess) pe = cudaMemcpyAsync(pad, x, esz * m->n * w, cudaMemcpyDeviceToDevice, s);
    if (pe != cudaSuccess) {  // free the padded copy on this exit path too
      cudaFreeAsync(pad, s);
      return cuda_fail(pe, "spmm input padding");
    }
    xin = pad;
  }
  const int threads = 256;
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device);
  const long long work = w <= 8 ? (long long)m->nb * 32 : (long long)m->nb * w;  // threads of work
  const int blocks = (int)std::min<long long>((work + threads - 1) / threads, (long long)nsm * 8);
  const bool aligned = (reinterpret_cast<uintptr_t>(xin) % 16) == 0 && (reinterpret_cast<uintptr_t>(y) % 16) == 0;
  const bool pow2 = (w & (w - 1)) == 0;
  const unsigned wblocks = (unsigned)((m->nb + 7) / 8);  // 8 warps = 8 block rows per CTA
  if (aligned && prec != GB_FP64 && w <= 2) {
    const float* A = which ? m->dm.sb_hi : m->dm.hb_hi;
    const auto* xq = static_cast<const float2*>(xin);
    auto* yq = static_cast<float2*>(y);
    if (w == 1)
      spmm_quad_kernel<1><<<wblocks, threads, 0, s>>>(m->dm, A, xq, yq);
    else
      spmm_quad_kernel<2><<<wblocks, threads, 0, s>>>(m->dm, A, xq, yq);
  } else if (aligned && prec != GB_FP64 && pow2) {  // w = 4 .. 64
    const float* A = which ? m->dm.sb_hi : m->dm.hb_hi;
    const auto* xq = static_cast<const float4*>(xin);
    auto* yq = static_cast<float4*>(y);
    switch (w) {
      case 4: spmm_wide_kernel<2><<<wblocks, threads, 0, s>>>(m->dm, A, xq, yq); break;
      case 8: spmm_wide_kernel<4><<<wblocks, threads, 0, s>>>(m->dm, A, xq, yq); break;
      case 16: spmm_wide_kernel<8><<<wblocks, threads, 0, s>>>(m->dm, A, xq, yq); break;
      case 32: spmm_wide_kernel<16><<<wblocks, threads, 0, s>>>(m->dm, A, xq, yq); break;
      default: spmm_wide_kernel<32><<<wblocks, threads, 0, s>>>(m->dm, A, xq, yq); break;
    }
  } else if (aligned && prec == GB_FP64 && pow2 && w <= 32) {
    const double* A = which ? m->dm.sb : m->dm.hb;
    const auto* xq = static_cast<const double2*>(xin);
    auto* yq = static_cast<double2*>(y);
    switch (w) {
      case 1: spmm_quad_d_kernel<1><<<wblocks, threads, 0, s>>>(m->dm, A, xq, yq); break;
      case 2: spmm_quad_d_kernel<2><<<wblocks, threads, 0, s>>>(m->dm, A, xq, yq); break;
      case 4: spmm_wide_d_kernel<4><<<wblocks, threads, 0, s>>>(m->dm, A, xq, yq); break;
      case 8: spmm_wide_d_kernel<8><<<wblocks, threads, 0, s>>>(m->dm, A, xq, yq); break;
      case 16: spmm_wide_d_kernel<16><<<wblocks, threads, 0, s>>>(m->dm, A, xq, yq); break;
      default: spmm_wide_d_kernel<32><<<wblocks, threads, 0, s>>>(m->dm, A, xq, yq); break;
    }
  } else if (prec == GB_FP64) {
    spmm_kernel<true><<<blocks, threads, 0, s>>>(m->dm, which, w, xin, y);
  } else {
    spmm_kernel<false><<<blocks, threads, 0, s>>>(m->dm, which, w, xin, y);
  }
  cudaError_t e = cudaGetLastError();
  if (pad) cudaFreeAsync(pad, s);
  if (e != cudaSuccess) return cuda_fail(e, "spmm launch");
  return GB_OK;
}

}  // extern "C"

// ------------------------------------------------------------ shifted solve
namespace {

// Inner solver: the exact block-bidiagonal Cholesky solve when S's
// half-bandwidth is at most 63 (both precisions), unless flags ask for an
// iteration.  Otherwise the mixed path runs Chebyshev when the spectrum bounds
// of the preconditioned S are known and positive (CG with flags bit 2), and
// the FP64 path runs CG.  K Chebyshev steps reduce the preconditioned residual
// below itol by the bound 2 sqrt(kappa) q^K (q = (sqrt(kappa) - 1) /
// (sqrt(kappa) + 1)), with the Lanczos bounds widened by 2% on each side.
constexpr int kFlagSmem = 2, kFlagCG = 4, kFlagCheb = 16, kFlagHpF32 = 32, kFlagStall = 64;
constexpr int kStallWindow = 3000;  // iterations without halving the best residual
void set_inner_method(const gb_matrix* m, const gb_solve_params* p, double itol, gbk::Args& a) {
  std::memset(&a, 0, sizeof a);
  a.hp_fp32 = (p->prec == GB_MIXED && (p->flags & kFlagHpF32)) ? 1 : 0;
  a.stall = (p->flags & kFlagStall) ? kStallWindow : 0;
  if (!(p->flags & (kFlagCG | kFlagCheb)) && m->dm.bf_bw > 0) {
    a.inner_bchol = 1;  // exact: block-bidiagonal Cholesky factor solves
    // mixed: FP32 factor solves on TF32 tensor cores with a three-term split,
    // each accurate to ~2e-6 (measured), refined around float-float
    // residuals: two levels for tol >= 1e-6, three down to 1e-9, four below
    // (measured: at tol 1e-10 a near-threshold pair of a 114-orbital chain
    // stagnated at 7.7e-10 with three levels and converged with four); an
    // explicit inner_tol asks for (2e-6)^levels <= inner_tol, two at least
    if (p->inner_tol > 0) {
      a.bc_levels = 2;
      while (a.bc_levels < 4 && std::pow(2e-6, a.bc_levels) > p->inner_tol) ++a.bc_levels;
    } else {
      a.bc_levels = p->tol >= 1e-6 ? 2 : (p->tol >= 1e-9 ? 3 : 4);
    }
    return;
  }
  const double lmin = m->dm.s_lam_min * 0.98, lmax = m->dm.s_lam_max * 1.02;
  if (p->prec != GB_MIXED || (p->flags & kFlagCG) || !(lmin > 0.0) || !(lmax > lmin)) return;
  const double kappa = lmax / lmin, sk = std::sqrt(kappa);
  const double q = (sk - 1.0) / (sk + 1.0);
  int K = (int)std::ceil(std::log(2.0 * sk / itol) / std::log(1.0 / q));
  K = std::max(1, std::min(K, 48));
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
  double rho = 1.0 / sigma;
  for (int k = 0; k < K; ++k) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    a.cheb_A[k] = (float)(rn * rho);
    a.cheb_B[k] = (float)(2.0 * rn / delta);
    rho = rn;
  }
  a.cheb_c0 = (float)(1.0 / theta);
  a.cheb_K = K;
  a.inner_cheb = 1;
}

struct Plan {
  int W, KG, npanels, teams, teams_per_sm, Mcap, inner_maxit, cg_smem;
  size_t dyn_smem;
  double itol;
  size_t team_bytes, header_bytes, total;
  size_t o_z, o_wr, o_we, o_cols, o_off, o_status, o_counter;
  gbk::Args a;
};

gb_status make_plan(const gb_matrix* m, const gb_solve_params* p, bool want_g, Plan* pl, bool full_hist = false) {
  if (!m) return fail(GB_EINVAL, "matrix is NULL");
  if (!p) return fail(GB_EINVAL, "params is NULL");
  if (p->nshift < 1 || p->nshift > 256) return fail(GB_EINVAL, "nshift must be in [1, 256]");
  if (!p->z_re || !p->z_im) return fail(GB_EINVAL, "shift arrays are NULL");
  for (int k = 0; k < p->nshift; ++k)
    if (!std::isfinite(p->z_re[k]) || !std::isfinite(p->z_im[k]) || !(p->z_im[k] > 0.0))
      return fail(GB_EINVAL, "shift %d must be finite with Im z > 0", k);
  if (p->nrhs < 1 || !p->rhs_cols) return fail(GB_EINVAL, "need nrhs >= 1 and rhs_cols");
  for (int i = 0; i < p->nrhs; ++i)
    if (p->rhs_cols[i] < 0 || p->rhs_cols[i] >= m->n) return fail(GB_EINVAL, "rhs_cols[%d] out of range", i);
  if (!(p->tol > 0.0) || !std::isfinite(p->tol)) return fail(GB_EINVAL, "tol must be > 0");
  if (p->maxit < 1 || p->maxit > 1000000) return fail(GB_EINVAL, "maxit must be in [1, 1e6]");
  if (p->prec != GB_FP64 && p->prec != GB_MIXED) return fail(GB_EINVAL, "bad precision");
  if (p->seed_shift >= p->nshift) return fail(GB_EINVAL, "seed_shift out of range");
  const double* ws[2] = {p->w_rho, p->w_edm};
  for (int q = 0; q < 2; ++q)
    if (ws[q])
      for (int k = 0; k < 2 * p->nshift; ++k)
        if (!std::isfinite(ws[q][k])) return fail(GB_EINVAL, "non-finite quadrature weight");

  cudaDeviceProp prop;
  cudaError_t e = cudaGetDeviceProperties(&prop, m->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
  const int nsm = prop.multiProcessorCount;

  // Panel width W and inner-CG placement.  The inner-CG vectors g, d, q of a
  // panel (3 x N4 x W elements) may live in shared memory (flag bit 1) when
  // they fit; by default they stay in global memory so that several teams
  // share each SM.  Auto W: the widest panel that still gives every resident
  // team a panel.
  const size_t n4 = 4 * (size_t)m->nb;
  const size_t cg_esz = p->prec == GB_FP64 ? 16 : 8;
  const size_t smem_budget = (size_t)prop.sharedMemPerBlockOptin - 40 * 1024;
  // the exact factor solve keeps its partial sums, its current block and (FP32)
  // two staged factor tiles in dynamic shared memory instead
  const bool bchol = !(p->flags & (kFlagCG | kFlagCheb)) && m->dm.bf_bw > 0;
  const bool want_smem = (p->flags & kFlagSmem) != 0 && !bchol;
  auto fits = [&](int w) { return want_smem && 3 * n4 * (size_t)w * cg_esz + gbk::kRedBytes <= smem_budget; };
  auto dyn_bytes = [&](int w) -> size_t {
    const unsigned cg = fits(w) ? (unsigned)(3 * n4 * (size_t)w * cg_esz) : 0u;
    return gbk::dyn_layout(p->prec == GB_FP64, w, bchol, cg, m->dm.bf_bw).bytes;
  };
  auto occupancy = [&](size_t dyn) {
    int per_sm = 1;
    const void* fn = p->prec == GB_FP64 ? (const void*)gbk::team_kernel<false> : (const void*)gbk::team_kernel<true>;
    if (dyn > 0) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    const cudaError_t oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, gbk::TPB, dyn);
    return (oe != cudaSuccess || per_sm < 1) ? 1 : per_sm;
  };
  int W = p->panel;
  if (W <= 0) {
    // one wave that fills >= 3/4 of the team slots beats 1.5 waves of half-size
    // panels (measured on the 1900-orbital chain: W = 8, 238 panels on 304
    // slots, ~20% faster than W = 4)
    W = 1;
    for (int cand : {32, 16, 8, 4, 2}) {
      const size_t dyn = dyn_bytes(cand);
      if (4LL * ((p->nrhs + cand - 1) / cand) >= 3LL * nsm * occupancy(dyn)) {
        W = cand;
        break;
      }
    }
  }
  if (W != 1 && W != 2 && W != 4 && W != 8 && W != 16 && W != 32)
    return fail(GB_EINVAL, "panel must be 1, 2, 4, 8, 16 or 32");
  pl->W = W;
  pl->cg_smem = fits(W) ? 1 : 0;
  pl->dyn_smem = dyn_bytes(W);
  pl->teams_per_sm = occupancy(pl->dyn_smem);
  pl->KG = (p->nshift + 31) / 32;
  pl->npanels = (p->nrhs + W - 1) / W;
  pl->teams = std::min(pl->npanels, nsm * pl->teams_per_sm);
  pl->Mcap = full_hist ? W * 4 * (int)m->nb : W * m->max_row;
  pl->inner_maxit = 500;
  // Inner-solve accuracy: the seed recurrence treats w = S^{-1} H p as exact,
  // and each iteration's error enters the shifted residual gap, so the inner
  // solve runs close to working precision (FP64: 1e-14; mixed: 1e-7 per FP32
  // refinement level, ~1e-14 after the float-float residual step).
  if (p->prec == GB_FP64)
    pl->itol = p->inner_tol > 0 ? p->inner_tol : 1e-14;
  else
    pl->itol = p->inner_tol > 0 ? p->inner_tol : 1e-7;

  set_inner_method(m, p, pl->itol, pl->a);
  pl->a.bc_bw_alloc = m->dm.bf_bw;
  const size_t K = p->nshift, Wz = W, maxit = p->maxit, N4 = 4 * (size_t)m->nb;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  gbk::Args& a = pl->a;
  const size_t vec = N4 * Wz * 16;
  a.o_r = take(vec);
  a.o_rt = take(vec);
  a.o_p = take(vec);
  a.o_sp = take(vec);
  a.o_u = take(vec);
  a.o_w = take(vec);
  a.o_g = take(vec);
  a.o_d = take(vec);
  a.o_q = take(vec);
  a.o_x = take(vec);
  a.o_hr = take((maxit + 1) * (size_t)pl->Mcap * 16);
  a.o_ab = take(maxit * Wz * 2 * 16);
  a.o_L = take((maxit + 1) * Wz * sizeof(int));
  a.o_t = take((maxit + 1) * Wz * 16);
  a.o_ck = take((maxit / gbk::CK + 1) * Wz * K * 2 * 16);
  a.o_pi = take(Wz * K * 2 * 16);
  a.o_nk = take(Wz * K * sizeof(int));
  a.o_res = take(Wz * K * sizeof(double));
  a.o_buf = take((gbk::CK + 1) * Wz * K * 16);
  a.o_cp = take((maxit + 1) * Wz * pl->KG * 2 * 16);
  a.o_cf = take((maxit + 1) * Wz * 2 * 16);
  a.o_cg = want_g ? take((maxit + 1) * Wz * K * 16) : 0;
  pl->team_bytes = off;

  off = 0;
  pl->o_z = take(K * 16);
  pl->o_wr = take(K * 16);
  pl->o_we = take(K * 16);
  pl->o_cols = take(sizeof(int) * p->nrhs);
  pl->o_off = take(sizeof(long long) * (p->nrhs + 1));
  pl->o_status = take(sizeof(int) * p->nrhs);
  pl->o_counter = take(sizeof(int));
  pl->header_bytes = off;
  pl->total = pl->header_bytes + pl->team_bytes * pl->teams + 256;
  return GB_OK;
}

}  // namespace

extern "C" {

gb_status gb_solve_plan(const gb_matrix* m, const gb_solve_params* p, int32_t* plan) {
  clear_error();
  if (!plan) return fail(GB_EINVAL, "plan is NULL");
  Plan pl;
  gb_status st = make_plan(m, p, false, &pl);
  if (st != GB_OK) return st;
  plan[0] = pl.W;
  plan[1] = pl.teams;
  plan[2] = pl.cg_smem;
  plan[3] = (int32_t)pl.dyn_smem;
  plan[4] = pl.a.inner_bchol ? 2 : (pl.a.inner_cheb ? 1 : 0);
  plan[5] = pl.teams_per_sm;
  return GB_OK;
}

size_t gb_solve_workspace_size(const gb_matrix* m, const gb_solve_params* p) {
  clear_error();
  Plan pl;
  if (make_plan(m, p, true, &pl) != GB_OK) return 0;
  return pl.total;
}

gb_status gb_shifted_solve(const gb_matrix* m, const gb_solve_params* p, const gb_outputs* out, void* workspace,
                           size_t workspace_bytes, void* stream) {
  clear_error();
  if (!out) return fail(GB_EINVAL, "outputs is NULL");
  if (check_outputs(out) != GB_OK) return GB_EINVAL;
  Plan pl;
  const bool want_g = out->g_proj != nullptr;
  gb_status st = make_plan(m, p, want_g, &pl);
  if (st != GB_OK) return st;
  if (!workspace) return fail(GB_EINVAL, "workspace is NULL");
  if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0) return fail(GB_EINVAL, "workspace must be 256-byte aligned");
  if (workspace_bytes < pl.total)
    return fail(GB_ENOMEM, "workspace too small: %zu < %zu bytes", workspace_bytes, pl.total);
  int dev = 0;
  GB_CUDA(cudaGetDevice(&dev));
  if (dev != m->device) return fail(GB_EINVAL, "current device %d differs from the matrix's device %d", dev, m->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  const int K = p->nshift, nrhs = p->nrhs;
  // packed output offsets: prefix sums of |R_j|
  std::vector<char> hdr(pl.header_bytes, 0);
  double2* hz = reinterpret_cast<double2*>(hdr.data() + pl.o_z);
  double2* hwr = reinterpret_cast<double2*>(hdr.data() + pl.o_wr);
  double2* hwe = reinterpret_cast<double2*>(hdr.data() + pl.o_we);
  for (int k = 0; k < K; ++k) {
    hz[k] = make_double2(p->z_re[k], p->z_im[k]);
    hwr[k] = p->w_rho ? make_double2(p->w_rho[2 * k], p->w_rho[2 * k + 1]) : make_double2(0, 0);
    hwe[k] = p->w_edm ? make_double2(p->w_edm[2 * k], p->w_edm[2 * k + 1]) : make_double2(0, 0);
  }
  std::memcpy(hdr.data() + pl.o_cols, p->rhs_cols, sizeof(int) * nrhs);
  const std::vector<int64_t>& rp = m->h_row_ptr;
  long long* ho = reinterpret_cast<long long*>(hdr.data() + pl.o_off);
  ho[0] = 0;
  for (int i = 0; i < nrhs; ++i) {
    const int j = p->rhs_cols[i];
    ho[i + 1] = ho[i] + (rp[j + 1] - rp[j]);
  }
  char* wsb = static_cast<char*>(workspace);
  GB_CUDA(cudaMemcpyAsync(wsb, hdr.data(), pl.header_bytes, cudaMemcpyHostToDevice, s));

  gbk::Args& a = pl.a;
  a.m = m->dm;
  a.K = K;
  a.W = pl.W;
  a.KG = pl.KG;
  a.nrhs = nrhs;
  a.npanels = pl.npanels;
  a.maxit = p->maxit;
  a.inner_maxit = pl.inner_maxit;
  a.has_rho = p->w_rho != nullptr;
  a.has_edm = p->w_edm != nullptr;
  a.want_g = want_g;
  a.tol = p->tol;
  a.itol = pl.itol;
  const int seed = p->seed_shift >= 0 ? p->seed_shift : K / 2;
  a.sigma = make_double2(p->z_re[seed], p->z_im[seed]);
  a.z = reinterpret_cast<const double2*>(wsb + pl.o_z);
  a.w_rho = reinterpret_cast<const double2*>(wsb + pl.o_wr);
  a.w_edm = reinterpret_cast<const double2*>(wsb + pl.o_we);
  a.rhs_cols = reinterpret_cast<const int*>(wsb + pl.o_cols);
  a.out_off = reinterpret_cast<const long long*>(wsb + pl.o_off);
  a.status = reinterpret_cast<int*>(wsb + pl.o_status);
  a.panel_counter = reinterpret_cast<int*>(wsb + pl.o_counter);
  a.team_ws = wsb + align256(pl.header_bytes);
  a.team_bytes = pl.team_bytes;
  a.Mcap = pl.Mcap;
  a.ldos = out->ldos;
  a.rho = out->rho;
  a.edm = out->edm;
  a.q = out->q;
  a.e_loc = out->e_loc;
  a.iters = out->iters;
  a.inner_iters = out->inner_iters;
  a.col_status = out->col_status;
  a.conv = out->converged;
  a.resid = out->resid;
  a.g_proj = reinterpret_cast<double2*>(out->g_proj);
  a.P = ho[nrhs];

  a.cg_smem = pl.cg_smem;
  if (p->prec == GB_FP64) {
    GB_CUDA(cudaFuncSetAttribute(gbk::team_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)pl.dyn_smem));
    gbk::team_kernel<false><<<pl.teams, gbk::TPB, pl.dyn_smem, s>>>(a);
  } else {
    GB_CUDA(cudaFuncSetAttribute(gbk::team_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)pl.dyn_smem));
    gbk::team_kernel<true><<<pl.teams, gbk::TPB, pl.dyn_smem, s>>>(a);
  }
  GB_CUDA(cudaGetLastError());
  std::vector<int> hst(nrhs);
  GB_CUDA(cudaMemcpyAsync(hst.data(), a.status, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, s));
  GB_CUDA(cudaStreamSynchronize(s));
  int any = 0;
  for (int v : hst) any |= v;
  if (any & gbk::kStTimeout) return fail(GB_ETIMEOUT, "a bounded wait for a staged factor tile gave up");
  if (any & gbk::kStNotSPD) return fail(GB_ENOTSPD, "inner CG found S not positive definite");
  if (any & gbk::kStBreakdown) return fail(GB_EBREAKDOWN, "COCG breakdown in at least one column");
  if (any & (gbk::kStNoConv | gbk::kStInner))
    return fail(GB_ENOCONV, "some (shift, column) pairs did not reach tol within maxit%s",
                (any & gbk::kStInner) ? " (inner CG hit its cap)" : "");
  return GB_OK;
}

}  // extern "C"

// ------------------------------------------------------------ standalone exact S^-1
// One team applies the block-bidiagonal Cholesky solve to a panel of W
// columns (the inner solve of the shifted recurrence, on its own: for tests
// and for timing the factor solve).
namespace {

template <typename T>
__global__ void __launch_bounds__(gbk::TPB, 1)
    sinv_kernel(const __grid_constant__ gbk::Args a, const typename gbk::CplxOf<T>::type* x,
                typename gbk::CplxOf<T>::type* y, typename gbk::CplxOf<T>::type* t1,
                typename gbk::CplxOf<T>::type* t2, int* status) {
  __shared__ gbk::Smem sm;
  extern __shared__ __align__(16) char dyn_smem[];
  gbk::team_init(sm, dyn_smem);
  if (threadIdx.x < gbk::WMAX) sm.act[threadIdx.x] = threadIdx.x < a.W ? 1 : 0;
  if (threadIdx.x == 0) sm.inner_count = 0;
  __syncthreads();
  gbk::bc_solve<T>(a, sm, x, y, t1, t2, dyn_smem);
  if (threadIdx.x == 0) *status = sm.bc_fail ? gbk::kStTimeout : 0;
}

}  // namespace

extern "C" {

gb_status gb_apply_sinv(const gb_matrix* m, gb_precision prec, int32_t w, const void* x, void* y, void* stream) {
  clear_error();
  if (!m || !x || !y) return fail(GB_EINVAL, "NULL argument");
  if (w != 1 && w != 2 && w != 4 && w != 8 && w != 16 && w != 32)
    return fail(GB_EINVAL, "w must be 1, 2, 4, 8, 16 or 32");
  if (prec != GB_FP64 && prec != GB_MIXED) return fail(GB_EINVAL, "bad precision");
  if (m->dm.bf_bw <= 0) return fail(GB_EINVAL, "no factor: S's half-bandwidth exceeds 63");
  if (misaligned(x, prec == GB_FP64 ? 16 : 8) || misaligned(y, prec == GB_FP64 ? 16 : 8))
    return fail(GB_EINVAL, "x and y must be aligned to their complex element");
  int dev = 0;
  GB_CUDA(cudaGetDevice(&dev));
  if (dev != m->device) return fail(GB_EINVAL, "current device %d differs from the matrix's device %d", dev, m->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool f64 = prec == GB_FP64;
  const size_t esz = f64 ? 16 : 8, n4 = 4 * (size_t)m->nb, panel = esz * n4 * w;
  // padded input, output and two scratch panels, plus the status word
  char* buf = nullptr;
  GB_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&buf), 4 * panel + 256, s));
  char* xin = buf;
  char* yout = buf + panel;
  int* st = reinterpret_cast<int*>(buf + 4 * panel);
  cudaError_t e = cudaMemsetAsync(buf, 0, 4 * panel + 256, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(xin, x, esz * m->n * w, cudaMemcpyDeviceToDevice, s);
  gbk::Args a;
  std::memset(&a, 0, sizeof a);
  a.m = m->dm;
  a.W = w;
  a.inner_bchol = 1;
  a.bc_bw_alloc = m->dm.bf_bw;
  const size_t dyn = gbk::dyn_layout(f64, w, true, 0, m->dm.bf_bw).bytes;
  if (e == cudaSuccess) {
    if (f64) {
      e = cudaFuncSetAttribute(sinv_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
      if (e == cudaSuccess)
        sinv_kernel<double><<<1, gbk::TPB, dyn, s>>>(a, reinterpret_cast<const double2*>(xin),
                                                      reinterpret_cast<double2*>(yout),
                                                      reinterpret_cast<double2*>(buf + 2 * panel),
                                                      reinterpret_cast<double2*>(buf + 3 * panel), st);
    } else {
      e = cudaFuncSetAttribute(sinv_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
      if (e == cudaSuccess)
        sinv_kernel<float><<<1, gbk::TPB, dyn, s>>>(a, reinterpret_cast<const float2*>(xin),
                                                    reinterpret_cast<float2*>(yout),
                                                    reinterpret_cast<float2*>(buf + 2 * panel),
                                                    reinterpret_cast<float2*>(buf + 3 * panel), st);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  int hst = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(y, yout, esz * m->n * w, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hst, st, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFreeAsync(buf, s);
  if (e != cudaSuccess) return cuda_fail(e, "gb_apply_sinv");
  if (hst & gbk::kStTimeout) return fail(GB_ETIMEOUT, "a bounded wait for a staged factor tile gave up");
  return GB_OK;
}

}  // extern "C"

// ------------------------------------------------------------ true-residual check
// The recursive estimate ||rt_n|| / |pi^k_n| equals the true residual only
// while every inner solve is exact; an inexact S^-1 makes them drift apart.
// The check re-runs the listed columns in the same precision with the full
// history r_m kept on every row, forms x^k = sum_m c^k_m r_m for every shift
// (a complex GEMM of the history with the coefficients) and evaluates
// ||e_j - (z_k S - H) x^k||_2 in FP64 from the scalar CSR.
namespace {

// X[v][i][k] = sum_{m < nk[k]} c[m][k] r_m[i] for verified column v (panel
// v / W, slot v % W): 64 rows x 32 shifts per block, 16 history steps staged
// in shared memory per round, each thread 4 rows x 2 shifts.
__global__ void __launch_bounds__(256) xk_kernel(int N4, int K, int W, int Mcap, int nver, const char* team_ws,
                                                 size_t team_bytes, size_t o_hr, size_t o_cg, size_t o_nk,
                                                 const int* iters_max, double2* __restrict__ X) {
  __shared__ double2 Rs[16][64];
  __shared__ double2 Cs[16][32];
  const int v = blockIdx.z, t = v / W, cc = v % W;
  const int i0 = blockIdx.x * 64, k0 = blockIdx.y * 32;
  const char* ws = team_ws + (size_t)t * team_bytes;
  const double2* hr = reinterpret_cast<const double2*>(ws + o_hr);
  const double2* cg = reinterpret_cast<const double2*>(ws + o_cg);
  const int* nk = reinterpret_cast<const int*>(ws + o_nk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double2 acc[4][2];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 2; ++b) acc[a][b] = make_double2(0.0, 0.0);
  const int M = iters_max[v];
  for (int m0 = 0; m0 < M; m0 += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += 256) {
      const int mm = e >> 6, i = e & 63;
      const int m = m0 + mm, row = i0 + i;
      Rs[mm][i] = (m < M && row < N4) ? hr[(size_t)m * Mcap + (size_t)cc * N4 + row] : make_double2(0.0, 0.0);
    }
    for (int e = threadIdx.x; e < 16 * 32; e += 256) {
      const int mm = e >> 5, kk = e & 31;
      const int m = m0 + mm, k = k0 + kk;
      Cs[mm][kk] = (k < K && m < nk[cc * K + k]) ? cg[((size_t)m * W + cc) * K + k] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int mm = 0; mm < 16; ++mm) {
      double2 r[4], c[2];
      for (int a = 0; a < 4; ++a) r[a] = Rs[mm][ty * 4 + a];
      for (int b = 0; b < 2; ++b) c[b] = Cs[mm][tx * 2 + b];
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 2; ++b) {
          acc[a][b].x = fma(r[a].x, c[b].x, fma(-r[a].y, c[b].y, acc[a][b].x));
          acc[a][b].y = fma(r[a].x, c[b].y, fma(r[a].y, c[b].x, acc[a][b].y));
        }
    }
    __syncthreads();
  }
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 2; ++b) {
      const int row = i0 + ty * 4 + a, k = k0 + tx * 2 + b;
      if (row < N4 && k < K) X[((size_t)v * N4 + row) * K + k] = acc[a][b];
    }
}

// res[k][v] = || e_j - (z_k S - H) x^k ||_2 from the scalar CSR, FP64; one
// block per (column, 32 shifts), lane = shift, warps split the rows, fixed
// reduction order.
__global__ void __launch_bounds__(256) true_resid_kernel(const gbk::DevMat mt, int N4, int K, int nver,
                                                         const int* __restrict__ cols, const double2* __restrict__ z,
                                                         const double2* __restrict__ X, double* __restrict__ res) {
  __shared__ double part[8][32];
  const int v = blockIdx.x, k = blockIdx.y * 32 + (threadIdx.x & 31), warp = threadIdx.x >> 5;
  const int j = cols[v];
  double acc = 0.0;
  if (k < K) {
    const double2 zk = z[k];
    const double2* Xv = X + (size_t)v * N4 * K;
    for (int i = warp; i < mt.n; i += 8) {
      double2 sx = make_double2(0.0, 0.0), hx = make_double2(0.0, 0.0);
      for (int t = mt.row_ptr[i]; t < mt.row_ptr[i + 1]; ++t) {
        const double2 xv = Xv[(size_t)mt.col_idx[t] * K + k];
        const double sv = mt.s_val[t], hv = mt.h_val[t];
        sx.x = fma(sv, xv.x, sx.x);
        sx.y = fma(sv, xv.y, sx.y);
        hx.x = fma(hv, xv.x, hx.x);
        hx.y = fma(hv, xv.y, hx.y);
      }
      // r_i = delta_ij - z_k (S x)_i + (H x)_i
      double rr = (i == j ? 1.0 : 0.0) - (zk.x * sx.x - zk.y * sx.y) + hx.x;
      double ri = -(zk.x * sx.y + zk.y * sx.x) + hx.y;
      acc = fma(rr, rr, fma(ri, ri, acc));
    }
  }
  part[warp][threadIdx.x & 31] = acc;
  __syncthreads();
  if (warp == 0 && k < K) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += part[w][threadIdx.x];
    res[(size_t)k * nver + v] = sqrt(s);
  }
}

struct VerLayout {
  Plan pl;
  int W;
  size_t o_x, o_im, o_cols, total;
};

gb_status ver_layout(const gb_matrix* m, const gb_solve_params* p, int32_t nver, VerLayout* L,
                     std::vector<int32_t>* cols_out, const int32_t* ver) {
  if (nver < 1 || nver > 1024) return fail(GB_EINVAL, "nver must be in [1, 1024]");
  gb_solve_params q = *p;
  std::vector<int32_t> cols(nver, 0);
  if (ver) {
    for (int i = 0; i < nver; ++i) {
      if (ver[i] < 0 || ver[i] >= p->nrhs) return fail(GB_EINVAL, "verify index %d out of range", i);
      cols[i] = p->rhs_cols[ver[i]];
    }
  } else {
    for (int i = 0; i < nver; ++i) cols[i] = p->rhs_cols[0];
  }
  int W = 1;
  while (W < 8 && W < nver) W <<= 1;
  q.nrhs = nver;
  q.rhs_cols = cols.data();
  q.panel = W;
  gb_status st = make_plan(m, &q, true, &L->pl, true);
  if (st != GB_OK) return st;
  L->W = W;
  L->pl.teams = L->pl.npanels;  // verification: every panel at once, one team each
  size_t off = align256(L->pl.header_bytes) + L->pl.team_bytes * L->pl.teams;
  off = align256(off);
  L->o_x = off;
  off = align256(off + (size_t)nver * 4 * m->nb * p->nshift * 16);
  L->o_im = off;
  off = align256(off + sizeof(int) * nver);
  L->o_cols = off;
  off = align256(off + sizeof(int) * nver);
  L->total = off + 256;
  if (cols_out) *cols_out = cols;
  return GB_OK;
}

}  // namespace

extern "C" {

size_t gb_true_residual_workspace_size(const gb_matrix* m, const gb_solve_params* p, int32_t nver) {
  clear_error();
  if (!m || !p) {
    fail(GB_EINVAL, "NULL argument");
    return 0;
  }
  VerLayout L;
  if (ver_layout(m, p, nver, &L, nullptr, nullptr) != GB_OK) return 0;
  return L.total;
}

gb_status gb_true_residual(const gb_matrix* m, const gb_solve_params* p, int32_t nver, const int32_t* ver,
                           double* resid_true, const gb_outputs* out, void* workspace, size_t workspace_bytes,
                           void* stream, int32_t* nflagged) {
  clear_error();
  if (nflagged) *nflagged = 0;
  if (!m || !p || !ver || !resid_true) return fail(GB_EINVAL, "NULL argument");
  {
    Plan full;  // validates the parameters of the solve being checked
    const gb_status st = make_plan(m, p, false, &full);
    if (st != GB_OK) return st;
  }
  if (out && (!out->resid || !out->col_status))
    return fail(GB_EINVAL, "updating outputs needs their resid and col_status arrays");
  VerLayout L;
  std::vector<int32_t> cols;
  gb_status st = ver_layout(m, p, nver, &L, &cols, ver);
  if (st != GB_OK) return st;
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
    return fail(GB_EINVAL, "workspace must be a 256-byte aligned device pointer");
  if (workspace_bytes < L.total)
    return fail(GB_ENOMEM, "workspace too small: %zu < %zu bytes", workspace_bytes, L.total);
  int dev = 0;
  GB_CUDA(cudaGetDevice(&dev));
  if (dev != m->device) return fail(GB_EINVAL, "current device %d differs from the matrix's device %d", dev, m->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int K = p->nshift, N4 = 4 * (int)m->nb;
  const Plan& pl = L.pl;
  char* wsb = static_cast<char*>(workspace);
  // header: shifts (no weights), columns, offsets, status, counter
  std::vector<char> hdr(pl.header_bytes, 0);
  double2* hz = reinterpret_cast<double2*>(hdr.data() + pl.o_z);
  for (int k = 0; k < K; ++k) hz[k] = make_double2(p->z_re[k], p->z_im[k]);
  std::memcpy(hdr.data() + pl.o_cols, cols.data(), sizeof(int) * nver);
  long long* ho = reinterpret_cast<long long*>(hdr.data() + pl.o_off);
  ho[0] = 0;
  for (int i = 0; i < nver; ++i) ho[i + 1] = ho[i] + (m->h_row_ptr[cols[i] + 1] - m->h_row_ptr[cols[i]]);
  GB_CUDA(cudaMemcpyAsync(wsb, hdr.data(), pl.header_bytes, cudaMemcpyHostToDevice, s));
  GB_CUDA(cudaMemcpyAsync(wsb + L.o_cols, cols.data(), sizeof(int) * nver, cudaMemcpyHostToDevice, s));
  gbk::Args a = pl.a;
  a.m = m->dm;
  a.K = K;
  a.W = pl.W;
  a.KG = pl.KG;
  a.nrhs = nver;
  a.npanels = pl.npanels;
  a.maxit = p->maxit;
  a.inner_maxit = pl.inner_maxit;
  a.has_rho = 0;
  a.has_edm = 0;
  a.want_g = 1;
  a.full_hist = 1;
  a.tol = p->tol;
  a.itol = pl.itol;
  const int seed = p->seed_shift >= 0 ? p->seed_shift : K / 2;
  a.sigma = make_double2(p->z_re[seed], p->z_im[seed]);
  a.z = reinterpret_cast<const double2*>(wsb + pl.o_z);
  a.w_rho = reinterpret_cast<const double2*>(wsb + pl.o_wr);
  a.w_edm = reinterpret_cast<const double2*>(wsb + pl.o_we);
  a.rhs_cols = reinterpret_cast<const int*>(wsb + pl.o_cols);
  a.out_off = reinterpret_cast<const long long*>(wsb + pl.o_off);
  a.status = reinterpret_cast<int*>(wsb + pl.o_status);
  a.panel_counter = reinterpret_cast<int*>(wsb + pl.o_counter);
  a.team_ws = wsb + align256(pl.header_bytes);
  a.team_bytes = pl.team_bytes;
  a.Mcap = pl.Mcap;
  a.iters = reinterpret_cast<int*>(wsb + L.o_im);
  a.cg_smem = pl.cg_smem;
  if (p->prec == GB_FP64) {
    GB_CUDA(cudaFuncSetAttribute(gbk::team_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)pl.dyn_smem));
    gbk::team_kernel<false><<<pl.teams, gbk::TPB, pl.dyn_smem, s>>>(a);
  } else {
    GB_CUDA(cudaFuncSetAttribute(gbk::team_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)pl.dyn_smem));
    gbk::team_kernel<true><<<pl.teams, gbk::TPB, pl.dyn_smem, s>>>(a);
  }
  GB_CUDA(cudaGetLastError());
  double2* X = reinterpret_cast<double2*>(wsb + L.o_x);
  {
    const dim3 grid((unsigned)((N4 + 63) / 64), (unsigned)((K + 31) / 32), (unsigned)nver);
    xk_kernel<<<grid, 256, 0, s>>>(N4, K, pl.W, pl.Mcap, nver, a.team_ws, pl.team_bytes, a.o_hr, a.o_cg, a.o_nk,
                                   a.iters, X);
    GB_CUDA(cudaGetLastError());
  }
  {
    const dim3 grid((unsigned)nver, (unsigned)((K + 31) / 32));
    true_resid_kernel<<<grid, 256, 0, s>>>(m->dm, N4, K, nver, reinterpret_cast<const int*>(wsb + L.o_cols), a.z, X,
                                           resid_true);
    GB_CUDA(cudaGetLastError());
  }
  std::vector<int> vst(nver);
  GB_CUDA(cudaMemcpyAsync(vst.data(), a.status, sizeof(int) * nver, cudaMemcpyDeviceToHost, s));
  GB_CUDA(cudaStreamSynchronize(s));
  int any = 0;
  for (int v : vst) any |= v;
  if (any & gbk::kStTimeout) return fail(GB_ETIMEOUT, "a bounded wait for a staged factor tile gave up");
  if (out) {  // columns whose true residual misses tol become unconverged in `out`
    const int nrhs = p->nrhs;
    std::vector<double> rt((size_t)K * nver);
    GB_CUDA(cudaMemcpyAsync(rt.data(), resid_true, sizeof(double) * K * nver, cudaMemcpyDeviceToHost, s));
    std::vector<int32_t> cst(nrhs);
    GB_CUDA(cudaMemcpyAsync(cst.data(), out->col_status, sizeof(int32_t) * nrhs, cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    int flagged = 0;
    for (int v = 0; v < nver; ++v) {
      const int c = ver[v];
      bool miss = false;
      for (int k = 0; k < K; ++k) miss |= !(rt[(size_t)k * nver + v] <= p->tol);
      if (!miss) continue;
      ++flagged;
      cst[c] |= gbk::kStNoConv;
      for (int k = 0; k < K; ++k) {
        const double r = rt[(size_t)k * nver + v];
        GB_CUDA(cudaMemcpyAsync(out->resid + (size_t)k * nrhs + c, &rt[(size_t)k * nver + v], sizeof(double),
                                cudaMemcpyHostToDevice, s));
        if (out->converged) {
          static const uint8_t zero = 0, one = 1;
          GB_CUDA(cudaMemcpyAsync(out->converged + (size_t)k * nrhs + c, r <= p->tol ? &one : &zero, 1,
                                  cudaMemcpyHostToDevice, s));
        }
      }
      GB_CUDA(cudaMemcpyAsync(out->col_status + c, &cst[c], sizeof(int32_t), cudaMemcpyHostToDevice, s));
    }
    GB_CUDA(cudaStreamSynchronize(s));
    if (nflagged) *nflagged = flagged;
  }
  return GB_OK;
}

}  // extern "C"

// ------------------------------------------------------------ chemical potential
// mu from the electron count and the Fermi-weighted rho / P^E of a finished
// solve of every orbital (Quantum molecular dynamics simulation: the density
// matrix of each MD step).  Real-axis rule on an evenly spaced shift grid
// z_k = eps_k + i eta, spacing d: c_k = -(s / pi) f((eps_k - mu) / kT) d,
// c^E_k = eps_k c_k, and N(mu) = sum_j q_j = -pi sum_k c_k D_k with the total
// DOS D_k = sum_j ldos[k][j], increasing in mu: bisection on the host over the
// K values D_k, then the reductions of rho / P^E / q / E on the device from
// the kept G_ij(z_k).
namespace {

__global__ void __launch_bounds__(256) dos_sum_kernel(const double* __restrict__ ldos, int K, int nrhs,
                                                      double* __restrict__ dos) {
  __shared__ double part[256];
  const int k = blockIdx.x;
  double acc = 0.0;
  for (int j = threadIdx.x; j < nrhs; j += 256) acc += ldos[(size_t)k * nrhs + j];
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {  // fixed-order tree
    if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) dos[k] = part[0];
}

// rho_e = sum_k c_k Im G_e(z_k), edm_e = sum_k eps_k c_k Im G_e(z_k) for every
// kept pattern entry e (the weights are real).
__global__ void __launch_bounds__(256) fermi_density_kernel(const double2* __restrict__ g, long long P, int K,
                                                            const double* __restrict__ c,
                                                            const double* __restrict__ eps,
                                                            double* __restrict__ rho, double* __restrict__ edm) {
  const long long e = blockIdx.x * 256LL + threadIdx.x;
  if (e >= P) return;
  double r = 0.0, en = 0.0;
  for (int k = 0; k < K; ++k) {
    const double im = g[(size_t)k * P + e].y;
    r = fma(c[k], im, r);
    en = fma(eps[k] * c[k], im, en);
  }
  if (rho) rho[e] = r;
  if (edm) edm[e] = en;
}

__global__ void __launch_bounds__(256) local_sums_kernel(const gbk::DevMat m, const int* __restrict__ cols,
                                                         const long long* __restrict__ off, int nrhs,
                                                         const double* __restrict__ rho, double* __restrict__ q,
                                                         double* __restrict__ el) {
  const int c = blockIdx.x * 256 + threadIdx.x;
  if (c >= nrhs) return;
  const int j = cols[c], base = m.row_ptr[j], mc = m.row_ptr[j + 1] - base;
  double qs = 0.0, es = 0.0;
  for (int t = 0; t < mc; ++t) {
    const double r = rho[off[c] + t];
    qs = fma(r, m.s_val[base + t], qs);
    es = fma(r, m.h_val[base + t], es);
  }
  if (q) q[c] = qs;
  if (el) el[c] = es;
}

double fermi_f(double x) { return x >= 0 ? std::exp(-x) / (1.0 + std::exp(-x)) : 1.0 / (1.0 + std::exp(x)); }

}  // namespace

extern "C" {

size_t gb_fermi_workspace_size(const gb_matrix* m, const gb_solve_params* p) {
  clear_error();
  if (!m || !p || p->nshift < 1 || p->nrhs < 1) {
    fail(GB_EINVAL, "NULL argument or empty problem");
    return 0;
  }
  return align256(8 * (size_t)p->nshift) * 3 + align256(4 * (size_t)p->nrhs) + align256(8 * ((size_t)p->nrhs + 1)) +
         256;
}

gb_status gb_fermi_density(const gb_matrix* m, const gb_solve_params* p, const double* g_proj, const double* ldos,
                           double n_electrons, double kT, double spin, double* mu, const gb_outputs* out,
                           void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  if (!m || !p || !g_proj || !ldos || !mu || !out) return fail(GB_EINVAL, "NULL argument");
  if (misaligned(g_proj, 16) || misaligned(ldos, 8) || check_outputs(out) != GB_OK)
    return fail(GB_EINVAL, "g_proj must be 16-byte aligned and every other array to its element");
  const int K = p->nshift, nrhs = p->nrhs;
  if (K < 2 || !p->z_re || !p->z_im) return fail(GB_EINVAL, "need at least two shifts");
  if (nrhs != m->n || !p->rhs_cols) return fail(GB_EINVAL, "the electron count needs every orbital solved (nrhs = n)");
  {
    std::vector<char> seen(m->n, 0);
    for (int c = 0; c < nrhs; ++c) {
      const int j = p->rhs_cols[c];
      if (j < 0 || j >= m->n || seen[j]) return fail(GB_EINVAL, "rhs_cols must hold every orbital once");
      seen[j] = 1;
    }
  }
  const double d = (p->z_re[K - 1] - p->z_re[0]) / (K - 1);
  if (!(d > 0.0)) return fail(GB_EINVAL, "shift real parts must increase");
  for (int k = 0; k < K; ++k)
    if (!std::isfinite(p->z_re[k]) || std::fabs(p->z_re[k] - (p->z_re[0] + k * d)) > 1e-9 * std::fabs(d) * K ||
        !(p->z_im[k] > 0.0))
      return fail(GB_EINVAL, "the shifts must be evenly spaced in Re z with Im z > 0");
  if (!(kT > 0.0) || !(spin > 0.0) || !(n_electrons > 0.0) || !(n_electrons < spin * m->n))
    return fail(GB_EINVAL, "need kT > 0, spin > 0 and 0 < n_electrons < spin * n");
  const size_t need = gb_fermi_workspace_size(m, p);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
    return fail(GB_EINVAL, "workspace must be a 256-byte aligned device pointer");
  if (workspace_bytes < need) return fail(GB_ENOMEM, "workspace too small: %zu < %zu bytes", workspace_bytes, need);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(workspace);
  double* d_dos = reinterpret_cast<double*>(w);
  double* d_c = reinterpret_cast<double*>(w + align256(8 * (size_t)K));
  double* d_eps = reinterpret_cast<double*>(w + 2 * align256(8 * (size_t)K));
  int* d_cols = reinterpret_cast<int*>(w + 3 * align256(8 * (size_t)K));
  long long* d_off = reinterpret_cast<long long*>(w + 3 * align256(8 * (size_t)K) + align256(4 * (size_t)nrhs));
  dos_sum_kernel<<<K, 256, 0, s>>>(ldos, K, nrhs, d_dos);
  GB_CUDA(cudaGetLastError());
  std::vector<double> dos(K);
  GB_CUDA(cudaMemcpyAsync(dos.data(), d_dos, sizeof(double) * K, cudaMemcpyDeviceToHost, s));
  GB_CUDA(cudaStreamSynchronize(s));
  auto count = [&](double x) {
    double n = 0.0;
    for (int k = 0; k < K; ++k) n += spin * fermi_f((p->z_re[k] - x) / kT) * d * dos[k];  // -pi c_k D_k
    return n;
  };
  double lo = p->z_re[0] - 40.0 * kT, hi = p->z_re[K - 1] + 40.0 * kT;
  if (!(count(lo) <= n_electrons && n_electrons <= count(hi)))
    return fail(GB_EINVAL, "the electron count is outside what the shift grid can hold (%g..%g)", count(lo), count(hi));
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (count(mid) < n_electrons)
      lo = mid;
    else
      hi = mid;
  }
  *mu = 0.5 * (lo + hi);
  std::vector<double> c(K), eps(K);
  for (int k = 0; k < K; ++k) {
    eps[k] = p->z_re[k];
    c[k] = -(spin / 3.141592653589793238462643383279502884) * fermi_f((eps[k] - *mu) / kT) * d;
  }
  std::vector<long long> off(nrhs + 1, 0);
  for (int i = 0; i < nrhs; ++i) {
    const int j = p->rhs_cols[i];
    off[i + 1] = off[i] + (m->h_row_ptr[j + 1] - m->h_row_ptr[j]);
  }
  const long long P = off[nrhs];
  GB_CUDA(cudaMemcpyAsync(d_c, c.data(), sizeof(double) * K, cudaMemcpyHostToDevice, s));
  GB_CUDA(cudaMemcpyAsync(d_eps, eps.data(), sizeof(double) * K, cudaMemcpyHostToDevice, s));
  GB_CUDA(cudaMemcpyAsync(d_cols, p->rhs_cols, sizeof(int) * nrhs, cudaMemcpyHostToDevice, s));
  GB_CUDA(cudaMemcpyAsync(d_off, off.data(), sizeof(long long) * (nrhs + 1), cudaMemcpyHostToDevice, s));
  fermi_density_kernel<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(reinterpret_cast<const double2*>(g_proj), P, K,
                                                                   d_c, d_eps, out->rho, out->edm);
  GB_CUDA(cudaGetLastError());
  if (out->rho && (out->q || out->e_loc)) {
    local_sums_kernel<<<(unsigned)((nrhs + 255) / 256), 256, 0, s>>>(m->dm, d_cols, d_off, nrhs, out->rho, out->q,
                                                                     out->e_loc);
    GB_CUDA(cudaGetLastError());
  }
  GB_CUDA(cudaStreamSynchronize(s));  // the host vectors above are this call's locals
  return GB_OK;
}

}  // extern "C"

// ------------------------------------------------------------ correction solve
// Shifted COCG with one seed can stagnate for a shift whose shifted residual
// loses attainable accuracy (observed near the gap of some PPV-like chains at
// eta = 0.02).  The correction re-solves each such column alone in plain FP64
// (exact factor inner solve) with its worst unconverged shift as the seed, so
// that shift's residual is the seed's own.  If shifts still miss tol, it
// repeats with the worst remaining shift as the next seed (up to six seeds)
// and keeps, per shift, the result of the seed that served it best; the
// column's outputs are then formed from those G_ij(z_k).
namespace {

struct CorrLayout {
  size_t plan_total, o_ldos, o_rho, o_edm, o_q, o_e, o_it, o_conv, o_res, o_g, o_in, o_st, total;
};

// Workspace of one single-column FP64 correction solve (its plan depends on
// maxit, the shift count and the longest pattern row, not on the column)
// followed by that column's temporary outputs.
gb_status corr_layout(const gb_matrix* m, const gb_solve_params* p, bool want_g, CorrLayout* L) {
  if (!p->rhs_cols || p->nrhs < 1) return fail(GB_EINVAL, "rhs_cols must hold nrhs >= 1 columns");
  gb_solve_params q = *p;
  const int32_t col0 = p->rhs_cols[0];
  q.nrhs = 1;
  q.rhs_cols = &col0;
  q.prec = GB_FP64;
  q.seed_shift = -1;
  q.panel = 1;
  q.flags = 0;
  q.inner_tol = 0.0;
  Plan pl;
  (void)want_g;
  const gb_status st = make_plan(m, &q, true, &pl);
  if (st != GB_OK) return st;
  const size_t K = p->nshift, mr = (size_t)std::max(m->max_row, 1);
  size_t off = align256(pl.total);
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  L->plan_total = pl.total;
  L->o_ldos = take(K * 8);
  L->o_rho = take(mr * 8);
  L->o_edm = take(mr * 8);
  L->o_q = take(8);
  L->o_e = take(8);
  L->o_it = take(4);
  L->o_conv = take(K);
  L->o_res = take(K * 8);
  L->o_g = take(K * mr * 16);  // always: the per-shift merge over seeds needs G on the pattern row
  L->o_in = take(4);
  L->o_st = take(4);
  L->total = off + 256;
  return GB_OK;
}

}  // namespace

extern "C" {

size_t gb_correct_workspace_size(const gb_matrix* m, const gb_solve_params* p, int32_t want_g) {
  clear_error();
  if (!m || !p) {
    fail(GB_EINVAL, "NULL argument");
    return 0;
  }
  CorrLayout L;
  if (corr_layout(m, p, want_g != 0, &L) != GB_OK) return 0;
  return L.total;
}

gb_status gb_correct_unconverged(const gb_matrix* m, const gb_solve_params* p, const gb_outputs* out,
                                 void* workspace, size_t workspace_bytes, void* stream, int32_t* ncorrected) {
  clear_error();
  if (ncorrected) *ncorrected = 0;
  if (!m || !p || !out) return fail(GB_EINVAL, "NULL argument");
  if (!out->col_status || !out->resid) return fail(GB_EINVAL, "col_status and resid of the first solve are required");
  {
    Plan full;  // validates every parameter of the first solve
    const gb_status st = make_plan(m, p, out->g_proj != nullptr, &full);
    if (st != GB_OK) return st;
  }
  const bool want_g = out->g_proj != nullptr;
  CorrLayout L;
  gb_status st = corr_layout(m, p, want_g, &L);
  if (st != GB_OK) return st;
  if (!workspace) return fail(GB_EINVAL, "workspace is NULL");
  if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0) return fail(GB_EINVAL, "workspace must be 256-byte aligned");
  if (workspace_bytes < L.total)
    return fail(GB_ENOMEM, "workspace too small: %zu < %zu bytes", workspace_bytes, L.total);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int K = p->nshift, nrhs = p->nrhs;
  std::vector<int32_t> hst(nrhs);
  std::vector<double> hres((size_t)K * nrhs);
  std::vector<uint8_t> hconv(out->converged ? (size_t)K * nrhs : 0);
  GB_CUDA(cudaMemcpyAsync(hst.data(), out->col_status, sizeof(int32_t) * nrhs, cudaMemcpyDeviceToHost, s));
  GB_CUDA(cudaMemcpyAsync(hres.data(), out->resid, sizeof(double) * K * nrhs, cudaMemcpyDeviceToHost, s));
  if (out->converged)
    GB_CUDA(cudaMemcpyAsync(hconv.data(), out->converged, (size_t)K * nrhs, cudaMemcpyDeviceToHost, s));
  GB_CUDA(cudaStreamSynchronize(s));
  const std::vector<int64_t>& rp = m->h_row_ptr;
  std::vector<long long> off(nrhs + 1, 0);
  for (int c = 0; c < nrhs; ++c) {
    const int j = p->rhs_cols[c];
    off[c + 1] = off[c] + (rp[j + 1] - rp[j]);
  }
  const long long P = off[nrhs];
  char* wsb = static_cast<char*>(workspace);
  int fixed = 0, left = 0;
  constexpr int kMaxSeeds = 6;
  for (int c = 0; c < nrhs; ++c) {
    const int sc = hst[c];
    if (!(sc & gbk::kStNoConv) || (sc & (gbk::kStBreakdown | gbk::kStNotSPD))) continue;
    const int32_t col = p->rhs_cols[c];
    const long long mc = off[c + 1] - off[c];
    // per shift, the best FP64 result over the seeds tried so far
    std::vector<double> best(K, INFINITY), tres(K);
    std::vector<double2> bestg((size_t)K * mc), tg((size_t)K * mc);
    std::vector<double> cur(K);  // residuals that pick the next seed
    for (int k = 0; k < K; ++k) {
      const size_t e = (size_t)k * nrhs + c;
      const bool conv = out->converged ? hconv[e] != 0 : hres[e] <= p->tol;
      cur[k] = conv ? 0.0 : hres[e];
    }
    int it_sum = 0, in_sum = 0, rounds = 0;
    bool done = false;
    std::vector<char> tried(K, 0);
    for (int round = 0; round < kMaxSeeds && !done; ++round) {
      // First the first solve's own seed, now in FP64 with the exact inner
      // solve (this alone converges most stalled columns); then the worst
      // shift still missing tol that has not been a seed yet.  (A shift that
      // stalls as a non-seed shift can stall as the seed too, so the worst
      // shift is not the first choice.)
      int kw = -1;
      if (round == 0) {
        kw = p->seed_shift >= 0 ? p->seed_shift : K / 2;
      } else {
        double rw = -1.0;
        for (int k = 0; k < K; ++k)
          if (!tried[k] && cur[k] > p->tol && cur[k] > rw) {
            rw = cur[k];
            kw = k;
          }
        if (kw < 0) break;  // every failing shift has been a seed
      }
      tried[kw] = 1;
      gb_solve_params q = *p;
      q.nrhs = 1;
      q.rhs_cols = &col;
      q.prec = GB_FP64;
      q.seed_shift = kw;
      q.panel = 1;
      q.flags = kFlagStall;  // a stalled column stops early and tries the next seed
      q.inner_tol = 0.0;
      gb_outputs t{};
      t.ldos = out->ldos ? reinterpret_cast<double*>(wsb + L.o_ldos) : nullptr;
      t.rho = out->rho ? reinterpret_cast<double*>(wsb + L.o_rho) : nullptr;
      t.edm = out->edm ? reinterpret_cast<double*>(wsb + L.o_edm) : nullptr;
      t.q = out->q ? reinterpret_cast<double*>(wsb + L.o_q) : nullptr;
      t.e_loc = out->e_loc ? reinterpret_cast<double*>(wsb + L.o_e) : nullptr;
      t.iters = reinterpret_cast<int32_t*>(wsb + L.o_it);
      t.converged = out->converged ? reinterpret_cast<uint8_t*>(wsb + L.o_conv) : nullptr;
      t.resid = reinterpret_cast<double*>(wsb + L.o_res);
      t.g_proj = reinterpret_cast<double*>(wsb + L.o_g);
      t.inner_iters = reinterpret_cast<int32_t*>(wsb + L.o_in);
      t.col_status = reinterpret_cast<int32_t*>(wsb + L.o_st);
      const gb_status sub = gb_shifted_solve(m, &q, &t, workspace, L.plan_total, stream);
      if (sub != GB_OK && sub != GB_ENOCONV) return sub;
      int hit = 0, hin = 0;
      GB_CUDA(cudaMemcpyAsync(tres.data(), t.resid, sizeof(double) * K, cudaMemcpyDeviceToHost, s));
      GB_CUDA(cudaMemcpyAsync(tg.data(), t.g_proj, sizeof(double2) * K * mc, cudaMemcpyDeviceToHost, s));
      GB_CUDA(cudaMemcpyAsync(&hit, t.iters, sizeof(int), cudaMemcpyDeviceToHost, s));
      GB_CUDA(cudaMemcpyAsync(&hin, t.inner_iters, sizeof(int), cudaMemcpyDeviceToHost, s));
      GB_CUDA(cudaStreamSynchronize(s));
      it_sum += hit;
      in_sum += hin;
      ++rounds;
      if (round == 0 && sub == GB_OK) {
        // one seed converged every shift: the solve's own outputs are the column's
        auto column = [&](void* dst, const void* src, size_t esz) {  // [K][nrhs] column c <- [K][1]
          return cudaMemcpy2DAsync(static_cast<char*>(dst) + esz * c, esz * nrhs, src, esz, esz, K,
                                   cudaMemcpyDeviceToDevice, s);
        };
        auto one = [&](void* dst, const void* src, size_t esz) {
          return cudaMemcpyAsync(static_cast<char*>(dst) + esz * c, src, esz, cudaMemcpyDeviceToDevice, s);
        };
        if (out->ldos) GB_CUDA(column(out->ldos, t.ldos, sizeof(double)));
        if (out->converged) GB_CUDA(column(out->converged, t.converged, 1));
        GB_CUDA(column(out->resid, t.resid, sizeof(double)));
        if (out->rho) GB_CUDA(cudaMemcpyAsync(out->rho + off[c], t.rho, sizeof(double) * mc, cudaMemcpyDeviceToDevice, s));
        if (out->edm) GB_CUDA(cudaMemcpyAsync(out->edm + off[c], t.edm, sizeof(double) * mc, cudaMemcpyDeviceToDevice, s));
        if (out->q) GB_CUDA(one(out->q, t.q, sizeof(double)));
        if (out->e_loc) GB_CUDA(one(out->e_loc, t.e_loc, sizeof(double)));
        if (out->iters) GB_CUDA(one(out->iters, t.iters, sizeof(int32_t)));
        if (out->inner_iters) GB_CUDA(one(out->inner_iters, t.inner_iters, sizeof(int32_t)));
        GB_CUDA(one(out->col_status, t.col_status, sizeof(int32_t)));
        if (want_g)
          GB_CUDA(cudaMemcpy2DAsync(out->g_proj + 2 * off[c], 16 * (size_t)P, t.g_proj, 16 * (size_t)mc,
                                    16 * (size_t)mc, K, cudaMemcpyDeviceToDevice, s));
        // the next column's solve reuses the temporaries: stream-ordered after these copies
        GB_CUDA(cudaStreamSynchronize(s));
        done = true;
        break;
      }
      bool all = true;
      for (int k = 0; k < K; ++k) {
        if (tres[k] < best[k]) {
          best[k] = tres[k];
          for (long long t2 = 0; t2 < mc; ++t2) bestg[(size_t)k * mc + t2] = tg[(size_t)k * mc + t2];
        }
        cur[k] = best[k];
        all &= best[k] <= p->tol;
      }
      if (all) done = true;
    }
    if (rounds > 1 || !done) {
      // Several seeds: every shift keeps the result of the seed that served it
      // best, and the column's outputs are formed from those G_ij(z_k) on the
      // pattern row (the same reductions as the solve's final phase).
      std::vector<double> sv(mc), hv(mc);
      const int base = (int)rp[col];
      GB_CUDA(cudaMemcpyAsync(sv.data(), m->dm.s_val + base, sizeof(double) * mc, cudaMemcpyDeviceToHost, s));
      GB_CUDA(cudaMemcpyAsync(hv.data(), m->dm.h_val + base, sizeof(double) * mc, cudaMemcpyDeviceToHost, s));
      GB_CUDA(cudaStreamSynchronize(s));
      std::vector<double> ldos(K), rho(mc, 0.0), edm(mc, 0.0);
      std::vector<uint8_t> conv(K);
      for (int k = 0; k < K; ++k) {
        double im = 0.0;
        for (long long t2 = 0; t2 < mc; ++t2) im += bestg[(size_t)k * mc + t2].y * sv[t2];
        ldos[k] = -im / 3.141592653589793238462643383279502884;
        conv[k] = best[k] <= p->tol ? 1 : 0;
        const double wr_re = p->w_rho ? p->w_rho[2 * k] : 0.0, wr_im = p->w_rho ? p->w_rho[2 * k + 1] : 0.0;
        const double we_re = p->w_edm ? p->w_edm[2 * k] : 0.0, we_im = p->w_edm ? p->w_edm[2 * k + 1] : 0.0;
        for (long long t2 = 0; t2 < mc; ++t2) {
          const double2 g = bestg[(size_t)k * mc + t2];
          rho[t2] += wr_re * g.y + wr_im * g.x;  // Im(c g)
          edm[t2] += we_re * g.y + we_im * g.x;
        }
      }
      double qs = 0.0, es = 0.0;
      for (long long t2 = 0; t2 < mc; ++t2) {
        qs += rho[t2] * sv[t2];
        es += rho[t2] * hv[t2];
      }
      const bool allc = std::all_of(conv.begin(), conv.end(), [](uint8_t v) { return v != 0; });
      const int32_t cst = allc ? 0 : gbk::kStNoConv;
      done = allc;
      for (int k = 0; k < K; ++k) {
        const size_t e = (size_t)k * nrhs + c;
        if (out->ldos) GB_CUDA(cudaMemcpyAsync(out->ldos + e, &ldos[k], sizeof(double), cudaMemcpyHostToDevice, s));
        if (out->converged) GB_CUDA(cudaMemcpyAsync(out->converged + e, &conv[k], 1, cudaMemcpyHostToDevice, s));
        GB_CUDA(cudaMemcpyAsync(out->resid + e, &best[k], sizeof(double), cudaMemcpyHostToDevice, s));
        if (want_g)
          GB_CUDA(cudaMemcpyAsync(out->g_proj + 2 * ((size_t)k * P + off[c]), &bestg[(size_t)k * mc],
                                  sizeof(double2) * mc, cudaMemcpyHostToDevice, s));
      }
      if (out->rho && p->w_rho)
        GB_CUDA(cudaMemcpyAsync(out->rho + off[c], rho.data(), sizeof(double) * mc, cudaMemcpyHostToDevice, s));
      if (out->edm && p->w_edm)
        GB_CUDA(cudaMemcpyAsync(out->edm + off[c], edm.data(), sizeof(double) * mc, cudaMemcpyHostToDevice, s));
      if (out->q && p->w_rho) GB_CUDA(cudaMemcpyAsync(out->q + c, &qs, sizeof(double), cudaMemcpyHostToDevice, s));
      if (out->e_loc && p->w_rho) GB_CUDA(cudaMemcpyAsync(out->e_loc + c, &es, sizeof(double), cudaMemcpyHostToDevice, s));
      if (out->iters) GB_CUDA(cudaMemcpyAsync(out->iters + c, &it_sum, sizeof(int32_t), cudaMemcpyHostToDevice, s));
      if (out->inner_iters)
        GB_CUDA(cudaMemcpyAsync(out->inner_iters + c, &in_sum, sizeof(int32_t), cudaMemcpyHostToDevice, s));
      GB_CUDA(cudaMemcpyAsync(out->col_status + c, &cst, sizeof(int32_t), cudaMemcpyHostToDevice, s));
      GB_CUDA(cudaStreamSynchronize(s));  // the host buffers above are this iteration's locals
    }
    if (done)
      ++fixed;
    else
      ++left;
  }
  GB_CUDA(cudaStreamSynchronize(s));
  if (ncorrected) *ncorrected = fixed;
  if (left > 0)
    return fail(GB_ENOCONV, "%d column(s) still miss tol after the FP64 correction solve", left);
  return GB_OK;
}

}  // extern "C"

// ------------------------------------------------------------ allocation-free solve
// gb_shifted_solve_static: the same solve for callers that may not allocate
// memory once they are running — e.g. an application whose device memory is
// owned by another runtime's pool that claims the whole GPU, or a latency-
// critical loop in which cudaMalloc's implicit device synchronisation is not
// acceptable.  Its device scratch is one file-scope array below; its host-side
// staging uses fixed static buffers.  Nothing here calls cudaMalloc, cudaFree
// or any other allocating routine.
#include <mutex>

namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;  // 32 MiB per device
constexpr int kStaticMaxRhs = 4096;
constexpr int kMaxDevices = 64;

// Device scratch shared by every gb_shifted_solve_static call on a device.  In
// host code this name is only a stand-in for the symbol: its device address is
// obtained once per device with cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;                      // guards the table and the host staging buffers
void* g_static_addr[kMaxDevices] = {nullptr};  // device address of g_static_scratch per device
alignas(256) char g_static_hdr[256 * 1024];  // host staging of the launch header
int g_static_status[kStaticMaxRhs];          // host copy of the per-column status

}  // namespace

extern "C" {

gb_status gb_shifted_solve_static(const gb_matrix* m, const gb_solve_params* p, const gb_outputs* out,
                                  void* stream) {
  clear_error();
  if (!out) return fail(GB_EINVAL, "outputs is NULL");
  if (!p) return fail(GB_EINVAL, "params is NULL");
  if (check_outputs(out) != GB_OK) return GB_EINVAL;
  if (p->nrhs > kStaticMaxRhs) return fail(GB_EINVAL, "nrhs %d exceeds the static limit %d", p->nrhs, kStaticMaxRhs);
  Plan pl;
  const bool want_g = out->g_proj != nullptr;
  gb_status st = make_plan(m, p, want_g, &pl);
  if (st != GB_OK) return st;
  int dev = 0;
  GB_CUDA(cudaGetDevice(&dev));
  if (dev != m->device) return fail(GB_EINVAL, "current device %d differs from the matrix's device %d", dev, m->device);
  if (dev < 0 || dev >= kMaxDevices) return fail(GB_EINVAL, "device ordinal %d out of range", dev);
  if (pl.header_bytes > sizeof(g_static_hdr)) return fail(GB_EINVAL, "too many shifts/columns for the static path");
  // fewer teams than the allocating path if needed: results do not depend on it
  const size_t hdr_al = align256(pl.header_bytes);
  if (hdr_al + pl.team_bytes > kStaticScratchBytes)
    return fail(GB_ENOMEM, "problem needs %zu bytes of scratch per team; the static scratch holds %zu bytes",
                hdr_al + pl.team_bytes, kStaticScratchBytes);
  const int teams = (int)std::min<size_t>(pl.teams, (kStaticScratchBytes - hdr_al) / pl.team_bytes);

  std::lock_guard<std::mutex> lock(g_static_mu);
  if (g_static_addr[dev] == nullptr) {  // first call on this device: look up the scratch address
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess || ptr == nullptr) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
    g_static_addr[dev] = ptr;
  }
  char* wsb = static_cast<char*>(g_static_addr[dev]);
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  const int K = p->nshift, nrhs = p->nrhs;
  std::memset(g_static_hdr, 0, pl.header_bytes);  // includes the panel counter, which must start at 0
  double2* hz = reinterpret_cast<double2*>(g_static_hdr + pl.o_z);
  double2* hwr = reinterpret_cast<double2*>(g_static_hdr + pl.o_wr);
  double2* hwe = reinterpret_cast<double2*>(g_static_hdr + pl.o_we);
  for (int k = 0; k < K; ++k) {
    hz[k] = make_double2(p->z_re[k], p->z_im[k]);
    hwr[k] = p->w_rho ? make_double2(p->w_rho[2 * k], p->w_rho[2 * k + 1]) : make_double2(0, 0);
    hwe[k] = p->w_edm ? make_double2(p->w_edm[2 * k], p->w_edm[2 * k + 1]) : make_double2(0, 0);
  }
  std::memcpy(g_static_hdr + pl.o_cols, p->rhs_cols, sizeof(int) * nrhs);
  long long* ho = reinterpret_cast<long long*>(g_static_hdr + pl.o_off);
  ho[0] = 0;
  for (int i = 0; i < nrhs; ++i) {
    const int j = p->rhs_cols[i];
    ho[i + 1] = ho[i] + (m->h_row_ptr[j + 1] - m->h_row_ptr[j]);
  }
  GB_CUDA(cudaMemcpyAsync(wsb, g_static_hdr, pl.header_bytes, cudaMemcpyHostToDevice, s));

  gbk::Args& a = pl.a;
  a.m = m->dm;
  a.K = K;
  a.W = pl.W;
  a.KG = pl.KG;
  a.nrhs = nrhs;
  a.npanels = pl.npanels;
  a.maxit = p->maxit;
  a.inner_maxit = pl.inner_maxit;
  a.has_rho = p->w_rho != nullptr;
  a.has_edm = p->w_edm != nullptr;
  a.want_g = want_g;
  a.tol = p->tol;
  a.itol = pl.itol;
  const int seed = p->seed_shift >= 0 ? p->seed_shift : K / 2;
  a.sigma = make_double2(p->z_re[seed], p->z_im[seed]);
  a.z = reinterpret_cast<const double2*>(wsb + pl.o_z);
  a.w_rho = reinterpret_cast<const double2*>(wsb + pl.o_wr);
  a.w_edm = reinterpret_cast<const double2*>(wsb + pl.o_we);
  a.rhs_cols = reinterpret_cast<const int*>(wsb + pl.o_cols);
  a.out_off = reinterpret_cast<const long long*>(wsb + pl.o_off);
  a.status = reinterpret_cast<int*>(wsb + pl.o_status);
  a.panel_counter = reinterpret_cast<int*>(wsb + pl.o_counter);
  a.team_ws = wsb + hdr_al;
  a.team_bytes = pl.team_bytes;
  a.Mcap = pl.Mcap;
  a.ldos = out->ldos;
  a.rho = out->rho;
  a.edm = out->edm;
  a.q = out->q;
  a.e_loc = out->e_loc;
  a.iters = out->iters;
  a.inner_iters = out->inner_iters;
  a.col_status = out->col_status;
  a.conv = out->converged;
  a.resid = out->resid;
  a.g_proj = reinterpret_cast<double2*>(out->g_proj);
  a.P = ho[nrhs];
  a.cg_smem = pl.cg_smem;
  if (p->prec == GB_FP64) {
    GB_CUDA(cudaFuncSetAttribute(gbk::team_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)pl.dyn_smem));
    gbk::team_kernel<false><<<teams, gbk::TPB, pl.dyn_smem, s>>>(a);
  } else {
    GB_CUDA(cudaFuncSetAttribute(gbk::team_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)pl.dyn_smem));
    gbk::team_kernel<true><<<teams, gbk::TPB, pl.dyn_smem, s>>>(a);
  }
  GB_CUDA(cudaGetLastError());
  GB_CUDA(cudaMemcpyAsync(g_static_status, a.status, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, s));
  GB_CUDA(cudaStreamSynchronize(s));
  int any = 0;
  for (int i = 0; i < nrhs; ++i) any |= g_static_status[i];
  if (any & gbk::kStTimeout) return fail(GB_ETIMEOUT, "a bounded wait for a staged factor tile gave up");
  if (any & gbk::kStNotSPD) return fail(GB_ENOTSPD, "inner CG found S not positive definite");
  if (any & gbk::kStBreakdown) return fail(GB_EBREAKDOWN, "COCG breakdown in at least one column");
  if (any & (gbk::kStNoConv | gbk::kStInner))
    return fail(GB_ENOCONV, "some (shift, column) pairs did not reach tol within maxit%s",
                (any & gbk::kStInner) ? " (inner CG hit its cap)" : "");
  return GB_OK;
}

size_t gb_static_scratch_bytes(void) { return kStaticScratchBytes; }

}  // extern "C"

// ------------------------------------------------------------ batched solve
// Many independent systems in one persistent launch (team_kernel_batched).
namespace {

// Team-workspace layout for the given maxima (same regions as a single solve).
size_t layout_team(size_t N4, int W, int K, int KG, int maxit, int Mcap, bool want_g, gbk::Args& a) {
  const size_t Kz = K, Wz = W, mx = maxit;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  const size_t vec = N4 * Wz * 16;
  a.o_r = take(vec);
  a.o_rt = take(vec);
  a.o_p = take(vec);
  a.o_sp = take(vec);
  a.o_u = take(vec);
  a.o_w = take(vec);
  a.o_g = take(vec);
  a.o_d = take(vec);
  a.o_q = take(vec);
  a.o_x = take(vec);
  a.o_hr = take((mx + 1) * (size_t)Mcap * 16);
  a.o_ab = take(mx * Wz * 2 * 16);
  a.o_L = take((mx + 1) * Wz * sizeof(int));
  a.o_t = take((mx + 1) * Wz * 16);
  a.o_ck = take((mx / gbk::CK + 1) * Wz * Kz * 2 * 16);
  a.o_pi = take(Wz * Kz * 2 * 16);
  a.o_nk = take(Wz * Kz * sizeof(int));
  a.o_res = take(Wz * Kz * sizeof(double));
  a.o_buf = take((gbk::CK + 1) * Wz * Kz * 16);
  a.o_cp = take((mx + 1) * Wz * KG * 2 * 16);
  a.o_cf = take((mx + 1) * Wz * 2 * 16);
  a.o_cg = want_g ? take((mx + 1) * Wz * Kz * 16) : 0;
  return off;
}

struct BatchPlan {
  int W, teams, total_panels, maxK, maxit, Mcap, KG;
  bool mixed, want_g;
  size_t N4, team_bytes, header_bytes, total, dyn_smem;
  std::vector<int> order;  // systems, largest estimated cost first
  gbk::Args proto;
};

gb_status make_batch_plan(int32_t nsys, const gb_matrix* const* mats, const gb_solve_params* params,
                          const gb_outputs* outs, int32_t panel, BatchPlan* bp) {
  if (nsys < 1 || !mats || !params) return fail(GB_EINVAL, "need nsys >= 1, mats and params");
  const gb_precision prec = params[0].prec;
  size_t n4max = 0;
  int kmax = 0, itmax = 0, rowmax = 0, dev = -1;
  long long cols = 0;
  bool want_g = false;
  for (int s = 0; s < nsys; ++s) {
    Plan pl;
    gb_status st = make_plan(mats[s], &params[s], false, &pl);
    if (st != GB_OK) {
      char msg[sizeof(gb::g_err)];
      std::snprintf(msg, sizeof msg, "%s", gb::g_err);
      return fail(st, "system %d: %s", s, msg);
    }
    if (params[s].prec != prec) return fail(GB_EINVAL, "all systems must use the same precision");
    if (dev >= 0 && mats[s]->device != dev) return fail(GB_EINVAL, "all matrices must live on one device");
    dev = mats[s]->device;
    n4max = std::max(n4max, 4 * (size_t)mats[s]->nb);
    kmax = std::max(kmax, (int)params[s].nshift);
    itmax = std::max(itmax, (int)params[s].maxit);
    rowmax = std::max(rowmax, (int)mats[s]->max_row);
    cols += params[s].nrhs;
    if (outs && outs[s].g_proj) want_g = true;
  }
  cudaDeviceProp prop;
  cudaError_t e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
  const int nsm = prop.multiProcessorCount;
  const void* fn = prec == GB_FP64 ? (const void*)gbk::team_kernel_batched<false>
                                   : (const void*)gbk::team_kernel_batched<true>;
  // dynamic shared memory: the factor solve's buffers (systems without a
  // factor leave them unused)
  auto dyn_bytes = [&](int w) -> size_t { return gbk::dyn_layout(prec == GB_FP64, w, true, 0, 63).bytes; };
  auto occupancy = [&](size_t dyn) {
    int per_sm = 1;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, gbk::TPB, dyn) != cudaSuccess || per_sm < 1)
      per_sm = 1;
    return per_sm;
  };
  int W = panel;
  if (W <= 0) {  // widest panel that still gives every resident team a work item
    W = 1;
    for (int cand : {32, 16, 8, 4, 2}) {
      long long np = 0;
      for (int s = 0; s < nsys; ++s) np += (params[s].nrhs + cand - 1) / cand;
      if (4 * np >= 3LL * nsm * occupancy(dyn_bytes(cand))) {
        W = cand;
        break;
      }
    }
  }
  if (W != 1 && W != 2 && W != 4 && W != 8 && W != 16 && W != 32)
    return fail(GB_EINVAL, "panel must be 1, 2, 4, 8, 16 or 32");
  bp->dyn_smem = dyn_bytes(W);
  const int per_sm = occupancy(bp->dyn_smem);
  bp->W = W;
  bp->mixed = prec == GB_MIXED;
  bp->want_g = want_g;
  bp->N4 = n4max;
  bp->maxK = kmax;
  bp->KG = (kmax + 31) / 32;
  bp->maxit = itmax;
  bp->Mcap = W * rowmax;
  std::memset(&bp->proto, 0, sizeof bp->proto);
  bp->team_bytes = layout_team(n4max, W, kmax, bp->KG, itmax, bp->Mcap, want_g, bp->proto);
  bp->total_panels = 0;
  for (int s = 0; s < nsys; ++s) bp->total_panels += (params[s].nrhs + W - 1) / W;
  bp->teams = std::min(bp->total_panels, nsm * per_sm);
  // largest systems first (cost ~ basis size x shifts) for load balance
  bp->order.resize(nsys);
  for (int s = 0; s < nsys; ++s) bp->order[s] = s;
  std::stable_sort(bp->order.begin(), bp->order.end(), [&](int x, int y) {
    return (double)mats[x]->n * params[x].nshift > (double)mats[y]->n * params[y].nshift;
  });
  // header: descriptors, panel prefix, counter, then per-system arrays
  size_t hb = align256(sizeof(gbk::Args) * nsys) + align256(sizeof(int) * (nsys + 1)) + 256;
  for (int s = 0; s < nsys; ++s)
    hb += 3 * align256(16 * (size_t)params[s].nshift) + align256(sizeof(int) * params[s].nrhs) +
          align256(sizeof(long long) * (params[s].nrhs + 1)) + align256(sizeof(int) * params[s].nrhs);
  bp->header_bytes = hb;
  bp->total = hb + bp->team_bytes * bp->teams + 256;
  return GB_OK;
}

}  // namespace

extern "C" {

size_t gb_batched_workspace_size(int32_t nsys, const gb_matrix* const* mats, const gb_solve_params* params,
                                 int32_t panel, int32_t want_g) {
  clear_error();
  BatchPlan bp;
  std::vector<gb_outputs> fake;
  if (want_g && nsys > 0) {
    fake.assign(nsys, gb_outputs{});
    for (auto& f : fake) f.g_proj = reinterpret_cast<double*>(1);
  }
  if (make_batch_plan(nsys, mats, params, want_g ? fake.data() : nullptr, panel, &bp) != GB_OK) return 0;
  return bp.total;
}

gb_status gb_shifted_solve_batched(int32_t nsys, const gb_matrix* const* mats, const gb_solve_params* params,
                                   const gb_outputs* outs, int32_t panel, void* workspace, size_t workspace_bytes,
                                   void* stream) {
  clear_error();
  if (!outs) return fail(GB_EINVAL, "outputs is NULL");
  for (int i = 0; i < nsys; ++i)
    if (check_outputs(&outs[i]) != GB_OK) return GB_EINVAL;
  BatchPlan bp;
  gb_status st = make_batch_plan(nsys, mats, params, outs, panel, &bp);
  if (st != GB_OK) return st;
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
    return fail(GB_EINVAL, "workspace must be a 256-byte aligned device pointer");
  if (workspace_bytes < bp.total) return fail(GB_ENOMEM, "workspace too small: %zu < %zu bytes", workspace_bytes, bp.total);
  int dev = 0;
  GB_CUDA(cudaGetDevice(&dev));
  if (dev != mats[0]->device) return fail(GB_EINVAL, "current device differs from the matrices' device");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* wsb = static_cast<char*>(workspace);
  std::vector<char> hdr(bp.header_bytes, 0);
  gbk::Args* desc = reinterpret_cast<gbk::Args*>(hdr.data());
  size_t off = align256(sizeof(gbk::Args) * nsys);
  int* prefix = reinterpret_cast<int*>(hdr.data() + off);
  const size_t o_prefix = off;
  off += align256(sizeof(int) * (nsys + 1));
  const size_t o_counter = off;
  off += 256;
  std::vector<size_t> o_status(nsys);
  prefix[0] = 0;
  char* team_ws = wsb + align256(bp.header_bytes);
  for (int q = 0; q < nsys; ++q) {
    const int sidx = bp.order[q];
    const gb_matrix* m = mats[sidx];
    const gb_solve_params* p = &params[sidx];
    const gb_outputs* out = &outs[sidx];
    const int K = p->nshift, nrhs = p->nrhs;
    const size_t o_z = off;
    off += align256(16 * (size_t)K);
    const size_t o_wr = off;
    off += align256(16 * (size_t)K);
    const size_t o_we = off;
    off += align256(16 * (size_t)K);
    const size_t o_cols = off;
    off += align256(sizeof(int) * nrhs);
    const size_t o_off = off;
    off += align256(sizeof(long long) * (nrhs + 1));
    o_status[sidx] = off;
    off += align256(sizeof(int) * nrhs);
    double2* hz = reinterpret_cast<double2*>(hdr.data() + o_z);
    double2* hwr = reinterpret_cast<double2*>(hdr.data() + o_wr);
    double2* hwe = reinterpret_cast<double2*>(hdr.data() + o_we);
    for (int k = 0; k < K; ++k) {
      hz[k] = make_double2(p->z_re[k], p->z_im[k]);
      hwr[k] = p->w_rho ? make_double2(p->w_rho[2 * k], p->w_rho[2 * k + 1]) : make_double2(0, 0);
      hwe[k] = p->w_edm ? make_double2(p->w_edm[2 * k], p->w_edm[2 * k + 1]) : make_double2(0, 0);
    }
    std::memcpy(hdr.data() + o_cols, p->rhs_cols, sizeof(int) * nrhs);
    long long* ho = reinterpret_cast<long long*>(hdr.data() + o_off);
    ho[0] = 0;
    for (int i = 0; i < nrhs; ++i) {
      const int j = p->rhs_cols[i];
      ho[i + 1] = ho[i] + (m->h_row_ptr[j + 1] - m->h_row_ptr[j]);
    }
    gbk::Args a = bp.proto;  // workspace regions laid out for the maxima
    {
      gbk::Args im;
      set_inner_method(m, p, p->inner_tol > 0 ? p->inner_tol : (p->prec == GB_FP64 ? 1e-14 : 1e-7), im);
      a.inner_cheb = im.inner_cheb;
      a.inner_bchol = im.inner_bchol;
      a.bc_levels = im.bc_levels;
      a.hp_fp32 = im.hp_fp32;
      a.stall = im.stall;
      a.bc_bw_alloc = 63;  // the launch's shared memory is sized for any band
      a.cheb_K = im.cheb_K;
      a.cheb_c0 = im.cheb_c0;
      std::memcpy(a.cheb_A, im.cheb_A, sizeof a.cheb_A);
      std::memcpy(a.cheb_B, im.cheb_B, sizeof a.cheb_B);
    }
    a.m = m->dm;
    a.K = K;
    a.W = bp.W;
    a.KG = (K + 31) / 32;
    a.nrhs = nrhs;
    a.npanels = (nrhs + bp.W - 1) / bp.W;
    a.maxit = p->maxit;
    a.inner_maxit = 500;
    a.has_rho = p->w_rho != nullptr;
    a.has_edm = p->w_edm != nullptr;
    a.want_g = out->g_proj != nullptr;
    a.tol = p->tol;
    a.itol = p->inner_tol > 0 ? p->inner_tol : (p->prec == GB_FP64 ? 1e-14 : 1e-7);
    const int seed = p->seed_shift >= 0 ? p->seed_shift : K / 2;
    a.sigma = make_double2(p->z_re[seed], p->z_im[seed]);
    a.z = reinterpret_cast<const double2*>(wsb + o_z);
    a.w_rho = reinterpret_cast<const double2*>(wsb + o_wr);
    a.w_edm = reinterpret_cast<const double2*>(wsb + o_we);
    a.rhs_cols = reinterpret_cast<const int*>(wsb + o_cols);
    a.out_off = reinterpret_cast<const long long*>(wsb + o_off);
    a.status = reinterpret_cast<int*>(wsb + o_status[sidx]);
    a.panel_counter = reinterpret_cast<int*>(wsb + o_counter);
    a.team_ws = team_ws;
    a.team_bytes = bp.team_bytes;
    a.Mcap = bp.W * m->max_row;
    a.cg_smem = 0;
    a.ldos = out->ldos;
    a.rho = out->rho;
    a.edm = out->edm;
    a.q = out->q;
    a.e_loc = out->e_loc;
    a.iters = out->iters;
    a.inner_iters = out->inner_iters;
    a.col_status = out->col_status;
    a.conv = out->converged;
    a.resid = out->resid;
    a.g_proj = reinterpret_cast<double2*>(out->g_proj);
    a.P = ho[nrhs];
    desc[q] = a;
    prefix[q + 1] = prefix[q] + a.npanels;
  }
  GB_CUDA(cudaMemcpyAsync(wsb, hdr.data(), bp.header_bytes, cudaMemcpyHostToDevice, s));
  const gbk::Args* d_desc = reinterpret_cast<const gbk::Args*>(wsb);
  const int* d_prefix = reinterpret_cast<const int*>(wsb + o_prefix);
  int* d_counter = reinterpret_cast<int*>(wsb + o_counter);
  if (bp.mixed) {
    GB_CUDA(cudaFuncSetAttribute(gbk::team_kernel_batched<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bp.dyn_smem));
    gbk::team_kernel_batched<true><<<bp.teams, gbk::TPB, bp.dyn_smem, s>>>(d_desc, d_prefix, nsys, d_counter,
                                                                           team_ws, bp.team_bytes);
  } else {
    GB_CUDA(cudaFuncSetAttribute(gbk::team_kernel_batched<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bp.dyn_smem));
    gbk::team_kernel_batched<false><<<bp.teams, gbk::TPB, bp.dyn_smem, s>>>(d_desc, d_prefix, nsys, d_counter,
                                                                            team_ws, bp.team_bytes);
  }
  GB_CUDA(cudaGetLastError());
  GB_CUDA(cudaMemcpyAsync(hdr.data(), wsb, bp.header_bytes, cudaMemcpyDeviceToHost, s));
  GB_CUDA(cudaStreamSynchronize(s));
  int any = 0;
  for (int q = 0; q < nsys; ++q) {
    const int* hs = reinterpret_cast<const int*>(hdr.data() + o_status[q]);
    for (int i = 0; i < params[q].nrhs; ++i) any |= hs[i];
  }
  if (any & gbk::kStTimeout) return fail(GB_ETIMEOUT, "a bounded wait for a staged factor tile gave up");
  if (any & gbk::kStNotSPD) return fail(GB_ENOTSPD, "inner CG found S not positive definite");
  if (any & gbk::kStBreakdown) return fail(GB_EBREAKDOWN, "COCG breakdown in at least one column");
  if (any & (gbk::kStNoConv | gbk::kStInner))
    return fail(GB_ENOCONV, "some (shift, column) pairs did not reach tol within maxit%s",
                (any & gbk::kStInner) ? " (inner CG hit its cap)" : "");
  return GB_OK;
}

gb_status gb_tune_panel_batched(int32_t nsys, const gb_matrix* const* mats, const gb_solve_params* params,
                                const gb_outputs* outs, int32_t probe_maxit, void* workspace,
                                size_t workspace_bytes, void* stream, int32_t* best_panel, float* times_ms) {
  clear_error();
  if (!best_panel || nsys < 1 || probe_maxit < 1) return fail(GB_EINVAL, "bad tuner arguments");
  std::vector<gb_solve_params> probe(params, params + nsys);
  for (auto& p : probe) p.maxit = std::min(p.maxit, probe_maxit);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  GB_CUDA(cudaEventCreate(&e0));
  GB_CUDA(cudaEventCreate(&e1));
  // the configuration's panel widths {8, 16, 32, 64} less 64: a 64-column
  // panel's per-column shared state next to the factor solve's buffers would
  // leave one team per SM instead of two
  const int cands[3] = {8, 16, 32};
  float best = 1e30f;
  *best_panel = 0;
  for (int i = 0; i < 3; ++i) {
    if (times_ms) times_ms[i] = -1.f;
    BatchPlan bp;
    if (make_batch_plan(nsys, mats, probe.data(), outs, cands[i], &bp) != GB_OK || bp.total > workspace_bytes)
      continue;
    cudaEventRecord(e0, s);
    const gb_status st = gb_shifted_solve_batched(nsys, mats, probe.data(), outs, cands[i], workspace,
                                                  workspace_bytes, stream);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    if (st != GB_OK && st != GB_ENOCONV) continue;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (times_ms) times_ms[i] = ms;
    if (ms < best) {
      best = ms;
      *best_panel = cands[i];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  clear_error();
  if (*best_panel == 0) return fail(GB_ENOMEM, "no candidate panel width fits the workspace");
  return GB_OK;
}

}  // extern "C"

// ------------------------------------------------------------ batched correction
// The correction of a finished batched launch: every column that missed tol,
// of every system, is solved again in one batched FP64 launch (exact inner
// solve, the first solve's seed, one column per panel), and the columns that
// now meet tol are copied into the batch's outputs.  Columns that still miss
// tol then go through gb_correct_unconverged (seed switching), system by
// system.  The layout of the temporaries depends on which columns failed, so
// the plan reads every system's col_status first.
namespace {

struct CorrBatch {
  std::vector<int> sys;                      // sub-system -> system
  std::vector<std::vector<int32_t>> cols;    // failing orbital columns per sub-system
  std::vector<std::vector<int>> cidx;        // their positions in the system's column list
  std::vector<std::vector<long long>> soff;  // packed pattern offsets of the sub-system
  std::vector<gb_solve_params> q;
  std::vector<gb_outputs> t;                 // temporaries, as offsets from the workspace base
  size_t tmp_bytes = 0, batch_bytes = 0, single_bytes = 0, total = 0;
};

gb_status corr_batch_plan(int32_t nsys, const gb_matrix* const* mats, const gb_solve_params* params,
                          const gb_outputs* outs, cudaStream_t s, CorrBatch* cb) {
  if (nsys < 1 || !mats || !params || !outs) return fail(GB_EINVAL, "NULL argument or empty batch");
  for (int i = 0; i < nsys; ++i) {
    const gb_solve_params* p = &params[i];
    if (!mats[i] || !outs[i].col_status || !outs[i].resid || !p->rhs_cols || p->nrhs < 1)
      return fail(GB_EINVAL, "system %d: matrix, col_status, resid and rhs_cols are required", i);
    std::vector<int32_t> st(p->nrhs);
    GB_CUDA(cudaMemcpyAsync(st.data(), outs[i].col_status, sizeof(int32_t) * p->nrhs, cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    std::vector<int32_t> fc;
    std::vector<int> ci;
    for (int c = 0; c < p->nrhs; ++c)
      if ((st[c] & gbk::kStNoConv) && !(st[c] & (gbk::kStBreakdown | gbk::kStNotSPD))) {
        fc.push_back(p->rhs_cols[c]);
        ci.push_back(c);
      }
    if (fc.empty()) continue;
    cb->sys.push_back(i);
    cb->cols.push_back(std::move(fc));
    cb->cidx.push_back(std::move(ci));
  }
  const int nsub = (int)cb->sys.size();
  size_t off = 0;
  cb->q.resize(nsub);
  cb->t.assign(nsub, gb_outputs{});
  cb->soff.resize(nsub);
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align256(bytes);
    return reinterpret_cast<void*>(o + 256);  // +256: a null offset stays distinguishable
  };
  for (int u = 0; u < nsub; ++u) {
    const int i = cb->sys[u];
    const gb_matrix* m = mats[i];
    const gb_outputs& o = outs[i];
    gb_solve_params q = params[i];
    q.nrhs = (int32_t)cb->cols[u].size();
    q.rhs_cols = cb->cols[u].data();
    q.prec = GB_FP64;
    q.panel = 1;
    q.flags = kFlagStall;  // a stalled column stops early and tries the next seed
    q.inner_tol = 0.0;
    cb->q[u] = q;
    const size_t K = q.nshift, n = q.nrhs;
    std::vector<long long>& so = cb->soff[u];
    so.assign(n + 1, 0);
    for (size_t c = 0; c < n; ++c) {
      const int j = cb->cols[u][c];
      so[c + 1] = so[c] + (m->h_row_ptr[j + 1] - m->h_row_ptr[j]);
    }
    const size_t P = so[n];
    gb_outputs& t = cb->t[u];
    if (o.ldos) t.ldos = static_cast<double*>(take(8 * K * n));
    if (o.rho) t.rho = static_cast<double*>(take(8 * P));
    if (o.edm) t.edm = static_cast<double*>(take(8 * P));
    if (o.q) t.q = static_cast<double*>(take(8 * n));
    if (o.e_loc) t.e_loc = static_cast<double*>(take(8 * n));
    t.iters = static_cast<int32_t*>(take(4 * n));
    t.inner_iters = static_cast<int32_t*>(take(4 * n));
    t.col_status = static_cast<int32_t*>(take(4 * n));
    if (o.converged) t.converged = static_cast<uint8_t*>(take(K * n));
    t.resid = static_cast<double*>(take(8 * K * n));
    if (o.g_proj) t.g_proj = static_cast<double*>(take(16 * K * P));
  }
  cb->tmp_bytes = align256(off + 256);
  bool want_g = false;
  for (int u = 0; u < nsub; ++u) want_g |= outs[cb->sys[u]].g_proj != nullptr;
  if (nsub > 0) {
    std::vector<const gb_matrix*> sm(nsub);
    for (int u = 0; u < nsub; ++u) sm[u] = mats[cb->sys[u]];
    cb->batch_bytes = gb_batched_workspace_size(nsub, sm.data(), cb->q.data(), 1, want_g ? 1 : 0);
    if (cb->batch_bytes == 0) return GB_EINVAL;  // error text set by the size call
    for (int u = 0; u < nsub; ++u) {
      const int i = cb->sys[u];
      const size_t b = gb_correct_workspace_size(mats[i], &params[i], outs[i].g_proj != nullptr);
      if (b == 0) return GB_EINVAL;
      cb->single_bytes = std::max(cb->single_bytes, b);
    }
  }
  cb->total = std::max(cb->tmp_bytes + cb->batch_bytes, cb->single_bytes);
  return GB_OK;
}

template <typename T>
T* at(void* base, T* rel) {
  return rel ? reinterpret_cast<T*>(static_cast<char*>(base) + (reinterpret_cast<uintptr_t>(rel) - 256)) : nullptr;
}

}  // namespace

extern "C" {

size_t gb_correct_batched_workspace_size(int32_t nsys, const gb_matrix* const* mats, const gb_solve_params* params,
                                         const gb_outputs* outs, void* stream) {
  clear_error();
  CorrBatch cb;
  if (corr_batch_plan(nsys, mats, params, outs, static_cast<cudaStream_t>(stream), &cb) != GB_OK) return 0;
  return std::max<size_t>(cb.total, 256);
}

gb_status gb_correct_batched(int32_t nsys, const gb_matrix* const* mats, const gb_solve_params* params,
                             const gb_outputs* outs, void* workspace, size_t workspace_bytes, void* stream,
                             int32_t* ncorrected) {
  clear_error();
  if (ncorrected) *ncorrected = 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CorrBatch cb;
  gb_status st = corr_batch_plan(nsys, mats, params, outs, s, &cb);
  if (st != GB_OK) return st;
  const int nsub = (int)cb.sys.size();
  if (nsub == 0) return GB_OK;
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
    return fail(GB_EINVAL, "workspace must be a 256-byte aligned device pointer");
  if (workspace_bytes < cb.total) return fail(GB_ENOMEM, "workspace too small: %zu < %zu bytes", workspace_bytes, cb.total);
  char* base = static_cast<char*>(workspace);
  std::vector<gb_outputs> tv(nsub);
  std::vector<const gb_matrix*> sm(nsub);
  for (int u = 0; u < nsub; ++u) {
    const gb_outputs& r = cb.t[u];
    gb_outputs& t = tv[u];
    t.ldos = at(base, r.ldos);
    t.rho = at(base, r.rho);
    t.edm = at(base, r.edm);
    t.q = at(base, r.q);
    t.e_loc = at(base, r.e_loc);
    t.iters = at(base, r.iters);
    t.inner_iters = at(base, r.inner_iters);
    t.col_status = at(base, r.col_status);
    t.converged = at(base, r.converged);
    t.resid = at(base, r.resid);
    t.g_proj = at(base, r.g_proj);
    sm[u] = mats[cb.sys[u]];
  }
  st = gb_shifted_solve_batched(nsub, sm.data(), cb.q.data(), tv.data(), 1, base + cb.tmp_bytes, cb.batch_bytes,
                                stream);
  if (st != GB_OK && st != GB_ENOCONV) return st;
  int fixed = 0;
  std::vector<int> left;
  for (int u = 0; u < nsub; ++u) {
    const int i = cb.sys[u];
    const gb_solve_params* p = &params[i];
    const gb_outputs& o = outs[i];
    const gb_outputs& t = tv[u];
    const int n = cb.q[u].nrhs, K = p->nshift, nrhs = p->nrhs;
    std::vector<int32_t> tst(n);
    GB_CUDA(cudaMemcpyAsync(tst.data(), t.col_status, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    // packed offsets of the system's own column list
    std::vector<long long> ooff(nrhs + 1, 0);
    for (int c = 0; c < nrhs; ++c) {
      const int j = p->rhs_cols[c];
      ooff[c + 1] = ooff[c] + (mats[i]->h_row_ptr[j + 1] - mats[i]->h_row_ptr[j]);
    }
    const long long Po = ooff[nrhs], Pt = cb.soff[u][n];
    bool rest = false;
    for (int a = 0; a < n; ++a) {
      if (tst[a] & (gbk::kStNoConv | gbk::kStBreakdown | gbk::kStNotSPD)) {
        rest = true;
        continue;
      }
      const int c = cb.cidx[u][a];
      const long long mc = ooff[c + 1] - ooff[c];
      auto col2d = [&](void* dst, const void* src, size_t esz) {  // [K][nrhs] column c <- [K][n] column a
        return cudaMemcpy2DAsync(static_cast<char*>(dst) + esz * c, esz * nrhs,
                                 static_cast<const char*>(src) + esz * a, esz * n, esz, K, cudaMemcpyDeviceToDevice, s);
      };
      auto one = [&](void* dst, const void* src, size_t esz) {
        return cudaMemcpyAsync(static_cast<char*>(dst) + esz * c, static_cast<const char*>(src) + esz * a, esz,
                               cudaMemcpyDeviceToDevice, s);
      };
      if (o.ldos) GB_CUDA(col2d(o.ldos, t.ldos, 8));
      if (o.converged) GB_CUDA(col2d(o.converged, t.converged, 1));
      GB_CUDA(col2d(o.resid, t.resid, 8));
      if (o.rho)
        GB_CUDA(cudaMemcpyAsync(o.rho + ooff[c], t.rho + cb.soff[u][a], 8 * mc, cudaMemcpyDeviceToDevice, s));
      if (o.edm)
        GB_CUDA(cudaMemcpyAsync(o.edm + ooff[c], t.edm + cb.soff[u][a], 8 * mc, cudaMemcpyDeviceToDevice, s));
      if (o.q) GB_CUDA(one(o.q, t.q, 8));
      if (o.e_loc) GB_CUDA(one(o.e_loc, t.e_loc, 8));
      if (o.iters) GB_CUDA(one(o.iters, t.iters, 4));
      if (o.inner_iters) GB_CUDA(one(o.inner_iters, t.inner_iters, 4));
      GB_CUDA(one(o.col_status, t.col_status, 4));
      if (o.g_proj)
        GB_CUDA(cudaMemcpy2DAsync(o.g_proj + 2 * ooff[c], 16 * (size_t)Po, t.g_proj + 2 * cb.soff[u][a],
                                  16 * (size_t)Pt, 16 * (size_t)mc, K, cudaMemcpyDeviceToDevice, s));
      ++fixed;
    }
    if (rest) left.push_back(i);
  }
  GB_CUDA(cudaStreamSynchronize(s));  // the temporaries are reused below
  bool all = true;
  for (const int i : left) {
    int32_t f = 0;
    const gb_status r = gb_correct_unconverged(mats[i], &params[i], &outs[i], workspace, workspace_bytes, stream, &f);
    fixed += f;
    if (r == GB_ENOCONV) {
      all = false;
    } else if (r != GB_OK) {
      if (ncorrected) *ncorrected = fixed;
      return r;
    }
  }
  if (ncorrected) *ncorrected = fixed;
  if (!all) return fail(GB_ENOCONV, "some columns still miss tol after the FP64 correction solves");
  return GB_OK;
}

}  // extern "C"

// ------------------------------------------------------------ atomic forces
// F_a = -Tr[rho dH/dR_a] + Tr[P^E dS/dR_a] (Quantum molecular dynamics
// simulation: the forces of each MD step) from the rho / P^E of a solve of
// every orbital.  For two-center elements the gradient of entry (j, i) with
// respect to the atom of row j is grad[:, e] (e its CSR position) and with
// respect to the atom of i its negative; the element (i, j) is the same
// function, so the trace over both orders gives
//   F_a = -sum_{j in a} sum_{i in R_j, atom(i) != a} ((rho_ij + rho_ji) gH_e - (P^E_ij + P^E_ji) gS_e),
// rho_ij read from column j of the packed output and rho_ji from column i (the
// two differ by the solve's rounding; the sum keeps the trace exact for the
// matrix as computed).  One warp per atom; the lanes take the entries of its
// orbitals' pattern rows and reduce in a fixed order (deterministic).
namespace {

__global__ void __launch_bounds__(256) forces_kernel(const gbk::DevMat m, const int* __restrict__ atom_off,
                                                     const int* __restrict__ orb_atom, const int* __restrict__ col_of,
                                                     const long long* __restrict__ off,
                                                     const long long* __restrict__ tpos, const double* __restrict__ rho,
                                                     const double* __restrict__ edm, const double* __restrict__ gh,
                                                     const double* __restrict__ gs, long long nnz, int n_atoms,
                                                     double* __restrict__ F) {
  const int a = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  if (a >= n_atoms) return;  // uniform per warp
  const int lane = threadIdx.x & 31;
  double fx = 0.0, fy = 0.0, fz = 0.0;
  for (int j = atom_off[a]; j < atom_off[a + 1]; ++j) {
    const int c = col_of[j], e0 = m.row_ptr[j], e1 = m.row_ptr[j + 1];
    const long long base = off[c] - e0;  // packed index of entry e in column j: base + e
    for (int e = e0 + lane; e < e1; e += 32) {
      if (orb_atom[m.col_idx[e]] == a) continue;
      const long long o = tpos[e];  // the same element in column i
      const double r = rho[base + e] + rho[o], q = edm[base + e] + edm[o];
      fx = fma(q, gs[e], fma(-r, gh[e], fx));
      fy = fma(q, gs[nnz + e], fma(-r, gh[nnz + e], fy));
      fz = fma(q, gs[2 * nnz + e], fma(-r, gh[2 * nnz + e], fz));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    fx += __shfl_xor_sync(0xffffffffu, fx, o);
    fy += __shfl_xor_sync(0xffffffffu, fy, o);
    fz += __shfl_xor_sync(0xffffffffu, fz, o);
  }
  if (lane == 0) {
    F[3 * a] = fx;
    F[3 * a + 1] = fy;
    F[3 * a + 2] = fz;
  }
}

}  // namespace

extern "C" {

size_t gb_forces_workspace_size(const gb_matrix* m, const gb_solve_params* p, int32_t n_atoms) {
  clear_error();
  if (!m || !p || p->nrhs < 1 || n_atoms < 1) {
    fail(GB_EINVAL, "NULL argument, no columns or no atoms");
    return 0;
  }
  return align256(4 * ((size_t)n_atoms + 1)) + 2 * align256(4 * (size_t)m->n) +
         align256(8 * ((size_t)p->nrhs + 1)) + align256(8 * (size_t)m->nnz) + 256;
}

gb_status gb_forces(const gb_matrix* m, const gb_solve_params* p, const double* rho, const double* edm,
                    const double* grad_h, const double* grad_s, const int64_t* atom_off, int32_t n_atoms,
                    double* forces, void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  if (!m || !p || !rho || !edm || !grad_h || !grad_s || !atom_off || !forces) return fail(GB_EINVAL, "NULL argument");
  if (misaligned(rho, 8) || misaligned(edm, 8) || misaligned(grad_h, 8) || misaligned(grad_s, 8) ||
      misaligned(forces, 8))
    return fail(GB_EINVAL, "arrays must be aligned to their element");
  const int n = (int)m->n, nrhs = p->nrhs;
  if (n_atoms < 1 || atom_off[0] != 0 || atom_off[n_atoms] != n)
    return fail(GB_EINVAL, "atom_off must run from 0 to n over n_atoms atoms");
  for (int a = 0; a < n_atoms; ++a)
    if (atom_off[a + 1] <= atom_off[a]) return fail(GB_EINVAL, "atom %d has no orbitals", a);
  if (nrhs != n || !p->rhs_cols) return fail(GB_EINVAL, "forces need every orbital solved (nrhs = n)");
  std::vector<int> col_of(n, -1), orb_atom(n), aoff(n_atoms + 1);
  for (int c = 0; c < nrhs; ++c) {
    const int j = p->rhs_cols[c];
    if (j < 0 || j >= n || col_of[j] >= 0) return fail(GB_EINVAL, "rhs_cols must hold every orbital once");
    col_of[j] = c;
  }
  for (int a = 0; a < n_atoms; ++a) {
    aoff[a] = (int)atom_off[a];
    for (int64_t j = atom_off[a]; j < atom_off[a + 1]; ++j) orb_atom[j] = a;
  }
  aoff[n_atoms] = n;
  const size_t need = gb_forces_workspace_size(m, p, n_atoms);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
    return fail(GB_EINVAL, "workspace must be a 256-byte aligned device pointer");
  if (workspace_bytes < need) return fail(GB_ENOMEM, "workspace too small: %zu < %zu bytes", workspace_bytes, need);
  std::vector<long long> off(nrhs + 1, 0);
  for (int c = 0; c < nrhs; ++c) {
    const int j = p->rhs_cols[c];
    off[c + 1] = off[c] + (m->h_row_ptr[j + 1] - m->h_row_ptr[j]);
  }
  // packed index of every CSR element's transpose: entry e = (row j, column i)
  // lies in column j; the element (i, j) lies in column i at the position of j in R_i
  const std::vector<int64_t>& rp = m->h_row_ptr;
  std::vector<int32_t> ci(m->nnz);
  GB_CUDA(cudaMemcpy(ci.data(), m->dm.col_idx, 4 * (size_t)m->nnz, cudaMemcpyDeviceToHost));
  std::vector<long long> tp(m->nnz);
  for (int j = 0; j < n; ++j)
    for (int64_t e = rp[j]; e < rp[j + 1]; ++e) {
      const int i = ci[e];
      const int32_t* r0 = ci.data() + rp[i];
      const int32_t* r1 = ci.data() + rp[i + 1];
      const int32_t* hit = std::lower_bound(r0, r1, j);
      if (hit == r1 || *hit != j) return fail(GB_EINVAL, "the pattern is not symmetric");
      tp[e] = off[col_of[i]] + (hit - r0);
    }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(workspace);
  int* d_aoff = reinterpret_cast<int*>(w);
  int* d_atom = reinterpret_cast<int*>(w + align256(4 * ((size_t)n_atoms + 1)));
  int* d_col = reinterpret_cast<int*>(w + align256(4 * ((size_t)n_atoms + 1)) + align256(4 * (size_t)n));
  long long* d_off =
      reinterpret_cast<long long*>(w + align256(4 * ((size_t)n_atoms + 1)) + 2 * align256(4 * (size_t)n));
  GB_CUDA(cudaMemcpyAsync(d_aoff, aoff.data(), 4 * ((size_t)n_atoms + 1), cudaMemcpyHostToDevice, s));
  GB_CUDA(cudaMemcpyAsync(d_atom, orb_atom.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, s));
  GB_CUDA(cudaMemcpyAsync(d_col, col_of.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, s));
  GB_CUDA(cudaMemcpyAsync(d_off, off.data(), 8 * ((size_t)nrhs + 1), cudaMemcpyHostToDevice, s));
  long long* d_tp = reinterpret_cast<long long*>(reinterpret_cast<char*>(d_off) + align256(8 * ((size_t)nrhs + 1)));
  GB_CUDA(cudaMemcpyAsync(d_tp, tp.data(), 8 * (size_t)m->nnz, cudaMemcpyHostToDevice, s));
  const unsigned blocks = (unsigned)(((long long)n_atoms * 32 + 255) / 256);
  forces_kernel<<<blocks, 256, 0, s>>>(m->dm, d_aoff, d_atom, d_col, d_off, d_tp, rho, edm, grad_h, grad_s,
                                       (long long)m->nnz, n_atoms, forces);
  GB_CUDA(cudaGetLastError());
  GB_CUDA(cudaStreamSynchronize(s));  // the host staging vectors are this call's locals
  return GB_OK;
}

}  // extern "C"

// ------------------------------------------------------------ S^-1 terms
// A pole expansion of the Fermi function leaves, besides the resolvents the
// shifted solve forms, multiples of S^-1 (in rho and P^E) and of S^-1 H S^-1
// (in P^E).  gb_add_sinv_terms adds them on the pattern: one team per chunk of
// 32 columns forms X = S^-1 E (E the unit columns), Y = H X and Z = S^-1 Y with
// the FP64 factor, then rho_ij += a X_ij and P^E_ij += b X_ij + c Z_ij on the
// pattern rows of each column; q and E are then recomputed from rho.
namespace {

__global__ void __launch_bounds__(gbk::TPB, 1)
    sinv_terms_kernel(const __grid_constant__ gbk::Args a, const int* __restrict__ cols,
                      const long long* __restrict__ off, int nrhs, double a_rho, double b_edm, double c_shs,
                      double* __restrict__ rho, double* __restrict__ edm, char* __restrict__ scratch,
                      size_t panel_bytes, int* __restrict__ status) {
  __shared__ gbk::Smem sm;
  extern __shared__ __align__(16) char dyn_smem[];
  gbk::team_init(sm, dyn_smem);
  constexpr int W = 32;
  const int c0 = blockIdx.x * W, tid = threadIdx.x;
  const int N4 = 4 * a.m.nb;
  char* base = scratch + (size_t)blockIdx.x * 5 * panel_bytes;
  double2* E = reinterpret_cast<double2*>(base);
  double2* X = reinterpret_cast<double2*>(base + panel_bytes);
  double2* Z = reinterpret_cast<double2*>(base + 2 * panel_bytes);
  double2* t1 = reinterpret_cast<double2*>(base + 3 * panel_bytes);
  double2* t2 = reinterpret_cast<double2*>(base + 4 * panel_bytes);
  if (tid < gbk::WMAX) sm.act[tid] = (tid < W && c0 + tid < nrhs) ? 1 : 0;
  if (tid == 0) sm.inner_count = 0;
  for (size_t e = tid; e < (size_t)N4 * W; e += gbk::TPB) {
    const int row = (int)(e / W), l = (int)(e - (size_t)row * W);
    E[e] = make_double2((c0 + l < nrhs && cols[c0 + l] == row) ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  gbk::bc_solve<double>(a, sm, E, X, t1, t2, dyn_smem);  // X = S^-1 E (ends with a barrier)
  for (int it = tid; it < a.m.nb * W; it += gbk::TPB) {  // E <- H X
    const int I = it / W, l = it - I * W;
    double2 acc[4];
    gbk::bsr_row_d(a.m, a.m.hb, X, W, l, I, acc);
#pragma unroll
    for (int r = 0; r < 4; ++r) E[(size_t)(4 * I + r) * W + l] = acc[r];
  }
  __syncthreads();
  gbk::bc_solve<double>(a, sm, E, Z, t1, t2, dyn_smem);  // Z = S^-1 H S^-1 E
  for (int l = 0; l < W && c0 + l < nrhs; ++l) {
    const int c = c0 + l, j = cols[c], e0 = a.m.row_ptr[j], len = a.m.row_ptr[j + 1] - e0;
    for (int t = tid; t < len; t += gbk::TPB) {
      const int i = a.m.col_idx[e0 + t];
      const double x = X[(size_t)i * W + l].x, zv = Z[(size_t)i * W + l].x;
      const long long o = off[c] + t;
      if (rho) rho[o] += a_rho * x;
      if (edm) edm[o] += b_edm * x + c_shs * zv;
    }
  }
  if (tid == 0 && sm.bc_fail) atomicOr(status, gbk::kStTimeout);
}

}  // namespace

extern "C" {

size_t gb_add_sinv_terms_workspace_size(const gb_matrix* m, const gb_solve_params* p) {
  clear_error();
  if (!m || !p || p->nrhs < 1) {
    fail(GB_EINVAL, "NULL argument or no columns");
    return 0;
  }
  const size_t chunks = ((size_t)p->nrhs + 31) / 32, panel = align256(16 * 4 * (size_t)m->nb * 32);
  return align256(4 * (size_t)p->nrhs) + align256(8 * ((size_t)p->nrhs + 1)) + 256 + chunks * 5 * panel;
}

gb_status gb_add_sinv_terms(const gb_matrix* m, const gb_solve_params* p, double a_rho, double b_edm, double c_shs,
                            const gb_outputs* out, void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  if (!m || !p || !out || !p->rhs_cols || p->nrhs < 1) return fail(GB_EINVAL, "NULL argument or no columns");
  if (m->dm.bf_bw <= 0) return fail(GB_EINVAL, "no factor: S's half-bandwidth exceeds 63");
  if (check_outputs(out) != GB_OK) return GB_EINVAL;
  const int nrhs = p->nrhs;
  for (int c = 0; c < nrhs; ++c)
    if (p->rhs_cols[c] < 0 || p->rhs_cols[c] >= m->n) return fail(GB_EINVAL, "rhs_cols[%d] out of range", c);
  const size_t need = gb_add_sinv_terms_workspace_size(m, p);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
    return fail(GB_EINVAL, "workspace must be a 256-byte aligned device pointer");
  if (workspace_bytes < need) return fail(GB_ENOMEM, "workspace too small: %zu < %zu bytes", workspace_bytes, need);
  int dev = 0;
  GB_CUDA(cudaGetDevice(&dev));
  if (dev != m->device) return fail(GB_EINVAL, "current device differs from the matrix's device");
  std::vector<long long> off(nrhs + 1, 0);
  for (int c = 0; c < nrhs; ++c) {
    const int j = p->rhs_cols[c];
    off[c + 1] = off[c] + (m->h_row_ptr[j + 1] - m->h_row_ptr[j]);
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(workspace);
  int* d_cols = reinterpret_cast<int*>(w);
  long long* d_off = reinterpret_cast<long long*>(w + align256(4 * (size_t)nrhs));
  int* d_st = reinterpret_cast<int*>(w + align256(4 * (size_t)nrhs) + align256(8 * ((size_t)nrhs + 1)));
  char* scratch = w + align256(4 * (size_t)nrhs) + align256(8 * ((size_t)nrhs + 1)) + 256;
  const size_t panel = align256(16 * 4 * (size_t)m->nb * 32);
  GB_CUDA(cudaMemcpyAsync(d_cols, p->rhs_cols, 4 * (size_t)nrhs, cudaMemcpyHostToDevice, s));
  GB_CUDA(cudaMemcpyAsync(d_off, off.data(), 8 * ((size_t)nrhs + 1), cudaMemcpyHostToDevice, s));
  GB_CUDA(cudaMemsetAsync(d_st, 0, sizeof(int), s));
  GB_CUDA(cudaMemsetAsync(scratch, 0, (size_t)((nrhs + 31) / 32) * 5 * panel, s));
  gbk::Args a;
  std::memset(&a, 0, sizeof a);
  a.m = m->dm;
  a.W = 32;
  a.inner_bchol = 1;
  a.bc_bw_alloc = m->dm.bf_bw;
  const size_t dyn = gbk::dyn_layout(true, 32, true, 0, m->dm.bf_bw).bytes;
  GB_CUDA(cudaFuncSetAttribute(sinv_terms_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
  const unsigned chunks = (unsigned)((nrhs + 31) / 32);
  sinv_terms_kernel<<<chunks, gbk::TPB, dyn, s>>>(a, d_cols, d_off, nrhs, a_rho, b_edm, c_shs, out->rho, out->edm,
                                                   scratch, panel, d_st);
  GB_CUDA(cudaGetLastError());
  if (out->rho && (out->q || out->e_loc)) {
    local_sums_kernel<<<(unsigned)((nrhs + 255) / 256), 256, 0, s>>>(m->dm, d_cols, d_off, nrhs, out->rho, out->q,
                                                                     out->e_loc);
    GB_CUDA(cudaGetLastError());
  }
  int hst = 0;
  GB_CUDA(cudaMemcpyAsync(&hst, d_st, sizeof(int), cudaMemcpyDeviceToHost, s));
  GB_CUDA(cudaStreamSynchronize(s));
  if (hst & gbk::kStTimeout) return fail(GB_ETIMEOUT, "a bounded wait for a staged factor tile gave up");
  return GB_OK;
}

}  // extern "C"

// ------------------------------------------------------------ wavepacket propagation
// i S dc/dt = H c (time in hbar / eV): the transport simulations propagate a
// hole wavepacket with a Schroedinger-type equation (Quantum wavepacket
// dynamics).  One step c <- exp(-i tau S^-1 H) c is a Chebyshev series: with
// A = S^-1 H, spec(A) in [e_min, e_max], b = (e_max + e_min) / 2,
// a = (e_max - e_min) / 2 and A~ = (A - b) / a, the Jacobi-Anger expansion
//   exp(-i tau A) = e^{-i b tau} [J_0(a tau) + 2 sum_{k>=1} (-i)^k J_k(a tau) T_k(A~)]
// with T_{k+1} = 2 A~ T_k - T_{k-1}.  Each term costs one H product and one
// FP64 factor solve; the series stops where |J_k(a tau)| < 1e-17.  One team
// per chunk of W wavepackets runs every step (persistent); W is the smallest
// power of two that spreads the packets over the SMs (at most 32).
namespace {

constexpr int kWpMaxTerms = 256;

__global__ void __launch_bounds__(gbk::TPB, 1)
    wavepacket_kernel(const __grid_constant__ gbk::Args a, double2* __restrict__ psi, int nwp, int nsteps,
                      const double2* __restrict__ coef, int nterms, double ca, double cb, double2 phase,
                      char* __restrict__ scratch, size_t panel_bytes, int* __restrict__ status) {
  __shared__ gbk::Smem sm;
  extern __shared__ __align__(16) char dyn_smem[];
  gbk::team_init(sm, dyn_smem);
  const int W = a.W;  // columns per team (1 .. 32)
  const int c0 = blockIdx.x * W, tid = threadIdx.x, n = a.m.n;
  const size_t NW = (size_t)4 * a.m.nb * W;
  char* base = scratch + (size_t)blockIdx.x * 7 * panel_bytes;
  double2* P = reinterpret_cast<double2*>(base);
  double2* Tm = reinterpret_cast<double2*>(base + panel_bytes);      // T_{k-1}
  double2* Tk = reinterpret_cast<double2*>(base + 2 * panel_bytes);  // T_k
  double2* Y = reinterpret_cast<double2*>(base + 3 * panel_bytes);
  double2* HX = reinterpret_cast<double2*>(base + 4 * panel_bytes);
  double2* t1 = reinterpret_cast<double2*>(base + 5 * panel_bytes);
  double2* t2 = reinterpret_cast<double2*>(base + 6 * panel_bytes);
  if (tid < gbk::WMAX) sm.act[tid] = (tid < W && c0 + tid < nwp) ? 1 : 0;
  if (tid == 0) sm.inner_count = 0;
  for (size_t e = tid; e < NW; e += gbk::TPB) {  // panel layout: row-major, W columns
    const int row = (int)(e / W), l = (int)(e - (size_t)row * W);
    P[e] = (row < n && c0 + l < nwp) ? psi[(size_t)row * nwp + c0 + l] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  auto cm = [](double2 x, double2 y) { return make_double2(x.x * y.x - x.y * y.y, x.x * y.y + x.y * y.x); };
  // Y <- S^-1 H X (ends with a barrier)
  auto apply_a = [&](const double2* X) {
    for (int it = tid; it < a.m.nb * W; it += gbk::TPB) {
      const int I = it / W, l = it - I * W;
      double2 acc[4];
      gbk::bsr_row_d(a.m, a.m.hb, X, W, l, I, acc);
#pragma unroll
      for (int r = 0; r < 4; ++r) HX[(size_t)(4 * I + r) * W + l] = acc[r];
    }
    __syncthreads();
    gbk::bc_solve<double>(a, sm, HX, Y, t1, t2, dyn_smem);
  };
  for (int step = 0; step < nsteps; ++step) {
    double2* tm = Tm;
    double2* tk = Tk;
    // T_0 = P, accumulate c_0 T_0 into P's replacement at the end (held in Tm / Tk roles)
    for (size_t e = tid; e < NW; e += gbk::TPB) tm[e] = P[e];
    __syncthreads();
    apply_a(tm);  // Y = A T_0
    for (size_t e = tid; e < NW; e += gbk::TPB) {  // T_1 = (A T_0 - b T_0) / a ; P <- c_0 T_0 + c_1 T_1
      const double2 t0 = tm[e];
      const double2 v = make_double2((Y[e].x - cb * t0.x) * ca, (Y[e].y - cb * t0.y) * ca);
      tk[e] = v;
      const double2 s0 = cm(coef[0], t0), s1 = cm(coef[1], v);
      P[e] = make_double2(s0.x + s1.x, s0.y + s1.y);
    }
    __syncthreads();
    for (int k = 2; k < nterms; ++k) {
      apply_a(tk);  // Y = A T_{k-1}
      const double2 ck = coef[k];
      for (size_t e = tid; e < NW; e += gbk::TPB) {  // T_k = 2 (A T_{k-1} - b T_{k-1}) / a - T_{k-2}
        const double2 t1v = tk[e], t0v = tm[e];
        const double2 v = make_double2(2.0 * (Y[e].x - cb * t1v.x) * ca - t0v.x, 2.0 * (Y[e].y - cb * t1v.y) * ca - t0v.y);
        tm[e] = v;  // the slot of T_{k-2} now holds T_k
        const double2 s = cm(ck, v);
        P[e] = make_double2(P[e].x + s.x, P[e].y + s.y);
      }
      __syncthreads();
      double2* sw = tm;  // T_k becomes the current term
      tm = tk;
      tk = sw;
    }
    for (size_t e = tid; e < NW; e += gbk::TPB) P[e] = cm(phase, P[e]);  // e^{-i b tau}
    __syncthreads();
  }
  for (size_t e = tid; e < NW; e += gbk::TPB) {
    const int row = (int)(e / W), l = (int)(e - (size_t)row * W);
    if (row < n && c0 + l < nwp) psi[(size_t)row * nwp + c0 + l] = P[e];
  }
  if (tid == 0 && sm.bc_fail) atomicOr(status, gbk::kStTimeout);
}

}  // namespace

extern "C" {

static int wp_width(const gb_matrix* m, int nwp) {
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device);
  int w = 1;
  while (w < 32 && (nwp + w - 1) / w > nsm) w <<= 1;
  return w;
}

size_t gb_wavepacket_workspace_size(const gb_matrix* m, int32_t nwp) {
  clear_error();
  if (!m || nwp < 1) {
    fail(GB_EINVAL, "NULL matrix or no wavepackets");
    return 0;
  }
  const int w = wp_width(m, nwp);
  const size_t chunks = ((size_t)nwp + w - 1) / w, panel = align256(16 * 4 * (size_t)m->nb * w);
  return align256(16 * (size_t)kWpMaxTerms) + 256 + chunks * 7 * panel;
}

gb_status gb_wavepacket(const gb_matrix* m, int32_t nwp, void* psi, int32_t nsteps, double tau, double e_min,
                        double e_max, int32_t* nterms_out, void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  if (!m || !psi || nwp < 1 || nsteps < 0) return fail(GB_EINVAL, "NULL argument, no wavepackets or nsteps < 0");
  if (misaligned(psi, 16)) return fail(GB_EINVAL, "psi must be 16-byte aligned (complex double)");
  if (m->dm.bf_bw <= 0) return fail(GB_EINVAL, "no factor: S's half-bandwidth exceeds 63");
  if (!(e_max > e_min) || !std::isfinite(e_min) || !std::isfinite(e_max) || !(tau > 0.0) || !std::isfinite(tau))
    return fail(GB_EINVAL, "need e_min < e_max and tau > 0");
  const double ca = 2.0 / (e_max - e_min), cb = 0.5 * (e_max + e_min), z = 0.5 * (e_max - e_min) * tau;
  // Jacobi-Anger coefficients c_0 = J_0(z), c_k = 2 (-i)^k J_k(z) up to |J_k| < 1e-17 past k > z
  std::vector<double2> coef;
  for (int k = 0; k < kWpMaxTerms; ++k) {
    const double j = std::cyl_bessel_j((double)k, z);
    const double mag = k == 0 ? j : 2.0 * j;
    const int r = k & 3;  // (-i)^k = 1, -i, -1, i
    coef.push_back(r == 0 ? make_double2(mag, 0.0)
                   : r == 1 ? make_double2(0.0, -mag)
                   : r == 2 ? make_double2(-mag, 0.0)
                            : make_double2(0.0, mag));
    if (k >= 2 && k > z && std::fabs(j) < 1e-17) break;
  }
  if ((int)coef.size() >= kWpMaxTerms)
    return fail(GB_EINVAL, "(e_max - e_min) tau / 2 = %g needs more than %d terms: take shorter steps", z, kWpMaxTerms);
  const int nterms = (int)coef.size();
  if (nterms_out) *nterms_out = nterms;
  const size_t need = gb_wavepacket_workspace_size(m, nwp);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
    return fail(GB_EINVAL, "workspace must be a 256-byte aligned device pointer");
  if (workspace_bytes < need) return fail(GB_ENOMEM, "workspace too small: %zu < %zu bytes", workspace_bytes, need);
  int dev = 0;
  GB_CUDA(cudaGetDevice(&dev));
  if (dev != m->device) return fail(GB_EINVAL, "current device differs from the matrix's device");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(workspace);
  double2* d_coef = reinterpret_cast<double2*>(w);
  int* d_st = reinterpret_cast<int*>(w + align256(16 * (size_t)kWpMaxTerms));
  char* scratch = w + align256(16 * (size_t)kWpMaxTerms) + 256;
  const int wc = wp_width(m, nwp);
  const size_t panel = align256(16 * 4 * (size_t)m->nb * wc);
  const unsigned chunks = (unsigned)((nwp + wc - 1) / wc);
  GB_CUDA(cudaMemcpyAsync(d_coef, coef.data(), 16 * (size_t)nterms, cudaMemcpyHostToDevice, s));
  GB_CUDA(cudaMemsetAsync(d_st, 0, sizeof(int), s));
  GB_CUDA(cudaMemsetAsync(scratch, 0, (size_t)chunks * 7 * panel, s));
  gbk::Args a;
  std::memset(&a, 0, sizeof a);
  a.m = m->dm;
  a.W = wc;
  a.inner_bchol = 1;
  a.bc_bw_alloc = m->dm.bf_bw;
  const size_t dyn = gbk::dyn_layout(true, wc, true, 0, m->dm.bf_bw).bytes;
  GB_CUDA(cudaFuncSetAttribute(wavepacket_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
  const double2 phase = make_double2(std::cos(cb * tau), -std::sin(cb * tau));
  wavepacket_kernel<<<chunks, gbk::TPB, dyn, s>>>(a, static_cast<double2*>(psi), nwp, nsteps, d_coef, nterms, ca, cb,
                                                   phase, scratch, panel, d_st);
  GB_CUDA(cudaGetLastError());
  int hst = 0;
  GB_CUDA(cudaMemcpyAsync(&hst, d_st, sizeof(int), cudaMemcpyDeviceToHost, s));
  GB_CUDA(cudaStreamSynchronize(s));
  if (hst & gbk::kStTimeout) return fail(GB_ETIMEOUT, "a bounded wait for a staged factor tile gave up");
  return GB_OK;
}

}  // extern "C"
