// Device building blocks of the shifted-COCG team solver.
//
// Layout used by every kernel: a panel of W right-hand sides is stored as an
// N4 x W array (N4 = 4 * block rows, row-major, complex interleaved), element
// (i, c) at index i * W + c.  A CTA ("team") owns a whole panel; thread t
// always works on column c = t % W (W divides 32 and the block size), so
// per-column partial sums stay in one lane position and reduce without
// atomics, in a fixed order (deterministic results).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "ffmath.cuh"

namespace gbk {

// Threads per team (CTA).  Several teams share an SM, so that one team's
// barrier and memory stalls are covered by another team's work.
#ifndef GB_TPB
#define GB_TPB 512
#endif
#ifndef GB_UNROLL
#define GB_UNROLL 2
#endif
constexpr int TPB = GB_TPB;
constexpr int kUnroll = GB_UNROLL;  // blocks of a block row in flight per thread
constexpr int NWARP = TPB / 32;
// Two 512-thread teams per SM (64 registers per thread): measured ~20% faster
// than one team with 128 registers on the 1900-orbital chain, despite a few
// spilled registers, because one team's barriers overlap the other's work.
#ifndef GB_MIN_TEAMS
#define GB_MIN_TEAMS ((1024 / GB_TPB) > 0 ? (1024 / GB_TPB) : 1)
#endif
#ifndef GB_WARP_SPMM
#define GB_WARP_SPMM 0
#endif
constexpr int MIN_TEAMS_PER_SM = GB_MIN_TEAMS;
constexpr int WMAX = 32;
constexpr int NVMAX = 4;

struct DevMat {
  int n, nb;
  const int* blk_ptr;
  const int* blk_col;
  const double* hb;  // FP64 4x4 blocks, row-major inside a block
  const double* sb;
  const float* hb_hi;  // float-float split of the same blocks: v = hi + lo
  const float* hb_lo;
  const float* sb_hi;
  const float* sb_lo;
  const double* minv;  // inverses of S's diagonal blocks (block Jacobi)
  const float* minv32;
  const int* row_ptr;  // scalar CSR pattern (for R_j and the reductions)
  const int* col_idx;
  const double* h_val;
  const double* s_val;
  double s_lam_min, s_lam_max;  // spectrum bounds of the block-Jacobi-preconditioned S
  // Block-bidiagonal Cholesky factor of S on 64-row blocks (bf_bw = 0: none).
  // FP64: four [bf_nblk][64][64] arrays, k-major (entry (r, k) at k * 64 + r):
  // D_i^-1, D_i^-T, E_i = D_i^-1 C_i, F_i = D_i^-T C_{i+1}^T.  FP32: per block
  // a FWD and a BWD tile of kMmaTileFloatsDev floats in tensor-core fragment
  // order (block_chol.cuh).
  int bf_bw, bf_nblk;
  const float* bfm;
  const double* bf64;
};
constexpr int kMmaTileFloatsDev = 52 * 128;

// ------------------------------------------------------------ complex FP64
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cinv(double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2(b.x / d, -b.y / d);
}
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) { return cmul(a, cinv(b)); }
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ bool cfinite(double2 a) { return isfinite(a.x) && isfinite(a.y); }

// ------------------------------------------------------------ block reduce
struct RedSmem {
  double scal[NVMAX * WMAX];
};

// Sum NV per-thread partials over all threads sharing column c = tid % W.
// Result for (value i, column c) lands in rs.scal[i * WMAX + c].  Fixed order.
// The per-warp partials (NWARP * NVMAX * 32 doubles) live at the start of the
// kernel's dynamic shared memory, which every team kernel sizes for them.
template <int NV>
__device__ __forceinline__ void block_reduce(double (&v)[NV], int W, RedSmem& rs) {
  extern __shared__ __align__(16) double br_dyn[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int off = W; off < 32; off <<= 1) {
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], off);
  }
  if (lane < W) {
#pragma unroll
    for (int i = 0; i < NV; ++i) br_dyn[(warp * NV + i) * 32 + lane] = v[i];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < NV * W; t += TPB) {
    const int i = t / W, c = t - i * W;
    double s = 0.0;
    for (int w = 0; w < NWARP; ++w) s += br_dyn[(w * NV + i) * 32 + c];
    rs.scal[i * WMAX + c] = s;
  }
  __syncthreads();
}

// ------------------------------------------------------------ BSR block-row products
// acc[r] = sum over stored blocks (I, J) of A_IJ[r][t] * x[4J + t][c]; FP64.
__device__ __forceinline__ void bsr_row_d(const DevMat& m, const double* __restrict__ A,
                                          const double2* __restrict__ x, int W, int c, int I,
                                          double2 (&acc)[4]) {
#pragma unroll
  for (int r = 0; r < 4; ++r) acc[r] = make_double2(0.0, 0.0);
  const int b1 = m.blk_ptr[I + 1];
#pragma unroll kUnroll
  for (int b = m.blk_ptr[I]; b < b1; ++b) {
    const int J = m.blk_col[b];
    const double2* xr = x + (size_t)(4 * J) * W + c;
    double2 xv[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) xv[t] = xr[(size_t)t * W];
    const double2* ab = reinterpret_cast<const double2*>(A + (size_t)b * 16);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const double2 a01 = __ldg(ab + 2 * r), a23 = __ldg(ab + 2 * r + 1);
      acc[r].x = fma(a01.x, xv[0].x, acc[r].x);
      acc[r].y = fma(a01.x, xv[0].y, acc[r].y);
      acc[r].x = fma(a01.y, xv[1].x, acc[r].x);
      acc[r].y = fma(a01.y, xv[1].y, acc[r].y);
      acc[r].x = fma(a23.x, xv[2].x, acc[r].x);
      acc[r].y = fma(a23.x, xv[2].y, acc[r].y);
      acc[r].x = fma(a23.y, xv[3].x, acc[r].x);
      acc[r].y = fma(a23.y, xv[3].y, acc[r].y);
    }
  }
}

// FP32 matrix (hi part) times FP32 complex vector, FP32 accumulation.
__device__ __forceinline__ void bsr_row_f(const DevMat& m, const float* __restrict__ A,
                                          const float2* __restrict__ x, int W, int c, int I,
                                          float2 (&acc)[4]) {
#pragma unroll
  for (int r = 0; r < 4; ++r) acc[r] = make_float2(0.f, 0.f);
  const int b1 = m.blk_ptr[I + 1];
#pragma unroll kUnroll
  for (int b = m.blk_ptr[I]; b < b1; ++b) {
    const int J = m.blk_col[b];
    const float2* xr = x + (size_t)(4 * J) * W + c;
    float2 xv[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) xv[t] = xr[(size_t)t * W];
    const float4* ab = reinterpret_cast<const float4*>(A + (size_t)b * 16);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const float4 a = __ldg(ab + r);
      acc[r].x = fmaf(a.x, xv[0].x, acc[r].x);
      acc[r].y = fmaf(a.x, xv[0].y, acc[r].y);
      acc[r].x = fmaf(a.y, xv[1].x, acc[r].x);
      acc[r].y = fmaf(a.y, xv[1].y, acc[r].y);
      acc[r].x = fmaf(a.z, xv[2].x, acc[r].x);
      acc[r].y = fmaf(a.z, xv[2].y, acc[r].y);
      acc[r].x = fmaf(a.w, xv[3].x, acc[r].x);
      acc[r].y = fmaf(a.w, xv[3].y, acc[r].y);
    }
  }
}

// FP32 matrix (hi part) times the hi parts of a float-float complex vector
// (float4 {re.hi, re.lo, im.hi, im.lo}), FP32 accumulation: the unrefined
// FP32 product (flags bit 5 of the mixed path).
__device__ __forceinline__ void bsr_row_fhi(const DevMat& m, const float* __restrict__ A,
                                            const float4* __restrict__ x, int W, int c, int I, float2 (&acc)[4]) {
#pragma unroll
  for (int r = 0; r < 4; ++r) acc[r] = make_float2(0.f, 0.f);
  const int b1 = m.blk_ptr[I + 1];
#pragma unroll kUnroll
  for (int b = m.blk_ptr[I]; b < b1; ++b) {
    const int J = m.blk_col[b];
    const float4* xr = x + (size_t)(4 * J) * W + c;
    float2 xv[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const float4 v = xr[(size_t)t * W];
      xv[t] = make_float2(v.x, v.z);
    }
    const float4* ab = reinterpret_cast<const float4*>(A + (size_t)b * 16);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const float4 a = __ldg(ab + r);
      acc[r].x = fmaf(a.x, xv[0].x, fmaf(a.y, xv[1].x, fmaf(a.z, xv[2].x, fmaf(a.w, xv[3].x, acc[r].x))));
      acc[r].y = fmaf(a.x, xv[0].y, fmaf(a.y, xv[1].y, fmaf(a.z, xv[2].y, fmaf(a.w, xv[3].y, acc[r].y))));
    }
  }
}

// float-float matrix (hi + lo) times float-float complex vector, compensated
// accumulation: acc_re[r] / acc_im[r] hold the row sums as hi + err.
__device__ __forceinline__ void bsr_row_ff(const DevMat& m, const float* __restrict__ Ahi,
                                           const float* __restrict__ Alo, const float4* __restrict__ x,
                                           int W, int c, int I, gbff::acc (&are)[4], gbff::acc (&aim)[4]) {
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    gbff::acc_init(are[r]);
    gbff::acc_init(aim[r]);
  }
  const int b1 = m.blk_ptr[I + 1];
#pragma unroll kUnroll
  for (int b = m.blk_ptr[I]; b < b1; ++b) {
    const int J = m.blk_col[b];
    const float4* xr = x + (size_t)(4 * J) * W + c;
    float4 xv[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) xv[t] = xr[(size_t)t * W];
    const float4* ah = reinterpret_cast<const float4*>(Ahi + (size_t)b * 16);
    const float4* al = reinterpret_cast<const float4*>(Alo + (size_t)b * 16);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const float4 h = __ldg(ah + r), l = __ldg(al + r);
      const float hv[4] = {h.x, h.y, h.z, h.w};
      const float lv[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const gbff::ff a = {hv[t], lv[t]};
        gbff::acc_mul_add(are[r], a, gbff::ff{xv[t].x, xv[t].y});
        gbff::acc_mul_add(aim[r], a, gbff::ff{xv[t].z, xv[t].w});
      }
    }
  }
}

// float-float matrix times FP32 complex vector (x exact in float), compensated.
__device__ __forceinline__ void bsr_row_ffx(const DevMat& m, const float* __restrict__ Ahi,
                                            const float* __restrict__ Alo, const float2* __restrict__ x,
                                            int W, int c, int I, gbff::acc (&are)[4], gbff::acc (&aim)[4]) {
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    gbff::acc_init(are[r]);
    gbff::acc_init(aim[r]);
  }
  const int b1 = m.blk_ptr[I + 1];
#pragma unroll kUnroll
  for (int b = m.blk_ptr[I]; b < b1; ++b) {
    const int J = m.blk_col[b];
    const float2* xr = x + (size_t)(4 * J) * W + c;
    float2 xv[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) xv[t] = xr[(size_t)t * W];
    const float4* ah = reinterpret_cast<const float4*>(Ahi + (size_t)b * 16);
    const float4* al = reinterpret_cast<const float4*>(Alo + (size_t)b * 16);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const float4 h = __ldg(ah + r), l = __ldg(al + r);
      const float hv[4] = {h.x, h.y, h.z, h.w};
      const float lv[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const gbff::ff a = {hv[t], lv[t]};
        gbff::acc_mul_add(are[r], a, xv[t].x);
        gbff::acc_mul_add(aim[r], a, xv[t].y);
      }
    }
  }
}


// ------------------------------------------------------------ warp-cooperative block rows
// The 32 lanes of a warp share one block row I: lane = slot * Wp + c with Wp a
// power of two >= W (Wp <= 32), column c = lane % Wp, and slot s = lane / Wp
// takes the stored blocks b = b0 + s, b0 + s + S, ... (S = 32 / Wp).  Each lane
// accumulates its share; xor shuffles over the slot bits then give every lane
// the full row sums of its column.  Lanes with `active` false (column beyond
// W, or a finished column) skip the loads but still take part in the shuffles.
__device__ __forceinline__ void wbsr_row_d(const DevMat& m, const double* __restrict__ A,
                                           const double2* __restrict__ x, int W, int Wp, int lane, int I,
                                           bool active, double2 (&acc)[4]) {
#pragma unroll
  for (int r = 0; r < 4; ++r) acc[r] = make_double2(0.0, 0.0);
  const int S = 32 / Wp, s = lane / Wp, c = lane - s * Wp;
  if (active) {
    const int b1 = m.blk_ptr[I + 1];
    for (int b = m.blk_ptr[I] + s; b < b1; b += S) {
      const int J = m.blk_col[b];
      const double2* xr = x + (size_t)(4 * J) * W + c;
      double2 xv[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) xv[t] = xr[(size_t)t * W];
      const double2* ab = reinterpret_cast<const double2*>(A + (size_t)b * 16);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const double2 a01 = __ldg(ab + 2 * r), a23 = __ldg(ab + 2 * r + 1);
        acc[r].x = fma(a01.x, xv[0].x, acc[r].x);
        acc[r].y = fma(a01.x, xv[0].y, acc[r].y);
        acc[r].x = fma(a01.y, xv[1].x, acc[r].x);
        acc[r].y = fma(a01.y, xv[1].y, acc[r].y);
        acc[r].x = fma(a23.x, xv[2].x, acc[r].x);
        acc[r].y = fma(a23.x, xv[2].y, acc[r].y);
        acc[r].x = fma(a23.y, xv[3].x, acc[r].x);
        acc[r].y = fma(a23.y, xv[3].y, acc[r].y);
      }
    }
  }
  for (int off = Wp; off < 32; off <<= 1) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      acc[r].x += __shfl_xor_sync(0xffffffffu, acc[r].x, off);
      acc[r].y += __shfl_xor_sync(0xffffffffu, acc[r].y, off);
    }
  }
}

__device__ __forceinline__ void wbsr_row_f(const DevMat& m, const float* __restrict__ A,
                                           const float2* __restrict__ x, int W, int Wp, int lane, int I,
                                           bool active, float2 (&acc)[4]) {
#pragma unroll
  for (int r = 0; r < 4; ++r) acc[r] = make_float2(0.f, 0.f);
  const int S = 32 / Wp, s = lane / Wp, c = lane - s * Wp;
  if (active) {
    const int b1 = m.blk_ptr[I + 1];
    int b = m.blk_ptr[I] + s;
    // groups of four blocks per lane: all block columns first, then every
    // matrix and x load of the group, then the FMAs (four times the loads in
    // flight of a block-at-a-time loop)
    for (; b + 3 * S < b1; b += 4 * S) {
      int J[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) J[u] = __ldg(m.blk_col + b + u * S);
      float4 a[4][4];
      float2 xv[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float4* ab = reinterpret_cast<const float4*>(A + (size_t)(b + u * S) * 16);
#pragma unroll
        for (int r = 0; r < 4; ++r) a[u][r] = __ldg(ab + r);
        const float2* xr = x + (size_t)(4 * J[u]) * W + c;
#pragma unroll
        for (int t = 0; t < 4; ++t) xv[u][t] = xr[(size_t)t * W];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          acc[r].x = fmaf(a[u][r].x, xv[u][0].x, acc[r].x);
          acc[r].y = fmaf(a[u][r].x, xv[u][0].y, acc[r].y);
          acc[r].x = fmaf(a[u][r].y, xv[u][1].x, acc[r].x);
          acc[r].y = fmaf(a[u][r].y, xv[u][1].y, acc[r].y);
          acc[r].x = fmaf(a[u][r].z, xv[u][2].x, acc[r].x);
          acc[r].y = fmaf(a[u][r].z, xv[u][2].y, acc[r].y);
          acc[r].x = fmaf(a[u][r].w, xv[u][3].x, acc[r].x);
          acc[r].y = fmaf(a[u][r].w, xv[u][3].y, acc[r].y);
        }
    }
    for (; b < b1; b += S) {
      const int J = m.blk_col[b];
      const float2* xr = x + (size_t)(4 * J) * W + c;
      float2 xv[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) xv[t] = xr[(size_t)t * W];
      const float4* ab = reinterpret_cast<const float4*>(A + (size_t)b * 16);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float4 a = __ldg(ab + r);
        acc[r].x = fmaf(a.x, xv[0].x, acc[r].x);
        acc[r].y = fmaf(a.x, xv[0].y, acc[r].y);
        acc[r].x = fmaf(a.y, xv[1].x, acc[r].x);
        acc[r].y = fmaf(a.y, xv[1].y, acc[r].y);
        acc[r].x = fmaf(a.z, xv[2].x, acc[r].x);
        acc[r].y = fmaf(a.z, xv[2].y, acc[r].y);
        acc[r].x = fmaf(a.w, xv[3].x, acc[r].x);
        acc[r].y = fmaf(a.w, xv[3].y, acc[r].y);
      }
    }
  }
  for (int off = Wp; off < 32; off <<= 1) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      acc[r].x += __shfl_xor_sync(0xffffffffu, acc[r].x, off);
      acc[r].y += __shfl_xor_sync(0xffffffffu, acc[r].y, off);
    }
  }
}

// compensated sum of two accumulators held by lanes `lane` and `lane ^ off`
__device__ __forceinline__ void acc_xor_combine(gbff::acc& a, int off) {
  const float oh = __shfl_xor_sync(0xffffffffu, a.hi, off);
  const float oe = __shfl_xor_sync(0xffffffffu, a.err, off);
  const gbff::ff sm = gbff::two_sum(a.hi, oh);
  a.hi = sm.hi;
  a.err = __fadd_rn(__fadd_rn(a.err, oe), sm.lo);
}

// float-float matrix (hi + lo) times float-float complex vector (float4 {re.hi,
// re.lo, im.hi, im.lo}), compensated accumulation and compensated combine.
__device__ __forceinline__ void wbsr_row_ff(const DevMat& m, const float* __restrict__ Ahi,
                                            const float* __restrict__ Alo, const float4* __restrict__ x, int W,
                                            int Wp, int lane, int I, bool active, gbff::acc (&are)[4],
                                            gbff::acc (&aim)[4]) {
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    gbff::acc_init(are[r]);
    gbff::acc_init(aim[r]);
  }
  const int S = 32 / Wp, s = lane / Wp, c = lane - s * Wp;
  if (active) {
    const int b1 = m.blk_ptr[I + 1];
    for (int b = m.blk_ptr[I] + s; b < b1; b += S) {
      const int J = m.blk_col[b];
      const float4* xr = x + (size_t)(4 * J) * W + c;
      float4 xv[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) xv[t] = xr[(size_t)t * W];
      const float4* ah = reinterpret_cast<const float4*>(Ahi + (size_t)b * 16);
      const float4* al = reinterpret_cast<const float4*>(Alo + (size_t)b * 16);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float4 h = __ldg(ah + r), l = __ldg(al + r);
        const float hv[4] = {h.x, h.y, h.z, h.w};
        const float lv[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const gbff::ff a = {hv[t], lv[t]};
          gbff::acc_mul_add(are[r], a, gbff::ff{xv[t].x, xv[t].y});
          gbff::acc_mul_add(aim[r], a, gbff::ff{xv[t].z, xv[t].w});
        }
      }
    }
  }
  for (int off = Wp; off < 32; off <<= 1) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      acc_xor_combine(are[r], off);
      acc_xor_combine(aim[r], off);
    }
  }
}

// float-float matrix times FP32 complex vector (exact in float), compensated.
__device__ __forceinline__ void wbsr_row_ffx(const DevMat& m, const float* __restrict__ Ahi,
                                             const float* __restrict__ Alo, const float2* __restrict__ x, int W,
                                             int Wp, int lane, int I, bool active, gbff::acc (&are)[4],
                                             gbff::acc (&aim)[4]) {
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    gbff::acc_init(are[r]);
    gbff::acc_init(aim[r]);
  }
  const int S = 32 / Wp, s = lane / Wp, c = lane - s * Wp;
  if (active) {
    const int b1 = m.blk_ptr[I + 1];
    for (int b = m.blk_ptr[I] + s; b < b1; b += S) {
      const int J = m.blk_col[b];
      const float2* xr = x + (size_t)(4 * J) * W + c;
      float2 xv[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) xv[t] = xr[(size_t)t * W];
      const float4* ah = reinterpret_cast<const float4*>(Ahi + (size_t)b * 16);
      const float4* al = reinterpret_cast<const float4*>(Alo + (size_t)b * 16);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float4 h = __ldg(ah + r), l = __ldg(al + r);
        const float hv[4] = {h.x, h.y, h.z, h.w};
        const float lv[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const gbff::ff a = {hv[t], lv[t]};
          gbff::acc_mul_add(are[r], a, xv[t].x);
          gbff::acc_mul_add(aim[r], a, xv[t].y);
        }
      }
    }
  }
  for (int off = Wp; off < 32; off <<= 1) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      acc_xor_combine(are[r], off);
      acc_xor_combine(aim[r], off);
    }
  }
}

}  // namespace gbk
