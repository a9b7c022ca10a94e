// Exact inner solve S x = f with the block-bidiagonal Cholesky factor of S.
//
// The shifted COCG recurrence applies S^{-1} once per outer iteration (and the
// mixed path two or more times, around float-float residuals).  An iterative
// inner solve leaves a relative error of its tolerance in every application,
// and near a spectral gap the shifted residuals amplify that error by ~1e9;
// the factor solve is exact to rounding instead.  For S with half-bandwidth
// bw <= 63 the Cholesky factor L, cut into 64-row blocks, is block lower
// bidiagonal (diagonal blocks D_i, sub-diagonal blocks C_i), and with the
// host-built products E_i = D_i^-1 C_i, F_i = D_i^-T C_{i+1}^T:
//   L y = f   :  t_i = D_i^-1 f_i (every block independent),  y_i = t_i - E_i y_{i-1}
//   L^T x = y :  u_i = D_i^-T y_i (every block independent),  x_i = u_i - F_i x_{i+1}
// The team walks the blocks in order for all four passes.  Every pass step
// multiplies one 64 x 64 (triangular) or 64 x bw (band) tile by a 64-row block
// of the W columns; in the FP32 levels the tiles are staged into shared memory
// by TMA bulk copies (cp.async.bulk + mbarrier), two tiles ahead of use, and
// the next block's vector inputs are prefetched into registers, so a step
// waits only for its own arithmetic and two barriers.  The FP64 solve is bound
// by the FP64 FMA rate and reads its tiles through L2.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "kernels.cuh"

namespace gbk {

template <typename T>
struct CplxOf;
template <>
struct CplxOf<float> {
  using type = float2;
};
template <>
struct CplxOf<double> {
  using type = double2;
};

// rows per thread (adjacent), columns per thread, TMA staging of the tiles
template <typename T>
struct BcCfg;
template <>
struct BcCfg<float> {
  static constexpr int RPT = 2, CW = 4;
  static constexpr bool TMA = true;
};
template <>
struct BcCfg<double> {
  static constexpr int RPT = 1, CW = 2;
  static constexpr bool TMA = false;
};

constexpr int kTileBufs = 3;                            // staged tiles: two in flight ahead of the one in use
constexpr unsigned kRedBytes = NWARP * NVMAX * 32 * 8;  // block_reduce's partials

// Dynamic shared memory of a team (host and device agree through this):
//   [partials: block_reduce's, or the chain's nks x 64 x (W+1) sums, or the
//    triangular pass's input block]  [y block: 64 x W]  [FP32: 3 tiles of 64 x 64]
//   or, for the iterative inner solve with its vectors in shared memory,
//   [partials] [g, d, q]
struct DynLayout {
  int cw, nchunk, nks, G;
  unsigned o_red, o_ysm, o_ebuf, o_cg, bytes;
};
__host__ __device__ inline DynLayout dyn_layout(bool fp64, int W, bool bchol, unsigned cg_bytes) {
  DynLayout L;
  const int RPT = fp64 ? 1 : 2, CW = fp64 ? 2 : 4;
  const unsigned esz = fp64 ? 16u : 8u;
  L.G = TPB / (64 / RPT);
  L.cw = W < CW ? W : CW;
  L.nchunk = W / L.cw;
  L.nks = L.nchunk >= L.G ? 1 : L.G / L.nchunk;
  unsigned red = kRedBytes;
  if (bchol) {
    const unsigned part = (unsigned)(L.nks * 64 * (W + 1)) * esz, xin = 64u * (unsigned)W * esz;
    red = red > part ? red : part;
    red = red > xin ? red : xin;
  }
  unsigned off = 0;
  L.o_red = off;
  off = (off + red + 127u) & ~127u;
  L.o_ysm = off;
  L.o_cg = off;
  if (bchol) {
    off = (off + 64u * (unsigned)W * esz + 127u) & ~127u;
    L.o_ebuf = off;
    if (!fp64) off += kTileBufs * 4096u * 4u;
  } else {
    L.o_ebuf = off;
    off += cg_bytes;
  }
  L.bytes = (off + 127u) & ~127u;
  return L;
}

// ------------------------------------------------------------ TMA bulk copy + mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// One thread: expect `bytes` on `bar` and start the copy global -> shared.
// src and dst 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void tma_bulk_g2s(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait: gives up after 0.2 s (a tile lands in microseconds) or 2^20
// polls, whichever comes first; the caller records the failure and later
// waits of the launch are skipped.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, uint32_t parity) {
  const unsigned long long t0 = global_ns();
  for (int it = 0; it < (1 << 20); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > 200000000ull) break;
  }
  return false;
}

// Tiles of one pass, staged through the kTileBufs buffers.  Tile number q of
// the launch (sm.tile_base + the pass-local index) lives in buffer q % 3 and
// completes barrier q % 3 for the (q / 3)-th time, so its wait parity is
// (q / 3) & 1.  Thread 0 issues; every issued tile is consumed in its pass.
struct TilePipe {
  float* ebuf;
  unsigned base;
};
__device__ __forceinline__ void tile_issue(const TilePipe& tp, Smem& sm, unsigned i, const float* src,
                                           uint32_t off, uint32_t bytes) {
  const unsigned q = tp.base + i;
  fence_proxy_async_smem();  // the generic-proxy reads of this buffer (a tile earlier) come first
  tma_bulk_g2s(tp.ebuf + (q % kTileBufs) * 4096 + off, src + off, bytes, &sm.bc_bar[q % kTileBufs]);
}
__device__ __forceinline__ const float* tile_wait(const TilePipe& tp, Smem& sm, unsigned i) {
  const unsigned q = tp.base + i;
  if (!sm.bc_fail && !mbar_wait_bounded(&sm.bc_bar[q % kTileBufs], (q / kTileBufs) & 1u)) sm.bc_fail = 1;
  return tp.ebuf + (q % kTileBufs) * 4096;
}

// ------------------------------------------------------------ element helpers
__device__ __forceinline__ float2 bc_in(const float2* p, size_t e) { return p[e]; }
__device__ __forceinline__ float2 bc_in(const float4* p, size_t e) {  // hi parts of a float-float vector
  const float4 v = p[e];
  return make_float2(v.x, v.z);
}
__device__ __forceinline__ double2 bc_in(const double2* p, size_t e) { return p[e]; }
__device__ __forceinline__ void cfma(float2& acc, float m, float2 v) {
  acc.x = fmaf(m, v.x, acc.x);
  acc.y = fmaf(m, v.y, acc.y);
}
__device__ __forceinline__ void cfma(double2& acc, double m, double2 v) {
  acc.x = fma(m, v.x, acc.x);
  acc.y = fma(m, v.y, acc.y);
}
template <typename C>
__device__ __forceinline__ C czero();
template <>
__device__ __forceinline__ float2 czero<float2>() {
  return make_float2(0.f, 0.f);
}
template <>
__device__ __forceinline__ double2 czero<double2>() {
  return make_double2(0.0, 0.0);
}
__device__ __forceinline__ float2 csub_(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 csub_(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cadd_(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cadd_(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// ------------------------------------------------------------ triangular pass, FP32
// out_i = M_i in_i for every block i in order (M_i = D_i^-1 lower, or D_i^-T
// upper, k-major).  Per step: the block's 64 x W inputs (prefetched into
// registers one step ahead) go to shared memory, the tile waits in its TMA
// buffer, and each thread forms two adjacent columns (one when W = 1) of one
// row over that row's triangle.  Ends with a barrier.
template <bool LOWER, typename InT>
__device__ __noinline__ void bc_tri_f32(const Args& a, Smem& sm, const float* __restrict__ Mall,
                                        const InT* __restrict__ in, float2* __restrict__ out, char* dyn) {
  const int W = a.W, N4 = 4 * a.m.nb, nblk = a.m.bf_nblk, tid = threadIdx.x;
  const DynLayout L = dyn_layout(false, W, true, 0);
  float2* xin = reinterpret_cast<float2*>(dyn + L.o_red);
  const TilePipe tp{reinterpret_cast<float*>(dyn + L.o_ebuf), sm.tile_base};
  const int per = 64 * W;          // inputs / outputs per block
  const int cw2 = W >= 2 ? 2 : 1;  // columns per thread
  const int nq = W / cw2;          // column groups per row
  constexpr int PF = 64 * WMAX / TPB;  // inputs per thread per block
  float2 pre[PF];
  auto load_block = [&](int i) {
#pragma unroll
    for (int m = 0; m < PF; ++m) {
      const int o = tid + m * TPB;
      const int row = 64 * i + o / W;
      pre[m] = (o < per && row < N4) ? bc_in(in, (size_t)64 * i * W + o) : make_float2(0.f, 0.f);
    }
  };
  if (tid == 0) {
    tile_issue(tp, sm, 0, Mall, 0, 4096u * 4u);
    if (nblk > 1) tile_issue(tp, sm, 1, Mall + 4096, 0, 4096u * 4u);
  }
  load_block(0);
  for (int i = 0; i < nblk; ++i) {
#pragma unroll
    for (int m = 0; m < PF; ++m) {
      const int o = tid + m * TPB;
      if (o < per) xin[o] = pre[m];
    }
    if (i + 1 < nblk) load_block(i + 1);
    if (tid == 0 && i + 2 < nblk) tile_issue(tp, sm, (unsigned)(i + 2), Mall + (size_t)(i + 2) * 4096, 0, 4096u * 4u);
    const float* Mt = tile_wait(tp, sm, (unsigned)i);
    __syncthreads();
    for (int o = tid; o < 64 * nq; o += TPB) {
      const int r = o / nq, c0 = (o - r * nq) * cw2;
      const int kb = LOWER ? 0 : r, ke = LOWER ? r + 1 : 64;
      float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
#pragma unroll 4
      for (int k = kb; k < ke; ++k) {
        const float mv = Mt[k * 64 + r];
        if (cw2 == 2) {
          const float4 v = *reinterpret_cast<const float4*>(xin + k * W + c0);
          cfma(acc0, mv, make_float2(v.x, v.y));
          cfma(acc1, mv, make_float2(v.z, v.w));
        } else {
          cfma(acc0, mv, xin[k * W + c0]);
        }
      }
      const int row = 64 * i + r;
      if (row < N4) {
        if (sm.act[c0]) out[(size_t)row * W + c0] = acc0;
        if (cw2 == 2 && sm.act[c0 + 1]) out[(size_t)row * W + c0 + 1] = acc1;
      }
    }
    // every thread read sm.tile_base at entry, before this pass's first
    // barrier; the next pass reads it after the barrier below
    if (tid == 0 && i + 1 == nblk) sm.tile_base = tp.base + (unsigned)nblk;
    __syncthreads();
  }
}

// ------------------------------------------------------------ triangular pass, FP64
// Same products in FP64: one warp per (block, column chunk), lane l owns rows
// l and l + 32, each over its triangle; tiles read through L2 (the pass is
// bound by the FP64 FMA rate).  No barrier at the end.
template <bool LOWER, int CWV, typename InT>
__device__ __noinline__ void bc_tri_f64(const Args& a, const Smem& sm, const double* __restrict__ Mall,
                                        const InT* __restrict__ in, double2* __restrict__ out) {
  const int W = a.W, N4 = 4 * a.m.nb, nblk = a.m.bf_nblk;
  const int nchunk = W / CWV, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int task = warp; task < nblk * nchunk; task += NWARP) {
    const int blk = task / nchunk, ch = task - blk * nchunk, c0 = ch * CWV, base = 64 * blk;
    const double* __restrict__ M = Mall + (size_t)blk * 4096;
    double2 acc0[CWV], acc1[CWV];
#pragma unroll
    for (int j = 0; j < CWV; ++j) {
      acc0[j] = czero<double2>();
      acc1[j] = czero<double2>();
    }
    const int kmax = min(64, N4 - base);
    const int k32 = min(32, kmax);
#pragma unroll 4
    for (int k = 0; k < k32; ++k) {  // LOWER: row l needs k <= l, row l+32 all; UPPER: only row l (k >= l)
      const size_t e = (size_t)(base + k) * W + c0;
      const bool u0 = LOWER ? k <= lane : k >= lane;
      const double m0 = u0 ? __ldg(M + k * 64 + lane) : 0.0;
      const double m1 = LOWER ? __ldg(M + k * 64 + 32 + lane) : 0.0;
#pragma unroll
      for (int j = 0; j < CWV; ++j) {
        const double2 v = bc_in(in, e + j);
        if (u0) cfma(acc0[j], m0, v);
        if (LOWER) cfma(acc1[j], m1, v);
      }
    }
#pragma unroll 4
    for (int k = 32; k < kmax; ++k) {  // LOWER: only row l+32 (k <= l+32); UPPER: row l all, row l+32 k >= l+32
      const size_t e = (size_t)(base + k) * W + c0;
      const bool u1 = LOWER ? k <= lane + 32 : k >= lane + 32;
      const double m0 = LOWER ? 0.0 : __ldg(M + k * 64 + lane);
      const double m1 = u1 ? __ldg(M + k * 64 + 32 + lane) : 0.0;
#pragma unroll
      for (int j = 0; j < CWV; ++j) {
        const double2 v = bc_in(in, e + j);
        if (!LOWER) cfma(acc0[j], m0, v);
        if (u1) cfma(acc1[j], m1, v);
      }
    }
#pragma unroll
    for (int j = 0; j < CWV; ++j) {
      if (!sm.act[c0 + j]) continue;
      if (base + lane < N4) out[(size_t)(base + lane) * W + c0 + j] = acc0[j];
      if (base + lane + 32 < N4) out[(size_t)(base + lane + 32) * W + c0 + j] = acc1[j];
    }
  }
}

// ------------------------------------------------------------ the sequential chain
// FWD: y_0 = t_0, y_i = t_i - E_i y_{i-1} (k over the last bw rows of y_{i-1});
// BWD: x_last = u_last, x_i = u_i - F_i x_{i+1} (k over the first bw rows).
// Thread = (row pair or row, column chunk, slice of k); partial sums meet in
// shared memory.  tin and yout may alias (each element is read, one step
// ahead, before it is written, by the same thread).  Ends with a barrier.
template <typename T, int CWV, int PF, bool FWD>
__device__ __noinline__ void bc_chain(const Args& a, Smem& sm, const T* __restrict__ Mall,
                                      const typename CplxOf<T>::type* tin, typename CplxOf<T>::type* yout,
                                      char* dyn) {
  using C = typename CplxOf<T>::type;
  using Cfg = BcCfg<T>;
  constexpr int RPT = Cfg::RPT;
  const int W = a.W, N4 = 4 * a.m.nb, nblk = a.m.bf_nblk, bw = a.m.bf_bw, tid = threadIdx.x;
  const DynLayout L = dyn_layout(sizeof(T) == 8, W, true, 0);
  C* red = reinterpret_cast<C*>(dyn + L.o_red);
  C* ysm = reinterpret_cast<C*>(dyn + L.o_ysm);
  const TilePipe tp{reinterpret_cast<float*>(dyn + L.o_ebuf), sm.tile_base};
  const int kbase = FWD ? 64 - bw : 0;
  const uint32_t tile_off = (uint32_t)kbase * 64u;  // elements
  const uint32_t tile_bytes = (uint32_t)bw * 64u * (uint32_t)sizeof(T);
  const int nsteps = nblk - 1;
  auto blk_of = [&](int s) { return FWD ? s : nblk - 1 - s; };  // s = 0: the chain's first block
  const bool stage = Cfg::TMA && bw > 0;
  {  // first block of the chain
    const int i0 = blk_of(0);
    for (int o = tid; o < 64 * W; o += TPB) {
      const int r = o / W, c = o - r * W, row = 64 * i0 + r;
      const C v = row < N4 ? tin[(size_t)64 * i0 * W + o] : czero<C>();
      ysm[o] = v;
      if (row < N4 && sm.act[c]) yout[(size_t)64 * i0 * W + o] = v;
    }
    if (stage && tid == 0)
      for (int s = 1; s <= 2 && s <= nsteps; ++s)
        tile_issue(tp, sm, (unsigned)(s - 1), reinterpret_cast<const float*>(Mall) + (size_t)blk_of(s) * 4096,
                   tile_off, tile_bytes);
    __syncthreads();
  }
  const int nrp = 64 / RPT, rp = tid % nrp, g = tid / nrp, r0 = rp * RPT;
  const int nks = L.nks, nchunk = L.nchunk;
  const int len = (bw + nks - 1) / nks;
  C tnext[PF];  // PF = ceil(64 W / TPB): t values per thread per block
  auto load_t = [&](int s) {  // this thread's t values, one step ahead of use
    const int i = blk_of(s);
#pragma unroll
    for (int m = 0; m < PF; ++m) {
      const int o = tid + m * TPB;
      const int row = 64 * i + o / W;
      tnext[m] = (o < 64 * W && row < N4) ? tin[(size_t)64 * i * W + o] : czero<C>();
    }
  };
  if (nsteps > 0) load_t(1);
  for (int s = 1; s <= nsteps; ++s) {
    const int i = blk_of(s);
    C tcur[PF];
#pragma unroll
    for (int m = 0; m < PF; ++m) tcur[m] = tnext[m];
    if (s + 1 <= nsteps) load_t(s + 1);
    const T* __restrict__ Mt;
    if constexpr (Cfg::TMA) {
      if (stage && tid == 0 && s + 2 <= nsteps)
        tile_issue(tp, sm, (unsigned)(s + 1), reinterpret_cast<const float*>(Mall) + (size_t)blk_of(s + 2) * 4096,
                   tile_off, tile_bytes);
      Mt = reinterpret_cast<const T*>(stage ? tile_wait(tp, sm, (unsigned)(s - 1)) : tp.ebuf);
    } else {
      Mt = Mall + (size_t)i * 4096;
    }
    // partial products over this thread's slice of k
    for (int ch = (nks == 1 ? g : g / nks); ch < nchunk; ch += (nks == 1 ? L.G : nchunk)) {
      const int ks = nks == 1 ? 0 : g % nks, c0 = ch * CWV;
      const int kb = kbase + ks * len, ke = min(kb + len, kbase + bw);
      C acc[RPT][CWV];
#pragma unroll
      for (int q = 0; q < RPT; ++q)
#pragma unroll
        for (int j = 0; j < CWV; ++j) acc[q][j] = czero<C>();
#pragma unroll 2
      for (int k = kb; k < ke; ++k) {
        T mv[RPT];
        if constexpr (RPT == 2) {
          const float2 m2 = *reinterpret_cast<const float2*>(Mt + k * 64 + r0);
          mv[0] = m2.x;
          mv[1] = m2.y;
        } else {
          mv[0] = Cfg::TMA ? Mt[k * 64 + r0] : __ldg(Mt + k * 64 + r0);
        }
        C yv[CWV];
        if constexpr (sizeof(T) == 4 && CWV == 4) {
          const float4* yp = reinterpret_cast<const float4*>(ysm + k * W + c0);
          const float4 y01 = yp[0], y23 = yp[1];
          yv[0] = make_float2(y01.x, y01.y);
          yv[1] = make_float2(y01.z, y01.w);
          yv[2] = make_float2(y23.x, y23.y);
          yv[3] = make_float2(y23.z, y23.w);
        } else {
#pragma unroll
          for (int j = 0; j < CWV; ++j) yv[j] = ysm[k * W + c0 + j];
        }
#pragma unroll
        for (int q = 0; q < RPT; ++q)
#pragma unroll
          for (int j = 0; j < CWV; ++j) cfma(acc[q][j], mv[q], yv[j]);
      }
#pragma unroll
      for (int q = 0; q < RPT; ++q)
#pragma unroll
        for (int j = 0; j < CWV; ++j) red[((size_t)ks * 64 + r0 + q) * (W + 1) + c0 + j] = acc[q][j];
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < PF; ++m) {
      const int o = tid + m * TPB;
      if (o >= 64 * W) break;
      const int r = o / W, c = o - r * W, row = 64 * i + r;
      C sacc = czero<C>();
      for (int ks = 0; ks < nks; ++ks) sacc = cadd_(sacc, red[((size_t)ks * 64 + r) * (W + 1) + c]);
      const C y = row < N4 ? csub_(tcur[m], sacc) : czero<C>();
      ysm[o] = y;
      if (row < N4 && sm.act[c]) yout[(size_t)64 * i * W + o] = y;
    }
    if (stage && tid == 0 && s == nsteps) sm.tile_base = tp.base + (unsigned)nsteps;  // see bc_tri_f32
    __syncthreads();
  }
}

// x = S^-1 f for every active column of the panel.  t1, t2: panel-sized
// scratch vectors (global).  f may be a float-float vector (its hi parts are
// solved).  Ends with a barrier.
template <typename T, int CWV, int PF, typename InT>
__device__ void bc_solve_w(const Args& a, Smem& sm, const InT* f, typename CplxOf<T>::type* x,
                           typename CplxOf<T>::type* t1, typename CplxOf<T>::type* t2, char* dyn) {
  const size_t part = (size_t)a.m.bf_nblk * 4096;
  if constexpr (sizeof(T) == 4) {
    const float* bf = a.m.bf32;
    bc_tri_f32<true>(a, sm, bf, f, t1, dyn);
    bc_chain<T, CWV, PF, true>(a, sm, bf + 2 * part, t1, t1, dyn);
    bc_tri_f32<false>(a, sm, bf + part, t1, t2, dyn);
    bc_chain<T, CWV, PF, false>(a, sm, bf + 3 * part, t2, x, dyn);
  } else {
    const double* bf = a.m.bf64;
    bc_tri_f64<true, CWV>(a, sm, bf, f, t1);
    __syncthreads();
    bc_chain<T, CWV, PF, true>(a, sm, bf + 2 * part, t1, t1, dyn);
    bc_tri_f64<false, CWV>(a, sm, bf + part, t1, t2);
    __syncthreads();
    bc_chain<T, CWV, PF, false>(a, sm, bf + 3 * part, t2, x, dyn);
  }
  if (threadIdx.x == 0) ++sm.inner_count;
}

template <typename T, typename InT>
__device__ void bc_solve(const Args& a, Smem& sm, const InT* f, typename CplxOf<T>::type* x,
                         typename CplxOf<T>::type* t1, typename CplxOf<T>::type* t2, char* dyn) {
  constexpr int CW = BcCfg<T>::CW;
  static_assert(TPB == 512, "outputs per thread assume 512-thread teams");
  if (a.W == 32)
    bc_solve_w<T, CW, 4>(a, sm, f, x, t1, t2, dyn);
  else if (a.W == 16)
    bc_solve_w<T, CW, 2>(a, sm, f, x, t1, t2, dyn);
  else if (a.W >= CW)
    bc_solve_w<T, CW, 1>(a, sm, f, x, t1, t2, dyn);
  else if (CW == 4 && a.W == 2)
    bc_solve_w<T, (CW == 4 ? 2 : 1), 1>(a, sm, f, x, t1, t2, dyn);
  else
    bc_solve_w<T, 1, 1>(a, sm, f, x, t1, t2, dyn);
}

}  // namespace gbk
