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

// columns per thread in the FP64 chain (the FP32 passes tile by 8 real columns)
template <typename T>
struct BcCfg;
template <>
struct BcCfg<float> {
  static constexpr int CW = 4;
};
template <>
struct BcCfg<double> {
  static constexpr int CW = 2;
};

constexpr int kTileBufs = 3;                            // FP32 factor tiles staged: two in flight ahead of the one in use
constexpr unsigned kRedBytes = NWARP * NVMAX * 32 * 8;  // block_reduce's partials

// Dynamic shared memory of a team (host and device agree through this):
//   FP32 factor passes: the tensor-core layout below (mma_layout);
//   FP64 factor chain: [partials: block_reduce's, or the chain's nks x 64 x
//   (W+1) sums]  [y block: 64 x W];
//   iterative inner solve with its vectors in shared memory: [partials] [g, d, q]
struct DynLayout {
  int cw, nchunk, nks, G;
  unsigned o_red, o_ysm, o_ebuf, o_cg, bytes;
};
// FP32 tensor-core passes: [S staged factor tiles][input block x 2][output
// block x 2], blocks of 64 rows x P floats (2 W real columns, padded so that
// the B-fragment loads are free of bank conflicts); S = 3 stages up to W = 8,
// 2 beyond.  A tile holds the 20 triangular fragments and the band fragments
// of a half-bandwidth bw (512 bytes each).  block_reduce's partials alias the
// first stage (the passes and the reductions never overlap).
struct MmaLayout {
  int P, nt, S;
  unsigned stage_floats, o_fin, o_ysm, o_xch, bytes;
};
__host__ __device__ inline MmaLayout mma_layout(int W, int bw) {
  MmaLayout L;
  L.P = 2 * W + 8 > 24 ? 2 * W + 8 : 24;
  L.nt = W >= 4 ? W / 4 : 1;  // n-tiles of 8 real columns
  L.S = W <= 8 ? 3 : 2;
  const int n2 = (bw + 7) / 8 > 8 - (64 - bw) / 8 ? (bw + 7) / 8 : 8 - (64 - bw) / 8;
  L.stage_floats = (unsigned)(20 + 4 * n2) * 128u;
  unsigned off = (unsigned)L.S * L.stage_floats * 4u;
  if (off < kRedBytes) off = kRedBytes;
  off = (off + 127u) & ~127u;
  L.o_fin = off;
  off += 2u * 64u * (unsigned)L.P * 4u;
  L.o_ysm = off;
  off += 2u * 64u * (unsigned)L.P * 4u;
  L.o_xch = off;  // band partials handed from one warp to its partner: 8 tiles x 32 lanes x 4
  off += 8u * 32u * 4u * 4u;
  L.bytes = (off + 127u) & ~127u;
  return L;
}

__host__ __device__ inline DynLayout dyn_layout(bool fp64, int W, bool bchol, unsigned cg_bytes, int bw = 63) {
  DynLayout L;
  if (bchol && !fp64) {
    const MmaLayout M = mma_layout(W, bw);
    L.cw = L.nchunk = L.nks = L.G = 0;
    L.o_red = 0;
    L.o_ysm = M.o_ysm;
    L.o_ebuf = 0;
    L.o_cg = M.bytes;
    L.bytes = M.bytes;
    return L;
  }
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
  if (bchol) {  // FP64 chain: the y block
    off = (off + 64u * (unsigned)W * esz + 127u) & ~127u;
    L.o_ebuf = off;
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

// ------------------------------------------------------------ FP32 passes on tensor cores
// One pass walks the blocks and forms, per block i (FWD, i ascending):
//   y_i = D_i^-1 f_i - E_i y_{i-1},
// (BWD, i descending: x_i = D_i^-T y_i - F_i x_{i+1}) as 64 x 2W products on
// m16n8k8 TF32 MMAs, one warp per 16 x 8 output tile.  FP32 accuracy from
// TF32 units: every operand is split into a TF32 head and a tail whose TF32
// part the units read (a = a_h + a_t to ~2^-21) and a b = a_h b_h + a_h b_t +
// a_t b_h is accumulated in FP32.  Per step: the block's tile (fragment order, built on
// the host) waits in its TMA stage, the input block was staged a step
// earlier, the previous output block sits in shared memory; one barrier.
// Head: x rounded to 11 significant bits (add half a TF32 unit to the bit
// pattern, clear the 13 low bits: exactly a TF32 value); tail: x - head,
// exact in FP32 and at most half a TF32 unit, of which the MMA reads the
// TF32 part (the units ignore the 13 low bits of a .tf32 operand).  Three
// full-rate integer / FP32 instructions per value.
__device__ __forceinline__ void split_tf32(float x, uint32_t& h, uint32_t& t) {
  h = (__float_as_uint(x) + 0x1000u) & 0xffffe000u;
  t = __float_as_uint(x - __uint_as_float(h));
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
// acc_h += A_h B_h, acc_t += A_h B_t + A_t B_h for one k-step: A fragment
// (four values of this lane) from the staged tile, B rows 8 ks + t, + 4 of
// column 8 ni + g of the block in shared memory (row stride P).
__device__ __forceinline__ void mma_kstep(float (&acc_h)[4], float (&acc_t)[4], float (&acc_u)[4],
                                          const float* __restrict__ frag, const float* __restrict__ B, int P, int ks,
                                          int ni, int lane) {
  const float4 av = *reinterpret_cast<const float4*>(frag + lane * 4);
  uint32_t ah[4], at[4];
  split_tf32(av.x, ah[0], at[0]);
  split_tf32(av.y, ah[1], at[1]);
  split_tf32(av.z, ah[2], at[2]);
  split_tf32(av.w, ah[3], at[3]);
  const int g = lane >> 2, t = lane & 3;
  uint32_t bh0, bt0, bh1, bt1;
  split_tf32(B[(8 * ks + t) * P + 8 * ni + g], bh0, bt0);
  split_tf32(B[(8 * ks + t + 4) * P + 8 * ni + g], bh1, bt1);
  mma_tf32(acc_h, ah, bh0, bh1);
  mma_tf32(acc_t, ah, bt0, bt1);
  mma_tf32(acc_u, at, bh0, bh1);
}
__device__ __forceinline__ void named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

template <bool FWD, int PF, typename InT>
__device__ __noinline__ void bc_pass_mma(const Args& a, Smem& sm, const InT* __restrict__ in, float2* __restrict__ out) {
  const int W = a.W, N4 = 4 * a.m.nb, nblk = a.m.bf_nblk, bw = a.m.bf_bw, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5, g = lane >> 2, t = lane & 3;
  const MmaLayout L = mma_layout(W, a.bc_bw_alloc);
  extern __shared__ __align__(16) char bc_dyn[];
  float* stage = reinterpret_cast<float*>(bc_dyn);
  float* fin = reinterpret_cast<float*>(bc_dyn + L.o_fin);
  float* ysm = reinterpret_cast<float*>(bc_dyn + L.o_ysm);
  float* xch = reinterpret_cast<float*>(bc_dyn + L.o_xch);
  const int P = L.P, S = L.S, ntile = 4 * L.nt;
  const int ksE0 = (64 - bw) / 8, nF = (bw + 7) / 8;
  const int n2 = FWD ? 8 - ksE0 : nF;  // band k-steps
  const uint32_t tile_bytes = (uint32_t)(20 + 4 * n2) * 512u;
  const float* tiles = a.m.bfm + (FWD ? 0 : kMmaTileFloatsDev);
  const unsigned base = sm.tile_base;
  auto blk_of = [&](int s) { return FWD ? s : nblk - 1 - s; };
  auto issue = [&](int s) {  // thread 0: the tile of step s into stage (base + s) % S
    const unsigned q = base + (unsigned)s;
    fence_proxy_async_smem();
    tma_bulk_g2s(stage + (q % S) * L.stage_floats, tiles + (size_t)(2 * blk_of(s)) * kMmaTileFloatsDev, tile_bytes,
                 &sm.bc_bar[q % S]);
  };
  // input blocks: this thread's PF complex values of a block, DEPTH blocks ahead
  constexpr int DEPTH = PF == 1 ? 3 : 2;
  float2 pq[DEPTH][PF];
  auto load_block = [&](float2 (&dst)[PF], int s) {
    const int i = blk_of(s);
#pragma unroll
    for (int m = 0; m < PF; ++m) {
      const int o = tid + m * TPB;
      const int row = 64 * i + o / W;
      dst[m] = (s < nblk && o < 64 * W && row < N4) ? bc_in(in, (size_t)64 * i * W + o) : make_float2(0.f, 0.f);
    }
  };
  auto store_block = [&](const float2 (&src)[PF], float* dst) {
#pragma unroll
    for (int m = 0; m < PF; ++m) {
      const int o = tid + m * TPB;
      if (o < 64 * W) {
        const int r = o / W, c = o - r * W;
        *reinterpret_cast<float2*>(dst + r * P + 2 * c) = src[m];
      }
    }
  };
  // prologue: zero both staging areas (padding columns stay zero), stage
  // block 0, queue blocks 1..DEPTH, issue the first tiles
  for (int e = tid; e < 4 * 64 * P; e += TPB) fin[e] = 0.f;  // fin and ysm are adjacent
  if (tid == 0)
    for (int s = 0; s < S - 1 && s < nblk; ++s) issue(s);
  {
    float2 b0[PF];
    load_block(b0, 0);
#pragma unroll
    for (int d = 0; d < DEPTH; ++d) load_block(pq[(1 + d) % DEPTH], 1 + d);
    __syncthreads();  // zeroing done before the stores below
    store_block(b0, fin);
  }
  __syncthreads();
  // One step per block.  The register queue of input blocks rotates by slot
  // (the loop is unrolled DEPTH times so the slots stay registers): step s
  // stages block s + 1 from slot (s + 1) % DEPTH and refills that slot with
  // block s + 1 + DEPTH.
  auto step = [&](int s, float2 (&slot)[PF]) {
    const int i = blk_of(s);
    const float* fcur = fin + (s & 1) * 64 * P;
    const float* yprev = ysm + ((s + 1) & 1) * 64 * P;
    float* ycur = ysm + (s & 1) * 64 * P;
    if (s + 1 < nblk) {  // stage the next input block (its buffer was read a step ago)
      store_block(slot, fin + ((s + 1) & 1) * 64 * P);
      load_block(slot, s + 1 + DEPTH);
    }
    if (tid == 0 && s + S - 1 < nblk) issue(s + S - 1);
    const unsigned q = base + (unsigned)s;
    if (!sm.bc_fail && !mbar_wait_bounded(&sm.bc_bar[q % S], (q / S) & 1u)) sm.bc_fail = 1;
    const float* T = stage + (q % S) * L.stage_floats;
    // Up to eight tiles (W <= 8): warp w < ntile forms the triangular part of
    // tile w, warp ntile + w its band part, and hands it over through shared
    // memory (a named barrier per pair); more tiles: one warp per tile.
    const bool split = 2 * ntile <= NWARP;
    const int nunits = split ? 2 * ntile : ntile;
    for (int u = warp; u < nunits; u += NWARP) {
      const int ot = split ? u % ntile : u, role = split ? u / ntile : 2;  // 0 tri, 1 band, 2 both
      // Warp w runs on sub-partition w mod 4.  The triangular part of m-tile
      // mi takes 2 mi + 2 (FWD) or 8 - 2 mi (BWD) k-steps, so odd n-tiles run
      // the m-tiles in reverse: every sub-partition then issues the same
      // number of tensor instructions per step (10 k-steps of triangle per
      // pair of n-tiles instead of 4 .. 16).
      const int ni = ot >> 2, mi = (ni & 1) ? 3 - (ot & 3) : (ot & 3);
      float dh[4] = {0.f, 0.f, 0.f, 0.f}, dt[4] = {0.f, 0.f, 0.f, 0.f}, du[4] = {0.f, 0.f, 0.f, 0.f};
      float e[4] = {0.f, 0.f, 0.f, 0.f};
      if (role != 0 && s > 0) {  // band part against the previous output block
        const int kb = FWD ? ksE0 : 0;
        for (int j = 0; j < n2; ++j) mma_kstep(dh, dt, du, T + (20 + 4 * j + mi) * 128, yprev, P, kb + j, ni, lane);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          e[v] = dh[v] + (dt[v] + du[v]);
          dh[v] = dt[v] = du[v] = 0.f;
        }
      }
      if (role == 1) {
        *reinterpret_cast<float4*>(xch + (ot * 32 + lane) * 4) = make_float4(e[0], e[1], e[2], e[3]);
        named_sync(1 + ot, 64);
        continue;
      }
      // triangular part: FWD lower (k-steps 0 .. 2 mi + 1), BWD upper (2 mi .. 7)
      const int k0 = FWD ? 0 : 2 * mi, k1 = FWD ? 2 * mi + 2 : 8;
      for (int ks = k0; ks < k1; ++ks) {
        // fragment index: FWD pairs (ks, mi >= ks / 2) after sum_{s < ks} (4 - s / 2);
        // BWD pairs (ks, mi <= ks / 2) after sum_{s < ks} (s / 2 + 1)
        const int h = ks >> 1;
        const int pre = FWD ? 4 * ks - (h * (h - 1) + (ks & 1) * h) : (h * (h + 1) + (ks & 1) * (h + 1));
        const int pair = FWD ? pre + mi - h : pre + mi;
        mma_kstep(dh, dt, du, T + pair * 128, fcur, P, ks, ni, lane);
      }
      if (role == 0) {
        named_sync(1 + ot, 64);
        const float4 ev = *reinterpret_cast<const float4*>(xch + (ot * 32 + lane) * 4);
        e[0] = ev.x;
        e[1] = ev.y;
        e[2] = ev.z;
        e[3] = ev.w;
      }
      const int cc = 4 * ni + t;  // complex column of this lane's outputs
#pragma unroll
      for (int hf = 0; hf < 2; ++hf) {
        const int r = 16 * mi + g + 8 * hf, row = 64 * i + r;
        float2 y = make_float2((dh[2 * hf] + (dt[2 * hf] + du[2 * hf])) - e[2 * hf],
                               (dh[2 * hf + 1] + (dt[2 * hf + 1] + du[2 * hf + 1])) - e[2 * hf + 1]);
        if (row >= N4) y = make_float2(0.f, 0.f);
        *reinterpret_cast<float2*>(ycur + r * P + 8 * ni + 2 * t) = y;
        if (cc < W && row < N4 && sm.act[cc]) out[(size_t)row * W + cc] = y;
      }
    }
    if (tid == 0 && s + 1 == nblk) sm.tile_base = base + (unsigned)nblk;  // every thread read it at entry
    __syncthreads();
  };
  for (int s0 = 0; s0 < nblk; s0 += DEPTH) {
#pragma unroll
    for (int j = 0; j < DEPTH; ++j)
      if (s0 + j < nblk) step(s0 + j, pq[(j + 1) % DEPTH]);
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

// ------------------------------------------------------------ the sequential chain, FP64
// FWD: y_0 = t_0, y_i = t_i - E_i y_{i-1} (k over the last bw rows of y_{i-1});
// BWD: x_last = u_last, x_i = u_i - F_i x_{i+1} (k over the first bw rows).
// Thread = (row, column chunk, slice of k); partial sums meet in shared
// memory; the tiles are read through L2 (the FP64 solve is bound by the FP64
// FMA rate).  tin and yout may alias (each element is read, a step ahead,
// before it is written, by the same thread).  Ends with a barrier.
template <int CWV, int PF, bool FWD>
__device__ __noinline__ void bc_chain64(const Args& a, Smem& sm, const double* __restrict__ Mall, const double2* tin,
                                        double2* yout) {
  using C = double2;
  const int W = a.W, N4 = 4 * a.m.nb, nblk = a.m.bf_nblk, bw = a.m.bf_bw, tid = threadIdx.x;
  const DynLayout L = dyn_layout(true, W, true, 0);
  extern __shared__ __align__(16) char bc_dyn[];
  C* red = reinterpret_cast<C*>(bc_dyn + L.o_red);
  C* ysm = reinterpret_cast<C*>(bc_dyn + L.o_ysm);
  const int kbase = FWD ? 64 - bw : 0;
  const int nsteps = nblk - 1;
  auto blk_of = [&](int s) { return FWD ? s : nblk - 1 - s; };  // s = 0: the chain's first block
  {  // first block of the chain
    const int i0 = blk_of(0);
    for (int o = tid; o < 64 * W; o += TPB) {
      const int r = o / W, c = o - r * W, row = 64 * i0 + r;
      const C v = row < N4 ? tin[(size_t)64 * i0 * W + o] : czero<C>();
      ysm[o] = v;
      if (row < N4 && sm.act[c]) yout[(size_t)64 * i0 * W + o] = v;
    }
    __syncthreads();
  }
  const int r0 = tid % 64, g = tid / 64;
  const int nks = L.nks, nchunk = L.nchunk;
  const int len = (bw + nks - 1) / nks;
  C tnext[PF];  // this thread's t values (PF per block), a step ahead of use
  auto load_t = [&](int s) {
    const int i = blk_of(s);
#pragma unroll
    for (int m = 0; m < PF; ++m) {
      const int o = tid + m * TPB;
      const int row = 64 * i + o / W;
      tnext[m] = (s <= nsteps && o < 64 * W && row < N4) ? tin[(size_t)64 * i * W + o] : czero<C>();
    }
  };
  load_t(1);
  for (int s = 1; s <= nsteps; ++s) {
    const int i = blk_of(s);
    C tcur[PF];
#pragma unroll
    for (int m = 0; m < PF; ++m) tcur[m] = tnext[m];
    load_t(s + 1);
    const double* __restrict__ Mt = Mall + (size_t)i * 4096;
    // partial products over this thread's slice of k
    for (int ch = (nks == 1 ? g : g / nks); ch < nchunk; ch += (nks == 1 ? L.G : nchunk)) {
      const int ks = nks == 1 ? 0 : g % nks, c0 = ch * CWV;
      const int kb = kbase + ks * len, ke = min(kb + len, kbase + bw);
      C acc[CWV];
#pragma unroll
      for (int j = 0; j < CWV; ++j) acc[j] = czero<C>();
#pragma unroll 2
      for (int k = kb; k < ke; ++k) {
        const double mv = __ldg(Mt + k * 64 + r0);
#pragma unroll
        for (int j = 0; j < CWV; ++j) cfma(acc[j], mv, ysm[k * W + c0 + j]);
      }
#pragma unroll
      for (int j = 0; j < CWV; ++j) red[((size_t)ks * 64 + r0) * (W + 1) + c0 + j] = acc[j];
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
    (void)t2;
    (void)part;
    bc_pass_mma<true, PF>(a, sm, f, t1);
    bc_pass_mma<false, PF>(a, sm, t1, x);
  } else {
    const double* bf = a.m.bf64;
    bc_tri_f64<true, CWV>(a, sm, bf, f, t1);
    __syncthreads();
    bc_chain64<CWV, PF, true>(a, sm, bf + 2 * part, t1, t1);
    bc_tri_f64<false, CWV>(a, sm, bf + part, t1, t2);
    __syncthreads();
    bc_chain64<CWV, PF, false>(a, sm, bf + 3 * part, t2, x);
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
