// Persistent team solver: shifted COCG in the S-bilinear form for a panel of
// W unit right-hand sides, all shifts at once, plus the Green's-function
// reductions.  One CTA is one team; teams pull panels from a device counter.
//
// Method (Introduction: generalized shifted linear equations (z S - H) x = b).
// With A = S^{-1} H the equations read (z I - A) x = S^{-1} b.  A is
// self-adjoint in the bilinear form <u, v> = u^T S v, so one COCG run for a
// seed shift sigma builds a Krylov space shared by every shift z_k (shift
// invariance) and the shifted residuals stay collinear, r^k_n = r_n / pi^k_n.
// Seed recurrence (rt = S r is carried instead of recomputed):
//   U = H p,  w = S^{-1} U                 (inner CG)
//   gamma = sigma (S p)^T p - p^T U,  alpha = rho / gamma
//   rt <- rt - alpha (sigma S p - U),  r <- r - alpha (sigma p - w)
//   beta = rho' / rho,  p <- r + beta p,  S p <- rt + beta S p
// Shift polynomials (delta_k = z_k - sigma, alpha_{-1} = 1, beta_{-1} = 0):
//   pi_{n+1} = (1 + alpha_n delta_k) pi_n + (alpha_n beta_{n-1}/alpha_{n-1}) (pi_n - pi_{n-1})
// Shift k has converged at n_k when ||rt_n|| / |pi^k_n| <= tol (= the true
// residual ||b - (z_k S - H) x^k|| for ||b|| = 1, since b - (zS-H)x = S r^k).
//
// Projected solutions without per-shift vector updates.  The shifted iterate
// x^k = sum_{n<n_k} alpha^k_n p^k_n, p^k_{n+1} = r_{n+1}/pi^k_{n+1} + beta^k_n p^k_n,
// alpha^k_n = (pi_n/pi_{n+1}) alpha_n, beta^k_n = (pi_n/pi_{n+1})^2 beta_n, is
// rewritten as x^k = sum_m c^k_m r_m with c^k_m = S^k_m / pi^k_m and the
// backward recurrence S^k_m = alpha^k_m + beta^k_m S^k_{m+1}, S^k_{n_k} = 0.
// Every output is a linear functional of x^k restricted to the rows R_j of the
// pattern, so the loop only records r_m[R_j] and the seed scalars; the final
// phase replays the pi recurrence from checkpoints and contracts.  This costs
// O(K) FP64 scalar work per iteration instead of O(K |R_j|) vector work.
#pragma once
#include "kernels.cuh"

namespace gbk {

constexpr int CK = 64;                      // checkpoint interval of the pi recurrence
// The seed vectors are rescaled by an exact power of two whenever ||rt|| drops
// below 2^-8, so that every vector of the mixed path (including the FP32
// inner-solve right-hand sides, ~1e-7 of ||U||) stays far above FP32 underflow.
constexpr double kRescaleBelow2 = 0x1p-16;  // rescale when ||rt||^2 < 2^-16
constexpr int kRescaleExp = 8;              // ... by 2^8 (exact)

struct Args {
  DevMat m;
  int K, W, KG, nrhs, npanels, maxit, inner_maxit, has_rho, has_edm, want_g;
  double tol, itol;
  double2 sigma;
  const double2* z;
  const double2* w_rho;
  const double2* w_edm;
  const int* rhs_cols;
  const long long* out_off;
  int* panel_counter;
  int* status;  // [nrhs] bit flags, see kSt*
  char* team_ws;
  size_t team_bytes;
  size_t o_r, o_rt, o_p, o_sp, o_u, o_w, o_g, o_d, o_q, o_x;
  size_t o_hr, o_ab, o_L, o_t, o_ck, o_pi, o_nk, o_res, o_buf, o_cp, o_cf, o_cg;
  int Mcap;
  int cg_smem;  // 1: the inner-CG vectors g, d, q live in dynamic shared memory
  // Chebyshev inner iteration of the mixed path (inner_cheb = 1): K steps per
  // FP32 level with d_{k+1} = A_k d_k + B_k M^-1 r_{k+1}, d_0 = c0 M^-1 r_0.
  int inner_cheb, cheb_K;
  int inner_bchol;  // 1: S x = f by the block-bidiagonal Cholesky factor (exact; block_chol.cuh)
  int bc_levels;    // mixed path: FP32 factor solves per application (refinement levels)
  int bc_bw_alloc;  // half-bandwidth the dynamic shared memory of the FP32 factor passes is sized for
  // Verification mode: team b solves panel b only and records r_m on every row
  // (history row = W columns x N4 rows, column-major) instead of the pattern
  // rows, for the true-residual check; only the coefficients (cgs), nk and
  // the iteration counts are produced.
  int full_hist;
  int hp_fp32;  // mixed path: H p as an unrefined FP32 product (flags bit 5)
  int stall;    // > 0: stop a column whose unconverged shifts all went this many
                // iterations without halving their best residual (flags bit 6)
  float cheb_c0;
  float cheb_A[48], cheb_B[48];
  double* ldos;
  double* rho;
  double* edm;
  double* q;
  double* e_loc;
  int* iters;
  int* inner_iters;
  int* col_status;
  unsigned char* conv;
  double* resid;
  double2* g_proj;
  long long P;
};

constexpr int kStBreakdown = 1;
constexpr int kStNotSPD = 2;
constexpr int kStNoConv = 4;
constexpr int kStInner = 8;
constexpr int kStTimeout = 16;  // a bounded wait for a staged factor tile gave up
constexpr int kStStall = 32;    // stopped early: no shift of the column was improving

struct Smem {
  RedSmem rs;
  int panel, Wp, flag, inner_count;
  int j[WMAX], mc[WMAX], off[WMAX + 1], act[WMAX], nc[WMAX], nact[WMAX], st[WMAX], nfresh[WMAX];
  double2 rho[WMAX], alpha[WMAX], beta[WMAX], aprev[WMAX], bprev[WMAX], gam[WMAX];
  double rt2[WMAX], scl[WMAX];
  double cg_rho[2 * WMAX], cg_un[2 * WMAX], cg_gg[2 * WMAX], cg_a[2 * WMAX], cg_b[2 * WMAX];
  unsigned long long bc_bar[3];  // mbarriers of the staged factor tiles (block_chol.cuh)
  unsigned tile_base;            // factor tiles consumed so far in this launch
  int bc_fail;                   // a bounded tile wait gave up
};

// Once per launch, before the team's first panel: the block-reduce scratch in
// dynamic shared memory and the tile barriers of the block Cholesky solve.
__device__ __forceinline__ void team_init(Smem& sm, char* dyn);

}  // namespace gbk

#include "block_chol.cuh"

namespace gbk {

__device__ __forceinline__ void team_init(Smem& sm, char* dyn) {
  (void)dyn;  // block_reduce finds its partials at the start of the dynamic shared memory
  if (threadIdx.x == 0) {
    for (int b = 0; b < kTileBufs; ++b) mbar_init(&sm.bc_bar[b], 1);
    fence_mbar_init();
    sm.tile_base = 0;
    sm.bc_fail = 0;
  }
  __syncthreads();
}

template <typename T>
__device__ __forceinline__ T* wsp(char* ws, size_t off) {
  return reinterpret_cast<T*>(ws + off);
}

// The same routine advances the pi recurrence in the loop and in the final
// replay, so both produce identical values.
__device__ __noinline__ double2 shift_coef(double2 a_n, double2 b_prev, double2 a_prev) {
  return cdiv(cmul(a_n, b_prev), a_prev);
}
__device__ __noinline__ double2 pi_step(double2 cur, double2 prev, double2 a_n, double2 coef, double2 delta) {
  double2 ad = cmul(a_n, delta);
  ad.x += 1.0;
  const double2 t = cmul(ad, cur);
  const double2 u = cmul(coef, csub(cur, prev));
  return cadd(t, u);
}

// ------------------------------------------------------------ inner CG, FP64
// Solves S x = f per real column (re, im parts separately), block-Jacobi
// preconditioned, zero initial guess, until ||g|| <= itol ||f|| for every
// active real column.
__device__ __noinline__ void cg64(const Args& a, Smem& sm, const double2* __restrict__ f, double2* __restrict__ x,
                     double2* __restrict__ g, double2* __restrict__ d, double2* __restrict__ q) {
  const int W = a.W, nb = a.m.nb, c = threadIdx.x % W;
  {
    double v[4] = {0, 0, 0, 0};
    for (int it = threadIdx.x; it < nb * W; it += TPB) {
      if (!sm.act[c]) continue;
      const int I = it / W;
      double2 gv[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) gv[r] = f[(size_t)(4 * I + r) * W + c];
      const double* Mi = a.m.minv + (size_t)I * 16;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        double2 zr = make_double2(0, 0);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          zr.x = fma(Mi[r * 4 + t], gv[t].x, zr.x);
          zr.y = fma(Mi[r * 4 + t], gv[t].y, zr.y);
        }
        const size_t e = (size_t)(4 * I + r) * W + c;
        g[e] = gv[r];
        d[e] = zr;
        x[e] = make_double2(0, 0);
        v[0] = fma(gv[r].x, zr.x, v[0]);
        v[1] = fma(gv[r].y, zr.y, v[1]);
        v[2] = fma(gv[r].x, gv[r].x, v[2]);
        v[3] = fma(gv[r].y, gv[r].y, v[3]);
      }
    }
    block_reduce<4>(v, W, sm.rs);
    if (threadIdx.x < 2 * W) {
      const int cc = threadIdx.x >> 1, p = threadIdx.x & 1;
      sm.cg_rho[threadIdx.x] = sm.rs.scal[p * WMAX + cc];
      sm.cg_un[threadIdx.x] = sm.rs.scal[(2 + p) * WMAX + cc];
      sm.cg_gg[threadIdx.x] = sm.cg_un[threadIdx.x];
    }
    __syncthreads();
  }
  const double it2 = a.itol * a.itol;
  for (int iter = 0;; ++iter) {
    // every thread evaluates the same test on the same shared scalars (the
    // preceding barrier published them), so no extra barrier is needed
    bool done = true;
    for (int k = 0; k < 2 * W; ++k)
      if (sm.act[k >> 1] && sm.cg_gg[k] > it2 * sm.cg_un[k]) done = false;
    if (!done && iter >= a.inner_maxit) {
      done = true;
      if (threadIdx.x < W && sm.act[threadIdx.x]) sm.st[threadIdx.x] |= kStInner;
    }
    if (done) break;
    if (threadIdx.x == 0) ++sm.inner_count;
    {  // q = S d, d^T q
      double v[2] = {0, 0};
#if GB_WARP_SPMM
      const int lane = threadIdx.x & 31;
      const bool act = sm.act[c] != 0;
      for (int I = threadIdx.x >> 5; I < nb; I += NWARP) {
        double2 acc[4];
        wbsr_row_d(a.m, a.m.sb, d, W, W, lane, I, act, acc);
        if (lane < W && act) {
#else
      for (int it = threadIdx.x; it < nb * W; it += TPB) {
        if (!sm.act[c]) continue;
        const int I = it / W;
        double2 acc[4];
        bsr_row_d(a.m, a.m.sb, d, W, c, I, acc);
        {
#endif
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const size_t e = (size_t)(4 * I + r) * W + c;
            const double2 dv = d[e];
            q[e] = acc[r];
            v[0] = fma(dv.x, acc[r].x, v[0]);
            v[1] = fma(dv.y, acc[r].y, v[1]);
          }
        }
      }
      block_reduce<2>(v, W, sm.rs);
      if (threadIdx.x < 2 * W) {
        const int cc = threadIdx.x >> 1, p = threadIdx.x & 1;
        const double dq = sm.rs.scal[p * WMAX + cc];
        double al = 0.0;
        if (dq > 0.0) al = sm.cg_rho[threadIdx.x] / dq;
        else if (dq < 0.0 && sm.act[cc]) sm.st[cc] |= kStNotSPD;
        sm.cg_a[threadIdx.x] = al;
      }
      __syncthreads();
    }
    {  // x += a d, g -= a q, z = M^-1 g (into q), g^T z, g^T g
      double v[4] = {0, 0, 0, 0};
      const double ar = sm.cg_a[2 * c], ai = sm.cg_a[2 * c + 1];
      for (int it = threadIdx.x; it < nb * W; it += TPB) {
        if (!sm.act[c]) continue;
        const int I = it / W;
        double2 gv[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const size_t e = (size_t)(4 * I + r) * W + c;
          const double2 dv = d[e], qv = q[e];
          double2 xv = x[e];
          xv.x = fma(ar, dv.x, xv.x);
          xv.y = fma(ai, dv.y, xv.y);
          x[e] = xv;
          double2 gg = g[e];
          gg.x = fma(-ar, qv.x, gg.x);
          gg.y = fma(-ai, qv.y, gg.y);
          g[e] = gg;
          gv[r] = gg;
        }
        const double* Mi = a.m.minv + (size_t)I * 16;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          double2 zr = make_double2(0, 0);
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            zr.x = fma(Mi[r * 4 + t], gv[t].x, zr.x);
            zr.y = fma(Mi[r * 4 + t], gv[t].y, zr.y);
          }
          q[(size_t)(4 * I + r) * W + c] = zr;
          v[0] = fma(gv[r].x, zr.x, v[0]);
          v[1] = fma(gv[r].y, zr.y, v[1]);
          v[2] = fma(gv[r].x, gv[r].x, v[2]);
          v[3] = fma(gv[r].y, gv[r].y, v[3]);
        }
      }
      block_reduce<4>(v, W, sm.rs);
      if (threadIdx.x < 2 * W) {
        const int cc = threadIdx.x >> 1, p = threadIdx.x & 1;
        const double rn = sm.rs.scal[p * WMAX + cc];
        const double ro = sm.cg_rho[threadIdx.x];
        sm.cg_b[threadIdx.x] = (ro != 0.0) ? rn / ro : 0.0;
        sm.cg_rho[threadIdx.x] = rn;
        sm.cg_gg[threadIdx.x] = sm.rs.scal[(2 + p) * WMAX + cc];
      }
      __syncthreads();
    }
    // d = z + b d
    const double br = sm.cg_b[2 * c], bi = sm.cg_b[2 * c + 1];
    for (int e = threadIdx.x; e < 4 * nb * W; e += TPB) {
      if (!sm.act[c]) continue;
      const double2 zv = q[e];
      double2 dv = d[e];
      dv.x = fma(br, dv.x, zv.x);
      dv.y = fma(bi, dv.y, zv.y);
      d[e] = dv;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ inner CG, FP32 loop
// Runs on (x, g, d) already initialised (x = 0, g = rhs, d = M^-1 g) with
// cg_rho / cg_un / cg_gg set.  FP32 vectors, FP64 scalars.
__device__ __noinline__ void cg32_loop(const Args& a, Smem& sm, float2* __restrict__ x, float2* __restrict__ g,
                          float2* __restrict__ d, float2* __restrict__ q, double itol) {
  const int W = a.W, nb = a.m.nb, c = threadIdx.x % W;
  const double it2 = itol * itol;
  for (int iter = 0;; ++iter) {
    // every thread evaluates the same test on the same shared scalars (the
    // preceding barrier published them), so no extra barrier is needed
    bool done = true;
    for (int k = 0; k < 2 * W; ++k)
      if (sm.act[k >> 1] && sm.cg_gg[k] > it2 * sm.cg_un[k]) done = false;
    if (!done && iter >= a.inner_maxit) {
      done = true;
      if (threadIdx.x < W && sm.act[threadIdx.x]) sm.st[threadIdx.x] |= kStInner;
    }
    if (done) break;
    if (threadIdx.x == 0) ++sm.inner_count;
    {
      double v[2] = {0, 0};
      float v0 = 0.f, v1 = 0.f;
#if GB_WARP_SPMM
      const int lane = threadIdx.x & 31;
      const bool act = sm.act[c] != 0;
      for (int I = threadIdx.x >> 5; I < nb; I += NWARP) {
        float2 acc[4];
        wbsr_row_f(a.m, a.m.sb_hi, d, W, W, lane, I, act, acc);
        if (lane < W && act) {
#else
      for (int it = threadIdx.x; it < nb * W; it += TPB) {
        if (!sm.act[c]) continue;
        const int I = it / W;
        float2 acc[4];
        bsr_row_f(a.m, a.m.sb_hi, d, W, c, I, acc);
        {
#endif
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const size_t e = (size_t)(4 * I + r) * W + c;
            const float2 dv = d[e];
            q[e] = acc[r];
            v0 = fmaf(dv.x, acc[r].x, v0);
            v1 = fmaf(dv.y, acc[r].y, v1);
          }
        }
      }
      v[0] = v0;
      v[1] = v1;
      block_reduce<2>(v, W, sm.rs);
      if (threadIdx.x < 2 * W) {
        const int cc = threadIdx.x >> 1, p = threadIdx.x & 1;
        const double dq = sm.rs.scal[p * WMAX + cc];
        double al = 0.0;
        if (dq > 0.0) {
          al = sm.cg_rho[threadIdx.x] / dq;
        } else if (sm.act[cc] && sm.cg_gg[threadIdx.x] > 0.0) {
          // no curvature left in FP32 (d^T S d <= 0 with a nonzero residual):
          // this real column cannot progress; stop it and report it
          sm.st[cc] |= (dq < 0.0 ? kStNotSPD : 0) | kStInner;
          sm.cg_gg[threadIdx.x] = 0.0;
        }
        sm.cg_a[threadIdx.x] = al;
      }
      __syncthreads();
    }
    {
      float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f;
      const float ar = (float)sm.cg_a[2 * c], ai = (float)sm.cg_a[2 * c + 1];
      for (int it = threadIdx.x; it < nb * W; it += TPB) {
        if (!sm.act[c]) continue;
        const int I = it / W;
        float2 gv[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const size_t e = (size_t)(4 * I + r) * W + c;
          const float2 dv = d[e], qv = q[e];
          float2 xv = x[e];
          xv.x = fmaf(ar, dv.x, xv.x);
          xv.y = fmaf(ai, dv.y, xv.y);
          x[e] = xv;
          float2 gg = g[e];
          gg.x = fmaf(-ar, qv.x, gg.x);
          gg.y = fmaf(-ai, qv.y, gg.y);
          g[e] = gg;
          gv[r] = gg;
        }
        const float4* Mi = reinterpret_cast<const float4*>(a.m.minv32 + (size_t)I * 16);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const float4 mr = __ldg(Mi + r);
          float2 zr;
          zr.x = mr.x * gv[0].x + mr.y * gv[1].x + mr.z * gv[2].x + mr.w * gv[3].x;
          zr.y = mr.x * gv[0].y + mr.y * gv[1].y + mr.z * gv[2].y + mr.w * gv[3].y;
          q[(size_t)(4 * I + r) * W + c] = zr;
          f0 = fmaf(gv[r].x, zr.x, f0);
          f1 = fmaf(gv[r].y, zr.y, f1);
          f2 = fmaf(gv[r].x, gv[r].x, f2);
          f3 = fmaf(gv[r].y, gv[r].y, f3);
        }
      }
      double v[4] = {f0, f1, f2, f3};
      block_reduce<4>(v, W, sm.rs);
      if (threadIdx.x < 2 * W) {
        const int cc = threadIdx.x >> 1, p = threadIdx.x & 1;
        const double rn = sm.rs.scal[p * WMAX + cc];
        const double ro = sm.cg_rho[threadIdx.x];
        sm.cg_b[threadIdx.x] = (ro != 0.0) ? rn / ro : 0.0;
        sm.cg_rho[threadIdx.x] = rn;
        sm.cg_gg[threadIdx.x] = sm.rs.scal[(2 + p) * WMAX + cc];
      }
      __syncthreads();
    }
    const float br = (float)sm.cg_b[2 * c], bi = (float)sm.cg_b[2 * c + 1];
    for (int e = threadIdx.x; e < 4 * nb * W; e += TPB) {
      if (!sm.act[c]) continue;
      const float2 zv = q[e];
      float2 dv = d[e];
      dv.x = fmaf(br, dv.x, zv.x);
      dv.y = fmaf(bi, dv.y, zv.y);
      d[e] = dv;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ inner Chebyshev, FP32
// Chebyshev semi-iteration on the block-Jacobi-preconditioned S (spectrum
// bounds from gb_build_bsr) for x (= 0 on entry), r (= rhs), d_0 (= c0 M^-1 r)
// already set: K fused steps, one barrier each, no reductions.
__device__ __noinline__ void cheb32_loop(const Args& a, Smem& sm, float2* __restrict__ x, float2* __restrict__ r,
                            float2* __restrict__ dA, float2* __restrict__ dB) {
  const int W = a.W, nb = a.m.nb, c = threadIdx.x % W;
  // x = sum_k d_k is updated every other step with two directions (d_k from
  // memory, d_{k+1} still in registers), so x is read and written half as
  // often as r; the directions ping-pong between dA and dB.
  for (int k = 0; k < a.cheb_K; ++k) {
    const float Ak = a.cheb_A[k], Bk = a.cheb_B[k];
    const bool last = k + 1 == a.cheb_K, even = !(k & 1);
    const float2* __restrict__ dk = (k & 1) ? dB : dA;
    float2* __restrict__ dn = (k & 1) ? dA : dB;
    for (int it = threadIdx.x; it < nb * W; it += TPB) {
      if (!sm.act[c]) continue;
      const int I = it / W;
      float2 acc[4];
      bsr_row_f(a.m, a.m.sb_hi, dk, W, c, I, acc);
      float2 rv[4], dv[4];
#pragma unroll
      for (int rr = 0; rr < 4; ++rr) {
        const size_t e = (size_t)(4 * I + rr) * W + c;
        dv[rr] = dk[e];
        float2 g = r[e];
        g.x -= acc[rr].x;
        g.y -= acc[rr].y;
        r[e] = g;
        rv[rr] = g;
      }
      if (last) {  // d_K is not formed; d_{K-1} is still owed to x when K-1 is even
        if (even) {
#pragma unroll
          for (int rr = 0; rr < 4; ++rr) {
            const size_t e = (size_t)(4 * I + rr) * W + c;
            float2 xv = x[e];
            xv.x += dv[rr].x;
            xv.y += dv[rr].y;
            x[e] = xv;
          }
        }
        continue;
      }
      const float4* Mi = reinterpret_cast<const float4*>(a.m.minv32 + (size_t)I * 16);
#pragma unroll
      for (int rr = 0; rr < 4; ++rr) {
        const float4 mr = __ldg(Mi + rr);
        float2 zr;
        zr.x = mr.x * rv[0].x + mr.y * rv[1].x + mr.z * rv[2].x + mr.w * rv[3].x;
        zr.y = mr.x * rv[0].y + mr.y * rv[1].y + mr.z * rv[2].y + mr.w * rv[3].y;
        float2 nd;
        nd.x = fmaf(Ak, dv[rr].x, Bk * zr.x);
        nd.y = fmaf(Ak, dv[rr].y, Bk * zr.y);
        const size_t e = (size_t)(4 * I + rr) * W + c;
        dn[e] = nd;
        if (even) {
          float2 xv = x[e];
          xv.x += dv[rr].x + nd.x;
          xv.y += dv[rr].y + nd.y;
          x[e] = xv;
        }
      }
    }
    if (threadIdx.x == 0) ++sm.inner_count;
    __syncthreads();
  }
}

// Stores the per-real-column CG start scalars from a reduced {g^T z, ||f||^2}.
__device__ __forceinline__ void cg_start_scalars(Smem& sm, int W) {
  if (threadIdx.x < 2 * W) {
    const int cc = threadIdx.x >> 1, p = threadIdx.x & 1;
    sm.cg_rho[threadIdx.x] = sm.rs.scal[p * WMAX + cc];
    sm.cg_un[threadIdx.x] = sm.rs.scal[(2 + p) * WMAX + cc];
    sm.cg_gg[threadIdx.x] = sm.cg_un[threadIdx.x];
  }
  __syncthreads();
}

// ------------------------------------------------------------ inner solve, mixed
// w = S^{-1} U to ~FP64 accuracy: FP32 CG on hi(U), a float-float residual
// e = U - S x1, FP32 CG on e, w = x1 + x2 (float-float).
__device__ __noinline__ void inner_mixed_factor(const Args& a, Smem& sm, const float4* __restrict__ U, float4* __restrict__ w,
                                   float2* __restrict__ x, float2* __restrict__ g, float2* __restrict__ d,
                                   float2* __restrict__ q, char* dyn);

__device__ __noinline__ void inner_mixed(const Args& a, Smem& sm, const float4* __restrict__ U, float4* __restrict__ w,
                            float2* __restrict__ x, float2* __restrict__ g, float2* __restrict__ d,
                            float2* __restrict__ q, char* dyn) {
  if (a.inner_bchol) {
    inner_mixed_factor(a, sm, U, w, x, g, d, q, dyn);
    return;
  }
  const int W = a.W, nb = a.m.nb, c = threadIdx.x % W;
  const double itol = a.itol;
  {  // level 1 start: g = hi(U), d = M^-1 g, x = 0
    float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f;
    for (int it = threadIdx.x; it < nb * W; it += TPB) {
      if (!sm.act[c]) continue;
      const int I = it / W;
      float2 gv[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float4 u = U[(size_t)(4 * I + r) * W + c];
        gv[r] = make_float2(u.x, u.z);
      }
      const float4* Mi = reinterpret_cast<const float4*>(a.m.minv32 + (size_t)I * 16);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float4 mr = __ldg(Mi + r);
        float2 zr;
        zr.x = mr.x * gv[0].x + mr.y * gv[1].x + mr.z * gv[2].x + mr.w * gv[3].x;
        zr.y = mr.x * gv[0].y + mr.y * gv[1].y + mr.z * gv[2].y + mr.w * gv[3].y;
        const size_t e = (size_t)(4 * I + r) * W + c;
        g[e] = gv[r];
        d[e] = a.inner_cheb ? make_float2(a.cheb_c0 * zr.x, a.cheb_c0 * zr.y) : zr;
        x[e] = make_float2(0.f, 0.f);
        f0 = fmaf(gv[r].x, zr.x, f0);
        f1 = fmaf(gv[r].y, zr.y, f1);
        f2 = fmaf(gv[r].x, gv[r].x, f2);
        f3 = fmaf(gv[r].y, gv[r].y, f3);
      }
    }
    double v[4] = {f0, f1, f2, f3};
    block_reduce<4>(v, W, sm.rs);
    cg_start_scalars(sm, W);
  }
  if (a.inner_cheb)
    cheb32_loop(a, sm, x, g, d, q);
  else
    cg32_loop(a, sm, x, g, d, q, itol);
  {  // e = U - S x1 (float-float); w = x1; level 2 start: g = e, d = M^-1 e, x = 0
    float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f;
    // x1 is read by neighbouring block rows: write w first, then overwrite x after a barrier.
#if GB_WARP_SPMM
    const int lane = threadIdx.x & 31;
    const bool act = sm.act[c] != 0;
    for (int I = threadIdx.x >> 5; I < nb; I += NWARP) {
      gbff::acc are[4], aim[4];
      wbsr_row_ffx(a.m, a.m.sb_hi, a.m.sb_lo, x, W, W, lane, I, act, are, aim);
      if (lane >= W || !act) continue;
#else
    for (int it = threadIdx.x; it < nb * W; it += TPB) {
      if (!sm.act[c]) continue;
      const int I = it / W;
      gbff::acc are[4], aim[4];
      bsr_row_ffx(a.m, a.m.sb_hi, a.m.sb_lo, x, W, c, I, are, aim);
#endif
      float2 ev[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const size_t e = (size_t)(4 * I + r) * W + c;
        const float4 u = U[e];
        const gbff::ff er = gbff::ff_sub(gbff::ff{u.x, u.y}, gbff::acc_get(are[r]));
        const gbff::ff ei = gbff::ff_sub(gbff::ff{u.z, u.w}, gbff::acc_get(aim[r]));
        ev[r] = make_float2(er.hi + er.lo, ei.hi + ei.lo);
        g[e] = ev[r];
      }
      const float4* Mi = reinterpret_cast<const float4*>(a.m.minv32 + (size_t)I * 16);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float4 mr = __ldg(Mi + r);
        float2 zr;
        zr.x = mr.x * ev[0].x + mr.y * ev[1].x + mr.z * ev[2].x + mr.w * ev[3].x;
        zr.y = mr.x * ev[0].y + mr.y * ev[1].y + mr.z * ev[2].y + mr.w * ev[3].y;
        d[(size_t)(4 * I + r) * W + c] = a.inner_cheb ? make_float2(a.cheb_c0 * zr.x, a.cheb_c0 * zr.y) : zr;
        f0 = fmaf(ev[r].x, zr.x, f0);
        f1 = fmaf(ev[r].y, zr.y, f1);
        f2 = fmaf(ev[r].x, ev[r].x, f2);
        f3 = fmaf(ev[r].y, ev[r].y, f3);
      }
    }
    double v[4] = {f0, f1, f2, f3};
    block_reduce<4>(v, W, sm.rs);  // contains the barrier that ends all reads of x1
    for (int e = threadIdx.x; e < 4 * nb * W; e += TPB) {
      if (!sm.act[c]) continue;
      const float2 xv = x[e];
      w[e] = make_float4(xv.x, 0.f, xv.y, 0.f);
      x[e] = make_float2(0.f, 0.f);
    }
    cg_start_scalars(sm, W);  // its barrier orders the x / w writes too
  }
  if (a.inner_cheb)
    cheb32_loop(a, sm, x, g, d, q);
  else
    cg32_loop(a, sm, x, g, d, q, itol);
  for (int e = threadIdx.x; e < 4 * nb * W; e += TPB) {
    if (!sm.act[c]) continue;
    const float4 wv = w[e];
    const float2 xv = x[e];
    const gbff::ff re = gbff::ff_add(gbff::ff{wv.x, wv.y}, gbff::ff{xv.x, 0.f});
    const gbff::ff im = gbff::ff_add(gbff::ff{wv.z, wv.w}, gbff::ff{xv.y, 0.f});
    w[e] = make_float4(re.hi, re.lo, im.hi, im.lo);
  }
  __syncthreads();
}

// ------------------------------------------------------------ inner solve, mixed, exact factor
// w = S^{-1} U to ~FP64 accuracy by refinement with FP32 factor solves:
// x1 = S^-1 hi(U), w = x1; then per further level the float-float residual
// e = U - S w and w += S^-1 e.  One FP32 solve is accurate to ~4e-7, so two
// levels give ~1e-13 and three ~1e-19 (a.bc_levels, set from the tolerance).
// g = U - S v (float-float) for the active columns; v is the FP32 vector x
// (XV = float2) or the float-float w (XV = float4).  No barrier.
template <typename XV>
__device__ __noinline__ void ff_residual(const Args& a, const Smem& sm, const float4* __restrict__ U,
                                         const XV* __restrict__ v, float2* __restrict__ g) {
  const int W = a.W, nb = a.m.nb, c = threadIdx.x % W;
  for (int it = threadIdx.x; it < nb * W; it += TPB) {
    if (!sm.act[c]) continue;
    const int I = it / W;
    gbff::acc are[4], aim[4];
    if constexpr (sizeof(XV) == 8)
      bsr_row_ffx(a.m, a.m.sb_hi, a.m.sb_lo, v, W, c, I, are, aim);
    else
      bsr_row_ff(a.m, a.m.sb_hi, a.m.sb_lo, v, W, c, I, are, aim);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const size_t e = (size_t)(4 * I + r) * W + c;
      const float4 u = U[e];
      const gbff::ff er = gbff::ff_sub(gbff::ff{u.x, u.y}, gbff::acc_get(are[r]));
      const gbff::ff ei = gbff::ff_sub(gbff::ff{u.z, u.w}, gbff::acc_get(aim[r]));
      g[e] = make_float2(er.hi + er.lo, ei.hi + ei.lo);
    }
  }
}

__device__ __noinline__ void inner_mixed_factor(const Args& a, Smem& sm, const float4* __restrict__ U, float4* __restrict__ w,
                                   float2* __restrict__ x, float2* __restrict__ g, float2* __restrict__ d,
                                   float2* __restrict__ q, char* dyn) {
  const int W = a.W, nb = a.m.nb, c = threadIdx.x % W;
  bc_solve<float>(a, sm, U, x, d, q, dyn);
  for (int lev = 1; lev < a.bc_levels; ++lev) {
    // e = U - S w into g; at the first refinement w = x1 is the FP32 vector x
    if (lev == 1)
      ff_residual(a, sm, U, x, g);
    else
      ff_residual(a, sm, U, w, g);
    __syncthreads();  // every read of x / w for the residual is done
    if (lev == 1) {
      for (int e = threadIdx.x; e < 4 * nb * W; e += TPB) {
        if (!sm.act[c]) continue;
        const float2 xv = x[e];
        w[e] = make_float4(xv.x, 0.f, xv.y, 0.f);
      }
      __syncthreads();
    }
    bc_solve<float>(a, sm, g, x, d, q, dyn);
    for (int e = threadIdx.x; e < 4 * nb * W; e += TPB) {
      if (!sm.act[c]) continue;
      const float4 wv = w[e];
      const float2 xv = x[e];
      const gbff::ff re = gbff::ff_add(gbff::ff{wv.x, wv.y}, gbff::ff{xv.x, 0.f});
      const gbff::ff im = gbff::ff_add(gbff::ff{wv.z, wv.w}, gbff::ff{xv.y, 0.f});
      w[e] = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
    __syncthreads();
  }
  if (a.bc_levels == 1) {
    for (int e = threadIdx.x; e < 4 * nb * W; e += TPB) {
      if (!sm.act[c]) continue;
      const float2 xv = x[e];
      w[e] = make_float4(xv.x, 0.f, xv.y, 0.f);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ inner solve, FP64
// w = S^{-1} f: the exact factor solve where the factor exists, else CG.
__device__ __noinline__ void inner64(const Args& a, Smem& sm, const double2* __restrict__ f, double2* __restrict__ x,
                        double2* __restrict__ g, double2* __restrict__ d, double2* __restrict__ q, char* dyn) {
  if (a.inner_bchol)
    bc_solve<double>(a, sm, f, x, d, q, dyn);
  else
    cg64(a, sm, f, x, g, d, q);
}

}  // namespace gbk
