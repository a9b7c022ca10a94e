// Panel driver of the team solver: seed COCG loop, shift polynomials,
// history, and the final Green's-function reductions (see team_solver.cuh).
#pragma once
#include <type_traits>

#include "team_solver.cuh"

namespace gbk {

// ------------------------------------------------------------ element helpers
template <bool MIX>
using SeedT = typename std::conditional<MIX, float4, double2>::type;

__device__ __forceinline__ double2 to_d2(double2 v) { return v; }
__device__ __forceinline__ double2 to_d2(float4 v) {
  return make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
}
template <bool MIX>
__device__ __forceinline__ SeedT<MIX> seed_unit(double v);
template <>
__device__ __forceinline__ double2 seed_unit<false>(double v) { return make_double2(v, 0.0); }
template <>
__device__ __forceinline__ float4 seed_unit<true>(double v) { return make_float4((float)v, 0.f, 0.f, 0.f); }

__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// r_m[R_j] for every column of the panel -> one history row (FP64).
template <bool MIX>
__device__ void gather_hist(const Args& a, const Smem& sm, const SeedT<MIX>* r, double2* row) {
  if (a.full_hist) {  // every row of every column: row[cc * N4 + i]
    const int N4 = 4 * a.m.nb, W = a.W;
    for (int e = threadIdx.x; e < N4 * W; e += TPB) {
      const int cc = e / N4, i = e - cc * N4;
      row[e] = to_d2(r[(size_t)i * W + cc]);
    }
    return;
  }
  const int M = sm.off[a.W];
  for (int e = threadIdx.x; e < M; e += TPB) {
    int cc = 0;
    while (sm.off[cc + 1] <= e) ++cc;
    const int t = e - sm.off[cc];
    const int i = a.m.col_idx[a.m.row_ptr[sm.j[cc]] + t];
    row[e] = to_d2(r[(size_t)i * a.W + cc]);
  }
}

struct PanelSmemExtra {
  int Mt[WMAX * 8];  // replay length per (column, 32-shift group)
  int Mc[WMAX];
  double rt2s[WMAX];  // last ||rt||^2 in the stored (scaled) units
  double2 coef[WMAX];
};

template <bool MIX>
__device__ void solve_panel(const Args& a, Smem& sm, PanelSmemExtra& sx, char* ws, char* dyn) {
  using V = SeedT<MIX>;
  const int W = a.W, K = a.K, nb = a.m.nb, tid = threadIdx.x, c = tid % W;
  const size_t NE = (size_t)4 * nb * W;
  V* r = wsp<V>(ws, a.o_r);
  V* rt = wsp<V>(ws, a.o_rt);
  V* p = wsp<V>(ws, a.o_p);
  V* sp = wsp<V>(ws, a.o_sp);
  V* U = wsp<V>(ws, a.o_u);
  V* w = wsp<V>(ws, a.o_w);
  double2* hr = wsp<double2>(ws, a.o_hr);
  double2* hab = wsp<double2>(ws, a.o_ab);
  int* hL = wsp<int>(ws, a.o_L);
  double2* ht = wsp<double2>(ws, a.o_t);
  double2* ck = wsp<double2>(ws, a.o_ck);
  double2* pis = wsp<double2>(ws, a.o_pi);
  int* nk = wsp<int>(ws, a.o_nk);
  double* resk = wsp<double>(ws, a.o_res);
  double2* buf = wsp<double2>(ws, a.o_buf);
  double2* cp = wsp<double2>(ws, a.o_cp);
  double2* cf = wsp<double2>(ws, a.o_cf);
  double2* cgs = a.want_g ? wsp<double2>(ws, a.o_cg) : nullptr;
  const double2 sigma = a.sigma;
  const int WK = W * K;
  // inner-CG vectors: shared memory when the panel fits (g, d, q), else global
  using CgT = typename std::conditional<MIX, float2, double2>::type;
  CgT* cg_x = wsp<CgT>(ws, a.o_x);
  CgT* cg_g = a.cg_smem ? reinterpret_cast<CgT*>(dyn + dyn_layout(!MIX, W, false, 0).o_cg) : wsp<CgT>(ws, a.o_g);
  CgT* cg_d = a.cg_smem ? cg_g + NE : wsp<CgT>(ws, a.o_d);
  CgT* cg_q = a.cg_smem ? cg_d + NE : wsp<CgT>(ws, a.o_q);

  // ---------------------------------------------------------------- set-up
  if (tid < WMAX) {
    const int col = sm.panel * W + tid;
    const bool ok = tid < W && col < a.nrhs;
    const int j = ok ? a.rhs_cols[col] : 0;
    sm.j[tid] = j;
    sm.act[tid] = ok ? 1 : 0;
    sm.mc[tid] = ok ? a.m.row_ptr[j + 1] - a.m.row_ptr[j] : 0;
    sm.nc[tid] = 0;
    sm.st[tid] = 0;
    sm.nact[tid] = 0;
    sm.nfresh[tid] = 0;
    sm.aprev[tid] = make_double2(1.0, 0.0);
    sm.bprev[tid] = make_double2(0.0, 0.0);
    sm.scl[tid] = 1.0;
    sx.rt2s[tid] = 1.0;
  }
  __syncthreads();
  if (tid == 0) {
    sm.off[0] = 0;
    int wp = 0;
    for (int i = 0; i < W; ++i) {
      sm.off[i + 1] = sm.off[i] + sm.mc[i];
      wp += sm.act[i];
    }
    sm.Wp = wp;
    sm.inner_count = 0;
  }
  for (int e = tid; e < WK; e += TPB) {
    const int cc = e / K;
    nk[e] = sm.act[cc] ? -1 : 0;
    resk[e] = 0.0;
    pis[2 * e] = make_double2(1.0, 0.0);
    pis[2 * e + 1] = make_double2(1.0, 0.0);
    ck[2 * e] = make_double2(1.0, 0.0);
    ck[2 * e + 1] = make_double2(1.0, 0.0);
  }
  if (tid < W) hL[tid] = 0;
  for (size_t e = tid; e < NE; e += TPB) {
    const int row = (int)(e / W);
    rt[e] = seed_unit<MIX>((sm.act[c] && row == sm.j[c]) ? 1.0 : 0.0);
  }
  __syncthreads();

  // r_0 = S^{-1} b
  if constexpr (MIX) {
    inner_mixed(a, sm, rt, r, cg_x, cg_g, cg_d, cg_q, dyn);
  } else {
    inner64(a, sm, rt, r, cg_g, cg_d, cg_q, dyn);
  }
  {  // p = r, Sp = rt, rho_0 = r^T rt
    double v[2] = {0, 0};
    gbff::acc ar, ai;
    gbff::acc_init(ar);
    gbff::acc_init(ai);
    for (size_t e = tid; e < NE; e += TPB) {
      if (!sm.act[c]) continue;
      const V rv = r[e], tv = rt[e];
      p[e] = rv;
      sp[e] = tv;
      if constexpr (MIX) {
        gbff::acc_mul_add(ar, gbff::ff{rv.x, rv.y}, gbff::ff{tv.x, tv.y});
        gbff::acc_mul_add(ar, gbff::ff{-rv.z, -rv.w}, gbff::ff{tv.z, tv.w});
        gbff::acc_mul_add(ai, gbff::ff{rv.x, rv.y}, gbff::ff{tv.z, tv.w});
        gbff::acc_mul_add(ai, gbff::ff{rv.z, rv.w}, gbff::ff{tv.x, tv.y});
      } else {
        v[0] = fma(rv.x, tv.x, fma(-rv.y, tv.y, v[0]));
        v[1] = fma(rv.x, tv.y, fma(rv.y, tv.x, v[1]));
      }
    }
    if constexpr (MIX) {
      v[0] = gbff::acc_to_double(ar);
      v[1] = gbff::acc_to_double(ai);
    }
    block_reduce<2>(v, W, sm.rs);
    if (tid < W) sm.rho[tid] = make_double2(sm.rs.scal[tid], sm.rs.scal[WMAX + tid]);
    gather_hist<MIX>(a, sm, r, hr);
    __syncthreads();
  }

  // ---------------------------------------------------------------- seed loop
  const double tol2 = a.tol * a.tol;
  int n = 0;
  for (; n < a.maxit; ++n) {
    if (tid == 0) {
      int any = 0;
      for (int i = 0; i < W; ++i) any |= sm.act[i];
      sm.flag = any;
    }
    __syncthreads();
    if (!sm.flag) break;

    {  // U = H p ; (S p)^T p and p^T U
      double v[4] = {0, 0, 0, 0};
      gbff::acc d0, d1, d2, d3;
      gbff::acc_init(d0);
      gbff::acc_init(d1);
      gbff::acc_init(d2);
      gbff::acc_init(d3);
#if GB_WARP_SPMM
      const int lane = tid & 31;
      const bool act = sm.act[c] != 0;
      for (int I = tid >> 5; I < nb; I += NWARP) {
#else
      for (int it = tid; it < nb * W; it += TPB) {
        if (!sm.act[c]) continue;
        const int I = it / W;
#endif
        if constexpr (MIX) {
          gbff::acc are[4], aim[4];
#if GB_WARP_SPMM
          wbsr_row_ff(a.m, a.m.hb_hi, a.m.hb_lo, p, W, W, lane, I, act, are, aim);
          if (lane >= W || !act) continue;
#else
          if (a.hp_fp32) {  // unrefined FP32 product: U = H hi(p), accumulated in FP32
            float2 acc[4];
            bsr_row_fhi(a.m, a.m.hb_hi, p, W, c, I, acc);
#pragma unroll
            for (int rr = 0; rr < 4; ++rr) {
              are[rr] = gbff::acc{acc[rr].x, 0.f};
              aim[rr] = gbff::acc{acc[rr].y, 0.f};
            }
          } else {
            bsr_row_ff(a.m, a.m.hb_hi, a.m.hb_lo, p, W, c, I, are, aim);
          }
#endif
#pragma unroll
          for (int rr = 0; rr < 4; ++rr) {
            const size_t e = (size_t)(4 * I + rr) * W + c;
            const gbff::ff ur = gbff::acc_get(are[rr]), ui = gbff::acc_get(aim[rr]);
            U[e] = make_float4(ur.hi, ur.lo, ui.hi, ui.lo);
            const float4 pv = p[e], sv = sp[e];
            const gbff::ff pr{pv.x, pv.y}, pim{pv.z, pv.w}, sr{sv.x, sv.y}, si{sv.z, sv.w};
            gbff::acc_mul_add(d0, sr, pr);
            gbff::acc_mul_add(d0, gbff::ff_neg(si), pim);
            gbff::acc_mul_add(d1, sr, pim);
            gbff::acc_mul_add(d1, si, pr);
            gbff::acc_mul_add(d2, pr, ur);
            gbff::acc_mul_add(d2, gbff::ff_neg(pim), ui);
            gbff::acc_mul_add(d3, pr, ui);
            gbff::acc_mul_add(d3, pim, ur);
          }
        } else {
          double2 acc[4];
#if GB_WARP_SPMM
          wbsr_row_d(a.m, a.m.hb, p, W, W, lane, I, act, acc);
          if (lane >= W || !act) continue;
#else
          bsr_row_d(a.m, a.m.hb, p, W, c, I, acc);
#endif
#pragma unroll
          for (int rr = 0; rr < 4; ++rr) {
            const size_t e = (size_t)(4 * I + rr) * W + c;
            U[e] = acc[rr];
            const double2 pv = p[e], sv = sp[e];
            v[0] = fma(sv.x, pv.x, fma(-sv.y, pv.y, v[0]));
            v[1] = fma(sv.x, pv.y, fma(sv.y, pv.x, v[1]));
            v[2] = fma(pv.x, acc[rr].x, fma(-pv.y, acc[rr].y, v[2]));
            v[3] = fma(pv.x, acc[rr].y, fma(pv.y, acc[rr].x, v[3]));
          }
        }
      }
      if constexpr (MIX) {
        v[0] = gbff::acc_to_double(d0);
        v[1] = gbff::acc_to_double(d1);
        v[2] = gbff::acc_to_double(d2);
        v[3] = gbff::acc_to_double(d3);
      }
      block_reduce<4>(v, W, sm.rs);
      if (tid < W) {
        const double2 spp = make_double2(sm.rs.scal[tid], sm.rs.scal[WMAX + tid]);
        const double2 pu = make_double2(sm.rs.scal[2 * WMAX + tid], sm.rs.scal[3 * WMAX + tid]);
        sm.gam[tid] = csub(cmul(sigma, spp), pu);
      }
      __syncthreads();
    }

    // w = S^{-1} U
    if constexpr (MIX) {
      inner_mixed(a, sm, U, w, cg_x, cg_g, cg_d, cg_q, dyn);
    } else {
      inner64(a, sm, U, w, cg_g, cg_d, cg_q, dyn);
    }

    if (tid < W && sm.act[tid]) {
      const double2 g = sm.gam[tid], rh = sm.rho[tid];
      const double2 al = cdiv(rh, g);
      if (cabs2(g) == 0.0 || cabs2(rh) == 0.0 || !cfinite(al)) {
        sm.st[tid] |= kStBreakdown;
        sm.act[tid] = 0;
        sm.nc[tid] = n;
      } else {
        sm.alpha[tid] = al;
      }
    }
    __syncthreads();

    {  // rt -= alpha (sigma Sp - U), r -= alpha (sigma p - w); rho' = r^T rt, ||rt||^2
      double v[3] = {0, 0, 0};
      gbff::acc d0, d1, d2;
      gbff::acc_init(d0);
      gbff::acc_init(d1);
      gbff::acc_init(d2);
      gbff::cff sg{}, al{};
      if constexpr (MIX) {
        sg = gbff::cff_from(sigma);
        al = gbff::cff_from(sm.alpha[c]);
      }
      const double2 ald = sm.alpha[c];
      for (size_t e = tid; e < NE; e += TPB) {
        if (!sm.act[c]) continue;
        if constexpr (MIX) {
          const gbff::cff spv = gbff::cff_load(sp[e]), uv = gbff::cff_load(U[e]);
          const gbff::cff pv = gbff::cff_load(p[e]), wv = gbff::cff_load(w[e]);
          gbff::cff tv = gbff::cff_load(rt[e]), rv = gbff::cff_load(r[e]);
          tv = gbff::cff_sub(tv, gbff::cff_mul(al, gbff::cff_sub(gbff::cff_mul(sg, spv), uv)));
          rv = gbff::cff_sub(rv, gbff::cff_mul(al, gbff::cff_sub(gbff::cff_mul(sg, pv), wv)));
          rt[e] = gbff::cff_store(tv);
          r[e] = gbff::cff_store(rv);
          gbff::acc_mul_add(d0, rv.re, tv.re);
          gbff::acc_mul_add(d0, gbff::ff_neg(rv.im), tv.im);
          gbff::acc_mul_add(d1, rv.re, tv.im);
          gbff::acc_mul_add(d1, rv.im, tv.re);
          gbff::acc_mul_add(d2, tv.re, tv.re);
          gbff::acc_mul_add(d2, tv.im, tv.im);
        } else {
          const double2 t1 = csub(cmul(sigma, sp[e]), U[e]);
          const double2 t2 = csub(cmul(sigma, p[e]), w[e]);
          const double2 tv = csub(rt[e], cmul(ald, t1));
          const double2 rv = csub(r[e], cmul(ald, t2));
          rt[e] = tv;
          r[e] = rv;
          v[0] = fma(rv.x, tv.x, fma(-rv.y, tv.y, v[0]));
          v[1] = fma(rv.x, tv.y, fma(rv.y, tv.x, v[1]));
          v[2] = fma(tv.x, tv.x, fma(tv.y, tv.y, v[2]));
        }
      }
      if constexpr (MIX) {
        v[0] = gbff::acc_to_double(d0);
        v[1] = gbff::acc_to_double(d1);
        v[2] = gbff::acc_to_double(d2);
      }
      block_reduce<3>(v, W, sm.rs);
      if (tid < W && sm.act[tid]) {
        const double2 rn = make_double2(sm.rs.scal[tid], sm.rs.scal[WMAX + tid]);
        const double rt2 = sm.rs.scal[2 * WMAX + tid];
        const double2 be = cdiv(rn, sm.rho[tid]);
        if (!cfinite(be) || !isfinite(rt2)) {
          sm.st[tid] |= kStBreakdown;
          sm.act[tid] = 0;
          sm.nc[tid] = n;
        } else {
          const double s = (rt2 < kRescaleBelow2 && rt2 > 0.0) ? scalbn(1.0, kRescaleExp) : 1.0;
          sm.scl[tid] = s;
          sm.beta[tid] = be;
          sm.rt2[tid] = rt2;
          sx.rt2s[tid] = rt2 * s * s;
          sm.rho[tid] = cscale(rn, s * s);
          hab[((size_t)n * W + tid) * 2] = sm.alpha[tid];
          hab[((size_t)n * W + tid) * 2 + 1] = be;
          hL[(size_t)(n + 1) * W + tid] = hL[(size_t)n * W + tid] + (s != 1.0 ? kRescaleExp : 0);
          sx.coef[tid] = shift_coef(sm.alpha[tid], sm.bprev[tid], sm.aprev[tid]);
          sm.nact[tid] = 0;
          sm.nfresh[tid] = 0;
        }
      }
      __syncthreads();
    }

    // p <- s (r + beta p), Sp <- s (rt + beta Sp), r, rt <- s r, s rt
    {
      const double2 be = sm.beta[c];
      const double s = sm.scl[c];
      gbff::cff bf{};
      if constexpr (MIX) bf = gbff::cff_from(be);
      for (size_t e = tid; e < NE; e += TPB) {
        if (!sm.act[c]) continue;
        if constexpr (MIX) {
          gbff::cff rv = gbff::cff_load(r[e]), tv = gbff::cff_load(rt[e]);
          gbff::cff pv = gbff::cff_add(rv, gbff::cff_mul(bf, gbff::cff_load(p[e])));
          gbff::cff qv = gbff::cff_add(tv, gbff::cff_mul(bf, gbff::cff_load(sp[e])));
          if (s != 1.0) {
            const float fs = (float)s;
            rv = gbff::cff_scale_pow2(rv, fs);
            tv = gbff::cff_scale_pow2(tv, fs);
            pv = gbff::cff_scale_pow2(pv, fs);
            qv = gbff::cff_scale_pow2(qv, fs);
            r[e] = gbff::cff_store(rv);
            rt[e] = gbff::cff_store(tv);
          }
          p[e] = gbff::cff_store(pv);
          sp[e] = gbff::cff_store(qv);
        } else {
          double2 rv = r[e], tv = rt[e];
          double2 pv = cadd(rv, cmul(be, p[e]));
          double2 qv = cadd(tv, cmul(be, sp[e]));
          if (s != 1.0) {
            rv = cscale(rv, s);
            tv = cscale(tv, s);
            pv = cscale(pv, s);
            qv = cscale(qv, s);
            r[e] = rv;
            rt[e] = tv;
          }
          p[e] = pv;
          sp[e] = qv;
        }
      }
      // shift polynomials, convergence, checkpoints
      for (int e = tid; e < WK; e += TPB) {
        const int cc = e / K, k = e - cc * K;
        if (!sm.act[cc] || nk[e] >= 0) continue;
        double2 cur = pis[2 * e], prev = pis[2 * e + 1];
        const double2 delta = csub(a.z[k], sigma);
        double2 nxt = pi_step(cur, prev, sm.alpha[cc], sx.coef[cc], delta);
        const double ap2 = cabs2(nxt);
        if (sm.rt2[cc] <= tol2 * ap2) {
          nk[e] = n + 1;
          resk[e] = sqrt(sm.rt2[cc] / ap2);
        } else {
          atomicAdd(&sm.nact[cc], 1);
          if (a.stall > 0) {
            // while the pair is open, resk holds its best squared residual so
            // far and nk = -2 - (iteration of that best); both are rewritten
            // when the column ends
            const double r2 = sm.rt2[cc] / ap2, best = resk[e];
            if (nk[e] == -1 || r2 < 0.25 * best) {
              resk[e] = r2;
              nk[e] = -2 - n;
            }
            if (n - (-2 - nk[e]) < a.stall) atomicAdd(&sm.nfresh[cc], 1);
          }
        }
        const double s = sm.scl[cc];
        if (s != 1.0) {
          nxt = cscale(nxt, s);
          cur = cscale(cur, s);
        }
        pis[2 * e] = nxt;
        pis[2 * e + 1] = cur;
        if ((n + 1) % CK == 0) {
          const size_t ce = ((size_t)((n + 1) / CK) * WK + e) * 2;
          ck[ce] = nxt;
          ck[ce + 1] = cur;
        }
      }
      __syncthreads();
    }
    gather_hist<MIX>(a, sm, r, hr + (size_t)(n + 1) * a.Mcap);
    if (tid < W && sm.act[tid]) {
      sm.aprev[tid] = sm.alpha[tid];
      sm.bprev[tid] = sm.beta[tid];
      if (sm.nact[tid] == 0) {
        sm.act[tid] = 0;
        sm.nc[tid] = n + 1;
      } else if (a.stall > 0 && sm.nfresh[tid] == 0) {  // every open shift has stalled
        sm.act[tid] = 0;
        sm.nc[tid] = n + 1;
        sm.st[tid] |= kStNoConv | kStStall;
      }
    }
    __syncthreads();
  }
  if (tid < W && sm.act[tid]) {  // iteration cap reached
    sm.act[tid] = 0;
    sm.nc[tid] = n;
    sm.st[tid] |= kStNoConv;
  }
  __syncthreads();
  for (int e = tid; e < WK; e += TPB) {
    const int cc = e / K;
    if (sm.off[cc + 1] == sm.off[cc] && sm.mc[cc] == 0) continue;  // padding column
    if (nk[e] < 0) {
      nk[e] = sm.nc[cc];
      const double2 pv = pis[2 * e];
      resk[e] = sqrt(sx.rt2s[cc] / cabs2(pv));
    }
  }
  __syncthreads();

  // ---------------------------------------------------------------- final phase
  const int KG = a.KG;
  // F0: t_m = sum_{i in R_j} S_ji r_m[i]  (not in verification mode: no LDOS)
  if (!a.full_hist) {
    int nmax = 0;
    for (int i = 0; i < W; ++i) nmax = max(nmax, sm.nc[i]);
    for (int e = tid; e < (nmax + 1) * W; e += TPB) {
      const int m = e / W, cc = e - m * W;
      if (sm.mc[cc] == 0 || m > sm.nc[cc]) continue;
      const int base = a.m.row_ptr[sm.j[cc]];
      const double2* hrow = hr + (size_t)m * a.Mcap + sm.off[cc];
      double2 s = make_double2(0, 0);
      for (int t = 0; t < sm.mc[cc]; ++t) {
        const double sv = a.m.s_val[base + t];
        const double2 x = hrow[t];
        s.x = fma(sv, x.x, s.x);
        s.y = fma(sv, x.y, s.y);
      }
      ht[(size_t)m * W + cc] = s;
    }
    __syncthreads();
  }
  // F1: backward coefficient recurrence per (column, 32 shifts), replayed from checkpoints
  {
    const int lane = tid & 31, warp = tid >> 5;
    for (int task = warp; task < W * KG; task += NWARP) {
      const int cc = task / KG, kg = task - cc * KG;
      if (sm.mc[cc] == 0) {
        if (lane == 0) sx.Mt[task] = 0;
        continue;
      }
      const int k = kg * 32 + lane;
      const bool valid = k < K;
      const int e = cc * K + (valid ? k : 0);
      const int nkk = valid ? nk[e] : 0;
      int M = nkk;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) M = max(M, __shfl_xor_sync(0xffffffffu, M, o));
      if (lane == 0) sx.Mt[task] = M;
      const double2 delta = valid ? csub(a.z[k], sigma) : make_double2(0, 0);
      const double2 wr = (valid && a.has_rho) ? a.w_rho[k] : make_double2(0, 0);
      const double2 we = (valid && a.has_edm) ? a.w_edm[k] : make_double2(0, 0);
      double2 S = make_double2(0, 0), lacc = make_double2(0, 0);
      for (int s = (M - 1) / CK; M > 0 && s >= 0; --s) {
        const int m0 = s * CK, mend = min(m0 + CK, M);
        const int lim = min(mend, nkk);
        if (valid && m0 < nkk) {
          const size_t ce = ((size_t)s * WK + e) * 2;
          double2 cur = ck[ce], prev = ck[ce + 1];
          buf[e] = cur;
          for (int mm = m0; mm < lim; ++mm) {
            const double2 am = hab[((size_t)mm * W + cc) * 2];
            const double2 bpm = mm > 0 ? hab[((size_t)(mm - 1) * W + cc) * 2 + 1] : make_double2(0, 0);
            const double2 apm = mm > 0 ? hab[((size_t)(mm - 1) * W + cc) * 2] : make_double2(1, 0);
            const double2 cf_ = shift_coef(am, bpm, apm);
            double2 nxt = pi_step(cur, prev, am, cf_, delta);
            const int dl = hL[(size_t)(mm + 1) * W + cc] - hL[(size_t)mm * W + cc];
            if (dl) {
              const double f = scalbn(1.0, dl);
              nxt = cscale(nxt, f);
              cur = cscale(cur, f);
            }
            prev = cur;
            cur = nxt;
            buf[(size_t)(mm + 1 - m0) * WK + e] = nxt;
          }
        }
        for (int mm = mend - 1; mm >= m0; --mm) {
          double2 cm = make_double2(0, 0);
          if (valid && mm < nkk) {
            const double2 pim = buf[(size_t)(mm - m0) * WK + e];
            const double2 pim1 = buf[(size_t)(mm + 1 - m0) * WK + e];
            double2 ratio = cdiv(pim, pim1);
            const int dl = hL[(size_t)(mm + 1) * W + cc] - hL[(size_t)mm * W + cc];
            if (dl) ratio = cscale(ratio, scalbn(1.0, dl));
            const double2 am = hab[((size_t)mm * W + cc) * 2];
            const double2 bm = hab[((size_t)mm * W + cc) * 2 + 1];
            const double2 ak = cmul(ratio, am);
            const double2 bk = cmul(cmul(ratio, ratio), bm);
            S = cadd(ak, cmul(bk, S));
            cm = cdiv(S, pim);
          }
          lacc = cadd(lacc, cmul(cm, ht[(size_t)mm * W + cc]));
          if (cgs && valid) cgs[((size_t)mm * W + cc) * K + k] = cm;
          const double2 vr = warp_sum(cmul(wr, cm));
          const double2 ve = warp_sum(cmul(we, cm));
          if (lane == 0) {
            const size_t pe = (((size_t)mm * W + cc) * KG + kg) * 2;
            cp[pe] = vr;
            cp[pe + 1] = ve;
          }
        }
      }
      if (valid) {
        const long long col = (long long)sm.panel * W + cc;
        const long long o = (long long)k * a.nrhs + col;
        if (a.ldos) a.ldos[o] = -lacc.y / 3.141592653589793238462643383279502884;
        if (a.resid) a.resid[o] = resk[e];
        if (a.conv) a.conv[o] = resk[e] <= a.tol ? 1 : 0;
      }
    }
    __syncthreads();
    if (tid < W) {
      int mc = 0;
      for (int g = 0; g < KG; ++g) mc = max(mc, sx.Mt[tid * KG + g]);
      sx.Mc[tid] = mc;
    }
    __syncthreads();
  }
  // F2: C_m = sum over shift groups
  if (a.has_rho || a.has_edm) {
    int mmax = 0;
    for (int i = 0; i < W; ++i) mmax = max(mmax, sx.Mc[i]);
    for (int e = tid; e < mmax * W; e += TPB) {
      const int m = e / W, cc = e - m * W;
      if (m >= sx.Mc[cc]) continue;
      double2 sr = make_double2(0, 0), se = make_double2(0, 0);
      for (int g = 0; g < KG; ++g) {
        if (m >= sx.Mt[cc * KG + g]) continue;
        const size_t pe = (((size_t)m * W + cc) * KG + g) * 2;
        sr = cadd(sr, cp[pe]);
        se = cadd(se, cp[pe + 1]);
      }
      cf[((size_t)m * W + cc) * 2] = sr;
      cf[((size_t)m * W + cc) * 2 + 1] = se;
    }
    __syncthreads();
    // F3: rho_ij = Im sum_m C^rho_m r_m[i], edm_ij likewise
    const int Mt_ = sm.off[W];
    for (int e = tid; e < Mt_; e += TPB) {
      int cc = 0;
      while (sm.off[cc + 1] <= e) ++cc;
      const int t = e - sm.off[cc];
      double2 xr = make_double2(0, 0), xe = make_double2(0, 0);
      for (int m = 0; m < sx.Mc[cc]; ++m) {
        const double2 rv = hr[(size_t)m * a.Mcap + e];
        xr = cadd(xr, cmul(cf[((size_t)m * W + cc) * 2], rv));
        xe = cadd(xe, cmul(cf[((size_t)m * W + cc) * 2 + 1], rv));
      }
      const long long col = (long long)sm.panel * W + cc;
      const long long o = a.out_off[col] + t;
      if (a.rho && a.has_rho) a.rho[o] = xr.y;
      if (a.edm && a.has_edm) a.edm[o] = xe.y;
    }
    __syncthreads();
  }
  // F4: per-column outputs
  if (tid < W && sm.mc[tid] > 0) {
    const long long col = (long long)sm.panel * W + tid;
    const int base = a.m.row_ptr[sm.j[tid]];
    if (a.has_rho && a.rho && (a.q || a.e_loc)) {
      double qs = 0.0, es = 0.0;
      for (int t = 0; t < sm.mc[tid]; ++t) {
        const double rv = a.rho[a.out_off[col] + t];
        qs = fma(rv, a.m.s_val[base + t], qs);
        es = fma(rv, a.m.h_val[base + t], es);
      }
      if (a.q) a.q[col] = qs;
      if (a.e_loc) a.e_loc[col] = es;
    }
    if (a.iters) a.iters[col] = sm.nc[tid];
    if (a.inner_iters) a.inner_iters[col] = sm.inner_count;
    int st = sm.st[tid] | (sm.bc_fail ? kStTimeout : 0);
    for (int k = 0; k < K; ++k)
      if (!(resk[tid * K + k] <= a.tol)) st |= kStNoConv;
    a.status[col] = st;
    if (a.col_status) a.col_status[col] = st;
  }
  if (cgs && a.g_proj) {
    __syncthreads();
    const int Mt_ = sm.off[W];
    for (int e = tid; e < Mt_ * K; e += TPB) {
      const int k = e / Mt_, f = e - k * Mt_;
      int cc = 0;
      while (sm.off[cc + 1] <= f) ++cc;
      const int t = f - sm.off[cc];
      const int nkk = nk[cc * K + k];
      double2 g = make_double2(0, 0);
      for (int m = 0; m < nkk; ++m) g = cadd(g, cmul(cgs[((size_t)m * W + cc) * K + k], hr[(size_t)m * a.Mcap + f]));
      const long long col = (long long)sm.panel * W + cc;
      a.g_proj[(long long)k * a.P + a.out_off[col] + t] = g;
    }
  }
  __syncthreads();
}

template <bool MIX>
__global__ void __launch_bounds__(TPB, MIN_TEAMS_PER_SM) team_kernel(const __grid_constant__ Args a) {
  __shared__ Smem sm;
  __shared__ PanelSmemExtra sx;
  extern __shared__ __align__(16) char dyn_smem[];
  char* ws = a.team_ws + (size_t)blockIdx.x * a.team_bytes;
  team_init(sm, dyn_smem);
  if (a.full_hist) {  // verification: one panel per team, panel = team
    if (threadIdx.x == 0) sm.panel = blockIdx.x;
    __syncthreads();
    if (sm.panel < a.npanels) solve_panel<MIX>(a, sm, sx, ws, dyn_smem);
    return;
  }
  for (;;) {
    if (threadIdx.x == 0) sm.panel = atomicAdd(a.panel_counter, 1);
    __syncthreads();
    if (sm.panel >= a.npanels) return;
    solve_panel<MIX>(a, sm, sx, ws, dyn_smem);
    __syncthreads();
  }
}

// Batched form: many independent systems (each with its own matrix, shifts,
// columns and outputs) in one persistent launch.  Work items are (system,
// panel) pairs numbered through panel_prefix (the host orders the systems,
// largest first); a team copies the item's system descriptor into shared
// memory and runs the same panel solver.  The team workspace is laid out for
// the largest system.
template <bool MIX>
__global__ void __launch_bounds__(TPB, MIN_TEAMS_PER_SM)
    team_kernel_batched(const Args* __restrict__ sys, const int* __restrict__ panel_prefix, int nsys,
                        int* __restrict__ counter, char* team_ws, size_t team_bytes) {
  __shared__ Smem sm;
  __shared__ PanelSmemExtra sx;
  __shared__ Args sa;
  __shared__ int s_sys;
  extern __shared__ __align__(16) char dyn_smem[];
  char* ws = team_ws + (size_t)blockIdx.x * team_bytes;
  team_init(sm, dyn_smem);
  const int total = panel_prefix[nsys];
  for (;;) {
    if (threadIdx.x == 0) {
      const int item = atomicAdd(counter, 1);
      int lo = 0;
      if (item < total) {
        int hi = nsys;  // panel_prefix[lo] <= item < panel_prefix[hi]
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (panel_prefix[mid] <= item) lo = mid;
          else hi = mid;
        }
      }
      s_sys = item < total ? lo : -1;
      sm.panel = item < total ? item - panel_prefix[lo] : 0;
    }
    __syncthreads();
    if (s_sys < 0) return;
    const unsigned* src = reinterpret_cast<const unsigned*>(sys + s_sys);
    unsigned* dst = reinterpret_cast<unsigned*>(&sa);
    for (int i = threadIdx.x; i < (int)(sizeof(Args) / sizeof(unsigned)); i += TPB) dst[i] = src[i];
    __syncthreads();
    solve_panel<MIX>(sa, sm, sx, ws, dyn_smem);
    __syncthreads();
  }
}

}  // namespace gbk
