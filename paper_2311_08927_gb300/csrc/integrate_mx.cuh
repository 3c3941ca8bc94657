// Mixed-precision integration with S_h2 algebraic (kernel form 4).
//
// The same W-method, queue and controller as integrate_impl.cuh, with the
// precision split chosen for a GPU whose FP32 rate is 64 times its FP64 rate:
//   * FP32: rates f(y) at every stage (Eq. 2-6), the split Jacobian J_d and
//     u = df/dS_H, the sparse LU of W_d and every solve;
//   * FP32: S_h2 from its mass balance (Eq. 8, the paper's DAE form), by
//     Newton on the coefficients that the FP32 rates already hold;
//   * two-float (about 48 bits, on the FP32 pipe): the stage right-hand
//     sides, the refinement residual r = b - W x of every solve (W x from
//     the FP32 rate partials in two-float arithmetic) and the error
//     combination k1 - 2 k2 + k3 of the FP32 stage vectors (exact);
//   * FP64: the charge-balance Newton for S_H (Eq. 7) at every rate
//     evaluation and the state y, y + h/2 k1 and y + h k2.
// One refinement step per solve: x0 = W^-1 b in FP32, x = x0 + W^-1 r.
//
// With S_h2 algebraic the fast hydrogen mode is not a state, so the FP32
// rounding of the stage rates (about 1e-7 relative) stays far below the
// error tolerance; as a state, S_h2 turns over at about 1e6 per day and its
// FP32 rate noise reaches the embedded error estimate (the reason the
// differential mixed forms keep FP64 stage rates).
//
// W = I - g J_eff, J_eff the Jacobian of the reduced system (S_h2 replaced
// by its root, S_H by the Eq. 7 root): W_d = I - g J_d without the S_h2 row
// and column, then two Sherman-Morrison levels, u v^T (S_H) and w zh^T
// (S_h2: w the S_h2 column of J_d, zh = dS_h2/dy including the path
// through S_H).  The residual's J_eff x is the product J_d x' + u (v^T x)
// of the rate partials with x' = x except x'_h2 = zh^T x, and a zero S_h2
// row.  W_d is factored by the generated LU over the 28 other states
// (sparse_lu_h2a_gen.cuh: 167 slots and 419 flops against 203 and 664 with
// S_h2 in it); the Jacobian scatter delivers S_h2's row into zh and its
// column into p2 directly (H2Split), so they never occupy LU slots.
#pragma once
#include "dfloat.cuh"
#include "integrate_impl.cuh"

namespace chad {
namespace integ {

// an opaque copy of an index (a digester's): loads through it are not
// hoisted out of the loop they are in
__device__ __forceinline__ int reread_i(int i) {
  asm volatile("" : "+r"(i));
  return i;
}

// the eight states that enter Eq. 7
__host__ __device__ constexpr bool in_eq7(int i) {
  return i == iS_va || i == iS_bu || i == iS_pro || i == iS_ac || i == iS_IC || i == iS_IN ||
         i == iS_cat || i == iS_an;
}

// binary64 -> float and float -> binary64 of the kernel (hardware conversions)
__device__ __forceinline__ float f32(double d) { return float(d); }
__device__ __forceinline__ double f64(float f) { return double(f); }

// Eq. 8 in FP32: root of E(S) from the guess by Newton; a non-decreasing
// slope, a growing |E| or an iterate leaving (0, inf) switches to bisection
// on [0, hi], hi doubled from the guess until E(hi) <= 0.  Converged when an
// update is below 1e-6 relative (FP32 Newton reaches the root to a few
// units in the last place, so a tighter test could stall on rounding).
__device__ __forceinline__ float solve_h2_f32(const H2Bal<float>& e, float guess, Cnt& cnt) {
  float S = (guess > 0.0f && guess < 1e30f) ? guess : 1e-8f;
  float prevE = INFINITY;
#pragma unroll 1
  for (int it = 0; it < 12; ++it) {
    float dE;
    const float E = h2_eval<float>(e, S, dE);
    cnt.h2++;
    if (!(fabsf(E) <= fabsf(prevE)) || !(dE < 0.0f)) break;
    const float dS = E * __frcp_rn(dE);
    const float Sn = S - dS;
    if (!(Sn > 0.0f) || !(Sn < 1e30f)) break;
    if (fabsf(dS) <= 1e-6f * Sn || E == 0.0f) return Sn;
    prevE = E;
    S = Sn;
  }
  cnt.fallback++;
  float lo = 0.0f, hi = fmaxf((guess > 0.0f && guess < 1e30f) ? guess : 0.0f, 1e-12f), dE;
  int k = 0;
  while (k < 120 && h2_eval<float>(e, hi, dE) > 0.0f) {
    hi *= 2.0f;
    ++k;
  }
  if (k == 120) {
    cnt.failed = 1;
    return (guess > 0.0f && guess < 1e30f) ? guess : 1e-8f;
  }
#pragma unroll 1
  for (int it = 0; it < 60; ++it) {
    const float mid = 0.5f * (lo + hi);
    if (!(mid > lo && mid < hi)) break;
    if (h2_eval<float>(e, mid, dE) > 0.0f) lo = mid; else hi = mid;
  }
  return 0.5f * (lo + hi);
}

// S_H (FP64 Newton at the FP64 state y) and S_h2 (FP32 Newton at the float
// state ys, written into ys[iS_h2]) at one evaluation point.
__device__ __forceinline__ void roots(const DigConst& c, const DigConstF& cf, const PartConst& q,
                                      const PartConstF& qf, const double* y, float* ys, float D,
                                      double& SHg, float& SH2g, int max_newton, Cnt& cnt,
                                      AcidBase& ab) {
  newton(c, q, y, SHg, max_newton, cnt, ab);
  H2Bal<float> e;
  h2_coeffs<float>(cf, qf, ys, D, ab, e);
  SH2g = solve_h2_f32(e, SH2g, cnt);
  ys[iS_h2] = SH2g;
}

// FP32 rate vector at ys (roots already in ab and ys[iS_h2]); S_h2 rate 0.
__device__ __forceinline__ void rates_f32(const DigConstF& cf, const PartConstF& qf,
                                          const float* ys, float D, const AcidBase& ab,
                                          float* f) {
  Rates<float> o;
  rates<float, false>(cf, qf, ys, ab, o);
  balances<float>(cf, ys, D, o, f);
  f[iS_h2] = 0.0f;
}

// x <- W^-1 x with the factored W_d and both Sherman-Morrison levels.
template <class W>
__device__ __forceinline__ void wsolve(W w, const float* qv,
                                       const float* vr, float inv_delta, const float* p2,
                                       const float* zh, float inv_delta2, float* x) {
  spa::solve<float>(w, x);
  rank1::update<float>(qv, vr, inv_delta, x);
  float s2 = 0.0f;
#pragma unroll
  for (int j = 0; j < NS; ++j) s2 = fmaf(zh[j], x[j], s2);
  s2 *= inv_delta2;
#pragma unroll
  for (int i = 0; i < NS; ++i) x[i] = fmaf(s2, p2[i], x[i]);
}

// IDX: contexts with more than one digester, whose warps hold particles of
// several digesters (the queue refills lanes one by one); there the
// per-thread-array shapes re-read the digester constants through an opaque
// copy of the digester index.
template <int BS, int MINB, bool WS, bool IDX>
__global__ void __launch_bounds__(BS, MINB) integrate_mx_kernel(StepArgs a) {
  __shared__ unsigned long long s_acc, s_rej, s_newton, s_fb, s_piv, s_redo, s_h2;
  __shared__ int s_min, s_max;
  if (threadIdx.x == 0) {
    s_acc = s_rej = s_newton = s_fb = s_piv = s_redo = s_h2 = 0ull;
    s_min = INT_MAX;
    s_max = 0;
  }
  __syncthreads();

  WStore<float, BS, WS, spa::kNNZ> wst;
  const auto w = wst.slots();
  float qv[NS];    // u = df/dS_H, then q = W_d^-1 (g u)
  float p2[NS], zh[NS];  // second level: W_1^-1 (g w) and dS_h2/dy
  double y[NS], y1[NS];  // state; evaluation point (only the eight states of Eq. 7)
  float ys[NS], y1s[NS]; // float copies (rates, error scale)
  float F0[NS];           // FP32 rates at y; after stage 1 e32 F1 + 2 F0
  float k1[NS], k2[NS], k3[NS];  // stage vectors (refined solutions, FP32)
  const double Tend = a.dt_days;
  const bool fixed = a.fixed_n > 0;
  Cnt tot{0, 0, 0, 0, 0, 0, 0};
  int min_steps = INT_MAX, max_steps = 0;

  int64_t p = -1;
  const DigConst* c = nullptr;
  const DigConstF* cf = nullptr;
  int dg = 0;  // digester of the particle
  // The digester constants, read again before each evaluation (see reread)
  // through an opaque copy of their pointer, or with IDX (several
  // digesters) and W_d in per-thread arrays of the digester index: the two
  // compile to different code, and measured on 64 digesters (one interval
  // pair of the 128-thread shape) the index copy took 1,141 ms against
  // 2,517 ms, while on one digester the pointer copy with W_d in shared
  // memory was the fastest shape.
  auto dcn = [&]() -> const DigConst& {
    if constexpr (IDX && !WS) return a.dc[reread_i(dg)];
    else return *reread(c);
  };
  auto dcfn = [&]() -> const DigConstF& {
    if constexpr (IDX && !WS) return a.dcf[reread_i(dg)];
    else return *reread(cf);
  };
  PartConst q;
  PartConstF qf;
  double SHg = 0.0, h = 0.0, t = 0.0;
  float Df = 0.0f, SH2g = 0.0f;
  int status = 0, attempts = 0, nacc = 0;
  bool rejected_prev = false, ys_stale = true;
  Cnt cnt{0, 0, 0, 0, 0, 0, 0};

  bool exhausted = false;
  while (true) {
    bool fresh = false;
    if (p < 0 && !exhausted) {
      p = queue_pop(a.queue);
      if (p >= a.n) {
        exhausted = true;
        p = -1;
      } else {
        if (a.order) p = a.order[p];
        fresh = true;
      }
    }
    if (!__syncthreads_or(p >= 0)) break;
    if (p < 0) continue;
    if (fresh) {
      cnt = Cnt{0, 0, 0, 0, 0, 0, 0, 0};
      dg = a.dig[p];
      c = &a.dc[dg];
      cf = &a.dcf[dg];
      pc_load(a.pc, a.ld, p, q);
      narrow_pc(q, qf);
#pragma unroll
      for (int i = 0; i < NS; ++i) y[i] = a.y[i * a.ld + p];
      SHg = a.SH[p];
      SH2g = f32(y[iS_h2]);
      h = a.h[p];
      if (a.SH_learned && !(h > 0.0 && isfinite(h))) {
        AcidBase abt;
        int it = 0;
        if (newton_only(*c, q, y, a.SH_learned[p], 4, 1e-10, abt, it))
          SHg = abt.SH;
        else
          cnt.redo++;
        cnt.newton += it;
        h = a.h_learned[p];
      }
      h = (h > 0.0 && isfinite(h)) ? h : kHdefault;
      if (fixed) h = Tend / a.fixed_n;
      Df = f32(a.D[p]);
      t = 0.0;
      status = 0;
      attempts = 0;
      nacc = 0;
      rejected_prev = false;
      ys_stale = true;
    }
    // ------------------------------------------------ one step attempt
    bool done = false;
    ++attempts;
    double hh = h;
    bool last = false;
    if (!fixed && hh >= (Tend - t) * (1.0 - 1e-12)) {
      hh = Tend - t;
      last = true;
    }
    const double g = hh * kRB_d;
    const float gf = f32(g);
    const df gd = df_of_double(g);
    if (ys_stale) {
#pragma unroll
      for (int i = 0; i < NS; ++i) ys[i] = f32(y[i]);
      ys_stale = false;
    }
    // roots, rates, J_d and u at y (all FP32 but the Eq. 7 Newton)
    AcidBase ab0;
    roots(dcn(), dcfn(), q, qf, y, ys, Df, SHg, SH2g, a.max_newton, cnt, ab0);
    {
      // the rate partials are recomputed for each refinement residual
      // (from ys and ab0) rather than kept across the stages
      Rates<float> ko;
      rates<float, true>(*cf, qf, ys, ab0, ko);
      balances<float>(*cf, ys, Df, ko, F0);
      F0[iS_h2] = 0.0f;
      jacobian<spa::Idx, float>(*cf, qf, ys, Df, ab0, ko,
                                H2Split<float, decltype(w)>{w, zh, p2}, qv);
    }
    const double SH0 = SHg;
    const float SH20 = SH2g;
    double vsh[8];
    sh_tangent(*c, q, ab0, vsh);
    float vr[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) vr[k] = f32(vsh[k]);
    // S_h2 leaves W_d: dS_h2/dy = -(J_h2,j + u_h2 v_j) / J_h2,h2 from its
    // row, g times its column becomes the second Sherman-Morrison vector
    {
      const float rjj = __frcp_rn(zh[iS_h2]);
#pragma unroll
      for (int j = 0; j < NS; ++j)
        zh[j] = (sp::slot(iS_h2, j) >= 0 && j != iS_h2) ? -zh[j] * rjj : 0.0f;
      const int hc[8] = {iS_va, iS_bu, iS_pro, iS_ac, iS_IC, iS_IN, iS_cat, iS_an};
#pragma unroll
      for (int k = 0; k < 8; ++k) zh[hc[k]] -= qv[iS_h2] * vr[k] * rjj;
#pragma unroll
      for (int i = 0; i < NS; ++i)
        p2[i] = (sp::slot(i, iS_h2) >= 0 && i != iS_h2) ? gf * p2[i] : 0.0f;
      qv[iS_h2] = 0.0f;
    }
    spa::form_w<float>(w, gf);
    const bool lu_ok = spa::factor<float>(w);
    float inv_delta = 0.0f, inv_delta2 = 0.0f;
    bool piv_ok = lu_ok;
    if (lu_ok || fixed) {
      // q = W_d^-1 (g u), then p2 = W_1^-1 (g w) with W_1 = W_d - g u v^T
#pragma unroll
      for (int i = 0; i < NS; ++i) qv[i] *= gf;
      spa::solve<float>(w, qv);
      piv_ok = rank1::denominator<float>(qv, vr, float(kPivTau), &inv_delta) && piv_ok;
      spa::solve<float>(w, p2);
      rank1::update<float>(qv, vr, inv_delta, p2);
      float s2 = 0.0f;
#pragma unroll
      for (int j = 0; j < NS; ++j) s2 = fmaf(zh[j], p2[j], s2);
      const float delta2 = 1.0f - s2;
      inv_delta2 = __frcp_rn(delta2);
      piv_ok = piv_ok && isfinite(delta2) && delta2 != 0.0f &&
               fabsf(delta2) >= float(kPivTau) * fmaxf(1.0f, fabsf(s2));
    }
    if (!piv_ok) cnt.pivot++;
    float norm = INFINITY;
    if (piv_ok || fixed) {
      // Stages (not unrolled: one copy of the rate evaluation and of the
      // solve pair in the kernel):
      //   0: b = F0                                  -> k1 = x
      //   1: F1 = f(y + h/2 k1), b = F1 - k1         -> k2 = x + k1
      //   2: F2 = f(y + h k2),   b = F2 - e32 (k2 - F1) - 2 (k1 - F0)
      //                                              -> k3 = x
      // The right-hand sides are formed in two-float from the FP32 rates and
      // stage vectors; the refined solution x0 + W^-1 r is kept in FP32 (the
      // stage rates it solves for are FP32).  After stage 1 the rates are
      // needed only as C = e32 F1 + 2 F0 (kept in F0's place), so that
      // b2 = F2 - e32 k2 - 2 k1 + C.
      const df e32 = df_of_double(kRB_e32);
#pragma unroll 1
      for (int st = 0; st < 3; ++st) {
        df b[NS];
        if (st == 0) {
#pragma unroll
          for (int i = 0; i < NS; ++i) b[i] = df_of(F0[i]);
        } else {
          // evaluation point y + (h/2) k1 or y + h k2.  Both need FP64 only
          // in the eight states of Eq. 7 (its Newton); stage 1's FP32 rates
          // take y + (h/2) k1 in float.  Stage 2's point is the new state:
          // its float copy is rounded from the FP64 sum, which is formed
          // again on acceptance rather than held through the stage.
          if (st == 1) {
            const double hs = 0.5 * hh;
            const float hsf = f32(hs);
            const int hc[8] = {iS_va, iS_bu, iS_pro, iS_ac, iS_IC, iS_IN, iS_cat, iS_an};
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              const int i = hc[k];
              y1[i] = fma(hs, f64(k1[i]), y[i]);
            }
#pragma unroll
            for (int i = 0; i < NS; ++i) y1s[i] = fmaf(hsf, k1[i], ys[i]);
          } else {
#pragma unroll
            for (int i = 0; i < NS; ++i) {
              const double yn = fma(hh, f64(k2[i]), y[i]);
              if (in_eq7(i)) y1[i] = yn;
              y1s[i] = f32(yn);
            }
          }
          {
            // tangent guess of the Eq. 7 root from the FP32 tangent and the
            // step's increment (h/2 k1 or h k2): only Newton's start moves
            const int hc[8] = {iS_va, iS_bu, iS_pro, iS_ac, iS_IC, iS_IN, iS_cat, iS_an};
            float ds = 0.0f;
#pragma unroll
            for (int k = 0; k < 8; ++k) ds = fmaf(vr[k], st == 1 ? k1[hc[k]] : k2[hc[k]], ds);
            const double g = fma(st == 1 ? 0.5 * hh : hh, f64(ds), SH0);
            SHg = (g > 0.5 * SH0 && g < 2.0 * SH0) ? g : SH0;
          }
          {
            float g2 = SH20;
#pragma unroll
            for (int j = 0; j < NS; ++j) g2 = fmaf(zh[j], y1s[j] - ys[j], g2);
            SH2g = (g2 > 0.5f * SH20 && g2 < 2.0f * SH20) ? g2 : SH20;
          }
          AcidBase ab;
          roots(dcn(), dcfn(), q, qf, y1, y1s, Df, SHg, SH2g, a.max_newton, cnt, ab);
          float Fs[NS];
          rates_f32(dcfn(), qf, y1s, Df, ab, Fs);
          if (st == 1) {
#pragma unroll
            for (int i = 0; i < NS; ++i) {
              b[i] = two_sum(Fs[i], -k1[i]);
              const df c1 = df_mul_f(e32, Fs[i]);
              F0[i] = c1.hi + fmaf(2.0f, F0[i], c1.lo);  // C = e32 F1 + 2 F0
            }
          } else {
#pragma unroll
            for (int i = 0; i < NS; ++i) {
              const df t1 = df_add_f(df_mul_f(e32, k2[i]), 2.0f * k1[i]);
              b[i] = df_add_f(df_sub(df_of(Fs[i]), t1), F0[i]);
            }
          }
        }
        // x0 = W^-1 b in FP32; r = b - x0 + g J_eff x0 in two-float; x = x0 + W^-1 r
        float x0[NS];
#pragma unroll
        for (int i = 0; i < NS; ++i) x0[i] = b[i].hi;
        wsolve(w, qv, vr, inv_delta, p2, zh, inv_delta2, x0);
        float xs[NS];
        {
          DF xp[NS], jx[NS];
#pragma unroll
          for (int i = 0; i < NS; ++i) xp[i] = DF(x0[i]);
          DF zx(0.0f);
#pragma unroll
          for (int j = 0; j < NS; ++j)
            if (j != iS_h2) zx = zx + zh[j] * xp[j];
          xp[iS_h2] = zx;
          DF sv(0.0f);
          {
            const int hc[8] = {iS_va, iS_bu, iS_pro, iS_ac, iS_IC, iS_IN, iS_cat, iS_an};
#pragma unroll
            for (int k = 0; k < 8; ++k) sv = sv + vr[k] * xp[hc[k]];
          }
          Rates<float> ko;
          const DigConstF& cfr = dcfn();
          rates<float, true>(cfr, qf, ys, ab0, ko);
          jvp<float, DF, DigConstF, float>(cfr, ys, Df, ko, xp, sv, jx);
          jx[iS_h2] = DF(0.0f);
          float r[NS];
#pragma unroll
          for (int i = 0; i < NS; ++i) {
            const df ri = df_add(df_add_f(b[i], -x0[i]), df_mul(gd, jx[i].v()));
            r[i] = ri.hi + ri.lo;
          }
          wsolve(w, qv, vr, inv_delta, p2, zh, inv_delta2, r);
#pragma unroll
          for (int i = 0; i < NS; ++i) xs[i] = x0[i] + r[i];
        }
        if (st == 0) {
#pragma unroll
          for (int i = 0; i < NS; ++i) k1[i] = xs[i];
        } else if (st == 1) {
#pragma unroll
          for (int i = 0; i < NS; ++i) k2[i] = xs[i] + k1[i];
        } else {
#pragma unroll
          for (int i = 0; i < NS; ++i) k3[i] = xs[i];
        }
      }
      // scaled error norm max_i |h/6 (k1 - 2 k2 + k3)_i| / (atol_i + rtol
      // max(|y_i|, |y1_i|)): the combination of the FP32 stage vectors exact
      // in two-float, the rest in FP32 (fixed steps need none)
      if (!fixed) {
        float nf = 0.0f;
        const float rtol = f32(a.rtol);
#pragma unroll
        for (int i = 0; i < NS; ++i) {
          const df ed = df_add_f(two_sum(k1[i], -2.0f * k2[i]), k3[i]);
          const float e = ed.hi + ed.lo;
          const float ym = fmaxf(fabsf(ys[i]), fabsf(y1s[i]));
          const float sc = fmaxf(fmaf(rtol, ym, f32(a.atol[i])), 1e-30f);
          const float r = fabsf(e) * __frcp_rn(sc);
          if (!(r <= nf)) nf = r;  // NaN propagates
        }
        norm = nf * (f32(hh) * (1.0f / 6.0f));
      }
    }
    const bool accept = fixed || norm <= 1.0f;
    if (accept) {
#pragma unroll
      for (int i = 0; i < NS; ++i) {
        y[i] = fma(hh, f64(k2[i]), y[i]);  // y + h k2, as at stage 2
        ys[i] = y1s[i];
      }
      y[iS_h2] = f64(SH2g);  // Eq. 8 root at the new state (last evaluation)
      ys[iS_h2] = SH2g;      // ys stays the float rounding of y
      cnt.acc++;
      ++nacc;
    }
    if (fixed) {
      // fixed steps need no error norm: a state that is not finite is
      // flagged when the particle is stored
      if (nacc >= a.fixed_n) done = true;
    } else if (accept) {
      t = last ? Tend : t + hh;
      float fac = (norm == 0.0f) ? 5.0f : fminf(5.0f, fmaxf(0.2f, 0.8f * powf(norm, -1.0f / 3.0f)));
      if (rejected_prev) fac = fminf(fac, 1.0f);
      h = hh * f64(fac);
      rejected_prev = false;
      if (last) done = true;
    } else {
      cnt.rej++;
      const float fac =
          !piv_ok ? 0.25f : (isfinite(norm) ? fmaxf(0.2f, 0.8f * powf(norm, -1.0f / 3.0f)) : 0.2f);
      h = hh * f64(fac);
      rejected_prev = true;
      if (h < kHmin) {
        status |= ST_HMIN;
        done = true;
      }
    }
    if (!done && !fixed && attempts >= a.max_steps) {
      status |= ST_STEPS;
      done = true;
    }
    // ------------------------------------------------ particle finished
    if (done) {
      if (cnt.failed) status |= ST_NEWTON;
#pragma unroll
      for (int i = 0; i < NS; ++i) {
        const long long yb = __double_as_longlong(y[i]);
        const long long mag = yb & 0x7fffffffffffffffll;
        if (mag >= 0x7ff0000000000000ll) status |= ST_NAN;
        if (yb < 0 && mag > __double_as_longlong(a.atol[i])) status |= ST_NEG;
      }
#pragma unroll
      for (int i = 0; i < NS; ++i) a.y[i * a.ld + p] = y[i];
      a.SH[p] = SHg;
      if (!fixed) a.h[p] = h;
      if (status) a.status[p] |= status;
      tot.acc += cnt.acc;
      tot.rej += cnt.rej;
      tot.newton += cnt.newton;
      tot.fallback += cnt.fallback;
      tot.pivot += cnt.pivot;
      tot.redo += cnt.redo;
      tot.h2 += cnt.h2;
      min_steps = min(min_steps, nacc);
      max_steps = max(max_steps, nacc);
      p = -1;
    }
  }

  atomicAdd(&s_acc, (unsigned long long)tot.acc);
  atomicAdd(&s_rej, (unsigned long long)tot.rej);
  atomicAdd(&s_newton, (unsigned long long)tot.newton);
  atomicAdd(&s_fb, (unsigned long long)tot.fallback);
  atomicAdd(&s_piv, (unsigned long long)tot.pivot);
  atomicAdd(&s_redo, (unsigned long long)tot.redo);
  atomicAdd(&s_h2, (unsigned long long)tot.h2);
  atomicMin(&s_min, min_steps);
  atomicMax(&s_max, max_steps);
  __syncthreads();
  if (threadIdx.x == 0 && a.counters) {
    atomicAdd(&a.counters->accepted, s_acc);
    atomicAdd(&a.counters->rejected, s_rej);
    atomicAdd(&a.counters->newton_iters, s_newton);
    atomicAdd(&a.counters->newton_fallbacks, s_fb);
    atomicAdd(&a.counters->pivot_rejects, s_piv);
    atomicAdd(&a.counters->mlp_redo, s_redo);
    atomicAdd(&a.counters->h2_iters, s_h2);
    if (s_min != INT_MAX) atomicMin(&a.counters->min_steps, s_min);
    atomicMax(&a.counters->max_steps, s_max);
  }
}

}  // namespace integ

template <int BS, int MINB, bool WS, bool IDX>
cudaError_t launch_variant_mx_k(const StepArgs& a, cudaStream_t s) {
  constexpr size_t smem = integ::wstore_smem_bytes<float, BS, WS, spa::kNNZ>();
  static int per_sm = -1, sms = 0;
  if (per_sm < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (smem > 0) {
      cudaError_t e = cudaFuncSetAttribute(integ::integrate_mx_kernel<BS, MINB, WS, IDX>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, integ::integrate_mx_kernel<BS, MINB, WS, IDX>, BS, smem);
    if (per_sm < 1) per_sm = 1;
    // The unified L1 / shared array: the smallest shared carve-out that holds
    // the resident blocks' tiles (none without a tile), so that the rest is
    // L1 for the spilled per-thread state whatever kernels ran before.  After
    // the MLP training kernels (large shared tiles) the register shapes had
    // less L1 otherwise: 1M workload 46,279 -> 51,212 particle-days/s with
    // the training in the same process.
    int smem_sm = 0;
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    const long long need = smem > 0 ? (long long)per_sm * ((long long)smem + 2048) : 0;
    const int pct = smem_sm > 0 ? (int)((need * 100 + smem_sm - 1) / smem_sm) : 100;
    cudaError_t e = cudaFuncSetAttribute(integ::integrate_mx_kernel<BS, MINB, WS, IDX>,
                                         cudaFuncAttributePreferredSharedMemoryCarveout,
                                         pct < 100 ? pct : 100);
    if (e != cudaSuccess) return e;
  }
  int64_t blocks = (int64_t)sms * per_sm;
  const int64_t need = (a.n + BS - 1) / BS;
  if (need < blocks) blocks = need;
  cudaError_t e = cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  integ::integrate_mx_kernel<BS, MINB, WS, IDX><<<(unsigned)blocks, BS, smem, s>>>(a);
  return cudaGetLastError();
}

template <int BS, int MINB, bool WS>
cudaError_t launch_variant_mx(const StepArgs& a, cudaStream_t s) {
  return a.n_dig > 1 ? launch_variant_mx_k<BS, MINB, WS, true>(a, s)
                     : launch_variant_mx_k<BS, MINB, WS, false>(a, s);
}

}  // namespace chad
