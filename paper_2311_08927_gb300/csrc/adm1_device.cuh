// Device-side ADM1 model for one particle per thread (Sec. 2.2-2.3).
//
//   * part_const   : temperature-dependent constants of a particle (van 't
//                    Hoff acid-base and Henry constants, Arrhenius kinetics).
//   * solve_SH     : Eq. 7 charge balance for S_H+ by Newton, with a
//                    bracketed geometric bisection fallback (FP64 always).
//   * model_f      : rate vector f(y) (Eq. 2 mass balances, Eq. 3-6 rates).
//   * model_fj     : f(y) and the analytic Jacobian df/dy, including the
//                    rank-1 coupling through S_H(y) given by the implicit
//                    function theorem on Eq. 7.
// R is the arithmetic type of rates, Jacobian and LU (double for the plain
// path, float for the mixed path); the charge balance is always FP64.
#pragma once
#include <cmath>
#include <cstdint>

#include "model.h"

#ifndef CHAD_HD
#define CHAD_HD __host__ __device__ __forceinline__
#endif

namespace chad {

// Dense row-major storage of a NS x NS matrix (slot of entry (r, c)).
struct DenseIdx {
  static CHAD_HD constexpr int at(int r, int c) { return r * NS + c; }
  static constexpr int size = NS * NS;
};

// Conversions between binary64 and binary32 (IEEE 754).  On the GPU a
// hardware FP64<->FP32 conversion occupies the FP64 pipe as long as an FP64
// FMA (measured on GB300: both ~600 G lane-ops/s, the DFMA rate), so the
// device versions below work on the bit patterns with integer operations:
//   widen  (float -> double): exact for normal numbers; zero and subnormal
//          inputs give a signed zero; Inf and NaN keep their class.
//   narrow (double -> float): the significand truncated to 23 bits (round
//          toward zero, relative error below 2^-23); magnitudes below the
//          normal float range give a signed zero, above it +-Inf; NaN stays
//          NaN.
// Host code and other types use the plain casts.
template <class To, class From>
CHAD_HD To cvt(From x) {
  return To(x);
}
#ifdef __CUDA_ARCH__
template <>
__device__ __forceinline__ double cvt<double, float>(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned m = (e == 0u) ? 0u : (u & 0x7fffffu);
  const unsigned ee = (e == 0u) ? 0u : ((e == 0xffu) ? 0x7ffu : e + 896u);
  const unsigned hi = (u & 0x80000000u) | (ee << 20) | (m >> 3);
  return __hiloint2double((int)hi, (int)(m << 29));
}
template <>
__device__ __forceinline__ float cvt<float, double>(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned sgn = hi & 0x80000000u;
  const int E = (int)((hi >> 20) & 0x7ffu);
  const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const int e = E - 896;
  const bool nan = (E == 0x7ff) && (((hi & 0xfffffu) | lo) != 0u);
  unsigned u = sgn | ((unsigned)e << 23) | m;
  u = (e <= 0) ? sgn : u;
  u = (e >= 255) ? (sgn | 0x7f800000u | (nan ? 0x400000u : 0u)) : u;
  return __uint_as_float(u);
}
#endif

// 1/d.  On the GPU in FP64: the FP32 hardware reciprocal of d as the seed
// r0 (relative error e = 1 - d r0 below 2^-22 with the truncated
// conversion), then one polynomial correction r0 (1 + e + e^2) of the
// Newton-Raphson family for the reciprocal, whose relative error is O(e^3)
// (below 1e-19): three FMAs.  Values outside the FP32 normal range use the
// division.  Elsewhere (host, FP32, counting types): the plain division.
template <class R>
CHAD_HD R rcp(R d) {
  return R(1) / d;
}
#ifdef __CUDA_ARCH__
template <>
__device__ __forceinline__ double rcp<double>(double d) {
  const float f = cvt<float, double>(d);
  const float af = fabsf(f);
  if (!(af > 1e-30f && af < 1e30f)) return 1.0 / d;
  const double r = cvt<double, float>(__frcp_rn(f));
  const double e = fma(-d, r, 1.0);
  return fma(r, fma(e, e, e), r);
}
#endif

// Threshold pivot test of the static-order LU: a pivot p is accepted when
// it is finite, nonzero and |p| >= 0.1 max_i |l_i| over its sub-column.
// key() maps an entry to a comparable magnitude, kmax() combines keys,
// good() takes the decision.  Host and counting types: the exact test.  On
// the GPU (FP64 and FP32) it runs on the IEEE-754 bit patterns with integer
// operations, because FP64 compares and min/max occupy the FP64 pipe: the
// sign-cleared pattern (the high word for a double) orders finite
// magnitudes like their values, and read as an integer it is a
// piecewise-linear log2 of the magnitude in units of 2^-20 (double high
// word) or 2^-23 (float), so the factor 0.1 becomes a shift by log2(10) in
// those units; the effective threshold is 0.1 up to the error of that
// linear log2, i.e. between 0.094 and 0.106.
template <class R>
struct PivTest {
  using K = R;
  static CHAD_HD K key(R x) { return fabs(x); }
  static CHAD_HD K kmax(K a, K b) { return fmax(a, b); }
  static CHAD_HD bool good(K p) { return p != R(0) && isfinite(p); }
  static CHAD_HD bool good(K p, K cm) { return good(p) && p >= R(0.1) * cm; }
};
#ifdef __CUDA_ARCH__
template <>
struct PivTest<double> {
  using K = unsigned;
  static __device__ __forceinline__ K key(double x) {
    return (unsigned)__double2hiint(x) & 0x7fffffffu;
  }
  static __device__ __forceinline__ K kmax(K a, K b) { return max(a, b); }
  static __device__ __forceinline__ bool good(K p) { return p != 0u && p < 0x7ff00000u; }
  static __device__ __forceinline__ bool good(K p, K cm) {
    return good(p) && p + 3483294u >= cm;  // log2(10) * 2^20
  }
};
template <>
struct PivTest<float> {
  using K = unsigned;
  static __device__ __forceinline__ K key(float x) { return __float_as_uint(x) & 0x7fffffffu; }
  static __device__ __forceinline__ K kmax(K a, K b) { return max(a, b); }
  static __device__ __forceinline__ bool good(K p) { return p != 0u && p < 0x7f800000u; }
  static __device__ __forceinline__ bool good(K p, K cm) {
    return good(p) && p + 27866353u >= cm;  // log2(10) * 2^23
  }
};
#endif

constexpr double kVfaCod_ac = 64.0, kVfaCod_pro = 112.0, kVfaCod_bu = 160.0, kVfaCod_va = 208.0;
constexpr double kC4Guard = 1e-6;  // division guard of the c4 uptake split
constexpr double kSH_lo = 1e-14, kSH_hi = 1.0;

template <class T>
struct PartConstT {
  T arr;  // Arrhenius factor of the kinetic constants
  T K_w, K_a_co2, K_a_IN, K_H_co2, K_H_ch4, K_H_h2, p_h2o, RT;
};
using PartConst = PartConstT<double>;
// float copy for FP32 rate evaluations (converted once per particle load
// instead of at every use)
using PartConstF = PartConstT<float>;
CHAD_HD void narrow_pc(const PartConst& q, PartConstF& f) {
  f.arr = float(q.arr);
  f.K_w = float(q.K_w);
  f.K_a_co2 = float(q.K_a_co2);
  f.K_a_IN = float(q.K_a_IN);
  f.K_H_co2 = float(q.K_H_co2);
  f.K_H_ch4 = float(q.K_H_ch4);
  f.K_H_h2 = float(q.K_H_h2);
  f.p_h2o = float(q.p_h2o);
  f.RT = float(q.RT);
}

CHAD_HD void part_const(const DigConst& c, double T, PartConst& q) {
  const double invT = 1.0 / T;
  const double dT = c.inv_T_base - invT;
  q.arr = exp(-c.Ea_over_R * (invT - c.inv_T_ref));
  q.K_w = c.K_w_b * exp(c.th_w * dT);
  q.K_a_co2 = c.K_a_co2_b * exp(c.th_a_co2 * dT);
  q.K_a_IN = c.K_a_IN_b * exp(c.th_a_IN * dT);
  q.K_H_co2 = c.K_H_co2_b * exp(c.th_H_co2 * dT);
  q.K_H_ch4 = c.K_H_ch4_b * exp(c.th_H_ch4 * dT);
  q.K_H_h2 = c.K_H_h2_b * exp(c.th_H_h2 * dT);
  q.p_h2o = c.p_h2o_b * exp(c.th_h2o * dT);
  q.RT = c.R * T;
}

// PartConst in structure-of-arrays form, field f of particle p at
// pc[f * ld + p]: computed once per load (the temperature of a particle is
// fixed while it is loaded) instead of by every lane that takes a new
// particle, which would leave the rest of its warp idle during nine FP64
// exponentials.
CHAD_HD void pc_store(const PartConst& q, double* pc, int64_t ld, int64_t p) {
  pc[0 * ld + p] = q.arr;
  pc[1 * ld + p] = q.K_w;
  pc[2 * ld + p] = q.K_a_co2;
  pc[3 * ld + p] = q.K_a_IN;
  pc[4 * ld + p] = q.K_H_co2;
  pc[5 * ld + p] = q.K_H_ch4;
  pc[6 * ld + p] = q.K_H_h2;
  pc[7 * ld + p] = q.p_h2o;
  pc[8 * ld + p] = q.RT;
}
CHAD_HD void pc_load(const double* pc, int64_t ld, int64_t p, PartConst& q) {
  q.arr = pc[0 * ld + p];
  q.K_w = pc[1 * ld + p];
  q.K_a_co2 = pc[2 * ld + p];
  q.K_a_IN = pc[3 * ld + p];
  q.K_H_co2 = pc[4 * ld + p];
  q.K_H_ch4 = pc[5 * ld + p];
  q.K_H_h2 = pc[6 * ld + p];
  q.p_h2o = pc[7 * ld + p];
  q.RT = pc[8 * ld + p];
}

// ----------------------------------------------------------- Eq. 7 (FP64)
struct AcidBase {
  double SH;     // root
  double dEdS;   // dE/dS_H at the root
  double r_IN, r_co2, r_ac, r_pro, r_bu, r_va;  // 1/(K_a + S_H) at the root
  double rS;     // 1/S_H
};

// E(S) and dE/dS of Eq. 7 from the reciprocals rS = 1/S and r = 1/(K_a + S)
// for IN, co2, ac, pro, bu, va.
template <class F>
CHAD_HD F charge_terms(const DigConst& c, const PartConst& q, const double* y, F S, F rS,
                       const F* r, F& dEdS) {
  const F nh3 = F(q.K_a_IN) * F(y[iS_IN]) * r[0];
  const F hco3 = F(q.K_a_co2) * F(y[iS_IC]) * r[1];
  const F ac = F(c.K_a_ac) * F(y[iS_ac]) * r[2] * F(1.0 / kVfaCod_ac);
  const F pro = F(c.K_a_pro) * F(y[iS_pro]) * r[3] * F(1.0 / kVfaCod_pro);
  const F bu = F(c.K_a_bu) * F(y[iS_bu]) * r[4] * F(1.0 / kVfaCod_bu);
  const F va = F(c.K_a_va) * F(y[iS_va]) * r[5] * F(1.0 / kVfaCod_va);
  const F kw = F(q.K_w) * rS;
  dEdS = F(1.0) + kw * rS + nh3 * r[0] + hco3 * r[1] + ac * r[2] + pro * r[3] + bu * r[4] +
         va * r[5];
  return (F(y[iS_cat]) - F(y[iS_an])) + (F(y[iS_IN]) - nh3) + S - hco3 - ac - pro - bu - va - kw;
}

// E(S) and dE/dS; fills the reciprocals used by the Jacobian.  Templated
// on the scalar type only so that its operations can be counted on the host.
template <class F>
CHAD_HD F charge_E_t(const DigConst& c, const PartConst& q, const double* y, F S, F* r, F& rS,
                     F& dEdS) {
  rS = rcp<F>(S);
  r[0] = rcp<F>(F(q.K_a_IN) + S);
  r[1] = rcp<F>(F(q.K_a_co2) + S);
  r[2] = rcp<F>(F(c.K_a_ac) + S);
  r[3] = rcp<F>(F(c.K_a_pro) + S);
  r[4] = rcp<F>(F(c.K_a_bu) + S);
  r[5] = rcp<F>(F(c.K_a_va) + S);
  return charge_terms<F>(c, q, y, S, rS, r, dEdS);
}

CHAD_HD double charge_E(const DigConst& c, const PartConst& q, const double* y, double S,
                        AcidBase& ab) {
  double r[6];
  const double E = charge_E_t<double>(c, q, y, S, r, ab.rS, ab.dEdS);
  ab.r_IN = r[0];
  ab.r_co2 = r[1];
  ab.r_ac = r[2];
  ab.r_pro = r[3];
  ab.r_bu = r[4];
  ab.r_va = r[5];
  return E;
}

// Move the reciprocals of charge_E_t from S to S + d to first order,
// 1/(K + S + d) = r / (1 + r d) ~ r (1 - r d) with relative error (r d)^2,
// and recompute dE/dS from them.  Templated for operation counting.
template <class F>
CHAD_HD void root_shift_t(const DigConst& c, const PartConst& q, const double* y, F S, F d, F* r,
                          F& rS, F& dEdS) {
  rS = rS - rS * rS * d;
#pragma unroll
  for (int k = 0; k < 6; ++k) r[k] = r[k] - r[k] * r[k] * d;
  charge_terms<F>(c, q, y, S + d, rS, r, dEdS);
}
CHAD_HD void root_shift(const DigConst& c, const PartConst& q, const double* y, AcidBase& ab,
                        double S, double d) {
  double r[6] = {ab.r_IN, ab.r_co2, ab.r_ac, ab.r_pro, ab.r_bu, ab.r_va};
  root_shift_t<double>(c, q, y, S, d, r, ab.rS, ab.dEdS);
  ab.r_IN = r[0];
  ab.r_co2 = r[1];
  ab.r_ac = r[2];
  ab.r_pro = r[3];
  ab.r_bu = r[4];
  ab.r_va = r[5];
}

struct NewtonCounters {
  int iters;
  int fallbacks;
  int failed;
};

// Newton from `guess` without a fallback: true if it converged within
// max_iters with |E| <= max_resid at the returned root (ab then describes it).
// E is increasing and concave, Newton converges quadratically with a
// relative contraction factor below 1 near the root: an update below 1e-8
// relative leaves the new iterate within ~1e-16 of the root.
__host__ __device__ inline bool newton_only(const DigConst& c, const PartConst& q,
                                            const double* y, double guess, int max_iters,
                                            double max_resid, AcidBase& ab, int& iters) {
  double S = (guess > 0.0 && isfinite(guess)) ? guess : 1e-7;
  double prevE = INFINITY;
  for (int it = 0; it < max_iters; ++it) {
    const double E = charge_E(c, q, y, S, ab);
    iters++;
    if (!isfinite(E) || fabs(E) > fabs(prevE)) return false;
    const double dS = E * rcp<double>(ab.dEdS);
    const double Sn = S - dS;
    if (!(Sn > 0.0) || !isfinite(Sn)) return false;
    if (fabs(dS) <= 1e-8 * Sn || fabs(E) <= 1e-15) {
      ab.SH = Sn;
      if (max_resid < INFINITY) {  // a residual bound is asked for: evaluate at the root
        const double Ef = charge_E(c, q, y, Sn, ab);
        return fabs(Ef) <= max_resid || fabs(E) <= max_resid;
      }
      // Otherwise move the reciprocals 1/S and 1/(K_a + S) to the root to
      // first order; |r dS| <= 1e-8, so their relative error (r dS)^2 is at
      // the FP64 rounding level, and dE/dS follows from them.
      root_shift(c, q, y, ab, S, -dS);
      return true;
    }
    prevE = E;
    S = Sn;
  }
  return false;
}

// Newton from `guess`; an iterate leaving (0, inf) or a growing |E| switches
// to bisection on [1e-14, 1] (geometric midpoint, at most 200 halvings).
// The same iterates as newton_only followed by the bisection, written as one
// loop around a single evaluation of Eq. 7: each evaluation inlines seven
// reciprocals, and one copy of it instead of seven keeps the integrator's
// code within reach of the instruction cache.
__host__ __device__ inline void solve_SH(const DigConst& c, const PartConst& q, const double* y,
                                         double guess, int max_iters, AcidBase& ab,
                                         NewtonCounters& nc) {
  enum { kNewton, kLo, kHi, kBisect, kFinal };
  const double start = (guess > 0.0 && isfinite(guess)) ? guess : 1e-7;
  int phase = max_iters > 0 ? kNewton : kLo;
  if (phase == kLo) nc.fallbacks++;
  double S = phase == kNewton ? start : kSH_lo;  // point of the next evaluation
  double prevE = INFINITY, lo = kSH_lo, hi = kSH_hi, elo = 0.0;
  int it = 0;
  for (;;) {
    const double E = charge_E(c, q, y, S, ab);
    if (phase == kFinal) {
      ab.SH = S;
      return;
    }
    if (phase == kNewton) {
      nc.iters++;
      bool fail = !isfinite(E) || fabs(E) > fabs(prevE);
      if (!fail) {
        const double dS = E * rcp<double>(ab.dEdS);
        const double Sn = S - dS;
        fail = !(Sn > 0.0) || !isfinite(Sn);
        if (!fail && (fabs(dS) <= 1e-8 * Sn || fabs(E) <= 1e-15)) {
          // converged: move the reciprocals 1/S and 1/(K_a + S) to the root
          // to first order (|r dS| <= 1e-8: relative error at the FP64
          // rounding level) and dE/dS with them
          ab.SH = Sn;
          root_shift(c, q, y, ab, S, -dS);
          return;
        }
        if (!fail) {
          prevE = E;
          S = Sn;
          fail = ++it >= max_iters;
        }
      }
      if (fail) {
        nc.fallbacks++;
        phase = kLo;
        S = lo;
      }
      continue;
    }
    if (phase == kLo) {
      elo = E;
      phase = kHi;
      S = hi;
      continue;
    }
    if (phase == kHi) {
      if (!(elo < 0.0 && E > 0.0)) {  // no sign change: keep the guess
        nc.failed = 1;
        phase = kFinal;
        S = start;
        continue;
      }
      phase = kBisect;
      it = 0;
    } else {  // kBisect: E at the midpoint S
      ++it;
      if (E == 0.0) {
        lo = hi = S;
      } else if (E < 0.0) {
        lo = S;
      } else {
        hi = S;
      }
    }
    const double mid = sqrt(lo * hi);
    if (lo == hi || it >= 200 || !(mid > lo && mid < hi)) {
      phase = kFinal;
      S = sqrt(lo * hi);
    } else {
      S = mid;
    }
  }
}

// dS_H/dy_k = -(dE/dy_k) / (dE/dS_H) (implicit function theorem on Eq. 7)
// for the 8 states that enter Eq. 7, in the order of kShStates.
constexpr int kShStates[8] = {iS_va, iS_bu, iS_pro, iS_ac, iS_IC, iS_IN, iS_cat, iS_an};
template <class DC, class PQ>
CHAD_HD void sh_tangent(const DC& c, const PQ& q, const AcidBase& ab, double* v) {
  const double inv = -rcp<double>(ab.dEdS);
  v[0] = inv * (-c.K_a_va * ab.r_va * (1.0 / kVfaCod_va));
  v[1] = inv * (-c.K_a_bu * ab.r_bu * (1.0 / kVfaCod_bu));
  v[2] = inv * (-c.K_a_pro * ab.r_pro * (1.0 / kVfaCod_pro));
  v[3] = inv * (-c.K_a_ac * ab.r_ac * (1.0 / kVfaCod_ac));
  v[4] = inv * (-q.K_a_co2 * ab.r_co2);
  v[5] = inv * (ab.SH * ab.r_IN);
  v[6] = inv;
  v[7] = -inv;
}

// ----------------------------------------------------------- inhibition helpers
// Hill pH inhibition I = 1 / (1 + (S/K)^n) and dI/dS
template <class R>
CHAD_HD void hill(R S, R invK, R n, int ni, R& I, R& dI) {
  const R x = S * invK;
  R xn1, xn;
  switch (ni) {
    case 1: xn1 = R(1); xn = x; break;
    case 2: xn1 = x; xn = x * x; break;
    case 3: xn1 = x * x; xn = xn1 * x; break;
    case 4: xn1 = x * x * x; xn = xn1 * x; break;
    default: xn = pow(x, n); xn1 = xn / x; break;
  }
  I = rcp<R>(R(1) + xn);
  dI = -n * xn1 * invK * I * I;
}

// ----------------------------------------------------------- Eq. 8 (FP64)
// S_h2 as an algebraic variable: its mass balance (Eq. 8) as a function of
// S_h2 alone, every other state and S_H fixed.  These are the hydrogen terms
// of rates() and balances() written out: the fa, c4 and pro uptakes carry
// the inhibition K_I/(K_I + S_h2), the hydrogen uptake the Monod factor
// S_h2/(K_S + S_h2), the transfer and the outflow are linear, so
//   E(S) = C0 + P_fa I_fa(S) + P_c4 I_c4(S) + P_pro I_pro(S) - P_h2 M(S) - kD S
// with P >= 0: E decreases in S and the root is unique.
template <class F>
struct H2Bal {
  F C0, Pfa, Pc4, Ppro, Ph2, kD, Kfa, Kc4, Kpro, Kh2;
};

template <class F, class DC, class PQ, class Y>
CHAD_HD void h2_coeffs(const DC& c, const PQ& q, const Y* y, F D, const AcidBase& ab,
                       H2Bal<F>& e) {
  const F a = F(q.arr);
  F Ipaa, dIpaa, Iph2, dIph2;
  hill<F>(F(ab.SH), F(c.inv_K_pH_aa), F(c.n_aa), c.ni_aa, Ipaa, dIpaa);
  hill<F>(F(ab.SH), F(c.inv_K_pH_h2), F(c.n_h2), c.ni_h2, Iph2, dIph2);
  const F S_IN = F(y[iS_IN]);
  const F IIN = S_IN * rcp<F>(S_IN + F(c.K_S_IN));
  const F msu = F(y[iS_su]) * rcp<F>(F(c.K_S_su) + F(y[iS_su]));
  const F maa = F(y[iS_aa]) * rcp<F>(F(c.K_S_aa) + F(y[iS_aa]));
  const F mfa = F(y[iS_fa]) * rcp<F>(F(c.K_S_fa) + F(y[iS_fa]));
  const F mva = F(y[iS_va]) * rcp<F>(F(c.K_S_c4) + F(y[iS_va]));
  const F mbu = F(y[iS_bu]) * rcp<F>(F(c.K_S_c4) + F(y[iS_bu]));
  const F mpo = F(y[iS_pro]) * rcp<F>(F(c.K_S_pro) + F(y[iS_pro]));
  const F rden = rcp<F>(F(y[iS_bu]) + F(y[iS_va]) + F(kC4Guard));
  const F gva = F(y[iS_va]) * rden, gbu = F(y[iS_bu]) * rden;
  const F B5 = Ipaa * IIN, B12 = Iph2 * IIN;
  const F r4 = F(c.k_m_su) * a * F(y[iX_su]) * msu * B5;
  const F r5 = F(c.k_m_aa) * a * F(y[iX_aa]) * maa * B5;
  const F kLa = F(c.k_La);
  const F KH2 = F(q.K_H_h2) * F(q.RT);
  e.C0 = D * F(c.y_in[iS_h2]) + F(c.su_h2) * r4 + F(c.aa_h2) * r5 + kLa * KH2 * F(y[iG_h2]);
  e.Pfa = F(c.fa_h2) * F(c.k_m_fa) * a * F(y[iX_fa]) * mfa * B5;
  e.Pc4 = (F(c.va_h2) * mva * gva + F(c.bu_h2) * mbu * gbu) * F(c.k_m_c4) * a * F(y[iX_c4]) * B5;
  e.Ppro = F(c.pro_h2) * F(c.k_m_pro) * a * F(y[iX_pro]) * mpo * B5;
  e.Ph2 = F(c.k_m_h2) * a * F(y[iX_h2]) * B12;
  e.kD = kLa + D;
  e.Kfa = F(c.K_I_h2_fa);
  e.Kc4 = F(c.K_I_h2_c4);
  e.Kpro = F(c.K_I_h2_pro);
  e.Kh2 = F(c.K_S_h2);
}

// E(S) and dE/dS of Eq. 8 from the coefficients.
template <class F>
CHAD_HD F h2_eval(const H2Bal<F>& e, F S, F& dE) {
  const F rfa = rcp<F>(e.Kfa + S), rc4 = rcp<F>(e.Kc4 + S), rpr = rcp<F>(e.Kpro + S);
  const F rh = rcp<F>(e.Kh2 + S);
  const F Ifa = e.Kfa * rfa, Ic4 = e.Kc4 * rc4, Ipr = e.Kpro * rpr;
  dE = F(0) - (e.Pfa * Ifa * rfa + e.Pc4 * Ic4 * rc4 + e.Ppro * Ipr * rpr +
               e.Ph2 * e.Kh2 * rh * rh + e.kD);
  return e.C0 + e.Pfa * Ifa + e.Pc4 * Ic4 + e.Ppro * Ipr - e.Ph2 * S * rh - e.kD * S;
}

// Root of Eq. 8 by Newton from the guess: an update below 1e-8 relative
// leaves the next iterate within ~1e-16 (quadratic convergence).  An iterate
// leaving (0, inf), a growing |E| or a non-negative slope switches to
// bisection on [0, hi], hi doubled from the guess until E(hi) <= 0 (E
// decreases, and E(0) >= 0: at S = 0 nothing removes hydrogen but the
// transfer from a gas that holds some).
__host__ __device__ inline double solve_h2(const H2Bal<double>& e, double guess, int max_iters,
                                           NewtonCounters& nc) {
  double S = (guess > 0.0 && isfinite(guess)) ? guess : 1e-8;
  double prevE = INFINITY;
  for (int it = 0; it < max_iters; ++it) {
    double dE;
    const double E = h2_eval<double>(e, S, dE);
    nc.iters++;
    if (!isfinite(E) || fabs(E) > fabs(prevE) || !(dE < 0.0)) break;
    const double dS = E * rcp<double>(dE);
    const double Sn = S - dS;
    if (!(Sn > 0.0) || !isfinite(Sn)) break;
    if (fabs(dS) <= 1e-8 * Sn || E == 0.0) return Sn;
    prevE = E;
    S = Sn;
  }
  nc.fallbacks++;
  double lo = 0.0, hi = fmax((guess > 0.0 && isfinite(guess)) ? guess : 0.0, 1e-12), dE;
  int k = 0;
  while (k < 200 && h2_eval<double>(e, hi, dE) > 0.0) {
    hi *= 2.0;
    ++k;
  }
  if (k == 200) {
    nc.failed = 1;
    return (guess > 0.0 && isfinite(guess)) ? guess : 1e-8;
  }
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (!(mid > lo && mid < hi)) break;
    if (h2_eval<double>(e, mid, dE) > 0.0) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

// Rates of the 19 biochemical processes, the 3 transfers and their partial
// derivatives.  Column lists are fixed per process.
template <class R>
struct Rates {
  R r[22];
  // partials (d*) -- only filled by the Jacobian variant
  R d1, d2, d3, d4;                                   // wrt X_c, X_ch, X_pr, X_li
  R d5[3], d6[3], d7[4], d8[5], d9[5], d10[4], d11[3], d12[3];
  R s5, s6, s7, s8, s9, s10, s11, s12;                // wrt S_H
  R ddec[7];
  R dT8[2], dT9[2], dT10[2], sT10;
  R qv, dqv;                                          // q_gas/V_gas, its dP derivative
  R P_h2, P_ch4, P_co2;                               // dP/dG
};

template <class R, bool J, class DC, class PQ>
CHAD_HD void rates(const DC& c, const PQ& q, const R* y, const AcidBase& ab, Rates<R>& o) {
  const R a = R(q.arr);
  const R SH = R(ab.SH);
  // inhibition factors (Eq. 3-6)
  R Ipaa, dIpaa, Ipac, dIpac, Iph2, dIph2;
  hill<R>(SH, R(c.inv_K_pH_aa), R(c.n_aa), c.ni_aa, Ipaa, dIpaa);
  hill<R>(SH, R(c.inv_K_pH_ac), R(c.n_ac), c.ni_ac, Ipac, dIpac);
  hill<R>(SH, R(c.inv_K_pH_h2), R(c.n_h2), c.ni_h2, Iph2, dIph2);
  const R S_IN = y[iS_IN], S_h2 = y[iS_h2];
  const R rIN = rcp<R>(S_IN + R(c.K_S_IN));
  const R IIN = S_IN * rIN;
  const R dIIN = R(c.K_S_IN) * rIN * rIN;
  const R rfa = rcp<R>(R(c.K_I_h2_fa) + S_h2), rc4 = rcp<R>(R(c.K_I_h2_c4) + S_h2);
  const R rpr = rcp<R>(R(c.K_I_h2_pro) + S_h2);
  const R Ih2fa = R(c.K_I_h2_fa) * rfa, Ih2c4 = R(c.K_I_h2_c4) * rc4, Ih2pro = R(c.K_I_h2_pro) * rpr;
  const R r_nh3 = R(q.K_a_IN) * R(ab.r_IN);
  const R nh3 = r_nh3 * S_IN;  // free ammonia
  const R rnh = rcp<R>(R(c.K_I_nh3) + nh3);
  const R Inh3 = R(c.K_I_nh3) * rnh;

  // first-order processes
  const R kdis = R(c.k_dis) * a, kch = R(c.k_hyd_ch) * a, kpr = R(c.k_hyd_pr) * a,
          kli = R(c.k_hyd_li) * a;
  o.r[0] = kdis * y[iX_c];
  o.r[1] = kch * y[iX_ch];
  o.r[2] = kpr * y[iX_pr];
  o.r[3] = kli * y[iX_li];
  // Monod terms m = S/(K+S), dm = K/(K+S)^2
  const R rsu = rcp<R>(R(c.K_S_su) + y[iS_su]), raa = rcp<R>(R(c.K_S_aa) + y[iS_aa]);
  const R rfs = rcp<R>(R(c.K_S_fa) + y[iS_fa]), rva = rcp<R>(R(c.K_S_c4) + y[iS_va]);
  const R rbu = rcp<R>(R(c.K_S_c4) + y[iS_bu]), rpo = rcp<R>(R(c.K_S_pro) + y[iS_pro]);
  const R rac = rcp<R>(R(c.K_S_ac) + y[iS_ac]), rh2 = rcp<R>(R(c.K_S_h2) + S_h2);
  const R msu = y[iS_su] * rsu, maa = y[iS_aa] * raa, mfa = y[iS_fa] * rfs, mva = y[iS_va] * rva;
  const R mbu = y[iS_bu] * rbu, mpo = y[iS_pro] * rpo, mac = y[iS_ac] * rac, mh2 = S_h2 * rh2;
  const R rden = rcp<R>(y[iS_bu] + y[iS_va] + R(kC4Guard));
  const R gva = y[iS_va] * rden, gbu = y[iS_bu] * rden;

  const R ksu = R(c.k_m_su) * a, kaa = R(c.k_m_aa) * a, kfa = R(c.k_m_fa) * a,
          kc4 = R(c.k_m_c4) * a, kpo = R(c.k_m_pro) * a, kac = R(c.k_m_ac) * a,
          kh2 = R(c.k_m_h2) * a;
  const R B5 = Ipaa * IIN;
  const R B7 = B5 * Ih2fa, B8 = B5 * Ih2c4, B10 = B5 * Ih2pro;
  const R B11 = Ipac * IIN * Inh3, B12 = Iph2 * IIN;
  const R A5 = ksu * y[iX_su], A6 = kaa * y[iX_aa], A7 = kfa * y[iX_fa], A8 = kc4 * y[iX_c4];
  const R A10 = kpo * y[iX_pro], A11 = kac * y[iX_ac], A12 = kh2 * y[iX_h2];
  o.r[4] = A5 * msu * B5;
  o.r[5] = A6 * maa * B5;
  o.r[6] = A7 * mfa * B7;
  o.r[7] = A8 * mva * gva * B8;
  o.r[8] = A8 * mbu * gbu * B8;
  o.r[9] = A10 * mpo * B10;
  o.r[10] = A11 * mac * B11;
  o.r[11] = A12 * mh2 * B12;
  R kd[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    kd[k] = R(c.k_dec[k]) * a;
    o.r[12 + k] = kd[k] * y[iX_su + k];
  }
  // gas phase
  const R RT = R(q.RT);
  const R P_h2 = RT * R(1.0 / 16.0), P_ch4 = RT * R(1.0 / 64.0), P_co2 = RT;
  const R P = P_h2 * y[iG_h2] + P_ch4 * y[iG_ch4] + P_co2 * y[iG_co2] + R(q.p_h2o);
  const R kpv = R(c.kp_over_Vgas), invPa = rcp<R>(R(c.P_atm));
  o.qv = kpv * (P - R(c.P_atm)) * P * invPa;
  const R kLa = R(c.k_La);
  const R KH2 = R(q.K_H_h2) * RT, KCH4 = R(q.K_H_ch4) * RT, KCO2 = R(q.K_H_co2) * RT;
  const R rco2 = R(ab.r_co2);
  const R fco2 = SH * rco2;  // S_co2 / S_IC
  o.r[19] = kLa * (S_h2 - KH2 * y[iG_h2]);
  o.r[20] = kLa * (y[iS_ch4] - KCH4 * y[iG_ch4]);
  o.r[21] = kLa * (y[iS_IC] * fco2 - KCO2 * y[iG_co2]);

  if (J) {
    o.d1 = kdis; o.d2 = kch; o.d3 = kpr; o.d4 = kli;
    // rho5: S_su, X_su, S_IN
    o.d5[0] = A5 * (R(c.K_S_su) * rsu * rsu) * B5;
    o.d5[1] = ksu * msu * B5;
    o.d5[2] = A5 * msu * Ipaa * dIIN;
    o.s5 = A5 * msu * dIpaa * IIN;
    // rho6: S_aa, X_aa, S_IN
    o.d6[0] = A6 * (R(c.K_S_aa) * raa * raa) * B5;
    o.d6[1] = kaa * maa * B5;
    o.d6[2] = A6 * maa * Ipaa * dIIN;
    o.s6 = A6 * maa * dIpaa * IIN;
    // rho7: S_fa, X_fa, S_IN, S_h2
    o.d7[0] = A7 * (R(c.K_S_fa) * rfs * rfs) * B7;
    o.d7[1] = kfa * mfa * B7;
    o.d7[2] = A7 * mfa * Ipaa * dIIN * Ih2fa;
    o.d7[3] = -A7 * mfa * B5 * Ih2fa * rfa;   // dI/dS_h2 = -K/(K+S)^2 = -I r
    o.s7 = A7 * mfa * dIpaa * IIN * Ih2fa;
    // rho8, rho9: S_va, S_bu, X_c4, S_IN, S_h2
    const R rd2 = rden * rden;
    const R dgva_va = (y[iS_bu] + R(kC4Guard)) * rd2, dgva_bu = -y[iS_va] * rd2;
    const R dgbu_bu = (y[iS_va] + R(kC4Guard)) * rd2, dgbu_va = -y[iS_bu] * rd2;
    const R dmva = R(c.K_S_c4) * rva * rva, dmbu = R(c.K_S_c4) * rbu * rbu;
    o.d8[0] = A8 * B8 * (dmva * gva + mva * dgva_va);
    o.d8[1] = A8 * B8 * mva * dgva_bu;
    o.d8[2] = kc4 * mva * gva * B8;
    o.d8[3] = A8 * mva * gva * Ipaa * dIIN * Ih2c4;
    o.d8[4] = -A8 * mva * gva * B5 * Ih2c4 * rc4;
    o.s8 = A8 * mva * gva * dIpaa * IIN * Ih2c4;
    o.d9[0] = A8 * B8 * mbu * dgbu_va;
    o.d9[1] = A8 * B8 * (dmbu * gbu + mbu * dgbu_bu);
    o.d9[2] = kc4 * mbu * gbu * B8;
    o.d9[3] = A8 * mbu * gbu * Ipaa * dIIN * Ih2c4;
    o.d9[4] = -A8 * mbu * gbu * B5 * Ih2c4 * rc4;
    o.s9 = A8 * mbu * gbu * dIpaa * IIN * Ih2c4;
    // rho10: S_pro, X_pro, S_IN, S_h2
    o.d10[0] = A10 * (R(c.K_S_pro) * rpo * rpo) * B10;
    o.d10[1] = kpo * mpo * B10;
    o.d10[2] = A10 * mpo * Ipaa * dIIN * Ih2pro;
    o.d10[3] = -A10 * mpo * B5 * Ih2pro * rpr;
    o.s10 = A10 * mpo * dIpaa * IIN * Ih2pro;
    // rho11: S_ac, X_ac, S_IN (I_IN and free ammonia)
    const R dInh3 = -Inh3 * rnh;  // dI_nh3 / dS_nh3
    o.d11[0] = A11 * (R(c.K_S_ac) * rac * rac) * B11;
    o.d11[1] = kac * mac * B11;
    o.d11[2] = A11 * mac * Ipac * (dIIN * Inh3 + IIN * dInh3 * r_nh3);
    o.s11 = A11 * mac * IIN * (dIpac * Inh3 - Ipac * dInh3 * nh3 * R(ab.r_IN));
    // rho12: S_h2, X_h2, S_IN
    o.d12[0] = A12 * (R(c.K_S_h2) * rh2 * rh2) * B12;
    o.d12[1] = kh2 * mh2 * B12;
    o.d12[2] = A12 * mh2 * Iph2 * dIIN;
    o.s12 = A12 * mh2 * dIph2 * IIN;
#pragma unroll
    for (int k = 0; k < 7; ++k) o.ddec[k] = kd[k];
    // transfers
    o.dT8[0] = kLa; o.dT8[1] = -kLa * KH2;
    o.dT9[0] = kLa; o.dT9[1] = -kLa * KCH4;
    o.dT10[0] = kLa * fco2; o.dT10[1] = -kLa * KCO2;
    o.sT10 = kLa * y[iS_IC] * R(q.K_a_co2) * rco2 * rco2;
    o.dqv = kpv * (R(2) * P - R(c.P_atm)) * invPa;
    o.P_h2 = P_h2; o.P_ch4 = P_ch4; o.P_co2 = P_co2;
  }
}

// Stoichiometric part of the mass balances of Eq. 2: f = dil + N r, where
// dil holds the transport terms of every state (liquid: dilution; gas:
// outflow) and N the ADM1 stoichiometry of the 19 processes and the three
// gas transfers (r[19..21]).
// C: type of the stoichiometric coefficients in the products (R itself,
// or float for a two-float accumulator R).
template <class R, class DC, class C = R>
CHAD_HD void stoich(const DC& c, const R* r, const R* dil, R* f) {
  const R dec = r[12] + r[13] + r[14] + r[15] + r[16] + r[17] + r[18];
  f[iS_su] = dil[iS_su] + r[1] + C(c.c_su_li) * r[3] - r[4];
  f[iS_aa] = dil[iS_aa] + r[2] - r[5];
  f[iS_fa] = dil[iS_fa] + C(c.f_fa_li) * r[3] - r[6];
  f[iS_va] = dil[iS_va] + C(c.aa_va) * r[5] - r[7];
  f[iS_bu] = dil[iS_bu] + C(c.su_bu) * r[4] + C(c.aa_bu) * r[5] - r[8];
  f[iS_pro] = dil[iS_pro] + C(c.su_pro) * r[4] + C(c.aa_pro) * r[5] + C(c.va_pro) * r[7] - r[9];
  f[iS_ac] = dil[iS_ac] + C(c.su_ac) * r[4] + C(c.aa_ac) * r[5] + C(c.fa_ac) * r[6] +
             C(c.va_ac) * r[7] + C(c.bu_ac) * r[8] + C(c.pro_ac) * r[9] - r[10];
  f[iS_h2] = dil[iS_h2] + C(c.su_h2) * r[4] + C(c.aa_h2) * r[5] + C(c.fa_h2) * r[6] +
             C(c.va_h2) * r[7] + C(c.bu_h2) * r[8] + C(c.pro_h2) * r[9] - r[11] - r[19];
  f[iS_ch4] = dil[iS_ch4] + C(c.ac_ch4) * r[10] + C(c.h2_ch4) * r[11] - r[20];
  R ic = dil[iS_IC] + C(c.cIC[12]) * dec - r[21];
#pragma unroll
  for (int j = 0; j < 12; ++j) ic += C(c.cIC[j]) * r[j];
  f[iS_IC] = ic;
  R in = dil[iS_IN] + C(c.nIN[0]) * r[0] + C(c.nIN[12]) * dec;
#pragma unroll
  for (int j = 4; j < 12; ++j) in += C(c.nIN[j]) * r[j];
  f[iS_IN] = in;
  f[iS_I] = dil[iS_I] + C(c.f_sI) * r[0];
  f[iX_c] = dil[iX_c] - r[0] + dec;
  f[iX_ch] = dil[iX_ch] + C(c.f_ch) * r[0] - r[1];
  f[iX_pr] = dil[iX_pr] + C(c.f_pr) * r[0] - r[2];
  f[iX_li] = dil[iX_li] + C(c.f_li) * r[0] - r[3];
  f[iX_su] = dil[iX_su] + C(c.Y_su) * r[4] - r[12];
  f[iX_aa] = dil[iX_aa] + C(c.Y_aa) * r[5] - r[13];
  f[iX_fa] = dil[iX_fa] + C(c.Y_fa) * r[6] - r[14];
  f[iX_c4] = dil[iX_c4] + C(c.Y_c4) * (r[7] + r[8]) - r[15];
  f[iX_pro] = dil[iX_pro] + C(c.Y_pro) * r[9] - r[16];
  f[iX_ac] = dil[iX_ac] + C(c.Y_ac) * r[10] - r[17];
  f[iX_h2] = dil[iX_h2] + C(c.Y_h2) * r[11] - r[18];
  f[iX_I] = dil[iX_I] + C(c.f_xI) * r[0];
  f[iS_cat] = dil[iS_cat];
  f[iS_an] = dil[iS_an];
  const C vr = C(c.Vliq_over_Vgas);
  f[iG_h2] = dil[iG_h2] + vr * r[19];
  f[iG_ch4] = dil[iG_ch4] + vr * r[20];
  f[iG_co2] = dil[iG_co2] + vr * r[21];
}

// Multiply every rate partial that enters the Jacobian (and u = df/dS_H) by
// sc.  The FP64 form scales by -g before the Jacobian scatter, which then
// yields -g J_d and -g u directly: W_d = I - g J_d needs only its diagonal
// ones, instead of a multiply per stored slot.
template <class R>
CHAD_HD void scale_partials(Rates<R>& o, R sc) {
  o.d1 *= sc; o.d2 *= sc; o.d3 *= sc; o.d4 *= sc;
#pragma unroll
  for (int k = 0; k < 3; ++k) { o.d5[k] *= sc; o.d6[k] *= sc; o.d11[k] *= sc; o.d12[k] *= sc; }
#pragma unroll
  for (int k = 0; k < 4; ++k) { o.d7[k] *= sc; o.d10[k] *= sc; }
#pragma unroll
  for (int k = 0; k < 5; ++k) { o.d8[k] *= sc; o.d9[k] *= sc; }
  o.s5 *= sc; o.s6 *= sc; o.s7 *= sc; o.s8 *= sc; o.s9 *= sc; o.s10 *= sc; o.s11 *= sc; o.s12 *= sc;
#pragma unroll
  for (int k = 0; k < 7; ++k) o.ddec[k] *= sc;
#pragma unroll
  for (int k = 0; k < 2; ++k) { o.dT8[k] *= sc; o.dT9[k] *= sc; o.dT10[k] *= sc; }
  o.sT10 *= sc;
  o.qv *= sc;
  o.dqv *= sc;
}

// f(y): mass balances of Eq. 2 with the ADM1 stoichiometry
template <class R, class DC>
CHAD_HD void balances(const DC& c, const R* y, R D, const Rates<R>& o, R* f) {
  R dil[NS];
#pragma unroll
  for (int i = 0; i < 26; ++i) dil[i] = D * (R(c.y_in[i]) - y[i]);
  dil[iG_h2] = -y[iG_h2] * o.qv;
  dil[iG_ch4] = -y[iG_ch4] * o.qv;
  dil[iG_co2] = -y[iG_co2] * o.qv;
  stoich<R>(c, o.r, dil, f);
}

// Jacobian-vector product J x = J_d x + u (v^T x) without a matrix: the
// rate partials of rates<RO, true> give the linearised rates
// dr = (d rho / dy) x + (d rho / dS_H) s with s = v^T x, which go through the
// same stoichiometry as the rates; the transport terms are linearised
// directly.  Arithmetic in precision RD (FP64 in the kernels) whatever the
// precision RO of the partials.
template <class RO, class RD, class DC, class C = RD>
CHAD_HD void jvp(const DC& c, const C* y, C D, const Rates<RO>& o, const RD* x, RD s,
                 RD* out) {
  RD dr[22];
  dr[0] = C(o.d1) * x[iX_c];
  dr[1] = C(o.d2) * x[iX_ch];
  dr[2] = C(o.d3) * x[iX_pr];
  dr[3] = C(o.d4) * x[iX_li];
  dr[4] = C(o.d5[0]) * x[iS_su] + C(o.d5[1]) * x[iX_su] + C(o.d5[2]) * x[iS_IN] +
          C(o.s5) * s;
  dr[5] = C(o.d6[0]) * x[iS_aa] + C(o.d6[1]) * x[iX_aa] + C(o.d6[2]) * x[iS_IN] +
          C(o.s6) * s;
  dr[6] = C(o.d7[0]) * x[iS_fa] + C(o.d7[1]) * x[iX_fa] + C(o.d7[2]) * x[iS_IN] +
          C(o.d7[3]) * x[iS_h2] + C(o.s7) * s;
  dr[7] = C(o.d8[0]) * x[iS_va] + C(o.d8[1]) * x[iS_bu] + C(o.d8[2]) * x[iX_c4] +
          C(o.d8[3]) * x[iS_IN] + C(o.d8[4]) * x[iS_h2] + C(o.s8) * s;
  dr[8] = C(o.d9[0]) * x[iS_va] + C(o.d9[1]) * x[iS_bu] + C(o.d9[2]) * x[iX_c4] +
          C(o.d9[3]) * x[iS_IN] + C(o.d9[4]) * x[iS_h2] + C(o.s9) * s;
  dr[9] = C(o.d10[0]) * x[iS_pro] + C(o.d10[1]) * x[iX_pro] +
          C(o.d10[2]) * x[iS_IN] + C(o.d10[3]) * x[iS_h2] + C(o.s10) * s;
  dr[10] = C(o.d11[0]) * x[iS_ac] + C(o.d11[1]) * x[iX_ac] +
           C(o.d11[2]) * x[iS_IN] + C(o.s11) * s;
  dr[11] = C(o.d12[0]) * x[iS_h2] + C(o.d12[1]) * x[iX_h2] +
           C(o.d12[2]) * x[iS_IN] + C(o.s12) * s;
#pragma unroll
  for (int k = 0; k < 7; ++k) dr[12 + k] = C(o.ddec[k]) * x[iX_su + k];
  dr[19] = C(o.dT8[0]) * x[iS_h2] + C(o.dT8[1]) * x[iG_h2];
  dr[20] = C(o.dT9[0]) * x[iS_ch4] + C(o.dT9[1]) * x[iG_ch4];
  dr[21] = C(o.dT10[0]) * x[iS_IC] + C(o.dT10[1]) * x[iG_co2] + C(o.sT10) * s;
  RD dil[NS];
#pragma unroll
  for (int i = 0; i < 26; ++i) dil[i] = -D * x[i];
  const C qv = C(o.qv);
  const RD dq =
      C(o.dqv) * (C(o.P_h2) * x[iG_h2] + C(o.P_ch4) * x[iG_ch4] + C(o.P_co2) * x[iG_co2]);
  dil[iG_h2] = -x[iG_h2] * qv - y[iG_h2] * dq;
  dil[iG_ch4] = -x[iG_ch4] * qv - y[iG_ch4] * dq;
  dil[iG_co2] = -x[iG_co2] * qv - y[iG_co2] * dq;
  stoich<RD, DC, C>(c, dr, dil, out);
}


// J[row][cols[k]] += coef * d[k]; u[row] += coef * s.  Idx maps (row, col)
// to a storage slot (negative: structurally absent, the write is dropped).
template <class Idx, class R, class JS>
CHAD_HD void jadd(JS Jm, int row, int col, R v) {
  const int s = Idx::at(row, col);
  if (s >= 0) Jm[s] += v;
}
template <class Idx, class R, class JS, int NC>
CHAD_HD void scat(JS Jm, R* u, int row, R coef, const int (&cols)[NC], const R (&d)[NC], R s) {
#pragma unroll
  for (int k = 0; k < NC; ++k) jadd<Idx>(Jm, row, cols[k], coef * d[k]);
  u[row] += coef * s;
}
template <class Idx, class R, class JS, int NC>
CHAD_HD void scat(JS Jm, int row, R coef, const int (&cols)[NC], const R (&d)[NC]) {
#pragma unroll
  for (int k = 0; k < NC; ++k) jadd<Idx>(Jm, row, cols[k], coef * d[k]);
}

// Analytic Jacobian (row-major NS x NS) from the rate partials.  The S_H
// dependence enters as the rank-1 term u v^T, u = df/dS_H (at fixed y),
// v = dS_H/dy = -(dE/dy) / (dE/dS_H) from Eq. 7.
// With u_out == nullptr the full J = J_d + u v^T is assembled; otherwise only
// the direct part J_d (S_H held fixed) goes into Jm and u = df/dS_H into
// u_out, for the Sherman-Morrison solve of W = W_d - g u v^T.
template <class Idx, class R, class JS, class DC, class PQ>
CHAD_HD void jacobian(const DC& c, const PQ& q, const R* y, R D, const AcidBase& ab,
                      const Rates<R>& o, JS Jm, R* u_out = nullptr) {
  R u[NS];
#pragma unroll
  for (int i = 0; i < Idx::size; ++i) Jm[i] = R(0);
#pragma unroll
  for (int i = 0; i < NS; ++i) u[i] = R(0);
#pragma unroll
  for (int i = 0; i < 26; ++i) jadd<Idx>(Jm, i, i, -D);
  const R one = R(1), mone = R(-1);
  const R cIC12 = R(c.cIC[12]), nIN12 = R(c.nIN[12]);
  {  // rho1 disintegration
    const int cols[1] = {iX_c};
    const R d[1] = {o.d1};
    scat<Idx>(Jm, iX_c, mone, cols, d);
    scat<Idx>(Jm, iS_I, R(c.f_sI), cols, d);
    scat<Idx>(Jm, iX_ch, R(c.f_ch), cols, d);
    scat<Idx>(Jm, iX_pr, R(c.f_pr), cols, d);
    scat<Idx>(Jm, iX_li, R(c.f_li), cols, d);
    scat<Idx>(Jm, iX_I, R(c.f_xI), cols, d);
    scat<Idx>(Jm, iS_IC, R(c.cIC[0]), cols, d);
    scat<Idx>(Jm, iS_IN, R(c.nIN[0]), cols, d);
  }
  {  // rho2-4 hydrolysis
    const int c2[1] = {iX_ch}, c3[1] = {iX_pr}, c4[1] = {iX_li};
    const R d2[1] = {o.d2}, d3[1] = {o.d3}, d4[1] = {o.d4};
    scat<Idx>(Jm, iX_ch, mone, c2, d2);
    scat<Idx>(Jm, iS_su, one, c2, d2);
    scat<Idx>(Jm, iS_IC, R(c.cIC[1]), c2, d2);
    scat<Idx>(Jm, iX_pr, mone, c3, d3);
    scat<Idx>(Jm, iS_aa, one, c3, d3);
    scat<Idx>(Jm, iS_IC, R(c.cIC[2]), c3, d3);
    scat<Idx>(Jm, iX_li, mone, c4, d4);
    scat<Idx>(Jm, iS_su, R(c.c_su_li), c4, d4);
    scat<Idx>(Jm, iS_fa, R(c.f_fa_li), c4, d4);
    scat<Idx>(Jm, iS_IC, R(c.cIC[3]), c4, d4);
  }
  {  // rho5 sugars
    const int cols[3] = {iS_su, iX_su, iS_IN};
    scat<Idx>(Jm, u, iS_su, mone, cols, o.d5, o.s5);
    scat<Idx>(Jm, u, iS_bu, R(c.su_bu), cols, o.d5, o.s5);
    scat<Idx>(Jm, u, iS_pro, R(c.su_pro), cols, o.d5, o.s5);
    scat<Idx>(Jm, u, iS_ac, R(c.su_ac), cols, o.d5, o.s5);
    scat<Idx>(Jm, u, iS_h2, R(c.su_h2), cols, o.d5, o.s5);
    scat<Idx>(Jm, u, iX_su, R(c.Y_su), cols, o.d5, o.s5);
    scat<Idx>(Jm, u, iS_IC, R(c.cIC[4]), cols, o.d5, o.s5);
    scat<Idx>(Jm, u, iS_IN, R(c.nIN[4]), cols, o.d5, o.s5);
  }
  {  // rho6 amino acids
    const int cols[3] = {iS_aa, iX_aa, iS_IN};
    scat<Idx>(Jm, u, iS_aa, mone, cols, o.d6, o.s6);
    scat<Idx>(Jm, u, iS_va, R(c.aa_va), cols, o.d6, o.s6);
    scat<Idx>(Jm, u, iS_bu, R(c.aa_bu), cols, o.d6, o.s6);
    scat<Idx>(Jm, u, iS_pro, R(c.aa_pro), cols, o.d6, o.s6);
    scat<Idx>(Jm, u, iS_ac, R(c.aa_ac), cols, o.d6, o.s6);
    scat<Idx>(Jm, u, iS_h2, R(c.aa_h2), cols, o.d6, o.s6);
    scat<Idx>(Jm, u, iX_aa, R(c.Y_aa), cols, o.d6, o.s6);
    scat<Idx>(Jm, u, iS_IC, R(c.cIC[5]), cols, o.d6, o.s6);
    scat<Idx>(Jm, u, iS_IN, R(c.nIN[5]), cols, o.d6, o.s6);
  }
  {  // rho7 LCFA
    const int cols[4] = {iS_fa, iX_fa, iS_IN, iS_h2};
    scat<Idx>(Jm, u, iS_fa, mone, cols, o.d7, o.s7);
    scat<Idx>(Jm, u, iS_ac, R(c.fa_ac), cols, o.d7, o.s7);
    scat<Idx>(Jm, u, iS_h2, R(c.fa_h2), cols, o.d7, o.s7);
    scat<Idx>(Jm, u, iX_fa, R(c.Y_fa), cols, o.d7, o.s7);
    scat<Idx>(Jm, u, iS_IC, R(c.cIC[6]), cols, o.d7, o.s7);
    scat<Idx>(Jm, u, iS_IN, R(c.nIN[6]), cols, o.d7, o.s7);
  }
  {  // rho8 valerate
    const int cols[5] = {iS_va, iS_bu, iX_c4, iS_IN, iS_h2};
    scat<Idx>(Jm, u, iS_va, mone, cols, o.d8, o.s8);
    scat<Idx>(Jm, u, iS_pro, R(c.va_pro), cols, o.d8, o.s8);
    scat<Idx>(Jm, u, iS_ac, R(c.va_ac), cols, o.d8, o.s8);
    scat<Idx>(Jm, u, iS_h2, R(c.va_h2), cols, o.d8, o.s8);
    scat<Idx>(Jm, u, iX_c4, R(c.Y_c4), cols, o.d8, o.s8);
    scat<Idx>(Jm, u, iS_IC, R(c.cIC[7]), cols, o.d8, o.s8);
    scat<Idx>(Jm, u, iS_IN, R(c.nIN[7]), cols, o.d8, o.s8);
  }
  {  // rho9 butyrate
    const int cols[5] = {iS_va, iS_bu, iX_c4, iS_IN, iS_h2};
    scat<Idx>(Jm, u, iS_bu, mone, cols, o.d9, o.s9);
    scat<Idx>(Jm, u, iS_ac, R(c.bu_ac), cols, o.d9, o.s9);
    scat<Idx>(Jm, u, iS_h2, R(c.bu_h2), cols, o.d9, o.s9);
    scat<Idx>(Jm, u, iX_c4, R(c.Y_c4), cols, o.d9, o.s9);
    scat<Idx>(Jm, u, iS_IC, R(c.cIC[8]), cols, o.d9, o.s9);
    scat<Idx>(Jm, u, iS_IN, R(c.nIN[8]), cols, o.d9, o.s9);
  }
  {  // rho10 propionate
    const int cols[4] = {iS_pro, iX_pro, iS_IN, iS_h2};
    scat<Idx>(Jm, u, iS_pro, mone, cols, o.d10, o.s10);
    scat<Idx>(Jm, u, iS_ac, R(c.pro_ac), cols, o.d10, o.s10);
    scat<Idx>(Jm, u, iS_h2, R(c.pro_h2), cols, o.d10, o.s10);
    scat<Idx>(Jm, u, iX_pro, R(c.Y_pro), cols, o.d10, o.s10);
    scat<Idx>(Jm, u, iS_IC, R(c.cIC[9]), cols, o.d10, o.s10);
    scat<Idx>(Jm, u, iS_IN, R(c.nIN[9]), cols, o.d10, o.s10);
  }
  {  // rho11 acetate
    const int cols[3] = {iS_ac, iX_ac, iS_IN};
    scat<Idx>(Jm, u, iS_ac, mone, cols, o.d11, o.s11);
    scat<Idx>(Jm, u, iS_ch4, R(c.ac_ch4), cols, o.d11, o.s11);
    scat<Idx>(Jm, u, iX_ac, R(c.Y_ac), cols, o.d11, o.s11);
    scat<Idx>(Jm, u, iS_IC, R(c.cIC[10]), cols, o.d11, o.s11);
    scat<Idx>(Jm, u, iS_IN, R(c.nIN[10]), cols, o.d11, o.s11);
  }
  {  // rho12 hydrogen
    const int cols[3] = {iS_h2, iX_h2, iS_IN};
    scat<Idx>(Jm, u, iS_h2, mone, cols, o.d12, o.s12);
    scat<Idx>(Jm, u, iS_ch4, R(c.h2_ch4), cols, o.d12, o.s12);
    scat<Idx>(Jm, u, iX_h2, R(c.Y_h2), cols, o.d12, o.s12);
    scat<Idx>(Jm, u, iS_IC, R(c.cIC[11]), cols, o.d12, o.s12);
    scat<Idx>(Jm, u, iS_IN, R(c.nIN[11]), cols, o.d12, o.s12);
  }
#pragma unroll
  for (int k = 0; k < 7; ++k) {  // rho13-19 decay
    const int col = iX_su + k;
    const R dk = o.ddec[k];
    jadd<Idx>(Jm, col, col, -dk);
    jadd<Idx>(Jm, (int)iX_c, col, dk);
    jadd<Idx>(Jm, (int)iS_IC, col, cIC12 * dk);
    jadd<Idx>(Jm, (int)iS_IN, col, nIN12 * dk);
  }
  const R vr = R(c.Vliq_over_Vgas);
  {  // transfers
    const int c8[2] = {iS_h2, iG_h2}, c9[2] = {iS_ch4, iG_ch4}, c10[2] = {iS_IC, iG_co2};
    scat<Idx>(Jm, iS_h2, mone, c8, o.dT8);
    scat<Idx>(Jm, iG_h2, vr, c8, o.dT8);
    scat<Idx>(Jm, iS_ch4, mone, c9, o.dT9);
    scat<Idx>(Jm, iG_ch4, vr, c9, o.dT9);
    scat<Idx>(Jm, u, iS_IC, mone, c10, o.dT10, o.sT10);
    scat<Idx>(Jm, u, iG_co2, vr, c10, o.dT10, o.sT10);
  }
  {  // gas outflow: f_G = -G q(P)
    const int g[3] = {iG_h2, iG_ch4, iG_co2};
    const R dP[3] = {o.P_h2, o.P_ch4, o.P_co2};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      jadd<Idx>(Jm, g[a], g[a], -o.qv);
      const R gq = y[g[a]] * o.dqv;
#pragma unroll
      for (int b = 0; b < 3; ++b) jadd<Idx>(Jm, g[a], g[b], -gq * dP[b]);
    }
  }
  if (u_out) {
#pragma unroll
    for (int i = 0; i < NS; ++i) u_out[i] = u[i];
    return;
  }
  // rank-1 S_H coupling: J += u v^T over the 8 states that enter Eq. 7
  const int hc[8] = {iS_va, iS_bu, iS_pro, iS_ac, iS_IC, iS_IN, iS_cat, iS_an};
  double vd[8];
  sh_tangent(c, q, ab, vd);
  R v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = R(vd[k]);
  const int ur[19] = {iS_su, iS_aa, iS_fa, iS_va, iS_bu, iS_pro, iS_ac, iS_h2, iS_ch4, iS_IC,
                      iS_IN, iX_su, iX_aa, iX_fa, iX_c4, iX_pro, iX_ac, iX_h2, iG_co2};
#pragma unroll
  for (int i = 0; i < 19; ++i)
#pragma unroll
    for (int k = 0; k < 8; ++k) jadd<Idx>(Jm, ur[i], hc[k], u[ur[i]] * v[k]);
}

}  // namespace chad
