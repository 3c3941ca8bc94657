// Per-particle stiff integration over one coupling interval (Sec. 2.3: each
// AD particle is integrated independently over every synchronised interval).
//
// Persistent kernel, one particle per thread at a time: a lane pulls the next
// particle from a device queue (warp-aggregated atomic) as soon as its own
// particle has reached the end of the interval, so warps stay full while
// particles take very different numbers of steps (substrate slugs).  The
// warps of a block start every step attempt together (one barrier per
// attempt): the kernel's straight-line code is much larger than the
// instruction cache, and warps at the same place share the fetched lines.
//
// The step is the linearly implicit Rosenbrock 2(3) W-method of Shampine &
// Reichelt (1997): d = 1/(2+sqrt 2), e32 = 6 + sqrt 2, W = I - h d J, three
// stages sharing one LU, embedded error h/6 (k1 - 2 k2 + k3), controller
// fac = min(5, max(0.2, 0.8 e^-1/3)) with growth capped at 1 after a
// rejection, last step clipped to the end of the interval.  S_H+ of Eq. 7 is
// re-solved by FP64 Newton at every rate evaluation.
//
// The Jacobian is split as J = J_d + u v^T (S_H held fixed in J_d; u =
// df/dS_H, v = dS_H/dy from Eq. 7): W_d = I - h d J_d is factored by the
// generated static-order sparse LU (sparse_lu_gen.cuh) and the rank-1 term
// is applied by the Sherman-Morrison formula (rank1.cuh).  A pivot failing
// the threshold test (or a Sherman-Morrison denominator failing the same
// test) rejects the attempt and shrinks h by 4, which moves W towards the
// identity, where the static order is stable.
//
// Forms: FP64 (J, LU, solves in FP64); MIXED (J, LU, solves in FP32, one
// FP64 refinement step r = b - W x per solve, stage rates FP64); MIXED with
// FP32 stage rates.  Newton, state accumulation and error estimate: FP64.
// The refinement residual needs W x = x - g J x: it is formed from the FP32
// rate partials kept from the Jacobian evaluation (jvp), not from a stored
// copy of J.
#pragma once
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <type_traits>

#include "adm1_device.cuh"
#include "kernels.h"
#include "rank1.cuh"
#include "sparse_lu_gen.cuh"
#include "sparse_lu_h2a_gen.cuh"

namespace chad {
namespace integ {

constexpr double kRB_d = 0.29289321881345247559915563789515;   // 1/(2+sqrt 2)
constexpr double kRB_e32 = 7.4142135623730950488016887242097;  // 6+sqrt 2
constexpr double kHmin = 1e-12;                                 // days
constexpr double kHdefault = 1e-6;                              // days
constexpr double kPivTau = 0.1;  // threshold of the Sherman-Morrison denominator test

struct Cnt {
  int acc, rej, newton, fallback, failed, pivot, redo, h2;
};

// The digester constants are read where they are used: an opaque copy of
// their pointer before each evaluation keeps the compiler from hoisting the
// loaded constants out of the stage loop and holding them through the LU
// and the solves (they are the same for every lane of a digester, and the
// loads come back from L1).
template <class T>
__device__ __forceinline__ const T* reread(const T* p) {
  asm volatile("" : "+l"(p));
  return p;
}

__device__ __forceinline__ int64_t queue_pop(unsigned long long* q) {
  const unsigned m = __activemask();
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(q, (unsigned long long)__popc(m));
  base = __shfl_sync(m, base, leader);
  return (int64_t)(base + (unsigned long long)__popc(m & ((1u << lane) - 1u)));
}

__device__ __forceinline__ void newton(const DigConst& c, const PartConst& q, const double* y,
                                       double& SHg, int max_newton, Cnt& cnt, AcidBase& ab) {
  NewtonCounters nc{0, 0, 0};
  solve_SH(c, q, y, SHg, max_newton, ab, nc);
  cnt.newton += nc.iters;
  cnt.fallback += nc.fallbacks;
  cnt.failed |= nc.failed;
  SHg = ab.SH;
}

// S_h2 from Eq. 8 at y (S_H given by ab), Newton from *SH2g, which receives
// the root (algebraic S_h2 form).
__device__ __forceinline__ void newton_h2(const DigConst& c, const PartConst& q, const double* y,
                                          double D, const AcidBase& ab, double* SH2g,
                                          int max_newton, Cnt& cnt) {
  H2Bal<double> e;
  h2_coeffs<double>(c, q, y, D, ab, e);
  NewtonCounters nc{0, 0, 0};
  *SH2g = solve_h2(e, *SH2g, max_newton, nc);
  cnt.h2 += nc.iters;
  cnt.fallback += nc.fallbacks;
  cnt.failed |= nc.failed;
}

// f(y) in precision RS (Newton in FP64).  H2A: S_h2 algebraic (Eq. 8), its
// root in *SH2g (guess in, root out) and a zero S_h2 rate.
template <class RS, bool H2A = false>
__device__ __forceinline__ void eval_f(const DigConst& c, const PartConst& q, const double* y,
                                       double D, double& SHg, int max_newton, Cnt& cnt,
                                       double* f, double* SH2g = nullptr) {
  AcidBase ab;
  newton(c, q, y, SHg, max_newton, cnt, ab);
  RS yr[NS];
#pragma unroll
  for (int i = 0; i < NS; ++i) yr[i] = RS(y[i]);
  if constexpr (H2A) {
    newton_h2(c, q, y, D, ab, SH2g, max_newton, cnt);
    yr[iS_h2] = RS(*SH2g);
  }
  Rates<RS> o;
  rates<RS, false>(c, q, yr, ab, o);
  RS fr[NS];
  balances<RS>(c, yr, RS(D), o, fr);
#pragma unroll
  for (int i = 0; i < NS; ++i) f[i] = double(fr[i]);
  if constexpr (H2A) f[iS_h2] = 0.0;
}

// f(y) in precision RS, J_d (sparse slots) and u = df/dS_H in precision R,
// one Newton solve.  SCALE (FP64 form only, where R is RS): J_d and u come
// out multiplied by jscale (the rate partials are scaled after f is formed).
// IX: the slot map of the Jacobian scatter (sp::Idx; with S_h2 algebraic
// spa::Idx, with w an H2Split that takes S_h2's row and column apart).
// The digester constants in the precision of the Jacobian evaluation.
template <class R>
struct DCSel;
template <>
struct DCSel<double> {
  static __device__ __forceinline__ const DigConst& get(const DigConst& c, const DigConstF*) {
    return c;
  }
};
template <>
struct DCSel<float> {
  static __device__ __forceinline__ const DigConstF& get(const DigConst&, const DigConstF* cf) {
    return *cf;
  }
};

template <class R, class RS, bool SCALE, bool H2A = false, class IX = sp::Idx, class W>
__device__ __forceinline__ void eval_fj(const DigConst& c, const DigConstF* cf, const PartConst& q,
                                        const double* y, double D, double& SHg, int max_newton,
                                        Cnt& cnt, double* f, W w, R* u, Rates<R>& o,
                                        AcidBase& ab, R jscale, double* SH2g = nullptr) {
  const auto& cr = DCSel<R>::get(c, cf);
  newton(c, q, y, SHg, max_newton, cnt, ab);
  if constexpr (H2A) newton_h2(c, q, y, D, ab, SH2g, max_newton, cnt);
  {
    R yr[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) yr[i] = R(y[i]);
    if constexpr (H2A) yr[iS_h2] = R(*SH2g);
    rates<R, true>(cr, q, yr, ab, o);
    if (std::is_same<R, RS>::value) {
      R fr[NS];
      balances<R>(cr, yr, R(D), o, fr);
#pragma unroll
      for (int i = 0; i < NS; ++i) f[i] = double(fr[i]);
      if constexpr (H2A) f[iS_h2] = 0.0;
    }
    if constexpr (SCALE) {
      scale_partials<R>(o, jscale);
      jacobian<IX, R>(cr, q, yr, R(D) * jscale, ab, o, w, u);
    } else {
      jacobian<IX, R>(cr, q, yr, R(D), ab, o, w, u);
    }
  }
  if (!std::is_same<R, RS>::value) {
    RS ys[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) ys[i] = RS(y[i]);
    Rates<RS> o;
    rates<RS, false>(c, q, ys, ab, o);
    RS fr[NS];
    balances<RS>(c, ys, RS(D), o, fr);
#pragma unroll
    for (int i = 0; i < NS; ++i) f[i] = double(fr[i]);
  }
}

// Newton guess for S_H at y + dy from the tangent dS_H/dy at y (Eq. 7
// differentiated implicitly); the root is unchanged, only the start moves.
__device__ __forceinline__ double sh_guess(double SH0, const double* v, const double* y0,
                                           const double* y1) {
  const double g = SH0 + v[0] * (y1[iS_va] - y0[iS_va]) + v[1] * (y1[iS_bu] - y0[iS_bu]) +
                   v[2] * (y1[iS_pro] - y0[iS_pro]) + v[3] * (y1[iS_ac] - y0[iS_ac]) +
                   v[4] * (y1[iS_IC] - y0[iS_IC]) + v[5] * (y1[iS_IN] - y0[iS_IN]) +
                   v[6] * (y1[iS_cat] - y0[iS_cat]) + v[7] * (y1[iS_an] - y0[iS_an]);
  return (g > 0.5 * SH0 && g < 2.0 * SH0) ? g : SH0;
}

// W x = b with the factored W_d and the Sherman-Morrison vector q (the FP64
// form calls it; the mixed form runs the same steps inside its merged stage
// loop).  Mixed: FP32 solve, FP64 residual r = b - x + g J x with J x from
// the kept FP32 rate partials ko at the step's start y, FP32 correction
// solve.
// v: dS_H/dy over the eight states of Eq. 7 in FP64 (residual) and in R
// (rank-1 update).  The FP32<->FP64 conversions here use the hardware
// instructions: there are ~120 per stage, and as integer sequences they
// cost more issue slots than they free on the FP64 pipe.
template <bool MIXED, class R, class LU, class W>
__device__ __forceinline__ void solve(W w, const R* qv, R inv_delta,
                                      const double* v, const R* vr, const DigConst& c,
                                      const double* y, double D, const Rates<R>& ko, double g,
                                      const double* b, double* x) {
  R t[NS];
#pragma unroll
  for (int i = 0; i < NS; ++i) t[i] = R(b[i]);
  LU::template sub<R>(w, t);
  rank1::update<R>(qv, vr, inv_delta, t);
#pragma unroll
  for (int i = 0; i < NS; ++i) x[i] = double(t[i]);
  if (MIXED) {
    double jx[NS];
    jvp<R, double>(c, y, D, ko, x, rank1::vdot<double>(v, x), jx);
#pragma unroll
    for (int i = 0; i < NS; ++i) t[i] = R(b[i] - x[i] + g * jx[i]);
    LU::template sub<R>(w, t);
    rank1::update<R>(qv, vr, inv_delta, t);
#pragma unroll
    for (int i = 0; i < NS; ++i) x[i] += double(t[i]);
  }
}

// Right-hand side of stage st of the W-method (Shampine & Reichelt):
//   st = 0: F0
//   st = 1: F1 - k1 with F1 = f(y + h/2 k1) (F1 kept)
//   st = 2: F2 - e32 (k2 - F1) - 2 (k1 - F0) with F2 = f(y + h k2)
// y1 holds the evaluation point (after st = 2: the new solution y + h k2)
// and SHg its Eq. 7 root.
template <class RS>
__device__ __forceinline__ void stage_rhs(int st, const DigConst& c, const PartConst& q,
                                          const double* y, double D, double hh, double SH0,
                                          const double* vsh, double& SHg, int max_newton,
                                          Cnt& cnt, const double* F0, double* F1,
                                          const double* k1, const double* k2, double* y1,
                                          double* out) {
  if (st == 0) {
#pragma unroll
    for (int i = 0; i < NS; ++i) out[i] = F0[i];
    return;
  }
  // separate loops per stage: a per-element select would evaluate both sides
  if (st == 1) {
    const double h2 = 0.5 * hh;
#pragma unroll
    for (int i = 0; i < NS; ++i) y1[i] = fma(h2, k1[i], y[i]);
  } else {
#pragma unroll
    for (int i = 0; i < NS; ++i) y1[i] = fma(hh, k2[i], y[i]);
  }
  SHg = sh_guess(SH0, vsh, y, y1);
  eval_f<RS>(c, q, y1, D, SHg, max_newton, cnt, out);
  if (st == 1) {
#pragma unroll
    for (int i = 0; i < NS; ++i) {
      F1[i] = out[i];
      out[i] = out[i] - k1[i];
    }
  } else {
#pragma unroll
    for (int i = 0; i < NS; ++i)
      out[i] = out[i] - kRB_e32 * (k2[i] - F1[i]) - 2.0 * (k1[i] - F0[i]);
  }
}

// Slot storage of W_d: a per-thread array (registers / local memory), or
// thread t's column of a [kNNZ][BS] tile in dynamic shared memory (slot s of
// consecutive threads in consecutive words: no bank conflicts).
extern __shared__ __align__(16) unsigned char chad_dyn_smem[];
template <class R, int BS>
struct SmemSlots {
  R* base;
  __device__ __forceinline__ R& operator[](int s) const { return base[s * BS]; }
};
// N: the LU's slots (sp::kNNZ, or spa::kNNZ for the forms with S_h2 algebraic).
template <class R, int BS, bool WS, int N = sp::kNNZ>
struct WStore;
template <class R, int BS, int N>
struct WStore<R, BS, false, N> {
  R a[N];
  __device__ __forceinline__ R* slots() { return a; }
};
template <class R, int BS, int N>
struct WStore<R, BS, true, N> {
  __device__ __forceinline__ SmemSlots<R, BS> slots() {
    return SmemSlots<R, BS>{reinterpret_cast<R*>(chad_dyn_smem) + threadIdx.x};
  }
};
template <class R, int BS, bool WS, int N = sp::kNNZ>
constexpr size_t wstore_smem_bytes() {
  return WS ? sizeof(R) * N * BS : 0;
}

// Storage of the Jacobian scatter for the LU without S_h2 (spa): the LU's
// slots in w, the S_h2 row (slot spa::kNNZ + c) in row[c] and the S_h2
// column (slot spa::kNNZ + NS + r) in col[r].  The slots are compile-time
// constants in the unrolled scatter, so the selection costs nothing.
template <class R, class W>
struct H2Split {
  W w;
  R* row;
  R* col;
  __device__ __forceinline__ R& operator[](int s) const {
    return s < spa::kNNZ ? w[s] : (s < spa::kNNZ + NS ? row[s - spa::kNNZ] : col[s - spa::kNNZ - NS]);
  }
};

// norm^(-1/3) of the step controller
__device__ __forceinline__ float inv_cbrt(float x) { return rcbrtf(x); }
__device__ __forceinline__ double inv_cbrt(double x) { return rcbrt(x); }

template <int FORM, int BS, int MINB, bool WS>
__global__ void __launch_bounds__(BS, MINB) integrate_kernel(StepArgs a) {
  constexpr bool MIXED = FORM == 1 || FORM == 2;
  constexpr bool H2A = FORM == 3;  // FP64 with S_h2 algebraic (Eq. 8)
  using R = typename std::conditional<MIXED, float, double>::type;
  using RS = typename std::conditional<FORM == 2, float, double>::type;
  __shared__ unsigned long long s_acc, s_rej, s_newton, s_fb, s_piv, s_redo, s_h2;
  __shared__ int s_min, s_max;
  if (threadIdx.x == 0) {
    s_acc = s_rej = s_newton = s_fb = s_piv = s_redo = s_h2 = 0ull;
    s_min = INT_MAX;
    s_max = 0;
  }
  __syncthreads();

  // S_h2 algebraic: the LU without S_h2's row and column (spa)
  using LU = typename std::conditional<H2A, spa::Lu, sp::Lu>::type;
  WStore<R, BS, WS, LU::nnz> wst;
  const auto w = wst.slots();
  R qv[NS];  // u = df/dS_H, then q = W_d^-1 (g u)
  Rates<R> ko;  // rates and partials at the step's start (mixed: kept for jvp)
  // algebraic S_h2: second rank-1 pair of W (p2 = W_1^-1 g w with w the S_h2
  // column of J_d, zh = dS_h2/dy) and the running Eq. 8 root
  double p2[H2A ? NS : 1], zh[H2A ? NS : 1];
  double inv_delta2 = 0.0, SH2g = 0.0;
  double y[NS], F0[NS], k1[NS], k2[NS], F1[NS], y1[NS], tmp[NS];
  const double Tend = a.dt_days;
  const bool fixed = a.fixed_n > 0;
  Cnt tot{0, 0, 0, 0, 0, 0, 0};
  int min_steps = INT_MAX, max_steps = 0;

  int64_t p = -1;
  const DigConst* c = nullptr;
  const DigConstF* cf = nullptr;
  PartConst q;
  double SHg = 0.0, h = 0.0, t = 0.0, D = 0.0;
  int status = 0, attempts = 0, nacc = 0;
  bool rejected_prev = false;
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
    // every thread of the block reaches this barrier once per iteration:
    // the block's warps start each attempt together (shared instruction
    // fetch); the loop ends when no thread of the block has a particle
    if (!__syncthreads_or(p >= 0)) break;
    if (p < 0) continue;
    if (fresh) {
      cnt = Cnt{0, 0, 0, 0, 0, 0, 0, 0};
      c = &a.dc[a.dig[p]];
      if constexpr (MIXED) cf = &a.dcf[a.dig[p]];
      pc_load(a.pc, a.ld, p, q);
#pragma unroll
      for (int i = 0; i < NS; ++i) y[i] = a.y[i * a.ld + p];
      SHg = a.SH[p];
      if constexpr (H2A) SH2g = y[iS_h2];
      h = a.h[p];
      if (a.SH_learned && !(h > 0.0 && isfinite(h))) {
        // no step-size history: learned guesses; Newton from the learned
        // S_H is bounded (4 iterations, |E| <= 1e-10) and the plain guess
        // takes over if it fails
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
      D = a.D[p];
      t = 0.0;
      status = 0;
      attempts = 0;
      nacc = 0;
      rejected_prev = false;
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
    AcidBase ab0;
    // FP64: J_d and u come out scaled by -g, so W_d = I + (-g J_d) and
    // q = W_d^-1 (g u) = -W_d^-1 (-g u)
    if constexpr (H2A)
      eval_fj<R, RS, true, true, spa::Idx>(*c, cf, q, y, D, SHg, a.max_newton, cnt, F0,
                                           H2Split<R, decltype(w)>{w, zh, p2}, qv, ko, ab0,
                                           R(-g), &SH2g);
    else
      eval_fj<R, RS, !MIXED>(*c, cf, q, y, D, SHg, a.max_newton, cnt, F0, w, qv, ko, ab0,
                             R(-g));
    const double SH0 = SHg;
    double vsh[8];
    sh_tangent(*c, q, ab0, vsh);
    R vr[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) vr[k] = R(vsh[k]);
    const double SH20 = SH2g;
    if constexpr (H2A) {
      // The S_h2 row of -g J_d (delivered into zh by the scatter) gives
      // dS_h2/dy = -(J_h2,j + u_h2 v_j) / J_h2,h2 (the scale cancels); its
      // column (into p2) times -1 is g w.  Neither is part of W_d (the LU
      // spa runs over the other states, S_h2's row of W_d is the
      // identity's), and u loses its S_h2 entry.  Entries outside the
      // Jacobian's pattern (sp::slot < 0) are zero.
      const double rjj = rcp<double>(zh[iS_h2]);
#pragma unroll
      for (int j = 0; j < NS; ++j)
        zh[j] = (sp::slot(iS_h2, j) >= 0 && j != iS_h2) ? -zh[j] * rjj : 0.0;
      const int hc[8] = {iS_va, iS_bu, iS_pro, iS_ac, iS_IC, iS_IN, iS_cat, iS_an};
#pragma unroll
      for (int k = 0; k < 8; ++k) zh[hc[k]] -= qv[iS_h2] * vsh[k] * rjj;
#pragma unroll
      for (int i = 0; i < NS; ++i) p2[i] = (sp::slot(i, iS_h2) >= 0 && i != iS_h2) ? -p2[i] : 0.0;
      qv[iS_h2] = R(0);
    }
    LU::template form<R>(w, MIXED ? R(g) : R(-1));
    const bool lu_ok = LU::template lu<R>(w);
    R inv_delta = R(0);
    // FP64: q and the Sherman-Morrison denominator here; mixed: in its loop
    const bool sm_ok = MIXED || rank1::setup<R, LU>(w, R(-1), vr, R(kPivTau), qv, &inv_delta);
    bool piv_ok = lu_ok && sm_ok;
    if constexpr (H2A) {
      // p2 = W_1^-1 (g w) with W_1 = W_d - g u v^T (first Sherman-Morrison
      // level), then the second level's denominator 1 - zh^T p2
      LU::template sub<double>(w, p2);
      rank1::update<double>(qv, vr, inv_delta, p2);
      double s2 = 0.0;
#pragma unroll
      for (int j = 0; j < NS; ++j) s2 += zh[j] * p2[j];
      const double delta2 = 1.0 - s2;
      inv_delta2 = rcp<double>(delta2);
      piv_ok = piv_ok && isfinite(delta2) && delta2 != 0.0 &&
               fabs(delta2) >= kPivTau * fmax(1.0, fabs(s2));
    }
    // error norm and controller: FP64 in the FP64 forms, FP32 in the mixed ones
    using NR = typename std::conditional<MIXED, float, double>::type;
    NR norm = NR(INFINITY);
    if (!MIXED && !piv_ok) cnt.pivot++;
    double xs[NS];
    if constexpr (MIXED) {
      // Mixed: one loop over q (st = -1) and the stages, and within a stage
      // two passes, the second with the FP64 residual r = b - x + g J x (J x
      // from the kept FP32 rate partials), so that the kernel holds one copy
      // of the FP32 solve instead of three (the straight-line code is much
      // larger than the instruction cache).  The FP32<->FP64 conversions use
      // the hardware instructions: ~120 per stage, which as integer
      // sequences cost more issue slots than they free on the FP64 pipe.
      if (lu_ok || fixed) {
        R t[NS];
#pragma unroll 1
        for (int st = -1; st < 3; ++st) {
          if (st == -1) {
#pragma unroll
            for (int i = 0; i < NS; ++i) t[i] = R(g) * qv[i];
          } else {
            stage_rhs<RS>(st, *c, q, y, D, hh, SH0, vsh, SHg, a.max_newton, cnt, F0, F1, k1, k2,
                          y1, tmp);
#pragma unroll
            for (int i = 0; i < NS; ++i) t[i] = R(tmp[i]);
          }
          const int npass = st >= 0 ? 2 : 1;
#pragma unroll 1
          for (int pass = 0; pass < npass; ++pass) {
            LU::template sub<R>(w, t);
            if (st < 0) break;
            rank1::update<R>(qv, vr, inv_delta, t);
            if (pass == 0) {
#pragma unroll
              for (int i = 0; i < NS; ++i) xs[i] = double(t[i]);
              double jx[NS];
              jvp<R, double>(*c, y, D, ko, xs, rank1::vdot<double>(vsh, xs), jx);
#pragma unroll
              for (int i = 0; i < NS; ++i) t[i] = R(tmp[i] - xs[i] + g * jx[i]);
            } else {
#pragma unroll
              for (int i = 0; i < NS; ++i) xs[i] += double(t[i]);
            }
          }
          if (st < 0) {
#pragma unroll
            for (int i = 0; i < NS; ++i) qv[i] = t[i];
            piv_ok = lu_ok && rank1::denominator<R>(qv, vr, R(kPivTau), &inv_delta);
            if (!piv_ok && !fixed) break;
            continue;
          }
          if (st == 0) {
#pragma unroll
            for (int i = 0; i < NS; ++i) k1[i] = xs[i];
          } else if (st == 1) {
#pragma unroll
            for (int i = 0; i < NS; ++i) k2[i] = xs[i] + k1[i];
          }
        }
      }
      if (!piv_ok) cnt.pivot++;
    } else if (piv_ok || fixed) {
      // The three stages share one factorisation.  They run as a loop that
      // is not unrolled, so the kernel holds a single copy of the solve and
      // of the rate evaluation (the straight-line code is large):
      //   stage 0: x = W^-1 F0                          -> k1
      //   stage 1: F1 = f(y + h/2 k1), x = W^-1 (F1 - k1) -> k2 = x + k1
      //   stage 2: F2 = f(y + h k2), x = W^-1 (F2 - e32 (k2 - F1) - 2 (k1 - F0))
      //            -> k3 = x (left in xs), y1 = y + h k2
#pragma unroll 1
      for (int st = 0; st < 3; ++st) {
        if (st == 0) {
#pragma unroll
          for (int i = 0; i < NS; ++i) tmp[i] = F0[i];
        } else {
          // separate loops per stage: a per-element select would evaluate both sides
          if (st == 1) {
            const double h2 = 0.5 * hh;
#pragma unroll
            for (int i = 0; i < NS; ++i) y1[i] = fma(h2, k1[i], y[i]);
          } else {
#pragma unroll
            for (int i = 0; i < NS; ++i) y1[i] = fma(hh, k2[i], y[i]);
          }
          SHg = sh_guess(SH0, vsh, y, y1);
          if constexpr (H2A) {
            // tangent guess of the Eq. 8 root at y1
            double g2 = SH20;
#pragma unroll
            for (int j = 0; j < NS; ++j) g2 += zh[j] * (y1[j] - y[j]);
            SH2g = (g2 > 0.5 * SH20 && g2 < 2.0 * SH20) ? g2 : SH20;
            eval_f<RS, true>(*c, q, y1, D, SHg, a.max_newton, cnt, tmp, &SH2g);
          } else {
            eval_f<RS>(*c, q, y1, D, SHg, a.max_newton, cnt, tmp);
          }
          if (st == 1) {
#pragma unroll
            for (int i = 0; i < NS; ++i) {
              F1[i] = tmp[i];
              tmp[i] = tmp[i] - k1[i];
            }
          } else {
#pragma unroll
            for (int i = 0; i < NS; ++i)
              tmp[i] = tmp[i] - kRB_e32 * (k2[i] - F1[i]) - 2.0 * (k1[i] - F0[i]);
          }
        }
        solve<MIXED, R, LU>(w, qv, inv_delta, vsh, vr, *c, y, D, ko, g, tmp, xs);
        if constexpr (H2A) {
          double s2 = 0.0;
#pragma unroll
          for (int j = 0; j < NS; ++j) s2 += zh[j] * xs[j];
          s2 *= inv_delta2;
#pragma unroll
          for (int i = 0; i < NS; ++i) xs[i] += s2 * p2[i];
        }
        if (st == 0) {
#pragma unroll
          for (int i = 0; i < NS; ++i) k1[i] = xs[i];
        } else if (st == 1) {
#pragma unroll
          for (int i = 0; i < NS; ++i) k2[i] = xs[i] + k1[i];
        }
      }
    }
    if (piv_ok || fixed) {
      // scaled error norm max_i |h/6 (k1 - 2 k2 + k3)_i| / (atol_i + rtol
      // max(|y_i|, |y1_i|)).  FP64 forms: all of it in FP64, as the oracle.
      // Mixed forms: the combination, which cancels, in FP64, everything
      // after it in FP32 (the accept test needs a few digits only).
      if constexpr (!MIXED) {
        // the largest ratio |e_i| / sc_i kept as the pair (en, sn), compared
        // by cross products (sc_i > 0), so that one reciprocal suffices
        double en = 0.0, sn = 1.0;
#pragma unroll
        for (int i = 0; i < NS; ++i) {
          const double e = fabs(fma(-2.0, k2[i], k1[i]) + xs[i]);
          const double sc = fma(a.rtol, fmax(fabs(y[i]), fabs(y1[i])), a.atol[i]);
          if (!(e * sn <= en * sc)) {  // NaN propagates as in the ratio form
            en = e;
            sn = sc;
          }
        }
        norm = en * rcp<double>(sn) * (hh * (1.0 / 6.0));
      } else {
        float nf = 0.0f;
        const float rtol = cvt<float>(a.rtol);
#pragma unroll
        for (int i = 0; i < NS; ++i) {
          const float e = cvt<float>(fma(-2.0, k2[i], k1[i]) + xs[i]);
          const float ym = fmaxf(fabsf(cvt<float>(y[i])), fabsf(cvt<float>(y1[i])));
          const float sc = fmaxf(fmaf(rtol, ym, cvt<float>(a.atol[i])), 1e-30f);
          const float r = fabsf(e) * __frcp_rn(sc);
          if (!(r <= nf)) nf = r;  // NaN propagates
        }
        norm = nf * (cvt<float>(hh) * (1.0f / 6.0f));
      }
    }
    if (fixed) {
#pragma unroll
      for (int i = 0; i < NS; ++i) y[i] = y1[i];
      if constexpr (H2A) y[iS_h2] = SH2g;  // Eq. 8 root at y1 (last evaluation)
      cnt.acc++;
      ++nacc;
      if (!isfinite(norm)) status |= ST_NAN;
      if (nacc >= a.fixed_n || (status & ST_NAN)) done = true;
    } else if (norm <= NR(1)) {
#pragma unroll
      for (int i = 0; i < NS; ++i) y[i] = y1[i];
      if constexpr (H2A) y[iS_h2] = SH2g;  // Eq. 8 root at y1 (last evaluation)
      t = last ? Tend : t + hh;
      cnt.acc++;
      ++nacc;
      NR fac = (norm == NR(0)) ? NR(5) : fmin(NR(5), fmax(NR(0.2), NR(0.8) * inv_cbrt(norm)));
      if (rejected_prev) fac = fmin(fac, NR(1));
      h = hh * cvt<double>(fac);
      rejected_prev = false;
      if (last) done = true;
    } else {
      cnt.rej++;
      const NR fac = !piv_ok ? NR(0.25)
                             : (isfinite(norm) ? fmax(NR(0.2), NR(0.8) * inv_cbrt(norm)) : NR(0.2));
      h = hh * cvt<double>(fac);
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
      // on the bit patterns (FP64 compares occupy the FP64 pipe): not
      // finite <=> exponent all ones; y < -atol (atol > 0) <=> y negative
      // with |y| > atol, and non-negative doubles order like their patterns
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

// Launch one kernel variant: persistent grid (resident blocks per SM x SMs,
// capped by the particle count), queue head reset first.
template <int FORM, int BS, int MINB, bool WS>
cudaError_t launch_variant(const StepArgs& a, cudaStream_t s) {
  using R = typename std::conditional<FORM == 1 || FORM == 2, float, double>::type;
  using LU = typename std::conditional<FORM == 3, spa::Lu, sp::Lu>::type;
  constexpr size_t smem = integ::wstore_smem_bytes<R, BS, WS, LU::nnz>();
  static int per_sm = -1, sms = 0;
  if (per_sm < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (smem > 0) {
      cudaError_t e = cudaFuncSetAttribute(integ::integrate_kernel<FORM, BS, MINB, WS>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, integ::integrate_kernel<FORM, BS, MINB, WS>,
                                                  BS, smem);
    if (per_sm < 1) per_sm = 1;
    // the smallest shared carve-out that holds the resident blocks' tiles
    // (none without a tile): the rest of the unified array is L1 for the
    // spilled per-thread state, whatever kernels ran before (a large-tile
    // kernel otherwise leaves the shared share large)
    int smem_sm = 0;
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    const long long need = smem > 0 ? (long long)per_sm * ((long long)smem + 2048) : 0;
    const int pct = smem_sm > 0 ? (int)((need * 100 + smem_sm - 1) / smem_sm) : 100;
    cudaError_t e = cudaFuncSetAttribute(integ::integrate_kernel<FORM, BS, MINB, WS>,
                                         cudaFuncAttributePreferredSharedMemoryCarveout,
                                         pct < 100 ? pct : 100);
    if (e != cudaSuccess) return e;
  }
  int64_t blocks = (int64_t)sms * per_sm;
  const int64_t need = (a.n + BS - 1) / BS;
  if (need < blocks) blocks = need;
  cudaError_t e = cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  integ::integrate_kernel<FORM, BS, MINB, WS><<<(unsigned)blocks, BS, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace chad
