// Per-particle stiff integration over one coupling interval (Sec. 2.3: each
// AD particle is integrated independently over every synchronised interval).
//
// One thread owns one particle.  The step is the linearly implicit
// Rosenbrock 2(3) W-method of Shampine & Reichelt (1997): d = 1/(2+sqrt 2),
// e32 = 6 + sqrt 2, W = I - h d J, three stages sharing one LU, embedded
// error h/6 (k1 - 2 k2 + k3), controller fac = min(5, max(0.2, 0.8 e^-1/3))
// with growth capped at 1 after a rejection, last step clipped to the end of
// the interval.  The S_H+ of Eq. 7 is re-solved (FP64 Newton) at every rate
// evaluation.
//
// Plain form (R = double): rates, Jacobian and LU in FP64.
// Mixed form (R = float): rates, Jacobian and LU in FP32; every linear solve
// is followed by one FP64 refinement step r = b - W x; Newton, the state
// accumulation and the error estimate stay FP64.
#include <cuda_runtime.h>

#include <cstdint>

#include "adm1_device.cuh"
#include "kernels.h"

namespace chad {

namespace {

constexpr double kRB_d = 0.29289321881345247559915563789515;   // 1/(2+sqrt 2)
constexpr double kRB_e32 = 7.4142135623730950488016887242097;  // 6+sqrt 2
constexpr double kHmin = 1e-12;                                 // days
constexpr double kHdefault = 1e-6;                              // days

struct Cnt {
  int acc, rej, newton, fallback, failed;
};

// Gaussian elimination with partial pivoting (lowest row wins ties),
// row-major, in place; dinv receives 1/U_kk.
template <class R>
__device__ bool lu_factor(R* A, int* piv, R* dinv) {
#pragma unroll 1
  for (int k = 0; k < NS; ++k) {
    int p = k;
    R best = fabs(A[k * NS + k]);
    for (int i = k + 1; i < NS; ++i) {
      const R v = fabs(A[i * NS + k]);
      if (v > best) { best = v; p = i; }
    }
    piv[k] = p;
    if (!(best > R(0)) || !isfinite(best)) return false;
    if (p != k) {
      for (int j = 0; j < NS; ++j) {
        const R t = A[k * NS + j];
        A[k * NS + j] = A[p * NS + j];
        A[p * NS + j] = t;
      }
    }
    const R inv = R(1) / A[k * NS + k];
    dinv[k] = inv;
    for (int i = k + 1; i < NS; ++i) {
      const R l = A[i * NS + k] * inv;
      A[i * NS + k] = l;
      for (int j = k + 1; j < NS; ++j) A[i * NS + j] -= l * A[k * NS + j];
    }
  }
  return true;
}

template <class R>
__device__ void lu_solve(const R* LU, const int* piv, const R* dinv, R* b) {
#pragma unroll 1
  for (int k = 0; k < NS; ++k) {
    const int p = piv[k];
    if (p != k) { const R t = b[k]; b[k] = b[p]; b[p] = t; }
  }
#pragma unroll 1
  for (int i = 1; i < NS; ++i) {
    R s = b[i];
    for (int j = 0; j < i; ++j) s -= LU[i * NS + j] * b[j];
    b[i] = s;
  }
#pragma unroll 1
  for (int i = NS - 1; i >= 0; --i) {
    R s = b[i];
    for (int j = i + 1; j < NS; ++j) s -= LU[i * NS + j] * b[j];
    b[i] = s * dinv[i];
  }
}

// rates at y (FP64 in), S_H solved in FP64; f returned in FP64
template <class R>
__device__ __forceinline__ void eval_f(const DigConst& c, const PartConst& q, const double* y,
                                       double D, double& SHg, int max_newton, Cnt& cnt,
                                       double* f) {
  AcidBase ab;
  NewtonCounters nc{0, 0, 0};
  solve_SH(c, q, y, SHg, max_newton, ab, nc);
  cnt.newton += nc.iters;
  cnt.fallback += nc.fallbacks;
  cnt.failed |= nc.failed;
  SHg = ab.SH;
  R yr[NS];
#pragma unroll
  for (int i = 0; i < NS; ++i) yr[i] = R(y[i]);
  Rates<R> o;
  rates<R, false>(c, q, yr, ab, o);
  R fr[NS];
  balances<R>(c, yr, R(D), o, fr);
#pragma unroll
  for (int i = 0; i < NS; ++i) f[i] = double(fr[i]);
}

template <class R>
__device__ __forceinline__ void eval_fj(const DigConst& c, const PartConst& q, const double* y,
                                        double D, double& SHg, int max_newton, Cnt& cnt,
                                        double* f, R* Jm) {
  AcidBase ab;
  NewtonCounters nc{0, 0, 0};
  solve_SH(c, q, y, SHg, max_newton, ab, nc);
  cnt.newton += nc.iters;
  cnt.fallback += nc.fallbacks;
  cnt.failed |= nc.failed;
  SHg = ab.SH;
  R yr[NS];
#pragma unroll
  for (int i = 0; i < NS; ++i) yr[i] = R(y[i]);
  Rates<R> o;
  rates<R, true>(c, q, yr, ab, o);
  R fr[NS];
  balances<R>(c, yr, R(D), o, fr);
#pragma unroll
  for (int i = 0; i < NS; ++i) f[i] = double(fr[i]);
  jacobian<R>(c, q, yr, R(D), ab, o, Jm);
}

// Linear solve W x = b with the factored W.  Mixed form: FP32 solve plus one
// FP64 refinement step using the kept FP32 Jacobian (W = I - g J).
template <bool MIXED, class R>
__device__ __forceinline__ void solve(const R* LU, const int* piv, const R* dinv, const R* Jk,
                                      double g, const double* b, double* x) {
  R t[NS];
#pragma unroll
  for (int i = 0; i < NS; ++i) t[i] = R(b[i]);
  lu_solve<R>(LU, piv, dinv, t);
#pragma unroll
  for (int i = 0; i < NS; ++i) x[i] = double(t[i]);
  if (MIXED) {
    // r = b - W x = b - x + g J x, in FP64
#pragma unroll 1
    for (int i = 0; i < NS; ++i) {
      double s = 0.0;
      for (int k = 0; k < NS; ++k) s = fma(double(Jk[i * NS + k]), x[k], s);
      t[i] = R(b[i] - x[i] + g * s);
    }
    lu_solve<R>(LU, piv, dinv, t);
#pragma unroll
    for (int i = 0; i < NS; ++i) x[i] += double(t[i]);
  }
}

template <bool MIXED>
__device__ int integrate_particle(const DigConst& c, const PartConst& q, double* y,
                                  double& SHg, double& h_io, double D, const StepArgs& a,
                                  Cnt& cnt) {
  using R = typename std::conditional<MIXED, float, double>::type;
  R Jm[NS * NS];                    // J, then W and its LU factors
  R Jk[MIXED ? NS * NS : 1];        // mixed: J kept for the refinement residual
  R dinv[NS];
  int piv[NS];
  double F0[NS], k1[NS], k2[NS], F1[NS], y1[NS], tmp[NS];
  int status = 0;
  const double Tend = a.dt_days;
  double t = 0.0;
  double h = (h_io > 0.0 && isfinite(h_io)) ? h_io : kHdefault;
  bool rejected_prev = false;
  int attempts = 0;
  const bool fixed = a.fixed_n > 0;
  if (fixed) h = Tend / a.fixed_n;
  int fixed_done = 0;
  while (fixed ? (fixed_done < a.fixed_n) : (t < Tend)) {
    if (!fixed && attempts >= a.max_steps) { status |= ST_STEPS; break; }
    ++attempts;
    double hh = h;
    bool last = false;
    if (!fixed && hh >= (Tend - t) * (1.0 - 1e-12)) { hh = Tend - t; last = true; }
    // F0 and J at the start of the step
    eval_fj<R>(c, q, y, D, SHg, a.max_newton, cnt, F0, Jm);
    const double g = hh * kRB_d;
    const R gr = R(g);
#pragma unroll 1
    for (int i = 0; i < NS; ++i)
      for (int j = 0; j < NS; ++j) {
        const R jij = Jm[i * NS + j];
        if (MIXED) Jk[i * NS + j] = jij;
        Jm[i * NS + j] = (i == j ? R(1) : R(0)) - gr * jij;
      }
    double norm;
    if (!lu_factor<R>(Jm, piv, dinv)) {
      norm = INFINITY;
      status |= fixed ? ST_NAN : 0;
    } else {
      solve<MIXED, R>(Jm, piv, dinv, Jk, g, F0, k1);
#pragma unroll
      for (int i = 0; i < NS; ++i) tmp[i] = y[i] + 0.5 * hh * k1[i];
      eval_f<R>(c, q, tmp, D, SHg, a.max_newton, cnt, F1);
#pragma unroll
      for (int i = 0; i < NS; ++i) tmp[i] = F1[i] - k1[i];
      solve<MIXED, R>(Jm, piv, dinv, Jk, g, tmp, k2);
#pragma unroll
      for (int i = 0; i < NS; ++i) {
        k2[i] += k1[i];
        y1[i] = y[i] + hh * k2[i];
      }
      eval_f<R>(c, q, y1, D, SHg, a.max_newton, cnt, tmp);  // F2
#pragma unroll
      for (int i = 0; i < NS; ++i)
        tmp[i] = tmp[i] - kRB_e32 * (k2[i] - F1[i]) - 2.0 * (k1[i] - F0[i]);
      solve<MIXED, R>(Jm, piv, dinv, Jk, g, tmp, F1);  // k3 (F1 no longer needed)
      norm = 0.0;
      const double h6 = hh / 6.0;
#pragma unroll
      for (int i = 0; i < NS; ++i) {
        const double e = h6 * (k1[i] - 2.0 * k2[i] + F1[i]);
        const double sc = a.atol[i] + a.rtol * fmax(fabs(y[i]), fabs(y1[i]));
        const double r = fabs(e) / sc;
        if (!(r <= norm)) norm = r;  // NaN propagates
      }
    }
    if (fixed) {
#pragma unroll
      for (int i = 0; i < NS; ++i) y[i] = y1[i];
      ++fixed_done;
      cnt.acc++;
      if (!isfinite(norm)) { status |= ST_NAN; break; }
      continue;
    }
    if (norm <= 1.0) {
#pragma unroll
      for (int i = 0; i < NS; ++i) y[i] = y1[i];
      t = last ? Tend : t + hh;
      cnt.acc++;
      double fac = (norm == 0.0) ? 5.0 : fmin(5.0, fmax(0.2, 0.8 * pow(norm, -1.0 / 3.0)));
      if (rejected_prev) fac = fmin(fac, 1.0);
      h = hh * fac;
      rejected_prev = false;
    } else {
      cnt.rej++;
      const double fac = isfinite(norm) ? fmax(0.2, 0.8 * pow(norm, -1.0 / 3.0)) : 0.2;
      h = hh * fac;
      rejected_prev = true;
      if (h < kHmin) { status |= ST_HMIN; break; }
    }
  }
  if (!fixed) h_io = h;
  if (cnt.failed) status |= ST_NEWTON;
#pragma unroll
  for (int i = 0; i < NS; ++i)
    if (!isfinite(y[i])) status |= ST_NAN;
#pragma unroll
  for (int i = 0; i < NS; ++i)
    if (y[i] < -a.atol[i]) status |= ST_NEG;
  return status;
}

template <bool MIXED>
__global__ void __launch_bounds__(128) integrate_kernel(StepArgs a) {
  __shared__ unsigned long long s_acc, s_rej, s_newton, s_fb;
  __shared__ int s_min, s_max;
  if (threadIdx.x == 0) {
    s_acc = s_rej = s_newton = s_fb = 0ull;
    s_min = 0x7fffffff;
    s_max = 0;
  }
  __syncthreads();
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < a.n) {
    const DigConst& c = a.dc[a.dig[p]];
    PartConst q;
    part_const(c, a.T[p], q);
    double y[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) y[i] = a.y[i * a.ld + p];
    double SHg = a.SH[p], h = a.h[p];
    Cnt cnt{0, 0, 0, 0, 0};
    const int st = integrate_particle<MIXED>(c, q, y, SHg, h, a.D[p], a, cnt);
#pragma unroll
    for (int i = 0; i < NS; ++i) a.y[i * a.ld + p] = y[i];
    a.SH[p] = SHg;
    a.h[p] = h;
    if (st) a.status[p] |= st;
    atomicAdd(&s_acc, (unsigned long long)cnt.acc);
    atomicAdd(&s_rej, (unsigned long long)cnt.rej);
    atomicAdd(&s_newton, (unsigned long long)cnt.newton);
    atomicAdd(&s_fb, (unsigned long long)cnt.fallback);
    atomicMin(&s_min, cnt.acc);
    atomicMax(&s_max, cnt.acc);
  }
  __syncthreads();
  if (threadIdx.x == 0 && a.counters) {
    atomicAdd(&a.counters->accepted, s_acc);
    atomicAdd(&a.counters->rejected, s_rej);
    atomicAdd(&a.counters->newton_iters, s_newton);
    atomicAdd(&a.counters->newton_fallbacks, s_fb);
    if (s_max > 0 || s_min != 0x7fffffff) {
      atomicMin(&a.counters->min_steps, s_min);
      atomicMax(&a.counters->max_steps, s_max);
    }
  }
}

}  // namespace

cudaError_t launch_integrate(const StepArgs& a, bool mixed, int block, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  block = 128;
  const int64_t grid = (a.n + block - 1) / block;
  if (mixed)
    integrate_kernel<true><<<(unsigned)grid, block, 0, s>>>(a);
  else
    integrate_kernel<false><<<(unsigned)grid, block, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace chad
