// Algorithmic operation counts of the integrator, taken from the kernel
// source itself: the templated model and linear-algebra routines are run on
// the host with a scalar type that counts every +, -, *, / (an FMA counts as
// two).  Comparisons, conversions and the per-interval temperature setup are
// not counted.  These counts are the numerator of the roofline.
#include <cstdint>
#include <cstring>

#include "adm1_device.cuh"
#include "chad.h"
#include "model.h"
#include "rank1.cuh"
#include "sparse_lu_gen.cuh"
#include "sparse_lu_h2a_gen.cuh"

namespace chad {
namespace {

// Counting scalar.  The operations are marked host-device only so that the
// host-device model templates accept them; they run on the host alone.
int64_t g_ops = 0;
#define HD __host__ __device__
struct Fc {
  double v;
  HD Fc() : v(0) {}
  HD Fc(double x) : v(x) {}
};
#ifdef __CUDA_ARCH__
#define CNT
#else
#define CNT ++g_ops;
#endif
HD inline Fc operator+(Fc a, Fc b) { CNT return Fc(a.v + b.v); }
HD inline Fc operator-(Fc a, Fc b) { CNT return Fc(a.v - b.v); }
HD inline Fc operator*(Fc a, Fc b) { CNT return Fc(a.v * b.v); }
HD inline Fc operator/(Fc a, Fc b) { CNT return Fc(a.v / b.v); }
HD inline Fc operator-(Fc a) { return Fc(-a.v); }
HD inline Fc& operator+=(Fc& a, Fc b) { a = a + b; return a; }
HD inline Fc& operator-=(Fc& a, Fc b) { a = a - b; return a; }
HD inline Fc& operator*=(Fc& a, Fc b) { a = a * b; return a; }
HD inline bool operator>=(Fc a, Fc b) { return a.v >= b.v; }
HD inline bool operator!=(Fc a, Fc b) { return a.v != b.v; }
HD inline Fc fabs(Fc a) { return Fc(a.v < 0 ? -a.v : a.v); }
HD inline Fc fmax(Fc a, Fc b) { return Fc(a.v > b.v ? a.v : b.v); }
HD inline Fc pow(Fc a, Fc b) { CNT return Fc(::pow(a.v, b.v)); }
HD inline bool isfinite(Fc a) { return ::isfinite(a.v); }

// Two-float accumulator with the operation counts of the kernel's DF type
// (dfloat.cuh), in FP32 flops (an FMA counts as two): a sum of two
// accumulators is TwoSum (6) plus the sum of the low parts (2); a product of
// a float coefficient and an accumulator is TwoProd (a product and an FMA,
// 3) plus an FMA for the low part (2).
struct DFc {
  double v;
  HD DFc() : v(0) {}
  HD DFc(double x) : v(x) {}
};
#ifdef __CUDA_ARCH__
#define CNT_N(k)
#else
#define CNT_N(k) g_ops += (k);
#endif
HD inline DFc operator+(DFc a, DFc b) { CNT_N(8) return DFc(a.v + b.v); }
HD inline DFc operator-(DFc a, DFc b) { CNT_N(8) return DFc(a.v - b.v); }
HD inline DFc operator-(DFc a) { return DFc(-a.v); }
HD inline DFc operator*(Fc c, DFc a) { CNT_N(5) return DFc(c.v * a.v); }
HD inline DFc operator*(DFc a, Fc c) { CNT_N(5) return DFc(c.v * a.v); }
HD inline DFc& operator+=(DFc& a, DFc b) { a = a + b; return a; }

}  // namespace
}  // namespace chad

using namespace chad;

// out[0] rate vector f (rates + mass balances)
// out[1] rate vector with rate partials, J_d and u (split Jacobian)
// out[2] one charge-balance evaluation E(S_H), dE/dS_H
// out[3] W_d = I - g J_d over the sparse slots
// out[4] sparse LU factorisation of W_d
// out[5] one sparse forward/back solve
// out[6] J x from the rate partials (jvp; mixed refinement residual)
// out[7] stage combinations and error norm of one W-method attempt
// out[8] refinement update of one mixed solve (besides J x)
// out[9] Sherman-Morrison set-up of one attempt (besides its solve)
// out[10] Sherman-Morrison update of one solve
// out[11] move of the acid-base reciprocals to a converged Newton root
// out[12] scaling of the rate partials by -g (FP64 form's W formation)
// With n >= 18, the mixed form with S_h2 algebraic (kernel form 4) also:
// out[13] J x from the FP32 rate partials in two-float arithmetic (FP32 flops)
// out[14] coefficients of the Eq. 8 balance (h2_coeffs)
// out[15] one Eq. 8 Newton iteration (h2_eval + update)
// out[16] FP32 work of one attempt besides rates, LU, solves, J x and Eq. 8
// out[17] FP64 work of one attempt besides the Eq. 7 Newton iterations
// With n >= 19: out[18] the rates with their partials alone (rates<., true>).
extern "C" chad_status chad_flop_counts(int64_t* out, int n) {
  if (!out || n < 13) return CHAD_E_INVALID;
  DigConst c;
  std::memset(&c, 0, sizeof(c));
  c.ni_aa = 2;
  c.ni_ac = 3;
  c.ni_h2 = 3;
  c.n_aa = 2;
  c.n_ac = 3;
  c.n_h2 = 3;
  c.inv_K_pH_aa = c.inv_K_pH_ac = c.inv_K_pH_h2 = 1.0;
  c.K_S_IN = c.K_S_su = c.K_S_aa = c.K_S_fa = c.K_S_c4 = c.K_S_pro = c.K_S_ac = c.K_S_h2 = 1.0;
  c.K_I_h2_fa = c.K_I_h2_c4 = c.K_I_h2_pro = c.K_I_nh3 = 1.0;
  c.P_atm = 1.0;
  PartConst q;
  std::memset(&q, 0, sizeof(q));
  q.arr = 1.0;
  AcidBase ab;
  std::memset(&ab, 0, sizeof(ab));
  ab.SH = 1e-7;
  ab.dEdS = 1.0;
  double yd[NS];
  Fc y[NS], f[NS];
  for (int i = 0; i < NS; ++i) { yd[i] = 1.0; y[i] = Fc(1.0); }
  Rates<Fc> o;
  g_ops = 0;
  rates<Fc, false>(c, q, y, ab, o);
  balances<Fc>(c, y, Fc(0.1), o, f);
  out[0] = g_ops;
  static Fc w[sp::kNNZ];
  Fc u[NS];
  g_ops = 0;
  rates<Fc, true>(c, q, y, ab, o);
  balances<Fc>(c, y, Fc(0.1), o, f);
  jacobian<sp::Idx, Fc>(c, q, y, Fc(0.1), ab, o, w, u);
  out[1] = g_ops;
  Fc r[6], rS, dE;
  g_ops = 0;
  charge_E_t<Fc>(c, q, yd, Fc(1e-7), r, rS, dE);
  out[2] = g_ops;
  for (int s = 0; s < sp::kNNZ; ++s) w[s] = Fc(0.0);
  g_ops = 0;
  sp::form_w<Fc>(w, Fc(1e-4));
  out[3] = g_ops;
  g_ops = 0;
  sp::factor<Fc>(w);
  out[4] = g_ops;
  Fc b[NS];
  for (int i = 0; i < NS; ++i) b[i] = Fc(1.0);
  g_ops = 0;
  sp::solve<Fc>(w, b);
  out[5] = g_ops;
  {
    Fc x[NS], jx[NS];
    for (int i = 0; i < NS; ++i) x[i] = Fc(1.0);
    g_ops = 0;
    jvp<Fc, Fc>(c, y, Fc(0.1), o, x, Fc(1.0), jx);
    out[6] = g_ops;
  }
  const Fc v[8] = {1, 1, 1, 1, 1, 1, 1, 1};
  Fc inv_delta;
  for (int i = 0; i < NS; ++i) u[i] = Fc(1.0);
  g_ops = 0;
  rank1::setup<Fc>(w, Fc(1e-4), v, Fc(0.1), u, &inv_delta);
  out[9] = g_ops - out[5];
  g_ops = 0;
  rank1::update<Fc>(u, v, inv_delta, b);
  out[10] = g_ops;
  g_ops = 0;
  root_shift_t<Fc>(c, q, yd, Fc(1e-7), Fc(1e-16), r, rS, dE);
  out[11] = g_ops;
  g_ops = 0;
  scale_partials<Fc>(o, Fc(-1e-4));
  out[12] = g_ops;
  // y + h/2 k1 (2/elt), F1 - k1 (1), k2 += k1 (1), y + h k2 (2), F2 - e32 (k2 - F1)
  // - 2 (k1 - F0) (5), h/6 (k1 - 2 k2 + k3) (4), atol + rtol max(..) (2), |e|/sc (1)
  out[7] = (int64_t)NS * 18;
  // s = v^T x (15), b - x + g jx (3/elt), x += dx (1/elt)
  out[8] = 15 + (int64_t)NS * 4;
  if (n >= 18) {
    {
      DFc x[NS], jx[NS];
      Fc ys[NS];
      for (int i = 0; i < NS; ++i) { x[i] = DFc(1.0); ys[i] = Fc(1.0); }
      g_ops = 0;
      jvp<Fc, DFc, DigConst, Fc>(c, ys, Fc(0.1), o, x, DFc(1.0), jx);
      out[13] = g_ops;
    }
    {
      H2Bal<Fc> e;
      g_ops = 0;
      h2_coeffs<Fc>(c, q, y, Fc(0.1), ab, e);
      out[14] = g_ops;
      e.Kfa = e.Kc4 = e.Kpro = e.Kh2 = Fc(1.0);
      Fc dE;
      g_ops = 0;
      h2_eval<Fc>(e, Fc(1e-6), dE);
      out[15] = g_ops + 2;  // + the Newton update S - E/E'
    }
    // FP32 flops of one form-4 attempt outside the counted blocks, from the
    // kernel source (two-float operations at their FP32 cost: TwoSum 6,
    // TwoProd 3, a sum with a float 10, a sum 11, a product 10, a product
    // with a float 8):
    //   S_h2 surgery of J_d: zh (29 + 3 x 8), p2 (29), its reciprocal (1)   83
    //   q scaling (29), second-level dot and denominator (58 + 3)           90
    //   per stage (x3): two wsolve level-2 updates (2 x (58 + 1 + 58)),
    //     x'_h2 = zh^T x (28 x 13), v^T x (8 x 13), residual b - x + g J x
    //     (29 x 32), x = x0 + dx (29)                          234 + 364 + 104 + 928 + 29
    //   k2 = x + k1 (29); right-hand sides: stage 1 (29 x 17 with
    //     C = e32 F1 + 2 F0), stage 2 (29 x 40), stage-1 float point (29 x 2)
    //   error norm: k1 - 2 k2 + k3 exact (17), hi + lo (1), scale (4)   29 x 22
    out[16] = 83 + 90 + 3 * (234 + 28 * 13 + 8 * 13 + (int64_t)NS * 32 + NS) + NS +
              (int64_t)NS * (17 + 40 + 2) + (int64_t)NS * 22;
    // FP64 flops of one form-4 attempt besides the Eq. 7 iterations (and the
    // three root moves, counted with them): evaluation points y + (h/2) k1 in
    // the 8 states of Eq. 7 and y + h k2 in all 29 (one FMA each), the two
    // tangent guesses of S_H (24 each), the tangent dS_H/dy (20) and g, h/2
    out[17] = 8 * 2 + (int64_t)NS * 2 + 2 * 24 + 20 + 2;
  }
  if (n >= 19) {
    // out[18] rates with their partials alone (no balances, no Jacobian):
    // the form-4 refinement residual recomputes them at each stage
    g_ops = 0;
    rates<Fc, true>(c, q, y, ab, o);
    out[18] = g_ops;
  }
  if (n >= 22) {
    // out[19..21] W formation, LU and one solve of the LU without S_h2's
    // row and column (spa), which the forms with S_h2 algebraic factor
    static Fc wa[spa::kNNZ];
    for (int s = 0; s < spa::kNNZ; ++s) wa[s] = Fc(0.0);
    g_ops = 0;
    spa::form_w<Fc>(wa, Fc(1e-4));
    out[19] = g_ops;
    g_ops = 0;
    spa::factor<Fc>(wa);
    out[20] = g_ops;
    Fc ba[NS];
    for (int i = 0; i < NS; ++i) ba[i] = Fc(1.0);
    g_ops = 0;
    spa::solve<Fc>(wa, ba);
    out[21] = g_ops;
  }
  return CHAD_OK;
}
