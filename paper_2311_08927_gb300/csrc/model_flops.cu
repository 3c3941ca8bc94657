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
  Fc dinv[NS];
  g_ops = 0;
  sp::factor<Fc>(w, dinv);
  out[4] = g_ops;
  Fc b[NS];
  for (int i = 0; i < NS; ++i) b[i] = Fc(1.0);
  g_ops = 0;
  sp::solve<Fc>(w, dinv, b);
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
  rank1::setup<Fc>(w, dinv, Fc(1e-4), v, Fc(0.1), u, &inv_delta);
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
  return CHAD_OK;
}
