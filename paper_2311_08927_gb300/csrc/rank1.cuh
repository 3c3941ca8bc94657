// Sherman-Morrison treatment of the Eq. 7 coupling in W = I - g J.
//
// With S_H+ the root of the charge balance (Eq. 7), the Jacobian of the
// rates splits as J = J_d + u v^T: J_d is df/dy with S_H held fixed, u =
// df/dS_H at fixed y (19 nonzero rows: the pH-inhibited uptakes and the CO2
// transfer) and v = dS_H/dy from Eq. 7 differentiated implicitly (nonzero in
// the eight states that enter Eq. 7).  W = W_d - g u v^T with W_d = I - g J_d,
// so with q = W_d^-1 (g u) and delta = 1 - v^T q:
//
//   W^-1 b = z + q (v^T z) / delta,   z = W_d^-1 b.
//
// Only the sparser W_d is factored; each attempt adds one solve for q and
// each stage an 8-term dot product and a 29-term update.  delta is the last
// pivot of the bordered matrix [[W_d, g u], [v^T, 1]] and takes the same
// threshold test as the pivots of W_d: |delta| >= tau max(1, |v^T q|).
#pragma once
#include "adm1_device.cuh"
#include "sparse_lu_gen.cuh"

namespace chad {
namespace rank1 {

// v^T x over the eight states of Eq. 7 (v[k] belongs to state hc[k]).
template <class R, class V, class X>
CHAD_HD R vdot(const V* v, const X* x) {
  const int hc[8] = {iS_va, iS_bu, iS_pro, iS_ac, iS_IC, iS_IN, iS_cat, iS_an};
  R s = R(v[0]) * R(x[hc[0]]);
#pragma unroll
  for (int k = 1; k < 8; ++k) s += R(v[k]) * R(x[hc[k]]);
  return s;
}

// delta = 1 - v^T q for an already solved q; *inv_delta = 1/delta.  Returns
// false when delta fails the threshold test or is not finite.
template <class R>
CHAD_HD bool denominator(const R* q, const R* v, R tau, R* inv_delta) {
  const R s = vdot<R>(v, q);
  const R delta = R(1) - s;
  *inv_delta = rcp<R>(delta);
  return isfinite(delta) && fabs(delta) >= tau * fmax(R(1), fabs(s)) && delta != R(0);
}

// u (in q) -> q = W_d^-1 (g u) with the factored W_d (slot storage w, LU
// one of the generated sparse LUs: sp::Lu, or spa::Lu without S_h2);
// *inv_delta = 1/delta.  Returns false when delta fails the threshold test or
// is not finite.
template <class R, class LU = sp::Lu, class W>
CHAD_HD bool setup(W w, R g, const R* v, R tau, R* q, R* inv_delta) {
#pragma unroll
  for (int i = 0; i < NS; ++i) q[i] *= g;
  LU::template sub<R>(w, q);
  const R s = vdot<R>(v, q);
  const R delta = R(1) - s;
  *inv_delta = rcp<R>(delta);
  return isfinite(delta) && fabs(delta) >= tau * fmax(R(1), fabs(s)) && delta != R(0);
}

// z = W_d^-1 b (already solved) -> W^-1 b in place.
template <class R>
CHAD_HD void update(const R* q, const R* v, R inv_delta, R* z) {
  const R s = vdot<R>(v, z) * inv_delta;
#pragma unroll
  for (int i = 0; i < NS; ++i) z[i] += s * q[i];
}

}  // namespace rank1
}  // namespace chad
