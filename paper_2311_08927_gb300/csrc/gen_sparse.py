"""Generate sparse_lu_gen.cuh: a static-order sparse LU of W_d = I - g J_d.

J_d is the ADM1 Jacobian with S_H held fixed; the full Jacobian is J_d + u v^T
(u = df/dS_H, v = dS_H/dy from Eq. 7), and the integrator applies that
rank-1 term by the Sherman-Morrison formula, so only W_d is factored.  The
structural pattern of J_d is taken from the library's own model
(chad_eval_model_split on the host, i.e. the same source as the kernels),
evaluated at random states and randomly perturbed parameter sets so that no
coefficient that happens to vanish for one parameter set is missed.  The
elimination order is Markowitz's (minimise (r-1)(c-1) of each pivot on the
remaining unsymmetric pattern, lowest state index on ties); its symbolic
fill gives the storage slots.  The emitted code is straight-line with static
slot indices:

  slot(r, c)         storage slot of W_rc (-1 when structurally zero)
  factor(w)          in-place LU in the static order, the reciprocal of each
                     pivot stored in its diagonal slot; returns false when a
                     pivot fails the threshold test |u_kk| >= 0.1 max_i |l_ik u_kk|
                     (equivalently |w_kk| >= 0.1 max_i |w_ik| before scaling,
                     PivTest in adm1_device.cuh) or is zero or not finite; the
                     caller then shrinks the step, which drives W towards the
                     identity where the order is safe
  solve(w, b)        forward / back substitution in the static order

A second header, sparse_lu_h2a_gen.cuh (namespace spa), serves the forms
with S_h2 algebraic (Eq. 8): there S_h2 is not a state of W_d (its row and
column go to the second Sherman-Morrison level), so its LU runs over the
other 28 states only and needs fewer slots and less fill.  Its slot()
returns, besides the LU slots, positions past them for the S_h2 row
(kNNZ + c) and the S_h2 column (kNNZ + NS + r), so that the Jacobian scatter
can deliver those two vectors apart from the factored matrix.

Each header also defines `struct Lu` with the same static members in both
namespaces, so that the kernels take the LU as a template parameter.

Run from the repository root:  python paper_2311_08927_gb300/csrc/gen_sparse.py
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from paper_2311_08927_gb300 import chad as CH  # noqa: E402
from paper_2311_08927_gb300 import inputs as I  # noqa: E402

NS = I.NS
OUT = os.path.join(HERE, "sparse_lu_gen.cuh")
OUT_H2A = os.path.join(HERE, "sparse_lu_h2a_gen.cuh")
I_H2 = I.STATE_NAMES.index("S_h2")


def jacobian_pattern(n_samples: int = 400, seed: int = 12345) -> np.ndarray:
    rng = np.random.default_rng(seed)
    base_p = I.default_params()
    base_y = I.x_ss()
    pat = np.eye(NS, dtype=bool)
    for k in range(n_samples):
        p = base_p * np.exp(0.3 * rng.standard_normal(base_p.size))
        # keep the parameters that must stay ordered or fixed
        for n in ("pH_LL_aa", "pH_UL_aa", "pH_LL_ac", "pH_UL_ac", "pH_LL_h2", "pH_UL_h2",
                  "R", "R_J", "T_base", "pK_w", "pK_a_va", "pK_a_bu", "pK_a_pro", "pK_a_ac",
                  "pK_a_co2", "pK_a_IN", "P_atm", "T_ref_kin", "V_liq_ref"):
            p[I.PIDX[n]] = base_p[I.PIDX[n]]
        y = base_y * np.exp(0.5 * rng.standard_normal(NS))
        T = rng.uniform(298.0, 318.0)
        D = rng.uniform(0.0, 1.0)
        yin = I.influent() * np.exp(0.3 * rng.standard_normal(NS)) + 1e-6
        _, Jd, _, _, _ = CH.eval_model_split(p, T, y, y_in=yin, D=D,
                                             V_liq=rng.uniform(1e-3, 1e4),
                                             V_gas=rng.uniform(1e-4, 1e3))
        pat |= (Jd != 0.0)
    return pat


def markowitz(pat: np.ndarray, states=None) -> list[int]:
    """Elimination order over `states` (all states by default)."""
    A = pat.copy()
    rem = list(range(NS)) if states is None else list(states)
    order = []
    while rem:
        best = None
        for v in rem:
            r = sum(A[v, u] for u in rem) - 1
            c = sum(A[u, v] for u in rem) - 1
            key = (r * c, v)
            if best is None or key < best[0]:
                best = (key, v)
        v = best[1]
        order.append(v)
        rows = [u for u in rem if u != v and A[u, v]]
        cols = [u for u in rem if u != v and A[v, u]]
        for i in rows:
            for j in cols:
                A[i, j] = True
        rem.remove(v)
    return order


def symbolic_fill(pat: np.ndarray, order: list[int]) -> np.ndarray:
    n = len(order)
    P = pat[np.ix_(order, order)].copy()  # permuted positions
    for k in range(n):
        rows = [i for i in range(k + 1, n) if P[i, k]]
        cols = [j for j in range(k + 1, n) if P[k, j]]
        for i in rows:
            for j in cols:
                P[i, j] = True
    return P


def generate(pat: np.ndarray, h2a: bool = False) -> str:
    """The full LU (namespace sp) or, with h2a, the LU without S_h2's row and
    column (namespace spa) for the forms with S_h2 algebraic."""
    ns = "spa" if h2a else "sp"
    if h2a:
        pat = pat.copy()
        pat[I_H2, :] = False
        pat[:, I_H2] = False
        states = [s for s in range(NS) if s != I_H2]
    else:
        states = list(range(NS))
    n_piv = len(states)
    order = markowitz(pat, states)
    F = symbolic_fill(pat, order)  # in permuted positions
    slot = -np.ones((NS, NS), dtype=int)
    n = 0
    for k in range(n_piv):           # row-major over permuted positions
        for j in range(n_piv):
            if F[k, j]:
                slot[order[k], order[j]] = n
                n += 1
    nnz = n
    if h2a:  # the S_h2 row and column, past the LU slots
        for c in range(NS):
            slot[I_H2, c] = nnz + c
        for r in range(NS):
            if r != I_H2:
                slot[r, I_H2] = nnz + NS + r
    n_store = nnz + (2 * NS if h2a else 0)
    nnz_j = int(pat.sum())
    flops = 0
    L = []
    w = L.append
    w("// GENERATED by gen_sparse.py from the library's own Jacobian pattern -- do not edit.")
    if h2a:
        w("// Static-order (Markowitz) sparse LU of W_d = I - g J_d without the S_h2 row and")
        w("// column (S_h2 algebraic, Eq. 8: those go to a second Sherman-Morrison level),")
        w(f"// over the other {n_piv} ADM1 states (J_d: the Jacobian with S_H held fixed).")
    else:
        w("// Static-order (Markowitz) sparse LU of W_d = I - g J_d for the 29 ADM1 states")
        w("// (J_d: the Jacobian with S_H held fixed).")
    w(f"// pattern nnz(J_d) = {nnz_j}, slots with fill = {nnz}")
    w("#pragma once")
    w('#include "adm1_device.cuh"')
    w("")
    w("namespace chad {")
    w(f"namespace {ns} {{")
    w("")
    w(f"constexpr int kNNZ = {nnz};")
    w(f"constexpr int kNNZ_J = {nnz_j};")
    if h2a:
        w(f"constexpr int kPiv = {n_piv};  // pivots (every state but S_h2)")
        w("// slots of the Jacobian scatter: the LU's, then the S_h2 row (kNNZ + c)")
        w("// and the S_h2 column (kNNZ + NS + r)")
        w(f"constexpr int kStore = {n_store};")
    else:
        w(f"constexpr int kPiv = {n_piv};")
        w(f"constexpr int kStore = {n_store};")
    w("// elimination position -> state index")
    w("constexpr int kOrder[kPiv] = {" + ", ".join(str(v) for v in order) + "};")
    w("")
    w("CHAD_HD constexpr int slot(int r, int c) {")
    w("  // row-major table over states, -1 = structurally zero")
    rows = []
    for r in range(NS):
        rows.append("      " + ", ".join(str(int(slot[r, c])) for c in range(NS)))
    w("  const int t[NS * NS] = {")
    w(",\n".join(rows))
    w("  };")
    w("  return t[r * NS + c];")
    w("}")
    w("")
    w("struct Idx {")
    w("  static CHAD_HD constexpr int at(int r, int c) { return slot(r, c); }")
    w("  static constexpr int size = kStore;")
    w("};")
    w("")
    w("// diagonal slots in elimination order")
    w("constexpr int kDiag[kPiv] = {" + ", ".join(str(int(slot[s, s])) for s in order) + "};")
    w("")
    # ------------------------------------------------------------- W formation
    w("// W_d = I - g J_d in place over the slots (fill slots hold zero in J_d).")
    w("// W: the slot storage, a pointer or any accessor whose w[s] is a reference.")
    w("template <class R, class W>")
    w("CHAD_HD void form_w(W w, R g) {")
    w("#pragma unroll")
    w("  for (int s = 0; s < kNNZ; ++s) w[s] = -g * w[s];")
    for sidx in order:
        w(f"  w[{int(slot[sidx, sidx])}] += R(1);")
    w("}")
    w("")
    # ------------------------------------------------------------- factor
    w("// In-place LU; the diagonal slots receive the reciprocals of the pivots")
    w("// (the only use the solve makes of them).  Returns false if a pivot fails")
    w("// the threshold test.")
    w("template <class R, class W>")
    w("CHAD_HD bool factor(W w) {")
    w("  using P = PivTest<R>;")
    w("  bool ok = true;")
    for k in range(n_piv):
        pv = order[k]
        d = slot[pv, pv]
        sub = [i for i in range(k + 1, n_piv) if F[i, k]]
        ucols = [j for j in range(k + 1, n_piv) if F[k, j]]
        w(f"  {{  // pivot {k}: state {pv} ({I.STATE_NAMES[pv]}), {len(sub)} rows x {len(ucols)} cols")
        w(f"    const R pv = w[{d}];")
        if sub:
            terms = [f"P::key(w[{slot[order[i], pv]}])" for i in sub]
            expr = terms[0]
            for t in terms[1:]:
                expr = f"P::kmax({expr}, {t})"
            w(f"    const typename P::K cm = {expr};")
            w("    ok = ok && P::good(P::key(pv), cm);")
        else:
            w("    ok = ok && P::good(P::key(pv));")
        w("    const R inv = rcp<R>(pv);")
        w(f"    w[{d}] = inv;")
        flops += 1
        for i in sub:
            sik = slot[order[i], pv]
            w(f"    {{ const R l = w[{sik}] * inv; w[{sik}] = l;")
            flops += 1
            for j in ucols:
                w(f"      w[{slot[order[i], order[j]]}] -= l * w[{slot[pv, order[j]]}];")
                flops += 2
            w("    }")
        w("  }")
    w("  return ok;")
    w("}")
    w("")
    # ------------------------------------------------------------- solve
    if h2a:
        w("// Solve W x = b in place (b indexed by state; b[S_h2] is left as it is:")
        w("// W_d's S_h2 row is the identity's).")
    else:
        w("// Solve W x = b in place (b indexed by state).")
    w("template <class R, class W>")
    w("CHAD_HD void solve(W w, R* b) {")
    for k in range(n_piv):
        w(f"  R z{k} = b[{order[k]}];")
    sflops = 0
    for k in range(n_piv):  # forward, unit lower
        terms = [(j, slot[order[k], order[j]]) for j in range(k) if F[k, j]]
        for j, s_ in terms:
            w(f"  z{k} -= w[{s_}] * z{j};")
            sflops += 2
    for k in reversed(range(n_piv)):  # back
        terms = [(j, slot[order[k], order[j]]) for j in range(k + 1, n_piv) if F[k, j]]
        for j, s_ in terms:
            w(f"  z{k} -= w[{s_}] * z{j};")
            sflops += 2
        w(f"  z{k} *= w[{int(slot[order[k], order[k]])}];")
        sflops += 1
    for k in range(n_piv):
        w(f"  b[{order[k]}] = z{k};")
    w("}")
    w("")
    w(f"constexpr int kFactorFlops = {flops};")
    w(f"constexpr int kSolveFlops = {sflops};")
    w("")
    w("// The LU as a type, so that the kernels can take it as a template parameter.")
    w("struct Lu {")
    w("  using Index = Idx;")
    w("  static constexpr int nnz = kNNZ;")
    w("  static constexpr int store = kStore;")
    w("  template <class R, class W>")
    w("  static CHAD_HD void form(W w, R g) { form_w<R>(w, g); }")
    w("  template <class R, class W>")
    w("  static CHAD_HD bool lu(W w) { return factor<R>(w); }")
    w("  template <class R, class W>")
    w("  static CHAD_HD void sub(W w, R* b) { solve<R>(w, b); }")
    w("};")
    w("")
    w(f"}}  // namespace {ns}")
    w("}  // namespace chad")
    return "\n".join(L) + "\n", dict(nnz=nnz, nnz_j=nnz_j, factor=flops, solve=sflops,
                                      order=[I.STATE_NAMES[s] for s in order])


def main():
    pat = jacobian_pattern()
    for out, h2a in ((OUT, False), (OUT_H2A, True)):
        src, info = generate(pat, h2a)
        with open(out, "w") as fh:
            fh.write(src)
        print(f"wrote {out}: {info}")


if __name__ == "__main__":
    main()
