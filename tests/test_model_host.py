"""The library's model code compiled for the host CPU (same source as the
kernels) against the oracle: rate vector and analytic Jacobian versus the
oracle's dual-number Jacobian, and the generated sparse LU against its
generator and the Jacobian's structural pattern.  No GPU needed."""
import os
import sys

import numpy as np
import pytest

import oracle as O
from paper_2311_08927_gb300 import build as B
from paper_2311_08927_gb300 import chad as CH
from paper_2311_08927_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


def _cases(n, seed):
    rng = np.random.default_rng(seed)
    for _ in range(n):
        p = I.default_params()
        kin = [I.PIDX[k] for k in I.KINETIC_PARAMS]
        p[kin] *= np.exp(0.2 * rng.standard_normal(len(kin)))
        y = I.x_ss() * np.exp(0.3 * rng.standard_normal(I.NS))
        yield p, rng.uniform(303.15, 313.15), y, rng.uniform(0, 1.0), rng.uniform(1e-2, 5e3)


def test_host_model_rates_and_analytic_jacobian_match_oracle():
    """Analytic J (hand-derived partials + rank-1 S_H coupling) equals the
    oracle's forward-mode AD Jacobian to round-off."""
    for p, T, y, D, V in _cases(30, 5):
        f, J, SH = CH.eval_model(p, T, y, y_in=I.influent(), D=D, V_liq=V, V_gas=V * 0.1)
        fo, SHo, _ = O.rhs(p, T, y, y_in=I.influent(), D=D, V_liq=V, V_gas=V * 0.1)
        Jo = O.jacobian(p, T, y, y_in=I.influent(), D=D, V_liq=V, V_gas=V * 0.1)
        assert abs(SH / SHo - 1) < 1e-13
        fs = np.abs(fo) + 1e-12 * np.abs(fo).max()
        assert np.max(np.abs(f - fo) / fs) < 1e-11
        cs = np.abs(Jo).max(axis=0, keepdims=True) + 1e-300
        assert np.max(np.abs(J - Jo) / cs) < 1e-12


def test_generated_sparse_lu_is_current():
    """Both generated LUs (all states; without S_h2 for the forms with S_h2
    algebraic) match what the generator makes of the model's pattern now."""
    sys.path.insert(0, os.path.join(ROOT, "paper_2311_08927_gb300", "csrc"))
    import gen_sparse as G
    pat = G.jacobian_pattern()
    for out, h2a in ((G.OUT, False), (G.OUT_H2A, True)):
        src, info = G.generate(pat, h2a)
        with open(out) as fh:
            assert fh.read() == src, f"{os.path.basename(out)} is stale: rerun gen_sparse.py"


def test_reduced_lu_leaves_out_s_h2_only():
    """The LU of the forms with S_h2 algebraic: 28 pivots (every state but
    S_h2), every structural nonzero of J_d outside S_h2's row and column has
    an LU slot, and S_h2's row and column map to the positions past the LU
    slots that the Jacobian scatter hands to the second Sherman-Morrison
    level."""
    sys.path.insert(0, os.path.join(ROOT, "paper_2311_08927_gb300", "csrc"))
    import gen_sparse as G
    pat = G.jacobian_pattern()
    src, info = G.generate(pat, True)
    NS = I.NS
    h2 = I.STATE_NAMES.index("S_h2")
    assert len(info["order"]) == NS - 1 and "S_h2" not in info["order"]
    import re
    nnz = int(re.search(r"constexpr int kNNZ = (\d+);", src).group(1))
    table = re.search(r"const int t\[NS \* NS\] = \{(.*?)\};", src, re.S).group(1)
    slot = np.array([int(x) for x in table.replace("\n", " ").split(",")]).reshape(NS, NS)
    for r in range(NS):
        for c in range(NS):
            if r == h2:
                assert slot[r, c] == nnz + c
            elif c == h2:
                assert slot[r, c] == nnz + NS + r
            elif pat[r, c]:
                assert 0 <= slot[r, c] < nnz
    lu = slot[np.ix_([i for i in range(NS) if i != h2], [i for i in range(NS) if i != h2])]
    assert sorted(lu[lu >= 0].tolist()) == list(range(nnz))
    # fewer slots and flops than the LU over all 29 states
    _, full = G.generate(pat, False)
    assert info["nnz"] < full["nnz"] and info["factor"] < full["factor"]


def test_direct_jacobian_nonzeros_have_sparse_slots():
    """The generated LU factors I - g J_d: every structural nonzero of J_d
    (S_H held fixed) has a slot, u = df/dS_H is nonzero only in the rows the
    kernels' rank-1 update covers and v = dS_H/dy only in the eight states of
    Eq. 7."""
    sys.path.insert(0, os.path.join(ROOT, "paper_2311_08927_gb300", "csrc"))
    import gen_sparse as G
    pat = G.jacobian_pattern()
    F = G.symbolic_fill(pat, G.markowitz(pat))
    eq7 = [I.SIDX[n] for n in ("S_va", "S_bu", "S_pro", "S_ac", "S_IC", "S_IN", "S_cat", "S_an")]
    for p, T, y, D, V in _cases(40, 17):
        _, Jd, u, v, _ = CH.eval_model_split(p, T, y, y_in=I.influent(), D=D)
        assert not np.any((Jd != 0) & ~pat)
        off = np.ones(I.NS, dtype=bool)
        off[eq7] = False
        assert np.all(v[off] == 0.0)
        assert np.count_nonzero(u) <= 19
    # fill only adds entries; the pattern includes the diagonal
    assert np.all(np.diag(pat)) and F.sum() >= pat.sum()


def _richardson(fun, x0, h):
    """Central difference with one Richardson step (error O(h^4))."""
    d1 = (fun(x0 + h) - fun(x0 - h)) / (2 * h)
    d2 = (fun(x0 + 2 * h) - fun(x0 - 2 * h)) / (4 * h)
    return (4 * d1 - d2) / 3


def test_split_jacobian_matches_oracle():
    """J_d + u v^T equals the oracle's dual-number Jacobian, and each part
    matches an independent (Richardson-extrapolated) central difference of
    the oracle: J_d and u of the rates at a fixed S_H (rhs_at), v of the
    Eq. 7 root (charge_solve)."""
    for p, T, y, D, V in _cases(8, 23):
        yin = I.influent()
        f, Jd, u, v, SH = CH.eval_model_split(p, T, y, y_in=yin, D=D, V_liq=V, V_gas=V * 0.1)
        Jo = O.jacobian(p, T, y, y_in=yin, D=D, V_liq=V, V_gas=V * 0.1)
        cs = np.abs(Jo).max(axis=0, keepdims=True) + 1e-300
        assert np.max(np.abs(Jd + np.outer(u, v) - Jo) / cs) < 1e-12
        SHo = O.charge_solve(p, T, y)[0]

        def fa(yy, S):
            return O.rhs_at(p, T, yy, S, y_in=yin, D=D, V_liq=V, V_gas=V * 0.1)

        uf = _richardson(lambda S: fa(y, S), SHo, 1e-2 * SHo)
        us = np.abs(uf) + 1e-9 * np.abs(uf).max()
        assert np.max(np.abs(u - uf) / us) < 2e-5
        for j in range(I.NS):
            hj = 1e-2 * max(abs(y[j]), 1e-8)
            e = np.zeros(I.NS)
            e[j] = 1.0
            col = _richardson(lambda t: fa(y + t * e, SHo), 0.0, hj)
            sc = np.abs(col).max() + 1e-300
            assert np.max(np.abs(Jd[:, j] - col)) / sc < 1e-6, j
            vf = _richardson(lambda t: O.charge_solve(p, T, y + t * e)[0], 0.0, 1e-2 * hj)
            assert abs(v[j] - vf) <= 1e-6 * abs(vf) + 1e-12 * SHo / max(abs(y[j]), 1e-8), j


def test_matrix_free_jacobian_vector_product():
    """The mixed form's refinement residual forms J x from the rate partials
    (no matrix).  It equals the oracle's dual-number Jacobian times x, for
    random directions x, to round-off."""
    rng = np.random.default_rng(41)
    for p, T, y, D, V in _cases(20, 29):
        yin = I.influent()
        x = rng.standard_normal(I.NS) * (np.abs(y) + 1e-6)
        *_, Jx = CH.eval_model_split(p, T, y, y_in=yin, D=D, V_liq=V, V_gas=V * 0.1, x=x)
        Jo = O.jacobian(p, T, y, y_in=yin, D=D, V_liq=V, V_gas=V * 0.1)
        ref = Jo @ x
        sc = np.abs(Jo) @ np.abs(x) + 1e-300
        assert np.max(np.abs(Jx - ref) / sc) < 1e-12


def test_flop_counts_of_the_reduced_lu_follow_the_generator():
    """The operation counter, run over the library's own templated LU code,
    agrees with the generator's static counts for both LUs, and the
    per-attempt counts of the forms with S_h2 algebraic use the 28-state LU
    (the FP64 form's count is the FP64 form 0's minus the LU savings plus its
    Eq. 8 work, counted per coefficient set and per extra solve)."""
    sys.path.insert(0, os.path.join(ROOT, "paper_2311_08927_gb300", "csrc"))
    import gen_sparse as G
    pat = G.jacobian_pattern()
    src_full, full = G.generate(pat, False)
    src_red, red = G.generate(pat, True)
    f = CH.flop_counts()
    assert f["solve"] == full["solve"] and f["solve_h2a"] == red["solve"]
    # the counter also counts the threshold test's 0.1 x max of every pivot
    # with a sub-column, which the generator's static count leaves out
    tests = "ok = ok && P::good(P::key(pv), cm);"
    assert f["factor"] - full["factor"] == src_full.count(tests)
    assert f["factor_h2a"] - red["factor"] == src_red.count(tests)
    assert f["form_w_h2a"] < f["form_w"]
    mx = CH.attempt_flops_h2_mixed()
    # 8 solves, one LU and one W formation of the 28-state LU in form 4
    lu_saving = (f["form_w"] - f["form_w_h2a"]) + (f["factor"] - f["factor_h2a"]) + \
        8 * (f["solve"] - f["solve_h2a"])
    full_lu = (f["rates_fj"] + 2 * f["rates_f"] + f["form_w"] + f["factor"] + 8 * f["solve"] +
               f["sm_setup"] + 7 * f["sm_update"] + 3 * f["h2_coeffs"] + 3 * f["jx_twofloat"] +
               3 * f["rates_partials"] + f["mx_fp32_extra"])
    assert mx["fp32"] == full_lu - lu_saving
    f3 = CH.attempt_flops(CH.PREC_FP64, True)
    f0 = CH.attempt_flops(CH.PREC_FP64, False)
    assert f3["fp64_per_h2_iter"] == f["h2_iter"]
    extra = f3["fp64"] - f0["fp64"]
    expect = (-(f["factor"] - f["factor_h2a"]) - 1            # LU; one diagonal one fewer
              + 5 * f["solve_h2a"] - 4 * f["solve"]          # the p2 solve, smaller solves
              + f["sm_update"] + 3 * f["h2_coeffs"] + 59 + 54 + 3 * 117 + 2 * 58)
    assert extra == expect


def _run_generated_lu(src, nnz, slot, W_vals, g, b):
    """Execute the generated form_w / factor / solve of one LU header on the
    host, statement by statement (the emitted code is straight-line with
    literal slot indices), in float64."""
    import re
    w = np.array(W_vals, dtype=np.float64)
    # form_w: w = -g w, then the diagonal ones
    body = src[src.index("CHAD_HD void form_w("):src.index("// In-place LU")]
    w *= -g
    for m in re.finditer(r"w\[(\d+)\] \+= R\(1\);", body):
        w[int(m.group(1))] += 1.0
    body = src[src.index("CHAD_HD bool factor("):src.index("return ok;")]
    inv = l = None
    for line in body.splitlines():
        line = line.strip()
        m = re.match(r"const R pv = w\[(\d+)\];", line)
        if m:
            pv = w[int(m.group(1))]
            inv = 1.0 / pv
            continue
        m = re.match(r"w\[(\d+)\] = inv;", line)
        if m:
            w[int(m.group(1))] = inv
            continue
        m = re.match(r"\{ const R l = w\[(\d+)\] \* inv; w\[(\d+)\] = l;", line)
        if m:
            l = w[int(m.group(1))] * inv
            w[int(m.group(2))] = l
            continue
        m = re.match(r"w\[(\d+)\] -= l \* w\[(\d+)\];", line)
        if m:
            w[int(m.group(1))] -= l * w[int(m.group(2))]
    body = src[src.index("CHAD_HD void solve("):src.index("constexpr int kFactorFlops")]
    b = np.array(b, dtype=np.float64)
    z = {}
    for line in body.splitlines():
        line = line.strip()
        m = re.match(r"R z(\d+) = b\[(\d+)\];", line)
        if m:
            z[int(m.group(1))] = b[int(m.group(2))]
            continue
        m = re.match(r"z(\d+) -= w\[(\d+)\] \* z(\d+);", line)
        if m:
            z[int(m.group(1))] -= w[int(m.group(2))] * z[int(m.group(3))]
            continue
        m = re.match(r"z(\d+) \*= w\[(\d+)\];", line)
        if m:
            z[int(m.group(1))] *= w[int(m.group(2))]
            continue
        m = re.match(r"b\[(\d+)\] = z(\d+);", line)
        if m:
            b[int(m.group(1))] = z[int(m.group(2))]
    return b


@pytest.mark.parametrize("h2a", [False, True])
def test_generated_lu_solves_like_a_dense_solver(h2a):
    """The generated static-order LU (all 29 states, or the 28 without S_h2),
    executed statement by statement on the host, solves (I - g J_d) x = b
    as numpy's dense solver does, for random J_d on the library's own
    pattern; without S_h2, W_d's S_h2 row is the identity's (b[S_h2] passes
    through) and S_h2's row and column of J_d take no part."""
    import re
    sys.path.insert(0, os.path.join(ROOT, "paper_2311_08927_gb300", "csrc"))
    import gen_sparse as G
    NS = I.NS
    h2 = I.STATE_NAMES.index("S_h2")
    pat = G.jacobian_pattern()
    src, info = G.generate(pat, h2a)
    nnz = int(re.search(r"constexpr int kNNZ = (\d+);", src).group(1))
    table = re.search(r"const int t\[NS \* NS\] = \{(.*?)\};", src, re.S).group(1)
    slot = np.array([int(x) for x in table.replace("\n", " ").split(",")]).reshape(NS, NS)
    rng = np.random.default_rng(7)
    for trial in range(5):
        J = np.where(pat, rng.standard_normal((NS, NS)), 0.0)
        J[np.diag_indices(NS)] = -np.abs(J[np.diag_indices(NS)]) - 1.0
        if h2a:
            J[h2, :] = 0.0
            J[:, h2] = 0.0
        g = [0.05, 0.3, 1.0, 3.0, 10.0][trial]
        vals = np.zeros(nnz)
        for r in range(NS):
            for c in range(NS):
                s = slot[r, c]
                if 0 <= s < nnz:
                    vals[s] = J[r, c]
        b = rng.standard_normal(NS)
        x = _run_generated_lu(src, nnz, slot, vals, g, b)
        ref = np.linalg.solve(np.eye(NS) - g * J, b)
        assert np.max(np.abs(x - ref)) <= 1e-10 * max(1.0, np.max(np.abs(ref))), (h2a, g)
        if h2a:
            assert x[h2] == b[h2]
