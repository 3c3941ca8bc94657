"""Pins of the CPU oracle against things other than itself.

Each test checks the oracle against a closed form, a conservation law the
paper's model must satisfy, a textbook value, an independent library routine
or brute force, so that a dropped term, a wrong sign or index or a transposed
operand in the oracle fails at least one of them.

Paper basis: Sec. 2.2 Eq. 2 (mass balance), Eq. 3-6 (inhibition), Eq. 7
(charge balance), Sec. 2.3 (AD particles), Sec. 3.1 (single particle = CSTR),
Sec. 4.2 (identical initial states stay identical without diffusion).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2311_08927_gb300 import inputs as I

S = I.SIDX
P = I.PIDX
BIO = ["X_su", "X_aa", "X_fa", "X_c4", "X_pro", "X_ac", "X_h2"]
COD_LIQ = ["S_su", "S_aa", "S_fa", "S_va", "S_bu", "S_pro", "S_ac", "S_h2", "S_ch4", "S_I",
           "X_c", "X_ch", "X_pr", "X_li"] + BIO + ["X_I"]


def params(**over):
    p = I.default_params()
    for k, v in over.items():
        p[P[k]] = v
    return p


def state(**kv):
    y = np.zeros(I.NS)
    for k, v in kv.items():
        y[S[k]] = v
    return y


def perturbed_ss(seed=0, n=1):
    rng = np.random.default_rng(seed)
    y = I.x_ss()[:, None] * np.exp(0.1 * rng.standard_normal((I.NS, n)))
    return y[:, 0] if n == 1 else y


# ----------------------------------------------------------------- layout
def test_param_layout_matches_input_generator():
    assert O.param_names() == I.PARAM_NAMES


# ----------------------------------------------------------------- stoichiometry
def test_parameter_closures():
    """COD fractions of each product group sum to 1; X_c's N and C contents
    equal the fraction-weighted contents of its products (ADM1 definition)."""
    p = I.default_params()
    g = lambda *n: sum(p[P[k]] for k in n)
    assert abs(g("f_sI_xc", "f_xI_xc", "f_ch_xc", "f_pr_xc", "f_li_xc") - 1) < 1e-15
    assert abs(g("f_h2_su", "f_bu_su", "f_pro_su", "f_ac_su") - 1) < 1e-15
    assert abs(g("f_h2_aa", "f_va_aa", "f_bu_aa", "f_pro_aa", "f_ac_aa") - 1) < 1e-15
    assert abs(g("f_ac_fa", "f_h2_fa") - 1) < 1e-15
    assert abs(g("f_pro_va", "f_ac_va", "f_h2_va") - 1) < 1e-15
    assert abs(g("f_ac_bu", "f_h2_bu") - 1) < 1e-15
    assert abs(g("f_ac_pro", "f_h2_pro") - 1) < 1e-15
    n_prod = (p[P["f_xI_xc"]] + p[P["f_sI_xc"]]) * p[P["N_I"]] + p[P["f_pr_xc"]] * p[P["N_aa"]]
    assert abs(p[P["N_xc"]] - n_prod) < 1e-15
    c_prod = (p[P["f_sI_xc"]] * p[P["C_sI"]] + p[P["f_ch_xc"]] * p[P["C_ch"]] +
              p[P["f_pr_xc"]] * p[P["C_pr"]] + p[P["f_li_xc"]] * p[P["C_li"]] +
              p[P["f_xI_xc"]] * p[P["C_xI"]])
    assert abs(p[P["C_xc"]] - c_prod) < 1e-15


def test_petersen_cod_closes_per_process():
    """Every biochemical process conserves COD: the COD-carrying rows of each
    Petersen column sum to zero (Eq. 2 with the standard ADM1 table)."""
    nu = O.petersen(I.default_params())
    rows = [S[k] for k in COD_LIQ]
    for j in range(19):
        assert abs(nu[rows, j].sum()) < 1e-15, j
    # every process consumes something (no all-zero column)
    assert np.all(np.abs(nu[:, :22]).sum(axis=0) > 0)


def test_petersen_nitrogen_matches_balance():
    """The S_IN coefficients equal the ADM1 nitrogen balance: biomass growth
    takes N_bac per unit yield, amino-acid uptake releases N_aa, decay
    releases N_bac - N_xc, disintegration releases N_xc minus its products' N."""
    p = I.default_params()
    nu = O.petersen(p)
    Nb = p[P["N_bac"]]
    expect = {4: -p[P["Y_su"]] * Nb, 5: p[P["N_aa"]] - p[P["Y_aa"]] * Nb,
              6: -p[P["Y_fa"]] * Nb, 7: -p[P["Y_c4"]] * Nb, 8: -p[P["Y_c4"]] * Nb,
              9: -p[P["Y_pro"]] * Nb, 10: -p[P["Y_ac"]] * Nb, 11: -p[P["Y_h2"]] * Nb}
    for j, v in expect.items():
        assert abs(nu[S["S_IN"], j] - v) < 1e-16, j
    for j in range(12, 19):
        assert abs(nu[S["S_IN"], j] - (Nb - p[P["N_xc"]])) < 1e-16
    for j in (1, 2, 3):
        assert nu[S["S_IN"], j] == 0.0


def invariants(y, p, V_liq=3400.0, V_gas=300.0):
    r = V_gas / V_liq
    cod = sum(y[S[k]] for k in COD_LIQ) + r * (y[S["S_gas_h2"]] + y[S["S_gas_ch4"]])
    nit = (y[S["S_IN"]] + p[P["N_aa"]] * (y[S["S_aa"]] + y[S["X_pr"]]) +
           p[P["N_bac"]] * sum(y[S[b]] for b in BIO) + p[P["N_xc"]] * y[S["X_c"]] +
           p[P["N_I"]] * (y[S["S_I"]] + y[S["X_I"]]))
    cc = {"S_su": "C_su", "S_aa": "C_aa", "S_fa": "C_fa", "S_va": "C_va", "S_bu": "C_bu",
          "S_pro": "C_pro", "S_ac": "C_ac", "S_ch4": "C_ch4", "S_I": "C_sI", "X_c": "C_xc",
          "X_ch": "C_ch", "X_pr": "C_pr", "X_li": "C_li", "X_I": "C_xI"}
    car = y[S["S_IC"]] + sum(p[P[c]] * y[S[k]] for k, c in cc.items())
    car += p[P["C_bac"]] * sum(y[S[b]] for b in BIO)
    car += r * (y[S["S_gas_co2"]] + p[P["C_ch4"]] * y[S["S_gas_ch4"]])
    return np.array([cod, nit, car, y[S["S_cat"]], y[S["S_an"]]])


@pytest.mark.parametrize("T", [308.15, 311.0])
def test_closed_batch_conserves_cod_n_c_charge(T):
    """No inflow and no gas venting (k_p = 0): total COD, N, C and the inert
    ions are linear invariants of Eq. 2, and a W-method with the exact
    Jacobian preserves them to round-off over a whole day."""
    p = params(k_p=0.0)
    y0 = perturbed_ss(1)
    inv0 = invariants(y0, p)
    y, SH, h, st, stats = O.integrate(p, T, y0, 1.0, rtol=1e-7, atol=I.atol_vector())
    assert st == 0 and stats[0] > 10
    inv1 = invariants(y, p)
    assert np.max(np.abs(inv1 - inv0) / np.abs(inv0)) < 1e-12


def test_open_cstr_balance_steady_state():
    """At the stored CSTR steady state with the Table 1 inflow, COD in = COD
    out (liquid effluent + vented CH4/H2) to the residual of the steady state."""
    p = I.default_params()
    y = I.x_ss()
    D = I.TABLE1["Q"] / I.TABLE1["V_liq"]
    f, SH, rho = O.rhs(p, I.T_OP, y, y_in=I.influent(), D=D)
    _, qv = O.rates_at(p, I.T_OP, y, SH)
    yin = I.influent()
    cod_in = D * sum(yin[S[k]] for k in COD_LIQ)
    cod_out = D * sum(y[S[k]] for k in COD_LIQ)
    vent = qv * (I.TABLE1["V_gas"] / I.TABLE1["V_liq"]) * (y[S["S_gas_h2"]] + y[S["S_gas_ch4"]])
    assert abs(cod_in - cod_out - vent) / cod_in < 1e-6


# ----------------------------------------------------------------- closed forms
@pytest.mark.parametrize("T", [308.15, 303.15])
def test_disintegration_hydrolysis_closed_form(T):
    """With no biomass, X_c decays as exp(-k_dis t) and each hydrolysis
    product follows the two-exponential solution of the linear chain."""
    p = I.default_params()
    arr = math.exp(-p[P["Ea_over_R"]] * (1.0 / T - 1.0 / p[P["T_ref_kin"]]))
    y0 = state(X_c=2.0, X_ch=1.0, X_pr=1.5, X_li=0.5, S_IC=0.1, S_IN=0.1, S_cat=0.04,
               S_an=0.02, S_gas_ch4=0.5, S_gas_co2=0.01)
    t = 1.0
    y, SH, h, st, _ = O.integrate(p, T, y0, t, rtol=1e-12, atol=np.full(I.NS, 1e-16))
    assert st == 0
    k = p[P["k_dis"]] * arr
    assert abs(y[S["X_c"]] / (2.0 * math.exp(-k * t)) - 1) < 1e-9
    for X, kh, fr in (("X_ch", "k_hyd_ch", "f_ch_xc"), ("X_pr", "k_hyd_pr", "f_pr_xc"),
                      ("X_li", "k_hyd_li", "f_li_xc")):
        kk = p[P[kh]] * arr
        exact = (y0[S[X]] * math.exp(-kk * t) +
                 p[P[fr]] * k * 2.0 * (math.exp(-k * t) - math.exp(-kk * t)) / (kk - k))
        # global error measured against the trajectory's scale (the value decays ~80x)
        assert abs(y[S[X]] - exact) < 1e-10 * max(exact, y0[S[X]]), X
    # the inert fractions accumulate exactly f * (X_c0 - X_c)
    for X, fr in (("X_I", "f_xI_xc"), ("S_I", "f_sI_xc")):
        assert abs(y[S[X]] - p[P[fr]] * (2.0 - y[S["X_c"]])) < 1e-12


def _vh(p, base, dH, T):
    return p[P[base]] * math.exp(p[P[dH]] / p[P["R_J"]] * (1 / p[P["T_base"]] - 1 / T))


@pytest.mark.parametrize("T", [308.15, 298.15])
def test_henry_equilibrium_closed_form(T):
    """Closed headspace, no biology: CH4 and H2 relax to Henry's law
    S = K_H p with COD conversions of 64 and 16 kgCOD/kmol, and the total
    amount S V_liq + G V_gas is conserved, fixing the equilibrium exactly."""
    p = params(k_p=0.0)
    y0 = state(S_ch4=0.05, S_h2=1e-5, S_gas_ch4=0.5, S_gas_h2=1e-4, S_IC=0.05, S_IN=0.05,
               S_cat=0.04, S_an=0.02)
    y, SH, h, st, _ = O.integrate(p, T, y0, 1.0, rtol=1e-10, atol=np.full(I.NS, 1e-16))
    assert st == 0
    Vl, Vg = 3400.0, 300.0
    RT = p[P["R"]] * T
    for s, g, base, dH in (("S_ch4", "S_gas_ch4", "K_H_ch4", "dH_K_H_ch4"),
                           ("S_h2", "S_gas_h2", "K_H_h2", "dH_K_H_h2")):
        KH = _vh(p, base, dH, T)
        M = y0[S[s]] * Vl + y0[S[g]] * Vg
        G = M / (Vl * KH * RT + Vg)
        assert abs(y[S[g]] / G - 1) < 1e-8, g
        assert abs(y[S[s]] / (KH * RT * G) - 1) < 1e-8, s


def test_gas_outflow_closed_form():
    """No transfer (k_La = 0): the dry headspace pressure p obeys
    dp/dt = -(k_p/V_gas) p (p + p_w - P_atm)(p + p_w) / P_atm, whose
    partial-fraction integral gives the elapsed time in closed form."""
    T = 308.15
    p = params(k_La=0.0)
    y0 = state(S_gas_ch4=2.0, S_gas_co2=0.02, S_gas_h2=1e-3, S_IC=0.05, S_IN=0.05,
               S_cat=0.04, S_an=0.02)
    t = 0.002
    y, SH, h, st, _ = O.integrate(p, T, y0, t, rtol=1e-13, atol=np.full(I.NS, 1e-18))
    assert st == 0
    RT = p[P["R"]] * T
    dry = lambda v: RT * (v[S["S_gas_h2"]] / 16 + v[S["S_gas_ch4"]] / 64 + v[S["S_gas_co2"]])
    a = p[P["p_h2o_base"]] * math.exp(p[P["p_h2o_theta"]] * (1 / p[P["T_base"]] - 1 / T))
    Pa = p[P["P_atm"]]
    b = a - Pa
    A, B, Cc = 1 / (a * b), 1 / (a * (a - b)), -1 / (b * (a - b))
    F = lambda x: A * math.log(x) + B * math.log(x + a) + Cc * math.log(x + b)
    kappa = p[P["k_p"]] / 300.0  # V_liq = V_liq_ref, V_gas = 300
    t_cf = Pa * (F(dry(y0)) - F(dry(y))) / kappa
    assert abs(t_cf / t - 1) < 5e-9  # global error of the rtol-1e-13 run
    # composition ratios are unchanged by a common outflow
    assert abs(y[S["S_gas_co2"]] / y[S["S_gas_ch4"]] / (0.02 / 2.0) - 1) < 1e-11


# ----------------------------------------------------------------- rate laws (Eq. 3-6)
def _uninhibited_state():
    return state(S_IN=1e6, S_IC=0.1, S_cat=0.04, S_an=0.02, X_su=1.0, X_aa=1.0, X_fa=1.0,
                 X_c4=1.0, X_pro=1.0, X_ac=1.0, X_h2=1.0)


@pytest.mark.parametrize("proc,sub,ks", [(4, "S_su", "K_S_su"), (5, "S_aa", "K_S_aa"),
                                         (6, "S_fa", "K_S_fa"), (9, "S_pro", "K_S_pro"),
                                         (10, "S_ac", "K_S_ac"), (11, "S_h2", "K_S_h2")])
def test_monod_half_saturation(proc, sub, ks):
    """Eq. 6 substrate limitation: the uptake rate at S = K_S is exactly half
    of its saturated value, identifying the half-saturation constant used."""
    p = params(K_I_nh3=1e300)
    y = _uninhibited_state()
    y[S[sub]] = p[P[ks]]
    r_half, _ = O.rates_at(p, 308.15, y, 1e-12)
    y[S[sub]] = p[P[ks]] * 1e12
    r_sat, _ = O.rates_at(p, 308.15, y, 1e-12)
    assert abs(r_half[proc] / r_sat[proc] - 0.5) < 1e-11


@pytest.mark.parametrize("proc,ki", [(6, "K_I_h2_fa"), (7, "K_I_h2_c4"), (8, "K_I_h2_c4"),
                                     (9, "K_I_h2_pro")])
def test_hydrogen_inhibition_half_point(proc, ki):
    """Eq. 5 non-competitive inhibition: S_h2 = K_I halves the rate."""
    p = I.default_params()
    y = _uninhibited_state()
    for s in ("S_fa", "S_va", "S_bu", "S_pro"):
        y[S[s]] = 1.0
    y[S["S_h2"]] = 0.0
    r0, _ = O.rates_at(p, 308.15, y, 1e-12)
    y[S["S_h2"]] = p[P[ki]]
    r1, _ = O.rates_at(p, 308.15, y, 1e-12)
    assert abs(r1[proc] / r0[proc] - 0.5) < 1e-12


@pytest.mark.parametrize("proc,ll,ul", [(4, "pH_LL_aa", "pH_UL_aa"), (10, "pH_LL_ac", "pH_UL_ac"),
                                        (11, "pH_LL_h2", "pH_UL_h2")])
def test_ph_inhibition_half_point_and_limits(proc, ll, ul):
    """Eq. 3-4: K_pH is the mid-point of the limits, where the Hill factor is
    1/2; it tends to 1 far above the upper pH limit and 0 far below."""
    p = params(K_I_nh3=1e300)
    y = _uninhibited_state()
    for s in ("S_su", "S_ac", "S_h2"):
        y[S[s]] = 1e6
    ref, _ = O.rates_at(p, 308.15, y, 1e-16)
    mid = 10 ** (-(p[P[ll]] + p[P[ul]]) / 2)
    r, _ = O.rates_at(p, 308.15, y, mid)
    assert abs(r[proc] / ref[proc] - 0.5) < 1e-12
    lo, _ = O.rates_at(p, 308.15, y, 10 ** (-(p[P[ll]] - 2)))
    assert lo[proc] / ref[proc] < 1e-3
    hi, _ = O.rates_at(p, 308.15, y, 10 ** (-(p[P[ul]] + 2)))
    assert hi[proc] / ref[proc] > 0.999


# ----------------------------------------------------------------- charge balance (Eq. 7)
def test_ph_pure_water_and_strong_base():
    p = I.default_params()
    T = 298.15  # van 't Hoff factors are 1 at T_base
    SH, _, _ = O.charge_solve(p, T, state())
    assert abs(-math.log10(SH) - 7.0) < 1e-10
    c = 0.01
    SH, _, _ = O.charge_solve(p, T, state(S_cat=c))
    exact = 2e-14 / (c + math.sqrt(c * c + 4e-14))  # root of S^2 + c S - K_w, stable form
    assert abs(SH / exact - 1) < 1e-9 and abs(-math.log10(SH) - 12.0) < 1e-6


def test_ph_acetic_acid_textbook():
    """0.1 M acetic acid (pK_a 4.76) has pH 2.88; Eq. 7 converts acetate COD
    by 64 kgCOD/kmol."""
    p = I.default_params()
    C = 0.1
    SH, _, _ = O.charge_solve(p, 298.15, state(S_ac=64.0 * C))
    Ka = 10 ** -4.76
    exact = (-Ka + math.sqrt(Ka * Ka + 4 * Ka * C)) / 2  # K_w negligible (<1e-8 rel.)
    assert abs(SH / exact - 1) < 1e-7
    assert abs(-math.log10(SH) - 2.88) < 0.005


@pytest.mark.parametrize("acid,cod,pka", [("S_pro", 112.0, 4.88), ("S_bu", 160.0, 4.82),
                                          ("S_va", 208.0, 4.86)])
def test_ph_other_vfa_cod_divisors(acid, cod, pka):
    """Each VFA enters Eq. 7 through its own COD-per-kmol divisor."""
    p = I.default_params()
    C = 0.02
    SH, _, _ = O.charge_solve(p, 298.15, state(**{acid: cod * C}))
    Ka = 10 ** -pka
    exact = (-Ka + math.sqrt(Ka * Ka + 4 * Ka * C)) / 2
    assert abs(SH / exact - 1) < 1e-7


def test_ph_ammonia_and_carbonate_polynomial_roots():
    """0.1 M NH3 solution: pH 11.12 (pK_b 4.75); the exact root of the cubic
    S^3 + (K_a + C) S^2 - K_w S - K_w K_a = 0 by numpy.roots.  Dissolved CO2
    with a strong base: cubic from the one-proton carbonate system."""
    p = I.default_params()
    C = 0.1
    SH, _, _ = O.charge_solve(p, 298.15, state(S_IN=C))
    Ka, Kw = 10 ** -9.25, 10 ** -14
    r = np.roots([1.0, Ka + C, -Kw, -Kw * Ka])
    root = max(x.real for x in r if abs(x.imag) < 1e-30 and x.real > 0)
    assert abs(SH / root - 1) < 1e-9
    assert abs(-math.log10(SH) - 11.12) < 0.01
    # S_IC + S_cat:  S^3 + (Ka + cat) S^2 + (cat Ka - Ka IC - Kw) S - Kw Ka = 0
    IC, cat = 0.1, 0.05
    Ka = 10 ** -6.35
    SH, _, _ = O.charge_solve(p, 298.15, state(S_IC=IC, S_cat=cat))
    r = np.roots([1.0, Ka + cat, cat * Ka - Ka * IC - Kw, -Kw * Ka])
    root = max(x.real for x in r if abs(x.imag) < 1e-30 and x.real > 0)
    assert abs(SH / root - 1) < 1e-8
    assert abs(-math.log10(SH) - 6.35) < 0.01  # half-neutralised: pH = pK_a


def test_newton_matches_bisection_on_realistic_states():
    """E is strictly increasing, so Newton and bisection find the same unique root."""
    p = I.default_params()
    ys = perturbed_ss(7, n=40)
    rng = np.random.default_rng(3)
    for k in range(ys.shape[1]):
        T = rng.uniform(303.15, 313.15)
        for guess in (1e-7, 1e-3, 1e-12, 0.5):
            SH, it, bis = O.charge_solve(p, T, ys[:, k], guess)
            SB = O.charge_bisect(p, T, ys[:, k])
            assert abs(SH / SB - 1) < 1e-12
        assert abs(O.charge_residual(p, T, ys[:, k], SH)) < 1e-14


def test_newton_iteration_limit_falls_back():
    p = I.default_params()
    y = I.x_ss()
    SH, it, bis = O.charge_solve(p, 308.15, y, 1e-3, max_iters=1)
    assert bis == 1
    SB = O.charge_bisect(p, 308.15, y)
    assert abs(SH / SB - 1) < 1e-15


# ----------------------------------------------------------------- Jacobian
def test_jacobian_ad_matches_central_differences():
    p = I.default_params()
    T = 310.0
    y = perturbed_ss(11)
    yin, D = I.influent(), 0.3
    J = O.jacobian(p, T, y, y_in=yin, D=D)
    Jfd = np.zeros_like(J)
    for k in range(I.NS):
        h = 1e-3 * max(abs(y[k]), 1e-9)  # balances Richardson truncation and round-off

        def d(hh):
            yp, ym = y.copy(), y.copy()
            yp[k] += hh
            ym[k] -= hh
            return (O.rhs(p, T, yp, y_in=yin, D=D)[0] - O.rhs(p, T, ym, y_in=yin, D=D)[0]) / (2 * hh)
        Jfd[:, k] = (4 * d(h / 2) - d(h)) / 3  # Richardson: O(h^4)
    scale = np.abs(J).max(axis=0, keepdims=True) + 1e-300
    assert np.max(np.abs(J - Jfd) / scale) < 1e-7


# ----------------------------------------------------------------- integrator
def test_rosenbrock_second_order_convergence():
    """Fixed-step W-method errors shrink 4x per halving of h (order 2)."""
    p = I.default_params()
    y0, SH, h, st, _ = O.integrate(p, 308.15, perturbed_ss(5), 0.05, rtol=1e-10,
                                   atol=I.atol_vector(1e-12))
    dt = 0.02
    ref = O.rk4(p, 308.15, y0, dt, 40000)
    errs = []
    for n in (4, 8, 16, 32):
        y, *_ = O.integrate(p, 308.15, y0, dt, fixed_n=n)
        errs.append(np.max(np.abs(y - ref) / (np.abs(ref) + 1e-6 * np.abs(ref).max())))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert all(1.7 < r < 2.4 for r in rates), (errs, rates)


def test_local_error_is_third_order_on_nonstiff_species():
    """One W-method step has an O(h^3) local error on the slow species (8x per
    halving), checked against brute-force RK4; the stiff S_h2 (h*lambda >> 1)
    shows the known order reduction of linearly implicit methods, but still
    at least O(h^2)."""
    p = I.default_params()
    y0, *_ = O.integrate(p, 308.15, perturbed_ss(6), 0.05, rtol=1e-10, atol=I.atol_vector(1e-12))
    errs = []
    for H in (150.0, 75.0, 37.5):
        dt = H / 86400
        ref = O.rk4(p, 308.15, y0, dt, int(H / 0.005))
        y1, *_ = O.integrate(p, 308.15, y0, dt, fixed_n=1)
        errs.append(np.abs(y1 - ref) / np.abs(y0))
    for sp in ("X_c", "S_IC", "X_ch", "S_ac"):
        r = [errs[i][S[sp]] / errs[i + 1][S[sp]] for i in range(2)]
        assert all(6.0 < x < 10.0 for x in r), (sp, r)
    r = [errs[i][S["S_h2"]] / errs[i + 1][S["S_h2"]] for i in range(2)]
    assert all(x > 3.5 for x in r), r


def test_rk4_brute_force_agreement():
    """Explicit RK4 at h = 0.005 s over 864 s agrees with the adaptive W-method
    at rtol 1e-12 on a steady-state particle and a 20x substrate slug."""
    p = I.default_params()
    for k, slug in enumerate((False, True)):
        y0 = perturbed_ss(20 + k)
        if slug:
            for s in ("S_su", "S_aa", "X_ch"):
                y0[S[s]] *= 20
        dt = 864.0 / 86400.0
        yr = O.rk4(p, 308.15, y0, dt, 172800)
        ya, *_ , st, stats = O.integrate(p, 308.15, y0, dt, rtol=1e-12, atol=I.atol_vector(1e-15),
                                         max_steps=10 ** 6)
        assert st == 0
        rel = np.abs(ya - yr) / np.maximum(np.abs(yr), 1e-12 * np.abs(yr).max())
        assert rel.max() < 1e-9, (slug, rel.max())


# ----------------------------------------------------------------- S_h2 algebraic (Eq. 8)
def test_h2_algebraic_root_zeroes_the_h2_balance():
    """The algebraic mode's S_h2 is the root of Eq. 8: the differential
    right-hand side at that S_h2 (same S_H) has a zero S_h2 rate, the balance
    changes sign across it (it decreases in S_h2), and every other rate is
    that right-hand side's."""
    p, T, yin, D = I.default_params(), 310.0, I.influent(), 0.3
    for seed in range(5):
        y = perturbed_ss(40 + seed)
        f, SH, SH2 = O.rhs_h2alg(p, T, y, y_in=yin, D=D)
        yy = y.copy()
        yy[S["S_h2"]] = SH2
        fo = O.rhs_at(p, T, yy, SH, y_in=yin, D=D)
        rho, _ = O.rates_at(p, T, yy, SH)
        assert abs(fo[S["S_h2"]]) <= 1e-13 * (abs(rho[11]) + abs(rho[19]))
        assert f[S["S_h2"]] == 0.0
        other = np.arange(I.NS) != S["S_h2"]
        assert np.array_equal(f[other], fo[other])
        for fac, sign in ((0.9, 1.0), (1.1, -1.0)):
            yy[S["S_h2"]] = fac * SH2
            assert sign * O.rhs_at(p, T, yy, SH, y_in=yin, D=D)[S["S_h2"]] > 0.0


def test_h2_algebraic_jacobian_matches_central_differences():
    """Dual-number Jacobian of the algebraic mode (through the Eq. 7 and Eq. 8
    roots) against Richardson central differences of its right-hand side,
    which re-solves both roots; the S_h2 row and column are zero."""
    p, T, yin, D = I.default_params(), 310.0, I.influent(), 0.3
    y = perturbed_ss(12)
    J = O.jacobian_h2alg(p, T, y, y_in=yin, D=D)
    Jfd = np.zeros_like(J)
    for k in range(I.NS):
        h = 1e-3 * max(abs(y[k]), 1e-9)

        def d(hh):
            yp, ym = y.copy(), y.copy()
            yp[k] += hh
            ym[k] -= hh
            return (O.rhs_h2alg(p, T, yp, y_in=yin, D=D)[0] -
                    O.rhs_h2alg(p, T, ym, y_in=yin, D=D)[0]) / (2 * hh)
        Jfd[:, k] = (4 * d(h / 2) - d(h)) / 3
    assert np.all(J[S["S_h2"], :] == 0.0) and np.all(J[:, S["S_h2"]] == 0.0)
    scale = np.abs(J).max(axis=0, keepdims=True) + 1e-300
    cols = np.arange(I.NS) != S["S_h2"]
    assert np.max(np.abs(J - Jfd)[:, cols] / scale[:, cols]) < 1e-7


def test_h2_algebraic_fixed_steps_converge_and_store_the_root():
    """Brute force in the algebraic mode: 2000 fixed W-method steps over one
    60-s interval agree with the adaptive integration at rtol 1e-11, and the
    S_h2 stored at the end is the Eq. 8 root of the final state."""
    p = I.default_params()
    y0 = perturbed_ss(50)
    dt = 60.0 / 86400.0
    ya, _, _, st, _ = O.integrate(p, 308.15, y0, dt, rtol=1e-11, atol=I.atol_vector(1e-14),
                                  max_steps=10 ** 6, h2_algebraic=True)
    assert st == 0
    yf, *_ = O.integrate(p, 308.15, y0, dt, fixed_n=2000, h2_algebraic=True)
    rel = np.abs(yf - ya) / np.maximum(np.abs(ya), 1e-12 * np.abs(ya).max())
    assert rel.max() < 1e-8, rel.max()
    _, _, SH2 = O.rhs_h2alg(p, 308.15, ya)
    assert abs(SH2 / ya[S["S_h2"]] - 1.0) < 1e-12


def test_h2_algebraic_and_differential_forms_agree():
    """Eq. 8 replaces a fast S_h2 (time scale well below a second) by its
    quasi-steady value; over one day of a closed batch the two forms agree to
    1e-5 in every species at a tight tolerance."""
    p = I.default_params()
    y0 = perturbed_ss(51)
    yo, *_ = O.integrate(p, 308.15, y0, 1.0, rtol=1e-10, atol=I.atol_vector(1e-13))
    yd, *_ = O.integrate(p, 308.15, y0, 1.0, rtol=1e-10, atol=I.atol_vector(1e-13),
                         h2_algebraic=True)
    rel = np.abs(yd - yo) / np.maximum(np.abs(yo), 1e-12 * np.abs(yo).max())
    assert rel.max() < 1e-5, rel.max()


# ----------------------------------------------------------------- particles (Sec. 2.3, 3.1, 4.2)
def _uniform_population(n, shared):
    p = I.default_params()
    y = np.repeat(perturbed_ss(31)[:, None], n, axis=1)
    D = I.TABLE1["Q"] / I.TABLE1["V_liq"]
    dg = [I.Digester(n=n, D=D)]
    pop = I.Population(dg, y, np.full(n, I.T_OP), np.zeros((3, n)), shared)
    return pop, p, D


@pytest.mark.parametrize("shared", [False, True])
def test_uniform_particles_equal_single_cstr(shared):
    """Sec. 3.1: one particle is a CSTR; Sec. 4.2: identical particles without
    diffusion stay identical.  N identical particles (per-particle or shared
    headspace) reproduce the single-CSTR solution of the Table 1 tank."""
    n = 8
    pop, p, D = _uniform_population(n, shared)
    r = O.run(pop, 60.0, 20, rtol=1e-6)
    y, SH, h = pop.y[:, 0].copy(), 1e-7, 0.0
    for _ in range(20):
        y, SH, h, st, _ = O.integrate(p, I.T_OP, y, 60.0 / 86400.0, rtol=1e-6,
                                      atol=I.atol_vector(), y_in=I.influent(), D=D, SH=SH, h=h)
    spread = np.abs(r["y"] - r["y"][:, :1]).max()
    assert spread == 0.0
    if shared:
        assert np.max(np.abs(r["y"][:, 0] - y) / np.abs(y)) < 1e-14
    else:
        assert np.array_equal(r["y"][:, 0], y)


# ----------------------------------------------------------------- advection
def test_philox_matches_numpy():
    """Philox4x64-10 agrees with numpy's independent implementation."""
    for key, ctr in (((0, 0), (0, 0, 0, 0)), ((123456789, 987654321), (5, 7, 11, 13)),
                     ((2**64 - 1, 2**63 + 5), (2**64 - 2, 1, 2, 3))):
        bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                              counter=np.array(ctr, dtype=np.uint64))
        got = bg.random_raw(4)
        # numpy increments the counter before producing a block
        c = list(ctr)
        c[0] = (c[0] + 1) % 2**64
        if c[0] == 0:
            c[1] = (c[1] + 1) % 2**64
        mine = O.philox4x64_10(c, key)
        assert np.array_equal(np.asarray(got, dtype=np.uint64), mine), (key, ctr)


def test_irwin_hall_moments():
    g = np.array([O.gauss(7, pid, 3, k, a) for pid in range(200) for k in range(10) for a in range(3)])
    assert abs(g.mean()) < 0.05 and abs(g.var() - 1.0) < 0.06
    assert np.all(np.abs(g) <= 6.0)


def _flow_population(n, sigma, seed=5):
    rng = np.random.default_rng(seed)
    R, H = 0.1, 0.3
    pos = I.cylinder_positions(n, R, H, rng)
    y = np.repeat(I.x_ss()[:, None], n, axis=1)
    V = math.pi * R * R * H
    dg = [I.Digester(n=n, V_liq=V, V_gas=V * 300 / 3400,
                     flow=I.swirl_flow(R=R, H=H, sigma=sigma, seed=seed))]
    return I.Population(dg, y, np.full(n, I.T_OP), pos, False), R, H


def test_advection_zero_noise_is_rigid_rotation():
    pop, R, H = _flow_population(16, 0.0)
    r = O.run(pop, 60.0, 2, rtol=1e-4)
    w = 0.05 / R
    th = 120 * w * 1.0
    x0, y0, z0 = pop.pos
    xe = x0 * math.cos(th) - y0 * math.sin(th)
    ye = x0 * math.sin(th) + y0 * math.cos(th)
    assert np.max(np.abs(r["pos"][0] - xe)) < 1e-12
    assert np.max(np.abs(r["pos"][1] - ye)) < 1e-12
    assert np.array_equal(r["pos"][2], z0)


def test_advection_stays_in_cylinder_and_moves():
    pop, R, H = _flow_population(64, 0.005)
    r = O.run(pop, 60.0, 5, rtol=1e-4)
    x, y, z = r["pos"]
    assert np.all(np.hypot(x, y) <= R * (1 + 1e-15))
    assert np.all((z >= 0) & (z <= H))
    assert np.abs(r["pos"] - pop.pos).max() > 1e-3


# ----------------------------------------------------------------- diffusion between particles
DIFF = ["S_su", "S_aa", "S_fa", "S_va", "S_bu", "S_pro", "S_ac", "S_h2", "S_ch4", "S_IC", "S_IN",
        "S_I", "S_cat", "S_an"]


def _lattice(n1, dx):
    g = np.arange(n1) * dx
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()])


def test_diffusion_conserves_and_leaves_uniform_fields():
    """Pairwise antisymmetric fluxes: the total of every diffusing species is
    conserved to round-off, a uniform field does not change, and the
    particulate and gas states are untouched."""
    rng = np.random.default_rng(3)
    n = 600
    pos = rng.uniform(0.0, 0.05, (3, n))
    y = perturbed_ss(60, n)
    y2 = O.diffuse(pos, y, V=(0.05 ** 3) / n, D=1e-6, h=0.006, dt_s=60.0, n_sub=20)
    for sp in DIFF:
        i = S[sp]
        assert abs(y2[i].sum() - y[i].sum()) <= 1e-13 * np.abs(y[i]).sum(), sp
        assert np.any(y2[i] != y[i]), sp
    others = [i for i in range(I.NS) if I.STATE_NAMES[i] not in DIFF]
    assert np.array_equal(y2[others], y[others])
    u = np.tile(I.x_ss()[:, None], (1, n))
    assert np.array_equal(O.diffuse(pos, u, (0.05 ** 3) / n, 1e-6, 0.006, 60.0, 20), u)


def test_diffusion_operator_approximates_the_laplacian():
    """On a cubic lattice the SPH operator applied to C = 1 + e sin(k x) gives
    dC/dt = D Laplacian(C) = -D k^2 e sin(k x) at particles farther than the
    kernel support from the walls, to the discretisation error (within 3 %
    at h = 1.6 dx, k h = 0.28)."""
    dx, n1 = 0.004, 18
    pos = _lattice(n1, dx)
    n = pos.shape[1]
    h, D = 1.6 * dx, 1e-6
    k = 2 * np.pi / (2 * n1 * dx)
    y = np.tile(I.x_ss()[:, None], (1, n))
    y[S["S_ac"]] = 1.0 + 1e-3 * np.sin(k * pos[0])
    dt = 1e-3
    y1 = O.diffuse(pos, y, dx ** 3, D, h, dt, 1)
    rate = (y1[S["S_ac"]] - y[S["S_ac"]]) / dt
    exact = -D * k * k * 1e-3 * np.sin(k * pos[0])
    inner = np.all((pos > 2 * h) & (pos < (n1 - 1) * dx - 2 * h), axis=0)
    sel = inner & (np.abs(np.sin(k * pos[0])) > 0.3)
    ratio = rate[sel] / exact[sel]
    assert sel.sum() > 100 and np.all(np.abs(ratio - 1.0) < 0.03), (ratio.min(), ratio.max())



def test_diffusion_row_sum_tends_to_the_continuum_integral():
    """The operator's row sum sum_j |w_ij| at an inner lattice particle is a
    quadrature of 8 pi D int_0^2h r^3 |W'(r)| / (r^2 + 0.01 h^2) dr, which
    for the Wendland C2 kernel without the 0.01 h^2 term is 7 D / h^2
    exactly (a Beta(3,4) integral); the quadrature error falls as h / dx
    grows."""
    quad = pytest.importorskip("scipy.integrate").quad
    D, dx = 1e-6, 0.004
    errs = []
    for f in (2.5, 4.5):
        n1 = int(4 * f) + 5
        pos, h = _lattice(n1, dx), f * dx
        alpha = 21.0 / (16.0 * np.pi * h ** 3)
        dw = lambda r: 5.0 * alpha * (r / h) * (1.0 - r / (2.0 * h)) ** 3 / h
        cont = quad(lambda r: 8 * np.pi * D * r ** 3 * dw(r) / (r * r + 0.01 * h * h), 0, 2 * h)[0]
        bare = quad(lambda r: 8 * np.pi * D * r * dw(r), 0, 2 * h)[0]
        assert abs(bare / (7.0 * D / h ** 2) - 1.0) < 1e-10
        errs.append(abs(O.diffusion_row_sum_max(pos, dx ** 3, D, h) / cont - 1.0))
    assert errs[1] < 0.005 and errs[1] < errs[0] < 0.03, errs


def test_diffusion_substep_rule_keeps_a_maximum_principle():
    """With ceil(dt S_max) substeps every Euler update is a convex
    combination of the old values, so no species leaves the range of its
    initial values, also for crowded particles (h about the spacing), where
    the continuum estimate 7 D / h^2 of the row sum is far too optimistic.
    A quarter of the substeps overshoots."""
    rng = np.random.default_rng(11)
    n, L, D, h, dt = 400, 0.02, 1e-5, 0.004, 2.0
    pos = rng.uniform(0.0, L, (3, n))
    pos[:, : n // 4] = pos[:, : n // 4] * 0.1 + 0.5 * L     # a dense cluster
    y = perturbed_ss(7, n)
    y[S["S_ac"]] = rng.uniform(0.0, 1.0, n)
    V = L ** 3 / n
    smax = O.diffusion_row_sum_max(pos, V, D, h)
    assert smax > 5 * 7 * D / h ** 2                            # crowding matters
    nsub = O.diffusion_substeps(dt, smax)
    y2 = O.diffuse(pos, y, V, D, h, dt, nsub)
    for sp in DIFF:
        i = S[sp]
        lo, hi = y[i].min(), y[i].max()
        assert y2[i].min() >= lo - 1e-12 * abs(lo) and y2[i].max() <= hi + 1e-12 * abs(hi), sp
    y3 = O.diffuse(pos, y, V, D, h, dt, max(1, nsub // 4))
    assert y3[S["S_ac"]].min() < 0.0 or y3[S["S_ac"]].max() > 1.0
