"""More pins of the CPU oracle: the rate-law factors and stoichiometric routes
that the conservation laws alone cannot see.

A swapped product fraction (say f_bu,su for f_pro,su) keeps COD, C and N
closed; a free-ammonia inhibition written on the ammonium ion, a c4 uptake
split with its states exchanged or a decay rate on the wrong biomass keep
every invariant too.  Each test below isolates one such term and checks it
against the definition of the standard ADM1 (Batstone et al. 2002, the
model the paper takes its Sec. 2.2 Eq. 2-6 from) or against printed
constants, so that such a mistake fails.

Paper basis: Sec. 2.2 Eq. 2 (mass balances with the ADM1 stoichiometry),
Eq. 3-6 (inhibition and limitation factors), Table 1 (35 C operation).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2311_08927_gb300 import inputs as I

S = I.SIDX
P = I.PIDX
BIO = ["X_su", "X_aa", "X_fa", "X_c4", "X_pro", "X_ac", "X_h2"]
T35 = 308.15  # the kinetic reference temperature: Arrhenius factor 1


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


# ----------------------------------------------------------------- Eq. 6: I_IN
@pytest.mark.parametrize("proc", [4, 5, 6, 7, 8, 9, 10, 11])
def test_inorganic_nitrogen_limitation_is_monod_in_S_IN(proc):
    """Every uptake carries I_IN = S_IN/(K_S,IN + S_IN): a Monod factor, so
    the rate at S_IN = K_S,IN is 1/2 of saturation and at 3 K_S,IN it is 3/4
    (ratio 2/3), whatever the rest of the rate.  Acetate uptake also carries
    the free-ammonia inhibition, which depends on S_IN; it is switched off
    here for that process only (its own pin follows)."""
    p = params(K_I_nh3=1e300)
    K = p[P["K_S_IN"]]
    y = state(S_su=1.0, S_aa=1.0, S_fa=1.0, S_va=1.0, S_bu=1.0, S_pro=1.0, S_ac=1.0,
              S_h2=1e-6, **{b: 1.0 for b in BIO})
    r = {}
    for m in (1.0, 3.0, 1e9):
        y[S["S_IN"]] = m * K
        r[m], _ = O.rates_at(p, T35, y, 1e-9)
    assert abs(r[1.0][proc] / r[3.0][proc] - 2.0 / 3.0) < 1e-13
    # and half of the saturated rate (1e9 K_S,IN: I_IN = 1 - 1e-9)
    assert abs(r[1.0][proc] / r[1e9][proc] - 0.5) < 2e-9


# ----------------------------------------------------------------- Eq. 5: I_nh3
@pytest.mark.parametrize("pH", [7.0, 7.5, 8.5])
def test_free_ammonia_inhibition_half_point(pH):
    """Acetoclastic uptake is inhibited by free ammonia, S_nh3 = K_a,IN S_IN /
    (K_a,IN + S_H), non-competitively: the rate halves where S_nh3 = K_I,nh3.
    At 25 C the van 't Hoff factor is 1 and K_a,IN is the textbook ammonium
    constant 10^-9.25.  The reference rate is the same state with the
    inhibition removed, so I_IN and the pH factor cancel.  Written on the
    ammonium ion S_IN - S_nh3 instead, the ratio would be far from 1/2 at
    every pH tested (the two differ by the factor S_H/K_a,IN)."""
    T = 298.15
    p = I.default_params()
    SH = 10.0 ** -pH
    Ka = 10.0 ** -9.25
    S_IN = p[P["K_I_nh3"]] * (Ka + SH) / Ka
    y = state(S_ac=10.0, X_ac=1.0, S_IN=S_IN)
    r, _ = O.rates_at(p, T, y, SH)
    r0, _ = O.rates_at(params(K_I_nh3=1e300), T, y, SH)
    assert abs(r[10] / r0[10] - 0.5) < 1e-12
    # the other uptakes do not see free ammonia
    y2 = state(S_su=1.0, X_su=1.0, S_h2=1e-6, X_h2=1.0, S_IN=S_IN)
    a, _ = O.rates_at(p, T, y2, SH)
    b, _ = O.rates_at(params(K_I_nh3=1e300), T, y2, SH)
    assert a[4] == b[4] and a[11] == b[11]


# ----------------------------------------------------------------- c4 uptake split
def test_c4_uptake_split_is_symmetric():
    """Valerate and butyrate degraders are one population X_c4 with one K_S;
    each uptake is weighted by its substrate's share of S_va + S_bu.  With
    equal concentrations the two rates are equal."""
    p = I.default_params()
    for c in (1e-3, 0.05, 2.0):
        y = state(S_va=c, S_bu=c, X_c4=1.0, S_IN=1.0)
        r, _ = O.rates_at(p, T35, y, 1e-9)
        assert r[7] > 0 and abs(r[7] / r[8] - 1) < 1e-15


def test_c4_uptake_tends_to_single_substrate_monod():
    """With one of the two acids absent, the other's share tends to 1 (the
    1e-6 guard of the standard form aside) and its uptake is the plain Monod
    rate k_m,c4 X_c4 S/(K_S,c4 + S) I_IN; the absent acid's uptake is 0.  An
    exchanged split (valerate weighted by butyrate's share) would give 0 and
    the Monod rate the other way round."""
    p = I.default_params()
    k, K, KIN = p[P["k_m_c4"]], p[P["K_S_c4"]], p[P["K_S_IN"]]
    X, S_IN = 2.0, 1.0
    for present, absent, proc, other in (("S_va", "S_bu", 7, 8), ("S_bu", "S_va", 8, 7)):
        for c in (0.01, 0.3, 5.0):
            y = state(X_c4=X, S_IN=S_IN, **{present: c})
            r, _ = O.rates_at(p, T35, y, 1e-10)  # pH 10: no pH inhibition
            monod = k * X * c / (K + c) * S_IN / (S_IN + KIN)
            assert r[other] == 0.0
            # share c/(c + 1e-6) and the pH factor (1 - ~1e-12) away from 1
            assert abs(r[proc] / monod - 1) < 1.5e-6 / c, (present, c)


# ----------------------------------------------------------------- decay
def test_biomass_decay_closed_form():
    """With uptake switched off (k_m = 0), each biomass decays at its own
    first-order rate, X(t) = X(0) exp(-k_dec t), and the decayed mass feeds
    the composite X_c, which disintegrates at k_dis: X_c(t) = sum over the
    populations of k_dec X(0) (e^(-k_dec t) - e^(-k_dis t)) / (k_dis - k_dec).
    The seven decay constants are made distinct, so a rate applied to the
    wrong population fails."""
    kdec = dict(zip(BIO, (0.011, 0.023, 0.037, 0.052, 0.068, 0.085, 0.103)))
    over = {f"k_dec_{b}": v for b, v in kdec.items()}
    over.update({k: 0.0 for k in ("k_m_su", "k_m_aa", "k_m_fa", "k_m_c4", "k_m_pro", "k_m_ac",
                                  "k_m_h2")})
    over["k_La"] = 0.0
    p = params(**over)
    X0 = dict(zip(BIO, (0.4, 0.9, 0.3, 0.5, 0.2, 0.7, 0.6)))
    y0 = state(S_IC=0.05, S_IN=0.05, S_cat=0.04, S_an=0.02, **X0)
    t = 2.0
    y, SH, h, st, _ = O.integrate(p, T35, y0, t, rtol=1e-12, atol=np.full(I.NS, 1e-16))
    assert st == 0
    kdis = p[P["k_dis"]]
    xc = 0.0
    for b in BIO:
        k = kdec[b]
        assert abs(y[S[b]] / (X0[b] * math.exp(-k * t)) - 1) < 1e-10, b
        xc += k * X0[b] * (math.exp(-k * t) - math.exp(-kdis * t)) / (kdis - k)
    assert abs(y[S["X_c"]] / xc - 1) < 1e-9


# ----------------------------------------------------------------- Petersen routing
# Standard ADM1 stoichiometry of each process, by name: (substrate, products
# with their yields per unit of substrate COD taken up).
def _routes(p):
    g = lambda k: p[P[k]]
    return {
        0: ("X_c", {"S_I": g("f_sI_xc"), "X_I": g("f_xI_xc"), "X_ch": g("f_ch_xc"),
                    "X_pr": g("f_pr_xc"), "X_li": g("f_li_xc")}),
        1: ("X_ch", {"S_su": 1.0}),
        2: ("X_pr", {"S_aa": 1.0}),
        3: ("X_li", {"S_su": 1.0 - g("f_fa_li"), "S_fa": g("f_fa_li")}),
        4: ("S_su", {"S_bu": (1 - g("Y_su")) * g("f_bu_su"), "S_pro": (1 - g("Y_su")) * g("f_pro_su"),
                     "S_ac": (1 - g("Y_su")) * g("f_ac_su"), "S_h2": (1 - g("Y_su")) * g("f_h2_su"),
                     "X_su": g("Y_su")}),
        5: ("S_aa", {"S_va": (1 - g("Y_aa")) * g("f_va_aa"), "S_bu": (1 - g("Y_aa")) * g("f_bu_aa"),
                     "S_pro": (1 - g("Y_aa")) * g("f_pro_aa"), "S_ac": (1 - g("Y_aa")) * g("f_ac_aa"),
                     "S_h2": (1 - g("Y_aa")) * g("f_h2_aa"), "X_aa": g("Y_aa")}),
        6: ("S_fa", {"S_ac": (1 - g("Y_fa")) * g("f_ac_fa"), "S_h2": (1 - g("Y_fa")) * g("f_h2_fa"),
                     "X_fa": g("Y_fa")}),
        7: ("S_va", {"S_pro": (1 - g("Y_c4")) * g("f_pro_va"), "S_ac": (1 - g("Y_c4")) * g("f_ac_va"),
                     "S_h2": (1 - g("Y_c4")) * g("f_h2_va"), "X_c4": g("Y_c4")}),
        8: ("S_bu", {"S_ac": (1 - g("Y_c4")) * g("f_ac_bu"), "S_h2": (1 - g("Y_c4")) * g("f_h2_bu"),
                     "X_c4": g("Y_c4")}),
        9: ("S_pro", {"S_ac": (1 - g("Y_pro")) * g("f_ac_pro"), "S_h2": (1 - g("Y_pro")) * g("f_h2_pro"),
                      "X_pro": g("Y_pro")}),
        10: ("S_ac", {"S_ch4": 1 - g("Y_ac"), "X_ac": g("Y_ac")}),
        11: ("S_h2", {"S_ch4": 1 - g("Y_h2"), "X_h2": g("Y_h2")}),
    }


_BIOMASS_OF = {4: "X_su", 5: "X_aa", 6: "X_fa", 7: "X_c4", 8: "X_c4", 9: "X_pro", 10: "X_ac",
               11: "X_h2"}


@pytest.mark.parametrize("proc", list(range(12)))
def test_petersen_routes_each_process_to_its_named_products(proc):
    """Isolate one process: only its substrate (and, for an uptake, its
    biomass) is present, gas transfer and decay are off, S_H is given.  Then
    f = nu rho for that process alone: the substrate falls at rho, each named
    product rises at its yield times rho, carbon and nitrogen go to S_IC and
    S_IN (their closure is pinned elsewhere), and nothing else moves.  The
    ADM1 default fractions of one process all differ, so exchanging two of
    them fails here."""
    over = {f"k_dec_{b}": 0.0 for b in BIO}
    over["k_La"] = 0.0
    p = params(**over)
    sub, prods = _routes(p)[proc]
    kv = {sub: 0.8, "S_IN": 1.0}
    if proc in _BIOMASS_OF:
        kv[_BIOMASS_OF[proc]] = 1.5
    if proc == 11:
        kv[sub] = 2e-5
    y = state(**kv)
    f = O.rhs_at(p, T35, y, 1e-9)
    rho = -f[S[sub]]
    assert rho > 0
    if proc in _BIOMASS_OF and _BIOMASS_OF[proc] not in prods:
        prods = dict(prods)
    seen = {sub, "S_IC", "S_IN"}
    for name, yld in prods.items():
        assert abs(f[S[name]] / rho - yld) < 1e-14 * max(1.0, yld), (proc, name)
        seen.add(name)
    for name, i in S.items():
        if name not in seen:
            assert f[i] == 0.0, (proc, name, f[i])


# ----------------------------------------------------------------- temperature
def test_van_t_hoff_constants_at_35C_match_printed_values():
    """The acid-base and Henry constants and the water vapour pressure at
    35 C, as printed (three significant figures) in the ADM1 benchmark
    literature (Rosen and Jeppsson's BSM2 ADM1 report): K_w 2.08e-14,
    K_a,co2 4.94e-7, K_a,IN 1.11e-9, K_H,co2 0.0271, K_H,ch4 0.00116,
    K_H,h2 7.38e-4 M/bar, p_gas,h2o 0.0557 bar.  Each is the 25 C value
    moved by its own enthalpy, so a wrong sign, a swapped enthalpy or a
    factor left out changes the printed digits."""
    c = O.constants(I.default_params(), 308.15)
    printed = {"K_w": 2.08e-14, "K_a_co2": 4.94e-7, "K_a_IN": 1.11e-9, "K_H_co2": 0.0271,
               "K_H_ch4": 0.00116, "K_H_h2": 7.38e-4, "p_h2o": 0.0557}
    for k, v in printed.items():
        assert float(f"{c[k]:.2e}") == v, (k, c[k], v)
    assert c["arrhenius"] == 1.0


def test_neutral_ph_at_35C():
    """Pure water at 35 C: S_H = sqrt(K_w), pH 6.84 (K_w = 2.08e-14)."""
    SH, _, _ = O.charge_solve(I.default_params(), 308.15, state())
    assert abs(-math.log10(SH) - 6.84) < 0.005


def test_kinetic_constants_follow_one_arrhenius_law():
    """Disintegration, hydrolysis, uptake and decay rates all scale with the
    same factor exp(-(E_a/R)(1/T - 1/T_ref)): ln(rate) is linear in 1/T with
    slope -E_a/R = -6000 K (the reading of the temperature dependence), and
    the half-saturation constants are not scaled (the Monod half-point stays
    at K_S at every temperature)."""
    p = I.default_params()
    y = state(X_c=1.0, X_ch=1.0, S_su=0.5, X_su=1.0, S_IN=1e6)
    Ts = (303.15, 308.15, 313.15)
    rs = [O.rates_at(p, T, y, 1e-12)[0] for T in Ts]
    for proc in (0, 1, 4, 12):
        lr = [math.log(r[proc]) for r in rs]
        s1 = (lr[1] - lr[0]) / (1 / Ts[1] - 1 / Ts[0])
        s2 = (lr[2] - lr[1]) / (1 / Ts[2] - 1 / Ts[1])
        assert abs(s1 + 6000.0) < 1e-6 and abs(s2 + 6000.0) < 1e-6, proc
    assert abs(rs[1][0] - p[P["k_dis"]]) < 1e-15  # factor 1 at T_ref
    for T in (303.15, 313.15):
        y2 = state(S_su=p[P["K_S_su"]], X_su=1.0, S_IN=1e6)
        half, _ = O.rates_at(p, T, y2, 1e-12)
        y2[S["S_su"]] = p[P["K_S_su"]] * 3.0
        three, _ = O.rates_at(p, T, y2, 1e-12)
        assert abs(half[4] / three[4] - 2.0 / 3.0) < 1e-13
