"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's source (a term written
on the wrong species, two stoichiometric fractions exchanged, a van 't Hoff
enthalpy with the wrong sign, ...), builds it into a separate library and
runs the pins that should see it: at least one must fail.  These are the
mistakes that keep COD, C and N closed, so the conservation pins alone would
pass them.  Everything runs on the CPU; the committed oracle is not touched.
"""
import contextlib
import os
import subprocess

import pytest

import oracle as O
import test_oracle_pins_kinetics as K

_SRC = open(O._SRC).read()

# name: (original text, planted text, pins that must see it)
MUTATIONS = {
    "free ammonia read as ammonium": (
        "R I_nh3 = R(1.0) / (R(1.0) + S_nh3 / m.K_I_nh3);",
        "R I_nh3 = R(1.0) / (R(1.0) + (y[S_IN] - S_nh3) / m.K_I_nh3);",
        [lambda: K.test_free_ammonia_inhibition_half_point(7.0)]),
    "c4 uptake split exchanged": (
        "(y[S_va] / (y[S_bu] + y[S_va] + 1e-6)) * I8;",
        "(y[S_bu] / (y[S_bu] + y[S_va] + 1e-6)) * I8;",
        [K.test_c4_uptake_tends_to_single_substrate_monod]),
    "decay constant of the next population": (
        "for (int k = 0; k < 7; ++k) rho[12 + k] = m.k_dec[k] * y[bio[k]];",
        "for (int k = 0; k < 7; ++k) rho[12 + k] = m.k_dec[(k + 1) % 7] * y[bio[k]];",
        [K.test_biomass_decay_closed_form]),
    "f_bu,su and f_pro,su exchanged": (
        "nu[S_bu][4] = (1.0 - Ysu) * p[P_f_bu_su];\n  nu[S_pro][4] = (1.0 - Ysu) * p[P_f_pro_su];",
        "nu[S_bu][4] = (1.0 - Ysu) * p[P_f_pro_su];\n  nu[S_pro][4] = (1.0 - Ysu) * p[P_f_bu_su];",
        [lambda: K.test_petersen_routes_each_process_to_its_named_products(4)]),
    "f_ac,bu and f_h2,bu exchanged": (
        "nu[S_ac][8] = (1.0 - Yc4) * p[P_f_ac_bu];\n  nu[S_h2][8] = (1.0 - Yc4) * p[P_f_h2_bu];",
        "nu[S_ac][8] = (1.0 - Yc4) * p[P_f_h2_bu];\n  nu[S_h2][8] = (1.0 - Yc4) * p[P_f_ac_bu];",
        [lambda: K.test_petersen_routes_each_process_to_its_named_products(8)]),
    "K_a,co2 enthalpy with the wrong sign": (
        "vant_hoff(p, p[P_dH_K_a_co2], T)", "vant_hoff(p, -p[P_dH_K_a_co2], T)",
        [K.test_van_t_hoff_constants_at_35C_match_printed_values]),
    "K_w without its van 't Hoff factor": (
        "m.K_w = std::pow(10.0, -p[P_pK_w]) * vant_hoff(p, p[P_dH_K_w], T);",
        "m.K_w = std::pow(10.0, -p[P_pK_w]);",
        [K.test_van_t_hoff_constants_at_35C_match_printed_values, K.test_neutral_ph_at_35C]),
    "I_IN dropped from propionate uptake": (
        "R I10 = I_pH_aa * I_IN * I_h2_pro;", "R I10 = I_pH_aa * I_h2_pro;",
        [lambda: K.test_inorganic_nitrogen_limitation_is_monod_in_S_IN(9)]),
    "K_H,ch4 moved by the H2 enthalpy": (
        "m.K_H_ch4 = p[P_K_H_ch4] * vant_hoff(p, p[P_dH_K_H_ch4], T);",
        "m.K_H_ch4 = p[P_K_H_ch4] * vant_hoff(p, p[P_dH_K_H_h2], T);",
        [K.test_van_t_hoff_constants_at_35C_match_printed_values]),
}


@contextlib.contextmanager
def _oracle_lib(lib_path):
    """Point the oracle binding at another build for the duration."""
    saved = (O._lib, O._LIB, O._SRC)
    O._lib, O._LIB, O._SRC = None, lib_path, lib_path  # an existing .so newer than "source"
    try:
        yield
    finally:
        O._lib, O._LIB, O._SRC = saved


@pytest.fixture(scope="module")
def mutants(tmp_path_factory):
    d = tmp_path_factory.mktemp("mutants")
    procs = {}
    for k, (name, (a, b, _)) in enumerate(MUTATIONS.items()):
        assert _SRC.count(a) == 1, name
        src, lib = d / f"m{k}.cpp", d / f"libm{k}.so"
        src.write_text(_SRC.replace(a, b))
        procs[name] = (subprocess.Popen(["g++", "-O1", "-std=c++17", "-fPIC", "-shared",
                                         "-ffp-contract=off", "-pthread", "-o", str(lib),
                                         str(src)]), str(lib))
    out = {}
    for name, (p, lib) in procs.items():
        assert p.wait() == 0, name
        out[name] = lib
    return out


def test_committed_oracle_passes_the_same_pins():
    for _, _, pins in MUTATIONS.values():
        for pin in pins:
            pin()


@pytest.mark.parametrize("name", list(MUTATIONS))
def test_planted_mistake_fails_a_pin(name, mutants):
    pins = MUTATIONS[name][2]
    failed = 0
    with _oracle_lib(mutants[name]):
        assert os.path.exists(O.lib()._name)
        for pin in pins:
            try:
                pin()
            except AssertionError:
                failed += 1
    assert failed >= 1, f"no pin saw: {name}"
