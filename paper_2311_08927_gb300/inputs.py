"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module holds values and recipes only: the ADM1 state and parameter
layouts, the parameter values of the mesophilic ADM1 set, the synthetic
influent, and the seeded generators for particle populations.  It contains
none of the method's arithmetic (no rates, no stoichiometry, no integrator),
so both the CUDA library and the CPU oracle can consume what it produces
without sharing any computation.

Paper basis: Sec. 2.2 (ADM1, Eq. 2-8), Sec. 2.3 (AD particles, V_p = V/N),
Table 1 (CSTR: V_liq 3400 m^3, V_gas 300 m^3, Q 178.45 m^3/d, 1.013 bar),
Sec. 4.3 (particles are independent).  The parameter values are the standard
ADM1 mesophilic set that the paper takes from its Ref. [14]; the paper itself
prints none of them.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# State layout (29 differential states; Sec. 2.2).  Units: kgCOD/m^3 unless
# noted; S_IC, S_IN, S_cat, S_an, S_gas_co2 in kmol/m^3.
STATE_NAMES = [
    "S_su", "S_aa", "S_fa", "S_va", "S_bu", "S_pro", "S_ac", "S_h2", "S_ch4",
    "S_IC", "S_IN", "S_I",
    "X_c", "X_ch", "X_pr", "X_li", "X_su", "X_aa", "X_fa", "X_c4", "X_pro",
    "X_ac", "X_h2", "X_I",
    "S_cat", "S_an",
    "S_gas_h2", "S_gas_ch4", "S_gas_co2",
]
NS = len(STATE_NAMES)
SIDX = {n: i for i, n in enumerate(STATE_NAMES)}

# --------------------------------------------------------------------------
# Parameter layout.  Every entry is a raw model constant; derived quantities
# (temperature scaling, stoichiometric sums) are computed by each consumer.
_PARAMS = [
    # disintegration fractions and N/C contents
    ("f_sI_xc", 0.1), ("f_xI_xc", 0.2), ("f_ch_xc", 0.2), ("f_pr_xc", 0.2),
    ("f_li_xc", 0.3),
    ("N_xc", 0.0376 / 14.0), ("N_I", 0.06 / 14.0), ("N_aa", 0.007),
    ("N_bac", 0.08 / 14.0),
    ("C_xc", 0.02786), ("C_sI", 0.03), ("C_ch", 0.0313), ("C_pr", 0.03),
    ("C_li", 0.022), ("C_xI", 0.03), ("C_su", 0.0313), ("C_aa", 0.03),
    ("C_fa", 0.0217), ("C_bu", 0.025), ("C_pro", 0.0268), ("C_ac", 0.0313),
    ("C_bac", 0.0313), ("C_va", 0.024), ("C_ch4", 0.0156),
    # product fractions
    ("f_fa_li", 0.95),
    ("f_h2_su", 0.19), ("f_bu_su", 0.13), ("f_pro_su", 0.27), ("f_ac_su", 0.41),
    ("f_h2_aa", 0.06), ("f_va_aa", 0.23), ("f_bu_aa", 0.26), ("f_pro_aa", 0.05),
    ("f_ac_aa", 0.40),
    ("f_ac_fa", 0.7), ("f_h2_fa", 0.3),
    ("f_pro_va", 0.54), ("f_ac_va", 0.31), ("f_h2_va", 0.15),
    ("f_ac_bu", 0.8), ("f_h2_bu", 0.2),
    ("f_ac_pro", 0.57), ("f_h2_pro", 0.43),
    # yields
    ("Y_su", 0.1), ("Y_aa", 0.08), ("Y_fa", 0.06), ("Y_c4", 0.06),
    ("Y_pro", 0.04), ("Y_ac", 0.05), ("Y_h2", 0.06),
    # first-order and uptake kinetics at the reference temperature, 1/d
    ("k_dis", 0.5), ("k_hyd_ch", 10.0), ("k_hyd_pr", 10.0), ("k_hyd_li", 10.0),
    ("k_m_su", 30.0), ("k_m_aa", 50.0), ("k_m_fa", 6.0), ("k_m_c4", 20.0),
    ("k_m_pro", 13.0), ("k_m_ac", 8.0), ("k_m_h2", 35.0),
    ("k_dec_X_su", 0.02), ("k_dec_X_aa", 0.02), ("k_dec_X_fa", 0.02),
    ("k_dec_X_c4", 0.02), ("k_dec_X_pro", 0.02), ("k_dec_X_ac", 0.02),
    ("k_dec_X_h2", 0.02),
    # half-saturation and inhibition constants
    ("K_S_IN", 1e-4), ("K_S_su", 0.5), ("K_S_aa", 0.3), ("K_S_fa", 0.4),
    ("K_S_c4", 0.2), ("K_S_pro", 0.1), ("K_S_ac", 0.15), ("K_S_h2", 7e-6),
    ("K_I_h2_fa", 5e-6), ("K_I_h2_c4", 1e-5), ("K_I_h2_pro", 3.5e-6),
    ("K_I_nh3", 0.0018),
    # pH inhibition limits (Eq. 3-4)
    ("pH_LL_aa", 4.0), ("pH_UL_aa", 5.5), ("pH_LL_ac", 6.0), ("pH_UL_ac", 7.0),
    ("pH_LL_h2", 5.0), ("pH_UL_h2", 6.0),
    # physico-chemical constants
    ("R", 0.083145), ("R_J", 8.3145), ("T_base", 298.15),
    ("pK_w", 14.0), ("pK_a_va", 4.86), ("pK_a_bu", 4.82), ("pK_a_pro", 4.88),
    ("pK_a_ac", 4.76), ("pK_a_co2", 6.35), ("pK_a_IN", 9.25),
    ("dH_K_w", 55900.0), ("dH_K_a_co2", 7646.0), ("dH_K_a_IN", 51965.0),
    ("K_H_co2", 0.035), ("K_H_ch4", 0.0014), ("K_H_h2", 7.8e-4),
    ("dH_K_H_co2", -19410.0), ("dH_K_H_ch4", -14240.0), ("dH_K_H_h2", -4180.0),
    ("p_h2o_base", 0.0313), ("p_h2o_theta", 5290.0),
    ("k_La", 200.0), ("k_p", 5.0e4), ("V_liq_ref", 3400.0), ("P_atm", 1.013),
    # Arrhenius scaling of the kinetic constants (project constant E_a/R)
    ("Ea_over_R", 6000.0), ("T_ref_kin", 308.15),
]
PARAM_NAMES = [n for n, _ in _PARAMS]
NP = len(PARAM_NAMES)
PIDX = {n: i for i, n in enumerate(PARAM_NAMES)}
# kinetic parameters that the 64-digester workload perturbs per digester
KINETIC_PARAMS = [n for n in PARAM_NAMES
                  if n.startswith(("k_dis", "k_hyd", "k_m_", "K_S_", "k_dec"))]


def default_params() -> np.ndarray:
    """The mesophilic ADM1 parameter vector (float64, length NP)."""
    return np.array([v for _, v in _PARAMS], dtype=np.float64)


# --------------------------------------------------------------------------
# Table 1 (single CSTR).  T_op reading: 308.15 K (35 degC).
TABLE1 = dict(V_liq=3400.0, V_gas=300.0, Q=178.45, T=308.15, P_atm=1.013)
T_OP = 308.15

# Synthetic constant influent: round project-chosen values of the magnitudes a
# municipal digester feed has (particulate COD of tens of kgCOD/m^3, soluble
# substrates 1e-3..1e-2, S_IC/S_IN ~1e-2..1e-1 kmol/m^3, S_cat > S_an).
INFLUENT = {
    "S_su": 0.01, "S_aa": 0.001, "S_fa": 0.001, "S_va": 0.001, "S_bu": 0.001,
    "S_pro": 0.001, "S_ac": 0.001, "S_h2": 1e-8, "S_ch4": 1e-5,
    "S_IC": 0.04, "S_IN": 0.01, "S_I": 0.02,
    "X_c": 2.0, "X_ch": 5.0, "X_pr": 20.0, "X_li": 5.0,
    "X_su": 0.0, "X_aa": 0.0, "X_fa": 0.0, "X_c4": 0.0, "X_pro": 0.0,
    "X_ac": 0.0, "X_h2": 0.0, "X_I": 25.0,
    "S_cat": 0.04, "S_an": 0.02,
    "S_gas_h2": 0.0, "S_gas_ch4": 0.0, "S_gas_co2": 0.0,
}


def influent() -> np.ndarray:
    return np.array([INFLUENT[n] for n in STATE_NAMES], dtype=np.float64)


def startup_state() -> np.ndarray:
    """Start vector of the steady-state run: digested sludge with an inoculum
    in every trophic group, little degradable particulate COD, moderate
    alkalinity and a methane-rich headspace.  (Starting from the raw feed
    instead is a shock load that acidifies the reactor.)"""
    y = np.full(NS, 1e-3)
    start = dict(S_h2=1e-7, S_ch4=1e-3, S_IC=0.1, S_IN=0.1, S_I=0.02,
                 X_c=0.5, X_ch=0.05, X_pr=0.05, X_li=0.05,
                 X_su=1.0, X_aa=1.0, X_fa=0.5, X_c4=0.4, X_pro=0.2, X_ac=1.0, X_h2=0.5,
                 X_I=25.0, S_cat=0.04, S_an=0.02,
                 S_gas_h2=1e-5, S_gas_ch4=1.0, S_gas_co2=0.01)
    for k, v in start.items():
        y[SIDX[k]] = v
    return y


_DATA = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")
X_SS_PATH = os.path.join(_DATA, "x_ss.json")


def x_ss() -> np.ndarray:
    """The single-CSTR steady state (Table 1, synthetic influent), written by
    oracle/make_x_ss.py.  Raises if that file has not been generated."""
    with open(X_SS_PATH) as fh:
        d = json.load(fh)
    return np.array([d["state"][n] for n in STATE_NAMES], dtype=np.float64)


def atol_vector(scale: float = 1e-9, floor: float = 1e-12) -> np.ndarray:
    """Absolute tolerances: scale * |x_ss_i| (floored) per species."""
    return np.maximum(np.abs(x_ss()), floor) * scale


# --------------------------------------------------------------------------
# Populations.
@dataclass
class Digester:
    n: int
    V_liq: float = TABLE1["V_liq"]
    V_gas: float = TABLE1["V_gas"]
    params: np.ndarray = field(default_factory=default_params)
    T: float = T_OP
    D: float = 0.0                 # uniform dilution rate (1/d) when there is no flow field
    flow: dict | None = None       # swirl field, see swirl_flow()
    y_in: np.ndarray = field(default_factory=lambda: influent())  # influent composition


@dataclass
class Population:
    digesters: list
    y: np.ndarray                  # (NS, N) float64, SoA
    T: np.ndarray                  # (N,)
    pos: np.ndarray                # (3, N)
    shared_headspace: bool = False
    note: str = ""

    @property
    def n(self) -> int:
        return self.y.shape[1]

    @property
    def offsets(self) -> np.ndarray:
        o = np.zeros(len(self.digesters) + 1, dtype=np.int64)
        o[1:] = np.cumsum([d.n for d in self.digesters])
        return o


def lognormal_states(base: np.ndarray, n: int, rng: np.random.Generator,
                     sigma: float = 0.1) -> np.ndarray:
    """y_i = base_i * exp(sigma z), z ~ N(0,1) per species and particle."""
    z = rng.standard_normal((NS, n))
    return base[:, None] * np.exp(sigma * z)


def cylinder_positions(n: int, R: float, H: float, rng: np.random.Generator) -> np.ndarray:
    """Uniform positions in a cylinder: r = R sqrt(u1), theta = 2 pi u2, z = H u3."""
    u = rng.random((3, n))
    r = R * np.sqrt(u[0])
    th = 2.0 * np.pi * u[1]
    return np.stack([r * np.cos(th), r * np.sin(th), H * u[2]])


def swirl_flow(U=0.05, R=0.1, H=0.3, sigma=0.005, slab=0.02, seed=0,
               V_tank=None, hrt_q_over_v=TABLE1["Q"] / TABLE1["V_liq"]) -> dict:
    """Prescribed swirl: rigid rotation u_theta = U r/R plus Gaussian noise of
    std sigma (m/s) per 1-s sub-step, reflecting walls; particles with
    z >= H - slab receive the influent at the Table 1 specific inflow."""
    if V_tank is None:
        V_tank = math.pi * R * R * H
    return dict(U=U, R=R, H=H, sigma=sigma, slab_zmin=H - slab,
                q_in=V_tank * hrt_q_over_v, seed=int(seed), y_in=influent())


SEED_BASE = 2311089270


def config_population(cfg: int, n: int | None = None, seed_offset: int = 0) -> Population:
    """Seeded population for one of the five workloads (n overrides the size).

    1: closed batch, N=1000, per-particle headspace, 308.15 K
    2: lab cylinder D=0.2 m, H=0.3 m, swirl + noise, inlet slab, shared headspace
    3: N=1e6, 5 % slugs (S_su, S_aa, X_ch x20), T ~ U(303.15, 313.15) K, no flow
    4: as 3 with N=2e6 and a new seed
    5: 64 digesters, N_d log-uniform in [1e4, 2e5], kinetic params x lognormal(0.2),
       own swirl speed and seed each, shared headspace per digester
    """
    rng = np.random.default_rng(SEED_BASE + cfg + seed_offset)
    base = x_ss()
    if cfg == 1:
        n = 1000 if n is None else n
        y = lognormal_states(base, n, rng)
        dg = [Digester(n=n)]
        return Population(dg, y, np.full(n, T_OP), np.zeros((3, n)), False, "closed batch")
    if cfg == 2:
        n = 100_000 if n is None else n
        R, H = 0.1, 0.3
        V = math.pi * R * R * H
        y = lognormal_states(base, n, rng)
        pos = cylinder_positions(n, R, H, rng)
        dg = [Digester(n=n, V_liq=V, V_gas=V * TABLE1["V_gas"] / TABLE1["V_liq"],
                       flow=swirl_flow(R=R, H=H, seed=SEED_BASE + 2))]
        return Population(dg, y, np.full(n, T_OP), pos, True, "lab cylinder, swirl")
    if cfg in (3, 4):
        n = (1_000_000 if cfg == 3 else 2_000_000) if n is None else n
        y = lognormal_states(base, n, rng)
        n_slug = max(1, n // 20) if n >= 20 else 0
        slugs = rng.permutation(n)[:n_slug]
        for s in ("S_su", "S_aa", "X_ch"):
            y[SIDX[s], slugs] *= 20.0
        T = rng.uniform(303.15, 313.15, n)
        dg = [Digester(n=n)]
        pop = Population(dg, y, T, np.zeros((3, n)), False, "heterogeneous stiffness")
        pop.slugs = np.sort(slugs)
        return pop
    if cfg == 5:
        nd = 64
        counts = np.floor(np.exp(rng.uniform(math.log(1e4), math.log(2e5), nd))).astype(np.int64)
        if n is not None:  # scale down keeping the log-uniform mix
            counts = np.maximum(1, np.round(counts * (n / counts.sum()))).astype(np.int64)
        R, H = 0.1, 0.3
        V = math.pi * R * R * H
        dgs = []
        kin = [PIDX[k] for k in KINETIC_PARAMS]
        for d in range(nd):
            p = default_params()
            p[kin] *= np.exp(0.2 * rng.standard_normal(len(kin)))
            U = 0.05 * math.exp(0.2 * rng.standard_normal())
            dgs.append(Digester(n=int(counts[d]), V_liq=V,
                                V_gas=V * TABLE1["V_gas"] / TABLE1["V_liq"], params=p,
                                flow=swirl_flow(U=U, R=R, H=H, seed=SEED_BASE + 500 + d)))
        N = int(counts.sum())
        y = lognormal_states(base, N, rng)
        pos = np.concatenate([cylinder_positions(int(c), R, H, rng) for c in counts], axis=1)
        return Population(dgs, y, np.full(N, T_OP), pos, True, "64 digesters")
    raise ValueError(f"unknown workload {cfg}")


# --------------------------------------------------------------------------
# Flow record layout shared by the oracle entry points and the C ABI struct.
FLOW_FIELDS = ["has_flow", "U", "R", "H", "sigma", "slab_zmin", "q_in"]


def flow_record(d: Digester) -> tuple[np.ndarray, int]:
    """Pack a digester's flow as FLOW_FIELDS + y_in (29) doubles and a seed.
    Without a flow field y_in is the digester's influent for its uniform
    dilution rate D."""
    if d.flow is None:
        rec = np.concatenate([np.zeros(len(FLOW_FIELDS)), np.asarray(d.y_in, dtype=np.float64)])
        return rec, 0
    f = d.flow
    rec = np.concatenate([[1.0, f["U"], f["R"], f["H"], f["sigma"], f["slab_zmin"], f["q_in"]],
                          np.asarray(f["y_in"], dtype=np.float64)])
    return rec, int(f["seed"])
