"""CPU FP64 oracle for the CHAD per-particle ADM1 hot path -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It wraps ``adm1_oracle.cpp`` (built with gcc,
no FMA contraction) through ctypes and shares no code with the CUDA library.

Pinned by: tests/test_oracle_pins.py (closed forms, conservation laws,
textbook pH values, AD-vs-finite-difference Jacobian, convergence order,
brute-force RK4, numpy's Philox) and tests/test_oracle_pins_kinetics.py
(each rate-law factor, the stoichiometric route of every process, the
temperature laws against printed 35 C constants); tests/test_oracle_mutations.py
checks that planted mistakes fail them.  Absolute trajectories against the paper's
Fig. 3 / Table 3: parity unpinned (the benchmark records are not available).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "adm1_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NS = 29
NPROC = 22
FLOW_N = 7 + NS

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_lp = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_up = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (FP contraction off, portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared",
                               "-ffp-contract=off", "-pthread", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.oracle_n_params.restype = C.c_int
            L.oracle_param_name.restype = C.c_char_p
            L.oracle_param_name.argtypes = [C.c_int]
            L.oracle_petersen.argtypes = [_dp, _dp]
            L.oracle_constants.argtypes = [_dp, C.c_double, _dp]
            L.oracle_charge_residual.restype = C.c_double
            L.oracle_charge_residual.argtypes = [_dp, C.c_double, _dp, C.c_double]
            L.oracle_charge_solve.restype = C.c_double
            L.oracle_charge_solve.argtypes = [_dp, C.c_double, _dp, C.c_double, C.c_int,
                                              C.POINTER(C.c_long), C.POINTER(C.c_long)]
            L.oracle_charge_bisect.restype = C.c_double
            L.oracle_charge_bisect.argtypes = [_dp, C.c_double, _dp]
            L.oracle_rhs.restype = C.c_int
            L.oracle_rhs.argtypes = [_dp, C.c_double, C.c_double, C.c_double, C.c_double,
                                     _dp, _dp, C.c_double, _dp,
                                     C.POINTER(C.c_double), _dp]
            L.oracle_rhs_at.argtypes = [_dp, C.c_double, C.c_double, C.c_double, C.c_double,
                                        _dp, _dp, C.c_double, _dp]
            L.oracle_rates_at.argtypes = [_dp, C.c_double, C.c_double, C.c_double, _dp,
                                          C.c_double, _dp]
            L.oracle_jacobian.restype = C.c_int
            L.oracle_jacobian.argtypes = [_dp, C.c_double, C.c_double, C.c_double, C.c_double,
                                          _dp, _dp, C.c_double, _dp]
            L.oracle_integrate.restype = C.c_int
            L.oracle_integrate.argtypes = [_dp, C.c_double, C.c_double, C.c_double, C.c_double,
                                           _dp, _dp, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                           C.c_double, C.c_double, _dp, C.c_long, C.c_int, _lp,
                                           C.c_int]
            L.oracle_diffuse.argtypes = [C.c_long, _dp, _dp, C.c_double, C.c_double, C.c_double,
                                         C.c_double, C.c_int]
            L.oracle_diffusion_row_sum_max.restype = C.c_double
            L.oracle_diffusion_row_sum_max.argtypes = [C.c_long, _dp, C.c_double, C.c_double,
                                                       C.c_double]
            L.oracle_rhs_h2alg.restype = C.c_int
            L.oracle_rhs_h2alg.argtypes = [_dp, C.c_double, C.c_double, C.c_double, C.c_double,
                                           _dp, _dp, C.c_double, _dp, C.POINTER(C.c_double),
                                           C.POINTER(C.c_double)]
            L.oracle_jacobian_h2alg.restype = C.c_int
            L.oracle_jacobian_h2alg.argtypes = [_dp, C.c_double, C.c_double, C.c_double,
                                                C.c_double, _dp, _dp, C.c_double, _dp]
            L.oracle_rk4.restype = C.c_int
            L.oracle_rk4.argtypes = [_dp, C.c_double, C.c_double, C.c_double, C.c_double,
                                     _dp, _dp, C.c_double, C.c_long]
            L.oracle_philox4x64_10.argtypes = [_up, _up, _up]
            L.oracle_gauss.restype = C.c_double
            L.oracle_gauss.argtypes = [C.c_uint64] * 5
            L.oracle_run.restype = C.c_int
            L.oracle_run.argtypes = [C.c_int, _lp, _dp, _dp, _dp, _dp, _dp, _up, C.c_int,
                                     C.c_long, _dp, _dp, _dp, _dp, _dp, _ip,
                                     C.c_double, C.c_int, C.c_long, C.c_double, _dp,
                                     C.c_long, C.c_int, C.c_int, _lp, C.c_int, _dp, _dp]
            _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def param_names() -> list[str]:
    L = lib()
    return [L.oracle_param_name(i).decode() for i in range(L.oracle_n_params())]


def petersen(params) -> np.ndarray:
    out = np.zeros(26 * NPROC)
    lib().oracle_petersen(_f64(params), out)
    return out.reshape(26, NPROC)


def constants(params, T) -> dict:
    out = np.zeros(8)
    lib().oracle_constants(_f64(params), float(T), out)
    keys = ["K_w", "K_a_co2", "K_a_IN", "K_H_co2", "K_H_ch4", "K_H_h2", "p_h2o", "arrhenius"]
    return dict(zip(keys, out))


def charge_residual(params, T, y, SH) -> float:
    return lib().oracle_charge_residual(_f64(params), float(T), _f64(y), float(SH))


def charge_solve(params, T, y, guess=1e-7, max_iters=50):
    it, bis = C.c_long(0), C.c_long(0)
    r = lib().oracle_charge_solve(_f64(params), float(T), _f64(y), float(guess), int(max_iters),
                                  C.byref(it), C.byref(bis))
    return r, it.value, bis.value


def charge_bisect(params, T, y) -> float:
    return lib().oracle_charge_bisect(_f64(params), float(T), _f64(y))


def rhs(params, T, y, y_in=None, D=0.0, V_liq=3400.0, V_gas=300.0, SH_guess=1e-7):
    """Returns (f, S_H, rho[22])."""
    f = np.zeros(NS)
    rho = np.zeros(NPROC)
    SH = C.c_double(0.0)
    y_in = np.zeros(NS) if y_in is None else y_in
    st = lib().oracle_rhs(_f64(params), float(T), float(V_liq), float(V_gas), float(D),
                          _f64(y_in), _f64(y), float(SH_guess), f, C.byref(SH), rho)
    if st:
        raise RuntimeError("charge balance failed")
    return f, SH.value, rho


def rhs_at(params, T, y, SH, y_in=None, D=0.0, V_liq=3400.0, V_gas=300.0):
    f = np.zeros(NS)
    y_in = np.zeros(NS) if y_in is None else y_in
    lib().oracle_rhs_at(_f64(params), float(T), float(V_liq), float(V_gas), float(D),
                        _f64(y_in), _f64(y), float(SH), f)
    return f


def rates_at(params, T, y, SH, V_liq=3400.0, V_gas=300.0):
    """The 22 process rates at a given S_H, and q_gas/V_gas."""
    out = np.zeros(NPROC + 1)
    lib().oracle_rates_at(_f64(params), float(T), float(V_liq), float(V_gas), _f64(y),
                          float(SH), out)
    return out[:NPROC], out[NPROC]


def jacobian(params, T, y, y_in=None, D=0.0, V_liq=3400.0, V_gas=300.0, SH_guess=1e-7):
    J = np.zeros(NS * NS)
    y_in = np.zeros(NS) if y_in is None else y_in
    lib().oracle_jacobian(_f64(params), float(T), float(V_liq), float(V_gas), float(D),
                          _f64(y_in), _f64(y), float(SH_guess), J)
    return J.reshape(NS, NS)


def integrate(params, T, y, dt_days, rtol=1e-6, atol=None, y_in=None, D=0.0,
              V_liq=3400.0, V_gas=300.0, SH=1e-7, h=0.0, max_steps=100000, fixed_n=0,
              h2_algebraic=False):
    """One particle over dt_days.  Returns (y, S_H, h, status, stats[4]).
    h2_algebraic: S_h2 from its mass balance (Eq. 8) instead of as a state."""
    y = _f64(y).copy()
    atol = np.full(NS, 1e-12) if atol is None else _f64(atol)
    y_in = np.zeros(NS) if y_in is None else y_in
    SHc, hc = C.c_double(SH), C.c_double(h)
    stats = np.zeros(4, dtype=np.int64)
    st = lib().oracle_integrate(_f64(params), float(T), float(V_liq), float(V_gas), float(D),
                                _f64(y_in), y, C.byref(SHc), C.byref(hc), float(dt_days),
                                float(rtol), atol, int(max_steps), int(fixed_n), stats,
                                int(bool(h2_algebraic)))
    return y, SHc.value, hc.value, st, stats


def rhs_h2alg(params, T, y, y_in=None, D=0.0, V_liq=3400.0, V_gas=300.0, SH_guess=1e-7):
    """f(y) with S_h2 algebraic (Eq. 8): returns (f, S_H, S_h2); f[S_h2] = 0."""
    f = np.zeros(NS)
    y_in = np.zeros(NS) if y_in is None else y_in
    SH, SH2 = C.c_double(0.0), C.c_double(0.0)
    st = lib().oracle_rhs_h2alg(_f64(params), float(T), float(V_liq), float(V_gas), float(D),
                                _f64(y_in), _f64(y), float(SH_guess), f, C.byref(SH),
                                C.byref(SH2))
    if st:
        raise RuntimeError("charge balance failed")
    return f, SH.value, SH2.value


def jacobian_h2alg(params, T, y, y_in=None, D=0.0, V_liq=3400.0, V_gas=300.0, SH_guess=1e-7):
    """J = df/dy with S_h2 algebraic (Eq. 8), through both roots."""
    J = np.zeros(NS * NS)
    y_in = np.zeros(NS) if y_in is None else y_in
    lib().oracle_jacobian_h2alg(_f64(params), float(T), float(V_liq), float(V_gas), float(D),
                                _f64(y_in), _f64(y), float(SH_guess), J)
    return J.reshape(NS, NS)


def rk4(params, T, y, dt_days, n_steps, y_in=None, D=0.0, V_liq=3400.0, V_gas=300.0):
    y = _f64(y).copy()
    y_in = np.zeros(NS) if y_in is None else y_in
    st = lib().oracle_rk4(_f64(params), float(T), float(V_liq), float(V_gas), float(D),
                          _f64(y_in), y, float(dt_days), int(n_steps))
    if st:
        raise RuntimeError("charge balance failed in RK4")
    return y


def philox4x64_10(ctr, key) -> np.ndarray:
    out = np.zeros(4, dtype=np.uint64)
    lib().oracle_philox4x64_10(np.asarray(ctr, dtype=np.uint64), np.asarray(key, dtype=np.uint64), out)
    return out


def gauss(seed, pid, interval, sub, axis) -> float:
    return lib().oracle_gauss(seed, pid, interval, sub, axis)


def run(pop, dt_coupling_s, n_intervals, interval0=0, rtol=1e-6, atol=None, SH=None, h=None,
        max_steps=100000, fixed_n=0, n_threads=0, status=None, h2_algebraic=False,
        diffusion=None):
    """Integrate a Population (see paper_2311_08927_gb300.inputs) in place.
    h2_algebraic: S_h2 from its mass balance (Eq. 8) instead of as a state.
    diffusion: (D m^2/s, h m) for every digester with a flow field, or a list
    with one such pair (or None) per digester: after the advection of each
    interval, SPH diffusion between its particles.

    Returns a dict with y, pos, S_H, h, status, stats (copies)."""
    from paper_2311_08927_gb300 import inputs as I  # seeded generators only
    N = pop.n
    nd = len(pop.digesters)
    params = np.ascontiguousarray(np.stack([d.params for d in pop.digesters]), dtype=np.float64)
    V_liq = _f64([d.V_liq for d in pop.digesters])
    V_gas = _f64([d.V_gas for d in pop.digesters])
    D_u = _f64([d.D for d in pop.digesters])
    recs, seeds = zip(*[I.flow_record(d) for d in pop.digesters])
    flow = np.ascontiguousarray(np.stack(recs), dtype=np.float64)
    seeds = np.asarray(seeds, dtype=np.uint64)
    y = np.ascontiguousarray(pop.y, dtype=np.float64).copy()
    pos = np.ascontiguousarray(pop.pos, dtype=np.float64).copy()
    T = _f64(pop.T)
    SH = np.full(N, 1e-7) if SH is None else _f64(SH).copy()
    h = np.zeros(N) if h is None else _f64(h).copy()
    status = np.zeros(N, dtype=np.int32) if status is None else np.ascontiguousarray(status, dtype=np.int32).copy()
    atol = I.atol_vector() if atol is None else _f64(atol)
    stats = np.zeros(4, dtype=np.int64)
    dD = np.zeros(nd)
    dh = np.zeros(nd)
    if diffusion is not None:
        per = diffusion if isinstance(diffusion, list) else [diffusion] * nd
        for k, dg in enumerate(pop.digesters):
            if dg.flow is not None and per[k] is not None:
                dD[k], dh[k] = per[k]
    lib().oracle_run(nd, np.ascontiguousarray(pop.offsets, dtype=np.int64), params, V_liq, V_gas,
                     D_u, flow, seeds, int(pop.shared_headspace), N, pos, y, T, SH, h, status,
                     float(dt_coupling_s), int(n_intervals), int(interval0), float(rtol), atol,
                     int(max_steps), int(fixed_n), int(n_threads), stats, int(bool(h2_algebraic)),
                     dD, dh)
    return dict(y=y, pos=pos, S_H=SH, h=h, status=status, stats=stats)


def diffusion_row_sum_max(pos, V, D, h):
    """max_i sum_j |w_ij| of the SPH diffusion operator (1/s) for particles
    at pos [3][n]; ceil(dt S) Euler substeps keep each update a convex
    combination of the old values."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    return float(lib().oracle_diffusion_row_sum_max(int(pos.shape[1]), pos, float(V), float(D),
                                                    float(h)))


def diffusion_substeps(dt_s, smax):
    """The substep rule run() applies each interval: ceil(dt S_max), >= 1."""
    return max(1, int(np.ceil(dt_s * smax)))


def diffuse(pos, y, V, D, h, dt_s, n_sub):
    """SPH diffusion between particles (brute force over all pairs): n_sub
    explicit Euler steps over dt_s seconds; returns the new y [NS][n]."""
    y = np.ascontiguousarray(y, dtype=np.float64).copy()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    lib().oracle_diffuse(int(y.shape[1]), pos, y, float(V), float(D), float(h), float(dt_s),
                         int(n_sub))
    return y
