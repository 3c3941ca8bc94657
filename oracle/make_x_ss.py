"""Write paper_2311_08927_gb300/data/x_ss.json: the oracle's single-CSTR
steady state under the synthetic constant influent.

Table 1 CSTR (V_liq 3400 m^3, V_gas 300 m^3, Q 178.45 m^3/d, 1.013 bar) at
T_op = 308.15 K, integrated 400 days from inputs.startup_state() in 1-day
intervals at rtol 1e-8.  Calls only the oracle; the CUDA path is not involved.
"""
import hashlib
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import oracle as O  # noqa: E402
from paper_2311_08927_gb300 import inputs as I  # noqa: E402


def main():
    p = I.default_params()
    t1 = I.TABLE1
    D = t1["Q"] / t1["V_liq"]
    y = I.startup_state()
    SH, h = 1e-7, 0.0
    atol = np.full(I.NS, 1e-12)
    for _ in range(400):
        y, SH, h, st, _ = O.integrate(p, I.T_OP, y, 1.0, rtol=1e-8, atol=atol,
                                      y_in=I.influent(), D=D, V_liq=t1["V_liq"],
                                      V_gas=t1["V_gas"], SH=SH, h=h)
        if st:
            raise SystemExit(f"oracle status {st}")
    f, SH, _ = O.rhs(p, I.T_OP, y, y_in=I.influent(), D=D, SH_guess=SH)
    resid = float(np.max(np.abs(f) / np.maximum(np.abs(y), 1e-12)))
    state = {n: float(v) for n, v in zip(I.STATE_NAMES, y)}
    blob = json.dumps(state, sort_keys=True).encode()
    out = dict(state=state, pH=float(-np.log10(SH)), S_H=float(SH),
               max_rel_rate_per_day=resid, days=400, rtol=1e-8,
               sha256=hashlib.sha256(blob).hexdigest(),
               note="oracle single-CSTR steady state, synthetic influent, Table 1 tank")
    os.makedirs(os.path.dirname(I.X_SS_PATH), exist_ok=True)
    with open(I.X_SS_PATH, "w") as fh:
        json.dump(out, fh, indent=1)
    print(f"wrote {I.X_SS_PATH}: pH {out['pH']:.4f}, residual {resid:.2e} /d")


if __name__ == "__main__":
    main()
