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
    sys.path.insert(0, os.path.join(ROOT, "paper_2311_08927_gb300", "csrc"))
    import gen_sparse as G
    src, info = G.generate(G.jacobian_pattern())
    with open(G.OUT) as fh:
        assert fh.read() == src, "sparse_lu_gen.cuh is stale: rerun gen_sparse.py"


def test_jacobian_nonzeros_have_sparse_slots():
    sys.path.insert(0, os.path.join(ROOT, "paper_2311_08927_gb300", "csrc"))
    import gen_sparse as G
    pat = G.jacobian_pattern()
    F = G.symbolic_fill(pat, G.markowitz(pat))
    for p, T, y, D, V in _cases(40, 17):
        _, J, _ = CH.eval_model(p, T, y, y_in=I.influent(), D=D)
        assert not np.any((J != 0) & ~pat)
    # fill only adds entries; the pattern includes the diagonal
    assert np.all(np.diag(pat)) and F.sum() >= pat.sum()
