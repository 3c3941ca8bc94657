"""Pins of the FP64 reference MLP: gradients against central finite
differences of its own loss (an independent route), and the bfloat16
rounding helper against exact bit patterns."""
import numpy as np

from oracle import mlp as M


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = rng.standard_normal(M.NPARAM) * 0.2
    X = rng.standard_normal((17, M.IN))
    Y = rng.standard_normal((17, M.OUT))
    loss, g = M.loss_and_grad(p, X, Y)
    idx = rng.choice(M.NPARAM, 60, replace=False)
    for k in idx:
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (M.loss_and_grad(pp, X, Y)[0] - M.loss_and_grad(pm, X, Y)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(g[k])), k
    assert M.NPARAM == 6402


def test_silu_network_shapes_and_zero_loss():
    p = np.zeros(M.NPARAM)
    out, _ = M.forward(p, np.ones((3, M.IN)))
    assert out.shape == (3, 2) and np.all(out == 0)
    loss, g = M.loss_and_grad(p, np.ones((3, M.IN)), np.zeros((3, 2)))
    assert loss == 0.0 and np.all(g == 0)


def test_bf16_rounding():
    v = np.array([1.0, 1.00390625, 1.005859375, -3.0, 0.0], dtype=np.float32)
    r = M.bf16_round(v)
    assert r[0] == 1.0 and r[1] == 1.0  # tie to even
    assert r[2] == np.float32(1.0078125) and r[3] == -3.0 and r[4] == 0.0
