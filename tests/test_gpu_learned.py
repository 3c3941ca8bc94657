"""Learned initial guesses on the GPU: the tensor-core MLP kernels against the
FP64 oracle MLP (forward and gradients with the same BF16 operands), training
on states the integrator produces, and the cold-restart comparison of the
method with and without the trained network."""
import numpy as np
import pytest

import oracle as O
from oracle import mlp as OM
from paper_2311_08927_gb300 import chad as CH
from paper_2311_08927_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_08927_gb300 import build
    build.build()
    CH.lib()


def _bf16_bits(a):
    """float32 array -> BF16 bit patterns (int16) with round-to-nearest-even."""
    r = OM.bf16_round(a)
    return (r.view(np.uint32) >> 16).astype(np.uint16).view(np.int16)


def _rand_case(n, seed):
    rng = np.random.default_rng(seed)
    p = OM.pack({"W1": rng.standard_normal((64, 32)) * 0.25, "b1": rng.standard_normal(64) * 0.1,
                 "W2": rng.standard_normal((64, 64)) * 0.18, "b2": rng.standard_normal(64) * 0.1,
                 "W3": rng.standard_normal((2, 64)) * 0.2, "b3": rng.standard_normal(2) * 0.1})
    X = rng.standard_normal((n, 32)).astype(np.float32)
    X[:, 30:] = 0.0
    Y = rng.standard_normal((n, 2)).astype(np.float32)
    return p.astype(np.float32), X, Y


def _weights_as_used(p32):
    """The GPU rounds weights (not biases) to BF16; the oracle uses the same."""
    w = OM.unpack(p32.astype(np.float64))
    for k in ("W1", "W2", "W3"):
        w[k] = OM.bf16_round(w[k].astype(np.float32)).astype(np.float64)
    return OM.pack(w)


def test_mlp_forward_matches_oracle():
    p, X, _ = _rand_case(1000, 1)
    Xb = torch.from_numpy(_bf16_bits(X)).cuda()
    P = torch.from_numpy(p).cuda()
    out = torch.empty((1000, 2), dtype=torch.float32, device="cuda")
    CH.chad_mlp_forward(Xb, P, out)
    ref, _ = OM.forward(_weights_as_used(p), OM.bf16_round(X).astype(np.float64))
    got = out.cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 2e-2


def test_mlp_gradients_match_oracle_per_tensor():
    n = 3000  # 12 blocks of 256 samples, ragged last block
    p, X, Y = _rand_case(n, 2)
    Xb = torch.from_numpy(_bf16_bits(X)).cuda()
    Yt = torch.from_numpy(Y).cuda()
    P = torch.from_numpy(p).cuda()
    g = torch.empty_like(P)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    sc = torch.empty(CH.mlp_grad_scratch_bytes(n) // 4 + 1, dtype=torch.float32, device="cuda")
    CH.chad_mlp_grad(Xb, Yt, P, g, loss, sc)
    ref_loss, ref = OM.loss_and_grad(_weights_as_used(p), OM.bf16_round(X).astype(np.float64),
                                     Y.astype(np.float64))
    got = g.cpu().numpy().astype(np.float64)
    assert abs(float(loss.item()) / ref_loss - 1) < 1e-2
    o = 0
    for name, shp in OM.SHAPES:
        k = int(np.prod(shp))
        rel = np.linalg.norm(got[o:o + k] - ref[o:o + k]) / np.linalg.norm(ref[o:o + k])
        assert rel < 1e-2, (name, rel)
        o += k
    # deterministic reduction
    g2 = torch.empty_like(P)
    CH.chad_mlp_grad(Xb, Yt, P, g2, loss, sc)
    assert torch.equal(g, g2)


@pytest.fixture(scope="module")
def trained():
    from paper_2311_08927_gb300 import learned as Lm
    pop = I.config_population(3, n=40000)
    y, T, SH, h = Lm.sample_states(pop, 6)
    X, Y, norm, onorm = Lm.build_dataset(y, T, SH, h)
    params, hist, test_loss = Lm.train(X, Y, epochs=12, batch=2048, lr=2e-3)
    model = Lm.TrainedMLP(params, norm.cpu().numpy(), onorm, hist)
    return model, hist, test_loss, (y, T, SH, h)


def test_training_reduces_loss_and_predicts_charge_balance_root(trained):
    """The validation loss falls well below its value before training, and
    the learned log10 S_H is within 0.05 decade (median) of the Newton root."""
    model, hist, test_loss, (y, T, SH, h) = trained
    assert hist[-1][2] < 0.6 * hist[0][2], hist
    from paper_2311_08927_gb300 import learned as Lm
    e_sh, e_h = Lm.prediction_errors(model, y, T, SH, h)
    assert e_sh < 0.05, (e_sh, e_h, hist)
    assert e_h < 0.5, (e_sh, e_h)


def _cold_restart(pop, relaxed, model, learned):
    sim = CH.Simulator(pop, precision=CH.PREC_MIXED, learned=1 if learned else 0)
    if learned:
        CH.chad_set_mlp(sim.ctx, model.params, model.feat_norm, model.out_norm)
    sim.load(y=relaxed)  # no S_H and no h: a restart without history
    sim.step(60.0, 1)
    out = sim.read()
    sim.close()
    return out


def test_learned_cold_restart_saves_work_and_keeps_the_solution(trained):
    model = trained[0]
    pop = I.config_population(3, n=20000, seed_offset=7)
    sim = CH.Simulator(pop, precision=CH.PREC_MIXED)
    sim.load()
    sim.step(60.0, 5)
    relaxed = sim.read()["y"]
    sim.close()
    plain = _cold_restart(pop, relaxed, model, False)
    lrn = _cold_restart(pop, relaxed, model, True)
    assert np.all(plain["status"] == 0) and np.all(lrn["status"] == 0)
    a_p = plain["stats"]["accepted_steps"] + plain["stats"]["rejected_steps"]
    a_l = lrn["stats"]["accepted_steps"] + lrn["stats"]["rejected_steps"]
    assert a_l < a_p, (a_l, a_p)
    assert lrn["stats"]["newton_iters"] < plain["stats"]["newton_iters"]
    assert lrn["stats"]["mlp_redo"] < 0.01 * pop.n
    # same solution within the production tolerance, and both against the oracle
    floor = 1e-12 * np.abs(plain["y"]).max(axis=1, keepdims=True)
    d = np.abs(lrn["y"] - plain["y"]) / np.maximum(np.abs(plain["y"]), floor)
    assert d.max() < 1e-4
    idx = np.arange(0, pop.n, 997)
    sub = I.Population([I.Digester(n=len(idx))], relaxed[:, idx].copy(), pop.T[idx].copy(),
                       np.zeros((3, len(idx))), False)
    o = O.run(sub, 60.0, 1, rtol=1e-10, atol=I.atol_vector(1e-13))
    floor = 1e-12 * np.abs(o["y"]).max(axis=1, keepdims=True)
    e = np.abs(lrn["y"][:, idx] - o["y"]) / np.maximum(np.abs(o["y"]), floor)
    assert e.max() < 1e-4


# ------------------------------------------------------------ full sizes with learned guesses
def _relerr(a, b):
    floor = 1e-12 * np.max(np.abs(b), axis=1, keepdims=True)
    return np.abs(a - b) / np.maximum(np.abs(b), floor + 1e-300)


def _learned_mixed_run(pop, model, n_intervals):
    """Learned + mixed form from a cold load (no S_H, no h: the network gives
    the first guesses), as the 2M and 64-digester workloads prescribe."""
    sim = CH.Simulator(pop, precision=CH.PREC_MIXED, learned=1)
    CH.chad_set_mlp(sim.ctx, model.params, model.feat_norm, model.out_norm)
    sim.load()
    sim.step(60.0, n_intervals)
    out = sim.read()
    sim.close()
    return out


def test_full_size_2M_learned_mixed_sampled(trained):
    """2,000,000 particles (the 1M recipe with a new seed) in the learned +
    mixed form from a cold load: every particle OK; under 5 % of the learned
    guesses redone plainly (this module's network sees 240k samples of one
    other seed; a cold load of unrelaxed states is its hardest input); and a
    seeded sample of 66 particles (slugs included) recomputed by the oracle
    within the mixed form's 1e-4 (oracle at the same rtol 1e-6; particles are
    independent, so a sample is exact)."""
    model = trained[0]
    pop = I.config_population(4)
    assert pop.n == 2_000_000
    g = _learned_mixed_run(pop, model, 2)
    assert np.all(g["status"] == 0)
    assert g["stats"]["mlp_redo"] < 0.05 * pop.n
    rng = np.random.default_rng(4)
    idx = np.sort(np.concatenate([rng.choice(pop.slugs, 16, replace=False),
                                  rng.choice(pop.n, 48, replace=False), [0, pop.n - 1]]))
    d0 = pop.digesters[0]
    sp = I.Population([I.Digester(n=len(idx), V_liq=d0.V_liq, V_gas=d0.V_gas, params=d0.params,
                                  D=d0.D, flow=d0.flow, y_in=d0.y_in)],
                      pop.y[:, idx].copy(), pop.T[idx].copy(), pop.pos[:, idx].copy(),
                      pop.shared_headspace)
    o = O.run(sp, 60.0, 2, rtol=1e-6)
    assert _relerr(g["y"][:, idx], o["y"]).max() < 1e-4


def test_full_size_64_digesters_learned_mixed(trained):
    """The 64-digester workload at full size (3.37M particles, log-uniform
    counts, per-digester kinetics, swirl fields and shared headspaces) in one
    learned + mixed run: every particle OK, the headspace states equal within
    each digester, every particle inside its cylinder, and the two smallest
    digesters recomputed whole by the oracle (each is self-contained: own
    flow, noise keys and headspace): positions bitwise, states within 1e-4."""
    model = trained[0]
    pop = I.config_population(5)
    g = _learned_mixed_run(pop, model, 2)
    assert np.all(g["status"] == 0)
    cnt = np.diff(pop.offsets)
    for d in range(64):
        a, b = pop.offsets[d], pop.offsets[d + 1]
        gas = g["y"][26:29, a:b]
        assert np.all(gas == gas[:, :1]), d
        x, y, z = g["pos"][:, a:b]
        f = pop.digesters[d].flow
        assert np.all(np.hypot(x, y) <= f["R"] * (1 + 1e-15)) and np.all((z >= 0) & (z <= f["H"]))
    for d in np.argsort(cnt)[:2]:
        a, b = pop.offsets[d], pop.offsets[d + 1]
        one = I.Population([pop.digesters[d]], pop.y[:, a:b].copy(), pop.T[a:b].copy(),
                           pop.pos[:, a:b].copy(), pop.shared_headspace)
        o = O.run(one, 60.0, 2, rtol=1e-6)
        assert np.array_equal(g["pos"][:, a:b], o["pos"]), d
        assert _relerr(g["y"][:, a:b], o["y"]).max() < 1e-4, d


# ------------------------------------------------------------ training data preparation
def test_feature_norm_and_targets_match_numpy():
    """The library's statistics against numpy in FP64: feature means and
    1/std (sample std) of log10 max(y, 1e-20) and T/100, target means and
    stds of log10 S_H and log10 h, and the standardised targets."""
    rng = np.random.default_rng(4)
    n = 70001  # not a multiple of the block size
    y = (I.x_ss()[:, None] * np.exp(0.3 * rng.standard_normal((I.NS, n))))
    y[3, :50] = 0.0  # below the log floor
    T = rng.uniform(303.15, 313.15, n)
    SH = 10 ** rng.uniform(-8, -6, n)
    h = 10 ** rng.uniform(-6, -3, n)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    sc = torch.empty(CH.mlp_prep_scratch_bytes() // 8 + 1, dtype=torch.float64, device="cuda")
    norm = torch.empty(64, dtype=torch.float32, device="cuda")
    CH.chad_mlp_feature_norm(d(y), d(T), norm, sc)
    f = np.vstack([np.log10(np.maximum(y.astype(np.float32), np.float32(1e-20))).astype(np.float64),
                   (T.astype(np.float32) * np.float32(0.01)).astype(np.float64)])
    nm = norm.cpu().numpy()
    np.testing.assert_allclose(nm[:30], f.mean(1), rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(nm[32:62], 1.0 / f.std(1, ddof=1), rtol=1e-5)
    assert np.all(nm[30:32] == 0) and np.all(nm[62:64] == 1)
    Y = torch.empty((n, 2), dtype=torch.float32, device="cuda")
    on = torch.empty(4, dtype=torch.float32, device="cuda")
    CH.chad_mlp_targets(d(SH), d(h), Y, on, sc)
    t = np.vstack([np.log10(SH), np.log10(h)])
    o = on.cpu().numpy()
    np.testing.assert_allclose(o[:2], t.mean(1), rtol=1e-6)
    np.testing.assert_allclose(o[2:], t.std(1, ddof=1), rtol=1e-5)
    ref = ((t.T - o[:2]) / o[2:]).astype(np.float32)
    np.testing.assert_allclose(Y.cpu().numpy(), ref, rtol=1e-5, atol=1e-5)


def test_gather_visits_every_row_of_a_split_once():
    """The keyed permutations are bijections: one pass over a split gathers
    each of its rows exactly once; the three splits partition the data; a
    different epoch key gives another order; the rows are copied intact."""
    M = 10007
    X = torch.arange(M * 32, dtype=torch.int32).remainder(30000).to(torch.int16).reshape(M, 32)
    X[:, 0] = torch.arange(M, dtype=torch.int32).remainder(30000).to(torch.int16)
    X = X.cuda().contiguous()
    ids = np.arange(M, dtype=np.float32)
    Y = torch.from_numpy(np.stack([ids, -ids], 1)).cuda()
    seen = []
    for off, n in ((0, 9000), (9000, 500), (9500, 507)):
        Xb = torch.empty((n, 32), dtype=torch.int16, device="cuda")
        Yb = torch.empty((n, 2), dtype=torch.float32, device="cuda")
        CH.chad_mlp_gather(X, Y, 12345, off, n, 777, 0, n, Xb, Yb)
        r = Yb.cpu().numpy()
        assert np.array_equal(r[:, 1], -r[:, 0])
        rows = r[:, 0].astype(np.int64)
        assert len(np.unique(rows)) == n
        np.testing.assert_array_equal(Xb.cpu().numpy(), X.cpu().numpy()[rows])
        seen.append(rows)
    allr = np.concatenate(seen)
    assert np.array_equal(np.sort(allr), np.arange(M))
    Xb = torch.empty((9000, 32), dtype=torch.int16, device="cuda")
    Yb = torch.empty((9000, 2), dtype=torch.float32, device="cuda")
    CH.chad_mlp_gather(X, Y, 12345, 0, 9000, 778, 0, 9000, Xb, Yb)
    other = Yb.cpu().numpy()[:, 0].astype(np.int64)
    assert np.array_equal(np.sort(other), np.sort(seen[0])) and not np.array_equal(other, seen[0])


def test_library_training_loop_reduces_the_loss():
    """The in-library loop (gather, asynchronous gradient, Adam, one wait per
    epoch) on a smooth synthetic target: the validation loss falls."""
    from paper_2311_08927_gb300 import learned as Lm
    rng = np.random.default_rng(9)
    M = 60000
    Xf = rng.standard_normal((M, 32)).astype(np.float32)
    Xf[:, 30:] = 0
    Yf = np.stack([np.tanh(Xf[:, 0] + 0.5 * Xf[:, 1]), Xf[:, 2] * Xf[:, 3] * 0.3], 1).astype(np.float32)
    X = torch.from_numpy(_bf16_bits(Xf)).cuda()
    Y = torch.from_numpy(Yf).cuda()
    params, hist, test_loss = Lm.train(X, Y, epochs=6, batch=4096, lr=3e-3)
    assert hist[-1][2] < 0.3 * hist[0][2], hist
    assert abs(test_loss - hist[-1][2]) < 0.5 * hist[-1][2] + 1e-3


def test_learned_cold_restart_with_algebraic_h2():
    """The mixed form with S_h2 algebraic (kernel form 4), network trained on
    states of the same model: a restart without history takes fewer attempts
    with the learned guesses, and both runs stay within 1e-4 of the tight
    algebraic oracle."""
    from paper_2311_08927_gb300 import learned as Lm
    pop = I.config_population(3, n=20000, seed_offset=11)
    y, T, SH, h = Lm.sample_states(I.config_population(3, n=30000, seed_offset=12), 5,
                                   h2_algebraic=True)
    X, Y, norm, onorm = Lm.build_dataset(y, T, SH, h)
    params, hist, _ = Lm.train(X, Y, epochs=10, batch=2048, lr=2e-3)
    model = Lm.TrainedMLP(params, norm.cpu().numpy(), onorm, hist)
    sim = CH.Simulator(pop, precision=CH.PREC_MIXED, h2_algebraic=True)
    sim.load()
    sim.step(60.0, 5)
    relaxed = sim.read()["y"]
    sim.close()
    runs = {}
    for learned in (False, True):
        s = CH.Simulator(pop, precision=CH.PREC_MIXED, h2_algebraic=True,
                         learned=1 if learned else 0)
        if learned:
            CH.chad_set_mlp(s.ctx, model.params, model.feat_norm, model.out_norm)
        s.load(y=relaxed)
        s.step(60.0, 1)
        runs[learned] = s.read()
        s.close()
    p, l = runs[False], runs[True]
    assert np.all(p["status"] == 0) and np.all(l["status"] == 0)
    att = lambda r: r["stats"]["accepted_steps"] + r["stats"]["rejected_steps"]
    assert att(l) < att(p), (att(l), att(p))
    # the test's small network (1.5e5 samples, 10 epochs): redo bound 5 %, as for
    # the other small-network test of this module
    assert l["stats"]["mlp_redo"] < 0.05 * pop.n
    idx = np.arange(0, pop.n, 997)
    sub = I.Population([I.Digester(n=len(idx))], relaxed[:, idx].copy(), pop.T[idx].copy(),
                       np.zeros((3, len(idx))), False)
    o = O.run(sub, 60.0, 1, rtol=1e-10, atol=I.atol_vector(1e-13), h2_algebraic=True)
    for r in (p, l):
        assert _relerr(r["y"][:, idx], o["y"]).max() < 1e-4


# ------------------------------------------------------------ full sizes, S_h2 algebraic
@pytest.fixture(scope="module")
def trained_h2():
    """A small network trained on states of the S_h2-algebraic model."""
    from paper_2311_08927_gb300 import learned as Lm
    y, T, SH, h = Lm.sample_states(I.config_population(3, n=40000), 6, h2_algebraic=True)
    X, Y, norm, onorm = Lm.build_dataset(y, T, SH, h)
    params, hist, _ = Lm.train(X, Y, epochs=12, batch=2048, lr=2e-3)
    return Lm.TrainedMLP(params, norm.cpu().numpy(), onorm, hist)


def _learned_mixed_h2_run(pop, model, n_intervals):
    sim = CH.Simulator(pop, precision=CH.PREC_MIXED, learned=1, h2_algebraic=True)
    CH.chad_set_mlp(sim.ctx, model.params, model.feat_norm, model.out_norm)
    sim.load()
    sim.step(60.0, n_intervals)
    out = sim.read()
    sim.close()
    return out


def test_full_size_2M_learned_mixed_h2_sampled(trained_h2):
    """2,000,000 particles, learned guesses from a cold load, kernel form 4
    (the form the 2M benchmark line runs): every particle OK, under 5 % of
    the guesses redone, and a seeded sample of 66 particles (slugs included)
    recomputed by the oracle's algebraic mode within 1e-4."""
    pop = I.config_population(4)
    g = _learned_mixed_h2_run(pop, trained_h2, 2)
    assert np.all(g["status"] == 0)
    assert g["stats"]["mlp_redo"] < 0.05 * pop.n
    rng = np.random.default_rng(14)
    idx = np.sort(np.concatenate([rng.choice(pop.slugs, 16, replace=False),
                                  rng.choice(pop.n, 48, replace=False), [0, pop.n - 1]]))
    sp = I.Population([I.Digester(n=len(idx))], pop.y[:, idx].copy(), pop.T[idx].copy(),
                      np.zeros((3, len(idx))), False)
    o = O.run(sp, 60.0, 2, rtol=1e-6, h2_algebraic=True)
    assert _relerr(g["y"][:, idx], o["y"]).max() < 1e-4


def test_full_size_64_digesters_learned_mixed_h2(trained_h2):
    """The 64-digester workload at full size in one learned form-4 run (the
    form its benchmark line runs): every particle OK, the headspace states
    equal within each digester, and the two smallest digesters recomputed
    whole by the oracle's algebraic mode: positions bitwise, states within
    1e-4."""
    pop = I.config_population(5)
    g = _learned_mixed_h2_run(pop, trained_h2, 2)
    assert np.all(g["status"] == 0)
    for d in range(64):
        a, b = pop.offsets[d], pop.offsets[d + 1]
        gas = g["y"][26:29, a:b]
        assert np.all(gas == gas[:, :1]), d
    cnt = np.diff(pop.offsets)
    for d in np.argsort(cnt)[:2]:
        a, b = pop.offsets[d], pop.offsets[d + 1]
        one = I.Population([pop.digesters[d]], pop.y[:, a:b].copy(), pop.T[a:b].copy(),
                           pop.pos[:, a:b].copy(), pop.shared_headspace)
        o = O.run(one, 60.0, 2, rtol=1e-6, h2_algebraic=True)
        assert np.array_equal(g["pos"][:, a:b], o["pos"]), d
        assert _relerr(g["y"][:, a:b], o["y"]).max() < 1e-4, d
