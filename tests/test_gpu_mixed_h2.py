"""The mixed form with S_h2 algebraic (kernel form 4) against the CPU oracle.

Form 4 evaluates the rates, the Jacobian and the LU in FP32, S_h2 from Eq. 8
in FP32, the refinement residual and the stage vectors in two-float
arithmetic, and keeps FP64 for the Eq. 7 Newton and the state.  Its
arithmetic is not the oracle's, so every comparison here is at the mixed
forms' tolerance: max relative species error 1e-4 against the oracle's
algebraic mode run at rtol 1e-10 (relative error |a - b| / max(|b|,
1e-12 max_p |b_i|), as in the other parity tests).
"""
import numpy as np
import pytest

import oracle as O
from paper_2311_08927_gb300 import chad as CH
from paper_2311_08927_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_08927_gb300 import build
    build.build()
    CH.lib()


def relerr(a, b):
    floor = 1e-12 * np.max(np.abs(b), axis=1, keepdims=True)
    return np.abs(a - b) / np.maximum(np.abs(b), floor + 1e-300)


def subset(pop, idx):
    idx = np.asarray(idx)
    d0 = pop.digesters[0]
    dg = [I.Digester(n=len(idx), V_liq=d0.V_liq, V_gas=d0.V_gas, params=d0.params, D=d0.D,
                     flow=d0.flow, y_in=d0.y_in)]
    return I.Population(dg, pop.y[:, idx].copy(), pop.T[idx].copy(), pop.pos[:, idx].copy(),
                        pop.shared_headspace)


def gpu_run(pop, dt, n, **kw):
    sim = CH.Simulator(pop, **kw)
    sim.load()
    sim.step(dt, n)
    out = sim.read()
    sim.close()
    return out


def tight_oracle(pop, dt, n):
    return O.run(pop, dt, n, rtol=1e-10, atol=I.atol_vector(1e-13), h2_algebraic=True)


def mixed_h2(pop, dt, n, **kw):
    return gpu_run(pop, dt, n, precision=CH.PREC_MIXED, h2_algebraic=True, **kw)


def _slug_sample(n_pop, n_slug, n_plain, seed_pop=3):
    pop = I.config_population(seed_pop, n=n_pop)
    idx = np.concatenate([pop.slugs[:n_slug], np.setdiff1d(np.arange(n_pop), pop.slugs)[:n_plain]])
    return subset(pop, idx)


def test_fixed_steps_within_mixed_tolerance():
    """Fixed steps (the same step sequence on both sides): the difference is
    the FP32 rounding of the rates and the LU, far below 1e-4; the stored
    S_h2 is the Eq. 8 root at the new state."""
    pop = I.config_population(3, n=700)  # ragged: 5 blocks of 128 + 60
    g = mixed_h2(pop, 60.0, 3, fixed_substeps=4)
    o = O.run(pop, 60.0, 3, fixed_n=4, h2_algebraic=True)
    assert np.all(g["status"] == 0)
    e = relerr(g["y"], o["y"])
    assert e.max() < TOL, (e.max(), I.STATE_NAMES[int(np.argmax(e.max(axis=1)))])
    assert np.max(np.abs(g["S_H"] / o["S_H"] - 1)) < TOL


def test_production_tolerance_against_tight_oracle():
    sp = _slug_sample(3000, 24, 72)
    g = mixed_h2(sp, 60.0, 20, rtol=1e-6)
    o = tight_oracle(sp, 60.0, 20)
    assert np.all(g["status"] == 0)
    e = relerr(g["y"], o["y"])
    assert e.max() < TOL, (e.max(), I.STATE_NAMES[int(np.argmax(e.max(axis=1)))])


def test_agrees_with_the_fp64_algebraic_and_differential_forms():
    """Same workload, rtol 1e-6: within 1e-4 of the FP64 form with S_h2
    algebraic (same model) and of the FP64 differential form (the models
    differ by the quasi-steady error of a sub-second S_h2)."""
    sp = _slug_sample(3000, 16, 48)
    g = mixed_h2(sp, 60.0, 10, rtol=1e-6)
    f3 = gpu_run(sp, 60.0, 10, rtol=1e-6, h2_algebraic=True)
    f0 = gpu_run(sp, 60.0, 10, rtol=1e-6)
    assert relerr(g["y"], f3["y"]).max() < TOL
    assert relerr(g["y"], f0["y"]).max() < TOL
    # FP32 rates do not inflate the step count: accepted steps within 10 % of
    # the FP64 algebraic form's, and few rejections
    ga, fa = g["stats"]["accepted_steps"], f3["stats"]["accepted_steps"]
    assert abs(ga - fa) <= 0.1 * fa, (ga, fa)
    assert g["stats"]["rejected_steps"] <= 0.1 * ga + 10


def test_flow_and_shared_headspace_whole_tank():
    """Lab cylinder (swirl + noise, inlet slab, shared headspace), whole
    tank: positions bit-identical to the oracle's, states within 1e-4 of
    the tight algebraic oracle."""
    pop = I.config_population(2, n=1500)
    g = mixed_h2(pop, 60.0, 3, rtol=1e-6)
    o = tight_oracle(pop, 60.0, 3)
    assert np.all(g["status"] == 0)
    assert np.array_equal(g["pos"], o["pos"])
    assert relerr(g["y"], o["y"]).max() < TOL


def test_many_digesters_within_tolerance():
    pop = I.config_population(5, n=2500)
    g = mixed_h2(pop, 60.0, 2, rtol=1e-6)
    o = tight_oracle(pop, 60.0, 2)
    assert np.all(g["status"] == 0)
    assert relerr(g["y"], o["y"]).max() < TOL


def test_autotuned_variants_and_graph_replay_agree():
    import torch
    pop = I.config_population(2, n=3000)
    outs = []
    for tune in (False, True):
        s = torch.cuda.Stream()
        sim = CH.Simulator(pop, precision=CH.PREC_MIXED, h2_algebraic=True,
                           stream=s.cuda_stream)
        sim.load()
        if tune:
            chosen, ms = CH.chad_autotune(sim.ctx, 60.0)
            assert 0 <= chosen < len(ms) and np.all(ms > 0)
        sim.step(60.0, 3)
        outs.append(sim.read())
        sim.close()
    assert np.array_equal(outs[0]["pos"], outs[1]["pos"])
    assert relerr(outs[1]["y"], outs[0]["y"]).max() < 1e-12


def test_full_size_1M_sampled():
    """The metric workload in the benchmark's launch configuration; a seeded
    sample (slugs, plain particles, both ends) recomputed by the tight
    algebraic oracle particle by particle."""
    pop = I.config_population(3)
    sim = CH.Simulator(pop, precision=CH.PREC_MIXED, h2_algebraic=True, rtol=1e-6)
    sim.load()
    sim.step(60.0, 2)
    g = sim.read()
    sim.close()
    assert np.all(g["status"] == 0)
    rng = np.random.default_rng(98)
    idx = np.sort(np.concatenate([rng.choice(pop.slugs, 16, replace=False),
                                  rng.choice(pop.n, 48, replace=False), [0, pop.n - 1]]))
    o = tight_oracle(subset(pop, idx), 60.0, 2)
    assert relerr(g["y"][:, idx], o["y"]).max() < TOL


def test_empty_digester_single_particle_and_step_limit():
    """Edge cases of the launch: a digester without particles next to one
    with a single particle (one thread of one block), and a step limit that
    sets the status bit instead of faulting."""
    y1 = I.x_ss()[:, None].copy()
    dg = [I.Digester(n=0), I.Digester(n=1)]
    pop = I.Population(dg, y1, np.array([I.T_OP]), np.zeros((3, 1)), False)
    g = mixed_h2(pop, 60.0, 3, fixed_substeps=2)
    o = O.run(pop, 60.0, 3, fixed_n=2, h2_algebraic=True)
    assert np.all(g["status"] == 0)
    assert relerr(g["y"], o["y"]).max() < TOL
    pop = I.config_population(1, n=64)
    sim = CH.Simulator(pop, precision=CH.PREC_MIXED, h2_algebraic=True, max_steps=1)
    sim.load()
    sim.step(60.0, 1)
    out = sim.read()
    sim.close()
    assert np.all(out["status"] & CH.P_STEPS)


def test_counters_split_eq7_and_eq8_iterations():
    """Eq. 7 (FP64) and Eq. 8 (FP32) Newton iterations are counted apart:
    at least one of each per rate evaluation (three per step attempt)."""
    pop = I.config_population(3, n=2000)
    g = mixed_h2(pop, 60.0, 2, rtol=1e-6)
    st = g["stats"]
    attempts = st["accepted_steps"] + st["rejected_steps"]
    full = 3 * (attempts - st["pivot_rejects"])  # an attempt stopped by a pivot test evaluates once
    assert st["newton_iters"] >= full and st["h2_newton_iters"] >= full
    d = gpu_run(pop, 60.0, 2, rtol=1e-6)  # S_h2 a state: no Eq. 8 iterations
    assert d["stats"]["h2_newton_iters"] == 0


def test_diffusion_between_particles_then_mixed_h2():
    """Diffusion between particles (SPH operator, before the ADM1 step of each
    interval) followed by form 4, whole lab-cylinder tank, adaptive: within
    1e-4 of the tight algebraic oracle with the same diffusion."""
    pop = I.config_population(2, n=1200)
    dif = (1e-5, 0.024)  # D m^2/s, h m: about 1.3 particle spacings at 1,200 particles
    g = mixed_h2(pop, 60.0, 3, rtol=1e-6, diffusion=dif)
    o = O.run(pop, 60.0, 3, rtol=1e-10, atol=I.atol_vector(1e-13), h2_algebraic=True,
              diffusion=dif)
    assert np.all(g["status"] == 0)
    assert np.array_equal(g["pos"], o["pos"])
    assert relerr(g["y"], o["y"]).max() < TOL


def test_full_size_lab_cylinder_100k_whole_tank():
    """The lab-cylinder workload at full size (100,000 particles, swirl +
    noise, inlet slab, shared headspace), one 60-s interval in form 4 at
    rtol 1e-6, against the oracle's algebraic mode on the whole tank at the
    same rtol: positions bitwise, states within 1e-4."""
    pop = I.config_population(2)
    assert pop.n == 100_000
    g = mixed_h2(pop, 60.0, 1, rtol=1e-6)
    o = O.run(pop, 60.0, 1, rtol=1e-6, h2_algebraic=True)
    assert np.all(g["status"] == 0) and np.all(o["status"] == 0)
    assert np.array_equal(g["pos"], o["pos"])
    assert relerr(g["y"], o["y"]).max() < TOL


@pytest.mark.parametrize("precision,h2", [(CH.PREC_FP64, False), (CH.PREC_FP64, True),
                                          (CH.PREC_MIXED, False), (CH.PREC_MIXED, True)])
def test_every_kernel_variant_gives_the_same_states(precision, h2):
    """Every launch shape the autotuner chooses from (threads per block,
    register budget, the factored matrix in registers or in shared memory),
    forced with chad_set_kernel_variant, integrates the same states: the
    arithmetic does not depend on the shape.  A ragged population (not a
    multiple of any block size) with slugs and a temperature spread."""
    pop = I.config_population(3, n=1500)
    outs = []
    for v in range(CH.NUM_VARIANTS):
        sim = CH.Simulator(pop, precision=precision, h2_algebraic=h2, rtol=1e-6)
        CH.chad_set_kernel_variant(sim.ctx, v)
        sim.load()
        sim.step(60.0, 2)
        outs.append(sim.read())
        sim.close()
    for v, o in enumerate(outs):
        assert np.all(o["status"] == 0), v
        assert relerr(o["y"], outs[0]["y"]).max() <= 1e-12, v
        assert o["stats"]["accepted_steps"] == outs[0]["stats"]["accepted_steps"], v
    with pytest.raises(CH.ChadError):
        sim = CH.Simulator(pop, precision=precision, h2_algebraic=h2)
        try:
            CH.chad_set_kernel_variant(sim.ctx, CH.NUM_VARIANTS)
        finally:
            sim.close()
