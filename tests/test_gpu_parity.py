"""GPU (CUDA, through the C ABI) versus the CPU oracle on identical seeded inputs.

Tolerances: the FP64 path must match the oracle to max relative error 1e-9
(fixed steps and tight adaptive tolerance, where both run the same
arithmetic); the production forms (FP64 at rtol 1e-6 and the mixed FP32/FP64
form) must stay within 1e-4 of the oracle run at rtol 1e-10.  The relative
error of species i is |a - b| / max(|b|, 1e-12 * max_p |b_i|), so species
near zero do not dominate.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle as O
from paper_2311_08927_gb300 import chad as CH
from paper_2311_08927_gb300 import inputs as I

pytestmark = pytest.mark.gpu


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
    """Population made of the given particles (single digester populations)."""
    idx = np.asarray(idx)
    dg = [I.Digester(n=len(idx), V_liq=pop.digesters[0].V_liq, V_gas=pop.digesters[0].V_gas,
                     params=pop.digesters[0].params, D=pop.digesters[0].D,
                     flow=pop.digesters[0].flow, y_in=pop.digesters[0].y_in)]
    return I.Population(dg, pop.y[:, idx].copy(), pop.T[idx].copy(), pop.pos[:, idx].copy(),
                        pop.shared_headspace)


def gpu_run(pop, dt, n, **kw):
    sim = CH.Simulator(pop, **kw)
    sim.load()
    sim.step(dt, n)
    out = sim.read()
    if kw.get("diffusion") is not None:
        out["diff_info"] = CH.chad_diffusion_info(sim.ctx)
    sim.close()
    return out


def oracle_run(pop, dt, n, rtol=1e-6, atol=None, fixed_n=0, h2_algebraic=False, diffusion=None):
    return O.run(pop, dt, n, rtol=rtol, atol=atol, fixed_n=fixed_n, h2_algebraic=h2_algebraic,
                 diffusion=diffusion)


# ------------------------------------------------------------ Gate A: same arithmetic
def test_fixed_step_fp64_matches_oracle():
    pop = I.config_population(1, n=300)          # ragged: 2 blocks of 128 + 44
    g = gpu_run(pop, 60.0, 10, fixed_substeps=4)
    o = oracle_run(pop, 60.0, 10, fixed_n=4)
    assert np.all(g["status"] == 0)
    e = relerr(g["y"], o["y"])
    assert e.max() < 1e-9, e.max()
    assert np.max(np.abs(g["S_H"] / o["S_H"] - 1)) < 1e-9


def test_fixed_step_fp64_heterogeneous_temperature_and_slugs():
    pop = I.config_population(3, n=4000)
    idx = np.concatenate([pop.slugs[:40], np.setdiff1d(np.arange(4000), pop.slugs)[:90]])
    sp = subset(pop, idx)
    g = gpu_run(sp, 60.0, 5, fixed_substeps=6)
    o = oracle_run(sp, 60.0, 5, fixed_n=6)
    assert relerr(g["y"], o["y"]).max() < 1e-9


# ------------------------------------------------------------ Gate B: adaptive, tight
def test_adaptive_tight_tolerance_fp64_matches_oracle():
    pop = I.config_population(3, n=2000)
    idx = np.concatenate([pop.slugs[:16], np.setdiff1d(np.arange(2000), pop.slugs)[:48]])
    sp = subset(pop, idx)
    atol = I.atol_vector(1e-13)
    g = gpu_run(sp, 60.0, 4, rtol=1e-10, atol=atol)
    o = oracle_run(sp, 60.0, 4, rtol=1e-10, atol=atol)
    assert np.all(g["status"] == 0) and np.all(o["status"] == 0)
    assert relerr(g["y"], o["y"]).max() < 1e-9
    # same step sequences (a round-off accept/reject flip would show here)
    assert abs(g["stats"]["accepted_steps"] - o["stats"][0]) <= 2


def test_production_fp64_same_tolerance_tracks_oracle():
    pop = I.config_population(1, n=256)
    g = gpu_run(pop, 60.0, 30, rtol=1e-6)
    o = oracle_run(pop, 60.0, 30, rtol=1e-6)
    e = relerr(g["y"], o["y"])
    assert np.median(e) < 1e-10 and e.max() < 1e-5
    # the next step size comes from the controller, FP64 on both sides: the
    # step sequences agree to the round-off of the (sparse vs dense) solves
    assert np.median(np.abs(g["h"] / o["h"] - 1)) < 1e-9


# ------------------------------------------------------------ Gate C: production forms
@pytest.mark.parametrize("precision", [CH.PREC_FP64, CH.PREC_MIXED])
def test_production_forms_within_1e4_of_tight_oracle(precision):
    pop = I.config_population(3, n=3000)
    idx = np.concatenate([pop.slugs[:24], np.setdiff1d(np.arange(3000), pop.slugs)[:72]])
    sp = subset(pop, idx)
    g = gpu_run(sp, 60.0, 20, rtol=1e-6, precision=precision)
    o = oracle_run(sp, 60.0, 20, rtol=1e-10, atol=I.atol_vector(1e-13))
    assert np.all(g["status"] == 0)
    e = relerr(g["y"], o["y"])
    assert e.max() < 1e-4, (e.max(), I.STATE_NAMES[int(np.argmax(e.max(axis=1)))])


# ------------------------------------------------------------ diffusion between particles
DIFFUSION = (1e-5, 0.024)  # D m^2/s, h m (about 1.3 particle spacings at 1,200 particles)


def test_diffusion_matches_oracle():
    """Interval = advect, SPH diffusion between the particles (grid neighbour
    search on the GPU, all pairs in the oracle), ADM1 in fixed steps (the
    same arithmetic on both sides): states to 1e-9 of the oracle, positions
    bitwise, and the diffusion visibly acts."""
    pop = I.config_population(2, n=1200)
    g = gpu_run(pop, 60.0, 3, diffusion=DIFFUSION, fixed_substeps=4)
    o = oracle_run(pop, 60.0, 3, diffusion=DIFFUSION, fixed_n=4)
    assert np.all(g["status"] == 0)
    assert np.array_equal(g["pos"], o["pos"])
    assert relerr(g["y"], o["y"]).max() < 1e-9
    smax = O.diffusion_row_sum_max(o["pos"], pop.digesters[0].V_liq / 1200, *DIFFUSION)
    assert g["diff_info"]["n_sub"] == O.diffusion_substeps(60.0, smax) > 1
    nd = gpu_run(pop, 60.0, 3, fixed_substeps=4)
    assert relerr(g["y"], nd["y"]).max() > 1e-6


def test_diffusion_production_tolerance_tracks_oracle():
    """Adaptive stepping at rtol 1e-6 on both sides after the same diffusion:
    the step sizes agree to the round-off of the (sparse vs dense) solves, so
    a rare accept/reject flip moves a particle by O(rtol) at worst; most agree
    to round-off (the bound of the production test above)."""
    pop = I.config_population(2, n=1200)
    g = gpu_run(pop, 60.0, 3, diffusion=DIFFUSION)
    o = oracle_run(pop, 60.0, 3, diffusion=DIFFUSION)
    assert np.all(g["status"] == 0)
    e = relerr(g["y"], o["y"])
    assert np.median(e) < 1e-10 and e.max() < 1e-5


def test_diffusion_with_algebraic_h2_matches_oracle():
    """Diffusion followed by the S_h2-algebraic FP64 form (Eq. 8): the
    diffused S_h2 is the root's starting point each interval; states to 1e-9
    of the oracle with both switched on."""
    pop = I.config_population(2, n=1200)
    g = gpu_run(pop, 60.0, 3, diffusion=DIFFUSION, h2_algebraic=True, fixed_substeps=4)
    o = oracle_run(pop, 60.0, 3, diffusion=DIFFUSION, h2_algebraic=True, fixed_n=4)
    assert np.all(g["status"] == 0) and np.all(o["status"] == 0)
    assert relerr(g["y"], o["y"]).max() < 1e-9


def test_diffusion_per_digester_settings_match_oracle():
    """64 digesters, each its own grid: diffusion off in every fourth, three
    (D, h) pairs in the rest, and a digester cut to one particle (no
    neighbours: S = 0, nothing moves).  One substep plan for all digesters,
    from the largest row sum over all of them."""
    pop = I.config_population(5, n=3000)
    a, b = pop.offsets[1], pop.offsets[2]
    keep = np.r_[0:a + 1, b:pop.n]           # digester 1 keeps one particle
    dgs = list(pop.digesters)
    dgs[1] = dataclasses.replace(dgs[1], n=1)
    pop = I.Population(dgs, pop.y[:, keep].copy(), pop.T[keep].copy(), pop.pos[:, keep].copy(),
                       pop.shared_headspace)
    pairs = [(1e-6, 0.05), (3e-6, 0.04), (1e-5, 0.06)]
    dif = [None if d % 4 == 0 else pairs[d % 3] for d in range(64)]
    g = gpu_run(pop, 60.0, 3, diffusion=dif, fixed_substeps=4)
    o = oracle_run(pop, 60.0, 3, diffusion=dif, fixed_n=4)
    assert np.all(g["status"] == 0) and np.all(o["status"] == 0)
    assert np.array_equal(g["pos"], o["pos"])
    assert relerr(g["y"], o["y"]).max() < 1e-9
    smax = 0.0
    for d in range(64):
        if dif[d] is None:
            continue
        lo, hi = pop.offsets[d], pop.offsets[d + 1]
        smax = max(smax, O.diffusion_row_sum_max(o["pos"][:, lo:hi], pop.digesters[d].V_liq / (hi - lo),
                                                 *dif[d]))
    assert g["diff_info"]["n_sub"] == O.diffusion_substeps(60.0, smax) > 1
    nd = gpu_run(pop, 60.0, 3, fixed_substeps=4)
    moved = np.abs(g["y"] - nd["y"]).max(axis=0) > 0
    for d in range(64):
        lo, hi = pop.offsets[d], pop.offsets[d + 1]
        if dif[d] is None or hi - lo == 1:
            assert not moved[lo:hi].any(), d
        else:
            assert moved[lo:hi].any(), d


def test_external_positions_each_interval_match_oracle():
    """The coupling loop of an external CFD: before every interval the caller
    supplies new positions (chad_set_positions) and the flow has U = 0 and no
    noise, so the library only uses them: inlet slab membership and diffusion
    follow the supplied positions, the states carry over.  Oracle chained
    interval by interval from the same positions; fixed ADM1 steps."""
    n = 1500
    base = I.config_population(2, n=n)
    fl = I.swirl_flow(U=0.0, sigma=0.0, R=0.1, H=0.3, seed=7)
    dg = dataclasses.replace(base.digesters[0], flow=fl)
    pop = I.Population([dg], base.y.copy(), base.T.copy(), base.pos.copy(), base.shared_headspace)
    frames = [I.config_population(2, n=n, seed_offset=10 + k).pos for k in range(4)]
    sim = CH.Simulator(pop, fixed_substeps=4, diffusion=DIFFUSION)
    sim.load()
    y, SH, h = pop.y.copy(), None, None
    for k, pos in enumerate(frames):
        sim.set_positions(pos)
        sim.step(60.0, 1)
        step_pop = I.Population([dg], y, pop.T.copy(), pos.copy(), pop.shared_headspace)
        o = O.run(step_pop, 60.0, 1, interval0=k, fixed_n=4, SH=SH, h=h, diffusion=DIFFUSION)
        y, SH, h = o["y"], o["S_H"], o["h"]
    g = sim.read()
    with pytest.raises(CH.ChadError) as ei:
        bad = frames[0].copy()
        bad[2, 5] = np.nan
        sim.set_positions(bad)
    assert ei.value.code == 1
    assert np.array_equal(sim.read()["pos"], g["pos"])
    sim.close()
    assert np.array_equal(g["pos"], frames[-1]) and np.array_equal(o["pos"], frames[-1])
    assert np.all(g["status"] == 0)
    assert relerr(g["y"], o["y"]).max() < 1e-9


def test_frames_scatter_by_id_and_refuse_bad_ids(tmp_path):
    """Frame files (FP64 and FP32, entries shuffled with their ids, as an SPH
    code writes them after re-sorting) land in particle order bitwise (FP32
    widened exactly); ids that repeat, run out of range or a frame of another
    size are refused and leave the positions as they were."""
    from paper_2311_08927_gb300 import frames as F
    pop = I.config_population(2, n=3000)
    sim = CH.Simulator(pop)
    sim.load()
    rng = np.random.default_rng(12)
    new = I.config_population(2, n=3000, seed_offset=21).pos
    perm = rng.permutation(3000)
    for dt in (np.float64, np.float32):
        f = tmp_path / f"f{np.dtype(dt).itemsize}.frm"
        F.write_frame(f, new[:, perm], ids=perm.astype(np.uint32), dtype=dt, step=5, time_s=2.5)
        assert CH.chad_load_frame(sim.ctx, 0, f) == (5, 2.5)
        assert np.array_equal(sim.read()["pos"], new.astype(dt).astype(np.float64))
    before = sim.read()["pos"]
    dup = perm.copy()
    dup[7] = dup[8]
    out = perm.copy()
    out[0] = 3000
    for ids, m in ((dup, 3000), (out, 3000), (np.arange(2999), 2999)):
        f = tmp_path / "bad.frm"
        F.write_frame(f, new[:, :m], ids=ids.astype(np.uint32))
        with pytest.raises(CH.ChadError) as ei:
            CH.chad_load_frame(sim.ctx, 0, f)
        assert ei.value.code == 1
        assert np.array_equal(sim.read()["pos"], before)
    sim.close()


def test_frames_each_interval_equal_set_positions(tmp_path):
    """Stepping from frame files (shuffled, with ids) gives bitwise the states
    of stepping from the same positions handed over in particle order."""
    from paper_2311_08927_gb300 import frames as F
    base = I.config_population(2, n=2000)
    dg = dataclasses.replace(base.digesters[0], flow=I.swirl_flow(U=0.0, sigma=0.0, seed=3))
    pop = I.Population([dg], base.y.copy(), base.T.copy(), base.pos.copy(), base.shared_headspace)
    frames = [I.config_population(2, n=2000, seed_offset=30 + k).pos for k in range(3)]
    a = CH.Simulator(pop, diffusion=DIFFUSION)
    b = CH.Simulator(pop, diffusion=DIFFUSION)
    a.load()
    b.load()
    rng = np.random.default_rng(1)
    for k, pos in enumerate(frames):
        a.set_positions(pos)
        perm = rng.permutation(2000)
        f = tmp_path / f"{k}.frm"
        F.write_frame(f, pos[:, perm], ids=perm.astype(np.uint32), step=k)
        CH.chad_load_frame(b.ctx, 0, f)
        a.step(60.0, 1)
        b.step(60.0, 1)
    ra, rb = a.read(), b.read()
    a.close()
    b.close()
    assert np.array_equal(ra["pos"], rb["pos"]) and np.array_equal(ra["y"], rb["y"])


def test_diffusion_kernel_timing_leaves_the_states_alone():
    """chad_diffusion_kernel_times re-runs the rows and one substep on the
    interval's scratch: positive times, states and positions unchanged, and
    the next interval identical to a run without the timing call."""
    pop = I.config_population(2, n=1500)
    a = CH.Simulator(pop, diffusion=DIFFUSION, fixed_substeps=2)
    b = CH.Simulator(pop, diffusion=DIFFUSION, fixed_substeps=2)
    for sim in (a, b):
        sim.load()
        sim.step(60.0, 1)
    before = a.read()
    rows_ms, step_ms = CH.chad_diffusion_kernel_times(a.ctx, 3)
    assert rows_ms > 0.0 and step_ms > 0.0
    after = a.read()
    assert np.array_equal(before["y"], after["y"]) and np.array_equal(before["pos"], after["pos"])
    a.step(60.0, 1)
    b.step(60.0, 1)
    ra, rb = a.read(), b.read()
    a.close()
    b.close()
    assert np.array_equal(ra["y"], rb["y"])


def test_diffusion_in_the_mixed_form_within_its_tolerance():
    """Diffusion runs before either precision form: the mixed form with
    diffusion stays within the mixed form's 1e-4 of the FP64 oracle."""
    pop = I.config_population(2, n=1200)
    g = gpu_run(pop, 60.0, 3, diffusion=DIFFUSION, precision=CH.PREC_MIXED, fixed_substeps=4)
    o = oracle_run(pop, 60.0, 3, diffusion=DIFFUSION, fixed_n=4)
    assert np.all(g["status"] == 0)
    assert relerr(g["y"], o["y"]).max() < 1e-4


def test_positions_by_id_from_device_buffers():
    """chad_set_positions_by_id with torch CUDA tensors (the in-memory form of
    a frame) lands the positions in particle order."""
    torch = pytest.importorskip("torch")
    pop = I.config_population(2, n=2000)
    sim = CH.Simulator(pop)
    sim.load()
    new = I.config_population(2, n=2000, seed_offset=41).pos
    perm = np.random.default_rng(2).permutation(2000)
    pos_d = torch.from_numpy(np.ascontiguousarray(new[:, perm])).cuda()
    ids_d = torch.from_numpy(perm.astype(np.int64)).cuda()
    CH.chad_set_positions_by_id(sim.ctx, 0, 2000, pos_d, ids_d)
    got = sim.read()["pos"]
    sim.close()
    assert np.array_equal(got, new)


def test_checkpoint_round_trip_is_bitwise(tmp_path):
    """Stop after two intervals, save y, pos, S_H, h and the interval index,
    restore into a fresh context and run two more: bitwise the states and
    positions of an uninterrupted four-interval run (flow with noise, inlet
    slab, shared headspace, diffusion)."""
    pop = I.config_population(2, n=1500)
    full = gpu_run(pop, 60.0, 4, diffusion=DIFFUSION)
    a = CH.Simulator(pop, diffusion=DIFFUSION)
    a.load()
    a.step(60.0, 2)
    mid = a.read()
    k = CH.chad_get_interval(a.ctx)
    a.close()
    assert k == 2
    b = CH.Simulator(pop, diffusion=DIFFUSION)
    b.load(y=mid["y"], pos=mid["pos"], T=pop.T, S_H=mid["S_H"], h=mid["h"])
    CH.chad_set_interval(b.ctx, k)
    b.step(60.0, 2)
    end = b.read()
    b.close()
    assert np.array_equal(end["pos"], full["pos"])
    assert np.array_equal(end["y"], full["y"])
    assert np.array_equal(end["S_H"], full["S_H"]) and np.array_equal(end["h"], full["h"])
    # the same through the binding's checkpoint file
    c = CH.Simulator(pop, diffusion=DIFFUSION)
    c.load()
    c.step(60.0, 2)
    c.checkpoint(tmp_path / "ck.npz")
    c.close()
    d = CH.Simulator(pop, diffusion=DIFFUSION)
    d.restore(tmp_path / "ck.npz")
    d.step(60.0, 2)
    end2 = d.read()
    d.close()
    assert np.array_equal(end2["y"], full["y"]) and np.array_equal(end2["pos"], full["pos"])


_BOUNDS_SCRIPT = r"""
import dataclasses, sys
import numpy as np
from paper_2311_08927_gb300 import chad as CH, inputs as I
assert CH.chad_debug_bounds(reset=True)[0] == 1
# diffusion: lab cylinder, then crowded particles (rows beyond the capacity
# formed on the fly) and a capped plan
for s_, dif in ((1.0, (1e-5, 0.024)), (0.15, (1e-6, 0.024)), (0.15, (6.5e-6, 0.024))):
    pop = I.config_population(2, n=1500)
    c = np.array([0.0, 0.0, 0.15])[:, None]
    pop.pos = c + s_ * (pop.pos - c)
    sim = CH.Simulator(pop, diffusion=dif)
    sim.load()
    sim.step(1.0 if s_ < 1.0 else 60.0, 2)
    sim.read()
    sim.close()
# positions by id, the adaptive integrator with its ordering pass, 64 digesters
pop = I.config_population(2, n=1000)
sim = CH.Simulator(pop)
sim.load()
perm = np.random.default_rng(1).permutation(1000)
CH.chad_set_positions_by_id(sim.ctx, 0, 1000, np.ascontiguousarray(pop.pos[:, perm]), perm.astype(np.int64))
sim.step(60.0, 2)
sim.close()
for cfg, n in ((3, 3000), (5, 3000)):
    sim = CH.Simulator(I.config_population(cfg, n=n))
    sim.load()
    sim.step(60.0, 2)
    sim.read()
    sim.close()
en, st = CH.chad_debug_bounds()
print("bounds", en, st)
sys.exit(0 if (en == 1 and st == 0) else 1)
"""


def test_bounds_check_build_records_no_violation():
    """The bounds-check build (libchad_debug.so) checks every data-dependent
    index of the diffusion, ordering and frame kernels and records a failed
    check instead of trapping; small runs of every path record none."""
    import os
    import subprocess
    import sys
    from paper_2311_08927_gb300 import build as B
    lib = B.build(debug_bounds=True)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, CHAD_LIB=lib, PYTHONPATH=root)
    r = subprocess.run([sys.executable, "-c", _BOUNDS_SCRIPT], env=env, cwd=root,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    assert "bounds 1 0" in r.stdout


def test_c_program_matches_the_binding(tmp_path):
    """A plain C99 program (tests/c/run_digester.c) drives the library through
    chad.h alone: on the same seeded inputs its states equal, bitwise, those
    of the same run through the Python binding."""
    import struct
    import subprocess
    from test_abi import _cc, build_c_caller
    if _cc() is None:
        pytest.skip("no C compiler")
    exe = build_c_caller(tmp_path / "run_digester")
    pop = I.config_population(1, n=64)
    d = pop.digesters[0]
    n, k, dt = pop.n, 3, 60.0
    with open(tmp_path / "in.bin", "wb") as f:
        f.write(struct.pack("<qqddddd", n, k, dt, d.V_liq, d.V_gas, d.D, 1e-6))
        for arr in (d.params, I.atol_vector(), d.y_in, pop.y, pop.T):
            f.write(np.ascontiguousarray(arr, dtype="<f8").tobytes())
    r = subprocess.run([exe, str(tmp_path / "in.bin"), str(tmp_path / "out.bin")],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    raw = (tmp_path / "out.bin").read_bytes()
    y = np.frombuffer(raw, dtype="<f8", count=29 * n).reshape(29, n)
    SH = np.frombuffer(raw, dtype="<f8", count=n, offset=8 * 29 * n)
    h = np.frombuffer(raw, dtype="<f8", count=n, offset=8 * 30 * n)
    st = np.frombuffer(raw, dtype="<i4", count=n, offset=8 * 31 * n)
    g = gpu_run(pop, dt, k)
    assert np.all(st == 0)
    assert np.array_equal(y, g["y"]) and np.array_equal(SH, g["S_H"]) and np.array_equal(h, g["h"])


def test_diffusion_settings_changed_between_steps_match_oracle():
    """Two intervals with one (D, h), two with another (a finer grid, more
    substeps), one with diffusion off: the library re-plans the grid, the
    operator's capacity and the interval graph at each change; the oracle is
    run the same way, chained interval by interval.  Fixed ADM1 steps."""
    pop = I.config_population(2, n=1500)
    plan = [((1e-6, 0.03), 2), ((1e-5, 0.02), 2), (None, 1)]
    sim = CH.Simulator(pop, fixed_substeps=4)
    sim.load()
    y, pos, SH, h, k0 = pop.y.copy(), pop.pos.copy(), None, None, 0
    for dif, k in plan:
        CH.chad_set_diffusion(sim.ctx, 0, dif[0] if dif else 0.0, dif[1] if dif else 0.0)
        sim.step(60.0, k)
        step_pop = I.Population(pop.digesters, y, pop.T, pos, pop.shared_headspace)
        o = O.run(step_pop, 60.0, k, interval0=k0, fixed_n=4, SH=SH, h=h, diffusion=dif)
        y, pos, SH, h, k0 = o["y"], o["pos"], o["S_H"], o["h"], k0 + k
    g = sim.read()
    sim.close()
    assert np.all(g["status"] == 0)
    assert np.array_equal(g["pos"], pos)
    assert relerr(g["y"], y).max() < 1e-9


def test_diffusion_rerun_is_bitwise_deterministic():
    """The cell lists are ordered by particle index after the atomic scatter,
    so the neighbour sums run in a fixed order."""
    pop = I.config_population(2, n=2000)
    a = gpu_run(pop, 60.0, 2, diffusion=DIFFUSION)
    b = gpu_run(pop, 60.0, 2, diffusion=DIFFUSION)
    assert np.array_equal(a["y"], b["y"])


def _crowded(n, s=0.15):
    """Config 2 with every particle pulled to within s of its distance from
    the tank's centre: neighbour counts far above the uniform fill."""
    pop = I.config_population(2, n=n)
    c = np.array([0.0, 0.0, 0.15])[:, None]
    pop.pos = c + s * (pop.pos - c)
    return pop


def test_diffusion_crowded_particles_match_oracle():
    """Crowded particles: the substep count comes from the operator's
    largest row sum at the interval's positions (computed on the GPU by an
    atomic max), several times the continuum estimate; states to 1e-9."""
    pop = _crowded(400)
    dif = (1e-6, 0.024)
    g = gpu_run(pop, 1.0, 2, diffusion=dif, fixed_substeps=2)
    o = oracle_run(pop, 1.0, 2, diffusion=dif, fixed_n=2)
    smax = O.diffusion_row_sum_max(o["pos"], pop.digesters[0].V_liq / 400, *dif)
    assert O.diffusion_substeps(1.0, smax) > 1 >= math.ceil(7.0 * dif[0] / dif[1] ** 2)
    assert np.all(g["status"] == 0)
    assert relerr(g["y"], o["y"]).max() < 1e-9
    # the last interval's plan: the same integer substep count, S_max to round-off
    info = g["diff_info"]
    assert info["n_sub"] == O.diffusion_substeps(1.0, smax) and info["capped"] == 0
    assert abs(info["s_max"] / smax - 1.0) < 1e-12


def test_diffusion_plan_above_the_cap_is_flagged():
    """A plan above the launched substeps (8 times the continuum estimate,
    at least 8) runs them all and marks every diffusing particle with
    CHAD_P_DIFFUSION (32); chosen just above the cap (dt_sub S_max about
    1.07), so the states stay finite."""
    pop = _crowded(400)
    dif = (6.5e-6, 0.024)
    o = oracle_run(pop, 1.0, 1, diffusion=dif)
    smax = O.diffusion_row_sum_max(o["pos"], pop.digesters[0].V_liq / 400, *dif)
    assert 8 < O.diffusion_substeps(1.0, smax) and 1.0 * smax / 8 < 1.1
    g = gpu_run(pop, 1.0, 1, diffusion=dif)
    assert g["diff_info"]["capped"] == 1 and g["diff_info"]["n_sub"] == 8
    assert np.all(g["status"] & 32)
    assert np.all(np.isfinite(g["y"]))
    ok = gpu_run(pop, 1.0, 1, diffusion=(1e-6, 0.024))
    assert np.all(ok["status"] == 0)


def test_diffusion_needs_flow_geometry():
    pop = I.config_population(1, n=16)
    sim = CH.Simulator(pop)
    with pytest.raises(CH.ChadError) as ei:
        CH.chad_set_diffusion(sim.ctx, 0, 1e-5, 0.01)
    assert ei.value.code == 4
    sim.close()


# ------------------------------------------------------------ S_h2 algebraic (Eq. 8)
def test_h2_algebraic_fixed_steps_match_oracle():
    """The FP64 kernel form with S_h2 from Eq. 8 at every evaluation against
    the oracle's algebraic mode, fixed steps: states (including the stored
    S_h2 root) to 1e-9, with temperature spread and slugs."""
    pop = I.config_population(3, n=2000)
    g = gpu_run(pop, 60.0, 3, fixed_substeps=4, h2_algebraic=True)
    o = oracle_run(pop, 60.0, 3, fixed_n=4, h2_algebraic=True)
    assert np.all(g["status"] == 0)
    assert relerr(g["y"], o["y"]).max() < 1e-9


def test_h2_algebraic_adaptive_tight_tolerance_matches_oracle():
    pop = I.config_population(3, n=2000)
    idx = np.concatenate([pop.slugs[:16], np.setdiff1d(np.arange(2000), pop.slugs)[:48]])
    sp = subset(pop, idx)
    atol = I.atol_vector(1e-13)
    g = gpu_run(sp, 60.0, 4, rtol=1e-10, atol=atol, h2_algebraic=True)
    o = oracle_run(sp, 60.0, 4, rtol=1e-10, atol=atol, h2_algebraic=True)
    assert np.all(g["status"] == 0) and np.all(o["status"] == 0)
    assert relerr(g["y"], o["y"]).max() < 1e-9
    assert abs(g["stats"]["accepted_steps"] - o["stats"][0]) <= 2


def test_h2_algebraic_production_tolerance_and_differential_form():
    """At rtol 1e-6 the algebraic form stays within 1e-4 of the tight
    algebraic oracle, and within 1e-4 of the differential form (the two
    models differ by the quasi-steady error of a sub-second S_h2)."""
    pop = I.config_population(3, n=3000)
    idx = np.concatenate([pop.slugs[:24], np.setdiff1d(np.arange(3000), pop.slugs)[:72]])
    sp = subset(pop, idx)
    g = gpu_run(sp, 60.0, 20, rtol=1e-6, h2_algebraic=True)
    o = oracle_run(sp, 60.0, 20, rtol=1e-10, atol=I.atol_vector(1e-13), h2_algebraic=True)
    assert np.all(g["status"] == 0)
    assert relerr(g["y"], o["y"]).max() < 1e-4
    d = gpu_run(sp, 60.0, 20, rtol=1e-6)
    assert relerr(g["y"], d["y"]).max() < 1e-4


def test_h2_algebraic_takes_the_fp64_and_mixed_forms_only():
    pop = I.config_population(1, n=16)
    with pytest.raises(CH.ChadError) as ei:
        CH.Simulator(pop, precision=CH.PREC_MIXED_F32RATES, h2_algebraic=True)
    assert ei.value.code == 1
    CH.Simulator(pop, precision=CH.PREC_MIXED, h2_algebraic=True).close()


# ------------------------------------------------------------ flow, headspace, digesters
def test_flow_positions_bitwise_and_shared_headspace_parity():
    pop = I.config_population(2, n=1500)
    g = gpu_run(pop, 60.0, 4, fixed_substeps=3)
    o = oracle_run(pop, 60.0, 4, fixed_n=3)
    assert np.array_equal(g["pos"], o["pos"])
    assert relerr(g["y"], o["y"]).max() < 1e-9
    gas = g["y"][26:29]
    assert np.all(gas == gas[:, :1])  # one headspace per digester
    # some particles sat in the inlet slab and were diluted
    assert np.any(pop.pos[2] >= pop.digesters[0].flow["slab_zmin"])


def test_paper_literal_stepping_matches_oracle():
    """Paper-literal stepping (Sec. 4.3): 0.5-s coupling intervals, each 10
    fixed substeps of 0.05 s, in the lab cylinder with swirl flow, inlet slab
    and shared headspace.  Positions bitwise, states to 1e-9 of the oracle."""
    pop = I.config_population(2, n=1500)
    g = gpu_run(pop, 0.5, 40, fixed_substeps=10)
    o = oracle_run(pop, 0.5, 40, fixed_n=10)
    assert np.all(g["status"] == 0)
    assert np.array_equal(g["pos"], o["pos"])
    assert relerr(g["y"], o["y"]).max() < 1e-9
    assert g["stats"]["accepted_steps"] == 1500 * 40 * 10


def test_many_digesters_parity():
    pop = I.config_population(5, n=2500)
    assert len(pop.digesters) == 64
    g = gpu_run(pop, 60.0, 3, fixed_substeps=2)
    o = oracle_run(pop, 60.0, 3, fixed_n=2)
    assert np.array_equal(g["pos"], o["pos"])
    assert relerr(g["y"], o["y"]).max() < 1e-9
    for d in range(64):
        a, b = pop.offsets[d], pop.offsets[d + 1]
        gas = g["y"][26:29, a:b]
        assert np.all(gas == gas[:, :1])


def test_uniform_population_reduces_to_single_cstr():
    """Sec. 3.1 / 4.2: identical particles with a shared headspace equal the CSTR."""
    n = 777
    base = I.x_ss()
    y = np.repeat(base[:, None], n, axis=1)
    D = I.TABLE1["Q"] / I.TABLE1["V_liq"]
    pop = I.Population([I.Digester(n=n, D=D)], y, np.full(n, I.T_OP), np.zeros((3, n)), True)
    g = gpu_run(pop, 60.0, 10, rtol=1e-8, atol=I.atol_vector(1e-11))
    assert np.all(g["y"] == g["y"][:, :1])
    yc, SH, h = base.copy(), 1e-7, 0.0
    for _ in range(10):
        yc, SH, h, st, _ = O.integrate(I.default_params(), I.T_OP, yc, 60.0 / 86400, rtol=1e-8,
                                       atol=I.atol_vector(1e-11), y_in=I.influent(), D=D, SH=SH, h=h)
    assert np.max(np.abs(g["y"][:, 0] - yc) / np.abs(yc)) < 1e-9


def test_rerun_is_bitwise_deterministic():
    pop = I.config_population(2, n=2000)
    a = gpu_run(pop, 60.0, 3)
    b = gpu_run(pop, 60.0, 3)
    assert np.array_equal(a["y"], b["y"]) and np.array_equal(a["pos"], b["pos"])


# ------------------------------------------------------------ full size, sampled
@pytest.mark.parametrize("precision,tol", [(CH.PREC_FP64, 1e-9), (CH.PREC_MIXED, 1e-4)])
def test_full_size_1M_sampled(precision, tol):
    """The metric workload (1M particles, slugs, T spread) in the benchmark's
    launch configuration; a seeded sample is recomputed particle by particle
    by the oracle (FP64 at the same rtol / the tight oracle for mixed)."""
    pop = I.config_population(3)
    sim = CH.Simulator(pop, precision=precision, rtol=1e-6)
    sim.load()
    sim.step(60.0, 2)
    g = sim.read()
    sim.close()
    assert np.all(g["status"] == 0)
    rng = np.random.default_rng(99)
    idx = np.sort(np.concatenate([rng.choice(pop.slugs, 16, replace=False),
                                  rng.choice(pop.n, 48, replace=False), [0, pop.n - 1]]))
    sp = subset(pop, idx)
    if precision == CH.PREC_FP64:
        o = oracle_run(sp, 60.0, 2, rtol=1e-6)
        e = relerr(g["y"][:, idx], o["y"])
        assert np.median(e) < tol and e.max() < 1e-5
    else:
        o = oracle_run(sp, 60.0, 2, rtol=1e-10, atol=I.atol_vector(1e-13))
        assert relerr(g["y"][:, idx], o["y"]).max() < tol


def test_full_size_lab_cylinder_100k_whole_tank():
    """The lab-cylinder workload at full size (100,000 particles, swirl +
    noise, inlet slab, shared headspace), one 60-s interval in the FP64 form
    at rtol 1e-6, against the oracle on the whole tank at the same rtol:
    positions bitwise, states to round-off for most particles and within the
    production bound for all (a round-off flip of an accept/reject decision
    moves a particle by O(rtol))."""
    pop = I.config_population(2)
    assert pop.n == 100_000
    g = gpu_run(pop, 60.0, 1, rtol=1e-6)
    o = oracle_run(pop, 60.0, 1, rtol=1e-6)
    assert np.all(g["status"] == 0) and np.all(o["status"] == 0)
    assert np.array_equal(g["pos"], o["pos"])
    e = relerr(g["y"], o["y"])
    assert np.median(e) < 1e-10 and e.max() < 1e-5


def test_runtime_is_linear_in_particles():
    """The paper reports ADM1 time linear in the particle count (Sec. 4.3):
    once the GPU is full, the time per particle-interval of the 1M recipe at
    1, 2 and 4 million particles agrees within 15 % (intervals 2-4, after a
    cold start and one warm interval)."""
    torch = pytest.importorskip("torch")
    per = []
    for n in (1_000_000, 2_000_000, 4_000_000):
        pop = I.config_population(3, n=n)
        s = torch.cuda.Stream()
        sim = CH.Simulator(pop, stream=s.cuda_stream)
        sim.load()
        sim.step(60.0, 2)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        sim.step(60.0, 3)
        e1.record(s)
        torch.cuda.synchronize()
        st = sim.read()
        sim.close()
        assert np.all(st["status"] == 0)
        per.append(e0.elapsed_time(e1) / (3 * n))
    assert max(per) / min(per) < 1.15, per


# ------------------------------------------------------------ failure handling
def test_step_limit_sets_status_without_faulting():
    pop = I.config_population(1, n=64)
    sim = CH.Simulator(pop, max_steps=1)
    sim.load()
    sim.step(60.0, 1)
    out = sim.read()
    assert np.all(out["status"] & CH.P_STEPS)
    code = CH.chad_read_states(sim.ctx, 0, status=np.zeros(64, dtype=np.int32))
    assert code == 5  # CHAD_E_PARTICLE
    sim.close()


def test_newton_iteration_limit_falls_back_to_bisection():
    pop = I.config_population(1, n=64)
    g = gpu_run(pop, 60.0, 2, max_newton=1, fixed_substeps=2)
    o = oracle_run(pop, 60.0, 2, fixed_n=2)
    assert np.all(g["status"] == 0)
    assert g["stats"]["newton_fallbacks"] > 0
    assert relerr(g["y"], o["y"]).max() < 1e-9


def test_call_order_and_argument_errors():
    pop = I.config_population(1, n=16)
    sim = CH.Simulator(pop)
    with pytest.raises(CH.ChadError) as ei:
        sim.step(60.0, 1)                              # not loaded
    assert ei.value.code == 4
    bad = pop.y.copy()
    bad[3, 5] = -1.0
    with pytest.raises(CH.ChadError) as ei:
        CH.chad_load_particles(sim.ctx, 0, 16, pop.pos, np.ascontiguousarray(bad), pop.T)
    assert ei.value.code == 1
    with pytest.raises(CH.ChadError):
        CH.chad_load_particles(sim.ctx, 0, 15, None, np.ascontiguousarray(pop.y[:, :15]))
    with pytest.raises(CH.ChadError):
        CH.chad_load_particles(sim.ctx, 1, 16, None, pop.y)
    sim.load()
    with pytest.raises(CH.ChadError):
        sim.step(-1.0, 1)
    sim.step(60.0, 0)
    sim.close()


def test_empty_digester_and_single_particle():
    y1 = I.x_ss()[:, None].copy()
    dg = [I.Digester(n=0), I.Digester(n=1)]
    pop = I.Population(dg, y1, np.array([I.T_OP]), np.zeros((3, 1)), False)
    g = gpu_run(pop, 60.0, 3, fixed_substeps=2)
    o = oracle_run(pop, 60.0, 3, fixed_n=2)
    assert relerr(g["y"], o["y"]).max() < 1e-9


def test_device_buffers_through_torch():
    torch = pytest.importorskip("torch")
    pop = I.config_population(1, n=100)
    sim = CH.Simulator(pop)
    y = torch.from_numpy(np.ascontiguousarray(pop.y)).cuda()
    T = torch.from_numpy(np.ascontiguousarray(pop.T)).cuda()
    CH.chad_load_particles(sim.ctx, 0, 100, None, y, T)
    sim.step(60.0, 2)
    out = torch.empty_like(y)
    st = torch.zeros(100, dtype=torch.int32, device="cuda")
    code = CH.chad_read_states(sim.ctx, 0, y=out, status=st)
    sim.close()
    assert code == 0
    ref = gpu_run(pop, 60.0, 2)
    assert np.array_equal(out.cpu().numpy(), ref["y"])


# ------------------------------------------------------------ model, tuning, graphs
def test_device_jacobian_matches_oracle_ad():
    """The kernels' analytic Jacobian, evaluated on the GPU, equals the
    oracle's dual-number Jacobian to 1e-12 (column-relative)."""
    rng = np.random.default_rng(8)
    for _ in range(10):
        y = I.x_ss() * np.exp(0.3 * rng.standard_normal(I.NS))
        T = rng.uniform(303.15, 313.15)
        f, J, SH = CH.eval_model(I.default_params(), T, y, y_in=I.influent(), D=0.2, on_device=True)
        Jo = O.jacobian(I.default_params(), T, y, y_in=I.influent(), D=0.2)
        assert np.max(np.abs(J - Jo) / (np.abs(Jo).max(axis=0, keepdims=True) + 1e-300)) < 1e-12


def test_device_conversions_and_reciprocal():
    """The integrator's integer bit-pattern conversions and its FP64
    reciprocal against exact references: narrowing truncates the significand
    to 24 bits (round toward zero; below the normal float range a signed
    zero, from 2^128 up +-Inf), widening reproduces the float exactly
    (subnormal floats become a signed zero), the reciprocal is within 2 ulp
    of the correctly rounded 1/x."""
    rng = np.random.default_rng(12)
    special = [0.0, -0.0, 1.0, -1.0, 2.0 ** -126, -(2.0 ** -126), 2.0 ** -127, 1e-40, 3.4e38,
               2.0 ** 128, -(2.0 ** 128), 1e39, np.inf, -np.inf, np.nan, np.nextafter(1.0, 2.0),
               np.nextafter(2.0 ** 128, 0.0), 1e-300, 1e300, 1e-31, 1e31]
    x = np.concatenate([rng.standard_normal(50000) * 10.0 ** rng.uniform(-40, 40, 50000),
                        np.asarray(special)])
    nar, wid, rec = CH.probe_numerics(x)
    with np.errstate(all="ignore"):
        m, e = np.frexp(np.abs(x))
        trunc = np.sign(x) * np.ldexp(np.floor(np.ldexp(m, 24)), e - 24)
        ref = np.where(np.abs(x) < 2.0 ** -126, np.copysign(0.0, x), trunc)
        ref = np.where(np.abs(x) >= 2.0 ** 128, np.copysign(np.inf, x), ref)
        ref = np.where(np.isnan(x), np.nan, ref)
    np.testing.assert_array_equal(nar.astype(np.float64), ref)
    assert np.array_equal(np.signbit(nar), np.signbit(ref))
    with np.errstate(all="ignore"):
        f32 = x.astype(np.float32).astype(np.float64)
        wref = np.where((np.abs(f32) < 2.0 ** -126) & (f32 != 0), np.copysign(0.0, f32), f32)
    np.testing.assert_array_equal(wid, wref)
    assert np.array_equal(np.signbit(wid), np.signbit(wref))
    with np.errstate(all="ignore"):
        exact = 1.0 / x
    fin = np.isfinite(exact) & (exact != 0)
    ulp = np.spacing(np.abs(exact[fin]))
    assert np.max(np.abs(rec[fin] - exact[fin]) / ulp) <= 2.0
    np.testing.assert_array_equal(rec[~fin], exact[~fin])


def _run_stream(pop, n, tune=False, graph=True, precision=CH.PREC_FP64):
    import torch
    s = torch.cuda.Stream() if graph else None
    sim = CH.Simulator(pop, precision=precision, stream=None if s is None else s.cuda_stream)
    sim.load()
    chosen = None
    if tune:
        chosen, ms = CH.chad_autotune(sim.ctx, 60.0)
        assert 0 <= chosen < len(ms) and np.all(ms > 0)
    sim.step(60.0, n)
    out = sim.read()
    sim.close()
    return out, chosen


@pytest.mark.parametrize("precision", [CH.PREC_FP64, CH.PREC_MIXED])
def test_autotune_and_graph_replay_leave_results_unchanged(precision):
    pop = I.config_population(2, n=3000)
    direct, _ = _run_stream(pop, 3, graph=False, precision=precision)
    graphed, _ = _run_stream(pop, 3, graph=True, precision=precision)
    tuned, chosen = _run_stream(pop, 3, tune=True, graph=True, precision=precision)
    assert np.array_equal(direct["y"], graphed["y"]) and np.array_equal(direct["pos"], graphed["pos"])
    assert relerr(tuned["y"], direct["y"]).max() < 1e-12
    assert np.array_equal(tuned["pos"], direct["pos"])


def test_mixed_f32_rates_form_within_tolerance():
    pop = I.config_population(3, n=3000)
    idx = np.concatenate([pop.slugs[:8], np.setdiff1d(np.arange(3000), pop.slugs)[:40]])
    sp = subset(pop, idx)
    g = gpu_run(sp, 60.0, 10, rtol=1e-6, precision=CH.PREC_MIXED_F32RATES)
    o = oracle_run(sp, 60.0, 10, rtol=1e-10, atol=I.atol_vector(1e-13))
    assert np.all(g["status"] == 0)
    assert relerr(g["y"], o["y"]).max() < 1e-4
