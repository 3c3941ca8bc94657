#!/usr/bin/env python3
"""Benchmark: particle-days simulated per second on the 1M-particle workload.

One step = one 60-s coupling interval of the whole hot path over the
1,000,000-particle heterogeneous-stiffness population (5 % substrate slugs,
per-particle temperature 303.15-313.15 K, per-particle headspace, no flow),
started from the seeded lognormal perturbation of the CSTR steady state.
Inputs stay resident in HBM (29 x 8 B x 1M = 232 MB of state > 129 MB L2).

Prints ONE JSON line (rank 0).  Under torchrun each rank integrates its own
1M-particle population (seed offset by rank; particles are independent, so
there is no data-path collective) and the slowest rank's time is reported.

--impl reference times the CPU oracle (FP64, all host cores) on a bounded
sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "adm1_particles_1M_heterogeneous"
METRIC = "particle-days simulated per second (1M particles, 60-s coupling intervals)"
UNIT = "particle-days/s"
DT_S = 60.0
N_PARTICLES = 1_000_000
STATE_BYTES = 29 * 8


# --------------------------------------------------------------------------- distributed
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(ws, backend):
    import torch.distributed as dist
    if ws > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return dist if ws > 1 else None


def barrier(dist, device=None):
    if dist is not None:
        if device is not None:
            dist.barrier(device_ids=[device])
        else:
            dist.barrier()


def max_over_ranks(dist, value: float, device="cpu") -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard_seed_offset(rank: int) -> int:
    """Weak scaling: each rank owns an independent 1M-particle population."""
    return 1000 * rank


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.samples = []
        self._stop = threading.Event()
        self._th = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits"],
                                     capture_output=True, text=True, timeout=5).stdout.strip()
                if out:
                    self.samples.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._th = threading.Thread(target=self._run, daemon=True)
        self._th.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self._th:
            self._th.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if len(s) > 5 + i and s[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


# --------------------------------------------------------------------------- algorithmic work
def work_per_launch(CH, precision, stats, steps, h2=False):
    """Algorithmic FP64 / FP32 operations of one integrator launch.

    Counts come from the kernel source (chad_flop_counts: the templated
    rate, Jacobian and sparse-LU routines run with an operation-counting
    scalar): per step attempt the W-method's rate evaluations, Jacobian,
    W formation, static-order sparse LU, three solves (mixed: FP32 solves
    plus FP64 refinement residuals J x) and stage combinations; per Newton
    iteration of Eq. 7 one charge-balance evaluation plus the update; per
    attempt three moves of the acid-base reciprocals to the converged root.
    The mixed form with S_h2 algebraic counts its two-float arithmetic at its
    FP32 cost and each FP32 Eq. 8 Newton iteration."""
    nf = CH.newton_flops()
    fin = CH.flop_counts()["sh_final"]
    attempts = stats["accepted_steps"] + stats["rejected_steps"]
    if h2 and precision == CH.PREC_MIXED:
        af = CH.attempt_flops_h2_mixed()
        f32 = attempts * af["fp32"] + stats["h2_newton_iters"] * af["fp32_per_h2_iter"]
    else:
        af = CH.attempt_flops(precision, h2)
        f32 = attempts * af["fp32"]
    f64 = attempts * (af["fp64"] + 3 * fin) + stats["newton_iters"] * nf
    if "fp64_per_h2_iter" in af:
        f64 += stats["h2_newton_iters"] * af["fp64_per_h2_iter"]
    return f64 / steps, f32 / steps, af


def alu_roofline(f64, f32, launch_ms, peak64, peak32):
    """The ALU roofline of a launch: the time the counted work needs on the
    pipe that bounds it, max(FP64 flops / FP64 peak, FP32 flops / FP32 peak),
    over the measured time.  achieved / peak are those of the bounding pipe."""
    t = launch_ms * 1e-3
    t64, t32 = f64 / (peak64 * 1e12), f32 / (peak32 * 1e12)
    if t64 >= t32:
        return {"pipe": "fp64", "achieved": f64 / t / 1e12, "peak": peak64, "frac": t64 / t}
    return {"pipe": "fp32", "achieved": f32 / t / 1e12, "peak": peak32, "frac": t32 / t}


def kernel_sources_hash():
    import hashlib
    h = hashlib.sha256()
    for f in ("adm1_device.cuh", "integrate_impl.cuh", "integrate_mx.cuh", "dfloat.cuh", "rank1.cuh",
              "sparse_lu_gen.cuh", "sparse_lu_h2a_gen.cuh", "model.h", "kernels.h"):
        with open(os.path.join(ROOT, "paper_2311_08927_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic_per_attempt(form: str):
    """DRAM bytes per step attempt from a committed ncu summary under
    profiles/, valid only while the kernel sources hash to the recorded value
    (otherwise None: the counters describe a different kernel)."""
    import glob
    cur = kernel_sources_hash()
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "integrate_*.md"))):
        rec = {}
        with open(path) as fh:
            for line in fh:
                if ":" in line and line.startswith("    "):
                    k, v = line.strip().split(":", 1)
                    rec[k.strip()] = v.strip()
        if rec.get("kernel_sources_sha256_16") == cur and f"{form}_dram_bytes_per_attempt" in rec:
            return float(rec[f"{form}_dram_bytes_per_attempt"]), os.path.basename(path)
    return None, None


def train_mlp(CH, I, args):
    """Train the learned-guess MLP on about 10^7 states from seeded runs of the
    lab-cylinder (100k particles) and heterogeneous (1M) workloads with seeds
    independent of the benchmark population; not timed as part of a step."""
    import torch
    from paper_2311_08927_gb300 import learned as Lm
    t0 = time.perf_counter()
    n3 = args.train_particles
    pops = [I.config_population(3, n=n3, seed_offset=100), I.config_population(2, seed_offset=100)]
    ys, Ts, SHs, hs = [], [], [], []
    for pop_t, k in zip(pops, (args.train_intervals, 11)):
        y, T, SH, h = Lm.sample_states(pop_t, k, h2_algebraic=(args.model == "h2alg"))
        ys.append(y); Ts.append(T); SHs.append(SH); hs.append(h)
    y, T, SH, h = torch.cat(ys, 1), torch.cat(Ts), torch.cat(SHs), torch.cat(hs)
    t1 = time.perf_counter()
    X, Y, norm, onorm = Lm.build_dataset(y, T, SH, h)
    params, hist, test_loss = Lm.train(X, Y, epochs=args.train_epochs, batch=16384, lr=2e-3)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    model = Lm.TrainedMLP(params, norm.cpu().numpy(), onorm, hist)
    e_sh, e_h = Lm.prediction_errors(model, y[:, -200000:].contiguous(), T[-200000:].contiguous(),
                                     SH[-200000:].contiguous(), h[-200000:].contiguous())
    info = {"samples": int(T.shape[0]), "epochs": args.train_epochs, "sampling_s": t1 - t0,
            "training_s": t2 - t1, "val_loss_before": hist[0][2], "val_loss_after": hist[-1][2],
            "test_loss": test_loss, "median_abs_log10_err_SH": e_sh,
            "median_abs_log10_err_h": e_h,
            "kernels": "chad_mlp_grad (BF16 tcgen05 fwd+bwd, TMEM accumulators) + chad_mlp_adam"}
    del X, Y, y, T, SH, h
    torch.cuda.empty_cache()
    return model, info


def cold_restart_ab(CH, pop, relaxed, model, stream, h2=False):
    """One interval after reloading relaxed states without S_H and h (as a
    coupling that reloads particle files would): plain start (S_H 1e-7, h
    1e-6 d) against the learned guesses, mixed form, CUDA-event timed."""
    import torch
    res = {}
    for name, learned in (("plain", False), ("learned", True)):
        sim = CH.Simulator(pop, precision=CH.PREC_MIXED, stream=stream.cuda_stream,
                           learned=1 if learned else 0, h2_algebraic=h2)
        if learned:
            CH.chad_set_mlp(sim.ctx, model.params, model.feat_norm, model.out_norm)
        sim.load(y=relaxed)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        sim.step(DT_S, 1)
        e1.record(stream)
        torch.cuda.synchronize()
        st = sim.read()["stats"]
        sim.close()
        res[name] = {"ms": e0.elapsed_time(e1),
                     "attempts_per_particle": (st["accepted_steps"] + st["rejected_steps"]) / pop.n,
                     "newton_iters_per_particle": st["newton_iters"] / pop.n,
                     "mlp_redo": st["mlp_redo"]}
    res["speedup"] = res["plain"]["ms"] / res["learned"]["ms"]
    return res


# --------------------------------------------------------------------------- our arm
# The five workloads: what each line reports and how its inputs meet the L2
# rule (state larger than the 129 MB L2, or a 256 MB flush before every
# timed interval, outside the interval's own events).
CONFIGS = {
    1: dict(workload="adm1_particles_1k_closed_batch", learned=False, flush=True,
            desc="1,000 particles, closed batch, 308.15 K, per-particle headspace, no flow",
            l2="state 0.3 MB fits in L2: 256 MB flush before every interval (not timed)"),
    2: dict(workload="lab_cylinder_100k_swirl_shared_headspace", learned=False, flush=True,
            desc="100,000 particles, lab cylinder D 0.2 m x H 0.3 m, swirl 0.05 m/s + noise "
                 "0.005 m/s, inlet slab, shared headspace",
            l2="state 30 MB fits in L2: 256 MB flush before every interval (not timed)"),
    3: dict(workload=WORKLOAD, learned=True, flush=False,
            desc="1,000,000 particles, 5 % slugs, T ~ U(303.15, 313.15) K, per-particle "
                 "headspace, no flow",
            l2="inputs larger than L2 (232 MB state)"),
    4: dict(workload="adm1_particles_2M_heterogeneous_learned", learned=True, flush=False,
            desc="2,000,000 particles as the 1M workload (new seed), learned guesses",
            l2="inputs larger than L2 (464 MB state)"),
    5: dict(workload="digesters_64_loguniform_learned_mixed", learned=True, flush=False,
            desc="64 digesters, particle counts log-uniform 1e4..2e5, kinetic parameters x "
                 "lognormal(0.2), own swirl each, shared headspace per digester, one "
                 "captured graph per interval",
            l2="inputs larger than L2 (~0.8 GB state)"),
}


# coupling intervals of 60 s in each workload's simulated duration
CONFIG_INTERVALS = {1: 1440, 2: 14400, 3: 7200, 4: 7200, 5: 2880}


def window_rates(per_ms, n_particles, k=20):
    """Particle-days/s over the first and the last k timed intervals."""
    d = n_particles * DT_S / 86400.0
    first, last = per_ms[:k], per_ms[-k:]
    return {"first_intervals": len(first), "first_value": d * len(first) / (sum(first) * 1e-3),
            "last_intervals": len(last), "last_value": d * len(last) / (sum(last) * 1e-3)}


def launches_per_interval(pop):
    """Kernels of one interval: ordering (2), integrator, interval bump; the
    advection when a digester has a flow; the headspace reduction (3) when
    it is shared."""
    k = 4
    if any(d.flow is not None for d in pop.digesters):
        k += 1
    if pop.shared_headspace:
        k += 3
    return k


def e2e_run(CH, pop, prec, stream, args, h2):
    """Host buffers through the C ABI: per interval and digester
    chad_load_particles from pinned host memory, chad_step, chad_read_states
    back into it; the copies are inside the timed region."""
    import torch
    N = pop.n
    sim = CH.Simulator(pop, precision=prec, rtol=1e-6, stream=stream.cuda_stream,
                       h2_algebraic=h2)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    flow = any(d.flow is not None for d in pop.digesters)
    off = pop.offsets
    bufs = []
    for d in range(len(pop.digesters)):
        a, b = off[d], off[d + 1]
        bufs.append(dict(n=b - a, y=pin(pop.y[:, a:b]), T=pin(pop.T[a:b]),
                         SH=pin(np.full(b - a, 1e-7)), h=pin(np.zeros(b - a)),
                         st=pin(np.zeros(b - a, dtype=np.int32)),
                         pos=pin(pop.pos[:, a:b]) if flow else None))

    def load():
        for d, B_ in enumerate(bufs):
            CH.chad_load_particles(sim.ctx, d, B_["n"], B_["pos"], B_["y"], B_["T"], B_["SH"],
                                   B_["h"])

    def read():
        for d, B_ in enumerate(bufs):
            CH.chad_read_states(sim.ctx, d, y=B_["y"], pos=B_["pos"], S_H=B_["SH"], h=B_["h"],
                                status=B_["st"])

    load()
    sim.step(DT_S, args.warmup)
    CH.chad_autotune(sim.ctx, DT_S)  # public API, as for the device-timed arm
    read()
    ksteps = max(1, min(args.steps, 20))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ksteps):
        load()
        sim.step(DT_S, 1)
        read()
    t1 = time.perf_counter()
    sim.close()
    pos_b = 3 * 8 if flow else 0
    h2d = N * (STATE_BYTES + 3 * 8 + pos_b)
    d2h = N * (STATE_BYTES + 2 * 8 + 4 + pos_b)
    return {"value": N * DT_S / 86400.0 * ksteps / (t1 - t0), "unit": UNIT,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": ksteps,
            "path": "chad_load_particles / chad_step / chad_read_states with pinned host "
                    "buffers, every digester, every interval"}


def run_ours(args, ws, rank, local, cfg=3):
    import torch
    torch.cuda.set_device(local)
    dist = init_dist(ws, "nccl")
    from paper_2311_08927_gb300 import build as B
    B.build()
    from paper_2311_08927_gb300 import chad as CH
    from paper_2311_08927_gb300 import inputs as I

    meta = CONFIGS[cfg]
    if args.full_run:
        # the workload's whole simulated duration: every interval after the
        # warm-up ones is timed
        args.steps = CONFIG_INTERVALS[cfg] - args.warmup
    pop = I.config_population(cfg, n=args.particles, seed_offset=shard_seed_offset(rank))
    N = pop.n
    dt_days = DT_S / 86400.0
    peak64 = CH.probe_alu_peak(True)
    peak32 = CH.probe_alu_peak(False)
    stream = torch.cuda.Stream()
    flush = (torch.empty(32 * 1024 * 1024, dtype=torch.float64, device="cuda")
             if meta["flush"] else None)

    h2m = args.model == "h2alg"
    model = None
    train_info = None
    if meta["learned"] and args.form in ("both", "mixed") and not args.no_learned:
        model, train_info = train_mlp(CH, I, args)

    def arm(precision, learned=False, h2=False):
        sim = CH.Simulator(pop, precision=precision, rtol=1e-6, stream=stream.cuda_stream,
                           learned=1 if learned else 0, h2_algebraic=h2)
        if learned:
            CH.chad_set_mlp(sim.ctx, model.params, model.feat_norm, model.out_norm)
        sim.load()
        sim.step(DT_S, args.warmup)
        CH.chad_synchronize(sim.ctx)
        variant, tune_ms = CH.chad_autotune(sim.ctx, DT_S)
        sim.read()  # resets the counters
        K = args.steps
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        barrier(dist, local)
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            ev[0].record(stream)
            for k in range(K):
                if flush is not None:
                    with torch.cuda.stream(stream):
                        flush.zero_()
                evs[k].record(stream)
                sim.step(DT_S, 1)
                ev[k + 1].record(stream)
            torch.cuda.synchronize()
        # per interval: from its own start (after any flush) to its end
        per = [evs[k].elapsed_time(ev[k + 1]) for k in range(K)]
        total_ms = sum(per) if flush is not None else ev[0].elapsed_time(ev[-1])
        total_ms = max_over_ranks(dist, total_ms, f"cuda:{local}")
        out = sim.read()
        st = out["stats"]
        attempts = st["accepted_steps"] + st["rejected_steps"]
        sim.close()
        launch_ms = statistics.mean(per)
        f64, f32, af = work_per_launch(CH, precision, st, K, h2)
        achieved = f64 / (launch_ms * 1e-3) / 1e12
        achieved32 = f32 / (launch_ms * 1e-3) / 1e12
        vinfo = CH.kernel_variant(precision, h2, variant)
        return dict(total_ms=total_ms, per_ms=per, launch_ms=launch_ms, stats=st,
                    f64_per_launch=f64, f32_per_launch=f32, attempt_flops=af,
                    achieved32_tflops=achieved32, variant_info=vinfo,
                    roof=alu_roofline(f64, f32, launch_ms, peak64, peak32),
                    variant=variant, tune_ms=[float(x) for x in tune_ms],
                    attempts=attempts, failed=int((out["status"] != 0).sum()),
                    clocks=clk.summary(), achieved_tflops=achieved,
                    y_final=out["y"])

    forms = {}
    for name, prec in (("mixed", CH.PREC_MIXED), ("fp64", CH.PREC_FP64)):
        if args.form in (name, "both"):
            forms[name] = arm(prec, learned=(name == "mixed" and model is not None), h2=h2m)
    if h2m and args.form == "both" and cfg == 3 and not args.no_differential:
        # the FP64 form of the other reading of S_h2 (a differential state)
        forms["fp64_differential"] = arm(CH.PREC_FP64, h2=False)
    if args.form == "fp64_h2alg":
        # S_h2 algebraic (Eq. 8): the counted attempt flops are those of the
        # differential FP64 form (the Eq. 8 solves and the second rank-1
        # level are not counted)
        forms["fp64_h2alg"] = arm(CH.PREC_FP64, h2=True)
    head = "mixed" if "mixed" in forms else ("fp64" if "fp64" in forms else "fp64_h2alg")
    H = forms[head]
    value = ws * N * dt_days * args.steps / (H["total_ms"] * 1e-3)

    # ---------------- learned guesses on a cold restart (reload without S_H, h)
    cold = None
    if model is not None and rank == 0 and cfg in (3, 4):
        cold = cold_restart_ab(CH, pop, H["y_final"], model, stream, h2m)

    # ---------------- e2e: host buffers through the C ABI, copies in the timed region
    e2e = None
    if rank == 0 and not args.no_e2e:
        prec = CH.PREC_MIXED if head == "mixed" else CH.PREC_FP64
        e2e = e2e_run(CH, pop, prec, stream, args, h2m or head == "fp64_h2alg")

    # ---------------- CPU baseline: the oracle on a bounded sample, same intervals
    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(pop, args.warmup, min(args.steps, 10), args.cpu_seconds, cfg,
                           h2m or head == "fp64_h2alg")

    if rank != 0:
        return None
    fr = H["clocks"]
    tkey = head + ("_h2alg" if (h2m and head != "fp64_h2alg") else "")
    tpa, tsrc = measured_traffic_per_attempt(tkey) if cfg == 3 else (None, None)
    traffic = None if tpa is None else tpa * H["attempts"] / args.steps
    default_n = {1: 1000, 2: 100_000, 3: N_PARTICLES, 4: 2_000_000, 5: None}[cfg]
    wl = meta["workload"] if (args.particles is None or N == default_n) else f"{meta['workload']}_n{N}"
    metric = METRIC if cfg == 3 else f"particle-days simulated per second ({meta['desc']})"
    res = {
        "metric": metric, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": H["total_ms"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if head == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": wl, "description": meta["desc"],
                   "particles_per_gpu": N, "digesters": len(pop.digesters),
                   "coupling_interval_s": DT_S,
                   "form": head + ((" (S_h2 algebraic, Eq. 8: FP32 rates, Jacobian and LU, "
                                    "two-float refinement residual, FP64 Eq. 7 Newton and state)"
                                    if h2m else " (FP32 Jacobian/LU + FP64 refinement)")
                                   if head == "mixed" else (" (S_h2 algebraic, Eq. 8)" if h2m else ""))
                + (" + learned guesses" if (head == "mixed" and model is not None) else ""),
                   "model": "S_h2 algebraic (Eq. 8)" if (h2m or head == "fp64_h2alg")
                            else "S_h2 a differential state",
                   "learned_guesses": model is not None, "rtol": 1e-6,
                   "l2": meta["l2"],
                   "parallelism": f"particles sharded, {ws} independent populations"},
        "roofline": {"bound": "alu", "achieved": H["roof"]["achieved"], "peak": H["roof"]["peak"],
                     "unit": "TFLOP/s", "frac": H["roof"]["frac"], "pipe": H["roof"]["pipe"],
                     "traffic": traffic,
                     "traffic_source": (f"profiles/{tsrc}: DRAM bytes per attempt x attempts per launch"
                                        if tsrc else "no capture of the current kernel on this workload"),
                     "kernel": ("integrate_mx_kernel" if (h2m and head == "mixed") else "integrate_kernel"),
                     "definition": "max(FP64 flops / FP64 peak, FP32 flops / FP32 peak) / launch time; "
                                   "achieved and peak of the bounding pipe",
                     "peak_source": "measured DFMA / FFMA chains on every SM (chad_probe_alu_peak)",
                     "fp64_tflops_achieved": H["achieved_tflops"],
                     "fp64_flops_per_launch": H["f64_per_launch"],
                     "attempt_flops": H["attempt_flops"],
                     "attempts_per_step": H["attempts"] / args.steps,
                     "fp32": {"achieved": H["achieved32_tflops"], "peak": peak32,
                              "frac": H["achieved32_tflops"] / peak32}},
        "peaks_measured": {"fp64_tflops": peak64, "fp32_tflops": peak32},
        "clocks": fr,
        "gpu_launches": launches_per_interval(pop) * args.steps,
        "steps_per_particle_interval": H["stats"]["accepted_steps"] / (N * args.steps),
        "rejected_per_particle_interval": H["stats"]["rejected_steps"] / (N * args.steps),
        "step_spread": [H["stats"]["min_steps"], H["stats"]["max_steps"]],
        "failed_particles": H["failed"],
        "kernel_variant": H["variant"], "kernel_variant_shape": H["variant_info"],
        "autotune_ms": H["tune_ms"],
        "pivot_rejects_per_step": H["stats"]["pivot_rejects"] / args.steps,
        "graph_per_interval": True,
        "windows": window_rates(H["per_ms"], ws * N),
    }
    if args.full_run:
        res["full_run"] = {"simulated_days": CONFIG_INTERVALS[cfg] * DT_S / 86400.0,
                           "timed_intervals": args.steps, "untimed_first_intervals": args.warmup}
    if "fp64" in forms and head != "fp64":
        F = forms["fp64"]
        def summary(F):
            return {
                "value": ws * N * dt_days * args.steps / (F["total_ms"] * 1e-3),
                "ms_per_step": F["total_ms"] / args.steps,
                "roofline": {"bound": "alu", "achieved": F["roof"]["achieved"],
                             "peak": F["roof"]["peak"], "unit": "TFLOP/s",
                             "frac": F["roof"]["frac"], "pipe": F["roof"]["pipe"],
                             "fp64_flops_per_launch": F["f64_per_launch"],
                             "attempt_flops": F["attempt_flops"]},
                "steps_per_particle_interval": F["stats"]["accepted_steps"] / (N * args.steps),
                "rejected_per_particle_interval": F["stats"]["rejected_steps"] / (N * args.steps),
                "kernel_variant": F["variant"], "kernel_variant_shape": F["variant_info"],
                "clocks": F["clocks"],
                "windows": window_rates(F["per_ms"], ws * N),
            }
        res["plain_fp64"] = summary(F)
        res["plain_fp64"]["model"] = "S_h2 algebraic (Eq. 8)" if h2m else "S_h2 a differential state"
        if "fp64_differential" in forms:
            res["plain_fp64_differential"] = summary(forms["fp64_differential"])
            res["plain_fp64_differential"]["model"] = "S_h2 a differential state"
            G = forms["fp64_differential"]
            d2 = np.abs(H["y_final"] - G["y_final"]) / np.maximum(
                np.abs(G["y_final"]), 1e-12 * np.abs(G["y_final"]).max(axis=1, keepdims=True))
            res["mixed_vs_fp64_differential_max_rel"] = float(d2.max())
        res["mixed_over_fp64"] = F["total_ms"] / H["total_ms"]
        d = np.abs(H["y_final"] - F["y_final"]) / np.maximum(
            np.abs(F["y_final"]), 1e-12 * np.abs(F["y_final"]).max(axis=1, keepdims=True))
        res["mixed_vs_fp64_max_rel"] = float(d.max())
    if train_info:
        res["learned_training"] = train_info
    if cold:
        res["learned_cold_restart"] = cold
    if e2e:
        res["e2e"] = e2e
    if cpu:
        res["cpu_baseline"] = cpu
    return res


def _oracle_sample(pop, n_s, seed=7):
    from paper_2311_08927_gb300 import inputs as I
    rng = np.random.default_rng(seed)
    n_s = min(n_s, pop.n)
    idx = np.sort(rng.choice(pop.n, n_s, replace=False))
    return I.Population([I.Digester(n=n_s)], pop.y[:, idx].copy(), pop.T[idx].copy(),
                        np.zeros((3, n_s)), False)


def _sampler(pop, cfg):
    """n -> a seeded oracle sample of the workload.  Independent particles
    (configs 1, 3, 4): n particles drawn from the population.  Flow and a
    shared headspace (configs 2, 5): the same recipe at n particles in all,
    whole tanks (every digester, its flow and its headspace mean), since a
    shared headspace couples the particles of a tank."""
    from paper_2311_08927_gb300 import inputs as I
    if cfg in (2, 5):
        return lambda n, seed=7: I.config_population(cfg, n=max(n, 64 if cfg == 2 else 640),
                                                     seed_offset=900 + seed)
    return lambda n, seed=7: _oracle_sample(pop, n, seed)


def _calibrate_sample(sample, intervals, budget_s, cores, cap, h2=False):
    """Sample size for about budget_s seconds of oracle work over `intervals`."""
    import oracle as O
    n_cal = min(cap, 64 * max(1, cores // 4))
    sub = sample(n_cal, 11)
    t0 = time.perf_counter()
    O.run(sub, DT_S, min(intervals, 3), rtol=1e-6, n_threads=cores, h2_algebraic=h2)
    per = (time.perf_counter() - t0) / (sub.n * min(intervals, 3))
    return int(max(128, min(cap, 50_000, budget_s / max(per, 1e-9) / intervals)))


def cpu_baseline(pop, warmup, k, budget_s, cfg=3, h2=False):
    """The oracle as it stands (FP64, std::thread equal chunks over all host
    cores) on a seeded sample of the workload, over the same intervals; the
    sample grows until the timed part takes about budget_s seconds."""
    import oracle as O
    from paper_2311_08927_gb300 import inputs as I
    cores = os.cpu_count() or 1
    sample = _sampler(pop, cfg)
    cap = pop.n if cfg == 1 else 200_000
    n_s = _calibrate_sample(sample, warmup + k, budget_s, cores, cap, h2)

    def timed(sub, threads):
        r = O.run(sub, DT_S, warmup, rtol=1e-6, n_threads=threads, h2_algebraic=h2)
        sub2 = I.Population(sub.digesters, r["y"], sub.T, r["pos"], sub.shared_headspace)
        t0 = time.perf_counter()
        O.run(sub2, DT_S, k, interval0=warmup, rtol=1e-6, SH=r["S_H"], h=r["h"],
              n_threads=threads, h2_algebraic=h2)
        return time.perf_counter() - t0

    for _ in range(3):
        sub = sample(n_s)
        dt = timed(sub, cores)
        if dt >= 0.5 * budget_s or n_s >= cap:
            break
        n_s = int(min(cap, n_s * budget_s / max(dt, 1e-3)))
    n_s = sub.n
    # the same timed intervals on one core, for a sample sized to ~1/4 of the budget
    s1 = sample(max(64, int(n_s * 0.25 / cores)), 13)
    dt1 = timed(s1, 1)
    what = lambda s_: (f"particles in {len(s_.digesters)} whole tank(s) of the same recipe"
                       if cfg in (2, 5) else "seeded particles of the workload")
    return {"value": n_s * k * DT_S / 86400.0 / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n_s} {what(sub)}, intervals {warmup}..{warmup + k - 1} "
                      f"(after {warmup} untimed), rtol 1e-6"
                      f"{', S_h2 algebraic' if h2 else ''}, {dt:.1f} s",
            "one_core": {"value": s1.n * k * DT_S / 86400.0 / dt1, "unit": UNIT, "cores": 1,
                         "sample": f"{s1.n} other {what(s1)}, same intervals, {dt1:.1f} s"}}


# --------------------------------------------------------------------------- paper-literal workload
FIG7_N = 110_929
FIG7_DT_S = 0.5
FIG7_SUB = 10


def run_fig7(args, ws, rank, local):
    """Paper-literal stepping, the shape of the paper's own timing (Sec. 4.3,
    Fig. 7): 110,929 particles, one coupling interval of 0.5 s integrated as
    10 fixed substeps of 0.05 s, here in the lab cylinder with the swirl
    flow, inlet slab and shared headspace, FP64.  Not the headline workload."""
    import torch
    torch.cuda.set_device(local)
    from paper_2311_08927_gb300 import build as B
    B.build()
    from paper_2311_08927_gb300 import chad as CH
    from paper_2311_08927_gb300 import inputs as I
    pop = I.config_population(2, n=FIG7_N)
    stream = torch.cuda.Stream()
    peak64 = CH.probe_alu_peak(True)
    sim = CH.Simulator(pop, precision=CH.PREC_FP64, fixed_substeps=FIG7_SUB,
                       stream=stream.cuda_stream)
    sim.load()
    sim.step(FIG7_DT_S, args.warmup)
    CH.chad_synchronize(sim.ctx)
    sim.read()
    k = 10 * args.steps
    # the state (~32 MB) fits in L2: flush it between intervals with a 256 MB
    # write, inside the timed region
    flush = torch.empty(32 * 1024 * 1024, dtype=torch.float64, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(k):
            with torch.cuda.stream(stream):
                flush.zero_()
            sim.step(FIG7_DT_S, 1)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st = sim.read()["stats"]
    sim.close()
    f64, _, af = work_per_launch(CH, CH.PREC_FP64, st, k)
    achieved = f64 / (ms / k * 1e-3) / 1e12
    days = FIG7_DT_S / 86400.0
    res = {"metric": "particle-days simulated per second (paper-literal stepping)",
           "value": FIG7_N * days * k / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": k,
           "warmup": args.warmup, "ms_per_step": ms / k, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "paper_fig7_110929_dt0.5s_10substeps", "particles": FIG7_N,
                      "coupling_interval_s": FIG7_DT_S, "substeps": FIG7_SUB,
                      "geometry": "lab cylinder, swirl + noise, inlet slab, shared headspace",
                      "l2": "state 32 MB fits in L2: 256 MB L2 flush before every interval, "
                            "inside the timed region"},
           "particle_steps_per_s": FIG7_N * FIG7_SUB * k / (ms * 1e-3),
           "roofline": {"bound": "alu", "achieved": achieved, "peak": peak64, "unit": "TFLOP/s",
                        "frac": achieved / peak64, "traffic": None,
                        "kernel": "whole interval (advect + integrate + headspace) FP64 flops",
                        "attempt_flops": af},
           "clocks": clk.summary(), "gpu_launches": k * 6}
    if not args.no_cpu:
        import oracle as O
        cores = os.cpu_count() or 1
        n_s = 2000
        for _ in range(3):
            sub = I.config_population(2, n=n_s)
            t0 = time.perf_counter()
            O.run(sub, FIG7_DT_S, 20, fixed_n=FIG7_SUB, n_threads=cores)
            dt = time.perf_counter() - t0
            if dt >= 0.5 * args.cpu_seconds or n_s >= 100_000:
                break
            n_s = int(min(100_000, n_s * args.cpu_seconds / max(dt, 1e-3)))
        res["cpu_baseline"] = {"value": n_s * days * 20 / dt, "unit": UNIT, "cores": cores,
                               "kind": "oracle",
                               "sample": f"{n_s} particles of the same recipe, 20 intervals of "
                                         f"0.5 s x 10 substeps, {dt:.1f} s"}
    return res


# --------------------------------------------------------------------------- diffusion workload
LAB_D, LAB_H = 1.0e-6, 0.006   # m^2/s; m (about 1.3 mean particle spacings at 100k particles)


def run_lab_diffusion(args, ws, rank, local):
    """Diffusion between particles (the paper's planned extension, Sec. 2.3):
    the lab cylinder (100k particles, swirl + noise, inlet slab, shared
    headspace), 60-s intervals of advection, SPH diffusion (D = 1e-6 m^2/s,
    h = 6 mm) and FP64 ADM1 (--form fp64_h2alg: with S_h2 from Eq. 8).  Not
    the headline workload.  The roofline object
    covers the diffusion substep kernel (FP64 multiply-adds of the sparse
    product), timed through chad_diffusion_kernel_times after the timed run."""
    import torch
    torch.cuda.set_device(local)
    from paper_2311_08927_gb300 import build as B
    B.build()
    from paper_2311_08927_gb300 import chad as CH
    from paper_2311_08927_gb300 import inputs as I
    pop = I.config_population(2)
    N = pop.n
    stream = torch.cuda.Stream()
    peak64 = CH.probe_alu_peak(True)
    h2 = args.form == "fp64_h2alg"
    sim = CH.Simulator(pop, precision=CH.PREC_FP64, stream=stream.cuda_stream,
                       diffusion=(LAB_D, LAB_H), h2_algebraic=h2)
    sim.load()
    sim.step(DT_S, args.warmup)
    CH.chad_synchronize(sim.ctx)
    sim.read()
    k = args.steps
    # state, operator and slot buffers (~150 MB) are about L2's size: flush it
    # with a 256 MB write before every interval, inside the timed region
    flush = torch.empty(32 * 1024 * 1024, dtype=torch.float64, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(k):
            with torch.cuda.stream(stream):
                flush.zero_()
            sim.step(DT_S, 1)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    out = sim.read()
    info = CH.chad_diffusion_info(sim.ctx)
    rows_ms, step_ms = [], []
    for _ in range(5):
        with torch.cuda.stream(stream):
            flush.zero_()
        r, t = CH.chad_diffusion_kernel_times(sim.ctx, 1)
        rows_ms.append(r)
        step_ms.append(t)
    sim.close()
    rows_ms, step_ms = statistics.median(rows_ms), statistics.median(step_ms)
    # one substep: a multiply-add per entry and species, and per particle and
    # species the update c + dt (acc - S c) (two more)
    flops_step = 2.0 * 14 * info["entries"] + 4.0 * 14 * N
    achieved = flops_step / (step_ms * 1e-3) / 1e12
    st = out["stats"]
    days = DT_S / 86400.0
    # kernels per interval: advect, 2 ordering, integrate, 3 headspace, bump;
    # diffusion: count, scan, scatter, sort, gather, rows, plan, the enqueued
    # substeps (8 x ceil(dt 7 D / h^2), at least 8) and store
    max_sub = max(8, 8 * math.ceil(DT_S * 7.0 * LAB_D / LAB_H ** 2))
    res = {"metric": "particle-days simulated per second (with diffusion between particles)",
           "value": N * days * k / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": k,
           "warmup": args.warmup, "ms_per_step": ms / k, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"lab_cylinder_{N}_diffusion_D{LAB_D:g}_h{LAB_H:g}",
                      "particles": N, "coupling_interval_s": DT_S, "rtol": 1e-6,
                      "form": "fp64, S_h2 algebraic (Eq. 8)" if h2 else "fp64, S_h2 a state",
                      "geometry": "lab cylinder, swirl + noise, inlet slab, shared headspace",
                      "l2": "256 MB L2 flush before every interval, inside the timed region"},
           "diffusion": {"substeps_last_interval": info["n_sub"], "entries": info["entries"],
                         "s_max_per_s": info["s_max"], "rows_ms": rows_ms,
                         "substep_ms": step_ms,
                         "share_of_interval": (rows_ms + info["n_sub"] * step_ms) / (ms / k)},
           "roofline": {"bound": "alu", "achieved": achieved, "peak": peak64, "unit": "TFLOP/s",
                        "frac": achieved / peak64, "traffic": None,
                        "kernel": "diffusion substep (diff_step), FP64 multiply-adds, entries "
                                  "= reserved bound",
                        "timing": "chad_diffusion_kernel_times after the timed run, L2 flushed "
                                  "before each of 5 launches, median"},
           "adm1": {"accepted_steps": st["accepted_steps"], "rejected_steps": st["rejected_steps"]},
           "clocks": clk.summary(), "gpu_launches": k * (8 + 8 + max_sub)}
    if not args.no_cpu:
        import oracle as O
        cores = os.cpu_count() or 1
        # all-pairs oracle: a sample of n_s particles in the same tank, h and D
        # scaled so the neighbours per particle and the substeps stay the same
        n_s = 2000
        scale = (N / n_s) ** (1.0 / 3.0)
        h_s, D_s = LAB_H * scale, LAB_D * scale ** 2
        sub = I.config_population(2, n=n_s)
        t0 = time.perf_counter()
        O.run(sub, DT_S, 2, n_threads=cores, diffusion=(D_s, h_s), h2_algebraic=h2)
        dt = time.perf_counter() - t0
        res["cpu_baseline"] = {"value": n_s * days * 2 / dt, "unit": UNIT, "cores": cores,
                               "kind": "oracle",
                               "sample": f"{n_s} particles of the same recipe with h = {h_s:.4f} m, "
                                         f"D = {D_s:.3g} m^2/s (same neighbours per particle and "
                                         f"substeps), 2 intervals, {dt:.1f} s"}
    return res


# --------------------------------------------------------------------------- frame files
FRAME_N = 1_000_000


def run_frames(args, ws, rank, local):
    """Particle frames from an external CFD (the paper's per-step particle
    files, Sec. 2.3): 1M particles of the lab cylinder, one FP32 frame file
    per coupling step with the entries shuffled and their uint32 ids (as an
    SPH code writes them), loaded with chad_load_frame and followed by the
    60-s interval (advection off: U = 0, no noise; FP64 ADM1).  Files are
    written before the timed region and read from the page cache.  Not the
    headline workload."""
    import dataclasses
    import tempfile
    import torch
    torch.cuda.set_device(local)
    from paper_2311_08927_gb300 import build as B
    B.build()
    from paper_2311_08927_gb300 import chad as CH
    from paper_2311_08927_gb300 import frames as F
    from paper_2311_08927_gb300 import inputs as I
    base = I.config_population(2, n=FRAME_N)
    dg = dataclasses.replace(base.digesters[0], flow=I.swirl_flow(U=0.0, sigma=0.0, seed=9))
    pop = I.Population([dg], base.y, base.T, base.pos, base.shared_headspace)
    stream = torch.cuda.Stream()
    k = args.steps
    rng = np.random.default_rng(5)
    tmp = tempfile.mkdtemp(prefix="chad_frames_")
    paths = []
    for j in range(args.warmup + k):
        pos = I.config_population(2, n=FRAME_N, seed_offset=200 + j).pos
        perm = rng.permutation(FRAME_N)
        path = os.path.join(tmp, f"{j:05d}.frm")
        F.write_frame(path, pos[:, perm], ids=perm.astype(np.uint32), dtype=np.float32, step=j,
                      time_s=DT_S * j)
        paths.append(path)
    file_bytes = os.path.getsize(paths[0])
    sim = CH.Simulator(pop, precision=CH.PREC_FP64, stream=stream.cuda_stream)
    sim.load()
    for j in range(args.warmup):
        CH.chad_load_frame(sim.ctx, 0, paths[j])
        sim.step(DT_S, 1)
    CH.chad_synchronize(sim.ctx)
    load_s, step_ms = [], []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        t_all = time.perf_counter()
        for j in range(args.warmup, args.warmup + k):
            t0 = time.perf_counter()
            CH.chad_load_frame(sim.ctx, 0, paths[j])   # returns after the GPU check
            load_s.append(time.perf_counter() - t0)
            e0.record(stream)
            sim.step(DT_S, 1)
            e1.record(stream)
            torch.cuda.synchronize()
            step_ms.append(e0.elapsed_time(e1))
        wall = time.perf_counter() - t_all
    out = sim.read()
    sim.close()
    for pth in paths:
        os.remove(pth)
    os.rmdir(tmp)
    load_ms = 1e3 * statistics.median(load_s)
    days = DT_S / 86400.0
    return {"metric": "particle-days simulated per second (positions from frame files)",
            "value": FRAME_N * days * k / wall, "unit": UNIT, "n_gpus": 1, "steps": k,
            "warmup": args.warmup, "ms_per_step": 1e3 * wall / k, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"frames_lab_cylinder_{FRAME_N}", "particles": FRAME_N,
                       "coupling_interval_s": DT_S,
                       "frame": f"FP32 positions + uint32 ids, entries shuffled, {file_bytes} bytes",
                       "geometry": "lab cylinder, positions from the frames (U = 0, no noise), "
                                   "inlet slab, shared headspace",
                       "l2": "state 300 MB > L2"},
            "frames": {"load_ms": load_ms, "file_MB_per_s": file_bytes / 1e6 / (load_ms * 1e-3),
                       "particles_per_s": FRAME_N / (load_ms * 1e-3),
                       "interval_ms": statistics.median(step_ms),
                       "load_share": load_ms / (1e3 * wall / k),
                       "timing": "host clock around chad_load_frame (read, widen, copy, GPU "
                                 "scatter and id check, blocking); page cache warm"},
            "roofline": None,
            "roofline_note": "the frame path is bound by host file reading and the pageable "
                             "host-to-device copy; its GPU scatter is in profiles/",
            "failed_particles": int((out["status"] != 0).sum()),
            "clocks": clk.summary(), "gpu_launches": k * (8 + 2)}


# --------------------------------------------------------------------------- reload coupling
def run_reload(args, ws, rank, local):
    """A coupling that hands the species over at every interval without the
    integrator's own history (the paper's file-based coupling reloads the
    particle data at every CFD step, Sec. 2.3): each interval starts with
    chad_load_particles from device buffers carrying y and T but no S_H and
    no step size, then chad_step.  The 1M-particle heterogeneous workload,
    mixed form, at rtol 1e-6.  Plain: Newton from S_H = 1e-7 and a first
    step of 1e-6 d.  Learned: both from the network (Newton bounded, plain
    restart when it fails, counted).  Load + interval timed with CUDA events."""
    import torch
    torch.cuda.set_device(local)
    from paper_2311_08927_gb300 import build as B
    B.build()
    from paper_2311_08927_gb300 import chad as CH
    from paper_2311_08927_gb300 import inputs as I
    pop = I.config_population(3, n=args.particles)
    N = pop.n
    stream = torch.cuda.Stream()
    model, train_info = train_mlp(CH, I, args)
    y0 = torch.from_numpy(np.ascontiguousarray(pop.y)).cuda()
    T = torch.from_numpy(np.ascontiguousarray(pop.T)).cuda()
    res_arms = {}
    finals = {}
    for name, learned in (("plain", False), ("learned", True)):
        sim = CH.Simulator(pop, precision=CH.PREC_MIXED, rtol=1e-6, stream=stream.cuda_stream,
                           learned=1 if learned else 0, h2_algebraic=(args.model == "h2alg"))
        if learned:
            CH.chad_set_mlp(sim.ctx, model.params, model.feat_norm, model.out_norm)
        y = y0.clone()
        torch.cuda.synchronize()
        for _ in range(args.warmup):
            CH.chad_load_particles(sim.ctx, 0, N, None, y, T)
            sim.step(DT_S, 1)
            CH.chad_read_states(sim.ctx, 0, y=y)
        CH.chad_synchronize(sim.ctx)
        sim.read()  # resets the counters
        K = args.steps
        e0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        e1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        with ClockSampler(local) as clk:
            for k in range(K):
                e0[k].record(stream)
                CH.chad_load_particles(sim.ctx, 0, N, None, y, T)
                sim.step(DT_S, 1)
                e1[k].record(stream)
                CH.chad_read_states(sim.ctx, 0, y=y)
            torch.cuda.synchronize()
        per = [e0[k].elapsed_time(e1[k]) for k in range(K)]
        st = sim.read()["stats"]
        finals[name] = y.cpu().numpy()
        sim.close()
        res_arms[name] = {"ms_per_interval": statistics.mean(per),
                          "value": N * DT_S / 86400.0 * K / (sum(per) * 1e-3),
                          "attempts_per_particle_interval":
                              (st["accepted_steps"] + st["rejected_steps"]) / (N * K),
                          "newton_iters_per_particle_interval": st["newton_iters"] / (N * K),
                          "mlp_redo": st["mlp_redo"], "mlp_redo_fraction": st["mlp_redo"] / (N * K),
                          "clocks": clk.summary()}
    L, P_ = res_arms["learned"], res_arms["plain"]
    a, b = finals["learned"], finals["plain"]
    d = np.abs(a - b) / np.maximum(np.abs(b), 1e-12 * np.abs(b).max(axis=1, keepdims=True))
    return {"metric": "particle-days simulated per second (species reloaded every interval)",
            "value": L["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": L["ms_per_interval"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"reload_coupling_{WORKLOAD}", "particles": N,
                       "coupling_interval_s": DT_S, "rtol": 1e-6,
                       "form": "mixed + learned guesses (network at every reload)",
                       "model": ("S_h2 algebraic (Eq. 8)" if args.model == "h2alg"
                                 else "S_h2 a differential state"),
                       "reload": "chad_load_particles (device buffers: y, T; no S_H, no h) "
                                 "before every interval, inside the timed region",
                       "l2": "inputs larger than L2 (232 MB state)"},
            "learned": L, "plain": P_, "learned_over_plain": P_["ms_per_interval"] / L["ms_per_interval"],
            "learned_vs_plain_max_rel": float(d.max()),
            "learned_training": train_info,
            "roofline": None,
            "roofline_note": "the integrator's roofline is reported by the default workload; "
                             "this line measures the work the guesses save",
            "clocks": L["clocks"],
            # load: part constants, 3 fills; step: MLP guesses, ordering (2), integrator, bump
            "gpu_launches": args.steps * 9}



# --------------------------------------------------------------------------- reference arm
def run_reference(args, ws, rank):
    dist = init_dist(ws, "gloo")
    if rank != 0:
        barrier(dist)
        return None
    from paper_2311_08927_gb300 import inputs as I
    import oracle as O
    pop = I.config_population(3)
    cores = os.cpu_count() or 1
    h2 = args.model == "h2alg"
    n_s = _calibrate_sample(_sampler(pop, 3), args.warmup + args.steps, 4 * args.cpu_seconds,
                            cores, 200_000, h2)
    sub = _oracle_sample(pop, n_s)
    r = O.run(sub, DT_S, args.warmup, rtol=1e-6, n_threads=cores, h2_algebraic=h2)
    y, SH, h = r["y"], r["S_H"], r["h"]
    times = []
    for k in range(args.steps):
        s2 = I.Population(sub.digesters, y, sub.T, sub.pos, False)
        t0 = time.perf_counter()
        r = O.run(s2, DT_S, 1, interval0=args.warmup + k, rtol=1e-6, SH=SH, h=h, n_threads=cores,
                  h2_algebraic=h2)
        times.append(time.perf_counter() - t0)
        y, SH, h = r["y"], r["S_H"], r["h"]
    tot = sum(times)
    value = n_s * args.steps * DT_S / 86400.0 / tot
    barrier(dist)
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "particles_per_step_sample": n_s,
                       "coupling_interval_s": DT_S, "rtol": 1e-6,
                       "model": "S_h2 algebraic (Eq. 8)" if h2 else "S_h2 a differential state"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{n_s} seeded particles of the 1M workload per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--form", choices=["both", "mixed", "fp64", "fp64_h2alg"], default="both",
                    help="fp64_h2alg: FP64 with S_h2 algebraic (Eq. 8), not the headline")
    ap.add_argument("--model", choices=["differential", "h2alg"], default="h2alg",
                    help="h2alg (default): S_h2 algebraic (Eq. 8, the paper's DAE form) in both "
                         "forms; differential: S_h2 a state")
    ap.add_argument("--full-run", action="store_true",
                    help="time every interval of the workload's whole simulated duration "
                         "(after the warm-up intervals), e.g. 7,200 for the 5-day 1M workload")
    ap.add_argument("--no-differential", action="store_true",
                    help="skip the extra FP64 arm with S_h2 a differential state")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-learned", action="store_true", help="skip the learned guesses")
    ap.add_argument("--train-particles", type=int, default=1_000_000)
    ap.add_argument("--train-intervals", type=int, default=10)
    ap.add_argument("--train-epochs", type=int, default=20)
    ap.add_argument("--workload", choices=["default", "c1", "c2", "c3", "c4", "c5", "fig7",
                                           "lab_diffusion", "frames", "reload"],
                    default="default",
                    help="default = c3 (the 1M-particle headline); c1..c5: the five workloads, "
                         "each with both forms side by side; reload: species reloaded without "
                         "S_H and h every interval, learned against plain guesses; fig7: paper-literal stepping, "
                         "110,929 particles, 0.5-s intervals of 10 substeps; lab_diffusion: "
                         "100k particles with diffusion between them")
    ap.add_argument("--particles", type=int, default=None,
                    help="override the 1M particles (profiling captures only)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    ws, rank, local = dist_env()
    if args.impl == "reference":
        res = run_reference(args, ws, rank)
    elif args.workload == "fig7":
        res = run_fig7(args, ws, rank, local) if rank == 0 else None
    elif args.workload == "lab_diffusion":
        res = run_lab_diffusion(args, ws, rank, local) if rank == 0 else None
    elif args.workload == "frames":
        res = run_frames(args, ws, rank, local) if rank == 0 else None
    elif args.workload == "reload":
        res = run_reload(args, ws, rank, local) if rank == 0 else None
    else:
        cfg = 3 if args.workload == "default" else int(args.workload[1])
        res = run_ours(args, ws, rank, local, cfg)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)
    if ws > 1:
        # every rank leaves together, after rank 0's untimed extras
        import torch.distributed as dist
        if dist.is_initialized():
            dist.barrier()
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
