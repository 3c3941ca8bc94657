"""Learned initial guesses (an AI-systems pattern layered on the method).

A small MLP maps the log-scaled ADM1 state and the temperature of a particle
to log10 S_H+ (the Eq. 7 root) and log10 of a good next step size.  It is
trained on states the integrator itself produces (accepted interval ends of
seeded runs), with the library's own tensor-core forward/backward kernels
and Adam (chad_mlp_grad, chad_mlp_adam), and installed with chad_set_mlp.
The Newton solver and the step controller remain the judges: a learned S_H
that Newton cannot confirm in 4 iterations (|E| <= 1e-10) is redone from the
plain guess, and a poor step size is simply rejected by the controller.

Where it helps: particles that start an interval without history (loaded
without S_H and h -- e.g. a coupling that reloads particle states from a CFD
frame), whose plain start is S_H = 1e-7 and h = 1e-6 d.

Torch is used for device memory only; every numerical step runs in the
library's kernels: feature and target statistics, standardisation, the
shuffled batches (keyed permutations, no stored index arrays), the
tensor-core forward/backward and Adam.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import chad as CH
from . import inputs as I

NS = I.NS


@dataclass
class TrainedMLP:
    params: np.ndarray      # [NPARAM] float32
    feat_norm: np.ndarray   # [64] float32: mean[32], 1/std[32]
    out_norm: np.ndarray    # [4] float32: mean log10 S_H, mean log10 h, std, std
    history: list           # (epoch, train loss, validation loss)


def sample_states(pop: I.Population, intervals: int, precision=CH.PREC_MIXED, skip: int = 1,
                  max_samples: int | None = None, stream=None, initial: bool = True,
                  h2_algebraic: bool = False):
    """Run the integrator on `pop` and collect (y, T, S_H, h) at every interval
    end after the first `skip` ones.  With `initial`, the loaded states are
    sampled too (a cold load is where the network is consulted): a first
    1-ms interval makes the stored S_H the Eq. 7 root at the loaded state,
    and their step-size target is the controller's proposal at the end of
    the first full interval.  Returns device tensors y [29][M], T [M],
    S_H [M], h [M]."""
    import torch
    sim = CH.Simulator(pop, precision=precision, stream=stream, h2_algebraic=h2_algebraic)
    sim.load()
    n = pop.n
    T = torch.from_numpy(np.ascontiguousarray(pop.T)).cuda()
    ys, Ts, SHs, hs = [], [], [], []
    total = 0
    first = None
    if initial:
        sim.step(1e-3, 1)
        y0 = torch.empty((NS, n), dtype=torch.float64, device="cuda")
        SH0 = torch.empty(n, dtype=torch.float64, device="cuda")
        CH.chad_read_states(sim.ctx, 0, y=y0, S_H=SH0)
        first = (y0, SH0)
    for k in range(intervals):
        sim.step(60.0, 1)
        if first is not None:
            h1 = torch.empty(n, dtype=torch.float64, device="cuda")
            CH.chad_read_states(sim.ctx, 0, h=h1)
            ys.append(first[0])
            Ts.append(T)
            SHs.append(first[1])
            hs.append(h1)
            total += n
            first = None
        if k < skip:
            continue
        y = torch.empty((NS, n), dtype=torch.float64, device="cuda")
        SH = torch.empty(n, dtype=torch.float64, device="cuda")
        h = torch.empty(n, dtype=torch.float64, device="cuda")
        CH.chad_read_states(sim.ctx, 0, y=y, S_H=SH, h=h)
        ys.append(y)
        Ts.append(T)
        SHs.append(SH)
        hs.append(h)
        total += n
        if max_samples and total >= max_samples:
            break
    sim.close()
    return torch.cat(ys, 1), torch.cat(Ts), torch.cat(SHs), torch.cat(hs)


def _prep_scratch():
    import torch
    return torch.empty(CH.mlp_prep_scratch_bytes() // 8 + 1, dtype=torch.float64, device="cuda")


def feature_norm(y, T):
    """Mean and inverse std of the features (log10 max(y, 1e-20), T/100),
    computed by the library (chad_mlp_feature_norm)."""
    import torch
    norm = torch.empty(64, dtype=torch.float32, device="cuda")
    CH.chad_mlp_feature_norm(y, T, norm, _prep_scratch())
    return norm


def build_dataset(y, T, SH, h, norm=None):
    """Features X [M][32] (BF16 bits in int16) and standardised targets Y [M][2],
    both formed by the library's kernels."""
    import torch
    if norm is None:
        norm = feature_norm(y, T)
    M = T.shape[0]
    X = torch.empty((M, 32), dtype=torch.int16, device="cuda")
    CH.chad_mlp_features(y, T, norm, X)
    Y = torch.empty((M, 2), dtype=torch.float32, device="cuda")
    on = torch.empty(4, dtype=torch.float32, device="cuda")
    CH.chad_mlp_targets(SH, h, Y, on, _prep_scratch())
    return X, Y, norm, on.cpu().numpy().astype(np.float32)


def init_params(seed=0):
    """He-style initialisation of the 32-64-64-2 network (float32)."""
    rng = np.random.default_rng(seed)
    parts = [rng.standard_normal((64, 32)) * np.sqrt(2.0 / 32), np.zeros(64),
             rng.standard_normal((64, 64)) * np.sqrt(2.0 / 64), np.zeros(64),
             rng.standard_normal((2, 64)) * np.sqrt(1.0 / 64), np.zeros(2)]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def _key(seed, k):
    """64-bit permutation key number k of a training run (SplitMix64 of seed, k)."""
    z = (seed * 0x9E3779B97F4A7C15 + (k + 1) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
    return z ^ (z >> 31)


def train(X, Y, epochs=20, batch=32768, lr=3e-3, seed=0, split=(0.90, 0.05)):
    """Adam on the mean-squared error, train/validation/test split 90/5/5;
    the learning rate halves every 8 epochs.  Returns (params float32,
    history [(epoch, train loss, validation loss)], test loss); epoch -1 is
    the validation loss before training.

    Every step runs in the library: the split and the per-epoch order are
    keyed permutations applied by chad_mlp_gather, the batch gradient is
    chad_mlp_grad_async, the update chad_mlp_adam; each batch loss lands in
    its own device slot and the host waits once per epoch (chad_mlp_wait)."""
    import torch
    M = X.shape[0]
    n_tr, n_va = int(split[0] * M), int(split[1] * M)
    n_te = M - n_tr - n_va
    split_key = _key(seed, 0)
    P = torch.from_numpy(init_params(seed)).cuda()
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    grad = torch.zeros_like(P)
    Xb = torch.empty((batch, 32), dtype=torch.int16, device="cuda")
    Yb = torch.empty((batch, 2), dtype=torch.float32, device="cuda")
    scratch = torch.empty(CH.mlp_grad_scratch_bytes(batch) // 4 + 1, dtype=torch.float32,
                          device="cuda")
    bs = max(1, min(batch, n_tr))
    nb = n_tr // bs
    losses = torch.zeros(max(nb, (max(n_va, n_te) + batch - 1) // batch), dtype=torch.float32,
                         device="cuda")

    def eval_loss(off, n):
        cnts = []
        for k, s in enumerate(range(0, n, batch)):
            c = min(batch, n - s)
            CH.chad_mlp_gather(X, Y, split_key, off, n, 0, s, c, Xb, Yb)
            CH.chad_mlp_grad_async(Xb[:c], Yb[:c], P, grad, losses[k:k + 1], scratch)
            cnts.append(c)
        CH.chad_mlp_wait()
        lv = losses[:len(cnts)].cpu().numpy()
        return float(np.dot(lv, cnts) / max(n, 1))

    hist = [(-1, float("nan"), eval_loss(n_tr, n_va))]  # before training
    step = 0
    for ep in range(epochs):
        ek = _key(seed, ep + 1)
        for b in range(nb):
            CH.chad_mlp_gather(X, Y, split_key, 0, n_tr, ek, b * bs, bs, Xb, Yb)
            CH.chad_mlp_grad_async(Xb[:bs], Yb[:bs], P, grad, losses[b:b + 1], scratch)
            step += 1
            CH.chad_mlp_adam(P, grad, m, v, step, lr * (0.5 ** (ep // 8)))
        CH.chad_mlp_wait()
        run = float(losses[:nb].cpu().numpy().astype(np.float64).mean())  # a copy, no kernel
        hist.append((ep, run, eval_loss(n_tr, n_va)))
    return P.cpu().numpy(), hist, eval_loss(n_tr + n_va, n_te)


def train_from_runs(pops, intervals=10, epochs=20, batch=32768, lr=3e-3, max_samples=None,
                    seed=0) -> tuple[TrainedMLP, float]:
    """Sample states from runs of the given populations and train the MLP."""
    import torch
    ys, Ts, SHs, hs = [], [], [], []
    for pop in pops:
        y, T, SH, h = sample_states(pop, intervals, max_samples=max_samples)
        ys.append(y)
        Ts.append(T)
        SHs.append(SH)
        hs.append(h)
    y, T, SH, h = torch.cat(ys, 1), torch.cat(Ts), torch.cat(SHs), torch.cat(hs)
    X, Y, norm, out_norm = build_dataset(y, T, SH, h)
    params, hist, test_loss = train(X, Y, epochs=epochs, batch=batch, lr=lr, seed=seed)
    return TrainedMLP(params, norm.cpu().numpy(), out_norm, hist), test_loss


def prediction_errors(model: TrainedMLP, y, T, SH, h, n=20000):
    """Median |log10 error| of the learned S_H and h on n states (device)."""
    import torch
    n = min(n, T.shape[0])
    X = torch.empty((n, 32), dtype=torch.int16, device="cuda")
    CH.chad_mlp_features(y[:, :n].contiguous(), T[:n].contiguous(),
                         torch.from_numpy(model.feat_norm).cuda(), X)
    out = torch.empty((n, 2), dtype=torch.float32, device="cuda")
    CH.chad_mlp_forward(X, torch.from_numpy(model.params).cuda(), out)
    o = out.cpu().numpy().astype(np.float64)
    on = model.out_norm
    e_sh = np.abs(o[:, 0] * on[2] + on[0] - np.log10(SH[:n].cpu().numpy()))
    e_h = np.abs(o[:, 1] * on[3] + on[1] - np.log10(h[:n].cpu().numpy()))
    return float(np.median(e_sh)), float(np.median(e_h))


def install(sim: CH.Simulator, model: TrainedMLP) -> None:
    CH.chad_set_mlp(sim.ctx, model.params, model.feat_norm, model.out_norm)
