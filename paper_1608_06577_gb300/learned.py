"""Training driver of the learned root-find start (argument marshalling and the loop; every
arithmetic step runs in libkt's CUDA kernels).

Data: cells sampled uniformly from trajectories of the hotspot workload (the 128^3 grid of
the benchmark by default), every `every` steps, seeds distinct from the evaluation seed.
The network corrects the conformal root e_conf: y = 10 ln(e / e_conf) = r^2 z with r^2 = M^2/E^2
(feature 1), applied where r^2 > GATE_R2 (the same threshold as the kernels, KT_MLP_GATE_R2);
it is trained on z = y / r^2 over those cells.  Training: Adam on the mean squared error of z,
BF16 forward pass.
"""
from __future__ import annotations

import math

import numpy as np

from .binding import KT, KT_MIXED, MLP_NPARAM, mlp_adam, mlp_batch, mlp_grad, mlp_predict, mlp_targets

GATE_R2 = 1e-3  # KT_MLP_GATE_R2


def init_params(seed=0):
    """He-uniform initial weights (seeded), zero biases, as float32 numpy."""
    rng = np.random.default_rng(seed)
    p = np.zeros(MLP_NPARAM, dtype=np.float32)
    o = 0
    for fan_in, fan_out in ((6, 32), (32, 32), (32, 1)):
        lim = math.sqrt(6.0 / fan_in)
        p[o:o + fan_in * fan_out] = rng.uniform(-lim, lim, fan_in * fan_out)
        o += fan_in * fan_out + fan_out
    return p


def collect(problem_factory, seeds, n_samples, steps=100, every=10, sample_seed=1234):
    """Sample n_samples cells uniformly over the snapshots of the given seeds' trajectories: the
    features and targets are written by kt_mlp_features straight into the preallocated set."""
    import torch
    snaps = len(seeds) * (steps // every)
    per = int(math.ceil(n_samples / snaps))
    rng = np.random.default_rng(sample_seed)
    X = torch.empty((snaps * per, 6), dtype=torch.float32, device="cuda")
    Y = torch.empty(snaps * per, dtype=torch.float32, device="cuda")
    E = torch.empty(per, dtype=torch.float64, device="cuda")
    k = 0
    for seed in seeds:
        prob = problem_factory(seed)
        kt = KT(prob, precision=KT_MIXED)
        kt.set_problem_state()
        for _ in range(steps // every):
            kt.step(every)
            cells = torch.as_tensor(rng.integers(0, prob.ncells, per), device="cuda")
            kt.mlp_features(cells, out=(X[k * per:(k + 1) * per], Y[k * per:(k + 1) * per], E))
            k += 1
        del kt
    return X[:n_samples], Y[:n_samples]


def train(X, Y, epochs=20, batch=8192, lr=3e-3, lr_min=1e-4, seed=0, log=None):
    """Adam with cosine learning-rate decay over shuffled epochs (kt_mlp_batch draws each mini-batch
    of a keyed permutation, kt_mlp_grad and kt_mlp_adam do the rest); returns float32 CUDA
    parameters and the loss after each epoch."""
    import torch
    params = torch.as_tensor(init_params(seed), device="cuda")
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    n = X.shape[0]
    batch = min(batch, n)
    xb = torch.empty((batch, 6), dtype=torch.float32, device="cuda")
    yb = torch.empty(batch, dtype=torch.float32, device="cuda")
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    steps_per_epoch = max(1, n // batch)
    total = epochs * steps_per_epoch
    step = 0
    losses = []
    for ep in range(epochs):
        for b in range(steps_per_epoch):
            rows = mlp_batch(X, Y, seed + 1, ep, b, batch, xb, yb, flag)
            g, loss = mlp_grad(params, xb[:rows], yb[:rows], bf16_forward=True)
            step += 1
            cur = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * step / total))
            mlp_adam(params, g, m, v, step, cur)
        losses.append(float(loss.item()))
        if log:
            log(f"epoch {ep}: loss {losses[-1]:.3e}")
    if int(flag.item()):
        raise RuntimeError("kt_mlp_batch: a permutation walk exceeded its bound")
    return params, losses


def network_targets(X, Y):
    """The cells the network corrects (r^2 > GATE_R2) and their targets z = y / r^2 (kt_mlp_targets)."""
    return mlp_targets(X, Y)


def predict_y(params, X):
    """The correction y of the learned start for feature rows X (tensor-core inference of z), as a
    host array: y = r^2 z where r^2 > GATE_R2, else 0."""
    z = mlp_predict(params, X).cpu().numpy().astype(np.float64)
    r2 = X[:, 1].cpu().numpy().astype(np.float64)
    return np.where(r2 > GATE_R2, r2 * z, 0.0)


def evaluate(params, X, Y):
    """Max and rms error in y of the learned start (tensor-core inference) on (X, Y), on the host."""
    d = predict_y(params, X) - Y.cpu().numpy().astype(np.float64)
    return float(np.max(np.abs(d))), float(np.sqrt(np.mean(d * d)))


def train_default(n=128, seeds=range(2, 12), n_samples=1_000_000, epochs=20, log=None):
    """The network used by the benchmark: trajectories of the n^3 hotspot workload, seeds 2-11."""
    from workload.problem import hotspot_problem
    X, Y = collect(lambda s: hotspot_problem(nx=n, ny=n, neta=n, seed=s), list(seeds), n_samples)
    params, losses = train(*network_targets(X, Y), epochs=epochs, log=log)
    return params, losses, (X, Y)
