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

from .binding import KT, KT_MIXED, MLP_NPARAM, mlp_adam, mlp_grad, mlp_predict

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
    """Sample n_samples cells uniformly over the snapshots of the given seeds' trajectories."""
    import torch
    snaps = len(seeds) * (steps // every)
    per = int(math.ceil(n_samples / snaps))
    rng = np.random.default_rng(sample_seed)
    xs, ys, es = [], [], []
    for seed in seeds:
        prob = problem_factory(seed)
        kt = KT(prob, precision=KT_MIXED)
        kt.set_problem_state()
        for _ in range(steps // every):
            kt.step(every)
            cells = torch.as_tensor(rng.integers(0, prob.ncells, per), device="cuda")
            x, y, e = kt.mlp_features(cells)
            xs.append(x)
            ys.append(y)
            es.append(e)
        del kt
    X, Y = torch.cat(xs)[:n_samples], torch.cat(ys)[:n_samples]
    return X.contiguous(), Y.contiguous()


def train(X, Y, epochs=20, batch=8192, lr=3e-3, lr_min=1e-4, seed=0, log=None):
    """Adam with cosine learning-rate decay; returns float32 CUDA parameters and the loss log."""
    import torch
    params = torch.as_tensor(init_params(seed), device="cuda")
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    n = X.shape[0]
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    steps_per_epoch = max(1, n // batch)
    total = epochs * steps_per_epoch
    step = 0
    losses = []
    for ep in range(epochs):
        perm = torch.randperm(n, device="cuda", generator=gen)
        for b in range(steps_per_epoch):
            idx = perm[b * batch:(b + 1) * batch]
            xb, yb = X[idx].contiguous(), Y[idx].contiguous()
            g, loss = mlp_grad(params, xb, yb, bf16_forward=True)
            step += 1
            cur = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * step / total))
            mlp_adam(params, g, m, v, step, cur)
        losses.append(float(loss.item()))
        if log:
            log(f"epoch {ep}: loss {losses[-1]:.3e}")
    return params, losses


def network_targets(X, Y):
    """The cells the network corrects (r^2 > GATE_R2) and their targets z = y / r^2."""
    r2 = X[:, 1]
    keep = r2 > GATE_R2
    return X[keep].contiguous(), (Y[keep] / r2[keep]).contiguous()


def predict_y(params, X):
    """The correction y of the learned start for feature rows X (tensor-core inference of z)."""
    r2 = X[:, 1]
    return (mlp_predict(params, X) * r2) * (r2 > GATE_R2)


def evaluate(params, X, Y):
    """Max and rms error in y of the learned start (tensor-core inference) on (X, Y)."""
    d = (predict_y(params, X) - Y).double()
    return float(d.abs().max().item()), float(d.pow(2).mean().sqrt().item())


def train_default(n=128, seeds=range(2, 12), n_samples=1_000_000, epochs=20, log=None):
    """The network used by the benchmark: trajectories of the n^3 hotspot workload, seeds 2-11."""
    from workload.problem import hotspot_problem
    X, Y = collect(lambda s: hotspot_problem(nx=n, ny=n, neta=n, seed=s), list(seeds), n_samples)
    params, losses = train(*network_targets(X, Y), epochs=epochs, log=log)
    return params, losses, (X, Y)
