"""Surrogate-assisted design screening.

1. Label voxel designs with the batched simulator (locomotion = centre-of-mass
   x-travel after a rollout).
2. Train the MLP surrogate on (one-hot materials -> travel) with the
   tensor-core kernels.
3. Screen a large candidate population with the surrogate, and re-simulate
   the best fraction with the simulator, which has the final word.

Everything numerical runs in the library (Population, Surrogate); this
module only orchestrates batches.
"""
from __future__ import annotations

import numpy as np

from .batch import Population
from .surrogate import Surrogate

__all__ = ["phase_field", "simulate_travel", "train", "screen", "top_indices", "r2"]


def phase_field(side: int = 8):
    """The fixed travelling-wave actuation phase phi(x) = 2 pi x / side shared
    by every surrogate design (so the label is a function of the materials)."""
    xs = (2 * np.pi * np.arange(side) / side).astype(np.float32)
    return np.broadcast_to(xs[None, None, :], (side, side, side)).copy()


def simulate_travel(materials, material_table, freq, voxel_edge, voxel_mass, params, nsteps,
                    chunk: int = 4096, autotune: bool = True):
    """x-travel of every design [N, side, side, side] after nsteps, batched."""
    mats = np.asarray(materials, np.uint8)
    side = mats.shape[-1]
    ph = phase_field(side)
    out = np.empty(len(mats), np.float32)
    for s in range(0, len(mats), chunk):
        part = mats[s:s + chunk]
        designs = [(m, ph) for m in part]
        with Population(designs, material_table, freq, voxel_edge, voxel_mass, params) as pop:
            if autotune:
                pop.autotune(sample_steps=50)
            pop.run(nsteps)
            out[s:s + len(part)] = pop.com_travel()
    return out


def r2(pred, target):
    pred = np.asarray(pred, np.float64); target = np.asarray(target, np.float64)
    ss_res = np.sum((pred - target) ** 2)
    ss_tot = np.sum((target - target.mean()) ** 2)
    return 1.0 - ss_res / ss_tot


def train(materials, labels, epochs: int = 20, batch: int = 1024, lr: float = 1e-3, seed: int = 0,
          hidden: int = 512, net: Surrogate | None = None):
    """Train (or continue training) a surrogate on standardised labels.
    Returns (net, mean, std) with prediction = mean + std * net output."""
    import torch
    mats = np.asarray(materials, np.uint8).reshape(len(materials), -1)
    y = np.asarray(labels, np.float64)
    mu, sd = float(y.mean()), float(y.std() or 1.0)
    yt = ((y - mu) / sd).astype(np.float32)
    n = (len(mats) // batch) * batch
    if n == 0:
        raise ValueError("need at least one full batch of designs")
    dm = torch.tensor(mats, device="cuda")
    dy = torch.tensor(yt, device="cuda")
    # the model's buffers also serve screening, which runs forward passes of
    # 65536 designs (fewer, fuller waves of GEMM tiles than smaller passes)
    net = net or Surrogate(mats.shape[1] * 4, hidden, max_batch=max(batch, 65536), seed=seed)
    rng = np.random.default_rng(seed)
    for _ in range(epochs):
        perm = torch.tensor(rng.permutation(len(mats))[:n], device="cuda")
        for s in range(0, n, batch):
            idx = perm[s:s + batch]
            net.train_step(dm[idx].contiguous(), dy[idx].contiguous(), lr=lr)
    net.sync()
    return net, mu, sd


def predict(net: Surrogate, materials, mu: float, sd: float):
    import torch
    mats = np.asarray(materials, np.uint8).reshape(len(materials), -1)
    n = len(mats)
    pad = (-n) % 128
    if pad:
        mats = np.concatenate([mats, np.zeros((pad, mats.shape[1]), np.uint8)])
    dm = torch.tensor(mats, device="cuda")
    out = net.predict(dm).cpu().numpy()[:n]
    return mu + sd * out


def top_indices(pred, top_frac: float):
    """Indices of the top_frac (at least one) largest entries of pred, largest first."""
    pred = np.asarray(pred)
    k = max(1, int(round(top_frac * len(pred))))
    top = np.argpartition(-pred, k - 1)[:k]
    return top[np.argsort(-pred[top], kind="stable")]


def screen(net: Surrogate, candidates, mu: float, sd: float, top_frac: float = 0.01):
    """Indices of the top_frac candidates by predicted travel, best first."""
    pred = predict(net, candidates, mu, sd)
    return top_indices(pred, top_frac), pred
