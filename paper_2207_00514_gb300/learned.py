"""Training driver of the learned search radius (the arithmetic runs in the
library's CUDA kernels: pair logging, forward + backward, Adam, inference).

    params = train(seeds=range(100, 132), n=1_000_000)   # on the GPU
    save(params, path); params = load(path)
    emst_compute_ex(points, mlp_params=params)           # same tree, other cutoffs

Parameter vector layout: see include/emst.h (EMST_MLP_PARAMS floats).
"""
from __future__ import annotations

import os

import numpy as np

from . import (EMST_MLP_FEATURES, EMST_MLP_PARAMS, emst_learned_samples, emst_mlp_adam,
               emst_mlp_forward, emst_mlp_grad)

HID = 64
_OFF_W1 = 20
MODEL_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "models")
DEFAULT_MODEL = os.path.join(MODEL_DIR, "learned_radius_halos3d.npy")


def initial_params(seed: int, in_mu, in_sigma, out_mu: float, out_sigma: float) -> np.ndarray:
    """He-initialised network with the given normalisation (zero biases)."""
    g = np.random.default_rng(seed)
    parts = [np.asarray(in_mu, np.float64), np.asarray(in_sigma, np.float64),
             [out_mu, out_sigma, 0.0, 0.0],
             g.standard_normal(HID * EMST_MLP_FEATURES) * np.sqrt(2.0 / EMST_MLP_FEATURES), np.zeros(HID),
             g.standard_normal(HID * HID) * np.sqrt(2.0 / HID), np.zeros(HID),
             g.standard_normal(HID * HID) * np.sqrt(2.0 / HID), np.zeros(HID),
             g.standard_normal(HID) * np.sqrt(1.0 / HID), [0.0]]
    p = np.concatenate([np.asarray(x, np.float64).reshape(-1) for x in parts]).astype(np.float32)
    assert p.size == EMST_MLP_PARAMS
    return p


def collect(point_sets, every: int = 8, capacity_per_set: int = 400_000):
    """Training pairs from plain runs on each point set (device tensors)."""
    import torch
    feats, targs = [], []
    for pts in point_sets:
        t = torch.from_numpy(np.ascontiguousarray(pts, np.float32)).cuda()
        f, y = emst_learned_samples(t, every, capacity_per_set)
        feats.append(f.clone())
        targs.append(y.clone())
    return torch.cat(feats), torch.cat(targs)


def fit(features, targets, epochs: int = 6, batch: int = 4096, lr: float = 2e-3, seed: int = 0,
        coverage: float = 0.95, log=None):
    """Train on (features, targets) with the library's kernels; returns the
    parameter tensor (device) with the margin set so that `coverage` of a
    held-out tenth is predicted at or above its target."""
    import torch
    dev = features.device
    m = features.shape[0]
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    order = torch.randperm(m, device=dev, generator=g)
    hold = order[: m // 10]
    train_idx = order[m // 10:]
    ftr, ttr = features[train_idx], targets[train_idx]
    mu = ftr.mean(0).double().cpu().numpy()
    sd = ftr.std(0).clamp_min(1e-3).double().cpu().numpy()
    p = torch.from_numpy(initial_params(seed, mu, sd, float(ttr.mean()), float(ttr.std().clamp_min(1e-3)))).to(dev)
    grad = torch.zeros(EMST_MLP_PARAMS, dtype=torch.float32, device=dev)
    m1 = torch.zeros_like(grad)
    m2 = torch.zeros_like(grad)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    step = 0
    history = []
    nt = ftr.shape[0]
    for ep in range(epochs):
        perm = torch.randperm(nt, device=dev, generator=g)
        fe, te = ftr[perm].contiguous(), ttr[perm].contiguous()
        loss.zero_()
        nb = 0
        for s in range(0, nt - batch + 1, batch):
            emst_mlp_grad(fe[s:s + batch], te[s:s + batch], p, grad, loss)
            step += 1
            emst_mlp_adam(p, grad, m1, m2, step, lr * (0.5 ** (ep // 2)))
            nb += 1
        history.append(float(loss.item()) / max(nb, 1))
        if log:
            log(f"epoch {ep}: mean batch loss {history[-1]:.4f}")
    # margin: the `coverage` quantile of (target - prediction) on held-out pairs
    pred = emst_mlp_forward(features[hold].contiguous(), p)
    resid = (targets[hold] - pred).double().cpu().numpy()
    p[18] = float(np.quantile(resid, coverage))
    return p, history


def train(seeds=range(100, 132), n: int = 1_000_000, every: int = 8, epochs: int = 6, log=None):
    """The recipe: pairs from plain runs on the 3D halo generator at n points
    for each seed, then fit."""
    import synth
    feats, targs = collect((synth.halos(n, s) for s in seeds), every=every)
    if log:
        log(f"{feats.shape[0]} training pairs")
    return fit(feats, targs, epochs=epochs, log=log)


def save(params, path: str = DEFAULT_MODEL) -> str:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.save(path, params.detach().cpu().numpy().astype(np.float32))
    return path


def load(path: str = DEFAULT_MODEL, device="cuda"):
    import torch
    a = np.load(path).astype(np.float32)
    if a.size != EMST_MLP_PARAMS:
        raise ValueError(f"{path}: expected {EMST_MLP_PARAMS} parameters")
    return torch.from_numpy(a).to(device)
