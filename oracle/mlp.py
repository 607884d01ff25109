"""FP64 oracle for the learned-radius network -- TEST INFRASTRUCTURE ONLY.

The network (not in the paper; it only proposes search radii, the method
stays exact): 8 input features -> 64 -> 64 -> 64 -> 1, ReLU between layers,
squared-error loss on the normalised log2 of the nearest other-component
weight.  Parameters travel as one flat FP32 vector in this order:

    in_mu[8], in_sigma[8], out_mu, out_sigma, margin, pad,
    W1[64][8], b1[64], W2[64][64], b2[64], W3[64][64], b3[64], w4[64], b4

Features are normalised as (f - in_mu) / in_sigma inside the network.

Everything here is plain numpy in float64 with an explicit backward pass;
``grad_fd`` differentiates the loss numerically (central differences) and is
the check on ``loss_and_grad``.  ``forward_bf16`` models the inference kernel's
rounding (inputs, weights and hidden activations rounded to BF16, sums exact)
so that kernel can be compared tightly.
"""
from __future__ import annotations

import numpy as np

IN, HID = 8, 64
SIZES = [("in_mu", IN), ("in_sigma", IN), ("out_mu", 1), ("out_sigma", 1), ("margin", 1),
         ("pad", 1), ("W1", HID * IN), ("b1", HID), ("W2", HID * HID), ("b2", HID),
         ("W3", HID * HID), ("b3", HID), ("w4", HID), ("b4", 1)]
NPARAM = sum(s for _, s in SIZES)
TRAINABLE_FROM = sum(s for name, s in SIZES[:6])


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, s in SIZES:
        out[name] = p[o:o + s]
        o += s
    out["W1"] = out["W1"].reshape(HID, IN)
    out["W2"] = out["W2"].reshape(HID, HID)
    out["W3"] = out["W3"].reshape(HID, HID)
    return out


def pack(d) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], np.float64).reshape(-1) for name, _ in SIZES])


def init_params(seed: int, in_mu=None, in_sigma=None, out_mu=0.0, out_sigma=1.0, margin=0.0):
    g = np.random.default_rng(seed)
    d = {"in_mu": np.zeros(IN) if in_mu is None else in_mu,
         "in_sigma": np.ones(IN) if in_sigma is None else in_sigma,
         "out_mu": [out_mu], "out_sigma": [out_sigma], "margin": [margin], "pad": [0.0],
         "W1": g.standard_normal((HID, IN)) * np.sqrt(2.0 / IN), "b1": np.zeros(HID),
         "W2": g.standard_normal((HID, HID)) * np.sqrt(2.0 / HID), "b2": np.zeros(HID),
         "W3": g.standard_normal((HID, HID)) * np.sqrt(2.0 / HID), "b3": np.zeros(HID),
         "w4": g.standard_normal(HID) * np.sqrt(1.0 / HID), "b4": [0.0]}
    return pack(d)


def forward(p, feat):
    """Normalised prediction y (before de-normalisation) and the activations."""
    d = unpack(p)
    x = (np.asarray(feat, np.float64) - d["in_mu"]) / d["in_sigma"]
    z1 = x @ d["W1"].T + d["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ d["W2"].T + d["b2"]
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ d["W3"].T + d["b3"]
    h3 = np.maximum(z3, 0.0)
    y = h3 @ d["w4"] + d["b4"][0]
    return y, (x, h1, h2, h3)


def loss(p, feat, target):
    """Mean squared error against the normalised target."""
    d = unpack(p)
    y, _ = forward(p, feat)
    t = (np.asarray(target, np.float64) - d["out_mu"][0]) / d["out_sigma"][0]
    return float(np.mean((y - t) ** 2))


def loss_and_grad(p, feat, target):
    """Loss and its gradient with respect to the flat parameter vector (the
    normalisation entries get zero gradient)."""
    d = unpack(p)
    y, (x, h1, h2, h3) = forward(p, feat)
    t = (np.asarray(target, np.float64) - d["out_mu"][0]) / d["out_sigma"][0]
    m = len(y)
    L = float(np.mean((y - t) ** 2))
    dy = 2.0 * (y - t) / m
    g = {name: np.zeros(s) for name, s in SIZES}
    g["w4"] = h3.T @ dy
    g["b4"] = np.array([dy.sum()])
    dz3 = np.outer(dy, d["w4"]) * (h3 > 0)
    g["W3"] = (dz3.T @ h2).reshape(-1)
    g["b3"] = dz3.sum(0)
    dz2 = (dz3 @ d["W3"]) * (h2 > 0)
    g["W2"] = (dz2.T @ h1).reshape(-1)
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ d["W2"]) * (h1 > 0)
    g["W1"] = (dz1.T @ x).reshape(-1)
    g["b1"] = dz1.sum(0)
    return L, np.concatenate([np.asarray(g[name], np.float64).reshape(-1) for name, _ in SIZES])


def grad_fd(p, feat, target, idx, h=1e-6):
    """Central-difference derivative of the loss for the parameters in idx."""
    p = np.asarray(p, np.float64)
    out = np.zeros(len(idx))
    for k, i in enumerate(idx):
        a = p.copy()
        b = p.copy()
        a[i] += h
        b[i] -= h
        out[k] = (loss(a, feat, target) - loss(b, feat, target)) / (2 * h)
    return out


def bf16(a):
    """Round float64/float32 values to BF16 (nearest, ties to even), returned as float64."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(p, feat):
    """Inference as the tensor-core kernel does it: features normalised in
    FP32 as (f - mu) * (1 / sigma), then they, all weights and each hidden
    activation but the last rounded to BF16; biases and sums in high
    precision.  Returns the predicted log2 weight (de-normalised, plus the
    margin)."""
    d = unpack(p)
    mu32 = np.asarray(d["in_mu"], np.float32)
    inv32 = (np.float32(1.0) / np.asarray(d["in_sigma"], np.float32)).astype(np.float32)
    x = bf16(((np.asarray(feat, np.float32) - mu32).astype(np.float32) * inv32).astype(np.float32))
    h1 = bf16(np.maximum(x @ bf16(d["W1"]).T + d["b1"], 0.0))
    h2 = bf16(np.maximum(h1 @ bf16(d["W2"]).T + d["b2"], 0.0))
    h3 = np.maximum(h2 @ bf16(d["W3"]).T + d["b3"], 0.0)
    y = h3 @ d["w4"] + d["b4"][0]
    return y * d["out_sigma"][0] + d["out_mu"][0] + d["margin"][0]
