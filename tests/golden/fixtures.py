"""Reader for the small text fixtures in this folder (``key: values`` lines,
``#`` comments carry each fixture's citation and derivation)."""
from __future__ import annotations

import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def load(name: str) -> dict:
    out = {}
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(":", 1)
            out[k.strip()] = v.split()
    return out


def floats(tokens, dim=None):
    a = np.array([float(t) for t in tokens], dtype=np.float32)
    return a.reshape(-1, dim) if dim else a


def ints(tokens, dtype=np.int64):
    return np.array([int(t) for t in tokens], dtype=dtype)


def edges(tokens):
    t = list(tokens)
    return [(int(t[k]), int(t[k + 1]), np.float32(float(t[k + 2]))) for k in range(0, len(t), 3)]
