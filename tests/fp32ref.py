"""Independent FP32 arithmetic for the tests (not used by the oracle or the product).

``fma32(a, b, c)`` returns the correctly rounded FP32 value of a*b + c for FP32
inputs, vectorised in numpy: the product of two FP32 numbers is exact in FP64,
TwoSum gives the FP64 sum plus its exact error, and a sum that lands exactly on
an FP32 rounding midpoint is nudged by the sign of the error (the only case in
which rounding FP64 -> FP32 can differ from rounding the exact value).
``exact_fma32`` does the same with Python fractions and is the check on it.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def _round_f64_to_f32(s: np.ndarray, e: np.ndarray) -> np.ndarray:
    r = s.astype(np.float32)
    rd = r.astype(np.float64)
    up = np.nextafter(r, np.float32(np.inf)).astype(np.float64)
    dn = np.nextafter(r, np.float32(-np.inf)).astype(np.float64)
    nb = np.where(s > rd, up, dn)
    mid = (rd + nb) * 0.5
    on_mid = (s != rd) & (s == mid) & (e != 0)
    hi = np.maximum(rd, nb)
    lo = np.minimum(rd, nb)
    fixed = np.where(e > 0, hi, lo).astype(np.float32)
    return np.where(on_mid, fixed, r)


def fma32(a, b, c) -> np.ndarray:
    a = np.asarray(a, np.float32).astype(np.float64)
    b = np.asarray(b, np.float32).astype(np.float64)
    c = np.asarray(c, np.float32).astype(np.float64)
    p = a * b  # exact: 24 + 24 significant bits
    s = p + c
    bp = s - p
    e = (p - (s - bp)) + (c - bp)  # TwoSum error: s + e == p + c exactly
    return _round_f64_to_f32(s, e)


def mul32(a, b) -> np.ndarray:
    a = np.asarray(a, np.float32)
    b = np.asarray(b, np.float32)
    return (a * b).astype(np.float32)


def weight32(p, q) -> np.ndarray:
    """FP32 squared distance in the order fma(dz,dz, fma(dy,dy, dx*dx))."""
    p = np.asarray(p, np.float32)
    q = np.asarray(q, np.float32)
    d = (p - q).astype(np.float32)
    s = mul32(d[..., 0], d[..., 0])
    s = fma32(d[..., 1], d[..., 1], s)
    if p.shape[-1] == 3:
        s = fma32(d[..., 2], d[..., 2], s)
    return s


def exact_round32(x: Fraction) -> np.float32:
    """Round a rational to the nearest FP32 (ties to even), no double rounding."""
    f = np.float32(float(x))
    cands = {f, np.nextafter(f, np.float32(np.inf)), np.nextafter(f, np.float32(-np.inf))}
    best = None
    for c in cands:
        d = abs(Fraction(float(c)) - x)
        key = (d, int(np.frombuffer(np.float32(c).tobytes(), np.uint32)[0]) & 1)
        if best is None or key < best[0]:
            best = (key, c)
    return np.float32(best[1])


def exact_fma32(a, b, c) -> np.float32:
    return exact_round32(Fraction(float(np.float32(a))) * Fraction(float(np.float32(b)))
                         + Fraction(float(np.float32(c))))


def exact_weight32(p, q) -> np.float32:
    p = [np.float32(x) for x in p]
    q = [np.float32(x) for x in q]
    d = [exact_round32(Fraction(float(a)) - Fraction(float(b))) for a, b in zip(p, q)]
    s = exact_round32(Fraction(float(d[0])) ** 2)
    s = exact_fma32(d[1], d[1], s)
    if len(p) == 3:
        s = exact_fma32(d[2], d[2], s)
    return s


def pairwise_weights(pts: np.ndarray) -> np.ndarray:
    """Dense n x n FP32 weight matrix (tests only, small n)."""
    p = np.asarray(pts, np.float32)
    return weight32(p[:, None, :], p[None, :, :])
