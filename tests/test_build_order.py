"""The one-pass build's order of work, modelled on the CPU, against the oracle.

The GPU builds Karras's radix tree (Fig. 4 numbering) from the leaves up: a
node covering chunks [l, r] hangs under the split r (as the left child) when
the keys of chunks r and r + 1 share more leading bits than those of l - 1
and l, else under the split l - 1 (as the right child); so a left child's
index is its right end and a right child's its left end.  Splits between two
chunks of one CTA meet in shared memory; a split at a CTA's edge is met in
global memory and, once both children are there, listed for a second launch;
a split inside a CTA that only one child reached hands that child's far end
to the second launch.  This test runs that protocol sequentially, threads in
random order (any order is a valid interleaving: each split has exactly two
arrivals and the first one stops), over random, heavily duplicated and
skewed keys and several CTA sizes, and checks every node's range and
children against the oracle's radix tree, and that fewer splits are listed
than there are CTAs.
"""
from __future__ import annotations

import random

import numpy as np
import pytest

import oracle


def _delta(keys, nc, i, j):
    """Leading bits shared by the augmented keys (code, index) of chunks i, j."""
    if i < 0 or j < 0 or i >= nc or j >= nc:
        return -1
    a, b = int(keys[i]), int(keys[j])
    if a != b:
        return 64 - (a ^ b).bit_length()
    return 64 + 32 - (i ^ j).bit_length()


def _parent(l, r, nc, keys):
    if l == 0 and r == nc - 1:
        return None
    dl, dr = _delta(keys, nc, l - 1, l), _delta(keys, nc, r, r + 1)
    left = l == 0 or (r != nc - 1 and dr > dl)
    return (r, 0) if left else (l - 1, 1)


def _model(keys, cta, rng):
    nc = len(keys)
    nodes = {}
    far = [[None, None] for _ in range(nc - 1)]
    arrivals = [0] * (nc - 1)
    ready = []

    def write(L, g, R, up):
        idx = 0 if up is None else (R if up[1] == 0 else L)
        assert idx not in nodes, "a node written twice"
        nodes[idx] = (L, g, R)

    for first in range(0, nc, cta):
        last = min(first + cta - 1, nc - 1)
        s_far, s_arr = {}, {}
        order = list(range(first, last + 1))
        rng.shuffle(order)
        for k in order:
            l = r = k
            up = _parent(l, r, nc, keys)
            while up is not None:
                ps, side = up
                f = l if side == 0 else r
                if ps < first or ps >= last:  # a split at the CTA's edge
                    assert far[ps][side] is None
                    far[ps][side] = f
                    arrivals[ps] += 1
                    if arrivals[ps] == 2:
                        ready.append(ps)
                    break
                s_far.setdefault(ps, [None, None])[side] = f
                s_arr[ps] = s_arr.get(ps, 0) + 1
                if s_arr[ps] == 1:
                    break
                sib = s_far[ps][side ^ 1]
                L, R = (l, sib) if side == 0 else (sib, r)
                assert first <= L <= ps < R <= last
                up2 = _parent(L, R, nc, keys)
                write(L, ps, R, up2)
                l, r, up = L, R, up2
        for s in range(first, last):  # one child arrived: hand its far end on
            if s_arr.get(s, 0) == 1:
                side = 0 if s_far[s][0] is not None else 1
                far[s][side] = s_far[s][side]
                arrivals[s] = 1
    assert len(ready) < (nc + cta - 1) // cta or len(ready) == 0
    rng.shuffle(ready)
    for ps in ready:
        L, R = far[ps]
        assert L <= ps < R
        while True:
            up = _parent(L, R, nc, keys)
            write(L, ps, R, up)
            if up is None:
                break
            ps, side = up
            far[ps][side] = L if side == 0 else R
            arrivals[ps] += 1
            if arrivals[ps] == 1:
                break
            sib = far[ps][side ^ 1]
            if side == 0:
                R = sib
            else:
                L = sib
    return nodes


@pytest.mark.parametrize("cta", [1, 2, 3, 8, 128])
@pytest.mark.parametrize("kind", ["random", "duplicates", "skewed"])
def test_bottom_up_build_gives_the_karras_tree(cta, kind):
    rng = random.Random(cta * 7 + len(kind))
    g = np.random.default_rng(cta * 13 + len(kind))
    for _ in range(3):
        n = int(g.integers(2, 700))
        if kind == "random":
            keys = np.sort(g.integers(0, 2**63, n, dtype=np.uint64))
        elif kind == "duplicates":
            keys = np.sort(g.integers(0, 20, n).astype(np.uint64))
        else:  # gaps that grow along the curve: a deep, lopsided tree
            keys = np.sort((np.cumsum(g.integers(1, 4, n)) ** 3).astype(np.uint64))
        nodes = _model(keys, cta, rng)
        left, right, first, last = oracle.radix_tree(keys)
        assert len(nodes) == n - 1
        for idx in range(n - 1):
            L, s, R = nodes[idx]
            assert (first[idx], last[idx]) == (L, R)
            assert left[idx] == (n - 1 + s if L == s else s)
            assert right[idx] == (n - 1 + s + 1 if R == s + 1 else s + 1)
