"""The search's lower bound for the next round, modelled on the CPU.

From the second round after the first on, a search that finds nothing
within its cutoff r0 leaves as the point's lower bound the smallest weight
bound (box distance) of the children of other components it rejected by
distance, instead of r0 itself; the next round skips the point when that
bound exceeds its component's cutoff.  That is exact only if the bound never
exceeds the point's true nearest other-component weight: every point of
another component lies in a child the search rejected by distance, or in a
leaf it saw.  This test runs the search of Algorithm 2 as the GPU does it
(nearer child first; a child of the query's own component skipped; a child
within the cutoff accepted, inclusive; a leaf taken and the cutoff shrunk)
over the oracle's hierarchy of seeded point sets with several labellings and
cutoffs, and checks against brute force that a found neighbour is the
nearest one and that an empty search's bound lies above r0 and at or below
the true nearest other-component weight.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth


def _tree(pts):
    lo, hi, _ = oracle.scene_box(pts)
    perm = oracle.sort_perm(oracle.morton(pts, lo, hi))
    sp = pts[perm].astype(np.float64)
    left, right, first, last = oracle.radix_tree(oracle.morton(pts, lo, hi)[perm])
    blo, bhi = oracle.node_boxes(pts[perm], first, last)
    return sp, left, right, first, last, blo.astype(np.float64), bhi.astype(np.float64)


def _box_d2(q, lo, hi):
    c = np.minimum(np.maximum(q, lo), hi)
    return float(((q - c) ** 2).sum())


def _search(q, i, me, r0, labels, nlab, sp, left, right, blo, bhi):
    """Returns (found weight or None, the bound an empty search leaves)."""
    n = len(sp)
    radius, best = r0, None
    rejected = np.inf
    stack = []
    node = 0
    while True:
        kids = []
        for ref in (left[node], right[node]):
            if ref >= n - 1:  # leaf: one point
                k = ref - (n - 1)
                lab = labels[k]
                d = float(((q - sp[k]) ** 2).sum())
                kids.append((d, lab, True, k))
            else:
                kids.append((_box_d2(q, blo[ref], bhi[ref]), nlab[ref], False, ref))
        nxt = []
        for d, lab, leaf, ref in kids:
            if lab == me:
                continue
            if d > radius:
                rejected = min(rejected, d)
                continue
            if leaf:
                if best is None or d < best:
                    best, radius = d, d
            else:
                nxt.append((d, ref))
        nxt = [(d, ref) for d, ref in nxt if d <= radius]
        nxt.sort()
        if len(nxt) == 2:
            stack.append(nxt[1])
        if nxt:
            node = nxt[0][1]
            continue
        node = None
        while stack:
            d, ref = stack.pop()
            if d <= radius:
                node = ref
                break
        if node is None:
            break
    if best is not None:
        return best, best
    return None, (rejected if np.isfinite(rejected) else r0)


@pytest.mark.parametrize("kind", ["halos3", "blobs2"])
@pytest.mark.parametrize("labelling", ["runs", "random"])
def test_empty_search_bound_is_a_lower_bound(kind, labelling):
    g = np.random.default_rng(len(kind) * 10 + len(labelling))
    pts = synth.halos(1500, 9) if kind == "halos3" else synth.blobs(1500, 2, 9)
    sp, left, right, first, last, blo, bhi = _tree(pts)
    n = len(sp)
    if labelling == "runs":  # components as runs of curve positions, as Boruvka makes them early
        cuts = np.sort(g.choice(np.arange(1, n), size=40, replace=False))
        labels = np.zeros(n, np.int64)
        labels[cuts] = 1
        labels = np.cumsum(labels)
    else:
        labels = g.integers(0, 25, n)
    nlab = oracle.node_labels(labels.astype(np.uint32), first, last).astype(np.int64)
    nlab[nlab == 0xFFFFFFFF] = -1
    empty = 0
    for i in g.choice(n, size=300, replace=False):
        q = sp[i]
        d2 = ((sp - q) ** 2).sum(1)
        other = labels != labels[i]
        true = float(d2[other].min())
        for factor in (0.25, 0.9, 1.0, 3.0):
            r0 = true * factor
            found, lb = _search(q, i, labels[i], r0, labels, nlab, sp, left, right, blo, bhi)
            if true <= r0:
                assert found == true
            else:
                assert found is None
                assert r0 < lb <= true
                empty += 1
    assert empty > 0
