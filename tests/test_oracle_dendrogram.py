"""Pins of the oracle's single-linkage dendrogram (oracle_dendrogram) against
things other than itself: hand-derived hierarchies, scipy's single linkage
of the same points, a brute-force divisive reading of the definition (the
cluster of edge k is the component of the edges ranked <= k that holds it),
and the cophenetic property (two points join at the largest weight on their
tree path)."""
from __future__ import annotations

import collections

import numpy as np
import pytest

import oracle
import synth

INV = 0xFFFFFFFF


def rows(link):
    return [(int(r["a"]), int(r["b"]), float(r["w"]), int(r["size"])) for r in link]


def test_hand_line():
    # points at 0, 1, 3, 6, 10: each gap is larger than the one before, so
    # every merge adds the next point to the one growing cluster
    pts = np.array([[0, 0], [1, 0], [3, 0], [6, 0], [10, 0]], np.float32)
    link, parent = oracle.dendrogram(oracle.prim(pts), 5)
    assert rows(link) == [(0, 1, 1.0, 2), (2, 5, 4.0, 3), (3, 6, 9.0, 4), (4, 7, 16.0, 5)]
    assert list(parent) == [5, 5, 6, 7, 8, 6, 7, 8, INV]


def test_hand_two_pairs():
    # two tight pairs {0,1} and {2,3} joined at 25, then the far point 4
    pts = np.array([[0, 0], [0, 1], [5, 0], [5, 2], [20, 0]], np.float32)
    link, parent = oracle.dendrogram(oracle.prim(pts), 5)
    assert rows(link) == [(0, 1, 1.0, 2), (2, 3, 4.0, 2), (5, 6, 25.0, 4), (4, 7, 225.0, 5)]
    assert list(parent) == [5, 5, 6, 6, 8, 7, 7, 8, INV]


def test_trivial_sizes():
    link, parent = oracle.dendrogram(np.zeros(0, oracle.EDGE_DTYPE), 1)
    assert len(link) == 0 and list(parent) == [INV]
    e = np.array([(0, 1, 2.5)], oracle.EDGE_DTYPE)
    link, parent = oracle.dendrogram(e, 2)
    assert rows(link) == [(0, 1, 2.5, 2)] and list(parent) == [2, 2, INV]


@pytest.mark.parametrize("dim,seed", [(2, 3), (3, 4), (3, 5)])
def test_matches_scipy_single_linkage(dim, seed):
    hier = pytest.importorskip("scipy.cluster.hierarchy")
    pts = synth.uniform(400, dim, seed)
    tree = oracle.prim(pts)
    # the pin is valid only where FP32 squared and FP64 Euclidean weights
    # order the tree's edges the same way (no near-ties)
    p64 = pts.astype(np.float64)
    d64 = np.linalg.norm(p64[tree["i"]] - p64[tree["j"]], axis=1)
    assert np.all(np.diff(d64) > 0)
    link, _ = oracle.dendrogram(tree, len(pts))
    Z = hier.linkage(p64, method="single")
    assert np.array_equal(link["a"], Z[:, 0].astype(np.uint32))
    assert np.array_equal(link["b"], Z[:, 1].astype(np.uint32))
    assert np.array_equal(link["size"], Z[:, 3].astype(np.uint32))
    np.testing.assert_allclose(np.sqrt(link["w"].astype(np.float64)), Z[:, 2], rtol=2e-7)


def divisive(edges, n):
    """The hierarchy read straight off the definition, no union-find: the
    cluster of edge k is the vertex set of the component of edges 0..k that
    holds edge k; its children are the components of edges 0..k-1 at its two
    ends; each point hangs under its lowest-ranked edge."""
    m = n - 1

    def component(v, upto):
        adj = collections.defaultdict(list)
        for r in range(upto):
            adj[int(edges[r]["i"])].append((int(edges[r]["j"]), r))
            adj[int(edges[r]["j"])].append((int(edges[r]["i"]), r))
        seen, top, stack = {v}, -1, [v]
        while stack:
            x = stack.pop()
            for y, r in adj[x]:
                top = max(top, r)
                if y not in seen:
                    seen.add(y)
                    stack.append(y)
        return seen, top

    link, parent = [], [INV] * (2 * n - 1)
    for k in range(m):
        i, j = int(edges[k]["i"]), int(edges[k]["j"])
        kids = []
        for v in (i, j):
            _, top = component(v, k)
            kids.append(v if top < 0 else n + top)
        verts, _ = component(i, k + 1)
        link.append((min(kids), max(kids), float(edges[k]["w"]), len(verts)))
        for c in kids:
            parent[c] = n + k
    return link, parent


@pytest.mark.parametrize("shape", synth.TREE_SHAPES)
@pytest.mark.parametrize("ties", [0, 4])
def test_matches_divisive_definition(shape, ties):
    for seed in range(3):
        n = 60 + 7 * seed
        e = synth.tree_edges(n, seed, shape, ties=ties)
        link, parent = oracle.dendrogram(e, n)
        want_link, want_parent = divisive(e, n)
        assert rows(link) == want_link, (shape, ties, seed)
        assert list(parent) == want_parent, (shape, ties, seed)


def test_cophenetic_is_minimax_path_weight():
    pts = synth.blobs(150, 2, 6)
    tree = oracle.prim(pts)
    n = len(pts)
    link, parent = oracle.dendrogram(tree, n)
    adj = collections.defaultdict(list)
    for e in tree:
        adj[int(e["i"])].append((int(e["j"]), e["w"]))
        adj[int(e["j"])].append((int(e["i"]), e["w"]))

    def ancestors(v):
        out = []
        while v != INV:
            out.append(v)
            v = int(parent[v])
        return out

    anc = [ancestors(v) for v in range(n)]
    for u in range(0, n, 7):
        # largest weight on the tree path from u to every v
        best = {u: np.float32(0)}
        stack = [u]
        while stack:
            x = stack.pop()
            for y, w in adj[x]:
                if y not in best:
                    best[y] = max(best[x], w)
                    stack.append(y)
        au = set(anc[u])
        for v in range(n):
            if v == u:
                continue
            lca = next(c for c in anc[v] if c in au)
            assert link[lca - n]["w"] == best[v], (u, v)


def test_invalid_inputs():
    e = synth.tree_edges(50, 1, "random")
    bad = e.copy()
    bad[10]["j"] = 50  # id out of range
    with pytest.raises(ValueError):
        oracle.dendrogram(bad, 50)
    bad = e.copy()
    bad[[3, 30]] = bad[[30, 3]]  # weights out of order
    with pytest.raises(ValueError):
        oracle.dendrogram(bad, 50)
    bad = e.copy()
    bad[20]["i"], bad[20]["j"] = bad[19]["i"], bad[19]["j"]  # a repeated edge closes a cycle
    bad[20]["w"] = bad[19]["w"]
    with pytest.raises(ValueError):
        oracle.dendrogram(bad, 50)
    bad = e.copy()
    bad[0]["w"] = np.nan
    with pytest.raises(ValueError):
        oracle.dendrogram(bad, 50)


@pytest.mark.parametrize("shape", synth.TREE_SHAPES)
def test_tree_generator_gives_spanning_trees_in_merge_order(shape):
    for n, ties in ((1, 0), (2, 0), (257, 0), (1000, 3)):
        e = synth.tree_edges(n, n + ties, shape, ties=ties)
        assert len(e) == max(n - 1, 0)
        if n < 2:
            continue
        assert np.all(e["i"] < e["j"]) and np.all(e["j"] < n)
        assert np.all(np.diff(e["w"].astype(np.float64)) >= 0)
        comps, cycle = oracle.count_components(e, n)
        assert comps == 1 and not cycle
    # the deep case: along the path the weights rise, so every merge adds one point
    e = synth.tree_edges(300, 5, "path_sorted")
    link, _ = oracle.dendrogram(e, 300)
    assert list(link["size"]) == list(range(2, 301))
