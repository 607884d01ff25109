"""Pins of the mutual-reachability oracle (§4.5): core distances and the
mutual-reachability MST, checked against facts other than the oracle itself."""
import numpy as np
import pytest

import oracle
import synth
from fp32ref import pairwise_weights


def _core_from_weights(W, k):
    """k-th nearest neighbour counting the point itself: the (k-1)-th smallest
    off-diagonal weight of each row (numpy partition on independent weights)."""
    n = len(W)
    if k == 1:
        return np.zeros(n, np.float32)
    off = W + np.diag(np.full(n, np.inf, np.float32))
    return np.partition(off, k - 2, axis=1)[:, k - 2]


@pytest.mark.parametrize("k", [1, 2, 3, 8, 16])
def test_core_distance_definition(k):
    p = synth.blobs(400, 3, 7)
    W = pairwise_weights(p)
    got = oracle.core_dist2(p, k, brute=True)
    assert np.array_equal(got, _core_from_weights(W, k))
    # the value is one of the row's weights, with at most k-2 others strictly
    # below it and at least k-1 at or below it
    off = W + np.diag(np.full(len(p), np.inf, np.float32))
    if k > 1:
        below = (off < got[:, None]).sum(1)
        at_or_below = (off <= got[:, None]).sum(1)
        assert np.all(below <= k - 2) and np.all(at_or_below >= k - 1)
    else:
        assert np.all(got == 0)


def test_core_k2_is_nearest_other_point():
    p = synth.uniform(500, 2, 3)
    ids = np.arange(len(p), dtype=np.uint32)
    w, j = oracle.nn_other(p, ids, ids, np.full(len(p), np.inf, np.float32))
    assert np.array_equal(oracle.core_dist2(p, 2, brute=True), w)


@pytest.mark.parametrize("gen", ["blobs", "lattice"])
def test_kd_core_equals_full_selection(gen):
    if gen == "blobs":
        p = synth.blobs(5000, 3, 2)
    else:  # many equal weights and duplicates
        g = np.random.default_rng(4)
        p = (g.integers(0, 12, size=(4000, 3)) / 12.0).astype(np.float32)
    for k in (1, 2, 5, 16):
        assert np.array_equal(oracle.core_dist2(p, k, threads=4), oracle.core_dist2(p, k, brute=True))


def test_mrd_hand_case_changes_the_tree():
    # 1D points 0, 1, 3 with k = 3: every core distance is the farther of the
    # two others (9, 4, 9), so all three weights are 9 and the id order picks
    # (0,1), (0,2) -- the Euclidean tree is (0,1), (1,2)
    p = np.array([[0, 0], [1, 0], [3, 0]], np.float32)
    c = oracle.core_dist2(p, 3, brute=True)
    assert list(c) == [9, 4, 9]
    e = oracle.prim_mrd(p, c)
    assert [(int(a), int(b), float(w)) for a, b, w in e] == [(0, 1, 9.0), (0, 2, 9.0)]
    assert [(int(a), int(b)) for a, b, _ in oracle.prim(p)] == [(0, 1), (1, 2)]


def test_mrd_k1_is_the_emst():
    p = synth.blobs(2000, 3, 9)
    c = oracle.core_dist2(p, 1)
    assert np.array_equal(oracle.prim_mrd(p, c), oracle.prim(p))
    assert np.array_equal(oracle.kd_boruvka_mrd(p, c, threads=2), oracle.kd_boruvka(p, threads=2))


def _tree_path_max(n, edges, keys):
    adj = [[] for _ in range(n)]
    for (a, b), key in zip(edges, keys):
        adj[a].append((b, key))
        adj[b].append((a, key))
    best = {}
    for s in range(n):  # max key on the path from s to every vertex
        mx = {s: None}
        stack = [s]
        while stack:
            u = stack.pop()
            for v, key in adj[u]:
                if v not in mx:
                    mx[v] = key if mx[u] is None or key > mx[u] else mx[u]
                    stack.append(v)
        best[s] = mx
    return best


@pytest.mark.parametrize("k", [2, 4])
def test_mrd_cycle_property_brute_force(k):
    p = synth.blobs(120, 2, 11)
    n = len(p)
    W = pairwise_weights(p)
    c = _core_from_weights(W, k)
    M = np.maximum(np.maximum(W, c[:, None]), c[None, :])
    e = oracle.prim_mrd(p, c)
    assert len(e) == n - 1
    tree = [(int(a), int(b)) for a, b, _ in e]
    for (a, b), (_, _, w) in zip(tree, e):
        assert w == M[a, b]
    keys = [(float(M[a, b]), min(a, b), max(a, b)) for a, b in tree]
    pm = _tree_path_max(n, tree, keys)
    in_tree = set(tree)
    for u in range(n):
        for v in range(u + 1, n):
            if (u, v) in in_tree:
                continue
            assert (float(M[u, v]), u, v) > pm[u][v]  # every other edge closes a cycle it tops


@pytest.mark.parametrize("k", [2, 5, 16])
def test_mrd_three_algorithms_agree(k):
    p = synth.blobs(1500, 3, 13)
    c = oracle.core_dist2(p, k)
    a = oracle.prim_mrd(p, c)
    assert np.array_equal(a, oracle.kruskal_mrd(p, c))
    assert np.array_equal(a, oracle.kd_boruvka_mrd(p, c, threads=4))
    assert np.all(a["w"] >= np.sort(c)[0])
