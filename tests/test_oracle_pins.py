"""Pins of the CPU oracle to things other than itself (runs without a GPU).

Each test ties one oracle function to a value the paper prints, a hand-worked
case, a closed form, an invariant, an independent library routine or brute
force, chosen so that a plausible slip (a dropped term, a wrong sign or index,
a transposed operand, a wrong tie rule) fails at least one of them.
"""
from __future__ import annotations

import numpy as np
import pytest

import synth
from fp32ref import exact_fma32, exact_weight32, fma32, pairwise_weights, weight32
from golden import fixtures as fx

INVALID = 0xFFFFFFFF


def as_tuples(e):
    return [(int(x["i"]), int(x["j"]), np.float32(x["w"])) for x in e]


def same_edges(a, b):
    return np.array_equal(np.asarray(a).view(np.uint8), np.asarray(b).view(np.uint8))


# --------------------------------------------------------------------------
# Independent FP32 reference used below: check it against exact rationals.
# --------------------------------------------------------------------------
def test_fp32ref_fma_matches_exact_rationals():
    g = np.random.default_rng(5)
    a = g.standard_normal(400).astype(np.float32) * np.float32(2.0) ** g.integers(-20, 20, 400)
    b = g.standard_normal(400).astype(np.float32)
    c = g.standard_normal(400).astype(np.float32) * np.float32(2.0) ** g.integers(-30, 5, 400)
    # adversarial: products that land near FP32 midpoints
    a[:50] = np.float32(1.0) + np.float32(2.0 ** -12)
    b[:50] = np.float32(1.0) + np.float32(2.0 ** -12)
    c[:50] = np.float32(2.0 ** -40) * np.arange(1, 51, dtype=np.float32)
    got = fma32(a, b, c)
    want = np.array([exact_fma32(x, y, z) for x, y, z in zip(a, b, c)], np.float32)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


# --------------------------------------------------------------------------
# Edge weight (FP32 squared distance in the fixed fma order)
# --------------------------------------------------------------------------
def test_weight_closed_forms(oracle_lib):
    assert oracle_lib.weight([0, 0, 0], [1, 2, 2]) == np.float32(9.0)
    assert oracle_lib.weight([0, 0], [3, 4]) == np.float32(25.0)
    assert oracle_lib.weight([1.5, -2, 7], [1.5, -2, 7]) == np.float32(0.0)


def test_weight_exact_fma_order(oracle_lib):
    g = np.random.default_rng(1)
    for dim in (2, 3):
        p = g.random((300, dim)).astype(np.float32)
        q = (p + g.standard_normal((300, dim)).astype(np.float32) * np.float32(1e-3)).astype(np.float32)
        for k in range(300):
            w = oracle_lib.weight(p[k], q[k])
            assert w.view(np.uint32) == exact_weight32(p[k], q[k]).view(np.uint32)
            # symmetric bit for bit: (-x)^2 == x^2
            assert oracle_lib.weight(q[k], p[k]).view(np.uint32) == w.view(np.uint32)
        # and the vectorised reference agrees with the exact one
        wv = weight32(p, q)
        assert np.array_equal(wv.view(np.uint32),
                              np.array([exact_weight32(p[k], q[k]) for k in range(300)],
                                       np.float32).view(np.uint32))


def test_weight_order_is_not_plain_sum(oracle_lib):
    # a pair where fma(dy,dy, dx*dx) and round(round(dx*dx) + round(dy*dy))
    # round to different FP32 values: the oracle must give the fused one
    dx = np.array([1050244054], np.uint32).view(np.float32)[0]  # 0.29971188
    dy = np.array([1054370422], np.uint32).view(np.float32)[0]  # 0.42268723
    p = np.array([dx, dy], np.float32)
    q = np.zeros(2, np.float32)
    w = oracle_lib.weight(p, q)
    fused = fma32(dy, dy, np.float32(dx * dx))
    plain = np.float32(np.float32(dx * dx) + np.float32(dy * dy))
    assert fused != plain
    assert w == fused


# --------------------------------------------------------------------------
# Whole EMST: hand cases from the fixtures
# --------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["unit_square.txt", "collinear.txt"])
def test_emst_hand_cases(oracle_lib, name):
    f = fx.load(name)
    dim = int(f["dim"][0])
    pts = fx.floats(f["points"], dim)
    want = fx.edges(f["edges"])
    for algo in (oracle_lib.prim, oracle_lib.kruskal, oracle_lib.kd_boruvka, oracle_lib.boruvka_steps):
        got = as_tuples(algo(pts))
        assert got == want, (algo.__name__, got)


def test_equilateral_fp32_ties(oracle_lib):
    # Equilateral in exact arithmetic; in FP32 the three weights may differ.
    # Brute force on three edges with the exact FP32 weights and the §2 key.
    pts = np.array([[0, 0], [1, 0], [0.5, np.sqrt(3) / 2]], np.float32)
    ws = {(a, b): exact_weight32(pts[a], pts[b]) for a, b in [(0, 1), (0, 2), (1, 2)]}
    order = sorted(ws, key=lambda e: (ws[e], e[0], e[1]))
    want = sorted([(a, b, ws[(a, b)]) for a, b in order[:2]], key=lambda t: (t[2], t[0], t[1]))
    for algo in (oracle_lib.prim, oracle_lib.kruskal, oracle_lib.kd_boruvka):
        assert as_tuples(algo(pts)) == want


def test_exact_ties_pick_smaller_ids(oracle_lib):
    # Four points at the corners of a square scaled by 2^-3 (weights exact):
    # the same tree as the unit square, whatever the scale.
    pts = np.array([[0, 0], [1, 0], [0, 1], [1, 1]], np.float32) * np.float32(0.125)
    got = as_tuples(oracle_lib.prim(pts))
    w = np.float32(0.015625)
    assert got == [(0, 1, w), (0, 2, w), (1, 3, w)]
    # relabel the corners: the chosen sides follow the ids, not the positions
    perm = [3, 2, 1, 0]
    got2 = as_tuples(oracle_lib.prim(pts[perm]))
    assert got2 == [(0, 1, w), (0, 2, w), (1, 3, w)]


def test_lattice_massive_ties(oracle_lib):
    k = np.stack(np.meshgrid(np.arange(4), np.arange(4), np.arange(4), indexing="ij"), -1).reshape(-1, 3)
    pts = k.astype(np.float32)
    e = oracle_lib.prim(pts)
    assert len(e) == 63 and np.all(e["w"] == np.float32(1.0))
    comps, cyc = oracle_lib.count_components(e, 64)
    assert comps == 1 and not cyc
    for algo in (oracle_lib.kruskal, oracle_lib.kd_boruvka, oracle_lib.boruvka_steps):
        assert same_edges(algo(pts), e)
    # under the (w, min, max) rule, vertex 0 keeps all of its unit edges
    s = set(zip(e["i"].tolist(), e["j"].tolist()))
    assert {(0, 1), (0, 4), (0, 16)} <= s


def test_duplicates_zero_weight(oracle_lib):
    pts = np.array([[0.5, 0.5, 0.5]] * 4 + [[0.75, 0.5, 0.5]], np.float32)
    e = as_tuples(oracle_lib.prim(pts))
    # coincident points join at weight 0; ties broken by (min, max): a star from 0
    assert e[:3] == [(0, 1, np.float32(0)), (0, 2, np.float32(0)), (0, 3, np.float32(0))]
    assert e[3] == (0, 4, np.float32(0.0625))


# --------------------------------------------------------------------------
# Whole EMST: invariants, brute-force cycle property, library cross-checks
# --------------------------------------------------------------------------
def _cycle_property_holds(pts, edges):
    n = len(pts)
    W = pairwise_weights(pts)
    adj = [[] for _ in range(n)]
    for i, j, w in zip(edges["i"], edges["j"], edges["w"]):
        adj[int(i)].append((int(j), (np.float32(w), min(i, j), max(i, j))))
        adj[int(j)].append((int(i), (np.float32(w), min(i, j), max(i, j))))
    tree = set((int(i), int(j)) for i, j in zip(edges["i"], edges["j"]))
    for s in range(n):
        # max key on the tree path from s to every vertex
        best = {s: None}
        stack = [s]
        while stack:
            u = stack.pop()
            for v, key in adj[u]:
                if v in best:
                    continue
                best[v] = key if best[u] is None or key > best[u] else best[u]
                stack.append(v)
        assert len(best) == n
        for t in range(s + 1, n):
            if (s, t) in tree:
                continue
            key = (W[s, t], s, t)
            if not key > best[t]:
                return False
    return True


@pytest.mark.parametrize("n,dim,seed", [(60, 2, 11), (120, 3, 12), (150, 2, 13)])
def test_cycle_property_bruteforce(oracle_lib, n, dim, seed):
    pts = synth.uniform(n, dim, seed)
    e = oracle_lib.prim(pts)
    assert len(e) == n - 1
    comps, cyc = oracle_lib.count_components(e, n)
    assert comps == 1 and not cyc
    assert _cycle_property_holds(pts, e)


def test_cycle_property_detects_a_planted_mistake(oracle_lib):
    pts = synth.uniform(40, 2, 3)
    e = oracle_lib.prim(pts).copy()
    # swap the heaviest tree edge for a heavier non-tree edge that keeps a tree
    W = pairwise_weights(pts)
    k = int(np.argmax(e["w"]))
    a, b = int(e["i"][k]), int(e["j"][k])
    rest = np.delete(e, k)
    comps = {}
    par = list(range(40))

    def find(x):
        while par[x] != x:
            x = par[x]
        return x
    for i, j in zip(rest["i"], rest["j"]):
        par[find(int(i))] = find(int(j))
    side = [find(v) == find(a) for v in range(40)]
    cands = [(W[u, v], u, v) for u in range(40) for v in range(u + 1, 40)
             if side[u] != side[v] and (u, v) != (min(a, b), max(a, b))]
    w2, u, v = min(cands)
    bad = np.concatenate([rest, np.array([(u, v, w2)], dtype=e.dtype)])
    assert not _cycle_property_holds(pts, bad)


@pytest.mark.parametrize("n,dim,seed", [(800, 3, 21), (1500, 2, 22)])
def test_total_weight_matches_scipy_mst(oracle_lib, n, dim, seed):
    """Every MST has the same multiset of weights; scipy's routine on the
    independent FP32 weight matrix must give the same sorted weights, and the
    FP64 total length must agree with an FP64-metric MST within 1e-6."""
    sp = pytest.importorskip("scipy.sparse.csgraph")
    pts = synth.uniform(n, dim, seed)
    e = oracle_lib.prim(pts)
    W = pairwise_weights(pts).astype(np.float64)
    T = sp.minimum_spanning_tree(W).tocoo()
    assert np.array_equal(np.sort(T.data.astype(np.float32)), np.sort(e["w"]))
    d64 = np.sqrt(((pts[:, None, :].astype(np.float64) - pts[None, :, :]) ** 2).sum(-1))
    T64 = sp.minimum_spanning_tree(d64)
    ours = np.sqrt(e["w"].astype(np.float64)).sum()
    assert abs(ours - T64.sum()) <= 1e-6 * T64.sum()


@pytest.mark.parametrize("n,dim,seed", [(300, 3, 31), (2000, 2, 32), (2000, 3, 33)])
def test_prim_kruskal_kd_steps_agree(oracle_lib, n, dim, seed):
    pts = synth.blobs(n, dim, seed, n_blobs=5)
    a = oracle_lib.prim(pts)
    assert same_edges(a, oracle_lib.kruskal(pts))
    assert same_edges(a, oracle_lib.kd_boruvka(pts))
    assert same_edges(a, oracle_lib.kd_boruvka(pts, threads=4))
    e, rounds = oracle_lib.boruvka_steps(pts, return_rounds=True)
    assert same_edges(a, e)
    assert rounds <= int(np.ceil(np.log2(n)))  # Algorithm 1's bound


@pytest.mark.parametrize("cfg", [1, 2, 3])
def test_kd_boruvka_matches_prim_on_workload_shapes(oracle_lib, cfg):
    n = 20000
    pts = synth.config_points(cfg, n=n, seed=100 + cfg)
    assert same_edges(oracle_lib.prim(pts), oracle_lib.kd_boruvka(pts, threads=4))


def test_kd_boruvka_lattice_ties(oracle_lib):
    pts = synth.lattice_ties(n_sites=3000, n_dup=200, side=20, seed=7)
    assert same_edges(oracle_lib.prim(pts), oracle_lib.kd_boruvka(pts, threads=2))


# --------------------------------------------------------------------------
# Per-step definitions
# --------------------------------------------------------------------------
def test_scene_box(oracle_lib):
    pts = synth.uniform(1000, 3, 4)
    lo, hi, fin = oracle_lib.scene_box(pts)
    assert fin and np.array_equal(lo, pts.min(0)) and np.array_equal(hi, pts.max(0))
    bad = pts.copy()
    bad[17, 1] = np.nan
    assert not oracle_lib.scene_box(bad)[2]


@pytest.mark.parametrize("dim", [3, 2])
def test_morton_hand_values(oracle_lib, dim):
    f = fx.load("morton_hand.txt")
    pts = fx.floats(f[f"dim{dim}_points"], dim)
    want = np.array([int(t) for t in f[f"dim{dim}_codes"]], dtype=np.uint64)
    lo, hi, _ = oracle_lib.scene_box(pts)
    assert np.array_equal(oracle_lib.morton(pts, lo, hi), want)


@pytest.mark.parametrize("dim", [3, 2])
def test_morton_deinterleave_and_monotone(oracle_lib, dim):
    pts = synth.uniform(3000, dim, 8)
    lo, hi, _ = oracle_lib.scene_box(pts)
    codes = oracle_lib.morton(pts, lo, hi)
    B = 21 if dim == 3 else 32
    q = np.zeros((len(pts), dim), np.uint64)
    for b in range(B):
        for d in range(dim):
            q[:, d] |= ((codes >> np.uint64(dim * b + dim - 1 - d)) & np.uint64(1)) << np.uint64(b)
    # the de-interleaved cells are non-decreasing in each coordinate
    for d in range(dim):
        o = np.argsort(pts[:, d], kind="stable")
        assert np.all(np.diff(q[o, d].astype(np.int64)) >= 0)
    # and equal the FP32 quantisation written out independently
    twoB = np.float32(2.0 ** B)
    s = (twoB / (hi - lo)).astype(np.float32)
    t = ((pts - lo).astype(np.float32) * s).astype(np.float32)
    qq = np.where(t >= twoB, np.uint64(2 ** B - 1), np.floor(t).astype(np.uint64))
    assert np.array_equal(q, qq)


def test_sort_perm_is_stable_argsort(oracle_lib):
    g = np.random.default_rng(3)
    codes = g.integers(0, 50, 5000).astype(np.uint64) << np.uint64(40)
    assert np.array_equal(oracle_lib.sort_perm(codes), np.argsort(codes, kind="stable"))


def test_radix_tree_fig4(oracle_lib):
    f = fx.load("fig4_node_labels.txt")
    codes = fx.ints(f["codes"], np.uint64)
    left, right, first, last = oracle_lib.radix_tree(codes)
    assert first.tolist() == fx.ints(f["node_first"]).tolist()
    assert last.tolist() == fx.ints(f["node_last"]).tolist()
    n = 8
    L = lambda k: n - 1 + k  # leaf ref
    assert left.tolist() == [3, L(0), L(2), 1, L(4), 6, L(5)]
    assert right.tolist() == [4, L(1), L(3), 2, 5, L(7), L(6)]


def _check_radix_tree(codes, left, right, first, last):
    n = len(codes)
    seen = np.zeros(2 * n - 1, np.int64)
    for v in range(n - 1):
        a, b = first[v], last[v]
        assert v in (a, b) or v == 0  # Karras numbering: a node is one end of its range
        for c in (left[v], right[v]):
            seen[c] += 1
        lf = (left[v] - (n - 1), left[v] - (n - 1)) if left[v] >= n - 1 else (first[left[v]], last[left[v]])
        rt = (right[v] - (n - 1), right[v] - (n - 1)) if right[v] >= n - 1 else (first[right[v]], last[right[v]])
        assert lf[0] == a and rt[1] == b and lf[1] + 1 == rt[0]

        # augmented keys: code then position; the split bit is 0 on the left, 1 on the right
        def key(k):
            return (int(codes[k]) << 32) | int(k)
        common = 96 - (key(a) ^ key(b)).bit_length()
        bit = 95 - common
        assert all(((key(k) >> bit) & 1) == 0 for k in range(lf[0], lf[1] + 1))
        assert all(((key(k) >> bit) & 1) == 1 for k in range(rt[0], rt[1] + 1))
    assert seen[0] == 0 and np.all(seen[1:] == 1)


@pytest.mark.parametrize("seed,dups", [(1, False), (2, True)])
def test_radix_tree_invariants(oracle_lib, seed, dups):
    g = np.random.default_rng(seed)
    codes = np.sort(g.integers(0, 2 ** 20 if dups else 2 ** 62, 300).astype(np.uint64))
    if dups:
        codes = np.sort(np.concatenate([codes, codes[:100]]))
    left, right, first, last = oracle_lib.radix_tree(codes)
    _check_radix_tree(codes, left, right, first, last)


def test_node_boxes_union_of_children(oracle_lib):
    pts = synth.uniform(500, 3, 9)
    r = oracle_lib.bvh_reference(pts)
    n = 500
    lo, hi = r["box_lo"], r["box_hi"]
    sp = r["sorted_points"]
    for v in range(n - 1):
        cl = [sp[c - (n - 1)] if c >= n - 1 else lo[c] for c in (r["left"][v], r["right"][v])]
        ch = [sp[c - (n - 1)] if c >= n - 1 else hi[c] for c in (r["left"][v], r["right"][v])]
        assert np.array_equal(lo[v], np.minimum(cl[0], cl[1]))
        assert np.array_equal(hi[v], np.maximum(ch[0], ch[1]))
    assert np.array_equal(lo[0], r["lo"]) and np.array_equal(hi[0], r["hi"])


def test_node_labels_fig4(oracle_lib):
    f = fx.load("fig4_node_labels.txt")
    labels = fx.ints(f["leaf_labels"], np.uint32)
    want = [INVALID if t == "INVALID" else int(t) for t in f["node_labels"]]
    got = oracle_lib.node_labels(labels, fx.ints(f["node_first"]), fx.ints(f["node_last"]))
    assert got.tolist() == want


def test_upper_bounds_bound_the_true_minimum(oracle_lib):
    pts = synth.uniform(400, 3, 10)
    g = np.random.default_rng(0)
    labels = np.maximum.accumulate(np.where(g.random(400) < 0.2, np.arange(400), 0))
    labels = labels.astype(np.uint32)  # runs of equal labels, label = first index
    ub = oracle_lib.upper_bounds(pts, labels)
    W = pairwise_weights(pts)
    for c in np.unique(labels):
        inside = labels == c
        true_min = W[np.ix_(inside, ~inside)].min()
        assert ub[c] >= true_min
        adj = [W[k, k + 1] for k in range(399) if labels[k] != labels[k + 1] and c in (labels[k], labels[k + 1])]
        assert ub[c] == min(adj)


def test_nn_other_bruteforce(oracle_lib):
    g = np.random.default_rng(4)
    pts = synth.uniform(200, 2, 12)
    ids = g.permutation(200).astype(np.uint32)
    labels = (np.arange(200) // 7 * 7).astype(np.uint32)
    W = pairwise_weights(pts)
    radius = np.where(g.random(200) < 0.5, np.float32(np.inf), np.float32(0.003)).astype(np.float32)
    w, j = oracle_lib.nn_other(pts, ids, labels, radius)
    for i in range(200):
        cand = [(W[i, k], ids[k], k) for k in range(200) if labels[k] != labels[i] and W[i, k] <= radius[i]]
        if not cand:
            assert j[i] == -1
        else:
            best = min(cand)
            assert j[i] == best[2] and w[i] == best[0]


def test_merge_chain_fixture(oracle_lib):
    f = fx.load("merge_chain.txt")
    pts = fx.floats(f["points"], 3)
    ids = np.arange(5, dtype=np.uint32)
    labels = np.arange(5, dtype=np.uint32)
    w, j = oracle_lib.nn_other(pts, ids, labels, np.full(5, np.inf, np.float32))
    assert j.tolist() == fx.ints(f["nn"]).tolist()
    assert w.tolist() == fx.floats(f["nn_w"]).tolist()
    cw, ca, cb = oracle_lib.component_min(labels, ids, w, j)
    new, e = oracle_lib.merge(labels, ca, cb, cw, ids)
    assert new.tolist() == fx.ints(f["new_labels"]).tolist()
    assert sorted(as_tuples(e)) == sorted(fx.edges(f["edges"]))


def test_component_min_uses_full_key(oracle_lib):
    # two points of one component tie on w and on min id; max id decides
    pts = np.array([[0, 0], [1, 0], [0, 1], [5, 5]], np.float32)
    labels = np.array([0, 1, 1, 3], np.uint32)
    ids = np.array([0, 1, 2, 3], np.uint32)
    # component 1 = {1, 2}: both are at w = 1 from point 0 -> keys (1,0,1), (1,0,2)
    w = np.array([1, 1, 1, 50], np.float32)
    j = np.array([1, 0, 0, 1], np.int64)
    cw, ca, cb = oracle_lib.component_min(labels, ids, w, j)
    assert (ca[1], cb[1]) == (1, 0)


# ---------------------------------------------------------------------------
# 128-bit Morton codes (§4.1's finer grid): codes, order, radix tree
# ---------------------------------------------------------------------------
def test_morton128_hand_values(oracle_lib):
    # lo = 0, hi = 1 on every axis: (0.5, 0.25, 0.75) quantises to x = 2^41,
    # y = 2^40, z = 2^41 + 2^40 on the 42-bit grid; interleaved (x first) those
    # are bits 125, 121, 123 and 120 of the 128-bit code
    p = np.array([[0, 0, 0], [1, 1, 1], [0.5, 0.25, 0.75]], np.float32)
    lo, hi, _ = oracle_lib.scene_box(p)
    ch, cl = oracle_lib.morton128(p, lo, hi)
    assert [int(x) for x in ch] == [0, 2 ** 62 - 1, (1 << 61) | (1 << 59) | (1 << 57) | (1 << 56)]
    assert [int(x) for x in cl] == [0, 2 ** 64 - 1, 0]


@pytest.mark.parametrize("dim", [2, 3])
def test_morton128_extends_the_64bit_code_on_a_dyadic_grid(oracle_lib, dim):
    # coordinates k / 2^10 in [0, 1] with both corners present: both quantisers
    # are exact, the 64-bit cell is the top half of the 128-bit cell's bits,
    # so the 128-bit code starts with the 64-bit one
    g = np.random.default_rng(5)
    p = (g.integers(0, 1024, size=(2000, dim)) / 1024.0).astype(np.float32)
    p[0] = 0.0
    p[1] = 1.0
    lo, hi, _ = oracle_lib.scene_box(p)
    c64 = oracle_lib.morton(p, lo, hi)
    ch, cl = oracle_lib.morton128(p, lo, hi)
    wide = [(int(h) << 64) | int(l) for h, l in zip(ch, cl)]
    shift = 128 - 64 if dim == 2 else 126 - 63
    assert [w >> shift for w in wide] == [int(c) for c in c64]


@pytest.mark.parametrize("dim", [2, 3])
def test_morton128_deinterleave_monotone_and_finer(oracle_lib, dim):
    # clusters denser than the 3D 64-bit grid (cells of 2^-21) but resolved by
    # FP32: the de-interleaved cells are monotone in each coordinate, and in
    # 3D the 128-bit codes separate many points the 64-bit codes do not (2D
    # 64-bit codes already have 32 bits per axis)
    g = np.random.default_rng(6)
    centres = g.random((20, dim))
    p = (centres[g.integers(0, 20, 4000)] + g.normal(0, 2e-7, (4000, dim))).astype(np.float32)
    lo, hi, _ = oracle_lib.scene_box(p)
    ch, cl = oracle_lib.morton128(p, lo, hi)
    B = 42 if dim == 3 else 64
    wide = [(int(h) << 64) | int(l) for h, l in zip(ch, cl)]
    q = np.zeros((len(p), dim), dtype=object)
    for i, w in enumerate(wide):
        for d in range(dim):
            v = 0
            for b in range(B):
                v |= ((w >> (dim * b + dim - 1 - d)) & 1) << b
            q[i, d] = v
    for d in range(dim):
        o = np.argsort(p[:, d], kind="stable")
        assert all(q[o[k], d] <= q[o[k + 1], d] for k in range(len(p) - 1))
    c64 = oracle_lib.morton(p, lo, hi)
    n128, n64 = len(set(wide)), len(set(int(c) for c in c64))
    assert n128 >= n64
    if dim == 3:
        assert n128 > 2 * n64


def test_sort_perm128_is_lexsort(oracle_lib):
    g = np.random.default_rng(7)
    ch = g.integers(0, 8, 4000).astype(np.uint64)
    cl = g.integers(0, 8, 4000).astype(np.uint64) << np.uint64(50)
    assert np.array_equal(oracle_lib.sort_perm128(ch, cl), np.lexsort((np.arange(4000), cl, ch)))


def test_radix_tree128_reduces_to_64bit_and_keeps_invariants(oracle_lib):
    g = np.random.default_rng(8)
    lo = np.sort(g.integers(0, 2 ** 62, 300).astype(np.uint64))
    want = oracle_lib.radix_tree(lo)
    got = oracle_lib.radix_tree128(np.zeros(300, np.uint64), lo)
    for a, b in zip(got, want):
        assert np.array_equal(a, b)
    # with duplicates in both words: the split bit of the augmented
    # (hi, lo, position) key is 0 on the left and 1 on the right
    hi = np.sort(g.integers(0, 4, 200).astype(np.uint64))
    lw = g.integers(0, 3, 200).astype(np.uint64) << np.uint64(63)
    o = np.lexsort((lw, hi))
    hi, lw = hi[o], lw[o]
    left, right, first, last = oracle_lib.radix_tree128(hi, lw)
    n = len(hi)

    def key(k):
        return (int(hi[k]) << 96) | (int(lw[k]) << 32) | int(k)
    for v in range(n - 1):
        a, b = first[v], last[v]
        lf = (left[v] - (n - 1),) * 2 if left[v] >= n - 1 else (first[left[v]], last[left[v]])
        rt = (right[v] - (n - 1),) * 2 if right[v] >= n - 1 else (first[right[v]], last[right[v]])
        assert lf[0] == a and rt[1] == b and lf[1] + 1 == rt[0]
        bit = (key(a) ^ key(b)).bit_length() - 1
        assert all(((key(k) >> bit) & 1) == 0 for k in range(lf[0], lf[1] + 1))
        assert all(((key(k) >> bit) & 1) == 1 for k in range(rt[0], rt[1] + 1))
