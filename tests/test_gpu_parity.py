"""Parity of the CUDA path with the CPU oracle, through the C ABI.

Bit-exact throughout: the tree build (codes, order, hierarchy, boxes), every
step of one Boruvka round, and whole spanning trees (edge ids and FP32 weight
bits), on seeded inputs shaped like the paper's workloads, at sizes that span
several sort tiles and CTAs with ragged tails, plus the degenerate cases.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

INVALID = 0xFFFFFFFF


@pytest.fixture(scope="module")
def pkg():
    import paper_2207_00514_gb300 as p
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p.load_library()
    return p


def dev_pts(pts):
    return torch.from_numpy(np.ascontiguousarray(pts)).cuda()


def gpu_emst(pkg, pts):
    e = pkg.emst_compute(dev_pts(pts))
    torch.cuda.synchronize()
    return pkg.edges_numpy(e)


def assert_same_edges(got, want, what=""):
    g = got.view(np.uint8).reshape(-1, 12)
    w = want.view(np.uint8).reshape(-1, 12)
    assert g.shape == w.shape, (what, g.shape, w.shape)
    rows = np.nonzero((g != w).any(1))[0]
    assert len(rows) == 0, f"{what}: {len(rows)} edges differ, first {rows[:5]}: got {got[rows[:3]]} want {want[rows[:3]]}"


def u32(t):
    return t.cpu().numpy().view(np.uint32)


# ---------------------------------------------------------------------------
# A1-A4: tree build
# ---------------------------------------------------------------------------
BUILD_CASES = [
    ("uniform3", lambda: synth.uniform(5000, 3, 1)),
    ("blobs2", lambda: synth.blobs(7001, 2, 2)),
    ("halos3", lambda: synth.halos(9000, 3)),
    ("lattice_dups", lambda: synth.lattice_ties(n_sites=3000, n_dup=400, side=16, seed=4)),
    ("tiny2", lambda: synth.uniform(2, 3, 5)),
    ("tiny3", lambda: synth.uniform(3, 2, 6)),
    ("one_tile_plus_one", lambda: synth.uniform(3073, 3, 7)),
]


def chunk_ranges(refs, n, nc, leaf, first, last):
    """Point ranges [a, b] of children given as refs (internal id, or leaf
    chunk c as nc-1+c) of the oracle's tree over chunk keys."""
    is_leaf = refs >= nc - 1
    c = np.clip(refs - (nc - 1), 0, nc - 1)
    v = np.clip(refs, 0, max(nc - 2, 0))
    cf = np.where(is_leaf, c, first[v])
    cl = np.where(is_leaf, c, last[v])
    return cf * leaf, np.minimum((cl + 1) * leaf, n) - 1


@pytest.mark.parametrize("leaf", [1, 4])
@pytest.mark.parametrize("name,make", BUILD_CASES, ids=[c[0] for c in BUILD_CASES])
def test_bvh_matches_oracle(pkg, name, make, leaf):
    pts = make()
    n = len(pts)
    if (n + leaf - 1) // leaf < 2:
        pytest.skip("fewer than two leaf chunks")
    ref = oracle.bvh_reference(pts)
    out = pkg.emst_build_bvh(dev_pts(pts), leaf_size=leaf)
    torch.cuda.synchronize()
    codes = out["codes"].cpu().numpy().view(np.uint64)
    perm = u32(out["perm"])
    assert np.array_equal(codes, ref["sorted_codes"])
    assert np.array_equal(perm, ref["perm"])
    # the hierarchy is the radix tree over the chunks' first codes
    nc = (n + leaf - 1) // leaf
    left, right, first, last = oracle.radix_tree(ref["sorted_codes"][::leaf])
    ch = u32(out["children"]).astype(np.int64)
    conv = np.where(ch & 0x80000000, (nc - 1) + (ch & 0x7FFFFFFF), ch)
    assert np.array_equal(conv[:, 0], left)
    assert np.array_equal(conv[:, 1], right)
    boxes = out["boxes"].cpu().numpy()
    sp = ref["sorted_points"]
    d = pts.shape[1]
    for side, refs in ((0, left), (1, right)):
        a, b = chunk_ranges(refs, n, nc, leaf, first, last)
        lo = np.stack([sp[x:y + 1].min(0) for x, y in zip(a, b)])
        hi = np.stack([sp[x:y + 1].max(0) for x, y in zip(a, b)])
        assert np.array_equal(boxes[:, side, 0:d], lo)
        assert np.array_equal(boxes[:, side, 3:3 + d], hi)
        if d == 2:
            assert np.all(boxes[:, side, 2] == 0) and np.all(boxes[:, side, 5] == 0)
    if leaf == 1:  # one point per leaf: the oracle's own node boxes
        for side, refs in ((0, left), (1, right)):
            inner = refs < n - 1
            assert np.array_equal(boxes[inner, side, 0:d], ref["box_lo"][refs[inner]])
            assert np.array_equal(boxes[inner, side, 3:3 + d], ref["box_hi"][refs[inner]])


# ---------------------------------------------------------------------------
# A5-A9: one round from given labels
# ---------------------------------------------------------------------------
def _labels_from_groups(groups):
    """Curve-order labels: each group's label is its smallest curve index."""
    n = len(groups)
    first = {}
    lab = np.empty(n, np.uint32)
    for k in range(n):
        g = int(groups[k])
        if g not in first:
            first[g] = k
        lab[k] = first[g]
    return lab


ROUND_CASES = [
    ("singletons", 3000, 3, lambda n, g: np.arange(n)),
    ("runs", 4000, 3, lambda n, g: np.maximum.accumulate(np.where(g.random(n) < 0.05, np.arange(n), 0))),
    ("scattered", 2500, 2, lambda n, g: g.integers(0, 40, n)),
    ("two", 1500, 3, lambda n, g: (np.arange(n) > n // 3).astype(np.int64)),
]


@pytest.mark.parametrize("leaf", [1, 4])
@pytest.mark.parametrize("name,n,dim,groups", ROUND_CASES, ids=[c[0] for c in ROUND_CASES])
@pytest.mark.parametrize("given_radius", [False, True])
def test_round_step_matches_oracle(pkg, name, n, dim, groups, given_radius, leaf):
    g = np.random.default_rng(n + dim)
    pts = synth.blobs(n, dim, n, n_blobs=6)
    ref = oracle.bvh_reference(pts)
    sp, perm = ref["sorted_points"], ref["perm"]
    labels = _labels_from_groups(groups(n, g))
    radius = None
    if given_radius:
        radius = np.where(g.random(n) < 0.5, np.float32(np.inf),
                          np.float32(g.random(n) * 0.002)).astype(np.float32)
    out = pkg.emst_round_step(dev_pts(pts), torch.from_numpy(labels.view(np.int32)),
                              None if radius is None else torch.from_numpy(radius), leaf_size=leaf)
    torch.cuda.synchronize()
    # A5 node labels (per child of each internal node): the label shared by
    # every point of the child's range, else invalid
    if leaf == 1:
        node_lab = oracle.node_labels(labels, ref["first"], ref["last"])
        for side, refs in ((0, ref["left"]), (1, ref["right"])):
            want = np.where(refs >= n - 1, labels[np.clip(refs - (n - 1), 0, n - 1)],
                            node_lab[np.clip(refs, 0, n - 2)])
            assert np.array_equal(u32(out["node_labels"])[:, side], want.astype(np.uint32))
    else:
        nc = (n + leaf - 1) // leaf
        left, right, first, last = oracle.radix_tree(ref["sorted_codes"][::leaf])
        for side, refs in ((0, left), (1, right)):
            a, b = chunk_ranges(refs, n, nc, leaf, first, last)
            want = np.array([labels[x] if np.all(labels[x:y + 1] == labels[x]) else INVALID
                             for x, y in zip(a, b)], dtype=np.uint32)
            assert np.array_equal(u32(out["node_labels"])[:, side], want)
    # A6 upper bounds
    ub = oracle.upper_bounds(sp, labels)
    assert np.array_equal(out["upper_bound"].cpu().numpy().view(np.uint32), ub.view(np.uint32))
    # A7 queries
    rad = ub[labels] if radius is None else radius
    w, j = oracle.nn_other(sp, perm, labels, rad)
    assert np.array_equal(out["nn_w"].cpu().numpy().view(np.uint32), w.view(np.uint32))
    jj = np.where(j < 0, INVALID, j).astype(np.uint32)
    assert np.array_equal(u32(out["nn_j"]), jj)
    # A8 + A9
    cw, ca, cb = oracle.component_min(labels, perm, w, j)
    new, e = oracle.merge(labels, ca, cb, cw, perm)
    assert np.array_equal(u32(out["labels"]), new)
    got_e = np.sort(pkg.edges_numpy(out["edges"]), order=["w", "i", "j"])
    want_e = np.sort(e, order=["w", "i", "j"])
    assert_same_edges(got_e, want_e, "round edges")


# ---------------------------------------------------------------------------
# Whole EMST
# ---------------------------------------------------------------------------
EMST_CASES = [
    ("n2", lambda: synth.uniform(2, 3, 0)),
    ("n3_2d", lambda: synth.uniform(3, 2, 1)),
    ("n5", lambda: synth.uniform(5, 3, 2)),
    ("n100_2d", lambda: synth.uniform(100, 2, 3)),
    ("tile_plus_one", lambda: synth.uniform(3073, 3, 4)),
    ("config1_uniform10k", lambda: synth.uniform(10_000, 3, 0)),
    ("blobs2d_12k", lambda: synth.blobs(12_345, 2, 1)),
    ("halos3d_15k", lambda: synth.halos(15_000, 2)),
    ("lattice_ties_dups", lambda: synth.lattice_ties(n_sites=6000, n_dup=250, side=20, seed=3)),
    ("all_identical", lambda: np.full((257, 3), 0.25, np.float32)),
    ("collinear", lambda: np.stack([np.arange(1000, dtype=np.float32) ** 1.5 / 1e4,
                                    np.zeros(1000, np.float32), np.zeros(1000, np.float32)], 1)),
    ("flat_dimension", lambda: np.concatenate([synth.uniform(2000, 2, 9), np.full((2000, 1), 0.5, np.float32)], 1)),
    ("negative_coords", lambda: (synth.uniform(3000, 3, 10) * 200 - 100).astype(np.float32)),
]


def equal_weight_pairs(n=20_000, pairs=40, triples=3, seed=12):
    """Uniform points plus `pairs` pairs (a, a + d) and `triples` triples
    (p - d, p, p + d), d = 2^-14 along x, all in [0.5, 1)^3 where both
    endpoints and their difference are exact in FP32: many MST edges of one
    exactly equal weight d^2 between different points (one run of equal
    weights the output must put in (i, j) order), far shorter than the
    uniform points' spacing."""
    g = np.random.default_rng(seed)
    d = np.float32(2.0 ** -14)
    base = synth.uniform(n, 3, seed)
    a = (0.5 + 0.45 * g.random((pairs, 3))).astype(np.float32)
    b = a.copy()
    b[:, 0] += d
    p = (0.5 + 0.45 * g.random((triples, 3))).astype(np.float32)
    lo, hi = p.copy(), p.copy()
    lo[:, 0] -= d
    hi[:, 0] += d
    pts = np.concatenate([base, a, b, lo, p, hi])
    return np.ascontiguousarray(pts[g.permutation(len(pts))])


EMST_CASES += [
    ("equal_weight_run", equal_weight_pairs),
    # equal weights by the million and no identical points: the output's
    # sort by weight alone meets runs too long to fix in place and falls back
    ("lattice_no_duplicates", lambda: synth.lattice_ties(n_sites=12_000, n_dup=0, side=30, seed=6)),
]


@pytest.mark.parametrize("name,make", EMST_CASES, ids=[c[0] for c in EMST_CASES])
def test_emst_matches_oracle(pkg, name, make):
    pts = np.ascontiguousarray(make(), dtype=np.float32)
    got = gpu_emst(pkg, pts)
    want = oracle.prim(pts) if len(pts) <= 4000 else oracle.kd_boruvka(pts, threads=os.cpu_count() or 4)
    assert_same_edges(got, want, name)


def test_host_buffers_match_device_buffers(pkg):
    pts = synth.halos(20_000, 5)
    dev = gpu_emst(pkg, pts)
    pinned = torch.from_numpy(pts).pin_memory()
    e_pinned = pkg.emst_compute(pinned)
    assert e_pinned.device.type == "cpu"
    assert_same_edges(pkg.edges_numpy(e_pinned), dev, "pinned host")
    pageable = torch.from_numpy(pts.copy())
    out = torch.empty((len(pts) - 1, 3), dtype=torch.int32)
    pkg.emst_compute(pageable, out_edges=out)
    assert_same_edges(pkg.edges_numpy(out), dev, "pageable host")


def test_repeatable_and_stats(pkg):
    pts = synth.blobs(50_000, 3, 11)
    t = dev_pts(pts)
    a, st = pkg.emst_compute_ex(t, count_visits=True)
    b = pkg.emst_compute(t)
    torch.cuda.synchronize()
    assert_same_edges(pkg.edges_numpy(a), pkg.edges_numpy(b), "repeat")
    assert 1 <= st["rounds"] <= int(np.ceil(np.log2(len(pts))))
    assert st["components_per_round"][0] == len(pts)
    assert st["node_visits"] > 0 and st["kernel_launches"] > 0
    c, _ = pkg.emst_compute_ex(t, carried_radius=False, block_size=128)
    assert_same_edges(pkg.edges_numpy(c), pkg.edges_numpy(b), "options")
    for block in (64, 192, 256):
        d, _ = pkg.emst_compute_ex(t, block_size=block)
        assert_same_edges(pkg.edges_numpy(d), pkg.edges_numpy(b), f"block {block}")
    # larger CTAs than the traversal is compiled for are refused, not run
    with pytest.raises(pkg.EmstError) as ei:
        pkg.emst_compute_ex(t, block_size=512)
    assert ei.value.status == -1
    for leaf in (1, 2, 8, 16):
        d, _ = pkg.emst_compute_ex(t, leaf_size=leaf)
        assert_same_edges(pkg.edges_numpy(d), pkg.edges_numpy(b), f"leaf size {leaf}")


def test_degenerate_sizes_and_errors(pkg):
    for n in (0, 1):
        e = pkg.emst_compute(dev_pts(np.zeros((n, 3), np.float32)))
        assert e.shape == (0, 3)
    bad = synth.uniform(1000, 3, 1)
    bad[123, 2] = np.nan
    with pytest.raises(pkg.EmstError) as ei:
        pkg.emst_compute(dev_pts(bad))
    assert ei.value.status == -2
    bad[123, 2] = np.inf
    with pytest.raises(pkg.EmstError):
        pkg.emst_compute(dev_pts(bad))
    # the context is still usable after a reported error
    ok = gpu_emst(pkg, synth.uniform(500, 2, 3))
    assert len(ok) == 499


@pytest.mark.parametrize("cfg", [2])
def test_full_size_config_vs_kd_oracle(pkg, cfg):
    """Config 2 at full size (1,000,000 2D blob points): the whole tree."""
    pts = synth.config_points(cfg)
    got = gpu_emst(pkg, pts)
    want = oracle.kd_boruvka(pts, threads=os.cpu_count() or 4)
    assert_same_edges(got, want, f"config {cfg}")


def test_full_size_halos_37M_vs_kd_oracle(pkg):
    """Config 3 at full size (37,000,000 3D halo points, seed 2): the whole
    tree against the k-d tree Boruvka oracle (all host threads)."""
    pts = synth.config_points(3)
    got = gpu_emst(pkg, pts)
    want = oracle.kd_boruvka(pts, threads=os.cpu_count() or 4)
    assert_same_edges(got, want, "config 3")


def test_full_size_lattice_ties_vs_kd_oracle(pkg):
    """Config 5's tie-stress set at full size: 7,680,000 distinct sites of
    {0..199}^3 plus 320,000 duplicates (massive equal weights, zero weights)."""
    pts = synth.lattice_ties()
    got = gpu_emst(pkg, pts)
    want = oracle.kd_boruvka(pts, threads=os.cpu_count() or 4)
    assert_same_edges(got, want, "lattice ties")


def test_full_size_halos_100M_vs_kd_oracle(pkg):
    """Config 5 at full size (100,000,000 3D halo points, seed 3): the whole
    tree against the k-d tree Boruvka oracle (Algorithm 1 with the §2
    tie-break, all host threads), edge for edge.  Before that, what holds at
    any size without the oracle: n-1 edges, one connected acyclic tree,
    (w, i, j) order, weights equal to the FP32 weight of their endpoints
    (sampled), and the cut property on sampled single-vertex cuts: for a
    vertex v the smallest edge (w, min id, max id) incident to v separates {v}
    from the rest, so it must be in the tree -- found here by brute force over
    all n points."""
    from fp32ref import weight32
    pts = synth.config_points(5)
    n = len(pts)
    e = gpu_emst(pkg, pts)
    assert len(e) == n - 1
    assert np.all(e["i"] < e["j"])
    w_bits = e["w"].view(np.uint32).astype(np.uint64)
    ii, jj = e["i"].astype(np.uint64), e["j"].astype(np.uint64)
    later = (w_bits[1:] > w_bits[:-1]) | ((w_bits[1:] == w_bits[:-1]) &
             ((ii[1:] > ii[:-1]) | ((ii[1:] == ii[:-1]) & (jj[1:] > jj[:-1]))))
    assert np.all(later)
    del w_bits, ii, jj, later
    comps, cyc = oracle.count_components(e, n)
    assert comps == 1 and not cyc
    g = np.random.default_rng(5)
    idx = g.choice(n - 1, 200_000, replace=False)
    w = weight32(pts[e["i"][idx]], pts[e["j"][idx]])
    assert np.array_equal(w.view(np.uint32), e["w"][idx].view(np.uint32))
    for v in g.choice(n, 12, replace=False):
        wv = weight32(np.broadcast_to(pts[v], pts.shape), pts)
        wv[v] = np.inf
        m = wv.min()
        j = int(np.nonzero(wv == m)[0].min())  # equal weights: the smaller id (the key's order)
        a, b = min(int(v), j), max(int(v), j)
        hit = np.nonzero((e["i"] == a) & (e["j"] == b))[0]
        assert len(hit) == 1 and e["w"][hit[0]] == m, (v, j)
        del wv
    want = oracle.kd_boruvka(pts, threads=os.cpu_count() or 4)
    assert_same_edges(e, want, "config 5 (100M)")


def test_massive_duplicate_group(pkg):
    """20,000 copies of one point among 30,000 others: the zero-weight ties
    resolve by id without every copy visiting every other (the traversal's
    tie pruning), and the tree is the oracle's."""
    g = np.random.default_rng(21)
    pts = np.concatenate([np.full((20_000, 3), 0.25, np.float32),
                          g.random((30_000, 3)).astype(np.float32)])
    pts = pts[g.permutation(len(pts))]
    got = gpu_emst(pkg, pts)
    want = oracle.kd_boruvka(pts, threads=os.cpu_count() or 4)
    assert_same_edges(got, want, "duplicates")
    assert np.count_nonzero(got["w"] == 0) == 19_999


@pytest.mark.parametrize("case", ["halos3", "blobs2", "lattice_dups", "uniform3_ragged"])
def test_persistent_traversal_matches_oracle(pkg, case):
    """The persistent work-queue form of Algorithm 2 (traversal = 2: warps
    refill lanes from a global queue of curve positions) gives the oracle's
    tree, as the one-thread-per-point form does; with counting on, the
    per-round counts add up."""
    pts = {"halos3": lambda: synth.halos(120_000, 31),
           "blobs2": lambda: synth.blobs(90_001, 2, 32),
           "lattice_dups": lambda: synth.lattice_ties(n_sites=40_000, n_dup=2_000, side=40, seed=33),
           "uniform3_ragged": lambda: synth.uniform(70_003, 3, 34)}[case]()
    want = oracle.kd_boruvka(pts, threads=os.cpu_count() or 4)
    t = dev_pts(pts)
    for count in (False, True):
        e, st = pkg.emst_compute_ex(t, traversal=2, count_visits=count)
        assert_same_edges(pkg.edges_numpy(e), want, f"persistent {case}")
        if count:
            assert sum(st["round_visits"]) == st["node_visits"]
            assert st["round_queries"][0] == len(pts)  # the first round searches every point
            assert all(0 < d <= len(pts) - 1 for d in st["round_distinct_nodes"][:2])


def test_batched_persistent_matches_oracle(pkg):
    sizes = [0, 1, 2, 3, 700, 2500, 3073, 17, 4000]
    parts = [synth.blobs(s, 3, 700 + k, n_blobs=3) if s > 0 else np.zeros((0, 3), np.float32)
             for k, s in enumerate(sizes)]
    pts = np.ascontiguousarray(np.concatenate(parts), dtype=np.float32)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    e, eo, st = pkg.emst_compute_batched_ex(dev_pts(pts), offsets, traversal=2)
    got = pkg.edges_numpy(e)
    for k, s in enumerate(sizes):
        if s >= 2:
            assert_same_edges(got[eo[k]:eo[k + 1]], oracle.prim(parts[k]), f"instance {k}")


@pytest.mark.parametrize("n,dim", [(70_001, 3), (50_002, 2), (4, 3), (2, 2)])
def test_pinned_host_buffers_match_oracle(pkg, n, dim):
    """Pinned host input and output are read and written in place (the
    scene-box pass reads the points through their device mapping, 16 bytes
    at a time with a ragged tail; the last output kernel writes four edges
    per thread straight into the host buffer, the rest one by one): the tree
    is the oracle's, and pageable host buffers give the same."""
    pts = synth.halos(n, 41) if dim == 3 else synth.blobs(n, 2, 42)
    want = oracle.kd_boruvka(pts, threads=os.cpu_count() or 4) if n > 10 else oracle.prim(pts)
    hp = torch.from_numpy(pts).pin_memory()
    ho = torch.empty((n - 1, 3), dtype=torch.int32).pin_memory()
    pkg.emst_compute(hp, out_edges=ho)
    torch.cuda.synchronize()
    assert_same_edges(pkg.edges_numpy(ho), want, f"pinned n={n} dim={dim}")
    po = torch.empty((n - 1, 3), dtype=torch.int32)  # pageable
    pkg.emst_compute(torch.from_numpy(pts.copy()), out_edges=po)
    torch.cuda.synchronize()
    assert_same_edges(pkg.edges_numpy(po), want, f"pageable n={n} dim={dim}")
