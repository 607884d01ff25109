"""Single-linkage dendrogram on the GPU (emst_dendrogram) against the CPU
oracle's Kruskal merge sequence, bit-exact: every linkage row (children,
weight bits, size) and every parent.  Inputs: seeded random trees of every
shape (with and without tied weights) at sizes that span the rank-split
levels and leave ragged blocks, the EMSTs and mutual-reachability trees the
library computes, host buffers, and invalid trees."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2207_00514_gb300 as p
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p.load_library()
    return p


def edges_tensor(e, device="cuda"):
    a = np.ascontiguousarray(e).view(np.int32).reshape(-1, 3)
    t = torch.from_numpy(a.copy())
    return t.to(device) if device == "cuda" else t.pin_memory()


def gpu_dendrogram(pkg, edges_t, n):
    link, parent = pkg.emst_dendrogram(edges_t, n)
    torch.cuda.synchronize()
    return pkg.linkage_numpy(link), parent.cpu().numpy().view(np.uint32)


def assert_same(pkg, got, want, what):
    gl, gp = got
    wl, wp = want
    g = gl.view(np.uint32).reshape(-1, 4)
    w = wl.view(np.uint32).reshape(-1, 4)
    assert g.shape == w.shape, what
    bad = np.nonzero((g != w).any(1))[0]
    assert len(bad) == 0, f"{what}: {len(bad)} linkage rows differ, first {bad[:5]}: {g[bad[:3]]} vs {w[bad[:3]]}"
    bad = np.nonzero(gp != wp)[0]
    assert len(bad) == 0, f"{what}: {len(bad)} parents differ, first {bad[:5]}"


SIZES = [1, 2, 3, 255, 256, 257, 511, 512, 513, 1000, 4097, 100_003]


@pytest.mark.parametrize("shape", synth.TREE_SHAPES)
@pytest.mark.parametrize("ties", [0, 5])
def test_random_trees(pkg, shape, ties):
    for idx, n in enumerate(SIZES):
        e = synth.tree_edges(n, 10 * idx + ties, shape, ties=ties)
        got = gpu_dendrogram(pkg, edges_tensor(e), n)
        assert_same(pkg, got, oracle.dendrogram(e, n), f"{shape} ties={ties} n={n}")


def test_deep_and_wide_trees_large(pkg):
    # a path whose weights rise along it (every merge adds one point: the
    # hierarchy is as deep as it gets), a star (one vertex on every edge) and
    # a random tree, each with 2M points
    for shape in ("path_sorted", "star", "random", "caterpillar"):
        n = 2_000_000
        e = synth.tree_edges(n, 77, shape)
        got = gpu_dendrogram(pkg, edges_tensor(e), n)
        assert_same(pkg, got, oracle.dendrogram(e, n), shape)


def test_untagged_levels(pkg, monkeypatch):
    # Trees below 2^26 edges keep the level number in each union-find, top
    # and lowest-heavy entry, so no level clears them; larger trees clear
    # them every level.  The environment switch selects the cleared form at
    # any size: both must give the oracle's hierarchy.
    monkeypatch.setenv("EMST_DENDROGRAM_UNTAGGED", "1")
    for shape in ("random", "path_sorted", "star", "caterpillar"):
        for ties in (0, 5):
            for idx, n in enumerate((257, 4097, 100_003, 1_000_000)):
                e = synth.tree_edges(n, 500 + 10 * idx + ties, shape, ties=ties)
                got = gpu_dendrogram(pkg, edges_tensor(e), n)
                assert_same(pkg, got, oracle.dendrogram(e, n), f"untagged {shape} ties={ties} n={n}")


@pytest.mark.parametrize("name,make", [
    ("blobs2", lambda: synth.blobs(300_000, 2, 1)),
    ("halos3", lambda: synth.halos(1_000_000, 2)),
    ("lattice_ties", lambda: synth.lattice_ties(200_000, 8_000, side=100)),
])
def test_on_the_emst(pkg, name, make):
    pts = make()
    edges = pkg.emst_compute(torch.from_numpy(pts).cuda())
    torch.cuda.synchronize()
    got = gpu_dendrogram(pkg, edges, len(pts))
    want = oracle.dendrogram(pkg.edges_numpy(edges), len(pts))
    assert_same(pkg, got, want, name)


def test_on_the_mutual_reachability_tree(pkg):
    # HDBSCAN*'s hierarchy: the dendrogram of the §4.5 tree (many equal
    # weights: every point's edges at or below its core distance tie)
    pts = synth.halos(300_000, 5)
    edges, _ = pkg.emst_compute_ex(torch.from_numpy(pts).cuda(), mrd_k=8)
    torch.cuda.synchronize()
    got = gpu_dendrogram(pkg, edges, len(pts))
    want = oracle.dendrogram(pkg.edges_numpy(edges), len(pts))
    assert_same(pkg, got, want, "mrd k=8")


def test_host_buffers_and_partial_outputs(pkg):
    n = 50_000
    e = synth.tree_edges(n, 3, "random", ties=20)
    want = oracle.dendrogram(e, n)
    link, parent = pkg.emst_dendrogram(edges_tensor(e, "cpu"), n)
    assert link.device.type == "cpu" and parent.device.type == "cpu"
    assert_same(pkg, (pkg.linkage_numpy(link), parent.numpy().view(np.uint32)), want, "host")
    link, parent = pkg.emst_dendrogram(edges_tensor(e), n, parent=False)
    torch.cuda.synchronize()
    assert parent is None
    assert np.array_equal(pkg.linkage_numpy(link).view(np.uint32), want[0].view(np.uint32))
    link, parent = pkg.emst_dendrogram(edges_tensor(e), n, linkage=False)
    torch.cuda.synchronize()
    assert link is None
    assert np.array_equal(parent.cpu().numpy().view(np.uint32), want[1])


def test_trivial_sizes(pkg):
    link, parent = pkg.emst_dendrogram(torch.zeros((0, 3), dtype=torch.int32, device="cuda"), 1)
    torch.cuda.synchronize()
    assert link.shape == (0, 4) and parent.cpu().tolist() == [-1]
    link, parent = pkg.emst_dendrogram(torch.zeros((0, 3), dtype=torch.int32, device="cuda"), 0)
    assert link.shape == (0, 4) and parent.shape == (0,)


def test_invalid_trees(pkg):
    n = 3000
    e = synth.tree_edges(n, 9, "random")
    cases = {}
    bad = e.copy(); bad[100]["j"] = n; cases["id out of range"] = bad
    bad = e.copy(); bad[[5, 2000]] = bad[[2000, 5]]; cases["weights out of order"] = bad
    bad = e.copy(); bad[700]["j"] = bad[700]["i"]; cases["loop edge"] = bad
    bad = e.copy(); bad[0]["w"] = np.nan; cases["nan weight"] = bad
    # a repeated edge: ids and order valid, but it closes a cycle (and some
    # point is left without an edge)
    bad = e.copy(); bad[1501] = bad[1500]; cases["cycle"] = bad
    for what, b in cases.items():
        with pytest.raises(ValueError):
            oracle.dendrogram(b, n)
        with pytest.raises(pkg.EmstError) as ei:
            pkg.emst_dendrogram(edges_tensor(b), n)
        assert ei.value.status == -1, what
    # the context is still usable afterwards
    got = gpu_dendrogram(pkg, edges_tensor(e), n)
    assert_same(pkg, got, oracle.dendrogram(e, n), "after errors")


def test_full_size_halos_37M(pkg):
    """The hierarchy of the 37,000,000-point halo EMST (seed 2), as the
    dendrogram benchmark computes it, against the oracle's merge sequence."""
    pts = synth.config_points(3)
    edges = pkg.emst_compute(torch.from_numpy(pts).cuda())
    torch.cuda.synchronize()
    got = gpu_dendrogram(pkg, edges, len(pts))
    want = oracle.dendrogram(pkg.edges_numpy(edges), len(pts))
    assert_same(pkg, got, want, "37M halos")
