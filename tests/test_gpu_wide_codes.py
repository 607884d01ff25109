"""128-bit Morton codes (§4.1's finer Z-curve grid) on the GPU against the
CPU oracle, through the C ABI: codes, order, hierarchy and boxes bit-exact,
and the spanning tree identical to the 64-bit one (the tree does not depend
on the code width)."""
from __future__ import annotations

import os

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


def dev_pts(pts):
    return torch.from_numpy(np.ascontiguousarray(pts)).cuda()


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def dense_clusters(n, dim, seed, sigma=2e-7, n_clusters=40, far=True):
    """Clusters far denser than the 64-bit grid in 3D (cells of 2^-21), at
    positions spread over a large box: the regime §4.1 describes."""
    g = np.random.default_rng(seed)
    scale = 1000.0 if far else 1.0
    centres = g.random((n_clusters, dim)) * scale
    pts = centres[g.integers(0, n_clusters, n)] + g.normal(0, sigma * scale, (n, dim))
    return pts.astype(np.float32)


CASES = [
    ("uniform3", lambda: synth.uniform(5000, 3, 1)),
    ("blobs2", lambda: synth.blobs(7001, 2, 2)),
    ("dense3", lambda: dense_clusters(6000, 3, 3)),
    ("dense2_near_zero", lambda: dense_clusters(4000, 2, 4, sigma=1e-9, far=False)),
    ("lattice_dups", lambda: synth.lattice_ties(n_sites=3000, n_dup=400, side=16, seed=4)),
    ("tiny2", lambda: synth.uniform(2, 3, 5)),
]


def chunk_ranges(refs, n, nc, leaf, first, last):
    is_leaf = refs >= nc - 1
    c = np.clip(refs - (nc - 1), 0, nc - 1)
    v = np.clip(refs, 0, max(nc - 2, 0))
    cf = np.where(is_leaf, c, first[v])
    cl = np.where(is_leaf, c, last[v])
    return cf * leaf, np.minimum((cl + 1) * leaf, n) - 1


@pytest.mark.parametrize("leaf", [1, 4])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_wide_bvh_matches_oracle(pkg, name, make, leaf):
    pts = make()
    n = len(pts)
    if (n + leaf - 1) // leaf < 2:
        pytest.skip("fewer than two leaf chunks")
    ref = oracle.bvh_reference(pts, morton_bits=128)
    out = pkg.emst_build_bvh(dev_pts(pts), leaf_size=leaf, morton_bits=128)
    torch.cuda.synchronize()
    codes = out["codes"].cpu().numpy().view(np.uint64).reshape(n, 2)
    assert np.array_equal(codes, ref["sorted_codes"])
    assert np.array_equal(u32(out["perm"]), ref["perm"])
    nc = (n + leaf - 1) // leaf
    sc = ref["sorted_codes"][::leaf]
    left, right, first, last = oracle.radix_tree128(sc[:, 0], sc[:, 1])
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


@pytest.mark.parametrize("name,make", CASES[:5], ids=[c[0] for c in CASES[:5]])
def test_wide_codes_same_tree(pkg, name, make):
    pts = make()
    a = pkg.edges_numpy(pkg.emst_compute_ex(dev_pts(pts), morton_bits=128)[0])
    b = pkg.edges_numpy(pkg.emst_compute(dev_pts(pts)))
    torch.cuda.synchronize()
    want = oracle.kd_boruvka(pts, threads=os.cpu_count() or 4)
    assert np.array_equal(a.view(np.uint8), want.view(np.uint8)), name
    assert np.array_equal(b.view(np.uint8), want.view(np.uint8)), name


def test_wide_codes_large_dense(pkg):
    pts = dense_clusters(400_000, 3, 9, n_clusters=300)
    a, st = pkg.emst_compute_ex(dev_pts(pts), morton_bits=128, count_visits=True)
    torch.cuda.synchronize()
    want = oracle.kd_boruvka(pts, threads=os.cpu_count() or 4)
    assert np.array_equal(pkg.edges_numpy(a).view(np.uint8), want.view(np.uint8))


def test_wide_codes_with_mrd_and_errors(pkg):
    pts = dense_clusters(5000, 3, 10)
    a = pkg.edges_numpy(pkg.emst_compute_ex(dev_pts(pts), morton_bits=128, mrd_k=4)[0])
    torch.cuda.synchronize()
    want = oracle.prim_mrd(pts, oracle.core_dist2(pts, 4, threads=os.cpu_count() or 4))
    assert np.array_equal(a.view(np.uint8), want.view(np.uint8))
    with pytest.raises(pkg.EmstError) as ei:
        pkg.emst_compute_ex(dev_pts(pts), morton_bits=96)
    assert ei.value.status == -1


def test_automatic_width(pkg):
    dense = synth.dense(200_000, 3, 5)
    a, st = pkg.emst_compute_ex(dev_pts(dense))
    torch.cuda.synchronize()
    assert st["morton_bits"] == 128 and st["code_collisions"] * 64 > len(dense)
    want = oracle.kd_boruvka(dense, threads=os.cpu_count() or 4)
    assert np.array_equal(pkg.edges_numpy(a).view(np.uint8), want.view(np.uint8))
    halos = synth.halos(200_000, 2)
    b, st = pkg.emst_compute_ex(dev_pts(halos))
    c, st64 = pkg.emst_compute_ex(dev_pts(halos), morton_bits=64)
    torch.cuda.synchronize()
    assert st["morton_bits"] == 64 and st["code_collisions"] * 64 <= len(halos)
    assert st64["morton_bits"] == 64 and st64["code_collisions"] == st["code_collisions"]
    assert np.array_equal(pkg.edges_numpy(b).view(np.uint8), pkg.edges_numpy(c).view(np.uint8))
