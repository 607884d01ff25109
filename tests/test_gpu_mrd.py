"""Mutual reachability distance (§4.5) on the GPU against the CPU oracle,
through the C ABI: core distances bit-exact, and the mutual-reachability
minimum spanning tree bit-exact (ids and FP32 weight bits)."""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
import synth
from fp32ref import weight32

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


def assert_same_edges(got, want, what=""):
    g = got.view(np.uint8).reshape(-1, 12)
    w = want.view(np.uint8).reshape(-1, 12)
    assert g.shape == w.shape, (what, g.shape, w.shape)
    rows = np.nonzero((g != w).any(1))[0]
    assert len(rows) == 0, f"{what}: {len(rows)} edges differ, first {rows[:5]}"


def gpu_core(pkg, pts, k):
    c = pkg.emst_core_distances(dev_pts(pts), k)
    torch.cuda.synchronize()
    return c.cpu().numpy()


def gpu_mrd(pkg, pts, k, **kw):
    e, st = pkg.emst_compute_ex(dev_pts(pts), mrd_k=k, **kw)
    torch.cuda.synchronize()
    return pkg.edges_numpy(e), st


def _lattice(n, side, seed):
    g = np.random.default_rng(seed)
    return (g.integers(0, side, size=(n, 3)) / float(side)).astype(np.float32)


CORE_CASES = [
    ("uniform3", lambda: synth.uniform(3001, 3, 1)),
    ("blobs2", lambda: synth.blobs(4099, 2, 2)),
    ("halos3", lambda: synth.halos(5000, 7)),
    ("lattice_dups", lambda: _lattice(3000, 10, 3)),
]


@pytest.mark.parametrize("name,make", CORE_CASES)
def test_core_distances_small(pkg, name, make):
    p = make()
    for k in (1, 2, 3, 5, 8, 9, 16, 17, 32):
        got = gpu_core(pkg, p, k)
        want = oracle.core_dist2(p, k, threads=os.cpu_count() or 4)
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), (name, k)


def test_core_distances_large(pkg):
    p = synth.halos(400_000, 11)
    for k in (2, 4, 16):
        got = gpu_core(pkg, p, k)
        want = oracle.core_dist2(p, k, threads=os.cpu_count() or 4)
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), k


def test_core_distances_host_buffers_and_tiny(pkg):
    p = synth.uniform(700, 2, 5)
    out = torch.empty(len(p), dtype=torch.float32).pin_memory()
    pkg.emst_core_distances(torch.from_numpy(p), 6, out=out)
    torch.cuda.synchronize()
    assert np.array_equal(out.numpy(), oracle.core_dist2(p, 6, brute=True))
    one = pkg.emst_core_distances(dev_pts(np.zeros((1, 3), np.float32)), 1)
    assert float(one.cpu()[0]) == 0.0
    two = gpu_core(pkg, np.array([[0, 0], [3, 4]], np.float32), 2)
    assert list(two) == [25.0, 25.0]


@pytest.mark.parametrize("name,make", CORE_CASES)
def test_mrd_tree_small(pkg, name, make):
    p = make()
    for k in (2, 4, 16):
        got, st = gpu_mrd(pkg, p, k)
        want = oracle.prim_mrd(p, oracle.core_dist2(p, k, threads=os.cpu_count() or 4))
        assert_same_edges(got, want, f"{name} k={k}")
        assert st["core_ms"] > 0


def test_mrd_k1_is_the_emst(pkg):
    p = synth.blobs(20_000, 3, 4)
    got, _ = gpu_mrd(pkg, p, 1)
    plain = pkg.edges_numpy(pkg.emst_compute(dev_pts(p)))
    torch.cuda.synchronize()
    assert_same_edges(got, plain, "k=1")


@pytest.mark.parametrize("k,leaf", [(2, 1), (5, 1), (16, 1), (4, 4)])
def test_mrd_tree_large_vs_kd_oracle(pkg, k, leaf):
    p = synth.halos(300_000, 12)
    got, _ = gpu_mrd(pkg, p, k, leaf_size=leaf)
    threads = os.cpu_count() or 4
    c = oracle.core_dist2(p, k, threads=threads)
    want = oracle.kd_boruvka_mrd(p, c, threads=threads)
    assert_same_edges(got, want, f"k={k} leaf={leaf}")
    # every weight is the mutual reachability of its endpoints
    i, j = got["i"].astype(np.int64), got["j"].astype(np.int64)
    ew = np.maximum(np.maximum(c[i], c[j]), weight32(p[i], p[j]))
    assert np.array_equal(got["w"], ew)


def test_mrd_host_buffers(pkg):
    p = synth.blobs(5000, 2, 8)
    out = torch.empty((len(p) - 1, 3), dtype=torch.int32).pin_memory()
    pkg.emst_compute_ex(torch.from_numpy(p), out_edges=out, mrd_k=3)
    torch.cuda.synchronize()
    want = oracle.prim_mrd(p, oracle.core_dist2(p, 3, brute=True))
    assert_same_edges(pkg.edges_numpy(out), want, "host")


def test_mrd_argument_errors(pkg):
    p = dev_pts(synth.uniform(100, 3, 1))
    for kw in (dict(mrd_k=33), dict(mrd_k=-1), dict(mrd_k=101)):
        with pytest.raises(pkg.EmstError) as ei:
            pkg.emst_compute_ex(p, **kw)
        assert ei.value.status == -1
    for k in (0, 33, 101):
        with pytest.raises(pkg.EmstError):
            pkg.emst_core_distances(p, k)
