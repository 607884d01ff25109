"""emst_compute_noalloc: the allocation-free entry point, through the C ABI.

It serves callers that cannot allocate device memory where they need the
tree (an execute hook that must not allocate, a process under a device-memory
budget it does not own, a latency-critical loop).  Its scratch is one fixed
array inside the library, shared by every call on a device and left holding
the previous call's contents, so the test calls it twice in a row on
different inputs and compares each result, edge for edge and bit for bit,
with emst_compute on the same points.  This file is collected last on
purpose: if it fails, every other test has already run.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    import paper_2207_00514_gb300 as pkg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return pkg, pkg.load_library()


def _run(lib_, fn, pts):
    n, dim = pts.shape
    out = torch.empty((n - 1, 3), dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = fn(ctypes.c_void_p(pts.data_ptr()), n, dim, ctypes.c_void_p(out.data_ptr()), stream)
    torch.cuda.synchronize()
    return rc, out.cpu().numpy()


def _run_host(fn, pts_np):
    """The same call with plain (pageable) host buffers for the points and
    the edges: the library stages both through its scratch."""
    n, dim = pts_np.shape
    pts_np = np.ascontiguousarray(pts_np, dtype=np.float32)
    out = np.zeros((n - 1, 3), np.int32)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = fn(ctypes.c_void_p(pts_np.ctypes.data), n, dim, ctypes.c_void_p(out.ctypes.data), stream)
    torch.cuda.synchronize()
    return rc, out


@pytest.mark.gpu
def test_noalloc_matches_emst_compute_twice_in_a_row(lib):
    pkg, L = lib
    cases = [synth.halos(40_000, 21), synth.blobs(65_536, 2, 22)]  # the second fills the limit
    for pts_np in cases:
        pts = torch.from_numpy(pts_np).cuda()
        rc_ref, ref = _run(L, L.emst_compute, pts)
        rc_na, got = _run(L, L.emst_compute_noalloc, pts)
        assert rc_ref == 0 and rc_na == 0
        assert np.array_equal(got, ref)


@pytest.mark.gpu
def test_noalloc_host_buffers_at_the_size_limit(lib):
    """Host input and host output at exactly EMST_NOALLOC_MAX_POINTS in 3D:
    the largest layout the fixed scratch has to hold (the point and edge
    staging copies included), twice in a row."""
    pkg, L = lib
    n = pkg.EMST_NOALLOC_MAX_POINTS
    for seed in (23, 24):
        pts_np = synth.halos(n, seed)
        rc_ref, ref = _run_host(L.emst_compute, pts_np)
        rc_na, got = _run_host(L.emst_compute_noalloc, pts_np)
        assert rc_ref == 0 and rc_na == 0
        assert np.array_equal(got, ref)


@pytest.mark.gpu
def test_noalloc_on_code_collisions_and_duplicates(lib):
    """Very dense clusters, where emst_compute rebuilds with 128-bit codes
    and the allocation-free path keeps 64-bit ones, and a lattice with
    duplicate points (zero-weight ties): the same trees, bit for bit."""
    pkg, L = lib
    dense = synth.dense(pkg.EMST_NOALLOC_MAX_POINTS, 3, 7, n_clusters=200)
    _, st = pkg.emst_compute_ex(torch.from_numpy(dense).cuda())
    assert st["morton_bits"] == 128  # the case really takes the other code width there
    lattice = synth.lattice_ties(n_sites=62_915, n_dup=2_621, side=40, seed=8)
    for pts_np in (dense, lattice):
        pts = torch.from_numpy(pts_np).cuda()
        rc_ref, ref = _run(L, L.emst_compute, pts)
        rc_na, got = _run(L, L.emst_compute_noalloc, pts)
        assert rc_ref == 0 and rc_na == 0
        assert np.array_equal(got, ref)


@pytest.mark.gpu
def test_noalloc_rejects_sizes_beyond_its_limit(lib):
    pkg, L = lib
    n = pkg.EMST_NOALLOC_MAX_POINTS + 1
    pts = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    rc, _ = _run(L, L.emst_compute_noalloc, pts)
    assert rc == -7
    assert "noalloc" in pkg.emst_status_string(rc)
