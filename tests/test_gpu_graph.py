"""Graph rounds (emst_options.use_graph): the rounds after the first run as
one CUDA graph whose while node is ended by a flag the device sets.  The
tree must be the oracle's, bit for bit, and the same as the host loop's, in
every form the rounds serve (single, batched, mutual reachability, the
persistent traversal), on the caller's stream whatever it is.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 4


@pytest.fixture(scope="module")
def pkg():
    import paper_2207_00514_gb300 as p
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p.load_library()
    return p


def same(a, b):
    return np.array_equal(np.asarray(a).view(np.uint8), np.asarray(b).view(np.uint8))


def run(pkg, pts, **opt):
    e, st = pkg.emst_compute_ex(torch.from_numpy(np.ascontiguousarray(pts)).cuda(), **opt)
    torch.cuda.synchronize()
    return pkg.edges_numpy(e), st


CASES = [
    ("uniform3_10k", lambda: synth.uniform(10_000, 3, 0)),
    ("blobs2_30k", lambda: synth.blobs(30_001, 2, 1)),
    ("halos3_200k", lambda: synth.halos(200_003, 5)),
    ("lattice_ties", lambda: synth.lattice_ties(n_sites=7000, n_dup=600, side=20, seed=9)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_graph_rounds_match_oracle_and_host_loop(pkg, name, make):
    pts = make()
    want = oracle.emst(pts, threads=THREADS)
    got, st = run(pkg, pts, use_graph=True)
    assert same(got, want), name
    host, st_host = run(pkg, pts, use_graph=False)
    assert same(host, want), name
    # the device-side loop ran exactly the host loop's rounds
    assert st["rounds"] == st_host["rounds"], (st["rounds"], st_host["rounds"])


@pytest.mark.parametrize("n", [2, 3, 5, 33, 1000])
def test_graph_rounds_small(pkg, n):
    # n = 2 finishes in round 0 (no graph); the others in a few graph rounds,
    # including an odd and an even number of them
    pts = synth.uniform(n, 3, 100 + n)
    got, _ = run(pkg, pts, use_graph=True)
    assert same(got, oracle.prim(pts)), n


def test_graph_rounds_persistent_traversal(pkg):
    pts = synth.halos(150_000, 6)
    got, st = run(pkg, pts, use_graph=True, traversal=2, ignore_tuning=True)
    assert st["traversal_used"] == 2
    assert same(got, oracle.emst(pts, threads=THREADS))


def test_graph_rounds_mutual_reachability(pkg):
    pts = synth.blobs(20_000, 3, 8)
    got, _ = run(pkg, pts, use_graph=True, mrd_k=5)
    host, _ = run(pkg, pts, use_graph=False, mrd_k=5)
    assert same(got, host)
    core2 = pkg.emst_core_distances(torch.from_numpy(pts).cuda(), 5)
    torch.cuda.synchronize()
    want = oracle.kd_boruvka_mrd(pts, core2.cpu().numpy(), threads=THREADS)
    assert same(got, want)


def test_graph_rounds_batched(pkg):
    sizes = synth.batched_sizes(48, seed=11, lo=2, hi=30_000)
    pts, offsets = synth.batched_instances(sizes, seed=11)
    dp = torch.from_numpy(pts).cuda()
    e, eo, st = pkg.emst_compute_batched_ex(dp, offsets, use_graph=True)
    e0, eo0, st0 = pkg.emst_compute_batched_ex(dp, offsets, use_graph=False)
    torch.cuda.synchronize()
    got, host = pkg.edges_numpy(e), pkg.edges_numpy(e0)
    assert np.array_equal(eo, eo0)
    assert same(got, host)
    assert st["rounds"] == st0["rounds"]
    for k in (0, 7, 47):
        part = pts[offsets[k]:offsets[k + 1]]
        assert same(got[eo[k]:eo[k + 1]], oracle.emst(part, threads=THREADS)), k


def test_graph_rounds_on_streams(pkg):
    # the legacy default stream cannot be captured: the library captures on
    # streams of its own and launches the graph on the caller's
    pts = synth.halos(60_000, 12)
    want = oracle.emst(pts, threads=THREADS)
    dp = torch.from_numpy(pts).cuda()
    s = torch.cuda.Stream()
    for stream in (None, s):
        out = torch.empty((pts.shape[0] - 1, 3), dtype=torch.int32, device="cuda")
        if stream is None:
            pkg.emst_compute_ex(dp, out_edges=out, use_graph=True)
        else:
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                pkg.emst_compute_ex(dp, out_edges=out, stream=s, use_graph=True)
        torch.cuda.synchronize()
        assert same(pkg.edges_numpy(out), want)


def test_graph_rounds_host_buffers_repeated(pkg):
    pts = synth.blobs(40_000, 3, 13)
    want = oracle.emst(pts, threads=THREADS)
    for _ in range(3):
        got, _ = pkg.emst_compute_ex(torch.from_numpy(pts), use_graph=True)
        assert same(pkg.edges_numpy(got), want)
