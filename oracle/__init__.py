"""CPU oracle for the single-tree Boruvka EMST -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (the CUDA library and its
Python binding) never imports it and shares no code with it.

The arithmetic lives in ``emst_oracle.c`` (plain C, compiled here with gcc and
``-ffp-contract=off``); this module only builds it and marshals numpy arrays.
Every C function cites the passage of the paper it follows.  Parity pins: see
``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "emst_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

EDGE_DTYPE = np.dtype([("i", np.uint32), ("j", np.uint32), ("w", np.float32)])
INVALID = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, no fma contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
               _SRC, "-o", tmp, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            I = ctypes.c_int
            sig = {
                "oracle_weight": (ctypes.c_float, [P, P, I]),
                "oracle_canonical_sort": (None, [P, I64]),
                "oracle_prim": (I, [P, I64, I, P]),
                "oracle_kruskal": (I, [P, I64, I, P]),
                "oracle_scene_box": (I, [P, I64, I, P, P]),
                "oracle_morton": (None, [P, I64, I, P, P, P]),
                "oracle_sort_perm": (None, [P, I64, P]),
                "oracle_radix_tree": (None, [P, I64, P, P, P, P]),
                "oracle_node_boxes": (None, [P, P, P, I64, I, P, P]),
                "oracle_node_labels": (None, [P, P, P, I64, P]),
                "oracle_upper_bounds": (None, [P, P, I64, I, P]),
                "oracle_nn_other": (None, [P, P, P, P, I64, I, P, P]),
                "oracle_component_min": (None, [P, P, P, P, I64, P, P, P]),
                "oracle_merge": (I64, [P, P, P, P, P, I64, P, P]),
                "oracle_boruvka_steps": (I, [P, P, I64, I, P, P]),
                "oracle_kd_boruvka": (I, [P, I64, I, P, I, P]),
                "oracle_prim_mrd": (I, [P, P, I64, I, P]),
                "oracle_kruskal_mrd": (I, [P, P, I64, I, P]),
                "oracle_kd_boruvka_mrd": (I, [P, P, I64, I, P, I, P]),
                "oracle_core_dist2_brute": (I, [P, I64, I, I, P]),
                "oracle_kd_core_dist2": (I, [P, I64, I, I, P, I]),
                "oracle_morton128": (None, [P, I64, I, P, P, P, P]),
                "oracle_sort_perm128": (None, [P, P, I64, P]),
                "oracle_radix_tree128": (None, [P, P, I64, P, P, P, P]),
                "oracle_count_components": (I64, [P, I64, I64, P]),
                "oracle_dendrogram": (I, [P, I64, P, P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else ctypes.c_void_p(0)


def _pts(points):
    p = np.ascontiguousarray(points, dtype=np.float32)
    assert p.ndim == 2 and p.shape[1] in (2, 3)
    return p


def _edges(m):
    return np.zeros(max(m, 0), dtype=EDGE_DTYPE)


def weight(p, q) -> np.float32:
    p = np.ascontiguousarray(p, dtype=np.float32)
    q = np.ascontiguousarray(q, dtype=np.float32)
    return np.float32(_load().oracle_weight(_p(p), _p(q), len(p)))


def canonical(edges) -> np.ndarray:
    e = np.array(edges, dtype=EDGE_DTYPE, copy=True)
    _load().oracle_canonical_sort(_p(e), len(e))
    return e


def prim(points) -> np.ndarray:
    """EMST by O(n^2) Prim, canonical order."""
    p = _pts(points)
    n = len(p)
    e = _edges(n - 1)
    rc = _load().oracle_prim(_p(p), n, p.shape[1], _p(e))
    assert rc == 0
    return canonical(e)


def kruskal(points) -> np.ndarray:
    p = _pts(points)
    n = len(p)
    e = _edges(n - 1)
    rc = _load().oracle_kruskal(_p(p), n, p.shape[1], _p(e))
    assert rc == 0, rc
    return canonical(e)


def kd_boruvka(points, threads: int = 1, return_rounds: bool = False):
    p = _pts(points)
    n = len(p)
    e = _edges(n - 1)
    rounds = np.zeros(1, dtype=np.int64)
    rc = _load().oracle_kd_boruvka(_p(p), n, p.shape[1], _p(e), int(threads), _p(rounds))
    assert rc == 0, rc
    e = canonical(e)
    return (e, int(rounds[0])) if return_rounds else e


def core_dist2(points, k: int, brute: bool = False, threads: int = 1) -> np.ndarray:
    """Squared core distances (§4.5): the (k-1)-th smallest FP32 weight from
    each point to the others (the point itself is the first neighbour), by a
    full selection (brute) or the k-d tree."""
    p = _pts(points)
    n = len(p)
    out = np.zeros(n, dtype=np.float32)
    if brute:
        rc = _load().oracle_core_dist2_brute(_p(p), n, p.shape[1], int(k), _p(out))
    else:
        rc = _load().oracle_kd_core_dist2(_p(p), n, p.shape[1], int(k), _p(out), int(threads))
    assert rc == 0, rc
    return out


def _core(core2, n):
    c = np.ascontiguousarray(core2, dtype=np.float32)
    assert c.shape == (n,)
    return c


def prim_mrd(points, core2) -> np.ndarray:
    """Mutual-reachability MST (§4.5) by O(n^2) Prim, canonical order."""
    p = _pts(points)
    n = len(p)
    e = _edges(n - 1)
    rc = _load().oracle_prim_mrd(_p(p), _p(_core(core2, n)), n, p.shape[1], _p(e))
    assert rc == 0
    return canonical(e)


def kruskal_mrd(points, core2) -> np.ndarray:
    p = _pts(points)
    n = len(p)
    e = _edges(n - 1)
    rc = _load().oracle_kruskal_mrd(_p(p), _p(_core(core2, n)), n, p.shape[1], _p(e))
    assert rc == 0
    return canonical(e)


def kd_boruvka_mrd(points, core2, threads: int = 1) -> np.ndarray:
    p = _pts(points)
    n = len(p)
    e = _edges(n - 1)
    rounds = np.zeros(1, dtype=np.int64)
    rc = _load().oracle_kd_boruvka_mrd(_p(p), _p(_core(core2, n)), n, p.shape[1], _p(e),
                                       int(threads), _p(rounds))
    assert rc == 0, rc
    return canonical(e)


def boruvka_steps(points, orig_ids=None, return_rounds: bool = False):
    """Boruvka through the per-step definitions with brute-force queries."""
    p = _pts(points)
    n = len(p)
    e = _edges(n - 1)
    ids = None if orig_ids is None else np.ascontiguousarray(orig_ids, dtype=np.uint32)
    rounds = np.zeros(1, dtype=np.int64)
    rc = _load().oracle_boruvka_steps(_p(p), _p(ids), n, p.shape[1], _p(e), _p(rounds))
    assert rc == 0, rc
    e = canonical(e)
    return (e, int(rounds[0])) if return_rounds else e


def emst(points, threads: int = 1) -> np.ndarray:
    """The oracle's EMST: Prim for n <= 20000, else the k-d tree Boruvka."""
    p = _pts(points)
    if len(p) <= 20000:
        return prim(p)
    return kd_boruvka(p, threads=threads)


def scene_box(points):
    p = _pts(points)
    d = p.shape[1]
    lo = np.zeros(d, np.float32)
    hi = np.zeros(d, np.float32)
    finite = _load().oracle_scene_box(_p(p), len(p), d, _p(lo), _p(hi))
    return lo, hi, bool(finite)


def morton(points, lo, hi) -> np.ndarray:
    p = _pts(points)
    lo = np.ascontiguousarray(lo, np.float32)
    hi = np.ascontiguousarray(hi, np.float32)
    codes = np.zeros(len(p), np.uint64)
    _load().oracle_morton(_p(p), len(p), p.shape[1], _p(lo), _p(hi), _p(codes))
    return codes


def morton128(points, lo, hi):
    """128-bit codes (42 bits per dimension in 3D, 64 in 2D, FP64 quantiser):
    (high words, low words)."""
    p = _pts(points)
    lo = np.ascontiguousarray(lo, np.float32)
    hi = np.ascontiguousarray(hi, np.float32)
    ch = np.zeros(len(p), np.uint64)
    cl = np.zeros(len(p), np.uint64)
    _load().oracle_morton128(_p(p), len(p), p.shape[1], _p(lo), _p(hi), _p(ch), _p(cl))
    return ch, cl


def sort_perm128(code_hi, code_lo) -> np.ndarray:
    h = np.ascontiguousarray(code_hi, np.uint64)
    l = np.ascontiguousarray(code_lo, np.uint64)
    perm = np.zeros(len(h), np.uint32)
    _load().oracle_sort_perm128(_p(h), _p(l), len(h), _p(perm))
    return perm


def radix_tree128(sorted_hi, sorted_lo):
    h = np.ascontiguousarray(sorted_hi, np.uint64)
    l = np.ascontiguousarray(sorted_lo, np.uint64)
    n = len(h)
    m = max(n - 1, 0)
    left, right, first, last = (np.zeros(m, np.int64) for _ in range(4))
    _load().oracle_radix_tree128(_p(h), _p(l), n, _p(left), _p(right), _p(first), _p(last))
    return left, right, first, last


def sort_perm(codes) -> np.ndarray:
    c = np.ascontiguousarray(codes, np.uint64)
    perm = np.zeros(len(c), np.uint32)
    _load().oracle_sort_perm(_p(c), len(c), _p(perm))
    return perm


def radix_tree(sorted_codes):
    """(left, right, first, last) per internal node; child refs: internal id
    in [0, n-1), leaf k as n-1+k."""
    c = np.ascontiguousarray(sorted_codes, np.uint64)
    n = len(c)
    m = max(n - 1, 0)
    left = np.zeros(m, np.int64)
    right = np.zeros(m, np.int64)
    first = np.zeros(m, np.int64)
    last = np.zeros(m, np.int64)
    _load().oracle_radix_tree(_p(c), n, _p(left), _p(right), _p(first), _p(last))
    return left, right, first, last


def node_boxes(sorted_points, first, last):
    p = _pts(sorted_points)
    n, d = p.shape
    lo = np.zeros((max(n - 1, 0), d), np.float32)
    hi = np.zeros((max(n - 1, 0), d), np.float32)
    f = np.ascontiguousarray(first, np.int64)
    l = np.ascontiguousarray(last, np.int64)
    _load().oracle_node_boxes(_p(p), _p(f), _p(l), n, d, _p(lo), _p(hi))
    return lo, hi


def node_labels(labels, first, last):
    lab = np.ascontiguousarray(labels, np.uint32)
    n = len(lab)
    out = np.zeros(max(n - 1, 0), np.uint32)
    f = np.ascontiguousarray(first, np.int64)
    l = np.ascontiguousarray(last, np.int64)
    _load().oracle_node_labels(_p(lab), _p(f), _p(l), n, _p(out))
    return out


def upper_bounds(sorted_points, labels):
    p = _pts(sorted_points)
    lab = np.ascontiguousarray(labels, np.uint32)
    ub = np.zeros(len(p), np.float32)
    _load().oracle_upper_bounds(_p(p), _p(lab), len(p), p.shape[1], _p(ub))
    return ub


def nn_other(sorted_points, orig_ids, labels, radius):
    p = _pts(sorted_points)
    n = len(p)
    ids = np.ascontiguousarray(orig_ids, np.uint32)
    lab = np.ascontiguousarray(labels, np.uint32)
    rad = np.ascontiguousarray(radius, np.float32)
    w = np.zeros(n, np.float32)
    j = np.zeros(n, np.int64)
    _load().oracle_nn_other(_p(p), _p(ids), _p(lab), _p(rad), n, p.shape[1], _p(w), _p(j))
    return w, j


def component_min(labels, orig_ids, res_w, res_j):
    lab = np.ascontiguousarray(labels, np.uint32)
    n = len(lab)
    ids = np.ascontiguousarray(orig_ids, np.uint32)
    rw = np.ascontiguousarray(res_w, np.float32)
    rj = np.ascontiguousarray(res_j, np.int64)
    cw = np.zeros(n, np.float32)
    ca = np.zeros(n, np.int64)
    cb = np.zeros(n, np.int64)
    _load().oracle_component_min(_p(lab), _p(ids), _p(rw), _p(rj), n, _p(cw), _p(ca), _p(cb))
    return cw, ca, cb


def merge(labels, comp_a, comp_b, comp_w, orig_ids):
    lab = np.ascontiguousarray(labels, np.uint32)
    n = len(lab)
    ca = np.ascontiguousarray(comp_a, np.int64)
    cb = np.ascontiguousarray(comp_b, np.int64)
    cw = np.ascontiguousarray(comp_w, np.float32)
    ids = np.ascontiguousarray(orig_ids, np.uint32)
    new = np.zeros(n, np.uint32)
    e = _edges(n)
    m = _load().oracle_merge(_p(lab), _p(ca), _p(cb), _p(cw), _p(ids), n, _p(new), _p(e))
    assert m >= 0
    return new, e[:m]


def count_components(edges, n):
    e = np.ascontiguousarray(edges, dtype=EDGE_DTYPE)
    cyc = ctypes.c_int(0)
    comps = _load().oracle_count_components(_p(e), len(e), int(n), ctypes.byref(cyc))
    return int(comps), bool(cyc.value)


LINKAGE_DTYPE = np.dtype([("a", np.uint32), ("b", np.uint32), ("w", np.float32), ("size", np.uint32)])


def dendrogram(edges, n):
    """Single-linkage hierarchy of a spanning tree given in merge order:
    (linkage rows {a, b, w, size}, parent of each of the 2n - 1 clusters).
    Raises ValueError on an invalid tree or a decreasing weight."""
    e = np.ascontiguousarray(edges, dtype=EDGE_DTYPE)
    n = int(n)
    assert len(e) == max(n - 1, 0)
    link = np.zeros(max(n - 1, 0), dtype=LINKAGE_DTYPE)
    parent = np.zeros(max(2 * n - 1, 0), dtype=np.uint32)
    rc = _load().oracle_dendrogram(_p(e), n, _p(link), _p(parent))
    if rc != 0:
        raise ValueError(f"not a spanning tree in weight order (rc {rc})")
    return link, parent


def bvh_reference(points, morton_bits: int = 64):
    """Steps A1-A4 end to end: scene box, codes, stable order, radix tree and
    node boxes.  Returns a dict of numpy arrays (sorted order throughout);
    with 128-bit codes `codes` / `sorted_codes` hold (high, low) word pairs."""
    p = _pts(points)
    lo, hi, finite = scene_box(p)
    if morton_bits == 128:
        ch, cl = morton128(p, lo, hi)
        perm = sort_perm128(ch, cl)
        codes = np.stack([ch, cl], 1)
        sc = codes[perm]
        left, right, first, last = radix_tree128(sc[:, 0], sc[:, 1])
        sp = p[perm]
        blo, bhi = node_boxes(sp, first, last)
        return dict(lo=lo, hi=hi, codes=codes, perm=perm, sorted_codes=sc, left=left,
                    right=right, first=first, last=last, box_lo=blo, box_hi=bhi,
                    sorted_points=sp)
    codes = morton(p, lo, hi)
    perm = sort_perm(codes)
    sc = codes[perm]
    left, right, first, last = radix_tree(sc)
    sp = p[perm]
    blo, bhi = node_boxes(sp, first, last)
    return dict(lo=lo, hi=hi, codes=codes, perm=perm, sorted_codes=sc, left=left, right=right,
                first=first, last=last, box_lo=blo, box_hi=bhi, sorted_points=sp)
