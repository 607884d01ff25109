"""Python binding of libemst.so (include/emst.h): single-tree Boruvka EMST on a GB300.

Argument marshalling only: every step of the method runs in the CUDA library.
Tensors are torch tensors (device memory, or host memory for the end-to-end
path); the CUDA stream defaults to torch's current stream.  There is no CPU
fallback: a missing or unloadable library raises ``EmstLibraryError``.

Edges come back as an (m, 3) int32 tensor: columns i, j (original indices,
i < j) and the FP32 bits of w (``edges_w(t)`` views them as float32), in
(w, i, j) order.  ``edges_numpy`` turns them into a structured numpy array
with fields i, j, w.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

__all__ = [
    "EmstError",
    "EmstLibraryError",
    "EMST_MAX_POINTS",
    "library_path",
    "load_library",
    "emst_compute",
    "emst_compute_ex",
    "emst_compute_batched",
    "emst_compute_batched_ex",
    "emst_core_distances",
    "EMST_MRD_MAX_K",
    "emst_compute_noalloc",
    "EMST_NOALLOC_MAX_POINTS",
    "emst_status_string",
    "emst_build_bvh",
    "emst_build_bvh_ex",
    "emst_round_step",
    "edges_w",
    "EMST_MLP_PARAMS",
    "EMST_MLP_FEATURES",
    "emst_mlp_forward",
    "emst_mlp_grad",
    "emst_mlp_adam",
    "emst_learned_samples",
    "edges_numpy",
    "EDGE_DTYPE",
    "emst_dendrogram",
    "linkage_numpy",
    "LINKAGE_DTYPE",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libemst.so")
_HEADER = os.path.join(os.path.dirname(_HERE), "include", "emst.h")
EMST_MAX_POINTS = (1 << 30) - 1
EMST_MLP_PARAMS = 8981
EMST_MLP_FEATURES = 8
EMST_MRD_MAX_K = 32
EDGE_DTYPE = np.dtype([("i", np.uint32), ("j", np.uint32), ("w", np.float32)])
LINKAGE_DTYPE = np.dtype([("a", np.uint32), ("b", np.uint32), ("w", np.float32), ("size", np.uint32)])
INVALID = 0xFFFFFFFF


class EmstError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: emst status {status} ({emst_status_string(status)})")


class EmstLibraryError(RuntimeError):
    pass


class _Options(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_int32), ("block_size", ctypes.c_int32),
                ("carried_radius", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("count_visits", ctypes.c_int32), ("leaf_size", ctypes.c_int32),
                ("mlp_params", ctypes.c_void_p), ("mrd_k", ctypes.c_int32),
                ("morton_bits", ctypes.c_int32), ("traversal", ctypes.c_int32),
                ("refill_lanes", ctypes.c_int32), ("queue_chunk", ctypes.c_int32),
                ("ignore_tuning", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2)]


class _Stats(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_int32), ("rounds", ctypes.c_int32),
                ("kernel_launches", ctypes.c_int32), ("morton_bits", ctypes.c_int32),
                ("total_ms", ctypes.c_double), ("build_ms", ctypes.c_double),
                ("rounds_ms", ctypes.c_double), ("output_ms", ctypes.c_double),
                ("node_visits", ctypes.c_int64), ("components_per_round", ctypes.c_int64 * 40),
                ("traverse_ms", ctypes.c_double), ("traverse_launches", ctypes.c_int32),
                ("reserved1", ctypes.c_int32), ("round_traverse_ms", ctypes.c_double * 40),
                ("queried_points", ctypes.c_int64), ("rerun_points", ctypes.c_int64),
                ("learned_search_ms", ctypes.c_double), ("core_ms", ctypes.c_double),
                ("code_collisions", ctypes.c_int64), ("reserved", ctypes.c_int64 * 1),
                ("round_visits", ctypes.c_int64 * 40), ("round_queries", ctypes.c_int64 * 40),
                ("round_distinct_nodes", ctypes.c_int64 * 40),
                ("traversal_used", ctypes.c_int32), ("block_used", ctypes.c_int32),
                ("leaf_used", ctypes.c_int32), ("tuned", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _LIB_PATH


def load_library(path: str | None = None):
    """Load libemst.so (built in-tree by ``__graft_entry__.build()``)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or _LIB_PATH
        if not os.path.exists(p):
            raise EmstLibraryError(f"libemst.so not built ({p}); run __graft_entry__.build()")
        try:
            lib = ctypes.CDLL(p)
        except OSError as e:  # pragma: no cover - depends on the machine
            raise EmstLibraryError(f"cannot load {p}: {e}") from e
        V, I64, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        lib.emst_compute.argtypes = [V, I64, I, V, V]
        lib.emst_compute.restype = I
        lib.emst_compute_ex.argtypes = [V, I64, I, V, V, ctypes.POINTER(_Options), ctypes.POINTER(_Stats)]
        lib.emst_compute_ex.restype = I
        lib.emst_compute_batched.argtypes = [V, V, I, I, V, V, V]
        lib.emst_compute_batched.restype = I
        lib.emst_compute_batched_ex.argtypes = [V, V, I, I, V, V, V, ctypes.POINTER(_Options),
                                                ctypes.POINTER(_Stats)]
        lib.emst_compute_batched_ex.restype = I
        lib.emst_build_bvh_ex.argtypes = [V, I64, I, I, I, V, V, V, V, V]
        lib.emst_build_bvh_ex.restype = I
        lib.emst_core_distances.argtypes = [V, I64, I, I, V, V]
        lib.emst_dendrogram.restype = I
        lib.emst_dendrogram.argtypes = [V, I64, V, V, V]
        lib.emst_core_distances.restype = I
        lib.emst_status_string.argtypes = [I]
        lib.emst_status_string.restype = ctypes.c_char_p
        lib.emst_build_bvh.argtypes = [V, I64, I, I, V, V, V, V, V]
        lib.emst_build_bvh.restype = I
        lib.emst_round_step.argtypes = [V, I64, I, I, V, V, V, V, V, V, V, V, ctypes.POINTER(I64), V]
        lib.emst_round_step.restype = I
        lib.emst_compute_noalloc.argtypes = [V, I64, I, V, V]
        lib.emst_compute_noalloc.restype = I
        lib.emst_mlp_forward.argtypes = [V, I64, V, V, V]
        lib.emst_mlp_forward.restype = I
        lib.emst_mlp_grad.argtypes = [V, V, I64, V, V, V, V]
        lib.emst_mlp_grad.restype = I
        F = ctypes.c_float
        lib.emst_mlp_adam.argtypes = [V, V, V, V, I, F, F, F, F, V]
        lib.emst_mlp_adam.restype = I
        lib.emst_learned_samples.argtypes = [V, I64, I, I, V, V, I64, ctypes.POINTER(I64), V]
        lib.emst_learned_samples.restype = I
        if path is None:
            _lib = lib
        return lib


def declared_functions(header: str = _HEADER):
    """Names of the functions include/emst.h declares."""
    txt = open(header).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(emst_[a-z_]+)\s*\(", txt)))


def emst_status_string(status: int) -> str:
    try:
        return load_library().emst_status_string(int(status)).decode()
    except EmstLibraryError:
        return "library not loaded"


# ----------------------------------------------------------------------------
def _torch():
    import torch
    return torch


def _stream_ptr(stream, device):
    torch = _torch()
    if stream is None:
        if device.type == "cuda":
            return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _check_points(points):
    torch = _torch()
    if not isinstance(points, torch.Tensor):
        raise TypeError("points must be a torch tensor")
    if points.dtype != torch.float32 or points.dim() != 2 or points.shape[1] not in (2, 3):
        raise ValueError("points must be an (n, 2|3) float32 tensor")
    if not points.is_contiguous():
        raise ValueError("points must be contiguous")
    return points.shape[0], points.shape[1]


def _edges_out(n, like, out_edges):
    torch = _torch()
    m = max(n - 1, 0)
    if out_edges is None:
        pin = like.device.type == "cpu" and torch.cuda.is_available()
        out_edges = torch.empty((m, 3), dtype=torch.int32, device=like.device, pin_memory=pin)
    elif out_edges.dtype != torch.int32 or tuple(out_edges.shape) != (m, 3) or not out_edges.is_contiguous():
        raise ValueError(f"out_edges must be a contiguous ({m}, 3) int32 tensor")
    return out_edges


def emst_compute(points, out_edges=None, stream=None):
    """EMST of an (n, dim) float32 tensor (device or host); returns the edges."""
    n, dim = _check_points(points)
    out_edges = _edges_out(n, points, out_edges)
    rc = load_library().emst_compute(_ptr(points), n, dim, _ptr(out_edges),
                                     _stream_ptr(stream, points.device))
    if rc != 0:
        raise EmstError(rc, "emst_compute")
    return out_edges


EMST_NOALLOC_MAX_POINTS = 65536


def emst_compute_noalloc(points, out_edges=None, stream=None):
    """emst_compute without any device allocation inside the call: scratch is
    the library's fixed device array (n <= EMST_NOALLOC_MAX_POINTS).  For
    callers that cannot allocate device memory where they need the tree.
    Calls that overlap on one GPU share that array and race: serialise them.
    (Passing out_edges=None still lets this binding allocate the result.)"""
    n, dim = _check_points(points)
    out_edges = _edges_out(n, points, out_edges)
    rc = load_library().emst_compute_noalloc(_ptr(points), n, dim, _ptr(out_edges),
                                             _stream_ptr(stream, points.device))
    if rc != 0:
        raise EmstError(rc, "emst_compute_noalloc")
    return out_edges


def _make_options(block_size=0, carried_radius=True, use_graph=False, count_visits=False,
                  leaf_size=0, mlp_params=None, mrd_k=0, morton_bits=0, traversal=0,
                  refill_lanes=0, queue_chunk=0, ignore_tuning=False):
    opt = _Options()
    opt.struct_size = ctypes.sizeof(_Options)
    opt.block_size = int(block_size)
    opt.carried_radius = 1 if carried_radius else 0
    opt.use_graph = 1 if use_graph else 0
    opt.count_visits = 1 if count_visits else 0
    opt.leaf_size = int(leaf_size)
    opt.mrd_k = int(mrd_k)
    opt.morton_bits = int(morton_bits)
    opt.traversal = int(traversal)
    opt.refill_lanes = int(refill_lanes)
    opt.queue_chunk = int(queue_chunk)
    opt.ignore_tuning = 1 if ignore_tuning else 0
    if mlp_params is not None:
        if mlp_params.dtype != _torch().float32 or mlp_params.numel() != EMST_MLP_PARAMS:
            raise ValueError(f"mlp_params must hold {EMST_MLP_PARAMS} float32 values")
        opt.mlp_params = mlp_params.data_ptr()
    return opt


def _new_stats():
    st = _Stats()
    st.struct_size = ctypes.sizeof(_Stats)
    return st


def _stats_dict(st):
    r = min(st.rounds, 40)
    return dict(rounds=st.rounds, kernel_launches=st.kernel_launches, total_ms=st.total_ms,
                build_ms=st.build_ms, rounds_ms=st.rounds_ms, output_ms=st.output_ms,
                node_visits=st.node_visits, traverse_ms=st.traverse_ms,
                traverse_launches=st.traverse_launches,
                round_traverse_ms=[float(st.round_traverse_ms[k]) for k in range(r)],
                components_per_round=[int(st.components_per_round[k]) for k in range(r)],
                queried_points=st.queried_points, rerun_points=st.rerun_points,
                learned_search_ms=st.learned_search_ms, core_ms=st.core_ms,
                morton_bits=st.morton_bits, code_collisions=st.code_collisions,
                round_visits=[int(st.round_visits[k]) for k in range(r)],
                round_queries=[int(st.round_queries[k]) for k in range(r)],
                round_distinct_nodes=[int(st.round_distinct_nodes[k]) for k in range(r)],
                traversal_used=st.traversal_used, block_used=st.block_used,
                leaf_used=st.leaf_used, tuned=bool(st.tuned))


def emst_compute_ex(points, out_edges=None, stream=None, **options):
    """emst_compute with options (keywords of emst_options: block_size,
    carried_radius, count_visits, leaf_size, mlp_params, mrd_k, morton_bits,
    traversal); returns (edges, stats dict).  mrd_k >= 2: the
    mutual-reachability MST (squared MRD weights).  traversal: 0 default,
    1 one thread per point, 2 persistent work queue."""
    n, dim = _check_points(points)
    out_edges = _edges_out(n, points, out_edges)
    opt = _make_options(**options)
    st = _new_stats()
    rc = load_library().emst_compute_ex(_ptr(points), n, dim, _ptr(out_edges),
                                        _stream_ptr(stream, points.device), ctypes.byref(opt),
                                        ctypes.byref(st))
    if rc != 0:
        raise EmstError(rc, "emst_compute_ex")
    return out_edges, _stats_dict(st)


def emst_core_distances(points, k, out=None, stream=None):
    """Squared core distances (k-th nearest neighbour, the point itself
    first) of the mutual reachability distance, in the points' order."""
    torch = _torch()
    n, dim = _check_points(points)
    if out is None:
        pin = points.device.type == "cpu" and torch.cuda.is_available()
        out = torch.empty(n, dtype=torch.float32, device=points.device, pin_memory=pin)
    rc = load_library().emst_core_distances(_ptr(points), n, dim, int(k), _ptr(out),
                                            _stream_ptr(stream, points.device))
    if rc != 0:
        raise EmstError(rc, "emst_core_distances")
    return out


def emst_compute_batched(points, offsets, out_edges=None, stream=None):
    """Independent EMSTs of the row blocks [offsets[k], offsets[k+1]).
    Returns (edges, edge_offsets) with instance-local ids.  ``offsets`` may be
    a CUDA int64 tensor: then the library reads it from device memory and the
    edge offsets come back as a CUDA tensor too."""
    e, eo, _ = _batched(points, offsets, out_edges, stream, None)
    return e, eo


def emst_compute_batched_ex(points, offsets, out_edges=None, stream=None, **options):
    """emst_compute_batched with options (see emst_compute_ex); returns
    (edges, edge_offsets, stats dict)."""
    return _batched(points, offsets, out_edges, stream, _make_options(**options))


def _batched(points, offsets, out_edges, stream, opt):
    torch = _torch()
    n, dim = _check_points(points)
    st = _new_stats() if opt is not None else None
    lib = load_library()

    def call(p_off, p_out_off, k):
        if opt is None:
            return lib.emst_compute_batched(_ptr(points), p_off, k, dim, _ptr(out_edges), p_out_off,
                                            _stream_ptr(stream, points.device))
        return lib.emst_compute_batched_ex(_ptr(points), p_off, k, dim, _ptr(out_edges), p_out_off,
                                           _stream_ptr(stream, points.device), ctypes.byref(opt),
                                           ctypes.byref(st))

    if isinstance(offsets, torch.Tensor) and offsets.is_cuda:
        if offsets.dtype != torch.int64 or offsets.dim() != 1 or not offsets.is_contiguous():
            raise ValueError("device offsets must be a contiguous 1-D int64 tensor")
        k = offsets.numel() - 1
        m = int((offsets[1:] - offsets[:-1] - 1).clamp(min=0).sum()) if k > 0 else 0
        if out_edges is None:
            out_edges = torch.empty((m, 3), dtype=torch.int32, device=points.device)
        out_offs = torch.empty(k + 1, dtype=torch.int64, device=offsets.device)
        rc = call(_ptr(offsets), _ptr(out_offs), k)
    else:
        offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        if offs.ndim != 1 or len(offs) < 1 or offs[0] != 0 or offs[-1] != n or np.any(np.diff(offs) < 0):
            raise ValueError("offsets must start at 0, end at n and be non-decreasing")
        k = len(offs) - 1
        m = int(np.maximum(np.diff(offs) - 1, 0).sum())
        if out_edges is None:
            pin = points.device.type == "cpu" and torch.cuda.is_available()
            out_edges = torch.empty((m, 3), dtype=torch.int32, device=points.device, pin_memory=pin)
        out_offs = np.zeros(k + 1, dtype=np.int64)
        rc = call(ctypes.c_void_p(offs.ctypes.data), ctypes.c_void_p(out_offs.ctypes.data), k)
    if rc != 0:
        raise EmstError(rc, "emst_compute_batched")
    return out_edges, out_offs, (_stats_dict(st) if st is not None else None)


def emst_build_bvh(points, leaf_size=1, stream=None, morton_bits=64):
    """The built hierarchy over leaf chunks of `leaf_size` curve positions:
    dict(codes, perm, children (m-1, 2), boxes (m-1, 2, 6)), m = ceil(n/leaf_size).
    With morton_bits=128, codes is (n, 2): (high, low) words."""
    torch = _torch()
    n, dim = _check_points(points)
    dev = points.device if points.device.type == "cuda" else torch.device("cuda")
    m = max((n + leaf_size - 1) // leaf_size, 1)
    codes = torch.empty((n, 2) if morton_bits == 128 else n, dtype=torch.int64, device=dev)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    children = torch.empty((m - 1, 2), dtype=torch.int32, device=dev)
    boxes = torch.empty((m - 1, 2, 6), dtype=torch.float32, device=dev)
    rc = load_library().emst_build_bvh_ex(_ptr(points), n, dim, int(leaf_size), int(morton_bits),
                                          _ptr(codes), _ptr(perm), _ptr(children), _ptr(boxes),
                                          _stream_ptr(stream, dev))
    if rc != 0:
        raise EmstError(rc, "emst_build_bvh_ex")
    return dict(codes=codes, perm=perm, children=children, boxes=boxes)


def emst_round_step(points, labels, radius=None, leaf_size=1, stream=None):
    """One Boruvka round from curve-order labels; see include/emst.h."""
    torch = _torch()
    n, dim = _check_points(points)
    dev = points.device if points.device.type == "cuda" else torch.device("cuda")
    labels = labels.to(device=dev, dtype=torch.int32).contiguous()
    if radius is not None:
        radius = radius.to(device=dev, dtype=torch.float32).contiguous()
    m = max((n + leaf_size - 1) // leaf_size, 1)
    node_labels = torch.empty((m - 1, 2), dtype=torch.int32, device=dev)
    ub = torch.empty(n, dtype=torch.float32, device=dev)
    nn_w = torch.empty(n, dtype=torch.float32, device=dev)
    nn_j = torch.empty(n, dtype=torch.int32, device=dev)
    new_labels = torch.empty(n, dtype=torch.int32, device=dev)
    edges = torch.empty((n, 3), dtype=torch.int32, device=dev)
    m = ctypes.c_int64(0)
    rc = load_library().emst_round_step(_ptr(points), n, dim, int(leaf_size), _ptr(labels), _ptr(radius),
                                        _ptr(node_labels), _ptr(ub), _ptr(nn_w), _ptr(nn_j),
                                        _ptr(new_labels), _ptr(edges), ctypes.byref(m),
                                        _stream_ptr(stream, dev))
    if rc != 0:
        raise EmstError(rc, "emst_round_step")
    return dict(node_labels=node_labels, upper_bound=ub, nn_w=nn_w, nn_j=nn_j, labels=new_labels,
                edges=edges[: m.value])


def edges_w(edges):
    return edges[:, 2].view(_torch().float32)


def emst_dendrogram(edges, n=None, out_linkage=None, out_parent=None, stream=None,
                    linkage=True, parent=True):
    """Single-linkage dendrogram of a spanning tree given as (n-1, 3) int32
    edges in merge order (weights not decreasing; emst_compute's output
    qualifies), device or host.  Returns (linkage, parent): linkage is an
    (n-1, 4) int32 tensor of rows {a, b, w bits, size} (linkage_numpy views
    it), parent a (2n-1,) int32 tensor (-1 for the root); either is None when
    not requested."""
    torch = _torch()
    if not isinstance(edges, torch.Tensor) or edges.dtype != torch.int32 or edges.dim() != 2 \
            or edges.shape[1] != 3 or not edges.is_contiguous():
        raise ValueError("edges must be a contiguous (m, 3) int32 tensor")
    m = edges.shape[0]
    n = m + 1 if n is None else int(n)
    if m != max(n - 1, 0):
        raise ValueError(f"a spanning tree of {n} points has {max(n - 1, 0)} edges, got {m}")
    pin = edges.device.type == "cpu" and torch.cuda.is_available()
    if linkage and out_linkage is None:
        out_linkage = torch.empty((m, 4), dtype=torch.int32, device=edges.device, pin_memory=pin)
    if parent and out_parent is None:
        out_parent = torch.empty(max(2 * n - 1, 0), dtype=torch.int32, device=edges.device,
                                 pin_memory=pin)
    for t, shape in ((out_linkage, (m, 4)), (out_parent, (max(2 * n - 1, 0),))):
        if t is not None and (t.dtype != torch.int32 or tuple(t.shape) != shape or not t.is_contiguous()):
            raise ValueError(f"output must be a contiguous {shape} int32 tensor")
    rc = load_library().emst_dendrogram(_ptr(edges), n, _ptr(out_linkage), _ptr(out_parent),
                                        _stream_ptr(stream, edges.device))
    if rc != 0:
        raise EmstError(rc, "emst_dendrogram")
    return out_linkage, out_parent


def linkage_numpy(linkage) -> np.ndarray:
    a = linkage.detach().cpu().contiguous().numpy()
    return np.ascontiguousarray(a).view(LINKAGE_DTYPE).reshape(-1)


def edges_numpy(edges) -> np.ndarray:
    a = edges.detach().cpu().contiguous().numpy()
    return np.ascontiguousarray(a).view(EDGE_DTYPE).reshape(-1)


# ----------------------------------------------------------------------------
# Learned search radius: network pieces (see include/emst.h)
# ----------------------------------------------------------------------------
def _dev_f32(t, numel=None):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float32 or not t.is_contiguous() or t.device.type != "cuda":
        raise ValueError("expected a contiguous float32 CUDA tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"expected {numel} values")
    return t


def emst_mlp_forward(features, params, out=None, stream=None):
    """Predicted log2 weights for an (m, 8) float32 feature tensor (BF16 tensor-core inference)."""
    torch = _torch()
    _dev_f32(features)
    _dev_f32(params, EMST_MLP_PARAMS)
    m = features.shape[0]
    if out is None:
        out = torch.empty(m, dtype=torch.float32, device=features.device)
    rc = load_library().emst_mlp_forward(_ptr(features), m, _ptr(params), _ptr(out),
                                         _stream_ptr(stream, features.device))
    if rc != 0:
        raise EmstError(rc, "emst_mlp_forward")
    return out


def emst_mlp_grad(features, targets, params, grad, loss, stream=None):
    """Adds the batch's mean-squared-error gradient to grad and the loss to loss[0]."""
    for t in (features, targets, params, grad, loss):
        _dev_f32(t)
    rc = load_library().emst_mlp_grad(_ptr(features), _ptr(targets), features.shape[0], _ptr(params),
                                      _ptr(grad), _ptr(loss), _stream_ptr(stream, features.device))
    if rc != 0:
        raise EmstError(rc, "emst_mlp_grad")


def emst_mlp_adam(params, grad, m1, m2, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    for t in (params, grad, m1, m2):
        _dev_f32(t, EMST_MLP_PARAMS)
    rc = load_library().emst_mlp_adam(_ptr(params), _ptr(grad), _ptr(m1), _ptr(m2), int(step),
                                      float(lr), float(beta1), float(beta2), float(eps),
                                      _stream_ptr(stream, params.device))
    if rc != 0:
        raise EmstError(rc, "emst_mlp_adam")


def emst_learned_samples(points, every, capacity, stream=None):
    """(features (k, 8), targets (k,)) training pairs logged from a plain run."""
    torch = _torch()
    n, dim = _check_points(points)
    dev = points.device if points.device.type == "cuda" else torch.device("cuda")
    feat = torch.empty((capacity, EMST_MLP_FEATURES), dtype=torch.float32, device=dev)
    targ = torch.empty(capacity, dtype=torch.float32, device=dev)
    cnt = ctypes.c_int64(0)
    rc = load_library().emst_learned_samples(_ptr(points), n, dim, int(every), _ptr(feat), _ptr(targ),
                                             int(capacity), ctypes.byref(cnt), _stream_ptr(stream, dev))
    if rc != 0:
        raise EmstError(rc, "emst_learned_samples")
    k = min(cnt.value, capacity)
    return feat[:k], targ[:k]
