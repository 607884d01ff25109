"""Seeded synthetic point sets shaped like the paper's workloads (§4, "Datasets").

The paper measures on HACC cosmology particles, GPS traces and generated
uniform / normal clouds.  None of those files exist here, so these generators
stand in for them with the same dimension, size and kind of structure:

* ``uniform``      -- i.i.d. uniform in [0,1)^d (the Uniform* sets).
* ``blobs``        -- isotropic Gaussian blobs plus a uniform background
                      (VisualVar / trajectory-like clustered 2D data).
* ``halos``        -- NFW-profile halos with a power-law mass function plus a
                      uniform background (stands in for Hacc37M / Hacc497M).
* ``lattice_ties`` -- points of the integer lattice {0..199}^3 / 200 with 4 %
                      duplicates: a tie-stress set (massive equal weights).
* ``batched_sizes`` / ``batched_instances`` -- many independent instances of
                      uneven size.
* ``tree_edges``   -- a random spanning tree of a given shape with weights,
                      listed by non-decreasing weight (input for the
                      single-linkage dendrogram; not point data).

This module holds no arithmetic of the EMST method: it only draws numbers.
Everything is generated in FP64 from ``numpy.random.Generator(PCG64(seed))``
and cast to FP32 C-contiguous (n, d) arrays.  Points that leave the unit box
are wrapped modulo 1 (a periodic box, as in a cosmology volume).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "tree_edges",
    "uniform",
    "blobs",
    "halos",
    "lattice_ties",
    "batched_sizes",
    "batched_instances",
    "config_points",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _wrap_f32(x: np.ndarray) -> np.ndarray:
    x = np.mod(x, 1.0)
    out = x.astype(np.float32)
    # FP32 rounding of a value just below 1 can land on 1.0; keep [0,1).
    out[out >= np.float32(1.0)] = np.float32(0.0)
    return np.ascontiguousarray(out)


def uniform(n: int, dim: int, seed: int) -> np.ndarray:
    """n points i.i.d. uniform in [0,1)^dim."""
    g = _rng(seed)
    return _wrap_f32(g.random((n, dim)))


def blobs(n: int, dim: int, seed: int, n_blobs: int = 50, frac_background: float = 0.10,
          sigma_range=(1e-3, 5e-2)) -> np.ndarray:
    """Gaussian blobs + uniform background.

    (1 - frac_background)·n points come from ``n_blobs`` isotropic Gaussians with
    centres uniform in the unit box, sigma log-uniform in ``sigma_range`` and
    mixture weights Dirichlet(1); the rest are uniform.  Rows are shuffled.
    """
    g = _rng(seed)
    n_bg = int(round(frac_background * n))
    n_cl = n - n_bg
    centres = g.random((n_blobs, dim))
    lo, hi = np.log(sigma_range[0]), np.log(sigma_range[1])
    sigmas = np.exp(g.uniform(lo, hi, n_blobs))
    weights = g.dirichlet(np.ones(n_blobs))
    counts = g.multinomial(n_cl, weights)
    which = np.repeat(np.arange(n_blobs), counts)
    pts = centres[which] + sigmas[which, None] * g.standard_normal((n_cl, dim))
    bg = g.random((n_bg, dim))
    allp = np.concatenate([pts, bg], axis=0)
    allp = allp[g.permutation(n)]
    return _wrap_f32(allp)


def dense(n: int, dim: int, seed: int, n_clusters: int = 20_000,
          sigma_range=(1e-9, 1e-6), frac_background: float = 0.10) -> np.ndarray:
    """Extremely dense clusters (the under-resolved regime §4.1 describes for
    a GPS-trace dataset): (1 - frac_background)·n points in ``n_clusters``
    isotropic Gaussians with centres uniform in the unit box, sigma
    log-uniform in ``sigma_range`` (below the 2^-21 cells of 64-bit 3D codes)
    and sizes from a power law p(m) ∝ m^-2 (Dirichlet-free: counts drawn by
    multinomial on those weights); the rest uniform.  Rows are shuffled."""
    g = _rng(seed)
    n_bg = int(round(frac_background * n))
    n_cl = n - n_bg
    centres = g.random((n_clusters, dim))
    lo, hi = np.log(sigma_range[0]), np.log(sigma_range[1])
    sigmas = np.exp(g.uniform(lo, hi, n_clusters))
    w = (1.0 - g.random(n_clusters)) ** (-1.0)  # Pareto, p(m) ∝ m^-2
    counts = g.multinomial(n_cl, w / w.sum())
    which = np.repeat(np.arange(n_clusters), counts)
    pts = centres[which] + sigmas[which, None] * g.standard_normal((n_cl, dim))
    bg = g.random((n_bg, dim))
    allp = np.concatenate([pts, bg], axis=0)
    allp = allp[g.permutation(n)]
    return _wrap_f32(allp)


def _nfw_mass(x):
    return np.log1p(x) - x / (1.0 + x)


def _nfw_inverse(y: np.ndarray, c: float) -> np.ndarray:
    """Solve ln(1+x) - x/(1+x) = y for x in [0, c] (table guess + Newton)."""
    grid = np.linspace(0.0, c, 8193)
    mg = _nfw_mass(grid)
    x = np.interp(y, mg, grid)
    for _ in range(4):
        f = _nfw_mass(x) - y
        fp = x / (1.0 + x) ** 2
        step = np.where(fp > 1e-300, f / np.maximum(fp, 1e-300), 0.0)
        x = np.clip(x - step, 0.0, c)
    return x


def halos(n: int, seed: int, frac_background: float = 0.20, alpha: float = 1.9,
          m_min: float = 10.0, m_max: float = 1e5, concentration: float = 5.0,
          r_vir_max: float = 0.01) -> np.ndarray:
    """3D cosmology-shaped clustering.

    (1 - frac_background)·n points are placed in halos.  Halo member counts m
    follow p(m) ∝ m^-alpha on [m_min, m_max] (inverse-CDF draws, floored), drawn
    until the budget is used (the last halo is truncated).  Centres are uniform,
    the radial profile is NFW with the given concentration and
    r_vir = r_vir_max·(m/m_max)^(1/3); the radius comes from inverting the
    enclosed-mass profile, the direction is isotropic.  The rest is uniform.
    """
    g = _rng(seed)
    n_bg = int(round(frac_background * n))
    n_cl = n - n_bg
    a1 = 1.0 - alpha
    lo_p, hi_p = m_min ** a1, m_max ** a1
    sizes = []
    used = 0
    while used < n_cl:
        u = g.random(4096)
        m = np.floor((lo_p + u * (hi_p - lo_p)) ** (1.0 / a1)).astype(np.int64)
        m = np.maximum(m, 1)
        for mi in m:
            take = int(min(mi, n_cl - used))
            sizes.append(take)
            used += take
            if used >= n_cl:
                break
    sizes = np.asarray(sizes, dtype=np.int64)
    masses = sizes.astype(np.float64)
    n_h = len(sizes)
    centres = g.random((n_h, 3))
    r_vir = r_vir_max * (masses / m_max) ** (1.0 / 3.0)
    which = np.repeat(np.arange(n_h), sizes)
    y = g.random(n_cl) * _nfw_mass(concentration)
    x = _nfw_inverse(y, concentration)
    r = x / concentration * r_vir[which]
    v = g.standard_normal((n_cl, 3))
    v /= np.maximum(np.linalg.norm(v, axis=1, keepdims=True), 1e-300)
    pts = centres[which] + r[:, None] * v
    bg = g.random((n_bg, 3))
    allp = np.concatenate([pts, bg], axis=0)
    allp = allp[g.permutation(n)]
    return _wrap_f32(allp)


def lattice_ties(n_sites: int = 7_680_000, n_dup: int = 320_000, side: int = 200,
                 seed: int = 3) -> np.ndarray:
    """Tie-stress set: distinct lattice sites of {0..side-1}^3 (without
    replacement) plus ``n_dup`` repeats of drawn sites, shuffled, scaled by 1/side."""
    g = _rng(seed)
    total = side ** 3
    sites = g.choice(total, size=n_sites, replace=False)
    dups = sites[g.integers(0, n_sites, n_dup)]
    allsites = np.concatenate([sites, dups])
    allsites = allsites[g.permutation(len(allsites))]
    k = np.stack([allsites // (side * side), (allsites // side) % side, allsites % side], axis=1)
    pts = k.astype(np.float64) / float(side)
    return np.ascontiguousarray(pts.astype(np.float32))


def batched_sizes(num_instances: int, seed: int, lo: int = 100, hi: int = 1_000_000) -> np.ndarray:
    """Instance sizes log-uniform in [lo, hi] (integers)."""
    g = _rng(seed)
    s = np.exp(g.uniform(np.log(lo), np.log(hi), num_instances))
    return np.floor(s).astype(np.int64)


def _fill_instances(job):
    """Worker of batched_instances: draw instances [k0, k1) into the shared
    output buffer (each instance has its own seed, so the result does not
    depend on how the work is split)."""
    from multiprocessing import shared_memory
    name, total, sizes, offsets, k0, k1, seed, n_blobs, frac_background = job
    shm = shared_memory.SharedMemory(name=name)
    try:
        out = np.ndarray((total, 3), dtype=np.float32, buffer=shm.buf)
        for k in range(k0, k1):
            out[offsets[k]:offsets[k + 1]] = blobs(int(sizes[k]), 3, seed * 1_000_003 + k,
                                                   n_blobs=n_blobs, frac_background=frac_background)
        del out
    finally:
        shm.close()
    return k1 - k0


def batched_instances(sizes, seed: int, n_blobs: int = 20, frac_background: float = 0.10,
                      workers: int = 1):
    """Concatenated 3D instances (blobs generator, 20 blobs, 10 % uniform) and
    the int64 offsets array of length len(sizes)+1.  Instance k is drawn with
    seed ``seed * 1_000_003 + k``; ``workers`` > 1 draws the instances in that
    many processes (spawned, so it is safe after CUDA is initialised) with the
    same result."""
    sizes = np.asarray(sizes, dtype=np.int64)
    offsets = np.zeros(len(sizes) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    total = int(offsets[-1])
    if workers <= 1 or len(sizes) < 2 or total == 0:
        out = np.empty((total, 3), dtype=np.float32)
        for k, s in enumerate(sizes):
            out[offsets[k]:offsets[k + 1]] = blobs(int(s), 3, seed * 1_000_003 + k, n_blobs=n_blobs,
                                                   frac_background=frac_background)
        return out, offsets
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    from multiprocessing import shared_memory
    shm = shared_memory.SharedMemory(create=True, size=total * 3 * 4)
    try:
        # contiguous runs of instances with about equal point counts
        bounds = np.searchsorted(offsets, np.linspace(0, total, 4 * workers + 1)[1:-1])
        cuts = np.unique(np.concatenate([[0], bounds, [len(sizes)]]))
        jobs = [(shm.name, total, sizes, offsets, int(a), int(b), seed, n_blobs, frac_background)
                for a, b in zip(cuts[:-1], cuts[1:]) if b > a]
        with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            done = sum(ex.map(_fill_instances, jobs))
        assert done == len(sizes)
        out = np.ndarray((total, 3), dtype=np.float32, buffer=shm.buf).copy()
    finally:
        shm.close()
        shm.unlink()
    return out, offsets


def config_points(config: int, n: int | None = None, seed: int | None = None) -> np.ndarray:
    """The five workload shapes, optionally resized (same generator, other n)."""
    if config == 1:
        return uniform(10_000 if n is None else n, 3, 0 if seed is None else seed)
    if config == 2:
        return blobs(1_000_000 if n is None else n, 2, 1 if seed is None else seed)
    if config == 3:
        return halos(37_000_000 if n is None else n, 2 if seed is None else seed)
    if config == 5:
        return halos(100_000_000 if n is None else n, 3 if seed is None else seed)
    raise ValueError(f"no single point set for config {config}")


TREE_SHAPES = ("random", "path", "path_sorted", "star", "caterpillar", "binary")


def tree_edges(n: int, seed: int, shape: str = "random", ties: int = 0) -> np.ndarray:
    """A spanning tree on n vertices as an (n-1)-row structured array
    (i, j: uint32 vertex ids, w: float32), listed by non-decreasing w with
    equal weights in random order.

    shape: "random" (each vertex k > 0 attaches to a uniform earlier vertex),
    "path" (a random vertex order, random weights), "path_sorted" (a path whose
    weights increase along it: the deepest possible hierarchy), "star" (one
    centre), "caterpillar" (a path with a leaf on every vertex), "binary"
    (vertex k attaches to (k-1)//2).  Vertex ids are shuffled.
    ties: 0 for distinct weights (FP32 of uniform draws), else the weights are
    drawn from that many distinct values."""
    g = _rng(seed)
    n = int(n)
    m = max(n - 1, 0)
    k = np.arange(1, n, dtype=np.int64)
    if shape == "random":
        parent = np.floor(g.random(m) * k).astype(np.int64)
    elif shape in ("path", "path_sorted"):
        parent = k - 1
    elif shape == "star":
        parent = np.zeros(m, dtype=np.int64)
    elif shape == "caterpillar":
        spine = (n + 1) // 2
        parent = np.where(k < spine, k - 1, k - spine)
    elif shape == "binary":
        parent = (k - 1) // 2
    else:
        raise ValueError(shape)
    if ties:
        w = (g.integers(0, int(ties), size=m) + 1).astype(np.float64) / float(ties)
    else:
        w = g.random(m) + 1e-3
    if shape == "path_sorted":
        w = np.sort(w)
    ids = g.permutation(n).astype(np.uint32)
    e = np.zeros(m, dtype=[("i", np.uint32), ("j", np.uint32), ("w", np.float32)])
    a, b = ids[parent], ids[k]
    e["i"] = np.minimum(a, b)
    e["j"] = np.maximum(a, b)
    e["w"] = w.astype(np.float32)
    order = np.lexsort((g.random(m), e["w"]))
    return e[order]
