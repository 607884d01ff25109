"""Autotuner of the traversal (Algorithm 2) parameters.

For every class -- dimension, form (one problem or a batch of independent
instances) and a range of sizes -- it times the exact variants of the search
on a seeded synthetic input shaped like the workloads of that class:

* the one-thread-per-point kernel (traversal 1) at CTA sizes 64 / 128 / 256
  and leaf-bucket sizes 1 / 2 (one problem only: a batch keeps one point per
  leaf);
* the persistent work-queue kernel (traversal 2) at refill thresholds
  8 / 16 / 24 idle lanes and queue chunks of 64 / 128 curve positions.

The search stack needs no tuning: it is a local array whose depth is fixed by
the hierarchy's key width (its untouched tail costs nothing); a shared-memory
ring for its top entries was measured slower at every size (it takes L1
capacity from the node records).

Each candidate runs once to warm up and three times timed (whole-call device
time from the library's CUDA events, best of three), with the tuning file
ignored.  The fastest candidate of each class is written as one line of the
tuning file the library reads (see include/emst.h); every candidate's time is
printed as a JSON line, so the choices are logged.

    python -m paper_2207_00514_gb300.tune [--out FILE] [--quick]
"""
from __future__ import annotations

import argparse
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
DEFAULT_OUT = os.path.join(HERE, "emst_tuning.txt")
BIG = 1 << 30

# (dim, form, nmin, nmax, representative n or number of instances)
CLASSES = [
    (3, "single", 0, 30_000, 10_000),
    (3, "single", 30_000, 300_000, 100_000),
    (3, "single", 300_000, 3_000_000, 1_000_000),
    (3, "single", 3_000_000, 20_000_000, 10_000_000),
    (3, "single", 20_000_000, BIG, 37_000_000),
    (2, "single", 0, 30_000, 10_000),
    (2, "single", 30_000, 300_000, 100_000),
    (2, "single", 300_000, 3_000_000, 1_000_000),
    (2, "single", 3_000_000, BIG, 10_000_000),
    (3, "batched", 0, BIG, 4096),
]


def candidates(form: str):
    out = []
    for block in (64, 128, 256):
        for leaf in ((1, 2) if form == "single" else (1,)):
            out.append({"traversal": 1, "block_size": block, "leaf_size": leaf})
    for refill in (8, 16, 24):
        for chunk in (64, 128):
            out.append({"traversal": 2, "refill_lanes": refill, "queue_chunk": chunk})
    return out


def make_input(dim, form, size):
    sys.path.insert(0, ROOT)
    import synth
    if form == "batched":
        sizes = synth.batched_sizes(size, seed=4, lo=100, hi=1_000_000)
        return synth.batched_instances(sizes, seed=4, workers=os.cpu_count() or 4)
    if dim == 3:
        return synth.halos(size, 2), None
    return synth.blobs(size, 2, 1), None


def time_candidate(pkg, torch, pts, offs, opts, reps=3):
    def call():
        if offs is None:
            return pkg.emst_compute_ex(pts, ignore_tuning=True, **opts)[1]
        return pkg.emst_compute_batched_ex(pts, offs, ignore_tuning=True, **opts)[2]
    call()
    torch.cuda.synchronize()
    best = None
    for _ in range(reps):
        st = call()
        best = st["total_ms"] if best is None else min(best, st["total_ms"])
    return best


def tune(out_path: str, quick: bool = False) -> list[dict]:
    import torch
    import paper_2207_00514_gb300 as pkg

    pkg.load_library()
    gpu = torch.cuda.get_device_name().replace(" ", "_")
    lines, chosen = [], []
    classes = CLASSES
    if quick:
        classes = [c for c in CLASSES if c[1] == "single" and c[4] <= 1_000_000]
        classes.append((3, "batched", 0, BIG, 256))
    for dim, form, nmin, nmax, size in classes:
        pts_np, offs = make_input(dim, form, size)
        pts = torch.from_numpy(pts_np).cuda()
        results = []
        for opts in candidates(form):
            ms = time_candidate(pkg, torch, pts, offs, opts)
            results.append((ms, opts))
            print(json.dumps({"gpu": gpu, "dim": dim, "form": form, "n": len(pts_np), "ms": round(ms, 4),
                              **opts}), flush=True)
        results.sort(key=lambda r: r[0])
        ms, best = results[0]
        default_ms = next(r[0] for r in results
                          if r[1] == {"traversal": 1, "block_size": 128, "leaf_size": 1})
        rec = {"gpu": gpu, "dim": dim, "form": form, "nmin": nmin, "nmax": nmax, "n": len(pts_np),
               "best_ms": round(ms, 4), "default_ms": round(default_ms, 4), **best}
        chosen.append(rec)
        print(json.dumps({"chosen": rec}), flush=True)
        lines.append(f"gpu={gpu} dim={dim} form={form} nmin={nmin} nmax={nmax} "
                     f"traversal={best['traversal']} block={best.get('block_size', 0)} "
                     f"leaf={best.get('leaf_size', 0)} refill={best.get('refill_lanes', 0)} "
                     f"chunk={best.get('queue_chunk', 0)}  # {ms:.3f} ms at n={len(pts_np)} "
                     f"(default kernel {default_ms:.3f} ms)")
        del pts
        torch.cuda.empty_cache()
    with open(out_path, "w") as f:
        f.write("# emst tuning file (written by paper_2207_00514_gb300/tune.py): per GPU, dimension,\n"
                "# form and size range, the fastest exact traversal variant measured.\n")
        for ln in lines:
            f.write(ln + "\n")
    return chosen


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_OUT)
    ap.add_argument("--quick", action="store_true", help="small classes only (a smoke run)")
    a = ap.parse_args()
    tune(a.out, a.quick)


if __name__ == "__main__":
    main()
