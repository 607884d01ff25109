#!/usr/bin/env python3
"""Benchmark: EMST throughput (Mpoints/s) of the single-tree Boruvka method on
one GB300, on the 37M-point clustered 3D workload (the cosmology-shaped
generator standing in for the paper's Hacc37M).

One step = one full emst_compute call (scene box, codes, sort, hierarchy,
refit, every Boruvka round, output ordering) on one batch of points that is
already resident in HBM.  Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--n N_POINTS] [--no-cpu-baseline]

--impl reference times the CPU oracle (k-d tree Boruvka) as it stands on the
host cores, on a bounded random sample of the same workload per step.
Multi-GPU: the single EMST does not shard, so N GPUs run N independent
replicas (weak scaling); only a timing barrier / max crosses ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "EMST Mpoints/s at 37M 3D clustered, plain vs learned-radius; % HBM roofline"
WORKLOAD = ("37,000,000 FP32 3D points: 80% in NFW halos (power-law member counts m^-1.9 on "
            "[10, 1e5], c = 5, r_vir = 0.01 (m/1e5)^(1/3)), 20% uniform, unit box, seed 2")
# DRAM bytes (read + write) of each round's traversal on this workload (37M
# halo points, seed 2): its k_traverse launch, plus from round 2 on the
# k_active launches that list the queries to search (inside the round's CUDA
# events), from one ncu capture of one whole call of the kernels as they are
# now:
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum
#       --clock-control none -k regex:"k_traverse|k_active" -c 24 --csv
#       python bench.py --workload once
# (one pass per launch).  Set back to None whenever those kernels change.
TRAVERSE_DRAM_BYTES_PER_ROUND = [5220.5e6, 6216.1e6, 6480.0e6, 3833.9e6, 1894.4e6, 1398.3e6,
                                 818.0e6, 537.6e6, 472.7e6, 455.1e6, 444.7e6]
PAPER_CONTEXT = ("paper: Hacc37M (real 37M 3D cosmology points) on one A100 in < 0.5 s, best-case "
                 "270 MFeatures/s ~ 90 Mpoints/s; other data, other GPU: context only")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=37_000_000)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--cpu-sample", type=int, default=3_000_000,
                    help="reference arm: points per step in the oracle's spatial-window sample")
    ap.add_argument("--cpu-single-sample", type=int, default=500_000,
                    help="cpu_baseline: also time the oracle on one thread on a spatial window of "
                         "about this many points (0: skip)")
    ap.add_argument("--cpu-full", type=int, default=1,
                    help="cpu_baseline: 1 = the oracle on the whole workload (all host threads)")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--traversal", type=int, default=0,
                    help="once workload: the traversal kernel (0 default, 1 one thread per point, "
                         "2 persistent work queue)")
    ap.add_argument("--no-batched-summary", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="halos37M",
                    choices=["halos37M", "batched", "sweep", "mrd", "dense", "dendrogram", "once"],
                    help="batched: 4,096 independent 3D instances (sizes log-uniform in [100, 1e6]) "
                         "in one emst_compute_batched call, against one emst_compute per instance")
    ap.add_argument("--instances", type=int, default=4096)
    ap.add_argument("--dense-n", type=int, default=24_000_000)
    ap.add_argument("--mrd-k", default="1,2,4,8,16",
                    help="mrd workload: the k_pts values to time, comma-separated")
    ap.add_argument("--clocks-dir", default=None,
                    help="keep the raw nvidia-smi clock samples of the timed region there "
                         "(default: a temporary file; the JSON line carries their summary)")
    ap.add_argument("--dg-tree", default="all", choices=["all", "emst", "mrd", "random"],
                    help="dendrogram workload: which tree(s) to time")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, keep_dir: str | None = None):
        import tempfile
        self.idx = gpu_index
        self.proc = None
        d = keep_dir or tempfile.gettempdir()
        self.path = os.path.join(d, f"emst_clocks_rank{gpu_index}_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [s for s, p in zip(sm, power) if p > 150.0] or sm
        return {"sm_mhz": float(np.median(load)), "sm_max_mhz": float(max(smax)),
                "samples": len(sm), "power_w_max": float(max(power)), "reasons": sorted(reasons)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# Algorithmic bytes of one traversal launch (Algorithm 2 over every point), by
# what the method must read or write at least once:
#  round 0 (every label is the point's own index, every query searches):
#    per query 56 B -- its point (16), label (4), component bound (4), the
#    component's best so far (8), its result (8), the update of the
#    component's 16-byte (w, min id, max id, outside label) minimum (16) --
#    and per distinct internal node visited its 64-B record;
#  later rounds: per point 24 B to decide whether to search at all -- label
#    (4), component bound (4) and best so far (8), its previous result (8)
#    (a skipped query rewrites its result only when it held a neighbour,
#    not counted) -- plus per query that searches 44 B -- its point (16),
#    its previous neighbour's label (4), its new result (8), the minimum's
#    update (16) -- and per distinct internal node visited 72 B: the record
#    (64) and its child labels (8).
BYTES_FIRST_QUERY = 56
BYTES_POINT = 24
BYTES_SEARCH = 44
BYTES_RECORD_FIRST = 64
BYTES_RECORD = 72


def traversal_round_bytes(n: int, queries, distinct):
    out = []
    for r, (q, d) in enumerate(zip(queries, distinct)):
        if r == 0:
            out.append(float(q * BYTES_FIRST_QUERY + d * BYTES_RECORD_FIRST))
        else:
            out.append(float(n * BYTES_POINT + q * BYTES_SEARCH + d * BYTES_RECORD))
    return out


def cpu_oracle_run(pts_sample, threads):
    import oracle
    t0 = time.perf_counter()
    oracle.kd_boruvka(pts_sample, threads=threads)
    return time.perf_counter() - t0


def make_points(n, seed):
    import synth
    return synth.halos(n, seed)


def workload_name(n: int, seed: int) -> str:
    if n == 37_000_000 and seed == 2:
        return WORKLOAD
    return f"{n:,} FP32 3D points of the same halo generator (seed {seed})"


def config_of(n: int, seed: int) -> dict:
    """The workload, the same for both arms of the benchmark."""
    return {"workload": workload_name(n, seed), "n": n, "dim": 3,
            "l2": "inputs and working set larger than L2 (no flush between steps)"}


def window_sample(pts, m, g):
    """A spatial window of the point set: the points inside a sub-cube of the
    unit box expected to hold about m of them, at a seeded random place.
    Unlike a random subsample it keeps the set's local density and
    clustering, so the oracle's rate on it stands for its rate on the whole
    set."""
    n = len(pts)
    side = min(1.0, (m / n) ** (1.0 / 3.0))
    o = g.random(3) * (1.0 - side)
    inside = np.all((pts >= o) & (pts < o + side), axis=1)
    return np.ascontiguousarray(pts[inside])


def run_reference(args, rank, world):
    """The oracle as it stands, on the host cores: each step one spatial
    window of the workload (about --cpu-sample points; the untimed warm-up
    steps a tenth of that), all host threads."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    pts = make_points(args.n, args.seed)
    g = np.random.default_rng(12345)
    threads = os.cpu_count() or 1
    done, secs = 0, 0.0
    for step in range(args.warmup + args.steps):
        m = args.cpu_sample if step >= args.warmup else max(args.cpu_sample // 10, 1000)
        sample = window_sample(pts, m, g)
        dt = cpu_oracle_run(sample, threads)
        if step >= args.warmup:
            done += len(sample)
            secs += dt
    value = done / secs / 1e6
    sample_desc = (f"per step the points of a seeded random sub-cube of the unit box holding about "
                   f"{args.cpu_sample:,} of the {args.n:,} points (same density and clustering); "
                   f"k-d tree Boruvka, {threads} threads; {done:,} points in {secs:.1f} s over "
                   f"{args.steps} steps")
    line = {
        "metric": METRIC, "value": value, "unit": "Mpoints/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "impl": "reference",
        "config": config_of(args.n, args.seed),
        "cpu_baseline": {"value": value, "unit": "Mpoints/s", "cores": threads, "kind": "oracle",
                         "sample": sample_desc},
        "e2e": {"value": value, "unit": "Mpoints/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_batched(args, rank, world, local):
    """The batched form: independent instances in one call per GPU.  With N
    GPUs one batch is split across the ranks by size (shard.partition_instances;
    no collective inside the method), timed from a barrier to the slowest
    rank.  Against the same instances one call each (identical output
    checked on every rank)."""
    import torch
    import paper_2207_00514_gb300 as pkg
    from paper_2207_00514_gb300 import shard
    import synth

    pkg.load_library()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    sizes = synth.batched_sizes(args.instances, seed=4, lo=100, hi=1_000_000)
    all_pts, all_offs = synth.batched_instances(sizes, seed=4)
    mine = shard.partition_instances(sizes, world)[rank]
    pts_np, offs = shard.local_batch(all_pts, all_offs, mine)
    del all_pts
    pts = torch.from_numpy(pts_np).to(dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        pkg.emst_compute_batched(pts, offs, stream=stream)
    torch.cuda.synchronize(dev)
    shard.barrier(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        eb, eo = pkg.emst_compute_batched(pts, offs, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = shard.max_over_ranks(e0.elapsed_time(e1) / args.steps, device=dev)
    e0.record(stream)
    singles = []
    for k in range(len(mine)):
        a, b = int(offs[k]), int(offs[k + 1])
        singles.append(pkg.emst_compute(pts[a:b], stream=stream) if b > a else None)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_seq = shard.max_over_ranks(e0.elapsed_time(e1), device=dev)
    ebn = pkg.edges_numpy(eb)
    same = all(s is None or np.array_equal(ebn[eo[k]:eo[k + 1]].view(np.uint8), pkg.edges_numpy(s).view(np.uint8))
               for k, s in enumerate(singles))
    differs = shard.max_over_ranks(0.0 if same else 1.0, device=dev)
    n = int(all_offs[-1])
    if rank == 0:
        print(json.dumps({
            "metric": f"batched EMST Mpoints/s ({len(sizes):,} independent 3D instances, one call per GPU)",
            "value": n / (ms / 1e3) / 1e6, "unit": "Mpoints/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{len(sizes)} instances, sizes log-uniform [100, 1e6] (seed 4), "
                                   "each 20 Gaussian blobs (sigma log-U[1e-3, 5e-2]) + 10% uniform, "
                                   "split across the GPUs by size",
                       "points": n, "points_rank0": len(pts_np)},
            "one_call_per_instance_ms": ms_seq,
            "speedup_over_one_call_per_instance": ms_seq / ms,
            "identical_output": differs == 0.0}), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_sweep(args, rank, world, local):
    """Throughput against n (1e4 .. 1e8) on the 2D blob and 3D halo
    generators: one JSON line per (generator, n), whole-call CUDA-event time
    with the input resident, best of the timed calls."""
    if rank != 0:
        return
    import torch
    import synth
    import paper_2207_00514_gb300 as pkg

    pkg.load_library()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    sizes = [10_000, 30_000, 100_000, 300_000, 1_000_000, 3_000_000, 10_000_000, 30_000_000,
             100_000_000]
    gens = {"2D blobs (config 2 generator, seed 1)": lambda n: synth.blobs(n, 2, 1),
            "3D halos (config 3 generator, seed 2)": lambda n: synth.halos(n, 2)}
    for name, gen in gens.items():
        for n in sizes:
            pts = torch.from_numpy(gen(n)).to(dev)
            out = torch.empty((n - 1, 3), dtype=torch.int32, device=dev)
            for _ in range(max(args.warmup, 2)):
                pkg.emst_compute(pts, out_edges=out, stream=stream)
            torch.cuda.synchronize(dev)
            best, rounds = None, 0
            for _ in range(max(args.steps, 3)):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                st = pkg.emst_compute_ex(pts, out_edges=out, stream=stream)[1]
                e1.record(stream)
                torch.cuda.synchronize(dev)
                ms = e0.elapsed_time(e1)
                rounds = st["rounds"]
                best = ms if best is None else min(best, ms)
            print(json.dumps({"workload": name, "n": n, "ms": round(best, 4),
                              "mpoints_per_s": round(n / best / 1e3, 2), "rounds": rounds}),
                  flush=True)
            del pts, out
            torch.cuda.empty_cache()


def run_mrd(args, rank, world, local):
    """The mutual-reachability MST (§4.5) on the 37M halo workload for
    k_pts = 1 (the EMST), 2, 4, 8, 16: whole-call time (core distances
    included) and the core-distance time alone, best of the timed calls."""
    if rank != 0:
        return
    import torch
    import paper_2207_00514_gb300 as pkg

    pkg.load_library()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    pts = torch.from_numpy(make_points(args.n, args.seed)).to(dev)
    n = pts.shape[0]
    out = torch.empty((n - 1, 3), dtype=torch.int32, device=dev)
    for k in [int(x) for x in args.mrd_k.split(",")]:
        for _ in range(max(args.warmup, 1)):
            pkg.emst_compute_ex(pts, out_edges=out, stream=stream, mrd_k=k)
        torch.cuda.synchronize(dev)
        best = None
        for _ in range(max(args.steps, 3)):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = pkg.emst_compute_ex(pts, out_edges=out, stream=stream, mrd_k=k)[1]
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1)
            if best is None or ms < best[0]:
                best = (ms, st)
        ms, st = best
        print(json.dumps({"workload": WORKLOAD, "n": n, "k_pts": k, "ms": round(ms, 3),
                          "core_ms": round(st["core_ms"], 3), "traverse_ms": round(st["traverse_ms"], 3),
                          "rounds": st["rounds"], "mpoints_per_s": round(n / ms / 1e3, 2)}), flush=True)


def run_dense(args, rank, world, local):
    """64- against 128-bit Morton codes on very dense clusters (synth.dense,
    --dense-n 3D points, seed 5): whole-call time, traversal time and node
    visits per query per round, best of the timed calls."""
    if rank != 0:
        return
    import torch
    import synth
    import paper_2207_00514_gb300 as pkg

    pkg.load_library()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    n = args.dense_n
    pts = torch.from_numpy(synth.dense(n, 3, 5)).to(dev)
    out = torch.empty((n - 1, 3), dtype=torch.int32, device=dev)
    for bits in (64, 128, 0):
        if bits == 64 and n > 4_000_000:
            print(json.dumps({"morton_bits": 64, "n": n, "skipped": "each query scans its whole "
                              "over-full 64-bit cell: minutes per call at this size"}), flush=True)
            continue
        for _ in range(max(args.warmup, 1)):
            pkg.emst_compute_ex(pts, out_edges=out, stream=stream, morton_bits=bits)
        torch.cuda.synchronize(dev)
        best = None
        for _ in range(max(args.steps, 3)):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = pkg.emst_compute_ex(pts, out_edges=out, stream=stream, morton_bits=bits)[1]
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1)
            if best is None or ms < best[0]:
                best = (ms, st)
        ms, st = best
        vis = pkg.emst_compute_ex(pts, out_edges=out, stream=stream, morton_bits=bits,
                                  count_visits=True)[1]
        print(json.dumps({"workload": f"{n:,} 3D points, 90% in 20,000 clusters with sigma "
                                      "log-U[1e-9, 1e-6] and power-law sizes, 10% uniform, seed 5",
                          "morton_bits": bits if bits else f"automatic ({st['morton_bits']})",
                          "code_collisions": st["code_collisions"], "ms": round(ms, 3),
                          "build_ms": round(st["build_ms"], 3),
                          "traverse_ms": round(st["traverse_ms"], 3), "rounds": st["rounds"],
                          "visits_per_query_round": round(vis["node_visits"] / n / vis["rounds"], 2),
                          "mpoints_per_s": round(n / ms / 1e3, 2)}), flush=True)


def run_dendrogram(args, rank, world, local):
    """The single-linkage dendrogram (emst_dendrogram) of the trees the
    library computes on the 37M halo workload -- the EMST and the
    mutual-reachability tree for k_pts = 8 (HDBSCAN*'s hierarchy) -- and of a
    seeded random tree of the same size: best and median device time of the
    timed calls (edges and outputs resident on the device), against the
    oracle's serial merge sequence on the same edges (one host core)."""
    if rank != 0:
        return
    import torch
    import synth
    import oracle
    import paper_2207_00514_gb300 as pkg

    pkg.load_library()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    pts = torch.from_numpy(make_points(args.n, args.seed)).to(dev)
    n = pts.shape[0]
    what = workload_name(n, args.seed)
    trees = [("EMST of " + what, lambda: pkg.emst_compute(pts)),
             ("mutual-reachability tree (k_pts = 8) of " + what,
              lambda: pkg.emst_compute_ex(pts, mrd_k=8)[0]),
             (f"random tree on {n:,} points (synth.tree_edges, seed 4)",
              lambda: torch.from_numpy(np.ascontiguousarray(synth.tree_edges(n, 4, "random"))
                                       .view(np.int32).reshape(-1, 3).copy()).to(dev))]
    if args.dg_tree != "all":
        trees = [trees[["emst", "mrd", "random"].index(args.dg_tree)]]
    link = torch.empty((n - 1, 4), dtype=torch.int32, device=dev)
    parent = torch.empty(2 * n - 1, dtype=torch.int32, device=dev)
    peak, peak_kind = measured_peaks()
    for name, make in trees:
        edges = make()
        torch.cuda.synchronize(dev)
        for _ in range(max(args.warmup, 1)):
            pkg.emst_dendrogram(edges, n, out_linkage=link, out_parent=parent, stream=stream)
        torch.cuda.synchronize(dev)
        times = []
        for _ in range(max(args.steps, 3)):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pkg.emst_dendrogram(edges, n, out_linkage=link, out_parent=parent, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            times.append(e0.elapsed_time(e1))
        e_np = pkg.edges_numpy(edges)
        t0 = time.perf_counter()
        oracle.dendrogram(e_np, n)
        cpu_s = time.perf_counter() - t0
        ms = min(times)
        # compulsory traffic: read the edges (12 B), write the rows (16 B) and
        # the parents (2 x 4 B) once per edge
        alg = (n - 1) * 36.0
        print(json.dumps({"workload": name, "n": n, "ms": round(ms, 3),
                          "median_ms": round(float(np.median(times)), 3),
                          "mpoints_per_s": round(n / ms / 1e3, 2),
                          "roofline": {"bound": "hbm", "algorithmic_bytes": alg,
                                       "achieved_gbs": round(alg / ms / 1e6, 1), "peak_gbs": peak,
                                       "peak_kind": peak_kind, "frac": round(alg / ms / 1e6 / peak, 4)},
                          "cpu_oracle_s": round(cpu_s, 3), "cpu_cores": 1}), flush=True)
        del edges


def run_once(args, rank, world, local):
    """One emst_compute call on the halo workload (--n, --seed) and nothing
    else: the command the profiler captures."""
    if rank != 0:
        return
    import torch
    import paper_2207_00514_gb300 as pkg
    pkg.load_library()
    torch.cuda.set_device(local)
    pts = torch.from_numpy(make_points(args.n, args.seed)).cuda()
    e = pkg.emst_compute_ex(pts, traversal=args.traversal)[0]
    torch.cuda.synchronize()
    print(json.dumps({"workload": workload_name(args.n, args.seed), "edges": int(e.shape[0])}), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.workload == "once":
        run_once(args, rank, world, local)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "batched":
        run_batched(args, rank, world, local)
        return
    if args.workload == "sweep":
        run_sweep(args, rank, world, local)
        return
    if args.workload == "mrd":
        run_mrd(args, rank, world, local)
        return
    if args.workload == "dense":
        run_dense(args, rank, world, local)
        return
    if args.workload == "dendrogram":
        run_dendrogram(args, rank, world, local)
        return

    import torch
    import paper_2207_00514_gb300 as pkg
    from paper_2207_00514_gb300 import shard

    pkg.load_library()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    seed = args.seed + 1000 * rank if world > 1 else args.seed
    pts_np = make_points(args.n, seed)
    n = len(pts_np)
    pts = torch.from_numpy(pts_np).to(dev)
    out = torch.empty((n - 1, 3), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    params = None
    if not args.no_learned:
        try:
            from paper_2207_00514_gb300 import learned
            params = learned.load(device=dev)
        except FileNotFoundError:
            params = None

    def timed(call, steps):
        """Run `call` (returning a stats dict) `steps` times between CUDA
        events on the launching stream, after a barrier; max over ranks."""
        shard.barrier(dev)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sts = [call() for _ in range(steps)]
        e1.record(stream)
        torch.cuda.synchronize(dev)
        shard.barrier(dev)
        return shard.max_over_ranks(e0.elapsed_time(e1) / steps, device=dev), sts

    plain = lambda: pkg.emst_compute_ex(pts, out_edges=out, stream=stream)[1]
    for _ in range(args.warmup):
        plain()
    torch.cuda.synchronize(dev)

    clocks = ClockSampler(local, args.clocks_dir)
    clocks.start()
    time.sleep(0.3)
    ms, sts = timed(plain, args.steps)
    clk = clocks.stop()
    value = world * n / (ms / 1e3) / 1e6
    launches = sum(st["kernel_launches"] for st in sts)
    rounds = sts[-1]["rounds"]
    phases = {k: float(np.mean([st[k + "_ms"] for st in sts])) for k in ("build", "rounds", "output", "traverse")}
    round_ms = [float(np.mean([st["round_traverse_ms"][r] for st in sts])) for r in range(rounds)]
    ref_edges = out.clone()

    # the learned-radius form (committed network) in its own timed region
    learned_form = None
    if params is not None:
        lcall = lambda: pkg.emst_compute_ex(pts, out_edges=out, stream=stream, mlp_params=params)[1]
        for _ in range(max(args.warmup, 1)):
            lcall()
        lms, lsts = timed(lcall, args.steps)
        launches += sum(st["kernel_launches"] for st in lsts)
        same = bool(torch.equal(out, ref_edges))
        lst = lsts[-1]
        learned_form = {"value": world * n / (lms / 1e3) / 1e6, "unit": "Mpoints/s", "ms_per_step": lms,
                        "vs_plain": ms / lms, "identical_tree": same,
                        "traverse_ms": round(float(np.mean([x["traverse_ms"] for x in lsts])), 3),
                        "search_with_proposed_cutoffs_ms": round(float(np.mean([x["learned_search_ms"] for x in lsts])), 3),
                        "rerun_fraction": lst["rerun_points"] / max(lst["queried_points"], 1)}

    # end to end through the C ABI with pinned host buffers (copies inside)
    e2e = None
    if not args.no_e2e:
        hpts = torch.from_numpy(pts_np).pin_memory()
        hout = torch.empty((n - 1, 3), dtype=torch.int32).pin_memory()
        hcall = lambda: pkg.emst_compute_ex(hpts, out_edges=hout, stream=stream)[1]
        hcall()
        ems, ests = timed(hcall, args.steps)
        launches += sum(st["kernel_launches"] for st in ests)
        e2e = {"value": world * n / (ems / 1e3) / 1e6, "unit": "Mpoints/s",
               "h2d_bytes_per_step": int(n * 3 * 4), "d2h_bytes_per_step": int((n - 1) * 12),
               "ms_per_step": ems}

    # per-round counts of the traversal (one extra, untimed call with counting on)
    vis = pkg.emst_compute_ex(pts, out_edges=out, stream=stream, count_visits=True)[1]
    torch.cuda.synchronize(dev)
    same_counted = bool(torch.equal(out, ref_edges))
    peak, peak_kind = measured_peaks()
    rb = traversal_round_bytes(n, vis["round_queries"], vis["round_distinct_nodes"])
    rr = min(len(rb), len(round_ms))
    tot_bytes, tot_ms = sum(rb[:rr]), sum(round_ms[:rr])
    achieved = tot_bytes / (tot_ms / 1e3) / 1e9 if tot_ms > 0 else 0.0
    per_round = {
        "ms": [round(x, 4) for x in round_ms[:rr]],
        "algorithmic_bytes": rb[:rr],
        "achieved_gbs": [round(b / (t / 1e3) / 1e9, 1) if t > 0 else None for b, t in zip(rb, round_ms)],
        "frac": [round(b / (t / 1e3) / 1e9 / peak, 4) if t > 0 else None for b, t in zip(rb, round_ms)],
        "queries": vis["round_queries"][:rr],
        "distinct_nodes": vis["round_distinct_nodes"][:rr],
        "visits": vis["round_visits"][:rr],
    }
    measured = (TRAVERSE_DRAM_BYTES_PER_ROUND if n == 37_000_000 and seed == 2
                and TRAVERSE_DRAM_BYTES_PER_ROUND and len(TRAVERSE_DRAM_BYTES_PER_ROUND) == rr else None)
    traffic = sum(measured) / rr if measured else None
    if measured:
        per_round["dram_bytes"] = measured
        per_round["dram_over_algorithmic"] = [round(d / b, 3) for d, b in zip(measured, rb)]
    roofline = {"bound": "hbm", "kernel": "k_traverse (Algorithm 2 queries, one thread per point)",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic,
                "peak_kind": (f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs copy)" if peak_kind == "measured"
                              else "fallback 6.8 TB/s"),
                "avg_launch_ms": tot_ms / max(rr, 1), "launches": rr,
                "algorithmic_bytes_per_launch": tot_bytes / max(rr, 1),
                "bytes_model": (f"round 0: {BYTES_FIRST_QUERY} B per query + {BYTES_RECORD_FIRST} B per distinct "
                                f"internal node visited; later rounds: {BYTES_POINT} B per point + "
                                f"{BYTES_SEARCH} B per query that searches + {BYTES_RECORD} B per distinct "
                                "internal node visited (counted by an instrumented call); time = the "
                                "round's traversal CUDA events in the timed calls"),
                "per_round": per_round}

    # the batched form (4,096 instances), one call, against one call per instance
    batched = None
    if rank == 0 and world == 1 and not args.no_batched_summary:
        batched = batched_summary(args, pkg, torch, dev, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        threads = os.cpu_count() or 1
        if args.cpu_full:
            dt = cpu_oracle_run(pts_np, threads)
            cpu = {"value": n / dt / 1e6, "unit": "Mpoints/s", "cores": threads, "kind": "oracle",
                   "sample": f"the whole workload ({n:,} points), k-d tree Boruvka, {threads} threads, {dt:.1f} s"}
        else:
            g = np.random.default_rng(12345)
            sample = window_sample(pts_np, args.cpu_sample, g)
            dt = cpu_oracle_run(sample, threads)
            cpu = {"value": len(sample) / dt / 1e6, "unit": "Mpoints/s", "cores": threads, "kind": "oracle",
                   "sample": f"a spatial window of {len(sample):,} points, k-d tree Boruvka, {threads} threads, {dt:.1f} s"}
        if args.cpu_single_sample > 0:
            g = np.random.default_rng(54321)
            sample = window_sample(pts_np, args.cpu_single_sample, g)
            dt1 = cpu_oracle_run(sample, 1)
            cpu["single_thread"] = {
                "value": len(sample) / dt1 / 1e6, "unit": "Mpoints/s", "cores": 1,
                "sample": f"a spatial window of {len(sample):,} points (same density and clustering), "
                          f"k-d tree Boruvka, 1 thread, {dt1:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Mpoints/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": config_of(args.n, args.seed),
            "form": "plain",
            "parallelism": f"{world} independent replica(s)" if world > 1 else "1 GPU",
            "detail": {"rounds": rounds, "phases_ms": {k: round(v, 3) for k, v in phases.items()},
                       "components_per_round": sts[-1]["components_per_round"],
                       "node_visits_per_query_per_round": round(vis["node_visits"] / float(n * max(vis["rounds"], 1)), 2),
                       "counted_call_identical_tree": same_counted,
                       "mfeatures_per_s": value * 3, "leaf_size": 1},
            "learned_form": learned_form,
            "batched_form": batched,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
            "paper_context": PAPER_CONTEXT,
        }
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


def batched_summary(args, pkg, torch, dev, stream):
    """The batched workload (4,096 independent 3D instances, sizes
    log-uniform in [100, 1e6], seed 4) in one emst_compute_batched call,
    against one emst_compute call per instance on the same device-resident
    points (identical output checked); CUDA events on the stream."""
    import synth
    sizes = synth.batched_sizes(args.instances, seed=4, lo=100, hi=1_000_000)
    pts_np, offs = synth.batched_instances(sizes, seed=4, workers=os.cpu_count() or 4)
    pts = torch.from_numpy(pts_np).to(dev)
    del pts_np
    pkg.emst_compute_batched(pts, offs, stream=stream)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    e0.record(stream)
    for _ in range(reps):
        eb, eo = pkg.emst_compute_batched(pts, offs, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / reps
    e0.record(stream)
    singles = []
    for k in range(len(sizes)):
        a, b = int(offs[k]), int(offs[k + 1])
        singles.append(pkg.emst_compute(pts[a:b], stream=stream) if b - a > 1 else None)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_seq = e0.elapsed_time(e1)
    same = all(s is None or torch.equal(eb[int(eo[k]):int(eo[k + 1])], s) for k, s in enumerate(singles))
    npts = int(offs[-1])
    del pts, eb, singles
    torch.cuda.empty_cache()
    return {"workload": f"{len(sizes):,} instances, sizes log-uniform [100, 1e6] (seed 4), each 20 "
                        "Gaussian blobs (sigma log-U[1e-3, 5e-2]) + 10% uniform",
            "points": npts, "ms": ms, "mpoints_per_s": npts / ms / 1e3,
            "one_call_per_instance_ms": ms_seq, "speedup_over_one_call_per_instance": ms_seq / ms,
            "identical_output": same}


if __name__ == "__main__":
    main()
