#!/usr/bin/env python3
"""JP-ADG benchmark: undirected edges coloured per second (ADG + JP) on GB300.

One step = one gc_color_graph call on a graph resident in HBM: every ADG
round (partition, UPDATE, threshold) and the whole JP colouring, with the
batch ids and colours written to device buffers.  `value` is m * steps / time
over the timed region (CUDA events on the launching stream, max over ranks).
`e2e` is the same metric through gc_color_graph_host with the graph in
page-locked host memory: the host->device copy of the CSR and the
device->host copy of the colours are inside every timed step.

Default workload: R-MAT scale 24, edge factor 16, (a,b,c,d) =
(.57,.19,.19,.05), duplicates and self-loops removed, eps = 1/100, tie-break
seed 42.  The CSR (2 GB of col_idx) is larger than the 129 MB L2, so no L2
flush is needed between steps.

--impl reference times the CPU oracle (plain single-threaded C: ADG with
fresh degree sums, then Greedy in priority order) on a bounded sample of the
same family.  With --gpus N > 1 each rank colours its own replica (the
single-graph path has no exchange step here): weak scaling, no collective on
the data path; a barrier and a max-reduction of the elapsed time bracket the
timed region.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "undirected edges colored/s (ADG+JP) and HBM GB/s vs peak; graphs/s batched vs per-graph"

WORKLOADS = {
    "rmat24": dict(kind="rmat", scale=24, ef=16, gen_seed=1, eps=(1, 100), seed=42,
                   desc="R-MAT scale 24, edge factor 16, (a,b,c,d)=(.57,.19,.19,.05), dedup, "
                        "no self-loops, eps=1/100, tie-break seed 42"),
    "rmat20": dict(kind="rmat", scale=20, ef=16, gen_seed=1, eps=(1, 100), seed=42,
                   desc="R-MAT scale 20, edge factor 16, (a,b,c,d)=(.57,.19,.19,.05), eps=1/100, seed 42"),
    "rmat22": dict(kind="rmat", scale=22, ef=16, gen_seed=1, eps=(1, 100), seed=42,
                   desc="R-MAT scale 22, edge factor 16, (a,b,c,d)=(.57,.19,.19,.05), eps=1/100, seed 42"),
    "grid256": dict(kind="grid3", k=256, perm_seed=7, eps=(1, 100), seed=42,
                    desc="3D 7-point grid 256^3, seeded vertex permutation, eps=1/100, seed 42"),
    "er": dict(kind="er", n=16384, m=81920, gen_seed=1, eps=(1, 100), seed=42,
               desc="Erdos-Renyi G(n=16384, m=81920), eps=1/100, seed 42"),
    "serve": dict(kind="serve", requests=1000, pool=48, n_lo=1000, n_hi=2_000_000, seed=42, budget=40 << 30,
                  load=0.5,
                  desc="serving: 1000 requests, Poisson arrivals at half the measured capacity; graphs drawn from "
                       "a pool of 48 generated ones, n log-uniform in [1000, 2000000], R-MAT (.57,.19,.19,.05, "
                       "edge factor 8-32) or Barabasi-Albert (m 2-16) 50/50; eps 1/100 or 1/10 50/50, seed per "
                       "request; 40 GB device-memory budget"),
    "batch4096": dict(kind="batch", count=4096, n_lo=100, n_hi=200_000, seed=42, eps=(1, 100),
                      desc="4096 graphs, n log-uniform in [100, 200000], Erdos-Renyi (avg deg 8) / "
                           "Barabasi-Albert (m=4) / 2D grid, packed as one disjoint union, eps=1/100, "
                           "seed 42+g"),
}

# Algorithmic bytes (what the method must move; random touches at 4 B) of the
# three kernel groups that take the time, summed over their launches in one
# step.  ADG's UPDATE sweeps every directed edge once over all rounds: the
# neighbour id and the neighbour's state (8 B per edge) plus one decrement
# per surviving neighbour (4 B).  The JP bulk kernels read, per vertex outside
# the core, its row offsets, own batch, list entry and colour write (28 B), per
# directed edge the neighbour id and its batch (8 B) and per predecessor edge
# its colour (4 B; half of the edges).  The core block reads its compacted
# 16-bit predecessor lists, the 8-byte list offsets and writes the colours.
def group_bytes(n_nonisolated, nnz, st):
    upd = 8 * nnz + 4 * st["sum_decrements"]
    n_bulk = n_nonisolated - st["core_vertices"]
    e_bulk = nnz - st["core_degree_sum"]
    bulk = 28 * n_bulk + 8 * e_bulk + 4 * (e_bulk // 2)
    core = 2 * st["core_preds"] + 12 * st["core_vertices"]
    return {"adg_update_kernel": upd, "jp_color_kernel": bulk, "jpf_core_solve_kernel": core}


# Whole path (ADG + JP), algorithmic bytes: ADG reads D and writes the
# survivor list per vertex-round (8 * sum|U|), writes the batch (4n), reads the
# row offsets of removed vertices (16n), streams col_idx and the neighbours'
# state (8 nnz) and decrements survivors (4 per decrement); JP reads row
# offsets, own batch and writes the colour per vertex (28n), streams col_idx
# and the neighbours' batch (8 nnz) and reads the predecessors' colours (2 nnz).
def path_bytes(n, nnz, sum_u, decrements):
    adg = 8 * sum_u + 4 * n + 16 * n + 8 * nnz + 4 * decrements
    jp = 28 * n + 8 * nnz + 4 * (nnz // 2)
    return adg + jp


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of a
# kernel, from a one-kernel ncu capture, keyed by (workload, kernel).  Each
# entry carries the SHA-256 prefix of the source file the kernel was built
# from at capture time; once that file changes the figure no longer
# describes the kernel and kernel_traffic() reports None.
KERNEL_TRAFFIC = {
    # R-MAT scale 24, the fourth call of `bench.py --steps 1 --warmup 3`; mean
    # over the launches of one call (4 bulk, 7 UPDATE, 1 core)
    ("rmat24", "jp_color_kernel"): (1119338816, "gc_jp.cu", "cab66866d06a1d97"),
    ("rmat24", "adg_update_kernel"): (355431424, "gc_adg.cu", "ee04c8d9eef69878"),
    ("rmat24", "jpf_core_solve_kernel"): (34953472, "gc_jp.cu", "cab66866d06a1d97"),
}


def kernel_traffic(workload, kernel):
    ent = KERNEL_TRAFFIC.get((workload, kernel))
    if not ent:
        return None
    nbytes, src, sha = ent
    import hashlib
    try:
        with open(os.path.join(ROOT, "paper_2008_11321_gb300", "csrc", src), "rb") as f:
            cur = hashlib.sha256(f.read()).hexdigest()[:16]
    except OSError:
        return None
    return nbytes if cur == sha else None


def load_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def sync_ranks(world, dev=None):
    """Bracket of a timed region: a barrier across the ranks (when there are
    several) and a synchronise of this rank's device."""
    import torch
    import torch.distributed as dist
    if world > 1:
        dist.barrier()
    if dev is not None:
        torch.cuda.synchronize(dev)


def max_over_ranks(seconds, world, device="cpu"):
    """The slowest rank's time: every rank passes its own and gets the max."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_step, steps, world, t_max):
    """Whole-job throughput of `world` replicas that each processed
    units_per_step units per step for `steps` steps in t_max seconds."""
    return units_per_step * steps * world / t_max


def make_graph(w, pinned=False):
    import graphgen as gg
    if w["kind"] == "rmat":
        return gg.rmat(w["scale"], w["ef"], seed=w["gen_seed"], pinned=pinned)
    if w["kind"] == "grid3":
        k = w["k"]
        return gg.grid(k, k, k, perm_seed=w["perm_seed"], pinned=pinned)
    if w["kind"] == "er":
        return gg.erdos_renyi(w["n"], w["m"], w["gen_seed"], pinned=pinned)
    raise ValueError(w["kind"])


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id: str):
        self.proc = None
        self.device_id = device_id

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", self.device_id],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sms, maxs, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                maxs.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sms:
            return None
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": max(maxs), "reasons": sorted(reasons),
                "samples": len(sms)}


def cpu_baseline(w_name, seconds_target=10.0, median=False, dec=False, ordered=False, itr=False, kind=None,
                 graph=None):
    """The oracle as it stands, single-threaded: on the benchmark's own
    R-MAT scale 24 graph (one run, about 8 s) for the default JP-ADG line,
    else on a bounded sample of the same family (R-MAT scale 22 for the
    R-MAT workloads)."""
    import numpy as np

    import graphgen as gg
    import oracle
    w = WORKLOADS[w_name]
    plain = not (median or dec or ordered or itr or kind is not None)
    if graph is not None and plain and w_name == "rmat24":
        g = graph
        desc = w["desc"] + " (the benchmarked graph itself)"
        seconds_target = 0.0  # one run
    elif w["kind"] == "rmat":
        sample = dict(w, scale=min(w["scale"], 22))
        g = make_graph(sample)
        desc = f"R-MAT scale {sample['scale']} edge factor {w['ef']} (same a,b,c,d), eps=1/100"
    elif w["kind"] == "grid3":
        g = gg.grid(128, 128, 128, perm_seed=w["perm_seed"])
        desc = "3D grid 128^3, seeded permutation, eps=1/100"
    else:
        g = make_graph(w)
        desc = w["desc"]
    p, q = w["eps"]
    reps, total = 0, 0.0
    while (reps == 0 or total < seconds_target) and reps < 50:
        t0 = time.perf_counter()
        if kind is not None:
            oracle.jp_color(g, oracle.priority_kind(g, kind, w["seed"]))
        elif median:
            oracle.jp_adg_m(g, w["seed"])
        elif itr:
            oracle.dec_itr(g, np.ones(g.n, dtype=np.int32), 1, w["seed"])
        elif dec:
            oracle.dec_adg_itr(g, p, q, w["seed"])
        elif ordered:
            oracle.jp_adg_o(g, p, q)
        else:
            oracle.jp_adg(g, p, q, w["seed"])
        total += time.perf_counter() - t0
        reps += 1
    what = ("ADG-M + Greedy" if median else "ITR (one partition)" if itr else "ADG + DEC-ADG-ITR" if dec
            else "ADG-O + Greedy" if ordered else f"priority kind {kind} + Greedy" if kind is not None
            else "ADG + Greedy")
    return {"value": g.m * reps / total, "unit": "edges/s", "cores": 1, "kind": "oracle",
            "sample": f"{desc}: n={g.n}, m={g.m}, {reps} run(s) of {what}, {total:.1f} s"}


PRIORITIES = {"r": (0, "JP-R"), "ff": (1, "JP-FF"), "lf": (2, "JP-LF"), "llf": (3, "JP-LLF"), "sl": (4, "JP-SL")}


def run_variant(args, rank, world):
    """A JP variant other than JP-ADG (Section 4.1): one step is the priority
    (gc_make_priority_kind) plus JP (gc_jp_color) on the resident graph."""
    import torch
    import torch.distributed as dist
    from paper_2008_11321_gb300 import _build
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    if rank == 0:
        _build.build()
    if world > 1:
        dist.barrier()
    import paper_2008_11321_gb300 as gcp
    kind, name = PRIORITIES[args.priority]
    w = WORKLOADS[args.workload]
    seed = w["seed"]
    g = make_graph(w, pinned=True)
    n, nnz, m = g.n, g.nnz, g.m
    dg = gcp.DeviceGraph(torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col_idx).to(dev))
    key = torch.empty(n, dtype=torch.int64, device=dev)
    color = torch.empty(n, dtype=torch.int32, device=dev)
    ctx = gcp.Context(local, args.options)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        ctx.gc_make_priority_kind(dg, kind, seed, key)
        nc = ctx.gc_jp_color(dg, key, color)
    ctx.gc_set_timing(True)
    sampler = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0])
    sampler.start()
    time.sleep(0.3)
    sync_ranks(world, dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    launches, bulk_ms = 0, 0.0
    for _ in range(args.steps):
        ctx.gc_make_priority_kind(dg, kind, seed, key)
        launches += ctx.gc_get_stats().launches
        nc = ctx.gc_jp_color(dg, key, color)
        st = ctx.gc_get_stats()
        launches += st.launches
        bulk_ms += st.ms_jp_color
    ev1.record(stream)
    sync_ranks(world, dev)
    clocks = sampler.stop()
    t_max = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, world, dev)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    peak, peak_kind = load_peak()
    # JP bulk over all vertices: 28 B per vertex, 12 B per edge (neighbour id,
    # its 8-byte key), 4 B per predecessor edge (its colour; half the edges)
    kbytes = 28 * n + 12 * nnz + 2 * nnz
    kms = bulk_ms / args.steps
    achieved = kbytes / (kms / 1e3) / 1e9 if kms > 0 else 0.0
    line = {
        "metric": METRIC, "value": job_rate(m, args.steps, world, t_max), "unit": "edges/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": w["desc"].replace("eps=1/100, ", ""), "priority": name, "n": n, "m": m,
                   "seed": seed, "num_colors": nc,
                   "l2": f"inputs larger than L2 (col_idx {4 * nnz / 1e9:.2f} GB), no flush"},
        "roofline": {"bound": "hbm", "kernel": "jp_color_kernel", "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                     "algorithmic_bytes_per_launch": kbytes, "ms_per_launch": kms, "launches_per_step": 1},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, kind=kind)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_dec(args, rank, world):
    """DEC-ADG-ITR (Section 4.3): one step is gc_color_graph_dec_itr (ADG,
    then the partitions coloured from the top by SIM-COL in its ITR form) on
    the resident graph.  --algo itr: the same colouring with every vertex in
    one partition (plain ITR, the paper's point of comparison), through
    gc_dec_itr_color."""
    import torch
    import torch.distributed as dist
    from paper_2008_11321_gb300 import _build
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    if rank == 0:
        _build.build()
    if world > 1:
        dist.barrier()
    import paper_2008_11321_gb300 as gcp
    w = WORKLOADS[args.workload]
    p, q = w["eps"]
    seed = w["seed"]
    g = make_graph(w, pinned=True)
    n, nnz, m = g.n, g.nnz, g.m
    dg = gcp.DeviceGraph(torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col_idx).to(dev))
    color = torch.empty(n, dtype=torch.int32, device=dev)
    batch = torch.empty(n, dtype=torch.int32, device=dev)
    itr = args.algo == "itr"
    ones = torch.ones(n, dtype=torch.int32, device=dev)
    ctx = gcp.Context(local, args.options)
    stream = torch.cuda.current_stream(dev)

    def colour_step():
        if itr:
            return ctx.gc_dec_itr_color(dg, ones, 1, seed, color), 1
        return ctx.gc_color_graph_dec_itr(dg, p, q, seed, color, batch)

    for _ in range(args.warmup):
        nc, nr = colour_step()
    ctx.gc_set_timing(True)
    sampler = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0])
    sampler.start()
    time.sleep(0.3)
    sync_ranks(world, dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    steps = []
    for _ in range(args.steps):
        nc, nr = colour_step()
        st = ctx.gc_get_stats()
        steps.append({k: getattr(st, k) for k, _ in st._fields_})
    ev1.record(stream)
    sync_ranks(world, dev)
    clocks = sampler.stop()
    t_max = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, world, dev)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    mean = lambda k: statistics.mean(x[k] for x in steps)  # noqa: E731
    last = steps[-1]
    peak, peak_kind = load_peak()
    n_nonisolated = int((g.degrees() > 0).sum())
    inner = last["dec_internal_edges"]
    # extraction, summed over its one launch per partition: per non-isolated
    # vertex its row offsets, list entry and state write (24 B); per CSR entry
    # the neighbour id and its state word (8 B); per internal entry the copy
    # to the internal list (4 B).  UPDATE as in the JP-ADG line.
    gb = {"adg_update_kernel": 8 * nnz + 4 * last["sum_decrements"],
          "dec_extract_kernel": 24 * n_nonisolated + 8 * nnz + 4 * inner}
    groups = {"adg_update_kernel": (mean("ms_adg_update"), last["adg_rounds"]),
              "dec_extract_kernel": (mean("ms_dec_extract"), last["adg_rounds"])}
    if itr:
        groups.pop("adg_update_kernel")
    kname = max(groups, key=lambda k: groups[k][0])
    kms, kl = groups[kname]
    if itr:
        kl = 1
    achieved = gb[kname] / (kms / 1e3) / 1e9 if kms > 0 else 0.0
    line = {
        "metric": METRIC, "value": job_rate(m, args.steps, world, t_max), "unit": "edges/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": w["desc"], "algorithm": "ITR (one partition)" if itr else "DEC-ADG-ITR", "n": n,
                   "m": m, "eps": None if itr else f"{p}/{q}",
                   "seed": seed, "adg_rounds": nr, "num_colors": nc, "sim_iterations": last["sim_iterations"],
                   "internal_entries": inner,
                   "l2": f"inputs larger than L2 (col_idx {4 * nnz / 1e9:.2f} GB), no flush"},
        "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None if itr else kernel_traffic(args.workload, kname),
                     "algorithmic_bytes_per_launch": gb[kname] / kl, "ms_per_launch": kms / kl,
                     "launches_per_step": kl,
                     "groups_ms": {"adg_update_kernel": mean("ms_adg_update"),
                                   "dec_extract_kernel": mean("ms_dec_extract"),
                                   "dec_check_pick_kernels": mean("ms_dec_iterate")}},
        "path": {"ms_adg": mean("ms_adg"), "ms_color": mean("ms_jp")},
        "gpu_launches": sum(x["launches"] for x in steps),
        "clocks": clocks,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, dec=True, itr=itr)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import graphgen as gg  # noqa: F401
    import oracle
    w = WORKLOADS[args.workload]
    if w["kind"] == "serve":  # each step: the oracle on the 8 smallest requests
        pool, stream = serve_requests(w)
        reqs = sorted([(pool[k], e, sd) for k, e, sd in stream], key=lambda r: r[0].nnz)[:8]
        for _ in range(args.warmup):
            oracle.jp_adg(reqs[0][0], *reqs[0][1], reqs[0][2])
        t0 = time.perf_counter()
        for _ in range(args.steps):
            for g, e, sd in reqs:
                oracle.jp_adg(g, e[0], e[1], sd)
        dt = time.perf_counter() - t0
        value = sum(g.m for g, _, _ in reqs) * args.steps / dt
        desc = "the 8 smallest requests of the serving workload, ADG + Greedy each"
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": "edges/s",
                          "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                          "config": {"workload": w["desc"], "sample": desc},
                          "cpu_baseline": {"value": value, "unit": "edges/s", "cores": 1, "kind": "oracle",
                                           "sample": desc},
                          "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}), flush=True)
        return 0
    if w["kind"] == "batch":  # each step: the oracle on the first 64 graphs of the batch
        sample = [gg.make_batch_graph(f, nv, w["seed"] + i)
                  for i, (f, nv) in enumerate(gg.batch_recipe(64, w["n_lo"], w["n_hi"], w["seed"]))]
        p, q = w["eps"]
        for _ in range(args.warmup):
            oracle.jp_adg(sample[0], p, q, w["seed"])
        t0 = time.perf_counter()
        for _ in range(args.steps):
            for i, sg in enumerate(sample):
                oracle.jp_adg(sg, p, q, w["seed"] + i)
        dt = time.perf_counter() - t0
        value = len(sample) * args.steps / dt
        desc = "first 64 graphs of the batch, ADG + Greedy each"
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": "graphs/s",
                          "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                          "config": {"workload": w["desc"], "sample": desc},
                          "cpu_baseline": {"value": value, "unit": "graphs/s", "cores": 1, "kind": "oracle",
                                           "sample": desc},
                          "e2e": {"value": value, "unit": "graphs/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}), flush=True)
        return 0
    # each step: the oracle on a bounded sample (R-MAT scale 22 for R-MAT)
    if w["kind"] == "rmat":
        sample = dict(w, scale=min(w["scale"], 22))
        desc = f"R-MAT scale {sample['scale']} edge factor {w['ef']}"
    elif w["kind"] == "grid3":
        sample = dict(w, k=min(w["k"], 96))
        desc = f"3D grid {sample['k']}^3 permuted"
    else:
        sample = w
        desc = w["desc"]
    g = make_graph(sample)
    p, q = w["eps"]
    for _ in range(args.warmup):
        oracle.jp_adg(g, p, q, w["seed"])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.jp_adg(g, p, q, w["seed"])
    dt = time.perf_counter() - t0
    value = g.m * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": w["desc"], "sample": f"{desc}: n={g.n}, m={g.m}"},
            "cpu_baseline": {"value": value, "unit": "edges/s", "cores": 1, "kind": "oracle",
                             "sample": f"{desc}: n={g.n}, m={g.m}, ADG + Greedy per step"},
            "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _phase(name):
    """Synchronises the device and notes on stderr that a phase ended, so an
    asynchronous CUDA error surfaces in the phase that caused it."""
    import torch
    torch.cuda.synchronize()
    print(f"[bench] {name} done", file=sys.stderr, flush=True)


def _timed(stream, fn, steps):
    """Device time (s) of `steps` calls of fn on `stream`, CUDA events."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3


def measure_batch(w, dev, steps, warmup, options=None, world=1, tune_cache=None):
    """The batched workload: the persistent path (one launch), the segmented
    path, the autotuned options, and one gc_color_graph call per graph on
    the same graphs; colourings checked identical.  Returns a dict."""
    import numpy as np
    import torch
    import graphgen as gg
    import paper_2008_11321_gb300 as gcp
    from paper_2008_11321_gb300 import tuning
    G = w["count"]
    g, off = gg.batch(G, w["n_lo"], w["n_hi"], w["seed"], pinned=True)
    p, q = w["eps"]
    jobs = [(p, q, w["seed"] + i) for i in range(G)]
    db = gcp.DeviceBatch(torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col_idx).to(dev),
                         torch.from_numpy(off).to(dev))
    color = torch.empty(db.n, dtype=torch.int32, device=dev)
    ncol = torch.empty(G, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    ctx = gcp.Context(dev.index, options)
    res = {}
    launches = {}
    for name, mode in (("persistent", gcp.GC_BATCH_PERSISTENT), ("segmented", gcp.GC_BATCH_SEGMENTED)):
        ctx.gc_set_options(dict(ctx.gc_get_options().as_dict(), batch_mode=mode))
        for _ in range(warmup):
            ctx.gc_color_batch(db, jobs, color, None, ncol)
        ctx.gc_set_timing(True)
        t = _timed(stream, lambda: ctx.gc_color_batch(db, jobs, color, None, ncol), steps) / steps
        st = ctx.gc_get_stats()
        ctx.gc_set_timing(False)
        res[name] = {"ms_per_step": t * 1e3, "graphs_per_s": G / t, "kernel_ms": st.ms_adg_update,
                     "launches_per_step": st.launches}
        _phase(f"batch {name}")
        launches[name] = st.launches * steps
        ref_color = color.clone() if name == "persistent" else ref_color
    identical_paths = bool(torch.equal(ref_color, color))
    sum_u, dec = st.sum_U, st.sum_decrements
    # the autotuner's choice for this batch class (searched unless cached)
    ctx.gc_set_options(options or {})
    rec = tuning.tune_batch(ctx, db, jobs, cache=tune_cache, reps=2)
    _phase("batch tuning")
    for _ in range(warmup):
        ctx.gc_color_batch(db, jobs, color, None, ncol)
    sync_ranks(world, dev)
    t_tuned = max_over_ranks(_timed(stream, lambda: ctx.gc_color_batch(db, jobs, color, None, ncol), steps),
                             world, dev) / steps
    launches["tuned"] = ctx.gc_get_stats().launches * steps
    identical_tuned = bool(torch.equal(ref_color, color))
    _phase("batch tuned")
    # per-graph plain launches of the same graphs (local ids), one pass
    rp, ci = g.row_ptr, g.col_idx
    graphs = []
    for i in range(G):
        a, b = int(off[i]), int(off[i + 1])
        graphs.append(gcp.DeviceGraph(torch.from_numpy(rp[a:b + 1] - rp[a]).to(dev),
                                      torch.from_numpy(ci[rp[a]:rp[b]] - np.int32(a)).to(dev)))
    single = torch.empty(db.n, dtype=torch.int32, device=dev)
    for i in range(min(8, G)):
        ctx.gc_color_graph(graphs[i], p, q, w["seed"] + i, single[int(off[i]):int(off[i + 1])])
    t_single = _timed(stream, lambda: [ctx.gc_color_graph(graphs[i], p, q, w["seed"] + i,
                                                          single[int(off[i]):int(off[i + 1])]) for i in range(G)], 1)
    identical_single = bool(torch.equal(single, ref_color))
    _phase("batch per-graph")
    # end to end: packed CSR host -> device, batch call, colours device -> host
    hcolor = torch.empty(db.n, dtype=torch.int32, pin_memory=True)
    rp_h, ci_h, off_h = torch.from_numpy(g.row_ptr), torch.from_numpy(g.col_idx), torch.from_numpy(off)

    def e2e_step():
        db2 = gcp.DeviceBatch(rp_h.to(dev, non_blocking=True), ci_h.to(dev, non_blocking=True),
                              off_h.to(dev, non_blocking=True))
        ctx.gc_color_batch(db2, jobs, color, None, ncol)
        hcolor.copy_(color, non_blocking=True)
    sync_ranks(world, dev)
    t_e2e = max_over_ranks(_timed(stream, e2e_step, steps), world, dev) / steps
    ctx.close()
    _phase("batch e2e")
    peak, peak_kind = load_peak()
    pb = path_bytes(db.n, db.nnz, sum_u, dec)
    kms = res["persistent"]["kernel_ms"]
    achieved = pb / (kms / 1e3) / 1e9 if kms > 0 else 0.0
    return {
        "graphs": G, "n": db.n, "m": db.nnz // 2, "t_tuned": t_tuned, "t_e2e": t_e2e,
        "graphs_per_s": G / t_tuned, "edges_per_s": (db.nnz // 2) / t_tuned,
        "paths": res, "identical_colourings": identical_paths and identical_tuned and identical_single,
        "tuned": {"options": rec["options"], "searched": rec["searched"], "best_ms": rec["best_ms"],
                  "start_ms": rec["start_ms"]},
        "per_graph": {"value": G / t_single, "unit": "graphs/s", "ms_total": t_single * 1e3},
        "speedup_vs_per_graph": t_single / t_tuned,
        "e2e": {"value": G / t_e2e, "unit": "graphs/s", "h2d_bytes_per_step": 8 * (db.n + 1) + 4 * db.nnz + 8 * (G + 1),
                "d2h_bytes_per_step": 4 * db.n},
        "roofline": {"bound": "hbm", "kernel": "batch_persistent_kernel", "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                     "algorithmic_bytes_per_launch": pb, "ms_per_launch": kms, "launches_per_step": 1},
        "path": {"algorithmic_bytes_per_step": pb, "sum_U": sum_u, "decrements": dec},
        "gpu_launches": launches["tuned"],
    }


def run_batch_path(args):
    """One path of gc_color_batch on the batch workload, nothing else: W
    warm-up calls, then K timed calls (CUDA events).  For profiling a path's
    kernels; the default batch line compares both paths, the tuned options
    and per-graph calls."""
    import torch
    import graphgen as gg
    from paper_2008_11321_gb300 import _build
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    _build.build()
    import paper_2008_11321_gb300 as gcp
    w = WORKLOADS[args.workload]
    G = w["count"]
    g, off = gg.batch(G, w["n_lo"], w["n_hi"], w["seed"])
    p, q = w["eps"]
    jobs = [(p, q, w["seed"] + i) for i in range(G)]
    db = gcp.DeviceBatch(torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col_idx).to(dev),
                         torch.from_numpy(off).to(dev))
    color = torch.empty(db.n, dtype=torch.int32, device=dev)
    ncol = torch.empty(G, dtype=torch.int32, device=dev)
    mode = gcp.GC_BATCH_PERSISTENT if args.batch_path == "persistent" else gcp.GC_BATCH_SEGMENTED
    ctx = gcp.Context(0, dict(args.options or {}, batch_mode=mode))
    for _ in range(args.warmup):
        ctx.gc_color_batch(db, jobs, color, None, ncol)
    torch.cuda.synchronize()
    t = _timed(torch.cuda.current_stream(dev), lambda: ctx.gc_color_batch(db, jobs, color, None, ncol),
               args.steps) / args.steps
    st = ctx.gc_get_stats()
    ctx.close()
    print(json.dumps({"metric": METRIC, "value": G / t, "unit": "graphs/s", "n_gpus": 1, "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
                      "config": {"workload": w["desc"], "path": args.batch_path, "graphs": G, "n": db.n,
                                 "m": db.nnz // 2},
                      "gpu_launches": st.launches * args.steps}), flush=True)
    return 0


def run_batch(args, rank, world):
    """Batched form: gc_color_batch colours every graph of the packed batch
    (with the autotuned options: the persistent one-launch path or the
    segmented one); the comparison is one gc_color_graph call per graph on
    the same GPU (graphs/s both ways, colourings checked identical)."""
    import torch
    import torch.distributed as dist
    from paper_2008_11321_gb300 import _build, tuning
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    if world > 1:  # replicas: every rank colours its own copy of the batch
        dist.init_process_group("nccl", device_id=dev)
    if rank == 0:
        _build.build()
    if world > 1:
        dist.barrier()
    w = WORKLOADS[args.workload]
    sampler = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0])
    sampler.start()
    b = measure_batch(w, dev, args.steps, args.warmup, args.options, world, tuning.TuningCache(args.tune_cache))
    clocks = sampler.stop()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    line = {"metric": METRIC, "value": job_rate(b["graphs"], 1, world, b["t_tuned"]), "unit": "graphs/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": b["t_tuned"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": w["desc"], "graphs": b["graphs"], "n": b["n"], "m": b["m"],
                       "options": b["tuned"]["options"],
                       "l2": f"inputs larger than L2 (col_idx {8 * b['m'] / 1e9:.2f} GB), no flush"},
            "paths": b["paths"], "tuned": b["tuned"], "identical_colourings": b["identical_colourings"],
            "per_graph": b["per_graph"], "speedup_vs_per_graph": b["speedup_vs_per_graph"],
            "edges_per_s": job_rate(b["m"], 1, world, b["t_tuned"]),
            "e2e": dict(b["e2e"], value=job_rate(b["graphs"], 1, world, b["t_e2e"])),
            "roofline": b["roofline"], "path": b["path"], "gpu_launches": b["gpu_launches"], "clocks": clocks}
    if world > 1:
        line["config"]["parallelism"] = "replicas"
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def serve_requests(w):
    """The serving workload: a pool of generated graphs (n log-uniform in
    [n_lo, n_hi]; R-MAT with edge factor 8-32 or Barabasi-Albert with m 2-16,
    50/50) and the request stream drawn from it (graph, eps 1/100 or 1/10,
    seed).  Returns (pool, [(pool index, eps, seed)])."""
    import math
    import numpy as np
    import graphgen as gg
    rng = np.random.default_rng(w["seed"])
    pool = []
    lo, hi = math.log(w["n_lo"]), math.log(w["n_hi"])
    for i in range(w["pool"]):
        n = int(round(math.exp(lo + rng.random() * (hi - lo))))
        if rng.random() < 0.5:
            scale = max(1, int(round(math.log2(n))))
            pool.append(gg.rmat(scale, int(rng.integers(8, 33)), seed=w["seed"] + i))
        else:
            pool.append(gg.barabasi_albert(n, int(rng.integers(2, 17)), w["seed"] + i))
    reqs = [(int(rng.integers(len(pool))), (1, 100) if rng.random() < 0.5 else (1, 10), w["seed"] + 1000 + i)
            for i in range(w["requests"])]
    return pool, reqs


def _log_batch(slot, reqs, seconds, errors):
    """--debug: one stderr line per serving batch."""
    bad = [e for e in errors if e]
    print(f"[serve] slot {slot} graphs {len(reqs)} n {sum(r.n for r in reqs)} nnz {sum(r.nnz for r in reqs)} "
          f"max_nnz {max(r.nnz for r in reqs)} {seconds * 1e3:.1f} ms" + (f" ERROR {bad[0]}" if bad else ""),
          file=sys.stderr, flush=True)


def measure_serve(w, dev_index, world=1, slots=2, debug=False):
    """Continuous batching: the capacity with every request submitted at
    once, then Poisson arrivals at `load` x capacity (latency from submission
    to colours on the host), and the same requests as one gc_color_graph call
    each on resident graphs (device time)."""
    import numpy as np
    import torch
    import paper_2008_11321_gb300 as gcp
    from paper_2008_11321_gb300.serve import ColoringServer, latency_summary
    pool, reqs_in = serve_requests(w)
    edges = sum(pool[k].m for k, _, _ in reqs_in)
    with ColoringServer(dev_index, memory_budget=w["budget"], slots=slots,
                        on_batch=_log_batch if debug else None) as srv:
        # warm-up: single requests, then one closed loop (the contexts'
        # buffers grow once)
        for k, e, sd in reqs_in[:4]:
            srv.submit(pool[k].row_ptr, pool[k].col_idx, e[0], e[1], sd).result()
        _phase("serve warm-up singles")
        for r in [srv.submit(pool[k].row_ptr, pool[k].col_idx, e[0], e[1], sd) for k, e, sd in reqs_in]:
            r.result()
        _phase("serve warm-up closed loop")
        t0 = time.perf_counter()
        rs = [srv.submit(pool[k].row_ptr, pool[k].col_idx, e[0], e[1], sd) for k, e, sd in reqs_in]
        for r in rs:
            r.result()
        t_closed = time.perf_counter() - t0
        cap = len(reqs_in) / t_closed
        _phase("serve closed loop")
        rng = np.random.default_rng(w["seed"] + 1)
        rate = w["load"] * cap
        n_batches0 = len(srv.batches)
        srv.reset_occupancy()
        sync_ranks(world)
        t0 = time.perf_counter()
        rs = []
        for k, e, sd in reqs_in:
            rs.append(srv.submit(pool[k].row_ptr, pool[k].col_idx, e[0], e[1], sd))
            time.sleep(rng.exponential(1.0 / rate))
        for r in rs:
            r.result()
        t_open = time.perf_counter() - t0
        occ = srv.occupancy()
        batches = srv.batches[n_batches0:]
        _phase("serve open loop")
        served = {i: r.result() for i, r in enumerate(rs[:16])}
    # the same requests, one gc_color_graph call each on resident graphs
    dev = torch.device("cuda", dev_index)
    dpool = [gcp.DeviceGraph.from_host(gr, dev) for gr in pool]
    out = [torch.empty(gr.n, dtype=torch.int32, device=dev) for gr in pool]
    stream = torch.cuda.current_stream(dev)
    with gcp.Context(dev_index) as ctx:
        for k, e, sd in reqs_in[:4]:
            ctx.gc_color_graph(dpool[k], e[0], e[1], sd, out[k])
        t_single = _timed(stream, lambda: [ctx.gc_color_graph(dpool[k], e[0], e[1], sd, out[k])
                                           for k, e, sd in reqs_in], 1)
        identical = True
        for i in range(16):
            k, e, sd = reqs_in[i]
            ctx.gc_color_graph(dpool[k], e[0], e[1], sd, out[k])
            identical &= bool(np.array_equal(out[k].cpu().numpy(), served[i]))
    return {"requests": len(reqs_in), "pool_graphs": len(pool), "edges": edges, "t_open": t_open,
            "arrival_rate_per_s": rate, "latency": latency_summary(rs), "requests_per_s": len(reqs_in) / t_open,
            "edges_per_s": edges / t_open,
            "capacity": {"requests_per_s": cap, "edges_per_s": edges / t_closed},
            "per_graph": {"requests_per_s": len(reqs_in) / t_single, "edges_per_s": edges / t_single,
                          "unit": "device time of one gc_color_graph call per request, graphs resident"},
            "identical_colourings": identical, "slots": slots, "occupancy": occ,
            "batches": {"count": len(batches), "mean_graphs": float(np.mean([b[1] for b in batches]))}}


def run_serve(args, rank, world):
    import torch
    import torch.distributed as dist
    from paper_2008_11321_gb300 import _build
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    if world > 1:  # replicas: every rank serves its own copy of the request stream
        dist.init_process_group("nccl", device_id=torch.device("cuda", dev))
    if rank == 0:
        _build.build()
    if world > 1:
        dist.barrier()
    w = WORKLOADS[args.workload]
    sampler = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0])
    sampler.start()
    r = measure_serve(w, dev, world, debug=args.debug)
    clocks = sampler.stop()
    # the job's time is the slowest replica's (host clocks: latency is a host-side quantity)
    t_open = max_over_ranks(r["t_open"], world, torch.device("cuda", dev))
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    line = {"metric": METRIC, "value": job_rate(r["edges"], 1, world, t_open), "unit": "edges/s", "n_gpus": world,
            "steps": 1, "warmup": 1, "ms_per_step": t_open * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": w["desc"], "requests": r["requests"], "pool_graphs": r["pool_graphs"],
                       "edges": r["edges"], "arrival_rate_per_s": r["arrival_rate_per_s"],
                       "budget_bytes": w["budget"], "slots": r["slots"]},
            **{k: r[k] for k in ("latency", "requests_per_s", "capacity", "per_graph", "identical_colourings",
                                 "occupancy", "batches")},
            "clocks": clocks}
    if world > 1:
        line["config"]["parallelism"] = "replicas; latency of rank 0"
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="rmat24")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--priority", choices=["adg", "adg-m", "adg-o"] + sorted(PRIORITIES), default="adg",
                    help="JP priority: adg (JP-ADG, the default), adg-m (JP-ADG-M), adg-o (JP-ADG-O) or "
                         "another JP variant")
    ap.add_argument("--debug", action="store_true",
                    help="diagnostics: CUDA_LAUNCH_BLOCKING=1 and a stderr line per serving batch")
    ap.add_argument("--tune-cache", default=None,
                    help="JSON file of autotuned options (default: GC_TUNING_CACHE or ~/.cache/gcolor/tuning.json)")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner: time the given/default options")
    ap.add_argument("--no-extras", action="store_true",
                    help="R-MAT 24 line only: leave out the batch4096 and serve sub-objects")
    ap.add_argument("--options", default=None,
                    help="gc_options fields for the context, as JSON (e.g. '{\"jp_state16\": 0}'); default: "
                         "the library's defaults")
    ap.add_argument("--batch-path", choices=["persistent", "segmented"], default=None,
                    help="batch workload only: time just this path of gc_color_batch (no tuning, no per-graph "
                         "or end-to-end comparison), e.g. to profile it")
    ap.add_argument("--algo", choices=["jp", "dec-itr", "itr"], default="jp",
                    help="colouring: jp (JP with --priority, the default), dec-itr (DEC-ADG-ITR) or itr "
                         "(its SIM-COL on one partition: plain ITR)")
    args = ap.parse_args()
    args.options = json.loads(args.options) if args.options else None
    if args.debug:  # before CUDA is initialised: every launch synchronous, faults reported where they happen
        os.environ["CUDA_LAUNCH_BLOCKING"] = "1"
    if args.warmup < 3:
        print("warning: --warmup below 3 is outside the timing rules", file=sys.stderr)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.algo in ("dec-itr", "itr"):
        if WORKLOADS[args.workload]["kind"] in ("batch", "serve") or args.priority != "adg":
            ap.error("--algo dec-itr applies to the single-graph workloads, without --priority")
        return run_dec(args, rank, world)
    if args.priority != "adg":
        if WORKLOADS[args.workload]["kind"] in ("batch", "serve"):
            ap.error("--priority applies to the single-graph workloads")
        if args.priority not in ("adg-m", "adg-o"):
            return run_variant(args, rank, world)
    if WORKLOADS[args.workload]["kind"] == "batch":
        if args.batch_path:
            if world > 1:
                ap.error("--batch-path times one GPU")
            return run_batch_path(args)
        return run_batch(args, rank, world)
    if WORKLOADS[args.workload]["kind"] == "serve":
        return run_serve(args, rank, world)

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2008_11321_gb300 import _build
    if rank == 0:
        _build.build()
    if world > 1:
        dist.barrier()
    import paper_2008_11321_gb300 as gcp

    w = WORKLOADS[args.workload]
    p, q = w["eps"]
    seed = w["seed"]
    g = make_graph(w, pinned=True)
    n, nnz, m = g.n, g.nnz, g.m
    dg = gcp.DeviceGraph(torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col_idx).to(dev))
    color = torch.empty(n, dtype=torch.int32, device=dev)
    batch = torch.empty(n, dtype=torch.int32, device=dev)
    ctx = gcp.Context(local, args.options)
    stream = torch.cuda.current_stream(dev)

    median = args.priority == "adg-m"
    ordered = args.priority == "adg-o"

    def colour_step():
        if median:  # JP-ADG-M: ADG-M has no eps
            return ctx.gc_color_graph_m(dg, seed, color, batch)
        if ordered:  # JP-ADG-O: a total order, no tie-break seed
            return ctx.gc_color_graph_o(dg, p, q, color, batch)
        return ctx.gc_color_graph(dg, p, q, seed, color, batch)

    for _ in range(args.warmup):
        nc, nr = colour_step()
    tuned = None
    if not args.no_tune and not median and not ordered:
        # the autotuner's options for this graph class (searched unless
        # cached), applied to the context; then warm up again
        from paper_2008_11321_gb300 import tuning
        tuned = tuning.tune_graph(ctx, dg, p, q, seed, cache=tuning.TuningCache(args.tune_cache), reps=3)
        for _ in range(args.warmup):
            nc, nr = colour_step()
    ctx.gc_set_timing(True)

    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        dev_id = uuid if uuid.startswith("GPU-") else f"GPU-{uuid}"
    except Exception:
        dev_id = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local]
    sampler = ClockSampler(dev_id)
    sampler.start()
    time.sleep(0.3)

    steps = []
    n_nonisolated = int((g.degrees() > 0).sum())
    sync_ranks(world, dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        nc, nr = colour_step()
        st = ctx.gc_get_stats()
        steps.append({k: getattr(st, k) for k, _ in st._fields_})
    ev1.record(stream)
    sync_ranks(world, dev)
    clocks = sampler.stop()
    t_max = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, world, dev)
    value = job_rate(m, args.steps, world, t_max)

    # end to end through the public host-buffer entry point
    e2e = None
    if not args.no_e2e and not median and not ordered:
        hcolor = torch.empty(n, dtype=torch.int32, pin_memory=True).numpy()
        ctx.gc_set_timing(False)
        ctx.gc_color_graph_host(g.row_ptr, g.col_idx, p, q, seed, hcolor)  # grows buffers once
        sync_ranks(world, dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            ctx.gc_color_graph_host(g.row_ptr, g.col_idx, p, q, seed, hcolor)
        e1.record(stream)
        sync_ranks(world, dev)
        te = max_over_ranks(e0.elapsed_time(e1) / 1e3, world, dev)
        assert (hcolor == color.cpu().numpy()).all(), "host entry point disagrees with device path"
        e2e = {"value": job_rate(m, args.steps, world, te), "unit": "edges/s",
               "h2d_bytes_per_step": 8 * (n + 1) + 4 * nnz, "d2h_bytes_per_step": 4 * n}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    mean = lambda k: statistics.mean(x[k] for x in steps)  # noqa: E731
    launches = sum(x["launches"] for x in steps)
    last = steps[-1]
    sum_u, dec = last["sum_U"], last["sum_decrements"]
    peak, peak_kind = load_peak()
    gb = group_bytes(n_nonisolated, nnz, last)
    groups = {"adg_update_kernel": (mean("ms_adg_update"), last["adg_rounds"]),
              "jp_color_kernel": (mean("ms_jp_color"), max(1, last["bulk_launches"])),
              "jpf_core_solve_kernel": (mean("ms_core_solve"), 1)}
    kname = max(groups, key=lambda k: groups[k][0])
    kms, kl = groups[kname]
    achieved = gb[kname] / (kms / 1e3) / 1e9 if kms > 0 else 0.0
    pbytes = path_bytes(n, nnz, sum_u, dec)
    path_gbs = pbytes / (t_max / args.steps) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": (w["desc"].replace("eps=1/100", "JP-ADG-M (median)") if median else
                                (w["desc"] + ", JP-ADG-O (R sorted by degree)" if ordered else w["desc"])),
                   "n": n, "m": m, "eps": f"{p}/{q}" if not median else None, "seed": seed,
                   "adg_rounds": nr, "num_colors": nc, "sum_U": sum_u, "decrements": dec,
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "options": ctx.gc_get_options().as_dict(), "jp_state_bits": last["jp_state_bits"],
                   "adg_pull_rounds": last["adg_pull_rounds"],
                   "l2": f"inputs larger than L2 (col_idx {4 * nnz / 1e9:.2f} GB), no flush"},
        "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": kernel_traffic(args.workload, kname),
                     "algorithmic_bytes_per_launch": gb[kname] / kl, "ms_per_launch": kms / kl,
                     "launches_per_step": kl,
                     "groups_ms": {k: v[0] for k, v in groups.items()}},
        "path": {"algorithmic_bytes_per_step": pbytes, "gbs": path_gbs, "frac": path_gbs / peak,
                 "ms_adg": mean("ms_adg"), "ms_jp": mean("ms_jp"), "ms_core_preds": mean("ms_core_preds"),
                 "core_vertices": last["core_vertices"], "core_preds": last["core_preds"]},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if tuned:
        line["tuned"] = {"searched": tuned["searched"], "best_ms": tuned["best_ms"], "start_ms": tuned["start_ms"]}
    if e2e:
        line["e2e"] = e2e
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, median=median, ordered=ordered, graph=g)
    if world == 1 and not args.no_extras and args.workload == "rmat24" and not median and not ordered:
        # the batched and served forms, measured in the same run (compact)
        from paper_2008_11321_gb300 import tuning
        ctx.close()
        b = measure_batch(WORKLOADS["batch4096"], dev, 3, 3, args.options, 1, tuning.TuningCache(args.tune_cache))
        line["batch4096"] = {"workload": WORKLOADS["batch4096"]["desc"], "graphs_per_s": b["graphs_per_s"],
                             "edges_per_s": b["edges_per_s"], "per_graph_graphs_per_s": b["per_graph"]["value"],
                             "speedup_vs_per_graph": b["speedup_vs_per_graph"],
                             "identical_colourings": b["identical_colourings"],
                             "paths_graphs_per_s": {k: v["graphs_per_s"] for k, v in b["paths"].items()},
                             "tuned_batch_mode": b["tuned"]["options"]["batch_mode"], "e2e_graphs_per_s":
                             b["e2e"]["value"], "roofline_frac": b["roofline"]["frac"]}
        r = measure_serve(WORKLOADS["serve"], local)
        line["serve"] = {"workload": WORKLOADS["serve"]["desc"], "requests": r["requests"],
                         "p50_ms": r["latency"].get("p50_ms"), "p99_ms": r["latency"].get("p99_ms"),
                         "requests_per_s": r["requests_per_s"], "edges_per_s": r["edges_per_s"],
                         "capacity_requests_per_s": r["capacity"]["requests_per_s"],
                         "per_graph_requests_per_s": r["per_graph"]["requests_per_s"],
                         "identical_colourings": r["identical_colourings"],
                         "requests_in_flight_mean": r["occupancy"]["requests_in_flight_mean"],
                         "busy_slots_mean": r["occupancy"]["busy_slots_mean"], "slots": r["slots"]}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
