"""Cache of autotuned context options, per device and workload class.

The search itself is the library's (gc_autotune / gc_autotune_batch: timed
trials on the GPU, every candidate checked to reproduce the colouring).  This
module only remembers its answers in a JSON file, so that a process that
meets a workload class again applies the tuned options without searching.

A workload class is what the options depend on: the size of the graph
(log2 of its vertices), its density (log2 of the average degree) and eps for
a single graph; the number of graphs and their mean size for a batch.  The
file is keyed by device name, then class.  Its location is the argument, or
the GC_TUNING_CACHE environment variable, or ~/.cache/gcolor/tuning.json.
"""
from __future__ import annotations

import json
import math
import os
import threading

from . import gcolor

_LOCK = threading.Lock()


def default_path() -> str:
    return os.environ.get("GC_TUNING_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "gcolor",
                                                              "tuning.json")


def _lg(x: float) -> int:
    return int(round(math.log2(x))) if x > 0 else 0


def graph_class(n: int, nnz: int, eps_p: int, eps_q: int) -> str:
    return f"graph/n2^{_lg(n)}/deg2^{_lg(nnz / n if n else 0)}/eps{eps_p}:{eps_q}"


def batch_class(num_graphs: int, n: int, nnz: int) -> str:
    return f"batch/g2^{_lg(num_graphs)}/n2^{_lg(n / num_graphs if num_graphs else 0)}/deg2^{_lg(nnz / n if n else 0)}"


class TuningCache:
    def __init__(self, path: str | None = None):
        self.path = path or default_path()

    def _load(self) -> dict:
        try:
            with open(self.path) as f:
                return json.load(f)
        except (OSError, ValueError):
            return {}

    def get(self, device: str, cls: str) -> dict | None:
        with _LOCK:
            return self._load().get(device, {}).get(cls)

    def put(self, device: str, cls: str, record: dict) -> None:
        with _LOCK:
            data = self._load()
            data.setdefault(device, {})[cls] = record
            os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
            tmp = f"{self.path}.tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(data, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)


def device_name(device: int) -> str:
    import torch
    return torch.cuda.get_device_name(device)


def tune_graph(ctx: gcolor.Context, g: gcolor.DeviceGraph, eps_p: int, eps_q: int, seed: int,
               cache: TuningCache | None = None, reps: int = 3, budget_ms: float = 0.0, retune: bool = False):
    """Applies tuned options for this graph's class to ctx (searching with
    gc_autotune unless the cache has them) and returns the cache record:
    {"options": {...}, "best_ms": ..., "start_ms": ..., "searched": bool}."""
    cache = cache or TuningCache()
    dev, cls = device_name(ctx.device), graph_class(g.n, g.nnz, eps_p, eps_q)
    rec = None if retune else cache.get(dev, cls)
    if rec is not None:
        ctx.gc_set_options(rec["options"])
        return dict(rec, searched=False)
    best, best_ms, start_ms = ctx.gc_autotune(g, eps_p, eps_q, seed, reps, budget_ms)
    rec = {"options": best.as_dict(), "best_ms": best_ms, "start_ms": start_ms, "n": g.n, "nnz": g.nnz}
    cache.put(dev, cls, rec)
    return dict(rec, searched=True)


def tune_batch(ctx: gcolor.Context, b: gcolor.DeviceBatch, jobs, cache: TuningCache | None = None, reps: int = 3,
               budget_ms: float = 0.0, retune: bool = False):
    """tune_graph for gc_color_batch."""
    cache = cache or TuningCache()
    dev, cls = device_name(ctx.device), batch_class(b.num_graphs, b.n, b.nnz)
    rec = None if retune else cache.get(dev, cls)
    if rec is not None:
        ctx.gc_set_options(rec["options"])
        return dict(rec, searched=False)
    best, best_ms, start_ms = ctx.gc_autotune_batch(b, jobs, reps, budget_ms)
    rec = {"options": best.as_dict(), "best_ms": best_ms, "start_ms": start_ms, "graphs": b.num_graphs, "n": b.n,
           "nnz": b.nnz}
    cache.put(dev, cls, rec)
    return dict(rec, searched=True)
