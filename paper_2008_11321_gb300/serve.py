"""Continuous-batching colouring service on one GPU.

Requests (a graph in host CSR arrays, eps, seed) arrive at any time.  Two
threads share the GPU:

* the admission thread takes waiting requests in arrival order while their
  device-memory estimate fits the budget, and uploads each graph on a copy
  stream; the graph's CSR then stays resident on the device until its result
  is delivered;
* the compute thread repeatedly takes every graph uploaded so far and colours
  them together with one gc_color_batch_list call on a compute stream, then
  copies each result back and releases the request's memory.

So requests that arrive while a batch is running are admitted and uploaded
while it runs (their copies overlap its kernels) and join the next batch as
soon as it starts; memory freed by finished requests admits waiting ones.
Every result equals gc_color_graph on the same graph alone (the batch entry
point guarantees it; the serving tests check it).  Latency is measured from
submission to the colours being in host memory.
"""
from __future__ import annotations

import collections
import itertools
import threading
import time

import numpy as np

from . import gcolor


def device_bytes(n: int, nnz: int) -> int:
    """Device memory a request may need while admitted: its resident CSR and
    colours plus its share of a batch's packed copy and scratch (about 100
    bytes per vertex and 24 per CSR entry, an upper estimate)."""
    return 8 * (n + 1) + 4 * nnz + 4 * n + 100 * n + 24 * nnz


class Request:
    __slots__ = ("id", "row_ptr", "col_idx", "eps_p", "eps_q", "seed", "n", "nnz", "bytes",
                 "t_submit", "t_admit", "t_done", "colors", "error", "done", "_dev")

    def __init__(self, rid, row_ptr, col_idx, eps_p, eps_q, seed):
        self.id = rid
        self.row_ptr = row_ptr
        self.col_idx = col_idx
        self.eps_p, self.eps_q, self.seed = eps_p, eps_q, seed
        self.n = int(row_ptr.shape[0]) - 1
        self.nnz = int(col_idx.shape[0])
        self.bytes = device_bytes(self.n, self.nnz)
        self.t_submit = time.perf_counter()
        self.t_admit = self.t_done = None
        self.colors = None
        self.error = None
        self.done = threading.Event()
        self._dev = None

    @property
    def latency(self) -> float:
        return self.t_done - self.t_submit

    def result(self, timeout: float | None = None) -> np.ndarray:
        if not self.done.wait(timeout):
            raise TimeoutError(f"request {self.id} not finished")
        if self.error:
            raise RuntimeError(self.error)
        return self.colors


class ColoringServer:
    def __init__(self, device: int = 0, memory_budget: int = 40 << 30, max_batch_graphs: int = 4096):
        import torch
        self._torch = torch
        self.dev = torch.device("cuda", device)
        self.ctx = gcolor.Context(device)
        self.copy_stream = torch.cuda.Stream(self.dev)
        self.compute_stream = torch.cuda.Stream(self.dev)
        self.budget = memory_budget
        self.max_batch = max_batch_graphs
        self.used = 0
        self._ids = itertools.count()
        self._cv = threading.Condition()
        self._waiting: collections.deque = collections.deque()
        self._ready: collections.deque = collections.deque()
        self._running = True
        self._uploading = 0
        self.batches = []  # (number of graphs, seconds) per batch
        self._threads = [threading.Thread(target=self._admit_loop, daemon=True),
                         threading.Thread(target=self._compute_loop, daemon=True)]
        for t in self._threads:
            t.start()

    # -- client side -----------------------------------------------------------
    def submit(self, row_ptr: np.ndarray, col_idx: np.ndarray, eps_p: int = 1, eps_q: int = 100,
               seed: int = 42) -> Request:
        req = Request(next(self._ids), np.ascontiguousarray(row_ptr, dtype=np.int64),
                      np.ascontiguousarray(col_idx, dtype=np.int32), eps_p, eps_q, seed)
        with self._cv:
            if req.bytes > self.budget:
                req.error = f"request needs ~{req.bytes} device bytes, budget is {self.budget}"
                req.t_done = time.perf_counter()
                req.done.set()
                return req
            self._waiting.append(req)
            self._cv.notify_all()
        return req

    def close(self):
        with self._cv:
            self._running = False
            self._cv.notify_all()
        for t in self._threads:
            t.join()
        self.ctx.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- admission: memory budget, uploads on the copy stream ------------------
    def _admit_loop(self):
        torch = self._torch
        while True:
            with self._cv:
                # after close() the queue is still drained: memory freed by
                # finishing batches admits the rest
                while not (self._waiting and self.used + self._waiting[0].bytes <= self.budget) and \
                        (self._running or self._waiting):
                    self._cv.wait()
                if not self._waiting:
                    return
                req = self._waiting.popleft()
                self.used += req.bytes
                self._uploading += 1
            with torch.cuda.stream(self.copy_stream):
                rp = torch.from_numpy(req.row_ptr).to(self.dev)
                ci = torch.from_numpy(req.col_idx).to(self.dev)
                col = torch.empty(req.n, dtype=torch.int32, device=self.dev)
                ev = torch.cuda.Event()
                ev.record(self.copy_stream)
            req._dev = (gcolor.DeviceGraph(rp, ci), col, ev)
            req.t_admit = time.perf_counter()
            with self._cv:
                self._uploading -= 1
                self._ready.append(req)
                self._cv.notify_all()

    # -- compute: everything uploaded so far, one batch call ---------------------
    def _compute_loop(self):
        torch = self._torch
        while True:
            with self._cv:
                while not self._ready and (self._running or self._waiting or self._uploading):
                    self._cv.wait()
                if not self._ready:
                    return
                batch = []
                while self._ready and len(batch) < self.max_batch:
                    batch.append(self._ready.popleft())
            t0 = time.perf_counter()
            for r in batch:
                self.compute_stream.wait_event(r._dev[2])
            err = None
            try:
                self.ctx.gc_color_batch_list([r._dev[0] for r in batch],
                                             [(r.eps_p, r.eps_q, r.seed) for r in batch],
                                             [r._dev[1] for r in batch], stream=self.compute_stream)
                with torch.cuda.stream(self.compute_stream):
                    host = [r._dev[1].to("cpu", non_blocking=True) for r in batch]
                self.compute_stream.synchronize()
            except Exception as e:  # reported per request, the service keeps running
                err = str(e)
            t1 = time.perf_counter()
            self.batches.append((len(batch), t1 - t0))
            with self._cv:
                for i, r in enumerate(batch):
                    if err:
                        r.error = err
                    else:
                        r.colors = host[i].numpy()
                    r.t_done = t1
                    r._dev = None
                    self.used -= r.bytes
                    r.done.set()
                self._cv.notify_all()


def latency_summary(reqs):
    lat = np.array([r.latency for r in reqs if r.t_done is not None and not r.error])
    if lat.size == 0:
        return {}
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "max_ms": float(lat.max() * 1e3)}
