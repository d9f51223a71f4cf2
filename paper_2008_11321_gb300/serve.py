"""Continuous-batching colouring service on one GPU.

Requests (a graph in host CSR arrays, eps, seed) arrive at any time and are
coloured with JP-ADG; each result equals gc_color_graph on the same graph
alone.  The service runs

* one admission thread: it takes waiting requests in arrival order while
  their device-memory estimate fits the budget and uploads each graph on a
  copy stream; the graph then stays resident on the device until its colours
  are delivered;
* `slots` compute threads, each with its own library context and CUDA
  stream: a free slot takes every uploaded request not yet taken (up to
  max_batch_graphs) and colours them together with one gc_color_batch_list
  call, copies the colours back and frees the requests' memory.

With two or more slots, requests that arrive while a large batch runs start
on the GPU in another slot at once: their kernels overlap the running batch
on the device instead of waiting for it, and memory freed by finished
requests admits waiting ones.  Latency is measured from submission to the
colours being in host memory.

Failures stay with their request: an upload that fails (for example out of
device memory) fails that request only; if a batch call fails, its requests
are coloured again one by one so that only the failing ones report the
error.  A request still waiting for admission can be cancelled.

The GPU work sits behind an engine object (upload / colour / release), so the
host logic above can be exercised without a GPU.
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
                 "t_submit", "t_admit", "t_start", "t_done", "colors", "error", "done", "cancelled", "_dev")

    def __init__(self, rid, row_ptr, col_idx, eps_p, eps_q, seed):
        self.id = rid
        self.row_ptr = row_ptr
        self.col_idx = col_idx
        self.eps_p, self.eps_q, self.seed = eps_p, eps_q, seed
        self.n = int(row_ptr.shape[0]) - 1
        self.nnz = int(col_idx.shape[0])
        self.bytes = device_bytes(self.n, self.nnz)
        self.t_submit = time.perf_counter()
        self.t_admit = self.t_start = self.t_done = None
        self.colors = None
        self.error = None
        self.cancelled = False
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


class CudaEngine:
    """The GPU side of the service: uploads on a copy stream, one library
    context and stream per compute slot."""

    def __init__(self, device: int, slots: int, options=None):
        import torch
        self.torch = torch
        self.dev = torch.device("cuda", device)
        self.copy_stream = torch.cuda.Stream(self.dev)
        self.ctxs = [gcolor.Context(device, options) for _ in range(slots)]
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(slots)]

    def upload(self, req):
        torch = self.torch
        with torch.cuda.stream(self.copy_stream):
            rp = torch.from_numpy(req.row_ptr).to(self.dev, non_blocking=False)
            ci = torch.from_numpy(req.col_idx).to(self.dev, non_blocking=False)
            col = torch.empty(req.n, dtype=torch.int32, device=self.dev)
            ev = torch.cuda.Event()
            ev.record(self.copy_stream)
        return gcolor.DeviceGraph(rp, ci), col, ev

    def colour(self, slot: int, reqs):
        """Colours the requests together in `slot`; returns their colours as
        host arrays, in order."""
        torch = self.torch
        stream = self.streams[slot]
        for r in reqs:
            stream.wait_event(r._dev[2])
        self.ctxs[slot].gc_color_batch_list([r._dev[0] for r in reqs], [(r.eps_p, r.eps_q, r.seed) for r in reqs],
                                            [r._dev[1] for r in reqs], stream=stream)
        with torch.cuda.stream(stream):
            host = [r._dev[1].to("cpu", non_blocking=True) for r in reqs]
        stream.synchronize()
        return [h.numpy() for h in host]

    def release(self, req):
        req._dev = None

    def close(self):
        for c in self.ctxs:
            c.close()


class ColoringServer:
    def __init__(self, device: int = 0, memory_budget: int = 40 << 30, max_batch_graphs: int = 4096,
                 slots: int = 2, options=None, engine=None, on_batch=None):
        """on_batch(slot, requests, seconds, errors): called after every
        batch (for logging), errors being one string or None per request."""
        self.engine = engine if engine is not None else CudaEngine(device, slots, options)
        self.on_batch = on_batch
        self.slots = slots
        self.budget = memory_budget
        self.max_batch = max_batch_graphs
        self.used = 0
        self._ids = itertools.count()
        self._cv = threading.Condition()
        self._waiting: collections.deque = collections.deque()
        self._ready: collections.deque = collections.deque()
        self._running = True
        self._uploading = 0
        self._busy = 0                    # slots colouring right now
        self._inflight = 0                # requests on the device right now
        self._t0 = self._t_last = time.perf_counter()
        self._inflight_area = 0.0         # integral of requests in flight over time
        self._busy_area = 0.0             # integral of busy slots over time
        self.batches = []                 # (slot, number of graphs, seconds) per batch
        self._threads = [threading.Thread(target=self._admit_loop, daemon=True)]
        self._threads += [threading.Thread(target=self._compute_loop, args=(k,), daemon=True) for k in range(slots)]
        for t in self._threads:
            t.start()

    # -- client side -----------------------------------------------------------
    def submit(self, row_ptr: np.ndarray, col_idx: np.ndarray, eps_p: int = 1, eps_q: int = 100,
               seed: int = 42) -> Request:
        req = Request(next(self._ids), np.ascontiguousarray(row_ptr, dtype=np.int64),
                      np.ascontiguousarray(col_idx, dtype=np.int32), eps_p, eps_q, seed)
        bad = None
        if req.bytes > self.budget:
            bad = f"request needs ~{req.bytes} device bytes, budget is {self.budget}"
        elif not (1 <= eps_q <= 1 << 20 and 0 <= eps_p <= 1 << 20):
            bad = f"eps = {eps_p}/{eps_q} out of range"
        elif req.n < 0 or req.row_ptr[0] != 0 or req.row_ptr[-1] != req.nnz:
            bad = "row_ptr does not describe col_idx"
        if bad:  # rejected at once, never batched with others
            req.error = bad
            req.t_done = time.perf_counter()
            req.done.set()
            return req
        with self._cv:
            self._waiting.append(req)
            self._cv.notify_all()
        return req

    def cancel(self, req: Request) -> bool:
        """Cancels a request still waiting for admission (True), or reports
        that it is already uploaded or running (False)."""
        with self._cv:
            try:
                self._waiting.remove(req)
            except ValueError:
                return False
            req.cancelled = True
            req.error = "cancelled"
            req.t_done = time.perf_counter()
            req.done.set()
            self._cv.notify_all()
            return True

    def close(self):
        with self._cv:
            self._running = False
            self._cv.notify_all()
        for t in self._threads:
            t.join()
        self.engine.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def occupancy(self) -> dict:
        """Time-averaged requests on the device and busy slots so far."""
        with self._cv:
            self._account()
            span = max(time.perf_counter() - self._t0, 1e-9)
            return {"requests_in_flight_mean": self._inflight_area / span, "busy_slots_mean": self._busy_area / span}

    def reset_occupancy(self):
        with self._cv:
            self._account()
            self._t0 = time.perf_counter()
            self._inflight_area = self._busy_area = 0.0

    def _account(self):  # under the lock
        now = time.perf_counter()
        dt = now - self._t_last
        self._inflight_area += self._inflight * dt
        self._busy_area += self._busy * dt
        self._t_last = now

    def _finish(self, req, colors, error, t):  # under the lock
        if error:
            req.error = error
        else:
            req.colors = colors
        req.t_done = t
        self.engine.release(req)
        self.used -= req.bytes
        req.done.set()

    # -- admission: memory budget, uploads on the copy stream ------------------
    def _admit_loop(self):
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
            try:
                dev = self.engine.upload(req)
                err = None
            except Exception as e:  # this request fails alone; the service keeps running
                dev, err = None, f"upload failed: {e}"
            with self._cv:
                self._uploading -= 1
                if err:
                    self._finish(req, None, err, time.perf_counter())
                else:
                    req._dev = dev
                    req.t_admit = time.perf_counter()
                    self._ready.append(req)
                self._cv.notify_all()

    # -- compute: a free slot takes everything uploaded and not yet taken -------
    def _compute_loop(self, slot: int):
        while True:
            with self._cv:
                while not self._ready and (self._running or self._waiting or self._uploading):
                    self._cv.wait()
                if not self._ready:
                    self._cv.notify_all()
                    return
                batch = []
                while self._ready and len(batch) < self.max_batch:
                    batch.append(self._ready.popleft())
                self._account()
                self._busy += 1
                self._inflight += len(batch)
            t0 = time.perf_counter()
            for r in batch:
                r.t_start = t0
            results = self._colour(slot, batch)
            t1 = time.perf_counter()
            if self.on_batch is not None:
                self.on_batch(slot, batch, t1 - t0, [e for _, e in results])
            with self._cv:
                self._account()
                self._busy -= 1
                self._inflight -= len(batch)
                self.batches.append((slot, len(batch), t1 - t0))
                for r, (colors, err) in zip(batch, results):
                    self._finish(r, colors, err, t1)
                self._cv.notify_all()

    def _colour(self, slot, batch):
        """[(colours, error)] per request: the batch in one call, or, if that
        call fails with an error a request can cause (bad input, no memory),
        each request alone so that the error stays with the requests that
        cause it.  A CUDA error of the device itself fails the whole batch
        with that first error: retrying on a broken device cannot help."""
        try:
            return [(c, None) for c in self.engine.colour(slot, batch)]
        except Exception as e:
            first = str(e)
            status = getattr(e, "status", None)
            device_error = status == gcolor.GC_ERR_CUDA or (status is None and "CUDA error" in first)
            if len(batch) == 1 or device_error:
                return [(None, first)] * len(batch)
        out = []
        for r in batch:
            try:
                out.append((self.engine.colour(slot, [r])[0], None))
            except Exception as e:
                out.append((None, str(e)))
        return out


def latency_summary(reqs):
    lat = np.array([r.latency for r in reqs if r.t_done is not None and not r.error])
    if lat.size == 0:
        return {}
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "max_ms": float(lat.max() * 1e3)}
