"""Host logic of the colouring service, without a GPU: admission by the
memory budget, compute slots whose work overlaps, failures that stay with
their request, cancellation.  The engine is a stand-in that colours with the
CPU oracle and sleeps for the device time; the GPU engine is exercised by
tests/test_serve_gpu.py."""
from __future__ import annotations

import threading
import time

import numpy as np
import pytest

import graphgen as gg
import oracle
from paper_2008_11321_gb300.serve import ColoringServer, device_bytes, latency_summary


class FakeEngine:
    def __init__(self, device_s=0.05, fail_upload=(), fail_colour=()):
        self.device_s = device_s
        self.fail_upload, self.fail_colour = set(fail_upload), set(fail_colour)
        self.lock = threading.Lock()
        self.active = 0
        self.max_active = 0
        self.calls = []
        self.released = 0

    def upload(self, req):
        if req.seed in self.fail_upload:
            raise MemoryError("out of device memory")
        return ("dev", req.id)

    def colour(self, slot, reqs):
        with self.lock:
            self.active += 1
            self.max_active = max(self.max_active, self.active)
            self.calls.append((slot, [r.id for r in reqs]))
        try:
            time.sleep(self.device_s)
            if any(r.seed in self.fail_colour for r in reqs):
                raise RuntimeError("gc_color_batch_list: GC_ERR_INVALID_GRAPH")
            out = []
            for r in reqs:
                g = gg.Graph(r.row_ptr, r.col_idx, "req")
                out.append(oracle.jp_adg(g, r.eps_p, r.eps_q, r.seed)[1])
            return out
        finally:
            with self.lock:
                self.active -= 1

    def release(self, req):
        self.released += 1

    def close(self):
        pass


GRAPHS = [gg.erdos_renyi(400 + 50 * i, 1500 + 100 * i, i + 1) for i in range(8)]


def expected(g, p, q, seed):
    return oracle.jp_adg(g, p, q, seed)[1]


def test_results_equal_oracle_and_slots_overlap():
    eng = FakeEngine(device_s=0.08)
    with ColoringServer(slots=2, engine=eng) as srv:
        first = srv.submit(GRAPHS[0].row_ptr, GRAPHS[0].col_idx, 1, 100, 7)
        time.sleep(0.02)  # the first batch is running: later arrivals go to the other slot
        rest = [srv.submit(g.row_ptr, g.col_idx, 1, 10, 40 + i) for i, g in enumerate(GRAPHS[1:])]
        assert np.array_equal(first.result(10), expected(GRAPHS[0], 1, 100, 7))
        for i, (r, g) in enumerate(zip(rest, GRAPHS[1:])):
            assert np.array_equal(r.result(10), expected(g, 1, 10, 40 + i))
        occ = srv.occupancy()
    assert eng.max_active == 2                       # two batches on the device at once
    assert {s for s, _ in eng.calls} == {0, 1}
    assert occ["requests_in_flight_mean"] > 0
    assert srv.used == 0 and eng.released == len(GRAPHS)
    assert set(latency_summary([first] + rest)) == {"p50_ms", "p99_ms", "mean_ms", "max_ms"}


def test_upload_failure_fails_only_that_request():
    eng = FakeEngine(device_s=0.01, fail_upload={13})
    with ColoringServer(slots=2, engine=eng) as srv:
        rs = [srv.submit(g.row_ptr, g.col_idx, 1, 100, 10 + i) for i, g in enumerate(GRAPHS[:5])]
        for i, r in enumerate(rs):
            if r.seed == 13:
                with pytest.raises(RuntimeError, match="upload failed"):
                    r.result(10)
            else:
                assert np.array_equal(r.result(10), expected(GRAPHS[i], 1, 100, 10 + i))
    assert srv.used == 0


def test_failing_request_does_not_poison_its_batch():
    # one slot and a slow first batch: the next four requests are batched
    # together; the batch call fails because of one of them, the others are
    # coloured again alone and succeed
    eng = FakeEngine(device_s=0.05, fail_colour={22})
    with ColoringServer(slots=1, engine=eng) as srv:
        srv.submit(GRAPHS[0].row_ptr, GRAPHS[0].col_idx, 1, 100, 1)
        time.sleep(0.01)
        rs = [srv.submit(g.row_ptr, g.col_idx, 1, 100, 20 + i) for i, g in enumerate(GRAPHS[1:5])]
        for i, r in enumerate(rs):
            if r.seed == 22:
                with pytest.raises(RuntimeError, match="INVALID_GRAPH"):
                    r.result(10)
            else:
                assert np.array_equal(r.result(10), expected(GRAPHS[1 + i], 1, 100, 20 + i))
    assert any(len(ids) == 4 for _, ids in eng.calls)   # they were batched together first
    assert srv.used == 0


def test_budget_admission_and_cancel():
    g = GRAPHS[0]
    one = device_bytes(g.n, g.nnz)
    eng = FakeEngine(device_s=0.2)
    with ColoringServer(slots=2, memory_budget=one, engine=eng) as srv:
        a = srv.submit(g.row_ptr, g.col_idx, 1, 100, 1)
        b = srv.submit(g.row_ptr, g.col_idx, 1, 100, 2)   # waits: the budget holds one request
        c = srv.submit(g.row_ptr, g.col_idx, 1, 100, 3)
        time.sleep(0.05)
        assert srv.used == one
        assert srv.cancel(c) is True
        with pytest.raises(RuntimeError, match="cancelled"):
            c.result(1)
        assert np.array_equal(a.result(10), expected(g, 1, 100, 1))
        assert np.array_equal(b.result(10), expected(g, 1, 100, 2))
        assert srv.cancel(a) is False                      # already finished
    assert eng.max_active == 1                             # the budget kept them apart
    assert srv.used == 0


def test_invalid_requests_rejected_at_submit():
    g = GRAPHS[0]
    eng = FakeEngine(device_s=0.0)
    with ColoringServer(slots=1, memory_budget=1 << 30, engine=eng) as srv:
        for r in (srv.submit(g.row_ptr, g.col_idx, 1, 0, 1), srv.submit(g.row_ptr, g.col_idx, 1 << 21, 1, 1),
                  srv.submit(g.row_ptr[:-1], g.col_idx, 1, 100, 1)):
            with pytest.raises(RuntimeError):
                r.result(1)
        r = srv.submit(np.zeros(12 << 20, dtype=np.int64), np.zeros(0, dtype=np.int32), 1, 100, 1)
        with pytest.raises(RuntimeError, match="budget"):
            r.result(1)
    assert eng.calls == []


def test_device_error_fails_the_batch_without_retries():
    # a CUDA error of the device (not of one request) is not retried request
    # by request: every request of the batch reports that first error
    class BrokenDevice(FakeEngine):
        def colour(self, slot, reqs):
            self.calls.append((slot, [r.id for r in reqs]))
            time.sleep(0.03)
            raise RuntimeError("CUDA error: an illegal memory access was encountered")
    eng = BrokenDevice()
    with ColoringServer(slots=1, engine=eng) as srv:
        srv.submit(GRAPHS[0].row_ptr, GRAPHS[0].col_idx, 1, 100, 1)
        time.sleep(0.01)
        rs = [srv.submit(g.row_ptr, g.col_idx, 1, 100, 2 + i) for i, g in enumerate(GRAPHS[1:4])]
        for r in rs:
            with pytest.raises(RuntimeError, match="illegal memory access"):
                r.result(10)
    assert len(eng.calls) == 2  # one call per batch, no per-request retries
    assert srv.used == 0
