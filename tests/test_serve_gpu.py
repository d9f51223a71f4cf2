"""The continuous-batching service: requests arriving at random times while
others are on the GPU are coloured in shared batches, in compute slots whose
work overlaps on the device, and every result is the same as colouring that
graph alone (gc_color_graph) and as the oracle."""
from __future__ import annotations

import threading
import time

import numpy as np
import pytest

import graphgen as gg
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2008_11321_gb300 as gcp  # noqa: E402
from paper_2008_11321_gb300.serve import ColoringServer, device_bytes, latency_summary  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_11321_gb300 import _build
    _build.build()


def _requests(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        kind = rng.integers(3)
        if kind == 0:
            g = gg.rmat(int(rng.integers(8, 15)), int(rng.integers(8, 33)), seed=seed + i)
        elif kind == 1:
            g = gg.barabasi_albert(int(rng.integers(1000, 30000)), int(rng.integers(2, 17)), seed + i)
        else:
            g = gg.erdos_renyi(int(rng.integers(500, 20000)), int(rng.integers(1000, 80000)), seed + i)
        eps = (1, 100) if rng.integers(2) else (1, 10)
        out.append((g, eps, 42 + i))
    return out


def _alone(g, eps, seed):
    with gcp.Context(0) as ctx:
        dg = gcp.DeviceGraph.from_host(g, "cuda:0")
        c = torch.empty(g.n, dtype=torch.int32, device="cuda:0")
        ctx.gc_color_graph(dg, eps[0], eps[1], seed, c)
        return c.cpu().numpy()


def test_results_same_alone_and_in_the_mix():
    reqs_in = _requests(30, 11)
    rng = np.random.default_rng(3)
    with ColoringServer(0, memory_budget=8 << 30) as srv:
        reqs = []
        # arrivals in bursts of 6 (Poisson gaps between bursts) while earlier
        # requests run: a burst arrives faster than one request is coloured,
        # so requests share batches however fast the device is
        for i, (g, eps, seed) in enumerate(reqs_in):
            reqs.append(srv.submit(g.row_ptr, g.col_idx, eps[0], eps[1], seed))
            if i % 6 == 5:
                time.sleep(rng.exponential(0.002))
        results = [r.result(timeout=120) for r in reqs]
        batches = list(srv.batches)
    assert sum(b[1] for b in batches) == len(reqs_in)
    assert len(batches) < len(reqs_in)  # requests really shared batches
    for (g, eps, seed), col in zip(reqs_in, results):
        assert np.array_equal(col, _alone(g, eps, seed))
        _, oc, _, _ = oracle.jp_adg(g, eps[0], eps[1], seed)
        assert np.array_equal(col, oc)
    assert latency_summary(reqs)["p99_ms"] > 0


def test_memory_budget_admits_in_turn():
    reqs_in = _requests(12, 5)
    biggest = max(device_bytes(g.n, g.nnz) for g, _, _ in reqs_in)
    with ColoringServer(0, memory_budget=biggest + 1) as srv:  # about one graph at a time
        reqs = [srv.submit(g.row_ptr, g.col_idx, e[0], e[1], s) for g, e, s in reqs_in]
        results = [r.result(timeout=120) for r in reqs]
    for (g, eps, seed), col in zip(reqs_in, results):
        assert np.array_equal(col, oracle.jp_adg(g, eps[0], eps[1], seed)[1])


def test_request_over_budget_is_refused():
    g = gg.rmat(12, 16, seed=1)
    with ColoringServer(0, memory_budget=1000) as srv:
        r = srv.submit(g.row_ptr, g.col_idx)
        with pytest.raises(RuntimeError):
            r.result(timeout=10)


def test_concurrent_clients():
    reqs_in = _requests(16, 23)
    out = [None] * len(reqs_in)
    with ColoringServer(0) as srv:
        def client(k):
            for i in range(k, len(reqs_in), 4):
                g, e, s = reqs_in[i]
                out[i] = srv.submit(g.row_ptr, g.col_idx, e[0], e[1], s).result(timeout=120)
        ts = [threading.Thread(target=client, args=(k,)) for k in range(4)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
    for (g, eps, seed), col in zip(reqs_in, out):
        assert np.array_equal(col, oracle.jp_adg(g, eps[0], eps[1], seed)[1])


def test_small_request_overtakes_a_running_large_one():
    # a large graph is running in one slot when a small one arrives: the
    # small one starts in the other slot at once and finishes first, both
    # with the oracle's colours
    big = gg.rmat(21, 16, seed=3)
    small = gg.erdos_renyi(2000, 8000, 4)
    with ColoringServer(0, slots=2) as srv:
        srv.submit(small.row_ptr, small.col_idx, 1, 100, 1).result(timeout=60)  # warm both paths
        rb = srv.submit(big.row_ptr, big.col_idx, 1, 100, 5)
        t0 = time.perf_counter()
        while rb.t_start is None and time.perf_counter() - t0 < 30:
            time.sleep(0.0005)
        rs = srv.submit(small.row_ptr, small.col_idx, 1, 100, 6)
        cs, cb = rs.result(timeout=60), rb.result(timeout=120)
        slots = {k for k, _, _ in srv.batches}
    assert rs.t_done < rb.t_done
    assert slots == {0, 1}
    assert np.array_equal(cs, oracle.jp_adg(small, 1, 100, 6)[1])
    assert np.array_equal(cb, oracle.jp_adg(big, 1, 100, 5)[1])
