"""Error paths of the C ABI on the GPU, without faulting it.

Every device-side wait on a colour is bounded; a wait that runs out ends the
call with GC_ERR_TIMEOUT and leaves the device and later contexts usable.
The failure is made on purpose, through the context's failure injection (a
vertex that never publishes its colour, a short wait bound, allocations that
fail), never by a trap, a bad address or an endless loop.
"""
from __future__ import annotations

import os
import time

import numpy as np
import pytest

import graphgen as gg
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2008_11321_gb300 as gcp  # noqa: E402


def context(env, options=None):
    """A context created with `env` set (the library reads its failure
    injection variables at gc_create) and the given gc_options fields."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_11321_gb300 import _build
    _build.build()
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        return gcp.Context(0, options)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


@pytest.fixture(scope="module")
def graph():
    g = gg.erdos_renyi(16384, 81920, seed=1)
    ob, oc, onr, onc = oracle.jp_adg(g, 1, 100, 42)
    return g, ob, oc, onc


def colour(ctx, g):
    dg = gcp.DeviceGraph.from_host(g, "cuda:0")
    color = torch.zeros(g.n, dtype=torch.int32, device="cuda:0")
    nc, _ = ctx.gc_color_graph(dg, 1, 100, 42, color, None)
    torch.cuda.synchronize()
    return nc, color.cpu().numpy()


def test_no_core_matches_oracle(graph):
    # core_target = 0: every vertex goes through the bulk kernels
    g, _, oc, onc = graph
    with context({}, {"core_target": 0}) as ctx:
        nc, c = colour(ctx, g)
        assert nc == onc and np.array_equal(c, oc)
        assert ctx.gc_get_stats().core_vertices == 0


def test_wait_runs_out_and_device_stays_usable(graph):
    g, ob, oc, onc = graph
    # the highest-priority vertex with neighbours: all of them wait on it
    key = oracle.priority(ob, 42)
    deg = g.degrees()
    cand = np.flatnonzero(deg > 0)
    v = int(cand[np.lexsort((cand, key[cand]))[-1]])
    with context({"GC_INJECT_STALL": str(v)}, {"core_target": 0, "wait_limit_ms": 200}) as ctx:
        t0 = time.perf_counter()
        with pytest.raises(gcp.GcError) as err:
            colour(ctx, g)
        elapsed = time.perf_counter() - t0
        assert err.value.status == gcp.GC_ERR_TIMEOUT
        assert elapsed < 5.0
    with context({}) as ctx:  # the device and a fresh context work
        nc, c = colour(ctx, g)
        assert nc == onc and np.array_equal(c, oc)


def test_allocation_failure_reported(graph):
    g, _, oc, onc = graph
    with context({"GC_INJECT_OOM": "1"}) as ctx:
        with pytest.raises(gcp.GcError) as err:
            colour(ctx, g)
        assert err.value.status == gcp.GC_ERR_OOM
    with context({}) as ctx:
        nc, c = colour(ctx, g)
        assert nc == onc and np.array_equal(c, oc)


def test_core_wait_runs_out_and_device_stays_usable(graph):
    # a stalled vertex inside the core (the default core of 16384 vertices
    # holds the top of the priority order): the core cluster's waits on it
    # run out after the limit, the call returns GC_ERR_TIMEOUT, and the
    # device and a fresh context then colour correctly
    g, ob, oc, onc = graph
    key = oracle.priority(ob, 42)
    deg = g.degrees()
    cand = np.flatnonzero(deg > 0)
    v = int(cand[np.lexsort((cand, key[cand]))[-1]])  # the first vertex of the core
    with context({"GC_INJECT_STALL": str(v)}, {"wait_limit_ms": 300}) as ctx:
        t0 = time.perf_counter()
        with pytest.raises(gcp.GcError) as err:
            colour(ctx, g)
        elapsed = time.perf_counter() - t0
        assert err.value.status == gcp.GC_ERR_TIMEOUT
        assert ctx.gc_get_stats().core_vertices > 0
        assert elapsed < 5.0
    with context({}) as ctx:
        nc, c = colour(ctx, g)
        assert nc == onc and np.array_equal(c, oc)


def test_two_contexts_with_different_options_agree(graph):
    # tunables change speed only: two contexts with different options colour
    # the same graph identically, and as the oracle does
    g, ob, oc, onc = graph
    with context({}, {"core_target": 1024, "core_cluster": 4, "core_warps": 4, "update_mode": gcp.GC_UPDATE_PULL,
                      "bulk_blocks_per_sm": 1}) as a, \
            context({}, {"core_target": 32768, "update_mode": gcp.GC_UPDATE_PUSH}) as b:
        assert a.gc_get_options().core_target == 1024
        for ctx in (a, b):
            nc, c = colour(ctx, g)
            assert nc == onc and np.array_equal(c, oc)
        assert a.gc_get_stats().adg_pull_rounds > 0 and b.gc_get_stats().adg_pull_rounds == 0
