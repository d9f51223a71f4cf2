"""The tuning cache (host side, no GPU) and the library's autotuner on the
GPU: tuned options are applied to the context, reproduce the oracle's
colouring, and are never slower than the starting ones by the tuner's own
measurement."""
from __future__ import annotations

import json

import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_2008_11321_gb300 as gcp
from paper_2008_11321_gb300 import tuning


def test_classes_and_cache_round_trip(tmp_path):
    assert tuning.graph_class(1 << 24, 520_000_000, 1, 100) == "graph/n2^24/deg2^5/eps1:100"
    assert tuning.graph_class(0, 0, 1, 2) == "graph/n2^0/deg2^0/eps1:2"
    assert tuning.batch_class(4096, 108_000_000, 723_000_000) == "batch/g2^12/n2^15/deg2^3"
    path = tmp_path / "t.json"
    c = tuning.TuningCache(str(path))
    assert c.get("GB300", "x") is None
    c.put("GB300", "x", {"options": {"core_target": 8192}, "best_ms": 1.0})
    c.put("GB300", "y", {"options": {"core_target": 0}, "best_ms": 2.0})
    c.put("other", "x", {"options": {}, "best_ms": 3.0})
    assert c.get("GB300", "x")["options"] == {"core_target": 8192}
    assert json.loads(path.read_text())["GB300"]["y"]["best_ms"] == 2.0
    assert tuning.TuningCache(str(path)).get("other", "x")["best_ms"] == 3.0


def test_cache_path_from_environment(monkeypatch, tmp_path):
    monkeypatch.setenv("GC_TUNING_CACHE", str(tmp_path / "c.json"))
    assert tuning.default_path() == str(tmp_path / "c.json")


torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_11321_gb300 import _build
    _build.build()
    c = gcp.Context(0)
    yield c
    c.close()


@pytest.mark.gpu
def test_autotune_graph(ctx, tmp_path):
    g = gg.rmat(14, 16, seed=2)
    dg = gcp.DeviceGraph.from_host(g, "cuda:0")
    rec = tuning.tune_graph(ctx, dg, 1, 100, 42, cache=tuning.TuningCache(str(tmp_path / "t.json")), reps=1)
    assert rec["searched"] and rec["best_ms"] <= rec["start_ms"]
    assert ctx.gc_get_options().as_dict() == rec["options"]
    color = torch.empty(g.n, dtype=torch.int32, device="cuda:0")
    nc, _ = ctx.gc_color_graph(dg, 1, 100, 42, color)
    assert np.array_equal(color.cpu().numpy(), oracle.jp_adg(g, 1, 100, 42)[1])
    # the second time the cache answers without a search
    rec2 = tuning.tune_graph(ctx, dg, 1, 100, 42, cache=tuning.TuningCache(str(tmp_path / "t.json")))
    assert not rec2["searched"] and rec2["options"] == rec["options"]
    ctx.gc_set_options({})  # back to the defaults for the other tests


@pytest.mark.gpu
def test_autotune_batch(ctx, tmp_path):
    graphs = [gg.make_batch_graph(f, n, 5 + i) for i, (f, n) in enumerate(gg.batch_recipe(24, 100, 5000, 5))]
    jobs = [(1, 100, 9 + i) for i in range(len(graphs))]
    db = gcp.DeviceBatch.from_host(graphs, "cuda:0")
    rec = tuning.tune_batch(ctx, db, jobs, cache=tuning.TuningCache(str(tmp_path / "b.json")), reps=1)
    assert rec["options"]["batch_mode"] in (gcp.GC_BATCH_SEGMENTED, gcp.GC_BATCH_PERSISTENT)
    color = torch.empty(db.n, dtype=torch.int32, device="cuda:0")
    ctx.gc_color_batch(db, jobs, color)
    voff = db.graph_off.cpu().numpy()
    for i, g in enumerate(graphs):
        assert np.array_equal(color.cpu().numpy()[voff[i]:voff[i + 1]], oracle.jp_adg(g, *jobs[i])[1])
    ctx.gc_set_options({})


@pytest.mark.gpu
def test_autotune_budget_stops_early(ctx):
    g = gg.erdos_renyi(20000, 100000, 3)
    dg = gcp.DeviceGraph.from_host(g, "cuda:0")
    best, best_ms, start_ms = ctx.gc_autotune(dg, 1, 100, 42, 1, 0.001)  # the first trial exhausts the budget
    assert best.as_dict() == gcp.make_options().as_dict() and best_ms == start_ms
    ctx.gc_set_options({})
