"""gc_color_batch: every graph of a packed batch gets exactly the batches,
round count, colours and colour count that the oracle (and gc_color_graph
on the graph alone) give it with its own eps and seed -- on both paths: the
segmented one (GPU-wide launches per ADG round) and the persistent one (one
launch, a thread block per graph)."""
from __future__ import annotations

import numpy as np
import pytest

import graphgen as gg
import oracle
from _fixtures import complete, empty, path, star

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2008_11321_gb300 as gcp  # noqa: E402


MODES = {"auto": gcp.GC_BATCH_AUTO, "segmented": gcp.GC_BATCH_SEGMENTED, "persistent": gcp.GC_BATCH_PERSISTENT,
         "segmented-host-rounds": gcp.GC_BATCH_SEGMENTED}


@pytest.fixture(scope="module", params=sorted(MODES))
def ctx(request):
    # the segmented path runs ADG's rounds from round 2 on as one CUDA graph
    # launch by default; "segmented-host-rounds" launches each round from
    # the host (round_graph 0)
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_11321_gb300 import _build
    _build.build()
    c = gcp.Context(0, {"batch_mode": MODES[request.param], "round_graph": int(request.param != "segmented-host-rounds")})
    c.mode = MODES[request.param]
    yield c
    c.close()


def _mixed(count, seed):
    graphs = []
    for i, (fam, n) in enumerate(gg.batch_recipe(count, 100, 20000, seed)):
        graphs.append(gg.make_batch_graph(fam, n, seed + i))
    return graphs


def _run(ctx, graphs, jobs):
    db = gcp.DeviceBatch.from_host(graphs, "cuda:0")
    color = torch.full((db.n,), -5, dtype=torch.int32, device="cuda:0")
    batch = torch.full((db.n,), -5, dtype=torch.int32, device="cuda:0")
    ncol = torch.full((db.num_graphs,), -5, dtype=torch.int32, device="cuda:0")
    nrnd = torch.full((db.num_graphs,), -5, dtype=torch.int32, device="cuda:0")
    ctx.gc_color_batch(db, jobs, color, batch, ncol, nrnd)
    torch.cuda.synchronize()
    path = ctx.gc_get_stats().batch_path
    assert path == ctx.mode or (ctx.mode == gcp.GC_BATCH_AUTO and path in (1, 2)) or db.n == 0
    voff = db.graph_off.cpu().numpy()
    return color.cpu().numpy(), batch.cpu().numpy(), ncol.cpu().numpy(), nrnd.cpu().numpy(), voff


def test_batch_matches_oracle_per_graph(ctx):
    graphs = _mixed(40, 7) + [empty(0), empty(5), complete(30), star(40), path(7), gg.rmat(12, 8, seed=3)]
    jobs = [((1, 100) if i % 3 else (1, 10)) + (42 + i,) for i in range(len(graphs))]
    color, batch, ncol, nrnd, voff = _run(ctx, graphs, jobs)
    st = ctx.gc_get_stats()
    sum_u = dec = 0
    for i, g in enumerate(graphs):
        p, q, sd = jobs[i]
        ob, oc, onr, onc = oracle.jp_adg(g, p, q, sd)
        sl = slice(voff[i], voff[i + 1])
        assert np.array_equal(batch[sl], ob), i
        assert np.array_equal(color[sl], oc), i
        assert nrnd[i] == onr and ncol[i] == onc, (i, nrnd[i], onr, ncol[i], onc)
        if g.n:
            sum_u += int(oracle.adg(g, p, q, log=True)[2]["U"].sum())
            src = np.repeat(np.arange(g.n), g.degrees())
            dec += int(np.sum(ob[g.col_idx] > ob[src]))
    # ADG's work counters over the batch: sum of |U| over graphs and rounds,
    # and the degree decrements (edges into a later batch)
    assert st.sum_U == sum_u and st.sum_decrements == dec


def test_batch_equals_single_graph_calls(ctx):
    graphs = _mixed(12, 99)
    jobs = [(1, 100, 42 + i) for i in range(len(graphs))]
    color, batch, _, _, voff = _run(ctx, graphs, jobs)
    for i, g in enumerate(graphs):
        dg = gcp.DeviceGraph.from_host(g, "cuda:0")
        c1 = torch.empty(g.n, dtype=torch.int32, device="cuda:0")
        ctx.gc_color_graph(dg, 1, 100, 42 + i, c1)
        assert np.array_equal(color[voff[i]:voff[i + 1]], c1.cpu().numpy()), i


def test_batch_twice_same_result(ctx):
    graphs = _mixed(20, 5)
    jobs = [(1, 100, 7 * i) for i in range(len(graphs))]
    a = _run(ctx, graphs, jobs)
    b = _run(ctx, graphs, jobs)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_batch_hard_cases(ctx):
    # many ADG rounds (short paths, eps = 0), colours beyond the 1024-colour
    # window of the warp path (K_1100), hubs (stars, a BA graph), isolated
    # vertices and empty graphs, all in one batch
    graphs = [path(60), path(99), complete(1100), star(3000), empty(1), empty(0), gg.barabasi_albert(5000, 7, 4),
              gg.grid(40, 50, perm_seed=9), complete(33), gg.erdos_renyi(3000, 200, 2), path(600)]
    jobs = [(0, 1, 5), (1, 100, 6), (1, 100, 7), (1, 2, 8), (1, 100, 9), (1, 100, 10), (3, 1, 11), (1, 100, 12),
            (1, 100, 13), (1, 10, 14), (1, 1 << 20, 15)]  # the last: 300 rounds, beyond an 8-bit batch
    color, batch, ncol, nrnd, voff = _run(ctx, graphs, jobs)
    for i, g in enumerate(graphs):
        p, q, sd = jobs[i]
        ob, oc, onr, onc = oracle.jp_adg(g, p, q, sd)
        sl = slice(voff[i], voff[i + 1])
        assert np.array_equal(batch[sl], ob), i
        assert np.array_equal(color[sl], oc), i
        assert nrnd[i] == onr and ncol[i] == onc, (i, nrnd[i], onr, ncol[i], onc)


def test_batch_list_entry_point(ctx):
    # the separately-resident form the serving path uses
    graphs = _mixed(16, 31)
    jobs = [(1, 100, 3 + i) for i in range(len(graphs))]
    dgs = [gcp.DeviceGraph.from_host(g, "cuda:0") for g in graphs]
    outs = [torch.full((g.n,), -1, dtype=torch.int32, device="cuda:0") for g in graphs]
    ctx.gc_color_batch_list(dgs, jobs, outs)
    for g, (p, q, sd), o in zip(graphs, jobs, outs):
        assert np.array_equal(o.cpu().numpy(), oracle.jp_adg(g, p, q, sd)[1])


def test_auto_takes_persistent_for_many_small_graphs():
    # every graph holds at most 1/1024 of the batch's entries: one launch
    graphs = [gg.erdos_renyi(40, 100, 900 + i) for i in range(1500)]
    jobs = [(1, 100, 5 + i) for i in range(len(graphs))]
    with gcp.Context(0) as c:
        c.mode = gcp.GC_BATCH_AUTO
        color, batch, ncol, nrnd, voff = _run(c, graphs, jobs)
        assert c.gc_get_stats().batch_path == gcp.GC_BATCH_PERSISTENT
    for i in (0, 1, 700, 1499):
        ob, oc, onr, onc = oracle.jp_adg(graphs[i], *jobs[i])
        sl = slice(voff[i], voff[i + 1])
        assert np.array_equal(batch[sl], ob) and np.array_equal(color[sl], oc), i


def test_auto_falls_back_to_segmented_on_a_fresh_context():
    # AUTO with one graph too large for a block (more than 1/1024 of the
    # batch's entries) in a multi-graph batch, on a fresh context: the persistent
    # path's check grows the scratch, then the segmented path runs on the
    # grown scratch
    graphs = [gg.rmat(16, 16, seed=8), path(9), complete(6), gg.erdos_renyi(300, 900, 2)]
    jobs = [(1, 100, 70 + i) for i in range(len(graphs))]
    with gcp.Context(0) as c:
        c.mode = gcp.GC_BATCH_AUTO
        color, batch, ncol, nrnd, voff = _run(c, graphs, jobs)
        assert c.gc_get_stats().batch_path == gcp.GC_BATCH_SEGMENTED
    for i, g in enumerate(graphs):
        ob, oc, onr, onc = oracle.jp_adg(g, *jobs[i])
        sl = slice(voff[i], voff[i + 1])
        assert np.array_equal(batch[sl], ob) and np.array_equal(color[sl], oc), i
