"""Full-size workloads, in the configuration the benchmark times
(gc_color_graph on a device-resident graph, eps = 1/100, tie-break seed 42),
compared with the oracle on every vertex: batch ids, round count, colours
and colour count bit for bit; and R-MAT 24 through DEC-ADG-ITR and JP-ADG-O
in the configurations of their benchmark modes."""
from __future__ import annotations

import numpy as np
import pytest

import graphgen as gg
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2008_11321_gb300 as gcp  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_11321_gb300 import _build
    _build.build()
    c = gcp.Context(0)
    yield c
    c.close()


def _check(ctx, g):
    dg = gcp.DeviceGraph.from_host(g, "cuda:0")
    color = torch.empty(g.n, dtype=torch.int32, device="cuda:0")
    batch = torch.empty(g.n, dtype=torch.int32, device="cuda:0")
    nc, nr = ctx.gc_color_graph(dg, 1, 100, 42, color, batch)
    b, c = batch.cpu().numpy(), color.cpu().numpy()
    del dg, color, batch
    ob, nr_o, log = oracle.adg(g, 1, 100, log=True)
    assert nr == nr_o
    assert np.array_equal(b, ob)
    st = ctx.gc_get_stats()
    assert st.sum_U == int(log["U"].sum())
    oc, nc_o = oracle.jp_color(g, oracle.priority(ob, 42))
    assert nc == nc_o
    assert np.array_equal(c, oc)


@pytest.fixture(scope="module")
def rmat24():
    # R-MAT scale 24, edge factor 16, (a,b,c,d) = (.57,.19,.19,.05)
    return gg.rmat(24, 16, seed=1)


def test_rmat24_full(ctx, rmat24):
    _check(ctx, rmat24)


def test_rmat24_dec_itr_full(ctx, rmat24):
    # bench.py --algo dec-itr: gc_color_graph_dec_itr, eps = 1/100, seed 42
    g = rmat24
    dg = gcp.DeviceGraph.from_host(g, "cuda:0")
    color = torch.empty(g.n, dtype=torch.int32, device="cuda:0")
    nc, nr = ctx.gc_color_graph_dec_itr(dg, 1, 100, 42, color)
    it = ctx.gc_get_stats().sim_iterations
    c = color.cpu().numpy()
    del dg, color
    _, oc, onr, onc, oit, _ = oracle.dec_adg_itr(g, 1, 100, 42)
    assert (nr, nc, it) == (onr, onc, oit)
    assert np.array_equal(c, oc)


def test_rmat24_adg_o_full(ctx, rmat24):
    # bench.py --priority adg-o: gc_color_graph_o, eps = 1/100
    g = rmat24
    dg = gcp.DeviceGraph.from_host(g, "cuda:0")
    color = torch.empty(g.n, dtype=torch.int32, device="cuda:0")
    nc, nr = ctx.gc_color_graph_o(dg, 1, 100, color)
    c = color.cpu().numpy()
    del dg, color
    _, _, oc, onr, onc = oracle.jp_adg_o(g, 1, 100)
    assert (nr, nc) == (onr, onc)
    assert np.array_equal(c, oc)


def test_grid256_permuted_full(ctx):
    # 3D 7-point grid 256^3 with a seeded vertex permutation: a single round
    g = gg.grid(256, 256, 256, perm_seed=7)
    _check(ctx, g)
