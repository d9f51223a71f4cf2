"""Full-size workloads, in the configuration the benchmark times
(gc_color_graph on a device-resident graph, eps = 1/100, tie-break seed 42),
compared with the oracle on every vertex: batch ids, round count, colours
and colour count bit for bit."""
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


def test_rmat24_full(ctx):
    # R-MAT scale 24, edge factor 16, (a,b,c,d) = (.57,.19,.19,.05)
    _check(ctx, gg.rmat(24, 16, seed=1))


def test_grid256_permuted_full(ctx):
    # 3D 7-point grid 256^3 with a seeded vertex permutation: a single round
    g = gg.grid(256, 256, 256, perm_seed=7)
    _check(ctx, g)
