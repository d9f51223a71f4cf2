"""ADG-O and JP-ADG-O on the GPU vs the CPU oracle, bit for bit, through the
C ABI: batches, the total order rho, the higher-rho neighbour counts, and
the JP-ADG-O colouring, on families with ties in D (cliques, stars, paths,
grids), more than 255 iterations, constant keys (a single digit-free sort)
and the R-MAT shapes of the benchmark."""
from __future__ import annotations

import numpy as np
import pytest

import graphgen as gg
import oracle
from _fixtures import (case_graph, complete, complete_bipartite, cycle, empty, ints, path, petersen, random_small,
                       read_cases, star)

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


def dev(g):
    return gcp.DeviceGraph.from_host(g, "cuda:0")


def i32(n):
    return torch.full((n,), -7, dtype=torch.int32, device="cuda:0")


GRAPHS = [empty(1), empty(50), complete(2), complete(40), complete(1100), star(3), star(5000), path(7), path(100),
          path(101), cycle(999), complete_bipartite(7, 50), petersen(), random_small(80, 0.2, 3),
          gg.erdos_renyi(16384, 81920, 1), gg.rmat(12, 8, seed=3), gg.rmat(16, 16, seed=2),
          gg.barabasi_albert(20000, 5, 3), gg.grid(64, 64, 16, perm_seed=3), gg.rmat(20, 16, seed=1)]


@pytest.mark.parametrize("g", GRAPHS, ids=lambda g: g.name)
@pytest.mark.parametrize("p,q", [(1, 100), (1, 2)])
def test_adg_o_matches_oracle(ctx, g, p, q):
    dg = dev(g)
    b, rho, rank = i32(g.n), i32(g.n), i32(g.n)
    nr = ctx.gc_adg_o_order(dg, p, q, rho, b, rank)
    ob, orho, orank, onr = oracle.adg_o(g, p, q)
    assert nr == onr and np.array_equal(b.cpu().numpy(), ob), g.name
    assert np.array_equal(rho.cpu().numpy(), orho), g.name
    assert np.array_equal(rank.cpu().numpy(), orank), g.name
    color, b2 = i32(g.n), i32(g.n)
    nc, nr2 = ctx.gc_color_graph_o(dg, p, q, color, b2)
    _, _, oc, _, onc = oracle.jp_adg_o(g, p, q)
    assert nr2 == onr and np.array_equal(b2.cpu().numpy(), ob), g.name
    assert nc == onc and np.array_equal(color.cpu().numpy(), oc), g.name


@pytest.mark.parametrize("case", read_cases("adg_o_small.txt"), ids=lambda c: c["name"])
def test_adg_o_golden(ctx, case):
    # the hand-worked cases: rho, rank and the JP-ADG-O colours
    g = case_graph(case)
    dg = dev(g)
    rho, rank, color = i32(g.n), i32(g.n), i32(g.n)
    ctx.gc_adg_o_order(dg, 1, 100, rho, None, rank)
    ctx.gc_color_graph_o(dg, 1, 100, color)
    assert np.array_equal(rho.cpu().numpy(), ints(case["rho"]))
    assert np.array_equal(rank.cpu().numpy(), ints(case["rank"]))
    assert np.array_equal(color.cpu().numpy(), ints(case["color"]))


@pytest.mark.parametrize("n", [520, 1500])
def test_adg_o_many_iterations(ctx, n):
    # eps = 2^-20 peels a path two vertices per iteration: n/2 iterations
    g = path(n)
    dg = dev(g)
    rho = i32(n)
    assert ctx.gc_adg_o_order(dg, 1, 1 << 20, rho) == n // 2
    assert np.array_equal(rho.cpu().numpy(), oracle.adg_o(g, 1, 1 << 20)[1])
    color = i32(n)
    nc, _ = ctx.gc_color_graph_o(dg, 1, 1 << 20, color)
    assert np.array_equal(color.cpu().numpy(), oracle.jp_adg_o(g, 1, 1 << 20)[2]) and nc == 2


def test_adg_o_optional_outputs_and_empty(ctx):
    g = gg.rmat(14, 8, seed=4)
    dg = dev(g)
    rho = i32(g.n)
    ctx.gc_adg_o_order(dg, 1, 100, rho)  # no batch, no rank
    assert np.array_equal(rho.cpu().numpy(), oracle.adg_o(g, 1, 100)[1])
    e = dev(empty(0))
    z = torch.empty(0, dtype=torch.int32, device="cuda:0")
    assert ctx.gc_adg_o_order(e, 1, 100, z) == 0
    assert ctx.gc_color_graph_o(e, 1, 100, z) == (0, 0)
    with pytest.raises(gcp.GcError) as err:
        ctx.gc_adg_o_order(dg, 1, 0, rho)
    assert err.value.status == gcp.GC_ERR_INVALID_ARG
