"""DEC-ADG-ITR on the GPU vs the CPU oracle, bit for bit, through the C ABI.

Colours, colour counts and SIM-COL iteration counts are integers: exact
equality.  The graphs cover both extraction paths (degree <= 32 by a lane,
larger by a warp), both check/pick paths (at most 32 internal neighbours or
more), bitmaps of many words (cliques past 1,024 colours), partitions with and
without conflicts, more than 255 partitions (the batch then read from its
array instead of the state word), partitions given by the caller (ADG-M's, and
arbitrary ones with empty partitions), and the degenerate cases.
"""
from __future__ import annotations

import numpy as np
import pytest

import graphgen as gg
import oracle
from _fixtures import (case_graph, complete, complete_bipartite, cycle, empty, ints, path, petersen, random_small,
                       read_cases, star, wheel)

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


@pytest.fixture(scope="module")
def ctx_notail():
    # every SIM-COL iteration as GPU-wide launches
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = gcp.Context(0, {"dec_tail": 0})
    yield c
    c.close()


def dev(g):
    return gcp.DeviceGraph.from_host(g, "cuda:0")


def dec_graph(ctx, g, p, q, seed):
    dg = dev(g)
    color = torch.full((g.n,), -7, dtype=torch.int32, device="cuda:0")
    batch = torch.full((g.n,), -7, dtype=torch.int32, device="cuda:0")
    nc, nr = ctx.gc_color_graph_dec_itr(dg, p, q, seed, color, batch)
    st = ctx.gc_get_stats()
    return batch.cpu().numpy(), color.cpu().numpy(), nr, nc, st.sim_iterations, st.dec_internal_edges


def assert_dec_same(ctx, g, p=1, q=100, seed=42):
    b, c, nr, nc, it, inner = dec_graph(ctx, g, p, q, seed)
    ob, oc, onr, onc, oit, _ = oracle.dec_adg_itr(g, p, q, seed)
    assert nr == onr and np.array_equal(b, ob), g.name
    assert np.array_equal(c, oc), g.name
    assert nc == onc and it == oit, (g.name, nc, onc, it, oit)
    src = np.repeat(np.arange(g.n), g.degrees())
    assert inner == int((ob[src] == ob[g.col_idx]).sum()), g.name  # edges of the G(l), both directions
    return c


DEC_GRAPHS = [empty(1), empty(100), complete(2), complete(33), complete(40), star(3), star(32), star(33),
              star(5000), path(7), path(100), path(101), cycle(1000), complete_bipartite(7, 50),
              complete_bipartite(40, 41), petersen(), wheel(64), random_small(60, 0.3, 1),
              random_small(200, 0.05, 2), gg.erdos_renyi(16384, 81920, 1), gg.rmat(12, 8, seed=3),
              gg.rmat(16, 16, seed=2), gg.barabasi_albert(30000, 4, 5), gg.barabasi_albert(2046, 14, 43),
              gg.grid(64, 64, 16, perm_seed=3)]


def _twin_hubs(k):
    # two adjacent hubs sharing k leaves: both land in one partition above the
    # leaves and conflict there; each hub's adjacency spans several chunks
    edges = [(0, 1)] + [(h, 2 + i) for h in (0, 1) for i in range(k)]
    return gg.from_edges(k + 2, edges, f"twinhubs{k}")


DEC_GRAPHS += [star(12345), wheel(9000), _twin_hubs(9000), gg.rmat(18, 16, seed=9)]


@pytest.mark.parametrize("g", DEC_GRAPHS, ids=lambda g: g.name)
@pytest.mark.parametrize("p,q", [(1, 100), (1, 2)])
def test_dec_itr_matches_oracle(ctx, g, p, q):
    assert_dec_same(ctx, g, p, q)


@pytest.mark.parametrize("case", read_cases("dec_itr_small.txt"), ids=lambda c: c["name"])
def test_dec_itr_golden(ctx, case):
    # the hand-worked cases: colours and iterations as derived in the fixture
    g = case_graph(case)
    b, c, nr, nc, it, _ = dec_graph(ctx, g, 1, 100, 42)
    assert nr == int(case["rounds"]) and np.array_equal(b, ints(case["batch"]))
    assert np.array_equal(c, ints(case["color"])) and it == int(case["iterations"])


def test_dec_itr_clique_beyond_window(ctx):
    # K_1100 is one partition coloured one vertex per iteration: 1100
    # iterations, bitmaps of 35 words, colours 1..1100 by decreasing key
    c = assert_dec_same(ctx, complete(1100))
    assert sorted(c.tolist()) == list(range(1, 1101))


@pytest.mark.parametrize("p,q", [(1, 100), (1, 10), (1, 2)])
def test_dec_itr_rmat20(ctx, p, q):
    assert_dec_same(ctx, gg.rmat(20, 16, seed=1), p, q)


@pytest.mark.parametrize("seed", [0, 2**63 + 11])
def test_dec_itr_seeds(ctx, seed):
    assert_dec_same(ctx, gg.rmat(14, 16, seed=5), 1, 100, seed)


@pytest.mark.parametrize("n", [500, 600])
def test_dec_itr_many_partitions(ctx, n):
    # eps = 2^-20 peels a path from both ends: n/2 partitions, 250 (batch in
    # the state word) and 300 (batch read from its array)
    assert oracle.adg(path(n), 1, 1 << 20)[1] == n // 2
    assert_dec_same(ctx, path(n), 1, 1 << 20)


def _given(ctx, g, batch, rounds, seed=42):
    dg = dev(g)
    b = torch.from_numpy(np.ascontiguousarray(batch, dtype=np.int32)).to("cuda:0")
    color = torch.full((g.n,), -7, dtype=torch.int32, device="cuda:0")
    nc = ctx.gc_dec_itr_color(dg, b, rounds, seed, color)
    return color.cpu().numpy(), nc, ctx.gc_get_stats().sim_iterations


def test_dec_itr_given_partitions(ctx):
    # ADG-M's partitions (DEC-ADG-M-ITR), and arbitrary ones with empty
    # partitions and more partitions than vertices need
    for g in (gg.rmat(15, 16, seed=3), gg.barabasi_albert(5000, 6, 2), complete(70)):
        bm, rm = oracle.adg_m(g)
        oc, onc, oit, _ = oracle.dec_itr(g, bm, rm, 42)
        c, nc, it = _given(ctx, g, bm, rm)
        assert np.array_equal(c, oc) and nc == onc and it == oit, g.name
        rb = (np.random.default_rng(g.n).integers(1, 9, g.n) * 3).astype(np.int32)
        oc, onc, oit, _ = oracle.dec_itr(g, rb, 30, 7)
        c, nc, it = _given(ctx, g, rb, 30, 7)
        assert np.array_equal(c, oc) and nc == onc and it == oit, g.name


def test_dec_itr_sparse_partition_ids(ctx):
    # 3 non-empty partitions numbered up to 200,000 of num_rounds = 250,000:
    # only the partitions that hold vertices are visited (the call returns
    # quickly), and the colouring is the one of the same partitions
    # numbered 1..3, with the same iteration count
    import time
    g = gg.barabasi_albert(20000, 6, 5)
    dense = (np.random.default_rng(5).integers(1, 4, g.n)).astype(np.int32)
    sparse = np.array([0, 7, 90000, 200000], dtype=np.int32)[dense]
    oc, onc, oit, _ = oracle.dec_itr(g, dense, 3, 11)
    t0 = time.perf_counter()
    c, nc, it = _given(ctx, g, sparse, 250000, 11)
    elapsed = time.perf_counter() - t0
    assert np.array_equal(c, oc) and nc == onc and it == oit
    assert elapsed < 10.0


def test_itr_one_partition(ctx):
    # every vertex in one partition: plain ITR, the paper's comparison point
    for g in (gg.rmat(16, 16, seed=4), gg.barabasi_albert(20000, 8, 1), complete(200)):
        ones = np.ones(g.n, dtype=np.int32)
        oc, onc, oit, _ = oracle.dec_itr(g, ones, 1, 42)
        c, nc, it = _given(ctx, g, ones, 1)
        assert np.array_equal(c, oc) and nc == onc and it == oit, g.name


def test_dec_itr_rejects_bad_partitions(ctx):
    g = path(6)
    for batch, rounds in (([1, 2, 3, 3, 2, 1], 2), ([0, 1, 1, 1, 1, 1], 3), ([1] * 6, 0)):
        with pytest.raises(gcp.GcError) as e:
            _given(ctx, g, np.array(batch), rounds)
        assert e.value.status == gcp.GC_ERR_INVALID_ARG
    # the context stays usable
    assert_dec_same(ctx, gg.rmat(10, 8, seed=1))


def test_dec_itr_zero_vertices(ctx):
    dg = dev(empty(0))
    out = torch.empty(0, dtype=torch.int32, device="cuda:0")
    assert ctx.gc_color_graph_dec_itr(dg, 1, 100, 42, out) == (0, 0)
    assert ctx.gc_dec_itr_color(dg, out, 1, 42, out) == 0


TAIL_GRAPHS = [complete(300), complete(1100), gg.rmat(16, 16, seed=2), gg.rmat(18, 16, seed=9),
               gg.barabasi_albert(2046, 14, 43), _twin_hubs(9000), gg.rmat(20, 16, seed=1)]


@pytest.mark.parametrize("g", TAIL_GRAPHS, ids=lambda g: g.name)
def test_dec_itr_tail_and_launch_paths(ctx, ctx_notail, g):
    # the single-cluster tail and the GPU-wide iterations give the oracle's
    # colouring; the dense graphs here do reach the tail
    c1 = assert_dec_same(ctx, g)
    tails = ctx.gc_get_stats().dec_tail_partitions
    c2 = assert_dec_same(ctx_notail, g)
    assert ctx_notail.gc_get_stats().dec_tail_partitions == 0
    assert np.array_equal(c1, c2)
    if g.name.startswith(("K300", "K1100", "rmat")):
        assert tails >= 1, g.name
