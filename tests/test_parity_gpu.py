"""CUDA path vs the CPU oracle, bit for bit, through the C ABI.

Batch ids, round counts, colours and colour counts are integers, so the bar
is exact equality.  Graphs span several thread blocks and ragged tails,
vertices above the lane/warp split (degree 32), UPDATE tasks split at 1024
edges, colours above the 1024-colour window, and the degenerate cases of the
method (no vertices, no edges, isolated vertices, cliques, stars, paths).
"""
from __future__ import annotations

import numpy as np
import pytest

import graphgen as gg
import oracle
from _fixtures import (case_graph, complete, complete_bipartite, cycle, empty, ints, path, petersen,
                       random_small, read_cases, star)

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


def color_graph(ctx, g, p, q, seed):
    dg = dev(g)
    color = torch.full((g.n,), -7, dtype=torch.int32, device="cuda:0")
    batch = torch.full((g.n,), -7, dtype=torch.int32, device="cuda:0")
    nc, nr = ctx.gc_color_graph(dg, p, q, seed, color, batch)
    torch.cuda.synchronize()
    return batch.cpu().numpy(), color.cpu().numpy(), nr, nc


def assert_same_as_oracle(ctx, g, p=1, q=100, seed=42):
    b, c, nr, nc = color_graph(ctx, g, p, q, seed)
    ob, oc, onr, onc = oracle.jp_adg(g, p, q, seed)
    assert nr == onr, (g.name, nr, onr)
    assert np.array_equal(b, ob), g.name
    assert nc == onc, (g.name, nc, onc)
    assert np.array_equal(c, oc), g.name
    return b, c


SMALL = [empty(1), empty(100), complete(2), complete(5), complete(33), complete(40), star(3),
         star(31), star(32), star(33), star(5000), path(7), path(100), path(101), cycle(1000),
         complete_bipartite(7, 50), complete_bipartite(40, 41), petersen(),
         random_small(60, 0.3, 1), random_small(200, 0.05, 2)]


@pytest.mark.parametrize("g", SMALL, ids=lambda g: g.name)
def test_small_families(ctx, g):
    assert_same_as_oracle(ctx, g)


@pytest.mark.parametrize("case", read_cases("jp_adg_small.txt") + read_cases("lollipop_adg.txt"),
                         ids=lambda c: c.get("name", "lollipop"))
def test_golden_fixtures(ctx, case):
    g = case_graph(case)
    b, c = assert_same_as_oracle(ctx, g)
    assert np.array_equal(b, ints(case["batch"]))
    if "color" in case:
        assert np.array_equal(c, ints(case["color"]))


def test_zero_vertices(ctx):
    g = empty(0)
    dg = dev(g)
    color = torch.empty(0, dtype=torch.int32, device="cuda:0")
    assert ctx.gc_color_graph(dg, 1, 100, 42, color) == (0, 0)


@pytest.mark.parametrize("n,seed", [(2046, 43), (8000, 7)])
def test_large_core_buckets(ctx, n, seed):
    # Barabasi-Albert graphs small enough to be all core, with ~80% of the
    # vertices in ADG's first batch: core buckets of ~200 vertices, ordered by
    # the block-wide sort rather than the per-thread one.
    assert_same_as_oracle(ctx, gg.barabasi_albert(n, 14, seed), 1, 10)


@pytest.mark.parametrize("n", [500, 520, 1500])
def test_many_adg_rounds(ctx, n):
    # With eps = 2^-20 the ADG threshold on a path stays 1 (Algorithm 1), so
    # each round removes only the two ends: n/2 rounds.  JP-ADG keeps the batch
    # in 8 bits of the colour word up to 255 rounds and orders by the full
    # batch array beyond; 500 / 520 / 1500 vertices land on both sides.
    g = path(n)
    p, q = 1, 1 << 20
    _, _, onr, _ = oracle.jp_adg(g, p, q, 42)
    assert onr == n // 2
    assert_same_as_oracle(ctx, g, p, q)


def test_clique_beyond_colour_window(ctx):
    # K_1100: colours 1..1100 exceed one 1024-colour window of the warp path
    g = complete(1100)
    b, c = assert_same_as_oracle(ctx, g)
    assert sorted(c.tolist()) == list(range(1, 1101))


def test_er_config(ctx):
    # Erdos-Renyi G(n=16384, m=81920), eps = 1/100, tie-break seed 42
    assert_same_as_oracle(ctx, gg.erdos_renyi(16384, 81920, 1), 1, 100, 42)


@pytest.mark.parametrize("p,q", [(1, 100), (1, 10), (1, 2), (0, 1), (3, 1), (7, 1000)])
def test_eps_sweep(ctx, p, q):
    for g in (gg.rmat(14, 16, seed=3), gg.erdos_renyi(20000, 100000, 4), gg.barabasi_albert(8000, 6, 5)):
        assert_same_as_oracle(ctx, g, p, q, 42)


@pytest.mark.parametrize("scale,ef", [(8, 4), (10, 16), (12, 8), (15, 16), (16, 4)])
def test_rmat_ragged(ctx, scale, ef):
    assert_same_as_oracle(ctx, gg.rmat(scale, ef, seed=scale), 1, 100, scale)


@pytest.mark.parametrize("g", [gg.grid(100, 100), gg.grid(101, 101), gg.grid(33, 47, perm_seed=3),
                               gg.grid(24, 24, 24, perm_seed=5), gg.barabasi_albert(30000, 4, 9),
                               gg.barabasi_albert(3000, 40, 9)], ids=lambda g: g.name)
def test_grids_and_ba(ctx, g):
    assert_same_as_oracle(ctx, g)


@pytest.mark.parametrize("seed", [0, 1, 2**63 + 11])
def test_seeds(ctx, seed):
    assert_same_as_oracle(ctx, gg.rmat(13, 16, seed=7), 1, 100, seed)


@pytest.mark.parametrize("p,q", [(1, 100), (1, 10), (1, 2)])
def test_rmat20_config(ctx, p, q):
    # R-MAT scale 20, edge factor 16, (a,b,c,d) = (.57,.19,.19,.05)
    assert_same_as_oracle(ctx, gg.rmat(20, 16, seed=1), p, q, 42)


def test_adg_partition_and_stats(ctx):
    g = gg.rmat(16, 16, seed=2)
    dg = dev(g)
    batch = torch.empty(g.n, dtype=torch.int32, device="cuda:0")
    rounds = ctx.gc_adg_partition(dg, 1, 100, batch)
    ob, onr, log = oracle.adg(g, 1, 100, log=True)
    assert rounds == onr and np.array_equal(batch.cpu().numpy(), ob)
    st = ctx.gc_get_stats()
    assert st.adg_rounds == onr
    assert st.sum_U == int(log["U"].sum())
    src = np.repeat(np.arange(g.n), g.degrees())
    assert st.sum_decrements == int(np.sum(ob[g.col_idx] > ob[src]))


def test_make_priority(ctx):
    n = 100003
    rng = np.random.default_rng(1)
    b = rng.integers(0, 2**31 - 1, size=n).astype(np.int32)
    bt = torch.from_numpy(b).cuda()
    key = torch.empty(n, dtype=torch.int64, device="cuda:0")
    ctx.gc_make_priority(n, bt, 987654321, key)
    torch.cuda.synchronize()
    assert np.array_equal(key.cpu().numpy().view(np.uint64), oracle.priority(b, 987654321))


@pytest.mark.parametrize("kind", ["ties", "full64", "adg"])
def test_jp_color_given_priority(ctx, kind):
    g = gg.rmat(14, 16, seed=11)
    rng = np.random.default_rng(5)
    if kind == "ties":
        prio = rng.integers(0, 3, size=g.n).astype(np.uint64)
    elif kind == "full64":
        prio = rng.integers(0, 2**63, size=g.n, dtype=np.uint64) * np.uint64(2) + \
            rng.integers(0, 2, size=g.n).astype(np.uint64)
    else:
        prio = oracle.priority(oracle.adg(g, 1, 100)[0], 42)
    dg = dev(g)
    pt = torch.from_numpy(prio.view(np.int64)).cuda()
    color = torch.empty(g.n, dtype=torch.int32, device="cuda:0")
    nc = ctx.gc_jp_color(dg, pt, color)
    oc, onc = oracle.jp_color(g, prio)
    assert nc == onc and np.array_equal(color.cpu().numpy(), oc)


VARIANT_GRAPHS = [gg.erdos_renyi(20000, 100000, seed=3), gg.rmat(16, 16, seed=2),
                  gg.grid(64, 64, 16, perm_seed=3), gg.barabasi_albert(30000, 4, 5), star(5000), empty(50)]


@pytest.mark.parametrize("kind", [0, 1, 2, 3, 4], ids=["R", "FF", "LF", "LLF", "SL"])
def test_jp_variants(ctx, kind):
    # JP-R / FF / LF / LLF / SL (Section 4.1): keys bit for bit, then the
    # colouring; SL's key is the smallest-last removal index
    for g in VARIANT_GRAPHS:
        dg = dev(g)
        key = torch.zeros(g.n, dtype=torch.int64, device="cuda:0")
        ctx.gc_make_priority_kind(dg, kind, 42, key)
        ok = oracle.priority_kind(g, kind, 42)
        assert np.array_equal(key.cpu().numpy().view(np.uint64), ok), g.name
        color = torch.empty(g.n, dtype=torch.int32, device="cuda:0")
        nc = ctx.gc_jp_color(dg, key, color)
        oc, onc = oracle.jp_color(g, ok)
        assert nc == onc and np.array_equal(color.cpu().numpy(), oc), g.name


ADGM_GRAPHS = [empty(1), empty(77), path(2), path(3), complete(10), complete(1100), star(3), star(6), star(5000),
               cycle(999), gg.erdos_renyi(20000, 100000, seed=3), gg.rmat(16, 16, seed=2),
               gg.grid(64, 64, 16, perm_seed=3), gg.barabasi_albert(30000, 4, 5), gg.rmat(20, 16, seed=1)]


@pytest.mark.parametrize("g", ADGM_GRAPHS, ids=lambda g: g.name)
def test_adg_m_and_jp_adg_m(ctx, g):
    # ADG-M (Section 5 median variant): batches bit for bit, then JP-ADG-M
    dg = dev(g)
    batch = torch.full((g.n,), -7, dtype=torch.int32, device="cuda:0")
    nr = ctx.gc_adg_m_partition(dg, batch)
    ob, onr = oracle.adg_m(g)
    assert nr == onr and np.array_equal(batch.cpu().numpy(), ob), g.name
    color = torch.full((g.n,), -7, dtype=torch.int32, device="cuda:0")
    batch2 = torch.full((g.n,), -7, dtype=torch.int32, device="cuda:0")
    nc, nr2 = ctx.gc_color_graph_m(dg, 42, color, batch2)
    _, oc, _, onc = oracle.jp_adg_m(g, 42)
    assert nr2 == onr and np.array_equal(batch2.cpu().numpy(), ob), g.name
    assert nc == onc and np.array_equal(color.cpu().numpy(), oc), g.name


def test_adg_m_zero_vertices(ctx):
    dg = dev(empty(0))
    assert ctx.gc_adg_m_partition(dg, torch.empty(0, dtype=torch.int32, device="cuda:0")) == 0
    assert ctx.gc_color_graph_m(dg, 1, torch.empty(0, dtype=torch.int32, device="cuda:0")) == (0, 0)


def test_jp_variant_kind_rejected(ctx):
    dg = dev(path(5))
    key = torch.zeros(5, dtype=torch.int64, device="cuda:0")
    for bad in (-1, 5):
        with pytest.raises(gcp.GcError) as e:
            ctx.gc_make_priority_kind(dg, bad, 1, key)
        assert e.value.status == gcp.GC_ERR_INVALID_ARG


def test_three_calls_equal_one(ctx):
    # adg_partition + make_priority + jp_color == color_graph
    g = gg.barabasi_albert(20000, 5, 3)
    dg = dev(g)
    batch = torch.empty(g.n, dtype=torch.int32, device="cuda:0")
    ctx.gc_adg_partition(dg, 1, 10, batch)
    key = torch.empty(g.n, dtype=torch.int64, device="cuda:0")
    ctx.gc_make_priority(g.n, batch, 77, key)
    c1 = torch.empty(g.n, dtype=torch.int32, device="cuda:0")
    ctx.gc_jp_color(dg, key, c1)
    c2 = torch.empty(g.n, dtype=torch.int32, device="cuda:0")
    ctx.gc_color_graph(dg, 1, 10, 77, c2)
    assert torch.equal(c1, c2)


@pytest.mark.parametrize("scale", [15, 20])
def test_host_entry_point(ctx, scale):
    # scale 20: a 126 MB col_idx upload
    g = gg.rmat(scale, 16, seed=4)
    color = np.zeros(g.n, dtype=np.int32)
    batch = np.zeros(g.n, dtype=np.int32)
    nc, nr = ctx.gc_color_graph_host(g.row_ptr, g.col_idx, 1, 100, 42, color, batch)
    ob, oc, onr, onc = oracle.jp_adg(g, 1, 100, 42)
    assert (nc, nr) == (onc, onr)
    assert np.array_equal(batch, ob) and np.array_equal(color, oc)


@pytest.mark.parametrize("opts", [{}, {"host_upload": 0}, {"update_mode": gcp.GC_UPDATE_PULL}, {"update_hubs": 0}],
                         ids=["auto", "copy-engine", "pull", "nohubs"])
@pytest.mark.parametrize("g", [star(2_500_000), gg.rmat(18, 16, seed=8)], ids=lambda g: g.name)
def test_host_entry_point_ranges(g, opts):
    # from 2^22 entries on, col_idx is copied in vertex ranges on a copy
    # stream (SM copy by default, copy engine with host_upload 0) and round
    # 1's UPDATE sweeps each range once it has arrived (the star: one row
    # holds half the entries, so several ranges are empty); page-locked and
    # pageable buffers, three calls in a row
    rp = torch.empty(g.n + 1, dtype=torch.int64, pin_memory=True).numpy()
    ci = torch.empty(g.nnz, dtype=torch.int32, pin_memory=True).numpy()
    rp[:] = g.row_ptr
    ci[:] = g.col_idx
    ob, oc, onr, onc = oracle.jp_adg(g, 1, 100, 42)
    with gcp.Context(0, opts) as c:
        for r, k in ((rp, ci), (g.row_ptr, g.col_idx), (rp, ci)):
            color = np.zeros(g.n, dtype=np.int32)
            batch = np.zeros(g.n, dtype=np.int32)
            nc, nr = c.gc_color_graph_host(r, k, 1, 100, 42, color, batch)
            assert (nc, nr) == (onc, onr)
            assert np.array_equal(batch, ob) and np.array_equal(color, oc)


@pytest.mark.parametrize("opts", [{}, {"update_mode": gcp.GC_UPDATE_PULL}, {"update_mode": gcp.GC_UPDATE_AUTO,
                                  "pull_percent": 100000}, {"update_hubs": 0}, {"round_graph": 0}],
                         ids=["default", "pull", "auto-pull-often", "nohubs", "host-rounds"])
@pytest.mark.parametrize("g", [gg.rmat(16, 16, seed=41), gg.grid(60, 60, perm_seed=3), gg.barabasi_albert(20000, 5, 6)],
                         ids=lambda g: g.name)
def test_round_loop_graph(g, opts):
    # ADG's rounds from round 2 on run as one CUDA graph launch from the
    # second call with the same buffers on (the first call runs them from the
    # host): four calls in a row give the oracle's batches and colours
    ob, oc, onr, onc = oracle.jp_adg(g, 1, 100, 9)
    dg = dev(g)
    batch = torch.empty(g.n, dtype=torch.int32, device="cuda:0")
    color = torch.empty(g.n, dtype=torch.int32, device="cuda:0")
    with gcp.Context(0, opts) as c:
        for _ in range(4):  # the same buffers every call
            batch.fill_(-1)
            color.fill_(-1)
            nc, nr = c.gc_color_graph(dg, 1, 100, 9, color, batch)
            assert nr == onr and nc == onc
            assert np.array_equal(batch.cpu().numpy(), ob) and np.array_equal(color.cpu().numpy(), oc)
            st = c.gc_get_stats()
            assert st.adg_rounds == onr


def test_scratch_regrow_and_reuse(ctx):
    for g in (gg.rmat(10, 8, seed=1), gg.rmat(17, 16, seed=2), gg.rmat(11, 8, seed=3)):
        assert_same_as_oracle(ctx, g)


def test_user_stream(ctx):
    g = gg.rmat(14, 8, seed=6)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        dg = dev(g)
        color = torch.empty(g.n, dtype=torch.int32, device="cuda:0")
        ctx.gc_color_graph(dg, 1, 100, 42, color, stream=s)
    s.synchronize()
    assert np.array_equal(color.cpu().numpy(), oracle.jp_adg(g, 1, 100, 42)[1])


# ------------------------------------------------------------------ validation

def _raw(n, row_ptr, col_idx):
    rp = torch.tensor(row_ptr, dtype=torch.int64, device="cuda:0")
    ci = torch.tensor(col_idx if col_idx else [0], dtype=torch.int32, device="cuda:0")
    if not col_idx:
        ci = ci[:0]
    return gcp.DeviceGraph(rp, ci)


def test_validate_accepts_generated(ctx):
    for g in (gg.rmat(12, 16), gg.grid(5, 5, 5, perm_seed=2), empty(3), empty(0)):
        assert ctx.gc_validate_csr(dev(g)) == gcp.GC_OK


@pytest.mark.parametrize("name,rp,ci", [
    ("asymmetric", [0, 1, 1], [1]),
    ("self_loop", [0, 1, 2], [0, 0]),
    ("unsorted", [0, 2, 3, 4], [2, 1, 0, 0]),
    ("duplicate", [0, 2, 4], [1, 1, 0, 0]),
    ("id_out_of_range", [0, 1, 2], [5, 0]),
    ("negative_id", [0, 1, 2], [-1, 0]),
    ("row_ptr_decreasing", [0, 2, 1, 2], [1, 2]),
    ("row_ptr_bad_end", [0, 1, 3], [1, 0]),
])
def test_validate_rejects(ctx, name, rp, ci):
    g = _raw(len(rp) - 1, rp, ci)
    assert ctx.gc_validate_csr(g) == gcp.GC_ERR_INVALID_GRAPH


def test_invalid_eps_rejected(ctx):
    g = dev(path(5))
    color = torch.empty(5, dtype=torch.int32, device="cuda:0")
    for p, q in [(1, 0), (1, 2**20 + 1), (2**20 + 1, 1)]:
        with pytest.raises(gcp.GcError) as e:
            ctx.gc_color_graph(g, p, q, 42, color)
        assert e.value.status == gcp.GC_ERR_INVALID_ARG


# ---------------------------------------------------------------- UPDATE direction

@pytest.fixture(scope="module")
def ctx_push():
    c = gcp.Context(0, {"update_mode": gcp.GC_UPDATE_PUSH})
    yield c
    c.close()


@pytest.fixture(scope="module")
def ctx_pull():
    c = gcp.Context(0, {"update_mode": gcp.GC_UPDATE_PULL})
    yield c
    c.close()


DIRECTION_GRAPHS = [gg.rmat(14, 16, seed=3), gg.barabasi_albert(20000, 8, 5), gg.erdos_renyi(30000, 150000, 9),
                    gg.grid(120, 130), star(5000), complete(300), path(60), empty(40)]


@pytest.mark.parametrize("g", DIRECTION_GRAPHS, ids=lambda g: g.name)
@pytest.mark.parametrize("p,q", [(1, 100), (1, 2)])
def test_push_pull_auto_identical(ctx, ctx_push, ctx_pull, g, p, q):
    # Section 5, "Push vs. Pull": a pull round recounts every survivor's
    # degree instead of decrementing it; batches, rounds, colours and the
    # statistics the degree-sum rule carries (sum |U|, decrements) are the
    # same in every direction and equal the oracle's
    ob, oc, onr, onc = oracle.jp_adg(g, p, q, 42)
    _, _, log = oracle.adg(g, p, q, log=True)
    src = np.repeat(np.arange(g.n), g.degrees())
    stats = []
    for c in (ctx, ctx_push, ctx_pull):
        b, col, nr, nc = color_graph(c, g, p, q, 42)
        assert nr == onr and np.array_equal(b, ob)
        assert nc == onc and np.array_equal(col, oc)
        stats.append(c.gc_get_stats())
    assert len({(s.sum_U, s.sum_decrements) for s in stats}) == 1
    assert stats[0].sum_U == int(log["U"].sum())
    assert stats[0].sum_decrements == int(np.sum(ob[g.col_idx] > ob[src]))
    assert stats[1].adg_pull_rounds == 0
    if g.nnz > 0 and onr > 1:
        assert stats[2].adg_pull_rounds >= 1


def test_auto_pulls_when_r_outweighs_u():
    # eps = 1/2 on a Barabasi-Albert graph removes most of U every round:
    # the rows of U' hold fewer entries than the rows of R, so AUTO (here
    # pulling at up to 100 %) pulls
    ctx = gcp.Context(0, {"pull_percent": 100})
    g = gg.barabasi_albert(50000, 4, 11)
    b, c, nr, nc = color_graph(ctx, g, 1, 2, 42)
    ob, oc, onr, onc = oracle.jp_adg(g, 1, 2, 42)
    assert np.array_equal(b, ob) and np.array_equal(c, oc)
    assert 0 < ctx.gc_get_stats().adg_pull_rounds < nr


# ---------------------------------------------------------------- 16-bit JP state

@pytest.fixture(scope="module")
def ctx_state32():
    c = gcp.Context(0, {"jp_state16": 0})
    yield c
    c.close()


@pytest.fixture(scope="module")
def ctx_state16():
    c = gcp.Context(0, {"jp_state16": 1})
    yield c
    c.close()


@pytest.mark.parametrize("g", [gg.rmat(15, 16, seed=7), gg.barabasi_albert(30000, 6, 2), complete(300),
                               gg.grid(64, 64, 8, perm_seed=1)], ids=lambda g: g.name)
def test_state_word_16_and_32_bits_identical(ctx_state16, ctx_state32, g):
    # the batch|colour word of JP-ADG in 16 bits (when the colour bound
    # 1 + max degree at removal fits) or in 32 bits: identical colourings
    ob, oc, onr, onc = oracle.jp_adg(g, 1, 100, 42)
    for c, bits in ((ctx_state16, 16), (ctx_state32, 32)):
        b, col, nr, nc = color_graph(c, g, 1, 100, 42)
        assert nr == onr and np.array_equal(b, ob)
        assert nc == onc and np.array_equal(col, oc)
        assert c.gc_get_stats().jp_state_bits == bits


@pytest.mark.parametrize("n,bits", [(4000, 16), (4100, 32)])
def test_state_word_switch_on_cliques(ctx_state16, n, bits):
    ctx = ctx_state16
    # JP-ADG-M on K_n takes floor(log2 n) + 1 = 12 or 13 rounds (4 batch
    # bits), leaving 12 colour bits (at most 4095): K_4000's 4000 colours fit
    # the 16-bit word, K_4100's 4100 do not and the call falls back to 32 bits
    g = complete(n)
    dg = dev(g)
    color = torch.empty(g.n, dtype=torch.int32, device="cuda:0")
    batch = torch.empty(g.n, dtype=torch.int32, device="cuda:0")
    nc, nr = ctx.gc_color_graph_m(dg, 42, color, batch)
    ob, oc, onr, onc = oracle.jp_adg_m(g, 42)
    assert nr == onr and nc == onc == n
    assert np.array_equal(batch.cpu().numpy(), ob) and np.array_equal(color.cpu().numpy(), oc)
    assert ctx.gc_get_stats().jp_state_bits == bits


def test_jp_sl_small_graphs_and_limit(ctx):
    # the smallest-last order on the hand-derived cases and a graph with
    # several chunks of 2048 vertices, then the size limit
    from _fixtures import complete_bipartite
    for g in (path(7), cycle(6), complete(5), star(5), complete_bipartite(2, 5), gg.rmat(13, 8, seed=4)):
        dg = dev(g)
        key = torch.zeros(g.n, dtype=torch.int64, device="cuda:0")
        ctx.gc_make_priority_kind(dg, gcp.GC_PRIO_SL, 0, key)
        order = np.argsort(key.cpu().numpy())
        assert np.array_equal(order, oracle.smallest_last(g)), g.name
    big = gcp.DeviceGraph(torch.zeros((1 << 25) + 2, dtype=torch.int64, device="cuda:0"),
                          torch.zeros(0, dtype=torch.int32, device="cuda:0"))
    with pytest.raises(gcp.GcError) as err:
        ctx.gc_make_priority_kind(big, gcp.GC_PRIO_SL, 0, torch.empty(1, dtype=torch.int64, device="cuda:0"))
    assert err.value.status == gcp.GC_ERR_OVERFLOW


# ---------------------------------------------------------------- UPDATE hub merging

@pytest.mark.parametrize("hubs", [0, 1, 512, 4096])
@pytest.mark.parametrize("g", [gg.rmat(16, 16, seed=12), gg.barabasi_albert(40000, 8, 3), star(5000), complete(300),
                               gg.grid(90, 90), gg.erdos_renyi(20000, 100000, 6)], ids=lambda g: g.name)
def test_hub_merging_identical(g, hubs):
    # decrements aimed at hubs are counted per block in shared memory at the
    # hub's rank before they reach the degree words: batches, colours and
    # ADG's statistics are unchanged (K_300: every vertex is a hub, ranks
    # spanning several bitmap words; star: the centre; grid: none; hubs=1:
    # only vertices of the top degree class, if it holds one vertex)
    with gcp.Context(0, {"update_hubs": hubs, "update_mode": gcp.GC_UPDATE_PUSH}) as c:
        for p, q in ((1, 100), (1, 2)):
            b, col, nr, nc = color_graph(c, g, p, q, 42)
            ob, oc, onr, onc = oracle.jp_adg(g, p, q, 42)
            assert nr == onr and np.array_equal(b, ob)
            assert nc == onc and np.array_equal(col, oc)
            src = np.repeat(np.arange(g.n), g.degrees())
            assert c.gc_get_stats().sum_decrements == int(np.sum(ob[g.col_idx] > ob[src]))


@pytest.mark.parametrize("misalign", [0, 1])
def test_host_entry_point_kernel_upload(misalign):
    # host_upload = 1: the SMs read the page-locked host CSR directly; a
    # buffer that is not 16-byte aligned falls back to the copy engine
    g = gg.rmat(18, 16, seed=6)
    rp = torch.empty(g.n + 1 + 2 * misalign, dtype=torch.int64, pin_memory=True).numpy()[misalign:misalign + g.n + 1]
    ci = torch.empty(g.nnz + 4 * misalign, dtype=torch.int32, pin_memory=True).numpy()[misalign:misalign + g.nnz]
    rp[:] = g.row_ptr
    ci[:] = g.col_idx
    color = np.zeros(g.n, dtype=np.int32)
    with gcp.Context(0, {"host_upload": 1}) as c:
        nc, nr = c.gc_color_graph_host(rp, ci, 1, 100, 42, color)
    ob, oc, onr, onc = oracle.jp_adg(g, 1, 100, 42)
    assert (nc, nr) == (onc, onr) and np.array_equal(color, oc)
