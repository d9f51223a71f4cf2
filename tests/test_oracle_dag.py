"""Pins of the oracle's DAG helpers: pred_count (|pred(v)| in G_rho, the
initial counters of Algorithm 3, Section 4.1) and jp_depth (the longest path
of G_rho, i.e. the number of dependency steps JP needs, which the depth
bound of Section 4.1 is about).

Neither helper is compared with a retyped copy of itself.  They are pinned by
closed forms on graphs whose DAG is known by hand, by a synchronous execution
of Algorithm 3 (every vertex whose predecessors are all coloured is coloured
in the same step, so vertex v is coloured in step depth[v]), and by brute
force over every path of G_rho on tiny graphs.  A dropped +1, a missing
equal-key id rule or a reversed edge direction each fail one of these.
"""
from __future__ import annotations

import itertools

import numpy as np
import pytest

import graphgen as gg
import oracle
from _fixtures import complete, empty, neighbours, path, random_small, star

FF_TOP = 0xFFFFFFFF  # JP-FF key of vertex 0: 2^32 - 1 - v


def ff_keys(n):
    return np.array([FF_TOP - v for v in range(n)], dtype=np.uint64)


# ------------------------------------------------------------------ pred_count

def test_pred_count_clique_is_rank_from_the_top():
    rng = np.random.default_rng(3)
    n = 9
    prio = rng.permutation(n).astype(np.uint64) * 7 + 1
    cnt = oracle.pred_count(complete(n), prio)
    # on K_n every higher-priority vertex is a predecessor
    ranks = np.argsort(np.argsort(-prio.astype(np.int64)))
    assert np.array_equal(cnt, ranks)


def test_pred_count_equal_keys_fall_back_to_larger_id():
    n = 7
    cnt = oracle.pred_count(complete(n), np.zeros(n, dtype=np.uint64))
    assert cnt.tolist() == [n - 1 - v for v in range(n)]


def test_pred_count_star_and_path():
    k = 6
    hub_first = np.array([10] + [1] * k, dtype=np.uint64)
    assert oracle.pred_count(star(k), hub_first).tolist() == [0] + [1] * k
    hub_last = np.array([0] + [5] * k, dtype=np.uint64)
    assert oracle.pred_count(star(k), hub_last).tolist() == [k] + [0] * k
    n = 8
    assert oracle.pred_count(path(n), ff_keys(n)).tolist() == [0] + [1] * (n - 1)


# -------------------------------------------------------------------- jp_depth

def test_depth_empty_and_zero_vertices():
    assert oracle.jp_depth(empty(5), np.arange(5, dtype=np.uint64)) == 1
    assert oracle.jp_depth(empty(0), np.zeros(0, dtype=np.uint64)) == 0


@pytest.mark.parametrize("n", [1, 2, 5, 12])
def test_depth_clique_is_n_for_any_priority(n):
    g = complete(n)
    rng = np.random.default_rng(n)
    for prio in (rng.integers(0, 3, size=n).astype(np.uint64), np.zeros(n, dtype=np.uint64),
                 rng.permutation(n).astype(np.uint64)):
        best, depth = oracle.jp_depth(g, prio, per_vertex=True)
        assert best == n
        assert sorted(depth.tolist()) == list(range(1, n + 1))


def test_depth_star_is_two():
    k = 9
    for prio in (np.array([10] + [1] * k, dtype=np.uint64), np.array([0] + [4] * k, dtype=np.uint64)):
        assert oracle.jp_depth(star(k), prio) == 2


@pytest.mark.parametrize("n", [2, 7, 30])
def test_depth_path(n):
    # first-fit order: vertex i waits on vertex i - 1
    best, depth = oracle.jp_depth(path(n), ff_keys(n), per_vertex=True)
    assert best == n and depth.tolist() == list(range(1, n + 1))
    # all keys equal: the larger id goes first, so the chain runs from n-1 down
    best, depth = oracle.jp_depth(path(n), np.zeros(n, dtype=np.uint64), per_vertex=True)
    assert best == n and depth.tolist() == list(range(n, 0, -1))
    # alternating high/low keys: two steps
    alt = np.array([1 if i % 2 == 0 else 0 for i in range(n)], dtype=np.uint64)
    assert oracle.jp_depth(path(n), alt) == 2


def _synchronous_jp_steps(g, prio):
    """Algorithm 3 with every ready vertex coloured in the same step: the step
    number at which each vertex is coloured."""
    n = g.n
    key = [(int(prio[v]), v) for v in range(n)]
    pred = [{int(w) for w in neighbours(g, v) if key[w] > key[v]} for v in range(n)]
    step = [0] * n
    left = set(range(n))
    s = 0
    while left:
        s += 1
        ready = [v for v in left if all(step[w] for w in pred[v])]
        assert ready, "G_rho has a cycle"
        for v in ready:
            step[v] = s
        left.difference_update(ready)
    return np.array(step, dtype=np.int32)


@pytest.mark.parametrize("seed", range(5))
def test_depth_equals_synchronous_jp_steps(seed):
    rng = np.random.default_rng(seed)
    for g in (random_small(30, 0.25, seed), gg.erdos_renyi(200, 900, seed + 1),
              gg.barabasi_albert(200, 3, seed + 1)):
        for prio in (oracle.priority(oracle.adg(g, 1, 100)[0], seed),
                     rng.integers(0, 3, size=g.n).astype(np.uint64)):
            best, depth = oracle.jp_depth(g, prio, per_vertex=True)
            steps = _synchronous_jp_steps(g, prio)
            assert np.array_equal(depth, steps)
            assert best == (int(steps.max()) if g.n else 0)


def _longest_path_brute_force(g, prio):
    """Every vertex sequence v1, v2, ... with consecutive vertices adjacent
    and strictly decreasing (key, id): the longest one's length."""
    n = g.n
    key = [(int(prio[v]), v) for v in range(n)]
    adj = [set(int(w) for w in neighbours(g, v)) for v in range(n)]
    best = 1 if n else 0
    for r in range(2, n + 1):
        found = False
        for combo in itertools.combinations(range(n), r):
            seq = sorted(combo, key=lambda v: key[v], reverse=True)
            if all(seq[i + 1] in adj[seq[i]] for i in range(r - 1)):
                found = True
                break
        if not found:
            break
        best = r
    return best


@pytest.mark.parametrize("seed", range(8))
def test_depth_brute_force_tiny(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(3, 9))
    g = random_small(n, 0.45, seed)
    for prio in (rng.integers(0, 4, size=n).astype(np.uint64), rng.permutation(n).astype(np.uint64)):
        assert oracle.jp_depth(g, prio) == _longest_path_brute_force(g, prio)


# ----------------------------------------------------------- smallest-last order

def _sl_naive(g):
    """Smallest-last by recomputing every remaining degree from scratch at
    each step and taking the minimum (degree, id)."""
    left = set(range(g.n))
    nb = [set(int(w) for w in neighbours(g, v)) for v in range(g.n)]
    out = []
    while left:
        v = min(left, key=lambda u: (len(nb[u] & left), u))
        out.append(v)
        left.remove(v)
    return out


def test_sl_closed_forms():
    from _fixtures import complete_bipartite, cycle
    assert oracle.smallest_last(path(7)).tolist() == list(range(7))          # an end, then its neighbour...
    assert oracle.smallest_last(cycle(6)).tolist() == list(range(6))         # vertex 0, then the path 1..5
    assert oracle.smallest_last(complete(5)).tolist() == list(range(5))      # all degrees equal: by id
    assert oracle.smallest_last(star(5)).tolist() == [1, 2, 3, 4, 0, 5]      # leaves until the centre ties at 1
    assert oracle.smallest_last(empty(4)).tolist() == [0, 1, 2, 3]
    # K_{2,5}: the degree-2 side goes until the other side is down to 2
    assert oracle.smallest_last(complete_bipartite(2, 5)).tolist() == [2, 3, 4, 0, 5, 1, 6]


@pytest.mark.parametrize("seed", range(10))
def test_sl_matches_naive_peeling(seed):
    rng = np.random.default_rng(seed)
    g = random_small(int(rng.integers(5, 40)), float(rng.uniform(0.05, 0.5)), seed)
    assert oracle.smallest_last(g).tolist() == _sl_naive(g)


@pytest.mark.parametrize("g", [gg.rmat(12, 8, seed=1), gg.barabasi_albert(2000, 5, 2), gg.erdos_renyi(3000, 12000, 3),
                               gg.grid(30, 40)], ids=lambda g: g.name)
def test_sl_degeneracy_and_colour_bound(g):
    # the largest degree at removal in a smallest-last order is the
    # degeneracy d, and Greedy in reverse removal order (JP-SL) uses at most
    # d + 1 colours
    order = oracle.smallest_last(g)
    assert sorted(order.tolist()) == list(range(g.n))
    pos = np.empty(g.n, dtype=np.int64)
    pos[order] = np.arange(g.n)
    src = np.repeat(np.arange(g.n), g.degrees())
    later = np.bincount(src[pos[g.col_idx] > pos[src]], minlength=g.n)  # degree at removal
    d, _ = oracle.degeneracy(g)
    assert later.max() == d
    key = oracle.priority_kind(g, 4, 0)
    assert np.array_equal(key[order], np.arange(g.n, dtype=np.uint64))
    color, nc = oracle.jp_color(g, key)
    assert nc <= d + 1
    assert np.all(color[src] != color[g.col_idx])
