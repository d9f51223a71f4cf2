"""Readers for the hand-worked fixtures under tests/golden/ and small graph
builders used by several test files (no colouring arithmetic here)."""
from __future__ import annotations

import itertools
import os

import numpy as np

import graphgen as gg

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_cases(fname: str):
    """Parse 'key: value' blocks; a new block starts at each 'name:' key
    (or the file is one block).  Comment lines start with '#'."""
    cases, cur = [], {}
    with open(os.path.join(GOLDEN, fname)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(":", 1)
            k, v = k.strip(), v.strip()
            if k == "name" and cur:
                cases.append(cur)
                cur = {}
            cur[k] = v
    if cur:
        cases.append(cur)
    return cases


def case_graph(case) -> gg.Graph:
    n = int(case["n"])
    edges = [tuple(map(int, e.split("-"))) for e in case["edges"].split()]
    return gg.from_edges(n, edges, case.get("name", "golden"))


def ints(s: str) -> np.ndarray:
    return np.array([int(x) for x in s.split()], dtype=np.int64)


# ---- named small graphs -------------------------------------------------------

def complete(n):
    return gg.from_edges(n, list(itertools.combinations(range(n), 2)), f"K{n}")


def path(n):
    return gg.from_edges(n, [(i, i + 1) for i in range(n - 1)], f"P{n}")


def cycle(n):
    return gg.from_edges(n, [(i, (i + 1) % n) for i in range(n)], f"C{n}")


def star(k):
    return gg.from_edges(k + 1, [(0, i) for i in range(1, k + 1)], f"star{k}")


def complete_bipartite(a, b):
    return gg.from_edges(a + b, [(i, a + j) for i in range(a) for j in range(b)], f"K{a},{b}")


def empty(n):
    return gg.from_edges(n, [], f"empty{n}")


def petersen():
    outer = [(i, (i + 1) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    return gg.from_edges(10, outer + spokes + inner, "petersen")


def wheel(rim):
    edges = [(0, i) for i in range(1, rim + 1)] + [(i, i % rim + 1) for i in range(1, rim + 1)]
    return gg.from_edges(rim + 1, edges, f"W{rim}")


def random_small(n, p, seed):
    rng = np.random.default_rng(seed)
    edges = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < p]
    return gg.from_edges(n, edges, f"rand{n}_{seed}")


def neighbours(g, v):
    return g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]]
