"""Seeded synthetic graph inputs (CSR), shared by the oracle tests, the CUDA
parity tests and the benchmark.

This module makes inputs only; it contains none of the colouring method's
arithmetic.  The generators live in ``graphgen.cpp`` (compiled on first use
into ``libgraphgen.so`` beside it) and every one of them is a pure function of
its parameters and seed, so the CPU and GPU sides colour the same graph.

Workload recipes stand in for the paper's inputs (Section 6): the paper used
real SNAP/KONECT/DIMACS/WebGraph graphs and Kronecker power-law graphs, which
are not available here, so R-MAT (a 2x2 stochastic Kronecker model), Erdos-
Renyi, Barabasi-Albert and regular grids of the same scale are generated.
"""
from __future__ import annotations

import ctypes
import hashlib
import math
import os
import platform
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.cpp")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lib = None

RMAT_ABC = (0.57, 0.19, 0.19)  # d = 0.05


def build(force: bool = False) -> str:
    """Compile libgraphgen.so next to the source (host C++ only) unless a
    stamp beside it holds the hash of the source, the command and the host
    architecture."""
    cmd = ["g++", "-O3", "-std=c++17", "-shared", "-fPIC", "-pthread", _SRC]
    h = hashlib.sha256(platform.machine().encode() + "\0".join(cmd).encode())
    with open(_SRC, "rb") as f:
        h.update(f.read())
    digest = h.hexdigest()
    stamp = _LIB + ".stamp"
    fresh = os.path.exists(_LIB) and os.path.exists(stamp) and open(stamp).read().strip() == digest
    if force or not fresh:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(cmd + ["-o", tmp])
        os.replace(tmp, _LIB)
        with open(stamp, "w") as f:
            f.write(digest + "\n")
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp, i64, u64, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        lib.gg_n.restype = i64
        lib.gg_n.argtypes = [vp]
        lib.gg_nnz.restype = i64
        lib.gg_nnz.argtypes = [vp]
        lib.gg_export.restype = ctypes.c_int
        lib.gg_export.argtypes = [vp, vp, vp]
        lib.gg_free.restype = None
        lib.gg_free.argtypes = [vp]
        lib.gg_from_edges.restype = vp
        lib.gg_from_edges.argtypes = [i64, i64, vp, vp]
        lib.gg_er.restype = vp
        lib.gg_er.argtypes = [i64, i64, u64]
        lib.gg_rmat.restype = vp
        lib.gg_rmat.argtypes = [ctypes.c_int, i64, dbl, dbl, dbl, u64]
        lib.gg_ba.restype = vp
        lib.gg_ba.argtypes = [i64, i64, u64]
        lib.gg_grid.restype = vp
        lib.gg_grid.argtypes = [i64, i64, i64]
        lib.gg_permute.restype = vp
        lib.gg_permute.argtypes = [vp, u64]
        lib.gg_draw.restype = u64
        lib.gg_draw.argtypes = [u64, u64, u64]
        lib.gg_batch_recipe.restype = None
        lib.gg_batch_recipe.argtypes = [i64, i64, i64, u64, vp, vp]
        lib.gg_batch.restype = vp
        lib.gg_batch.argtypes = [i64, i64, i64, u64, vp]
        _lib = lib
    return _lib


@dataclass
class Graph:
    """Undirected simple graph in CSR: int64 row_ptr[n+1], int32 col_idx[nnz]."""
    row_ptr: np.ndarray
    col_idx: np.ndarray
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    @property
    def m(self) -> int:
        return self.nnz // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)


def _take(handle, name: str, pinned: bool = False) -> Graph:
    lib = _load()
    if not handle:
        raise ValueError(f"graph generator failed for {name}")
    try:
        n, nnz = lib.gg_n(handle), lib.gg_nnz(handle)
        if pinned:
            import torch
            rp_t = torch.empty(n + 1, dtype=torch.int64, pin_memory=True)
            ci_t = torch.empty(nnz, dtype=torch.int32, pin_memory=True)
            rp, ci = rp_t.numpy(), ci_t.numpy()
        else:
            rp = np.empty(n + 1, dtype=np.int64)
            ci = np.empty(nnz, dtype=np.int32)
        lib.gg_export(handle, rp.ctypes.data, ci.ctypes.data if nnz else None)
    finally:
        lib.gg_free(handle)
    return Graph(rp, ci, name)


def from_edges(n: int, edges, name: str = "edges") -> Graph:
    """Canonical CSR from an undirected edge list (loops/duplicates dropped)."""
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    if e.size and (e.min() < 0 or e.max() >= n):
        raise ValueError("edge endpoint out of range")
    src = np.ascontiguousarray(e[:, 0].astype(np.uint32))
    dst = np.ascontiguousarray(e[:, 1].astype(np.uint32))
    h = _load().gg_from_edges(n, len(src), src.ctypes.data if len(src) else None,
                              dst.ctypes.data if len(dst) else None)
    return _take(h, name)


def erdos_renyi(n: int, m: int, seed: int = 1, pinned: bool = False) -> Graph:
    return _take(_load().gg_er(n, m, seed), f"er_n{n}_m{m}", pinned)


def rmat(scale: int, edge_factor: int = 16, abc=RMAT_ABC, seed: int = 1,
         pinned: bool = False) -> Graph:
    a, b, c = abc
    return _take(_load().gg_rmat(scale, edge_factor, a, b, c, seed),
                 f"rmat{scale}_ef{edge_factor}", pinned)


def barabasi_albert(n: int, m: int, seed: int = 1, pinned: bool = False) -> Graph:
    return _take(_load().gg_ba(n, m, seed), f"ba_n{n}_m{m}", pinned)


def grid(k1: int, k2: int = 1, k3: int = 1, perm_seed: int | None = None,
         pinned: bool = False) -> Graph:
    lib = _load()
    h = lib.gg_grid(k1, k2, k3)
    name = f"grid{k1}x{k2}x{k3}"
    if perm_seed is not None and h:
        p = lib.gg_permute(h, perm_seed)
        lib.gg_free(h)
        h = p
        name += f"_perm{perm_seed}"
    return _take(h, name, pinned)


def draw(seed: int, stream: int, k: int) -> int:
    """Uniform 64-bit value k of the generator's stream (for recipes)."""
    return int(_load().gg_draw(seed, stream, k))


def batch_recipe(num_graphs: int, n_lo: int = 100, n_hi: int = 200_000, seed: int = 42):
    """Per-graph (family, n) for the batched workload: n log-uniform in
    [n_lo, n_hi]; family uniform over Erdos-Renyi (average degree 8),
    Barabasi-Albert (m=4) and 2D grids (k = ceil(sqrt(n)))."""
    fam = np.zeros(num_graphs, dtype=np.int32)
    nv = np.zeros(num_graphs, dtype=np.int64)
    _load().gg_batch_recipe(num_graphs, n_lo, n_hi, seed, fam.ctypes.data, nv.ctypes.data)
    names = ("er", "ba", "grid")
    return [(names[f], int(n)) for f, n in zip(fam, nv)]


def batch(num_graphs: int, n_lo: int = 100, n_hi: int = 200_000, seed: int = 42, pinned: bool = False):
    """The batched workload, generated in parallel and packed as the disjoint
    union: returns (Graph of the union, graph_off int64[num_graphs+1]).  Graph
    g equals make_batch_graph(*batch_recipe(...)[g], seed + g)."""
    off = np.zeros(num_graphs + 1, dtype=np.int64)
    h = _load().gg_batch(num_graphs, n_lo, n_hi, seed, off.ctypes.data)
    return _take(h, f"batch{num_graphs}", pinned), off


def make_batch_graph(fam: str, n: int, seed: int) -> Graph:
    if fam == "er":
        return erdos_renyi(n, 4 * n, seed)
    if fam == "ba":
        return barabasi_albert(n, 4, seed)
    if fam == "grid":
        k = int(math.ceil(math.sqrt(n)))
        return grid(k, k)
    raise ValueError(fam)
