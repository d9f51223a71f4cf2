"""CPU oracle for ADG and JP-ADG (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It wraps ``oracle.c`` (plain single-threaded C,
exact integer arithmetic) through ctypes and shares no code with the CUDA
library.  ``build()`` compiles ``liboracle.so`` next to the source with gcc.

Functions (each cites the passage of the paper it follows in ``oracle.c``):
  adg(g, p, q)                   Algorithm 1, fresh degree sums every round
  adg_naive(g, p, q)             Algorithm 1 with D recomputed from scratch
  adg_m(g), adg_m_naive(g)       ADG-M (median; R = ceil(|U|/2) smallest (D, id))
  adg_o(g, p, q)                 ADG-O (Algorithm 6: R sorted by D, total order rho)
  jp_adg_o(g, p, q)              JP with rho_ADG-O
  tiebreak(seed, v)              SplitMix64-based random tie-break rho_R
  priority(batch, seed)          (batch << 32) | tiebreak, ties by vertex id
  priority_kind(g, kind, seed)   JP-R / FF / LF / LLF / SL keys (kinds 0..4)
  smallest_last(g)               SL order: minimum (current degree, id) first
  greedy(g, order)               Greedy colouring in a given order
  jp_color(g, priority)          JP (Algorithm 3) == Greedy by decreasing key
  jp_adg(g, p, q, seed)          ADG then JP with <rho_ADG, rho_R>
  dec_itr(g, batch, rounds, seed)   DEC-ADG-ITR colouring of given partitions
  dec_adg_itr(g, p, q, seed)     ADG then DEC-ADG-ITR
  pred_count(g, priority)        |pred(v)| in the DAG G_rho
  jp_depth(g, priority)          longest path of G_rho (JP's step count)
  degeneracy(g)                  exact d and smallest-last order (Matula-Beck)
  chromatic_number(g)            exhaustive, n <= 16
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import platform
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so unless a stamp beside it holds the hash of the
    source, the command and the host architecture."""
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC]
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
        vp, i64, u64, u32, i32 = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64,
                                  ctypes.c_uint32, ctypes.c_int32)
        lib.oracle_splitmix64_output.restype = u64
        lib.oracle_splitmix64_output.argtypes = [u64, u64]
        lib.oracle_tiebreak.restype = u32
        lib.oracle_tiebreak.argtypes = [u64, i64]
        lib.oracle_adg.restype = ctypes.c_int
        lib.oracle_adg.argtypes = [i64, vp, vp, u32, u32, vp, vp, vp, vp, vp, vp, i64]
        lib.oracle_adg_naive.restype = ctypes.c_int
        lib.oracle_adg_naive.argtypes = [i64, vp, vp, u32, u32, vp, vp]
        lib.oracle_greedy.restype = ctypes.c_int
        lib.oracle_greedy.argtypes = [i64, vp, vp, vp, vp, vp]
        lib.oracle_priority.restype = None
        lib.oracle_priority.argtypes = [i64, vp, u64, vp]
        for fn in ("oracle_adg_m", "oracle_adg_m_naive"):
            getattr(lib, fn).restype = ctypes.c_int
            getattr(lib, fn).argtypes = [i64, vp, vp, vp, ctypes.POINTER(ctypes.c_int32)]
        lib.oracle_priority_kind.restype = ctypes.c_int
        lib.oracle_priority_kind.argtypes = [i64, vp, ctypes.c_int, u64, vp]
        lib.oracle_jp_color.restype = ctypes.c_int
        lib.oracle_jp_color.argtypes = [i64, vp, vp, vp, vp, vp]
        lib.oracle_jp_adg.restype = ctypes.c_int
        lib.oracle_jp_adg.argtypes = [i64, vp, vp, u32, u32, u64, vp, vp, vp, vp]
        lib.oracle_pred_count.restype = None
        lib.oracle_pred_count.argtypes = [i64, vp, vp, vp, vp]
        lib.oracle_smallest_last.restype = ctypes.c_int
        lib.oracle_smallest_last.argtypes = [i64, vp, vp, vp]
        lib.oracle_jp_depth.restype = i64
        lib.oracle_jp_depth.argtypes = [i64, vp, vp, vp, vp]
        lib.oracle_degeneracy.restype = i64
        lib.oracle_degeneracy.argtypes = [i64, vp, vp, vp]
        lib.oracle_adg_o.restype = ctypes.c_int
        lib.oracle_adg_o.argtypes = [i64, vp, vp, u32, u32, vp, vp, vp, ctypes.POINTER(ctypes.c_int32)]
        lib.oracle_dec_adg_itr.restype = ctypes.c_int
        lib.oracle_dec_adg_itr.argtypes = [i64, vp, vp, vp, i32, u64, vp, vp, vp, vp]
        lib.oracle_chromatic_number.restype = i32
        lib.oracle_chromatic_number.argtypes = [i64, vp, vp]
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data if a.size else None


def _csr(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(g.col_idx, dtype=np.int32)
    return rp.shape[0] - 1, rp, ci


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def splitmix64_output(seed: int, k: int) -> int:
    return int(_load().oracle_splitmix64_output(seed, k))


def tiebreak(seed: int, v: int) -> int:
    return int(_load().oracle_tiebreak(seed, v))


def adg(g, eps_p: int, eps_q: int, log: bool = False):
    """Returns (batch int32[n], num_rounds) or, with log=True,
    (batch, num_rounds, dict of per-round |U|, |R|, Sigma, T arrays)."""
    n, rp, ci = _csr(g)
    batch = np.zeros(n, dtype=np.int32)
    rounds = ctypes.c_int32(0)
    cap = 1 << 16 if log else 0
    logs = {k: np.zeros(max(cap, 1), dtype=np.int64) for k in ("U", "R", "sigma", "T")}
    lib = _load()
    _check(lib.oracle_adg(n, _p(rp), _p(ci), eps_p, eps_q, _p(batch), ctypes.byref(rounds),
                          logs["U"].ctypes.data if log else None,
                          logs["R"].ctypes.data if log else None,
                          logs["sigma"].ctypes.data if log else None,
                          logs["T"].ctypes.data if log else None, cap), "adg")
    if not log:
        return batch, rounds.value
    r = min(rounds.value, cap)
    return batch, rounds.value, {k: v[:r].copy() for k, v in logs.items()}


def adg_naive(g, eps_p: int, eps_q: int):
    n, rp, ci = _csr(g)
    batch = np.zeros(n, dtype=np.int32)
    rounds = ctypes.c_int32(0)
    _check(_load().oracle_adg_naive(n, _p(rp), _p(ci), eps_p, eps_q, _p(batch),
                                    ctypes.byref(rounds)), "adg_naive")
    return batch, rounds.value


def adg_m(g):
    n, rp, ci = _csr(g)
    batch = np.zeros(n, dtype=np.int32)
    rounds = ctypes.c_int32(0)
    _check(_load().oracle_adg_m(n, _p(rp), _p(ci), _p(batch), ctypes.byref(rounds)), "adg_m")
    return batch, rounds.value


def adg_m_naive(g):
    n, rp, ci = _csr(g)
    batch = np.zeros(n, dtype=np.int32)
    rounds = ctypes.c_int32(0)
    _check(_load().oracle_adg_m_naive(n, _p(rp), _p(ci), _p(batch), ctypes.byref(rounds)), "adg_m_naive")
    return batch, rounds.value


def adg_o(g, eps_p: int, eps_q: int):
    """ADG-O (Algorithm 6).  Returns (batch, rho int64[n], rank int64[n],
    num_rounds)."""
    n, rp, ci = _csr(g)
    batch = np.zeros(n, dtype=np.int32)
    rho = np.zeros(n, dtype=np.int64)
    rank = np.zeros(n, dtype=np.int64)
    rounds = ctypes.c_int32(0)
    _check(_load().oracle_adg_o(n, _p(rp), _p(ci), eps_p, eps_q, _p(batch), _p(rho), _p(rank),
                                ctypes.byref(rounds)), "adg_o")
    return batch, rho, rank, rounds.value


def jp_adg_o(g, eps_p: int, eps_q: int):
    """JP-ADG-O: JP with priority rho_ADG-O (a total order, no random
    tie-break).  Returns (batch, rho, color, num_rounds, num_colors)."""
    batch, rho, _, rounds = adg_o(g, eps_p, eps_q)
    color, nc = jp_color(g, rho.astype(np.uint64))
    return batch, rho, color, rounds, nc


def jp_adg_m(g, seed: int):
    """JP-ADG-M: ADG-M, then JP with <rho_ADG-M, rho_R>.  Returns (batch,
    color, num_rounds, num_colors)."""
    batch, rounds = adg_m(g)
    color, nc = jp_color(g, priority(batch, seed))
    return batch, color, rounds, nc


def priority(batch: np.ndarray, seed: int) -> np.ndarray:
    b = np.ascontiguousarray(batch, dtype=np.int32)
    key = np.zeros(b.shape[0], dtype=np.uint64)
    _load().oracle_priority(b.shape[0], _p(b), seed, _p(key))
    return key


PRIO_R, PRIO_FF, PRIO_LF, PRIO_LLF = 0, 1, 2, 3


def priority_kind(g, kind: int, seed: int) -> np.ndarray:
    """Keys of the JP variants: 0 JP-R, 1 JP-FF, 2 JP-LF, 3 JP-LLF (from the
    degrees and the seeded hash), 4 JP-SL (the smallest-last removal index:
    vertices removed later are coloured first; no seed)."""
    n, rp, _ = _csr(g)
    key = np.zeros(n, dtype=np.uint64)
    if kind == 4:
        key[smallest_last(g)] = np.arange(n, dtype=np.uint64)
        return key
    _check(_load().oracle_priority_kind(n, _p(rp), kind, seed, _p(key)), "priority_kind")
    return key


def smallest_last(g) -> np.ndarray:
    """int64[n]: the vertices in smallest-last removal order (minimum
    current degree first, then minimum id)."""
    n, rp, ci = _csr(g)
    order = np.zeros(n, dtype=np.int64)
    _check(_load().oracle_smallest_last(n, _p(rp), _p(ci), _p(order)), "smallest_last")
    return order


def greedy(g, order: np.ndarray):
    n, rp, ci = _csr(g)
    o = np.ascontiguousarray(order, dtype=np.int64)
    assert o.shape[0] == n
    color = np.zeros(n, dtype=np.int32)
    nc = ctypes.c_int32(0)
    _check(_load().oracle_greedy(n, _p(rp), _p(ci), _p(o), _p(color), ctypes.byref(nc)), "greedy")
    return color, nc.value


def jp_color(g, prio: np.ndarray):
    n, rp, ci = _csr(g)
    pr = np.ascontiguousarray(prio, dtype=np.uint64)
    color = np.zeros(n, dtype=np.int32)
    nc = ctypes.c_int32(0)
    _check(_load().oracle_jp_color(n, _p(rp), _p(ci), _p(pr), _p(color), ctypes.byref(nc)),
           "jp_color")
    return color, nc.value


def jp_adg(g, eps_p: int, eps_q: int, seed: int):
    """Returns (batch, color, num_rounds, num_colors)."""
    n, rp, ci = _csr(g)
    batch = np.zeros(n, dtype=np.int32)
    color = np.zeros(n, dtype=np.int32)
    nr, nc = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(_load().oracle_jp_adg(n, _p(rp), _p(ci), eps_p, eps_q, seed, _p(batch), _p(color),
                                 ctypes.byref(nr), ctypes.byref(nc)), "jp_adg")
    return batch, color, nr.value, nc.value


def dec_itr(g, batch: np.ndarray, rounds: int, seed: int):
    """DEC-ADG-ITR colouring of the partitions R(l) = {v : batch[v] = l}.
    Returns (color, num_colors, iterations, fixed_iter)."""
    n, rp, ci = _csr(g)
    b = np.ascontiguousarray(batch, dtype=np.int32)
    color = np.zeros(n, dtype=np.int32)
    fixed = np.zeros(n, dtype=np.int32)
    nc = ctypes.c_int32(0)
    iters = ctypes.c_int64(0)
    _check(_load().oracle_dec_adg_itr(n, _p(rp), _p(ci), _p(b), rounds, seed, _p(color), _p(fixed),
                                      ctypes.byref(nc), ctypes.byref(iters)), "dec_adg_itr")
    return color, nc.value, iters.value, fixed


def dec_adg_itr(g, eps_p: int, eps_q: int, seed: int):
    """ADG, then DEC-ADG-ITR.  Returns (batch, color, num_rounds, num_colors,
    iterations, fixed_iter)."""
    batch, rounds = adg(g, eps_p, eps_q)
    color, nc, iters, fixed = dec_itr(g, batch, rounds, seed)
    return batch, color, rounds, nc, iters, fixed


def pred_count(g, prio: np.ndarray) -> np.ndarray:
    n, rp, ci = _csr(g)
    pr = np.ascontiguousarray(prio, dtype=np.uint64)
    cnt = np.zeros(n, dtype=np.int32)
    _load().oracle_pred_count(n, _p(rp), _p(ci), _p(pr), _p(cnt))
    return cnt


def jp_depth(g, prio: np.ndarray, per_vertex: bool = False):
    """Longest path (in vertices) of G_rho; with per_vertex, also depth[v],
    the length of the longest path of G_rho that ends at v."""
    n, rp, ci = _csr(g)
    pr = np.ascontiguousarray(prio, dtype=np.uint64)
    depth = np.zeros(n, dtype=np.int32)
    best = int(_load().oracle_jp_depth(n, _p(rp), _p(ci), _p(pr), _p(depth)))
    return (best, depth) if per_vertex else best


def degeneracy(g):
    """Returns (d, smallest-last removal order int64[n])."""
    n, rp, ci = _csr(g)
    order = np.zeros(n, dtype=np.int64)
    d = _load().oracle_degeneracy(n, _p(rp), _p(ci), _p(order))
    return int(d), order


def chromatic_number(g) -> int:
    n, rp, ci = _csr(g)
    if n > 16:
        raise ValueError("chromatic_number is exhaustive; n <= 16 only")
    return int(_load().oracle_chromatic_number(n, _p(rp), _p(ci)))
