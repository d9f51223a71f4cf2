"""Python binding of the C ABI in include/gcolor.h (argument marshalling only).

Every function here forwards to the same-named entry point of libgcolor.so
through ctypes.  Device buffers are PyTorch CUDA tensors (their data
pointers are passed; PyTorch is used for device memory and streams only) and
the stream defaults to the caller's current PyTorch stream.  All computation
happens in the library's CUDA kernels; there is no fallback: if the library
cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgcolor.so")

GC_OK, GC_ERR_INVALID_ARG, GC_ERR_INVALID_GRAPH, GC_ERR_OOM = 0, 1, 2, 3
GC_ERR_CUDA, GC_ERR_TIMEOUT, GC_ERR_OVERFLOW = 4, 5, 6

# Every symbol declared in include/gcolor.h.
EXPORTS = ("gc_status_str", "gc_last_error", "gc_options_init", "gc_create", "gc_get_options", "gc_set_options", "gc_autotune",
           "gc_autotune_batch", "gc_destroy", "gc_get_stats", "gc_set_timing",
           "gc_validate_csr", "gc_adg_partition", "gc_make_priority", "gc_jp_color",
           "gc_color_graph", "gc_color_graph_host", "gc_adg_partition_noalloc", "gc_color_batch",
           "gc_color_batch_list", "gc_make_priority_kind", "gc_adg_m_partition", "gc_color_graph_m",
           "gc_dec_itr_color", "gc_color_graph_dec_itr", "gc_adg_o_order", "gc_color_graph_o")

# priority kinds of gc_make_priority_kind
GC_PRIO_R, GC_PRIO_FF, GC_PRIO_LF, GC_PRIO_LLF, GC_PRIO_SL = 0, 1, 2, 3, 4
# ADG UPDATE directions (gc_options.update_mode)
GC_UPDATE_AUTO, GC_UPDATE_PUSH, GC_UPDATE_PULL = 0, 1, 2
# gc_color_batch paths (gc_options.batch_mode, gc_stats.batch_path)
GC_BATCH_AUTO, GC_BATCH_SEGMENTED, GC_BATCH_PERSISTENT = 0, 1, 2


class GcError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        where = load().gc_last_error().decode() if status == GC_ERR_CUDA else ""
        super().__init__(f"{what}: {status_str(status)}" + (f" at {where}" if where else ""))


class gc_csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p)]


class gc_batch_csr(ctypes.Structure):
    _fields_ = [("num_graphs", ctypes.c_int64), ("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p), ("graph_off", ctypes.c_void_p)]


class gc_job(ctypes.Structure):
    _fields_ = [("eps_p", ctypes.c_uint32), ("eps_q", ctypes.c_uint32), ("seed", ctypes.c_uint64)]


class gc_options(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("core_target", ctypes.c_int32),
                ("core_cluster", ctypes.c_int32), ("core_warps", ctypes.c_int32), ("dec_tail", ctypes.c_int32),
                ("update_mode", ctypes.c_int32), ("pull_percent", ctypes.c_int32),
                ("bulk_blocks_per_sm", ctypes.c_int32), ("wait_limit_ms", ctypes.c_uint32),
                ("jp_state16", ctypes.c_int32), ("batch_mode", ctypes.c_int32), ("update_hubs", ctypes.c_int32),
                ("host_upload", ctypes.c_int32), ("round_graph", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "struct_size"}


def make_options(**fields) -> gc_options:
    """gc_options with the library's defaults, then the given fields."""
    o = gc_options()
    _check(load().gc_options_init(ctypes.byref(o)), "gc_options_init")
    for k, v in fields.items():
        if k not in dict(gc_options._fields_) or k == "struct_size":
            raise KeyError(f"gc_options has no field {k!r}")
        setattr(o, k, int(v))
    return o


class gc_stats(ctypes.Structure):
    _fields_ = [("adg_rounds", ctypes.c_int32), ("num_colors", ctypes.c_int32),
                ("sum_U", ctypes.c_int64), ("sum_decrements", ctypes.c_int64),
                ("jp_spins", ctypes.c_int64), ("ms_adg", ctypes.c_float), ("ms_jp", ctypes.c_float),
                ("ms_jp_color", ctypes.c_float), ("launches", ctypes.c_int32),
                ("ms_adg_update", ctypes.c_float), ("ms_core_solve", ctypes.c_float),
                ("ms_core_preds", ctypes.c_float), ("bulk_launches", ctypes.c_int32),
                ("core_vertices", ctypes.c_int64), ("core_preds", ctypes.c_int64),
                ("core_degree_sum", ctypes.c_int64), ("core_ctas", ctypes.c_int32),
                ("sim_iterations", ctypes.c_int64), ("dec_internal_edges", ctypes.c_int64),
                ("ms_dec_extract", ctypes.c_float), ("ms_dec_iterate", ctypes.c_float),
                ("dec_tail_partitions", ctypes.c_int64), ("adg_pull_rounds", ctypes.c_int32),
                ("jp_state_bits", ctypes.c_int32), ("batch_path", ctypes.c_int32)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libgcolor.so (build it first with __graft_entry__.build() or
    paper_2008_11321_gb300._build.build()).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libgcolor.so not built at {path}; run paper_2008_11321_gb300._build.build()")
    lib = ctypes.CDLL(path)
    vp, i32, i64, u32, u64 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                              ctypes.c_uint64)
    P = ctypes.POINTER
    lib.gc_status_str.restype = ctypes.c_char_p
    lib.gc_status_str.argtypes = [ctypes.c_int]
    lib.gc_last_error.restype = ctypes.c_char_p
    lib.gc_last_error.argtypes = []
    lib.gc_options_init.restype = ctypes.c_int
    lib.gc_options_init.argtypes = [P(gc_options)]
    lib.gc_create.restype = ctypes.c_int
    lib.gc_create.argtypes = [P(vp), ctypes.c_int, P(gc_options)]
    lib.gc_get_options.restype = ctypes.c_int
    lib.gc_get_options.argtypes = [vp, P(gc_options)]
    lib.gc_set_options.restype = ctypes.c_int
    lib.gc_set_options.argtypes = [vp, P(gc_options)]
    f32 = ctypes.c_float
    lib.gc_autotune.restype = ctypes.c_int
    lib.gc_autotune.argtypes = [vp, P(gc_csr), u32, u32, u64, i32, f32, P(gc_options), P(f32), P(f32), vp]
    lib.gc_autotune_batch.restype = ctypes.c_int
    lib.gc_autotune_batch.argtypes = [vp, P(gc_batch_csr), P(gc_job), i32, f32, P(gc_options), P(f32), P(f32), vp]
    lib.gc_destroy.restype = None
    lib.gc_destroy.argtypes = [vp]
    lib.gc_get_stats.restype = ctypes.c_int
    lib.gc_get_stats.argtypes = [vp, P(gc_stats)]
    lib.gc_set_timing.restype = ctypes.c_int
    lib.gc_set_timing.argtypes = [vp, ctypes.c_int]
    lib.gc_validate_csr.restype = ctypes.c_int
    lib.gc_validate_csr.argtypes = [vp, P(gc_csr), vp]
    lib.gc_adg_partition.restype = ctypes.c_int
    lib.gc_adg_partition.argtypes = [vp, P(gc_csr), u32, u32, vp, P(i32), vp]
    lib.gc_make_priority.restype = ctypes.c_int
    lib.gc_make_priority.argtypes = [vp, i64, vp, u64, vp, vp]
    lib.gc_jp_color.restype = ctypes.c_int
    lib.gc_jp_color.argtypes = [vp, P(gc_csr), vp, vp, P(i32), vp]
    lib.gc_adg_m_partition.restype = ctypes.c_int
    lib.gc_adg_m_partition.argtypes = [vp, P(gc_csr), vp, P(i32), vp]
    lib.gc_color_graph_m.restype = ctypes.c_int
    lib.gc_color_graph_m.argtypes = [vp, P(gc_csr), u64, vp, vp, P(i32), P(i32), vp]
    lib.gc_adg_o_order.restype = ctypes.c_int
    lib.gc_adg_o_order.argtypes = [vp, P(gc_csr), u32, u32, vp, vp, vp, P(i32), vp]
    lib.gc_color_graph_o.restype = ctypes.c_int
    lib.gc_color_graph_o.argtypes = [vp, P(gc_csr), u32, u32, vp, vp, P(i32), P(i32), vp]
    lib.gc_dec_itr_color.restype = ctypes.c_int
    lib.gc_dec_itr_color.argtypes = [vp, P(gc_csr), vp, i32, u64, vp, P(i32), vp]
    lib.gc_color_graph_dec_itr.restype = ctypes.c_int
    lib.gc_color_graph_dec_itr.argtypes = [vp, P(gc_csr), u32, u32, u64, vp, vp, P(i32), P(i32), vp]
    lib.gc_make_priority_kind.restype = ctypes.c_int
    lib.gc_make_priority_kind.argtypes = [vp, P(gc_csr), ctypes.c_int32, u64, vp, vp]
    lib.gc_color_graph.restype = ctypes.c_int
    lib.gc_color_graph.argtypes = [vp, P(gc_csr), u32, u32, u64, vp, vp, P(i32), P(i32), vp]
    lib.gc_adg_partition_noalloc.restype = ctypes.c_int
    lib.gc_adg_partition_noalloc.argtypes = [P(gc_csr), u32, u32, vp, P(i32), vp]
    lib.gc_color_batch.restype = ctypes.c_int
    lib.gc_color_batch.argtypes = [vp, P(gc_batch_csr), P(gc_job), vp, vp, vp, vp, vp]
    lib.gc_color_batch_list.restype = ctypes.c_int
    lib.gc_color_batch_list.argtypes = [vp, i64, P(gc_csr), P(gc_job), P(vp), vp]
    lib.gc_color_graph_host.restype = ctypes.c_int
    lib.gc_color_graph_host.argtypes = [vp, i64, i64, vp, vp, u32, u32, u64, vp, vp, P(i32), P(i32), vp]
    _lib = lib
    return lib


def status_str(status: int) -> str:
    return load().gc_status_str(status).decode()


def _check(status: int, what: str):
    if status != GC_OK:
        raise GcError(status, what)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


@dataclass
class DeviceGraph:
    """A CSR graph held in CUDA tensors (int64 row_ptr[n+1], int32 col_idx)."""
    row_ptr: "object"
    col_idx: "object"

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0]) - 1

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    def csr(self) -> gc_csr:
        return gc_csr(self.n, self.nnz, self.row_ptr.data_ptr(),
                      self.col_idx.data_ptr() if self.nnz else None)

    @classmethod
    def from_host(cls, g, device="cuda"):
        import torch
        rp = torch.from_numpy(np.ascontiguousarray(g.row_ptr, dtype=np.int64)).to(device)
        ci = torch.from_numpy(np.ascontiguousarray(g.col_idx, dtype=np.int32)).to(device)
        return cls(rp, ci)


@dataclass
class DeviceBatch:
    """Graphs packed as their disjoint union (CUDA tensors): row_ptr[n+1],
    col_idx[nnz] with union ids, graph_off[num_graphs+1]."""
    row_ptr: "object"
    col_idx: "object"
    graph_off: "object"

    @property
    def num_graphs(self) -> int:
        return int(self.graph_off.shape[0]) - 1

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0]) - 1

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    def csr(self) -> gc_batch_csr:
        return gc_batch_csr(self.num_graphs, self.n, self.nnz, self.row_ptr.data_ptr(),
                            self.col_idx.data_ptr() if self.nnz else None, self.graph_off.data_ptr())

    @staticmethod
    def pack_host(graphs):
        """Host arrays (row_ptr, col_idx, graph_off) of the disjoint union."""
        nv = np.array([g.n for g in graphs], dtype=np.int64)
        ne = np.array([g.nnz for g in graphs], dtype=np.int64)
        voff = np.concatenate([[0], np.cumsum(nv)]).astype(np.int64)
        eoff = np.concatenate([[0], np.cumsum(ne)]).astype(np.int64)
        rp = np.empty(int(voff[-1]) + 1, dtype=np.int64)
        ci = np.empty(int(eoff[-1]), dtype=np.int32)
        for i, g in enumerate(graphs):
            rp[voff[i]:voff[i + 1]] = g.row_ptr[:-1] + eoff[i]
            ci[eoff[i]:eoff[i + 1]] = g.col_idx + np.int32(voff[i])
        rp[-1] = eoff[-1]
        return rp, ci, voff

    @classmethod
    def from_host(cls, graphs, device="cuda"):
        import torch
        rp, ci, voff = cls.pack_host(graphs)
        return cls(torch.from_numpy(rp).to(device), torch.from_numpy(ci).to(device),
                   torch.from_numpy(voff).to(device))


class Context:
    """Owns a gc_context (scratch memory on one device).  `options` is a
    gc_options, a dict of its fields, or None for the defaults."""

    def __init__(self, device: int = 0, options=None):
        self._lib = load()
        if isinstance(options, dict):
            options = make_options(**options)
        h = ctypes.c_void_p()
        _check(self._lib.gc_create(ctypes.byref(h), device, ctypes.byref(options) if options is not None else None),
               "gc_create")
        self.handle = h
        self.device = device

    def close(self):
        if self.handle:
            self._lib.gc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- the C ABI, one method per entry point ------------------------------
    def gc_get_options(self) -> gc_options:
        o = gc_options()
        _check(self._lib.gc_get_options(self.handle, ctypes.byref(o)), "gc_get_options")
        return o

    def gc_set_options(self, options):
        """options: a gc_options or a dict of its fields (the rest default)."""
        if isinstance(options, dict):
            options = make_options(**options)
        _check(self._lib.gc_set_options(self.handle, ctypes.byref(options)), "gc_set_options")

    def gc_autotune(self, g: DeviceGraph, eps_p: int, eps_q: int, seed: int, reps: int = 3, budget_ms: float = 0.0,
                    stream=None):
        """Returns (best gc_options, best ms, starting ms); the best options
        are left applied to the context."""
        c = g.csr()
        best = gc_options()
        bm, sm = ctypes.c_float(0), ctypes.c_float(0)
        _check(self._lib.gc_autotune(self.handle, ctypes.byref(c), eps_p, eps_q, seed, reps, budget_ms,
                                     ctypes.byref(best), ctypes.byref(bm), ctypes.byref(sm), _stream(stream)),
               "gc_autotune")
        return best, bm.value, sm.value

    def gc_autotune_batch(self, b: "DeviceBatch", jobs, reps: int = 3, budget_ms: float = 0.0, stream=None):
        c = b.csr()
        arr = (gc_job * b.num_graphs)(*[gc_job(int(p), int(q), int(sd)) for p, q, sd in jobs])
        best = gc_options()
        bm, sm = ctypes.c_float(0), ctypes.c_float(0)
        _check(self._lib.gc_autotune_batch(self.handle, ctypes.byref(c), arr, reps, budget_ms, ctypes.byref(best),
                                           ctypes.byref(bm), ctypes.byref(sm), _stream(stream)), "gc_autotune_batch")
        return best, bm.value, sm.value

    def gc_set_timing(self, enable: bool):
        _check(self._lib.gc_set_timing(self.handle, int(enable)), "gc_set_timing")

    def gc_get_stats(self) -> gc_stats:
        st = gc_stats()
        _check(self._lib.gc_get_stats(self.handle, ctypes.byref(st)), "gc_get_stats")
        return st

    def gc_validate_csr(self, g: DeviceGraph, stream=None) -> int:
        """Returns GC_OK or GC_ERR_INVALID_GRAPH (other errors raise)."""
        c = g.csr()
        st = self._lib.gc_validate_csr(self.handle, ctypes.byref(c), _stream(stream))
        if st not in (GC_OK, GC_ERR_INVALID_GRAPH):
            _check(st, "gc_validate_csr")
        return st

    def gc_adg_partition(self, g: DeviceGraph, eps_p: int, eps_q: int, batch_out, stream=None) -> int:
        c = g.csr()
        rounds = ctypes.c_int32(0)
        _check(self._lib.gc_adg_partition(self.handle, ctypes.byref(c), eps_p, eps_q, _ptr(batch_out),
                                          ctypes.byref(rounds), _stream(stream)), "gc_adg_partition")
        return rounds.value

    def gc_make_priority(self, n: int, batch, seed: int, key_out, stream=None):
        _check(self._lib.gc_make_priority(self.handle, n, _ptr(batch), seed, _ptr(key_out),
                                          _stream(stream)), "gc_make_priority")

    def gc_adg_m_partition(self, g: DeviceGraph, batch_out, stream=None) -> int:
        c = g.csr()
        nr = ctypes.c_int32(0)
        _check(self._lib.gc_adg_m_partition(self.handle, ctypes.byref(c), _ptr(batch_out), ctypes.byref(nr),
                                            _stream(stream)), "gc_adg_m_partition")
        return nr.value

    def gc_color_graph_m(self, g: DeviceGraph, seed: int, color_out, batch_out=None, stream=None):
        """JP-ADG-M; returns (num_colors, num_rounds)."""
        c = g.csr()
        nc, nr = ctypes.c_int32(0), ctypes.c_int32(0)
        _check(self._lib.gc_color_graph_m(self.handle, ctypes.byref(c), seed, _ptr(color_out), _ptr(batch_out),
                                          ctypes.byref(nc), ctypes.byref(nr), _stream(stream)), "gc_color_graph_m")
        return nc.value, nr.value

    def gc_adg_o_order(self, g: DeviceGraph, eps_p: int, eps_q: int, rho_out, batch_out=None, rank_out=None,
                       stream=None) -> int:
        """ADG-O's total order rho (and batches, rank); returns the number of
        iterations."""
        c = g.csr()
        nr = ctypes.c_int32(0)
        _check(self._lib.gc_adg_o_order(self.handle, ctypes.byref(c), eps_p, eps_q, _ptr(batch_out), _ptr(rho_out),
                                        _ptr(rank_out), ctypes.byref(nr), _stream(stream)), "gc_adg_o_order")
        return nr.value

    def gc_color_graph_o(self, g: DeviceGraph, eps_p: int, eps_q: int, color_out, batch_out=None, stream=None):
        """JP-ADG-O; returns (num_colors, num_rounds)."""
        c = g.csr()
        nc, nr = ctypes.c_int32(0), ctypes.c_int32(0)
        _check(self._lib.gc_color_graph_o(self.handle, ctypes.byref(c), eps_p, eps_q, _ptr(color_out),
                                          _ptr(batch_out), ctypes.byref(nc), ctypes.byref(nr), _stream(stream)),
               "gc_color_graph_o")
        return nc.value, nr.value

    def gc_dec_itr_color(self, g: DeviceGraph, batch, num_rounds: int, seed: int, color_out, stream=None) -> int:
        """DEC-ADG-ITR colouring of the partitions batch = 1..num_rounds;
        returns the number of colours (SIM-COL iterations in stats())."""
        c = g.csr()
        nc = ctypes.c_int32(0)
        _check(self._lib.gc_dec_itr_color(self.handle, ctypes.byref(c), _ptr(batch), num_rounds, seed,
                                          _ptr(color_out), ctypes.byref(nc), _stream(stream)), "gc_dec_itr_color")
        return nc.value

    def gc_color_graph_dec_itr(self, g: DeviceGraph, eps_p: int, eps_q: int, seed: int, color_out,
                               batch_out=None, stream=None):
        """ADG then DEC-ADG-ITR; returns (num_colors, num_rounds)."""
        c = g.csr()
        nc, nr = ctypes.c_int32(0), ctypes.c_int32(0)
        _check(self._lib.gc_color_graph_dec_itr(self.handle, ctypes.byref(c), eps_p, eps_q, seed, _ptr(color_out),
                                                _ptr(batch_out), ctypes.byref(nc), ctypes.byref(nr),
                                                _stream(stream)), "gc_color_graph_dec_itr")
        return nc.value, nr.value

    def gc_make_priority_kind(self, g: DeviceGraph, kind: int, seed: int, key_out, stream=None):
        c = g.csr()
        _check(self._lib.gc_make_priority_kind(self.handle, ctypes.byref(c), kind, seed, _ptr(key_out),
                                               _stream(stream)), "gc_make_priority_kind")

    def gc_jp_color(self, g: DeviceGraph, priority, color_out, stream=None) -> int:
        c = g.csr()
        nc = ctypes.c_int32(0)
        _check(self._lib.gc_jp_color(self.handle, ctypes.byref(c), _ptr(priority), _ptr(color_out),
                                     ctypes.byref(nc), _stream(stream)), "gc_jp_color")
        return nc.value

    def gc_color_graph(self, g: DeviceGraph, eps_p: int, eps_q: int, seed: int, color_out,
                       batch_out=None, stream=None):
        """Returns (num_colors, num_rounds)."""
        c = g.csr()
        nc, nr = ctypes.c_int32(0), ctypes.c_int32(0)
        _check(self._lib.gc_color_graph(self.handle, ctypes.byref(c), eps_p, eps_q, seed,
                                        _ptr(color_out), _ptr(batch_out), ctypes.byref(nc),
                                        ctypes.byref(nr), _stream(stream)), "gc_color_graph")
        return nc.value, nr.value

    def gc_color_batch(self, b: DeviceBatch, jobs, color_out, batch_out=None, num_colors_out=None,
                       num_rounds_out=None, stream=None):
        """jobs: sequence of (eps_p, eps_q, seed), one per graph."""
        c = b.csr()
        arr = (gc_job * b.num_graphs)(*[gc_job(int(p), int(q), int(sd)) for p, q, sd in jobs])
        _check(self._lib.gc_color_batch(self.handle, ctypes.byref(c), arr, _ptr(color_out), _ptr(batch_out),
                                        _ptr(num_colors_out), _ptr(num_rounds_out), _stream(stream)),
               "gc_color_batch")

    def gc_color_batch_list(self, graphs, jobs, color_outs, stream=None):
        """graphs: DeviceGraph list; jobs: (eps_p, eps_q, seed) per graph;
        color_outs: CUDA int32 tensors, one per graph."""
        G = len(graphs)
        csrs = (gc_csr * G)(*[g.csr() for g in graphs])
        arr = (gc_job * G)(*[gc_job(int(p), int(q), int(sd)) for p, q, sd in jobs])
        outs = (ctypes.c_void_p * G)(*[c.data_ptr() if c.numel() else None for c in color_outs])
        _check(self._lib.gc_color_batch_list(self.handle, G, csrs, arr, outs, _stream(stream)),
               "gc_color_batch_list")

    def gc_color_graph_host(self, row_ptr: np.ndarray, col_idx: np.ndarray, eps_p: int, eps_q: int,
                            seed: int, color_out: np.ndarray, batch_out: np.ndarray | None = None,
                            stream=None):
        """Host arrays in and out (numpy, ideally in page-locked memory).
        Returns (num_colors, num_rounds)."""
        n = row_ptr.shape[0] - 1
        nnz = col_idx.shape[0]
        assert row_ptr.dtype == np.int64 and col_idx.dtype == np.int32 and color_out.dtype == np.int32
        nc, nr = ctypes.c_int32(0), ctypes.c_int32(0)
        _check(self._lib.gc_color_graph_host(
            self.handle, n, nnz, row_ptr.ctypes.data, col_idx.ctypes.data if nnz else None,
            eps_p, eps_q, seed, color_out.ctypes.data if n else None,
            batch_out.ctypes.data if batch_out is not None and n else None,
            ctypes.byref(nc), ctypes.byref(nr), _stream(stream)), "gc_color_graph_host")
        return nc.value, nr.value


def gc_adg_partition_noalloc(g: DeviceGraph, eps_p: int, eps_q: int, batch_out, stream=None) -> int:
    """ADG without a context and without any device allocation (a fixed
    scratch array inside the library bounds the graph to n <= 262144 and
    nnz <= 8388608).  For callers that cannot allocate device memory when they
    call in.  Runs on the current device; concurrent calls must not overlap
    on the GPU.  Returns the number of rounds."""
    c = g.csr()
    rounds = ctypes.c_int32(0)
    _check(load().gc_adg_partition_noalloc(ctypes.byref(c), eps_p, eps_q, _ptr(batch_out),
                                           ctypes.byref(rounds), _stream(stream)),
           "gc_adg_partition_noalloc")
    return rounds.value
