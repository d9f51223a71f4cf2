"""The C-ABI library builds, loads and exports every symbol that
include/gcolor.h declares (no GPU needed: only calls that make no CUDA
compute call are exercised)."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

import paper_2008_11321_gb300 as gcp
from paper_2008_11321_gb300 import _build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "gcolor.h")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(gc_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return gcp.load()


def test_header_declares_expected_calls():
    assert set(_declared()) == set(gcp.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_status_strings(lib):
    assert lib.gc_last_error() == b""
    assert gcp.status_str(gcp.GC_OK) == "GC_OK"
    assert gcp.status_str(gcp.GC_ERR_TIMEOUT) == "GC_ERR_TIMEOUT"
    assert gcp.status_str(99) == "GC_ERR_UNKNOWN"


def test_null_arguments_rejected_without_device_work(lib):
    rounds = ctypes.c_int32(0)
    csr = gcp.gcolor.gc_csr(10, 0, None, None)
    assert lib.gc_adg_partition(None, ctypes.byref(csr), 1, 100, None, ctypes.byref(rounds), None) == \
        gcp.GC_ERR_INVALID_ARG
    assert lib.gc_color_graph(None, None, 1, 100, 42, None, None, None, None, None) == gcp.GC_ERR_INVALID_ARG
    assert lib.gc_create(None, 0, None) == gcp.GC_ERR_INVALID_ARG
    for call in (lambda: lib.gc_dec_itr_color(None, None, None, 1, 42, None, None, None),
                 lambda: lib.gc_color_graph_dec_itr(None, None, 1, 100, 42, None, None, None, None, None),
                 lambda: lib.gc_adg_o_order(None, None, 1, 100, None, None, None, None, None),
                 lambda: lib.gc_color_graph_o(None, None, 1, 100, None, None, None, None, None),
                 lambda: lib.gc_adg_m_partition(None, None, None, None, None),
                 lambda: lib.gc_color_graph_m(None, None, 42, None, None, None, None, None)):
        assert call() == gcp.GC_ERR_INVALID_ARG
    st = gcp.gcolor.gc_stats()
    assert lib.gc_get_stats(None, ctypes.byref(st)) == gcp.GC_ERR_INVALID_ARG
    lib.gc_destroy(None)  # a no-op


def test_library_links_cuda_sm103a_only(lib):
    # the build compiles for exactly one real architecture
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def _prototypes():
    """{name: [parameter declarations]} from the header's prototypes."""
    text = re.sub(r"/\*.*?\*/", " ", open(HEADER).read(), flags=re.S)
    out = {}
    for name, params in re.findall(r"\b(?:gc_status|void|const char\s*\*)\s*(gc_\w+)\s*\(([^;]*?)\)\s*;", text,
                                   flags=re.S):
        ps = [" ".join(p.split()) for p in params.split(",")]
        out[name] = [] if ps == ["void"] or ps == [""] else ps
    return out


def _ctype_kind(t):
    """'ptr' for pointer-sized arguments, else the integer width and sign."""
    if t in (ctypes.c_void_p, ctypes.c_char_p) or (isinstance(t, type) and issubclass(t, ctypes._Pointer)):
        return "ptr"
    return {ctypes.c_int32: "i32", ctypes.c_uint32: "u32", ctypes.c_int64: "i64", ctypes.c_uint64: "u64",
            ctypes.c_float: "f32"}.get(t, t)


def _decl_kind(decl):
    if "*" in decl or decl.startswith("gc_stream"):
        return "ptr"
    base = decl.rsplit(" ", 1)[0].replace("const ", "")
    return {"int": "i32", "int32_t": "i32", "uint32_t": "u32", "int64_t": "i64", "uint64_t": "u64",
            "gc_status": "i32", "float": "f32"}[base]


def test_binding_signatures_match_header(lib):
    # the ctypes argument lists the binding installs have the header's arity
    # and, parameter by parameter, its pointer/integer kind and width
    protos = _prototypes()
    assert set(protos) == set(gcp.EXPORTS)
    for name, decls in protos.items():
        argtypes = getattr(lib, name).argtypes
        assert argtypes is not None and len(argtypes) == len(decls), (name, decls)
        for decl, t in zip(decls, argtypes):
            kind = _ctype_kind(t)
            want = _decl_kind(decl)
            assert kind == want or (want == "i32" and t is ctypes.c_int), (name, decl, t)


def test_options_defaults_and_range_checks(lib):
    # defaults come from the library; out-of-range fields are rejected by
    # gc_create before it touches any device
    o = gcp.make_options()
    assert o.struct_size == ctypes.sizeof(gcp.gc_options)
    assert o.as_dict() == {"core_target": 16384, "core_cluster": 16, "core_warps": 12, "dec_tail": 1,
                           "update_mode": gcp.GC_UPDATE_AUTO, "pull_percent": 25, "bulk_blocks_per_sm": 0,
                           "wait_limit_ms": 4000, "jp_state16": 0,
                           "batch_mode": gcp.GC_BATCH_AUTO, "update_hubs": 512,
                           "host_upload": 1, "round_graph": 1}
    h = ctypes.c_void_p()
    bad = [dict(core_target=-1), dict(core_target=32769), dict(core_cluster=0), dict(core_cluster=17),
           dict(core_warps=0), dict(core_warps=33), dict(dec_tail=2), dict(update_mode=3),
           dict(pull_percent=-1), dict(bulk_blocks_per_sm=33), dict(wait_limit_ms=0),
           dict(wait_limit_ms=600001), dict(jp_state16=2),
           dict(batch_mode=3), dict(update_hubs=-1), dict(update_hubs=4097),
           dict(host_upload=2), dict(round_graph=2)]
    for fields in bad:
        o = gcp.make_options(**fields)
        assert lib.gc_create(ctypes.byref(h), 0, ctypes.byref(o)) == gcp.GC_ERR_INVALID_ARG, fields
        assert not h.value
    o = gcp.make_options()
    o.struct_size = ctypes.sizeof(gcp.gc_options) + 4  # newer than the library
    assert lib.gc_create(ctypes.byref(h), 0, ctypes.byref(o)) == gcp.GC_ERR_INVALID_ARG
    with pytest.raises(KeyError):
        gcp.make_options(no_such_field=1)
    assert lib.gc_options_init(None) == gcp.GC_ERR_INVALID_ARG
    assert lib.gc_get_options(None, ctypes.byref(o)) == gcp.GC_ERR_INVALID_ARG
    assert lib.gc_set_options(None, ctypes.byref(o)) == gcp.GC_ERR_INVALID_ARG
    assert lib.gc_autotune(None, None, 1, 100, 42, 3, 0.0, None, None, None, None) == gcp.GC_ERR_INVALID_ARG
    assert lib.gc_autotune_batch(None, None, None, 3, 0.0, None, None, None, None) == gcp.GC_ERR_INVALID_ARG
