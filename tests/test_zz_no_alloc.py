"""The allocation-free ADG entry point (for callers that cannot allocate
device memory when they call in) against the ordinary gc_adg_partition and
against the CPU oracle, through the C ABI: the batch ids and round counts
must be identical (they are integers, so the tolerance is exact equality), on
two calls in a row, since every call reuses the same built-in scratch array.
Graphs at the fixed array's limits (n = 2^18, nnz up to 2^23) still fit; one
past either limit is refused with GC_ERR_OVERFLOW."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import graphgen as gg
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2008_11321_gb300 as gcp  # noqa: E402
from paper_2008_11321_gb300 import gcolor  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_11321_gb300 import _build
    _build.build()
    c = gcp.Context(0)
    yield c
    c.close()


MAX_N, MAX_NNZ = 1 << 18, 1 << 23

GRAPHS = [gg.erdos_renyi(16384, 81920, 1), gg.rmat(16, 16, seed=5), gg.barabasi_albert(200000, 4, 3),
          gg.grid(300, 300, perm_seed=2),
          # at the limits: n = 2^18 with nnz at 96% of 2^23, and nnz = 2^23 exactly
          gg.rmat(18, 17, seed=4), gg.erdos_renyi(MAX_N, MAX_NNZ // 2, 6)]


@pytest.mark.parametrize("g", GRAPHS, ids=lambda g: g.name)
@pytest.mark.parametrize("p,q", [(1, 100), (1, 2)])
def test_noalloc_matches_context_path_twice(ctx, g, p, q):
    dg = gcp.DeviceGraph.from_host(g, "cuda:0")
    ref = torch.empty(g.n, dtype=torch.int32, device="cuda:0")
    ref_rounds = ctx.gc_adg_partition(dg, p, q, ref)
    ob, onr = oracle.adg(g, p, q)
    assert g.n <= MAX_N and g.nnz <= MAX_NNZ
    for _ in range(2):
        out = torch.full((g.n,), -3, dtype=torch.int32, device="cuda:0")
        rounds = gcolor.gc_adg_partition_noalloc(dg, p, q, out)
        torch.cuda.synchronize()
        assert rounds == ref_rounds == onr
        assert torch.equal(out, ref)
        assert np.array_equal(out.cpu().numpy(), ob)


@pytest.mark.parametrize("g", [gg.erdos_renyi(MAX_N + 1, 1000, 7), gg.erdos_renyi(MAX_N, MAX_NNZ // 2 + 1, 8)],
                         ids=["n_over", "nnz_over"])
def test_noalloc_refuses_one_past_each_limit(g):
    # a real graph one vertex or one edge past the fixed array's bounds: the
    # call is refused before any device work and leaves batch_out untouched
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    assert g.n == MAX_N + 1 or g.nnz == MAX_NNZ + 2
    dg = gcp.DeviceGraph.from_host(g, "cuda:0")
    out = torch.full((g.n,), -3, dtype=torch.int32, device="cuda:0")
    with pytest.raises(gcp.GcError) as err:
        gcolor.gc_adg_partition_noalloc(dg, 1, 100, out)
    assert err.value.status == gcp.GC_ERR_OVERFLOW
    torch.cuda.synchronize()
    assert int(out.min()) == -3 and int(out.max()) == -3


def test_noalloc_rejects_graphs_over_its_limit():
    lib = gcp.load()
    rounds = ctypes.c_int32(0)
    big = gcolor.gc_csr(262145, 0, 1, None)  # never dereferenced: rejected on size
    assert lib.gc_adg_partition_noalloc(ctypes.byref(big), 1, 100, 1, ctypes.byref(rounds), None) == \
        gcp.GC_ERR_OVERFLOW
    dense = gcolor.gc_csr(1000, 8388609, 1, 1)
    assert lib.gc_adg_partition_noalloc(ctypes.byref(dense), 1, 100, 1, ctypes.byref(rounds), None) == \
        gcp.GC_ERR_OVERFLOW
