"""Failure paths, triggered without faulting or hanging the GPU.

* Round cap: a context limited to 2 peeling rounds gives ND_ETIMEOUT on a graph that needs more,
  in every launch mode of the peeling loop; the same context then decomposes correctly.
* Bounded grid-barrier wait: with ND_LIMIT_DROP_BLOCK the last block of the persistent peel
  kernel leaves before its first barrier, so the other blocks wait for an arrival that never
  comes; each wait is bounded (here 50 ms), every block leaves, and the call returns
  ND_ETIMEOUT within about a second. The context stays usable and the next decomposition
  matches the oracle.
* Count overflow: with a width-4 count limit below the graph's largest count, width 4 gives
  ND_EOVERFLOW, while width 8 (and the automatic choice) give the oracle's result.
"""
import time

import numpy as np
import pytest

import graphgen as gg
import oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nd():
    import paper_2111_10980_gb300 as nd

    nd.lib()
    return nd


def _decompose(nd, ctx, g, r, s, **kw):
    G = nd.nd_load_csr(ctx, g.rowptr, g.col)
    try:
        return nd.nd_decompose(G, r, s, **kw)
    finally:
        nd.nd_graph_free(G)


def test_round_cap_gives_etimeout(nd):
    g = gg.rmat(11, 16, 0.57, 0.19, 0.19, seed=61)
    want = orc.decompose(g, 2, 3)
    assert want.rho > 2
    ctx = nd.nd_ctx_create(0)
    try:
        nd.nd_ctx_set_limits(ctx, max_rounds=2)
        for flags in (nd.ND_PEEL_PERSISTENT, nd.ND_PEEL_LOOP_GRAPH, nd.ND_NO_GRAPH):
            with pytest.raises(nd.NdError) as ei:
                _decompose(nd, ctx, g, 2, 3, flags=flags)
            assert ei.value.code == nd.ND_ETIMEOUT, flags
            assert "round cap" in str(ei.value)
        # a cap above rho changes nothing
        nd.nd_ctx_set_limits(ctx, max_rounds=want.rho)
        core, rnd, st = _decompose(nd, ctx, g, 2, 3)
        assert np.array_equal(core, want.core) and st["rho"] == want.rho
        nd.nd_ctx_set_limits(ctx)
        core, rnd, _ = _decompose(nd, ctx, g, 2, 3)
        assert np.array_equal(core, want.core) and np.array_equal(rnd, want.round)
    finally:
        nd.nd_ctx_destroy(ctx)


@pytest.mark.parametrize("r,s", [(2, 3), (3, 4)])
def test_bounded_barrier_wait_gives_etimeout(nd, r, s):
    g = gg.chung_lu(3000, 20.0, 2.2, seed=62)
    want = orc.decompose(g, r, s)
    ctx = nd.nd_ctx_create(0)
    try:
        nd.nd_ctx_set_limits(ctx, barrier_timeout_ns=50_000_000, flags=nd.ND_LIMIT_DROP_BLOCK)
        t0 = time.perf_counter()
        with pytest.raises(nd.NdError) as ei:
            _decompose(nd, ctx, g, r, s, flags=nd.ND_PEEL_PERSISTENT)
        dt = time.perf_counter() - t0
        assert ei.value.code == nd.ND_ETIMEOUT
        assert "barrier" in str(ei.value)
        assert dt < 10.0, dt
        # the context is still usable: the next decompositions match the oracle
        nd.nd_ctx_set_limits(ctx)
        for flags in (nd.ND_PEEL_PERSISTENT, 0):
            core, rnd, st = _decompose(nd, ctx, g, r, s, flags=flags)
            assert np.array_equal(core, want.core) and np.array_equal(rnd, want.round)
            assert st["listed"] == want.n_s
    finally:
        nd.nd_ctx_destroy(ctx)


def test_width4_count_overflow_gives_eoverflow(nd):
    g = gg.complete(10)  # every triangle lies in 7 4-cliques, every edge in 8 triangles
    ctx = nd.nd_ctx_create(0)
    try:
        nd.nd_ctx_set_limits(ctx, count_limit=6)
        G = nd.nd_load_csr(ctx, g.rowptr, g.col)
        try:
            for fn in (lambda: nd.nd_count(G, 3, 4, count_width=4), lambda: nd.nd_decompose(G, 3, 4, count_width=4)):
                with pytest.raises(nd.NdError) as ei:
                    fn()
                assert ei.value.code == nd.ND_EOVERFLOW
            counts, _, _ = nd.nd_count(G, 3, 4, count_width=8)
            assert np.all(counts == 7)
            for width in (0, 8):
                core, _, st = nd.nd_decompose(G, 3, 4, count_width=width)
                assert np.all(core == 7) and st["count_width"] == 8
            # (2,3): counts of 8 also exceed the limit; (1,2) degrees of 9 too
            with pytest.raises(nd.NdError) as ei:
                nd.nd_decompose(G, 2, 3, count_width=4)
            assert ei.value.code == nd.ND_EOVERFLOW
        finally:
            nd.nd_graph_free(G)
        nd.nd_ctx_set_limits(ctx, count_limit=7)
        core, _, st = _decompose(nd, ctx, g, 3, 4, count_width=4)
        assert np.all(core == 7) and st["count_width"] == 4
    finally:
        nd.nd_ctx_destroy(ctx)


def test_limits_reject_bad_arguments(nd):
    ctx = nd.nd_ctx_create(0)
    try:
        with pytest.raises(nd.NdError) as ei:
            nd.nd_ctx_set_limits(ctx, max_rounds=-1)
        assert ei.value.code == nd.ND_EINVAL
        with pytest.raises(nd.NdError) as ei:
            nd.nd_ctx_set_limits(ctx, flags=0x100)
        assert ei.value.code == nd.ND_EINVAL
    finally:
        nd.nd_ctx_destroy(ctx)
