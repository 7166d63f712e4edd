"""Graph contraction for (2,3) (Section 5.6): the peel compacts the adjacency rows of vertices
that lost edges, so later Updates do not walk peeled edges; for (3,4) the same is done to the
triangle lists, whose entries of peeled triangles are removed (moving each kept entry's tag and
offset along). Neither may change any result.

Compared with the oracle element by element (cores, peel rounds, |A| and k per round, destroyed
triangles, decrements) with contraction forced before every round (every row that lost an entry
is compacted), with the paper's schedule (the default: after 2n peeled edges, rows that lost a
quarter of their entries) and with contraction off, in every launch mode of the peeling loop.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle as orc
from test_gpu_parity import assert_parity

pytestmark = pytest.mark.gpu

GRAPHS = [lambda: gg.fig1(), lambda: gg.complete(12), lambda: gg.chung_lu_2k(),
          lambda: gg.rmat(12, 16, 0.57, 0.19, 0.19, seed=81),
          lambda: gg.hubs_over_sparse(n_common=3000, hubs=3, p_hub=0.8, avg_deg=8.0, seed=82),
          lambda: gg.with_planted(gg.chung_lu(3000, 8.0, 2.3, seed=83), 30, 20, 50, 0.7, seed=84)]


@pytest.fixture(scope="module")
def nd():
    import paper_2111_10980_gb300 as nd

    nd.lib()
    return nd


@pytest.fixture(scope="module")
def ctx(nd):
    c = nd.nd_ctx_create(0)
    yield c
    nd.nd_ctx_destroy(c)


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_contraction_parity(nd, ctx, gi):
    g = GRAPHS[gi]()
    for mode in (0, nd.ND_PEEL_PERSISTENT, nd.ND_PEEL_LOOP_GRAPH, nd.ND_NO_GRAPH):
        for c in (nd.ND_CONTRACT_ALWAYS, 0, nd.ND_CONTRACT_OFF):
            got = assert_parity(nd, ctx, g, 2, 3, flags=mode | c)
            if c == nd.ND_CONTRACT_OFF:
                assert got["st"]["contractions"] == 0
            elif c == nd.ND_CONTRACT_ALWAYS and got["st"]["rho"] > 1:
                assert got["st"]["contractions"] >= 1


def test_contraction_schedule_follows_the_paper(nd, ctx):
    """By default a contraction runs only after at least 2n edges were peeled since the last one,
    so there are at most m / (2n) of them; forced contraction runs before every later round."""
    g = gg.rmat(13, 16, 0.57, 0.19, 0.19, seed=85)
    want = orc.decompose(g, 2, 3)
    G = nd.nd_load_csr(ctx, g.rowptr, g.col)
    try:
        core, rnd, st = nd.nd_decompose(G, 2, 3)
        assert np.array_equal(core, want.core) and np.array_equal(rnd, want.round)
        assert 1 <= st["contractions"] <= g.m // (2 * g.n)
        core, rnd, st = nd.nd_decompose(G, 2, 3, flags=nd.ND_CONTRACT_ALWAYS)
        assert np.array_equal(core, want.core) and np.array_equal(rnd, want.round)
        assert st["contractions"] == want.rho - 1
    finally:
        nd.nd_graph_free(G)


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_list_contraction_parity_34(nd, ctx, gi):
    g = GRAPHS[gi]()
    for mode in (0, nd.ND_PEEL_PERSISTENT, nd.ND_PEEL_LOOP_GRAPH, nd.ND_NO_GRAPH):
        for c in (nd.ND_CONTRACT_ALWAYS, 0, nd.ND_CONTRACT_OFF):
            got = assert_parity(nd, ctx, g, 3, 4, flags=mode | c)
            if c == nd.ND_CONTRACT_OFF:
                assert got["st"]["contractions"] == 0
            elif c == nd.ND_CONTRACT_ALWAYS and got["st"]["rho"] > 1:
                assert got["st"]["contractions"] >= 1


def test_list_contraction_with_dense_buckets_and_no_directory(nd):
    """(3,4) list contraction next to the dense buckets, and without the hash directory (every
    list bisected over its compacted length)."""
    import torch

    g = gg.rmat(12, 16, 0.57, 0.19, 0.19, seed=86)
    ctx = nd.nd_ctx_create(0)
    try:
        for c in (nd.ND_CONTRACT_ALWAYS, 0):
            assert_parity(nd, ctx, g, 3, 4, flags=nd.ND_DENSE_BUCKETS | c)
    finally:
        nd.nd_ctx_destroy(ctx)
    alloc, free = nd.torch_allocator_hooks(0)

    def small_only(nbytes, stream):
        return 0 if nbytes > 16 << 20 else alloc(nbytes, stream)

    ctx = nd.nd_ctx_create(0, stream=torch.cuda.Stream())
    nd.nd_ctx_set_allocator(ctx, small_only, free)
    try:
        for c in (nd.ND_CONTRACT_ALWAYS, 0):
            assert_parity(nd, ctx, g, 3, 4, flags=c)
    finally:
        nd.nd_ctx_destroy(ctx)
