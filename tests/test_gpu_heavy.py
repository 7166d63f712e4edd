"""Parity on the paths an Update takes for r-cliques with very long driving lists.

The light Update phase gives one warp to each r-clique of A; an r-clique whose driving list is
longer than the variant's threshold (4,096 entries for (1,2), (1,3) and (3,4); 256 for (2,3); 96
for (2,4)) is deferred to the heavy phase, which gives it a whole block. The graphs here are
built so that this happens for every (r,s) while the oracle still finishes in a second: a sparse
power-law graph plus a few mutually adjacent hub vertices adjacent to most of it, so that hub
vertices have degree > 4,096 ((1,2), (1,3)), hub edges have > 4,096 common neighbours, and the
triangles of three hubs have three lists longer than 4,096 ((3,4)). Every output is compared
with the oracle element by element (cores, peel rounds, |A| and k of every round, decrements,
s-cliques destroyed), in every launch mode of the peeling loop.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle as orc
from test_gpu_parity import assert_parity

pytestmark = pytest.mark.gpu

HEAVY = 4096

GRAPHS = {
    "4 hubs, p 0.9": dict(n_common=6000, hubs=4, p_hub=0.9, avg_deg=8.0, seed=51),
    "5 hubs, p 0.85": dict(n_common=6500, hubs=5, p_hub=0.85, avg_deg=6.0, seed=52),
}


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


@pytest.fixture(scope="module", params=list(GRAPHS))
def hub_graph(request):
    return gg.hubs_over_sparse(**GRAPHS[request.param])


def test_the_graphs_reach_the_heavy_threshold(hub_graph):
    """Hub vertices, and all three edges of every hub triangle, exceed 4,096 (checked with the
    oracle's counts: the (1,2) count of a vertex is its degree, the (2,3) count of an edge its
    number of common neighbours)."""
    g = hub_graph
    deg, _ = orc.count(g, 1, 2)
    n_hubs = int((deg > HEAVY).sum())
    assert n_hubs >= 4
    sup, _ = orc.count(g, 2, 3)
    edges = orc.list_cliques(g, 2)
    tris = orc.list_cliques(g, 3)
    hubs = set(np.nonzero(deg > HEAVY)[0].tolist())
    pos = {tuple(e): i for i, e in enumerate(edges.tolist())}
    heavy_tris = 0
    for t in tris.tolist():
        if all(v in hubs for v in t):
            lists = [sup[pos[(t[0], t[1])]], sup[pos[(t[0], t[2])]], sup[pos[(t[1], t[2])]]]
            assert min(lists) > HEAVY
            heavy_tris += 1
    assert heavy_tris >= 4


@pytest.mark.parametrize("r,s", [(1, 2), (1, 3), (2, 3), (2, 4), (3, 4)])
def test_heavy_phase_parity(nd, ctx, hub_graph, r, s):
    for flags in (0, nd.ND_PEEL_PERSISTENT, nd.ND_PEEL_LOOP_GRAPH, nd.ND_NO_GRAPH):
        assert_parity(nd, ctx, hub_graph, r, s, flags=flags)


def test_heavy_phase_with_degeneracy_orientation(nd, ctx, hub_graph):
    for r, s in [(1, 3), (3, 4), (2, 4)]:
        assert_parity(nd, ctx, hub_graph, r, s, orient=nd.ND_ORIENT_DEGENERACY)
