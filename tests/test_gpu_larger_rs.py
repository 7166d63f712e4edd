"""(r,s) beyond the five with kernels of their own: (1,4), (2,5), (3,5), (3,6), (4,5), (4,6),
through the generic listing of the (s-r)-cliques of each r-clique's common neighbourhood, with the
4-clique index for r = 4 (Section 6 evaluates every r < s <= 7). Compared with the oracle element by element (counts, cores, peel rounds, |A|
and k per round, s-cliques destroyed, decrements), including graphs whose hubs send r-cliques to
the heavy phase and the K_n closed form C(n-r, s-r)."""
import math

import numpy as np
import pytest

import graphgen as gg
import oracle as orc
from test_gpu_parity import assert_parity

pytestmark = pytest.mark.gpu

RS = [(1, 4), (2, 5), (3, 5), (3, 6), (4, 5), (4, 6)]


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


@pytest.mark.parametrize("r,s", RS)
def test_figure1_and_complete_graphs(nd, ctx, r, s):
    assert_parity(nd, ctx, gg.fig1(), r, s)
    for n in (1, 4, 5, 6, 8, 13):
        got = assert_parity(nd, ctx, gg.complete(n), r, s)
        if n >= s:
            assert np.all(got["core"] == math.comb(n - r, s - r)) and got["rho"] == 1


@pytest.mark.parametrize("r,s", RS)
def test_random_small_graphs(nd, ctx, r, s):
    for seed in range(12):
        n = 8 + (seed * 5) % 22
        assert_parity(nd, ctx, gg.gnp(n, [0.4, 0.6, 0.8][seed % 3], 7000 + seed), r, s)


@pytest.mark.parametrize("r,s", RS)
def test_power_law_rmat_and_communities(nd, ctx, r, s):
    assert_parity(nd, ctx, gg.chung_lu(1500, 12.0, 2.2, seed=101), r, s)
    assert_parity(nd, ctx, gg.rmat(11, 16, 0.5, 0.1, 0.1, seed=102), r, s)
    assert_parity(nd, ctx, gg.with_planted(gg.chung_lu(1500, 6.0, 2.3, seed=103), 12, 12, 24, 0.7, seed=104), r, s)


@pytest.mark.parametrize("r,s", [(1, 4), (2, 5), (3, 5), (4, 5)])
def test_heavy_phase(nd, ctx, r, s):
    g = gg.hubs_over_sparse(n_common=5000, hubs=4, p_hub=0.9, avg_deg=4.0, seed=105)
    for flags in (nd.ND_PEEL_PERSISTENT, nd.ND_NO_GRAPH):
        assert_parity(nd, ctx, g, r, s, flags=flags)


@pytest.mark.parametrize("r,s", RS)
def test_launch_modes_and_dense_buckets(nd, ctx, r, s):
    g = gg.chung_lu(800, 14.0, 2.1, seed=106)
    for flags in (nd.ND_PEEL_LOOP_GRAPH, nd.ND_NO_GRAPH, nd.ND_DENSE_BUCKETS):
        assert_parity(nd, ctx, g, r, s, flags=flags)
    assert_parity(nd, ctx, g, r, s, count_width=8)


def test_4clique_index_and_batches(nd, ctx):
    """The 4-clique index: tuples in canonical order (compared with the oracle's listing), and
    (4,5) requests inside a batch get the numbers they get alone."""
    g = gg.with_planted(gg.chung_lu(1200, 8.0, 2.2, seed=107), 10, 12, 20, 0.8, seed=108)
    G = nd.nd_load_csr(ctx, g.rowptr, g.col)
    try:
        got = nd.nd_rcliques(G, 4)
    finally:
        nd.nd_graph_free(G)
    assert np.array_equal(got.reshape(-1, 4), orc.list_cliques(g, 4).reshape(-1, 4))
    items = [(gg.complete(7), 4, 5), (g, 4, 5), (gg.fig1(), 4, 5), (gg.gnp(25, 0.7, 109), 4, 6), (g, 3, 5)]
    outs, n_r, status, _ = nd.nd_batch_run(ctx, [(x.rowptr, x.col, r, s) for x, r, s in items])
    assert all(st == nd.ND_OK for st in status)
    for (x, r, s), out in zip(items, outs):
        assert np.array_equal(out, orc.decompose(x, r, s).core), (x.name, r, s)
