"""Dense buckets with the doubling search (Section 4.2, Discussion): the peel finds each new level
as the first non-empty bucket of an array indexed by count, searching regions of sizes 1, 2, 4,
... above the current level, instead of taking the minimum over the bucket window. The buckets
are kept exact by the decrements (a count above k + 1 moves down one bucket; at k + 1 the
r-clique is scheduled and leaves) and by the selection of A. Results must be the oracle's,
element by element, for every (r,s), every launch mode, and together with the (2,3) contraction.
"""
import numpy as np
import pytest

import graphgen as gg
from test_gpu_parity import assert_parity

pytestmark = pytest.mark.gpu

RS = [(1, 2), (1, 3), (2, 3), (2, 4), (3, 4)]
GRAPHS = [lambda: gg.fig1(), lambda: gg.complete(10), lambda: gg.gnp(30, 0.5, 91), lambda: gg.chung_lu_2k(),
          lambda: gg.rmat(11, 16, 0.57, 0.19, 0.19, seed=92),
          lambda: gg.hubs_over_sparse(n_common=5000, hubs=4, p_hub=0.9, avg_deg=6.0, seed=93),
          lambda: gg.csr_from_edges(5, np.zeros(0, np.int32), np.zeros(0, np.int32), "isolated5")]


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
@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_dense_buckets_parity(nd, ctx, gi, r, s):
    g = GRAPHS[gi]()
    for mode in (nd.ND_PEEL_PERSISTENT, nd.ND_PEEL_LOOP_GRAPH, nd.ND_NO_GRAPH):
        assert_parity(nd, ctx, g, r, s, flags=mode | nd.ND_DENSE_BUCKETS)


def test_dense_buckets_with_contraction(nd, ctx):
    g = gg.rmat(12, 16, 0.57, 0.19, 0.19, seed=94)
    for c in (nd.ND_CONTRACT_ALWAYS, 0):
        assert_parity(nd, ctx, g, 2, 3, flags=nd.ND_DENSE_BUCKETS | c)


def test_dense_buckets_int64_counts(nd, ctx):
    g = gg.with_planted(gg.chung_lu(3000, 10.0, 2.3, seed=95), 30, 20, 60, 0.7, seed=96)
    for r, s in [(3, 4), (2, 4)]:
        assert_parity(nd, ctx, g, r, s, count_width=8, flags=nd.ND_DENSE_BUCKETS)
