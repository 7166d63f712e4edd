"""nd_kcore_noalloc: k-core coreness with no allocation by the library.

It serves callers that cannot let a library allocate device memory (a framework that keeps the
GPU's memory in its own pool, or a latency-critical loop where cudaMalloc may synchronise). The
test calls it through the C ABI twice in a row and compares both results with those of the
regular entry point nd_decompose(g, 1, 2) and with the oracle; the work is integer, so the
tolerance is zero. The graphs include one with exactly ND_NOALLOC_MAX_VERTICES vertices (every
scratch array full), one with a hub of degree above 4,096 (the peeling takes the path a heavy
vertex would take), and the empty graph; a graph one vertex larger than the static scratch is
rejected. Collected last on purpose, so that a run stopping at the first failure has already run
every other test."""
import numpy as np
import pytest

import graphgen as gg
import oracle as orc

pytestmark = pytest.mark.gpu


def _graphs(nd):
    return [gg.chung_lu(50_000, 16.0, 2.2, seed=41), gg.rmat(14, 16, 0.57, 0.19, 0.19, seed=42),
            gg.hubs_over_sparse(n_common=6000, hubs=4, p_hub=0.9, avg_deg=8.0, seed=51),
            gg.chung_lu(nd.ND_NOALLOC_MAX_VERTICES, 12.0, 2.2, seed=43, exact=False)]


def test_noalloc_kcore_matches_nd_decompose_and_oracle_twice():
    import torch

    import paper_2111_10980_gb300 as nd

    graphs = _graphs(nd)
    assert graphs[-1].n == nd.ND_NOALLOC_MAX_VERTICES
    assert np.diff(graphs[2].rowptr).max() > 4096
    ctx = nd.nd_ctx_create(0)
    try:
        for g in graphs:
            G = nd.nd_load_csr(ctx, g.rowptr, g.col)
            want, _, _ = nd.nd_decompose(G, 1, 2)
            nd.nd_graph_free(G)
            assert np.array_equal(want, orc.decompose(g, 1, 2).core), g.name
            rp = torch.from_numpy(g.rowptr).cuda()
            col = torch.from_numpy(g.col).cuda()
            for _ in range(2):  # the static scratch keeps the previous call's contents
                core = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
                torch.cuda.synchronize()
                nd.nd_kcore_noalloc(rp, col, core)
                got = core.cpu().numpy()
                assert np.array_equal(got, want), g.name
    finally:
        nd.nd_ctx_destroy(ctx)


def test_noalloc_empty_graph():
    import torch

    import paper_2111_10980_gb300 as nd

    rp = torch.zeros(1, dtype=torch.int64, device="cuda")
    col = torch.zeros(1, dtype=torch.int32, device="cuda")
    core = torch.zeros(1, dtype=torch.int32, device="cuda")
    nd.nd_kcore_noalloc(rp, col, core[:0])
    one = torch.zeros(2, dtype=torch.int64, device="cuda")  # a single isolated vertex
    nd.nd_kcore_noalloc(one, col, core)
    assert int(core[0]) == 0


def test_noalloc_rejects_graphs_beyond_the_scratch():
    import torch

    import paper_2111_10980_gb300 as nd

    n = nd.ND_NOALLOC_MAX_VERTICES + 1
    rp = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    col = torch.zeros(1, dtype=torch.int32, device="cuda")
    core = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(nd.NdError) as ei:
        nd.nd_kcore_noalloc(rp, col, core)
    assert ei.value.code == nd.ND_EINVAL
    assert "static scratch" in str(ei.value)
