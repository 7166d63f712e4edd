"""Connected nuclei (Section 2, footnote): the components, through s-cliques whose r-subsets all
have core >= c, of the r-cliques with core >= c. The library's labels (smallest id of each
component, -1 outside) and component counts are compared with the oracle's sequential union-find
element by element, at every level of each decomposition, for every supported (r,s), on host and
device pointers, including disjoint unions (components that must stay apart) and graphs with hubs.
The core arrays given to both sides are the oracle's."""
import numpy as np
import pytest

import graphgen as gg
import oracle as orc

pytestmark = pytest.mark.gpu

RS = [(1, 2), (1, 3), (1, 4), (2, 3), (2, 4), (2, 5), (3, 4), (3, 5), (3, 6), (4, 5), (4, 6)]


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


def levels_of(core, cap=12):
    """0, every distinct core value (capped to `cap` of them, spread evenly) and max + 1."""
    vals = np.unique(core) if core.size else np.zeros(0, np.int64)
    if vals.size > cap:
        vals = vals[np.linspace(0, vals.size - 1, cap).astype(np.int64)]
    top = int(core.max()) + 1 if core.size else 1
    return sorted({0, top, *[int(v) for v in vals]})


def check(nd, ctx, g, r, s, device=False, cap=12):
    core = orc.decompose(g, r, s).core.astype(np.int32)
    G = nd.nd_load_csr(ctx, g.rowptr, g.col, flags=nd.ND_VALIDATE)
    try:
        for c in levels_of(core, cap):
            want, nw = orc.nuclei(g, r, s, core, c)
            if device:
                import torch

                got, ng = nd.nd_nuclei(G, r, s, torch.from_numpy(core).cuda(), c)
                got = got.cpu().numpy()
            else:
                got, ng = nd.nd_nuclei(G, r, s, core, c)
            assert ng == nw, (r, s, c, ng, nw)
            np.testing.assert_array_equal(got, want, err_msg=f"(r,s)=({r},{s}) level {c}")
    finally:
        nd.nd_graph_free(G)


@pytest.mark.parametrize("r,s", RS)
def test_small_graphs(nd, ctx, r, s):
    check(nd, ctx, gg.fig1(), r, s)
    check(nd, ctx, gg.disjoint_union(gg.complete(7), gg.fig1(), gg.complete(s), gg.complete(s + 2)), r, s)
    for seed in range(6):
        check(nd, ctx, gg.gnp(10 + 4 * seed, [0.3, 0.5, 0.7][seed % 3], 9100 + seed), r, s)


@pytest.mark.parametrize("r,s", RS)
def test_power_law_and_communities(nd, ctx, r, s):
    check(nd, ctx, gg.with_planted(gg.chung_lu(1200, 5.0, 2.3, seed=9201), 10, 8, 20, 0.7, seed=9202), r, s)
    if s - r == 1:
        check(nd, ctx, gg.rmat(11, 8, seed=9203), r, s, device=True)
    elif s - r == 2:
        check(nd, ctx, gg.rmat(9, 8, seed=9204), r, s, device=True)


@pytest.mark.parametrize("r,s,scale,ef", [(1, 2, 14, 16), (2, 3, 14, 8), (2, 4, 12, 8), (3, 4, 12, 8)])
def test_larger_graphs(nd, ctx, r, s, scale, ef):
    # 10^4 to 10^5 r-cliques; hubs whose r-cliques list long neighbourhoods
    check(nd, ctx, gg.rmat(scale, ef, seed=9301), r, s, device=True, cap=6)
    check(nd, ctx, gg.hubs_over_sparse(n_common=4000, hubs=4, p_hub=0.9, avg_deg=4.0, seed=9302), r, s)


def test_empty_and_edgeless(nd, ctx):
    for g in (gg.complete(1), gg.gnp(30, 0.0, 1)):
        for r, s in [(1, 2), (2, 3), (3, 4)]:
            check(nd, ctx, g, r, s)


def test_bad_arguments(nd, ctx):
    g = gg.fig1()
    G = nd.nd_load_csr(ctx, g.rowptr, g.col)
    try:
        core = np.zeros(g.n, np.int32)
        with pytest.raises(nd.NdError):
            nd.nd_nuclei(G, 4, 7, core, 0)
        with pytest.raises(ValueError):
            import torch

            nd.nd_nuclei(G, 1, 2, core, 0, out=torch.zeros(g.n, dtype=torch.int32, device="cuda"))
    finally:
        nd.nd_graph_free(G)


def check_hierarchy(nd, ctx, g, r, s, device=False):
    core = orc.decompose(g, r, s).core.astype(np.int32)
    want = orc.hierarchy(g, r, s, core)
    G = nd.nd_load_csr(ctx, g.rowptr, g.col, flags=nd.ND_VALIDATE)
    try:
        if device:
            import torch

            got = nd.nd_hierarchy(G, r, s, torch.from_numpy(core).cuda())
            got = [x.cpu().numpy() for x in got[:3]] + [got[3]]
        else:
            got = nd.nd_hierarchy(G, r, s, core)
        for name, a, b in zip(("comp", "parent_level", "parent_comp"), got[:3], want):
            np.testing.assert_array_equal(a, b, err_msg=f"(r,s)=({r},{s}) {name}")
        nodes = {(int(c), int(x)) for c, x in zip(core, want[0])}
        assert got[3] == len(nodes)
    finally:
        nd.nd_graph_free(G)


@pytest.mark.parametrize("r,s", RS)
def test_hierarchy_small_graphs(nd, ctx, r, s):
    check_hierarchy(nd, ctx, gg.fig1(), r, s)
    check_hierarchy(nd, ctx, gg.disjoint_union(gg.complete(7), gg.fig1(), gg.complete(s), gg.complete(s + 2)), r, s)
    for seed in range(4):
        check_hierarchy(nd, ctx, gg.gnp(10 + 4 * seed, [0.3, 0.5, 0.7][seed % 3], 9400 + seed), r, s, device=seed % 2 == 1)


@pytest.mark.parametrize("r,s", [(1, 2), (2, 3), (2, 4), (3, 4)])
def test_hierarchy_power_law_and_hubs(nd, ctx, r, s):
    check_hierarchy(nd, ctx, gg.with_planted(gg.chung_lu(1200, 5.0, 2.3, seed=9501), 10, 8, 20, 0.7, seed=9502), r, s)
    check_hierarchy(nd, ctx, gg.hubs_over_sparse(n_common=1500, hubs=3, p_hub=0.9, avg_deg=4.0, seed=9503), r, s,
                    device=True)
    if s - r == 1:
        check_hierarchy(nd, ctx, gg.rmat(11, 8, seed=9504), r, s)


def test_hierarchy_empty_and_bad_core(nd, ctx):
    g = gg.gnp(30, 0.0, 1)
    check_hierarchy(nd, ctx, g, 2, 3)  # no edges: nothing to build
    check_hierarchy(nd, ctx, g, 1, 2)  # isolated vertices: one root node each
    G = nd.nd_load_csr(ctx, g.rowptr, g.col)
    try:
        with pytest.raises(nd.NdError):
            nd.nd_hierarchy(G, 1, 2, np.full(g.n, -1, np.int32))
        with pytest.raises(nd.NdError):
            nd.nd_hierarchy(G, 4, 7, np.zeros(g.n, np.int32))
    finally:
        nd.nd_graph_free(G)
