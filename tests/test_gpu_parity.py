"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, bit for bit.

Compared element by element: core numbers, the peel round of every r-clique, rho, the
per-round |A| and level k, the s-clique counts and the r-clique tuples (canonical order).
Graphs span several warps/blocks and ragged tails, plus the degenerate cases (no vertices, no
edges, no triangles, a single edge, stars, complete graphs).
"""
import math

import numpy as np
import pytest

import graphgen as gg
import oracle as orc

pytestmark = pytest.mark.gpu

RS = [(1, 2), (1, 3), (2, 3), (2, 4), (3, 4)]


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


def run_gpu(nd, ctx, g, r, s, flags=0, count_width=0, orient=None):
    G = nd.nd_load_csr(ctx, g.rowptr, g.col, flags=nd.ND_VALIDATE)
    try:
        if orient is not None:
            nd.nd_orient(G, orient)
        core, rnd, st = nd.nd_decompose(G, r, s, count_width=count_width, flags=flags)
        sizes, levels, rho = nd.nd_rounds(G)
        counts, n_r, n_s = nd.nd_count(G, r, s, count_width=8)
        tuples = nd.nd_rcliques(G, r)
    finally:
        nd.nd_graph_free(G)
    return dict(core=core, round=rnd, st=st, sizes=sizes, levels=levels, rho=rho, counts=counts, n_r=n_r, n_s=n_s,
                tuples=tuples)


def assert_parity(nd, ctx, g, r, s, **kw):
    want = orc.decompose(g, r, s)
    wcounts, wn_s = orc.count(g, r, s)
    got = run_gpu(nd, ctx, g, r, s, **kw)
    tag = f"{g.name} ({r},{s})"
    assert got["n_r"] == want.core.size, tag
    assert np.array_equal(got["tuples"].reshape(-1, r), orc.list_cliques(g, r).reshape(-1, r)), tag
    assert got["n_s"] == wn_s, tag
    assert np.array_equal(got["counts"], wcounts), tag
    assert np.array_equal(got["core"], want.core), tag
    assert np.array_equal(got["round"], want.round), tag
    assert got["rho"] == want.rho and got["st"]["rho"] == want.rho, tag
    assert np.array_equal(got["sizes"], want.sizes), tag
    assert np.array_equal(got["levels"], want.levels), tag
    assert got["st"]["n_s"] == wn_s and got["st"]["n_r"] == want.core.size, tag
    assert got["st"]["listed"] == wn_s, tag  # every s-clique destroyed exactly once
    assert got["st"]["decrements"] == want.decs, tag
    if want.core.size:
        assert got["st"]["max_core"] == int(want.core.max()), tag
    return got


@pytest.mark.parametrize("r,s", RS)
def test_figure1(nd, ctx, r, s):
    assert_parity(nd, ctx, gg.fig1(), r, s)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 9, 33])
def test_complete_graphs(nd, ctx, n):
    g = gg.complete(n)
    for r, s in RS:
        got = assert_parity(nd, ctx, g, r, s)
        if s <= n:
            assert np.all(got["core"] == math.comb(n - r, s - r))
            assert got["rho"] == 1


@pytest.mark.parametrize("r,s", RS)
def test_random_small_graphs(nd, ctx, r, s):
    for seed in range(25):
        n = 6 + (seed * 7) % 30
        p = [0.2, 0.4, 0.6, 0.85][seed % 4]
        assert_parity(nd, ctx, gg.gnp(n, p, 5000 + seed), r, s)


@pytest.mark.parametrize("r,s", RS)
def test_chung_lu_2k_workload(nd, ctx, r, s):
    """The n = 2,000 power-law workload (avg degree 20, exponent 2.1, max expected degree 200)."""
    assert_parity(nd, ctx, gg.chung_lu_2k(), r, s)


@pytest.mark.parametrize("r,s", RS)
def test_power_law_and_rmat(nd, ctx, r, s):
    assert_parity(nd, ctx, gg.chung_lu(3000, 24.0, 2.2, seed=17), r, s)
    assert_parity(nd, ctx, gg.rmat(11, 16, 0.57, 0.19, 0.19, seed=3), r, s)


@pytest.mark.parametrize("r,s", [(2, 3), (3, 4), (2, 4)])
def test_planted_communities(nd, ctx, r, s):
    base = gg.chung_lu(4000, 10.0, 2.3, seed=8)
    g = gg.with_planted(base, 40, 20, 60, 0.7, seed=9)
    assert_parity(nd, ctx, g, r, s)


def test_degenerate_graphs(nd, ctx):
    empty = gg.csr_from_edges(0, np.zeros(0, np.int32), np.zeros(0, np.int32), "empty")
    isolated = gg.csr_from_edges(5, np.zeros(0, np.int32), np.zeros(0, np.int32), "isolated5")
    single = gg.csr_from_edges(2, np.array([0], np.int32), np.array([1], np.int32), "K2")
    star = gg.csr_from_edges(40, np.zeros(39, np.int32), np.arange(1, 40, dtype=np.int32), "star40")
    bip = gg.csr_from_edges(60, np.repeat(np.arange(30), 30).astype(np.int32),
                            np.tile(np.arange(30, 60), 30).astype(np.int32), "K30,30")
    for g in [empty, isolated, single, star, bip]:
        for r, s in RS:
            assert_parity(nd, ctx, g, r, s)


@pytest.mark.parametrize("r,s", RS)
def test_count_width_and_launch_modes_agree(nd, ctx, r, s):
    g = gg.chung_lu(1500, 18.0, 2.1, seed=23)
    want = orc.decompose(g, r, s)
    for kw in [dict(count_width=4), dict(count_width=8), dict(flags=nd.ND_NO_GRAPH),
               dict(flags=nd.ND_PEEL_LOOP_GRAPH), dict(flags=nd.ND_PEEL_PERSISTENT),
               dict(orient=nd.ND_ORIENT_DEGENERACY)]:
        got = run_gpu(nd, ctx, g, r, s, **kw)
        assert np.array_equal(got["core"], want.core), kw
        assert np.array_equal(got["round"], want.round), kw
        assert got["rho"] == want.rho, kw
        assert got["st"]["listed"] == want.n_s, kw


@pytest.mark.parametrize("mode", ["NO_GRAPH", "PEEL_LOOP_GRAPH", "PEEL_PERSISTENT"])
def test_launch_modes_on_rmat(nd, ctx, mode):
    """Every way of launching the peeling rounds gives the oracle's result, rounds included."""
    g = gg.rmat(12, 16, 0.57, 0.19, 0.19, seed=6)
    for r, s in [(2, 3), (3, 4), (1, 2)]:
        assert_parity(nd, ctx, g, r, s, flags=getattr(nd, "ND_" + mode))


def test_determinism(nd, ctx):
    g = gg.rmat(12, 16, 0.57, 0.19, 0.19, seed=4)
    first = run_gpu(nd, ctx, g, 3, 4)
    for _ in range(3):
        again = run_gpu(nd, ctx, g, 3, 4)
        assert np.array_equal(again["core"], first["core"])
        assert np.array_equal(again["round"], first["round"])


def test_device_pointers_and_torch_allocator(nd):
    import torch

    g = gg.chung_lu(2500, 16.0, 2.2, seed=29)
    want = orc.decompose(g, 2, 3)
    stream = torch.cuda.Stream()
    ctx = nd.nd_ctx_create(0, stream=stream)
    alloc, free = nd.torch_allocator_hooks(0)
    nd.nd_ctx_set_allocator(ctx, alloc, free)
    rp = torch.from_numpy(g.rowptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    torch.cuda.synchronize()
    G = nd.nd_load_csr(ctx, rp, col)
    core = torch.zeros(g.m, dtype=torch.int32, device="cuda")
    rnd = torch.zeros(g.m, dtype=torch.int32, device="cuda")
    nd.nd_decompose(G, 2, 3, core_out=core, round_out=rnd)
    assert np.array_equal(core.cpu().numpy(), want.core)
    assert np.array_equal(rnd.cpu().numpy(), want.round)
    assert nd.nd_ctx_bytes_in_use(ctx) > 0
    nd.nd_graph_free(G)
    assert nd.nd_ctx_bytes_in_use(ctx) == 0
    nd.nd_ctx_destroy(ctx)


def test_errors_are_reported(nd, ctx):
    g = gg.fig1()
    bad = g.col.copy()
    bad[[0, 1]] = bad[[1, 0]]  # row 0 no longer ascending
    with pytest.raises(nd.NdError) as ei:
        nd.nd_load_csr(ctx, g.rowptr, bad, flags=nd.ND_VALIDATE)
    assert ei.value.code == nd.ND_EINVAL
    asym = gg.csr_from_edges(3, np.array([0, 1], np.int32), np.array([1, 2], np.int32))
    col = asym.col.copy()
    col[-1] = 0  # vertex 2 lists 0 instead of 1
    with pytest.raises(nd.NdError):
        nd.nd_load_csr(ctx, asym.rowptr, col, flags=nd.ND_VALIDATE)
    G = nd.nd_load_csr(ctx, g.rowptr, g.col)
    for r, s in [(4, 7), (2, 6), (5, 6)]:
        with pytest.raises(nd.NdError) as ei:
            nd.nd_decompose(G, r, s)
        assert ei.value.code == nd.ND_EINVAL
    nd.nd_graph_free(G)
    small = nd.nd_ctx_create(0, mem_budget=1 << 12)
    with pytest.raises(nd.NdError) as ei:
        nd.nd_load_csr(small, gg.complete(60).rowptr, gg.complete(60).col)
    assert ei.value.code == nd.ND_ENOMEM
    nd.nd_ctx_destroy(small)


def test_phase_and_round_times(nd, ctx):
    """The persistent kernel's timing record: per-phase times add up to at most the peel's time,
    the per-round Update times add up to the Update phases, and every round is accounted for."""
    g = gg.rmat(12, 16, 0.57, 0.19, 0.19, seed=5)
    G = nd.nd_load_csr(ctx, g.rowptr, g.col)
    try:
        for r, s in [(2, 3), (3, 4)]:
            _, _, st = nd.nd_decompose(G, r, s, flags=nd.ND_PEEL_PERSISTENT)
            ph = st["t_phase_ms"]
            assert len(ph) == 6 and min(ph) >= 0.0
            assert 0.0 < sum(ph) <= st["t_peel_ms"] * 1.05
            sizes, _, rho = nd.nd_rounds(G)
            ns = nd.nd_round_times(G)
            assert ns.size == rho == sizes.size
            assert (ns >= 0).all()
            assert abs(ns.sum() / 1e6 - (ph[4] + ph[5])) <= 1e-3 * max(1.0, ph[4] + ph[5]) + 1e-3
            _, _, st = nd.nd_decompose(G, r, s, flags=nd.ND_NO_GRAPH)
            assert sum(st["t_phase_ms"]) == 0.0 and not nd.nd_round_times(G).any()
    finally:
        nd.nd_graph_free(G)


def test_34_without_room_for_the_hash_directory(nd):
    """When the lists' hash directory cannot be allocated (here: an allocator that refuses any
    block above 16 MB, which only the directory's tables reach), (3,4) runs with bisection and
    still gives the oracle's result."""
    import torch

    g = gg.rmat(12, 16, 0.57, 0.19, 0.19, seed=9)
    want = orc.decompose(g, 3, 4)
    alloc, free = nd.torch_allocator_hooks(0)
    refused = []

    def small_only(nbytes, stream):
        if nbytes > 16 << 20:
            refused.append(nbytes)
            return 0
        return alloc(nbytes, stream)

    stream = torch.cuda.Stream()
    ctx = nd.nd_ctx_create(0, stream=stream)
    nd.nd_ctx_set_allocator(ctx, small_only, free)
    G = nd.nd_load_csr(ctx, g.rowptr, g.col)
    try:
        core, rnd, st = nd.nd_decompose(G, 3, 4)
    finally:
        nd.nd_graph_free(G)
        nd.nd_ctx_destroy(ctx)
    assert refused, "the directory should not have fitted"
    assert np.array_equal(core, want.core) and np.array_equal(rnd, want.round)
    assert st["listed"] == want.n_s and st["decrements"] == want.decs
