"""Parity at full size -- R-MAT scale 20 ((2,3), (3,4)) in the launch configuration bench.py
times, and Chung-Lu n = 4,194,304 with 2,000 planted communities ((3,4), (2,4), int64 tallies)
-- where the oracle cannot run the whole peeling loop:

* the validity + elimination-order + level certificate (oracle.certify_all, the Section 2
  definition) over EVERY r-clique for R-MAT 20 (2,3) and for both Chung-Lu 4M decompositions,
  which proves every core number exact; for R-MAT 20 (3,4) (17e9 4-cliques) over a stratified
  sample of more than 1e5 triangles: every triangle whose three lists exceed the heavy-phase
  threshold (4,096 entries), every triangle of the last round (the top level), and 1e5 random
  ones;
* sampled outputs the oracle computes one by one: the s-clique count of sampled r-cliques
  (oracle.local_counts, from the definition of the count);
* properties that hold at any size: canonical order of the r-clique tuples, every sampled tuple
  is an r-clique, sum of round sizes = n_r, levels non-decreasing, core <= count, and the
  statistic sum(count) = C(s,r) n_s.
"""
import math

import numpy as np
import pytest

import graphgen as gg
import oracle as orc

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

SAMPLE_COUNTS = 3000


@pytest.fixture(scope="module")
def big():
    return gg.rmat_scale20(seed=2)


@pytest.fixture(scope="module")
def cl4m():
    return gg.chung_lu_4m_planted(seed=3)


@pytest.fixture(scope="module")
def nd():
    import paper_2111_10980_gb300 as nd

    nd.lib()
    return nd


def neighbours(g, v):
    return g.col[g.rowptr[v]:g.rowptr[v + 1]]


def is_clique(g, t):
    return all(np.isin(t[j], neighbours(g, t[i])) for i in range(len(t)) for j in range(i + 1, len(t)))


def run_full(nd, g, r, s, width=0):
    import torch

    ctx = nd.nd_ctx_create(0)
    rp = torch.from_numpy(g.rowptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    torch.cuda.synchronize()
    G = nd.nd_load_csr(ctx, rp, col)
    import ctypes

    k = ctypes.c_int64()
    assert nd.lib().nd_rcliques(G.ptr, r, None, 0, ctypes.byref(k)) == nd.ND_OK
    n_r = k.value
    core = torch.empty(n_r, dtype=torch.int32, device="cuda")
    rnd = torch.empty(n_r, dtype=torch.int32, device="cuda")
    _, _, st = nd.nd_decompose(G, r, s, count_width=width, core_out=core, round_out=rnd)
    sizes, levels, rho = nd.nd_rounds(G)
    cnt = torch.empty(n_r, dtype=torch.int64, device="cuda")
    _, _, n_s = nd.nd_count(G, r, s, out=cnt)
    tuples = torch.empty((n_r, r), dtype=torch.int32, device="cuda")
    nd.nd_rcliques(G, r, out=tuples)
    edge_support = None
    if r == 3:
        edge_support = torch.empty(g.m, dtype=torch.int64, device="cuda")
        nd.nd_count(G, 2, 3, out=edge_support)
    nd.nd_graph_free(G)
    nd.nd_ctx_destroy(ctx)
    return dict(core=core, round=rnd, st=st, sizes=sizes, levels=levels, rho=rho, count=cnt, n_s=n_s,
                tuples=tuples, n_r=n_r, edge_support=edge_support)


def edge_keys(g):
    """a * n + b for every canonical edge (a < b), ascending (device tensor)."""
    import torch

    e = g.edges().astype(np.int64)
    return torch.from_numpy(e[:, 0] * g.n + e[:, 1]).cuda()


def lex_keys(t, n, ek):
    """Order-preserving int64 keys of ascending r-tuples (device int64 tensor [k, r]): a*n + b for
    r = 2; (rank of edge (a,b)) * n + c for r = 3, which stays below 2^63 for any int32 graph."""
    import torch

    if t.shape[1] == 1:
        return t[:, 0].clone()
    ab = t[:, 0] * n + t[:, 1]
    if t.shape[1] == 2:
        return ab
    rank = torch.searchsorted(ek, ab)
    return rank * n + t[:, 2]


@pytest.mark.parametrize("r,s", [(2, 3), (3, 4)])
def test_rmat_scale20(nd, big, r, s):
    res = check_sampled(nd, big, r, s, 0)
    if (r, s) == (2, 3):
        certify_every(big, r, s, res)
    else:
        certify_stratified(big, res)


@pytest.mark.parametrize("r,s", [(3, 4), (2, 4)])
def test_chung_lu_4m_planted(nd, cl4m, r, s):
    res = check_sampled(nd, cl4m, r, s, 8)
    assert res["st"]["count_width"] == 8
    certify_every(cl4m, r, s, res)


def certify_every(g, r, s, res):
    """The certificate over every r-clique: no validity, order or level failure."""
    core = res["core"].cpu().numpy()
    rnd = res["round"].cpu().numpy()
    out = orc.certify_all(g, r, s, core, rnd, res["levels"])
    assert out["bad_valid"] == 0 and out["bad_order"] == 0 and out["bad_level"] == 0, out


def certify_stratified(g, res):
    """(3,4): the certificate over every heavy triangle, every triangle of the last round and
    1e5 random triangles."""
    import torch

    n_r = res["n_r"]
    t = res["tuples"]
    ek = edge_keys(g)
    # edge supports |N(a) ∩ N(b)| from the (2,3) counts, to find the triangles whose three lists
    # are all longer than the heavy threshold (any source may choose the sample: the certificate
    # does not depend on it)
    sup = res["edge_support"]
    heavy = []
    for lo in range(0, n_r, 1 << 26):
        tt = t[lo:lo + (1 << 26)].to(torch.int64)
        m = None
        for i, j in ((0, 1), (0, 2), (1, 2)):
            e = torch.searchsorted(ek, tt[:, i] * g.n + tt[:, j])
            x = sup[e] > 4096
            m = x if m is None else (m & x)
        heavy.append(torch.nonzero(m).flatten() + lo)
        del tt
    heavy = torch.cat(heavy).cpu().numpy()
    top = torch.nonzero(res["round"] == int(res["rho"]) - 1).flatten().cpu().numpy()
    rng = np.random.default_rng(11)
    ids = np.unique(np.concatenate([heavy, top, rng.integers(0, n_r, 100_000)]))
    assert ids.size > 100_000 and heavy.size > 0
    core = res["core"].cpu().numpy()
    rnd = res["round"].cpu().numpy()
    out = orc.certify_all(g, 3, 4, core, rnd, res["levels"], ids=ids)
    assert out["bad_valid"] == 0 and out["bad_order"] == 0 and out["bad_level"] == 0, out


def check_sampled(nd, g, r, s, width):
    import torch

    res = run_full(nd, g, r, s, width)
    n_r = res["n_r"]
    assert res["st"]["n_r"] == n_r and res["n_s"] == res["st"]["n_s"]
    # properties at any size
    assert int(res["sizes"].sum()) == n_r and res["rho"] == res["st"]["rho"]
    assert np.all(np.diff(res["levels"]) >= 0)
    assert int(res["count"].sum().item()) == math.comb(s, r) * res["n_s"]
    assert bool((res["core"].to(torch.int64) <= res["count"]).all().item())
    assert bool((res["core"] >= 0).all().item())
    ek = edge_keys(g)
    t = res["tuples"].to(torch.int64)
    if r == 3:  # every (a, b) of a triangle must be an edge for the rank key to be exact
        ab = t[:, 0] * g.n + t[:, 1]
        pos = torch.searchsorted(ek, ab)
        assert bool((ek[pos.clamp(max=ek.numel() - 1)] == ab).all().item())
    key = lex_keys(t, g.n, ek)
    del t
    assert bool((key[1:] > key[:-1]).all().item()), "tuples are not in canonical order"
    # sampled counts, one by one from the definition
    rng = np.random.default_rng(7 + r)
    ids = np.unique(rng.integers(0, n_r, size=SAMPLE_COUNTS))
    idt = torch.from_numpy(ids).cuda()
    tup = res["tuples"][idt].cpu().numpy()
    for q in range(0, len(ids), 97):
        assert is_clique(g, tup[q])
    want = orc.local_counts(g, r, s, tup)
    assert np.array_equal(res["count"][idt].cpu().numpy(), want)
    return res
