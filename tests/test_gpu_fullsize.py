"""Parity at full size -- R-MAT scale 20 ((2,3), (3,4)) in the launch configuration bench.py
times, and Chung-Lu n = 4,194,304 with 2,000 planted communities ((3,4), (2,4), int64 tallies)
-- where the oracle cannot run the whole decomposition:

* sampled outputs the oracle computes one by one: the s-clique count of sampled r-cliques
  (oracle.local_counts, from the definition of the count);
* the validity + elimination-order certificate (oracle.certify) on sampled r-cliques, which
  for every checked r-clique confirms that its core number is neither too high nor too low;
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
SAMPLE_CERT = 400


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
    nd.nd_graph_free(G)
    nd.nd_ctx_destroy(ctx)
    return dict(core=core, round=rnd, st=st, sizes=sizes, levels=levels, rho=rho, count=cnt, n_s=n_s,
                tuples=tuples, n_r=n_r)


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
def test_rmat_scale20_sampled(nd, big, r, s):
    check_sampled(nd, big, r, s, 0)


@pytest.mark.parametrize("r,s", [(3, 4), (2, 4)])
def test_chung_lu_4m_planted_sampled(nd, cl4m, r, s):
    st = check_sampled(nd, cl4m, r, s, 8)
    assert st["count_width"] == 8


def sibling_tuples(g, R, r, s):
    """Every r-subset of every s-clique containing R (R ascending), found from the graph."""
    common = neighbours(g, int(R[0]))
    for v in R[1:]:
        common = np.intersect1d(common, neighbours(g, int(v)), assume_unique=True)
    common = common[~np.isin(common, R)]
    out = []
    if s - r == 1:
        completions = [(w,) for w in common]
    else:  # s - r == 2: adjacent pairs inside the common neighbourhood
        completions = []
        for i, w in enumerate(common):
            nw = neighbours(g, int(w))
            for x in common[i + 1:][np.isin(common[i + 1:], nw)]:
                completions.append((w, x))
    for C in completions:
        S = np.sort(np.concatenate([R, np.array(C, R.dtype)]))
        for sub in __import__("itertools").combinations(range(s), r):
            out.append(S[list(sub)])
    return out


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
    # certificate on a smaller sample; sibling ids found by a batched search of the canonical keys
    pick = np.sort(rng.choice(ids.size, size=min(SAMPLE_CERT, ids.size), replace=False))
    cid = ids[pick]
    ctup = tup[pick]
    sib = []
    for R in ctup:
        sib.extend(sibling_tuples(g, R, r, s))
    sib = np.unique(np.array(sib, np.int64).reshape(-1, r), axis=0) if sib else np.zeros((0, r), np.int64)
    sk = lex_keys(torch.from_numpy(sib).cuda(), g.n, ek)
    pos = torch.searchsorted(key, sk)
    assert bool((key[pos.clamp(max=n_r - 1)] == sk).all().item()), "an r-subset of an s-clique is missing"
    lut = {tuple(x): int(p) for x, p in zip(sib.tolist(), pos.cpu().tolist())}
    sel = torch.from_numpy(np.unique(np.concatenate([cid, np.array(list(lut.values()), np.int64)]))).cuda()
    core_s = dict(zip(sel.cpu().tolist(), res["core"][sel].cpu().tolist()))
    rnd_s = dict(zip(sel.cpu().tolist(), res["round"][sel].cpu().tolist()))
    # dense small arrays indexed by position in `sel` for the C checker
    order = sel.cpu().numpy()
    remap = {int(x): i for i, x in enumerate(order)}
    core_small = np.array([core_s[int(x)] for x in order], np.int32)
    rnd_small = np.array([rnd_s[int(x)] for x in order], np.int32)
    sv, so = orc.certify(g, r, s, core_small, rnd_small, np.array([remap[int(i)] for i in cid], np.int64), ctup,
                         lambda tt: remap.get(lut.get(tuple(int(x) for x in tt), -1), -1))
    assert np.all(sv >= core_small[[remap[int(i)] for i in cid]]), "validity fails for a sampled r-clique"
    assert np.all(so <= core_small[[remap[int(i)] for i in cid]]), "elimination order fails for a sampled r-clique"
    return res["st"]
