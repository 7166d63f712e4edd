"""Pins for the CPU oracle: it is checked against things other than itself.

* the worked example of the paper (Figure 1, Section 4.2 Example, Figure 2 bucket contents);
* closed forms: in K_n every r-clique lies in C(n-r, s-r) s-cliques and that is its core
  number, reached in one round; disjoint unions of cliques and paths;
* textbook special cases: (1,2) = k-core coreness (networkx ``core_number``) and
  (2,3) = k-truss trussness - 2 (networkx ``k_truss``), Section 2;
* brute force: the maximal c-(r,s) nucleus as the union of all feasible subsets of
  r-cliques, enumerated exhaustively on tiny graphs (definition of Section 2);
* invariants: sum of counts = C(s,r) n_s, n_3 = trace(A^3)/6, clique totals against
  networkx, 0 <= core <= count, invariance under vertex relabelling;
* the two oracle algorithms (Algorithm 2 peeling with exact 1/a, and the definition's
  nested fixpoints) against each other on 1,200 seeded random graphs;
* the certificate checker accepts the oracle's results and rejects perturbed ones.
"""
import itertools
import math

import networkx as nx
import numpy as np
import pytest

import graphgen as gg
import oracle as orc
from golden_io import load

RS_ALL = [(r, s) for s in range(2, 6) for r in range(1, s)]


def to_nx(g):
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    G.add_edges_from(map(tuple, g.edges().tolist()))
    return G


def py_cliques(g, c):
    """Brute force: every c-subset of vertices that is pairwise adjacent (lexicographic)."""
    adj = [set(g.col[g.rowptr[v]:g.rowptr[v + 1]].tolist()) for v in range(g.n)]
    out = []
    for t in itertools.combinations(range(g.n), c):
        if all(b in adj[a] for a, b in itertools.combinations(t, 2)):
            out.append(t)
    return out


# ------------------------------------------------------------------------------------
# Worked example

@pytest.mark.parametrize("name", ["fig1_34.txt", "fig1_23.txt", "fig1_24.txt", "fig1_12.txt", "fig1_13.txt",
                                  "fig1_14.txt"])
def test_figure1_worked_example(name):
    gold = load(name)
    g = gg.fig1()
    r, s = gold["r"], gold["s"]
    tuples = orc.list_cliques(g, r)
    assert np.array_equal(tuples, gold["tuples"]), "canonical r-clique order"
    counts, n_s = orc.count(g, r, s)
    assert n_s == gold["n_s"]
    assert np.array_equal(counts, gold["count"])
    d = orc.decompose(g, r, s)
    assert d.rho == gold["rho"]
    assert d.sizes.tolist() == gold["sizes"]
    assert d.levels.tolist() == gold["levels"]
    assert np.array_equal(d.core, gold["core"])
    assert np.array_equal(d.round, gold["round"])
    assert d.decs == gold["decs"]
    assert np.array_equal(orc.decompose_fixpoint(g, r, s), gold["core"])


def test_figure1_graph_shape():
    g = gg.fig1()
    assert g.n == 7 and g.m == 15
    assert len(orc.list_cliques(g, 3)) == 14  # "14 total triangles" (Example, Section 4.2)
    assert len(orc.list_cliques(g, 4)) == 6


# ------------------------------------------------------------------------------------
# Closed forms

@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7, 9, 12])
def test_complete_graph_closed_form(n):
    g = gg.complete(n)
    for r, s in RS_ALL:
        if s > n:
            continue
        want = math.comb(n - r, s - r)
        counts, n_s = orc.count(g, r, s)
        assert n_s == math.comb(n, s)
        assert counts.size == math.comb(n, r)
        assert np.all(counts == want)
        d = orc.decompose(g, r, s)
        assert np.all(d.core == want), (n, r, s)
        assert d.rho == 1
        assert np.all(orc.decompose_fixpoint(g, r, s) == want)


@pytest.mark.parametrize("n,r,s", [(30, 1, 2), (30, 2, 3), (20, 2, 4), (16, 3, 4), (14, 3, 5), (12, 4, 5)])
def test_complete_graph_larger(n, r, s):
    d = orc.decompose(gg.complete(n), r, s)
    assert np.all(d.core == math.comb(n - r, s - r)) and d.rho == 1


def test_disjoint_cliques_and_paths():
    sizes = [3, 4, 5, 6, 8]
    parts = [gg.complete(k) for k in sizes] + [gg.path(6), gg.path(2)]
    g = gg.disjoint_union(*parts)
    for r, s in [(1, 2), (1, 3), (2, 3), (2, 4), (3, 4), (3, 5)]:
        tuples = orc.list_cliques(g, r)
        d = orc.decompose(g, r, s)
        want = np.zeros(len(tuples), np.int64)
        off = 0
        bounds = []
        for k in sizes:
            bounds.append((off, off + k, math.comb(k - r, s - r) if k >= s else 0))
            off += k
        for i, t in enumerate(tuples):
            for lo, hi, val in bounds:
                if lo <= t[0] < hi:
                    want[i] = val
        if r == 1:
            # path vertices: coreness 1 for (1,2) (every path vertex has an edge), 0 otherwise
            path_lo = sum(sizes)
            for i, t in enumerate(tuples):
                if t[0] >= path_lo:
                    want[i] = 1 if s == 2 else 0
        elif r == 2 and s == 3:
            pass  # path edges lie in no triangle: 0 (already)
        assert np.array_equal(d.core, want), (r, s)
        if (r, s) != (1, 2):
            # every level is peeled in exactly one round (the path in (1,2) needs one round
            # per vertex pair it sheds, so it is left out)
            assert d.rho == len(set(want.tolist())), (r, s, d.levels)


# ------------------------------------------------------------------------------------
# Textbook special cases

@pytest.mark.parametrize("seed", [1, 2, 3])
def test_12_equals_networkx_core_number(seed):
    g = gg.chung_lu(400, 12.0, 2.2, seed=seed)
    d = orc.decompose(g, 1, 2)
    cn = nx.core_number(to_nx(g))
    assert np.array_equal(d.core, np.array([cn[v] for v in range(g.n)]))


def test_12_config_graph_equals_networkx():
    g = gg.chung_lu_2k()
    d = orc.decompose(g, 1, 2)
    cn = nx.core_number(to_nx(g))
    assert np.array_equal(d.core, np.array([cn[v] for v in range(g.n)]))


def _trussness(G):
    """Classic trussness via networkx.k_truss: the largest k such that the edge survives in
    the k-truss (every edge in >= k-2 triangles of the subgraph)."""
    truss = {tuple(sorted(e)): 2 for e in G.edges()}
    k = 3
    H = G
    while H.number_of_edges() > 0:
        H = nx.k_truss(H, k)
        for e in H.edges():
            truss[tuple(sorted(e))] = k
        k += 1
    return truss


@pytest.mark.parametrize("seed", [1, 2])
def test_23_equals_networkx_truss_minus_two(seed):
    g = gg.chung_lu(300, 14.0, 2.2, seed=seed)
    d = orc.decompose(g, 2, 3)
    truss = _trussness(to_nx(g))
    edges = orc.list_cliques(g, 2)
    want = np.array([truss[(int(a), int(b))] - 2 for a, b in edges])
    assert np.array_equal(d.core, want)


# ------------------------------------------------------------------------------------
# Brute force over all subsets of r-cliques (definition of Section 2)

def brute_force_cores(g, r, s):
    rcl = py_cliques(g, r)
    idx = {t: i for i, t in enumerate(rcl)}
    nr = len(rcl)
    smasks = []
    for S in py_cliques(g, s):
        mask = 0
        for sub in itertools.combinations(S, r):
            mask |= 1 << idx[sub]
        smasks.append(mask)
    core = np.zeros(nr, np.int64)
    if nr == 0:
        return core
    maxc = len(smasks)
    for c in range(1, maxc + 1):
        union = 0
        for X in range(1, 1 << nr):
            ok = True
            for i in range(nr):
                if X >> i & 1:
                    sup = sum(1 for m in smasks if (m >> i & 1) and (m & X) == m)
                    if sup < c:
                        ok = False
                        break
            if ok:
                union |= X
        if union == 0:
            break
        for i in range(nr):
            if union >> i & 1:
                core[i] = c
    return core


def _tiny_graphs():
    out = [gg.fig1()]
    for seed in range(40):
        g = gg.gnp(6, 0.7, 1000 + seed)
        out.append(g)
    return out


@pytest.mark.parametrize("r,s", [(1, 2), (1, 3), (2, 3), (2, 4), (3, 4)])
def test_brute_force_subsets(r, s):
    checked = 0
    for g in _tiny_graphs():
        nr = len(py_cliques(g, r))
        if nr == 0 or nr > 12:
            continue
        want = brute_force_cores(g, r, s)
        d = orc.decompose(g, r, s)
        assert np.array_equal(d.core, want), (g.name, r, s)
        checked += 1
    assert checked >= 5


def test_brute_force_figure1_edges():
    g = gg.fig1()
    for s in (3, 4):
        assert np.array_equal(orc.decompose(g, 2, s).core, brute_force_cores(g, 2, s))


# ------------------------------------------------------------------------------------
# Invariants

@pytest.mark.parametrize("seed", [7, 8, 9])
def test_count_invariants(seed):
    g = gg.chung_lu(250, 16.0, 2.1, seed=seed)
    G = to_nx(g)
    A = nx.to_numpy_array(G, nodelist=range(g.n), dtype=np.int64)
    n3 = int(np.trace(A @ A @ A)) // 6
    assert len(orc.list_cliques(g, 3)) == n3
    totals = {}
    for cl in nx.enumerate_all_cliques(G):
        totals[len(cl)] = totals.get(len(cl), 0) + 1
    for c in range(1, 6):
        assert len(orc.list_cliques(g, c)) == totals.get(c, 0)
    for r, s in RS_ALL:
        counts, n_s = orc.count(g, r, s)
        assert n_s == totals.get(s, 0)
        assert int(counts.sum()) == math.comb(s, r) * n_s
        d = orc.decompose(g, r, s)
        assert np.all(d.core >= 0) and np.all(d.core <= counts)
        # levels never decrease; each round is non-empty
        assert np.all(np.diff(d.levels) >= 0) and np.all(d.sizes > 0)
        assert int(d.sizes.sum()) == counts.size
        # every re-listing of Update is one (s-clique, member r-clique) pair
        assert d.listed == math.comb(s, r) * n_s
        # an s-clique is live for the first round that peels any of its members, and for every
        # member peeled in that round: at least n_s and at most the listings
        assert n_s <= d.live <= d.listed
        # every s-clique is destroyed exactly once, lowering each member that survives that round
        # by exactly one: the decrements equal the counts taken by surviving members
        assert d.decs <= (math.comb(s, r) - 1) * n_s


def test_relabel_invariance():
    g = gg.chung_lu(200, 14.0, 2.2, seed=11)
    perm = np.random.default_rng(5).permutation(g.n).astype(np.int32)
    h = gg.relabel(g, perm)
    for r, s in [(1, 2), (2, 3), (2, 4), (3, 4)]:
        dg, dh = orc.decompose(g, r, s), orc.decompose(h, r, s)
        tg = orc.list_cliques(g, r)
        th = orc.list_cliques(h, r)
        pos = {tuple(t): i for i, t in enumerate(th.tolist())}
        mapped = [pos[tuple(sorted(perm[t].tolist()))] for t in tg]
        assert np.array_equal(dg.core, dh.core[mapped])
        assert np.array_equal(dg.round, dh.round[mapped])
        assert dg.rho == dh.rho


@pytest.mark.parametrize("r,s", RS_ALL)
def test_rounds_match_definition_on_random_graphs(r, s):
    """Algorithm 2's peeling (exact 1/a) and the definition's fixpoints agree."""
    for seed in range(120):
        n = 5 + seed % 6
        p = [0.3, 0.5, 0.7, 0.9][seed % 4]
        g = gg.gnp(n, p, 77 + 1000 * r + 100 * s + seed)
        d = orc.decompose(g, r, s)
        fp = orc.decompose_fixpoint(g, r, s)
        assert np.array_equal(d.core, fp), (seed, r, s)


@pytest.mark.parametrize("r,s", [(1, 2), (2, 3), (2, 4), (3, 4), (3, 5), (4, 5)])
def test_rounds_match_definition_on_power_law(r, s):
    g = gg.chung_lu(150, 12.0, 2.1, seed=r * 10 + s)
    assert np.array_equal(orc.decompose(g, r, s).core, orc.decompose_fixpoint(g, r, s))


def test_s_up_to_7():
    g = gg.disjoint_union(gg.complete(9), gg.gnp(9, 0.8, 3))
    for r, s in [(1, 7), (3, 7), (6, 7), (5, 6)]:
        d = orc.decompose(g, r, s)
        assert np.array_equal(d.core, orc.decompose_fixpoint(g, r, s))
        assert np.all(d.core[: math.comb(9, r)] == math.comb(9 - r, s - r))


# ------------------------------------------------------------------------------------
# Sampled checks used at full size

def test_local_counts_match_count():
    g = gg.chung_lu(300, 14.0, 2.2, seed=21)
    for r, s in [(1, 3), (2, 3), (2, 4), (3, 4)]:
        counts, _ = orc.count(g, r, s)
        tuples = orc.list_cliques(g, r)
        assert np.array_equal(orc.local_counts(g, r, s, tuples), counts)


def _lookup_for(g, r):
    tuples = orc.list_cliques(g, r)
    pos = {tuple(t): i for i, t in enumerate(tuples.tolist())}
    return tuples, (lambda t: pos.get(tuple(t), -1))


@pytest.mark.parametrize("r,s", [(1, 2), (2, 3), (2, 4), (3, 4)])
def test_certificate_accepts_oracle_and_rejects_perturbations(r, s):
    g = gg.chung_lu(250, 14.0, 2.2, seed=31)
    d = orc.decompose(g, r, s)
    tuples, lookup = _lookup_for(g, r)
    ids = np.arange(tuples.shape[0])
    sv, so = orc.certify(g, r, s, d.core, d.round, ids, tuples, lookup)
    assert np.all(sv >= d.core) and np.all(so <= d.core)
    # raising one core number breaks validity; lowering one breaks the order condition
    i = int(np.argmax(d.core))
    bad = d.core.copy()
    bad[i] += 1
    sv2, _ = orc.certify(g, r, s, bad, d.round, ids[i:i + 1], tuples[i:i + 1], lookup)
    assert sv2[0] < bad[i]
    tight = np.nonzero((so == d.core) & (d.core > 0))[0]
    assert tight.size > 0
    j = int(tight[0])
    bad = d.core.copy()
    bad[j] -= 1
    _, so2 = orc.certify(g, r, s, bad, d.round, ids[j:j + 1], tuples[j:j + 1], lookup)
    assert so2[0] > bad[j]


# ------------------------------------------------------------------------------------
# The parallel certificate (certify_all): its supports against brute force over the
# s-cliques, acceptance of the oracle's decomposition, rejection of perturbed claims.

def _brute_supports(g, r, s, core, rnd):
    """Per r-clique (canonical order): #{S containing R : min core over S's r-subsets >=
    core[R]} and #{S containing R : min round over S's r-subsets >= round[R]}, from every
    pairwise-adjacent vertex subset of size s."""
    rcl = py_cliques(g, r)
    pos = {t: i for i, t in enumerate(rcl)}
    sv = np.zeros(len(rcl), np.int64)
    so = np.zeros(len(rcl), np.int64)
    for S in py_cliques(g, s):
        ids = [pos[t] for t in itertools.combinations(S, r)]
        mc = min(core[i] for i in ids)
        mr = min(rnd[i] for i in ids)
        for i in ids:
            sv[i] += mc >= core[i]
            so[i] += mr >= rnd[i]
    return sv, so


@pytest.mark.parametrize("r,s", RS_ALL)
def test_certify_all_supports_match_brute_force(r, s):
    for seed in range(6):
        g = gg.gnp(9, [0.4, 0.6, 0.8][seed % 3], 900 + seed)
        d = orc.decompose(g, r, s)
        # a perturbed claim too, so that the supports are checked where they differ from n_s
        rng = np.random.default_rng(seed)
        core = d.core + rng.integers(-1, 2, d.core.size).astype(np.int32)
        rnd = np.maximum(d.round + rng.integers(-1, 2, d.round.size).astype(np.int32), 0)
        for c, t in [(d.core, d.round), (core, rnd)]:
            want_v, want_o = _brute_supports(g, r, s, c, t)
            got = orc.certify_all(g, r, s, c, t, d.levels, ids=np.arange(c.size))
            assert np.array_equal(got["sup_valid"], want_v)
            assert np.array_equal(got["sup_order"], want_o)


@pytest.mark.parametrize("r,s", [(1, 2), (1, 3), (2, 3), (2, 4), (3, 4), (2, 5), (3, 5), (4, 5)])
def test_certify_all_accepts_oracle_and_rejects_perturbations(r, s):
    for g in [gg.fig1(), gg.chung_lu(400, 16.0, 2.2, seed=37), gg.rmat(9, 16, 0.57, 0.19, 0.19, seed=38)]:
        d = orc.decompose(g, r, s)
        ok = orc.certify_all(g, r, s, d.core, d.round, d.levels)
        assert ok["bad_valid"] == ok["bad_order"] == ok["bad_level"] == 0 and ok["first_bad"] == -1
        if d.core.size == 0 or d.core.max() == 0:
            continue
        # a raised core number fails validity (and the level test)
        i = int(np.argmax(d.core))
        bad = d.core.copy()
        bad[i] += 1
        res = orc.certify_all(g, r, s, bad, d.round, d.levels)
        assert res["bad_valid"] >= 1 and res["first_bad"] <= i
        # an r-clique claimed one round later at a lower level than it has fails the order test
        # for the first r-clique of the top round
        top = int(d.rho - 1)
        j = int(np.nonzero(d.round == top)[0][0])
        lev = d.levels.copy()
        lev[top] -= 1
        bad = d.core.copy()
        bad[d.round == top] -= 1
        res = orc.certify_all(g, r, s, bad, d.round, lev)
        assert res["bad_order"] + res["bad_valid"] + res["bad_level"] >= 1
        # decreasing levels are rejected
        if d.rho >= 2 and d.levels[-1] > d.levels[0]:
            lev = d.levels.copy()
            lev[0] = lev[-1] + 1
            res = orc.certify_all(g, r, s, d.core, d.round, lev)
            assert res["bad_level"] >= 1
        # full mode and sample mode agree on the failures
        res_s = orc.certify_all(g, r, s, d.core, d.round, d.levels, ids=np.arange(d.core.size))
        assert res_s["bad_valid"] == res_s["bad_order"] == res_s["bad_level"] == 0
        assert j >= 0


# ------------------------------------------------------------------------------------
# Connectivity of nuclei (Section 2, footnote): components against networkx and brute force

def _brute_nuclei(g, r, s, core, level):
    """Components by breadth-first search over r-cliques, two of them adjacent when a vertex
    subset of size s that is pairwise adjacent contains both and has every r-subset at level."""
    rcl = py_cliques(g, r)
    pos = {t: i for i, t in enumerate(rcl)}
    adj = {i: set() for i in range(len(rcl))}
    for S in py_cliques(g, s):
        ids = [pos[t] for t in itertools.combinations(S, r)]
        if all(core[i] >= level for i in ids):
            for a in ids:
                adj[a].update(ids)
    comp = np.full(len(rcl), -1, np.int32)
    for i in range(len(rcl)):
        if core[i] < level or comp[i] >= 0:
            continue
        stack, members = [i], []
        comp[i] = i
        while stack:
            x = stack.pop()
            members.append(x)
            for y in adj[x]:
                if comp[y] < 0:
                    comp[y] = i
                    stack.append(y)
        comp[members] = min(members)
    return comp


def test_nuclei_12_equals_networkx_kcore_components():
    for seed in range(4):
        g = gg.chung_lu(400, 6.0, 2.2, seed=120 + seed)
        G = to_nx(g)
        core = orc.decompose(g, 1, 2).core
        for level in sorted(set(core.tolist()))[:6]:
            comp, nc = orc.nuclei(g, 1, 2, core, level)
            H = G.subgraph([v for v in range(g.n) if core[v] >= level])
            want = np.full(g.n, -1, np.int32)
            for cc in nx.connected_components(H):
                want[list(cc)] = min(cc)
            assert np.array_equal(comp, want) and nc == nx.number_connected_components(H)


@pytest.mark.parametrize("r,s", [(1, 2), (1, 3), (2, 3), (2, 4), (3, 4), (3, 5)])
def test_nuclei_brute_force(r, s):
    for seed in range(8):
        g = gg.disjoint_union(gg.gnp(8, 0.6, 1300 + seed), gg.gnp(7, 0.7, 1400 + seed))
        core = orc.decompose(g, r, s).core
        for level in sorted(set(core.tolist())):
            comp, nc = orc.nuclei(g, r, s, core, level)
            want = _brute_nuclei(g, r, s, core, level)
            assert np.array_equal(comp, want), (seed, r, s, level)
            assert nc == len(set(want[want >= 0].tolist()))


def test_nuclei_closed_forms():
    # K_n: at its one level every r-clique is in one nucleus; two disjoint copies give two
    g = gg.disjoint_union(gg.complete(6), gg.complete(6))
    for r, s in [(1, 2), (2, 3), (3, 4)]:
        core = orc.decompose(g, r, s).core
        comp, nc = orc.nuclei(g, r, s, core, int(core.max()))
        assert nc == 2 and np.all(comp >= 0)
        comp, nc = orc.nuclei(g, r, s, core, int(core.max()) + 1)
        assert nc == 0 and np.all(comp == -1)
    # bowtie: two triangles sharing only vertex 0. As (1,2) it is one 2-core; as (2,3) each
    # edge lies in one triangle (core 1), and no triangle holds edges of both, so two nuclei
    bow = gg.csr_from_edges(5, np.array([0, 0, 1, 0, 0, 3], np.int32), np.array([1, 2, 2, 3, 4, 4], np.int32))
    core = orc.decompose(bow, 1, 2).core
    assert list(core) == [2] * 5 and orc.nuclei(bow, 1, 2, core, 2)[1] == 1
    core = orc.decompose(bow, 2, 3).core
    comp, nc = orc.nuclei(bow, 2, 3, core, 1)
    # canonical edge ids: 01, 02, 03, 04, 12, 34
    assert list(core) == [1] * 6 and nc == 2 and list(comp) == [0, 0, 2, 2, 0, 2]


def _hierarchy_from_components(core, comp_at):
    """Checks the defining properties of a hierarchy output against per-level components
    comp_at[c] (smallest id per component, -1 outside X_c), computed independently."""
    levels = sorted(set(core.tolist()))
    nodes = {c: set(comp_at[c][core == c].tolist()) for c in levels}
    return levels, nodes


def _check_hierarchy(core, out, comp_at):
    comp, plev, pcomp = out
    levels, nodes = _hierarchy_from_components(core, comp_at)
    for R in range(core.size):
        c = int(core[R])
        # the node of R: its component at its own level, which holds an r-clique of core c
        assert comp[R] == comp_at[c][R] and comp[R] in nodes[c]
        below = [x for x in levels if x < c and comp_at[x][R] in nodes[x]]
        if not below:
            assert plev[R] == -1 and pcomp[R] == -1
            continue
        # the parent is the nearest lower node, and its component contains R's component
        assert plev[R] == max(below) and pcomp[R] == comp_at[plev[R]][R]
        members = np.flatnonzero(comp_at[c] == comp[R])
        assert np.all(comp_at[plev[R]][members] == pcomp[R])


def test_hierarchy_closed_forms():
    # Figure 1 as (1,2): the K5 (core 4) inside f's 3-core inside g's 2-core, a chain of three
    g = gg.fig1()
    core = orc.decompose(g, 1, 2).core
    comp, plev, pcomp = orc.hierarchy(g, 1, 2, core)
    assert list(core) == [4, 4, 4, 4, 4, 3, 2]
    assert list(comp) == [0] * 7 and list(plev) == [3] * 5 + [2, -1] and list(pcomp) == [0] * 6 + [-1]
    # Figure 1 as (3,4): cdg (core 0, in no 4-clique) is a node and a root of its own; the K5's
    # triangles (core 2) hang under the level-1 node of abf, aef, bef
    core = orc.decompose(g, 3, 4).core
    comp, plev, pcomp = orc.hierarchy(g, 3, 4, core)
    one = core == 1
    assert core[13] == 0 and comp[13] == 13 and plev[13] == -1
    assert np.all(plev[one] == -1) and np.all(plev[core == 2] == 1) and np.all(pcomp[core == 2] == 0)
    # two K5s (vertices 0-4, 5-9) joined through a vertex x = 10 of degree 2: as (1,2) two level-4
    # nodes, both children of the level-2 node that x closes
    u = [a for a in range(5) for b in range(a + 1, 5)]
    v = [b for a in range(5) for b in range(a + 1, 5)]
    uu = np.array(u + [a + 5 for a in u] + [0, 5], np.int32)
    vv = np.array(v + [b + 5 for b in v] + [10, 10], np.int32)
    g2 = gg.csr_from_edges(11, uu, vv)
    core = orc.decompose(g2, 1, 2).core
    comp, plev, pcomp = orc.hierarchy(g2, 1, 2, core)
    assert list(core) == [4] * 10 + [2]
    assert list(comp) == [0] * 5 + [5] * 5 + [0]
    assert list(plev) == [2] * 10 + [-1] and list(pcomp) == [0] * 10 + [-1]
    # the same graph as (2,3): every K5 edge has core 3 and the two connector edges core 0. No
    # triangle holds a connector, so each is a component of X_0 by itself (a level-0 node and a
    # root); the K5s' components of X_0 hold no core-0 edge, so the two level-3 nodes are roots too
    core = orc.decompose(g2, 2, 3).core
    comp, plev, pcomp = orc.hierarchy(g2, 2, 3, core)
    assert sorted(set(core.tolist())) == [0, 3]
    assert np.all(plev == -1) and len(set(comp.tolist())) == 4


@pytest.mark.parametrize("r,s", [(1, 2), (2, 3), (2, 4), (3, 4)])
def test_hierarchy_brute_force(r, s):
    # components from explicitly enumerated s-cliques (breadth-first search), not from the oracle
    for seed in range(6):
        g = gg.disjoint_union(gg.gnp(8, 0.6, 1500 + seed), gg.gnp(7, 0.75, 1600 + seed), gg.complete(s + 1))
        core = orc.decompose(g, r, s).core
        comp_at = {int(c): _brute_nuclei(g, r, s, core, int(c)) for c in set(core.tolist())}
        _check_hierarchy(core, orc.hierarchy(g, r, s, core), comp_at)


def test_hierarchy_12_networkx():
    for seed in range(3):
        g = gg.chung_lu(300, 6.0, 2.2, seed=170 + seed)
        G = to_nx(g)
        core = orc.decompose(g, 1, 2).core
        comp_at = {}
        for c in set(core.tolist()):
            H = G.subgraph([v for v in range(g.n) if core[v] >= c])
            want = np.full(g.n, -1, np.int32)
            for cc in nx.connected_components(H):
                want[list(cc)] = min(cc)
            comp_at[int(c)] = want
        _check_hierarchy(core, orc.hierarchy(g, 1, 2, core), comp_at)
