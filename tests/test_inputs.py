"""The seeded synthetic inputs that stand in for the paper's graphs: well-formed symmetric CSR,
determinism per seed, and the recipe's targets (Chung-Lu expected degrees, R-MAT sample counts,
planted dense communities). CPU only."""
import math

import numpy as np
import pytest

import graphgen as gg


def assert_valid_csr(g):
    rp, col = g.rowptr, g.col
    assert rp.dtype == np.int64 and col.dtype == np.int32
    assert rp[0] == 0 and rp[-1] == col.size and np.all(np.diff(rp) >= 0)
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(rp))
    assert np.all(col >= 0) and np.all(col < g.n)
    assert not np.any(rows == col), "self-loop"
    # strictly ascending within each row (no duplicates)
    same_row = rows[1:] == rows[:-1]
    assert np.all(col[1:][same_row] > col[:-1][same_row])
    # symmetric: the multiset of (u, v) equals that of (v, u)
    fwd = rows * g.n + col
    bwd = col.astype(np.int64) * g.n + rows
    assert np.array_equal(np.sort(fwd), np.sort(bwd))
    assert col.size % 2 == 0 and g.m == col.size // 2


@pytest.mark.parametrize("make", [
    lambda s: gg.chung_lu(3000, 12.0, 2.2, seed=s),
    lambda s: gg.rmat(12, 16, 0.57, 0.19, 0.19, seed=s),
    lambda s: gg.rmat_m(5000, seed=s),
    lambda s: gg.gnp(200, 0.1, s),
    lambda s: gg.with_planted(gg.chung_lu(2000, 8.0, 2.3, seed=s), 20, 20, 60, 0.7, s + 1),
])
def test_valid_and_deterministic(make):
    a, b, c = make(11), make(11), make(12)
    assert_valid_csr(a)
    assert np.array_equal(a.rowptr, b.rowptr) and np.array_equal(a.col, b.col)
    assert not (a.rowptr.size == c.rowptr.size and np.array_equal(a.col, c.col)), "seed has no effect"


def test_chung_lu_2k_degrees():
    """n = 2000, average degree 20, exponent 2.1, largest expected degree 200."""
    g = gg.chung_lu_2k(seed=1)
    assert g.n == 2000
    d = g.degrees()
    assert 17.0 <= d.mean() <= 21.0  # pair probabilities are capped at 1, so slightly below 20
    assert 120 <= d.max() <= 280
    # power law: the top 1% of vertices hold far more than 1% of the edge endpoints
    top = np.sort(d)[::-1][: g.n // 100].sum()
    assert top / d.sum() > 0.05


def test_power_law_weights_targets():
    w = gg.power_law_weights(100000, 30.0, 2.3, math.sqrt(100000 * 30.0))
    assert abs(w.mean() - 30.0) < 1e-6 * 30.0
    assert abs(w[0] - math.sqrt(100000 * 30.0)) < 1e-9 * w[0]
    assert np.all(np.diff(w) <= 0)


def test_rmat_sizes():
    """2^scale vertices from 16 * 2^scale directed samples; after dropping loops and duplicates
    the undirected edge count falls well below the sample count (skewed a = .57)."""
    g = gg.rmat(14, 16, 0.57, 0.19, 0.19, seed=2)
    assert g.n == 1 << 14
    ratio = g.m / (16 * g.n)
    assert 0.5 < ratio < 1.0
    d = g.degrees()
    assert d.max() > 20 * d.mean()  # heavy hubs


def test_rmat_m_hits_its_edge_count():
    """n = 2^ceil(log2(m/8)); sampling stops at m unique edges, or after 4m samples (on 16
    vertices the skewed sampler cannot find 100 distinct edges in 400 draws)."""
    for m in [100, 1000, 20000, 200000]:
        g = gg.rmat_m(m, seed=5)
        assert g.n == 1 << max(1, math.ceil(math.log2(max(m / 8.0, 2.0))))
        assert g.m <= m
        if m >= 1000:
            assert g.m == m


def test_planted_communities():
    """k disjoint communities with sizes in [smin, smax], each pair inside joined with p = 0.7."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components

    n, k, smin, smax, p = 20000, 200, 20, 60, 0.7
    u, v = gg.planted_edges(n, k, smin, smax, p, seed=3)
    adj = coo_matrix((np.ones(u.size), (u, v)), shape=(n, n)).tocsr()
    ncomp, lab = connected_components(adj, directed=False)
    sizes = np.bincount(lab)
    members = sizes[sizes > 1]
    assert members.size == k  # disjoint and (at p = 0.7) connected
    assert members.min() >= smin and members.max() <= smax
    pairs = sum(s * (s - 1) // 2 for s in members)
    e = np.unique(np.minimum(u, v).astype(np.int64) * n + np.maximum(u, v)).size
    assert abs(e / pairs - p) < 0.02


def test_batch_workload_recipe():
    items = gg.batch_workload(64, seed=4)
    assert len(items) == 64
    rs_seen = set()
    for g, rs in items:
        assert 50 <= g.n <= 5000 and rs in [(1, 2), (2, 3), (3, 4)]
        rs_seen.add(rs)
    assert rs_seen == {(1, 2), (2, 3), (3, 4)}
    for g, _ in items[:8]:
        assert_valid_csr(g)
    # a prefix does not depend on the count
    again = gg.batch_workload(16, seed=4)
    for (a, ra), (b, rb) in zip(items[:16], again):
        assert ra == rb and np.array_equal(a.col, b.col)


def test_serve_pool_recipe():
    pool = gg.serve_pool(48, seed=5, max_m=60_000)
    assert 0 < len(pool) < 48  # the draws above max_m are skipped
    ms = np.array([g.m for g in pool])
    assert ms.min() >= 50 and ms.max() <= 60_000 * 1.05
    for g in pool[:6]:
        assert_valid_csr(g)
    # max_m skips draws without changing the others
    full = [g for g in gg.serve_pool(48, seed=5, max_m=10**9) if g.m <= 60_000 * 1.05]
    assert len(full) >= len(pool)


def test_hubs_over_sparse_makes_long_lists():
    g = gg.hubs_over_sparse(n_common=3000, hubs=3, p_hub=0.9, avg_deg=4.0, seed=7)
    assert_valid_csr(g)
    deg = np.diff(g.rowptr)
    hub_deg = deg[-3:]
    assert np.all(hub_deg > 0.85 * 3000) and np.median(deg[:-3]) < 20
    # the hubs are mutually adjacent
    for h in range(3000, 3003):
        row = g.col[g.rowptr[h]:g.rowptr[h + 1]]
        assert set(range(3000, 3003)) - {h} <= set(row.tolist())
