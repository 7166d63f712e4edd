"""Batches and the continuous-batching server: every graph's result in a batch, or served in a
mix of concurrent requests, is the same as the graph decomposed alone and as the oracle's.
The work is integer, so "the same" means bit for bit."""
import time

import numpy as np
import pytest

import graphgen as gg
import oracle as orc

pytestmark = pytest.mark.gpu

MIX = [(1, 2), (2, 3), (3, 4), (2, 4)]


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


def mixed_graphs(count, seed):
    u = gg.uniform(seed, 4 * count)
    out = []
    for i in range(count):
        n = 30 + int(u[4 * i] * 400)
        d = 4.0 + u[4 * i + 1] * 12.0
        if u[4 * i + 2] < 0.5:
            g = gg.chung_lu(n, d, 2.2, seed=seed * 1000 + i)
        else:
            g = gg.rmat(max(5, int(np.log2(n))), 8, 0.57, 0.19, 0.19, seed=seed * 1000 + i)
        r, s = MIX[int(u[4 * i + 3] * len(MIX)) % len(MIX)]
        out.append((g, r, s))
    return out


def alone(nd, ctx, g, r, s):
    G = nd.nd_load_csr(ctx, g.rowptr, g.col)
    core, _, _ = nd.nd_decompose(G, r, s, want_round=False)
    nd.nd_graph_free(G)
    return core


def test_batch_equals_alone_and_oracle(nd, ctx):
    items = mixed_graphs(40, 7)
    # include degenerate members: no edges, a single vertex, a complete graph
    items.append((gg.csr_from_edges(6, np.zeros(0, np.int32), np.zeros(0, np.int32), "empty6"), 2, 3))
    items.append((gg.complete(1), 1, 2))
    items.append((gg.complete(9), 3, 4))
    outs, n_r, status, st = nd.nd_batch_run(ctx, [(g.rowptr, g.col, r, s) for g, r, s in items])
    assert all(x == nd.ND_OK for x in status)
    assert st["groups"] == len({(r, s) for _, r, s in items})
    for (g, r, s), got, k in zip(items, outs, n_r):
        want = orc.decompose(g, r, s).core
        assert k == want.size
        assert np.array_equal(got, want), (g.name, r, s)
        assert np.array_equal(got, alone(nd, ctx, g, r, s))


def test_batch_reports_bad_requests_individually(nd, ctx):
    good = gg.fig1()
    reqs = [(good.rowptr, good.col, 2, 3), (good.rowptr, good.col, 4, 7), (good.rowptr, good.col, 3, 4)]
    outs, n_r, status, _ = nd.nd_batch_run(ctx, reqs)
    assert status == [nd.ND_OK, nd.ND_EINVAL, nd.ND_OK]
    assert np.array_equal(outs[0], orc.decompose(good, 2, 3).core)
    assert np.array_equal(outs[2], orc.decompose(good, 3, 4).core)


def _serve(nd, ctx, items, **cfg):
    outs = []
    for g, r, s in items:  # output sizes first, so that the requests go out as one burst
        G = nd.nd_load_csr(ctx, g.rowptr, g.col)
        _, k, _ = nd.nd_count(G, r, s, count_width=8)
        nd.nd_graph_free(G)
        outs.append((np.full(max(k, 1), -1, np.int32), k))
    sv = nd.nd_server_create(ctx, **cfg)
    tickets = []
    try:
        for (g, r, s), (out, k) in zip(items, outs):
            tickets.append(sv.submit(g.rowptr, g.col, r, s, out))
        results = {}
        deadline = time.time() + 300
        while len(results) < len(tickets) and time.time() < deadline:
            for t in tickets:
                if t in results:
                    continue
                rc, res = sv.poll(t)
                if rc != nd.ND_PENDING:
                    results[t] = (rc, res)
            time.sleep(0.001)
        assert len(results) == len(tickets), "server did not finish"
    finally:
        sv.close()
    return tickets, outs, results


def test_server_results_equal_alone(nd, ctx):
    items = mixed_graphs(60, 11)
    # one worker: while it runs a batch, the rest of the burst waits and is merged
    tickets, outs, results = _serve(nd, ctx, items, workers=1, max_batch=16)
    batched = 0
    for (g, r, s), t, (out, k) in zip(items, tickets, outs):
        rc, res = results[t]
        assert rc == nd.ND_OK
        assert res["n_r"] == k
        assert np.array_equal(out[:k], alone(nd, ctx, g, r, s)), (g.name, r, s)
        assert res["latency_ms"] >= res["run_ms"] >= 0
        batched += res["batch_size"] > 1
    assert batched > 0, "requests submitted back to back should share batches"


def test_server_overlapping_workers_equal_alone(nd, ctx):
    items = mixed_graphs(48, 17)
    tickets, outs, results = _serve(nd, ctx, items, workers=4, max_batch=8)
    for (g, r, s), t, (out, k) in zip(items, tickets, outs):
        assert results[t][0] == nd.ND_OK
        assert np.array_equal(out[:k], orc.decompose(g, r, s).core), (g.name, r, s)


def test_server_memory_budget_and_queue(nd, ctx):
    items = mixed_graphs(12, 13)
    # a tight budget admits only a few small requests at a time; results are unchanged
    tickets, outs, results = _serve(nd, ctx, items, workers=2, max_batch=8, mem_budget=8 << 20)
    for (g, r, s), t, (out, k) in zip(items, tickets, outs):
        assert results[t][0] == nd.ND_OK
        assert np.array_equal(out[:k], orc.decompose(g, r, s).core)
    big = gg.complete(300)
    sv = nd.nd_server_create(ctx, mem_budget=1 << 16, workers=1, max_batch=4)
    with pytest.raises(nd.NdError) as ei:
        sv.submit(big.rowptr, big.col, 3, 4, np.zeros(10, np.int32))
    assert ei.value.code == nd.ND_ENOMEM
    sv.close()
    sv = nd.nd_server_create(ctx, workers=1, max_batch=1, queue_cap=1)
    g = gg.chung_lu(3000, 20.0, 2.1, seed=3)
    out = [np.zeros(g.m, np.int32) for _ in range(40)]
    busy = 0
    ts = []
    for o in out:
        try:
            ts.append(sv.submit(g.rowptr, g.col, 2, 3, o))
        except nd.NdError as e:
            assert e.code == nd.ND_EBUSY
            busy += 1
    sv.drain()
    for t in ts:
        assert sv.poll(t)[0] == nd.ND_OK
    sv.close()
    assert busy > 0


# ------------------------------------------------------------------------------------
# The batched and served workloads at their own size ranges, checked against the oracle

def _rs_draw(count, seed):
    choices = [(2, 3), (3, 4), (2, 4)]
    u = gg.uniform(seed, count)
    return [choices[min(2, int(x * 3))] for x in u]


@pytest.fixture(scope="module")
def batch_items():
    """The first 256 graphs of the batched workload (n up to 5,000, average degree up to 40,
    (r,s) from (1,2), (2,3), (3,4)) with their oracle core numbers."""
    from oracle_pool import oracle_cores

    items = [(g, r, s) for g, (r, s) in gg.batch_workload(256)]
    return items, oracle_cores(items)


@pytest.fixture(scope="module")
def serve_items():
    """256 graphs of the served stream's pool with at most 1e5 edges (Chung-Lu and R-MAT, edge
    count log-uniform), each with an (r,s) drawn from (2,3), (3,4), (2,4), with their oracle
    core numbers."""
    from oracle_pool import oracle_cores

    graphs = gg.serve_pool(420, max_m=100_000)[:256]
    items = [(g, r, s) for g, (r, s) in zip(graphs, _rs_draw(len(graphs), 77))]
    return items, oracle_cores(items)


def test_batch_workload_256_against_oracle_and_alone(nd, ctx, batch_items):
    items, want = batch_items
    assert len(items) == 256 and max(g.n for g, _, _ in items) > 4000
    outs, n_r, status, st = nd.nd_batch_run(ctx, [(g.rowptr, g.col, r, s) for g, r, s in items])
    assert all(x == nd.ND_OK for x in status)
    for (g, r, s), got, k, w in zip(items, outs, n_r, want):
        assert k == w.size, (g.name, r, s)
        assert np.array_equal(got, w), (g.name, r, s)
    for i in range(0, len(items), 5):  # one in five also against the graph decomposed alone
        g, r, s = items[i]
        assert np.array_equal(outs[i], alone(nd, ctx, g, r, s)), (g.name, r, s)


def test_server_on_the_serve_pool_against_oracle_and_alone(nd, ctx, serve_items):
    items, want = serve_items
    assert len(items) == 256 and max(g.m for g, _, _ in items) > 50_000
    tickets, outs, results = _serve(nd, ctx, items, workers=4, max_batch=64)
    shared = 0
    for (g, r, s), t, (out, k), w in zip(items, tickets, outs, want):
        rc, res = results[t]
        assert rc == nd.ND_OK
        assert res["n_r"] == k == w.size
        assert np.array_equal(out[:k], w), (g.name, r, s)
        shared += res["batch_size"] > 1
    assert shared > 0
    for i in range(0, len(items), 5):
        g, r, s = items[i]
        assert np.array_equal(outs[i][0][:outs[i][1]], alone(nd, ctx, g, r, s)), (g.name, r, s)


def test_malformed_requests_fail_alone(nd, ctx):
    """A request whose CSR breaks an invariant (an id out of range, an unsorted row, a
    self-loop, a missing reverse entry) fails alone with ND_EINVAL, in a batch and in the
    server, while the well-formed requests beside it still get the oracle's result. Ids out of
    range are caught on the host before the union is built; the other faults by the GPU
    validation of the union, after which the host checks each request in full."""
    good = [gg.chung_lu(300, 10.0, 2.2, seed=71), gg.rmat(8, 8, 0.57, 0.19, 0.19, seed=72)]
    base = gg.chung_lu(200, 8.0, 2.2, seed=73)
    row = int(np.argmax(np.diff(base.rowptr)))
    lo, hi = int(base.rowptr[row]), int(base.rowptr[row + 1])
    nbrs = set(base.col[lo:hi].tolist())
    bads = []
    c = base.col.copy()
    c[5] = base.n + 3  # id out of range
    bads.append(c)
    c = base.col.copy()
    c[[lo, lo + 1]] = c[[lo + 1, lo]]  # row not ascending
    bads.append(c)
    # a value between two neighbours of `row` that keeps the row ascending: `row` itself gives a
    # self-loop, any other non-neighbour an entry whose reverse is missing
    for target in (row, None):
        for q in range(lo + 1, hi - 1):
            cands = [x for x in range(int(base.col[q - 1]) + 1, int(base.col[q + 1]))
                     if x not in nbrs and (x == row if target is not None else x != row)]
            if cands:
                c = base.col.copy()
                c[q] = cands[0]
                bads.append(c)
                break
    assert len(bads) == 4
    reqs = [(good[0].rowptr, good[0].col, 2, 3)]
    for c in bads:
        reqs.append((base.rowptr, c, 2, 3))
    reqs.append((good[1].rowptr, good[1].col, 2, 3))
    reqs.append((good[1].rowptr, good[1].col, 3, 4))
    outs, n_r, status, _ = nd.nd_batch_run(ctx, reqs)
    assert status[0] == nd.ND_OK and status[-1] == nd.ND_OK and status[-2] == nd.ND_OK
    assert all(st == nd.ND_EINVAL for st in status[1:1 + len(bads)]), status
    assert np.array_equal(outs[0][:n_r[0]], orc.decompose(good[0], 2, 3).core)
    assert np.array_equal(outs[-2][:n_r[-2]], orc.decompose(good[1], 2, 3).core)
    assert np.array_equal(outs[-1][:n_r[-1]], orc.decompose(good[1], 3, 4).core)
    # the server accepts them (nd_submit checks only the arguments, in O(1)) and they fail with
    # ND_EINVAL in their batch, next to a good request that is served
    sv = nd.nd_server_create(ctx, workers=1, max_batch=8)
    try:
        out = np.zeros(good[0].m, np.int32)
        tickets = [sv.submit(base.rowptr, c, 2, 3, np.zeros(base.m, np.int32)) for c in bads]
        t = sv.submit(good[0].rowptr, good[0].col, 2, 3, out)
        sv.drain()
        for tb in tickets:
            assert sv.poll(tb)[0] == nd.ND_EINVAL
        assert sv.poll(t)[0] == nd.ND_OK
        assert np.array_equal(out, orc.decompose(good[0], 2, 3).core)
        bad_rp = base.rowptr.copy()
        bad_rp[0] = 1
        with pytest.raises(nd.NdError) as ei:
            sv.submit(bad_rp, base.col, 2, 3, np.zeros(base.m, np.int32))
        assert ei.value.code == nd.ND_EINVAL
    finally:
        sv.close()
