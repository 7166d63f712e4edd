"""bench.py's multi-process plumbing on the CPU with the gloo backend (world size 2): the
barrier and max-over-ranks timing, and the reference arm (the CPU oracle) printing exactly one
JSON line from rank 0 while the other rank exits without work. No GPU is involved."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench

    w, r, local, pg = bench.dist_setup(want_nccl=False)
    assert (w, r) == (world, rank)
    bench.barrier(pg)
    m = bench.max_over_ranks(pg, float(10 * (rank + 1)))
    q.put((rank, m))
    pg.destroy_process_group()


def test_max_over_ranks_gloo():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 20.0), (1, 20.0)]


def test_reference_arm_under_torchrun_prints_one_line():
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"), "--impl", "reference",
           "--workload", "cl2k", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["value"] > 0
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["cpu_baseline"]["cores"] == 1
    assert rec["e2e"]["h2d_bytes_per_step"] == 0


def test_units_formula():
    sys.path.insert(0, ROOT)
    import bench

    # (2,3): each triangle counted once and re-listed for each of its 3 edges
    assert bench.units_of(2, 3, 10) == 40
    assert bench.units_of(3, 4, 10) == 50
    assert bench.units_of(2, 4, 1) == 7


def _fake_stats(rs_list):
    st = {}
    for r, s in rs_list:
        st[(r, s)] = {"n_r": 1000, "n_s": 5000, "listed": 5000, "decrements": 12000, "count_width": 4,
                      "t_count_ms": 10.0, "t_peel_ms": 40.0}
    return [st]


SUMS = {"sum_deg": 800, "edge_min_deg": 900, "edge_dplus": 1100, "n3": 1000, "tri_min_deg": 2000,
        "tri_dplus_last": 700}


class _G:
    n, m = 100, 400


def test_byte_models_written_out():
    """The method's lower-bound model on hand-set sums: (3,4) peel = 4 sum_t min deg + C(4,3) n_4
    listings x 3 other triangles x 5 B + 2w per decrement + 8 B per triangle of A; count = 4 sum_e
    (d+(u) + d+(v)) + 4 sum_t d+(last) + 2w per count."""
    sys.path.insert(0, ROOT)
    import bench

    st = _fake_stats([(3, 4)])[0][(3, 4)]
    cm, pm, ci, pi = bench.byte_models(3, 4, st, SUMS, _G())
    assert pm == 4 * 2000 + 4 * 5000 * 3 * 5 + 8 * 12000 + 8 * 1000
    assert cm == 4 * 1100 + 4 * 700 + 8 * 1000
    assert ci == 64 * 1000 + 32 * 5000 and pi == 72 * 1000 + 28 * 5000 + 8 * 12000
    cm, pm, _, _ = bench.byte_models(2, 3, _fake_stats([(2, 3)])[0][(2, 3)], SUMS, _G())
    assert pm == 4 * 900 + 3 * 5000 * 2 * 5 + 8 * 12000 + 8 * 1000 and cm == 4 * 1100 + 8 * 1000
    cm, pm, _, _ = bench.byte_models(1, 2, _fake_stats([(1, 2)])[0][(1, 2)], SUMS, _G())
    assert cm == 8 * 101 and pm == 4 * 800 + 2 * 5000 * 1 * 5 + 8 * 12000 + 8 * 1000


def test_roofline_models_and_traffic_gate(monkeypatch):
    """Every benchmarked (r,s) has nonzero byte models; the ncu traffic figure is reported only
    while the library sources match the fingerprint the capture was taken on."""
    sys.path.insert(0, ROOT)
    import bench

    for name, rs_list in [("rmat20", [(2, 3), (3, 4)]), ("cl4m", [(3, 4), (2, 4)]),
                          ("rmat_dense", [(2, 5), (3, 5)])]:
        top = bench.roofline(name, rs_list, _fake_stats(rs_list), _G(), SUMS)
        for e in [top] + top["others"]:
            assert e["algorithmic_bytes_per_launch"] > 0 and e["implementation_bytes_per_launch"] > 0, e["kernel"]
            assert e["unit"] == "GB/s" and e["bound"] == "hbm"
            assert abs(e["frac"] - e["achieved"] / e["peak"]) < 1e-12
    table = {"f" * 16: {("rmat20", "k_peel_loop(3,4)"): 1.5e9, ("rmat20", "k_peel_loop(2,3)"): 2.5e8}}
    monkeypatch.setattr(bench, "NCU_TRAFFIC", table)
    monkeypatch.setattr(bench, "sources_fingerprint", lambda: "f" * 16)
    rs = [(2, 3), (3, 4)]
    top = bench.roofline("rmat20", rs, _fake_stats(rs), _G(), SUMS)
    assert top["traffic"] == table["f" * 16].get(("rmat20", top["kernel"]))
    monkeypatch.setattr(bench, "sources_fingerprint", lambda: "0" * 16)
    top = bench.roofline("rmat20", rs, _fake_stats(rs), _G(), SUMS)
    assert top["traffic"] is None and all(o["traffic"] is None for o in top["others"])
