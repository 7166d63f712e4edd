#!/usr/bin/env python
"""Benchmark of the (r,s) nucleus decomposition hot path on GB300.

One step = the whole hot path for every (r,s) of the workload on a graph already resident in
HBM: orientation and the edge index, the triangle index (r = 3), s-clique counting and the
device-resident peeling loop, results left in device memory. Default workload: seeded R-MAT
scale 20 (2^20 vertices, 16 * 2^20 edge samples, a=0.57 b=0.19 c=0.19), (2,3) then (3,4).

Prints ONE JSON line (rank 0). ``value`` is s-cliques processed per second, counting each
s-clique once for the count phase and once per member r-clique re-listed by Update:
(1 + C(s,r)) * n_s per (r,s), summed over the workload's (r,s) and over ranks.

    python bench.py [--gpus N --steps K --warmup W] [--impl ours|reference] [--workload NAME]

--impl reference times the CPU oracle (test infrastructure, single-threaded C) on a bounded
sample of the same workload (a smaller R-MAT with the same parameters), on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402

L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2

WORKLOADS = {
    "rmat20": dict(
        desc="R-MAT scale 20, edge factor 16, a=0.57 b=0.19 c=0.19, symmetrised+deduplicated; (2,3) and (3,4)",
        gen=lambda: gg.rmat_scale20(seed=2),
        rs=[(2, 3), (3, 4)],
        sample=lambda scale: gg.rmat(scale, 16, 0.57, 0.19, 0.19, seed=2),
        sample_desc="R-MAT scale {scale} (same edge factor, a, b, c and seed), (2,3) and (3,4)",
    ),
    "cl2k": dict(
        desc="Chung-Lu n=2000, avg degree 20, exponent 2.1, max expected degree 200; (2,3)",
        gen=lambda: gg.chung_lu_2k(seed=1),
        rs=[(2, 3)],
        sample=lambda scale: gg.chung_lu_2k(seed=1),
        sample_desc="the whole workload",
    ),
    "cl4m": dict(
        desc="Chung-Lu n=4,194,304, avg degree 30, exponent 2.3, w_max=sqrt(sum w), + 2000 planted communities "
             "(20-60 vertices, density 0.7); (3,4) and (2,4), int64 tallies",
        gen=lambda: gg.chung_lu_4m_planted(seed=3),
        rs=[(3, 4), (2, 4)],
        width=8,
        sample=lambda scale: gg.with_planted(gg.chung_lu(1 << scale, 30.0, 2.3, seed=3, exact=False), 20, 20, 60,
                                             0.7, 3 + 7919),
        sample_desc="Chung-Lu n=2^{scale} with the same parameters plus 20 planted communities, (3,4) and (2,4)",
    ),
}


def units_of(r: int, s: int, n_s: int) -> int:
    """s-cliques of Algorithm 2: each counted once, then re-listed once per member r-clique."""
    return (1 + math.comb(s, r)) * n_s


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["batch", "serve"], default="rmat20")
    ap.add_argument("--batch-graphs", type=int, default=4096)
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-pool", type=int, default=256)
    ap.add_argument("--serve-workers", type=int, default=4)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--peel-mode", choices=["default", "persistent", "loop_graph", "plain"], default="default",
                    help="how the peeling rounds are launched (default: the library's choice)")
    ap.add_argument("--contract", choices=["default", "off", "always"], default="default",
                    help="(2,3) graph contraction: the paper's schedule (default), off, or before every round")
    ap.add_argument("--dense-buckets", action="store_true", help="level advances by the dense-bucket search")
    ap.add_argument("--rs", default=None, help="only these (r,s) of the workload, e.g. 2,3 or 2,3:3,4")
    ap.add_argument("--scale", type=int, default=None,
                    help="R-MAT workload only: use scale S instead of 20 (profiling a smaller case)")
    return ap.parse_args()


# ------------------------------------------------------------------------------------------
# distributed plumbing (replicas: every rank runs the whole workload; no data-path collective)

def dist_setup(want_nccl: bool):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist

        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl" if want_nccl else "gloo")
        pg = dist
    return world, rank, local, pg


def barrier(pg, device=None):
    if pg is None:
        return
    if device is not None:
        pg.barrier(device_ids=[device])
    else:
        pg.barrier()


def max_over_ranks(pg, x: float, device=None) -> float:
    if pg is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=f"cuda:{device}" if device is not None else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="nd_clocks_", suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def gpu_uuid(device: int) -> str | None:
    try:
        import torch

        u = str(torch.cuda.get_device_properties(device).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


# ------------------------------------------------------------------------------------------
# CPU oracle timing (the baseline and the reference arm)

def oracle_sample_run(workload: dict, scale: int):
    import oracle as orc

    g = workload["sample"](scale)
    units = 0
    t0 = time.perf_counter()
    for r, s in workload["rs"]:
        d = orc.decompose(g, r, s)
        units += units_of(r, s, d.n_s)
    dt = time.perf_counter() - t0
    return units, dt, g


def pick_sample_scale(per_step_budget_s: float) -> int:
    # one-core oracle times on this R-MAT family: scale 12 ~ 27 s, scale 11 ~ 9 s, scale 10 ~ 3 s
    if per_step_budget_s >= 30:
        return 12
    if per_step_budget_s >= 10:
        return 11
    return 10


def run_reference(args, world, rank):
    """--impl reference: the CPU oracle, as it stands, on a bounded sample per step."""
    if rank != 0:
        return 0
    wl = WORKLOADS[args.workload]
    steps, warm = args.steps, args.warmup
    scale = pick_sample_scale(150.0 / max(1, steps + warm))
    for _ in range(warm):
        oracle_sample_run(wl, scale)
    tot_units, tot_t = 0, 0.0
    g = None
    for _ in range(steps):
        u, dt, g = oracle_sample_run(wl, scale)
        tot_units += u
        tot_t += dt
    value = tot_units / tot_t
    sample = wl["sample_desc"].format(scale=scale) + f": n={g.n}, m={g.m}"
    line = {"impl": "reference", "metric": "(r,s) s-cliques/sec", "value": value, "unit": "s-cliques/s",
            "n_gpus": args.gpus, "steps": steps, "warmup": warm, "ms_per_step": 1000.0 * tot_t / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": {"workload": args.workload, "desc": wl["desc"]},
            "cpu_baseline": {"value": value, "unit": "s-cliques/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "s-cliques/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------
# our arm

def main():
    args = parse_args()
    world, rank, local, pg = dist_setup(want_nccl=(args.impl == "ours"))
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import numpy as np
    import torch

    import paper_2111_10980_gb300 as nd

    torch.cuda.set_device(local)
    if args.workload == "batch":
        return run_batch(args, nd, world, rank, local, pg)
    if args.workload == "serve":
        return run_serve(args, nd, world, rank, local, pg)
    wl = dict(WORKLOADS[args.workload])
    width = wl.get("width", 0)
    workload_name = args.workload
    if args.scale is not None and args.workload == "rmat20":
        sc = args.scale
        wl["gen"] = lambda: gg.rmat(sc, 16, 0.57, 0.19, 0.19, seed=2)
        wl["desc"] = wl["desc"].replace("scale 20", f"scale {sc}")
        workload_name = f"rmat{sc}"
    if args.rs:
        wl["rs"] = [tuple(int(x) for x in p.split(",")) for p in args.rs.split(":")]
    wl["name"] = workload_name
    g = wl["gen"]()
    stream = torch.cuda.Stream(device=local)
    ctx = nd.nd_ctx_create(local, stream=stream)
    rp_d = torch.from_numpy(g.rowptr).to(f"cuda:{local}")
    col_d = torch.from_numpy(g.col).to(f"cuda:{local}")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=f"cuda:{local}")
    torch.cuda.synchronize()
    G = nd.nd_load_csr(ctx, rp_d, col_d)

    outs = {}
    pflags = {"default": 0, "persistent": nd.ND_PEEL_PERSISTENT, "loop_graph": nd.ND_PEEL_LOOP_GRAPH,
              "plain": nd.ND_NO_GRAPH}[args.peel_mode]
    pflags |= {"default": 0, "off": nd.ND_CONTRACT_OFF, "always": nd.ND_CONTRACT_ALWAYS}[args.contract]
    if args.dense_buckets:
        pflags |= nd.ND_DENSE_BUCKETS

    def step():
        nd.nd_graph_reset(G)  # every step rebuilds orientation and indexes
        stats = {}
        for r, s in wl["rs"]:
            core = outs.get((r, s))
            if core is None:  # first warm-up step: learn n_r, then keep a device output buffer
                _, _, st = nd.nd_decompose(G, r, s, count_width=width, want_round=False, flags=pflags)
                outs[(r, s)] = torch.empty(max(st["n_r"], 1), dtype=torch.int32, device=f"cuda:{local}")
            else:
                _, _, st = nd.nd_decompose(G, r, s, count_width=width, core_out=core, want_round=False,
                                           flags=pflags)
            stats[(r, s)] = st
        return stats

    for _ in range(args.warmup):
        step()

    # timed region
    sampler = ClockSampler(gpu_uuid(local))
    barrier(pg, local)
    torch.cuda.synchronize()
    sampler.start()
    launches0 = nd.nd_kernel_launches()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    per_step_stats = []
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)  # evict the previous step's data from L2 (not timed)
        with torch.cuda.stream(stream):
            ev0[i].record(stream)
            per_step_stats.append(step())
            ev1[i].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    launches = nd.nd_kernel_launches() - launches0
    clocks = sampler.stop()
    barrier(pg, local)
    t_ms = sum(a.elapsed_time(b) for a, b in zip(ev0, ev1))
    t_ms = max_over_ranks(pg, t_ms, local)

    stats = per_step_stats[-1]
    units_per_step = sum(units_of(r, s, stats[(r, s)]["n_s"]) for r, s in wl["rs"])
    rcl_per_step = sum(stats[(r, s)]["n_r"] for r, s in wl["rs"])
    value = units_per_step * args.steps * world / (t_ms / 1000.0)
    peel_ms = [sum(st[(r, s)]["t_peel_ms"] for r, s in wl["rs"]) for st in per_step_stats]
    peeled_per_s = rcl_per_step * args.steps * world / (sum(peel_ms) / 1000.0)

    roof = roofline(wl, per_step_stats, g)

    line = {"metric": "(r,s) s-cliques/sec", "value": value, "unit": "s-cliques/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int64" if width == 8 else "int32", "data": "synthetic",
            "config": {"workload": workload_name, "desc": wl["desc"], "n": g.n, "m": g.m,
                       "rs": [f"({r},{s})" for r, s in wl["rs"]], "parallelism": f"replicas x{world}",
                       "l2": "flushed between steps (256 MiB write, outside the step events)",
                       "peel_mode": args.peel_mode, "contract": args.contract,
                       "dense_buckets": bool(args.dense_buckets)},
            "r_cliques_peeled_per_s": peeled_per_s,
            "wall_s_timed": wall,
            "per_rs": {f"({r},{s})": dict(
                {k: stats[(r, s)][k] for k in
                 ("n_r", "n_s", "rho", "max_core", "listed", "decrements", "advances", "refills", "count_width",
                  "t_orient_ms", "t_index_ms", "t_count_ms", "t_peel_ms", "t_total_ms", "t_phase_ms",
                  "t_contract_ms", "contractions")},
                # the count phase alone (s-cliques counted per second) and the peel alone
                n_s_per_s_count=stats[(r, s)]["n_s"] / max(stats[(r, s)]["t_count_ms"], 1e-9) * 1e3,
                n_r_per_s_peel=stats[(r, s)]["n_r"] / max(stats[(r, s)]["t_peel_ms"], 1e-9) * 1e3)
                for r, s in wl["rs"]},
            "gpu_launches": launches,
            "roofline": roof,
            "clocks": clocks}

    # end to end through the C ABI with pinned host buffers (H2D of the CSR, D2H of every core array)
    if not args.no_e2e:
        line["e2e"] = e2e(nd, wl, g, local, width, args.e2e_steps, world, pg)

    nd.nd_graph_free(G)
    nd.nd_ctx_destroy(ctx)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        scale = 12 if args.workload == "rmat20" else 14
        units, dt, sg = oracle_sample_run(wl, scale)
        line["cpu_baseline"] = {"value": units / dt, "unit": "s-cliques/s", "cores": 1, "kind": "oracle",
                                "sample": wl["sample_desc"].format(scale=scale) + f": n={sg.n}, m={sg.m}, "
                                f"{dt:.1f} s single-threaded"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()
    return 0


# DRAM bytes per launch (read + write) from one-pass ncu captures of the bench workloads (metrics
# dram__bytes_read.sum and dram__bytes_write.sum over every launch of one warm-up and one timed
# step), keyed by the fingerprint of the library sources they were taken on; reported as
# roofline.traffic only while the sources still match.
NCU_TRAFFIC = {
    "fcd44b27ffba5a44": {
        ("rmat20", "k_peel_loop(3,4)"): 7.648e12,
        ("rmat20", "k_peel_loop(2,3)"): 115.7e9,
        ("rmat20", "k_count34"): 1164.0e9,
        ("rmat20", "k_count23"): 9.58e9,
    },
}


def sources_fingerprint():
    import glob
    import hashlib

    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_2111_10980_gb300", "csrc", "*"))):
        if f.endswith((".cu", ".cuh", ".h")):
            h.update(os.path.basename(f).encode())
            with open(f, "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def roofline(wl, per_step_stats, g):
    """HBM roofline of the dominant kernel (largest share of the step, from the library's CUDA
    events on the launching stream), with the algorithmic-byte models written out below (lower
    bounds of what each kernel must move). The other major kernels are reported beside it."""
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = peaks.get("hbm_gbs")
    src = "measured"
    if not peak:
        peak, src = 6800.0, "fallback"
    entries = []
    for r, s in wl["rs"]:
        st = per_step_stats[-1][(r, s)]
        n_r, n_s = st["n_r"], st["n_s"]
        destroyed, decs = st["listed"], st["decrements"]
        t_count = statistics.mean(x[(r, s)]["t_count_ms"] for x in per_step_stats) / 1000.0
        t_peel = statistics.mean(x[(r, s)]["t_peel_ms"] for x in per_step_stats) / 1000.0
        if (r, s) == (3, 4):
            # count: per triangle 3 edge ids (12 B) + 6 list bounds (48 B) + the count (4 B); per
            # (triangle, common neighbour) the entry in the two lists intersected (8 B); sum = 4 n_4
            count_b = 64 * n_r + 8 * 4 * n_s
            # peel: per triangle edge ids, list bounds, entry offsets (72 B); per destroyed
            # 4-clique its fourth vertex and the three sibling entries' tag and id (28 B); per
            # decrement a count read + write (8 B)
            peel_b = 72 * n_r + 28 * destroyed + 8 * decs
        elif (r, s) == (2, 3):
            # count: per edge endpoints (8 B) + 2 row bounds (32 B) + count (4 B); per (edge,
            # common neighbour) the entry in both rows (8 B); sum = 3 n_3
            count_b = 44 * n_r + 8 * 3 * n_s
            # peel: per edge endpoints + row bounds (40 B); per destroyed triangle the two other
            # edge ids and their rounds (16 B); per decrement read + write (8 B)
            peel_b = 40 * n_r + 16 * destroyed + 8 * decs
        elif (r, s) == (2, 4):
            w = st["count_width"]
            # count (DG listing): per edge its DG entry (8 B) and count (w B); per 4-clique the
            # fourth vertex's DG entry (8 B) and its six edge counts (read + write, 2w B each)
            count_b = (8 + w) * n_r + (8 + 12 * w) * n_s
            # peel: per edge endpoints + row bounds (40 B); per destroyed 4-clique the DG entry of
            # its last edge (8 B) and the rounds of its five other edges (20 B); per decrement a
            # count read + write
            peel_b = 40 * n_r + 28 * destroyed + 2 * w * decs
        else:
            count_b = peel_b = 0
        entries.append(("k_count%d%d" % (r, s), count_b, t_count))
        entries.append(("k_peel_loop(%d,%d)" % (r, s), peel_b, t_peel))
    entries.sort(key=lambda e: -e[2])
    traffic = NCU_TRAFFIC.get(sources_fingerprint(), {})

    def one(name, b, t):
        a = b / t / 1e9 if t > 0 else 0.0
        return {"bound": "hbm", "kernel": name, "achieved": a, "peak": peak, "unit": "GB/s", "frac": a / peak,
                "traffic": traffic.get((wl.get("name"), name)), "peak_source": src + " (hbm_gbs)",
                "algorithmic_bytes_per_launch": b, "avg_launch_ms": 1000.0 * t}

    top = one(*entries[0])
    top["others"] = [one(*e) for e in entries[1:]]
    return top


def e2e(nd, wl, g, local, width, steps, world, pg):
    import numpy as np
    import torch

    rp_h = torch.from_numpy(g.rowptr).pin_memory()
    col_h = torch.from_numpy(g.col).pin_memory()
    stream = torch.cuda.Stream(device=local)
    ctx = nd.nd_ctx_create(local, stream=stream)
    outs = {}
    h2d = rp_h.numel() * 8 + col_h.numel() * 4
    d2h = 0
    units = 0

    def one():
        nonlocal d2h, units
        G = nd.nd_load_csr(ctx, rp_h, col_h)
        d2h = 0
        units = 0
        for r, s in wl["rs"]:
            core = outs.get((r, s))
            if core is None:
                _, _, st = nd.nd_decompose(G, r, s, count_width=width, want_round=False)
                outs[(r, s)] = torch.empty(st["n_r"], dtype=torch.int32).pin_memory()
                core = outs[(r, s)]
            _, _, st = nd.nd_decompose(G, r, s, count_width=width, core_out=core, want_round=False)
            d2h += 4 * st["n_r"]
            units += units_of(r, s, st["n_s"])
        nd.nd_graph_free(G)

    one()  # warm-up (allocations, first-touch of pinned outputs)
    torch.cuda.synchronize()
    barrier(pg, local)
    t0 = time.perf_counter()
    for _ in range(steps):
        one()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    dt = max_over_ranks(pg, dt, local)
    nd.nd_ctx_destroy(ctx)
    return {"value": units * steps * world / dt, "unit": "s-cliques/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "steps": steps}


# ------------------------------------------------------------------------------------------
# batched and served workloads

def batch_graphs(count: int, seed: int = 4):
    """The batched workload: graphgen.batch_workload (Chung-Lu, n ~ U[50, 5000], average degree
    ~ U[8, 40], exponent 2.2; (r,s) uniform over (1,2), (2,3), (3,4))."""
    return gg.batch_workload(count, seed)


def run_batch(args, nd, world, rank, local, pg):
    """Config: 4,096 small graphs of mixed (r,s), one nd_batch_run per batch, against one
    load + decompose per graph (the plain path); host inputs and outputs in both."""
    import numpy as np

    items = batch_graphs(args.batch_graphs)
    ctx = nd.nd_ctx_create(local)
    graphs = [(g.rowptr, g.col, r, s) for g, (r, s) in items]
    # output buffers sized once
    outs, n_r, status, st0 = nd.nd_batch_run(ctx, graphs)
    assert all(x == nd.ND_OK for x in status)
    units = 0
    n_s_of = []
    for (g, (r, s)) in items:
        G = nd.nd_load_csr(ctx, g.rowptr, g.col)
        _, _, n_s = nd.nd_count(G, r, s)
        nd.nd_graph_free(G)
        n_s_of.append(n_s)
        units += units_of(r, s, n_s)
    bufs = [np.zeros(max(k, 1), np.int32) for k in n_r]
    for _ in range(args.warmup):
        nd.nd_batch_run(ctx, graphs, bufs)
    launches0 = nd.nd_kernel_launches()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _, _, _, st = nd.nd_batch_run(ctx, graphs, bufs)
    t_batch = (time.perf_counter() - t0) / args.steps
    launches_batch = (nd.nd_kernel_launches() - launches0) // args.steps
    # plain path: one graph at a time
    t0 = time.perf_counter()
    launches0 = nd.nd_kernel_launches()
    for (g, (r, s)), b in zip(items, bufs):
        G = nd.nd_load_csr(ctx, g.rowptr, g.col)
        nd.nd_decompose(G, r, s, core_out=b, want_round=False)
        nd.nd_graph_free(G)
    t_plain = time.perf_counter() - t0
    launches_plain = nd.nd_kernel_launches() - launches0
    nd.nd_ctx_destroy(ctx)
    t_batch = max_over_ranks(pg, t_batch, local)
    t_plain = max_over_ranks(pg, t_plain, local)
    line = {"metric": "batched (r,s) s-cliques/sec", "value": units * world / t_batch, "unit": "s-cliques/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t_batch,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": "batch", "graphs": len(items),
                       "desc": "Chung-Lu graphs, n~U[50,5000], avg degree~U[8,40], exponent 2.2, "
                               "(r,s) uniform over (1,2),(2,3),(3,4); host CSR in, host cores out",
                       "m_total": int(sum(g.m for g, _ in items))},
            "plain_one_graph_at_a_time": {"value": units * world / t_plain, "ms": 1000 * t_plain,
                                          "gpu_launches": launches_plain},
            "speedup_vs_plain": t_plain / t_batch, "gpu_launches": launches_batch,
            "batch_stats": {k: st[k] for k in ("groups", "requests", "n_r_total", "n_s_total", "rho_max")}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def serve_pool(count: int, seed: int = 5):
    """Graphs of the served stream: graphgen.serve_pool (Chung-Lu or R-MAT, edge count
    log-uniform in [1e2, 1e6])."""
    return gg.serve_pool(count, seed)


def run_serve(args, nd, world, rank, local, pg):
    """Config: a Poisson stream of requests against the continuous-batching server, compared
    with serial one-at-a-time handling of the same trace on the same GPU."""
    import threading

    import numpy as np

    pool = serve_pool(args.serve_pool)
    rs_choices = [(2, 3), (3, 4), (2, 4)]
    rng = np.random.default_rng(5 + rank)
    horizon = args.serve_seconds
    gaps = rng.exponential(1.0 / args.serve_rate, size=int(args.serve_rate * horizon * 1.2) + 16)
    arrivals = np.cumsum(gaps)
    arrivals = arrivals[arrivals < horizon]
    picks = rng.integers(0, len(pool), size=arrivals.size)
    rsi = rng.integers(0, 3, size=arrivals.size)
    ctx = nd.nd_ctx_create(local)
    # per (graph, rs): n_r, n_s and the plain service time (load + decompose + copy out)
    info = {}
    for gi, ri in set(zip(picks.tolist(), rsi.tolist())):
        g = pool[gi]
        r, s = rs_choices[ri]
        G = nd.nd_load_csr(ctx, g.rowptr, g.col)
        _, n_r, n_s = nd.nd_count(G, r, s)
        nd.nd_graph_free(G)
        info[(gi, ri)] = [n_r, n_s, 0.0]
    for key in info:  # warm, then time each distinct request once
        g = pool[key[0]]
        r, s = rs_choices[key[1]]
        for rep in range(2):
            t0 = time.perf_counter()
            G = nd.nd_load_csr(ctx, g.rowptr, g.col)
            nd.nd_decompose(G, r, s, want_round=False)
            nd.nd_graph_free(G)
            info[key][2] = time.perf_counter() - t0
    # serial FIFO on the same trace (Lindley recursion over measured service times)
    lat_fifo = np.zeros(arrivals.size)
    free_at = 0.0
    for i in range(arrivals.size):
        start = max(arrivals[i], free_at)
        free_at = start + info[(int(picks[i]), int(rsi[i]))][2]
        lat_fifo[i] = free_at - arrivals[i]
    fifo_span = free_at
    # live server
    sv = nd.nd_server_create(ctx, workers=args.serve_workers, max_batch=256, queue_cap=1 << 20)
    lat = []
    done = threading.Event()
    pending = {}
    lock = threading.Lock()

    def poller():
        while not done.is_set() or pending:
            with lock:
                items = list(pending.items())
            for t, _ in items:
                rc, res = sv.poll(t)
                if rc != nd.ND_PENDING:
                    with lock:
                        pending.pop(t, None)
                    if rc == nd.ND_OK:
                        lat.append(res["latency_ms"])
            time.sleep(0.0005)

    th = threading.Thread(target=poller, daemon=True)
    th.start()
    t0 = time.perf_counter()
    rejected = 0
    for i in range(arrivals.size):
        wait = arrivals[i] - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        g = pool[int(picks[i])]
        r, s = rs_choices[int(rsi[i])]
        out = np.empty(max(info[(int(picks[i]), int(rsi[i]))][0], 1), np.int32)
        try:
            t = sv.submit(g.rowptr, g.col, r, s, out)
            with lock:
                pending[t] = True
        except nd.NdError:
            rejected += 1
    done.set()
    sv.drain()
    th.join()
    span = time.perf_counter() - t0
    sv.close()
    nd.nd_ctx_destroy(ctx)
    units = sum(units_of(*rs_choices[int(rsi[i])], info[(int(picks[i]), int(rsi[i]))][1]) for i in range(arrivals.size))
    lat = np.array(lat)
    line = {"metric": "served (r,s) s-cliques/sec", "value": units * world / span, "unit": "s-cliques/s",
            "n_gpus": world, "steps": 1, "warmup": 0, "ms_per_step": 1000 * span, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "serve", "rate_per_s": args.serve_rate, "seconds": horizon,
                       "requests": int(arrivals.size), "pool_graphs": len(pool), "workers": args.serve_workers,
                       "desc": "Poisson arrivals; graphs Chung-Lu or R-MAT, m log-uniform [1e2, 1e6], "
                               "(r,s) uniform over (2,3),(3,4),(2,4); graphs pre-generated in host memory"},
            "served": {"requests_per_s": len(lat) / span, "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
                       "p99_ms": float(np.percentile(lat, 99)) if lat.size else None, "completed": int(lat.size),
                       "rejected": rejected, "span_s": span},
            "serial_fifo": {"requests_per_s": arrivals.size / fifo_span, "p50_ms": float(np.percentile(lat_fifo, 50) * 1000),
                            "p99_ms": float(np.percentile(lat_fifo, 99) * 1000), "span_s": fifo_span}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
