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

Beside ``value`` the line carries:
  * ``e2e``: the same metric through the C ABI with pinned host buffers (CSR upload and the
    core numbers' download inside the timed region);
  * ``roofline``: HBM roofline of the dominant kernel, with two algorithmic byte models (see
    ``byte_models``): the lower bound written from the method (smaller-list reads per r-clique,
    (C(s,r) - 1) x (1 B state + 4 B id probe) per listed s-clique, 2w per decrement, the A lists),
    and the tighter per-kernel model of the data this implementation must touch;
  * ``cpu_baseline``: the CPU oracle (single-threaded C) on R-MAT scale 12 of the same family, and
    the GPU on that identical graph in the same process, with the host's core count and model;
  * ``configs`` (single GPU, default workload): the other workloads -- Chung-Lu 2k (2,3), Chung-Lu
    4M with planted communities (3,4)+(2,4) in int64 tallies, the batch of 4,096 small graphs
    (autotuned nd_batch_run against one graph at a time), and the served Poisson stream at
    2,000 requests/s for 60 s against a live serial plain-GPU run of the same trace.

--impl reference times the CPU oracle (test infrastructure, single-threaded C) on a bounded
sample of the same workload (a smaller R-MAT with the same parameters), on the host cores.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import threading
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
    "rmat_dense": dict(
        desc="R-MAT scale 16, edge factor 32, a=0.5 b=0.1 c=0.1 (the denser family of Fig. 13); (2,5), (3,5)",
        gen=lambda: gg.rmat(16, 32, 0.5, 0.1, 0.1, seed=7),
        rs=[(2, 5), (3, 5)],
        sample=lambda scale: gg.rmat(scale, 32, 0.5, 0.1, 0.1, seed=7),
        sample_desc="R-MAT scale {scale}, edge factor 32, a=0.5 b=0.1 c=0.1, (2,5) and (3,5)",
    ),
}

# The density sweep of Fig. 13: R-MAT with a=0.5, b=c=0.1 (d=0.3), duplicate edges removed, at
# several edge factors, for (2,3), (3,4) and (4,5).
SWEEP_SCALE = 17
SWEEP_EDGE_FACTORS = [8, 16, 32, 64]
SWEEP_RS = [(2, 3), (3, 4), (4, 5)]


def units_of(r: int, s: int, n_s: int) -> int:
    """s-cliques of Algorithm 2: each counted once, then re-listed once per member r-clique."""
    return (1 + math.comb(s, r)) * n_s


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["batch", "serve", "sweep"], default="rmat20")
    ap.add_argument("--batch-graphs", type=int, default=4096)
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-pool", type=int, default=256)
    ap.add_argument("--serve-workers", type=int, default=4)
    ap.add_argument("--serve-batch", type=int, default=256, help="most requests merged into one server batch")
    ap.add_argument("--serve-mode", choices=["loop_graph", "persistent"], default="loop_graph",
                    help="how the server's workers launch a batch's peeling loop")
    ap.add_argument("--serve-queue", type=int, default=4096,
                    help="requests waiting for admission beyond which new ones are rejected (both arms)")
    ap.add_argument("--serve-drain", type=float, default=30.0,
                    help="seconds after the last arrival that each arm may take to finish its queue")
    ap.add_argument("--no-serial", action="store_true", help="serve workload: skip the serial arm")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the other workloads in the default run")
    ap.add_argument("--config-steps", type=int, default=3, help="timed steps of each secondary workload")
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


def cpu_info() -> dict:
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return {"cpu_model": model or platform.processor() or platform.machine(), "nproc": os.cpu_count(),
            "machine": platform.machine()}


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
    wl = WORKLOADS[args.workload] if args.workload in WORKLOADS else WORKLOADS["rmat20"]
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
            "cpu_baseline": dict({"value": value, "unit": "s-cliques/s", "cores": 1, "kind": "oracle",
                                  "sample": sample}, **cpu_info()),
            "e2e": {"value": value, "unit": "s-cliques/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------
# timed steps on a resident graph

def peel_flags(nd, args) -> int:
    f = {"default": 0, "persistent": nd.ND_PEEL_PERSISTENT, "loop_graph": nd.ND_PEEL_LOOP_GRAPH,
         "plain": nd.ND_NO_GRAPH}[args.peel_mode]
    f |= {"default": 0, "off": nd.ND_CONTRACT_OFF, "always": nd.ND_CONTRACT_ALWAYS}[args.contract]
    if args.dense_buckets:
        f |= nd.ND_DENSE_BUCKETS
    return f


class Resident:
    """A graph loaded once in device memory, stepped through the whole hot path."""

    def __init__(self, nd, g, local, stream):
        import torch

        self.nd, self.g, self.local, self.stream = nd, g, local, stream
        self.ctx = nd.nd_ctx_create(local, stream=stream)
        rp = torch.from_numpy(g.rowptr).to(f"cuda:{local}")
        col = torch.from_numpy(g.col).to(f"cuda:{local}")
        torch.cuda.synchronize()
        self.G = nd.nd_load_csr(self.ctx, rp, col)
        del rp, col
        self.outs = {}

    def step(self, rs, width, flags):
        import torch

        nd = self.nd
        nd.nd_graph_reset(self.G)  # every step rebuilds orientation and indexes
        stats = {}
        for r, s in rs:
            core = self.outs.get((r, s))
            if core is None:  # first warm-up step: learn n_r, then keep a device output buffer
                _, _, st = nd.nd_decompose(self.G, r, s, count_width=width, want_round=False, flags=flags)
                self.outs[(r, s)] = torch.empty(max(st["n_r"], 1), dtype=torch.int32, device=f"cuda:{self.local}")
            else:
                _, _, st = nd.nd_decompose(self.G, r, s, count_width=width, core_out=core, want_round=False,
                                           flags=flags)
            stats[(r, s)] = st
        return stats

    def timed(self, rs, width, flags, steps, warmup, flush, pg=None, sample_clocks=False):
        """W untimed steps, then K steps each bracketed by CUDA events on the library's stream, the
        L2 flushed before each (outside the events). Returns per-step stats, total ms, launches,
        host wall seconds and the clocks sampled meanwhile."""
        import torch

        nd = self.nd
        for _ in range(warmup):
            self.step(rs, width, flags)
        sampler = ClockSampler(gpu_uuid(self.local)) if sample_clocks else None
        barrier(pg, self.local)
        torch.cuda.synchronize()
        if sampler:
            sampler.start()
        launches0 = nd.nd_kernel_launches()
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        per_step = []
        wall0 = time.perf_counter()
        for i in range(steps):
            flush.fill_(i & 0xFF)  # evict the previous step's data from L2 (not timed)
            with torch.cuda.stream(self.stream):
                ev0[i].record(self.stream)
                per_step.append(self.step(rs, width, flags))
                ev1[i].record(self.stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        launches = nd.nd_kernel_launches() - launches0
        clocks = sampler.stop() if sampler else None
        barrier(pg, self.local)
        t_ms = sum(a.elapsed_time(b) for a, b in zip(ev0, ev1))
        return per_step, t_ms, launches, wall, clocks

    def close(self):
        self.nd.nd_graph_free(self.G)
        self.nd.nd_ctx_destroy(self.ctx)


STAT_KEYS = ("n_r", "n_s", "rho", "max_core", "listed", "decrements", "advances", "refills", "count_width",
             "t_orient_ms", "t_index_ms", "t_count_ms", "t_hash_ms", "t_peel_ms", "t_total_ms", "t_phase_ms", "t_contract_ms",
             "contractions")


def per_rs_summary(stats, rs):
    return {f"({r},{s})": dict(
        {k: stats[(r, s)][k] for k in STAT_KEYS},
        # the count phase alone (s-cliques counted per second) and the peel alone
        n_s_per_s_count=stats[(r, s)]["n_s"] / max(stats[(r, s)]["t_count_ms"], 1e-9) * 1e3,
        n_r_per_s_peel=stats[(r, s)]["n_r"] / max(stats[(r, s)]["t_peel_ms"], 1e-9) * 1e3) for r, s in rs}


# ------------------------------------------------------------------------------------------
# roofline

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of single-kernel ncu captures
# (one launch each, -k <kernel> -c 1, --clock-control none) on R-MAT scale 17 of the same family,
# scaled to a full R-MAT scale 20 launch by the s-cliques each processes (n_s of scale 20 / n_s of
# scale 17): the traffic of these kernels grows with the s-cliques listed. Keyed by the fingerprint
# of the library sources the captures were taken on; reported only while the sources still match.
NCU_TRAFFIC = {
    # R-MAT scale 17 (n_4 = 819,091,962): k_peel_loop (3,4) 247.50 GB read + 39.52 GB written, k_count34
    # 54.53 GB + 0.56 GB; scaled by 16,996,482,431 / 819,091,962 = 20.750. The (2,3) kernels are not
    # listed: at scale 17 their arrays fit in L2, so their DRAM bytes do not scale.
    "37514f67ef4c48be": {
        ("rmat20", "k_peel_loop(3,4)"): 5.9558e+12,
        ("rmat20", "k_count34"): 1.1432e+12,
    },
}


# translation units that no kernel of the timed step includes or calls (the connected nuclei and the
# hierarchy, run outside the step): a change there leaves the captured kernels' traffic as it was
NOT_IN_STEP = ("nd_nuclei.cu",)


def sources_fingerprint():
    import glob
    import hashlib

    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_2111_10980_gb300", "csrc", "*"))):
        if os.path.basename(f) in NOT_IN_STEP:
            continue
        if f.endswith((".cu", ".cuh", ".h")):
            h.update(os.path.basename(f).encode())
            with open(f, "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def graph_sums(nd, res: Resident, need_tri: bool) -> dict:
    """Exact sums over the graph that the byte models need, computed on the GPU with torch from the
    graph and the library's r-clique tuples (measurement plumbing, untimed): deg = degree, d+ =
    out-degree in the (degree, id) orientation; over edges sum min(deg) and sum (d+(u) + d+(v));
    over triangles sum min(deg) and sum d+(last vertex in the orientation)."""
    import numpy as np
    import torch

    g = res.g
    dev = f"cuda:{res.local}"
    n = g.n
    deg = torch.from_numpy(np.diff(g.rowptr)).to(dev)
    rows = torch.repeat_interleave(torch.arange(n, device=dev), deg)
    col = torch.from_numpy(g.col).to(dev).long()
    after = (deg[col] > deg[rows]) | ((deg[col] == deg[rows]) & (col > rows))
    dplus = torch.zeros(n, dtype=torch.int64, device=dev).scatter_add_(0, rows, after.long())
    up = col > rows
    eu, ev = rows[up], col[up]
    out = {"sum_deg": int(deg.sum().item()),
           "edge_min_deg": int(torch.minimum(deg[eu], deg[ev]).sum().item()),
           "edge_dplus": int((dplus[eu] + dplus[ev]).sum().item())}
    del rows, col, after, up, eu, ev
    if need_tri:
        c = ctypes.c_int64()
        nd.lib().nd_rcliques(res.G.ptr, 3, None, 0, ctypes.byref(c))
        n3 = c.value
        tmin, tdp = 0, 0
        if n3:
            t = torch.empty((n3, 3), dtype=torch.int32, device=dev)
            nd.nd_rcliques(res.G, 3, out=t)
            key = deg * n + torch.arange(n, device=dev)  # the orientation's total order
            for lo in range(0, n3, 1 << 26):
                tt = t[lo:lo + (1 << 26)].long()
                tmin += int(deg[tt].min(dim=1).values.sum().item())
                last = tt.gather(1, key[tt].argmax(dim=1, keepdim=True)).squeeze(1)
                tdp += int(dplus[last].sum().item())
                del tt, last
            del t
        out.update(n3=n3, tri_min_deg=tmin, tri_dplus_last=tdp)
    torch.cuda.empty_cache()
    return out


def byte_models(r, s, st, sums, g):
    """(count bytes, peel bytes) of two models for one (r,s) decomposition.

    "method": the lower bound written from the method. Count: s = 3, r = 2 reads both out-lists of
    every DG edge, 4 (d+(u) + d+(v)) B, and reads + writes each count (2w B); s = 4 adds the
    out-list of the last vertex of every triangle, 4 d+ B; r = 1 reads the row pointers. Peel: per
    r-clique its smaller neighbour list (4 min deg B, the intersection bound of Lemma 4.1), per
    listed s-clique -- each s-clique listed once per member r-clique, C(s,r) n_s listings -- 1 B of
    state and a 4 B id probe for each of its other C(s,r) - 1 r-subsets, per decrement a count read
    and write (2w B), and each r-clique written to and read from A once (8 B).

    "implementation": what these kernels must touch at the least in their own data layout: the
    peel of (3,4) per triangle its edge ids, list bounds and entry offsets (72 B), per destroyed
    4-clique its fourth vertex and the three sibling entries' tag and id (28 B), 8 B per decrement;
    (2,3) per edge endpoints and row bounds (40 B), per destroyed triangle the two other edge ids
    and their rounds (16 B), 8 B per decrement; (2,4) per edge 40 B, per destroyed 4-clique the DG
    entry of its last edge and the rounds of its five other edges (28 B), 2w per decrement.
    Counting: (2,3) 44 m + 8 (3 n_3); (3,4) 64 n_3 + 8 (4 n_4); (2,4) (8 + w) m + (8 + 12 w) n_4."""
    w = st["count_width"]
    n_r, n_s, decs, destroyed = st["n_r"], st["n_s"], st["decrements"], st["listed"]
    C = math.comb(s, r)
    if r == 1:
        count_m = 8 * (g.n + 1)
    elif s == r + 1 and r == 2:
        count_m = 4 * sums["edge_dplus"] + 2 * w * n_r
    else:
        count_m = 4 * sums["edge_dplus"] + 4 * sums.get("tri_dplus_last", 0) + 2 * w * n_r
    minsum = {1: sums["sum_deg"], 2: sums["edge_min_deg"], 3: sums.get("tri_min_deg", 0)}[r]
    peel_m = 4 * minsum + C * n_s * (C - 1) * 5 + 2 * w * decs + 8 * n_r
    if (r, s) == (3, 4):
        count_i, peel_i = 64 * n_r + 8 * 4 * n_s, 72 * n_r + 28 * destroyed + 8 * decs
    elif (r, s) == (2, 3):
        count_i, peel_i = 44 * n_r + 8 * 3 * n_s, 40 * n_r + 16 * destroyed + 8 * decs
    elif (r, s) == (2, 4):
        count_i, peel_i = (8 + w) * n_r + (8 + 12 * w) * n_s, 40 * n_r + 28 * destroyed + 2 * w * decs
    else:
        count_i, peel_i = count_m, peel_m
    return count_m, peel_m, count_i, peel_i


def roofline(wl_name, rs, per_step_stats, g, sums):
    """HBM roofline of the dominant kernel (largest share of the step, from the library's CUDA
    events on the launching stream), the other major kernels beside it. ``frac`` uses the method's
    lower-bound model; ``frac_implementation`` the tighter model of this implementation's data."""
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
    for r, s in rs:
        st = per_step_stats[-1][(r, s)]
        # the counting kernel alone: (3,4) builds the hash directory inside the counting interval
        t_count = statistics.mean(x[(r, s)]["t_count_ms"] - x[(r, s)].get("t_hash_ms", 0.0)
                                  for x in per_step_stats) / 1000.0
        t_peel = statistics.mean(x[(r, s)]["t_peel_ms"] for x in per_step_stats) / 1000.0
        cm, pm, ci, pi = byte_models(r, s, st, sums, g)
        entries.append(("k_count%d%d" % (r, s), cm, ci, t_count))
        entries.append(("k_peel_loop(%d,%d)" % (r, s), pm, pi, t_peel))
    entries.sort(key=lambda e: -e[3])
    traffic = NCU_TRAFFIC.get(sources_fingerprint(), {})

    def one(name, bm, bi, t):
        a = bm / t / 1e9 if t > 0 else 0.0
        ai = bi / t / 1e9 if t > 0 else 0.0
        return {"bound": "hbm", "kernel": name, "achieved": a, "peak": peak, "unit": "GB/s", "frac": a / peak,
                "traffic": traffic.get((wl_name, name)), "peak_source": src + " (hbm_gbs)",
                "algorithmic_bytes_per_launch": bm, "avg_launch_ms": 1000.0 * t,
                "model": "method lower bound", "achieved_implementation": ai, "frac_implementation": ai / peak,
                "implementation_bytes_per_launch": bi}

    top = one(*entries[0])
    top["others"] = [one(*e) for e in entries[1:]]
    top["graph_sums"] = sums
    return top


def e2e(nd, rs, g, local, width, steps, world, pg):
    """The same metric through the C ABI with host buffers: every step uploads the CSR from pinned
    host memory and downloads every core array to pinned host memory."""
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
        for r, s in rs:
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


def secondary(nd, name, steps, local, flush, stream, flags=0):
    """One of the other graph workloads, resident, timed like the main one (fewer steps)."""
    wl = WORKLOADS[name]
    t0 = time.perf_counter()
    g = wl["gen"]()
    gen_s = time.perf_counter() - t0
    width = wl.get("width", 0)
    res = Resident(nd, g, local, stream)
    per_step, t_ms, launches, wall, _ = res.timed(wl["rs"], width, flags, steps, 1, flush)
    stats = per_step[-1]
    units = sum(units_of(r, s, stats[(r, s)]["n_s"]) for r, s in wl["rs"])
    sums = graph_sums(nd, res, need_tri=any(r == 3 or s >= 4 for r, s in wl["rs"]))
    roof = roofline(name, wl["rs"], per_step, g, sums)
    res.close()
    peel_s = sum(x[(r, s)]["t_peel_ms"] for x in per_step for r, s in wl["rs"]) / 1000.0
    return {"workload": name, "desc": wl["desc"], "n": g.n, "m": g.m, "value": units * steps / (t_ms / 1000.0),
            "unit": "s-cliques/s", "ms_per_step": t_ms / steps, "steps": steps,
            "dtype": "int64" if width == 8 else "int32", "gpu_launches": launches,
            "r_cliques_peeled_per_s": sum(stats[(r, s)]["n_r"] for r, s in wl["rs"]) * steps / max(peel_s, 1e-9),
            "per_rs": per_rs_summary(stats, wl["rs"]), "roofline": roof, "generate_s": gen_s}


def density_sweep(nd, local, flush, stream, steps=2):
    """Fig. 13's R-MAT density sweep: s-cliques/s of (2,3), (3,4), (4,5) as the edge factor grows."""
    out = []
    for ef in SWEEP_EDGE_FACTORS:
        g = gg.rmat(SWEEP_SCALE, ef, 0.5, 0.1, 0.1, seed=7)
        res = Resident(nd, g, local, stream)
        row = {"scale": SWEEP_SCALE, "edge_factor": ef, "n": g.n, "m": g.m, "rs": {}}
        for r, s in SWEEP_RS:
            per_step, t_ms, _, _, _ = res.timed([(r, s)], 0, 0, steps, 1, flush)
            st = per_step[-1][(r, s)]
            row["rs"][f"({r},{s})"] = {"n_r": st["n_r"], "n_s": st["n_s"], "rho": st["rho"], "max_core": st["max_core"],
                                       "ms": t_ms / steps, "s_cliques_per_s": units_of(r, s, st["n_s"]) * steps /
                                       (t_ms / 1000.0)}
        res.close()
        out.append(row)
    return {"desc": f"R-MAT scale {SWEEP_SCALE}, a=0.5 b=0.1 c=0.1, edge factors {SWEEP_EDGE_FACTORS}, duplicates "
                    "removed; one step = index + count + peel of one (r,s)", "points": out}


# ------------------------------------------------------------------------------------------
# batched and served workloads

def batch_graphs(count: int, seed: int = 4):
    """The batched workload: graphgen.batch_workload (Chung-Lu, n ~ U[50, 5000], average degree
    ~ U[8, 40], exponent 2.2; (r,s) uniform over (1,2), (2,3), (3,4))."""
    return gg.batch_workload(count, seed)


def batch_result(nd, count, steps, warmup, local):
    """4,096 small graphs of mixed (r,s): nd_batch_run per batch (one union decomposition per (r,s),
    peel schedule autotuned on a sample of 512 of the graphs), against one load + decompose per
    graph (the plain path); host CSRs in and host core arrays out in both."""
    import numpy as np

    from paper_2111_10980_gb300 import autotune

    items = batch_graphs(count)
    ctx = nd.nd_ctx_create(local)
    graphs = [(g.rowptr, g.col, r, s) for g, (r, s) in items]
    t0 = time.perf_counter()
    tuning = autotune.tune(ctx, graphs[:512])
    tune_s = time.perf_counter() - t0
    try:
        autotune.save(tuning)
    except OSError:
        pass
    outs, n_r, status, _ = nd.nd_batch_run(ctx, graphs)
    assert all(x == nd.ND_OK for x in status)
    units = 0
    for (g, (r, s)) in items:
        G = nd.nd_load_csr(ctx, g.rowptr, g.col)
        _, _, n_s = nd.nd_count(G, r, s)
        nd.nd_graph_free(G)
        units += units_of(r, s, n_s)
    bufs = [np.zeros(max(k, 1), np.int32) for k in n_r]
    for _ in range(warmup):
        nd.nd_batch_run(ctx, graphs, bufs)
    launches0 = nd.nd_kernel_launches()
    t0 = time.perf_counter()
    for _ in range(steps):
        _, _, _, st = nd.nd_batch_run(ctx, graphs, bufs)
    t_batch = (time.perf_counter() - t0) / steps
    launches_batch = (nd.nd_kernel_launches() - launches0) // steps
    # plain path: one graph at a time, default settings
    for (r, s) in {(r, s) for _, (r, s) in items}:
        nd.nd_ctx_set_tuning(ctx, r, s, 0, 0)
    t0 = time.perf_counter()
    launches0 = nd.nd_kernel_launches()
    for (g, (r, s)), b in zip(items, bufs):
        G = nd.nd_load_csr(ctx, g.rowptr, g.col)
        nd.nd_decompose(G, r, s, core_out=b, want_round=False)
        nd.nd_graph_free(G)
    t_plain = time.perf_counter() - t0
    launches_plain = nd.nd_kernel_launches() - launches0
    nd.nd_ctx_destroy(ctx)
    return {"metric": "batched (r,s) s-cliques/sec", "value": units / t_batch, "unit": "s-cliques/s",
            "ms_per_batch": 1000 * t_batch, "steps": steps, "graphs": len(items),
            "desc": "Chung-Lu graphs, n~U[50,5000], avg degree~U[8,40], exponent 2.2, (r,s) uniform over "
                    "(1,2),(2,3),(3,4); host CSR in, host cores out",
            "m_total": int(sum(g.m for g, _ in items)),
            "plain_one_graph_at_a_time": {"value": units / t_plain, "ms": 1000 * t_plain,
                                          "gpu_launches": launches_plain},
            "speedup_vs_plain": t_plain / t_batch, "gpu_launches": launches_batch,
            "batch_stats": {k: st[k] for k in ("groups", "requests", "n_r_total", "n_s_total", "rho_max")},
            "autotune": {"seconds": tune_s, "sample_graphs": 512,
                         "choice": {k: {"heavy_work": v["heavy_work"], "dense_buckets": v["dense_buckets"],
                                        "ms": v["ms"]} for k, v in tuning["rs"].items()}}}


def serve_pool(count: int, seed: int = 5):
    """Graphs of the served stream: graphgen.serve_pool (Chung-Lu or R-MAT, edge count
    log-uniform in [1e2, 1e6])."""
    return gg.serve_pool(count, seed)


def _latency_summary(lat_ms, censored_ms, span_s, offered, rejected):
    import numpy as np

    lat = np.array(lat_ms)
    allv = np.concatenate([lat, np.array(censored_ms)]) if censored_ms else lat
    return {"completed": int(lat.size), "requests_per_s": lat.size / span_s if span_s > 0 else None,
            "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
            "rejected": int(rejected), "unfinished_at_cutoff": len(censored_ms),
            "p99_ms_lower_bound_all_admitted": float(np.percentile(allv, 99)) if allv.size else None,
            "offered": int(offered), "span_s": span_s}


def serve_result(nd, seconds, rate, pool_size, workers, queue_cap, drain_s, local, seed=5, max_batch=256,
                 mode="loop_graph", serial=True):
    """A Poisson stream of requests against the continuous-batching server, and the same trace served
    live one request at a time on the same GPU (load + decompose + copy out, FIFO). Both arms admit
    at most queue_cap waiting requests and reject the rest; both stop drain_s after the last
    arrival, counting what is still queued or running as unfinished (with a latency lower bound)."""
    import collections

    import numpy as np

    pool = serve_pool(pool_size)
    rs_choices = [(2, 3), (3, 4), (2, 4)]
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=int(rate * seconds * 1.2) + 16)
    arrivals = np.cumsum(gaps)
    arrivals = arrivals[arrivals < seconds]
    picks = rng.integers(0, len(pool), size=arrivals.size)
    rsi = rng.integers(0, 3, size=arrivals.size)
    ctx = nd.nd_ctx_create(local)
    info = {}
    for gi, ri in sorted(set(zip(picks.tolist(), rsi.tolist()))):
        g = pool[gi]
        r, s = rs_choices[ri]
        G = nd.nd_load_csr(ctx, g.rowptr, g.col)
        _, n_r, n_s = nd.nd_count(G, r, s)
        nd.nd_graph_free(G)
        info[(gi, ri)] = (n_r, n_s)
    outs = {key: np.empty(max(v[0], 1), np.int32) for key, v in info.items()}

    # --- the server
    sv = nd.nd_server_create(ctx, workers=workers, max_batch=max_batch, queue_cap=queue_cap,
                             flags=nd.ND_PEEL_PERSISTENT if mode == "persistent" else nd.ND_PEEL_LOOP_GRAPH)
    lat, units_done = [], [0]
    pending = {}
    lock = threading.Lock()
    stop = threading.Event()
    t0 = time.perf_counter()

    def poller():
        while not stop.is_set():
            with lock:
                items = list(pending.items())
            for t, (arr, key) in items:
                rc, res = sv.poll(t)
                if rc != nd.ND_PENDING:
                    with lock:
                        pending.pop(t, None)
                    if rc == nd.ND_OK:
                        lat.append(res["latency_ms"])
                        units_done[0] += units_of(*rs_choices[key[1]], info[key][1])
            time.sleep(0.0005)

    th = threading.Thread(target=poller, daemon=True)
    th.start()
    rejected = 0
    for i in range(arrivals.size):
        wait = arrivals[i] - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        key = (int(picks[i]), int(rsi[i]))
        g = pool[key[0]]
        r, s = rs_choices[key[1]]
        try:
            t = sv.submit(g.rowptr, g.col, r, s, outs[key])
            with lock:
                pending[t] = (arrivals[i], key)
        except nd.NdError:
            rejected += 1
    while time.perf_counter() - t0 < seconds + drain_s:
        with lock:
            if not pending:
                break
        time.sleep(0.01)
    now = time.perf_counter() - t0
    with lock:
        censored = [1000.0 * (now - a) for a, _ in pending.values()]
    stop.set()
    th.join()
    sv.close()  # finishes what was admitted (not timed)
    server = _latency_summary(lat, censored, now, arrivals.size, rejected)
    server["s_cliques_per_s"] = units_done[0] / max(now, 1e-9)
    server.update(workers=workers, max_batch=max_batch, peel_mode=mode)
    out = {"metric": "served (r,s) requests/sec, p50/p99 latency", "rate_per_s": rate, "seconds": seconds,
           "requests": int(arrivals.size), "pool_graphs": len(pool), "queue_cap": queue_cap, "drain_s": drain_s,
           "desc": "Poisson arrivals; graphs Chung-Lu or R-MAT, m log-uniform [1e2, 1e6], (r,s) uniform over "
                   "(2,3),(3,4),(2,4); graphs pre-generated in host memory",
           "server": server}
    if not serial:
        nd.nd_ctx_destroy(ctx)
        return out

    # --- serial plain-GPU handling of the same trace, live
    q = collections.deque()
    cv = threading.Condition()
    lat2, units2, done_flag = [], [0], [False]
    t0 = time.perf_counter()

    def worker():
        while True:
            with cv:
                while not q and not done_flag[0]:
                    cv.wait(0.01)
                if not q:
                    return
                arr, key = q.popleft()
            if time.perf_counter() - t0 > seconds + drain_s:
                with cv:
                    q.appendleft((arr, key))
                return
            g = pool[key[0]]
            r, s = rs_choices[key[1]]
            G = nd.nd_load_csr(ctx, g.rowptr, g.col)
            nd.nd_decompose(G, r, s, core_out=outs[key], want_round=False)
            nd.nd_graph_free(G)
            lat2.append(1000.0 * (time.perf_counter() - t0 - arr))
            units2[0] += units_of(r, s, info[key][1])

    wt = threading.Thread(target=worker, daemon=True)
    wt.start()
    rejected2 = 0
    for i in range(arrivals.size):
        wait = arrivals[i] - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        with cv:
            if len(q) >= queue_cap:
                rejected2 += 1
            else:
                q.append((arrivals[i], (int(picks[i]), int(rsi[i]))))
                cv.notify()
    with cv:
        done_flag[0] = True
        cv.notify()
    wt.join()
    now = time.perf_counter() - t0
    with cv:
        censored2 = [1000.0 * (now - a) for a, _ in q]
        q.clear()
    serial = _latency_summary(lat2, censored2, now, arrivals.size, rejected2)
    serial["s_cliques_per_s"] = units2[0] / max(now, 1e-9)
    nd.nd_ctx_destroy(ctx)
    out["serial_plain_gpu"] = serial
    return out


# ------------------------------------------------------------------------------------------
# CPU baseline: the oracle and the GPU on identical graphs

def cpu_baseline(nd, local, flush, stream):
    import oracle as orc

    out = {}
    for name, g, rs in [("rmat12", gg.rmat(12, 16, 0.57, 0.19, 0.19, seed=2), [(2, 3), (3, 4)]),
                        ("cl2k", gg.chung_lu_2k(seed=1), [(2, 3)])]:
        t0 = time.perf_counter()
        units = 0
        for r, s in rs:
            units += units_of(r, s, orc.decompose(g, r, s).n_s)
        dt = time.perf_counter() - t0
        res = Resident(nd, g, local, stream)
        per_step, t_ms, _, _, _ = res.timed(rs, 0, 0, 10, 3, flush)
        res.close()
        gpu = units * 10 / (t_ms / 1000.0)
        out[name] = {"graph": g.name, "rs": [f"({r},{s})" for r, s in rs], "oracle_s": dt,
                     "oracle_value": units / dt, "gpu_value": gpu, "gpu_over_cpu": gpu / (units / dt)}
    base = out["rmat12"]
    return dict({"value": base["oracle_value"], "unit": "s-cliques/s", "cores": 1, "kind": "oracle",
                 "sample": "the whole R-MAT scale 12 graph of the same family (n=4096), (2,3) and (3,4), "
                           "single-threaded; the GPU runs the identical graph in the same process",
                 "same_graph": out}, **cpu_info())


# ------------------------------------------------------------------------------------------
# our arm

def main():
    args = parse_args()
    world, rank, local, pg = dist_setup(want_nccl=(args.impl == "ours"))
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import torch

    import paper_2111_10980_gb300 as nd

    torch.cuda.set_device(local)
    if args.workload == "batch":
        line = batch_result(nd, args.batch_graphs, args.steps, args.warmup, local)
        line.update(n_gpus=1, warmup=args.warmup, higher_is_better=True, scaling="weak", vs_baseline=None,
                    dtype="int32", data="synthetic", config={"workload": "batch", "graphs": args.batch_graphs})
        if rank == 0:
            print(json.dumps(line), flush=True)
        return 0
    if args.workload == "sweep":
        stream = torch.cuda.Stream(device=local)
        flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=f"cuda:{local}")
        line = density_sweep(nd, local, flush, stream, steps=args.steps)
        line.update(metric="(r,s) s-cliques/sec over an R-MAT density sweep", n_gpus=1, data="synthetic",
                    config={"workload": "sweep"})
        if rank == 0:
            print(json.dumps(line), flush=True)
        return 0
    if args.workload == "serve":
        line = serve_result(nd, args.serve_seconds, args.serve_rate, args.serve_pool, args.serve_workers,
                            args.serve_queue, args.serve_drain, local, seed=5 + rank, max_batch=args.serve_batch,
                            mode=args.serve_mode, serial=not args.no_serial)
        line.update(value=line["server"]["requests_per_s"], unit="requests/s", n_gpus=1, steps=1, warmup=0,
                    higher_is_better=True, scaling="weak", vs_baseline=None, dtype="int32", data="synthetic",
                    config={"workload": "serve", "rate_per_s": args.serve_rate, "seconds": args.serve_seconds})
        if rank == 0:
            print(json.dumps(line), flush=True)
        return 0
    wl = dict(WORKLOADS[args.workload])
    width = wl.get("width", 0)
    workload_name = args.workload
    default_run = args.workload == "rmat20" and args.scale is None and args.rs is None
    if args.scale is not None and args.workload == "rmat20":
        sc = args.scale
        wl["gen"] = lambda: gg.rmat(sc, 16, 0.57, 0.19, 0.19, seed=2)
        wl["desc"] = wl["desc"].replace("scale 20", f"scale {sc}")
        workload_name = f"rmat{sc}"
    if args.rs:
        wl["rs"] = [tuple(int(x) for x in p.split(",")) for p in args.rs.split(":")]
    g = wl["gen"]()
    stream = torch.cuda.Stream(device=local)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=f"cuda:{local}")
    pflags = peel_flags(nd, args)
    res = Resident(nd, g, local, stream)
    per_step_stats, t_ms, launches, wall, clocks = res.timed(wl["rs"], width, pflags, args.steps, args.warmup, flush,
                                                             pg=pg, sample_clocks=True)
    t_ms = max_over_ranks(pg, t_ms, local)

    stats = per_step_stats[-1]
    units_per_step = sum(units_of(r, s, stats[(r, s)]["n_s"]) for r, s in wl["rs"])
    rcl_per_step = sum(stats[(r, s)]["n_r"] for r, s in wl["rs"])
    value = units_per_step * args.steps * world / (t_ms / 1000.0)
    peel_ms = [sum(st[(r, s)]["t_peel_ms"] for r, s in wl["rs"]) for st in per_step_stats]
    peeled_per_s = rcl_per_step * args.steps * world / (sum(peel_ms) / 1000.0)
    sums = graph_sums(nd, res, need_tri=any(r == 3 or s >= 4 for r, s in wl["rs"]))
    roof = roofline(workload_name, wl["rs"], per_step_stats, g, sums)
    res.close()

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
            "per_rs": per_rs_summary(stats, wl["rs"]),
            "gpu_launches": launches,
            "roofline": roof,
            "clocks": clocks}

    if not args.no_e2e:
        line["e2e"] = e2e(nd, wl["rs"], g, local, width, args.e2e_steps, world, pg)
    del g

    if world == 1 and default_run and not args.no_configs:
        cfg = {}
        for key, name in (("chung_lu_2k", "cl2k"), ("chung_lu_4m_planted", "cl4m")):
            try:
                cfg[key] = secondary(nd, name, args.config_steps if name == "cl4m" else 20, local, flush, stream)
            except Exception as e:  # report it, keep the main line
                cfg[key] = {"error": repr(e)}
        try:
            cfg["rmat_density_sweep"] = density_sweep(nd, local, flush, stream)
        except Exception as e:
            cfg["rmat_density_sweep"] = {"error": repr(e)}
        for key, fn in (("batched_4096", lambda: batch_result(nd, args.batch_graphs, args.config_steps, 1, local)),
                        ("served_2000_per_s", lambda: serve_result(nd, args.serve_seconds, args.serve_rate,
                                                                   args.serve_pool, args.serve_workers,
                                                                   args.serve_queue, args.serve_drain, local,
                                                                   max_batch=args.serve_batch,
                                                                   mode=args.serve_mode))):
            try:
                cfg[key] = fn()
            except Exception as e:
                cfg[key] = {"error": repr(e)}
        line["configs"] = cfg

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(nd, local, flush, stream)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
