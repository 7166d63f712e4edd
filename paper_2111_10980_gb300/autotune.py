"""Autotuner of the batched and served paths: for each (r,s) it chooses how r-cliques are
scheduled in Update -- one warp each up to a driving-list length, one block each above it (the
heavy phase) -- and whether level advances use the dense buckets, by timing nd_batch_run on a
sample of the workload with every candidate. The choice is stored per device in a JSON file and
applied to a context with nd_ctx_set_tuning. Host-side orchestration only: every candidate runs
the library's own kernels.

    import paper_2111_10980_gb300 as nd
    from paper_2111_10980_gb300 import autotune
    res = autotune.tune(ctx, [(rowptr, col, r, s), ...])   # times the candidates
    autotune.save(res); autotune.apply(ctx, autotune.load())
"""
from __future__ import annotations

import json
import os
import time

from . import ND_DENSE_BUCKETS, nd_batch_run, nd_ctx_set_tuning

# driving-list lengths at which an r-clique moves from a warp to a block (0: the built-in one)
HEAVY_CANDIDATES = [0, 64, 256, 1024, 4096]
# (2,4) stages a warp's common neighbourhood in 96 entries of shared memory
HEAVY_CANDIDATES_STAGED = [0, 32, 64, 96]


def device_key() -> str:
    import torch

    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name.replace(' ', '_')}_sm{p.major}{p.minor}_{p.multi_processor_count}sms"


def default_path() -> str:
    base = os.environ.get("ND_TUNING_DIR") or os.path.join(os.path.expanduser("~"), ".cache", "paper_2111_10980_gb300")
    return os.path.join(base, f"tuning_{device_key()}.json")


def _time_batch(ctx, graphs, outs, reps: int) -> float:
    best = float("inf")
    for _ in range(reps):
        t0 = time.perf_counter()
        _, _, status, _ = nd_batch_run(ctx, graphs, outs)
        dt = time.perf_counter() - t0
        if any(x != 0 for x in status):
            raise RuntimeError("autotune: a request of the sample failed")
        best = min(best, dt)
    return best


def tune(ctx, graphs, reps: int = 2) -> dict:
    """Times every candidate on ``graphs`` (a list of (rowptr, col, r, s) host arrays), (r,s)
    group by (r,s) group, and returns {"device": ..., "rs": {"r,s": choice}}. Leaves ctx tuned
    with the winners."""
    import numpy as np

    groups: dict[tuple[int, int], list] = {}
    for item in graphs:
        groups.setdefault((int(item[2]), int(item[3])), []).append(item)
    out = {"device": device_key(), "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()), "rs": {}}
    for (r, s), items in sorted(groups.items()):
        nd_ctx_set_tuning(ctx, r, s, 0, 0)
        outs0, n_r, _, _ = nd_batch_run(ctx, items)
        outs = [np.zeros(max(k, 1), np.int32) for k in n_r]
        _time_batch(ctx, items, outs, 1)  # warm
        heavy = HEAVY_CANDIDATES_STAGED if (r, s) == (2, 4) else HEAVY_CANDIDATES
        tried = []
        for h in heavy:
            for dense in (False, True):
                nd_ctx_set_tuning(ctx, r, s, h, ND_DENSE_BUCKETS if dense else 0)
                t = _time_batch(ctx, items, outs, reps)
                tried.append({"heavy_work": h, "dense_buckets": dense, "ms": 1000.0 * t})
        best = min(tried, key=lambda x: x["ms"])
        nd_ctx_set_tuning(ctx, r, s, best["heavy_work"], ND_DENSE_BUCKETS if best["dense_buckets"] else 0)
        out["rs"][f"{r},{s}"] = dict(best, graphs=len(items), tried=tried)
    return out


def save(result: dict, path: str | None = None) -> str:
    path = path or default_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(result, f, indent=1)
    os.replace(tmp, path)
    return path


def load(path: str | None = None) -> dict | None:
    path = path or default_path()
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f)


def apply(ctx, result: dict | None) -> int:
    """Applies a stored choice to ctx; returns how many (r,s) were tuned."""
    if not result:
        return 0
    k = 0
    for key, c in result.get("rs", {}).items():
        r, s = (int(x) for x in key.split(","))
        nd_ctx_set_tuning(ctx, r, s, int(c["heavy_work"]), ND_DENSE_BUCKETS if c["dense_buckets"] else 0)
        k += 1
    return k
