"""Oracle results for many graphs at once, in a pool of host processes started with spawn (a
process forked after the GPU was initialised could hang, so the pool never forks)."""
import multiprocessing as mp
import os

import numpy as np


class _G:
    def __init__(self, n, rowptr, col):
        self.n, self.rowptr, self.col = n, rowptr, col


def _core(args):
    import oracle as orc

    n, rowptr, col, r, s = args
    return orc.decompose(_G(n, rowptr, col), r, s).core


def oracle_cores(items, procs=None):
    """[oracle.decompose(g, r, s).core for g, r, s in items], computed in parallel."""
    procs = procs or min(16, os.cpu_count() or 1)
    jobs = [(g.n, np.ascontiguousarray(g.rowptr), np.ascontiguousarray(g.col), r, s) for g, r, s in items]
    # the longest jobs first, so that the pool's tail is short
    order = sorted(range(len(jobs)), key=lambda i: -(jobs[i][2].size * (jobs[i][4] - jobs[i][3] + jobs[i][3])))
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_core, [jobs[i] for i in order], chunksize=1)
    out = [None] * len(jobs)
    for i, c in zip(order, res):
        out[i] = c
    return out
