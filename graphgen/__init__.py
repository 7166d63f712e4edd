"""Seeded synthetic graph generators shared by the CPU oracle tests and the GPU library.

Every generator returns a canonical symmetric CSR: ``rowptr`` (int64, n+1) and ``col``
(int32, 2m) with each neighbour list sorted ascending, no self-loops and no duplicate
edges. None of the nucleus-decomposition arithmetic lives here.

The workloads follow the graph families the paper measures on (power-law social and
web graphs, and R-MAT graphs, Section 6.1), at the sizes of the benchmark configurations:

* ``chung_lu``      Chung-Lu with power-law expected degrees ``w_i = c (i + i0)^(-1/(gamma-1))``,
                    exact O(n^2) Bernoulli sampling for small n, Miller-Hagberg skip sampling
                    otherwise (identical distribution);
* ``rmat``          R-MAT with quadrant probabilities a, b, c, d = 1-a-b-c, symmetrised and
                    deduplicated;
* ``planted``       disjoint dense communities (edge density p) on top of another graph;
* ``complete``, ``fig1``, ``gnp``, ``disjoint_union``, ``relabel`` for tests.

Random numbers come from xoshiro256** seeded through SplitMix64 (in ``_gen.c``).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "_gen.c")
_LIB = os.path.join(_HERE, "_libgraphgen.so")
_lock = threading.Lock()
_lib = None


def build_lib(force: bool = False) -> str:
    """Compile ``_gen.c`` into ``_libgraphgen.so`` next to it (plain gcc, no -march)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build_lib()
            lib = ctypes.CDLL(_LIB)
            i32p = ctypes.POINTER(ctypes.c_int32)
            i32pp = ctypes.POINTER(i32p)
            dp = ctypes.POINTER(ctypes.c_double)
            i64p = ctypes.POINTER(ctypes.c_int64)
            lib.gg_chung_lu_exact.argtypes = [ctypes.c_int32, dp, ctypes.c_uint64, i32pp, i32pp]
            lib.gg_chung_lu_exact.restype = ctypes.c_int64
            lib.gg_chung_lu_fast.argtypes = [ctypes.c_int32, dp, ctypes.c_uint64, i32pp, i32pp]
            lib.gg_chung_lu_fast.restype = ctypes.c_int64
            lib.gg_rmat.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_uint64, i32p, i32p]
            lib.gg_rmat.restype = ctypes.c_int64
            lib.gg_planted.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_double, ctypes.c_uint64, i32pp, i32pp]
            lib.gg_planted.restype = ctypes.c_int64
            lib.gg_gnp.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_uint64, i32pp, i32pp]
            lib.gg_gnp.restype = ctypes.c_int64
            lib.gg_uniform.argtypes = [ctypes.c_uint64, ctypes.c_int64, dp]
            lib.gg_uniform.restype = None
            lib.gg_csr_from_edges.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i64p, i32pp]
            lib.gg_csr_from_edges.restype = ctypes.c_int64
            lib.gg_free.argtypes = [ctypes.c_void_p]
            lib.gg_free.restype = None
            _lib = lib
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _take_edges(m: int, pu, pv):
    lib = _L()
    if m < 0:
        raise MemoryError("graph generator ran out of memory")
    if m == 0:
        return np.zeros(0, np.int32), np.zeros(0, np.int32)
    u = np.ctypeslib.as_array(pu, shape=(m,)).copy()
    v = np.ctypeslib.as_array(pv, shape=(m,)).copy()
    lib.gg_free(ctypes.cast(pu, ctypes.c_void_p))
    lib.gg_free(ctypes.cast(pv, ctypes.c_void_p))
    return u, v


@dataclass
class Graph:
    """Canonical symmetric CSR graph on vertices 0..n-1."""

    n: int
    rowptr: np.ndarray  # int64[n+1]
    col: np.ndarray  # int32[2m], each row sorted ascending
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.rowptr[-1]) // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.rowptr)

    def edges(self) -> np.ndarray:
        """Undirected edges (u < v) in CSR order, shape (m, 2)."""
        src = np.repeat(np.arange(self.n, dtype=np.int32), self.degrees())
        keep = src < self.col
        return np.stack([src[keep], self.col[keep]], axis=1)


def csr_from_edges(n: int, u: np.ndarray, v: np.ndarray, name: str = "") -> Graph:
    """Canonical symmetric CSR from an undirected edge list (loops and duplicates dropped)."""
    u = np.ascontiguousarray(u, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.int32)
    if u.shape != v.shape:
        raise ValueError("edge arrays differ in length")
    rowptr = np.zeros(n + 1, dtype=np.int64)
    pcol = ctypes.POINTER(ctypes.c_int32)()
    lib = _L()
    w = lib.gg_csr_from_edges(int(n), int(u.size), _p(u, ctypes.c_int32), _p(v, ctypes.c_int32),
                              _p(rowptr, ctypes.c_int64), ctypes.byref(pcol))
    if w < 0:
        raise ValueError("edge list has an endpoint outside 0..n-1 (or out of memory)")
    col = np.ctypeslib.as_array(pcol, shape=(max(int(w), 1),))[: int(w)].copy()
    lib.gg_free(ctypes.cast(pcol, ctypes.c_void_p))
    return Graph(int(n), rowptr, col, name)


def power_law_weights(n: int, avg_deg: float, gamma: float, w_max: float) -> np.ndarray:
    """Expected degrees w_i = c (i + i0)^(-1/(gamma-1)), i = 0..n-1 (non-increasing), with
    c and i0 chosen so that w_0 = w_max and mean(w) = avg_deg (solved by bisection)."""
    beta = 1.0 / (gamma - 1.0)
    if w_max <= avg_deg:
        return np.full(n, float(avg_deg))
    idx = np.arange(n, dtype=np.float64)

    def mean_for(i0: float) -> float:
        return float(np.mean(w_max * (i0 / (idx + i0)) ** beta))

    lo, hi = 1e-9, 1.0
    while mean_for(hi) < avg_deg:
        hi *= 2.0
        if hi > 1e18:
            break
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mean_for(mid) < avg_deg:
            lo = mid
        else:
            hi = mid
    i0 = 0.5 * (lo + hi)
    return w_max * (i0 / (idx + i0)) ** beta


def chung_lu(n: int, avg_deg: float, gamma: float, w_max: float | None = None, seed: int = 1,
             exact: bool | None = None) -> Graph:
    """Seeded Chung-Lu graph with power-law expected degrees. ``w_max`` defaults to
    sqrt(sum w) = sqrt(n * avg_deg), capped at n-1, so every pair probability is <= 1."""
    if w_max is None:
        w_max = min(math.sqrt(n * avg_deg), n - 1.0)
    w = np.ascontiguousarray(power_law_weights(n, avg_deg, gamma, w_max), dtype=np.float64)
    if exact is None:
        exact = n <= 5000
    pu = ctypes.POINTER(ctypes.c_int32)()
    pv = ctypes.POINTER(ctypes.c_int32)()
    fn = _L().gg_chung_lu_exact if exact else _L().gg_chung_lu_fast
    m = fn(int(n), _p(w, ctypes.c_double), int(seed), ctypes.byref(pu), ctypes.byref(pv))
    u, v = _take_edges(int(m), pu, pv)
    return csr_from_edges(n, u, v, f"chung_lu(n={n},d={avg_deg},g={gamma},wmax={w_max:.1f},seed={seed})")


def rmat_edges(scale: int, samples: int, a: float, b: float, c: float, seed: int):
    u = np.empty(samples, np.int32)
    v = np.empty(samples, np.int32)
    _L().gg_rmat(int(scale), int(samples), float(a), float(b), float(c), int(seed),
                 _p(u, ctypes.c_int32), _p(v, ctypes.c_int32))
    return u, v


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 2) -> Graph:
    """Seeded R-MAT graph on 2^scale vertices from edge_factor * 2^scale directed samples,
    no noise and no permutation, symmetrised with loops and duplicates dropped."""
    n = 1 << scale
    u, v = rmat_edges(scale, edge_factor * n, a, b, c, seed)
    return csr_from_edges(n, u, v, f"rmat(scale={scale},ef={edge_factor},a={a},b={b},c={c},seed={seed})")


def rmat_m(m_target: int, a: float = 0.57, b: float = 0.19, c: float = 0.19, seed: int = 5) -> Graph:
    """R-MAT sized by edge count: n = 2^ceil(log2(m/8)); samples are drawn in chunks until
    m_target unique undirected edges exist or 4 * m_target samples were drawn."""
    scale = max(1, int(math.ceil(math.log2(max(m_target / 8.0, 2.0)))))
    n = 1 << scale
    us, vs = [], []
    drawn = 0
    g = None
    chunk = max(m_target, 16)
    k = 0
    while drawn < 4 * m_target:
        u, v = rmat_edges(scale, chunk, a, b, c, seed * 1000003 + k)
        us.append(u)
        vs.append(v)
        drawn += chunk
        k += 1
        g = csr_from_edges(n, np.concatenate(us), np.concatenate(vs))
        if g.m >= m_target:
            break
    if g.m > m_target:
        # keep the first m_target unique edges in sampling order
        uu, vv = np.concatenate(us), np.concatenate(vs)
        lo, hi = np.minimum(uu, vv), np.maximum(uu, vv)
        keep = lo != hi
        key = lo[keep].astype(np.int64) * n + hi[keep]
        _, first = np.unique(key, return_index=True)
        first.sort()
        sel = first[:m_target]
        g = csr_from_edges(n, lo[keep][sel], hi[keep][sel])
    g.name = f"rmat_m(m={m_target},scale={scale},seed={seed})"
    return g


def planted_edges(n: int, k: int, smin: int, smax: int, p: float, seed: int):
    pu = ctypes.POINTER(ctypes.c_int32)()
    pv = ctypes.POINTER(ctypes.c_int32)()
    m = _L().gg_planted(int(n), int(k), int(smin), int(smax), float(p), int(seed), ctypes.byref(pu),
                        ctypes.byref(pv))
    return _take_edges(int(m), pu, pv)


def with_planted(g: Graph, k: int, smin: int, smax: int, p: float, seed: int) -> Graph:
    """Union of ``g`` and ``k`` planted communities (sizes U[smin, smax], density p)."""
    e = g.edges()
    pu, pv = planted_edges(g.n, k, smin, smax, p, seed)
    u = np.concatenate([e[:, 0], pu])
    v = np.concatenate([e[:, 1], pv])
    return csr_from_edges(g.n, u, v, g.name + f"+planted(k={k},{smin}-{smax},p={p},seed={seed})")


def gnp(n: int, p: float, seed: int) -> Graph:
    pu = ctypes.POINTER(ctypes.c_int32)()
    pv = ctypes.POINTER(ctypes.c_int32)()
    m = _L().gg_gnp(int(n), float(p), int(seed), ctypes.byref(pu), ctypes.byref(pv))
    u, v = _take_edges(int(m), pu, pv)
    return csr_from_edges(n, u, v, f"gnp(n={n},p={p},seed={seed})")


def uniform(seed: int, count: int) -> np.ndarray:
    out = np.empty(count, np.float64)
    _L().gg_uniform(int(seed), int(count), _p(out, ctypes.c_double))
    return out


def complete(n: int) -> Graph:
    iu, ju = np.triu_indices(n, 1)
    return csr_from_edges(n, iu.astype(np.int32), ju.astype(np.int32), f"K{n}")


def fig1() -> Graph:
    """The example graph of the paper's Figure 1: K5 on a..e (0..4), f (5) adjacent to a, b, e
    and g (6) adjacent to c, d."""
    a, b, c, d, e, f, g = range(7)
    k5 = [(x, y) for x in range(5) for y in range(x + 1, 5)]
    extra = [(a, f), (b, f), (e, f), (c, g), (d, g)]
    ed = np.array(k5 + extra, dtype=np.int32)
    return csr_from_edges(7, ed[:, 0], ed[:, 1], "fig1")


def disjoint_union(*gs: Graph) -> Graph:
    us, vs, off = [], [], 0
    for g in gs:
        e = g.edges()
        us.append(e[:, 0] + off)
        vs.append(e[:, 1] + off)
        off += g.n
    return csr_from_edges(off, np.concatenate(us).astype(np.int32), np.concatenate(vs).astype(np.int32),
                          "union(" + ",".join(g.name for g in gs) + ")")


def path(n: int) -> Graph:
    a = np.arange(n - 1, dtype=np.int32)
    return csr_from_edges(n, a, a + 1, f"P{n}")


def relabel(g: Graph, perm: np.ndarray) -> Graph:
    """Graph with vertex v renamed perm[v]."""
    e = g.edges()
    perm = np.asarray(perm, dtype=np.int32)
    return csr_from_edges(g.n, perm[e[:, 0]], perm[e[:, 1]], g.name + "+relabel")


# --------------------------------------------------------------------------------------
# The benchmark workloads, by what they are.

def chung_lu_2k(seed: int = 1) -> Graph:
    """Chung-Lu, n = 2,000, average degree 20, exponent 2.1, maximum expected degree 200."""
    return chung_lu(2000, 20.0, 2.1, w_max=200.0, seed=seed, exact=True)


def rmat_scale20(seed: int = 2, scale: int = 20) -> Graph:
    """R-MAT scale 20, edge factor 16, a=0.57, b=0.19, c=0.19 (d=0.05)."""
    return rmat(scale, 16, 0.57, 0.19, 0.19, seed)


def chung_lu_4m_planted(seed: int = 3, n: int = 4_194_304) -> Graph:
    """Chung-Lu, n = 4,194,304, average degree 30, exponent 2.3, w_max = sqrt(sum w), plus 2,000
    planted communities of 20-60 vertices at internal density 0.7."""
    g = chung_lu(n, 30.0, 2.3, seed=seed, exact=False)
    return with_planted(g, 2000, 20, 60, 0.7, seed + 7919)


def batch_workload(count: int, seed: int = 4):
    """``count`` seeded Chung-Lu graphs with n ~ U[50, 5000], average degree ~ U[8, 40], exponent
    2.2, w_0 = min(sqrt(sum w), n - 1), each with (r, s) drawn uniformly from (1,2), (2,3), (3,4).
    Returns a list of (graph, (r, s)); the first k items do not depend on ``count``."""
    u = uniform(seed, 3 * count)
    rs = [(1, 2), (2, 3), (3, 4)]
    out = []
    for i in range(count):
        n = 50 + int(u[3 * i] * 4951)
        d = 8.0 + u[3 * i + 1] * 32.0
        g = chung_lu(n, d, 2.2, seed=seed + i, exact=False)
        out.append((g, rs[min(2, int(u[3 * i + 2] * 3))]))
    return out


def serve_pool(count: int, seed: int = 5, max_m: int | None = None):
    """Graphs of the served stream: Chung-Lu or R-MAT with probability 1/2 each, edge count
    log-uniform in [1e2, 1e6]; Chung-Lu with average degree ~ U[8, 40], exponent 2.2, n = 2m/d;
    R-MAT with n = 2^ceil(log2(m/8)) and a, b, c = 0.57, 0.19, 0.19. The first k graphs do not
    depend on ``count``. With ``max_m``, the draws whose edge count exceeds it are skipped (not
    generated), the others are the same graphs in the same order."""
    u = uniform(seed, 3 * count)
    out = []
    for i in range(count):
        m = int(round(math.exp(math.log(1e2) + u[3 * i] * (math.log(1e6) - math.log(1e2)))))
        if max_m is not None and m > max_m:
            continue
        if u[3 * i + 1] < 0.5:
            d = 8.0 + u[3 * i + 2] * 32.0
            n = max(16, int(2 * m / d))
            out.append(chung_lu(n, d, 2.2, seed=seed * 100003 + i, exact=False))
        else:
            out.append(rmat_m(m, seed=seed * 100003 + i))
    return out


def hubs_over_sparse(n_common: int = 6000, hubs: int = 4, p_hub: float = 0.9, avg_deg: float = 8.0,
                     seed: int = 51) -> Graph:
    """A sparse Chung-Lu graph (exponent 2.2) on ``n_common`` vertices plus ``hubs`` mutually
    adjacent hub vertices (ids n_common ..), each adjacent to every other vertex with probability
    p_hub. Hubs reach degree ~ p_hub * n_common, pairs of hubs share ~ p_hub^2 * n_common
    neighbours and triples ~ p_hub^3 * n_common, so hub vertices, hub edges and hub triangles
    have neighbour lists of thousands of entries while everything else stays sparse."""
    base = chung_lu(n_common, avg_deg, 2.2, seed=seed, exact=True)
    e = base.edges()
    u = uniform(seed * 7 + 1, hubs * n_common).reshape(hubs, n_common)
    us, vs = [e[:, 0]], [e[:, 1]]
    for h in range(hubs):
        nb = np.nonzero(u[h] < p_hub)[0].astype(np.int32)
        us.append(np.full(nb.size, n_common + h, np.int32))
        vs.append(nb)
        for h2 in range(h + 1, hubs):
            us.append(np.array([n_common + h], np.int32))
            vs.append(np.array([n_common + h2], np.int32))
    return csr_from_edges(n_common + hubs, np.concatenate(us).astype(np.int32), np.concatenate(vs).astype(np.int32),
                          f"hubs_over_sparse(n={n_common},hubs={hubs},p={p_hub},d={avg_deg},seed={seed})")
