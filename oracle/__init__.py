"""CPU oracle for the (r,s) nucleus decomposition -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use
this package. The CUDA library never imports, links or calls it, and the two share no code:
the only common module is the seeded input generator package ``graphgen``.

The arithmetic lives in ``nucleus_oracle.c`` (plain sequential C, exact integers); this
module only compiles it (gcc, no -march flags, so it builds on x86_64 and aarch64 alike)
and marshals numpy arrays through ctypes.

Functions (each follows the passage named in its docstring):

* ``list_cliques(g, c)``        all c-cliques, lexicographic order of ascending tuples
* ``count(g, r, s)``            s-clique count of every r-clique (Algorithm 2, Count-Func)
* ``decompose(g, r, s)``        Algorithm 2's peeling loop with Update/Update-Func, 1/a exact
* ``decompose_fixpoint(g, r, s)`` the definition of Section 2 written out as nested fixpoints
* ``local_counts(g, r, s, tuples)`` per-r-clique s-clique counts one by one (sampled checks)
* ``certify(...)``              validity + elimination-order certificate of a claimed result
* ``certify_all(...)``          the same certificate over every r-clique (or a sample), with the
                                oracle's own id lookups, split across host threads
* ``nuclei(g, r, s, core, c)``  the s-connected components of the c-(r,s) nucleus (Section 2,
                                footnote: the original definition's connectivity)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nucleus_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

LOOKUP_FN = ctypes.CFUNCTYPE(ctypes.c_int64, ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p)


def build_lib(force: bool = False) -> str:
    """Compile the oracle with plain gcc -O2 into ``_liboracle.so``."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        base = ["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-o", tmp, _SRC]
        # OpenMP only splits the certificate's loops across host threads; without it the same
        # code runs on one thread
        if subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True).returncode != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build_lib()
            lib = ctypes.CDLL(_LIB)
            i64p = ctypes.POINTER(ctypes.c_int64)
            i32p = ctypes.POINTER(ctypes.c_int32)
            g3 = [ctypes.c_int32, i64p, i32p]
            lib.orc_list_cliques.argtypes = g3 + [ctypes.c_int, i32p, ctypes.c_int64]
            lib.orc_list_cliques.restype = ctypes.c_int64
            lib.orc_count.argtypes = g3 + [ctypes.c_int, ctypes.c_int, i64p, i64p, i64p]
            lib.orc_count.restype = ctypes.c_int
            lib.orc_decompose.argtypes = g3 + [ctypes.c_int, ctypes.c_int, i32p, i32p, i64p, i64p, i64p,
                                               ctypes.c_int64, i64p, i64p, i64p, i64p]
            lib.orc_decompose.restype = ctypes.c_int
            lib.orc_decompose_fixpoint.argtypes = g3 + [ctypes.c_int, ctypes.c_int, i32p]
            lib.orc_decompose_fixpoint.restype = ctypes.c_int
            lib.orc_certify.argtypes = g3 + [ctypes.c_int, ctypes.c_int, i32p, i32p, i64p, i32p, ctypes.c_int64,
                                             LOOKUP_FN, ctypes.c_void_p, i64p, i64p]
            lib.orc_certify.restype = ctypes.c_int
            lib.orc_local_counts.argtypes = g3 + [ctypes.c_int, ctypes.c_int, i32p, ctypes.c_int64, i64p]
            lib.orc_local_counts.restype = ctypes.c_int
            lib.orc_certify_all.argtypes = g3 + [ctypes.c_int, ctypes.c_int, ctypes.c_int64, i32p, i32p, i64p,
                                                 ctypes.c_int64, i64p, ctypes.c_int64, ctypes.c_int, i64p, i64p, i64p]
            lib.orc_certify_all.restype = ctypes.c_int
            lib.orc_nuclei.argtypes = g3 + [ctypes.c_int, ctypes.c_int, i32p, ctypes.c_int32, i32p, i64p]
            lib.orc_nuclei.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _g(g):
    rp = np.ascontiguousarray(g.rowptr, dtype=np.int64)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    if col.size == 0:
        col = np.zeros(1, np.int32)
    return rp, col, [ctypes.c_int32(g.n), _p(rp, ctypes.c_int64), _p(col, ctypes.c_int32)]


def _check(rc: int, what: str):
    if rc == -1:
        raise ValueError(f"{what}: unsupported (r, s); the oracle takes 1 <= r < s <= 7")
    if rc == -2:
        raise MemoryError(f"{what}: out of memory")
    if rc != 0:
        raise RuntimeError(f"{what}: internal inconsistency (rc={rc})")


def list_cliques(g, c: int) -> np.ndarray:
    """All c-cliques as ascending tuples, lexicographic order; shape (n_c, c). Algorithm 1."""
    rp, col, a = _g(g)
    n_c = _L().orc_list_cliques(*a, int(c), None, 0)
    if n_c < 0:
        raise ValueError("bad clique size")
    out = np.zeros((max(int(n_c), 1), c), np.int32)
    _L().orc_list_cliques(*a, int(c), _p(out, ctypes.c_int32), int(n_c))
    return out[: int(n_c)]


def count(g, r: int, s: int):
    """(counts int64[n_r], n_s): Algorithm 2, Count-Func applied to every s-clique."""
    rp, col, a = _g(g)
    n_r = ctypes.c_int64()
    n_s = ctypes.c_int64()
    _check(_L().orc_count(*a, r, s, None, ctypes.byref(n_r), ctypes.byref(n_s)), "count")
    counts = np.zeros(max(n_r.value, 1), np.int64)
    _check(_L().orc_count(*a, r, s, _p(counts, ctypes.c_int64), ctypes.byref(n_r), ctypes.byref(n_s)), "count")
    return counts[: n_r.value], int(n_s.value)


@dataclass
class Decomposition:
    core: np.ndarray  # int32[n_r], canonical order
    round: np.ndarray  # int32[n_r], round in which each r-clique is peeled
    rho: int  # number of rounds
    sizes: np.ndarray  # |A| per round
    levels: np.ndarray  # k per round
    n_s: int
    listed: int  # (s-clique, peeled member) pairs re-listed by Update over the whole run
    live: int  # of those, the pairs whose s-clique had no r-subset peeled in an earlier round
    decs: int  # unit decrements: per live s-clique, its r-subsets outside A (counted once per S)
    extra: dict = field(default_factory=dict)


def decompose(g, r: int, s: int) -> Decomposition:
    """Algorithm 2 (arb-nucleus-decomp) with Update / Update-Func; exact 1/a."""
    rp, col, a = _g(g)
    n_r = ctypes.c_int64()
    _check(_L().orc_count(*a, r, s, None, ctypes.byref(n_r), None), "decompose")
    nr = n_r.value
    core = np.zeros(max(nr, 1), np.int32)
    rnd = np.zeros(max(nr, 1), np.int32)
    cap = max(nr, 1)
    sizes = np.zeros(cap, np.int64)
    levels = np.zeros(cap, np.int64)
    rho = ctypes.c_int64()
    n_s = ctypes.c_int64()
    listed = ctypes.c_int64()
    live = ctypes.c_int64()
    decs = ctypes.c_int64()
    _check(_L().orc_decompose(*a, r, s, _p(core, ctypes.c_int32), _p(rnd, ctypes.c_int32), ctypes.byref(rho),
                              _p(sizes, ctypes.c_int64), _p(levels, ctypes.c_int64), cap, ctypes.byref(n_s),
                              ctypes.byref(listed), ctypes.byref(live), ctypes.byref(decs)), "decompose")
    t = rho.value
    return Decomposition(core[:nr], rnd[:nr], t, sizes[:t].copy(), levels[:t].copy(), int(n_s.value),
                         int(listed.value), int(live.value), int(decs.value))


def decompose_fixpoint(g, r: int, s: int) -> np.ndarray:
    """Core numbers straight from the definition (Section 2): nested greatest fixpoints."""
    rp, col, a = _g(g)
    n_r = ctypes.c_int64()
    _check(_L().orc_count(*a, r, s, None, ctypes.byref(n_r), None), "fixpoint")
    core = np.zeros(max(n_r.value, 1), np.int32)
    _check(_L().orc_decompose_fixpoint(*a, r, s, _p(core, ctypes.c_int32)), "fixpoint")
    return core[: n_r.value]


def local_counts(g, r: int, s: int, tuples: np.ndarray) -> np.ndarray:
    """s-clique count of each given r-clique (ascending tuples), one by one."""
    rp, col, a = _g(g)
    t = np.ascontiguousarray(tuples, dtype=np.int32).reshape(-1, r)
    out = np.zeros(max(t.shape[0], 1), np.int64)
    _check(_L().orc_local_counts(*a, r, s, _p(t, ctypes.c_int32), t.shape[0], _p(out, ctypes.c_int64)),
           "local_counts")
    return out[: t.shape[0]]


def certify(g, r: int, s: int, core: np.ndarray, rnd: np.ndarray, ids: np.ndarray, tuples: np.ndarray, lookup):
    """Validity / elimination-order supports of the r-cliques ``ids`` (ascending ``tuples``)
    under a claimed (core, round). ``lookup(tuple) -> canonical id``. Returns two int64 arrays."""
    rp, col, a = _g(g)
    core = np.ascontiguousarray(core, dtype=np.int32)
    rnd = np.ascontiguousarray(rnd, dtype=np.int32)
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    t = np.ascontiguousarray(tuples, dtype=np.int32).reshape(-1, r)
    k = ids.size
    sv = np.zeros(max(k, 1), np.int64)
    so = np.zeros(max(k, 1), np.int64)

    def _cb(ptr, user):
        return int(lookup(tuple(ptr[i] for i in range(r))))

    cb = LOOKUP_FN(_cb)
    _check(_L().orc_certify(*a, r, s, _p(core, ctypes.c_int32), _p(rnd, ctypes.c_int32), _p(ids, ctypes.c_int64),
                            _p(t, ctypes.c_int32), k, cb, None, _p(sv, ctypes.c_int64), _p(so, ctypes.c_int64)),
           "certify")
    return sv[:k], so[:k]


def certify_all(g, r: int, s: int, core: np.ndarray, rnd: np.ndarray, levels: np.ndarray, ids=None,
                nthreads: int = 0) -> dict:
    """Validity / elimination-order / level certificate of a claimed decomposition (Section 2
    definition; see ``orc_certify_all``) over every r-clique, or over the r-cliques ``ids``.
    ``core`` and ``rnd`` cover all n_r r-cliques (canonical order); ``levels[t]`` is the level
    of round t. Returns the failure counts, the first failing id (-1 if none) and, for a
    sample, the two supports of each sampled r-clique."""
    rp, col, a = _g(g)
    core = np.ascontiguousarray(core, dtype=np.int32)
    rnd = np.ascontiguousarray(rnd, dtype=np.int32)
    levels = np.ascontiguousarray(levels, dtype=np.int64)
    if levels.size == 0:
        levels = np.zeros(1, np.int64)
        rho = 0
    else:
        rho = levels.size
    bad = np.zeros(4, np.int64)
    sv = so = None
    if ids is None:
        pids, k = None, 0
    else:
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        k = ids.size
        pids = _p(ids if k else np.zeros(1, np.int64), ctypes.c_int64)
        sv = np.zeros(max(k, 1), np.int64)
        so = np.zeros(max(k, 1), np.int64)
    rc = _L().orc_certify_all(*a, int(r), int(s), int(core.size), _p(core if core.size else np.zeros(1, np.int32),
                                                                      ctypes.c_int32),
                              _p(rnd if rnd.size else np.zeros(1, np.int32), ctypes.c_int32),
                              _p(levels, ctypes.c_int64), int(rho), pids, int(k), int(nthreads),
                              _p(bad, ctypes.c_int64), None if sv is None else _p(sv, ctypes.c_int64),
                              None if so is None else _p(so, ctypes.c_int64))
    if rc == -3:
        raise ValueError("certify_all: an r-subset of an s-clique is not an r-clique, or n_r does not match")
    _check(rc, "certify_all")
    out = {"bad_valid": int(bad[0]), "bad_order": int(bad[1]), "bad_level": int(bad[2]), "first_bad": int(bad[3])}
    if sv is not None:
        out["sup_valid"] = sv[:k]
        out["sup_order"] = so[:k]
    return out


def nuclei(g, r: int, s: int, core: np.ndarray, level: int):
    """(comp int32[n_r], n_components): comp[R] = smallest r-clique id of R's component among the
    r-cliques with core >= level, joined through s-cliques all of whose r-subsets have core >=
    level (Section 2, footnote); -1 where core < level."""
    rp, col, a = _g(g)
    core = np.ascontiguousarray(core, dtype=np.int32)
    out = np.zeros(max(core.size, 1), np.int32)
    nc = ctypes.c_int64()
    _check(_L().orc_nuclei(*a, int(r), int(s), _p(core if core.size else np.zeros(1, np.int32), ctypes.c_int32),
                           int(level), _p(out, ctypes.c_int32), ctypes.byref(nc)), "nuclei")
    return out[: core.size], int(nc.value)


def hierarchy(g, r: int, s: int, core: np.ndarray):
    """The nucleus hierarchy (Section 2, footnote), written out from its definition level by level.

    For every distinct core value c, the connected c-(r,s) nuclei are the components of
    X_c = {R : core[R] >= c} (`nuclei`). A node of the hierarchy is a component of X_c that holds an
    r-clique whose core number is exactly c; each r-clique belongs to the node of its own core
    number. The parent of node (c, C) is the node (c', C') at the largest distinct level c' < c for
    which the component C' of X_c' containing C holds an r-clique of core exactly c'. Returns
    (comp, parent_level, parent_comp), int32[n_r] each: comp[R] = smallest r-clique id of R's
    node's component; parent_level[R], parent_comp[R] = the level and smallest id of the parent
    node of R's node, -1 and -1 for a root node."""
    core = np.ascontiguousarray(core, dtype=np.int32)
    n_r = core.size
    comp = np.full(n_r, -1, np.int32)
    parent_level = np.full(n_r, -1, np.int32)
    parent_comp = np.full(n_r, -1, np.int32)
    if n_r == 0:
        return comp, parent_level, parent_comp
    levels = np.unique(core)  # ascending
    comps = {int(c): nuclei(g, r, s, core, int(c))[0] for c in levels}
    # nodes at each level: the components that hold an r-clique of exactly that core number
    nodes = {int(c): set(comps[int(c)][core == c].tolist()) for c in levels}
    for R in range(n_r):
        c = int(core[R])
        comp[R] = comps[c][R]
    for R in range(n_r):
        c = int(core[R])
        for c2 in reversed([int(x) for x in levels if x < c]):
            cc = int(comps[c2][R])
            if cc in nodes[c2]:
                parent_level[R] = c2
                parent_comp[R] = cc
                break
    return comp, parent_level, parent_comp
